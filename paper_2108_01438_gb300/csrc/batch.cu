// Batched reconstruction of several B-scans of different sizes (one plan each):
// every stage of the path -- the operator passes, the FISTA epilogues, the
// wavelet levels, the power iteration and the lambda rule -- runs as ONE launch
// over all scans, each CTA finding its scan from a prefix table of CTA offsets.
// A fixed-count FISTA loop (Sec. 2.3, Eq. alg) is captured once into a CUDA graph
// and replayed; the serving loop instead advances scans that sit at different
// iteration counts one batched iteration at a time.  A scan runs exactly the
// same kernel code whatever it is batched with (the adjoint gather is
// deterministic), so its result does not depend on the mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "operator.cuh"

namespace mbir {

constexpr int kBThreads = 256;
constexpr int kBBlocks = 64;    // CTAs per scan of the batched vector kernels

// Per-scan operands of the batched vector kernels.
struct ScanVec {
  void* v;
  void* w;
  size_t n;
  double* part;   // partial sums (pairs for the power iteration)
  double* scal;   // scalars
  int np;         // partial pairs b_power_finalize reads (0: kBBlocks)
};

__device__ __forceinline__ double bsum(double v) {
  __shared__ double ws[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ double bmax(double v) {
  __shared__ double ws[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// v = uniform [-1, 1) pseudo-random start of the power iteration (SplitMix64 of the index)
template <class R>
__global__ void b_fill_hash(const ScanVec* sv) {
  pdl_wait_release();
  const ScanVec s = sv[blockIdx.y];
  cplx_t<R>* v = reinterpret_cast<cplx_t<R>*>(s.v);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < s.n; i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t a = mix64(2 * i), b = mix64(2 * i + 1);
    v[i] = cmk<cplx_t<R>>(R((a >> 11) * 0x1.0p-53 * 2.0 - 1.0), R((b >> 11) * 0x1.0p-53 * 2.0 - 1.0));
  }
}

// part[2 b] = sum Re(conj(v) w), part[2 b + 1] = sum |w|^2
template <class R>
__global__ void b_dot_norm(const ScanVec* sv) {
  pdl_wait_release();
  const ScanVec s = sv[blockIdx.y];
  const cplx_t<R>* v = reinterpret_cast<const cplx_t<R>*>(s.v);
  const cplx_t<R>* w = reinterpret_cast<const cplx_t<R>*>(s.w);
  double d = 0.0, q = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < s.n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> a = v[i], b = w[i];
    d += double(a.x) * double(b.x) + double(a.y) * double(b.y);
    q += double(b.x) * double(b.x) + double(b.y) * double(b.y);
  }
  const double D = bsum(d), Q = bsum(q);
  if (threadIdx.x == 0) {
    s.part[2 * blockIdx.x] = D;
    s.part[2 * blockIdx.x + 1] = Q;
  }
}

// scal[0] = <v, w>, scal[1] = 1/||w||
__global__ void b_power_finalize(const ScanVec* sv, int nb) {
  pdl_wait_release();
  const ScanVec s = sv[blockIdx.y];
  if (s.np > 0) nb = s.np;
  double d = 0.0, q = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    d += s.part[2 * i];
    q += s.part[2 * i + 1];
  }
  const double D = bsum(d), Q = bsum(q);
  if (threadIdx.x == 0) {
    s.scal[0] = D;
    s.scal[1] = Q > 0 ? 1.0 / sqrt(Q) : 0.0;
  }
}

// v = w * scal[1]
template <class R>
__global__ void b_scale(const ScanVec* sv) {
  pdl_wait_release();
  const ScanVec s = sv[blockIdx.y];
  cplx_t<R>* v = reinterpret_cast<cplx_t<R>*>(s.v);
  const cplx_t<R>* w = reinterpret_cast<const cplx_t<R>*>(s.w);
  const R f = R(s.scal[1]);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < s.n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = cscale(w[i], f);
}

// scal[4] = max |v|
template <class R>
__global__ void b_maxabs(const ScanVec* sv) {
  pdl_wait_release();
  const ScanVec s = sv[blockIdx.y];
  const cplx_t<R>* v = reinterpret_cast<const cplx_t<R>*>(s.v);
  R m2 = R(0);   // largest |v|^2 of the thread, one square root at the end
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < s.n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> a = v[i];
    m2 = fmax(m2, a.x * a.x + a.y * a.y);
  }
  const double M = bmax(sqrt(double(m2)));
  if (threadIdx.x == 0) s.part[blockIdx.x] = M;
}

__global__ void b_max_finalize(const ScanVec* sv, int nb) {
  pdl_wait_release();
  const ScanVec s = sv[blockIdx.y];
  double m = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, s.part[i]);
  const double M = bmax(m);
  if (threadIdx.x == 0) s.scal[4] = M;
}


// Objective of each scan: out = 1/2 sum(part_data) + lam * sum(part_reg), written to
// the scan's trace entry and to the engine's per-slot array.
struct ObjArgs {
  const double* part_data;
  int n_data;
  const double* part_reg;
  int n_reg;
  double lam;
  double* trace_out;
  double* slot_out;
};

__global__ void b_objective(const ObjArgs* oa) {
  pdl_wait_release();
  const ObjArgs o = oa[blockIdx.x];
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < o.n_data; i += blockDim.x) s += o.part_data[i];
  for (int i = threadIdx.x; i < o.n_reg; i += blockDim.x) t += o.part_reg[i];
  const double S = bsum(s), T = bsum(t);
  if (threadIdx.x == 0) {
    const double f = 0.5 * S + o.lam * T;
    if (o.trace_out) *o.trace_out = f;
    *o.slot_out = f;
  }
}

// ------------------------------------------------------------------ contexts

int plan_ctx(mbir_plan p, int penalty, int trace_cap, Ctx* out) {
  int rc = ensure_state(p, trace_cap);
  if (rc) return rc;
  if (penalty == MBIR_PENALTY_DB4) {
    if (!wavelet_supported(p->nx, p->nz)) return MBIR_ERR_UNSUPPORTED_SIZE;
    rc = ensure_wavelet_scratch(p);
    if (rc) return rc;
  }
  SolveState* S = p->solve;
  Ctx c;
  c.wsA = p->wsA;
  c.wsB = p->wsB;
  c.zA = S->zA;
  c.zB = S->zB;
  c.v = S->v;
  c.pz = S->pz;
  c.r = S->r;
  c.wv_b1 = p->wv_b1;
  c.wv_b2 = p->wv_b2;
  c.wv_coef = p->wv_coef;
  c.part_data = S->part_data;
  c.part_reg = S->part_reg;
  c.part_tmp = S->part_tmp;
  c.scal = S->scal;
  c.objtrace = S->objtrace;
  c.n_data = S->n_data;
  c.n_reg = S->n_reg;
  c.trace_cap = S->trace_cap;
  c.nimg = S->nimg;
  c.nmeas = S->nmeas;
  c.owned = false;
  *out = c;
  return MBIR_OK;
}

static int reg_partials(mbir_plan p) {
  int nr = lateral_grid(p, p->nz);
  if (wavelet_supported(p->nx, p->nz)) nr = std::max(nr, wavelet_partial_count(p->nx, p->nz));
  return nr;
}

size_t ctx_bytes(mbir_plan p, int penalty, int trace_cap) {
  const size_t es = p->precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t rs = p->precision == MBIR_FP64 ? sizeof(double) : sizeof(float);
  const size_t img = (size_t)p->nx * p->nz, meas = (size_t)p->nx * p->m;
  size_t b = 2 * es * p->ws_elems + 3 * es * img + 2 * rs * meas;
  if (penalty == MBIR_PENALTY_DB4) b += es * (img / 4 + img / 16 + img);
  b += sizeof(double) * ((size_t)lateral_grid(p, p->m) + reg_partials(p) + 2 * (size_t)part_tmp_count(p) + 16 +
                         trace_cap);
  return b;
}

void ctx_free(Ctx* c) {
  if (!c->owned) return;
  void* ptrs[] = {c->wsA, c->wsB, c->zA, c->zB, c->v, c->pz, c->r, c->wv_b1, c->wv_b2, c->wv_coef,
                  c->part_data, c->part_reg, c->part_tmp, c->scal, c->objtrace};
  for (void* q : ptrs) cudaFree(q);
  *c = Ctx();
}

int ctx_alloc(mbir_plan p, int penalty, int trace_cap, Ctx* out) {
  Ctx c;
  c.owned = true;
  const size_t es = p->precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t rs = p->precision == MBIR_FP64 ? sizeof(double) : sizeof(float);
  c.nimg = (size_t)p->nx * p->nz;
  c.nmeas = (size_t)p->nx * p->m;
  c.n_data = lateral_grid(p, p->m);
  c.n_reg = reg_partials(p);
  c.trace_cap = trace_cap;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** q, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(q, bytes);
  };
  A(&c.wsA, es * p->ws_elems);
  A(&c.wsB, es * p->ws_elems);
  A(&c.zA, es * c.nimg);
  A(&c.zB, es * c.nimg);
  A(&c.v, es * c.nimg);
  A(&c.pz, rs * c.nmeas);
  A(&c.r, rs * c.nmeas);
  if (penalty == MBIR_PENALTY_DB4) {
    A(&c.wv_b1, es * (c.nimg / 4));
    A(&c.wv_b2, es * (c.nimg / 16));
    A(&c.wv_coef, es * c.nimg);
  }
  A((void**)&c.part_data, sizeof(double) * c.n_data);
  A((void**)&c.part_reg, sizeof(double) * c.n_reg);
  A((void**)&c.part_tmp, sizeof(double) * 2 * part_tmp_count(p));
  A((void**)&c.scal, sizeof(double) * 16);
  A((void**)&c.objtrace, sizeof(double) * std::max(trace_cap, 1));
  if (e != cudaSuccess) {
    ctx_free(&c);
    return set_cuda_error(e, "request context allocation");
  }
  *out = c;
  return MBIR_OK;
}

// ------------------------------------------------------------------ engine

Engine::~Engine() {
  cudaStreamSynchronize(st_);
  cudaFree(dbuf_);
  cudaFree(dobj_);
  for (Staging& r : ring_) {
    cudaFreeHost(r.h);
    if (r.ev) cudaEventDestroy(r.ev);
  }
}

int Engine::begin_build() {
  cur_ = (cur_ + 1) % kRing;
  Staging& r = ring_[cur_];
  if (r.pending) {
    MBIR_CUDA_TRY(cudaEventSynchronize(r.ev));
    r.pending = false;
  }
  hbuf_ = r.h;
  hcap_ = r.cap;
  hlen_ = 0;
  return MBIR_OK;
}

int Engine::check(const std::vector<BScan*>& scans) {
  for (BScan* s : scans) {
    if (prec_ < 0) {
      prec_ = s->p->precision;
      J_ = s->p->J;
      alpha_ = s->p->alpha;
      esz_ = prec_ == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
      rsz_ = prec_ == MBIR_FP64 ? sizeof(double) : sizeof(float);
    }
    if (s->p->precision != prec_ || s->p->J != J_ || s->p->alpha != alpha_) return MBIR_ERR_INVALID;
    if (s->o.penalty == MBIR_PENALTY_DB4 && !s->c.wv_coef) return MBIR_ERR_INVALID;
  }
  return MBIR_OK;
}

size_t Engine::push(const void* data, size_t bytes) {
  const size_t at = (hlen_ + 15) & ~size_t(15);
  if (at + bytes > hcap_) grow(at + bytes);
  if (grow_failed_ || at + bytes > hcap_) {
    grow_failed_ = true;
    return 0;
  }
  memcpy(hbuf_ + at, data, bytes);
  hlen_ = at + bytes;
  return at;
}

void Engine::grow(size_t need) {
  size_t cap = hcap_ ? hcap_ : (1 << 16);
  while (cap < need) cap *= 2;
  unsigned char* nb = nullptr;
  if (cudaMallocHost(&nb, cap) != cudaSuccess) {
    grow_failed_ = true;
    return;
  }
  if (hbuf_) {
    memcpy(nb, hbuf_, hlen_);
    cudaFreeHost(hbuf_);   // not pending: begin_build waited for its last upload
  }
  hbuf_ = nb;
  hcap_ = cap;
  ring_[cur_].h = nb;
  ring_[cur_].cap = cap;
}

int Engine::upload() {
  if (grow_failed_) return MBIR_ERR_OOM;
  if (hlen_ > dcap_) {
    // previous launches reading dbuf_ must be done before it is released
    MBIR_CUDA_TRY(cudaStreamSynchronize(st_));
    cudaFree(dbuf_);
    dbuf_ = nullptr;
    const size_t cap = std::max(hlen_, 2 * dcap_);
    MBIR_CUDA_TRY(cudaMalloc(&dbuf_, cap));
    dcap_ = cap;
  }
  MBIR_CUDA_TRY(cudaMemcpyAsync(dbuf_, hbuf_, hlen_, cudaMemcpyHostToDevice, st_));
  Staging& r = ring_[cur_];
  if (!r.ev) MBIR_CUDA_TRY(cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming));
  MBIR_CUDA_TRY(cudaEventRecord(r.ev, st_));
  r.pending = true;
  return MBIR_OK;
}

static LatFill lfill(const void* in, void* out, const uint8_t* mask, int cols, double scale) {
  LatFill f;
  memset(&f, 0, sizeof(f));
  f.in = in;
  f.out = out;
  f.mask = mask;
  f.cols = cols;
  f.scale = scale;
  return f;
}

template <class F>
int Engine::add_lateral(std::vector<Stage>& out, int mode, const std::vector<BScan*>& idx, F make, bool uses_mu) {
  if (idx.empty()) return MBIR_OK;
  const size_t ab = lat_args_bytes(prec_);
  std::vector<unsigned char> blocks(ab * idx.size());
  std::vector<int> off(idx.size() + 1, 0);
  size_t smem = 0;
  int blu = 0;
  for (size_t i = 0; i < idx.size(); ++i) {
    BScan& s = *idx[i];
    LatFill f = make(s);
    fill_lat_args(s.p, f, blocks.data() + i * ab);
    off[i + 1] = off[i] + lateral_grid(s.p, f.cols);
    smem = std::max(smem, lat_smem_bytes(s.p));
    if (s.p->chirp) blu = 1;
  }
  Stage g{0, mode, 0, 0, (int)idx.size(), off.back(), smem, uses_mu ? 1 : 0, blu};
  g.arg_off = push(blocks.data(), blocks.size());
  g.off_off = push(off.data(), off.size() * sizeof(int));
  out.push_back(g);
  return grow_failed_ ? MBIR_ERR_OOM : MBIR_OK;
}

// One launch per (row kernel, shared-memory size, fused passes or not) among the
// scans: each scan runs the kernel its own plan chooses (tuned or automatic), and
// scans with shorter rows keep the occupancy of their own footprint.
int Engine::add_row(std::vector<Stage>& out, bool adjoint, const std::vector<BScan*>& idx) {
  if (idx.empty()) return MBIR_OK;
  const size_t ab = row_args_bytes(prec_);
  using Key = std::tuple<int, size_t, bool>;
  auto key_of = [&](BScan* s) {
    const int k = row_kind(s->p, adjoint);
    // batched lean gathers keep the plain passes (their fused form spills)
    return Key(k, row_kind_smem(s->p, k), row_fusable(s->p) && k != ROW_GATHER_PAIR_LEAN);
  };
  std::vector<Key> keys;
  for (BScan* s : idx) {
    const Key k = key_of(s);
    if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
  }
  for (const Key& key : keys) {
    const int kind = std::get<0>(key);
    std::vector<BScan*> grp;
    for (BScan* s : idx)
      if (key_of(s) == key) grp.push_back(s);
    std::vector<unsigned char> blocks(ab * grp.size());
    std::vector<int> off(grp.size() + 1, 0);
    size_t smem = 0;
    for (size_t i = 0; i < grp.size(); ++i) {
      BScan& s = *grp[i];
      fill_row_args(s.p, s.c.wsA, s.c.wsB, blocks.data() + i * ab);
      off[i + 1] = off[i] + row_ctas(s.p, kind);
      smem = std::max(smem, row_kind_smem(s.p, kind));
    }
    Stage g{1, kind, 0, 0, (int)grp.size(), off.back(), smem, 0, 0, std::get<2>(key) ? 1 : 0};
    g.arg_off = push(blocks.data(), blocks.size());
    g.off_off = push(off.data(), off.size() * sizeof(int));
    out.push_back(g);
  }
  return grow_failed_ ? MBIR_ERR_OOM : MBIR_OK;
}

int Engine::add_dwt(std::vector<Stage>& out, int inverse, int level, const std::vector<BScan*>& idx,
                    const std::vector<const void*>& in, const std::vector<void*>& outp,
                    const std::vector<void*>& coefs, const std::vector<double*>& partial, bool thresh) {
  if (idx.empty()) return MBIR_OK;
  const size_t ab = dwt_args_bytes(prec_);
  std::vector<unsigned char> blocks(ab * idx.size());
  std::vector<int> off(idx.size() + 1, 0);
  for (size_t i = 0; i < idx.size(); ++i) {
    BScan& s = *idx[i];
    const int th = thresh ? (level == 2 ? 2 : 1) : 0;
    fill_dwt_args(s.p, level, inverse, in.empty() ? nullptr : in[i], outp.empty() ? nullptr : outp[i], coefs[i],
                  thresh ? s.tau : 0.0, th, partial.empty() ? nullptr : partial[i], s.c.wv_b1, s.c.wv_b2,
                  blocks.data() + i * ab);
    off[i + 1] = off[i] + dwt_level_ctas(s.p->nx >> level, s.p->nz >> level, inverse, level);
  }
  Stage g{inverse ? 3 : 2, level, 0, 0, (int)idx.size(), off.back(), dwt_smem_bytes(prec_, inverse, level), 0};
  g.arg_off = push(blocks.data(), blocks.size());
  g.off_off = push(off.data(), off.size() * sizeof(int));
  out.push_back(g);
  return grow_failed_ ? MBIR_ERR_OOM : MBIR_OK;
}

int Engine::run(const Stage& g, double mu) {
  if (g.kind == 4) {
    const ObjArgs* d = reinterpret_cast<const ObjArgs*>(static_cast<unsigned char*>(dbuf_) + g.arg_off);
    launch(b_objective, dim3(g.n), dim3(kBThreads), 0, st_, d);
    MBIR_LAUNCH_CHECK();
    return MBIR_OK;
  }
  BatchLaunch L;
  L.dargs = static_cast<unsigned char*>(dbuf_) + g.arg_off;
  L.doff = reinterpret_cast<const int*>(static_cast<unsigned char*>(dbuf_) + g.off_off);
  L.n = g.n;
  L.total = g.total;
  L.smem = g.smem;
  L.host0 = hbuf_ + g.arg_off;
  L.set_mu = g.uses_mu;
  L.mu = mu;
  L.blu = g.blu;
  L.fz = g.fz;
  switch (g.kind) {
    case 0: return batch_lateral(g.mode, prec_, L, st_);
    case 1: return batch_row(g.mode, prec_, J_, L, st_);
    case 2: return batch_dwt(0, g.mode, prec_, L, st_);
    default: return batch_dwt(1, g.mode, prec_, L, st_);
  }
}

int Engine::vec_kernel(int which, size_t off, int n) {
  dim3 grid(kBBlocks, n);
  const ScanVec* d = reinterpret_cast<const ScanVec*>(static_cast<unsigned char*>(dbuf_) + off);
  const bool f64 = prec_ == MBIR_FP64;
  switch (which) {
    case 0: f64 ? launch(b_fill_hash<double>, grid, dim3(kBThreads), 0, st_, d)
                : launch(b_fill_hash<float>, grid, dim3(kBThreads), 0, st_, d); break;
    case 1: f64 ? launch(b_dot_norm<double>, grid, dim3(kBThreads), 0, st_, d)
                : launch(b_dot_norm<float>, grid, dim3(kBThreads), 0, st_, d); break;
    case 2: launch(b_power_finalize, dim3(1, n), dim3(kBThreads), 0, st_, d, kBBlocks); break;
    case 3: f64 ? launch(b_scale<double>, grid, dim3(kBThreads), 0, st_, d)
                : launch(b_scale<float>, grid, dim3(kBThreads), 0, st_, d); break;
    case 4: f64 ? launch(b_maxabs<double>, grid, dim3(kBThreads), 0, st_, d)
                : launch(b_maxabs<float>, grid, dim3(kBThreads), 0, st_, d); break;
    default: launch(b_max_finalize, dim3(1, n), dim3(kBThreads), 0, st_, d, kBBlocks); break;
  }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

int Engine::setup(const std::vector<BScan*>& scans) {
  if (scans.empty()) return MBIR_OK;
  int rc = check(scans);
  if (rc) return rc;
  std::vector<BScan*> pw, lm, lm_db4;
  for (BScan* s : scans) {
    if (!(s->o.step > 0)) pw.push_back(s);
    if (s->o.lambda_is_relative) {
      lm.push_back(s);
      if (s->o.penalty == MBIR_PENALTY_DB4) lm_db4.push_back(s);
    }
  }
  if ((rc = begin_build())) return rc;
  std::vector<Stage> pst, lst;
  size_t v_self = 0, v_pair = 0, v_lam = 0;
  if (!pw.empty()) {
    // power iteration: w = start, then v = w/||w||, w = Phi^H s Phi v per step
    if ((rc = add_lateral(pst, LAT_POWER_FWD, pw, [](BScan& s) {
           LatFill f = lfill(s.c.zA, s.c.wsA, nullptr, s.p->nz, 1.0);
           f.vout = s.c.v;
           f.scal = s.c.scal;
           return f; }, false)))
      return rc;
    if ((rc = add_row(pst, false, pw))) return rc;
    if ((rc = add_lateral(pst, LAT_POWER_MID, pw, [](BScan& s) { return lfill(s.c.wsB, s.c.wsA, s.mask, s.p->m, 1.0 / s.p->nx); }, false))) return rc;
    if ((rc = add_row(pst, true, pw))) return rc;
    if ((rc = add_lateral(pst, LAT_POWER_ADJ, pw, [](BScan& s) {
           LatFill f = lfill(s.c.wsB, s.c.zA, nullptr, s.p->nz, 1.0);
           f.z1 = s.c.v;
           f.partial = s.c.part_tmp;
           return f; }, false)))
      return rc;
    std::vector<ScanVec> a, b;
    for (BScan* s : pw) {
      a.push_back({s->c.zA, s->c.zA, s->c.nimg, s->c.part_tmp, s->c.scal, 0});
      b.push_back({s->c.v, s->c.zA, s->c.nimg, s->c.part_tmp, s->c.scal, lateral_grid(s->p, s->p->nz)});
    }
    v_self = push(a.data(), a.size() * sizeof(ScanVec));
    v_pair = push(b.data(), b.size() * sizeof(ScanVec));
  }
  if (!lm.empty()) {
    if ((rc = add_lateral(lst, LAT_R2C_MASK, lm, [](BScan& s) { return lfill(s.y, s.c.wsA, s.mask, s.p->m, 1.0 / s.p->nx); }, false))) return rc;
    if ((rc = add_row(lst, true, lm))) return rc;
    if ((rc = add_lateral(lst, LAT_C2C_INV, lm, [](BScan& s) { return lfill(s.c.wsB, s.c.zA, nullptr, s.p->nz, 1.0); }, false))) return rc;
    if (!lm_db4.empty()) {
      // full analysis (no threshold) of Phi^H s y into v
      std::vector<const void*> in;
      std::vector<void*> coefs;
      for (BScan* s : lm_db4) {
        in.push_back(s->c.zA);
        coefs.push_back(s->c.v);
      }
      for (int lev = 0; lev < 3; ++lev)
        if ((rc = add_dwt(lst, 0, lev, lm_db4, in, {}, coefs, {}, false))) return rc;
    }
    std::vector<ScanVec> a;
    for (BScan* s : lm)
      a.push_back({s->o.penalty == MBIR_PENALTY_DB4 ? s->c.v : s->c.zA, nullptr, s->c.nimg, s->c.part_tmp, s->c.scal, 0});
    v_lam = push(a.data(), a.size() * sizeof(ScanVec));
  }
  if ((rc = upload())) return rc;
  if (!pw.empty()) {
    const int np = (int)pw.size();
    for (int w : {0, 1, 2})
      if ((rc = vec_kernel(w, v_self, np))) return rc;
    int iters = 0;
    for (BScan* s : pw) iters = std::max(iters, s->o.power_iters > 0 ? s->o.power_iters : 30);
    for (int it = 0; it < iters; ++it) {
      for (const Stage& g : pst)
        if ((rc = run(g, 0.0))) return rc;
      if ((rc = vec_kernel(2, v_pair, np))) return rc;
    }
  }
  if (!lm.empty()) {
    for (const Stage& g : lst)
      if ((rc = run(g, 0.0))) return rc;
    for (int w : {4, 5})
      if ((rc = vec_kernel(w, v_lam, (int)lm.size()))) return rc;
  }
  std::vector<double> hs(8 * scans.size(), 0.0);
  for (size_t i = 0; i < scans.size(); ++i)
    MBIR_CUDA_TRY(cudaMemcpyAsync(&hs[8 * i], scans[i]->c.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st_));
  MBIR_CUDA_TRY(cudaStreamSynchronize(st_));
  for (size_t i = 0; i < scans.size(); ++i) {
    BScan& s = *scans[i];
    s.L = 0.0;
    s.delta = s.o.step;
    if (!(s.delta > 0)) {
      s.L = hs[8 * i + 0];
      if (!(s.L > 0) || !isfinite(s.L)) return MBIR_ERR_INVALID;
      s.delta = 1.0 / (1.01 * s.L);
    }
    s.lam = s.o.lambda * (s.o.lambda_is_relative ? hs[8 * i + 4] : 1.0);
    s.tau = s.lam * s.delta;
    s.k = 0;
    s.f1 = s.f2 = 0.0;
    MBIR_CUDA_TRY(cudaMemsetAsync(s.c.pz, 0, rsz_ * s.c.nmeas, st_));
    MBIR_CUDA_TRY(cudaMemsetAsync(s.c.part_reg, 0, sizeof(double) * s.c.n_reg, st_));
    if (s.o.warm_start) {
      MBIR_CUDA_TRY(cudaMemcpyAsync(s.c.zA, s.x, esz_ * s.c.nimg, cudaMemcpyDeviceToDevice, st_));
      MBIR_CUDA_TRY(cudaMemcpyAsync(s.c.zB, s.x, esz_ * s.c.nimg, cudaMemcpyDeviceToDevice, st_));
    } else {
      MBIR_CUDA_TRY(cudaMemsetAsync(s.c.zA, 0, esz_ * s.c.nimg, st_));
      MBIR_CUDA_TRY(cudaMemsetAsync(s.c.zB, 0, esz_ * s.c.nimg, st_));
    }
  }
  return MBIR_OK;
}

static double momentum(int k) {
  // mu_{k-1} = (t^{k-1} - 1)/t^k used in iteration k (mu_0 = 0), t^1 = 1
  if (k < 2) return 0.0;
  double t = 1.0, tn = 1.0;
  for (int i = 1; i < k; ++i) {
    tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    if (i < k - 1) t = tn;
  }
  return (t - 1.0) / tn;
}

// Stages of one FISTA iteration.  parity_override >= 0 fixes which buffer holds
// z^{k-1} for every scan (the graph-captured loop); otherwise each scan's own k
// decides, and with per_scan_mu the momentum of its own k goes into its block.
int Engine::build_iteration(std::vector<Stage>& out, const std::vector<BScan*>& scans, int parity_override,
                            bool per_scan_mu, bool want_obj) {
  std::vector<BScan*> l1, db4;
  for (BScan* s : scans) (s->o.penalty == MBIR_PENALTY_L1 ? l1 : db4).push_back(s);
  auto par = [&](const BScan& s) { return parity_override >= 0 ? parity_override : (s.k & 1); };
  auto z1 = [&](const BScan& s) { return par(s) == 0 ? s.c.zA : s.c.zB; };
  auto z2 = [&](const BScan& s) { return par(s) == 0 ? s.c.zB : s.c.zA; };
  auto mu_of = [&](const BScan& s) { return per_scan_mu ? momentum(s.k + 1) : 0.0; };
  int rc;
  if ((rc = add_lateral(out, LAT_C2C_FWD, scans, [&](BScan& s) { return lfill(z1(s), s.c.wsA, nullptr, s.p->nz, 1.0); }, false))) return rc;
  if ((rc = add_row(out, false, scans))) return rc;
  if ((rc = add_lateral(out, LAT_SOLVE_MID, scans, [&](BScan& s) {
         LatFill f = lfill(s.c.wsB, s.c.wsA, s.mask, s.p->m, 1.0 / s.p->nx);
         f.y = s.y;
         f.pz = s.c.pz;
         f.partial = s.c.part_data;
         f.mu = mu_of(s);
         return f; }, !per_scan_mu)))
    return rc;
  if (want_obj) {
    if (dobj_cap_ < (int)scans.size()) {
      cudaFree(dobj_);
      dobj_ = nullptr;
      const int cap = std::max((int)scans.size(), 2 * dobj_cap_);
      MBIR_CUDA_TRY(cudaMalloc(&dobj_, sizeof(double) * cap));
      dobj_cap_ = cap;
    }
    std::vector<ObjArgs> oa;
    for (size_t i = 0; i < scans.size(); ++i) {
      BScan& s = *scans[i];
      s.slot = (int)i;
      const int nreg = s.o.penalty == MBIR_PENALTY_L1 ? lateral_grid(s.p, s.p->nz)
                                                      : wavelet_partial_count(s.p->nx, s.p->nz);
      oa.push_back({s.c.part_data, s.c.n_data, s.c.part_reg, nreg, s.lam,
                    s.k < s.c.trace_cap ? s.c.objtrace + s.k : nullptr, dobj_ + i});
    }
    Stage g{4, 0, 0, 0, (int)scans.size(), 0, 0, 0};
    g.arg_off = push(oa.data(), oa.size() * sizeof(ObjArgs));
    out.push_back(g);
  }
  if ((rc = add_row(out, true, scans))) return rc;
  if ((rc = add_lateral(out, LAT_SOLVE_ADJ_L1, l1, [&](BScan& s) {
         LatFill f = lfill(s.c.wsB, nullptr, nullptr, s.p->nz, 1.0);
         f.z1 = z1(s);
         f.z2 = z2(s);
         f.delta = s.delta;
         f.tau = s.tau;
         f.mu = mu_of(s);
         f.partial = s.c.part_reg;
         return f; }, !per_scan_mu)))
    return rc;
  if ((rc = add_lateral(out, LAT_SOLVE_ADJ_V, db4, [&](BScan& s) {
         LatFill f = lfill(s.c.wsB, nullptr, nullptr, s.p->nz, 1.0);
         f.z1 = z1(s);
         f.z2 = z2(s);
         f.vout = s.c.v;
         f.delta = s.delta;
         f.tau = s.tau;
         f.mu = mu_of(s);
         return f; }, !per_scan_mu)))
    return rc;
  if (!db4.empty()) {
    std::vector<const void*> in;
    std::vector<void*> outs, coefs;
    std::vector<double*> parts[3];
    for (BScan* s : db4) {
      in.push_back(s->c.v);
      outs.push_back(z2(*s));
      coefs.push_back(s->c.wv_coef);
      double* pr = s->c.part_reg;
      int P = s->p->nx, N = s->p->nz;
      for (int lev = 0; lev < 3; ++lev) {
        parts[lev].push_back(pr);
        pr += dwt_level_ctas(P, N, 0, lev);
        P /= 2;
        N /= 2;
      }
    }
    for (int lev = 0; lev < 3; ++lev)
      if ((rc = add_dwt(out, 0, lev, db4, in, {}, coefs, parts[lev], true))) return rc;
    for (int lev = 2; lev >= 0; --lev)
      if ((rc = add_dwt(out, 1, lev, db4, {}, outs, coefs, {}, false))) return rc;
  }
  return MBIR_OK;
}

int Engine::step(const std::vector<BScan*>& scans, bool want_obj) {
  if (scans.empty()) return MBIR_OK;
  int rc = check(scans);
  if (rc) return rc;
  if ((rc = begin_build())) return rc;
  std::vector<Stage> st;
  if ((rc = build_iteration(st, scans, -1, true, want_obj))) return rc;
  if ((rc = upload())) return rc;
  for (const Stage& g : st)
    if ((rc = run(g, 0.0))) return rc;
  for (BScan* s : scans) s->k += 1;
  return MBIR_OK;
}

int Engine::read_objectives(const std::vector<BScan*>& scans) {
  if (scans.empty()) return MBIR_OK;
  hobj_.resize(scans.size());
  MBIR_CUDA_TRY(cudaMemcpyAsync(hobj_.data(), dobj_, sizeof(double) * scans.size(), cudaMemcpyDeviceToHost, st_));
  MBIR_CUDA_TRY(cudaStreamSynchronize(st_));
  for (BScan* s : scans) {
    s->f2 = s->f1;
    s->f1 = hobj_[s->slot];
  }
  return MBIR_OK;
}

int Engine::solve_fixed(const std::vector<BScan*>& scans) {
  int rc = check(scans);
  if (rc) return rc;
  const int kmax = scans[0]->o.max_iter;
  for (BScan* s : scans)
    if (s->o.max_iter != kmax) return MBIR_ERR_INVALID;
  if ((rc = begin_build())) return rc;
  std::vector<Stage> it[2];
  for (int par = 0; par < 2; ++par)
    if ((rc = build_iteration(it[par], scans, par, false, false))) return rc;
  if ((rc = upload())) return rc;
  std::vector<double> mu(kmax + 2, 0.0);
  {
    double t = 1.0;
    for (int k = 0; k <= kmax; ++k) {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      mu[k] = (t - 1.0) / tn;
      t = tn;
    }
  }
  auto iterate = [&]() -> int {
    for (int k = 1; k <= kmax; ++k) {
      const double m = k >= 2 ? mu[k - 2] : 0.0;
      for (const Stage& g : it[(k - 1) & 1]) {
        const int r = run(g, m);
        if (r) return r;
      }
    }
    return MBIR_OK;
  };
  if (st_ != nullptr && st_ != cudaStreamLegacy && st_ != cudaStreamPerThread) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    MBIR_CUDA_TRY(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
    rc = iterate();
    cudaError_t e = cudaStreamEndCapture(st_, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return set_cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return set_cuda_error(e, "cudaGraphInstantiate");
    }
    e = cudaGraphLaunch(exec, st_);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGraphLaunch");
  } else if ((rc = iterate())) {
    return rc;
  }
  for (BScan* s : scans) s->k = kmax;
  return MBIR_OK;
}

int Engine::finish(BScan* s) {
  // z^k lives in zA when k is even, zB when odd
  void* zlast = (s->k & 1) ? s->c.zB : s->c.zA;
  MBIR_CUDA_TRY(cudaMemcpyAsync(s->x, zlast, esz_ * s->c.nimg, cudaMemcpyDeviceToDevice, st_));
  return MBIR_OK;
}

}  // namespace mbir

namespace mbir {

// A scan runs its own stages inside a batch when its row kernels alone give every
// SM at least three CTAs (nx/2 + 1 row pairs).
static bool runs_alone(mbir_plan p, int sms) { return p->nx / 2 + 1 >= 3 * sms; }

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_solve_batch(mbir_plan* plans, int32_t n, const void* const* y, const uint8_t* const* mask,
                     const mbir_solve_opts* opts, void* const* x, mbir_solve_info* info, void* stream) {
  if (!plans || n < 1 || !y || !opts || !x) return MBIR_ERR_INVALID;
  for (int i = 0; i < n; ++i)
    if (const int vrc = bscan_only(plans[i], "mbir_solve_batch")) return vrc;
  std::vector<BScan> scans(n);
  std::vector<BScan*> ptrs(n);
  for (int i = 0; i < n; ++i) {
    const mbir_solve_opts& o = opts[i];
    if (!plans[i] || !y[i] || !x[i]) return MBIR_ERR_INVALID;
    if (o.max_iter < 1 || o.penalty < MBIR_PENALTY_L1 || o.penalty > MBIR_PENALTY_DB4) return MBIR_ERR_INVALID;
    if (o.backprojection != MBIR_BACKPROJ_TRANSPOSE) return MBIR_ERR_INVALID;
    if (!(o.lambda >= 0) || !isfinite(o.lambda) || !isfinite(o.step) || o.rel_tol != 0.0) return MBIR_ERR_INVALID;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return MBIR_ERR_INVALID;   // each plan once: its buffers are per scan
    BScan& s = scans[i];
    s.p = plans[i];
    s.y = y[i];
    s.mask = mask ? mask[i] : nullptr;
    s.x = x[i];
    s.o = o;
    int rc = plan_ctx(s.p, o.penalty, o.max_iter, &s.c);
    if (rc) return rc;
    ptrs[i] = &s;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // Scans whose own row stage fills every SM several times run the single-scan
  // path: batching them only adds the batched kernels' per-CTA cost (argument
  // blocks in device memory, fewer resident warps), which outweighs the wave tails
  // it fills.  The other scans share batched stages on a second stream, where they
  // fill the idle SMs of the large scans' launches.  A scan's path depends on its
  // own size only, so its result does not depend on the rest of the batch.
  int dev = 0, sms = 0;
  MBIR_CUDA_TRY(cudaGetDevice(&dev));
  MBIR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  std::vector<BScan*> shared;
  std::vector<int> alone;
  for (int i = 0; i < n; ++i) {
    if (runs_alone(plans[i], sms)) alone.push_back(i);
    else shared.push_back(ptrs[i]);
  }
  // two created streams forked from `stream`: the large scans on a high-priority
  // one, the shared batch on another; the legacy and per-thread default streams
  // run everything on `stream`, one after the other
  const bool fork = !alone.empty() && !shared.empty() && st != nullptr && st != cudaStreamLegacy &&
                    st != cudaStreamPerThread;
  cudaStream_t sa = st, sb = st;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  auto release = [&]() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (sa != st) cudaStreamDestroy(sa);
    if (sb != st) cudaStreamDestroy(sb);
  };
  if (fork) {
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sa, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sb, cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sa, ev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sb, ev[0], 0);
    if (e != cudaSuccess) {
      release();
      return set_cuda_error(e, "mbir_solve_batch: streams");
    }
  }
  int rc = MBIR_OK;
  std::vector<mbir_solve_info> solo_info(alone.size());
  {
    Engine eng(sb);
    if (!shared.empty()) {
      // set-up (one read-back), then the captured iteration loop, queued on sb
      rc = eng.setup(shared);
      if (!rc) rc = eng.solve_fixed(shared);
      for (size_t i = 0; !rc && i < shared.size(); ++i) rc = eng.finish(shared[i]);
    }
    // the large scans on sa while the shared batch runs
    for (size_t j = 0; !rc && j < alone.size(); ++j) {
      const int i = alone[j];
      memset(&solo_info[j], 0, sizeof(mbir_solve_info));
      rc = solve_plan(plans[i], y[i], mask ? mask[i] : nullptr, &opts[i], x[i], info ? &solo_info[j] : nullptr, sa,
                      false);
    }
    if (fork) {
      cudaError_t e = cudaEventRecord(ev[1], sa);
      if (e == cudaSuccess) e = cudaEventRecord(ev[2], sb);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1], 0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[2], 0);
      if (e != cudaSuccess && !rc) rc = set_cuda_error(e, "mbir_solve_batch: join");
    }
    if (!rc && info) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = set_cuda_error(e, "cudaStreamSynchronize");
    }
  }
  release();
  if (rc) return rc;
  if (info) {
    for (int i = 0; i < n; ++i) {
      info[i].iters = scans[i].k;
      info[i].status = MBIR_OK;
      info[i].objective = NAN;
      info[i].lipschitz = scans[i].L;
      info[i].step = scans[i].delta;
      info[i].lambda_used = scans[i].lam;
    }
    for (size_t j = 0; j < alone.size(); ++j) {
      mbir_solve_info& d = info[alone[j]];
      const mbir_solve_info& s = solo_info[j];
      d.iters = s.iters;
      d.status = s.status;
      d.objective = NAN;
      d.lipschitz = s.lipschitz;
      d.step = s.step;
      d.lambda_used = s.lambda_used;
    }
  }
  return MBIR_OK;
}

}  // extern "C"
