// Batched reconstruction of several B-scans of different sizes (one plan each):
// every stage of the path -- the operator passes, the FISTA epilogues, the
// wavelet levels, the power iteration and the lambda rule -- runs as ONE launch
// over all scans, each CTA finding its scan from a prefix table of CTA offsets.
// The FISTA loop (Sec. 2.3, Eq. alg) is captured once into a CUDA graph and
// replayed.  A scan runs exactly the same kernel code whatever it is batched
// with (the adjoint gather is deterministic), so its result does not depend on
// the mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "operator.cuh"
#include "solve_state.cuh"

namespace mbir {

constexpr int kBThreads = 256;
constexpr int kBBlocks = 64;    // CTAs per scan of the batched vector kernels

// Per-scan operands of the batched vector kernels.
struct ScanVec {
  void* v;
  void* w;
  size_t n;
  double* part;   // 2 * kBBlocks doubles
  double* scal;   // scalars
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
  const ScanVec s = sv[blockIdx.y];
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
  const ScanVec s = sv[blockIdx.y];
  const cplx_t<R>* v = reinterpret_cast<const cplx_t<R>*>(s.v);
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < s.n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> a = v[i];
    m = fmax(m, sqrt(double(a.x) * double(a.x) + double(a.y) * double(a.y)));
  }
  const double M = bmax(m);
  if (threadIdx.x == 0) s.part[blockIdx.x] = M;
}

__global__ void b_max_finalize(const ScanVec* sv, int nb) {
  const ScanVec s = sv[blockIdx.y];
  double m = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, s.part[i]);
  const double M = bmax(m);
  if (threadIdx.x == 0) s.scal[4] = M;
}

// ------------------------------------------------------------------ engine

struct BScan {
  mbir_plan p;
  const void* y;
  const uint8_t* mask;
  void* x;
  mbir_solve_opts o;
  double L, lam, delta, tau;
};

class Engine {
 public:
  Engine(std::vector<BScan>& scans, cudaStream_t st) : sc_(scans), st_(st) {}
  ~Engine() {
    cudaFree(dbuf_);
    cudaFreeHost(hbuf_);
  }

  int prepare() {
    prec_ = sc_[0].p->precision;
    J_ = sc_[0].p->J;
    gather_ = true;
    for (auto& s : sc_) {
      if (s.p->precision != prec_ || s.p->J != J_ || s.p->alpha != sc_[0].p->alpha) return MBIR_ERR_INVALID;
      if (s.p->device != sc_[0].p->device) return MBIR_ERR_INVALID;
      gather_ = gather_ && plan_uses_gather(s.p);
      int rc = ensure_state(s.p, s.o.max_iter);
      if (rc) return rc;
      if (s.o.penalty == MBIR_PENALTY_DB4) {
        if (!wavelet_supported(s.p->nx, s.p->nz)) return MBIR_ERR_UNSUPPORTED_SIZE;
        rc = ensure_wavelet_scratch(s.p);
        if (rc) return rc;
      }
    }
    esz_ = prec_ == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
    rsz_ = prec_ == MBIR_FP64 ? sizeof(double) : sizeof(float);
    return MBIR_OK;
  }

  // ---- stage recording: argument blocks are appended to a host staging buffer,
  // uploaded once, then launched from the device copy.
  struct Stage {
    int kind;   // 0 lateral, 1 row, 2 dwt analysis, 3 dwt synthesis
    int mode;   // lateral mode / row kind
    size_t arg_off, off_off;
    int n, total;
    size_t smem;
    int uses_mu;
  };

  size_t push(const void* data, size_t bytes) {
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

  void grow(size_t need) {
    size_t cap = hcap_ ? hcap_ : (1 << 16);
    while (cap < need) cap *= 2;
    unsigned char* nb = nullptr;
    if (cudaMallocHost(&nb, cap) != cudaSuccess) {
      nb = nullptr;
      grow_failed_ = true;
      return;
    }
    if (hbuf_) {
      memcpy(nb, hbuf_, hlen_);
      cudaFreeHost(hbuf_);
    }
    hbuf_ = nb;
    hcap_ = cap;
  }

  // lateral stage over the scans `idx`
  template <class F>
  int add_lateral(std::vector<Stage>& out, int mode, const std::vector<int>& idx, F make, bool uses_mu) {
    if (idx.empty()) return MBIR_OK;
    const size_t ab = lat_args_bytes(prec_);
    std::vector<unsigned char> blocks(ab * idx.size());
    std::vector<int> off(idx.size() + 1, 0);
    size_t smem = 0;
    for (size_t i = 0; i < idx.size(); ++i) {
      BScan& s = sc_[idx[i]];
      LatFill f = make(s);
      fill_lat_args(s.p, f, blocks.data() + i * ab);
      off[i + 1] = off[i] + lateral_grid(s.p, f.cols);
      smem = std::max(smem, lat_smem_bytes(s.p));
    }
    Stage g{0, mode, 0, 0, (int)idx.size(), off.back(), smem, uses_mu ? 1 : 0};
    g.arg_off = push(blocks.data(), blocks.size());
    g.off_off = push(off.data(), off.size() * sizeof(int));
    out.push_back(g);
    return grow_failed_ ? MBIR_ERR_OOM : MBIR_OK;
  }

  int add_row(std::vector<Stage>& out, bool adjoint, const std::vector<int>& idx, int in_ws /*0: A->B*/) {
    if (idx.empty()) return MBIR_OK;
    const size_t ab = row_args_bytes(prec_);
    std::vector<unsigned char> blocks(ab * idx.size());
    std::vector<int> off(idx.size() + 1, 0);
    size_t smem = 0;
    const int kind = adjoint ? (gather_ ? 1 : 2) : 0;
    for (size_t i = 0; i < idx.size(); ++i) {
      BScan& s = sc_[idx[i]];
      fill_row_args(s.p, in_ws == 0 ? s.p->wsA : s.p->wsB, in_ws == 0 ? s.p->wsB : s.p->wsA,
                    blocks.data() + i * ab);
      off[i + 1] = off[i] + s.p->nx;
      smem = std::max(smem, row_smem_bytes(s.p, kind == 1));
    }
    Stage g{1, kind, 0, 0, (int)idx.size(), off.back(), smem, 0};
    g.arg_off = push(blocks.data(), blocks.size());
    g.off_off = push(off.data(), off.size() * sizeof(int));
    out.push_back(g);
    return grow_failed_ ? MBIR_ERR_OOM : MBIR_OK;
  }

  // one wavelet level over the scans `idx`
  int add_dwt(std::vector<Stage>& out, int inverse, int level, const std::vector<int>& idx,
              const void* const* in, void* const* outp, double* const* partial, bool thresh) {
    if (idx.empty()) return MBIR_OK;
    const size_t ab = dwt_args_bytes(prec_);
    std::vector<unsigned char> blocks(ab * idx.size());
    std::vector<int> off(idx.size() + 1, 0);
    for (size_t i = 0; i < idx.size(); ++i) {
      BScan& s = sc_[idx[i]];
      const int th = thresh ? (level == 2 ? 2 : 1) : 0;
      fill_dwt_args(s.p, level, inverse, in ? in[i] : nullptr, outp ? outp[i] : nullptr, s.p->wv_coef,
                    thresh ? s.tau : 0.0, th, partial ? partial[i] : nullptr, blocks.data() + i * ab);
      off[i + 1] = off[i] + dwt_level_ctas(s.p->nx >> level, s.p->nz >> level, inverse);
    }
    Stage g{inverse ? 3 : 2, 0, 0, 0, (int)idx.size(), off.back(), dwt_smem_bytes(prec_, inverse), 0};
    g.arg_off = push(blocks.data(), blocks.size());
    g.off_off = push(off.data(), off.size() * sizeof(int));
    out.push_back(g);
    return grow_failed_ ? MBIR_ERR_OOM : MBIR_OK;
  }

  int upload() {
    if (hlen_ > dcap_) {
      cudaFree(dbuf_);
      dbuf_ = nullptr;
      MBIR_CUDA_TRY(cudaMalloc(&dbuf_, hlen_));
      dcap_ = hlen_;
    }
    MBIR_CUDA_TRY(cudaMemcpyAsync(dbuf_, hbuf_, hlen_, cudaMemcpyHostToDevice, st_));
    return MBIR_OK;
  }

  int run(const Stage& g, double mu) {
    BatchLaunch L;
    L.dargs = static_cast<unsigned char*>(dbuf_) + g.arg_off;
    L.doff = reinterpret_cast<const int*>(static_cast<unsigned char*>(dbuf_) + g.off_off);
    L.n = g.n;
    L.total = g.total;
    L.smem = g.smem;
    L.host0 = hbuf_ + g.arg_off;
    L.set_mu = g.uses_mu;
    L.mu = mu;
    switch (g.kind) {
      case 0: return batch_lateral(g.mode, prec_, L, st_);
      case 1: return batch_row(g.mode, prec_, J_, L, st_);
      case 2: return batch_dwt(0, prec_, L, st_);
      default: return batch_dwt(1, prec_, L, st_);
    }
  }

  size_t push_scanvec(const std::vector<ScanVec>& v) { return push(v.data(), v.size() * sizeof(ScanVec)); }
  const ScanVec* dvec(size_t off) const {
    return reinterpret_cast<const ScanVec*>(static_cast<unsigned char*>(dbuf_) + off);
  }

  int vec_kernel(int which, size_t off, int n) {
    dim3 grid(kBBlocks, n);
    const ScanVec* d = dvec(off);
    const bool f64 = prec_ == MBIR_FP64;
    switch (which) {
      case 0: f64 ? b_fill_hash<double><<<grid, kBThreads, 0, st_>>>(d) : b_fill_hash<float><<<grid, kBThreads, 0, st_>>>(d); break;
      case 1: f64 ? b_dot_norm<double><<<grid, kBThreads, 0, st_>>>(d) : b_dot_norm<float><<<grid, kBThreads, 0, st_>>>(d); break;
      case 2: b_power_finalize<<<dim3(1, n), kBThreads, 0, st_>>>(d, kBBlocks); break;
      case 3: f64 ? b_scale<double><<<grid, kBThreads, 0, st_>>>(d) : b_scale<float><<<grid, kBThreads, 0, st_>>>(d); break;
      case 4: f64 ? b_maxabs<double><<<grid, kBThreads, 0, st_>>>(d) : b_maxabs<float><<<grid, kBThreads, 0, st_>>>(d); break;
      default: b_max_finalize<<<dim3(1, n), kBThreads, 0, st_>>>(d, kBBlocks); break;
    }
    MBIR_LAUNCH_CHECK();
    return MBIR_OK;
  }

  // ---- the solve
  int solve() {
    const int n = (int)sc_.size();
    std::vector<int> all(n), pow_idx, lam_idx, l1_idx, db4_idx;
    for (int i = 0; i < n; ++i) {
      all[i] = i;
      if (!(sc_[i].o.step > 0)) pow_idx.push_back(i);
      if (sc_[i].o.lambda_is_relative) lam_idx.push_back(i);
      (sc_[i].o.penalty == MBIR_PENALTY_L1 ? l1_idx : db4_idx).push_back(i);
    }
    int rc;
    // ---------------- set-up: power iteration and lambda, batched
    std::vector<Stage> pw, lm;
    size_t pw_vec = 0, lm_vec = 0, lm_vec2 = 0;
    if (!pow_idx.empty()) {
      rc = add_lateral(pw, LAT_C2C_FWD, pow_idx, [&](BScan& s) {
        return fill(s.p, s.p->solve->v, s.p->wsA, nullptr, s.p->nz, 1.0); }, false);
      if (rc) return rc;
      if ((rc = add_row(pw, false, pow_idx, 0))) return rc;
      rc = add_lateral(pw, LAT_C2R_INV_MASK, pow_idx, [&](BScan& s) {
        return fill(s.p, s.p->wsB, s.p->solve->r, s.mask, s.p->m, 1.0 / s.p->nx); }, false);
      if (rc) return rc;
      rc = add_lateral(pw, LAT_R2C_MASK, pow_idx, [&](BScan& s) {
        return fill(s.p, s.p->solve->r, s.p->wsA, s.mask, s.p->m, 1.0 / s.p->nx); }, false);
      if (rc) return rc;
      if ((rc = add_row(pw, true, pow_idx, 0))) return rc;
      rc = add_lateral(pw, LAT_C2C_INV, pow_idx, [&](BScan& s) {
        return fill(s.p, s.p->wsB, s.p->solve->zA, nullptr, s.p->nz, 1.0); }, false);
      if (rc) return rc;
      std::vector<ScanVec> vv, vw;
      for (int i : pow_idx) {
        SolveState* S = sc_[i].p->solve;
        vv.push_back({S->v, S->v, S->nimg, S->part_tmp, S->scal});
        vw.push_back({S->v, S->zA, S->nimg, S->part_tmp, S->scal});
      }
      pw_vec = push_scanvec(vv);
      lm_vec2 = push_scanvec(vw);   // (v, w) pairs
    }
    if (!lam_idx.empty()) {
      rc = add_lateral(lm, LAT_R2C_MASK, lam_idx, [&](BScan& s) {
        return fill(s.p, s.y, s.p->wsA, s.mask, s.p->m, 1.0 / s.p->nx); }, false);
      if (rc) return rc;
      if ((rc = add_row(lm, true, lam_idx, 0))) return rc;
      rc = add_lateral(lm, LAT_C2C_INV, lam_idx, [&](BScan& s) {
        return fill(s.p, s.p->wsB, s.p->solve->zA, nullptr, s.p->nz, 1.0); }, false);
      if (rc) return rc;
      std::vector<int> lam_db4;
      for (int i : lam_idx)
        if (sc_[i].o.penalty == MBIR_PENALTY_DB4) lam_db4.push_back(i);
      std::vector<const void*> ins;
      std::vector<void*> outs;
      for (int i : lam_db4) {
        ins.push_back(sc_[i].p->solve->zA);
        outs.push_back(sc_[i].p->solve->v);
      }
      for (int lev = 0; lev < 3; ++lev) {
        // analysis without threshold; the last level's low-low block lands in v
        std::vector<void*> coefs;
        for (size_t q = 0; q < lam_db4.size(); ++q) coefs.push_back(outs[q]);
        rc = add_dwt_coef(lm, lev, lam_db4, ins.data(), coefs.data());
        if (rc) return rc;
      }
      std::vector<ScanVec> vm;
      for (int i : lam_idx) {
        SolveState* S = sc_[i].p->solve;
        vm.push_back({sc_[i].o.penalty == MBIR_PENALTY_DB4 ? S->v : S->zA, nullptr, S->nimg, S->part_tmp, S->scal});
      }
      lm_vec = push_scanvec(vm);
    }
    if ((rc = upload())) return rc;
    if (!pow_idx.empty()) {
      const int np = (int)pow_idx.size();
      if ((rc = vec_kernel(0, pw_vec, np))) return rc;
      if ((rc = vec_kernel(1, pw_vec, np))) return rc;
      if ((rc = vec_kernel(2, pw_vec, np))) return rc;
      if ((rc = vec_kernel(3, pw_vec, np))) return rc;
      int iters = 0;
      for (int i : pow_idx) iters = std::max(iters, sc_[i].o.power_iters > 0 ? sc_[i].o.power_iters : 30);
      for (int it = 0; it < iters; ++it) {
        for (const Stage& g : pw)
          if ((rc = run(g, 0.0))) return rc;
        if ((rc = vec_kernel(1, lm_vec2, np))) return rc;
        if ((rc = vec_kernel(2, lm_vec2, np))) return rc;
        if ((rc = vec_kernel(3, lm_vec2, np))) return rc;
      }
    }
    if (!lam_idx.empty()) {
      for (const Stage& g : lm)
        if ((rc = run(g, 0.0))) return rc;
      if ((rc = vec_kernel(4, lm_vec, (int)lam_idx.size()))) return rc;
      if ((rc = vec_kernel(5, lm_vec, (int)lam_idx.size()))) return rc;
    }
    // read the scalars back (one sync for the whole batch)
    std::vector<double> hs(n * 8, 0.0);
    for (int i = 0; i < n; ++i)
      MBIR_CUDA_TRY(cudaMemcpyAsync(&hs[8 * i], sc_[i].p->solve->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st_));
    MBIR_CUDA_TRY(cudaStreamSynchronize(st_));
    for (int i = 0; i < n; ++i) {
      BScan& s = sc_[i];
      s.L = 0.0;
      s.delta = s.o.step;
      if (!(s.delta > 0)) {
        s.L = hs[8 * i + 0];
        if (!(s.L > 0) || !isfinite(s.L)) return MBIR_ERR_INVALID;
        s.delta = 1.0 / (1.01 * s.L);
      }
      s.lam = s.o.lambda * (s.o.lambda_is_relative ? hs[8 * i + 4] : 1.0);
      s.tau = s.lam * s.delta;
    }
    // ---------------- the FISTA iterations: stages for both parities of (z1, z2)
    hlen_ = 0;
    std::vector<Stage> it[2];
    for (int par = 0; par < 2; ++par) {
      auto z1 = [&](BScan& s) { return par == 0 ? s.p->solve->zA : s.p->solve->zB; };
      auto z2 = [&](BScan& s) { return par == 0 ? s.p->solve->zB : s.p->solve->zA; };
      rc = add_lateral(it[par], LAT_C2C_FWD, all, [&](BScan& s) {
        return fill(s.p, z1(s), s.p->wsA, nullptr, s.p->nz, 1.0); }, false);
      if (rc) return rc;
      if ((rc = add_row(it[par], false, all, 0))) return rc;
      rc = add_lateral(it[par], LAT_SOLVE_FWD, all, [&](BScan& s) {
        LatFill f = fill(s.p, s.p->wsB, nullptr, s.mask, s.p->m, 1.0 / s.p->nx);
        f.y = s.y;
        f.pz = s.p->solve->pz;
        f.r = s.p->solve->r;
        f.partial = s.p->solve->part_data;
        return f; }, true);
      if (rc) return rc;
      rc = add_lateral(it[par], LAT_R2C_MASK, all, [&](BScan& s) {
        return fill(s.p, s.p->solve->r, s.p->wsA, nullptr, s.p->m, 1.0 / s.p->nx); }, false);
      if (rc) return rc;
      if ((rc = add_row(it[par], true, all, 0))) return rc;
      rc = add_lateral(it[par], LAT_SOLVE_ADJ_L1, l1_idx, [&](BScan& s) {
        LatFill f = fill(s.p, s.p->wsB, nullptr, nullptr, s.p->nz, 1.0);
        f.z1 = z1(s);
        f.z2 = z2(s);
        f.delta = s.delta;
        f.tau = s.tau;
        f.partial = s.p->solve->part_reg;
        return f; }, true);
      if (rc) return rc;
      rc = add_lateral(it[par], LAT_SOLVE_ADJ_V, db4_idx, [&](BScan& s) {
        LatFill f = fill(s.p, s.p->wsB, nullptr, nullptr, s.p->nz, 1.0);
        f.z1 = z1(s);
        f.z2 = z2(s);
        f.vout = s.p->solve->v;
        f.delta = s.delta;
        f.tau = s.tau;
        return f; }, true);
      if (rc) return rc;
      if (!db4_idx.empty()) {
        std::vector<const void*> ins;
        std::vector<void*> outs;
        std::vector<double*> parts[3];
        for (int i : db4_idx) {
          BScan& s = sc_[i];
          ins.push_back(s.p->solve->v);
          outs.push_back(z2(s));
          double* pr = s.p->solve->part_reg;
          int P = s.p->nx, N = s.p->nz;
          for (int lev = 0; lev < 3; ++lev) {
            parts[lev].push_back(pr);
            pr += dwt_level_ctas(P, N, 0);
            P /= 2;
            N /= 2;
          }
        }
        for (int lev = 0; lev < 3; ++lev)
          if ((rc = add_dwt(it[par], 0, lev, db4_idx, ins.data(), nullptr, parts[lev].data(), true))) return rc;
        for (int lev = 2; lev >= 0; --lev)
          if ((rc = add_dwt(it[par], 1, lev, db4_idx, nullptr, outs.data(), nullptr, false))) return rc;
      }
    }
    if ((rc = upload())) return rc;
    int kmax = 0;
    for (auto& s : sc_) kmax = std::max(kmax, s.o.max_iter);
    for (auto& s : sc_)
      if (s.o.max_iter != kmax) return MBIR_ERR_INVALID;   // one iteration count per batch
    for (auto& s : sc_) {
      SolveState* S = s.p->solve;
      MBIR_CUDA_TRY(cudaMemsetAsync(S->pz, 0, rsz_ * S->nmeas, st_));
      if (s.o.warm_start) {
        MBIR_CUDA_TRY(cudaMemcpyAsync(S->zA, s.x, esz_ * S->nimg, cudaMemcpyDeviceToDevice, st_));
        MBIR_CUDA_TRY(cudaMemcpyAsync(S->zB, s.x, esz_ * S->nimg, cudaMemcpyDeviceToDevice, st_));
      } else {
        MBIR_CUDA_TRY(cudaMemsetAsync(S->zA, 0, esz_ * S->nimg, st_));
        MBIR_CUDA_TRY(cudaMemsetAsync(S->zB, 0, esz_ * S->nimg, st_));
      }
    }
    std::vector<double> mu(kmax + 1, 0.0);
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
      // capture the loop once and replay it as one graph launch
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
    } else {
      if ((rc = iterate())) return rc;
    }
    // z^kmax sits in zA when kmax is even, zB when odd
    for (auto& s : sc_) {
      void* zlast = (kmax & 1) ? s.p->solve->zB : s.p->solve->zA;
      MBIR_CUDA_TRY(cudaMemcpyAsync(s.x, zlast, esz_ * s.p->solve->nimg, cudaMemcpyDeviceToDevice, st_));
    }
    return MBIR_OK;
  }

  static LatFill fill(mbir_plan p, const void* in, void* out, const uint8_t* mask, int cols, double scale) {
    (void)p;
    LatFill f;
    memset(&f, 0, sizeof(f));
    f.in = in;
    f.out = out;
    f.mask = mask;
    f.cols = cols;
    f.scale = scale;
    return f;
  }

  // analysis level without threshold whose coefficient array is coefs[i]
  int add_dwt_coef(std::vector<Stage>& out, int level, const std::vector<int>& idx, const void* const* in,
                   void* const* coefs) {
    if (idx.empty()) return MBIR_OK;
    const size_t ab = dwt_args_bytes(prec_);
    std::vector<unsigned char> blocks(ab * idx.size());
    std::vector<int> off(idx.size() + 1, 0);
    for (size_t i = 0; i < idx.size(); ++i) {
      BScan& s = sc_[idx[i]];
      fill_dwt_args(s.p, level, 0, in[i], nullptr, coefs[i], 0.0, 0, nullptr, blocks.data() + i * ab);
      off[i + 1] = off[i] + dwt_level_ctas(s.p->nx >> level, s.p->nz >> level, 0);
    }
    Stage g{2, 0, 0, 0, (int)idx.size(), off.back(), dwt_smem_bytes(prec_, 0), 0};
    g.arg_off = push(blocks.data(), blocks.size());
    g.off_off = push(off.data(), off.size() * sizeof(int));
    out.push_back(g);
    return grow_failed_ ? MBIR_ERR_OOM : MBIR_OK;
  }

 private:
  std::vector<BScan>& sc_;
  cudaStream_t st_;
  int prec_ = 0, J_ = 6;
  bool gather_ = true;
  size_t esz_ = 8, rsz_ = 4;
  unsigned char* hbuf_ = nullptr;
  size_t hlen_ = 0, hcap_ = 0;
  bool grow_failed_ = false;
  void* dbuf_ = nullptr;
  size_t dcap_ = 0;
};

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_solve_batch(mbir_plan* plans, int32_t n, const void* const* y, const uint8_t* const* mask,
                     const mbir_solve_opts* opts, void* const* x, mbir_solve_info* info, void* stream) {
  if (!plans || n < 1 || !y || !opts || !x) return MBIR_ERR_INVALID;
  std::vector<BScan> scans(n);
  for (int i = 0; i < n; ++i) {
    const mbir_solve_opts& o = opts[i];
    if (!plans[i] || !y[i] || !x[i]) return MBIR_ERR_INVALID;
    if (o.max_iter < 1 || o.penalty < MBIR_PENALTY_L1 || o.penalty > MBIR_PENALTY_DB4) return MBIR_ERR_INVALID;
    if (!(o.lambda >= 0) || !isfinite(o.lambda) || !isfinite(o.step) || o.rel_tol != 0.0) return MBIR_ERR_INVALID;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return MBIR_ERR_INVALID;   // each plan once: its workspace is per scan
    scans[i] = BScan{plans[i], y[i], mask ? mask[i] : nullptr, x[i], o, 0, 0, 0, 0};
  }
  cudaStream_t st = (cudaStream_t)stream;
  Engine eng(scans, st);
  int rc = eng.prepare();
  if (rc) return rc;
  rc = eng.solve();
  if (rc) return rc;
  if (info) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaStreamSynchronize");
    for (int i = 0; i < n; ++i) {
      info[i].iters = scans[i].o.max_iter;
      info[i].status = MBIR_OK;
      info[i].objective = NAN;
      info[i].lipschitz = scans[i].L;
      info[i].step = scans[i].delta;
      info[i].lambda_used = scans[i].lam;
    }
  }
  return MBIR_OK;
}

}  // extern "C"
