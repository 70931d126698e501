// FISTA (Sec. 2.3, Eq. alg) around the fused operator passes, the power-iteration
// step-size bound, the relative lambda rule and the FP64 objective (Eqs. obj,
// ls_obj).
//
// One iteration k (x^1 = z^0 = 0, t^1 = 1, mu_{k-1} = (t^{k-1} - 1)/t^k, mu_0 = 0):
//   forward pass on z^{k-1}, epilogue: pz = Phi z^{k-1} (kept for the next
//     iteration), r = Phi x^k - s y = (1 + mu) pz - mu Phi z^{k-2} - s y
//     (Phi is real-linear and x^k = z^{k-1} + mu (z^{k-1} - z^{k-2})), and the FP64
//     partial sums of 1/2 ||pz - s y||^2, the data term of F(z^{k-1}); r never
//     leaves the chip: the same pass over the column tiles applies the first
//     (lateral) stage of Phi^H to it;
//   rest of the adjoint pass, epilogue: z^k = prox_{tau}(x^k - delta Phi^H r) with
//     tau = lambda delta (l1 fused; the wavelet prox follows as its own kernels),
//     and the partial sums of ||Psi z^k||_1.
// With the paper's back-projection Phi* (Eq. back_model) in place of Phi^H, the
// residual r is written out by the measurement pass and A(r) is formed along the
// spectrometer axis before the lateral stage of B^H.
// F(z^{k-1}) = data + lambda * reg is reduced on the device in a fixed order, so
// the objective trace is deterministic.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"
#include "solve_state.cuh"

namespace mbir {

int prox_partial_impl(mbir_plan p, int penalty, const void* v, double tau, void* z, double* partial,
                      cudaStream_t st);
int wavelet_partial_count(int nx, int nz);
int ensure_wavelet_scratch(mbir_plan p);

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ double block_sum_s(double v) {
  __shared__ double wsum[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? wsum[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ double block_max_s(double v) {
  __shared__ double wmax[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wmax[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? wmax[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
  }
  __syncthreads();
  return t;
}

// out = wa * sum(a[0..na)) + wb * sum(b[0..nb)), one block, fixed order.
__global__ void combine_kernel(const double* a, int na, double wa, const double* b, int nb, double wb,
                               double* out) {
  pdl_wait_release();
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < na; i += blockDim.x) s += a[i];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) t += b[i];
  const double S = block_sum_s(s);
  const double T = block_sum_s(t);
  if (threadIdx.x == 0) *out = wa * S + (nb > 0 ? wb * T : 0.0);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// Pseudo-random start vector of the power iteration: uniform in [-1, 1) from a
// counter-based hash (SplitMix64) of the element index.
template <class R>
__global__ void fill_hash_kernel(cplx_t<R>* v, size_t n) {
  pdl_wait_release();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(2 * i), b = splitmix64(2 * i + 1);
    v[i] = cmk<cplx_t<R>>(R((a >> 11) * 0x1.0p-53 * 2.0 - 1.0), R((b >> 11) * 0x1.0p-53 * 2.0 - 1.0));
  }
}

// part[2 blk] = sum Re(conj(v) w), part[2 blk + 1] = sum |w|^2
template <class R>
__global__ void dot_norm_kernel(const cplx_t<R>* v, const cplx_t<R>* w, size_t n, double* part) {
  pdl_wait_release();
  // a thread's few terms in the working precision, FP64 across the block (FP64
  // arithmetic per element is slow on this GPU)
  R d = R(0), q = R(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> a = v[i], b = w[i];
    d += a.x * b.x + a.y * b.y;
    q += b.x * b.x + b.y * b.y;
  }
  const double D = block_sum_s(double(d)), Q = block_sum_s(double(q));
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = D;
    part[2 * blockIdx.x + 1] = Q;
  }
}

// scal[0] = <v, w>, scal[1] = 1/||w||, scal[2] = ||w||^2
__global__ void power_finalize_kernel(const double* part, int nb, double* scal) {
  pdl_wait_release();
  double d = 0.0, q = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    d += part[2 * i];
    q += part[2 * i + 1];
  }
  const double D = block_sum_s(d), Q = block_sum_s(q);
  if (threadIdx.x == 0) {
    scal[0] = D;
    scal[1] = Q > 0 ? 1.0 / sqrt(Q) : 0.0;
    scal[2] = Q;
  }
}

template <class R>
__global__ void scale_kernel(cplx_t<R>* v, const cplx_t<R>* w, size_t n, const double* scal) {
  pdl_wait_release();
  const R s = R(scal[1]);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = cscale(w[i], s);
}

template <class R>
__global__ void maxabs_kernel(const cplx_t<R>* v, size_t n, double* part) {
  pdl_wait_release();
  R m2 = R(0);   // largest |v|^2 of the thread, one square root at the end
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> a = v[i];
    m2 = fmax(m2, a.x * a.x + a.y * a.y);
  }
  const double M = block_max_s(sqrt(double(m2)));
  if (threadIdx.x == 0) part[blockIdx.x] = M;
}

__global__ void max_finalize_kernel(const double* part, int nb, double* out) {
  pdl_wait_release();
  double m = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, part[i]);
  const double M = block_max_s(m);
  if (threadIdx.x == 0) *out = M;
}

template <class R>
__global__ void abs_sum_kernel(const cplx_t<R>* v, size_t n, double* part) {
  pdl_wait_release();
  R s = R(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> a = v[i];
    s += sqrt(a.x * a.x + a.y * a.y);
  }
  const double S = block_sum_s(double(s));
  if (threadIdx.x == 0) part[blockIdx.x] = S;
}

template <class R>
__global__ void resid_kernel(const R* pz, const R* y, const uint8_t* mask, size_t n, double* part) {
  pdl_wait_release();
  R s = R(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (mask && !mask[i]) continue;
    const R d = pz[i] - y[i];
    s += d * d;
  }
  const double S = block_sum_s(double(s));
  if (threadIdx.x == 0) part[blockIdx.x] = S;
}


// Volume FISTA (the operator of both lateral axes has no fused solver passes):
// r = s (Phi x) - s y; Phi x arrives masked, so r = 0 where s = 0.
template <class R>
__global__ void vol_resid_kernel(const R* pz, const R* y, const uint8_t* mask, size_t n, R* r) {
  pdl_wait_release();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    r[i] = (mask && !mask[i]) ? R(0) : pz[i] - y[i];
}

// z^k = prox_{tau |.|}(x^k - delta g) (modulus soft threshold), then the momentum
// point x^{k+1} = z^k + mu (z^k - z^{k-1}) over x in place (Eq. alg).
template <class R>
__global__ void vol_fista_kernel(cplx_t<R>* x, const cplx_t<R>* g, const cplx_t<R>* zprev, cplx_t<R>* znew,
                                 size_t n, R delta, R tau, R mu) {
  pdl_wait_release();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> xi = x[i], gi = g[i], zp = zprev[i];
    const R ux = xi.x - delta * gi.x, uy = xi.y - delta * gi.y;
    const R mag = sqrt(ux * ux + uy * uy);
    const R sh = mag > tau ? R(1) - tau / mag : R(0);
    const R zx = ux * sh, zy = uy * sh;
    znew[i] = cmk<cplx_t<R>>(zx, zy);
    x[i] = cmk<cplx_t<R>>(zx + mu * (zx - zp.x), zy + mu * (zy - zp.y));
  }
}

// ------------------------------------------------------------------ state

// doubles in part_tmp / 2: grid-stride reductions and the power iteration's two
// partials per lateral CTA
int part_tmp_count(mbir_plan p) {
  const int g = lateral_grid(p, p->nz);
  return g > kRedBlocks ? g : kRedBlocks;
}

static size_t elem_size(mbir_plan p) { return p->precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2); }
static size_t real_size(mbir_plan p) { return p->precision == MBIR_FP64 ? sizeof(double) : sizeof(float); }

void destroy_solve_state(mbir_plan p) {
  SolveState* s = p->solve;
  if (!s) return;
  cudaFree(s->zA);
  cudaFree(s->zB);
  cudaFree(s->v);
  cudaFree(s->pz);
  cudaFree(s->r);
  cudaFree(s->part_data);
  cudaFree(s->part_reg);
  cudaFree(s->part_tmp);
  cudaFree(s->scal);
  cudaFree(s->objtrace);
  cudaFree(s->g);
  delete s;
  p->solve = nullptr;
}

int ensure_state(mbir_plan p, int trace_cap) {
  if (p->solve && p->solve->trace_cap >= trace_cap) return MBIR_OK;
  if (p->solve) {
    cudaFree(p->solve->objtrace);
    p->solve->objtrace = nullptr;
    MBIR_CUDA_TRY(cudaMalloc(&p->solve->objtrace, sizeof(double) * trace_cap));
    p->solve->trace_cap = trace_cap;
    return MBIR_OK;
  }
  SolveState* s = new (std::nothrow) SolveState;
  if (!s) return MBIR_ERR_OOM;
  p->solve = s;
  s->nimg = (size_t)p->nx * p->ny * p->nz;
  s->nmeas = (size_t)p->nx * p->ny * p->m;
  s->n_data = lateral_grid(p, p->m);
  int nr = lateral_grid(p, p->nz);
  if (wavelet_supported(p->nx, p->nz)) {
    const int w = wavelet_partial_count(p->nx, p->nz);
    if (w > nr) nr = w;
  }
  if (tv_partial_count(p) > nr) nr = tv_partial_count(p);
  s->n_reg = nr;
  s->trace_cap = trace_cap;
  MBIR_CUDA_TRY(cudaMalloc(&s->zA, elem_size(p) * s->nimg));
  MBIR_CUDA_TRY(cudaMalloc(&s->zB, elem_size(p) * s->nimg));
  MBIR_CUDA_TRY(cudaMalloc(&s->v, elem_size(p) * s->nimg));
  MBIR_CUDA_TRY(cudaMalloc(&s->pz, real_size(p) * s->nmeas));
  MBIR_CUDA_TRY(cudaMalloc(&s->r, real_size(p) * s->nmeas));
  MBIR_CUDA_TRY(cudaMalloc(&s->part_data, sizeof(double) * s->n_data));
  MBIR_CUDA_TRY(cudaMalloc(&s->part_reg, sizeof(double) * s->n_reg));
  MBIR_CUDA_TRY(cudaMalloc(&s->part_tmp, sizeof(double) * 2 * part_tmp_count(p)));
  MBIR_CUDA_TRY(cudaMalloc(&s->scal, sizeof(double) * 16));
  MBIR_CUDA_TRY(cudaMalloc(&s->objtrace, sizeof(double) * trace_cap));
  if (p->ny > 1) MBIR_CUDA_TRY(cudaMalloc(&s->g, elem_size(p) * s->nimg));
  return MBIR_OK;
}

static int grid_for(size_t n) {
  size_t g = (n + kRedThreads - 1) / kRedThreads;
  return (int)(g < (size_t)kRedBlocks ? (g ? g : 1) : kRedBlocks);
}

// ------------------------------------------------------------------ pieces

// Power iteration for L = ||Phi^H diag(s) Phi|| (the step-size bound, Sec. 2.3): a
// counter-based pseudo-random start w, then per step v = w/||w||, w = Phi^H s Phi v
// and the Rayleigh quotient <v, w>.  The normalisation is folded into the first
// lateral pass and the two reductions into the last one.
// With the Hilbert-form back-projection the same iteration runs on Phi* s Phi.
template <class R>
static int lipschitz_t(mbir_plan p, const uint8_t* mask, int iters, double* out, cudaStream_t st,
                       bool hilbert = false) {
  using V = cplx_t<R>;
  SolveState* s = p->solve;
  const size_t n = s->nimg;
  const int gb = grid_for(n);
  V* v = (V*)s->v;
  V* w = (V*)s->zA;
  { ProfScope ps_(p, PC_REDUCE, st); launch(fill_hash_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, w, n); }
  { ProfScope ps_(p, PC_REDUCE, st); launch(dot_norm_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, w, w, n, s->part_tmp); }
  { ProfScope ps_(p, PC_REDUCE, st); launch(power_finalize_kernel, dim3(1), dim3(kRedThreads), 0, st, s->part_tmp, gb, s->scal); }
  MBIR_LAUNCH_CHECK();
  const int np = lateral_grid(p, p->nz);
  for (int it = 0; it < iters; ++it) {
    int rc = hilbert ? power_step_hilbert_impl(p, mask, w, v, s->r, s->scal, s->part_tmp, st)
                     : power_step_impl(p, mask, w, v, s->scal, s->part_tmp, st);
    if (rc) return rc;
    { ProfScope ps_(p, PC_REDUCE, st); launch(power_finalize_kernel, dim3(1), dim3(kRedThreads), 0, st, s->part_tmp, np, s->scal); }
    MBIR_LAUNCH_CHECK();
  }
  MBIR_CUDA_TRY(cudaMemcpyAsync(out, s->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  MBIR_CUDA_TRY(cudaStreamSynchronize(st));
  return MBIR_OK;
}

// max |Psi Phi^H (s y)| (Phi* in place of Phi^H for the Hilbert-form back-projection)
template <class R>
static int lambda_scale_t(mbir_plan p, const void* y, const uint8_t* mask, int penalty, double* out,
                          cudaStream_t st, bool hilbert = false) {
  using V = cplx_t<R>;
  SolveState* s = p->solve;
  const size_t n = s->nimg;
  int rc = hilbert ? adjoint_hilbert_impl(p, y, mask, s->zA, st) : adjoint_impl(p, y, mask, s->zA, st);
  if (rc) return rc;
  const V* src = (const V*)s->zA;
  if (penalty == MBIR_PENALTY_DB4) {
    rc = wavelet_impl(p, 0, s->zA, s->v, st);
    if (rc) return rc;
    src = (const V*)s->v;
  }
  const int gb = grid_for(n);
  { ProfScope ps_(p, PC_REDUCE, st); launch(maxabs_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, src, n, s->part_tmp); }
  { ProfScope ps_(p, PC_REDUCE, st); launch(max_finalize_kernel, dim3(1), dim3(kRedThreads), 0, st, s->part_tmp, gb, s->scal + 4); }
  MBIR_LAUNCH_CHECK();
  MBIR_CUDA_TRY(cudaMemcpyAsync(out, s->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
  MBIR_CUDA_TRY(cudaStreamSynchronize(st));
  return MBIR_OK;
}

// reg partials of z for the penalty, written as solve iterations would
template <class R>
static int reg_partials_t(mbir_plan p, int penalty, const void* z, cudaStream_t st) {
  SolveState* s = p->solve;
  if (penalty == MBIR_PENALTY_L1) {
    const int gb = lateral_grid(p, p->nz);
    { ProfScope ps_(p, PC_REDUCE, st); launch(abs_sum_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, (const cplx_t<R>*)z, s->nimg, s->part_reg); }
    MBIR_LAUNCH_CHECK();
    return MBIR_OK;
  }
  if (penalty == MBIR_PENALTY_TV) return tv_prox_impl(p, z, 0.0, 0, s->v, s->part_reg, st);
  return prox_partial_impl(p, penalty, z, 0.0, s->v, s->part_reg, st);
}

static int reg_count(mbir_plan p, int penalty) {
  if (penalty == MBIR_PENALTY_TV) return tv_partial_count(p);
  return penalty == MBIR_PENALTY_L1 ? lateral_grid(p, p->nz) : wavelet_partial_count(p->nx, p->nz);
}

template <class R>
static int solve_t(mbir_plan p, const void* y, const uint8_t* mask, const mbir_solve_opts* o, void* x,
                   mbir_solve_info* info, cudaStream_t st, bool final_objective) {
  SolveState* s = p->solve;
  const size_t es = elem_size(p);
  const bool hil = o->backprojection == MBIR_BACKPROJ_HILBERT;
  double L = 0.0, delta = o->step;
  if (!(delta > 0)) {
    const int pit = o->power_iters > 0 ? o->power_iters : 30;
    int rc = lipschitz_t<R>(p, mask, pit, &L, st, hil);
    if (rc) return rc;
    if (!(L > 0) || !isfinite(L)) return MBIR_ERR_INVALID;
    delta = 1.0 / (1.01 * L);
  }
  double lam = o->lambda;
  if (o->lambda_is_relative) {
    double m = 0.0;
    int rc = lambda_scale_t<R>(p, y, mask, o->penalty, &m, st, hil);
    if (rc) return rc;
    lam *= m;
  }
  const double tau = lam * delta;
  // momentum sequence mu_k = (t^k - 1)/t^{k+1}
  std::vector<double> mu(o->max_iter + 1, 0.0);
  {
    double t = 1.0;
    for (int k = 0; k <= o->max_iter; ++k) {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      mu[k] = (t - 1.0) / tn;
      t = tn;
    }
  }
  void* z1 = s->zA;
  void* z2 = s->zB;
  const int nreg = reg_count(p, o->penalty);
  MBIR_CUDA_TRY(cudaMemsetAsync(s->pz, 0, real_size(p) * s->nmeas, st));
  if (o->warm_start) {
    MBIR_CUDA_TRY(cudaMemcpyAsync(z1, x, es * s->nimg, cudaMemcpyDeviceToDevice, st));
    MBIR_CUDA_TRY(cudaMemcpyAsync(z2, x, es * s->nimg, cudaMemcpyDeviceToDevice, st));
    int rc = reg_partials_t<R>(p, o->penalty, z1, st);
    if (rc) return rc;
  } else {
    MBIR_CUDA_TRY(cudaMemsetAsync(z1, 0, es * s->nimg, st));
    MBIR_CUDA_TRY(cudaMemsetAsync(z2, 0, es * s->nimg, st));
    MBIR_CUDA_TRY(cudaMemsetAsync(s->part_reg, 0, sizeof(double) * s->n_reg, st));
  }
  int k = 0, status = MBIR_OK;
  const bool check = o->rel_tol > 0;
  // the objective of every iterate is reduced only when something reads it
  const bool want_trace = check || (info && info->objective_trace && info->trace_len > 0);
  if (check) status = MBIR_ERR_NOT_CONVERGED;
  for (k = 1; k <= o->max_iter; ++k) {
    const double m = k >= 2 ? mu[k - 2] : 0.0;
    int rc = hil ? forward_solve_hilbert_impl(p, z1, mask, y, s->pz, s->r, m, s->part_data, st)
                 : forward_solve_impl(p, z1, mask, y, s->pz, m, s->part_data, st);
    if (rc) return rc;
    if (want_trace) {
      ProfScope ps_(p, PC_REDUCE, st);
      launch(combine_kernel, dim3(1), dim3(kRedThreads), 0, st, s->part_data, s->n_data, 0.5, s->part_reg, nreg,
             lam, s->objtrace + (k - 1));
    }
    MBIR_LAUNCH_CHECK();
    if (o->penalty == MBIR_PENALTY_L1) {
      rc = adjoint_solve_impl(p, z1, z2, nullptr, m, delta, tau, s->part_reg, st);
      if (rc) return rc;
    } else {
      rc = adjoint_solve_impl(p, z1, z2, s->v, m, delta, tau, nullptr, st);
      if (rc) return rc;
      if (o->penalty == MBIR_PENALTY_TV)
        rc = tv_prox_impl(p, s->v, tau, o->tv_iters > 0 ? o->tv_iters : kTvDefaultIters, z2, s->part_reg, st);
      else
        rc = prox_partial_impl(p, o->penalty, s->v, tau, z2, s->part_reg, st);
      if (rc) return rc;
    }
    void* t = z1;
    z1 = z2;
    z2 = t;
    if (check && k >= 3 && k >= o->min_iter) {
      double f[2];
      MBIR_CUDA_TRY(cudaMemcpyAsync(f, s->objtrace + (k - 2), 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      MBIR_CUDA_TRY(cudaStreamSynchronize(st));
      if (fabs(f[1] - f[0]) <= o->rel_tol * fabs(f[0])) {
        status = MBIR_OK;
        break;
      }
    }
  }
  const int iters = k > o->max_iter ? o->max_iter : k;
  MBIR_CUDA_TRY(cudaMemcpyAsync(x, z1, es * s->nimg, cudaMemcpyDeviceToDevice, st));
  if (info) {
    double fin = NAN;
    if (final_objective) {
      // F(z^iters): one more forward pass for the data term
      int rc = forward_impl(p, z1, mask, s->r, st);
      if (rc) return rc;
      const int gb = grid_for(s->nmeas);
      { ProfScope ps_(p, PC_REDUCE, st); launch(resid_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, (const R*)s->r, (const R*)y, mask, s->nmeas, s->part_tmp); }
      { ProfScope ps_(p, PC_REDUCE, st); launch(combine_kernel, dim3(1), dim3(kRedThreads), 0, st, s->part_tmp, gb, 0.5, s->part_reg, nreg, lam, s->scal + 6); }
      MBIR_LAUNCH_CHECK();
      MBIR_CUDA_TRY(cudaMemcpyAsync(&fin, s->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (info->objective_trace && info->trace_len > 0) {
      const int n = info->trace_len < iters ? info->trace_len : iters;
      MBIR_CUDA_TRY(cudaMemcpyAsync(info->objective_trace, s->objtrace, sizeof(double) * n,
                                    cudaMemcpyDeviceToHost, st));
    }
    MBIR_CUDA_TRY(cudaStreamSynchronize(st));
    info->iters = iters;
    info->status = status;
    info->objective = fin;
    info->lipschitz = L;
    info->step = delta;
    info->lambda_used = lam;
  }
  return status;
}


// FISTA (Eq. alg) on a volume plan with the l1 penalty, in the oracle's form:
// z^k = prox(x^k - delta Phi^H(s Phi x^k - s y)), x^{k+1} = z^k + mu_k (z^k - z^{k-1}),
// x^1 = z^0 = 0 (or the warm start), the step from the power iteration on
// Phi^H s Phi and the relative lambda from max|Phi^H s y|.  Each iteration is one
// volume forward, one volume adjoint and two elementwise passes.
template <class R>
static int solve_vol_t(mbir_plan p, const void* y, const uint8_t* mask, const mbir_solve_opts* o, void* x,
                       mbir_solve_info* info, cudaStream_t st, bool final_objective) {
  using V = cplx_t<R>;
  SolveState* s = p->solve;
  const size_t n = s->nimg, nm = s->nmeas;
  const int gb = grid_for(n), gm = grid_for(nm);
  const size_t es = elem_size(p);
  V* G = (V*)s->g;
  double L = 0.0, delta = o->step;
  if (!(delta > 0)) {
    const int pit = o->power_iters > 0 ? o->power_iters : 30;
    V* w = (V*)s->zA;
    V* v = (V*)s->v;
    { ProfScope ps_(p, PC_REDUCE, st); launch(fill_hash_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, w, n); }
    { ProfScope ps_(p, PC_REDUCE, st); launch(dot_norm_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, w, w, n, s->part_tmp); }
    { ProfScope ps_(p, PC_REDUCE, st); launch(power_finalize_kernel, dim3(1), dim3(kRedThreads), 0, st, s->part_tmp, gb, s->scal); }
    MBIR_LAUNCH_CHECK();
    for (int it = 0; it < pit; ++it) {
      { ProfScope ps_(p, PC_REDUCE, st); launch(scale_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, v, (const V*)w, n, (const double*)s->scal); }
      MBIR_LAUNCH_CHECK();
      int rc = forward_impl(p, v, mask, s->pz, st);
      if (!rc) rc = adjoint_impl(p, s->pz, mask, w, st);
      if (rc) return rc;
      { ProfScope ps_(p, PC_REDUCE, st); launch(dot_norm_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, (const V*)v, (const V*)w, n, s->part_tmp); }
      { ProfScope ps_(p, PC_REDUCE, st); launch(power_finalize_kernel, dim3(1), dim3(kRedThreads), 0, st, s->part_tmp, gb, s->scal); }
      MBIR_LAUNCH_CHECK();
    }
    MBIR_CUDA_TRY(cudaMemcpyAsync(&L, s->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    MBIR_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(L > 0) || !isfinite(L)) return MBIR_ERR_INVALID;
    delta = 1.0 / (1.01 * L);
  }
  double lam = o->lambda;
  if (o->lambda_is_relative) {
    int rc = adjoint_impl(p, y, mask, G, st);
    if (rc) return rc;
    { ProfScope ps_(p, PC_REDUCE, st); launch(maxabs_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, (const V*)G, n, s->part_tmp); }
    { ProfScope ps_(p, PC_REDUCE, st); launch(max_finalize_kernel, dim3(1), dim3(kRedThreads), 0, st, (const double*)s->part_tmp, gb, s->scal + 4); }
    MBIR_LAUNCH_CHECK();
    double m = 0.0;
    MBIR_CUDA_TRY(cudaMemcpyAsync(&m, s->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    MBIR_CUDA_TRY(cudaStreamSynchronize(st));
    lam *= m;
  }
  const double tau = lam * delta;
  V* X = (V*)s->v;                       // the momentum point x^k
  V* Z[2] = {(V*)s->zA, (V*)s->zB};      // z^{k-1}, z^k alternate
  if (o->warm_start) {
    MBIR_CUDA_TRY(cudaMemcpyAsync(X, x, es * n, cudaMemcpyDeviceToDevice, st));
    MBIR_CUDA_TRY(cudaMemcpyAsync(Z[0], x, es * n, cudaMemcpyDeviceToDevice, st));
  } else {
    MBIR_CUDA_TRY(cudaMemsetAsync(X, 0, es * n, st));
    MBIR_CUDA_TRY(cudaMemsetAsync(Z[0], 0, es * n, st));
  }
  double t = 1.0;
  int cur = 0;   // Z[cur] holds z^{k-1}
  for (int k = 1; k <= o->max_iter; ++k) {
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const double mu = (t - 1.0) / tn;
    t = tn;
    int rc = forward_impl(p, X, mask, s->pz, st);
    if (rc) return rc;
    { ProfScope ps_(p, PC_REDUCE, st); launch(vol_resid_kernel<R>, dim3(gm), dim3(kRedThreads), 0, st, (const R*)s->pz, (const R*)y, mask, nm, (R*)s->r); }
    MBIR_LAUNCH_CHECK();
    if ((rc = adjoint_impl(p, s->r, mask, G, st))) return rc;
    { ProfScope ps_(p, PC_SOFT, st); launch(vol_fista_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, X, (const V*)G, (const V*)Z[cur], Z[cur ^ 1], n, R(delta), R(tau), R(mu)); }
    MBIR_LAUNCH_CHECK();
    cur ^= 1;
  }
  MBIR_CUDA_TRY(cudaMemcpyAsync(x, Z[cur], es * n, cudaMemcpyDeviceToDevice, st));
  if (info) {
    double fin = NAN;
    if (final_objective) {
      // F(z) = 1/2 ||s Phi z - s y||^2 + lambda ||z||_1
      int rc = forward_impl(p, Z[cur], mask, s->pz, st);
      if (rc) return rc;
      double* pd = s->part_tmp;
      double* pr = s->part_tmp + gm;
      { ProfScope ps_(p, PC_REDUCE, st); launch(resid_kernel<R>, dim3(gm), dim3(kRedThreads), 0, st, (const R*)s->pz, (const R*)y, mask, nm, pd); }
      { ProfScope ps_(p, PC_REDUCE, st); launch(abs_sum_kernel<R>, dim3(gb), dim3(kRedThreads), 0, st, (const V*)Z[cur], n, pr); }
      { ProfScope ps_(p, PC_REDUCE, st); launch(combine_kernel, dim3(1), dim3(kRedThreads), 0, st, (const double*)pd, gm, 0.5, (const double*)pr, gb, lam, s->scal + 6); }
      MBIR_LAUNCH_CHECK();
      MBIR_CUDA_TRY(cudaMemcpyAsync(&fin, s->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    MBIR_CUDA_TRY(cudaStreamSynchronize(st));
    info->iters = o->max_iter;
    info->status = MBIR_OK;
    info->objective = fin;
    info->lipschitz = L;
    info->step = delta;
    info->lambda_used = lam;
  }
  return MBIR_OK;
}

// mbir_solve; final_objective = false leaves info->objective NaN (no extra forward pass).
int solve_plan(mbir_plan p, const void* y, const uint8_t* mask, const mbir_solve_opts* o, void* x,
               mbir_solve_info* info, cudaStream_t st, bool final_objective) {
  if (!p || !y || !o || !x) return MBIR_ERR_INVALID;
  if (p->ny > 1) {
    // volume plans: l1 penalty, the transpose back-projection, a fixed iteration count
    if (o->max_iter < 1 || o->penalty != MBIR_PENALTY_L1 || o->backprojection != MBIR_BACKPROJ_TRANSPOSE ||
        o->rel_tol != 0.0 || !(o->lambda >= 0) || !isfinite(o->lambda) || !isfinite(o->step)) {
      set_error_text("mbir_solve: a volume plan takes the l1 penalty, the transpose back-projection and "
                     "rel_tol = 0");
      return MBIR_ERR_INVALID;
    }
    int rc = ensure_state(p, 1);
    if (rc) return rc;
    return p->precision == MBIR_FP64 ? solve_vol_t<double>(p, y, mask, o, x, info, st, final_objective)
                                     : solve_vol_t<float>(p, y, mask, o, x, info, st, final_objective);
  }
  if (o->max_iter < 1 || o->min_iter < 0) return MBIR_ERR_INVALID;
  if (o->penalty != MBIR_PENALTY_L1 && o->penalty != MBIR_PENALTY_DB4 && o->penalty != MBIR_PENALTY_TV)
    return MBIR_ERR_INVALID;
  if (!(o->lambda >= 0) || !isfinite(o->lambda) || !isfinite(o->step) || !(o->rel_tol >= 0))
    return MBIR_ERR_INVALID;
  if (o->backprojection != MBIR_BACKPROJ_TRANSPOSE && o->backprojection != MBIR_BACKPROJ_HILBERT)
    return MBIR_ERR_INVALID;
  if (o->penalty == MBIR_PENALTY_DB4 && !wavelet_supported(p->nx, p->nz)) return MBIR_ERR_UNSUPPORTED_SIZE;
  int rc = ensure_state(p, o->max_iter);
  if (rc) return rc;
  if (o->backprojection == MBIR_BACKPROJ_HILBERT) {
    rc = ensure_hilbert(p);
    if (rc) return rc;
  }
  if (o->penalty == MBIR_PENALTY_DB4) {
    rc = ensure_wavelet_scratch(p);
    if (rc) return rc;
  }
  return p->precision == MBIR_FP64 ? solve_t<double>(p, y, mask, o, x, info, st, final_objective)
                                   : solve_t<float>(p, y, mask, o, x, info, st, final_objective);
}

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_lipschitz(mbir_plan p, const uint8_t* mask, int32_t iters, double* out, void* stream) {
  if (const int vrc = bscan_only(p, "mbir_lipschitz")) return vrc;
  if (!p || !out || iters < 1) return MBIR_ERR_INVALID;
  int rc = ensure_state(p, 1);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  return p->precision == MBIR_FP64 ? lipschitz_t<double>(p, mask, iters, out, st)
                                   : lipschitz_t<float>(p, mask, iters, out, st);
}

int mbir_solve(mbir_plan p, const void* y, const uint8_t* mask, const mbir_solve_opts* o, void* x,
               mbir_solve_info* info, void* stream) {
  return solve_plan(p, y, mask, o, x, info, (cudaStream_t)stream, true);
}

}  // extern "C"
