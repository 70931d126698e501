// The ISAM system operator Phi and its adjoint Phi^H (Sec. 2.1, Eqs. for_model and
// back_model) as three kernels each:
//
//   forward  x[p][n] --lateral FFT over p-->  X[l][n]                    (Eq. 4)
//            X[l][.] --row kernel: c_n, centred zero-pad to K, K-point FFT,
//                      J-tap KB interpolation at t_lm, filter f_lm--> S[l][m]   (Eq. 5, "u = Kx")
//            S[.][m] --inverse lateral FFT, 1/nx, real part, mask-->  y[p][m]  (Re, diag(s))
//   adjoint  the transpose of each stage in reverse order: masked y embedded as
//            complex, (1/nx) lateral FFT; per row conj(f), KB spreading (shared-
//            memory atomics), unnormalised inverse K-point FFT, keep the nz centred
//            samples, c_n; unnormalised inverse lateral FFT.
//
// Lateral stages work on tiles of TC adjacent columns with all nx rows staged in
// shared memory; row stages give one CTA per lateral frequency l and keep the
// K-point row (K = 2 nz) in shared memory.
#include "common.cuh"
#include "fft.cuh"
#include "operator.cuh"

namespace mbir {

// --------------------------------------------------------------- lateral FFT

// Deterministic block sum of one double per thread (fixed shuffle tree).
__device__ __forceinline__ double block_sum(double v) {
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
  return t;   // valid in thread 0
}

template <class R, int MODE>
__global__ void __launch_bounds__(kLatThreads)
lateral_kernel(LatArgs<R> a) {
  using V = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s = reinterpret_cast<V*>(smem_raw);
  const int TC = a.tc, nx = a.nx, C = a.cols;
  const int c0 = blockIdx.x * TC;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int total = nx * TC;
  for (int e = tid; e < total; e += nthr) {
    const int p = e / TC, b = e - p * TC;
    const int c = c0 + b;
    V v = cmk<V>(R(0), R(0));
    if (c < C) {
      const size_t off = (size_t)p * C + c;
      if constexpr (MODE == LAT_R2C_MASK) {
        const R r = reinterpret_cast<const R*>(a.in)[off];
        v.x = (a.mask == nullptr || a.mask[off]) ? r : R(0);
      } else {
        v = reinterpret_cast<const V*>(a.in)[off];
      }
    }
    s[p * TC + b] = v;
  }
  __syncthreads();
  constexpr bool INV = (MODE != LAT_C2C_FWD && MODE != LAT_R2C_MASK);
  fft_dif<INV>(s, TC, a.rad, reinterpret_cast<const V*>(a.tw));
  double part = 0.0;
  for (int e = tid; e < total; e += nthr) {
    const int p = e / TC, b = e - p * TC;
    const int c = c0 + b;
    if (c >= C) continue;
    const size_t off = (size_t)p * C + c;
    const V v = s[a.perm[p] * TC + b];
    if constexpr (MODE == LAT_C2R_INV_MASK) {
      const R r = v.x * a.scale;
      reinterpret_cast<R*>(a.out)[off] = (a.mask == nullptr || a.mask[off]) ? r : R(0);
    } else if constexpr (MODE == LAT_SOLVE_FWD) {
      const bool meas = (a.mask == nullptr || a.mask[off]);
      const R pz = meas ? v.x * a.scale : R(0);
      const R yv = meas ? a.y[off] : R(0);
      const R prev = a.pz[off];
      const R d = pz - yv;
      part += double(d) * double(d);
      a.pz[off] = pz;
      a.r[off] = (R(1) + a.mu) * pz - a.mu * prev - yv;
    } else if constexpr (MODE == LAT_SOLVE_ADJ_L1 || MODE == LAT_SOLVE_ADJ_V) {
      const V z1 = reinterpret_cast<const V*>(a.z1)[off];
      const V z2 = reinterpret_cast<const V*>(a.z2)[off];
      V xv;
      xv.x = z1.x + a.mu * (z1.x - z2.x) - a.delta * v.x;
      xv.y = z1.y + a.mu * (z1.y - z2.y) - a.delta * v.y;
      if constexpr (MODE == LAT_SOLVE_ADJ_L1) {
        const R mag = sqrt(xv.x * xv.x + xv.y * xv.y);
        const R sh = mag > a.tau ? R(1) - a.tau / mag : R(0);
        xv.x *= sh;
        xv.y *= sh;
        part += mag > a.tau ? double(mag - a.tau) : 0.0;
        reinterpret_cast<V*>(a.z2)[off] = xv;
      } else {
        reinterpret_cast<V*>(a.vout)[off] = xv;
      }
    } else {
      reinterpret_cast<V*>(a.out)[off] = cscale(v, a.scale);
    }
  }
  if constexpr (MODE == LAT_SOLVE_FWD || MODE == LAT_SOLVE_ADJ_L1) {
    const double t = block_sum(part);
    if (tid == 0) a.partial[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------- KB weights

template <class R>
__device__ __forceinline__ R kb_weight(R u, const float* kb, int J, R alpha, R inv_i0a) {
  const R au = u < R(0) ? -u : u;
  if constexpr (sizeof(R) == 4) {
    const float x = au * float(kKbRes);
    const int i = (int)x;
    const float f = x - float(i);
    const float a0 = kb[i], a1 = kb[i + 1];
    return fmaf(f, a1 - a0, a0);
  } else {
    const double r = 1.0 - (2.0 * au / J) * (2.0 * au / J);
    if (r < 0.0) return 0.0;
    return cyl_bessel_i0(alpha * sqrt(r)) * inv_i0a;
  }
}

// --------------------------------------------------------- row kernels (NUFFT)

template <class R>
__global__ void __launch_bounds__(kRowThreads)
row_forward_kernel(RowArgs<R> a) {
  using V = cplx_t<R>;
  using Tab = typename TabOf<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  float* kb = reinterpret_cast<float*>(buf + a.K);
  const int l = blockIdx.x;
  const int lp = l <= a.nx - l ? l : a.nx - l;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int K = a.K, nz = a.nz, n0 = a.n0, J = a.J, M = a.m;
  if (sizeof(R) == 4)
    for (int i = tid; i < a.nkb; i += nthr) kb[i] = a.kbtab[i];
  const V* X = reinterpret_cast<const V*>(a.in) + (size_t)l * nz;
  const R* cdep = reinterpret_cast<const R*>(a.cdep);
  // centred zero-padded row, element i = (n - n0) mod K holding c_n X[l][n],
  // stored digit-reversed for the decimation-in-time transform
  for (int i = tid; i < K; i += nthr) {
    int n = i + n0;
    if (n >= K) n -= K;
    buf[a.perm[i]] = (n < nz) ? cscale(X[n], cdep[n]) : cmk<V>(R(0), R(0));
  }
  __syncthreads();
  fft_dit<false>(buf, 1, a.rad, reinterpret_cast<const V*>(a.tw));
  const Tab* tab = reinterpret_cast<const Tab*>(a.tab) + (size_t)lp * M;
  V* S = reinterpret_cast<V*>(a.out) + (size_t)l * M;
  const int h = J / 2;
  for (int mm = tid; mm < M; mm += nthr) {
    const Tab e = tab[mm];
    V acc = cmk<V>(R(0), R(0));
    for (int j = 0; j < J; ++j) {
      const R u = R(e.frac) + R(h - 1 - j);
      const R w = kb_weight<R>(u, kb, J, R(a.alpha), R(a.inv_i0a));
      int idx = e.i0 - h + 1 + j;
      if (idx < 0) idx += K;
      if (idx >= K) idx -= K;
      const V b = buf[idx];
      acc.x += w * b.x;
      acc.y += w * b.y;
    }
    S[mm] = cmul(acc, cmk<V>(R(e.fre), R(e.fim)));
  }
}

template <class R>
__global__ void __launch_bounds__(kRowThreads)
row_adjoint_kernel(RowArgs<R> a) {
  using V = cplx_t<R>;
  using Tab = typename TabOf<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  float* kb = reinterpret_cast<float*>(buf + a.K);
  const int l = blockIdx.x;
  const int lp = l <= a.nx - l ? l : a.nx - l;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int K = a.K, nz = a.nz, n0 = a.n0, J = a.J, M = a.m;
  if (sizeof(R) == 4)
    for (int i = tid; i < a.nkb; i += nthr) kb[i] = a.kbtab[i];
  for (int i = tid; i < K; i += nthr) buf[i] = cmk<V>(R(0), R(0));
  __syncthreads();
  const Tab* tab = reinterpret_cast<const Tab*>(a.tab) + (size_t)lp * M;
  const V* Rh = reinterpret_cast<const V*>(a.in) + (size_t)l * M;
  const int h = J / 2;
  R* bufr = reinterpret_cast<R*>(buf);
  for (int mm = tid; mm < M; mm += nthr) {
    const Tab e = tab[mm];
    const V v = cmulc(Rh[mm], cmk<V>(R(e.fre), R(e.fim)));
    for (int j = 0; j < J; ++j) {
      const R u = R(e.frac) + R(h - 1 - j);
      const R w = kb_weight<R>(u, kb, J, R(a.alpha), R(a.inv_i0a));
      int idx = e.i0 - h + 1 + j;
      if (idx < 0) idx += K;
      if (idx >= K) idx -= K;
      atomicAdd(&bufr[2 * idx], w * v.x);
      atomicAdd(&bufr[2 * idx + 1], w * v.y);
    }
  }
  __syncthreads();
  fft_dif<true>(buf, 1, a.rad, reinterpret_cast<const V*>(a.tw));
  const R* cdep = reinterpret_cast<const R*>(a.cdep);
  V* Wo = reinterpret_cast<V*>(a.out) + (size_t)l * nz;
  for (int n = tid; n < nz; n += nthr) {
    int i = n - n0;
    if (i < 0) i += K;
    Wo[n] = cscale(buf[a.perm[i]], cdep[n]);
  }
}

// ------------------------------------------------------------------ launch

int lateral_grid(mbir_plan p, int cols);

template <class R>
LatArgs<R> lat_args(mbir_plan p, const void* in, void* out, const uint8_t* mask, int cols, R scale) {
  LatArgs<R> a;
  a.in = in;
  a.out = out;
  a.mask = mask;
  a.nx = p->nx;
  a.cols = cols;
  a.tc = p->tile_c;
  a.rad = p->rad_x;
  a.tw = p->tw_x;
  a.perm = p->perm_x;
  a.scale = scale;
  a.y = nullptr;
  a.pz = nullptr;
  a.r = nullptr;
  a.z1 = nullptr;
  a.z2 = nullptr;
  a.vout = nullptr;
  a.mu = a.delta = a.tau = R(0);
  a.partial = nullptr;
  return a;
}

constexpr int lat_class(int mode) {
  return mode == LAT_C2C_FWD ? PC_LAT_FWD
         : mode == LAT_R2C_MASK ? PC_LAT_R2C
         : (mode == LAT_C2R_INV_MASK || mode == LAT_SOLVE_FWD) ? PC_LAT_INV
                                                               : PC_LAT_ADJ;
}

template <class R>
size_t lat_smem(mbir_plan p) {
  return sizeof(cplx_t<R>) * p->nx * p->tile_c;
}

template <class R, int MODE>
int launch_lateral(mbir_plan p, const void* in, void* out, const uint8_t* mask, int cols, R scale,
                   cudaStream_t st) {
  LatArgs<R> a = lat_args<R>(p, in, out, mask, cols, scale);
  { ProfScope ps_(p, lat_class(MODE), st); lateral_kernel<R, MODE><<<lateral_grid(p, cols), kLatThreads, lat_smem<R>(p), st>>>(a); }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

template <class R>
RowArgs<R> row_args(mbir_plan p, const void* in, void* out) {
  RowArgs<R> a;
  a.in = in;
  a.out = out;
  a.tab = p->tab;
  a.cdep = p->cdep;
  a.kbtab = p->kbtab;
  a.tw = p->tw_k;
  a.rad = p->rad_k;
  a.perm = p->perm_k;
  a.nx = p->nx;
  a.nz = p->nz;
  a.m = p->m;
  a.K = p->K;
  a.J = p->J;
  a.n0 = p->n0;
  a.nkb = kKbRes * p->J / 2 + 2;
  a.alpha = p->alpha;
  a.inv_i0a = 1.0 / host_bessel_i0(p->alpha);
  return a;
}

template <class R>
size_t row_smem(mbir_plan p) {
  return sizeof(cplx_t<R>) * p->K + sizeof(float) * (kKbRes * p->J / 2 + 2);
}

template <class R>
int forward_t(mbir_plan p, const void* x, const uint8_t* mask, void* y, cudaStream_t st) {
  int rc = launch_lateral<R, LAT_C2C_FWD>(p, x, p->wsA, nullptr, p->nz, R(1), st);
  if (rc) return rc;
  RowArgs<R> a = row_args<R>(p, p->wsA, p->wsB);
  { ProfScope ps_(p, PC_ROW_FWD, st); row_forward_kernel<R><<<p->nx, kRowThreads, row_smem<R>(p), st>>>(a); }
  MBIR_LAUNCH_CHECK();
  return launch_lateral<R, LAT_C2R_INV_MASK>(p, p->wsB, y, mask, p->m, R(1) / R(p->nx), st);
}

template <class R>
int adjoint_t(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st) {
  int rc = launch_lateral<R, LAT_R2C_MASK>(p, y, p->wsA, mask, p->m, R(1) / R(p->nx), st);
  if (rc) return rc;
  RowArgs<R> a = row_args<R>(p, p->wsA, p->wsB);
  { ProfScope ps_(p, PC_ROW_ADJ, st); row_adjoint_kernel<R><<<p->nx, kRowThreads, row_smem<R>(p), st>>>(a); }
  MBIR_LAUNCH_CHECK();
  return launch_lateral<R, LAT_C2C_INV>(p, p->wsB, x, nullptr, p->nz, R(1), st);
}

template <class R>
int forward_solve_t(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, void* r,
                    double mu, double* partial, cudaStream_t st) {
  int rc = launch_lateral<R, LAT_C2C_FWD>(p, z1, p->wsA, nullptr, p->nz, R(1), st);
  if (rc) return rc;
  RowArgs<R> ra = row_args<R>(p, p->wsA, p->wsB);
  { ProfScope ps_(p, PC_ROW_FWD, st); row_forward_kernel<R><<<p->nx, kRowThreads, row_smem<R>(p), st>>>(ra); }
  MBIR_LAUNCH_CHECK();
  LatArgs<R> a = lat_args<R>(p, p->wsB, nullptr, mask, p->m, R(1) / R(p->nx));
  a.y = reinterpret_cast<const R*>(y);
  a.pz = reinterpret_cast<R*>(pz);
  a.r = reinterpret_cast<R*>(r);
  a.mu = R(mu);
  a.partial = partial;
  { ProfScope ps_(p, PC_LAT_INV, st); lateral_kernel<R, LAT_SOLVE_FWD><<<lateral_grid(p, p->m), kLatThreads, lat_smem<R>(p), st>>>(a); }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

template <class R>
int adjoint_solve_t(mbir_plan p, const void* r, const void* z1, void* z2, void* vout, double mu,
                    double delta, double tau, double* partial, cudaStream_t st) {
  // r is already zero where the mask is zero
  int rc = launch_lateral<R, LAT_R2C_MASK>(p, r, p->wsA, nullptr, p->m, R(1) / R(p->nx), st);
  if (rc) return rc;
  RowArgs<R> ra = row_args<R>(p, p->wsA, p->wsB);
  { ProfScope ps_(p, PC_ROW_ADJ, st); row_adjoint_kernel<R><<<p->nx, kRowThreads, row_smem<R>(p), st>>>(ra); }
  MBIR_LAUNCH_CHECK();
  LatArgs<R> a = lat_args<R>(p, p->wsB, nullptr, nullptr, p->nz, R(1));
  a.z1 = z1;
  a.z2 = z2;
  a.vout = vout;
  a.mu = R(mu);
  a.delta = R(delta);
  a.tau = R(tau);
  a.partial = partial;
  if (vout)
    { ProfScope ps_(p, PC_LAT_ADJ, st); lateral_kernel<R, LAT_SOLVE_ADJ_V><<<lateral_grid(p, p->nz), kLatThreads, lat_smem<R>(p), st>>>(a); }
  else
    { ProfScope ps_(p, PC_LAT_ADJ, st); lateral_kernel<R, LAT_SOLVE_ADJ_L1><<<lateral_grid(p, p->nz), kLatThreads, lat_smem<R>(p), st>>>(a); }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

int forward_solve_impl(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, void* r,
                       double mu, double* partial, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? forward_solve_t<double>(p, z1, mask, y, pz, r, mu, partial, st)
                                   : forward_solve_t<float>(p, z1, mask, y, pz, r, mu, partial, st);
}

int adjoint_solve_impl(mbir_plan p, const void* r, const void* z1, void* z2, void* vout, double mu,
                       double delta, double tau, double* partial, cudaStream_t st) {
  return p->precision == MBIR_FP64
             ? adjoint_solve_t<double>(p, r, z1, z2, vout, mu, delta, tau, partial, st)
             : adjoint_solve_t<float>(p, r, z1, z2, vout, mu, delta, tau, partial, st);
}

int lateral_grid(mbir_plan p, int cols) { return (cols + p->tile_c - 1) / p->tile_c; }

int forward_impl(mbir_plan p, const void* x, const uint8_t* mask, void* y, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? forward_t<double>(p, x, mask, y, st)
                                   : forward_t<float>(p, x, mask, y, st);
}

int adjoint_impl(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? adjoint_t<double>(p, y, mask, x, st)
                                   : adjoint_t<float>(p, y, mask, x, st);
}

template <class R>
static int configure_t(mbir_plan p) {
  const int lat = (int)(sizeof(cplx_t<R>) * kLatElems);
  const int row = (int)(sizeof(cplx_t<R>) * kMaxFFT + sizeof(float) * (kKbRes * 4 + 2));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(lateral_kernel<R, LAT_C2C_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lat));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(lateral_kernel<R, LAT_C2C_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, lat));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(lateral_kernel<R, LAT_R2C_MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, lat));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(lateral_kernel<R, LAT_C2R_INV_MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, lat));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(lateral_kernel<R, LAT_SOLVE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lat));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(lateral_kernel<R, LAT_SOLVE_ADJ_L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lat));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(lateral_kernel<R, LAT_SOLVE_ADJ_V>, cudaFuncAttributeMaxDynamicSharedMemorySize, lat));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(row_forward_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, row));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(row_adjoint_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, row));
  return MBIR_OK;
}

int configure_operator_kernels(mbir_plan p) {
  return p->precision == MBIR_FP64 ? configure_t<double>(p) : configure_t<float>(p);
}

}  // namespace mbir

using namespace mbir;

extern "C" {

static int check_common(mbir_plan p, const void* a, const void* b) {
  if (!p || !a || !b) return MBIR_ERR_INVALID;
  return MBIR_OK;
}

int mbir_forward(mbir_plan p, const void* x, const uint8_t* mask, void* y, void* stream) {
  const int rc = check_common(p, x, y);
  if (rc) return rc;
  return forward_impl(p, x, mask, y, (cudaStream_t)stream);
}

int mbir_adjoint(mbir_plan p, const void* y, const uint8_t* mask, void* x, void* stream) {
  const int rc = check_common(p, y, x);
  if (rc) return rc;
  return adjoint_impl(p, y, mask, x, (cudaStream_t)stream);
}

}  // extern "C"
