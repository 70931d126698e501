// The conjugate analytic signal of the paper's back-projection (Sec. 2.1, Eq.
// back_model): Phi*(y) = B^H A(s y), A(r) = r - j d H(r) along the spectrometer
// axis of every A-scan, H the discrete Hilbert transform (DFT multiplier
// -j sgn(f), zero at DC and at the Nyquist bin), d = +1 when the wavenumbers
// ascend with the pixel index (the printed sign) and -1 when they descend.
//
// One CTA takes two A-scans a, b and transforms z = r_a + j r_b once: H is real,
// so the inverse transform of -j sgn(f) Z(f) is H r_a + j H r_b.  The forward
// transform runs as a dif (spectrum left digit-reversed), the multiplier is
// applied in place through the digit-reversal table, and the inverse runs as a
// dit (natural order out), so no reordering pass is needed.  HBM traffic per
// sample: y and the mask in (5 bytes in FP32), c out (8 bytes); the measurements
// are read a second time for the real part, from L2.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
#include "operator.cuh"

namespace mbir {

constexpr int kHilThreads = 256;

template <class R>
__global__ void __launch_bounds__(kHilThreads)
    hilbert_kernel(const R* __restrict__ y, const uint8_t* __restrict__ mask, cplx_t<R>* __restrict__ c, int nx,
                   int m, Radix rad, const cplx_t<R>* __restrict__ twg, const int* __restrict__ perm, R side,
                   int sw) {
  using V = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s = reinterpret_cast<V*>(smem_raw);
  const Tw2<V> tw = load_twiddles(s + m, twg, rad);
  const bool on = sw != 0;
  const int pa = 2 * blockIdx.x;
  const bool hb = pa + 1 < nx;
  const size_t oa = (size_t)pa * m, ob = oa + m;
  pdl_wait_release();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    R a = y[oa + i];
    R b = hb ? y[ob + i] : R(0);
    if (mask) {
      if (!mask[oa + i]) a = R(0);
      if (hb && !mask[ob + i]) b = R(0);
    }
    s[swz(i, on)] = cmk<V>(a, b);
  }
  __syncthreads();
  fft_dif<false>(s, 1, rad, tw, on);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int q = swz(perm[k], on);
    const V v = s[q];
    const R g = (k == 0 || 2 * k == m) ? R(0) : (2 * k < m ? R(1) : R(-1));
    s[q] = cmk<V>(g * v.y, -g * v.x);   // -j g (v.x + j v.y)
  }
  __syncthreads();
  fft_dit<true>(s, 1, rad, tw, on);
  const R f = -side / R(m);   // the inverse transform is unnormalised
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const V h = s[swz(i, on)];
    R a = y[oa + i];
    R b = hb ? y[ob + i] : R(0);
    if (mask) {
      if (!mask[oa + i]) a = R(0);
      if (hb && !mask[ob + i]) b = R(0);
    }
    c[oa + i] = cmk<V>(a, f * h.x);
    if (hb) c[ob + i] = cmk<V>(b, f * h.y);
  }
}

template <class R>
static size_t hilbert_smem(mbir_plan p) {
  return sizeof(cplx_t<R>) * ((size_t)p->m + p->rad_m.tw_lo + p->rad_m.tw_hi);
}

int ensure_hilbert(mbir_plan p) {
  if (p->tw_m) return MBIR_OK;
  Radix r;
  if (p->m > kMaxFFT || !plan_factor_radix(p->m, &r, 8)) return MBIR_ERR_UNSUPPORTED_SIZE;
  const size_t es = p->precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t smem = es * ((size_t)p->m + r.tw_lo + r.tw_hi);
  if (smem > (size_t)kMaxDynSmem) return MBIR_ERR_UNSUPPORTED_SIZE;
  int rc = plan_fft_tables(p, p->m, &p->rad_m, &p->tw_m, &p->perm_m);
  if (rc) {
    cudaFree(p->tw_m);
    cudaFree(p->perm_m);
    p->tw_m = nullptr;
    p->perm_m = nullptr;
    return rc;
  }
  // the cap, not this plan's size: plans of other lengths share the kernel
  if (p->precision == MBIR_FP64)
    MBIR_CUDA_TRY(cudaFuncSetAttribute(hilbert_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
  else
    MBIR_CUDA_TRY(cudaFuncSetAttribute(hilbert_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
  return MBIR_OK;
}

template <class R>
static int hilbert_t(mbir_plan p, const void* y, const uint8_t* mask, void* c, cudaStream_t st) {
  const int grid = (p->nx + 1) / 2;
  const R side = p->k_ascending ? R(1) : R(-1);
  {
    ProfScope ps_(p, PC_HILBERT, st);
    launch(hilbert_kernel<R>, dim3(grid), dim3(kHilThreads), hilbert_smem<R>(p), st, static_cast<const R*>(y), mask,
           static_cast<cplx_t<R>*>(c), p->nx, p->m, p->rad_m, static_cast<const cplx_t<R>*>(p->tw_m),
           (const int*)p->perm_m, side, (p->m & 15) == 0 ? 1 : 0);
  }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

int hilbert_impl(mbir_plan p, const void* y, const uint8_t* mask, void* c, cudaStream_t st) {
  int rc = ensure_hilbert(p);
  if (rc) return rc;
  return p->precision == MBIR_FP64 ? hilbert_t<double>(p, y, mask, c, st) : hilbert_t<float>(p, y, mask, c, st);
}

}  // namespace mbir
