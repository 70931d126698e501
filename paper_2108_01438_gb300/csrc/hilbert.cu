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
//
// The interpolating variant (the baseline of Sec. 3, direct ISAM on linearly
// interpolated measurements) first fills every unmeasured sample from the nearest
// measured ones on either side, in the pixel index.  Thread t owns a contiguous
// chunk of the row: it finds the last and first measured sample of its chunk,
// a block-wide max-scan (min-scan) of those gives the last measured sample
// before (first after) the chunk, a forward walk records each sample's previous
// measured index, and a backward walk interpolates.  Both rows of the CTA are
// handled at once (int2 indices); the filled rows are kept for the real part.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
#include "operator.cuh"

namespace mbir {

constexpr int kHilThreads = 256;
// resident CTAs an SM for FP32 (the launch-bounds register cap): four fit the
// 1024 x 2048 B-scan's 512 row pairs in one wave on 152 SMs
#ifndef MBIR_HIL_MINB
#define MBIR_HIL_MINB 4
#endif

// Linear interpolation at i between the measured samples p < i < n of one row
// (lane 0: the .x component of s, lane 1: .y); p < 0 or n >= m: hold the other
// end, neither: zero.
template <class R, class V>
__device__ __forceinline__ R interp_at(const V* s, bool on, int lane, int i, int p, int n, int m) {
  auto val = [&](int j) { const V v = s[swz(j, on)]; return lane == 0 ? v.x : v.y; };
  if (p < 0) return n < m ? val(n) : R(0);
  if (n >= m) return val(p);
  const R yp = val(p), yn = val(n);
  return yp + (yn - yp) * (R(i - p) / R(n - p));
}

// Fill the unmeasured samples of the two staged rows in s (flags in M: bit 0 row
// a measured, bit 1 row b) into Q, which first holds each sample's previous
// measured indices; scan: 2 * blockDim.x int2.
template <class R>
__device__ void interp_rows(const cplx_t<R>* s, cplx_t<R>* Q, const uint8_t* M, int2* scan, int m, bool on) {
  using V = cplx_t<R>;
  const int T = blockDim.x, t = threadIdx.x;
  const int chunk = (m + T - 1) / T;
  const int c0 = min(m, t * chunk), c1 = min(m, c0 + chunk);
  int2 last = make_int2(-1, -1), first = make_int2(m, m);
  for (int i = c0; i < c1; ++i) {
    const int f = M[i];
    if (f & 1) {
      last.x = i;
      first.x = min(first.x, i);
    }
    if (f & 2) {
      last.y = i;
      first.y = min(first.y, i);
    }
  }
  int2* smax = scan;
  int2* smin = scan + T;
  smax[t] = last;
  smin[t] = first;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {   // inclusive scans, Hillis-Steele
    int2 a = smax[t], b = smin[t];
    if (t >= off) {
      const int2 o = smax[t - off];
      a = make_int2(max(a.x, o.x), max(a.y, o.y));
    }
    if (t + off < T) {
      const int2 o = smin[t + off];
      b = make_int2(min(b.x, o.x), min(b.y, o.y));
    }
    __syncthreads();
    smax[t] = a;
    smin[t] = b;
    __syncthreads();
  }
  int2 prev = t > 0 ? smax[t - 1] : make_int2(-1, -1);
  int2 next = t + 1 < T ? smin[t + 1] : make_int2(m, m);
  for (int i = c0; i < c1; ++i) {
    const int f = M[i];
    if (f & 1) prev.x = i;
    if (f & 2) prev.y = i;
    *reinterpret_cast<int2*>(Q + i) = prev;
  }
  for (int i = c1 - 1; i >= c0; --i) {
    const int f = M[i];
    if (f & 1) next.x = i;
    if (f & 2) next.y = i;
    const int2 pv = *reinterpret_cast<const int2*>(Q + i);
    const V cur = s[swz(i, on)];
    const R va = (f & 1) ? cur.x : interp_at<R>(s, on, 0, i, pv.x, next.x, m);
    const R vb = (f & 2) ? cur.y : interp_at<R>(s, on, 1, i, pv.y, next.y, m);
    Q[i] = cmk<V>(va, vb);
  }
}

// Shared-memory layout (bytes): the row pair s [m], the twiddles, the
// digit-reversal table [m], then for the interpolating variant Q [m], the scans
// and the flags.
struct HilLayout {
  size_t tw, perm, q, scan, flags, total;
};
__host__ __device__ inline HilLayout hil_layout(size_t es, int m, int tw_n, int threads, bool interp) {
  HilLayout L;
  L.tw = es * (size_t)m;
  L.perm = L.tw + es * (size_t)tw_n;
  L.q = (L.perm + sizeof(int) * (size_t)m + 15) & ~size_t(15);
  L.scan = L.q + (interp ? es * (size_t)m : 0);
  L.flags = L.scan + (interp ? 2 * sizeof(int2) * (size_t)threads : 0);
  L.total = L.flags + (interp ? (size_t)m : 0);
  return L;
}

// vec (FP32 only, m % 4 == 0, 16-byte aligned rows): four samples per access.
template <class R, bool INTERP>
__global__ void __launch_bounds__(kHilThreads, sizeof(R) == 4 ? MBIR_HIL_MINB : 2)
    hilbert_kernel(const R* __restrict__ y, const uint8_t* __restrict__ mask, cplx_t<R>* __restrict__ c, int nx,
                   int m, Radix rad, const cplx_t<R>* __restrict__ twg, const int* __restrict__ perm, R side,
                   int sw, int vec) {
  using V = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const HilLayout L = hil_layout(sizeof(V), m, rad.tw_lo + rad.tw_hi, blockDim.x, INTERP);
  V* s = reinterpret_cast<V*>(smem_raw);
  const Tw2<V> tw = load_twiddles(reinterpret_cast<V*>(smem_raw + L.tw), twg, rad);
  int* sperm = reinterpret_cast<int*>(smem_raw + L.perm);
  for (int i = threadIdx.x; i < m; i += blockDim.x) sperm[i] = perm[i];
  // interpolating variant: Q [m] (indices, then the filled rows), scan, flags
  V* Q = reinterpret_cast<V*>(smem_raw + L.q);
  int2* scan = reinterpret_cast<int2*>(smem_raw + L.scan);
  uint8_t* M = smem_raw + L.flags;
  const bool interp = INTERP && mask != nullptr;
  const bool on = sw != 0;
  const int pa = 2 * blockIdx.x;
  const bool hb = pa + 1 < nx;
  const size_t oa = (size_t)pa * m, ob = oa + m;
  pdl_wait_release();
  // one sample of both rows: mask, flags, staging
  auto stage = [&](int i, R a, R b, bool ma, bool mb) {
    if (!ma) a = R(0);
    if (!mb) b = R(0);
    if (interp) M[i] = (uint8_t)((ma ? 1 : 0) | (mb ? 2 : 0));
    s[swz(i, on)] = cmk<V>(a, b);
  };
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    if (vec) {
      for (int i = 4 * threadIdx.x; i < m; i += 4 * blockDim.x) {
        const float4 a4 = *reinterpret_cast<const float4*>(y + oa + i);
        const float4 b4 = hb ? *reinterpret_cast<const float4*>(y + ob + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        uchar4 ma = make_uchar4(1, 1, 1, 1), mb = hb ? ma : make_uchar4(0, 0, 0, 0);
        if (mask) {
          ma = *reinterpret_cast<const uchar4*>(mask + oa + i);
          if (hb) mb = *reinterpret_cast<const uchar4*>(mask + ob + i);
        }
        stage(i, a4.x, b4.x, ma.x != 0, mb.x != 0);
        stage(i + 1, a4.y, b4.y, ma.y != 0, mb.y != 0);
        stage(i + 2, a4.z, b4.z, ma.z != 0, mb.z != 0);
        stage(i + 3, a4.w, b4.w, ma.w != 0, mb.w != 0);
      }
      done = true;
    }
  }
  if (!done) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const R a = y[oa + i];
      const R b = hb ? y[ob + i] : R(0);
      const bool ma = !mask || mask[oa + i] != 0;
      const bool mb = hb && (!mask || mask[ob + i] != 0);
      stage(i, a, b, ma, mb);
    }
  }
  __syncthreads();
  if (interp) {
    interp_rows<R>(s, Q, M, scan, m, on);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) s[swz(i, on)] = Q[i];
    __syncthreads();
  }
  fft_dif<false>(s, 1, rad, tw, on);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int q = swz(sperm[k], on);
    const V v = s[q];
    const R g = (k == 0 || 2 * k == m) ? R(0) : (2 * k < m ? R(1) : R(-1));
    s[q] = cmk<V>(g * v.y, -g * v.x);   // -j g (v.x + j v.y)
  }
  __syncthreads();
  fft_dit<true>(s, 1, rad, tw, on);
  const R f = -side / R(m);   // the inverse transform is unnormalised
  // the real part of one sample of both rows: the filled rows, or y again (L2)
  auto real_part = [&](int i, R& a, R& b) {
    if (interp) {
      a = Q[i].x;
      b = Q[i].y;
    } else {
      a = y[oa + i];
      b = hb ? y[ob + i] : R(0);
      if (mask) {
        if (!mask[oa + i]) a = R(0);
        if (hb && !mask[ob + i]) b = R(0);
      }
    }
  };
  if constexpr (sizeof(R) == 4) {
    if (vec) {
      for (int i = 4 * threadIdx.x; i < m; i += 4 * blockDim.x) {
        float a[4], b[4], ha[4], hbv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          real_part(i + j, a[j], b[j]);
          const V h = s[swz(i + j, on)];
          ha[j] = f * h.x;
          hbv[j] = f * h.y;
        }
        float4* ca = reinterpret_cast<float4*>(c + oa + i);
        ca[0] = make_float4(a[0], ha[0], a[1], ha[1]);
        ca[1] = make_float4(a[2], ha[2], a[3], ha[3]);
        if (hb) {
          float4* cb = reinterpret_cast<float4*>(c + ob + i);
          cb[0] = make_float4(b[0], hbv[0], b[1], hbv[1]);
          cb[1] = make_float4(b[2], hbv[2], b[3], hbv[3]);
        }
      }
      return;
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const V h = s[swz(i, on)];
    R a, b;
    real_part(i, a, b);
    c[oa + i] = cmk<V>(a, f * h.x);
    if (hb) c[ob + i] = cmk<V>(b, f * h.y);
  }
}

static size_t hilbert_smem_bytes(size_t es, int m, const Radix& r, bool interp) {
  return hil_layout(es, m, r.tw_lo + r.tw_hi, kHilThreads, interp).total;
}

int ensure_hilbert(mbir_plan p) {
  if (p->tw_m) return MBIR_OK;
  Radix r;
  if (p->m > kMaxFFT || !plan_factor_radix(p->m, &r, 8)) return MBIR_ERR_UNSUPPORTED_SIZE;
  const size_t es = p->precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
  if (hilbert_smem_bytes(es, p->m, r, false) > (size_t)kMaxDynSmem) return MBIR_ERR_UNSUPPORTED_SIZE;
  int rc = plan_fft_tables(p, p->m, &p->rad_m, &p->tw_m, &p->perm_m);
  if (rc) {
    cudaFree(p->tw_m);
    cudaFree(p->perm_m);
    p->tw_m = nullptr;
    p->perm_m = nullptr;
    return rc;
  }
  // the cap, not this plan's size: plans of other lengths share the kernel
#define MBIR_HIL_ATTR(fn) MBIR_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem))
  if (p->precision == MBIR_FP64) {
    MBIR_HIL_ATTR((hilbert_kernel<double, false>));
    MBIR_HIL_ATTR((hilbert_kernel<double, true>));
  } else {
    MBIR_HIL_ATTR((hilbert_kernel<float, false>));
    MBIR_HIL_ATTR((hilbert_kernel<float, true>));
  }
#undef MBIR_HIL_ATTR
  return MBIR_OK;
}

template <class R>
static int hilbert_t(mbir_plan p, const void* y, const uint8_t* mask, void* c, bool interp, cudaStream_t st) {
  const int grid = (p->nx + 1) / 2;
  const R side = p->k_ascending ? R(1) : R(-1);
  const bool iv = interp && mask != nullptr;
  const size_t smem = hilbert_smem_bytes(sizeof(cplx_t<R>), p->m, p->rad_m, iv);
  if (smem > (size_t)kMaxDynSmem) return MBIR_ERR_UNSUPPORTED_SIZE;
  const auto al = [](const void* q, uintptr_t b) { return (reinterpret_cast<uintptr_t>(q) & (b - 1)) == 0; };
  const int vec = sizeof(R) == 4 && (p->m & 3) == 0 && al(y, 16) && al(c, 16) && (!mask || al(mask, 4)) ? 1 : 0;
  {
    ProfScope ps_(p, PC_HILBERT, st);
    auto kernel = iv ? hilbert_kernel<R, true> : hilbert_kernel<R, false>;
    launch(kernel, dim3(grid), dim3(kHilThreads), smem, st, static_cast<const R*>(y), mask,
           static_cast<cplx_t<R>*>(c), p->nx, p->m, p->rad_m, static_cast<const cplx_t<R>*>(p->tw_m),
           (const int*)p->perm_m, side, (p->m & 15) == 0 ? 1 : 0, vec);
  }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

int hilbert_impl(mbir_plan p, const void* y, const uint8_t* mask, void* c, cudaStream_t st, bool interp) {
  int rc = ensure_hilbert(p);
  if (rc) return rc;
  return p->precision == MBIR_FP64 ? hilbert_t<double>(p, y, mask, c, interp, st)
                                   : hilbert_t<float>(p, y, mask, c, interp, st);
}

}  // namespace mbir
