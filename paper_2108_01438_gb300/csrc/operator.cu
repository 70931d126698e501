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
// K-point row (K = 2 nz) in shared memory.  FP32 KB weights come from per-tap
// degree-9 polynomials in the fractional grid position (fitted in FP64 per plan);
// FP64 plans evaluate the Bessel function directly.
#include "common.cuh"
#include "fft.cuh"
#include "operator.cuh"
#include <string.h>

namespace mbir {

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

// This CTA's argument block (the by-value one, or its scan's block in a batch)
// and its index within its scan's grid.
template <class Args>
__device__ __forceinline__ const Args* resolve_args(const Args* a0, const BatchRef<Args>& B, int& blk) {
  blk = blockIdx.x;
  if (B.args == nullptr) return a0;
  int lo = 0, hi = B.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.off[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  blk -= B.off[lo];
  return B.args + lo;
}

// Copy a radix plan into shared memory (no barrier inside).
__device__ __forceinline__ void copy_radix(Radix* dst, const Radix* src) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Radix) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

// Operands of the lateral load/store phases, held in registers.
template <class R>
struct LatEp {
  const void* in;
  void* out;
  const uint8_t* mask;
  const R* y;
  R* pz;
  R* r;
  const void* z1;
  void* z2;
  void* vout;
  const double* scal;
  const void* chirp;
  const void* bhat;
  R scale, mu, delta, tau;
};

// --------------------------------------------------------- column pairs
//
// A lateral tile is moved as column pairs (c, c + 1): with an even row length
// and suitably aligned bases one pair is one vector access.

template <class T> struct PairOf { using V = void; };
template <> struct PairOf<float> { using V = float2; };
template <> struct PairOf<double> { using V = double2; };
template <> struct PairOf<float2> { using V = float4; };
template <> struct PairOf<uint8_t> { using V = uchar2; };

// a = p[o], b = p[o + 1] where in range (unchanged otherwise)
template <class T>
__device__ __forceinline__ void ld2(const T* p, size_t o, bool v2, bool ok0, bool ok1, T& a, T& b) {
  using PV = typename PairOf<T>::V;
  if constexpr (!std::is_same<PV, void>::value) {
    if (v2) {
      const PV t = *reinterpret_cast<const PV*>(p + o);
      memcpy(&a, &t, sizeof(T));
      memcpy(&b, reinterpret_cast<const unsigned char*>(&t) + sizeof(T), sizeof(T));
      return;
    }
  }
  if (ok0) a = p[o];
  if (ok1) b = p[o + 1];
}

template <class T>
__device__ __forceinline__ void st2(T* p, size_t o, bool v2, bool ok0, bool ok1, T a, T b) {
  using PV = typename PairOf<T>::V;
  if constexpr (!std::is_same<PV, void>::value) {
    if (v2) {
      PV t;
      memcpy(&t, &a, sizeof(T));
      memcpy(reinterpret_cast<unsigned char*>(&t) + sizeof(T), &b, sizeof(T));
      *reinterpret_cast<PV*>(p + o) = t;
      return;
    }
  }
  if (ok0) p[o] = a;
  if (ok1) p[o + 1] = b;
}

// The column pair (c, c + 1) of a tile row in shared memory, at an even index i.
// FP32 tiles hold the pair in split form {re_c, re_c+1, im_c, im_c+1} (the
// layout of the paired transform); FP64 tiles hold two complex numbers.
template <class V>
__device__ __forceinline__ void lds2(const V* s, int i, V& a, V& b) {
  if constexpr (sizeof(V) == 8) {
    const float4 t = *reinterpret_cast<const float4*>(s + i);
    a = cmk<V>(t.x, t.z);
    b = cmk<V>(t.y, t.w);
  } else {
    a = s[i];
    b = s[i + 1];
  }
}

template <class V>
__device__ __forceinline__ void sts2(V* s, int i, V a, V b) {
  if constexpr (sizeof(V) == 8) {
    *reinterpret_cast<float4*>(s + i) = make_float4(a.x, b.x, a.y, b.y);
  } else {
    s[i] = a;
    s[i + 1] = b;
  }
}

// The lateral transforms of a tile: FP32 tiles as TC/2 interleaved split pairs
// through the paired transform, FP64 tiles as TC interleaved sequences.
template <class R>
struct LatFFT {
  Tw2<cplx_t<R>> tw;
  TwP twp;
};

template <class R>
__device__ __forceinline__ LatFFT<R> lat_twiddles(cplx_t<R>* tws, const void* twg, const Radix& rad) {
  LatFFT<R> f;
  if constexpr (sizeof(R) == 4)
    f.twp = load_twiddles_p(reinterpret_cast<float4*>(tws), reinterpret_cast<const float2*>(twg), rad);
  else
    f.tw = load_twiddles(tws, reinterpret_cast<const cplx_t<R>*>(twg), rad);
  return f;
}

template <class R, bool INV, bool DIT>
__device__ __forceinline__ void lat_fft(cplx_t<R>* s, int TC, const Radix& rad, const LatFFT<R>& f) {
  if constexpr (sizeof(R) == 4) {
    if constexpr (DIT) fft_p_dit<INV>(reinterpret_cast<float4*>(s), TC >> 1, rad, f.twp);
    else fft_p_dif<INV>(reinterpret_cast<float4*>(s), TC >> 1, rad, f.twp);
  } else {
    if constexpr (DIT) fft_dit<INV>(s, TC, rad, f.tw, false);
    else fft_dif<INV>(s, TC, rad, f.tw, false);
  }
}

// Bluestein (chirp-z) form of the lateral transform, for widths nx that do not
// factor into radices 2..8: with c_k = e^{-j pi k^2 / nx},
//   X_l = sum_p x_p e^{-2 pi j l p / nx} = c_l sum_p (x_p c_p) conj(c)_{l-p},
// a linear convolution that an nxl-point transform pair computes exactly
// (nxl = rad.n >= 2 nx - 1, so indices l - p never wrap onto each other).  The
// tile holds rows [0, nxl): rows p < nx are multiplied by the chirp and the rest
// zeroed, a forward dif transform leaves the spectrum digit-reversed, where it
// is multiplied by the plan's transformed conjugate chirp (stored digit-reversed,
// divided by nxl), and an inverse dit transform brings the convolution back to
// natural order, multiplied by the chirp again.  The inverse transform is
// conj(forward(conj x)).  Output rows [0, nx) are in natural order.
template <class R, bool INV>
__device__ __noinline__ void lat_bluestein(cplx_t<R>* s, int TC, int nx, const Radix& rad, const LatFFT<R>& tw,
                                           const cplx_t<R>* chirp, const cplx_t<R>* bhat) {
  using V = cplx_t<R>;
  const int half = TC >> 1, hs = __ffs(half) - 1;
  const int npairs = rad.n * half;
  const V zero = cmk<V>(R(0), R(0));
  for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
    const int p = i >> hs, idx = p * TC + 2 * (i & (half - 1));
    V va = zero, vb = zero;
    if (p < nx) {
      lds2(s, idx, va, vb);
      if (INV) {
        va = cconj(va);
        vb = cconj(vb);
      }
      const V c = chirp[p];
      va = cmul(va, c);
      vb = cmul(vb, c);
    }
    sts2(s, idx, va, vb);
  }
  __syncthreads();
  lat_fft<R, false, false>(s, TC, rad, tw);
  for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
    const int p = i >> hs, idx = p * TC + 2 * (i & (half - 1));
    V va, vb;
    lds2(s, idx, va, vb);
    const V h = bhat[p];
    sts2(s, idx, cmul(va, h), cmul(vb, h));
  }
  __syncthreads();
  lat_fft<R, true, true>(s, TC, rad, tw);
  for (int i = threadIdx.x; i < nx * half; i += blockDim.x) {
    const int p = i >> hs, idx = p * TC + 2 * (i & (half - 1));
    V va, vb;
    lds2(s, idx, va, vb);
    const V c = chirp[p];
    va = cmul(va, c);
    vb = cmul(vb, c);
    if (INV) {
      va = cconj(va);
      vb = cconj(vb);
    }
    sts2(s, idx, va, vb);
  }
  __syncthreads();
}

// The lateral transform of a tile: the plan's mixed-radix FFT (dif: digit-reversed
// out; dit: digit-reversed in, natural out), or the Bluestein form when the plan
// has a chirp (natural order in and out either way).
// Kernels instantiated with BLU = false never contain the Bluestein code (it
// would raise their register pressure); BLU = true kernels check per plan.
template <class R, bool INV, bool DIT, bool BLU>
__device__ __forceinline__ void lat_xform(cplx_t<R>* s, int TC, int nx, const Radix& rad, const LatFFT<R>& tw,
                                          const void* chirp, const void* bhat) {
  if constexpr (BLU) {
    if (chirp) {
      lat_bluestein<R, INV>(s, TC, nx, rad, tw, static_cast<const cplx_t<R>*>(chirp),
                            static_cast<const cplx_t<R>*>(bhat));
      return;
    }
  }
  lat_fft<R, INV, DIT>(s, TC, rad, tw);
}

__device__ __forceinline__ bool al(const void* p, unsigned bytes) {
  return p == nullptr || (reinterpret_cast<uintptr_t>(p) & (bytes - 1)) == 0;
}

// Every base a mode touches allows pair accesses.
template <class R, int MODE, class A>
__device__ __forceinline__ bool lat_pairs_aligned(const A& a) {
  const unsigned c2 = 2 * sizeof(cplx_t<R>) <= 16 ? 2 * sizeof(cplx_t<R>) : 16, r2 = 2 * sizeof(R);
  const bool real_in = MODE == LAT_R2C_MASK;
  bool ok = al(a.in, real_in ? r2 : c2) && al(a.mask, 2);
  if constexpr (MODE == LAT_C2R_INV_MASK) ok = ok && al(a.out, r2);
  else ok = ok && al(a.out, c2);
  if constexpr (MODE == LAT_SOLVE_FWD || MODE == LAT_SOLVE_MID) ok = ok && al(a.y, r2) && al(a.pz, r2) && al(a.r, r2);
  if constexpr (MODE == LAT_SOLVE_ADJ_L1 || MODE == LAT_SOLVE_ADJ_V || MODE == LAT_POWER_ADJ || MODE == LAT_POWER_FWD)
    ok = ok && al(a.z1, c2) && al(a.z2, c2) && al(a.vout, c2);
  return ok;
}

// --------------------------------------------------------------- lateral FFT

// Load the pair (p, c), (p, c + 1) of the lateral input as complex.
template <class R, int MODE, class A>
__device__ __forceinline__ void lat_load2(const A& a, size_t off, bool v2, bool ok0, bool ok1, cplx_t<R>& va,
                                          cplx_t<R>& vb) {
  using V = cplx_t<R>;
  if constexpr (MODE == LAT_R2C_MASK) {
    R x0 = R(0), x1 = R(0);
    ld2(reinterpret_cast<const R*>(a.in), off, v2, ok0, ok1, x0, x1);
    if (a.mask != nullptr) {
      uint8_t m0 = 0, m1 = 0;
      ld2(a.mask, off, v2, ok0, ok1, m0, m1);
      if (!m0) x0 = R(0);
      if (!m1) x1 = R(0);
    }
    va = cmk<V>(x0, R(0));
    vb = cmk<V>(x1, R(0));
  } else {
    ld2(reinterpret_cast<const V*>(a.in), off, v2, ok0, ok1, va, vb);
  }
}

// Operands an epilogue reads besides the transform output, fetched ahead of use
// so that several rows' loads are in flight at once.
template <class R>
struct EpOps {
  R y, prev;
  cplx_t<R> z1, z2;
  uint8_t meas;
};

template <class R, int MODE, class A>
__device__ __forceinline__ void lat_prefetch2(const A& a, size_t off, bool v2, bool ok0, bool ok1, EpOps<R>& o0,
                                              EpOps<R>& o1) {
  using V = cplx_t<R>;
  if constexpr (MODE == LAT_C2R_INV_MASK || MODE == LAT_SOLVE_FWD || MODE == LAT_SOLVE_MID ||
                MODE == LAT_POWER_MID) {
    o0.meas = o1.meas = 1;
    if (a.mask != nullptr) ld2(a.mask, off, v2, ok0, ok1, o0.meas, o1.meas);
  }
  if constexpr (MODE == LAT_SOLVE_FWD || MODE == LAT_SOLVE_MID) {
    o0.y = o1.y = o0.prev = o1.prev = R(0);
    ld2(a.y, off, v2, ok0, ok1, o0.y, o1.y);
    ld2(static_cast<const R*>(a.pz), off, v2, ok0, ok1, o0.prev, o1.prev);
  } else if constexpr (MODE == LAT_SOLVE_ADJ_L1 || MODE == LAT_SOLVE_ADJ_V) {
    ld2(reinterpret_cast<const V*>(a.z1), off, v2, ok0, ok1, o0.z1, o1.z1);
    ld2(reinterpret_cast<const V*>(a.z2), off, v2, ok0, ok1, o0.z2, o1.z2);
  } else if constexpr (MODE == LAT_POWER_ADJ) {
    o0.z1 = o1.z1 = cmk<V>(R(0), R(0));
    ld2(reinterpret_cast<const V*>(a.z1), off, v2, ok0, ok1, o0.z1, o1.z1);
  }
}

// The epilogue operands of the CTA's columns [c0, c0 + TC) that the kernel just
// before this one does not write -- the measurements, the mask, Phi z^{k-2}, the
// iterates z^{k-1}, z^{k-2} -- pulled into L2 ahead of the dependency wait.
template <class R, int MODE, class A>
__device__ __forceinline__ void lat_prefetch_l2(const A& a, int nx, int C, int c0, int TC) {
  using V = cplx_t<R>;
  const int ncol = C - c0 < TC ? C - c0 : TC;
  if (ncol <= 0) return;
  if constexpr (MODE == LAT_C2R_INV_MASK || MODE == LAT_SOLVE_FWD || MODE == LAT_SOLVE_MID ||
                MODE == LAT_POWER_MID)
    prefetch_l2_rows(a.mask, nx, (size_t)C, (size_t)c0, ncol);
  if constexpr (MODE == LAT_SOLVE_FWD || MODE == LAT_SOLVE_MID) {
    prefetch_l2_rows(a.y, nx, sizeof(R) * C, sizeof(R) * c0, (int)sizeof(R) * ncol);
    prefetch_l2_rows(a.pz, nx, sizeof(R) * C, sizeof(R) * c0, (int)sizeof(R) * ncol);
  }
  if constexpr (MODE == LAT_SOLVE_ADJ_L1 || MODE == LAT_SOLVE_ADJ_V || MODE == LAT_POWER_ADJ)
    prefetch_l2_rows(a.z1, nx, sizeof(V) * C, sizeof(V) * c0, (int)sizeof(V) * ncol);
  if constexpr (MODE == LAT_SOLVE_ADJ_L1 || MODE == LAT_SOLVE_ADJ_V)
    prefetch_l2_rows(a.z2, nx, sizeof(V) * C, sizeof(V) * c0, (int)sizeof(V) * ncol);
}

// Measurement-side FISTA epilogue of one element (Eq. alg): pz = s Re{S}/nx,
// r = (1 + mu) pz - mu pz_prev - s y; accumulates (pz - s y)^2.
template <class R, class A>
__device__ __forceinline__ R solve_meas(const A& a, R sre, const EpOps<R>& o, R& pz, R& part) {
  pz = o.meas ? sre * a.scale : R(0);
  const R yv = o.meas ? o.y : R(0);
  const R d = pz - yv;
  part += d * d;
  return (R(1) + a.mu) * pz - a.mu * o.prev - yv;
}

// Image-side epilogue of one element: x^k - delta g, then the l1 prox (ADJ_L1) or
// the pre-prox image v (ADJ_V).
template <class R, int MODE, class A>
__device__ __forceinline__ cplx_t<R> solve_img(const A& a, cplx_t<R> g, const EpOps<R>& o, R& part) {
  using V = cplx_t<R>;
  V xv;
  xv.x = o.z1.x + a.mu * (o.z1.x - o.z2.x) - a.delta * g.x;
  xv.y = o.z1.y + a.mu * (o.z1.y - o.z2.y) - a.delta * g.y;
  if constexpr (MODE == LAT_SOLVE_ADJ_L1) {
    const R mag = sqrt(xv.x * xv.x + xv.y * xv.y);
    const R sh = mag > a.tau ? R(1) - a.tau / mag : R(0);
    xv.x *= sh;
    xv.y *= sh;
    part += mag > a.tau ? mag - a.tau : R(0);
  }
  return xv;
}

// Store the pair of transform outputs (va, vb) at (p, c), (p, c + 1).
template <class R, int MODE, class A>
__device__ __forceinline__ void lat_store2(const A& a, size_t off, bool v2, bool ok0, bool ok1, cplx_t<R> va,
                                           cplx_t<R> vb, const EpOps<R>& o0, const EpOps<R>& o1, R& part,
                                           R& part2) {
  using V = cplx_t<R>;
  if constexpr (MODE == LAT_C2R_INV_MASK) {
    st2(reinterpret_cast<R*>(a.out), off, v2, ok0, ok1, o0.meas ? va.x * a.scale : R(0),
        o1.meas ? vb.x * a.scale : R(0));
  } else if constexpr (MODE == LAT_SOLVE_FWD) {
    R pa, pb;
    R pa_part = R(0), pb_part = R(0);
    const R ra = solve_meas<R>(a, va.x, o0, pa, pa_part);
    const R rb = solve_meas<R>(a, vb.x, o1, pb, pb_part);
    if (ok0) part += pa_part;
    if (ok1) part += pb_part;
    st2(a.pz, off, v2, ok0, ok1, pa, pb);
    st2(a.r, off, v2, ok0, ok1, ra, rb);
  } else if constexpr (MODE == LAT_SOLVE_ADJ_L1 || MODE == LAT_SOLVE_ADJ_V) {
    R qa = R(0), qb = R(0);
    const V xa = solve_img<R, MODE>(a, va, o0, qa);
    const V xb = solve_img<R, MODE>(a, vb, o1, qb);
    if (ok0) part += qa;
    if (ok1) part += qb;
    st2(reinterpret_cast<V*>(MODE == LAT_SOLVE_ADJ_L1 ? a.z2 : a.vout), off, v2, ok0, ok1, xa, xb);
  } else if constexpr (MODE == LAT_POWER_ADJ) {
    // w = Phi^H Phi v, with <v, w> and ||w||^2 partial sums
    if (ok0) {
      part += o0.z1.x * va.x + o0.z1.y * va.y;
      part2 += va.x * va.x + va.y * va.y;
    }
    if (ok1) {
      part += o1.z1.x * vb.x + o1.z1.y * vb.y;
      part2 += vb.x * vb.x + vb.y * vb.y;
    }
    st2(reinterpret_cast<V*>(a.out), off, v2, ok0, ok1, va, vb);
  } else {
    st2(reinterpret_cast<V*>(a.out), off, v2, ok0, ok1, cscale(va, a.scale), cscale(vb, a.scale));
  }
}

template <int MODE>
constexpr bool lat_is_mid() {
  return MODE == LAT_SOLVE_MID || MODE == LAT_POWER_MID;
}

// The input pair (p, c), (p, c + 1) of a lateral tile as the transform takes it:
// loaded (masked for R2C), scaled by 1/||w|| and written out as v for the power
// iteration's first pass, conjugated for the middle passes (their inverse
// transform runs as a forward transform of conj S).
template <class R, int MODE, class A>
__device__ __forceinline__ void lat_in2(const A& a, size_t off, bool v2, bool ok0, bool ok1, R fscale,
                                        cplx_t<R>& va, cplx_t<R>& vb) {
  using V = cplx_t<R>;
  va = vb = cmk<V>(R(0), R(0));
  lat_load2<R, MODE>(a, off, v2, ok0, ok1, va, vb);
  if constexpr (MODE == LAT_POWER_FWD) {
    va = cscale(va, fscale);
    vb = cscale(vb, fscale);
    st2(reinterpret_cast<V*>(a.vout), off, v2, ok0, ok1, va, vb);
  }
  if constexpr (lat_is_mid<MODE>()) {
    va.y = -va.y;
    vb.y = -vb.y;
  }
}

// Pass 0 of the FP32 dif transform (radix RR, span N/RR) run on the way in from
// global memory: each thread loads the RR rows of its butterflies straight into
// registers, so the tile is written to shared memory once, already through that
// pass (staging would write it, and the pass read and write it again).
template <int RR, bool INV, int MODE, class A>
__device__ __forceinline__ void lat_first_pass_p(const A& a, float4* s4, int N, int half, int hs, int C, int c,
                                                 bool v2, bool ok0, bool ok1, float fscale, const TwP& tw) {
  const int M = N / RR, q = threadIdx.x & (half - 1);
  for (int j = threadIdx.x >> hs; j < M; j += (int)blockDim.x >> hs) {
    PC v[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      float2 va, vb;
      lat_in2<float, MODE>(a, (size_t)(j + r * M) * C + c, v2, ok0, ok1, fscale, va, vb);
      v[r] = PC{make_float2(va.x, vb.x), make_float2(va.y, vb.y)};
    }
    dft_small_p<RR, INV>(v, tw, N);
    if (j != 0) apply_twiddles_p<RR, INV>(v, tw, j);
#pragma unroll
    for (int r = 0; r < RR; ++r) st_pc(s4, (j + r * M) * half + q, v[r]);
  }
}

// The last pass (pass 0, span N/RR) of the FP32 forward dit transform run on the
// way out: its outputs are in natural row order, so each thread writes the RR rows
// of its butterflies, scaled, straight to global memory.
template <int RR, class A>
__device__ __forceinline__ void lat_last_pass_store_p(const A& a, const float4* s4, int N, int half, int hs, int C,
                                                      int c, bool v2, bool ok0, bool ok1, const TwP& tw) {
  const int M = N / RR, q = threadIdx.x & (half - 1);
  const float sc = a.scale;
  for (int j = threadIdx.x >> hs; j < M; j += (int)blockDim.x >> hs) {
    PC v[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) v[r] = ld_pc(s4, (j + r * M) * half + q);
    if (j != 0) apply_twiddles_p<RR, false>(v, tw, j);
    dft_small_p<RR, false>(v, tw, N);
#pragma unroll
    for (int r = 0; r < RR; ++r)
      st2(reinterpret_cast<float2*>(a.out), (size_t)(j + r * M) * C + c, v2, ok0, ok1,
          make_float2(v[r].re.x * sc, v[r].im.x * sc), make_float2(v[r].re.y * sc, v[r].im.y * sc));
  }
}

// The last pass (span 1, radix RL) of an FP32 dif transform run on the way out:
// its outputs sit at positions blk RL + r, natural row siperm[pos]; the mode's
// epilogue runs there and writes straight to global memory (a read-out would
// read the tile back after that pass wrote it).
template <int RL, bool INV, int MODE, class A>
__device__ __forceinline__ void lat_last_pass_epi_p(const A& a, const float4* s4, int N, int half, int hs, int C,
                                                    int c, bool v2, bool ok0, bool ok1, const int* siperm,
                                                    const TwP& tw, float& part, float& part2) {
  const int q = threadIdx.x & (half - 1);
  constexpr bool kHoist = RL <= kEpHoistMax;
  for (int blk = threadIdx.x >> hs; blk < N / RL; blk += (int)blockDim.x >> hs) {
    // with a small radix the epilogue operands are loaded first, so that their
    // latency overlaps the shared-memory reads and the butterfly
    EpOps<float> o0[kHoist ? RL : 1], o1[kHoist ? RL : 1];
    if constexpr (kHoist) {
#pragma unroll
      for (int r = 0; r < RL; ++r)
        lat_prefetch2<float, MODE>(a, (size_t)siperm[blk * RL + r] * C + c, v2, ok0, ok1, o0[r], o1[r]);
    }
    PC v[RL];
#pragma unroll
    for (int r = 0; r < RL; ++r) v[r] = ld_pc(s4, (blk * RL + r) * half + q);
    dft_small_p<RL, INV>(v, tw, N);
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const size_t off = (size_t)siperm[blk * RL + r] * C + c;
      const int k = kHoist ? r : 0;
      if constexpr (!kHoist) lat_prefetch2<float, MODE>(a, off, v2, ok0, ok1, o0[0], o1[0]);
      lat_store2<float, MODE>(a, off, v2, ok0, ok1, make_float2(v[r].re.x, v[r].im.x),
                              make_float2(v[r].re.y, v[r].im.y), o0[k], o1[k], part, part2);
    }
  }
}

// The middle of the measurement pass in registers: the last dif pass of the
// inverse transform (span 1, radix RL), the measurement epilogue at the natural
// rows of its outputs, and the first dit pass of the forward transform, which
// works on the same RL positions (span 1, no twiddles).  The tile is read and
// written once for the three.
template <int RL, int MODE, class A>
__device__ __forceinline__ void lat_mid_center_p(const A& a, float4* s4, int N, int half, int hs, int C, int c,
                                                 bool v2, bool ok0, bool ok1, const int* siperm, const TwP& tw,
                                                 float& part) {
  const int q = threadIdx.x & (half - 1);
  constexpr bool kHoist = RL <= kEpHoistMax;
  for (int blk = threadIdx.x >> hs; blk < N / RL; blk += (int)blockDim.x >> hs) {
    EpOps<float> e0[kHoist ? RL : 1], e1[kHoist ? RL : 1];
    if constexpr (kHoist) {
#pragma unroll
      for (int r = 0; r < RL; ++r)
        lat_prefetch2<float, MODE>(a, (size_t)siperm[blk * RL + r] * C + c, v2, ok0, ok1, e0[r], e1[r]);
    }
    PC v[RL];
#pragma unroll
    for (int r = 0; r < RL; ++r) v[r] = ld_pc(s4, (blk * RL + r) * half + q);
    dft_small_p<RL, false>(v, tw, N);
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const size_t off = (size_t)siperm[blk * RL + r] * C + c;
      const int k = kHoist ? r : 0;
      if constexpr (!kHoist) lat_prefetch2<float, MODE>(a, off, v2, ok0, ok1, e0[0], e1[0]);
      const EpOps<float>& o0 = e0[k];
      const EpOps<float>& o1 = e1[k];
      float ra, rb;
      if constexpr (MODE == LAT_SOLVE_MID) {
        float pa, pb, qa = 0.f, qb = 0.f;
        ra = solve_meas<float>(a, v[r].re.x, o0, pa, qa);
        rb = solve_meas<float>(a, v[r].re.y, o1, pb, qb);
        if (ok0) part += qa;
        if (ok1) part += qb;
        st2(a.pz, off, v2, ok0, ok1, pa, pb);
      } else {
        ra = o0.meas ? v[r].re.x * a.scale : 0.f;
        rb = o1.meas ? v[r].re.y * a.scale : 0.f;
      }
      v[r] = PC{make_float2(ok0 ? ra : 0.f, ok1 ? rb : 0.f), make_float2(0.f, 0.f)};
    }
    dft_small_p<RL, false>(v, tw, N);
#pragma unroll
    for (int r = 0; r < RL; ++r) st_pc(s4, (blk * RL + r) * half + q, v[r]);
  }
  __syncthreads();
}

// One lateral tile: `a` supplies the operands (the launch's argument block, or a
// register copy of a batched scan's block), `rad` the nx-point radix plan.
// Thread t owns the column pair b = 2 (t mod TC/2) of rows p0 = t / (TC/2),
// p0 + pstep, ...; the staging loops keep U rows of loads in flight per thread.
//
// Single-transform modes: stage in natural order, one decimation-in-frequency
// FFT, epilogue on the digit-reversed result.  Mid modes (the measurement side of
// Phi^H Phi): inverse FFT (dif), the measurement epilogue in place on the
// digit-reversed tile, forward FFT (dit, digit-reversed in, natural out).
// FZ: 0 the plain staging, transform and read-out; 1 the fused first and last
// passes only (the launch checked that the plan's radices allow them); 2 either,
// chosen per tile (batched launches, whose scans may differ).
template <class R, int MODE, bool BLU, int FZ, class A>
__device__ __forceinline__ void lateral_body(const A& a, const Radix& rad, int nx, int TC, int C, int blk,
                                             const void* twg, const int* perm, double* partial) {
  using V = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s = reinterpret_cast<V*>(smem_raw);
  V* tws = s + rad.n * TC;   // rad.n = nx, or the Bluestein length
  const int tid = threadIdx.x;
  const LatFFT<R> tw = lat_twiddles<R>(tws, twg, rad);
  // digit-reversal table in shared memory: the read-out and the middle epilogue
  // index the tile with it once per row, and a global load there would stall
  // the dependent shared-memory read (first read after the transform's barriers)
  int* sperm = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(tws) + 16 * (rad.tw_lo + rad.tw_hi));
  // and its inverse, the natural row of each tile position (the fused last passes)
  int* siperm = sperm + nx;
  for (int i = tid; i < nx; i += blockDim.x) {
    const int pi = perm[i];
    sperm[i] = pi;
    siperm[pi] = i;
  }
  const int half = TC >> 1, hs = __ffs(half) - 1;
  const int b = 2 * (tid & (half - 1));
  const int p0 = tid >> hs, pstep = (int)blockDim.x >> hs;
  const int c = blk * TC + b;
  const bool ok0 = c < C, ok1 = c + 1 < C;
  const bool v2 = ok1 && (C & 1) == 0 && lat_pairs_aligned<R, MODE>(a);
  constexpr int U = kLatUnroll;
  constexpr bool kMid = lat_is_mid<MODE>();
  constexpr bool INV = !(MODE == LAT_C2C_FWD || MODE == LAT_R2C_MASK || MODE == LAT_POWER_FWD);
  // FP32 mixed-radix tiles whose first radix is 2, 4 or 8 run the transform's
  // pass 0 on the way in (and the middle passes' last dit pass on the way out)
  static_assert(FZ == 0 || (sizeof(R) == 4 && !BLU), "fused passes: FP32 mixed-radix tiles only");
  int r0 = 0;
  if constexpr (FZ == 1) {
    r0 = rad.r[0];
  } else if constexpr (FZ == 2) {
    const int rl = rad.r[rad.npass - 1];
    if (rad.npass >= 2 && (rad.r[0] == 8 || rad.r[0] == 4 || rad.r[0] == 2) && (rl == 8 || rl == 4 || rl == 2))
      r0 = rad.r[0];
  }
  lat_prefetch_l2<R, MODE>(a, nx, C, blk * TC, TC);
  pdl_wait_release();
  R fscale = R(1);
  if constexpr (MODE == LAT_POWER_FWD) fscale = R(a.scal[1]);
  if constexpr (FZ != 0) {
    if (r0) {
      // the pass's twiddles come from the table the CTA's threads just staged
      __syncthreads();
      float4* s4 = reinterpret_cast<float4*>(s);
      constexpr bool INV0 = kMid ? false : INV;
      if (r0 == 8) lat_first_pass_p<8, INV0, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, fscale, tw.twp);
      else if (r0 == 4) lat_first_pass_p<4, INV0, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, fscale, tw.twp);
      else lat_first_pass_p<2, INV0, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, fscale, tw.twp);
    }
  }
  if (FZ != 1 && !r0) {
    const V zero = cmk<V>(R(0), R(0));
    for (int p = p0; p < nx; p += U * pstep) {
      V va[U], vb[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        va[u] = vb[u] = zero;
        const int pp = p + u * pstep;
        if (pp < nx) lat_load2<R, MODE>(a, (size_t)pp * C + c, v2, ok0, ok1, va[u], vb[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int pp = p + u * pstep;
        if (pp < nx) {
          if constexpr (MODE == LAT_POWER_FWD) {
            va[u] = cscale(va[u], fscale);
            vb[u] = cscale(vb[u], fscale);
            st2(reinterpret_cast<V*>(a.vout), (size_t)pp * C + c, v2, ok0, ok1, va[u], vb[u]);
          }
          if constexpr (kMid) {
            // inverse transform as conj(FFT(conj S)); the epilogue reads only its real part
            va[u].y = -va[u].y;
            vb[u].y = -vb[u].y;
          }
          sts2(s, pp * TC + b, va[u], vb[u]);
        }
      }
    }
  }
  __syncthreads();

  // per-thread partial sums in the working precision (a thread adds a few dozen
  // terms; FP64 arithmetic is a small fraction of FP32 throughput on this GPU),
  // the block and grid reductions in FP64
  R part = R(0), part2 = R(0);
  bool fused = false;
  if constexpr (FZ != 0) {
    if (r0) {
      // pass 0 ran on the way in; the last pass runs on the way out (and, in the
      // middle passes, together with the epilogue and the forward transform's first)
      float4* s4 = reinterpret_cast<float4*>(s);
      const int rl = rad.r[rad.npass - 1];
      if constexpr (kMid) {
        fft_p_dif<false>(s4, half, rad, tw.twp, 1, rad.npass - 1);
        if (rl == 8) lat_mid_center_p<8, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, siperm, tw.twp, part);
        else if (rl == 4) lat_mid_center_p<4, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, siperm, tw.twp, part);
        else lat_mid_center_p<2, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, siperm, tw.twp, part);
        fft_p_dit<false>(s4, half, rad, tw.twp, 1, rad.npass - 2);
        if (r0 == 8) lat_last_pass_store_p<8>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, tw.twp);
        else if (r0 == 4) lat_last_pass_store_p<4>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, tw.twp);
        else lat_last_pass_store_p<2>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, tw.twp);
      } else {
        fft_p_dif<INV>(s4, half, rad, tw.twp, 1, rad.npass - 1);
        if (rl == 8)
          lat_last_pass_epi_p<8, INV, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, siperm, tw.twp, part, part2);
        else if (rl == 4)
          lat_last_pass_epi_p<4, INV, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, siperm, tw.twp, part, part2);
        else
          lat_last_pass_epi_p<2, INV, MODE>(a, s4, nx, half, hs, C, c, v2, ok0, ok1, siperm, tw.twp, part, part2);
      }
      fused = true;
    }
  }
  if (FZ == 1 || fused) {
    // done
  } else if constexpr (kMid) {
    // inverse as a forward dif of conj S, the epilogue in place on the
    // digit-reversed tile, then the forward dit
    lat_xform<R, false, false, BLU>(s, TC, nx, rad, tw, a.chirp, a.bhat);
    constexpr int UM = 2;
    for (int p = p0; p < nx; p += UM * pstep) {
      EpOps<R> oa[UM], ob[UM];
#pragma unroll
      for (int u = 0; u < UM; ++u) {
        const int pp = p + u * pstep;
        if (pp < nx) lat_prefetch2<R, MODE>(a, (size_t)pp * C + c, v2, ok0, ok1, oa[u], ob[u]);
      }
#pragma unroll
      for (int u = 0; u < UM; ++u) {
        const int pp = p + u * pstep;
        if (pp >= nx) continue;
        const size_t off = (size_t)pp * C + c;
        const int slot = sperm[pp] * TC + b;
        V xa, xb;
        lds2(s, slot, xa, xb);
        R ra, rb;
        if constexpr (MODE == LAT_SOLVE_MID) {
          R pa, pb;
          R qa = R(0), qb = R(0);
          ra = solve_meas<R>(a, xa.x, oa[u], pa, qa);
          rb = solve_meas<R>(a, xb.x, ob[u], pb, qb);
          if (ok0) part += qa;
          if (ok1) part += qb;
          st2(a.pz, off, v2, ok0, ok1, pa, pb);
        } else {
          ra = oa[u].meas ? xa.x * a.scale : R(0);
          rb = ob[u].meas ? xb.x * a.scale : R(0);
        }
        sts2(s, slot, cmk<V>(ok0 ? ra : R(0), R(0)), cmk<V>(ok1 ? rb : R(0), R(0)));
      }
    }
    __syncthreads();
    lat_xform<R, false, true, BLU>(s, TC, nx, rad, tw, a.chirp, a.bhat);
    for (int p = p0; p < nx; p += pstep) {
      V xa, xb;
      lds2(s, p * TC + b, xa, xb);
      st2(reinterpret_cast<V*>(a.out), (size_t)p * C + c, v2, ok0, ok1, cscale(xa, a.scale), cscale(xb, a.scale));
    }
  } else {
    lat_xform<R, INV, false, BLU>(s, TC, nx, rad, tw, a.chirp, a.bhat);
    constexpr int UE = 4;
    for (int p = p0; p < nx; p += UE * pstep) {
      EpOps<R> oa[UE], ob[UE];
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int pp = p + u * pstep;
        if (pp < nx) lat_prefetch2<R, MODE>(a, (size_t)pp * C + c, v2, ok0, ok1, oa[u], ob[u]);
      }
#pragma unroll
      for (int u = 0; u < UE; ++u) {
        const int pp = p + u * pstep;
        if (pp >= nx) continue;
        V xa, xb;
        lds2(s, sperm[pp] * TC + b, xa, xb);
        lat_store2<R, MODE>(a, (size_t)pp * C + c, v2, ok0, ok1, xa, xb, oa[u], ob[u], part, part2);
      }
    }
  }
  if constexpr (MODE == LAT_SOLVE_FWD || MODE == LAT_SOLVE_MID || MODE == LAT_SOLVE_ADJ_L1) {
    const double t = block_sum(double(part));
    if (tid == 0) partial[blk] = t;
  } else if constexpr (MODE == LAT_POWER_ADJ) {
    const double t = block_sum(double(part));
    __syncthreads();
    const double t2 = block_sum(double(part2));
    if (tid == 0) {
      partial[2 * blk] = t;
      partial[2 * blk + 1] = t2;
    }
  }
}

template <class R, int MODE, bool BAT, bool BLU, int FZ = 0>
__global__ void __launch_bounds__(BAT ? kLatThreadsBatch : kLatThreads, sizeof(R) == 4 ? kLatMinBlocks : 1)
lateral_kernel(const __grid_constant__ LatArgs<R> a0, const BatchRef<LatArgs<R>> B) {
  if constexpr (!BAT) {
    lateral_body<R, MODE, BLU, FZ>(a0, a0.rad, a0.nx, a0.tc, a0.cols, (int)blockIdx.x, a0.tw, a0.perm, a0.partial);
  } else {
    int blk;
    const LatArgs<R>& A = *resolve_args(&a0, B, blk);
    __shared__ Radix rad;
    copy_radix(&rad, &A.rad);
    // the scan's operands in shared memory, where the body reads them as it needs
    // them (a register copy of all of them made the kernel spill)
    __shared__ LatEp<R> e;
    if (threadIdx.x == 0) {
      e.in = A.in;
      e.out = A.out;
      e.mask = A.mask;
      e.y = A.y;
      e.pz = A.pz;
      e.r = A.r;
      e.z1 = A.z1;
      e.z2 = A.z2;
      e.vout = A.vout;
      e.scal = A.scal;
      e.chirp = A.chirp;
      e.bhat = A.bhat;
      e.scale = A.scale;
      e.mu = B.set_mu ? R(B.mu) : A.mu;
      e.delta = A.delta;
      e.tau = A.tau;
    }
    __syncthreads();
    lateral_body<R, MODE, BLU, FZ>(e, rad, A.nx, A.tc, A.cols, blk, A.tw, A.perm, A.partial);
  }
}

// The y-axis transform of a volume: lateral_body over the ny rows of every px slab
// (blockIdx.y) of an [nx][ny][cols] array, in place or not (each CTA stages its
// whole tile before it writes).  Complex transforms only.  Like the batched
// kernels it works from a register copy of its operands, in 256-thread CTAs.
template <class R, int MODE, bool BLU>
__global__ void __launch_bounds__(kLatThreadsBatch, sizeof(R) == 4 ? kLatMinBlocks : 1)
lateral_slab_kernel(const __grid_constant__ LatArgs<R> a0, long long slab) {
  static_assert(MODE == LAT_C2C_FWD || MODE == LAT_C2C_INV, "complex slab transforms only");
  const size_t off = (size_t)blockIdx.y * (size_t)slab;
  LatEp<R> e;
  e.in = static_cast<const cplx_t<R>*>(a0.in) + off;
  e.out = static_cast<cplx_t<R>*>(a0.out) + off;
  e.mask = nullptr;
  e.y = nullptr;
  e.pz = nullptr;
  e.r = nullptr;
  e.z1 = nullptr;
  e.z2 = nullptr;
  e.vout = nullptr;
  e.scal = nullptr;
  e.chirp = a0.chirp;
  e.bhat = a0.bhat;
  e.scale = a0.scale;
  e.mu = e.delta = e.tau = R(0);
  lateral_body<R, MODE, BLU, 0>(e, a0.rad, a0.nx, a0.tc, a0.cols, (int)blockIdx.x, a0.tw, a0.perm, nullptr);
}

// ------------------------------------------------------------- KB weights

// Weights of the J taps at fractional grid position frac (tap j at offset
// J/2 - 1 - j + frac from the point).  The kernel is even, so tap J-1-j at x is
// tap j at -x: one polynomial per mirrored pair, split into its even and odd
// halves in x^2, gives both weights (w = E(x^2) +- x O(x^2)).
template <class R, int J>
__device__ __forceinline__ void kb_weights(R frac, const RowArgs<R>& a, R (&w)[J]) {
  if constexpr (sizeof(R) == 4) {
    static_assert(kKbDeg % 2 == 1 && J % 2 == 0, "paired taps need an odd degree and an even width");
    const float x = frac - 0.5f, x2 = x * x;
#pragma unroll
    for (int j = 0; j < J / 2; ++j) {
      float e = a.kbpoly[j][kKbDeg - 1], o = a.kbpoly[j][kKbDeg];
#pragma unroll
      for (int d = kKbDeg - 3; d >= 0; d -= 2) {
        e = fmaf(e, x2, a.kbpoly[j][d]);
        o = fmaf(o, x2, a.kbpoly[j][d + 1]);
      }
      w[j] = fmaf(x, o, e);
      w[J - 1 - j] = fmaf(-x, o, e);
    }
  } else {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const double u = frac + double(J / 2 - 1 - j);
      const double r = 1.0 - (2.0 * u / J) * (2.0 * u / J);
      w[j] = r < 0.0 ? 0.0 : cyl_bessel_i0(a.alpha * sqrt(r)) * a.inv_i0a;
    }
  }
}

// Position of index i after a dif transform (the plan's digit-reversal table).
__device__ __forceinline__ int row_pos(int i, const int* perm) { return perm[i]; }

// Accumulator of sum_i w_i b_i: plain, or error-compensated (two-product of
// each term by FMA, two-sum of the running total; Ogita, Rump & Oishi's Dot2)
// for the FP32-compensated precision mode.
template <class R, bool COMP>
struct DotAcc {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R w, R b) {
    if constexpr (!COMP) {
      s += w * b;
    } else {
      const R p = w * b;
      const R ep = fma(w, b, -p);
      const R t = s + p;
      const R bp = t - s;
      c += ((s - (t - bp)) + (p - bp)) + ep;
      s = t;
    }
  }
  __device__ __forceinline__ R value() const { return COMP ? s + c : s; }
};

// --------------------------------------------------------- row kernels (NUFFT)

// Table row of lateral-frequency row l: |l~| for a B-scan; (|lx|, |ly|) with
// (lx, ly) = (l / ny, l % ny) for a volume.
template <class A>
__device__ __forceinline__ int table_row(const A& a, int l) {
  if (a.ny == 1) return l <= a.nx - l ? l : a.nx - l;
  const int lx = l / a.ny, ly = l - lx * a.ny;
  const int ix = lx <= a.nx - lx ? lx : a.nx - lx, iy = ly <= a.ny - ly ? ly : a.ny - ly;
  return ix * (a.ny / 2 + 1) + iy;
}

template <class R, int J, bool COMP>
__device__ __forceinline__ void row_forward_body(const RowArgs<R>& a, const Radix& rad, int blk, const RowArgs<R>& a0) {
  using V = cplx_t<R>;
  using Tab = typename TabOf<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  V* tws = buf + a.K;
  const int l = blk;
  const int lp = table_row(a, l);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int K = a.K, nz = a.nz, n0 = a.n0, M = a.m;
  const bool sw = (K & 15) == 0;
  const int* perm = a.perm;
  const Tw2<V> tw = load_twiddles(tws, reinterpret_cast<const V*>(a.tw), rad);
  const V* X = reinterpret_cast<const V*>(a.in) + (size_t)l * nz;
  const R* cdep = reinterpret_cast<const R*>(a.cdep);
  pdl_wait_release();
  // centred zero-padded row, element i = (n - n0) mod K holding c_n X[l][n],
  // placed digit-reversed for the decimation-in-time transform
  constexpr int U = 4;
  for (int i0 = tid; i0 < K; i0 += U * nthr) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nthr;
      int n = i + n0;
      if (n >= K) n -= K;
      v[u] = (i < K && n < nz) ? cscale(X[n], cdep[n]) : cmk<V>(R(0), R(0));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nthr;
      if (i < K) buf[swz(row_pos(i, perm), sw)] = v[u];
    }
  }
  __syncthreads();
  fft_dit<false>(buf, 1, rad, tw, sw);
  const Tab* tab = reinterpret_cast<const Tab*>(a.tab) + (size_t)lp * M;
  V* S = reinterpret_cast<V*>(a.out) + (size_t)l * M;
  constexpr int UM = 2;
  for (int m0 = tid; m0 < M; m0 += UM * nthr) {
    Tab e[UM];
#pragma unroll
    for (int u = 0; u < UM; ++u) {
      const int mm = m0 + u * nthr;
      if (mm < M) e[u] = tab[mm];
    }
#pragma unroll
    for (int u = 0; u < UM; ++u) {
      const int mm = m0 + u * nthr;
      if (mm >= M) continue;
      R w[J];
      kb_weights<R, J>(R(e[u].frac), a0, w);
      const int pc = e[u].cell & 0xFFFF;
      DotAcc<R, COMP> ax, ay;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        int idx = pc + j;
        if (idx >= K) idx -= K;
        const V b = buf[swz(idx, sw)];
        ax.add(w[j], b.x);
        ay.add(w[j], b.y);
      }
      S[mm] = cmul(cmk<V>(ax.value(), ay.value()), cmk<V>(R(e[u].fre), R(e[u].fim)));
    }
  }
}

template <class R, int J, bool BAT, bool COMP = false>
__global__ void __launch_bounds__(kRowThreads, sizeof(R) == 4 ? kRowMinBlocks : 1)
row_forward_kernel(const __grid_constant__ RowArgs<R> a0, const BatchRef<RowArgs<R>> B) {
  if constexpr (!BAT) {
    row_forward_body<R, J, COMP>(a0, a0.rad, (int)blockIdx.x, a0);
  } else {
    int blk;
    const RowArgs<R>& A = *resolve_args(&a0, B, blk);
    __shared__ Radix rad;
    copy_radix(&rad, &A.rad);
    __syncthreads();
    row_forward_body<R, J, COMP>(A, rad, blk, a0);
  }
}

template <class R, int J>
__device__ __forceinline__ void row_adjoint_body(const RowArgs<R>& a, const Radix& rad, int blk, const RowArgs<R>& a0) {
  using V = cplx_t<R>;
  using Tab = typename TabOf<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  V* tws = buf + a.K;
  const int l = blk;
  const int lp = table_row(a, l);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int K = a.K, nz = a.nz, n0 = a.n0, M = a.m;
  const bool sw = (K & 15) == 0;
  const int* perm = a.perm;
  const Tw2<V> tw = load_twiddles(tws, reinterpret_cast<const V*>(a.tw), rad);
  for (int i = tid; i < K; i += nthr) buf[i] = cmk<V>(R(0), R(0));
  pdl_wait_release();
  __syncthreads();
  const Tab* tab = reinterpret_cast<const Tab*>(a.tab) + (size_t)lp * M;
  const V* Rh = reinterpret_cast<const V*>(a.in) + (size_t)l * M;
  R* bufr = reinterpret_cast<R*>(buf);
  constexpr int UM = 2;
  for (int m0 = tid; m0 < M; m0 += UM * nthr) {
    Tab e[UM];
    V r[UM];
#pragma unroll
    for (int u = 0; u < UM; ++u) {
      const int mm = m0 + u * nthr;
      if (mm < M) {
        e[u] = tab[mm];
        r[u] = Rh[mm];
      }
    }
#pragma unroll
    for (int u = 0; u < UM; ++u) {
      const int mm = m0 + u * nthr;
      if (mm >= M) continue;
      const V v = cmulc(r[u], cmk<V>(R(e[u].fre), R(e[u].fim)));
      R w[J];
      kb_weights<R, J>(R(e[u].frac), a0, w);
      const int pc = e[u].cell & 0xFFFF;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        int idx = pc + j;
        if (idx >= K) idx -= K;
        const int q = swz(idx, sw);
        atomicAdd(&bufr[2 * q], w[j] * v.x);
        atomicAdd(&bufr[2 * q + 1], w[j] * v.y);
      }
    }
  }
  __syncthreads();
  fft_dif<true>(buf, 1, rad, tw, sw);
  const R* cdep = reinterpret_cast<const R*>(a.cdep);
  V* Wo = reinterpret_cast<V*>(a.out) + (size_t)l * nz;
  for (int n = tid; n < nz; n += nthr) {
    int i = n - n0;
    if (i < 0) i += K;
    Wo[n] = cscale(buf[swz(row_pos(i, perm), sw)], cdep[n]);
  }
}

template <class R, int J, bool BAT>
__global__ void __launch_bounds__(kRowThreads, sizeof(R) == 4 ? kRowMinBlocks : 1)
row_adjoint_kernel(const __grid_constant__ RowArgs<R> a0, const BatchRef<RowArgs<R>> B) {
  if constexpr (!BAT) {
    row_adjoint_body<R, J>(a0, a0.rad, (int)blockIdx.x, a0);
  } else {
    int blk;
    const RowArgs<R>& A = *resolve_args(&a0, B, blk);
    __shared__ Radix rad;
    copy_radix(&rad, &A.rad);
    __syncthreads();
    row_adjoint_body<R, J>(A, rad, blk, a0);
  }
}

// Adjoint row kernel without atomics: the transpose of the J-tap interpolation
// as a segmented gather.  Within a row the first-tap cells of the pixels,
// unwrapped to u (plan table), are monotone in m, so the pixels reaching grid
// cell c (those with c - J + 1 <= u <= c) form a contiguous run once the row is
// staged in increasing-u order.  first[c] = min{s : u_s >= c} is built by a
// conflict-free scatter (each cell written once); cell c then sums its run in a
// fixed order, so the result is deterministic.
template <class R, int J, bool COMP>
__device__ __forceinline__ void row_adjoint_gather_body(const RowArgs<R>& a, const Radix& rad, int blk, const RowArgs<R>& a0) {
  using V = cplx_t<R>;
  using Tab = typename TabOf<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.K, nz = a.nz, n0 = a.n0, M = a.m;
  V* buf = reinterpret_cast<V*>(smem_raw);
  V* tws = buf + K;
  V* sv = tws + rad.tw_lo + rad.tw_hi;                          // [M] conj(f) R
  // FP32 with kGatherPrecomp: the J weights of every pixel [M][J]; otherwise frac [M]
  R* sfrac = reinterpret_cast<R*>(sv + M);
  constexpr bool kPre = kGatherPrecomp && sizeof(R) == 4;
  float* spoly = reinterpret_cast<float*>(sfrac + (kPre ? M * J : M));   // [J][kKbDeg + 1]
  uint16_t* su = reinterpret_cast<uint16_t*>(spoly + J * (kKbDeg + 1));   // [M]
  uint16_t* sfirst = su + M + (M & 1);                              // [span + 1]
  const int l = blk;
  const int lp = table_row(a, l);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool sw = (K & 15) == 0;
  const int* perm = a.perm;
  const Tw2<V> tw = load_twiddles(tws, reinterpret_cast<const V*>(a.tw), rad);
  if (sizeof(R) == 4)
    for (int i = tid; i < J * (kKbDeg + 1); i += nthr) spoly[i] = a0.kbpoly[i / (kKbDeg + 1)][i % (kKbDeg + 1)];
  const int4 meta = a.rowmeta[lp];
  const int base = meta.x, span = meta.y, dir = meta.z;
  const Tab* tab = reinterpret_cast<const Tab*>(a.tab) + (size_t)lp * M;
  const V* Rh = reinterpret_cast<const V*>(a.in) + (size_t)l * M;
  pdl_wait_release();
  // stage the row in increasing-u order
  constexpr int UM = 4;
  for (int m0 = tid; m0 < M; m0 += UM * nthr) {
    Tab e[UM];
    V r[UM];
#pragma unroll
    for (int q = 0; q < UM; ++q) {
      const int mm = m0 + q * nthr;
      if (mm < M) {
        e[q] = tab[mm];
        r[q] = Rh[mm];
      }
    }
#pragma unroll
    for (int q = 0; q < UM; ++q) {
      const int mm = m0 + q * nthr;
      if (mm < M) {
        const int sidx = dir > 0 ? mm : M - 1 - mm;
        sv[sidx] = cmulc(r[q], cmk<V>(R(e[q].fre), R(e[q].fim)));
        if constexpr (kPre) {
          R w[J];
          kb_weights<R, J>(R(e[q].frac), a0, w);
#pragma unroll
          for (int j = 0; j < J; ++j) sfrac[sidx * J + j] = w[j];
        } else {
          sfrac[sidx] = R(e[q].frac);
        }
        su[sidx] = (uint16_t)((unsigned)e[q].cell >> 16);
      }
    }
  }
  __syncthreads();
  // first[c] = min{s : u_s >= c} for c in [0, span]: pixel s owns the cells
  // (u_{s-1}, u_s] (u_{-1} = -1); the last pixel also owns (u_{M-1}, span] -> M
  for (int sidx = tid; sidx < M; sidx += nthr) {
    const int lo = sidx == 0 ? 0 : int(su[sidx - 1]) + 1;
    const int hi = su[sidx];
    for (int c = lo; c <= hi; ++c) sfirst[c] = (uint16_t)sidx;
    if (sidx == M - 1)
      for (int c = hi + 1; c <= span; ++c) sfirst[c] = (uint16_t)M;
  }
  __syncthreads();
  // each physical cell i: unwrapped c = (i - base) mod K; sum its run of pixels
  for (int i = tid; i < K; i += nthr) {
    int c = i - base;
    if (c < 0) c += K;
    DotAcc<R, COMP> ax, ay;
    if (c < span) {
      const int slo = c - J + 1 <= 0 ? 0 : int(sfirst[c - J + 1]);
      const int shi = int(sfirst[c + 1]) - 1;
      for (int sidx = slo; sidx <= shi; ++sidx) {
        const int j = c - int(su[sidx]);
        R w;
        if constexpr (kPre) {
          w = sfrac[sidx * J + j];
        } else if constexpr (sizeof(R) == 4) {
          const float x = sfrac[sidx] - 0.5f;
          const float* cf = spoly + j * (kKbDeg + 1);
          float t = cf[kKbDeg];
#pragma unroll
          for (int d = kKbDeg - 1; d >= 0; --d) t = fmaf(t, x, cf[d]);
          w = t;
        } else {
          const double uu = sfrac[sidx] + double(J / 2 - 1 - j);
          const double rr = 1.0 - (2.0 * uu / J) * (2.0 * uu / J);
          w = rr < 0.0 ? 0.0 : cyl_bessel_i0(a0.alpha * sqrt(rr)) * a0.inv_i0a;
        }
        const V v = sv[sidx];
        ax.add(w, v.x);
        ay.add(w, v.y);
      }
    }
    buf[swz(i, sw)] = cmk<V>(ax.value(), ay.value());
  }
  __syncthreads();
  fft_dif<true>(buf, 1, rad, tw, sw);
  const R* cdep = reinterpret_cast<const R*>(a.cdep);
  V* Wo = reinterpret_cast<V*>(a.out) + (size_t)l * nz;
  for (int n = tid; n < nz; n += nthr) {
    int i = n - n0;
    if (i < 0) i += K;
    Wo[n] = cscale(buf[swz(row_pos(i, perm), sw)], cdep[n]);
  }
}

template <class R, int J, bool BAT, bool COMP = false>
__global__ void __launch_bounds__(kGatherThreads, sizeof(R) == 4 ? kGatherMinBlocks : 1)
row_adjoint_gather_kernel(const __grid_constant__ RowArgs<R> a0, const BatchRef<RowArgs<R>> B) {
  if constexpr (!BAT) {
    row_adjoint_gather_body<R, J, COMP>(a0, a0.rad, (int)blockIdx.x, a0);
  } else {
    int blk;
    const RowArgs<R>& A = *resolve_args(&a0, B, blk);
    __shared__ Radix rad;
    copy_radix(&rad, &A.rad);
    __syncthreads();
    row_adjoint_gather_body<R, J, COMP>(A, rad, blk, a0);
  }
}

// --------------------------------------------- paired row kernels (FP32)
//
// Rows l and nx - l of the lateral spectrum share |l~| and with it the resampling
// table, the KB weights and the filter (the model sees the lateral frequency
// only through q^2).  One CTA runs both rows: the table, the weights and the
// gather's index arithmetic serve two rows, and the K-point transform runs on
// split pairs {re_l, re_l', im_l, im_l'} with paired FP32 instructions.  CTA lp
// (0 <= lp <= nx/2) takes rows lp and nx - lp; rows 0 and nx/2 are their own
// mirror and run alone (lane b repeats lane a and is not stored).

// The filter of pixel m on table row lp formed from its factors (plan otf):
// fp = {Re, Im of A e^{j(Omega - 2k z_f + 2k (z_f - z_c))}, 1/(2 k^2 NA^2), 2k},
// times exp(-q^2 / (2 k^2 NA^2)) e^{-j (2k - beta)(z_f - z_c)}, with
// 2k - beta = q^2 / (beta + 2k) (no cancellation in FP32); 0 where 4k^2 <= q^2.
__device__ __forceinline__ float2 otf_filter(const float4& fp, float q2, float dzf) {
  const float b2 = fp.w * fp.w - q2;
  if (!(b2 > 0.f)) return make_float2(0.f, 0.f);
  const float d = q2 / (sqrtf(b2) + fp.w);
  const float G = expf(-q2 * fp.z);
  float sn, cs;
  sincosf(-d * dzf, &sn, &cs);
  return make_float2(G * (fp.x * cs - fp.y * sn), G * (fp.x * sn + fp.y * cs));
}

// Table entry of pixel mm on table row lp: grid position and filter, read whole
// (OTF = false) or position read and filter formed (OTF = true).
template <bool OTF>
__device__ __forceinline__ void row_entry_load(const RowArgs<float>& a, int lp, int mm, TabF& e, float4& fp) {
  if constexpr (OTF) {
    const TabP t = a.tabp[(size_t)lp * a.m + mm];
    e.cell = t.cell;
    e.frac = t.frac;
    fp = a.fpix[mm];
  } else {
    e = reinterpret_cast<const TabF*>(a.tab)[(size_t)lp * a.m + mm];
  }
}

template <bool OTF>
__device__ __forceinline__ float2 row_entry_filter(const RowArgs<float>& a, const TabF& e, const float4& fp, float q2) {
  if constexpr (OTF) return otf_filter(fp, q2, a.dzf);
  else return make_float2(e.fre, e.fim);
}

__device__ __forceinline__ int pair_row_b(int lp, int nx) {
  const int lb = nx - lp;
  return (lp == 0 || lb == lp) ? -1 : lb;
}

// Fused first and last passes of the K-point row transforms (the pair kernels'
// FZ = 1; the host launches them for plans whose transform starts and ends with a
// radix 2, 4 or 8, and batches only when every scan of the launch qualifies).  With R the radix of
// the last dif pass (the first dit pass), the positions b' R + r of a
// digit-reversed row hold the natural elements b + r K/R, where perm[b] = b' R
// (b < K/R: the last digit of k is its most significant one).  So a butterfly of
// that pass is addressed from its natural base b with one table read.

// The first dit pass (span 1, no twiddles) run on the way in: load(i) gives the
// natural element i of the row.
template <int R, class F>
__device__ __forceinline__ void row_first_pass_dit(float4* buf, int K, const int* perm, const TwP& tw, F&& load) {
  const int B = K / R;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int p0 = perm[b];
    PC v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = load(b + r * B);
    dft_small_p<R, false>(v, tw, K);
#pragma unroll
    for (int r = 0; r < R; ++r) st_pc(buf, swz8(p0 + r), v[r]);
  }
}

// The first dif pass (span K/R, twiddles after the butterfly) with its inputs,
// the natural cells j + r K/R, computed in registers by cell(i).
template <int R, class F>
__device__ __forceinline__ void row_first_pass_dif(float4* buf, int K, const TwP& tw, F&& cell) {
  const int B = K / R;
  for (int j = threadIdx.x; j < B; j += blockDim.x) {
    PC v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cell(j + r * B);
    dft_small_p<R, true>(v, tw, K);
    if (j != 0) apply_twiddles_p<R, true>(v, tw, j);
#pragma unroll
    for (int r = 0; r < R; ++r) st_pc(buf, swz8(j + r * B), v[r]);
  }
}

// The last dif pass (span 1, no twiddles) run on the way out: out(i, v) takes the
// natural output i.
template <int R, class F>
__device__ __forceinline__ void row_last_pass_dif(const float4* buf, int K, const int* perm, const TwP& tw,
                                                  F&& out) {
  const int B = K / R;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int p0 = perm[b];
    PC v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld_pc(buf, swz8(p0 + r));
    dft_small_p<R, true>(v, tw, K);
#pragma unroll
    for (int r = 0; r < R; ++r) out(b + r * B, v[r]);
  }
}

// f(RadixC<r>()) for a radix r in {2, 4, 8}
template <int N> struct RadixC { static constexpr int value = N; };
template <class F>
__device__ __forceinline__ void with_radix248(int r, F&& f) {
  if (r == 8) f(RadixC<8>());
  else if (r == 4) f(RadixC<4>());
  else f(RadixC<2>());
}

template <int J, bool OTF, int FZ>
__device__ __forceinline__ void row_forward_pair_body(const RowArgs<float>& a, const Radix& rad, int lp,
                                                      const RowArgs<float>& a0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.K, nz = a.nz, n0 = a.n0, M = a.m;
  const int K8 = (K + 7) & ~7;
  float4* buf = reinterpret_cast<float4*>(smem_raw);   // [K8], swizzled
  int la = lp, lb = pair_row_b(lp, a.nx);
  if (a.rowmap) {   // a volume: the CTA's rows and table row from the plan's map
    const int4 rm = a.rowmap[lp];
    la = rm.x;
    lb = rm.y;
    lp = rm.z;
  }
  const int lbr = lb < 0 ? la : lb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const TwP tw = load_twiddles_p(buf + K8, reinterpret_cast<const float2*>(a.tw), rad);
  const float2* Xa = reinterpret_cast<const float2*>(a.in) + (size_t)la * nz;
  const float2* Xb = reinterpret_cast<const float2*>(a.in) + (size_t)lbr * nz;
  const float* cdep = reinterpret_cast<const float*>(a.cdep);
  const int* perm = a.perm;
  if (!OTF) prefetch_l2_range(reinterpret_cast<const TabF*>(a.tab) + (size_t)lp * M, sizeof(TabF) * M);
  pdl_wait_release();
  // centred zero-padded rows, element i = (n - n0) mod K holding c_n X[l][n],
  // placed digit-reversed for the decimation-in-time transform
  if constexpr (FZ != 0) {
    // the first dit pass on the way in (its butterflies read no twiddles)
    with_radix248(rad.r[rad.npass - 1], [&](auto rc) {
      row_first_pass_dit<decltype(rc)::value>(buf, K, perm, tw, [&](int i) {
        int n = i + n0;
        if (n >= K) n -= K;
        PC v{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (n < nz) {
          const float c = cdep[n];
          const float2 xa = Xa[n], xb = Xb[n];
          v = PC{make_float2(xa.x * c, xb.x * c), make_float2(xa.y * c, xb.y * c)};
        }
        return v;
      });
    });
    __syncthreads();
    fft_p_dit<false, true>(buf, 1, rad, tw, 0, rad.npass - 2);
  } else {
    constexpr int U = 4;
    for (int i0 = tid; i0 < K; i0 += U * nthr) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * nthr;
        int n = i + n0;
        if (n >= K) n -= K;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < K && n < nz) {
          const float c = cdep[n];
          const float2 xa = Xa[n], xb = Xb[n];
          v[u] = make_float4(xa.x * c, xb.x * c, xa.y * c, xb.y * c);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * nthr;
        if (i < K) buf[swz8(perm[i])] = v[u];
      }
    }
    __syncthreads();
    fft_p_dit<false, true>(buf, 1, rad, tw);
  }
  float2* Sa = reinterpret_cast<float2*>(a.out) + (size_t)la * M;
  float2* Sb = reinterpret_cast<float2*>(a.out) + (size_t)lbr * M;
  const float q2 = OTF ? a.q2row[lp] : 0.f;
  constexpr int UM = 2;
  for (int m0 = tid; m0 < M; m0 += UM * nthr) {
    TabF e[UM];
    float4 fp[UM];
#pragma unroll
    for (int u = 0; u < UM; ++u) {
      const int mm = m0 + u * nthr;
      if (mm < M) row_entry_load<OTF>(a, lp, mm, e[u], fp[u]);
    }
#pragma unroll
    for (int u = 0; u < UM; ++u) {
      const int mm = m0 + u * nthr;
      if (mm >= M) continue;
      float w[J];
      kb_weights<float, J>(e[u].frac, a0, w);
      const int pc = e[u].cell & 0xFFFF;
      float2 ar = make_float2(0.f, 0.f), ai = ar;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        int idx = pc + j;
        if (idx >= K) idx -= K;
        const float4 t = buf[swz8(idx)];
        const float2 ww = make_float2(w[j], w[j]);
        ar = fma2(make_float2(t.x, t.y), ww, ar);
        ai = fma2(make_float2(t.z, t.w), ww, ai);
      }
      const float2 f = row_entry_filter<OTF>(a, e[u], fp[u], q2);
      Sa[mm] = cmul(make_float2(ar.x, ai.x), f);
      if (lb >= 0) Sb[mm] = cmul(make_float2(ar.y, ai.y), f);
    }
  }
}

template <int J, bool BAT, bool OTF, int FZ = 0>
__global__ void __launch_bounds__(kRowPairThreads, kRowPairMinBlocks)
row_forward_pair_kernel(const __grid_constant__ RowArgs<float> a0, const BatchRef<RowArgs<float>> B) {
  if constexpr (!BAT) {
    row_forward_pair_body<J, OTF, FZ>(a0, a0.rad, (int)blockIdx.x, a0);
  } else {
    int blk;
    const RowArgs<float>& A = *resolve_args(&a0, B, blk);
    __shared__ Radix rad;
    copy_radix(&rad, &A.rad);
    __syncthreads();
    row_forward_pair_body<J, OTF, FZ>(A, rad, blk, a0);
  }
}

// The adjoint gather of row_adjoint_gather_body for a row pair: the pixels' KB
// weights, unwrapped cells and run boundaries are built once, each cell sums its
// run for both rows in the two lanes of split pairs.
// The end of a paired gather once its pixels are staged: the K grid cells of both
// rows (cell(i), after a barrier), the inverse K-point dif transform and the
// read-out of the nz depth samples n (natural output (n - n0) mod K, times c_n).
// FZ: the cells feed the first pass's butterflies in registers and the last pass
// writes the read-out, so the row crosses shared memory two times fewer.
template <int FZ, class F>
__device__ __forceinline__ void row_gather_pair_finish(const RowArgs<float>& a, const Radix& rad, const TwP& tw,
                                                       float4* buf, int la, int lb, int lbr, F&& cell) {
  const int K = a.K, nz = a.nz, n0 = a.n0;
  const float* cdep = reinterpret_cast<const float*>(a.cdep);
  const int* perm = a.perm;
  float2* Wa = reinterpret_cast<float2*>(a.out) + (size_t)la * nz;
  float2* Wb = reinterpret_cast<float2*>(a.out) + (size_t)lbr * nz;
  if constexpr (FZ != 0) {
    with_radix248(rad.r[0], [&](auto rc) { row_first_pass_dif<decltype(rc)::value>(buf, K, tw, cell); });
    __syncthreads();
    fft_p_dif<true, true>(buf, 1, rad, tw, 1, rad.npass - 1);
    with_radix248(rad.r[rad.npass - 1], [&](auto rc) {
      row_last_pass_dif<decltype(rc)::value>(buf, K, perm, tw, [&](int i, const PC& v) {
        int n = i + n0;
        if (n >= K) n -= K;
        if (n < nz) {
          const float cn = cdep[n];
          Wa[n] = make_float2(v.re.x * cn, v.im.x * cn);
          if (lb >= 0) Wb[n] = make_float2(v.re.y * cn, v.im.y * cn);
        }
      });
    });
  } else {
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      const PC v = cell(i);
      buf[swz8(i)] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
    }
    __syncthreads();
    fft_p_dif<true, true>(buf, 1, rad, tw);
    for (int n = threadIdx.x; n < nz; n += blockDim.x) {
      int i = n - n0;
      if (i < 0) i += K;
      const float4 t = buf[swz8(perm[i])];
      const float cn = cdep[n];
      Wa[n] = make_float2(t.x * cn, t.z * cn);
      if (lb >= 0) Wb[n] = make_float2(t.y * cn, t.w * cn);
    }
  }
}

template <int J, bool OTF, int FZ>
__device__ __forceinline__ void row_gather_pair_body(const RowArgs<float>& a, const Radix& rad, int lp,
                                                     const RowArgs<float>& a0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.K, M = a.m;
  const int K8 = (K + 7) & ~7;
  float4* buf = reinterpret_cast<float4*>(smem_raw);         // [K8], swizzled
  float4* tws = buf + K8;
  float4* sv = tws + rad.tw_lo + rad.tw_hi;                  // [M] conj(f) R of both rows, split
  float* sw = reinterpret_cast<float*>(sv + M);              // [M][J] weights
  uint16_t* su = reinterpret_cast<uint16_t*>(sw + M * J);    // [M]
  uint16_t* sfirst = su + M + (M & 1);                       // [span + 1]
  int la = lp, lb = pair_row_b(lp, a.nx);
  if (a.rowmap) {   // a volume: the CTA's rows and table row from the plan's map
    const int4 rm = a.rowmap[lp];
    la = rm.x;
    lb = rm.y;
    lp = rm.z;
  }
  const int lbr = lb < 0 ? la : lb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const TwP tw = load_twiddles_p(tws, reinterpret_cast<const float2*>(a.tw), rad);
  const int4 meta = a.rowmeta[lp];
  const int base = meta.x, span = meta.y, dir = meta.z;
  const float q2 = OTF ? a.q2row[lp] : 0.f;
  const float2* Ra = reinterpret_cast<const float2*>(a.in) + (size_t)la * M;
  const float2* Rb = reinterpret_cast<const float2*>(a.in) + (size_t)lbr * M;
  if (!OTF) prefetch_l2_range(reinterpret_cast<const TabF*>(a.tab) + (size_t)lp * M, sizeof(TabF) * M);
  pdl_wait_release();
  // stage both rows in increasing-u order
  constexpr int UM = 2;
  for (int m0 = tid; m0 < M; m0 += UM * nthr) {
    TabF e[UM];
    float4 fp[UM];
    float2 ra[UM], rb[UM];
#pragma unroll
    for (int q = 0; q < UM; ++q) {
      const int mm = m0 + q * nthr;
      if (mm < M) {
        row_entry_load<OTF>(a, lp, mm, e[q], fp[q]);
        ra[q] = Ra[mm];
        rb[q] = Rb[mm];
      }
    }
#pragma unroll
    for (int q = 0; q < UM; ++q) {
      const int mm = m0 + q * nthr;
      if (mm >= M) continue;
      const int sidx = dir > 0 ? mm : M - 1 - mm;
      const float2 f = row_entry_filter<OTF>(a, e[q], fp[q], q2);
      const float2 va = cmulc(ra[q], f), vb = cmulc(rb[q], f);
      sv[sidx] = make_float4(va.x, vb.x, va.y, vb.y);
      float w[J];
      kb_weights<float, J>(e[q].frac, a0, w);
#pragma unroll
      for (int j = 0; j < J; ++j) sw[sidx * J + j] = w[j];
      su[sidx] = (uint16_t)((unsigned)e[q].cell >> 16);
    }
  }
  __syncthreads();
  // first[c] = min{s : u_s >= c} for c in [0, span], as in the single-row kernel
  for (int sidx = tid; sidx < M; sidx += nthr) {
    const int lo = sidx == 0 ? 0 : int(su[sidx - 1]) + 1;
    const int hi = su[sidx];
    for (int c = lo; c <= hi; ++c) sfirst[c] = (uint16_t)sidx;
    if (sidx == M - 1)
      for (int c = hi + 1; c <= span; ++c) sfirst[c] = (uint16_t)M;
  }
  __syncthreads();
  auto cell = [&](int i) {
    int c = i - base;
    if (c < 0) c += K;
    float2 ar = make_float2(0.f, 0.f), ai = ar;
    if (c < span) {
      const int slo = c - J + 1 <= 0 ? 0 : int(sfirst[c - J + 1]);
      const int shi = int(sfirst[c + 1]) - 1;
#pragma unroll 4
      for (int sidx = slo; sidx <= shi; ++sidx) {
        const float w = sw[sidx * J + (c - int(su[sidx]))];
        const float4 t = sv[sidx];
        const float2 ww = make_float2(w, w);
        ar = fma2(make_float2(t.x, t.y), ww, ar);
        ai = fma2(make_float2(t.z, t.w), ww, ai);
      }
    }
    return PC{ar, ai};
  };
  row_gather_pair_finish<FZ>(a, rad, tw, buf, la, lb, lbr, cell);
}

template <int J, bool BAT, bool OTF, int FZ = 0>
__global__ void __launch_bounds__(kGatherPairThreads, 1)
row_gather_pair_kernel(const __grid_constant__ RowArgs<float> a0, const BatchRef<RowArgs<float>> B) {
  if constexpr (!BAT) {
    row_gather_pair_body<J, OTF, FZ>(a0, a0.rad, (int)blockIdx.x, a0);
  } else {
    int blk;
    const RowArgs<float>& A = *resolve_args(&a0, B, blk);
    __shared__ Radix rad;
    copy_radix(&rad, &A.rad);
    __syncthreads();
    row_gather_pair_body<J, OTF, FZ>(A, rad, blk, a0);
  }
}

// The paired gather without per-pixel weight and cell arrays, so that two CTAs
// fit an SM (about 110 KB at K = 4096, M = 2048 instead of 162 KB).  Staging keeps
// conj(f) R of both rows and the fractional position of each pixel in
// increasing-u order, and first[v] = min{s : u_s >= v}, built directly from the
// table (pixel s writes the entries (u_{s-1}, u_s]).  Cell c then sums, tap by tap,
// the run of pixels whose first-tap cell is v = c - j, [first[v], first[v+1]),
// with the tap's weight evaluated from the pixel's fractional position by its
// polynomial.  The order of the terms of a cell is fixed (taps in order, pixels
// in order), so the result is deterministic; it differs from the other gathers
// only in rounding order.
template <int J>
__device__ __forceinline__ float kb_tap_weight(float frac, const RowArgs<float>& a0, int j) {
  const float x = frac - 0.5f;
  float t = a0.kbpoly[j][kKbDeg];
#pragma unroll
  for (int d = kKbDeg - 1; d >= 0; --d) t = fmaf(t, x, a0.kbpoly[j][d]);
  return t;
}

template <int J, bool OTF, int FZ>
__device__ __forceinline__ void row_gather_pair_lean_body(const RowArgs<float>& a, const Radix& rad, int lp,
                                                          const RowArgs<float>& a0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.K, M = a.m;
  const int K8 = (K + 7) & ~7;
  float4* buf = reinterpret_cast<float4*>(smem_raw);         // [K8], swizzled
  float4* tws = buf + K8;
  float4* sv = tws + rad.tw_lo + rad.tw_hi;                  // [M] conj(f) R of both rows, split
  float* sfrac = reinterpret_cast<float*>(sv + M);           // [M]
  uint16_t* sfirst = reinterpret_cast<uint16_t*>(sfrac + M); // [span - J + 2]
  int la = lp, lb = pair_row_b(lp, a.nx);
  if (a.rowmap) {   // a volume: the CTA's rows and table row from the plan's map
    const int4 rm = a.rowmap[lp];
    la = rm.x;
    lb = rm.y;
    lp = rm.z;
  }
  const int lbr = lb < 0 ? la : lb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const TwP tw = load_twiddles_p(tws, reinterpret_cast<const float2*>(a.tw), rad);
  const int4 meta = a.rowmeta[lp];
  const int base = meta.x, span = meta.y, dir = meta.z;
  const int vmax = span - J;                                 // largest u of the row
  const float q2 = OTF ? a.q2row[lp] : 0.f;
  const float2* Ra = reinterpret_cast<const float2*>(a.in) + (size_t)la * M;
  const float2* Rb = reinterpret_cast<const float2*>(a.in) + (size_t)lbr * M;
  if (!OTF) prefetch_l2_range(reinterpret_cast<const TabF*>(a.tab) + (size_t)lp * M, sizeof(TabF) * M);
  pdl_wait_release();
  constexpr int UM = 2;
  for (int m0 = tid; m0 < M; m0 += UM * nthr) {
    TabF e[UM];
    float4 fp[UM];
    float2 ra[UM], rb[UM];
    int uprev[UM];
#pragma unroll
    for (int q = 0; q < UM; ++q) {
      const int mm = m0 + q * nthr;
      uprev[q] = -1;
      if (mm < M) {
        row_entry_load<OTF>(a, lp, mm, e[q], fp[q]);
        ra[q] = Ra[mm];
        rb[q] = Rb[mm];
        // the previous pixel in increasing-u order
        const int mp = dir > 0 ? mm - 1 : mm + 1;
        if (mp >= 0 && mp < M) {
          const int cp = OTF ? a.tabp[(size_t)lp * M + mp].cell
                             : reinterpret_cast<const TabF*>(a.tab)[(size_t)lp * M + mp].cell;
          uprev[q] = (int)((unsigned)cp >> 16);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < UM; ++q) {
      const int mm = m0 + q * nthr;
      if (mm >= M) continue;
      const int sidx = dir > 0 ? mm : M - 1 - mm;
      const float2 f = row_entry_filter<OTF>(a, e[q], fp[q], q2);
      const float2 va = cmulc(ra[q], f), vb = cmulc(rb[q], f);
      sv[sidx] = make_float4(va.x, vb.x, va.y, vb.y);
      sfrac[sidx] = e[q].frac;
      const int u = (int)((unsigned)e[q].cell >> 16);
      for (int v = uprev[q] + 1; v <= u; ++v) sfirst[v] = (uint16_t)sidx;
      if (sidx == M - 1)
        for (int v = u + 1; v <= vmax + 1; ++v) sfirst[v] = (uint16_t)M;
    }
  }
  __syncthreads();
  // grid cell i of both rows
  auto cell = [&](int i) {
    int c = i - base;
    if (c < 0) c += K;
    float2 ar = make_float2(0.f, 0.f), ai = ar;
    if (c < span) {
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int v = c - j;
        if (v < 0 || v > vmax) continue;
        const int s1 = sfirst[v + 1];
        for (int sidx = sfirst[v]; sidx < s1; ++sidx) {
          const float w = kb_tap_weight<J>(sfrac[sidx], a0, j);
          const float4 t = sv[sidx];
          const float2 ww = make_float2(w, w);
          ar = fma2(make_float2(t.x, t.y), ww, ar);
          ai = fma2(make_float2(t.z, t.w), ww, ai);
        }
      }
    }
    return PC{ar, ai};
  };
  row_gather_pair_finish<FZ>(a, rad, tw, buf, la, lb, lbr, cell);
}

template <int J, bool BAT, bool OTF, int FZ = 0>
__global__ void __launch_bounds__(kGatherLeanThreads, kGatherLeanMinBlocks)
row_gather_pair_lean_kernel(const __grid_constant__ RowArgs<float> a0, const BatchRef<RowArgs<float>> B) {
  if constexpr (!BAT) {
    row_gather_pair_lean_body<J, OTF, FZ>(a0, a0.rad, (int)blockIdx.x, a0);
  } else {
    int blk;
    const RowArgs<float>& A = *resolve_args(&a0, B, blk);
    __shared__ Radix rad;
    copy_radix(&rad, &A.rad);
    __syncthreads();
    row_gather_pair_lean_body<J, OTF, FZ>(A, rad, blk, a0);
  }
}

// ------------------------------------------------------------------ launch

int lateral_grid(mbir_plan p, int cols) { return (cols + p->tile_c - 1) / p->tile_c; }

constexpr int lat_class(int mode) {
  return (mode == LAT_C2C_FWD || mode == LAT_POWER_FWD) ? PC_LAT_FWD
         : mode == LAT_R2C_MASK ? PC_LAT_R2C
         : (mode == LAT_C2R_INV_MASK || mode == LAT_SOLVE_FWD) ? PC_LAT_INV
         : (mode == LAT_SOLVE_MID || mode == LAT_POWER_MID) ? PC_LAT_MID
                                                            : PC_LAT_ADJ;
}

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
  a.nxl = p->nxl;
  a.chirp = p->chirp;
  a.bhat = p->bhat;
  a.scale = scale;
  a.y = nullptr;
  a.pz = nullptr;
  a.r = nullptr;
  a.z1 = nullptr;
  a.z2 = nullptr;
  a.vout = nullptr;
  a.mu = a.delta = a.tau = R(0);
  a.partial = nullptr;
  a.scal = nullptr;
  return a;
}

// tile, the twiddle tables (16 bytes an entry: FP64 complex or FP32 broadcast) and
// the digit-reversal table
template <class R>
size_t lat_smem(mbir_plan p) {
  return sizeof(cplx_t<R>) * (size_t)p->nxl * p->tile_c + 16 * (size_t)(p->rad_x.tw_lo + p->rad_x.tw_hi) +
         2 * sizeof(int) * (size_t)p->nx;
}

// The fused first and last passes apply to FP32 mixed-radix plans whose first and
// last radices are 2, 4 or 8 (at least two passes).
static bool lat_fusable(mbir_plan p) {
  const Radix& r = p->rad_x;
  auto ok = [](int x) { return x == 2 || x == 4 || x == 8; };
  return kLatFuse && p->precision != MBIR_FP64 && !p->chirp && r.npass >= 2 && ok(r.r[0]) && ok(r.r[r.npass - 1]);
}

// The fused row passes apply to FP32 plans whose K-point transform starts and
// ends with a radix 2, 4 or 8 (at least two passes).
bool row_fusable(mbir_plan p) {
  const Radix& r = p->rad_k;
  auto ok = [](int x) { return x == 2 || x == 4 || x == 8; };
  return kRowFuse && p->precision == MBIR_FP32 && !p->otf && r.npass >= 2 && ok(r.r[0]) && ok(r.r[r.npass - 1]);
}

template <class R, int MODE>
int launch_lateral_args(mbir_plan p, const LatArgs<R>& a, int cols, cudaStream_t st) {
  {
    ProfScope ps_(p, lat_class(MODE), st);
    const dim3 grid(lateral_grid(p, cols)), block(kLatThreads);
    if (p->chirp) {
      launch(lateral_kernel<R, MODE, false, true>, grid, block, lat_smem<R>(p), st, a, no_batch<LatArgs<R>>());
    } else {
      bool fused = false;
      if constexpr (sizeof(R) == 4) {
        if (lat_fusable(p)) {
          launch(lateral_kernel<R, MODE, false, false, 1>, grid, block, lat_smem<R>(p), st, a, no_batch<LatArgs<R>>());
          fused = true;
        }
      }
      if (!fused)
        launch(lateral_kernel<R, MODE, false, false>, grid, block, lat_smem<R>(p), st, a, no_batch<LatArgs<R>>());
    }
  }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

template <class R, int MODE>
int launch_lateral(mbir_plan p, const void* in, void* out, const uint8_t* mask, int cols, R scale,
                   cudaStream_t st) {
  return launch_lateral_args<R, MODE>(p, lat_args<R>(p, in, out, mask, cols, scale), cols, st);
}

template <class R>
RowArgs<R> row_args(mbir_plan p, const void* in, void* out) {
  RowArgs<R> a;
  a.in = in;
  a.out = out;
  a.tab = p->tab;
  a.cdep = p->cdep;
  a.tw = p->tw_k;
  a.perm = p->perm_k;
  a.rad = p->rad_k;
  a.nx = p->nx;
  a.nz = p->nz;
  a.m = p->m;
  a.K = p->K;
  a.n0 = p->n0;
  a.rowmeta = p->rowmeta;
  a.rowmap = p->rowmap;
  a.ny = p->ny;
  a.otf = p->otf;
  a.tabp = p->tabp;
  a.fpix = p->fpix;
  a.q2row = p->q2row;
  a.dzf = p->dzf;
  a.alpha = p->alpha;
  a.inv_i0a = 1.0 / host_bessel_i0(p->alpha);
  for (int j = 0; j < kMaxJ; ++j)
    for (int d = 0; d <= kKbDeg; ++d) a.kbpoly[j][d] = p->kbpoly[j][d];
  return a;
}

template <class R>
size_t row_smem(mbir_plan p) {
  return sizeof(cplx_t<R>) * ((size_t)p->K + p->rad_k.tw_lo + p->rad_k.tw_hi);
}

template <class R>
size_t row_gather_smem(mbir_plan p) {
  const size_t M = p->m;
  const size_t nw = (kGatherPrecomp && sizeof(R) == 4) ? M * p->J : M;
  return sizeof(cplx_t<R>) * ((size_t)p->K + p->rad_k.tw_lo + p->rad_k.tw_hi + M) + sizeof(R) * nw +
         sizeof(float) * p->J * (kKbDeg + 1) + sizeof(uint16_t) * (M + (M & 1) + p->K + 2);
}

// paired FP32 row kernels: the row pair (16 bytes a cell, padded to a multiple of
// 8 cells) and the broadcast twiddles; the gather adds its pixel staging
size_t row_pair_smem(mbir_plan p) {
  const size_t K8 = (size_t)((p->K + 7) & ~7);
  return 16 * (K8 + p->rad_k.tw_lo + p->rad_k.tw_hi);
}
size_t row_gather_pair_smem(mbir_plan p) {
  const size_t M = p->m;
  return row_pair_smem(p) + 16 * M + sizeof(float) * M * p->J + sizeof(uint16_t) * (M + (M & 1) + p->K + 2);
}
size_t row_gather_pair_lean_smem(mbir_plan p) {
  const size_t M = p->m;
  return row_pair_smem(p) + 16 * M + sizeof(float) * M + sizeof(uint16_t) * (size_t)(p->max_span - p->J + 2);
}

size_t row_smem_bytes(mbir_plan p, int adjoint_gather);

bool row_kind_fits(mbir_plan p, int kind) {
  switch (kind) {
    case ROW_GATHER_PAIR:
      return p->precision == MBIR_FP32 && p->gather_ok && row_gather_pair_smem(p) <= (size_t)kMaxDynSmem;
    case ROW_GATHER_PAIR_LEAN:
      return p->precision == MBIR_FP32 && p->gather_ok && row_gather_pair_lean_smem(p) <= (size_t)kMaxDynSmem;
    case ROW_GATHER: return p->gather_ok && row_smem_bytes(p, 1) <= (size_t)kMaxDynSmem;
    case ROW_ATOMIC: return true;
    default: return false;
  }
}

int row_kind(mbir_plan p, bool adjoint) {
  const bool pair = p->precision == MBIR_FP32;
  if (!adjoint) return pair ? ROW_FWD_PAIR : ROW_FWD;
  if (p->adj_kind >= 0 && row_kind_fits(p, p->adj_kind)) return p->adj_kind;
  if (kAdjAtomic || !p->gather_ok) return ROW_ATOMIC;
  if (pair && kGatherLeanDefault && row_kind_fits(p, ROW_GATHER_PAIR_LEAN)) return ROW_GATHER_PAIR_LEAN;
  if (pair && row_gather_pair_smem(p) <= (size_t)kMaxDynSmem) return ROW_GATHER_PAIR;
  if (row_smem_bytes(p, 1) <= (size_t)kMaxDynSmem) return ROW_GATHER;
  return ROW_ATOMIC;
}

int row_ctas(mbir_plan p, int kind) { return kind >= ROW_FWD_PAIR ? p->npair : p->nx * p->ny; }

size_t row_kind_smem(mbir_plan p, int kind) {
  switch (kind) {
    case ROW_FWD_PAIR: return row_pair_smem(p);
    case ROW_GATHER_PAIR: return row_gather_pair_smem(p);
    case ROW_GATHER_PAIR_LEAN: return row_gather_pair_lean_smem(p);
    case ROW_GATHER: return row_smem_bytes(p, 1);
    default: return row_smem_bytes(p, 0);
  }
}

template <class R, int J, bool BAT, bool COMP>
static void row_launch_j(int kind, const RowArgs<R>& a, const BatchRef<RowArgs<R>>& B, int grid, size_t smem,
                         cudaStream_t st, bool fz) {
  if constexpr (sizeof(R) == 4 && !COMP) {
    // FP32 pair kernels with the fused first and last transform passes
    if (fz && a.otf == 0) {
      if (kind == ROW_FWD_PAIR) {
        launch(row_forward_pair_kernel<J, BAT, false, 1>, dim3(grid), dim3(kRowPairThreads), smem, st, a, B);
        return;
      }
      if (kind == ROW_GATHER_PAIR) {
        launch(row_gather_pair_kernel<J, BAT, false, 1>, dim3(grid), dim3(kGatherPairThreads), smem, st, a, B);
        return;
      }
      if constexpr (!BAT) {   // batched: the lean gather keeps its plain passes (it would spill)
        if (kind == ROW_GATHER_PAIR_LEAN) {
          launch(row_gather_pair_lean_kernel<J, false, false, 1>, dim3(grid), dim3(kGatherLeanThreads), smem, st, a,
                 B);
          return;
        }
      }
    }
  }
  if constexpr (sizeof(R) == 4 && !COMP) {
    const bool otf = a.otf != 0;
    if (kind == ROW_FWD_PAIR) {
      if constexpr (kFilterOtf) {
        if (otf) {
          launch(row_forward_pair_kernel<J, BAT, true>, dim3(grid), dim3(kRowPairThreads), smem, st, a, B);
          return;
        }
      }
      launch(row_forward_pair_kernel<J, BAT, false>, dim3(grid), dim3(kRowPairThreads), smem, st, a, B);
      return;
    }
    if (kind == ROW_GATHER_PAIR) {
      if constexpr (kFilterOtf) {
        if (otf) {
          launch(row_gather_pair_kernel<J, BAT, true>, dim3(grid), dim3(kGatherPairThreads), smem, st, a, B);
          return;
        }
      }
      launch(row_gather_pair_kernel<J, BAT, false>, dim3(grid), dim3(kGatherPairThreads), smem, st, a, B);
      return;
    }
    if (kind == ROW_GATHER_PAIR_LEAN) {
      if constexpr (kFilterOtf) {
        if (otf) {
          launch(row_gather_pair_lean_kernel<J, BAT, true>, dim3(grid), dim3(kGatherLeanThreads), smem, st, a, B);
          return;
        }
      }
      launch(row_gather_pair_lean_kernel<J, BAT, false>, dim3(grid), dim3(kGatherLeanThreads), smem, st, a, B);
      return;
    }
  }
  if (kind == ROW_FWD) launch(row_forward_kernel<R, J, BAT, COMP>, dim3(grid), dim3(kRowThreads), smem, st, a, B);
  else if (kind == ROW_GATHER)
    launch(row_adjoint_gather_kernel<R, J, BAT, COMP>, dim3(grid), dim3(kGatherThreads), smem, st, a, B);
  else launch(row_adjoint_kernel<R, J, BAT>, dim3(grid), dim3(kRowThreads), smem, st, a, B);
}

template <class R, bool BAT>
static void row_launch(int kind, int J, bool comp, const RowArgs<R>& a, const BatchRef<RowArgs<R>>& B, int grid,
                       size_t smem, cudaStream_t st, bool fz = false) {
  if (comp && sizeof(R) == 4) {
    switch (J) {
      case 4: row_launch_j<R, 4, BAT, true>(kind, a, B, grid, smem, st, fz); break;
      case 6: row_launch_j<R, 6, BAT, true>(kind, a, B, grid, smem, st, fz); break;
      default: row_launch_j<R, 8, BAT, true>(kind, a, B, grid, smem, st, fz); break;
    }
  } else {
    switch (J) {
      case 4: row_launch_j<R, 4, BAT, false>(kind, a, B, grid, smem, st, fz); break;
      case 6: row_launch_j<R, 6, BAT, false>(kind, a, B, grid, smem, st, fz); break;
      default: row_launch_j<R, 8, BAT, false>(kind, a, B, grid, smem, st, fz); break;
    }
  }
}

template <class R>
int launch_row(mbir_plan p, bool adjoint, const void* in, void* out, cudaStream_t st) {
  RowArgs<R> a = row_args<R>(p, in, out);
  const int kind = row_kind(p, adjoint);
  {
    ProfScope ps_(p, adjoint ? PC_ROW_ADJ : PC_ROW_FWD, st);
    row_launch<R, false>(kind, p->J, p->precision == MBIR_FP32_COMPENSATED, a, no_batch<RowArgs<R>>(),
                         row_ctas(p, kind), row_kind_smem(p, kind), st, row_fusable(p));
  }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

template <class R>
int forward_t(mbir_plan p, const void* x, const uint8_t* mask, void* y, cudaStream_t st) {
  int rc = launch_lateral<R, LAT_C2C_FWD>(p, x, p->wsA, nullptr, p->nz, R(1), st);
  if (rc) return rc;
  rc = launch_row<R>(p, false, p->wsA, p->wsB, st);
  if (rc) return rc;
  return launch_lateral<R, LAT_C2R_INV_MASK>(p, p->wsB, y, mask, p->m, R(1) / R(p->nx), st);
}

template <class R>
int adjoint_t(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st) {
  int rc = launch_lateral<R, LAT_R2C_MASK>(p, y, p->wsA, mask, p->m, R(1) / R(p->nx), st);
  if (rc) return rc;
  rc = launch_row<R>(p, true, p->wsA, p->wsB, st);
  if (rc) return rc;
  return launch_lateral<R, LAT_C2C_INV>(p, p->wsB, x, nullptr, p->nz, R(1), st);
}

// FISTA forward pass on z^{k-1} through the fused middle: pz = Phi z^{k-1}, the
// data-term partials, and R = the first stage of Phi^H on the residual, left in wsA.
template <class R>
int forward_solve_t(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, double mu,
                    double* partial, cudaStream_t st) {
  int rc = launch_lateral<R, LAT_C2C_FWD>(p, z1, p->wsA, nullptr, p->nz, R(1), st);
  if (rc) return rc;
  rc = launch_row<R>(p, false, p->wsA, p->wsB, st);
  if (rc) return rc;
  LatArgs<R> a = lat_args<R>(p, p->wsB, p->wsA, mask, p->m, R(1) / R(p->nx));
  a.y = reinterpret_cast<const R*>(y);
  a.pz = reinterpret_cast<R*>(pz);
  a.mu = R(mu);
  a.partial = partial;
  return launch_lateral_args<R, LAT_SOLVE_MID>(p, a, p->m, st);
}

// The rest of the FISTA adjoint pass: row adjoint of wsA, then the image epilogue.
template <class R>
int adjoint_solve_t(mbir_plan p, const void* z1, void* z2, void* vout, double mu, double delta, double tau,
                    double* partial, cudaStream_t st) {
  int rc = launch_row<R>(p, true, p->wsA, p->wsB, st);
  if (rc) return rc;
  LatArgs<R> a = lat_args<R>(p, p->wsB, nullptr, nullptr, p->nz, R(1));
  a.z1 = z1;
  a.z2 = z2;
  a.vout = vout;
  a.mu = R(mu);
  a.delta = R(delta);
  a.tau = R(tau);
  a.partial = partial;
  if (vout) return launch_lateral_args<R, LAT_SOLVE_ADJ_V>(p, a, p->nz, st);
  return launch_lateral_args<R, LAT_SOLVE_ADJ_L1>(p, a, p->nz, st);
}

// One power-iteration step: v = w scal[1] (written), w = Phi^H s Phi v, partial
// sums of <v, w> and ||w||^2 (two per lateral CTA of the image) into part.
template <class R>
int power_step_t(mbir_plan p, const uint8_t* mask, void* w, void* v, const double* scal, double* part,
                 cudaStream_t st) {
  LatArgs<R> a = lat_args<R>(p, w, p->wsA, nullptr, p->nz, R(1));
  a.vout = v;
  a.scal = scal;
  int rc = launch_lateral_args<R, LAT_POWER_FWD>(p, a, p->nz, st);
  if (rc) return rc;
  if ((rc = launch_row<R>(p, false, p->wsA, p->wsB, st))) return rc;
  if ((rc = launch_lateral<R, LAT_POWER_MID>(p, p->wsB, p->wsA, mask, p->m, R(1) / R(p->nx), st))) return rc;
  if ((rc = launch_row<R>(p, true, p->wsA, p->wsB, st))) return rc;
  LatArgs<R> b = lat_args<R>(p, p->wsB, w, nullptr, p->nz, R(1));
  b.z1 = v;
  b.partial = part;
  return launch_lateral_args<R, LAT_POWER_ADJ>(p, b, p->nz, st);
}

// ------------------------------------------- Hilbert-form back-projection
//
// Phi*(y) = B^H A(s y) (Eq. back_model): A along the spectrometer axis into wsB,
// then B^H of a complex array: the (1/nx) lateral FFT of wsB into wsA, the row
// adjoint and the inverse lateral FFT.

// c = A(s y) into wsB (interp: unmeasured samples filled first), R = (1/nx)
// lateral FFT of c into wsA
template <class R>
static int hilbert_lateral_t(mbir_plan p, const void* y, const uint8_t* mask, cudaStream_t st, bool interp = false) {
  int rc = hilbert_impl(p, y, mask, p->wsB, st, interp);
  if (rc) return rc;
  return launch_lateral<R, LAT_C2C_FWD>(p, p->wsB, p->wsA, nullptr, p->m, R(1) / R(p->nx), st);
}

template <class R>
int adjoint_hilbert_t(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st, bool interp) {
  int rc = hilbert_lateral_t<R>(p, y, mask, st, interp);
  if (rc) return rc;
  rc = launch_row<R>(p, true, p->wsA, p->wsB, st);
  if (rc) return rc;
  return launch_lateral<R, LAT_C2C_INV>(p, p->wsB, x, nullptr, p->nz, R(1), st);
}

// FISTA forward pass for Phi*: pz = Phi z^{k-1}, the data-term partials and the
// residual r written out (the Hilbert transform runs along m, across the
// lateral column tiles, so r leaves the chip), then A(r) and its lateral FFT
// into wsA for adjoint_solve_impl.  r is zero where the mask is.
template <class R>
int forward_solve_hilbert_t(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, void* r,
                            double mu, double* partial, cudaStream_t st) {
  int rc = launch_lateral<R, LAT_C2C_FWD>(p, z1, p->wsA, nullptr, p->nz, R(1), st);
  if (rc) return rc;
  rc = launch_row<R>(p, false, p->wsA, p->wsB, st);
  if (rc) return rc;
  LatArgs<R> a = lat_args<R>(p, p->wsB, nullptr, mask, p->m, R(1) / R(p->nx));
  a.y = reinterpret_cast<const R*>(y);
  a.pz = reinterpret_cast<R*>(pz);
  a.r = reinterpret_cast<R*>(r);
  a.mu = R(mu);
  a.partial = partial;
  rc = launch_lateral_args<R, LAT_SOLVE_FWD>(p, a, p->m, st);
  if (rc) return rc;
  return hilbert_lateral_t<R>(p, r, nullptr, st);
}

// Power-iteration step for Phi* Phi: v = w scal[1] (written), w = Phi*(s Phi v)
// through the measurement buffer r, partial sums of <v, w> and ||w||^2.
template <class R>
int power_step_hilbert_t(mbir_plan p, const uint8_t* mask, void* w, void* v, void* r, const double* scal,
                         double* part, cudaStream_t st) {
  LatArgs<R> a = lat_args<R>(p, w, p->wsA, nullptr, p->nz, R(1));
  a.vout = v;
  a.scal = scal;
  int rc = launch_lateral_args<R, LAT_POWER_FWD>(p, a, p->nz, st);
  if (rc) return rc;
  if ((rc = launch_row<R>(p, false, p->wsA, p->wsB, st))) return rc;
  if ((rc = launch_lateral<R, LAT_C2R_INV_MASK>(p, p->wsB, r, mask, p->m, R(1) / R(p->nx), st))) return rc;
  if ((rc = hilbert_lateral_t<R>(p, r, nullptr, st))) return rc;
  if ((rc = launch_row<R>(p, true, p->wsA, p->wsB, st))) return rc;
  LatArgs<R> b = lat_args<R>(p, p->wsB, w, nullptr, p->nz, R(1));
  b.z1 = v;
  b.partial = part;
  return launch_lateral_args<R, LAT_POWER_ADJ>(p, b, p->nz, st);
}

int adjoint_hilbert_impl(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st, bool interp) {
  return p->precision == MBIR_FP64 ? adjoint_hilbert_t<double>(p, y, mask, x, st, interp)
                                   : adjoint_hilbert_t<float>(p, y, mask, x, st, interp);
}

int forward_solve_hilbert_impl(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, void* r,
                               double mu, double* partial, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? forward_solve_hilbert_t<double>(p, z1, mask, y, pz, r, mu, partial, st)
                                   : forward_solve_hilbert_t<float>(p, z1, mask, y, pz, r, mu, partial, st);
}

int power_step_hilbert_impl(mbir_plan p, const uint8_t* mask, void* w, void* v, void* r, const double* scal,
                            double* part, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? power_step_hilbert_t<double>(p, mask, w, v, r, scal, part, st)
                                   : power_step_hilbert_t<float>(p, mask, w, v, r, scal, part, st);
}

// ------------------------------------------------------------------ volumes
//
// Phi of a volume x[px][py][n] (Sec. 2.1 with both lateral axes): the 2-D lateral
// transform as the x pass (nx rows, columns (py, n)) and the y pass (ny rows on
// every px slab), the row kernels over the nx * ny rows (lx, ly) with |q|^2 =
// qx^2 + qy^2, then the inverse y pass and the inverse x pass with 1/(nx ny), the
// real part and the mask.  Phi^H is the transpose of each pass in reverse order.

template <class R>
LatArgs<R> lat_args_y(mbir_plan p, const void* in, void* out, int cols) {
  LatArgs<R> a = lat_args<R>(p, in, out, nullptr, cols, R(1));
  a.nx = p->ny;
  a.tc = p->tile_y;
  a.rad = p->rad_y;
  a.tw = p->tw_y;
  a.perm = p->perm_y;
  a.nxl = p->nyl;
  a.chirp = p->chirp_y;
  a.bhat = p->bhat_y;
  return a;
}

template <class R>
size_t lat_smem_y(mbir_plan p) {
  return sizeof(cplx_t<R>) * (size_t)p->nyl * p->tile_y + 16 * (size_t)(p->rad_y.tw_lo + p->rad_y.tw_hi) +
         2 * sizeof(int) * (size_t)p->ny;
}

// in-place y pass of an [nx][ny][cols] complex array
template <class R, int MODE>
int launch_slab(mbir_plan p, void* buf, int cols, cudaStream_t st) {
  const LatArgs<R> a = lat_args_y<R>(p, buf, buf, cols);
  {
    ProfScope ps_(p, MODE == LAT_C2C_FWD ? PC_LAT_FWD : PC_LAT_ADJ, st);
    const dim3 grid((cols + p->tile_y - 1) / p->tile_y, p->nx);
    if (p->chirp_y)
      launch(lateral_slab_kernel<R, MODE, true>, grid, dim3(kLatThreadsBatch), lat_smem_y<R>(p), st, a,
             (long long)p->ny * cols);
    else
      launch(lateral_slab_kernel<R, MODE, false>, grid, dim3(kLatThreadsBatch), lat_smem_y<R>(p), st, a,
             (long long)p->ny * cols);
  }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

template <class R>
int forward_vol_t(mbir_plan p, const void* x, const uint8_t* mask, void* y, cudaStream_t st) {
  const int ny = p->ny;
  int rc = launch_lateral<R, LAT_C2C_FWD>(p, x, p->wsA, nullptr, ny * p->nz, R(1), st);
  if (!rc) rc = launch_slab<R, LAT_C2C_FWD>(p, p->wsA, p->nz, st);
  if (!rc) rc = launch_row<R>(p, false, p->wsA, p->wsB, st);
  if (!rc) rc = launch_slab<R, LAT_C2C_INV>(p, p->wsB, p->m, st);
  if (!rc) rc = launch_lateral<R, LAT_C2R_INV_MASK>(p, p->wsB, y, mask, ny * p->m, R(1) / R(p->nx * ny), st);
  return rc;
}

template <class R>
int adjoint_vol_t(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st) {
  const int ny = p->ny;
  int rc = launch_lateral<R, LAT_R2C_MASK>(p, y, p->wsA, mask, ny * p->m, R(1) / R(p->nx * ny), st);
  if (!rc) rc = launch_slab<R, LAT_C2C_FWD>(p, p->wsA, p->m, st);
  if (!rc) rc = launch_row<R>(p, true, p->wsA, p->wsB, st);
  if (!rc) rc = launch_slab<R, LAT_C2C_INV>(p, p->wsB, p->nz, st);
  if (!rc) rc = launch_lateral<R, LAT_C2C_INV>(p, p->wsB, x, nullptr, ny * p->nz, R(1), st);
  return rc;
}

int forward_impl(mbir_plan p, const void* x, const uint8_t* mask, void* y, cudaStream_t st) {
  if (p->ny > 1)
    return p->precision == MBIR_FP64 ? forward_vol_t<double>(p, x, mask, y, st)
                                     : forward_vol_t<float>(p, x, mask, y, st);
  return p->precision == MBIR_FP64 ? forward_t<double>(p, x, mask, y, st)
                                   : forward_t<float>(p, x, mask, y, st);
}

int adjoint_impl(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st) {
  if (p->ny > 1)
    return p->precision == MBIR_FP64 ? adjoint_vol_t<double>(p, y, mask, x, st)
                                     : adjoint_vol_t<float>(p, y, mask, x, st);
  return p->precision == MBIR_FP64 ? adjoint_t<double>(p, y, mask, x, st)
                                   : adjoint_t<float>(p, y, mask, x, st);
}

int forward_solve_impl(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, double mu,
                       double* partial, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? forward_solve_t<double>(p, z1, mask, y, pz, mu, partial, st)
                                   : forward_solve_t<float>(p, z1, mask, y, pz, mu, partial, st);
}

int adjoint_solve_impl(mbir_plan p, const void* z1, void* z2, void* vout, double mu, double delta, double tau,
                       double* partial, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? adjoint_solve_t<double>(p, z1, z2, vout, mu, delta, tau, partial, st)
                                   : adjoint_solve_t<float>(p, z1, z2, vout, mu, delta, tau, partial, st);
}

int power_step_impl(mbir_plan p, const uint8_t* mask, void* w, void* v, const double* scal, double* part,
                    cudaStream_t st) {
  return p->precision == MBIR_FP64 ? power_step_t<double>(p, mask, w, v, scal, part, st)
                                   : power_step_t<float>(p, mask, w, v, scal, part, st);
}

template <class R>
static int configure_t() {
  const int lat = (int)(sizeof(cplx_t<R>) * kLatElems + 16 * 512 + 2 * sizeof(int) * 4096);
  const int row = (int)(sizeof(cplx_t<R>) * (kMaxFFT + 512));
  const int gat = kMaxDynSmem;
#define MBIR_SMEM_ATTR(fn, bytes)                                                                  \
  MBIR_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));    \
  MBIR_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100))
#define MBIR_LAT_ATTRS(M)                                                                   \
  MBIR_SMEM_ATTR((lateral_kernel<R, M, false, false>), lat);                                \
  MBIR_SMEM_ATTR((lateral_kernel<R, M, true, false>), lat);                                 \
  MBIR_SMEM_ATTR((lateral_kernel<R, M, false, true>), lat);                                 \
  MBIR_SMEM_ATTR((lateral_kernel<R, M, true, true>), lat);                                  \
  if constexpr (sizeof(R) == 4 && kLatFuse) {                                               \
    MBIR_SMEM_ATTR((lateral_kernel<R, M, false, false, sizeof(R) == 4 ? 1 : 0>), lat);     \
    MBIR_SMEM_ATTR((lateral_kernel<R, M, true, false, sizeof(R) == 4 ? 2 : 0>), lat);      \
  }
  MBIR_LAT_ATTRS(LAT_C2C_FWD);
  MBIR_LAT_ATTRS(LAT_C2C_INV);
  MBIR_LAT_ATTRS(LAT_R2C_MASK);
  MBIR_LAT_ATTRS(LAT_C2R_INV_MASK);
  MBIR_LAT_ATTRS(LAT_SOLVE_FWD);
  MBIR_LAT_ATTRS(LAT_SOLVE_ADJ_L1);
  MBIR_LAT_ATTRS(LAT_SOLVE_ADJ_V);
  MBIR_LAT_ATTRS(LAT_SOLVE_MID);
  MBIR_LAT_ATTRS(LAT_POWER_MID);
  MBIR_LAT_ATTRS(LAT_POWER_FWD);
  MBIR_LAT_ATTRS(LAT_POWER_ADJ);
  MBIR_SMEM_ATTR((lateral_slab_kernel<R, LAT_C2C_FWD, false>), lat);
  MBIR_SMEM_ATTR((lateral_slab_kernel<R, LAT_C2C_INV, false>), lat);
  MBIR_SMEM_ATTR((lateral_slab_kernel<R, LAT_C2C_FWD, true>), lat);
  MBIR_SMEM_ATTR((lateral_slab_kernel<R, LAT_C2C_INV, true>), lat);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 4, false>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 4, true>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 6, false>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 6, true>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 8, false>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 8, true>), row);
  MBIR_SMEM_ATTR((row_adjoint_kernel<R, 4, false>), row);
  MBIR_SMEM_ATTR((row_adjoint_kernel<R, 4, true>), row);
  MBIR_SMEM_ATTR((row_adjoint_kernel<R, 6, false>), row);
  MBIR_SMEM_ATTR((row_adjoint_kernel<R, 6, true>), row);
  MBIR_SMEM_ATTR((row_adjoint_kernel<R, 8, false>), row);
  MBIR_SMEM_ATTR((row_adjoint_kernel<R, 8, true>), row);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 4, false>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 4, true>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 6, false>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 6, true>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 8, false>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 8, true>), gat);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 4, false, true>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 6, false, true>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 8, false, true>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 4, true, true>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 6, true, true>), row);
  MBIR_SMEM_ATTR((row_forward_kernel<R, 8, true, true>), row);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 4, false, true>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 6, false, true>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 8, false, true>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 4, true, true>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 6, true, true>), gat);
  MBIR_SMEM_ATTR((row_adjoint_gather_kernel<R, 8, true, true>), gat);
  if constexpr (sizeof(R) == 4) {
    MBIR_SMEM_ATTR((row_forward_pair_kernel<4, false, false>), gat);
    MBIR_SMEM_ATTR((row_forward_pair_kernel<4, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_forward_pair_kernel<4, false, true>), gat); }
    MBIR_SMEM_ATTR((row_forward_pair_kernel<4, true, false>), gat);
    MBIR_SMEM_ATTR((row_forward_pair_kernel<4, true, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_forward_pair_kernel<4, true, true>), gat); }
    MBIR_SMEM_ATTR((row_forward_pair_kernel<6, false, false>), gat);
    MBIR_SMEM_ATTR((row_forward_pair_kernel<6, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_forward_pair_kernel<6, false, true>), gat); }
    MBIR_SMEM_ATTR((row_forward_pair_kernel<6, true, false>), gat);
    MBIR_SMEM_ATTR((row_forward_pair_kernel<6, true, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_forward_pair_kernel<6, true, true>), gat); }
    MBIR_SMEM_ATTR((row_forward_pair_kernel<8, false, false>), gat);
    MBIR_SMEM_ATTR((row_forward_pair_kernel<8, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_forward_pair_kernel<8, false, true>), gat); }
    MBIR_SMEM_ATTR((row_forward_pair_kernel<8, true, false>), gat);
    MBIR_SMEM_ATTR((row_forward_pair_kernel<8, true, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_forward_pair_kernel<8, true, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_kernel<4, false, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_kernel<4, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_kernel<4, false, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_kernel<4, true, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_kernel<4, true, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_kernel<4, true, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_kernel<6, false, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_kernel<6, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_kernel<6, false, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_kernel<6, true, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_kernel<6, true, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_kernel<6, true, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_kernel<8, false, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_kernel<8, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_kernel<8, false, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_kernel<8, true, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_kernel<8, true, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_kernel<8, true, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<4, false, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<4, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<4, false, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<4, true, false>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<4, true, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<6, false, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<6, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<6, false, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<6, true, false>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<6, true, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<8, false, false>), gat);
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<8, false, false, 1>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<8, false, true>), gat); }
    MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<8, true, false>), gat);
    if constexpr (kFilterOtf) { MBIR_SMEM_ATTR((row_gather_pair_lean_kernel<8, true, true>), gat); }
  }
#undef MBIR_LAT_ATTRS
#undef MBIR_SMEM_ATTR
  return MBIR_OK;
}

int configure_operator_kernels(mbir_plan p) {
  return p->precision == MBIR_FP64 ? configure_t<double>() : configure_t<float>();
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

int mbir_adjoint_hilbert(mbir_plan p, const void* y, const uint8_t* mask, void* x, void* stream) {
  if (const int vrc = bscan_only(p, "mbir_adjoint_hilbert")) return vrc;
  const int rc = check_common(p, y, x);
  if (rc) return rc;
  return adjoint_hilbert_impl(p, y, mask, x, (cudaStream_t)stream);
}

int mbir_isam_interpolated(mbir_plan p, const void* y, const uint8_t* mask, void* x, void* stream) {
  if (const int vrc = bscan_only(p, "mbir_isam_interpolated")) return vrc;
  const int rc = check_common(p, y, x);
  if (rc) return rc;
  return adjoint_hilbert_impl(p, y, mask, x, (cudaStream_t)stream, true);
}

}  // extern "C"

// ------------------------------------------------------------ batched launches
//
// Helpers for the batch engine (batch.cu): build a scan's argument block into
// host memory and launch one stage over a device array of such blocks.

namespace mbir {

size_t lat_args_bytes(int precision) {
  return precision == MBIR_FP64 ? sizeof(LatArgs<double>) : sizeof(LatArgs<float>);
}
size_t row_args_bytes(int precision) {
  return precision == MBIR_FP64 ? sizeof(RowArgs<double>) : sizeof(RowArgs<float>);
}
size_t lat_smem_bytes(mbir_plan p) {
  return p->precision == MBIR_FP64 ? lat_smem<double>(p) : lat_smem<float>(p);
}
size_t row_smem_bytes(mbir_plan p, int adjoint_gather) {
  if (p->precision == MBIR_FP64) return adjoint_gather ? row_gather_smem<double>(p) : row_smem<double>(p);
  return adjoint_gather ? row_gather_smem<float>(p) : row_smem<float>(p);
}

template <class R>
static void fill_lat_t(mbir_plan p, const LatFill& f, void* dst) {
  LatArgs<R> a = lat_args<R>(p, f.in, f.out, f.mask, f.cols, R(f.scale));
  a.y = reinterpret_cast<const R*>(f.y);
  a.pz = reinterpret_cast<R*>(f.pz);
  a.r = reinterpret_cast<R*>(f.r);
  a.z1 = f.z1;
  a.z2 = f.z2;
  a.vout = f.vout;
  a.mu = R(f.mu);
  a.delta = R(f.delta);
  a.tau = R(f.tau);
  a.partial = f.partial;
  a.scal = f.scal;
  memcpy(dst, &a, sizeof(a));
}

void fill_lat_args(mbir_plan p, const LatFill& f, void* dst) {
  if (p->precision == MBIR_FP64) fill_lat_t<double>(p, f, dst);
  else fill_lat_t<float>(p, f, dst);
}

void fill_row_args(mbir_plan p, const void* in, void* out, void* dst) {
  if (p->precision == MBIR_FP64) {
    RowArgs<double> a = row_args<double>(p, in, out);
    memcpy(dst, &a, sizeof(a));
  } else {
    RowArgs<float> a = row_args<float>(p, in, out);
    memcpy(dst, &a, sizeof(a));
  }
}

template <class R, int MODE>
static void lat_batch_t(const BatchLaunch& L, cudaStream_t st) {
  BatchRef<LatArgs<R>> B;
  B.args = reinterpret_cast<const LatArgs<R>*>(L.dargs);
  B.off = L.doff;
  B.n = L.n;
  B.set_mu = L.set_mu;
  B.mu = L.mu;
  LatArgs<R> a0;
  memcpy(&a0, L.host0, sizeof(a0));
  if (L.blu)
    launch(lateral_kernel<R, MODE, true, true>, dim3(L.total), dim3(kLatThreadsBatch), L.smem, st, a0, B);
  else if (sizeof(R) == 4 && kLatFuse)
    launch(lateral_kernel<R, MODE, true, false, sizeof(R) == 4 ? 2 : 0>, dim3(L.total), dim3(kLatThreadsBatch), L.smem,
           st, a0, B);
  else
    launch(lateral_kernel<R, MODE, true, false>, dim3(L.total), dim3(kLatThreadsBatch), L.smem, st, a0, B);
}

int batch_lateral(int mode, int precision, const BatchLaunch& L, cudaStream_t st) {
  if (L.total <= 0) return MBIR_OK;
#define MBIR_LAT_CASE(M)                                                         \
  case M:                                                                        \
    if (precision == MBIR_FP64) lat_batch_t<double, M>(L, st);                   \
    else lat_batch_t<float, M>(L, st);                                           \
    break;
  switch (mode) {
    MBIR_LAT_CASE(LAT_C2C_FWD)
    MBIR_LAT_CASE(LAT_C2C_INV)
    MBIR_LAT_CASE(LAT_R2C_MASK)
    MBIR_LAT_CASE(LAT_C2R_INV_MASK)
    MBIR_LAT_CASE(LAT_SOLVE_FWD)
    MBIR_LAT_CASE(LAT_SOLVE_ADJ_L1)
    MBIR_LAT_CASE(LAT_SOLVE_ADJ_V)
    MBIR_LAT_CASE(LAT_SOLVE_MID)
    MBIR_LAT_CASE(LAT_POWER_MID)
    MBIR_LAT_CASE(LAT_POWER_FWD)
    MBIR_LAT_CASE(LAT_POWER_ADJ)
    default: return MBIR_ERR_INVALID;
  }
#undef MBIR_LAT_CASE
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

template <class R>
static void row_batch_t(int kind, int J, bool comp, const BatchLaunch& L, cudaStream_t st) {
  BatchRef<RowArgs<R>> B;
  B.args = reinterpret_cast<const RowArgs<R>*>(L.dargs);
  B.off = L.doff;
  B.n = L.n;
  B.set_mu = 0;
  B.mu = 0.0;
  RowArgs<R> a0;
  memcpy(&a0, L.host0, sizeof(a0));
  row_launch<R, true>(kind, J, comp, a0, B, L.total, L.smem, st, L.fz != 0);
}

int batch_row(int kind, int precision, int J, const BatchLaunch& L, cudaStream_t st) {
  if (L.total <= 0) return MBIR_OK;
  if (precision == MBIR_FP64) row_batch_t<double>(kind, J, false, L, st);
  else row_batch_t<float>(kind, J, precision == MBIR_FP32_COMPENSATED, L, st);
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

}  // namespace mbir
