// Orthonormal wavelet penalty transform Psi (Sec. 2.2): 3-level periodic 2-D
// Daubechies wavelet with 4 vanishing moments (8 taps), applied to the real and
// imaginary parts alike, and its proximal map Psi^T soft(Psi v, tau) (Sec. 2.3).
//
// Layout (Mallat): at each level the current low-low block of size P x N, stored
// at the top-left of an [nx][nz] array, becomes [[LL, LH], [HL, HH]] with blocks
// of P/2 x N/2; the first letter is the filter along the lateral axis p, the
// second along depth n.  One analysis level:
//   lo_n / hi_n[i][b] = sum_t h_t / g_t  x[i][(2b + t) mod N]
//   LL / HL[a][b]     = sum_t h_t / g_t  lo_n[(2a + t) mod P][b]
//   LH / HH[a][b]     = sum_t h_t / g_t  hi_n[(2a + t) mod P][b]
// with g_t = (-1)^t h_{7-t}.  Synthesis is the transpose, written as a gather:
// output index X receives from coefficient (X - t)/2 for the four t of X's parity.
#include <math.h>
#include <string.h>

#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace mbir {

// threads per CTA: 256 for the finest level, 128 for the coarse levels' tiles
template <bool SMALL>
constexpr int wav_threads() { return SMALL ? 128 : 256; }

// Tiles.  Analysis computes a TA x TB block of every band's coefficients from a
// (2 TA + 6) x (2 TB + 6) input block; synthesis a TR x TC block of output pixels
// from (TR/2 + 3) x (TC/2 + 3) coefficients per band.  The coarse levels (level >=
// 1, a quarter and a sixteenth of the image) use half-width tiles in half-size
// CTAs so that their grids still cover the SMs and every thread has work.
template <bool SMALL>
struct FwdTile {
  static constexpr int TA = 16, TB = SMALL ? 16 : 32;
  static constexpr int Rows = 2 * TA + 6, Cols = 2 * TB + 6;
};
template <bool SMALL>
struct InvTile {
  static constexpr int TR = 32, TC = SMALL ? 32 : 64;
  static constexpr int Rows = TR / 2 + 3, Cols = TC / 2 + 3;
};
constexpr bool dwt_small(int level) { return level > 0; }

template <class R>
struct WArgs {
  const void* in;
  int istride;      // analysis: input block; synthesis: LL block
  void* out;
  int ostride;      // analysis: LL output; synthesis: output block
  void* coef;
  int cstride;      // detail bands at their Mallat positions (level block at the origin)
  int P, N;         // level block size (analysis input / synthesis output)
  const R* h;       // 8 low-pass taps
  R tau;
  int thresh;       // analysis: 0 none, 1 details, 2 details and LL
  double* partial;  // analysis with thresh: sum |soft(c)| per CTA
  int gx;           // CTAs along the columns (the grid is flattened row-major)
};

template <class Args>
__device__ __forceinline__ Args resolve_wargs(const Args& a0, const BatchRef<Args>& B, int& blk) {
  blk = blockIdx.x;
  if (B.args == nullptr) return a0;
  int lo = 0, hi = B.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.off[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  blk -= B.off[lo];
  return B.args[lo];
}

template <class R>
__device__ __forceinline__ cplx_t<R> soft_c(cplx_t<R> c, R tau, R& acc) {
  const R mag = sqrt(c.x * c.x + c.y * c.y);
  const R s = mag > tau ? R(1) - tau / mag : R(0);
  if (mag > tau) acc += mag - tau;
  return cmk<cplx_t<R>>(c.x * s, c.y * s);
}

__device__ __forceinline__ double block_sum_w(double v) {
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
  return t;
}

// acc += w x for a complex x and a real tap given broadcast ({w, w}): one paired
// FP32 instruction (FFMA2) in single precision.
template <class V>
__device__ __forceinline__ void tap(V& acc, V wb, V x) {
  if constexpr (sizeof(V) == 8) {
    acc = __ffma2_rn(x, wb, acc);
  } else {
    acc.x += wb.x * x.x;
    acc.y += wb.y * x.y;
  }
}

// The 8 low-pass taps h and the high-pass taps g_t = (-1)^t h_{7-t}, broadcast.
template <class R>
__device__ __forceinline__ void load_taps(const R* hsrc, cplx_t<R>* hb, cplx_t<R>* gb) {
  const int t = threadIdx.x;
  if (t < 8) {
    const R hv = hsrc[t], gv = ((t & 1) ? R(-1) : R(1)) * hsrc[7 - t];
    hb[t] = cmk<cplx_t<R>>(hv, hv);
    gb[t] = cmk<cplx_t<R>>(gv, gv);
  }
}

// Every thread computes two neighbouring outputs of a filter stage: they share
// 6 of their 8 inputs (analysis) or all 4 coefficient positions (synthesis),
// which are loaded from shared memory once.
template <class R, bool SMALL>
__global__ void __launch_bounds__(wav_threads<SMALL>())
dwt_fwd_kernel(const __grid_constant__ WArgs<R> arg0, const BatchRef<WArgs<R>> B) {
  using V = cplx_t<R>;
  constexpr int kTA = FwdTile<SMALL>::TA, kTB = FwdTile<SMALL>::TB;
  constexpr int kRows = FwdTile<SMALL>::Rows, kCols = FwdTile<SMALL>::Cols;
  int blk;
  const WArgs<R> a = resolve_wargs(arg0, B, blk);
  const int bx = blk % a.gx, by = blk / a.gx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tin = reinterpret_cast<V*>(smem_raw);        // [kRows][kCols]
  V* tL = tin + kRows * kCols;                    // [kRows][kTB]
  V* tH = tL + kRows * kTB;
  __shared__ V hb[8], gb[8];
  const int tid = threadIdx.x, nthr = blockDim.x;
  load_taps<R>(a.h, hb, gb);
  const int P = a.P, N = a.N;
  const int a0 = by * kTA, b0 = bx * kTB;
  const V* in = reinterpret_cast<const V*>(a.in);
  pdl_wait_release();
  // stage the input tile with every load of a thread in flight at once.  The
  // window starts inside the block, so one subtraction of P (N) wraps it when the
  // block is at least as large as the window; the coarse levels of small images,
  // whose window can span the block several times, take the remainder as well
  // (a branch that is the same for the whole grid)
  constexpr int kFwdPer = (kRows * kCols + wav_threads<SMALL>() - 1) / wav_threads<SMALL>();
  auto stage = [&](auto small_block) {
    V vv[kFwdPer];
#pragma unroll
    for (int q = 0; q < kFwdPer; ++q) {
      const int e = tid + q * nthr;
      if (e < kRows * kCols) {
        const int i = e / kCols, j = e - i * kCols;
        int row = 2 * a0 + i, col = 2 * b0 + j;
        if (row >= P) row -= P;
        if (col >= N) col -= N;
        if constexpr (decltype(small_block)::value) {
          row %= P;
          col %= N;
        }
        vv[q] = in[(size_t)row * a.istride + col];
      }
    }
#pragma unroll
    for (int q = 0; q < kFwdPer; ++q) {
      const int e = tid + q * nthr;
      if (e < kRows * kCols) tin[e] = vv[q];
    }
  };
  if (P < kRows || N < kCols) stage(std::true_type());
  else stage(std::false_type());
  __syncthreads();
  // along depth: outputs b, b + 1 of row i from inputs 2b .. 2b + 9
  for (int e = tid; e < kRows * (kTB / 2); e += nthr) {
    const int i = e / (kTB / 2), bp = e - i * (kTB / 2);
    const V* src = tin + i * kCols + 4 * bp;
    const V z = cmk<V>(R(0), R(0));
    V lo0 = z, hi0 = z, lo1 = z, hi1 = z;
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      const V x = src[t];
      if (t < 8) {
        tap(lo0, hb[t], x);
        tap(hi0, gb[t], x);
      }
      if (t >= 2) {
        tap(lo1, hb[t - 2], x);
        tap(hi1, gb[t - 2], x);
      }
    }
    tL[i * kTB + 2 * bp] = lo0;
    tL[i * kTB + 2 * bp + 1] = lo1;
    tH[i * kTB + 2 * bp] = hi0;
    tH[i * kTB + 2 * bp + 1] = hi1;
  }
  __syncthreads();
  const int Ph = P / 2, Nh = N / 2;
  V* coef = reinterpret_cast<V*>(a.coef);
  V* llo = reinterpret_cast<V*>(a.out);
  R acc = R(0);   // a thread's few terms in the working precision; FP64 across the block
  // along the A-scans: outputs ai, ai + 1 of column b from rows 2 ai .. 2 ai + 9
  for (int e = tid; e < (kTA / 2) * kTB; e += nthr) {
    const int ap = e / kTB, b = e - ap * kTB;
    const V z = cmk<V>(R(0), R(0));
    V ll[2] = {z, z}, hl[2] = {z, z}, lh[2] = {z, z}, hh[2] = {z, z};
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      const V xl = tL[(4 * ap + t) * kTB + b];
      const V xh = tH[(4 * ap + t) * kTB + b];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int tt = t - 2 * k;
        if (tt < 0 || tt >= 8) continue;
        tap(ll[k], hb[tt], xl);
        tap(hl[k], gb[tt], xl);
        tap(lh[k], hb[tt], xh);
        tap(hh[k], gb[tt], xh);
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int A = a0 + 2 * ap + k, Bc = b0 + b;
      if (A >= Ph || Bc >= Nh) continue;
      V vll = ll[k], vhl = hl[k], vlh = lh[k], vhh = hh[k];
      if (a.thresh >= 1) {
        vlh = soft_c<R>(vlh, a.tau, acc);
        vhl = soft_c<R>(vhl, a.tau, acc);
        vhh = soft_c<R>(vhh, a.tau, acc);
      }
      if (a.thresh == 2) vll = soft_c<R>(vll, a.tau, acc);
      llo[(size_t)A * a.ostride + Bc] = vll;
      coef[(size_t)A * a.cstride + Nh + Bc] = vlh;
      coef[(size_t)(Ph + A) * a.cstride + Bc] = vhl;
      coef[(size_t)(Ph + A) * a.cstride + Nh + Bc] = vhh;
    }
  }
  if (a.partial) {
    const double t = block_sum_w(double(acc));
    if (tid == 0) a.partial[blk] = t;
  }
}

template <class R, bool SMALL>
__global__ void __launch_bounds__(wav_threads<SMALL>())
dwt_inv_kernel(const __grid_constant__ WArgs<R> arg0, const BatchRef<WArgs<R>> B) {
  using V = cplx_t<R>;
  constexpr int kTR = InvTile<SMALL>::TR, kTC = InvTile<SMALL>::TC;
  constexpr int kRows = InvTile<SMALL>::Rows, kCols = InvTile<SMALL>::Cols;
  int blk;
  const WArgs<R> a = resolve_wargs(arg0, B, blk);
  const int bx = blk % a.gx, by = blk / a.gx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* cLL = reinterpret_cast<V*>(smem_raw);        // [kRows][kCols] each
  V* cLH = cLL + kRows * kCols;
  V* cHL = cLH + kRows * kCols;
  V* cHH = cHL + kRows * kCols;
  V* tlo = cHH + kRows * kCols;                   // [kTR][kCols]
  V* thi = tlo + kTR * kCols;
  __shared__ V hb[8], gb[8];
  const int tid = threadIdx.x, nthr = blockDim.x;
  load_taps<R>(a.h, hb, gb);
  const int P = a.P, N = a.N, Ph = P / 2, Nh = N / 2;
  const int r0 = by * kTR, c0 = bx * kTC;
  const V* ll = reinterpret_cast<const V*>(a.in);
  const V* coef = reinterpret_cast<const V*>(a.coef);
  pdl_wait_release();
  constexpr int kInvPer = (kRows * kCols + wav_threads<SMALL>() - 1) / wav_threads<SMALL>();
  {
    V v0[kInvPer], v1[kInvPer], v2[kInvPer], v3[kInvPer];
#pragma unroll
    for (int q = 0; q < kInvPer; ++q) {
      const int e = tid + q * nthr;
      if (e < kRows * kCols) {
        const int ia = e / kCols, ib = e - ia * kCols;
        // r0/2 - 3 + ia lies in [-3, Ph + kRows): one wrap up (Ph, Nh >= 4), and
        // as many down as the window spans the block
        int A = r0 / 2 - 3 + ia, Bc = c0 / 2 - 3 + ib;
        if (A < 0) A += Ph;
        while (A >= Ph) A -= Ph;
        if (Bc < 0) Bc += Nh;
        while (Bc >= Nh) Bc -= Nh;
        v0[q] = ll[(size_t)A * a.istride + Bc];
        v1[q] = coef[(size_t)A * a.cstride + Nh + Bc];
        v2[q] = coef[(size_t)(Ph + A) * a.cstride + Bc];
        v3[q] = coef[(size_t)(Ph + A) * a.cstride + Nh + Bc];
      }
    }
#pragma unroll
    for (int q = 0; q < kInvPer; ++q) {
      const int e = tid + q * nthr;
      if (e < kRows * kCols) {
        cLL[e] = v0[q];
        cLH[e] = v1[q];
        cHL[e] = v2[q];
        cHH[e] = v3[q];
      }
    }
  }
  __syncthreads();
  // along the A-scans: output rows r = 2 rp (taps 0, 2, 4, 6) and r + 1 (taps
  // 1, 3, 5, 7) read the same coefficient rows rp + 3 - q, q = 0 .. 3
  for (int e = tid; e < (kTR / 2) * kCols; e += nthr) {
    const int rp = e / kCols, ib = e - rp * kCols;
    const V z = cmk<V>(R(0), R(0));
    V lo0 = z, hi0 = z, lo1 = z, hi1 = z;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ia = rp + 3 - q;
      const V vll = cLL[ia * kCols + ib], vhl = cHL[ia * kCols + ib];
      const V vlh = cLH[ia * kCols + ib], vhh = cHH[ia * kCols + ib];
      tap(lo0, hb[2 * q], vll);
      tap(lo0, gb[2 * q], vhl);
      tap(hi0, hb[2 * q], vlh);
      tap(hi0, gb[2 * q], vhh);
      tap(lo1, hb[2 * q + 1], vll);
      tap(lo1, gb[2 * q + 1], vhl);
      tap(hi1, hb[2 * q + 1], vlh);
      tap(hi1, gb[2 * q + 1], vhh);
    }
    tlo[(2 * rp) * kCols + ib] = lo0;
    thi[(2 * rp) * kCols + ib] = hi0;
    tlo[(2 * rp + 1) * kCols + ib] = lo1;
    thi[(2 * rp + 1) * kCols + ib] = hi1;
  }
  __syncthreads();
  V* out = reinterpret_cast<V*>(a.out);
  // along depth: output columns c = 2 cp and c + 1 share the coefficient columns
  for (int e = tid; e < kTR * (kTC / 2); e += nthr) {
    const int r = e / (kTC / 2), cp = e - r * (kTC / 2);
    if (r0 + r >= P) continue;
    const V z = cmk<V>(R(0), R(0));
    V x0 = z, x1 = z;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ib = cp + 3 - q;
      const V lo = tlo[r * kCols + ib], hi = thi[r * kCols + ib];
      tap(x0, hb[2 * q], lo);
      tap(x0, gb[2 * q], hi);
      tap(x1, hb[2 * q + 1], lo);
      tap(x1, gb[2 * q + 1], hi);
    }
    const int c = c0 + 2 * cp;
    if (c < N) out[(size_t)(r0 + r) * a.ostride + c] = x0;
    if (c + 1 < N) out[(size_t)(r0 + r) * a.ostride + c + 1] = x1;
  }
}

template <class R>
__global__ void soft_kernel(const cplx_t<R>* v, cplx_t<R>* z, size_t n, R tau, double* partial) {
  pdl_wait_release();
  R acc = R(0);   // a thread's few terms in the working precision; FP64 across the block
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    z[i] = soft_c<R>(v[i], tau, acc);
  if (partial) {
    const double t = block_sum_w(double(acc));
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

template <bool SMALL>
static size_t fwd_smem_t(size_t vs) {
  using T = FwdTile<SMALL>;
  return vs * (T::Rows * T::Cols + 2 * T::Rows * T::TB);
}
template <bool SMALL>
static size_t inv_smem_t(size_t vs) {
  using T = InvTile<SMALL>;
  return vs * (4 * T::Rows * T::Cols + 2 * T::TR * T::Cols);
}
static size_t fwd_smem(size_t vs, int level) { return dwt_small(level) ? fwd_smem_t<true>(vs) : fwd_smem_t<false>(vs); }
static size_t inv_smem(size_t vs, int level) { return dwt_small(level) ? inv_smem_t<true>(vs) : inv_smem_t<false>(vs); }

// CTAs along the columns and in total of analysis (inverse = 0) or synthesis of a
// level whose block (analysis input / synthesis output) is P x N.
static int dwt_gx(int N, int inverse, int level) {
  if (inverse) {
    const int tc = dwt_small(level) ? InvTile<true>::TC : InvTile<false>::TC;
    return (N + tc - 1) / tc;
  }
  const int tb = dwt_small(level) ? FwdTile<true>::TB : FwdTile<false>::TB;
  return (N / 2 + tb - 1) / tb;
}
static int dwt_gy(int P, int inverse, int level) {
  if (inverse) {
    const int tr = dwt_small(level) ? InvTile<true>::TR : InvTile<false>::TR;
    return (P + tr - 1) / tr;
  }
  const int ta = dwt_small(level) ? FwdTile<true>::TA : FwdTile<false>::TA;
  return (P / 2 + ta - 1) / ta;
}

int wavelet_partial_count(int nx, int nz) {
  int total = 0, P = nx, N = nz;
  for (int lev = 0; lev < 3; ++lev) {
    total += dwt_gx(N, 0, lev) * dwt_gy(P, 0, lev);
    P /= 2;
    N /= 2;
  }
  return total;
}

int ensure_wavelet_scratch(mbir_plan p) {
  if (p->wv_b1) return MBIR_OK;
  const size_t es = p->precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t n = (size_t)p->nx * p->nz;
  MBIR_CUDA_TRY(cudaMalloc(&p->wv_b1, es * (n / 4)));
  MBIR_CUDA_TRY(cudaMalloc(&p->wv_b2, es * (n / 16)));
  MBIR_CUDA_TRY(cudaMalloc(&p->wv_coef, es * n));
  return MBIR_OK;
}

template <class R>
static int analysis_t(mbir_plan p, const void* in, void* coef, bool thresh, R tau, double* partial,
                      cudaStream_t st) {
  const int nx = p->nx, nz = p->nz;
  const void* src = in;
  int sstride = nz;
  int P = nx, N = nz;
  double* part = partial;
  void* lls[3] = {p->wv_b1, p->wv_b2, coef};
  int lstr[3] = {nz / 2, nz / 4, nz};
  for (int lev = 0; lev < 3; ++lev) {
    WArgs<R> a;
    a.in = src;
    a.istride = sstride;
    a.out = lls[lev];
    a.ostride = lstr[lev];
    a.coef = coef;
    a.cstride = nz;
    a.P = P;
    a.N = N;
    a.h = p->precision == MBIR_FP64 ? reinterpret_cast<const R*>(p->h_db4) : reinterpret_cast<const R*>(p->h_db4f);
    a.tau = tau;
    a.thresh = thresh ? (lev == 2 ? 2 : 1) : 0;
    a.partial = thresh ? part : nullptr;
    const int gx = dwt_gx(N, 0, lev), gy = dwt_gy(P, 0, lev);
    a.gx = gx;
    {
      ProfScope ps_(p, PC_DWT_FWD, st);
      launch(dwt_small(lev) ? dwt_fwd_kernel<R, true> : dwt_fwd_kernel<R, false>, dim3(gx * gy),
             dim3(dwt_small(lev) ? wav_threads<true>() : wav_threads<false>()),
             fwd_smem(sizeof(cplx_t<R>), lev), st, a, no_batch<WArgs<R>>());
    }
    MBIR_LAUNCH_CHECK();
    if (part) part += gx * gy;
    src = lls[lev];
    sstride = lstr[lev];
    P /= 2;
    N /= 2;
  }
  return MBIR_OK;
}

template <class R>
static int synthesis_t(mbir_plan p, const void* coef, void* out, cudaStream_t st) {
  const int nx = p->nx, nz = p->nz;
  const void* lls[3] = {p->wv_b1, p->wv_b2, coef};
  const int lstr[3] = {nz / 2, nz / 4, nz};
  void* outs[3] = {out, p->wv_b1, p->wv_b2};
  const int ostr[3] = {nz, nz / 2, nz / 4};
  for (int lev = 2; lev >= 0; --lev) {
    WArgs<R> a;
    a.in = lls[lev];
    a.istride = lstr[lev];
    a.out = outs[lev];
    a.ostride = ostr[lev];
    a.coef = const_cast<void*>(coef);
    a.cstride = nz;
    a.P = nx >> lev;
    a.N = nz >> lev;
    a.h = p->precision == MBIR_FP64 ? reinterpret_cast<const R*>(p->h_db4) : reinterpret_cast<const R*>(p->h_db4f);
    a.tau = R(0);
    a.thresh = 0;
    a.partial = nullptr;
    const int gx = dwt_gx(a.N, 1, lev), gy = dwt_gy(a.P, 1, lev);
    a.gx = gx;
    {
      ProfScope ps_(p, PC_DWT_INV, st);
      launch(dwt_small(lev) ? dwt_inv_kernel<R, true> : dwt_inv_kernel<R, false>, dim3(gx * gy),
             dim3(dwt_small(lev) ? wav_threads<true>() : wav_threads<false>()),
             inv_smem(sizeof(cplx_t<R>), lev), st, a, no_batch<WArgs<R>>());
    }
    MBIR_LAUNCH_CHECK();
  }
  return MBIR_OK;
}

bool wavelet_supported(int nx, int nz) { return nx % 8 == 0 && nz % 8 == 0 && nx >= 32 && nz >= 32; }

template <class R>
static int configure_wavelet_t() {
  MBIR_CUDA_TRY(cudaFuncSetAttribute(dwt_fwd_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)fwd_smem_t<false>(sizeof(cplx_t<R>))));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(dwt_fwd_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)fwd_smem_t<true>(sizeof(cplx_t<R>))));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(dwt_inv_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)inv_smem_t<false>(sizeof(cplx_t<R>))));
  MBIR_CUDA_TRY(cudaFuncSetAttribute(dwt_inv_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)inv_smem_t<true>(sizeof(cplx_t<R>))));
  return MBIR_OK;
}

int configure_wavelet_kernels(mbir_plan p) {
  return p->precision == MBIR_FP64 ? configure_wavelet_t<double>() : configure_wavelet_t<float>();
}

int wavelet_impl(mbir_plan p, int inverse, const void* in, void* out, cudaStream_t st) {
  if (!wavelet_supported(p->nx, p->nz)) return MBIR_ERR_UNSUPPORTED_SIZE;
  int rc = ensure_wavelet_scratch(p);
  if (rc) return rc;
  if (p->precision == MBIR_FP64)
    return inverse ? synthesis_t<double>(p, in, out, st) : analysis_t<double>(p, in, out, false, 0.0, nullptr, st);
  return inverse ? synthesis_t<float>(p, in, out, st) : analysis_t<float>(p, in, out, false, 0.0f, nullptr, st);
}

// z = prox of tau ||Psi .||_1 at v; partial (may be null) receives per-CTA sums of
// |Psi z| (wavelet_partial_count entries for DB4, soft_grid entries for L1).
int prox_partial_impl(mbir_plan p, int penalty, const void* v, double tau, void* z, double* partial,
                      cudaStream_t st) {
  const bool f64 = p->precision == MBIR_FP64;
  if (penalty == MBIR_PENALTY_TV) {
    // the TV stencil reads neighbouring tiles of v: an aliased v is copied first
    if (v == z) {
      MBIR_CUDA_TRY(cudaMemcpyAsync(p->wsA, v, (f64 ? sizeof(double2) : sizeof(float2)) * (size_t)p->nx * p->nz,
                                    cudaMemcpyDeviceToDevice, st));
      v = p->wsA;
    }
    return tv_prox_impl(p, v, tau, kTvDefaultIters, z, partial, st);
  }
  if (penalty == MBIR_PENALTY_L1) {
    const size_t n = (size_t)p->nx * p->nz;
    if (f64)
      { ProfScope ps_(p, PC_SOFT, st); launch(soft_kernel<double>, dim3(kSoftGrid), dim3(256), 0, st, (const double2*)v, (double2*)z, n, tau, partial); }
    else
      { ProfScope ps_(p, PC_SOFT, st); launch(soft_kernel<float>, dim3(kSoftGrid), dim3(256), 0, st, (const float2*)v, (float2*)z, n, (float)tau, partial); }
    MBIR_LAUNCH_CHECK();
    return MBIR_OK;
  }
  if (penalty != MBIR_PENALTY_DB4) return MBIR_ERR_INVALID;
  if (!wavelet_supported(p->nx, p->nz)) return MBIR_ERR_UNSUPPORTED_SIZE;
  int rc = ensure_wavelet_scratch(p);
  if (rc) return rc;
  if (f64) {
    rc = analysis_t<double>(p, v, p->wv_coef, true, tau, partial, st);
    if (rc) return rc;
    return synthesis_t<double>(p, p->wv_coef, z, st);
  }
  rc = analysis_t<float>(p, v, p->wv_coef, true, (float)tau, partial, st);
  if (rc) return rc;
  return synthesis_t<float>(p, p->wv_coef, z, st);
}

// ------------------------------------------------- allocation-free variant
//
// The wavelet transform without a plan, for callers that must not allocate
// device memory at all (see mbir_wavelet_static in mbir.h).  Its scratch -- the
// filter taps and the level-1 and level-2 low-low blocks -- lives in one
// file-scope device array that every GPU loading the library keeps until exit.

void daubechies8_taps(double h[8]);

constexpr size_t kStaticMaxPixels = size_t(1) << 21;          // nx * nz limit
constexpr size_t kStaticTapSlots = 32;                         // 256 bytes for the 8 taps
constexpr size_t kStaticElems = kStaticTapSlots + kStaticMaxPixels / 4 + kStaticMaxPixels / 16;
static __device__ __align__(256) float2 g_static_scratch[kStaticElems];

// The array's device address belongs to a CUDA context: it is looked up once per
// context (the primary context of each device, or a context the caller made
// current) and kept in this table.
typedef int (*CtxGetCurrentFn)(void** ctx);   // the driver's cuCtxGetCurrent
constexpr int kStaticMaxContexts = 64;
struct StaticSlot {
  void* ctx;
  float2* base;
};
static std::mutex g_static_mutex;
static StaticSlot g_static_slots[kStaticMaxContexts];
static int g_static_nslots = 0;
static CtxGetCurrentFn g_ctx_get_current = nullptr;

// The context current on this thread, or null when the runtime has made none yet.
static void* current_context() {
  if (!g_ctx_get_current) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  void* ctx = nullptr;
  return g_ctx_get_current(&ctx) == 0 ? ctx : nullptr;
}

// The db4 taps, passed by value to a one-CTA kernel that writes them into the
// array: no host-to-device copy is involved.
struct Taps8 {
  float h[8];
};

__global__ void static_taps_kernel(Taps8 t, float* dst) {
  if (threadIdx.x < 8) dst[threadIdx.x] = t.h[threadIdx.x];
}

// Once per context, with the caller's device current: the array's device address
// (its name in host code is only a host-side stand-in), the kernels' shared
// memory attributes and the taps.
static int static_scratch_setup(float2** base) {
  std::lock_guard<std::mutex> lock(g_static_mutex);
  void* ctx = current_context();
  for (int i = 0; ctx && i < g_static_nslots; ++i)
    if (g_static_slots[i].ctx == ctx) {
      *base = g_static_slots[i].base;
      return MBIR_OK;
    }
  // the lookup loads the library's module into the context if it is not yet (lazy
  // module loading), which is when the array is placed in device memory
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess) {
    const int rc = set_cuda_error(e, "cudaGetSymbolAddress(static wavelet scratch)");
    set_error_text(std::string("mbir_wavelet_static: the 5 MiB static scratch array could not be placed on the "
                               "device (the module loads at the first call; make it at start-up, before other "
                               "allocators take the memory): ") + cudaGetErrorString(e));
    return rc;
  }
  const int rc = configure_wavelet_t<float>();
  if (rc) return rc;
  // the taps, written once per context and waited for: the transform kernels read
  // them in their prologue, before they wait on the previous kernel of the stream
  Taps8 taps;
  {
    double h[8];
    daubechies8_taps(h);
    for (int i = 0; i < 8; ++i) taps.h[i] = (float)h[i];
  }
  static_taps_kernel<<<1, 32>>>(taps, static_cast<float*>(ptr));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_cuda_error(e, "static wavelet taps");
  if (!ctx) ctx = current_context();   // the lookup made the runtime's context current
  if (ctx) {
    if (g_static_nslots >= kStaticMaxContexts) {
      set_error_text("mbir_wavelet_static: more than 64 CUDA contexts used the static scratch");
      return MBIR_ERR_INVALID;
    }
    g_static_slots[g_static_nslots++] = {ctx, static_cast<float2*>(ptr)};
  }
  *base = static_cast<float2*>(ptr);
  return MBIR_OK;
}

int wavelet_static_impl(int nx, int nz, int inverse, const void* in, void* out, cudaStream_t st) {
  if (!in || !out || in == out || nx <= 0 || nz <= 0) return MBIR_ERR_INVALID;
  if (!wavelet_supported(nx, nz)) return MBIR_ERR_UNSUPPORTED_SIZE;
  if ((size_t)nx * (size_t)nz > kStaticMaxPixels) {
    set_error_text("mbir_wavelet_static: nx * nz exceeds the static scratch limit of 2^21 pixels");
    return MBIR_ERR_UNSUPPORTED_SIZE;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  float2* base = nullptr;
  int rc = static_scratch_setup(&base);
  if (rc) return rc;
  // a plan-shaped view onto the static scratch: no tables, no allocation
  mbir_plan_s view;
  memset(&view, 0, sizeof(view));
  view.nx = nx;
  view.nz = nz;
  view.precision = MBIR_FP32;
  view.device = dev;
  view.h_db4f = reinterpret_cast<float*>(base);
  view.wv_b1 = base + kStaticTapSlots;
  view.wv_b2 = base + kStaticTapSlots + (size_t)nx * nz / 4;
  return inverse ? synthesis_t<float>(&view, in, out, st)
                 : analysis_t<float>(&view, in, out, false, 0.0f, nullptr, st);
}

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_wavelet_static(int32_t nx, int32_t nz, int32_t inverse, const void* in, void* out, void* stream) {
  return wavelet_static_impl(nx, nz, inverse, in, out, (cudaStream_t)stream);
}

int mbir_prox(mbir_plan p, int32_t penalty, const void* v, double tau, void* z, void* stream) {
  if (const int vrc = bscan_only(p, "mbir_prox")) return vrc;
  if (!p || !v || !z || !(tau >= 0) || !isfinite(tau)) return MBIR_ERR_INVALID;
  if (penalty != MBIR_PENALTY_L1 && penalty != MBIR_PENALTY_DB4 && penalty != MBIR_PENALTY_TV) return MBIR_ERR_INVALID;
  return prox_partial_impl(p, penalty, v, tau, z, nullptr, (cudaStream_t)stream);
}

int mbir_wavelet(mbir_plan p, int32_t inverse, const void* in, void* out, void* stream) {
  if (const int vrc = bscan_only(p, "mbir_wavelet")) return vrc;
  if (!p || !in || !out || in == out) return MBIR_ERR_INVALID;
  return wavelet_impl(p, inverse, in, out, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------ batched launches

namespace mbir {

size_t dwt_args_bytes(int precision) {
  return precision == MBIR_FP64 ? sizeof(WArgs<double>) : sizeof(WArgs<float>);
}

int dwt_level_ctas(int P, int N, int inverse, int level) {
  return dwt_gx(N, inverse, level) * dwt_gy(P, inverse, level);
}

size_t dwt_smem_bytes(int precision, int inverse, int level) {
  const size_t vs = precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
  return inverse ? inv_smem(vs, level) : fwd_smem(vs, level);
}

// Argument block of analysis (inverse = 0) or synthesis level `level` (0 = finest)
// for plan p, laid out like the plan-path launches: analysis reads `in` at level
// 0 and the plan's low-low scratch above, synthesis writes `out` at level 0.
template <class R>
static void fill_dwt_t(mbir_plan p, int level, int inverse, const void* in, void* out, void* coef, double tau,
                       int thresh, double* partial, void* b1, void* b2, void* dst) {
  const int nx = p->nx, nz = p->nz;
  void* lls[3] = {b1, b2, coef};
  const int lstr[3] = {nz / 2, nz / 4, nz};
  WArgs<R> a;
  memset(&a, 0, sizeof(a));
  a.P = nx >> level;
  a.N = nz >> level;
  a.coef = coef;
  a.cstride = nz;
  a.h = p->precision == MBIR_FP64 ? reinterpret_cast<const R*>(p->h_db4) : reinterpret_cast<const R*>(p->h_db4f);
  a.tau = R(tau);
  a.partial = partial;
  if (!inverse) {
    a.in = level == 0 ? in : lls[level - 1];
    a.istride = level == 0 ? nz : lstr[level - 1];
    a.out = lls[level];
    a.ostride = lstr[level];
    a.thresh = thresh;
    a.gx = dwt_gx(a.N, 0, level);
  } else {
    a.in = lls[level];
    a.istride = lstr[level];
    a.out = level == 0 ? out : lls[level - 1];
    a.ostride = level == 0 ? nz : lstr[level - 1];
    a.thresh = 0;
    a.partial = nullptr;
    a.gx = dwt_gx(a.N, 1, level);
  }
  memcpy(dst, &a, sizeof(a));
}

void fill_dwt_args(mbir_plan p, int level, int inverse, const void* in, void* out, void* coef, double tau,
                   int thresh, double* partial, void* b1, void* b2, void* dst) {
  if (p->precision == MBIR_FP64) fill_dwt_t<double>(p, level, inverse, in, out, coef, tau, thresh, partial, b1, b2, dst);
  else fill_dwt_t<float>(p, level, inverse, in, out, coef, tau, thresh, partial, b1, b2, dst);
}

template <class R>
static void dwt_batch_t(int inverse, int level, const BatchLaunch& L, cudaStream_t st) {
  BatchRef<WArgs<R>> B;
  B.args = reinterpret_cast<const WArgs<R>*>(L.dargs);
  B.off = L.doff;
  B.n = L.n;
  B.set_mu = 0;
  B.mu = 0.0;
  WArgs<R> a0;
  memcpy(&a0, L.host0, sizeof(a0));
  const bool sm = dwt_small(level);
  const dim3 thr(sm ? wav_threads<true>() : wav_threads<false>());
  if (inverse) launch(sm ? dwt_inv_kernel<R, true> : dwt_inv_kernel<R, false>, dim3(L.total), thr, L.smem, st, a0, B);
  else launch(sm ? dwt_fwd_kernel<R, true> : dwt_fwd_kernel<R, false>, dim3(L.total), thr, L.smem, st, a0, B);
}

int batch_dwt(int inverse, int level, int precision, const BatchLaunch& L, cudaStream_t st) {
  if (L.total <= 0) return MBIR_OK;
  if (precision == MBIR_FP64) dwt_batch_t<double>(inverse, level, L, st);
  else dwt_batch_t<float>(inverse, level, L, st);
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

}  // namespace mbir
