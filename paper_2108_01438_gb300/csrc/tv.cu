// Isotropic total-variation penalty (Sec. 2.2) and its proximal map (the prox of
// Eq. alg with R = TV):
//
//   TV(x) = sum_ij sqrt(|x(i+1,j) - x(i,j)|^2 + |x(i,j+1) - x(i,j)|^2),
//
// differences that would leave the image taken as zero.  The prox
// argmin_x 1/2 ||x - v||^2 + tau TV(x) is x = v + tau div p for the dual field p
// (one complex number per direction and pixel, |p1|^2 + |p2|^2 <= 1) minimising
// 1/2 ||v + tau div p||^2, where div = -grad^T.  That smooth problem is solved by
// fast gradient projection from p = 0:
//
//   p_k     = project(r_k + grad(v + tau div r_k) / (8 tau))
//   r_{k+1} = p_k + m_k (p_k - p_{k-1}),   m_k = (t_k - 1)/t_{k+1}, FISTA's t,
//
// two steps per kernel over 8 x 64 pixel tiles (8 x 32 in FP64) with a two-pixel
// halo (tv_step2_kernel): step k runs on the tile plus a one-pixel ring so that
// step k + 1 can run on the tile.  p_k depends on r_k within one pixel, so the ring
// is recomputed by the neighbouring tiles instead of exchanged.  A pass reads
// p_{k-1}, p_{k-2} and v and writes p_k and p_{k+1}: 72 bytes a pixel (FP32) for
// two steps instead of 112 for two one-step passes.  An odd step count ends with
// one one-step pass (tv_step_kernel, one-pixel halo).  Four dual fields rotate.  A
// last kernel forms z = v + tau div p and the per-CTA sums of TV(z).
#include <math.h>

#include <vector>

#include "common.cuh"

namespace mbir {

// tile rows (lateral) x columns (depth): 16 x 64 in FP32, 16 x 32 in FP64 (the
// halo tiles of a step stay within 48 KB of static shared memory)
constexpr int kTvTI = 16;
template <class R>
constexpr int tv_tj() { return sizeof(R) == 4 ? 64 : 32; }
constexpr int kTvThreads = 256;

// dual pair at one pixel: p1 (lateral) and p2 (depth), complex each
template <class R>
struct Dual {
  cplx_t<R> p1, p2;
};

template <class R>
__device__ __forceinline__ Dual<R> dzero() {
  Dual<R> d;
  d.p1 = cmk<cplx_t<R>>(R(0), R(0));
  d.p2 = d.p1;
  return d;
}

// a pixel's dual pair moves as one 16-byte access in FP32 (two in FP64)
template <class R>
__device__ __forceinline__ Dual<R> dload(const void* base, size_t i) {
  Dual<R> d;
  if constexpr (sizeof(R) == 4) {
    const float4 t = reinterpret_cast<const float4*>(base)[i];
    d.p1 = make_float2(t.x, t.y);
    d.p2 = make_float2(t.z, t.w);
  } else {
    const cplx_t<R>* q = reinterpret_cast<const cplx_t<R>*>(base) + 2 * i;
    d.p1 = q[0];
    d.p2 = q[1];
  }
  return d;
}

template <class R>
__device__ __forceinline__ void dstore(void* base, size_t i, const Dual<R>& d) {
  if constexpr (sizeof(R) == 4) {
    reinterpret_cast<float4*>(base)[i] = make_float4(d.p1.x, d.p1.y, d.p2.x, d.p2.y);
  } else {
    cplx_t<R>* q = reinterpret_cast<cplx_t<R>*>(base) + 2 * i;
    q[0] = d.p1;
    q[1] = d.p2;
  }
}

__device__ __forceinline__ double tv_block_sum(double v) {
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
  return t;
}

// Load a dual field on the tile plus a one-pixel halo into shared memory:
// d[(ii + 1) * (TJ + 2) + jj + 1] for ii in [-1, TI], jj in [-1, TJ]; zero outside the
// image.  With pa: r = pa + m (pa - pb) (pb read only when m != 0); without: zero.
template <class R>
__device__ __forceinline__ void load_dual_halo(Dual<R>* d, const void* pa, const void* pb, R m, int i0, int j0,
                                               int P, int N) {
  constexpr int TJ = tv_tj<R>(), W = TJ + 2, H = kTvTI + 2;
  for (int e = threadIdx.x; e < W * H; e += blockDim.x) {
    const int ii = e / W - 1, jj = e - (e / W) * W - 1;
    const int gi = i0 + ii, gj = j0 + jj;
    Dual<R> r = dzero<R>();
    if (pa && gi >= 0 && gi < P && gj >= 0 && gj < N) {
      const size_t g = (size_t)gi * N + gj;
      r = dload<R>(pa, g);
      if (m != R(0)) {
        const Dual<R> b = dload<R>(pb, g);
        r.p1.x += m * (r.p1.x - b.p1.x);
        r.p1.y += m * (r.p1.y - b.p1.y);
        r.p2.x += m * (r.p2.x - b.p2.x);
        r.p2.y += m * (r.p2.y - b.p2.y);
      }
    }
    d[e] = r;
  }
}

// x = v + tau div r on tile rows [0, TI] and columns [0, TJ] (one beyond the tile
// for the forward differences); div r = r1(i) - r1(i-1) + r2(j) - r2(j-1) with the
// terms of p1 on the last row and p2 on the last column dropped (grad never fills
// them) and the terms outside the image zero.
template <class R>
__device__ __forceinline__ void form_x(cplx_t<R>* x, const Dual<R>* d, const cplx_t<R>* v, R tau, int i0, int j0,
                                       int P, int N) {
  using V = cplx_t<R>;
  constexpr int TJ = tv_tj<R>(), W = TJ + 2, XW = TJ + 1;
  for (int e = threadIdx.x; e < (kTvTI + 1) * XW; e += blockDim.x) {
    const int ii = e / XW, jj = e - (e / XW) * XW;
    const int gi = i0 + ii, gj = j0 + jj;
    V xv = cmk<V>(R(0), R(0));
    if (gi < P && gj < N) {
      const Dual<R>& c = d[(ii + 1) * W + jj + 1];
      const Dual<R>& up = d[ii * W + jj + 1];
      const Dual<R>& lf = d[(ii + 1) * W + jj];
      V dv = cmk<V>(R(0), R(0));
      if (gi < P - 1) dv = cadd(dv, c.p1);
      if (gi >= 1) dv = csub(dv, up.p1);
      if (gj < N - 1) dv = cadd(dv, c.p2);
      if (gj >= 1) dv = csub(dv, lf.p2);
      const V vv = v[(size_t)gi * N + gj];
      xv = cmk<V>(vv.x + tau * dv.x, vv.y + tau * dv.y);
    }
    x[e] = xv;
  }
}

// One FGP step: pout = project(r + grad(v + tau div r) / (8 tau)), r from pa, pb, m
// (pa = nullptr: r = 0, the first step).
template <class R>
__global__ void __launch_bounds__(kTvThreads)
tv_step_kernel(const void* v, const void* pa, const void* pb, R m, R tau, void* pout, int P, int N, int gx) {
  using V = cplx_t<R>;
  constexpr int TJ = tv_tj<R>();
  __shared__ Dual<R> d[(kTvTI + 2) * (TJ + 2)];
  __shared__ V x[(kTvTI + 1) * (TJ + 1)];
  const int bx = blockIdx.x % gx, by = blockIdx.x / gx;
  const int i0 = by * kTvTI, j0 = bx * TJ;
  pdl_wait_release();
  load_dual_halo<R>(d, pa, pb, m, i0, j0, P, N);
  __syncthreads();
  form_x<R>(x, d, reinterpret_cast<const V*>(v), tau, i0, j0, P, N);
  __syncthreads();
  constexpr int W = TJ + 2, XW = TJ + 1;
  const R step = R(1) / (R(8) * tau);
  for (int e = threadIdx.x; e < kTvTI * TJ; e += blockDim.x) {
    const int ii = e / TJ, jj = e - (e / TJ) * TJ;
    const int gi = i0 + ii, gj = j0 + jj;
    if (gi >= P || gj >= N) continue;
    const V xc = x[ii * XW + jj];
    const V g1 = gi < P - 1 ? csub(x[(ii + 1) * XW + jj], xc) : cmk<V>(R(0), R(0));
    const V g2 = gj < N - 1 ? csub(x[ii * XW + jj + 1], xc) : cmk<V>(R(0), R(0));
    Dual<R> q = d[(ii + 1) * W + jj + 1];
    q.p1 = cmk<V>(q.p1.x + step * g1.x, q.p1.y + step * g1.y);
    q.p2 = cmk<V>(q.p2.x + step * g2.x, q.p2.y + step * g2.y);
    const R n2 = q.p1.x * q.p1.x + q.p1.y * q.p1.y + q.p2.x * q.p2.x + q.p2.y * q.p2.y;
    if (n2 > R(1)) {
      const R s = R(1) / sqrt(n2);
      q.p1 = cscale(q.p1, s);
      q.p2 = cscale(q.p2, s);
    }
    dstore<R>(pout, (size_t)gi * N + gj, q);
  }
}

// Two FGP steps: p_k from r_k = pa + m1 (pa - pb) (pa = nullptr: r_k = 0; pb read
// only when m1 != 0), then r_{k+1} = p_k + m2 (p_k - pa) and p_{k+1}.  Shared
// memory (dynamic): r_k on the tile plus two pixels (rows and columns -2 .. T+1),
// p_{k-1} on the tile plus one (later r_{k+1}), and x on rows and columns -1 .. T+1.
// FP32 tile rows of the two-step pass (a build-time knob): 8 x 64 tiles take
// 30 KB of shared memory against 50 KB for 16 x 64, so more CTAs stay resident,
// and the prox took 0.533 ms against 0.580 ms at 1024 x 2048 (20 dual steps),
// although the two-pixel halo is a larger share of the tile
#ifndef MBIR_TV2_TI
#define MBIR_TV2_TI 8
#endif
template <class R>
constexpr int tv2_ti() { return sizeof(R) == 4 ? MBIR_TV2_TI : 8; }
template <class R>
constexpr int tv2_tj() { return sizeof(R) == 4 ? 64 : 32; }
template <class R>
constexpr size_t tv2_smem() {
  return sizeof(Dual<R>) * ((tv2_ti<R>() + 4) * (tv2_tj<R>() + 4) + (tv2_ti<R>() + 2) * (tv2_tj<R>() + 2)) +
         sizeof(cplx_t<R>) * (tv2_ti<R>() + 3) * (tv2_tj<R>() + 3);
}

template <class R>
__device__ __forceinline__ Dual<R> project_step(Dual<R> q, cplx_t<R> g1, cplx_t<R> g2, R step) {
  using V = cplx_t<R>;
  q.p1 = cmk<V>(q.p1.x + step * g1.x, q.p1.y + step * g1.y);
  q.p2 = cmk<V>(q.p2.x + step * g2.x, q.p2.y + step * g2.y);
  const R n2 = q.p1.x * q.p1.x + q.p1.y * q.p1.y + q.p2.x * q.p2.x + q.p2.y * q.p2.y;
  if (n2 > R(1)) {
    // 1/|q| by the library's reciprocal square root (a few ulp) rather than a
    // rounded square root and a division: the pass is bound by instruction issue
    const R s = rsqrt(n2);
    q.p1 = cscale(q.p1, s);
    q.p2 = cscale(q.p2, s);
  }
  return q;
}

template <class R>
__global__ void __launch_bounds__(kTvThreads)
tv_step2_kernel(const void* v, const void* pa, const void* pb, R m1, R m2, R tau, void* pout1, void* pout2, int P,
                int N, int gx) {
  using V = cplx_t<R>;
  constexpr int TI = tv2_ti<R>(), TJ = tv2_tj<R>();
  constexpr int W2 = TJ + 4, W1 = TJ + 2, XW = TJ + 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Dual<R>* d2 = reinterpret_cast<Dual<R>*>(smem_raw);      // r_k, rows/cols -2 .. T+1
  Dual<R>* d1 = d2 + (TI + 4) * W2;                         // p_{k-1}, then r_{k+1}, rows/cols -1 .. T
  V* x = reinterpret_cast<V*>(d1 + (TI + 2) * W1);          // x, rows/cols -1 .. T+1
  const int bx = blockIdx.x % gx, by = blockIdx.x / gx;
  const int i0 = by * TI, j0 = bx * TJ;
  const V* vv = reinterpret_cast<const V*>(v);
  const V zero = cmk<V>(R(0), R(0));
  const R step = R(1) / (R(8) * tau);
  pdl_wait_release();
  for (int e = threadIdx.x; e < (TI + 4) * W2; e += blockDim.x) {
    const int a = e / W2 - 2, b = e - (e / W2) * W2 - 2;
    const int gi = i0 + a, gj = j0 + b;
    Dual<R> pk1 = dzero<R>(), r = dzero<R>();
    if (pa && gi >= 0 && gi < P && gj >= 0 && gj < N) {
      const size_t g = (size_t)gi * N + gj;
      pk1 = dload<R>(pa, g);
      r = pk1;
      if (m1 != R(0)) {
        const Dual<R> q = dload<R>(pb, g);
        r.p1.x += m1 * (pk1.p1.x - q.p1.x);
        r.p1.y += m1 * (pk1.p1.y - q.p1.y);
        r.p2.x += m1 * (pk1.p2.x - q.p2.x);
        r.p2.y += m1 * (pk1.p2.y - q.p2.y);
      }
    }
    d2[e] = r;
    if (a >= -1 && a <= TI && b >= -1 && b <= TJ) d1[(a + 1) * W1 + b + 1] = pk1;
  }
  __syncthreads();
  // x_k = v + tau div r_k on rows and columns -1 .. T+1
  for (int e = threadIdx.x; e < (TI + 3) * XW; e += blockDim.x) {
    const int a = e / XW - 1, b = e - (e / XW) * XW - 1;
    const int gi = i0 + a, gj = j0 + b;
    V xv = zero;
    if (gi >= 0 && gi < P && gj >= 0 && gj < N) {
      const Dual<R>& c = d2[(a + 2) * W2 + b + 2];
      V dv = zero;
      if (gi < P - 1) dv = cadd(dv, c.p1);
      if (gi >= 1) dv = csub(dv, d2[(a + 1) * W2 + b + 2].p1);
      if (gj < N - 1) dv = cadd(dv, c.p2);
      if (gj >= 1) dv = csub(dv, d2[(a + 2) * W2 + b + 1].p2);
      const V v0 = vv[(size_t)gi * N + gj];
      xv = cmk<V>(v0.x + tau * dv.x, v0.y + tau * dv.y);
    }
    x[e] = xv;
  }
  __syncthreads();
  // p_k on the tile plus one (stored on the tile), r_{k+1} into d1
  for (int e = threadIdx.x; e < (TI + 2) * W1; e += blockDim.x) {
    const int a = e / W1 - 1, b = e - (e / W1) * W1 - 1;
    const int gi = i0 + a, gj = j0 + b;
    Dual<R> rn = dzero<R>();
    if (gi >= 0 && gi < P && gj >= 0 && gj < N) {
      const V xc = x[(a + 1) * XW + b + 1];
      const V g1 = gi < P - 1 ? csub(x[(a + 2) * XW + b + 1], xc) : zero;
      const V g2 = gj < N - 1 ? csub(x[(a + 1) * XW + b + 2], xc) : zero;
      const Dual<R> q = project_step<R>(d2[(a + 2) * W2 + b + 2], g1, g2, step);
      if (a >= 0 && a < TI && b >= 0 && b < TJ) dstore<R>(pout1, (size_t)gi * N + gj, q);
      const Dual<R> o = d1[e];
      rn.p1 = cmk<V>(q.p1.x + m2 * (q.p1.x - o.p1.x), q.p1.y + m2 * (q.p1.y - o.p1.y));
      rn.p2 = cmk<V>(q.p2.x + m2 * (q.p2.x - o.p2.x), q.p2.y + m2 * (q.p2.y - o.p2.y));
    }
    d1[e] = rn;
  }
  __syncthreads();
  // x_{k+1} = v + tau div r_{k+1} on rows and columns 0 .. T
  for (int e = threadIdx.x; e < (TI + 1) * (TJ + 1); e += blockDim.x) {
    const int a = e / (TJ + 1), b = e - (e / (TJ + 1)) * (TJ + 1);
    const int gi = i0 + a, gj = j0 + b;
    V xv = zero;
    if (gi < P && gj < N) {
      const Dual<R>& c = d1[(a + 1) * W1 + b + 1];
      V dv = zero;
      if (gi < P - 1) dv = cadd(dv, c.p1);
      if (gi >= 1) dv = csub(dv, d1[a * W1 + b + 1].p1);
      if (gj < N - 1) dv = cadd(dv, c.p2);
      if (gj >= 1) dv = csub(dv, d1[(a + 1) * W1 + b].p2);
      const V v0 = vv[(size_t)gi * N + gj];
      xv = cmk<V>(v0.x + tau * dv.x, v0.y + tau * dv.y);
    }
    x[(a + 1) * XW + b + 1] = xv;
  }
  __syncthreads();
  // p_{k+1} on the tile
  for (int e = threadIdx.x; e < TI * TJ; e += blockDim.x) {
    const int a = e / TJ, b = e - (e / TJ) * TJ;
    const int gi = i0 + a, gj = j0 + b;
    if (gi >= P || gj >= N) continue;
    const V xc = x[(a + 1) * XW + b + 1];
    const V g1 = gi < P - 1 ? csub(x[(a + 2) * XW + b + 1], xc) : zero;
    const V g2 = gj < N - 1 ? csub(x[(a + 1) * XW + b + 2], xc) : zero;
    dstore<R>(pout2, (size_t)gi * N + gj, project_step<R>(d1[(a + 1) * W1 + b + 1], g1, g2, step));
  }
}

// z = v + tau div p on the tile (p = nullptr: z = v), and the per-CTA sum of TV(z)
// (from z on the tile plus one row and column).
template <class R>
__global__ void __launch_bounds__(kTvThreads)
tv_finish_kernel(const void* v, const void* p, R tau, void* z, double* partial, int P, int N, int gx) {
  using V = cplx_t<R>;
  constexpr int TJ = tv_tj<R>();
  __shared__ Dual<R> d[(kTvTI + 2) * (TJ + 2)];
  __shared__ V x[(kTvTI + 1) * (TJ + 1)];
  const int bx = blockIdx.x % gx, by = blockIdx.x / gx;
  const int i0 = by * kTvTI, j0 = bx * TJ;
  pdl_wait_release();
  load_dual_halo<R>(d, p, nullptr, R(0), i0, j0, P, N);
  __syncthreads();
  form_x<R>(x, d, reinterpret_cast<const V*>(v), tau, i0, j0, P, N);
  __syncthreads();
  constexpr int XW = TJ + 1;
  R acc = R(0);   // a thread's few terms in the working precision, FP64 across the block
  V* zo = reinterpret_cast<V*>(z);
  for (int e = threadIdx.x; e < kTvTI * TJ; e += blockDim.x) {
    const int ii = e / TJ, jj = e - (e / TJ) * TJ;
    const int gi = i0 + ii, gj = j0 + jj;
    if (gi >= P || gj >= N) continue;
    const V xc = x[ii * XW + jj];
    zo[(size_t)gi * N + gj] = xc;
    const V g1 = gi < P - 1 ? csub(x[(ii + 1) * XW + jj], xc) : cmk<V>(R(0), R(0));
    const V g2 = gj < N - 1 ? csub(x[ii * XW + jj + 1], xc) : cmk<V>(R(0), R(0));
    acc += sqrt(g1.x * g1.x + g1.y * g1.y + g2.x * g2.x + g2.y * g2.y);
  }
  if (partial) {
    const double t = tv_block_sum(double(acc));
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// ------------------------------------------------------------------ host

static int tv_grid_x(mbir_plan p) {
  const int tj = p->precision == MBIR_FP64 ? tv_tj<double>() : tv_tj<float>();
  return (p->nz + tj - 1) / tj;
}
static int tv_grid_y(mbir_plan p) { return (p->nx + kTvTI - 1) / kTvTI; }

int tv_partial_count(mbir_plan p) { return tv_grid_x(p) * tv_grid_y(p); }

static int ensure_tv_scratch(mbir_plan p) {
  if (p->tv_p[0]) return MBIR_OK;
  const size_t bytes = (p->precision == MBIR_FP64 ? 4 * sizeof(double) : 4 * sizeof(float)) * (size_t)p->nx * p->nz;
  for (void*& q : p->tv_p) MBIR_CUDA_TRY(cudaMalloc(&q, bytes));
  if (p->precision == MBIR_FP64)
    MBIR_CUDA_TRY(cudaFuncSetAttribute(tv_step2_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tv2_smem<double>()));
  else
    MBIR_CUDA_TRY(cudaFuncSetAttribute(tv_step2_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tv2_smem<float>()));
  return MBIR_OK;
}

template <class R>
static int tv_prox_t(mbir_plan p, const void* v, double tau, int iters, void* z, double* partial, cudaStream_t st) {
  const int P = p->nx, N = p->nz, gx = tv_grid_x(p), grid = gx * tv_grid_y(p);
  if (!(tau > 0) || iters <= 0) {
    { ProfScope ps_(p, PC_TV, st); launch(tv_finish_kernel<R>, dim3(grid), dim3(kTvThreads), 0, st, v, (const void*)nullptr, R(0), z, partial, P, N, gx); }
    MBIR_LAUNCH_CHECK();
    return MBIR_OK;
  }
  int rc = ensure_tv_scratch(p);
  if (rc) return rc;
  // momenta m_j = (t_j - 1)/t_{j+1}, j = 1 .. iters (m_1 = 0)
  std::vector<double> mom(iters + 1, 0.0);
  {
    double t = 1.0;
    for (int j = 1; j <= iters; ++j) {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      mom[j] = (t - 1.0) / tn;
      t = tn;
    }
  }
  // p_j lives in buffer (j - 1) % 4: a pass never writes a field that it or a
  // neighbouring tile still reads
  auto buf = [&](int j) { return p->tv_p[(j - 1) & 3]; };
  constexpr int TI2 = tv2_ti<R>(), TJ2 = tv2_tj<R>();
  const int gx2 = (N + TJ2 - 1) / TJ2, grid2 = gx2 * ((P + TI2 - 1) / TI2);
  int k = 1;
  for (; k + 1 <= iters; k += 2) {   // steps k and k + 1
    const void* pa = k >= 2 ? buf(k - 1) : nullptr;
    const void* pb = k >= 3 ? buf(k - 2) : nullptr;
    const R m1 = k >= 3 ? R(mom[k - 1]) : R(0);
    {
      ProfScope ps_(p, PC_TV, st);
      launch(tv_step2_kernel<R>, dim3(grid2), dim3(kTvThreads), tv2_smem<R>(), st, v, pa, pb, m1, R(mom[k]),
             R(tau), buf(k), buf(k + 1), P, N, gx2);
    }
    MBIR_LAUNCH_CHECK();
  }
  if (k == iters) {   // an odd count ends with one one-step pass
    const void* pa = k >= 2 ? buf(k - 1) : nullptr;
    const void* pb = k >= 3 ? buf(k - 2) : nullptr;
    const R m = k >= 3 ? R(mom[k - 1]) : R(0);
    {
      ProfScope ps_(p, PC_TV, st);
      launch(tv_step_kernel<R>, dim3(grid), dim3(kTvThreads), 0, st, v, pa, pb, m, R(tau), buf(k), P, N, gx);
    }
    MBIR_LAUNCH_CHECK();
  }
  {
    ProfScope ps_(p, PC_TV, st);
    launch(tv_finish_kernel<R>, dim3(grid), dim3(kTvThreads), 0, st, v, (const void*)buf(iters), R(tau),
           z, partial, P, N, gx);
  }
  MBIR_LAUNCH_CHECK();
  return MBIR_OK;
}

int tv_prox_impl(mbir_plan p, const void* v, double tau, int iters, void* z, double* partial, cudaStream_t st) {
  return p->precision == MBIR_FP64 ? tv_prox_t<double>(p, v, tau, iters, z, partial, st)
                                   : tv_prox_t<float>(p, v, tau, iters, z, partial, st);
}

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_prox_tv(mbir_plan p, const void* v, double tau, int32_t iters, void* z, void* stream) {
  if (const int vrc = bscan_only(p, "mbir_prox_tv")) return vrc;
  if (!p || !v || !z || v == z || !(tau >= 0) || !isfinite(tau)) return MBIR_ERR_INVALID;
  return tv_prox_impl(p, v, tau, iters, z, nullptr, (cudaStream_t)stream);
}

}  // extern "C"
