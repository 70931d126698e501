// Shared-memory mixed-radix (2,3,4,5,7,8,16) in-place Cooley-Tukey FFT used by
// every transform of the operator: the lateral FFTs over A-scans (Eq. 4) and
// the oversampled axial FFT inside the NUFFT (Sec. 2.1).
//
// Data: `batch` interleaved sequences of length N in shared memory, element i of
// sequence b at s[sw(i) * batch + b], where sw is either the identity or, for
// batch = 1 and N divisible by 16, the XOR swizzle i ^ (((i >> 4) ^ (i >> 8)) & 15)
// (a permutation within each aligned group of 16).  It keeps the unit-stride
// last passes free of bank conflicts, and also the digit-reversed accesses
// (staging for dit, read-out after dif): for N = 4096 = 16^3, 16 consecutive
// indices land at positions 256 a + 16 b + c with a running and b, c fixed, and
// the (i >> 8) term spreads those over all 16 bank pairs.  With radices R_1..R_P:
//   decimation in frequency (dif): natural-order input; pass p works on blocks of
//     length L = N / (R_1 ... R_{p-1}): for j < M = L/R the R points
//     j + r M of a block go through an R-point DFT, output q is multiplied by
//     w_L^{q j}, and each point is written back where it was read.  The result
//     X[k] ends at position digit_reverse(k).
//   decimation in time (dit): the transpose, input x[k] placed at
//     digit_reverse(k), passes in reverse radix order, twiddles before the DFT,
//     natural-order output.
// Each butterfly owns its R slots, so threads run butterflies one at a time and
// only a barrier between passes is needed.  Twiddles w_N^e = e^{-2 pi j e / N}
// come from two small shared-memory tables, w_N^e = hi[e >> s] * lo[e & (2^s-1)];
// inverse transforms use the conjugate and are unnormalised.
#pragma once

#include "common.cuh"

namespace mbir {

// Position, after a dif transform with radices r[0..npass), of output index k:
// k = s_1 + s_2 R_1 + s_3 R_1 R_2 + ...  ->  pos = s_1 N/R_1 + s_2 N/(R_1 R_2) + ...
__host__ __device__ inline int digit_reverse(int k, const Radix& rad) {
  int L = rad.n, pos = 0;
  for (int p = 0; p < rad.npass; ++p) {
    const int R = rad.r[p];
    const int s = k % R;
    k /= R;
    L /= R;
    pos += s * L;
  }
  return pos;
}

template <class V>
struct Tw2 {
  const V* lo;   // w_N^i, i < 2^shift
  const V* hi;   // w_N^{i 2^shift}
  int shift, mask;
  __device__ __forceinline__ V operator()(int e) const { return cmul(hi[e >> shift], lo[e & mask]); }
};

__device__ __forceinline__ int swz(int i, bool on) { return on ? (i ^ (((i >> 4) ^ (i >> 8)) & 15)) : i; }

template <int R, bool INV, class V>
__device__ __forceinline__ void dft_small(V (&v)[R], const Tw2<V>& tw, int N) {
  using S = decltype(V{}.x);
  if constexpr (R == 2) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    V t2 = cadd(v[1], v[3]), t3 = mul_mj<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
  } else if constexpr (R == 8) {
    // radix-4 DFTs of the even and odd samples, combined with w_8^k
    V e0 = cadd(v[0], v[4]), e1 = csub(v[0], v[4]);
    V e2 = cadd(v[2], v[6]), e3 = mul_mj<INV>(csub(v[2], v[6]));
    V E0 = cadd(e0, e2), E2 = csub(e0, e2), E1 = cadd(e1, e3), E3 = csub(e1, e3);
    V o0 = cadd(v[1], v[5]), o1 = csub(v[1], v[5]);
    V o2 = cadd(v[3], v[7]), o3 = mul_mj<INV>(csub(v[3], v[7]));
    V O0 = cadd(o0, o2), O2 = csub(o0, o2), O1 = cadd(o1, o3), O3 = csub(o1, o3);
    const S h = S(0.70710678118654752440084436210485);
    // w_8^1 = (1 - j)/sqrt2 forward, (1 + j)/sqrt2 inverse; w_8^2 = -j / +j;
    // w_8^3 = (-1 - j)/sqrt2 forward, (-1 + j)/sqrt2 inverse
    V O1w = INV ? cmk<V>(h * (O1.x - O1.y), h * (O1.x + O1.y))
                : cmk<V>(h * (O1.x + O1.y), h * (O1.y - O1.x));
    V O2w = mul_mj<INV>(O2);
    V O3w = INV ? cmk<V>(-h * (O3.x + O3.y), h * (O3.x - O3.y))
                : cmk<V>(h * (O3.y - O3.x), -h * (O3.x + O3.y));
    v[0] = cadd(E0, O0);  v[4] = csub(E0, O0);
    v[1] = cadd(E1, O1w); v[5] = csub(E1, O1w);
    v[2] = cadd(E2, O2w); v[6] = csub(E2, O2w);
    v[3] = cadd(E3, O3w); v[7] = csub(E3, O3w);
  } else if constexpr (R == 16) {
    // 16 = 4 x 4: radix-4 DFTs over n1 of x[4 n1 + n2], twiddle w_16^{n2 k1},
    // radix-4 DFTs over n2; output k1 + 4 k2
    V y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      V a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
      dft_small<4, INV>(a, tw, N);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = a[k1];
    }
    const S c1 = S(0.92387953251128675612818318939679);   // cos(pi/8)
    const S s1 = S(0.38268343236508977172845998403040);   // sin(pi/8)
    const S h = S(0.70710678118654752440084436210485);
    // w_16^e for e = n2 k1 in {1, 2, 3, 4, 6, 9}; forward sign -, inverse +
    const S sg = INV ? S(1) : S(-1);
    auto rot = [&](V a, S c, S s) { return cmk<V>(a.x * c - a.y * s, a.x * s + a.y * c); };
    y[1][1] = rot(y[1][1], c1, sg * s1);                 // e = 1
    y[1][2] = rot(y[1][2], h, sg * h);                   // e = 2
    y[1][3] = rot(y[1][3], s1, sg * c1);                 // e = 3
    y[2][1] = rot(y[2][1], h, sg * h);                   // e = 2
    y[2][2] = mul_mj<INV>(y[2][2]);                      // e = 4
    y[2][3] = rot(y[2][3], -h, sg * h);                  // e = 6
    y[3][1] = rot(y[3][1], s1, sg * c1);                 // e = 3
    y[3][2] = rot(y[3][2], -h, sg * h);                  // e = 6
    y[3][3] = rot(y[3][3], -c1, -sg * s1);               // e = 9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      V a[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      dft_small<4, INV>(a, tw, N);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = a[k2];
    }
  } else {
    // direct R-point DFT, roots of unity from the N-point twiddles
    V out[R];
    const int stride = N / R;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      V acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = tw(((r * q) % R) * stride);
        if (INV) w = cconj(w);
        acc = cadd(acc, cmul(v[r], w));
      }
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = out[q];
  }
}

// v[q] *= w_N^{q e1} (conjugated for inverse transforms), q = 1 .. R-1.  For the
// power-of-two radices only w^{e1} (and w^{4 e1} for R = 16) come from the
// tables; the other powers are products of those, at most three multiplications
// deep, which costs one complex multiplication per twiddle instead of a two-table
// lookup and a multiplication.
template <int R, bool INV, class V>
__device__ __forceinline__ void apply_twiddles(V (&v)[R], const Tw2<V>& tw, int e1) {
  auto get = [&](int e) {
    const V w = tw(e);
    return INV ? cconj(w) : w;
  };
  if constexpr (R == 2) {
    v[1] = cmul(v[1], get(e1));
  } else if constexpr (R == 4 || R == 8 || R == 16) {
    const V w1 = get(e1);
    const V w2 = cmul(w1, w1);
    const V w3 = cmul(w2, w1);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    if constexpr (R >= 8) {
      const V w4 = R == 16 ? get(4 * e1) : cmul(w2, w2);
      v[4] = cmul(v[4], w4);
      v[5] = cmul(v[5], cmul(w4, w1));
      v[6] = cmul(v[6], cmul(w4, w2));
      v[7] = cmul(v[7], cmul(w4, w3));
      if constexpr (R == 16) {
        const V w8 = cmul(w4, w4);
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w8, w1));
        v[10] = cmul(v[10], cmul(w8, w2));
        v[11] = cmul(v[11], cmul(w8, w3));
        const V w12 = cmul(w8, w4);
        v[12] = cmul(v[12], w12);
        v[13] = cmul(v[13], cmul(w12, w1));
        v[14] = cmul(v[14], cmul(w12, w2));
        v[15] = cmul(v[15], cmul(w12, w3));
      }
    }
  } else {
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = cmul(v[q], get(q * e1));
  }
}

// x = a / d and a - x d, with a shift when d is a power of two (uniform branch).
__device__ __forceinline__ void divmod_u(int a, int d, int d_shift, int& q, int& r) {
  if (d_shift >= 0) {
    q = a >> d_shift;
    r = a & (d - 1);
  } else {
    q = a / d;
    r = a - q * d;
  }
}

__device__ __forceinline__ int log2_if_pow2(int d) {
  return (d & (d - 1)) == 0 ? __ffs(d) - 1 : -1;
}

template <int R, bool INV, bool DIT, class V>
__device__ __forceinline__ void ct_pass(V* s, int N, int batch, int bshift, int L, const Tw2<V>& tw,
                                        bool sw, int tid, int nthr) {
  const int M = L / R;
  const int mshift = log2_if_pow2(M);
  const int nb = batch * (N / R);
  const int tstep = N / L;
  for (int idx = tid; idx < nb; idx += nthr) {
    int t, b, blk, j;
    divmod_u(idx, batch, bshift, t, b);
    divmod_u(t, M, mshift, blk, j);
    const int base = blk * L + j;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[swz(base + r * M, sw) * batch + b];
    if (DIT && j != 0) apply_twiddles<R, INV>(v, tw, j * tstep);
    dft_small<R, INV>(v, tw, N);
    if (!DIT && j != 0) apply_twiddles<R, INV>(v, tw, j * tstep);
#pragma unroll
    for (int r = 0; r < R; ++r) s[swz(base + r * M, sw) * batch + b] = v[r];
  }
  __syncthreads();
}

template <bool INV, bool DIT, class V>
__device__ __forceinline__ void ct_dispatch(int R, V* s, int N, int batch, int bshift, int L,
                                            const Tw2<V>& tw, bool sw, int tid, int nthr) {
  switch (R) {
    case 16: ct_pass<16, INV, DIT>(s, N, batch, bshift, L, tw, sw, tid, nthr); break;
    case 8: ct_pass<8, INV, DIT>(s, N, batch, bshift, L, tw, sw, tid, nthr); break;
    case 4: ct_pass<4, INV, DIT>(s, N, batch, bshift, L, tw, sw, tid, nthr); break;
    case 2: ct_pass<2, INV, DIT>(s, N, batch, bshift, L, tw, sw, tid, nthr); break;
    case 3: ct_pass<3, INV, DIT>(s, N, batch, bshift, L, tw, sw, tid, nthr); break;
    case 5: ct_pass<5, INV, DIT>(s, N, batch, bshift, L, tw, sw, tid, nthr); break;
    case 7: ct_pass<7, INV, DIT>(s, N, batch, bshift, L, tw, sw, tid, nthr); break;
    default: break;
  }
}

// Decimation in frequency: natural order in, digit-reversed order out.
// Caller must __syncthreads() between filling s and this call.
template <bool INV, class V>
__device__ void fft_dif(V* s, int batch, const Radix& rad, const Tw2<V>& tw, bool sw) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bshift = log2_if_pow2(batch);
  int L = rad.n;
  for (int p = 0; p < rad.npass; ++p) {
    const int R = rad.r[p];
    ct_dispatch<INV, false>(R, s, rad.n, batch, bshift, L, tw, sw, tid, nthr);
    L /= R;
  }
}

// Decimation in time: digit-reversed order in, natural order out.
template <bool INV, class V>
__device__ void fft_dit(V* s, int batch, const Radix& rad, const Tw2<V>& tw, bool sw) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bshift = log2_if_pow2(batch);
  int L = 1;
  for (int p = rad.npass - 1; p >= 0; --p) {
    const int R = rad.r[p];
    L *= R;
    ct_dispatch<INV, true>(R, s, rad.n, batch, bshift, L, tw, sw, tid, nthr);
  }
}

// ------------------------------------------------------------------ paired
//
// Two complex sequences a, b that share every twiddle (two adjacent columns of a
// lateral tile) in split form: one float4 {re_a, re_b, im_a, im_b} per index.
// Every butterfly then runs on float2 lanes with the paired FP32 instructions of
// sm_100 and later (FADD2 / FMUL2 / FFMA2), so one instruction does the work
// of two scalar ones.  Twiddles are held broadcast ({c, c}, {s, s}) so that they
// multiply both lanes.  Same algorithms, orders and twiddle tables as above.

struct PC {
  float2 re, im;   // lanes: sequence a, sequence b
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ PC padd(PC a, PC b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ PC psub(PC a, PC b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }
// times -j (forward) or +j (inverse)
template <bool INV>
__device__ __forceinline__ PC pmul_mj(PC a) {
  return INV ? PC{neg2(a.im), a.re} : PC{a.im, neg2(a.re)};
}
// a times the broadcast twiddle w (also the product of two broadcast twiddles)
__device__ __forceinline__ PC pmulw(PC a, PC w) {
  return {fma2(a.re, w.re, mul2(neg2(a.im), w.im)), fma2(a.re, w.im, mul2(a.im, w.re))};
}
__device__ __forceinline__ PC pconj(PC w) { return {w.re, neg2(w.im)}; }

__device__ __forceinline__ PC ld_pc(const float4* s, int i) {
  const float4 t = s[i];
  return {make_float2(t.x, t.y), make_float2(t.z, t.w)};
}
__device__ __forceinline__ void st_pc(float4* s, int i, PC v) { s[i] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }

// Swizzle of single split-pair sequences (a row pair in shared memory, 16-byte
// elements): i ^ (((i >> 3) ^ (i >> 9)) & 7), a permutation within each aligned
// group of 8.  For K = 4096 with radix 8 every pass and the digit-reversed staging
// and read-out touch 8 distinct 16-byte bank groups per quarter warp (bank model
// of the access patterns).  The buffer is padded to a multiple of 8 elements.
__device__ __forceinline__ int swz8(int i) { return i ^ (((i >> 3) ^ (i >> 9)) & 7); }
template <bool SW>
__device__ __forceinline__ int psw(int i) { return SW ? swz8(i) : i; }

struct TwP {
  const float4* lo;   // broadcast w_N^i, i < 2^shift
  const float4* hi;   // broadcast w_N^{i 2^shift}
  int shift, mask;
  __device__ __forceinline__ PC operator()(int e) const {
    const float4 h = hi[e >> shift], l = lo[e & mask];
    return pmulw(PC{make_float2(h.x, h.y), make_float2(h.z, h.w)}, PC{make_float2(l.x, l.y), make_float2(l.z, l.w)});
  }
};

template <int R, bool INV>
__device__ __forceinline__ void dft_small_p(PC (&v)[R], const TwP& tw, int N) {
  if constexpr (R == 2) {
    const PC a = v[0], b = v[1];
    v[0] = padd(a, b);
    v[1] = psub(a, b);
  } else if constexpr (R == 4) {
    const PC t0 = padd(v[0], v[2]), t1 = psub(v[0], v[2]);
    const PC t2 = padd(v[1], v[3]), t3 = pmul_mj<INV>(psub(v[1], v[3]));
    v[0] = padd(t0, t2);
    v[2] = psub(t0, t2);
    v[1] = padd(t1, t3);
    v[3] = psub(t1, t3);
  } else if constexpr (R == 8) {
    const PC e0 = padd(v[0], v[4]), e1 = psub(v[0], v[4]);
    const PC e2 = padd(v[2], v[6]), e3 = pmul_mj<INV>(psub(v[2], v[6]));
    const PC E0 = padd(e0, e2), E2 = psub(e0, e2), E1 = padd(e1, e3), E3 = psub(e1, e3);
    const PC o0 = padd(v[1], v[5]), o1 = psub(v[1], v[5]);
    const PC o2 = padd(v[3], v[7]), o3 = pmul_mj<INV>(psub(v[3], v[7]));
    const PC O0 = padd(o0, o2), O2 = psub(o0, o2), O1 = padd(o1, o3), O3 = psub(o1, o3);
    const float2 h = make_float2(0.70710678118654752440f, 0.70710678118654752440f);
    // w_8^1, w_8^2 = -+j, w_8^3 as in the scalar transform
    const PC O1w = INV ? PC{mul2(h, sub2(O1.re, O1.im)), mul2(h, add2(O1.re, O1.im))}
                       : PC{mul2(h, add2(O1.re, O1.im)), mul2(h, sub2(O1.im, O1.re))};
    const PC O2w = pmul_mj<INV>(O2);
    const PC O3w = INV ? PC{neg2(mul2(h, add2(O3.re, O3.im))), mul2(h, sub2(O3.re, O3.im))}
                       : PC{mul2(h, sub2(O3.im, O3.re)), neg2(mul2(h, add2(O3.re, O3.im)))};
    v[0] = padd(E0, O0);
    v[4] = psub(E0, O0);
    v[1] = padd(E1, O1w);
    v[5] = psub(E1, O1w);
    v[2] = padd(E2, O2w);
    v[6] = psub(E2, O2w);
    v[3] = padd(E3, O3w);
    v[7] = psub(E3, O3w);
  }
}

// v[q] *= w_N^{q e1} (conjugated for inverse transforms), as apply_twiddles.
template <int R, bool INV>
__device__ __forceinline__ void apply_twiddles_p(PC (&v)[R], const TwP& tw, int e1) {
  auto get = [&](int e) {
    const PC w = tw(e);
    return INV ? pconj(w) : w;
  };
  if constexpr (R == 2) {
    v[1] = pmulw(v[1], get(e1));
  } else if constexpr (R == 4 || R == 8) {
    const PC w1 = get(e1);
    const PC w2 = pmulw(w1, w1);
    v[1] = pmulw(v[1], w1);
    v[2] = pmulw(v[2], w2);
    v[3] = pmulw(v[3], pmulw(w2, w1));
    if constexpr (R == 8) {
      const PC w4 = pmulw(w2, w2);
      v[4] = pmulw(v[4], w4);
      v[5] = pmulw(v[5], pmulw(w4, w1));
      v[6] = pmulw(v[6], pmulw(w4, w2));
      v[7] = pmulw(v[7], pmulw(pmulw(w4, w2), w1));
    }
  } else {
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = pmulw(v[q], get(q * e1));
  }
}

// One pass of an odd radix R (3, 5, 7) on split pairs.  With s_r = v_r + v_{R-r},
// d_r = v_r - v_{R-r} (r = 1 .. (R-1)/2) and w^{rq} = c + i sigma,
//   X_0 = v_0 + sum s_r,  X_q = A + i B,  X_{R-q} = A - i B,
//   A = v_0 + sum c s_r,  B = sum sigma d_r,
// so the sums and differences replace the inputs in place and each output pair
// is twiddled (dif) and stored as soon as it is formed: no second array of R
// values is held in registers.
template <int R, bool INV, bool DIT, bool SW>
__device__ __forceinline__ void ct_pass_p_odd(float4* s, int N, int batch, int bshift, int L, const TwP& tw,
                                              int tid, int nthr) {
  static_assert(R % 2 == 1, "odd radix");
  constexpr int H = (R - 1) / 2;
  const int M = L / R;
  const int mshift = log2_if_pow2(M);
  const int nb = batch * (N / R);
  const int tstep = N / L;
  const int stride = N / R;
  auto get = [&](int e) {
    const PC w = tw(e);
    return INV ? pconj(w) : w;
  };
  for (int idx = tid; idx < nb; idx += nthr) {
    int t, b, blk, j;
    divmod_u(idx, batch, bshift, t, b);
    divmod_u(t, M, mshift, blk, j);
    const int i0 = (blk * L + j) * batch + b, di = M * batch;
    const int e1 = j * tstep;
    PC v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld_pc(s, psw<SW>(i0 + r * di));
    if (DIT && j != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = pmulw(v[r], get(r * e1));
    }
    PC x0 = v[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const PC a = v[r], c = v[R - r];
      v[r] = padd(a, c);
      v[R - r] = psub(a, c);
      x0 = padd(x0, v[r]);
    }
    st_pc(s, psw<SW>(i0), x0);
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      PC A = v[0], B = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        const PC w = get(((r * q) % R) * stride);
        A.re = fma2(v[r].re, w.re, A.re);
        A.im = fma2(v[r].im, w.re, A.im);
        B.re = fma2(v[R - r].re, w.im, B.re);
        B.im = fma2(v[R - r].im, w.im, B.im);
      }
      PC xq = {sub2(A.re, B.im), add2(A.im, B.re)};        // A + i B
      PC xr = {add2(A.re, B.im), sub2(A.im, B.re)};        // A - i B
      if (!DIT && j != 0) {
        xq = pmulw(xq, get(q * e1));
        xr = pmulw(xr, get((R - q) * e1));
      }
      st_pc(s, psw<SW>(i0 + q * di), xq);
      st_pc(s, psw<SW>(i0 + (R - q) * di), xr);
    }
  }
  __syncthreads();
}

#ifndef MBIR_FFT_ILP
#define MBIR_FFT_ILP 1
#endif
// Butterflies a thread keeps in flight per pass of the paired transform: 2 loads
// both butterflies' inputs before computing either, so that the shared-memory
// latency of one overlaps the arithmetic of the other (twice the registers).
constexpr int kFftIlp = MBIR_FFT_ILP;

template <int R, bool INV, bool DIT, bool SW>
__device__ __forceinline__ void ct_pass_p(float4* s, int N, int batch, int bshift, int L, const TwP& tw, int tid,
                                          int nthr) {
  const int M = L / R;
  const int mshift = log2_if_pow2(M);
  const int nb = batch * (N / R);
  const int tstep = N / L;
  if constexpr (kFftIlp >= 2) {
    for (int idx = tid; idx < nb; idx += 2 * nthr) {
      const bool two = idx + nthr < nb;
      int ia[2], ja[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        int t, b, blk, j;
        divmod_u(q && two ? idx + nthr : idx, batch, bshift, t, b);
        divmod_u(t, M, mshift, blk, j);
        ia[q] = (blk * L + j) * batch + b;
        ja[q] = j;
      }
      const int di = M * batch;
      PC v[2][R];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = ld_pc(s, psw<SW>(ia[q] + r * di));
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (DIT && ja[q] != 0) apply_twiddles_p<R, INV>(v[q], tw, ja[q] * tstep);
        dft_small_p<R, INV>(v[q], tw, N);
        if (!DIT && ja[q] != 0) apply_twiddles_p<R, INV>(v[q], tw, ja[q] * tstep);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) st_pc(s, psw<SW>(ia[0] + r * di), v[0][r]);
      if (two) {
#pragma unroll
        for (int r = 0; r < R; ++r) st_pc(s, psw<SW>(ia[1] + r * di), v[1][r]);
      }
    }
  } else {
    for (int idx = tid; idx < nb; idx += nthr) {
      int t, b, blk, j;
      divmod_u(idx, batch, bshift, t, b);
      divmod_u(t, M, mshift, blk, j);
      const int i0 = (blk * L + j) * batch + b, di = M * batch;
      PC v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = ld_pc(s, psw<SW>(i0 + r * di));
      if (DIT && j != 0) apply_twiddles_p<R, INV>(v, tw, j * tstep);
      dft_small_p<R, INV>(v, tw, N);
      if (!DIT && j != 0) apply_twiddles_p<R, INV>(v, tw, j * tstep);
#pragma unroll
      for (int r = 0; r < R; ++r) st_pc(s, psw<SW>(i0 + r * di), v[r]);
    }
  }
  __syncthreads();
}

// Radices up to 8 (a radix-16 butterfly of split pairs would hold 64 registers).
template <bool INV, bool DIT, bool SW>
__device__ __forceinline__ void ct_dispatch_p(int R, float4* s, int N, int batch, int bshift, int L, const TwP& tw,
                                              int tid, int nthr) {
  switch (R) {
    case 8: ct_pass_p<8, INV, DIT, SW>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 4: ct_pass_p<4, INV, DIT, SW>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 2: ct_pass_p<2, INV, DIT, SW>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 3: ct_pass_p_odd<3, INV, DIT, SW>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 5: ct_pass_p_odd<5, INV, DIT, SW>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 7: ct_pass_p_odd<7, INV, DIT, SW>(s, N, batch, bshift, L, tw, tid, nthr); break;
    default: break;
  }
}

// `batch` interleaved pair-sequences, element i of pair-sequence b at
// s[psw<SW>(i * batch + b)] (SW only with batch = 1).
// Passes [first, end) (end < 0: to the last): a caller that runs pass 0 on its
// way in from global memory starts at 1, one that runs the last pass on its way
// out ends before it.
template <bool INV, bool SW = false>
__device__ void fft_p_dif(float4* s, int batch, const Radix& rad, const TwP& tw, int first = 0, int end = -1) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bshift = log2_if_pow2(batch);
  if (end < 0) end = rad.npass;
  int L = rad.n;
  for (int p = 0; p < first; ++p) L /= rad.r[p];
  for (int p = first; p < end; ++p) {
    const int R = rad.r[p];
    ct_dispatch_p<INV, false, SW>(R, s, rad.n, batch, bshift, L, tw, tid, nthr);
    L /= R;
  }
}

// Passes top, top - 1, ..., last (top < 0: from the first dit pass, npass - 1): a
// caller that runs pass 0 on its way out to global memory stops at 1, one that
// ran pass npass - 1 itself starts at npass - 2.
template <bool INV, bool SW = false>
__device__ void fft_p_dit(float4* s, int batch, const Radix& rad, const TwP& tw, int last = 0, int top = -1) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bshift = log2_if_pow2(batch);
  if (top < 0) top = rad.npass - 1;
  int L = 1;
  for (int p = rad.npass - 1; p > top; --p) L *= rad.r[p];
  for (int p = top; p >= last; --p) {
    const int R = rad.r[p];
    L *= R;
    ct_dispatch_p<INV, true, SW>(R, s, rad.n, batch, bshift, L, tw, tid, nthr);
  }
}

// Twiddle tables of a transform (global [lo | hi], float2) into shared memory in
// broadcast form.  No barrier inside.
__device__ __forceinline__ TwP load_twiddles_p(float4* smem, const float2* __restrict__ g, const Radix& rad) {
  const int n = rad.tw_lo + rad.tw_hi;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 w = g[i];
    smem[i] = make_float4(w.x, w.x, w.y, w.y);
  }
  TwP t;
  t.lo = smem;
  t.hi = smem + rad.tw_lo;
  t.shift = rad.tw_shift;
  t.mask = rad.tw_lo - 1;
  return t;
}

// Copy the two twiddle tables of a transform (tw2 = [lo | hi] in global memory)
// into shared memory and return the accessor.  No barrier inside.
template <class V>
__device__ __forceinline__ Tw2<V> load_twiddles(V* smem, const V* __restrict__ g, const Radix& rad) {
  const int n = rad.tw_lo + rad.tw_hi;
  for (int i = threadIdx.x; i < n; i += blockDim.x) smem[i] = g[i];
  Tw2<V> t;
  t.lo = smem;
  t.hi = smem + rad.tw_lo;
  t.shift = rad.tw_shift;
  t.mask = rad.tw_lo - 1;
  return t;
}

}  // namespace mbir
