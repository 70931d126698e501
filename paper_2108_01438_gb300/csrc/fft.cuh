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
