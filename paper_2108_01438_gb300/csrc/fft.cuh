// Shared-memory mixed-radix (2,3,4,5,7,8) in-place Cooley-Tukey FFT used by
// every transform of the operator: the lateral FFTs over A-scans (Eq. 4) and
// the oversampled axial FFT inside the NUFFT (Sec. 2.1).
//
// Data: `batch` interleaved sequences of length N in shared memory, element i of
// sequence b at s[i * batch + b].  With the radices R_1..R_P of the plan:
//   decimation in frequency (dif): natural-order input; pass p works on blocks of
//     length L = N / (R_1 ... R_{p-1}): for j < M = L/R the R points
//     j + r M of a block go through an R-point DFT, output q is multiplied by
//     w_L^{q j}, and each point is written back where it was read.  The result
//     X[k] ends at position digit_reverse(k) (see digit_reverse below).
//   decimation in time (dit): the transpose, input x[k] placed at
//     digit_reverse(k), passes in reverse radix order, twiddles before the DFT,
//     natural-order output.
// Each butterfly owns its R slots, so threads run butterflies one at a time and
// only a barrier between passes is needed.  The twiddle table holds
// w_N^i = e^{-2 pi j i / N}; inverse transforms use its conjugate, unnormalised.
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

template <int R, bool INV, class V>
__device__ __forceinline__ void dft_small(V (&v)[R], const V* __restrict__ tw, int N) {
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
  } else {
    // direct R-point DFT, roots of unity taken from the N-point table
    V out[R];
    const int stride = N / R;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      V acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = tw[((r * q) % R) * stride];
        if (INV) w = cconj(w);
        acc = cadd(acc, cmul(v[r], w));
      }
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = out[q];
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
__device__ __forceinline__ void ct_pass(V* s, int N, int batch, int bshift, int L,
                                        const V* __restrict__ tw, int tid, int nthr) {
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
    for (int r = 0; r < R; ++r) v[r] = s[(base + r * M) * batch + b];
    if (DIT && j != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = tw[r * j * tstep];
        if (INV) w = cconj(w);
        v[r] = cmul(v[r], w);
      }
    }
    dft_small<R, INV>(v, tw, N);
    if (!DIT && j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        V w = tw[q * j * tstep];
        if (INV) w = cconj(w);
        v[q] = cmul(v[q], w);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) s[(base + r * M) * batch + b] = v[r];
  }
  __syncthreads();
}

template <bool INV, bool DIT, class V>
__device__ __forceinline__ void ct_dispatch(int R, V* s, int N, int batch, int bshift, int L,
                                            const V* __restrict__ tw, int tid, int nthr) {
  switch (R) {
    case 8: ct_pass<8, INV, DIT>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 4: ct_pass<4, INV, DIT>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 2: ct_pass<2, INV, DIT>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 3: ct_pass<3, INV, DIT>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 5: ct_pass<5, INV, DIT>(s, N, batch, bshift, L, tw, tid, nthr); break;
    case 7: ct_pass<7, INV, DIT>(s, N, batch, bshift, L, tw, tid, nthr); break;
    default: break;
  }
}

// Decimation in frequency: natural order in, digit-reversed order out.
// Caller must __syncthreads() between filling s and this call.
template <bool INV, class V>
__device__ void fft_dif(V* s, int batch, const Radix& rad, const V* __restrict__ tw) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bshift = log2_if_pow2(batch);
  int L = rad.n;
  for (int p = 0; p < rad.npass; ++p) {
    const int R = rad.r[p];
    ct_dispatch<INV, false>(R, s, rad.n, batch, bshift, L, tw, tid, nthr);
    L /= R;
  }
}

// Decimation in time: digit-reversed order in, natural order out.
template <bool INV, class V>
__device__ void fft_dit(V* s, int batch, const Radix& rad, const V* __restrict__ tw) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bshift = log2_if_pow2(batch);
  int L = 1;
  for (int p = rad.npass - 1; p >= 0; --p) {
    const int R = rad.r[p];
    L *= R;
    ct_dispatch<INV, true>(R, s, rad.n, batch, bshift, L, tw, tid, nthr);
  }
}

}  // namespace mbir
