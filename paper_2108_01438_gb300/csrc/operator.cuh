// Launch-argument blocks and tuning constants of the operator kernels.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace mbir {

// Launch shapes (overridable at build time for tuning sweeps).
#ifndef MBIR_LAT_THREADS
#define MBIR_LAT_THREADS 512
#endif
#ifndef MBIR_LAT_ELEMS
#define MBIR_LAT_ELEMS 8192
#endif
#ifndef MBIR_ROW_THREADS
#define MBIR_ROW_THREADS 256
#endif
#ifndef MBIR_ROW_MINB
#define MBIR_ROW_MINB 4
#endif
#ifndef MBIR_GATHER_THREADS
#define MBIR_GATHER_THREADS 512
#endif
#ifndef MBIR_GATHER_MINB
#define MBIR_GATHER_MINB 2
#endif
#ifndef MBIR_GATHER_PRECOMP
#define MBIR_GATHER_PRECOMP 1
#endif
#ifndef MBIR_ADJ_ATOMIC
#define MBIR_ADJ_ATOMIC 0
#endif
#ifndef MBIR_LAT_MINB
#define MBIR_LAT_MINB 2
#endif
constexpr int kLatThreads = MBIR_LAT_THREADS;   // lateral FFT block size
// Batched lateral kernels read their scan's argument block from device memory
// and keep a register copy of its operands; at 512 threads and 64 registers they
// spilled 130-400 bytes a thread, so they run 256-thread CTAs with up to 128
// registers (two an SM, the same tiles).
#ifndef MBIR_LAT_THREADS_BATCH
#define MBIR_LAT_THREADS_BATCH 256
#endif
constexpr int kLatThreadsBatch = MBIR_LAT_THREADS_BATCH;
constexpr int kLatElems = MBIR_LAT_ELEMS;       // nx * columns staged per lateral CTA (max)
constexpr int kRowThreads = MBIR_ROW_THREADS;   // row (NUFFT) block size
constexpr int kRowMinBlocks = MBIR_ROW_MINB;    // resident CTAs per SM the register budget targets
constexpr int kLatMinBlocks = MBIR_LAT_MINB;
// the adjoint gather keeps per-pixel weights in shared memory (about 110 KB per row
// at K = 4096), so two CTAs fit an SM; wider CTAs keep more warps resident
constexpr int kGatherThreads = MBIR_GATHER_THREADS;
constexpr int kGatherMinBlocks = MBIR_GATHER_MINB;
// paired FP32 row kernels (two rows per CTA): the forward keeps a 16-byte-per-cell
// row pair (66 KB at K = 4096) in 512-thread CTAs, two an SM (a sweep of 256 x 3,
// 256 x 2 and 512 x 2 favoured the last); the gather's staging and row pair take
// about 160 KB, one CTA an SM, of 512 threads: a radix-8 pass of a 4096-point row
// has 512 butterflies, and with 1024 threads half of them waited at every pass
// barrier (51.99 vs 53.53 us at 1024 x 2048)
#ifndef MBIR_ROWPAIR_THREADS
#define MBIR_ROWPAIR_THREADS 512
#endif
#ifndef MBIR_ROWPAIR_MINB
#define MBIR_ROWPAIR_MINB 2
#endif
constexpr int kRowPairThreads = MBIR_ROWPAIR_THREADS;
constexpr int kRowPairMinBlocks = MBIR_ROWPAIR_MINB;
#ifndef MBIR_GATHERPAIR_THREADS
#define MBIR_GATHERPAIR_THREADS 512
#endif
#ifndef MBIR_LAT_UNROLL
#define MBIR_LAT_UNROLL 4
#endif
constexpr int kGatherPairThreads = MBIR_GATHERPAIR_THREADS;
// the lean paired gather (weights evaluated per term, no per-pixel cell array)
// fits two CTAs an SM at K = 4096
#ifndef MBIR_GATHERLEAN_THREADS
#define MBIR_GATHERLEAN_THREADS 512
#endif
#ifndef MBIR_GATHERLEAN_MINB
#define MBIR_GATHERLEAN_MINB 2
#endif
// FP32 plans form the filter in the row kernels from per-pixel and per-row
// constants (8-byte table entries) instead of reading it (16-byte entries)
#ifndef MBIR_FILTER_OTF
#define MBIR_FILTER_OTF 0
#endif
constexpr bool kFilterOtf = MBIR_FILTER_OTF != 0;
#ifndef MBIR_GATHERLEAN_DEFAULT
#define MBIR_GATHERLEAN_DEFAULT 0
#endif
constexpr int kGatherLeanThreads = MBIR_GATHERLEAN_THREADS;
constexpr int kGatherLeanMinBlocks = MBIR_GATHERLEAN_MINB;
constexpr bool kGatherLeanDefault = MBIR_GATHERLEAN_DEFAULT != 0;
constexpr int kLatUnroll = MBIR_LAT_UNROLL;   // rows of loads in flight per thread when staging a lateral tile
// FP32 lateral tiles run the transform's first pass on the way in from global
// memory and the middle passes' last pass on the way out
#ifndef MBIR_LAT_FUSE
#define MBIR_LAT_FUSE 1
#endif
constexpr bool kLatFuse = MBIR_LAT_FUSE != 0;
// FP32 paired row kernels: the forward runs its first transform pass on the way in
// from global memory; the gathers sum the cells of the first pass's butterflies in
// registers and run the last pass on the way out
#ifndef MBIR_ROW_FUSE
#define MBIR_ROW_FUSE 1
#endif
constexpr bool kRowFuse = MBIR_ROW_FUSE != 0;
// fused last lateral passes of radix <= this load their epilogue operands before
// the butterfly (more radix means more registers held across it)
#ifndef MBIR_EP_HOIST
#define MBIR_EP_HOIST 4
#endif
constexpr int kEpHoistMax = MBIR_EP_HOIST;
constexpr int kMaxDynSmem = 200 * 1024;   // dynamic shared memory cap (static use stays below the rest)
constexpr bool kGatherPrecomp = MBIR_GATHER_PRECOMP != 0;   // adjoint gather keeps per-pixel weights
constexpr bool kAdjAtomic = MBIR_ADJ_ATOMIC != 0;           // adjoint spreads with atomics

enum LatMode {
  LAT_C2C_FWD = 0,        // X = lateral FFT of x
  LAT_C2C_INV = 1,        // x = unnormalised inverse lateral FFT of W
  LAT_R2C_MASK = 2,       // R = (1/nx) lateral FFT of (s * y)
  LAT_C2R_INV_MASK = 3,   // y = s * Re{(1/nx) inverse lateral FFT of S}
  // FISTA epilogues (Eq. alg), fused into the last stage of Phi / Phi^H:
  LAT_SOLVE_FWD = 4,      // pz = Phi z^{k-1}; r = (1+mu) pz - mu pz_prev - s y; data term
  LAT_SOLVE_ADJ_L1 = 5,   // g = Phi^H r; z^k = soft(z1 + mu (z1 - z2) - delta g, tau); |z^k| sum
  LAT_SOLVE_ADJ_V = 6,    // g = Phi^H r; v = z1 + mu (z1 - z2) - delta g (wavelet prox follows)
  // measurement side of Phi^H Phi in one pass over the column tiles: the inverse
  // lateral FFT ending Phi, an epilogue in p-space, the lateral FFT starting Phi^H
  LAT_SOLVE_MID = 7,      // SOLVE_FWD's epilogue, then R = (1/nx) lateral FFT of r (r stays on chip)
  LAT_POWER_MID = 8,      // s Re{(1/nx) inverse lateral FFT of S}, then (1/nx) lateral FFT
  // power iteration (step-size bound) around Phi^H Phi
  LAT_POWER_FWD = 9,      // v = w / ||w|| (1/||w|| = scal[1]) written out, X = lateral FFT of v
  LAT_POWER_ADJ = 10      // w = inverse lateral FFT of W; partial sums of <v, w> and ||w||^2
};

template <class R>
struct LatArgs {
  const void* in;
  void* out;
  const uint8_t* mask;
  int nx, cols, tc;
  Radix rad;
  const void* tw;
  const int* perm;   // [nx] tile row of lateral output p (digit reversal, or the identity)
  int nxl;           // transform length (rad.n): nx, or the Bluestein length
  const void* chirp; // Bluestein: [nx] chirp e^{-j pi p^2/nx}, else null
  const void* bhat;  // Bluestein: [nxl] transformed conjugate chirp / nxl, digit-reversed
  R scale;
  // solver epilogue operands (LAT_SOLVE_*)
  const R* y;          // measurements [nx][m]
  R* pz;               // in: Phi z^{k-2}, out: Phi z^{k-1}   [nx][m]
  R* r;                // residual out [nx][m]
  const void* z1;      // z^{k-1} [nx][nz]
  void* z2;            // in: z^{k-2}; out: z^k (ADJ_L1) -- may be read before written
  void* vout;          // v out (ADJ_V)
  R mu, delta, tau;
  double* partial;     // one FP64 partial sum per CTA (two for LAT_POWER_ADJ)
  const double* scal;  // LAT_POWER_FWD: scal[1] = 1/||w||
};

template <class R>
struct RowArgs {
  const void* in;
  void* out;
  const void* tab;
  const void* cdep;
  const void* tw;
  const int* perm;   // digit reversal of the K-point transform
  const int4* rowmeta;   // per table row {base, span, direction, 0} of the unwrapped tap cells
  const int4* rowmap;    // volumes: per paired CTA {row a, row b or -1, table row, 0}; null for a B-scan
  Radix rad;
  int nx, nz, m, K, n0;
  int ny;                // volumes: rows are (lx, ly) = (r / ny, r % ny); 1 for a B-scan
  // FP32 pair kernels with the filter formed per (row, pixel) instead of read
  // from the table (the plan's otf): tab then points at TabP entries
  int otf;
  const TabP* tabp;
  const float4* fpix;
  const float* q2row;
  float dzf;
  double alpha, inv_i0a;
  float kbpoly[kMaxJ][kKbDeg + 1];   // FP32 KB weight of tap j: polynomial in (frac - 1/2)
};

double host_bessel_i0(double x);

}  // namespace mbir
