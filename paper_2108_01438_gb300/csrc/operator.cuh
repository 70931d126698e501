// Launch-argument blocks and tuning constants of the operator kernels.
#pragma once

#include "common.cuh"

namespace mbir {

constexpr int kLatThreads = 256;    // lateral FFT block size
constexpr int kLatElems = 8192;     // nx * columns staged per lateral CTA
constexpr int kRowThreads = 512;    // row (NUFFT) block size

enum LatMode {
  LAT_C2C_FWD = 0,        // X = lateral FFT of x
  LAT_C2C_INV = 1,        // x = unnormalised inverse lateral FFT of W
  LAT_R2C_MASK = 2,       // R = (1/nx) lateral FFT of (s * y)
  LAT_C2R_INV_MASK = 3,   // y = s * Re{(1/nx) inverse lateral FFT of S}
  // FISTA epilogues (Eq. alg), fused into the last stage of Phi / Phi^H:
  LAT_SOLVE_FWD = 4,      // pz = Phi z^{k-1}; r = (1+mu) pz - mu pz_prev - s y; data term
  LAT_SOLVE_ADJ_L1 = 5,   // g = Phi^H r; z^k = soft(z1 + mu (z1 - z2) - delta g, tau); |z^k| sum
  LAT_SOLVE_ADJ_V = 6     // g = Phi^H r; v = z1 + mu (z1 - z2) - delta g (wavelet prox follows)
};

template <class R>
struct LatArgs {
  const void* in;
  void* out;
  const uint8_t* mask;
  int nx, cols, tc;
  Radix rad;
  const void* tw;
  const int* perm;   // digit reversal of the nx-point transform
  R scale;
  // solver epilogue operands (LAT_SOLVE_*)
  const R* y;          // measurements [nx][m]
  R* pz;               // in: Phi z^{k-2}, out: Phi z^{k-1}   [nx][m]
  R* r;                // residual out [nx][m]
  const void* z1;      // z^{k-1} [nx][nz]
  void* z2;            // in: z^{k-2}; out: z^k (ADJ_L1) -- may be read before written
  void* vout;          // v out (ADJ_V)
  R mu, delta, tau;
  double* partial;     // one FP64 partial sum per CTA
};

template <class R>
struct RowArgs {
  const void* in;
  void* out;
  const void* tab;
  const void* cdep;
  const float* kbtab;
  const void* tw;
  const int* perm;   // digit reversal of the K-point transform
  Radix rad;
  int nx, nz, m, K, J, n0, nkb;
  double alpha, inv_i0a;
};

double host_bessel_i0(double x);

}  // namespace mbir
