// Launch-argument blocks and tuning constants of the operator kernels.
#pragma once

#include "common.cuh"

namespace mbir {

constexpr int kLatThreads = 256;    // lateral FFT block size
constexpr int kLatElems = 8192;     // nx * columns staged per lateral CTA
constexpr int kRowThreads = 512;    // row (NUFFT) block size

enum LatMode { LAT_C2C_FWD = 0, LAT_C2C_INV = 1, LAT_R2C_MASK = 2, LAT_C2R_INV_MASK = 3 };

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
