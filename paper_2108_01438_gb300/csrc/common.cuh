// Internal helpers shared by the library's translation units: complex
// arithmetic on float2/double2, status plumbing and the plan layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "mbir.h"

namespace mbir {

// ------------------------------------------------------------------ complex

template <class R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };
template <class R> using cplx_t = typename Cplx<R>::T;

template <class V> __host__ __device__ __forceinline__ V cmk(decltype(V{}.x) a, decltype(V{}.x) b) {
  V v; v.x = a; v.y = b; return v;
}
template <class V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <class V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <class V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <class V> __device__ __forceinline__ V cmulc(V a, V b) {
  return cmk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <class V> __device__ __forceinline__ V cscale(V a, decltype(V{}.x) s) { return cmk<V>(a.x * s, a.y * s); }
template <class V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
// multiply by -j (forward) or +j (inverse)
template <bool INV, class V> __device__ __forceinline__ V mul_mj(V a) {
  return INV ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x);
}

// ------------------------------------------------------------------ plan

constexpr int kMaxPasses = 16;
constexpr int kKbRes = 1024;          // KB table samples per grid cell
constexpr int kMaxFFT = 8192;         // largest transform length (K = 2 nz)

struct Radix {
  int n;                  // transform length
  int npass;
  int r[kMaxPasses];      // radix of each pass, in decimation-in-frequency order
};

// One entry of the per-(|l~|, m) resampling table: integer grid cell of
// t = K/(2 pi) (beta dz mod 2 pi), its fractional part and the complex filter.
struct TabF { int i0; float frac; float fre, fim; };
struct TabD { int i0; int pad; double frac; double fre, fim; };

template <class R> struct TabOf;
template <> struct TabOf<float> { using T = TabF; };
template <> struct TabOf<double> { using T = TabD; };

struct SolveState;   // defined in solve.cu
struct BatchCache;

}  // namespace mbir

struct mbir_plan_s {
  int nx, nz, m, K, J, n0, nlh, precision;
  int device;
  double dx, dz, alpha;
  mbir::Radix rad_x, rad_k;
  int tile_c;                 // lateral FFT columns per CTA
  // device tables (one precision, per plan)
  void* tw_x;                 // nx twiddles e^{-2 pi j i / nx}
  void* tw_k;                 // K twiddles
  int* perm_x;                // digit reversal of the nx-point transform
  int* perm_k;                // digit reversal of the K-point transform
  void* cdep;                 // [nz] falloff / KB deapodisation
  void* tab;                  // [nlh][m] TabF or TabD
  float* kbtab;               // KB kernel samples (FP32 path)
  double* h_db4;              // 8 wavelet taps (device, double)
  float* h_db4f;              // same, float
  // workspace: two [nx][max(nz, m)] complex buffers
  void* wsA;
  void* wsB;
  size_t ws_elems;
  // wavelet scratch (lazily allocated): level-1/2 low-low blocks, coefficients
  void* wv_b1;
  void* wv_b2;
  void* wv_coef;
  // reductions: partial sums
  double* red;                // kRedSlots doubles
  mbir::SolveState* solve;    // lazily created
};

namespace mbir {

constexpr int kRedSlots = 4096;
constexpr int kSoftGrid = 1024;

int set_cuda_error(cudaError_t e, const char* where);
void set_error_text(const std::string& s);

#define MBIR_CUDA_TRY(call)                                         \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::mbir::set_cuda_error(e_, #call); \
  } while (0)

#define MBIR_LAUNCH_CHECK()                                                     \
  do {                                                                          \
    cudaError_t e_ = cudaGetLastError();                                        \
    if (e_ != cudaSuccess) return ::mbir::set_cuda_error(e_, "kernel launch");   \
  } while (0)

// operator.cu
int forward_impl(mbir_plan p, const void* x, const uint8_t* mask, void* y, cudaStream_t st);
int adjoint_impl(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st);
int configure_operator_kernels(mbir_plan p);
int forward_solve_impl(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, void* r,
                       double mu, double* partial, cudaStream_t st);
// vout == nullptr: l1 prox fused (z^k written over z2); else v written to vout
int adjoint_solve_impl(mbir_plan p, const void* r, const void* z1, void* z2, void* vout, double mu,
                       double delta, double tau, double* partial, cudaStream_t st);
int lateral_grid(mbir_plan p, int cols);

// wavelet.cu
int wavelet_impl(mbir_plan p, int inverse, const void* in, void* out, cudaStream_t st);
int prox_impl(mbir_plan p, int penalty, const void* v, double tau, void* z, cudaStream_t st);
bool wavelet_supported(int nx, int nz);
int configure_wavelet_kernels(mbir_plan p);

// solve.cu
void destroy_solve_state(mbir_plan p);

}  // namespace mbir
