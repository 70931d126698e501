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
constexpr int kMaxFFT = 8192;         // largest transform length (K = 2 nz)
constexpr int kMaxJ = 8;              // largest KB width
constexpr int kKbDeg = 9;             // degree of the per-tap KB weight polynomials

struct Radix {
  int n;                  // transform length
  int npass;
  int r[kMaxPasses];      // radix of each pass, in decimation-in-frequency order
  int lg[kMaxPasses];     // log2 of each radix when pow2
  int pow2;               // every radix a power of two
  int log2n;
  int tw_shift;           // twiddles: w^e = hi[e >> tw_shift] * lo[e & (tw_lo - 1)]
  int tw_lo, tw_hi;       // table lengths
};

// One entry of the per-(|l~|, m) resampling table for t = K/(2 pi) (beta dz mod 2 pi):
// cell = (u << 16) | pc, pc = floor(t) - J/2 + 1 (mod K) the first tap's grid cell
// and u its unwrapped offset within the row (see the plan), the fractional part
// of t and the complex filter.
struct TabF { int cell; float frac; float fre, fim; };
// The same grid position without the filter (FP32 plans whose row kernels form
// the filter from per-pixel and per-row constants, see RowArgs::otf).
struct TabP { int cell; float frac; };
struct TabD { int cell; int pad; double frac; double fre, fim; };

template <class R> struct TabOf;
template <> struct TabOf<float> { using T = TabF; };
template <> struct TabOf<double> { using T = TabD; };

struct SolveState;   // defined in solve.cu

// Batched launches: one grid covers several B-scans.  args[s] is scan s's
// argument block (device memory) and off[s] .. off[s+1]-1 its CTAs; a null args
// means a single scan whose block is passed by value.  mu (when set_mu) replaces
// the momentum of every block, the one value that changes per FISTA iteration.
template <class Args>
struct BatchRef {
  const Args* args;
  const int* off;
  int n;
  int set_mu;
  double mu;
};

template <class Args>
inline BatchRef<Args> no_batch() {
  BatchRef<Args> b;
  b.args = nullptr;
  b.off = nullptr;
  b.n = 0;
  b.set_mu = 0;
  b.mu = 0.0;
  return b;
}

// Kernel classes for the event profiler (mbir_profile_begin / _end).
enum ProfClass {
  PC_LAT_FWD = 0,     // lateral FFT of the image (first stage of Phi)
  PC_ROW_FWD,         // row NUFFT forward
  PC_LAT_INV,         // inverse lateral FFT + real part (+ FISTA measurement epilogue)
  PC_LAT_R2C,         // lateral FFT of the masked residual (first stage of Phi^H)
  PC_ROW_ADJ,         // row NUFFT adjoint
  PC_LAT_ADJ,         // inverse lateral FFT of the adjoint (+ FISTA image epilogue)
  PC_DWT_FWD,         // wavelet analysis level (+ soft-threshold)
  PC_DWT_INV,         // wavelet synthesis level
  PC_SOFT,            // elementwise soft-threshold
  PC_REDUCE,          // reductions, scalars, power-iteration helpers
  PC_LAT_MID,         // inverse lateral FFT + measurement epilogue + lateral FFT (Phi^H Phi middle)
  PC_TV,              // TV prox: dual projected-gradient steps and the finishing pass
  PC_HILBERT,         // conjugate analytic signal along the spectrometer axis
  PC_COUNT
};

struct Profiler {
  int cap = 0, n = 0;
  cudaEvent_t* ev = nullptr;   // 2 * cap
  int* cls = nullptr;          // cap
  unsigned mask = ~0u;         // kernel classes that record (bit per ProfClass)
};

const char* prof_class_name(int c);
struct BatchCache;

}  // namespace mbir

struct mbir_plan_s {
  int nx, nz, m, K, J, n0, nlh, precision;
  // volumes (mbir_volume_plan_create): a second lateral axis of ny pixels; ny = 1
  // for a B-scan.  The resampling table has ntab rows, one per (|lx|, |ly|); the
  // paired row kernels run npair CTAs, CTA c on rows rowmap[c].x and rowmap[c].y
  // (-1: none) with table row rowmap[c].z (rowmap null for a B-scan: CTA l' runs
  // rows l' and nx - l' with table row l')
  int ny, ntab, npair;
  double dy;
  int4* rowmap;
  mbir::Radix rad_y;          // the y-axis transform, of length nyl
  int nyl, tile_y;
  void* tw_y;
  int* perm_y;
  void* chirp_y;
  void* bhat_y;
  int device;
  double dx, dz, alpha;
  mbir::Radix rad_x, rad_k;   // rad_x: the lateral transform, of length nxl
  int nxl;                    // lateral transform length: nx, or the Bluestein length when nx is not 7-smooth
  void* chirp;                // Bluestein: [nx] e^{-j pi p^2 / nx} (plan precision complex), else null
  void* bhat;                 // Bluestein: [nxl] DFT of the conjugate chirp / nxl, digit-reversed
  int tile_c;                 // lateral FFT columns per CTA
  int lat_order;              // lateral radix order: 0 largest radix first, 1 smallest first
  int adj_kind;               // row adjoint kernel override (RowKind), -1: automatic
  int k_ascending;            // wavenumbers increase with the spectrometer pixel index
  // device tables (one precision, per plan)
  void* tw_x;                 // nxl-point twiddle tables [lo | hi]
  void* tw_k;                 // K-point twiddle tables [lo | hi]
  int* perm_x;                // [nx] tile row of lateral output p: digit reversal of the nx-point
                              // transform, the identity for Bluestein (natural-order output)
  int* perm_k;                // digit reversal of the K-point transform
  void* cdep;                 // [nz] falloff / KB deapodisation
  void* tab;                  // [ntab][m] TabF or TabD
  // FP32 plans, filter formed in the row kernels (otf != 0): the grid positions
  // [ntab][m] TabP, per pixel {Re, Im of A e^{j(Omega - 2k z_f + 2k (z_f - z_c))},
  // 1/(2 k^2 NA^2), 2k} and per table row q^2; z_f - z_c
  int otf;
  mbir::TabP* tabp;
  float4* fpix;
  float* q2row;
  float dzf;
  int4* rowmeta;              // [ntab] {base cell of u = 0, span of u + J, direction, 0}
  int gather_ok;              // every row monotone with span <= K: deterministic adjoint gather
  int max_span;               // largest row span (rowmeta .y) of the plan
  float kbpoly[mbir::kMaxJ][mbir::kKbDeg + 1];   // FP32 KB weight polynomials per tap
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
  // TV prox scratch (lazily allocated): four dual fields [nx][nz] x 4 reals
  void* tv_p[4];
  // m-point transform of the Hilbert-form back-projection (built on first use)
  mbir::Radix rad_m;
  void* tw_m;
  int* perm_m;
  double* ncc_scratch;        // NCC partial sums and scalars (lazily allocated)
  // reductions: partial sums
  double* red;                // kRedSlots doubles
  mbir::SolveState* solve;    // lazily created
  mbir::Profiler* prof;       // non-null while profiling
};

namespace mbir {

constexpr int kRedSlots = 4096;
constexpr int kSoftGrid = 1024;

int set_cuda_error(cudaError_t e, const char* where);
void set_error_text(const std::string& s);

// Volume plans (ny > 1) run the operator only: the B-scan calls refuse them.
inline int bscan_only(mbir_plan p, const char* call) {
  if (p && p->ny > 1) {
    set_error_text(std::string(call) + ": a volume plan takes mbir_forward and mbir_adjoint only");
    return MBIR_ERR_UNSUPPORTED_SIZE;
  }
  return MBIR_OK;
}

#define MBIR_CUDA_TRY(call)                                         \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::mbir::set_cuda_error(e_, #call); \
  } while (0)

// Programmatic dependent launch: every kernel of the path is launched with
// programmatic stream serialisation, so its CTAs can be scheduled while the
// previous kernel drains and run their prologue (plan constants, twiddles into
// shared memory); each calls pdl_wait_release() before it touches any data that
// an earlier kernel writes, which waits for the previous grid to complete and
// flush, then lets the next kernel be scheduled.  Without the attribute the
// instructions are no-ops.
#ifndef MBIR_PDL
#define MBIR_PDL 1
#endif
constexpr bool kPdl = MBIR_PDL != 0;

__device__ __forceinline__ void pdl_wait_release() {
  asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory");
}

// Before its dependency wait a kernel may pull into L2 the operands that no
// kernel still in flight writes (measurements, masks, tables, iterates of earlier
// iterations): its CTAs that start while the previous grid drains then find them
// there.  A prefetch is a hint: it returns no data, leaves L1 alone and cannot
// expose a stale value, since L2 is the point of coherence.
#ifndef MBIR_L2_PREFETCH
#define MBIR_L2_PREFETCH 1
#endif
constexpr bool kL2Prefetch = MBIR_L2_PREFETCH != 0;

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// The 128-byte lines of bytes [0, len) from base, spread over the CTA's threads.
__device__ __forceinline__ void prefetch_l2_range(const void* base, size_t len) {
  if (!kL2Prefetch || base == nullptr) return;
  const uintptr_t s = reinterpret_cast<uintptr_t>(base) & ~uintptr_t(127);
  const uintptr_t e = reinterpret_cast<uintptr_t>(base) + len;
  for (uintptr_t l = s + 128 * (uintptr_t)threadIdx.x; l < e; l += 128 * (uintptr_t)blockDim.x)
    prefetch_l2(reinterpret_cast<const void*>(l));
}

// The 128-byte lines of rows [0, rows) of a row-major array (row pitch `pitch`
// bytes), bytes [off, off + len) of each row; the CTA's threads share the rows.
__device__ __forceinline__ void prefetch_l2_rows(const void* base, int rows, size_t pitch, size_t off, int len) {
  if (!kL2Prefetch || base == nullptr || len <= 0) return;
  const char* b = static_cast<const char*>(base) + off;
  for (int p = threadIdx.x; p < rows; p += blockDim.x) {
    const uintptr_t s = reinterpret_cast<uintptr_t>(b + (size_t)p * pitch);
    for (uintptr_t l = s & ~uintptr_t(127); l < s + len; l += 128) prefetch_l2(reinterpret_cast<const void*>(l));
  }
}

template <class... KArgs, class... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   const Args&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = kPdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kernel, args...) == cudaErrorNotSupported && kPdl) {
    // a stream that does not take the attribute: plain stream order
    (void)cudaGetLastError();
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
  }
}

#define MBIR_LAUNCH_CHECK()                                                     \
  do {                                                                          \
    cudaError_t e_ = cudaGetLastError();                                        \
    if (e_ != cudaSuccess) return ::mbir::set_cuda_error(e_, "kernel launch");   \
  } while (0)

// Event profiler: prof_begin returns a slot (or -1 when not recording).
inline int prof_begin(mbir_plan p, int cls, cudaStream_t st) {
  Profiler* pr = p->prof;
  if (!pr || pr->n >= pr->cap || !((pr->mask >> cls) & 1u)) return -1;
  const int i = pr->n++;
  pr->cls[i] = cls;
  cudaEventRecord(pr->ev[2 * i], st);
  return i;
}
inline void prof_end(mbir_plan p, int slot, cudaStream_t st) {
  if (slot >= 0) cudaEventRecord(p->prof->ev[2 * slot + 1], st);
}
struct ProfScope {
  mbir_plan p;
  cudaStream_t st;
  int slot;
  ProfScope(mbir_plan p_, int cls, cudaStream_t st_) : p(p_), st(st_), slot(prof_begin(p_, cls, st_)) {}
  ~ProfScope() { prof_end(p, slot, st); }
};
void destroy_profiler(mbir_plan p);

// Batched launch descriptor: device array of per-scan argument blocks, CTA
// prefix offsets (n + 1 entries), total CTAs, dynamic shared memory (the
// maximum over the scans), the by-value block (uniform fields) and the momentum.
struct BatchLaunch {
  const void* dargs;
  const int* doff;
  int n, total;
  size_t smem;
  const void* host0;
  int set_mu;
  double mu;
  int blu;   // a scan of the launch runs its lateral transform in the Bluestein form
  int fz;    // row launches: every scan's K-point transform takes the fused first and last passes
};

// Operands of one lateral stage for one scan (batch.cu fills these).
struct LatFill {
  const void* in;
  void* out;
  const uint8_t* mask;
  int cols;
  double scale;
  const void* y;
  void* pz;
  void* r;
  const void* z1;
  void* z2;
  void* vout;
  double mu, delta, tau;
  double* partial;
  const double* scal;
};

// operator.cu (batch helpers)
size_t lat_args_bytes(int precision);
size_t row_args_bytes(int precision);
size_t lat_smem_bytes(mbir_plan p);
size_t row_smem_bytes(mbir_plan p, int adjoint_gather);
// Row (NUFFT) kernel of a plan: FP32 plans pair rows l and nx - l in one CTA
enum RowKind { ROW_FWD = 0, ROW_GATHER = 1, ROW_ATOMIC = 2, ROW_FWD_PAIR = 3, ROW_GATHER_PAIR = 4,
               ROW_GATHER_PAIR_LEAN = 5 };
int row_kind(mbir_plan p, bool adjoint);
bool row_kind_fits(mbir_plan p, int kind);     // adjoint kinds a plan can run
int row_ctas(mbir_plan p, int kind);           // CTAs of one scan
size_t row_kind_smem(mbir_plan p, int kind);
void fill_lat_args(mbir_plan p, const LatFill& f, void* dst);
void fill_row_args(mbir_plan p, const void* in, void* out, void* dst);
int batch_lateral(int mode, int precision, const BatchLaunch& L, cudaStream_t st);
int batch_row(int kind, int precision, int J, const BatchLaunch& L, cudaStream_t st);
// FP32 plan whose paired row kernels run the fused first and last transform passes
bool row_fusable(mbir_plan p);

// wavelet.cu (batch helpers)
size_t dwt_args_bytes(int precision);
// P x N: the level's block (analysis input / synthesis output); level 0 = finest
int dwt_level_ctas(int P, int N, int inverse, int level);
size_t dwt_smem_bytes(int precision, int inverse, int level);
void fill_dwt_args(mbir_plan p, int level, int inverse, const void* in, void* out, void* coef, double tau,
                   int thresh, double* partial, void* b1, void* b2, void* dst);
int batch_dwt(int inverse, int level, int precision, const BatchLaunch& L, cudaStream_t st);

// operator.cu
int forward_impl(mbir_plan p, const void* x, const uint8_t* mask, void* y, cudaStream_t st);
int adjoint_impl(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st);
int configure_operator_kernels(mbir_plan p);
// FISTA forward pass on z1 with the fused middle: pz = Phi z1, data-term partials,
// R = first stage of Phi^H on r = (1 + mu) pz - mu pz_prev - s y left in wsA
int forward_solve_impl(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, double mu,
                       double* partial, cudaStream_t st);
// rest of Phi^H from wsA; vout == nullptr: l1 prox fused (z^k written over z2); else v written to vout
int adjoint_solve_impl(mbir_plan p, const void* z1, void* z2, void* vout, double mu, double delta, double tau,
                       double* partial, cudaStream_t st);
// power-iteration step: v = w scal[1], w = Phi^H s Phi v, partials of <v, w>, ||w||^2
int power_step_impl(mbir_plan p, const uint8_t* mask, void* w, void* v, const double* scal, double* part,
                    cudaStream_t st);
int lateral_grid(mbir_plan p, int cols);

// wavelet.cu
int wavelet_impl(mbir_plan p, int inverse, const void* in, void* out, cudaStream_t st);
int prox_impl(mbir_plan p, int penalty, const void* v, double tau, void* z, cudaStream_t st);
bool wavelet_supported(int nx, int nz);
int configure_wavelet_kernels(mbir_plan p);

// tune.cu: a recorded tuning for the plan's shape class, applied at creation
int apply_class_tuning(mbir_plan p);
// plan.cu: radix plan of an n-point transform, radices at most max_radix
bool plan_factor_radix(int n, Radix* r, int max_radix);

// plan.cu: radix plan, [lo | hi] twiddles (plan precision) and digit-reversal
// table of an n-point transform, uploaded; UNSUPPORTED_SIZE unless n is 7-smooth
int plan_fft_tables(mbir_plan p, int n, Radix* rad, void** tw, int** perm);

// hilbert.cu: c = A(s y) = s y - j d H(s y) along the spectrometer axis, c [nx][m]
// complex (d = +1 for ascending wavenumbers); interp: the unmeasured samples are
// first filled by linear interpolation (the baseline of Sec. 3); the tables are
// built on first use
int hilbert_impl(mbir_plan p, const void* y, const uint8_t* mask, void* c, cudaStream_t st, bool interp = false);
int ensure_hilbert(mbir_plan p);
// operator.cu: the paper's back-projection Phi*(y) = B^H A(s y), and its FISTA /
// power-iteration passes (the residual is written to r, then A, then B^H)
int adjoint_hilbert_impl(mbir_plan p, const void* y, const uint8_t* mask, void* x, cudaStream_t st,
                         bool interp = false);
int forward_solve_hilbert_impl(mbir_plan p, const void* z1, const uint8_t* mask, const void* y, void* pz, void* r,
                               double mu, double* partial, cudaStream_t st);
int power_step_hilbert_impl(mbir_plan p, const uint8_t* mask, void* w, void* v, void* r, const double* scal,
                            double* part, cudaStream_t st);

// eval.cu: NCC of magnitudes of two [nx][nz] images (Eq. ncc), synchronous
int ncc_impl(mbir_plan p, const void* x, const void* z, double* r, cudaStream_t st);

// tv.cu: z = prox_{tau TV}(v) by `iters` FGP steps; partial (may be null) receives
// per-CTA sums of TV(z), tv_partial_count(p) of them
int tv_prox_impl(mbir_plan p, const void* v, double tau, int iters, void* z, double* partial, cudaStream_t st);
int tv_partial_count(mbir_plan p);
constexpr int kTvDefaultIters = 20;

// solve.cu
void destroy_solve_state(mbir_plan p);
int part_tmp_count(mbir_plan p);

}  // namespace mbir
