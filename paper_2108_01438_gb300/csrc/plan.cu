// Plan creation: validation of the optical geometry and the FP64 host
// derivation of every table the kernels read (Sec. 2.1).
//
// Per lateral frequency magnitude l' = |l~| (q = 2 pi l'/(nx dx); the tables only
// depend on q^2) and spectrometer pixel m:
//   beta  = sqrt(4 k_m^2 - q^2)                         ISAM resampling, Eq. 5
//   t     = K/(2 pi) (beta dz mod 2 pi)  -> (i0 = floor t, frac = t - i0)
//   f     = A(k) G(q,k) e^{j [Omega(k) - 2 k z_f + beta (z_f - n0 dz)]}
// where G = exp(-q^2/(2 k^2 NA^2)) is the focused Gaussian beam filter (the
// paper's f^, Eq. 5), Omega the dispersion phase and the last term moves the
// phase reference of the depth sum from the NUFFT centre n0 dz to the focus.
// Per depth pixel n:  c_n = w(z_n) / Psi((n - n0)/K)  (falloff x deapodisation).
// All phases are reduced in FP64 before rounding to the kernel precision.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <complex>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "operator.cuh"

namespace mbir {

static thread_local std::string g_last_error;

int set_cuda_error(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return MBIR_ERR_OOM;
  return MBIR_ERR_CUDA;
}

void set_error_text(const std::string& s) { g_last_error = s; }

// Modified Bessel function I0 by its power series sum ((x/2)^k / k!)^2.
static double bessel_i0(double x) {
  const double h = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= h / (double(k) * double(k));
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

double host_bessel_i0(double x) { return bessel_i0(x); }

// Kaiser-Bessel kernel psi(u) = I0(alpha sqrt(1 - (2u/J)^2)) / I0(alpha), |u| <= J/2.
static double kb_psi(double u, int J, double alpha) {
  const double r = 1.0 - (2.0 * u / J) * (2.0 * u / J);
  if (r < 0.0) return 0.0;
  return bessel_i0(alpha * sqrt(r)) / bessel_i0(alpha);
}

// Its Fourier transform at nu cycles per cell:
// J sinh(sqrt(alpha^2 - (pi J nu)^2)) / sqrt(...) / I0(alpha)  (sin form beyond alpha).
static double kb_hat(double nu, int J, double alpha) {
  const double s2 = alpha * alpha - (M_PI * J * nu) * (M_PI * J * nu);
  double v;
  if (s2 > 1e-30) {
    const double s = sqrt(s2);
    v = sinh(s) / s;
  } else if (s2 < -1e-30) {
    const double s = sqrt(-s2);
    v = sin(s) / s;
  } else {
    v = 1.0;
  }
  return J * v / bessel_i0(alpha);
}

// max_radix 16 or 8 (the paired FP32 transforms keep a butterfly's split pairs
// in registers, which radix 16 would overflow)
static bool factor_radix(int n, Radix* r, int max_radix = 16) {
  memset(r, 0, sizeof(*r));
  r->n = n;
  int rem = n;
  const int order[] = {16, 8, 4, 2, 3, 5, 7};
  for (int f : order) {
    if (f > max_radix) continue;
    while (rem % f == 0) {
      if (r->npass >= kMaxPasses) return false;
      r->r[r->npass++] = f;
      rem /= f;
    }
  }
  if (rem != 1) return false;
  // a lone radix-2 pass next to a radix-16 or radix-8 pass: 16*2 -> 8*4, 8*2 -> 4*4
  for (int i = 0; i < r->npass; ++i) {
    if (r->r[i] != 2) continue;
    for (int j = 0; j < r->npass; ++j) {
      if (r->r[j] == 16) { r->r[j] = 8; r->r[i] = 4; break; }
      if (r->r[j] == 8) { r->r[j] = 4; r->r[i] = 4; break; }
    }
    break;
  }
  r->pow2 = (n & (n - 1)) == 0;
  r->log2n = 0;
  while ((1 << r->log2n) < n) ++r->log2n;
  for (int i = 0; i < r->npass; ++i) {
    int b = 0;
    while ((1 << b) < r->r[i]) ++b;
    r->lg[i] = b;
  }
  // two-level twiddle tables: lo = w^i (i < 2^s), hi = w^{i 2^s}
  int s = (r->log2n + 1) / 2;
  if (s < 1) s = 1;
  r->tw_shift = s;
  r->tw_lo = 1 << s;
  r->tw_hi = (n + r->tw_lo - 1) / r->tw_lo;
  return true;
}

bool plan_factor_radix(int n, Radix* r, int max_radix) { return factor_radix(n, r, max_radix); }

template <class V>
static void make_twiddles(const Radix& rad, std::vector<V>& out);

int plan_fft_tables(mbir_plan p, int n, Radix* rad, void** tw, int** perm) {
  if (n < 1 || n > kMaxFFT || !factor_radix(n, rad, 8)) return MBIR_ERR_UNSUPPORTED_SIZE;
  std::vector<int> pr(n);
  for (int i = 0; i < n; ++i) pr[i] = digit_reverse(i, *rad);
  size_t bytes;
  std::vector<double2> t64;
  std::vector<float2> t32;
  const void* src;
  if (p->precision == MBIR_FP64) {
    make_twiddles(*rad, t64);
    bytes = sizeof(double2) * t64.size();
    src = t64.data();
  } else {
    make_twiddles(*rad, t32);
    bytes = sizeof(float2) * t32.size();
    src = t32.data();
  }
  MBIR_CUDA_TRY(cudaMalloc(tw, bytes));
  MBIR_CUDA_TRY(cudaMalloc(perm, sizeof(int) * n));
  MBIR_CUDA_TRY(cudaMemcpy(*tw, src, bytes, cudaMemcpyHostToDevice));
  MBIR_CUDA_TRY(cudaMemcpy(*perm, pr.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  // a copy from pageable memory may return before its DMA lands, and it is
  // ordered only against the legacy default stream: wait for it, so that kernels
  // on any stream of the caller see the tables
  MBIR_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
  return MBIR_OK;
}

// [lo | hi] twiddle tables of an n-point transform, w = e^{-2 pi j / n}, in FP64.
template <class V>
static void make_twiddles(const Radix& rad, std::vector<V>& out) {
  const int n = rad.n;
  out.resize(rad.tw_lo + rad.tw_hi);
  for (int i = 0; i < rad.tw_lo; ++i) {
    const double a = -2.0 * M_PI * double(i % n) / double(n);
    out[i].x = cos(a);
    out[i].y = sin(a);
  }
  for (int i = 0; i < rad.tw_hi; ++i) {
    const double a = -2.0 * M_PI * double(((int64_t)i * rad.tw_lo) % n) / double(n);
    out[rad.tw_lo + i].x = cos(a);
    out[rad.tw_lo + i].y = sin(a);
  }
}

// FP64 fit of the KB weight of each tap j as a degree-kKbDeg polynomial in
// x = frac - 1/2 (tap offset J/2 - 1 - j + frac), interpolating at Chebyshev
// nodes on [-1/2, 1/2] (Vandermonde system by Gaussian elimination).
static void fit_kb_polynomials(int J, double alpha, float out[kMaxJ][kKbDeg + 1]) {
  constexpr int D = kKbDeg + 1;
  memset(out, 0, sizeof(float) * kMaxJ * D);
  for (int j = 0; j < J; ++j) {
    double A[D][D + 1];
    for (int q = 0; q < D; ++q) {
      const double x = 0.5 * cos(M_PI * (q + 0.5) / D);
      double pw = 1.0;
      for (int d = 0; d < D; ++d) {
        A[q][d] = pw;
        pw *= x;
      }
      A[q][D] = kb_psi(x + 0.5 + (J / 2 - 1 - j), J, alpha);
    }
    for (int c = 0; c < D; ++c) {
      int piv = c;
      for (int q = c + 1; q < D; ++q)
        if (fabs(A[q][c]) > fabs(A[piv][c])) piv = q;
      for (int d = 0; d <= D; ++d) {
        const double t = A[c][d];
        A[c][d] = A[piv][d];
        A[piv][d] = t;
      }
      for (int q = c + 1; q < D; ++q) {
        const double f = A[q][c] / A[c][c];
        for (int d = c; d <= D; ++d) A[q][d] -= f * A[c][d];
      }
    }
    double coef[D];
    for (int c = D - 1; c >= 0; --c) {
      double acc = A[c][D];
      for (int d = c + 1; d < D; ++d) acc -= A[c][d] * coef[d];
      coef[c] = acc / A[c][c];
    }
    for (int d = 0; d < D; ++d) out[j][d] = (float)coef[d];
  }
}

// Lateral transform length of an nx-point axis: nx itself when it factors into
// radices 2..8, else the smallest 7-smooth length >= 2 nx - 1 for the Bluestein
// (chirp-z) form; 0 when that exceeds the largest transform or its tile of two
// columns exceeds the lateral shared-memory tile.
static int lateral_length(int nx) {
  Radix r;
  if (factor_radix(nx, &r, 8)) return nx;
  for (int n = 2 * nx - 1; n <= kMaxFFT && 2 * n <= kLatElems; ++n)
    if (factor_radix(n, &r, 8)) return n;
  return 0;
}

static int validate(const mbir_geometry* g) {
  if (!g || !g->k) return MBIR_ERR_INVALID;
  if (g->nx <= 0 || g->nz <= 0 || g->m <= 0) return MBIR_ERR_INVALID;
  if (!(g->dx_um > 0) || !(g->dz_um >= 0) || !isfinite(g->dx_um) || !isfinite(g->dz_um))
    return MBIR_ERR_INVALID;
  if (!isfinite(g->na) || !isfinite(g->z_focus_um) || !isfinite(g->disp_a) || !isfinite(g->disp_b) ||
      !isfinite(g->k0) || !isfinite(g->falloff_half_um) || !isfinite(g->kb_alpha) || g->kb_alpha < 0)
    return MBIR_ERR_INVALID;
  if (g->precision < MBIR_FP32 || g->precision > MBIR_FP64) return MBIR_ERR_INVALID;
  for (int i = 0; i < g->m; ++i) {
    if (!isfinite(g->k[i]) || g->k[i] <= 0) return MBIR_ERR_INVALID;
    if (g->source && (!isfinite(g->source[i]) || g->source[i] < 0)) return MBIR_ERR_INVALID;
  }
  if (g->m > 1) {
    const bool inc = g->k[1] > g->k[0];
    for (int i = 1; i < g->m; ++i) {
      if (inc ? !(g->k[i] > g->k[i - 1]) : !(g->k[i] < g->k[i - 1])) return MBIR_ERR_INVALID;
    }
  } else if (g->dz_um == 0) {
    return MBIR_ERR_INVALID;   // the default dz needs a wavenumber step
  }
  if (g->kb_width < 4 || g->kb_width > 8 || (g->kb_width & 1)) return MBIR_ERR_UNSUPPORTED_SIZE;
  if (g->kb_oversamp != 2.0) return MBIR_ERR_UNSUPPORTED_SIZE;
  if (g->nx < 2 || g->nx > 4096 || g->nz < 8 || g->nz > 4096 || g->m > 65536)
    return MBIR_ERR_UNSUPPORTED_SIZE;
  if ((int64_t)g->nx * g->nz >= (int64_t(1) << 31) || (int64_t)g->nx * g->m >= (int64_t(1) << 31))
    return MBIR_ERR_UNSUPPORTED_SIZE;
  Radix r;
  if (!lateral_length(g->nx) || !factor_radix(2 * g->nz, &r)) return MBIR_ERR_UNSUPPORTED_SIZE;
  return MBIR_OK;
}

// Tables of one lateral axis of n pixels whose transform has length nl (rad):
// twiddles, the tile row of each output (digit reversal, or the identity for the
// Bluestein form) and, when nl != n, the Bluestein chirp and the transformed
// conjugate chirp.  Uploaded on st, which is synchronised before returning.
template <class R>
static int lateral_axis_tables(int n, const Radix& rad, void** tw, int** perm, void** chirp, void** bhat,
                               cudaStream_t st) {
  using V = cplx_t<R>;
  const int nl = rad.n;
  const bool blu = nl != n;
  std::vector<V> twv;
  make_twiddles(rad, twv);
  std::vector<int> pv(n);
  for (int i = 0; i < n; ++i) pv[i] = blu ? i : digit_reverse(i, rad);
  MBIR_CUDA_TRY(cudaMalloc(tw, sizeof(V) * twv.size()));
  MBIR_CUDA_TRY(cudaMalloc(perm, sizeof(int) * n));
  MBIR_CUDA_TRY(cudaMemcpyAsync(*tw, twv.data(), sizeof(V) * twv.size(), cudaMemcpyHostToDevice, st));
  MBIR_CUDA_TRY(cudaMemcpyAsync(*perm, pv.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  std::vector<V> ch, bh;
  if (blu) {
    // Bluestein: X_l = c_l sum_p (x_p c_p) conj(c)_{l-p}, c_k = e^{-j pi k^2 / n}; the
    // convolution runs through nl-point transforms (nl >= 2 n - 1, no wrap-around)
    ch.resize(n);
    bh.resize(nl);
    std::vector<std::complex<double>> b(nl, 0.0), w(nl);
    for (int k = 0; k < n; ++k) {
      const double a = M_PI * double(((int64_t)k * k) % (2 * (int64_t)n)) / n;
      ch[k].x = R(cos(a));
      ch[k].y = R(-sin(a));
      b[k] = std::complex<double>(cos(a), sin(a));
      if (k) b[nl - k] = b[k];
    }
    for (int k = 0; k < nl; ++k) w[k] = std::polar(1.0, -2.0 * M_PI * k / nl);
    for (int j = 0; j < nl; ++j) {
      std::complex<double> acc = 0.0;
      for (int k = 0; k < nl; ++k) acc += b[k] * w[((int64_t)j * k) % nl];
      acc /= double(nl);
      V& e = bh[digit_reverse(j, rad)];
      e.x = R(acc.real());
      e.y = R(acc.imag());
    }
    MBIR_CUDA_TRY(cudaMalloc(chirp, sizeof(V) * n));
    MBIR_CUDA_TRY(cudaMalloc(bhat, sizeof(V) * nl));
    MBIR_CUDA_TRY(cudaMemcpyAsync(*chirp, ch.data(), sizeof(V) * n, cudaMemcpyHostToDevice, st));
    MBIR_CUDA_TRY(cudaMemcpyAsync(*bhat, bh.data(), sizeof(V) * nl, cudaMemcpyHostToDevice, st));
  }
  MBIR_CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors die here
  return MBIR_OK;
}

template <class R>
static int upload_tables(mbir_plan p, const mbir_geometry* g, cudaStream_t st) {
  using V = cplx_t<R>;
  using Tab = typename TabOf<R>::T;
  const int nx = p->nx, nz = p->nz, m = p->m, K = p->K, J = p->J;
  std::vector<V> twk;
  make_twiddles(p->rad_k, twk);
  int rc = lateral_axis_tables<R>(nx, p->rad_x, &p->tw_x, &p->perm_x, &p->chirp, &p->bhat, st);
  if (rc) return rc;
  if (p->ny > 1) {
    rc = lateral_axis_tables<R>(p->ny, p->rad_y, &p->tw_y, &p->perm_y, &p->chirp_y, &p->bhat_y, st);
    if (rc) return rc;
  }
  std::vector<R> cdep(nz);
  for (int n = 0; n < nz; ++n) {
    const double z = n * p->dz;
    double w = 1.0;
    if (g->falloff_half_um > 0) w = exp(-M_LN2 * (z / g->falloff_half_um) * (z / g->falloff_half_um));
    cdep[n] = R(w / kb_hat(double(n - p->n0) / K, J, p->alpha));
  }
  // Resampling table.  Per row l' and pixel m: the first tap cell pc = floor(t) -
  // J/2 + 1 (mod K), frac, and the filter.  For the adjoint's segmented gather the
  // first-tap cells of a row are also unwrapped into a monotone sequence U_m (the
  // beta mapping is monotone in k); u = U_m - min U is packed above pc.  Rows whose
  // unwrapped cells are not monotone or span more than K cells make the plan use
  // shared-memory atomics in the adjoint instead.
  std::vector<Tab> tab((size_t)p->ntab * m);
  std::vector<int4> meta(p->ntab);
  const int nyh = p->ny / 2 + 1;
  const int h = J / 2;
  bool gather_ok = m <= 65535 && K <= 32768;
  std::vector<int> pc(m), valid(m);
  std::vector<double> fr(m);
  std::vector<long long> U(m);
  for (int lp = 0; lp < p->ntab; ++lp) {
    // table row lp: lateral frequency (|lx|, |ly|) = (lp / nyh, lp % nyh); |ly| = 0 for a B-scan
    const double qx = 2.0 * M_PI * (lp / nyh) / (nx * p->dx);
    const double qy = p->ny > 1 ? 2.0 * M_PI * (lp % nyh) / (p->ny * p->dy) : 0.0;
    const double q2 = qx * qx + qy * qy;
    for (int mm = 0; mm < m; ++mm) {
      const double k = g->k[mm];
      const double b2 = 4.0 * k * k - q2;
      Tab e;
      memset(&e, 0, sizeof(e));
      valid[mm] = b2 > 0;
      pc[mm] = 0;
      fr[mm] = 0.0;
      if (b2 > 0) {
        const double beta = sqrt(b2);
        double t = (K / (2.0 * M_PI)) * fmod(beta * p->dz, 2.0 * M_PI);
        double i0 = floor(t);
        fr[mm] = t - i0;
        long long first = (long long)i0 - h + 1;
        first %= K;
        if (first < 0) first += K;
        pc[mm] = (int)first;
        const double A = g->source ? g->source[mm] : 1.0;
        const double G = g->na > 0 ? exp(-q2 / (2.0 * k * k * g->na * g->na)) : 1.0;
        const double dk = k - g->k0;
        const double omega = g->disp_a * dk * dk + g->disp_b * dk * dk * dk;
        const double phase = fmod(omega - 2.0 * k * g->z_focus_um, 2.0 * M_PI) +
                             fmod(beta * (g->z_focus_um - p->n0 * p->dz), 2.0 * M_PI);
        e.fre = (decltype(e.fre))(A * G * cos(phase));
        e.fim = (decltype(e.fim))(A * G * sin(phase));
      }
      tab[(size_t)lp * m + mm] = e;
    }
    // evanescent pixels (filter 0) borrow a neighbour's position to keep the row monotone
    int first_valid = -1, last = -1;
    for (int mm = 0; mm < m; ++mm) {
      if (valid[mm]) {
        if (first_valid < 0) first_valid = mm;
        last = mm;
      } else if (last >= 0) {
        pc[mm] = pc[last];
        fr[mm] = fr[last];
      }
    }
    for (int mm = 0; mm < first_valid; ++mm) {
      pc[mm] = pc[first_valid];
      fr[mm] = fr[first_valid];
    }
    // unwrap and check monotonicity / span
    U[0] = pc[0];
    int dir = 0;
    bool mono = true;
    for (int mm = 1; mm < m; ++mm) {
      long long d = (long long)pc[mm] - pc[mm - 1];
      if (d > K / 2) d -= K;
      if (d <= -(K + 1) / 2) d += K;
      U[mm] = U[mm - 1] + d;
      if (d > 0) {
        if (dir < 0) mono = false;
        dir = 1;
      } else if (d < 0) {
        if (dir > 0) mono = false;
        dir = -1;
      }
    }
    long long umin = U[0], umax = U[0];
    for (int mm = 1; mm < m; ++mm) {
      umin = U[mm] < umin ? U[mm] : umin;
      umax = U[mm] > umax ? U[mm] : umax;
    }
    const long long span = umax - umin + J;
    if (!mono || span > K) gather_ok = false;
    if (span > p->max_span) p->max_span = (int)span;
    long long base = umin % K;
    if (base < 0) base += K;
    meta[lp] = make_int4((int)base, (int)span, dir >= 0 ? 1 : -1, 0);
    for (int mm = 0; mm < m; ++mm) {
      Tab& e = tab[(size_t)lp * m + mm];
      const long long u = (mono && span <= K) ? U[mm] - umin : 0;
      e.cell = (int)((u << 16) | (long long)pc[mm]);
      e.frac = (decltype(e.frac))fr[mm];
    }
  }
  p->gather_ok = gather_ok ? 1 : 0;
  MBIR_CUDA_TRY(cudaMalloc(&p->rowmeta, sizeof(int4) * meta.size()));
  MBIR_CUDA_TRY(cudaMemcpyAsync(p->rowmeta, meta.data(), sizeof(int4) * meta.size(), cudaMemcpyHostToDevice, st));
  MBIR_CUDA_TRY(cudaMalloc(&p->tw_k, sizeof(V) * twk.size()));
  MBIR_CUDA_TRY(cudaMalloc(&p->cdep, sizeof(R) * nz));
  MBIR_CUDA_TRY(cudaMalloc(&p->tab, sizeof(Tab) * tab.size()));
  if (sizeof(R) == 4 && kFilterOtf) {
    // the filter's factors: per pixel A e^{j(Omega - 2k z_f + 2k (z_f - z_c))}, the beam
    // filter's 1/(2 k^2 NA^2) and 2k; per table row q^2; the row kernels form
    // A G(q, k) e^{j(Omega - 2k z_f + beta (z_f - z_c))} as that times
    // exp(-q^2 / (2 k^2 NA^2)) e^{-j (2k - beta)(z_f - z_c)}, 2k - beta = q^2 / (beta + 2k)
    std::vector<TabP> tp(tab.size());
    for (size_t i = 0; i < tab.size(); ++i) {
      tp[i].cell = tab[i].cell;
      tp[i].frac = (float)tab[i].frac;
    }
    std::vector<float4> fp(m);
    const double zc = p->n0 * p->dz, dzf = g->z_focus_um - zc;
    for (int mm = 0; mm < m; ++mm) {
      const double k = g->k[mm];
      const double A = g->source ? g->source[mm] : 1.0;
      const double dk = k - g->k0;
      const double omega = g->disp_a * dk * dk + g->disp_b * dk * dk * dk;
      const double ph = fmod(omega - 2.0 * k * g->z_focus_um, 2.0 * M_PI) + fmod(2.0 * k * dzf, 2.0 * M_PI);
      fp[mm] = make_float4((float)(A * cos(ph)), (float)(A * sin(ph)),
                           g->na > 0 ? (float)(1.0 / (2.0 * k * k * g->na * g->na)) : 0.0f, (float)(2.0 * k));
    }
    std::vector<float> q2v(p->ntab);
    for (int lp = 0; lp < p->ntab; ++lp) {
      const double qx = 2.0 * M_PI * (lp / nyh) / (nx * p->dx);
      const double qy = p->ny > 1 ? 2.0 * M_PI * (lp % nyh) / (p->ny * p->dy) : 0.0;
      q2v[lp] = (float)(qx * qx + qy * qy);
    }
    p->otf = 1;
    p->dzf = (float)dzf;
    MBIR_CUDA_TRY(cudaMalloc(&p->tabp, sizeof(TabP) * tp.size()));
    MBIR_CUDA_TRY(cudaMalloc(&p->fpix, sizeof(float4) * fp.size()));
    MBIR_CUDA_TRY(cudaMalloc(&p->q2row, sizeof(float) * q2v.size()));
    MBIR_CUDA_TRY(cudaMemcpyAsync(p->tabp, tp.data(), sizeof(TabP) * tp.size(), cudaMemcpyHostToDevice, st));
    MBIR_CUDA_TRY(cudaMemcpyAsync(p->fpix, fp.data(), sizeof(float4) * fp.size(), cudaMemcpyHostToDevice, st));
    MBIR_CUDA_TRY(cudaMemcpyAsync(p->q2row, q2v.data(), sizeof(float) * q2v.size(), cudaMemcpyHostToDevice, st));
    MBIR_CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors die here
  }
  MBIR_CUDA_TRY(cudaMemcpyAsync(p->tw_k, twk.data(), sizeof(V) * twk.size(), cudaMemcpyHostToDevice, st));
  MBIR_CUDA_TRY(cudaMemcpyAsync(p->cdep, cdep.data(), sizeof(R) * nz, cudaMemcpyHostToDevice, st));
  MBIR_CUDA_TRY(cudaMemcpyAsync(p->tab, tab.data(), sizeof(Tab) * tab.size(), cudaMemcpyHostToDevice, st));
  std::vector<int> pk(K);
  for (int i = 0; i < K; ++i) pk[i] = digit_reverse(i, p->rad_k);
  MBIR_CUDA_TRY(cudaMalloc(&p->perm_k, sizeof(int) * K));
  MBIR_CUDA_TRY(cudaMemcpyAsync(p->perm_k, pk.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
  MBIR_CUDA_TRY(cudaStreamSynchronize(st));
  return MBIR_OK;
}

// Daubechies low-pass filter with 4 vanishing moments, derived by spectral
// factorisation: z^3 P((2 - z - 1/z)/4), P(u) = 1 + 4u + 10u^2 + 20u^3, has three
// reciprocal root pairs; the roots inside the unit circle (found by Durand-Kerner
// iteration) together with four roots at z = -1 give the minimum-phase filter,
// scaled to sum sqrt(2).
static void daubechies8(double h[8]) {
  // polynomial coefficients, highest power first, of z^3 P(u(z))
  // u z = (-z^2 + 2z - 1)/4
  double poly[7] = {0, 0, 0, 0, 0, 0, 0};
  const double binom[4] = {1, 4, 10, 20};
  for (int kk = 0; kk < 4; ++kk) {
    double term[7] = {1, 0, 0, 0, 0, 0, 0};
    int deg = 0;
    for (int r = 0; r < kk; ++r) {
      double nt[7] = {0, 0, 0, 0, 0, 0, 0};
      const double uz[3] = {-0.25, 0.5, -0.25};
      for (int a = 0; a <= deg; ++a)
        for (int b = 0; b < 3; ++b) nt[a + b] += term[a] * uz[b];
      deg += 2;
      for (int a = 0; a <= deg; ++a) term[a] = nt[a];
    }
    // term (degree 2kk) times z^(3-kk), aligned in a degree-6 array
    const int lead = 3 - kk;
    for (int a = 0; a <= deg; ++a) poly[lead + a] += binom[kk] * term[a];
  }
  // Durand-Kerner on the monic version
  double re[6], im[6];
  for (int i = 0; i < 6; ++i) {
    const double ang = 0.4 + 2.0 * M_PI * i / 6.0;
    re[i] = 0.9 * cos(ang);
    im[i] = 0.9 * sin(ang);
  }
  for (int it = 0; it < 2000; ++it) {
    double maxd = 0;
    for (int i = 0; i < 6; ++i) {
      // p(z_i)
      double pr = 1.0, pi = 0.0;
      for (int a = 1; a <= 6; ++a) {
        const double nr = pr * re[i] - pi * im[i] + poly[a] / poly[0];
        const double ni = pr * im[i] + pi * re[i];
        pr = nr; pi = ni;
      }
      double dr = 1.0, di = 0.0;
      for (int j = 0; j < 6; ++j) {
        if (j == i) continue;
        const double xr = re[i] - re[j], xi = im[i] - im[j];
        const double nr = dr * xr - di * xi, ni = dr * xi + di * xr;
        dr = nr; di = ni;
      }
      const double den = dr * dr + di * di;
      const double qr = (pr * dr + pi * di) / den, qi = (pi * dr - pr * di) / den;
      re[i] -= qr;
      im[i] -= qi;
      maxd = fmax(maxd, fabs(qr) + fabs(qi));
    }
    if (maxd < 1e-16) break;
  }
  // product (z+1)^4 * prod_{|r|<1} (z - r), highest power first
  double cr[8] = {1, 0, 0, 0, 0, 0, 0, 0}, ci[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int deg = 0;
  auto mul_root = [&](double rr, double ri) {
    double nr[8] = {0}, ni[8] = {0};
    for (int a = 0; a <= deg; ++a) {
      nr[a] += cr[a];
      ni[a] += ci[a];
      nr[a + 1] -= cr[a] * rr - ci[a] * ri;
      ni[a + 1] -= cr[a] * ri + ci[a] * rr;
    }
    ++deg;
    for (int a = 0; a <= deg; ++a) { cr[a] = nr[a]; ci[a] = ni[a]; }
  };
  for (int i = 0; i < 4; ++i) mul_root(-1.0, 0.0);
  for (int i = 0; i < 6; ++i)
    if (re[i] * re[i] + im[i] * im[i] < 1.0) mul_root(re[i], im[i]);
  double s = 0;
  for (int a = 0; a < 8; ++a) s += cr[a];
  for (int a = 0; a < 8; ++a) h[a] = cr[a] * (M_SQRT2 / s);
}

void daubechies8_taps(double h[8]) { daubechies8(h); }

const char* prof_class_name(int c) {
  static const char* names[PC_COUNT] = {"lateral_forward", "row_forward", "lateral_inverse_real",
                                        "lateral_residual", "row_adjoint", "lateral_adjoint",
                                        "dwt_analysis", "dwt_synthesis", "soft_threshold", "reduce",
                                        "lateral_mid", "tv_prox", "hilbert"};
  return (c >= 0 && c < PC_COUNT) ? names[c] : "unknown";
}

void destroy_profiler(mbir_plan p) {
  Profiler* pr = p->prof;
  if (!pr) return;
  for (int i = 0; i < 2 * pr->cap; ++i) cudaEventDestroy(pr->ev[i]);
  delete[] pr->ev;
  delete[] pr->cls;
  delete pr;
  p->prof = nullptr;
}

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_profile_begin(mbir_plan p, int32_t capacity) {
  if (!p || capacity < 1 || capacity > (1 << 22)) return MBIR_ERR_INVALID;
  destroy_profiler(p);
  Profiler* pr = new (std::nothrow) Profiler;
  if (!pr) return MBIR_ERR_OOM;
  pr->ev = new (std::nothrow) cudaEvent_t[2 * (size_t)capacity];
  pr->cls = new (std::nothrow) int[capacity];
  if (!pr->ev || !pr->cls) {
    delete[] pr->ev;
    delete[] pr->cls;
    delete pr;
    return MBIR_ERR_OOM;
  }
  int made = 0;
  for (; made < 2 * capacity; ++made) {
    if (cudaEventCreate(&pr->ev[made]) != cudaSuccess) break;
  }
  if (made < 2 * capacity) {
    for (int i = 0; i < made; ++i) cudaEventDestroy(pr->ev[i]);
    delete[] pr->ev;
    delete[] pr->cls;
    delete pr;
    return set_cuda_error(cudaGetLastError(), "cudaEventCreate");
  }
  pr->cap = capacity;
  pr->n = 0;
  p->prof = pr;
  return MBIR_OK;
}

int mbir_profile_only(mbir_plan p, const char* kernel_class) {
  if (!p || !p->prof) return MBIR_ERR_INVALID;
  if (!kernel_class) {
    p->prof->mask = ~0u;
    return MBIR_OK;
  }
  for (int c = 0; c < PC_COUNT; ++c) {
    if (strcmp(prof_class_name(c), kernel_class) == 0) {
      p->prof->mask = 1u << c;
      return MBIR_OK;
    }
  }
  return MBIR_ERR_INVALID;
}

int mbir_profile_end(mbir_plan p, mbir_profile_entry* out, int32_t max_entries, int32_t* n_entries) {
  if (!p || !p->prof) return MBIR_ERR_INVALID;
  Profiler* pr = p->prof;
  int64_t launches[PC_COUNT] = {0};
  double total[PC_COUNT] = {0};
  int rc = MBIR_OK;
  for (int i = 0; i < pr->n; ++i) {
    cudaError_t e = cudaEventSynchronize(pr->ev[2 * i + 1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr->ev[2 * i], pr->ev[2 * i + 1]);
    if (e != cudaSuccess) {
      rc = set_cuda_error(e, "profile events");
      break;
    }
    launches[pr->cls[i]] += 1;
    total[pr->cls[i]] += ms;
  }
  int n = 0;
  for (int c = 0; c < PC_COUNT; ++c) {
    if (!launches[c]) continue;
    if (out && n < max_entries) {
      out[n].name = prof_class_name(c);
      out[n].launches = launches[c];
      out[n].total_ms = total[c];
    }
    ++n;
  }
  if (n_entries) *n_entries = n;
  destroy_profiler(p);
  return rc;
}

const char* mbir_status_string(int s) {
  switch (s) {
    case MBIR_OK: return "ok";
    case MBIR_ERR_INVALID: return "invalid argument";
    case MBIR_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case MBIR_ERR_OOM: return "out of device memory";
    case MBIR_ERR_CUDA: return "CUDA error";
    case MBIR_ERR_TIMEOUT: return "device wait timed out";
    case MBIR_ERR_NOT_CONVERGED: return "not converged";
    default: return "unknown status";
  }
}

const char* mbir_last_error(void) { return g_last_error.c_str(); }

void mbir_plan_destroy(mbir_plan p) {
  if (!p) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  destroy_profiler(p);
  destroy_solve_state(p);
  cudaFree(p->tw_x);
  cudaFree(p->tw_k);
  cudaFree(p->perm_x);
  cudaFree(p->chirp);
  cudaFree(p->bhat);
  cudaFree(p->rowmap);
  cudaFree(p->tabp);
  cudaFree(p->fpix);
  cudaFree(p->q2row);
  cudaFree(p->tw_y);
  cudaFree(p->perm_y);
  cudaFree(p->chirp_y);
  cudaFree(p->bhat_y);
  cudaFree(p->rowmeta);
  cudaFree(p->perm_k);
  cudaFree(p->cdep);
  cudaFree(p->tab);
  cudaFree(p->h_db4);
  cudaFree(p->h_db4f);
  cudaFree(p->wv_b1);
  cudaFree(p->wv_b2);
  cudaFree(p->wv_coef);
  for (void* q : p->tv_p) cudaFree(q);
  cudaFree(p->tw_m);
  cudaFree(p->perm_m);
  cudaFree(p->ncc_scratch);
  cudaFree(p->wsA);
  cudaFree(p->wsB);
  cudaFree(p->red);
  if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
  delete p;
}

}  // extern "C"

// A B-scan plan (ny = 1) or a volume plan with a second lateral axis of ny pixels
// spaced dy.
static int plan_create(const mbir_geometry* g, int ny, double dy, void* stream, mbir_plan* out) {
  if (!out) return MBIR_ERR_INVALID;
  *out = nullptr;
  const int v = validate(g);
  if (v != MBIR_OK) return v;
  if (ny < 1 || (ny > 1 && !(dy > 0 && isfinite(dy)))) return MBIR_ERR_INVALID;
  if (ny > 4096) return MBIR_ERR_UNSUPPORTED_SIZE;
  if (ny > 1 && ((int64_t)g->nx * ny * g->nz >= (int64_t(1) << 31) ||
                 (int64_t)g->nx * ny * g->m >= (int64_t(1) << 31) || !lateral_length(ny)))
    return MBIR_ERR_UNSUPPORTED_SIZE;
  cudaStream_t st = (cudaStream_t)stream;

  mbir_plan p = new (std::nothrow) mbir_plan_s;
  if (!p) return MBIR_ERR_OOM;
  memset(p, 0, sizeof(*p));
  p->nx = g->nx;
  p->nz = g->nz;
  p->m = g->m;
  p->K = 2 * g->nz;
  p->J = g->kb_width;
  p->n0 = g->nz / 2;
  p->nlh = g->nx / 2 + 1;
  p->ny = ny;
  p->dy = ny > 1 ? dy : 0.0;
  p->ntab = p->nlh * (ny / 2 + 1);
  p->npair = p->nlh;
  p->precision = g->precision;
  p->dx = g->dx_um;
  if (g->dz_um > 0) {
    p->dz = g->dz_um;
  } else {
    double dkmax = 0;
    for (int i = 1; i < g->m; ++i) dkmax = fmax(dkmax, fabs(g->k[i] - g->k[i - 1]));
    p->dz = M_PI / (2.0 * g->nz * dkmax);
  }
  p->alpha = g->kb_alpha > 0 ? g->kb_alpha : 2.34 * g->kb_width;
  p->k_ascending = g->m < 2 || g->k[g->m - 1] > g->k[0];
  p->nxl = lateral_length(p->nx);
  factor_radix(p->nxl, &p->rad_x, 8);
  factor_radix(p->K, &p->rad_k, 8);
  // lateral tile: keep nxl * tile_c <= kLatElems elements, at most 16 columns
  int tc = kLatElems / p->nxl;
  if (tc > 16) tc = 16;
  int pw = 1;
  while (pw * 2 <= tc) pw *= 2;
  p->tile_c = pw;
  if (ny > 1) {
    p->nyl = lateral_length(ny);
    factor_radix(p->nyl, &p->rad_y, 8);
    int ty = kLatElems / p->nyl;
    if (ty > 16) ty = 16;
    int py = 1;
    while (py * 2 <= ty) py *= 2;
    p->tile_y = py;
  }

  int rc = MBIR_OK;
  auto fail = [&](int code) { mbir_plan_destroy(p); return code; };
  if (cudaGetDevice(&p->device) != cudaSuccess) return fail(set_cuda_error(cudaGetLastError(), "cudaGetDevice"));
  if (ny > 1) {
    // row pairs of the 2-D lateral spectrum [lx][ly]: a row and its point reflection
    // (-lx, -ly) share |q| and so the table row (|lx|, |ly|); a row that is its own
    // reflection runs alone
    const int nx = p->nx, nyh = ny / 2 + 1;
    std::vector<int4> map;
    for (int lx = 0; lx < nx; ++lx)
      for (int ly = 0; ly < ny; ++ly) {
        const int r = lx * ny + ly, mr = ((nx - lx) % nx) * ny + (ny - ly) % ny;
        if (mr < r) continue;
        const int ix = lx <= nx - lx ? lx : nx - lx, iy = ly <= ny - ly ? ly : ny - ly;
        map.push_back(make_int4(r, mr == r ? -1 : mr, ix * nyh + iy, 0));
      }
    p->npair = (int)map.size();
    cudaError_t e = cudaMalloc(&p->rowmap, sizeof(int4) * map.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->rowmap, map.data(), sizeof(int4) * map.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) return fail(set_cuda_error(e, "volume row map"));
  }

  rc = (p->precision == MBIR_FP64) ? upload_tables<double>(p, g, st) : upload_tables<float>(p, g, st);
  if (rc != MBIR_OK) return fail(rc);

  fit_kb_polynomials(p->J, p->alpha, p->kbpoly);
  {
    double h[8];
    daubechies8(h);
    float hf[8];
    for (int i = 0; i < 8; ++i) hf[i] = (float)h[i];
    cudaError_t e = cudaMalloc(&p->h_db4, sizeof(h));
    if (e == cudaSuccess) e = cudaMalloc(&p->h_db4f, sizeof(hf));
    if (e == cudaSuccess) e = cudaMemcpy(p->h_db4, h, sizeof(h), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->h_db4f, hf, sizeof(hf), cudaMemcpyHostToDevice);
    // pageable copies: wait until they have landed (see plan_fft_tables)
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) return fail(set_cuda_error(e, "wavelet filter upload"));
  }
  {
    const size_t cols = (size_t)(p->nz > p->m ? p->nz : p->m);
    p->ws_elems = (size_t)p->nx * p->ny * cols;
    const size_t esz = (p->precision == MBIR_FP64) ? sizeof(double2) : sizeof(float2);
    cudaError_t e = cudaMalloc(&p->wsA, esz * p->ws_elems);
    if (e == cudaSuccess) e = cudaMalloc(&p->wsB, esz * p->ws_elems);
    if (e == cudaSuccess) e = cudaMalloc(&p->red, sizeof(double) * kRedSlots);
    if (e != cudaSuccess) return fail(set_cuda_error(e, "workspace allocation"));
  }
  rc = configure_operator_kernels(p);
  if (rc != MBIR_OK) return fail(rc);
  rc = configure_wavelet_kernels(p);
  if (rc != MBIR_OK) return fail(rc);
  p->adj_kind = -1;
  if (ny == 1) {
    rc = apply_class_tuning(p);
    if (rc != MBIR_OK) return fail(rc);
  }
  *out = p;
  return MBIR_OK;
}

extern "C" {

int mbir_plan_create(const mbir_geometry* g, void* stream, mbir_plan* out) {
  return plan_create(g, 1, 0.0, stream, out);
}

int mbir_volume_plan_create(const mbir_geometry* g, int32_t ny, double dy_um, void* stream, mbir_plan* out) {
  if (ny < 2 || !isfinite(dy_um)) return MBIR_ERR_INVALID;
  return plan_create(g, ny, dy_um > 0 ? dy_um : (g ? g->dx_um : 0.0), stream, out);
}

int mbir_volume_dims(mbir_plan p, int32_t* ny) {
  if (!p || !ny) return MBIR_ERR_INVALID;
  *ny = p->ny;
  return MBIR_OK;
}

int mbir_plan_dims(mbir_plan p, int32_t* nx, int32_t* nz, int32_t* m, int32_t* precision) {
  if (!p) return MBIR_ERR_INVALID;
  if (nx) *nx = p->nx;
  if (nz) *nz = p->nz;
  if (m) *m = p->m;
  if (precision) *precision = p->precision;
  return MBIR_OK;
}

}  // extern "C"
