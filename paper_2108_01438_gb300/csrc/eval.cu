// The evaluation loop of Sec. 3: the normalised cross-correlation of magnitudes
// (Eq. ncc) and the golden-section search of lambda that maximises it.
//
// NCC: two grid-stride passes over the two images, each CTA writing FP64 partial
// sums (first sum|x| and sum|z|, then the centred products), each pass closed by
// a one-CTA kernel that adds the partials in a fixed order, so the value is
// deterministic.  The images are read twice: 4 x 8 bytes per pixel in FP32.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace mbir {

constexpr int kNccThreads = 256;
constexpr int kNccBlocks = 1024;

__device__ __forceinline__ double ncc_block_sum(double v) {
  __shared__ double wsum[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = lane < nw ? wsum[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// stat == nullptr: part[2 b] = sum |x|, part[2 b + 1] = sum |z| over this CTA's pixels;
// else, with a = |x| - stat[0], c = |z| - stat[1]: part[3 b ..] = sum a c, sum a^2, sum c^2.
template <class R>
__global__ void __launch_bounds__(kNccThreads)
    ncc_pass_kernel(const cplx_t<R>* __restrict__ x, const cplx_t<R>* __restrict__ z, size_t n,
                    const double* __restrict__ stat, double* __restrict__ part) {
  pdl_wait_release();
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const double mx = stat ? stat[0] : 0.0, mz = stat ? stat[1] : 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cplx_t<R> u = x[i], v = z[i];
    const double ax = sqrt(double(u.x) * u.x + double(u.y) * u.y);
    const double az = sqrt(double(v.x) * v.x + double(v.y) * v.y);
    if (stat) {
      const double a = ax - mx, c = az - mz;
      s0 += a * c;
      s1 += a * a;
      s2 += c * c;
    } else {
      s0 += ax;
      s1 += az;
    }
  }
  const double t0 = ncc_block_sum(s0), t1 = ncc_block_sum(s1);
  if (stat) {
    const double t2 = ncc_block_sum(s2);
    if (threadIdx.x == 0) {
      part[3 * blockIdx.x] = t0;
      part[3 * blockIdx.x + 1] = t1;
      part[3 * blockIdx.x + 2] = t2;
    }
  } else if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t0;
    part[2 * blockIdx.x + 1] = t1;
  }
}

// stage 0: stat[0..1] = the mean magnitudes; stage 1: stat[2] = r (0 if a
// denominator vanishes)
__global__ void __launch_bounds__(kNccThreads)
    ncc_finalize_kernel(const double* __restrict__ part, int nb, int stage, double n, double* __restrict__ stat) {
  pdl_wait_release();
  const int w = stage == 0 ? 2 : 3;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    for (int k = 0; k < w; ++k) s[k] += part[w * b + k];
  double t[3];
  for (int k = 0; k < w; ++k) t[k] = ncc_block_sum(s[k]);
  if (threadIdx.x == 0) {
    if (stage == 0) {
      stat[0] = t[0] / n;
      stat[1] = t[1] / n;
    } else {
      const double den = sqrt(t[1]) * sqrt(t[2]);
      stat[2] = den > 0.0 ? t[0] / den : 0.0;
    }
  }
}

// Device scratch of one NCC: 3 * kNccBlocks partials and 4 scalars, on the plan.
static int ensure_ncc_scratch(mbir_plan p) {
  if (p->ncc_scratch) return MBIR_OK;
  MBIR_CUDA_TRY(cudaMalloc(&p->ncc_scratch, sizeof(double) * (3 * kNccBlocks + 4)));
  return MBIR_OK;
}

template <class R>
static int ncc_t(mbir_plan p, const void* x, const void* z, double* r, cudaStream_t st) {
  const size_t n = (size_t)p->nx * p->nz;
  size_t g = (n + kNccThreads - 1) / kNccThreads;
  const int nb = (int)(g < (size_t)kNccBlocks ? g : kNccBlocks);
  double* part = p->ncc_scratch;
  double* stat = part + 3 * kNccBlocks;
  using V = cplx_t<R>;
  const V* xv = static_cast<const V*>(x);
  const V* zv = static_cast<const V*>(z);
  {
    ProfScope ps_(p, PC_REDUCE, st);
    launch(ncc_pass_kernel<R>, dim3(nb), dim3(kNccThreads), 0, st, xv, zv, n, (const double*)nullptr, part);
  }
  { ProfScope ps_(p, PC_REDUCE, st); launch(ncc_finalize_kernel, dim3(1), dim3(kNccThreads), 0, st, (const double*)part, nb, 0, double(n), stat); }
  { ProfScope ps_(p, PC_REDUCE, st); launch(ncc_pass_kernel<R>, dim3(nb), dim3(kNccThreads), 0, st, xv, zv, n, (const double*)stat, part); }
  { ProfScope ps_(p, PC_REDUCE, st); launch(ncc_finalize_kernel, dim3(1), dim3(kNccThreads), 0, st, (const double*)part, nb, 1, double(n), stat); }
  MBIR_LAUNCH_CHECK();
  MBIR_CUDA_TRY(cudaMemcpyAsync(r, stat + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
  MBIR_CUDA_TRY(cudaStreamSynchronize(st));
  return MBIR_OK;
}

int ncc_impl(mbir_plan p, const void* x, const void* z, double* r, cudaStream_t st) {
  int rc = ensure_ncc_scratch(p);
  if (rc) return rc;
  return p->precision == MBIR_FP64 ? ncc_t<double>(p, x, z, r, st) : ncc_t<float>(p, x, z, r, st);
}

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_ncc(mbir_plan p, const void* x, const void* z, double* r, void* stream) {
  if (const int vrc = bscan_only(p, "mbir_ncc")) return vrc;
  if (!p || !x || !z || !r) return MBIR_ERR_INVALID;
  return ncc_impl(p, x, z, r, (cudaStream_t)stream);
}

int mbir_lambda_search(mbir_plan p, const void* y, const uint8_t* mask, const void* z_true,
                       const mbir_solve_opts* opts, double log10_lo, double log10_hi, int32_t n_eval, void* x,
                       mbir_lambda_search_info* info, void* stream) {
  if (!p || !y || !z_true || !opts || !x || !info || n_eval < 2) return MBIR_ERR_INVALID;
  if (const int vrc = bscan_only(p, "mbir_lambda_search")) return vrc;
  if (!isfinite(log10_lo) || !isfinite(log10_hi) || !(log10_lo < log10_hi)) return MBIR_ERR_INVALID;
  if (log10_lo < -30 || log10_hi > 30) return MBIR_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = p->precision == MBIR_FP64 ? sizeof(double2) : sizeof(float2);
  void* xs = nullptr;
  MBIR_CUDA_TRY(cudaMalloc(&xs, es * (size_t)p->nx * p->nz));
  struct Free {
    void* q;
    ~Free() { cudaFree(q); }
  } free_xs{xs};

  mbir_solve_opts o = *opts;
  double step = opts->step, scale = 0.0, best_f = -INFINITY, best_t = 0.0;
  int evals = 0;
  bool have_scale = false;
  // one evaluation: a solve at 10^t (relative), its NCC; keeps the best in x
  auto eval = [&](double t, double* f) -> int {
    const double rel = pow(10.0, t);
    int rc;
    if (!have_scale) {
      o.lambda = rel;
      o.lambda_is_relative = 1;
      mbir_solve_info si = {};
      rc = mbir_solve(p, y, mask, &o, xs, &si, stream);
      if (rc != MBIR_OK && rc != MBIR_ERR_NOT_CONVERGED) return rc;
      step = si.step;
      scale = rel > 0 ? si.lambda_used / rel : 0.0;
      have_scale = true;
    } else {
      o.lambda = scale * rel;
      o.lambda_is_relative = 0;
      o.step = step;
      rc = mbir_solve(p, y, mask, &o, xs, nullptr, stream);
      if (rc != MBIR_OK && rc != MBIR_ERR_NOT_CONVERGED) return rc;
    }
    if ((rc = ncc_impl(p, xs, z_true, f, st))) return rc;
    if (info->trace_lambda_rel) info->trace_lambda_rel[evals] = rel;
    if (info->trace_ncc) info->trace_ncc[evals] = *f;
    ++evals;
    if (*f > best_f) {
      best_f = *f;
      best_t = t;
      MBIR_CUDA_TRY(cudaMemcpyAsync(x, xs, es * (size_t)p->nx * p->nz, cudaMemcpyDeviceToDevice, st));
    }
    return MBIR_OK;
  };
  const double g = (sqrt(5.0) - 1.0) / 2.0;
  double a = log10_lo, b = log10_hi;
  double c = b - g * (b - a), d = a + g * (b - a), fc = 0.0, fd = 0.0;
  int rc = eval(c, &fc);
  if (!rc) rc = eval(d, &fd);
  while (!rc && evals < n_eval) {
    if (fc >= fd) {
      b = d;
      d = c;
      fd = fc;
      c = b - g * (b - a);
      rc = eval(c, &fc);
    } else {
      a = c;
      c = d;
      fc = fd;
      d = a + g * (b - a);
      rc = eval(d, &fd);
    }
  }
  if (rc) return rc;
  MBIR_CUDA_TRY(cudaStreamSynchronize(st));
  info->lambda_rel = pow(10.0, best_t);
  info->lambda = scale * info->lambda_rel;
  info->ncc = best_f;
  info->step = step;
  info->evaluations = evals;
  return MBIR_OK;
}

}  // extern "C"
