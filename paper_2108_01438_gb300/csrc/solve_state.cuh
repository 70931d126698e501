// Per-plan solver state shared by the single-scan solver (solve.cu) and the
// batch engine (batch.cu).
#pragma once

#include "common.cuh"

namespace mbir {

struct SolveState {
  size_t nimg = 0, nmeas = 0;
  void* zA = nullptr;        // z^{k-1} / z^{k-2}, swapped every iteration
  void* zB = nullptr;
  void* v = nullptr;         // gradient-step image before the wavelet prox; power-iteration vector
  void* pz = nullptr;        // Phi z^{k-1} (measurement space)
  void* r = nullptr;         // residual Phi x^k - s y
  double* part_data = nullptr;   // per-CTA partial sums of the data term
  double* part_reg = nullptr;    // per-CTA partial sums of ||Psi z||_1
  double* part_tmp = nullptr;
  double* scal = nullptr;        // device scalars (power iteration, lambda, objective)
  double* objtrace = nullptr;
  void* g = nullptr;              // volume plans: the gradient image Phi^H (s Phi x - s y)
  int n_data = 0, n_reg = 0, trace_cap = 0;
};

int ensure_state(mbir_plan p, int trace_cap);
int wavelet_partial_count(int nx, int nz);
int ensure_wavelet_scratch(mbir_plan p);
// mbir_solve on a cudaStream_t; final_objective = false skips the extra forward
// pass that evaluates F(z^iters) for info (info->objective stays NaN).
int solve_plan(mbir_plan p, const void* y, const uint8_t* mask, const mbir_solve_opts* o, void* x,
               mbir_solve_info* info, cudaStream_t st, bool final_objective);

}  // namespace mbir
