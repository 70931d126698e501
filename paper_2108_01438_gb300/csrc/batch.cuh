// Batch engine shared by mbir_solve_batch (batch.cu) and the serving loop
// (serve.cu): batched set-up, one batched FISTA iteration over scans that are at
// different iteration counts, and the graph-captured fixed-count loop.
#pragma once

#include <vector>

#include "common.cuh"
#include "solve_state.cuh"

namespace mbir {

// Device buffers one reconstruction runs in: the plan's own (plan API and batch
// API) or a request's (serving), so requests sharing a geometry do not collide.
struct Ctx {
  void* wsA = nullptr;       // operator workspace [nx][max(nz, m)] complex
  void* wsB = nullptr;
  void* zA = nullptr;        // z^{k-1} / z^{k-2} images
  void* zB = nullptr;
  void* v = nullptr;         // image before the wavelet prox; power-iteration vector
  void* pz = nullptr;        // Phi z^{k-1}
  void* r = nullptr;         // residual
  void* wv_b1 = nullptr;     // wavelet level-1/2 low-low blocks and coefficients
  void* wv_b2 = nullptr;
  void* wv_coef = nullptr;
  double* part_data = nullptr;
  double* part_reg = nullptr;
  double* part_tmp = nullptr;
  double* scal = nullptr;
  double* objtrace = nullptr;
  int n_data = 0, n_reg = 0, trace_cap = 0;
  size_t nimg = 0, nmeas = 0;
  bool owned = false;
};

struct BScan {
  mbir_plan p;
  Ctx c;
  const void* y;
  const uint8_t* mask;
  void* x;
  mbir_solve_opts o;
  double L = 0, lam = 0, delta = 0, tau = 0;
  int k = 0;                 // iterations done
  double f1 = 0, f2 = 0;     // F(z^{k-1}), F(z^{k-2}) of the last two iterations
  int slot = 0;              // row of the engine's objective array
};

// Buffers of the plan itself (allocating the solver state / wavelet scratch on first use).
int plan_ctx(mbir_plan p, int penalty, int trace_cap, Ctx* out);
// Device bytes a request-owned context for plan p needs, and its allocation.
size_t ctx_bytes(mbir_plan p, int penalty, int trace_cap);
int ctx_alloc(mbir_plan p, int penalty, int trace_cap, Ctx* out);
void ctx_free(Ctx* c);

class Engine {
 public:
  explicit Engine(cudaStream_t st) : st_(st) {}
  ~Engine();
  // all scans of an engine share precision, KB width and shape
  int check(const std::vector<BScan*>& scans);
  // power iteration and lambda rule for `scans` (batched; one read-back), then the
  // FISTA start (z = 0 or the warm start, Phi z^{-1} = 0)
  int setup(const std::vector<BScan*>& scans);
  // one FISTA iteration for every scan at its own count k (advances k); with
  // want_obj the objective F(z^{k-1}) of each scan lands in its trace and in the
  // engine's objective array (read it with read_objectives)
  int step(const std::vector<BScan*>& scans, bool want_obj);
  int read_objectives(const std::vector<BScan*>& scans);
  // max_iter iterations of every scan (all equal), captured into one graph when
  // the stream allows it
  int solve_fixed(const std::vector<BScan*>& scans);
  // copy z^k of a scan to its output
  int finish(BScan* s);

 private:
  struct Stage {
    int kind;   // 0 lateral, 1 row, 2 dwt analysis, 3 dwt synthesis, 4 objective
    int mode;
    size_t arg_off, off_off;
    int n, total;
    size_t smem;
    int uses_mu;
    int blu;    // lateral stages: some scan's plan uses the Bluestein form
    int fz;     // row stages: every scan's row transform takes the fused passes
  };
  size_t push(const void* data, size_t bytes);
  void grow(size_t need);
  // start recording argument blocks into the next staging buffer of the ring,
  // waiting until that buffer's previous upload has been consumed
  int begin_build();
  int upload();
  int run(const Stage& g, double mu);
  int vec_kernel(int which, size_t off, int n);
  int build_iteration(std::vector<Stage>& out, const std::vector<BScan*>& scans, int parity_override,
                      bool per_scan_mu, bool want_obj);
  template <class F>
  int add_lateral(std::vector<Stage>& out, int mode, const std::vector<BScan*>& idx, F make, bool uses_mu);
  int add_row(std::vector<Stage>& out, bool adjoint, const std::vector<BScan*>& idx);
  int add_dwt(std::vector<Stage>& out, int inverse, int level, const std::vector<BScan*>& idx,
              const std::vector<const void*>& in, const std::vector<void*>& outp,
              const std::vector<void*>& coefs, const std::vector<double*>& partial, bool thresh);

  cudaStream_t st_;
  int prec_ = -1, J_ = 6;
  double alpha_ = 0;
  bool gather_ = true;
  size_t esz_ = 8, rsz_ = 4;
  // Host staging ring: an upload is an async copy from a pinned buffer, so a
  // buffer is rewritten only after the event recorded behind its last copy.
  static constexpr int kRing = 3;
  struct Staging {
    unsigned char* h = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
  };
  Staging ring_[kRing];
  int cur_ = 0;
  unsigned char* hbuf_ = nullptr;
  size_t hlen_ = 0, hcap_ = 0;
  bool grow_failed_ = false;
  void* dbuf_ = nullptr;
  size_t dcap_ = 0;
  double* dobj_ = nullptr;     // objective per engine slot
  int dobj_cap_ = 0;
  std::vector<double> hobj_;
};

}  // namespace mbir
