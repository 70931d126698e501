// Serving loop with continuous batching: B-scan reconstruction requests arrive
// at any time; each server step (tick) admits pending requests in arrival order
// while their device state fits the HBM budget, runs the set-up (power iteration,
// lambda rule) of the newly admitted ones as one batch, then advances EVERY
// active request by one FISTA iteration (Sec. 2.3, Eq. alg) in one batched pass,
// whatever iteration each one is at, and retires those that met their stopping
// rule.  Requests keep their iterates, momentum, step size and objective history
// on the device for their whole life; a request's result does not depend on the
// requests it shared ticks with.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "batch.cuh"
#include "common.cuh"

namespace mbir {

// Byte-budget admission: first come, first served, no overtaking.
class Admission {
 public:
  explicit Admission(size_t budget) : budget_(budget) {}
  bool fits(size_t b) const { return b <= budget_ && in_use_ + b <= budget_; }
  bool ever_fits(size_t b) const { return b <= budget_; }
  void take(size_t b) {
    in_use_ += b;
    peak_ = std::max(peak_, in_use_);
  }
  void give(size_t b) { in_use_ -= std::min(b, in_use_); }
  size_t in_use() const { return in_use_; }
  size_t peak() const { return peak_; }
  size_t budget() const { return budget_; }

 private:
  size_t budget_, in_use_ = 0, peak_ = 0;
};

struct Request {
  int64_t id;
  BScan s;
  size_t bytes = 0;
  int state = 0;       // 0 pending, 1 active, 2 done, 3 failed
  int status = MBIR_OK;
  double t_submit = 0, t_done = 0;
};

}  // namespace mbir

struct mbir_server_s {
  explicit mbir_server_s(size_t budget, cudaStream_t st) : adm(budget), stream(st), eng(st) {}
  mbir::Admission adm;
  cudaStream_t stream;
  mbir::Engine eng;
  std::deque<mbir::Request*> pending;
  std::vector<mbir::Request*> active;
  std::map<int64_t, mbir::Request*> all;
  int64_t next_id = 1;
  int64_t completed = 0;
  int precision = -1;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace mbir {

static int server_step(mbir_server_s* srv, int32_t* n_active, int32_t* n_pending, int32_t* n_done) {
  int done_now = 0;
  // 1. admission in arrival order while the budget allows
  std::vector<Request*> fresh;
  while (!srv->pending.empty()) {
    Request* r = srv->pending.front();
    if (!srv->adm.ever_fits(r->bytes)) {
      r->state = 3;
      r->status = MBIR_ERR_OOM;
      r->t_done = srv->now();
      srv->pending.pop_front();
      continue;
    }
    if (!srv->adm.fits(r->bytes)) break;
    const int rc = ctx_alloc(r->s.p, r->s.o.penalty, r->s.o.max_iter, &r->s.c);
    if (rc == MBIR_ERR_OOM) break;   // the device itself is full: retry next tick
    if (rc) return rc;
    srv->adm.take(r->bytes);
    r->state = 1;
    srv->pending.pop_front();
    fresh.push_back(r);
  }
  std::vector<BScan*> sc;
  for (Request* r : fresh) sc.push_back(&r->s);
  int rc = srv->eng.setup(sc);
  if (rc) return rc;
  for (Request* r : fresh) srv->active.push_back(r);
  // 2. one batched iteration for every active request
  if (!srv->active.empty()) {
    sc.clear();
    bool want_obj = false;
    for (Request* r : srv->active) {
      sc.push_back(&r->s);
      want_obj = want_obj || r->s.o.rel_tol > 0;
    }
    if ((rc = srv->eng.step(sc, want_obj))) return rc;
    if (want_obj && (rc = srv->eng.read_objectives(sc))) return rc;
    // 3. retire the requests that met their stopping rule
    std::vector<Request*> keep, finished;
    for (Request* r : srv->active) {
      const BScan& s = r->s;
      bool stop = s.k >= s.o.max_iter;
      if (!stop && s.o.rel_tol > 0 && s.k >= std::max(s.o.min_iter, 3))
        stop = fabs(s.f1 - s.f2) <= s.o.rel_tol * fabs(s.f2);
      if (stop) {
        r->status = (s.o.rel_tol > 0 && s.k >= s.o.max_iter && !(fabs(s.f1 - s.f2) <= s.o.rel_tol * fabs(s.f2)))
                        ? MBIR_ERR_NOT_CONVERGED
                        : MBIR_OK;
        if ((rc = srv->eng.finish(&r->s))) return rc;
        finished.push_back(r);
      } else {
        keep.push_back(r);
      }
    }
    if (!finished.empty()) {
      MBIR_CUDA_TRY(cudaStreamSynchronize(srv->stream));
      const double t = srv->now();
      for (Request* r : finished) {
        r->t_done = t;
        r->state = 2;
        ctx_free(&r->s.c);
        srv->adm.give(r->bytes);
        ++srv->completed;
        ++done_now;
      }
    }
    srv->active.swap(keep);
  }
  if (n_active) *n_active = (int32_t)srv->active.size();
  if (n_pending) *n_pending = (int32_t)srv->pending.size();
  if (n_done) *n_done = done_now;
  return MBIR_OK;
}

}  // namespace mbir

using namespace mbir;

extern "C" {

int mbir_server_create(size_t hbm_budget_bytes, void* stream, mbir_server* out) {
  if (!out || hbm_budget_bytes == 0) return MBIR_ERR_INVALID;
  *out = nullptr;
  mbir_server_s* s = new (std::nothrow) mbir_server_s(hbm_budget_bytes, (cudaStream_t)stream);
  if (!s) return MBIR_ERR_OOM;
  *out = s;
  return MBIR_OK;
}

void mbir_server_destroy(mbir_server srv) {
  if (!srv) return;
  cudaStreamSynchronize(srv->stream);
  for (auto& kv : srv->all) {
    ctx_free(&kv.second->s.c);
    delete kv.second;
  }
  delete srv;
}

int mbir_server_submit(mbir_server srv, mbir_plan plan, const void* y, const uint8_t* mask,
                       const mbir_solve_opts* o, void* x, int64_t* ticket) {
  if (!srv || !plan || !y || !o || !x || !ticket) return MBIR_ERR_INVALID;
  if (const int vrc = bscan_only(plan, "mbir_server_submit")) return vrc;
  if (o->max_iter < 1 || o->min_iter < 0 || o->penalty < MBIR_PENALTY_L1 || o->penalty > MBIR_PENALTY_DB4)
    return MBIR_ERR_INVALID;
  if (o->backprojection != MBIR_BACKPROJ_TRANSPOSE) return MBIR_ERR_INVALID;
  if (!(o->lambda >= 0) || !isfinite(o->lambda) || !isfinite(o->step) || !(o->rel_tol >= 0))
    return MBIR_ERR_INVALID;
  if (o->penalty == MBIR_PENALTY_DB4 && !wavelet_supported(plan->nx, plan->nz)) return MBIR_ERR_UNSUPPORTED_SIZE;
  if (srv->precision >= 0 && plan->precision != srv->precision) return MBIR_ERR_INVALID;
  srv->precision = plan->precision;
  Request* r = new (std::nothrow) Request;
  if (!r) return MBIR_ERR_OOM;
  r->id = srv->next_id++;
  r->s.p = plan;
  r->s.y = y;
  r->s.mask = mask;
  r->s.x = x;
  r->s.o = *o;
  r->bytes = ctx_bytes(plan, o->penalty, o->max_iter);
  r->t_submit = srv->now();
  srv->pending.push_back(r);
  srv->all[r->id] = r;
  *ticket = r->id;
  return MBIR_OK;
}

int mbir_server_step(mbir_server srv, int32_t* n_active, int32_t* n_pending, int32_t* n_completed) {
  if (!srv) return MBIR_ERR_INVALID;
  return server_step(srv, n_active, n_pending, n_completed);
}

int mbir_server_poll(mbir_server srv, int64_t ticket, int32_t* done, mbir_solve_info* info, double* latency_s) {
  if (!srv) return MBIR_ERR_INVALID;
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) return MBIR_ERR_INVALID;
  Request* r = it->second;
  const bool fin = r->state >= 2;
  if (done) *done = fin ? 1 : 0;
  if (fin && info) {
    info->iters = r->s.k;
    info->status = r->status;
    info->objective = r->s.f1;
    info->lipschitz = r->s.L;
    info->step = r->s.delta;
    info->lambda_used = r->s.lam;
  }
  if (latency_s) *latency_s = fin ? r->t_done - r->t_submit : srv->now() - r->t_submit;
  if (fin) {
    srv->all.erase(it);
    delete r;
  }
  return MBIR_OK;
}

int mbir_server_stats(mbir_server srv, size_t* bytes_in_use, size_t* peak_bytes, int64_t* completed) {
  if (!srv) return MBIR_ERR_INVALID;
  if (bytes_in_use) *bytes_in_use = srv->adm.in_use();
  if (peak_bytes) *peak_bytes = srv->adm.peak();
  if (completed) *completed = srv->completed;
  return MBIR_OK;
}

int mbir_server_request_bytes(mbir_plan plan, int32_t penalty, int32_t max_iter, size_t* bytes) {
  if (!plan || !bytes || max_iter < 1) return MBIR_ERR_INVALID;
  if (const int vrc = bscan_only(plan, "mbir_server_request_bytes")) return vrc;
  *bytes = ctx_bytes(plan, penalty, max_iter);
  return MBIR_OK;
}

int mbir_admission_simulate(size_t budget, int32_t n, const int64_t* bytes, const int32_t* arrive_tick,
                            const int32_t* service_ticks, int32_t* admit_tick, int32_t* done_tick,
                            int64_t* peak_bytes) {
  if (n < 0 || (n > 0 && (!bytes || !arrive_tick || !service_ticks || !admit_tick || !done_tick)))
    return MBIR_ERR_INVALID;
  Admission adm(budget);
  struct Item {
    int i;
    int left;
  };
  std::deque<int> pend;
  std::vector<Item> act;
  int next = 0, finished = 0;
  for (int i = 0; i < n; ++i) admit_tick[i] = done_tick[i] = -1;
  for (int tick = 0; finished < n && tick < (1 << 30); ++tick) {
    while (next < n && arrive_tick[next] <= tick) pend.push_back(next++);
    // the server's rule: arrival order, stop at the first that does not fit,
    // drop requests larger than the whole budget
    while (!pend.empty()) {
      const int i = pend.front();
      if (!adm.ever_fits((size_t)bytes[i])) {
        pend.pop_front();
        ++finished;
        continue;
      }
      if (!adm.fits((size_t)bytes[i])) break;
      adm.take((size_t)bytes[i]);
      admit_tick[i] = tick;
      act.push_back({i, std::max(1, service_ticks[i])});
      pend.pop_front();
    }
    std::vector<Item> keep;
    for (Item& it : act) {
      if (--it.left == 0) {
        done_tick[it.i] = tick;
        adm.give((size_t)bytes[it.i]);
        ++finished;
      } else {
        keep.push_back(it);
      }
    }
    act.swap(keep);
    if (next >= n && pend.empty() && act.empty()) break;
  }
  if (peak_bytes) *peak_bytes = (int64_t)adm.peak();
  return MBIR_OK;
}

}  // extern "C"
