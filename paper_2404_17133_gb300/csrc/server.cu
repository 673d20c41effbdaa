// Serving: continuous admission of independent solves under a device-memory
// budget.  Host-only code; every solve runs through the context API of
// capi.cu, each admitted request on its slot's own stream so that the kernels
// of different requests overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "ctx.cuh"
#include "small.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Entry {
  tddft_serve_request* r = nullptr;
  unsigned long long bytes = 0;
  bool done = false;
  tddft_status status = TDDFT_PENDING;
};

struct Server {
  int device = 0;
  unsigned long long budget = 0, in_use = 0, peak_in_use = 0;
  int max_active = 1, active = 0;
  bool stopping = false;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_admit, cv_done;
  std::deque<unsigned long long> queue;
  std::map<unsigned long long, Entry> entries;
  unsigned long long next_ticket = 1, n_done = 0;
  std::vector<std::thread> slots;
  std::vector<cudaStream_t> streams;
  cudaMemPool_t pool = nullptr;
  unsigned long long pool_used0 = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

int work_vectors(const tddft_serve_request& q) {
  if (q.kind == 2) return std::max(1, q.req.n_dip * q.req.n_freq);
  int extra = q.req.opts.n_extra_guess >= 0 ? q.req.opts.n_extra_guess
                                            : std::min(q.req.opts.n_states, 3);
  return std::max(1, q.req.opts.n_states + extra);
}

void copy_error(tddft_serve_request* r, const char* msg) {
  std::strncpy(r->error, msg ? msg : "", sizeof(r->error) - 1);
  r->error[sizeof(r->error) - 1] = 0;
}

tddft_status run_one(tddft_serve_request* q, cudaStream_t s) {
  tddft_ctx* ctx = q->ctx;
  bool own = false;
  if (!ctx) {
    tddft_status st = tddft_create(&q->desc, q->eps_occ, q->eps_vir, q->L_oo, q->L_ov, q->L_vv, q->Lr_oo,
                                   q->Lr_ov, q->Lr_vv, q->ris_K_index, q->dtype, q->inputs_on_device, s, &ctx);
    if (st != TDDFT_OK) {
      copy_error(q, tddft_last_error(nullptr));
      return st;
    }
    own = true;
  }
  tddft_request& r = q->req;
  tddft_status st;
  if (q->kind == 0) st = tddft_solve_tda(ctx, &r.opts, r.omega, r.X, r.resid, &r.stats);
  else if (q->kind == 1) st = tddft_solve_rpa(ctx, &r.opts, r.omega, r.X, r.Y, r.resid, &r.stats);
  else st = tddft_solve_polar(ctx, &r.opts, r.mu, r.n_dip, r.freqs, r.n_freq, r.alpha, &r.stats);
  if (st != TDDFT_OK) copy_error(q, tddft_last_error(ctx));
  if (own) tddft_destroy(ctx);
  return st;
}

void slot_loop(Server* sv, int slot) {
  cudaSetDevice(sv->device);
  cudaStream_t s = sv->streams[slot];
  for (;;) {
    unsigned long long t;
    tddft_serve_request* q;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      // first in, first out: the oldest request starts once its estimate fits
      sv->cv_admit.wait(lk, [&] {
        if (sv->stopping && sv->queue.empty()) return true;
        if (sv->queue.empty()) return false;
        const Entry& e = sv->entries[sv->queue.front()];
        return sv->in_use + e.bytes <= sv->budget;
      });
      if (sv->queue.empty()) return;   // stopping
      t = sv->queue.front();
      sv->queue.pop_front();
      Entry& e = sv->entries[t];
      q = e.r;
      sv->in_use += e.bytes;
      sv->peak_in_use = std::max(sv->peak_in_use, sv->in_use);
      ++sv->active;
      q->t_start_s = sv->now();
    }
    sv->cv_admit.notify_all();   // the next request may fit as well
    tddft_status st;
    try {
      st = run_one(q, s);
    } catch (const std::exception& ex) {
      copy_error(q, ex.what());
      st = TDDFT_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      Entry& e = sv->entries[t];
      q->t_end_s = sv->now();
      sv->in_use -= e.bytes;
      --sv->active;
      e.status = st;
      e.done = true;
      ++sv->n_done;
    }
    sv->cv_admit.notify_all();
    sv->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

tddft_status tddft_estimate_bytes(const tddft_desc* desc, int kind, const tddft_opts* opts, int n_dip,
                                  int n_freq, unsigned long long* factor_bytes,
                                  unsigned long long* work_bytes) {
  if (!desc || !opts || kind < 0 || kind > 2) return TDDFT_ERR_ARG;
  const tddft_desc& d = *desc;
  if (d.n_occ < 1 || d.n_vir < 1 || d.n_aux < 1) return TDDFT_ERR_ARG;
  if (factor_bytes) *factor_bytes = tddft::factor_copy_bytes(d);
  if (work_bytes) {
    tddft_serve_request q;
    std::memset(&q, 0, sizeof(q));
    q.kind = kind;
    q.req.opts = *opts;
    q.req.n_dip = n_dip;
    q.req.n_freq = n_freq;
    const double ov = (double)d.n_occ * d.n_vir;
    const double k = work_vectors(q);
    const double cap = opts->max_subspace > 0 ? std::min(opts->max_subspace, tddft::kSmallMax)
                                              : tddft::kSmallMax;
    const double inner_es = opts->precision == TDDFT_MIXED ? 4.0 : 8.0;
    // Outer subspace (paired: V, U, W of cap rows in FP64) and its ~24 k-row
    // work vectors; the rid inner space (cap + 2k rows and ~24 k-row vectors in
    // the inner precision); operator intermediates (at most three P-chunks of
    // 512 MiB, fewer for small problems); 64 MiB for the small algebra.
    const double outer = 8.0 * ov * (3.0 * cap + 24.0 * k);
    const double inner = opts->precond == TDDFT_PRECOND_RID ? inner_es * ov * (4.0 * cap + 26.0 * k) : 0.0;
    const double inter = 3.0 * std::min(512.0 * 1048576.0, (double)d.n_aux * cap * ov * 8.0);
    *work_bytes = (unsigned long long)(outer + inner + inter + 64.0 * 1048576.0);
  }
  return TDDFT_OK;
}

tddft_status tddft_server_create(double hbm_budget_gb, int max_active, tddft_server** out) {
  if (!out || max_active < 1 || max_active > 64 || !(hbm_budget_gb >= 0.0)) return TDDFT_ERR_ARG;
  *out = nullptr;
  Server* sv = new Server();
  try {
    TD_CUDA(cudaGetDevice(&sv->device));
    size_t fr = 0, tot = 0;
    TD_CUDA(cudaMemGetInfo(&fr, &tot));
    const double cap = (double)fr - 2e9;
    sv->budget = (unsigned long long)(hbm_budget_gb > 0 ? std::min(hbm_budget_gb * 1e9, cap) : cap);
    sv->max_active = max_active;
    sv->t0 = Clock::now();
    // the device's stream-ordered pool serves every work buffer: record its use
    // now and restart its high-water mark, so state->pool_high_bytes measures
    // what the requests really took
    TD_CUDA(cudaDeviceGetDefaultMemPool(&sv->pool, sv->device));
    uint64_t used = 0;
    TD_CUDA(cudaMemPoolGetAttribute(sv->pool, cudaMemPoolAttrUsedMemCurrent, &used));
    sv->pool_used0 = used;
    uint64_t zero = 0;
    TD_CUDA(cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrUsedMemHigh, &zero));
    for (int i = 0; i < max_active; ++i) {
      cudaStream_t s;
      TD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      sv->streams.push_back(s);
    }
    for (int i = 0; i < max_active; ++i) sv->slots.emplace_back(slot_loop, sv, i);
  } catch (const std::exception&) {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stopping = true;
    }
    sv->cv_admit.notify_all();
    for (auto& th : sv->slots)
      if (th.joinable()) th.join();
    for (auto s : sv->streams) cudaStreamDestroy(s);
    delete sv;
    return TDDFT_ERR_CUDA;
  }
  *out = reinterpret_cast<tddft_server*>(sv);
  return TDDFT_OK;
}

tddft_status tddft_server_submit(tddft_server* server, tddft_serve_request* req, unsigned long long* ticket) {
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv || !req || !ticket || req->kind < 0 || req->kind > 2) return TDDFT_ERR_ARG;
  req->error[0] = 0;
  req->t_start_s = req->t_end_s = 0.0;
  unsigned long long fb = 0, wb = 0;
  if (!req->ctx) {
    tddft_status st = tddft_estimate_bytes(&req->desc, req->kind, &req->req.opts, req->req.n_dip,
                                           req->req.n_freq, &fb, &wb);
    if (st != TDDFT_OK) {
      copy_error(req, "bad tddft_desc or request kind");
      return st;
    }
  } else {
    // the context's factors are already resident: charge the solve's workspace only
    tddft_desc d;
    tddft_ctx_desc(req->ctx, &d);
    tddft_status st = tddft_estimate_bytes(&d, req->kind, &req->req.opts, req->req.n_dip, req->req.n_freq,
                                           nullptr, &wb);
    if (st != TDDFT_OK) {
      copy_error(req, "bad request kind");
      return st;
    }
  }
  req->charged_bytes = fb + wb;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (req->charged_bytes > sv->budget) {
    copy_error(req, "request needs more device memory than the server's whole budget");
    return TDDFT_ERR_OOM;
  }
  if (sv->stopping) return TDDFT_ERR_BUSY;
  if (sv->queue.size() >= 65536) return TDDFT_ERR_BUSY;
  unsigned long long t = sv->next_ticket++;
  Entry e;
  e.r = req;
  e.bytes = req->charged_bytes;
  sv->entries[t] = e;
  sv->queue.push_back(t);
  req->t_submit_s = sv->now();
  *ticket = t;
  sv->cv_admit.notify_all();
  return TDDFT_OK;
}

tddft_status tddft_server_poll(tddft_server* server, unsigned long long ticket, int timeout_ms) {
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv) return TDDFT_ERR_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->entries.find(ticket);
  if (it == sv->entries.end()) return TDDFT_ERR_ARG;
  if (!it->second.done && timeout_ms > 0) {
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
      auto j = sv->entries.find(ticket);
      return j != sv->entries.end() && j->second.done;
    });
    it = sv->entries.find(ticket);
  }
  if (!it->second.done) return timeout_ms > 0 ? TDDFT_ERR_TIMEOUT : TDDFT_PENDING;
  tddft_status st = it->second.status;
  sv->entries.erase(it);
  return st;
}

tddft_status tddft_server_info(const tddft_server* server, tddft_server_state* st) {
  Server* sv = reinterpret_cast<Server*>(const_cast<tddft_server*>(server));
  if (!sv || !st) return TDDFT_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  st->budget_bytes = sv->budget;
  st->in_use_bytes = sv->in_use;
  st->peak_in_use_bytes = sv->peak_in_use;
  st->active = sv->active;
  st->max_active = sv->max_active;
  st->queued = (int)sv->queue.size();
  st->completed = sv->n_done;
  uint64_t high = 0;
  if (cudaMemPoolGetAttribute(sv->pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess) return TDDFT_ERR_CUDA;
  st->pool_used_at_create_bytes = sv->pool_used0;
  st->pool_high_bytes = high;
  return TDDFT_OK;
}

void tddft_server_destroy(tddft_server* server) {
  Server* sv = reinterpret_cast<Server*>(server);
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
  }
  sv->cv_admit.notify_all();
  for (auto& th : sv->slots)
    if (th.joinable()) th.join();
  for (auto s : sv->streams) {
    cudaStreamSynchronize(s);
    tddft::pool_trim(s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete sv;
}

}  // extern "C"
