// Continuous-batching server: CC solves submitted at any time are admitted as soon as a
// slot and device memory are free, run concurrently on the device (one stream and one
// memory pool per slot, so kernels of different requests overlap), and complete
// independently. Every kernel is deterministic, so a request's result does not depend on
// what else runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "handles.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int o = 0, v = 0, naux = 0;
  std::vector<double> fock, B;  // host copies taken at submit
  cc_solve_opts opts{};
  size_t footprint = 0;  // admission estimate (bytes)
  double cost = 0;       // work estimate of one residual evaluation ((naux + o^2) v^4)
  // results
  bool done = false, released = false;
  int status = CC_PENDING;
  cc_report report{};
  std::vector<double> t1, t2;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  std::string err;
  std::atomic<int> cancel{0};  // set by cc_serve_cancel; a running solve stops at its next iteration
};

// Device bytes a solve is expected to hold: the resident problem, the engine's intermediates
// and tangents, the ladder slab, the Krylov bases (outer and inner) and the tensor-core staging.
size_t footprint_bytes(int o, int v, int naux, const cc_solve_opts& op) {
  const double n = o + v, ov = (double)o * v, oovv = ov * ov;
  const double namp = ov + oovv;
  const double lb = ccpnk::ladder_block_for(v);
  double doubles = 0;
  doubles += 3.0 * naux * n * n;                            // B (upload, blocks)
  doubles += 36.0 * oovv + 8.0 * naux * n * n;              // engine values + tangents
  doubles += 2.0 * lb * v * v * v;                          // ladder slab and its (c, d) split
  if (op.prec != CC_FP64 && op.prec != CC_DF64 && op.prec != CC_FP64_EMU) {  // its tensor-core staging copy,
    doubles += std::ceil(lb * v / 256.0) * 256.0 * 3.0 * std::ceil((double)v * v / 64.0) * 64.0 / 2.0;
    doubles += ccpnk::stage_cache_cap(o, v, naux) / 8.0;    // and kept value-side operands
  }
  doubles += (op.m_max + 8.0) * namp;                       // outer Krylov basis and vectors
  doubles += (op.af_direct ? 2.0 : (op.inner_max + 2.0)) * namp;  // A_F inverse work
  doubles += 4.0 * oovv;                                    // split-k partials, staging
  if (op.prec == CC_FP64_EMU || op.outer_prec == CC_FP64_EMU)  // digit slices and exact partial sums
    doubles += 2.0 * lb * v * v * v + 8.0 * naux * v * v;
  return (size_t)(doubles * 8.0 * 1.15) + (64u << 20);
}

}  // namespace

struct cc_server {
  int device = 0;
  size_t budget = 0;  // 0: no limit
  int max_slots = 1;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  int running = 0, max_running = 0;
  bool stop = false;
  int group_max = 1;  // > 1: a slot solves up to this many compatible requests together
  int policy = CC_SERVE_FIFO;
  std::vector<std::thread> workers;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// The waiting request a free slot takes next (called with the lock held, queue not empty):
// the oldest (FIFO), or the one with the least work, its estimate divided by (1 + seconds
// waited) so that a large request is not passed over for ever (shortest first).
std::deque<Request*>::iterator next_request(cc_server* srv) {
  if (srv->policy != CC_SERVE_SHORTEST_FIRST) return srv->queue.begin();
  const double now = srv->now();
  auto best = srv->queue.begin();
  double bv = 1e300;
  for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it) {
    const double v = (*it)->cost / (1.0 + std::max(0.0, now - (*it)->t_submit));
    if (v < bv) {
      bv = v;
      best = it;
    }
  }
  return best;
}

// Requests a slot may solve together: NK or PNK with identical options (so one lockstep batch
// runs them all exactly as each would run alone).
bool groupable(const Request& a, const Request& b) {
  const cc_solve_opts &x = a.opts, &y = b.opts;
  return (x.method == CC_NK || x.method == CC_PNK) && x.method == y.method && x.prec == y.prec && x.tol == y.tol &&
         x.max_outer == y.max_outer && x.m_max == y.m_max && x.gamma == y.gamma && x.alpha == y.alpha &&
         x.eta_max == y.eta_max && x.jvp_fd == 0 && y.jvp_fd == 0 && x.inner_rtol == y.inner_rtol &&
         x.inner_max == y.inner_max && x.af_direct == y.af_direct && x.ccd == y.ccd &&
         x.max_seconds == y.max_seconds && x.outer_prec == y.outer_prec;
}

// Posts a finished request's result (called with the server's lock held).
void post(cc_server* srv, Request* r, int status, const cc_report& rep, std::vector<double>& t1,
          std::vector<double>& t2, const std::string& err) {
  r->status = status;
  r->report = rep;
  r->t1.swap(t1);
  r->t2.swap(t2);
  r->err = err;
  r->t_finish = srv->now();
  r->done = true;
  r->fock.clear();
  r->fock.shrink_to_fit();
  r->B.clear();
  r->B.shrink_to_fit();
  srv->in_use -= r->footprint;
  srv->running -= 1;
}

void worker_main(cc_server* srv, int slot) {
  (void)slot;
  cudaSetDevice(srv->device);
  cc_ctx* ctx = nullptr;
  int st = cc_ctx_create(&ctx, srv->device, 0, nullptr);
  for (;;) {
    std::vector<Request*> batch;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      // admission: the request the policy puts first goes once its memory estimate fits
      srv->cv.wait(lk, [&] {
        if (srv->stop) return true;
        if (srv->queue.empty()) return false;
        Request* h = *next_request(srv);
        return srv->budget == 0 || srv->in_use + h->footprint <= srv->budget || srv->running == 0;
      });
      if (srv->stop) break;
      auto head = next_request(srv);
      batch.push_back(*head);
      srv->queue.erase(head);
      if (srv->policy == CC_SERVE_SHORTEST_FIRST)  // group the cheapest compatible ones with it
        std::stable_sort(srv->queue.begin(), srv->queue.end(), [](const Request* a, const Request* b) {
          return a->cost < b->cost;
        });
      size_t fp = batch[0]->footprint;
      // grouped mode: later waiting requests that can run in the same lockstep batch and fit
      for (auto it = srv->queue.begin(); (int)batch.size() < srv->group_max && it != srv->queue.end();) {
        Request* c = *it;
        if (groupable(*batch[0], *c) && (srv->budget == 0 || srv->in_use + fp + c->footprint <= srv->budget)) {
          fp += c->footprint;
          batch.push_back(c);
          it = srv->queue.erase(it);
        } else {
          ++it;
        }
      }
      for (Request* r : batch) {
        srv->in_use += r->footprint;
        srv->running += 1;
        r->t_admit = srv->now();
      }
      srv->max_running = std::max(srv->max_running, srv->running);
    }
    const int nb = (int)batch.size();
    std::vector<std::vector<double>> t1(nb), t2(nb);
    for (int k = 0; k < nb; ++k) {
      t1[k].assign((size_t)batch[k]->o * batch[k]->v, 0.0);
      t2[k].assign((size_t)batch[k]->o * batch[k]->o * batch[k]->v * batch[k]->v, 0.0);
    }
    if (st != CC_OK || !ctx) {
      std::lock_guard<std::mutex> lk(srv->mu);
      for (int k = 0; k < nb; ++k) post(srv, batch[k], CC_ERR_CUDA, cc_report{}, t1[k], t2[k], "no device context for this slot");
      srv->cv.notify_all();
      continue;
    }
    // the problems (a request whose input the library rejects fails on its own)
    std::vector<cc_sys*> sys(nb, nullptr);
    std::vector<int> live;
    for (int k = 0; k < nb; ++k) {
      Request* r = batch[k];
      const int cs = cc_sys_create(ctx, r->o, r->v, r->naux, r->fock.data(), r->B.data(), &sys[k]);
      if (cs == CC_OK) {
        live.push_back(k);
      } else {
        std::lock_guard<std::mutex> lk(srv->mu);
        post(srv, r, cs, cc_report{}, t1[k], t2[k], cc_last_error(ctx));
        srv->cv.notify_all();
      }
    }
    if (live.size() == 1) {
      const int k = live[0];
      Request* r = batch[k];
      cc_report rep{};
      const int status = ccpnk::solve_cancellable(ctx, sys[k], &r->opts, t1[k].data(), t2[k].data(), 0, &rep, &r->cancel);
      std::string err;
      if (status < 0 && status != CC_ERR_NOT_CONVERGED && status != CC_ERR_DIVERGED && status != CC_ERR_CANCELLED)
        err = cc_last_error(ctx);
      std::lock_guard<std::mutex> lk(srv->mu);
      post(srv, r, status, rep, t1[k], t2[k], err);
    } else if (!live.empty()) {
      // one lockstep batch; each request is posted as soon as it has finished
      const int nl = (int)live.size();
      std::vector<cc_sys*> ls;
      std::vector<double*> p1, p2;
      std::vector<const std::atomic<int>*> cancels;
      std::vector<cc_report> reps(nl);
      for (int k : live) {
        ls.push_back(sys[k]);
        p1.push_back(t1[k].data());
        p2.push_back(t2[k].data());
        cancels.push_back(&batch[k]->cancel);
      }
      auto notify = [&](int j, int status) {
        const int k = live[j];
        std::lock_guard<std::mutex> lk(srv->mu);
        post(srv, batch[k], status, reps[j], t1[k], t2[k], "");
        srv->cv.notify_all();
      };
      const int bs = ccpnk::solve_batch_notify(ctx, nl, ls.data(), &batch[live[0]]->opts, p1.data(), p2.data(),
                                               reps.data(), notify, &cancels);
      if (bs != CC_OK) {  // the batch itself failed: every request not yet posted gets its error
        std::lock_guard<std::mutex> lk(srv->mu);
        for (int k : live)
          if (!batch[k]->done) post(srv, batch[k], bs, cc_report{}, t1[k], t2[k], cc_last_error(ctx));
      }
    }
    for (cc_sys* s : sys)
      if (s) cc_sys_destroy(s);
    srv->cv.notify_all();
  }
  if (ctx) cc_ctx_destroy(ctx);
}

}  // namespace

extern "C" {

int cc_server_create(cc_server** out, int device, size_t mem_budget, int max_slots) {
  if (!out || max_slots < 1) return CC_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return CC_ERR_INVALID;
  std::unique_ptr<cc_server> s(new cc_server);
  s->device = device;
  s->budget = mem_budget;
  s->max_slots = max_slots;
  s->t0 = Clock::now();
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_main, s.get(), i);
  *out = s.release();
  return CC_OK;
}

void cc_server_destroy(cc_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  for (auto& w : srv->workers) w.join();
  delete srv;
}

int cc_serve_submit(cc_server* srv, int o, int v, int naux, const double* fock, const double* B,
                    const cc_solve_opts* opts, uint64_t* ticket) {
  if (!srv || !fock || !B || !opts || !ticket || o < 1 || v < 1 || naux < 1) return CC_ERR_INVALID;
  std::unique_ptr<Request> r(new Request);
  const size_t n = (size_t)o + v;
  r->o = o;
  r->v = v;
  r->naux = naux;
  r->fock.assign(fock, fock + n * n);
  r->B.assign(B, B + (size_t)naux * n * n);
  r->opts = *opts;
  r->footprint = footprint_bytes(o, v, naux, *opts);
  r->cost = ((double)naux + (double)o * o) * std::pow((double)v, 4.0);
  if (srv->budget && r->footprint > srv->budget) return CC_ERR_OOM;  // never admissible
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    r->ticket = srv->next_ticket++;
    r->t_submit = srv->now();
    *ticket = r->ticket;
    srv->queue.push_back(r.get());
    srv->all[r->ticket] = std::move(r);
  }
  srv->cv.notify_all();
  return CC_OK;
}

int cc_serve_poll(cc_server* srv, uint64_t ticket, cc_report* report, double* t1, double* t2) {
  if (!srv) return CC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end() || it->second->released) return CC_ERR_INVALID;
  Request* r = it->second.get();
  if (!r->done) return CC_PENDING;
  if (report) *report = r->report;
  if (t1) memcpy(t1, r->t1.data(), r->t1.size() * sizeof(double));
  if (t2) memcpy(t2, r->t2.data(), r->t2.size() * sizeof(double));
  r->released = true;
  r->t1.clear();
  r->t1.shrink_to_fit();
  r->t2.clear();
  r->t2.shrink_to_fit();
  return r->status;
}

int cc_server_set_policy(cc_server* srv, int policy) {
  if (!srv || (policy != CC_SERVE_FIFO && policy != CC_SERVE_SHORTEST_FIRST)) return CC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->policy = policy;
  return CC_OK;
}

int cc_server_set_grouping(cc_server* srv, int group_max) {
  if (!srv || group_max < 1 || group_max > 64) return CC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->group_max = group_max;
  return CC_OK;
}

int cc_serve_cancel(cc_server* srv, uint64_t ticket) {
  if (!srv) return CC_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end() || it->second->released) return CC_ERR_INVALID;
    Request* r = it->second.get();
    if (r->done) return CC_OK;  // finished already: its own status stands
    auto q = std::find(srv->queue.begin(), srv->queue.end(), r);
    if (q != srv->queue.end()) {  // still waiting: drop it without running
      srv->queue.erase(q);
      r->status = CC_ERR_CANCELLED;
      r->report = cc_report{};
      r->report.status = CC_ERR_CANCELLED;
      r->t1.assign((size_t)r->o * r->v, 0.0);
      r->t2.assign((size_t)r->o * r->o * r->v * r->v, 0.0);
      r->t_admit = r->t_finish = srv->now();
      r->done = true;
      r->fock.clear();
      r->fock.shrink_to_fit();
      r->B.clear();
      r->B.shrink_to_fit();
    } else {
      r->cancel.store(1);  // running: the solve stops between outer iterations
    }
  }
  srv->cv.notify_all();
  return CC_OK;
}

int cc_serve_times(cc_server* srv, uint64_t ticket, double* t_submit, double* t_admit, double* t_finish) {
  if (!srv) return CC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) return CC_ERR_INVALID;
  Request* r = it->second.get();
  if (t_submit) *t_submit = r->t_submit;
  if (t_admit) *t_admit = r->t_admit;
  if (t_finish) *t_finish = r->t_finish;
  return r->done ? CC_OK : CC_PENDING;
}

int cc_server_stats(cc_server* srv, int* running, int* queued, int* max_running, size_t* bytes_admitted) {
  if (!srv) return CC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (running) *running = srv->running;
  if (queued) *queued = (int)srv->queue.size();
  if (max_running) *max_running = srv->max_running;
  if (bytes_admitted) *bytes_admitted = srv->in_use;
  return CC_OK;
}

}  // extern "C"
