// The C ABI (include/ccpnk.h): contexts, resident problems, residual / JVP / A_F entry
// points and the solver. Every entry point converts exceptions into a status code and a
// per-context error message; no exception crosses the ABI.
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>

#include "handles.h"


namespace ccpnk {

void fail(int status, const std::string& msg) { throw Error{status, msg}; }

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) fail(CC_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    fail(CC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

Pool::~Pool() {
  for (auto& b : blocks_) cudaFree(b.p);
}

void* Pool::get(size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  // best fit among free blocks no more than twice the request
  int best = -1;
  for (size_t i = 0; i < blocks_.size(); ++i) {
    const Block& b = blocks_[i];
    if (!b.used && !b.pins && b.bytes >= bytes && b.bytes <= 2 * bytes + 4096 &&
        (best < 0 || b.bytes < blocks_[best].bytes))
      best = (int)i;
  }
  if (best >= 0) {
    blocks_[best].used = true;
    if (record) record->push_back(blocks_[best].p);
    return blocks_[best].p;
  }
  if (budget_ && held_ + bytes > budget_) release_free();
  if (budget_ && held_ + bytes > budget_)
    fail(CC_ERR_OOM, "device memory budget exceeded (" + std::to_string(held_ + bytes) + " > " +
                         std::to_string(budget_) + " bytes)");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_free();
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(CC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
  }
  blocks_.push_back({p, bytes, true, 0});
  held_ += bytes;
  if (record) record->push_back(p);
  return p;
}

void Pool::pin(void* p) {
  for (auto& b : blocks_)
    if (b.p == p) b.pins += 1;
}

void Pool::unpin(void* p) {
  for (auto& b : blocks_)
    if (b.p == p && b.pins > 0) b.pins -= 1;
}

void Pool::put(void* p) {
  for (auto& b : blocks_)
    if (b.p == p) {
      b.used = false;
      return;
    }
}

void Exec::mark_begin(cudaEvent_t* a) const {
  CC_CUDA(cudaEventCreate(a));
  CC_CUDA(cudaEventRecord(*a, stream));
}

void Exec::mark_end(const char* tag, cudaEvent_t a, double flops) const {
  cudaEvent_t b;
  CC_CUDA(cudaEventCreate(&b));
  CC_CUDA(cudaEventRecord(b, stream));
  prof->pending.push_back({tag, a, b, flops});
}

void Prof::resolve() {
  for (auto& r : pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    Sum* s = nullptr;
    for (auto& d : done)
      if (d.first == r.tag) s = &d.second;
    if (!s) {
      done.push_back({r.tag, Sum{}});
      s = &done.back().second;
    }
    s->launches += 1;
    s->ms += ms;
    s->flops += r.flops;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  pending.clear();
}

void Prof::reset() {
  for (auto& r : pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  pending.clear();
  done.clear();
}

void Pool::release_free() {
  std::vector<Block> keep;
  for (auto& b : blocks_) {
    if (b.used || b.pins) keep.push_back(b);
    else {
      cudaFree(b.p);
      held_ -= b.bytes;
    }
  }
  blocks_.swap(keep);
}

}  // namespace ccpnk

using namespace ccpnk;

namespace {

// Reads and clears the device error flag after the context's work has completed.
void check_device_flag(cc_ctx* ctx) {
  if (!ctx || !ctx->dflag) return;
  int h = 0;
  CC_CUDA(cudaMemcpyAsync(&h, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CC_CUDA(cudaStreamSynchronize(ctx->stream));
  if (h) {
    CC_CUDA(cudaMemsetAsync(ctx->dflag, 0, sizeof(int), ctx->stream));
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    fail(CC_ERR_TIMEOUT, "a bounded device wait gave up (tensor-core pipeline)");
  }
}

template <typename F>
int guarded(cc_ctx* ctx, F&& f) {
  try {
    if (ctx) CC_CUDA(cudaSetDevice(ctx->device));
    int st = f();
    check_device_flag(ctx);
    return st;
  } catch (const Error& e) {
    if (ctx) ctx->err = e.msg;
    return e.status;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    return CC_ERR_CUDA;
  }
}

bool is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_in(cc_ctx* ctx, double* dst, const double* src, size_t n) {
  if (!n) return;
  CC_REQUIRE(src, CC_ERR_INVALID, "NULL input pointer");
  CC_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), is_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          ctx->stream));
}

void copy_out(cc_ctx* ctx, double* dst, const double* src, size_t n) {
  if (!n || !dst) return;
  CC_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), is_device(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          ctx->stream));
}

Engine& engine(cc_sys* sys) {
  if (!sys->eng) sys->eng.reset(new Engine(sys->ctx->ex(), sys->s));
  else sys->eng->rebind(sys->ctx->ex());  // the context's options may have changed
  return *sys->eng;
}

void check_prec(cc_precision p) {
  CC_REQUIRE(p == CC_FP64 || p == CC_MIXED_TF32 || p == CC_MIXED_TF32X3 || p == CC_MIXED_BF16X3 || p == CC_DF64 ||
                 p == CC_FP64_EMU,
             CC_ERR_INVALID, "unknown precision");
}

// Precision of the value-side intermediates a JVP linearises around: FP64 for the FP64 and
// double-float JVPs, the tensor-core FP64 emulation (FP64-accurate) for the other precisions.
cc_precision value_prec(cc_precision prec) {
  return prec == CC_FP64 || prec == CC_DF64 ? CC_FP64 : CC_FP64_EMU;
}

// [t1 | t2] with t2 symmetrised: T2 only depends on t_ij^ab + t_ji^ba
void load_amplitudes(cc_ctx* ctx, const System& s, const double* t1, const double* t2, double* dst) {
  const size_t ov = (size_t)s.o * s.v;
  copy_in(ctx, dst, t1, ov);
  DBuf<double> raw(ctx->pool.get(), s.namp() - ov);
  copy_in(ctx, raw.p, t2, s.namp() - ov);
  Exec ex = ctx->ex();
  k_sym_add(ex, s.o, s.v, raw.p, dst + ov, 0.0);
  k_scale(ex, s.namp() - ov, 0.5, dst + ov);
}

}  // namespace

extern "C" {

void cc_solve_opts_default(cc_solve_opts* o, cc_method method, cc_precision prec) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->method = method;
  o->prec = prec;
  o->tol = 1e-8;
  o->max_outer = method == CC_FP_DIIS ? 500 : 100;
  o->m_max = 30;
  o->gamma = 0.9;
  o->alpha = 1.5;
  o->eta_max = 0.9;
  o->level_shift = 0.0;
  o->diis_size = 8;
  o->jvp_fd = 0;
  o->inner_rtol = prec == CC_MIXED_TF32 ? 1e-6 : prec == CC_MIXED_BF16X3 ? 1e-7 : prec == CC_MIXED_TF32X3 ? 1e-8 : 1e-12;
  o->inner_max = 50;
  o->af_direct = 0;
  o->verbose = 0;
}

int cc_ctx_create(cc_ctx** out, int device, size_t mem_budget, void* stream) {
  if (!out) return CC_ERR_INVALID;
  *out = nullptr;
  std::unique_ptr<cc_ctx> c(new cc_ctx);
  c->device = device;
  int st = guarded(c.get(), [&]() {
    int ndev = 0;
    CC_CUDA(cudaGetDeviceCount(&ndev));
    CC_REQUIRE(device >= 0 && device < ndev, CC_ERR_INVALID, "no such device");
    CC_CUDA(cudaSetDevice(device));
    CC_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    if (stream) {
      c->stream = (cudaStream_t)stream;
    } else {
      CC_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    c->pool.reset(new Pool(mem_budget));
    CC_CUDA(cudaMalloc(&c->dflag, sizeof(int)));
    CC_CUDA(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->stream));
    CC_CUDA(cudaStreamSynchronize(c->stream));
    return CC_OK;
  });
  if (st == CC_OK) *out = c.release();
  return st;
}

void cc_ctx_destroy(cc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  ctx->pool.reset();
  if (ctx->dflag) cudaFree(ctx->dflag);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* cc_last_error(const cc_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

size_t cc_ctx_device_bytes(const cc_ctx* ctx) { return ctx && ctx->pool ? ctx->pool->held() : 0; }

uint64_t cc_ctx_launches(const cc_ctx* ctx) { return ctx ? ctx->launches : 0; }

uint64_t cc_ctx_launch_calls(const cc_ctx* ctx) { return ctx ? ctx->launch_calls : 0; }

int cc_ctx_set_option(cc_ctx* ctx, int option, long long value) {
  if (!ctx) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    if (option == CC_OPT_STAGE_CACHE_BYTES) {
      CC_REQUIRE(value >= -1, CC_ERR_INVALID, "CC_OPT_STAGE_CACHE_BYTES: -1 (default) or a byte count");
      ctx->stage_cap = value;
    } else if (option == CC_OPT_WAIT_LIMIT_NS) {
      CC_REQUIRE(value >= 100000, CC_ERR_INVALID, "CC_OPT_WAIT_LIMIT_NS: at least 1e5 ns");
      ctx->wait_ns = (unsigned long long)value;
    } else if (option == CC_OPT_EMU_CHUNK) {
      CC_REQUIRE(value >= 1 && value <= 64, CC_ERR_INVALID, "CC_OPT_EMU_CHUNK: 1 to 64 k blocks");
      ctx->emu_chunk = (int)value;
    } else if (option == CC_OPT_EMU_ONCHIP) {
      CC_REQUIRE(value >= -1 && value <= 1, CC_ERR_INVALID, "CC_OPT_EMU_ONCHIP: -1 (by shape), 0 or 1");
      ctx->emu_onchip = (int)value;
    } else if (option == CC_OPT_LADDER_PACK) {
      CC_REQUIRE(value >= -1 && value <= 1, CC_ERR_INVALID, "CC_OPT_LADDER_PACK: -1 (by shape), 0 or 1");
      ctx->ladder_pack = (int)value;
    } else if (option == CC_OPT_GRAPHS) {
      CC_REQUIRE(value == 0 || value == 1, CC_ERR_INVALID, "CC_OPT_GRAPHS: 0 or 1");
      ctx->graphs = (int)value;
    } else {
      fail(CC_ERR_INVALID, "unknown option");
    }
    return CC_OK;
  });
}

int cc_ctx_selftest_wait(cc_ctx* ctx) {
  if (!ctx) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    k_wait_selftest(ctx->ex());
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    return CC_OK;  // the flag the kernel set turns this into CC_ERR_TIMEOUT
  });
}

int cc_ctx_profile(cc_ctx* ctx, int enable) {
  if (!ctx) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->prof.reset();
    ctx->prof.on = enable != 0;
    ctx->prof.all = enable >= 2;
    return CC_OK;
  });
}

int cc_ctx_profile_get(cc_ctx* ctx, const char* tag, uint64_t* launches, double* total_ms, double* flops) {
  if (!ctx || !tag) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    ctx->prof.resolve();
    uint64_t l = 0;
    double ms = 0.0, fl = 0.0;
    for (auto& d : ctx->prof.done)
      if (d.first == tag) {
        l = d.second.launches;
        ms = d.second.ms;
        fl = d.second.flops;
      }
    if (launches) *launches = l;
    if (total_ms) *total_ms = ms;
    if (flops) *flops = fl;
    return CC_OK;
  });
}

int cc_ctx_profile_list(cc_ctx* ctx, char* buf, size_t cap, size_t* needed) {
  if (!ctx || (!buf && cap)) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    ctx->prof.resolve();
    std::string all;
    size_t fit = 0;  // length of the whole lines that fit in buf
    for (auto& d : ctx->prof.done) {
      char line[512];
      snprintf(line, sizeof line, "%s\t%llu\t%.6f\t%.6e\n", d.first.c_str(), (unsigned long long)d.second.launches,
               d.second.ms, d.second.flops);
      all += line;
      if (all.size() < cap) fit = all.size();
    }
    if (cap) {
      memcpy(buf, all.data(), fit);
      buf[fit] = '\0';
    }
    if (needed) *needed = all.size() + 1;
    return CC_OK;
  });
}

int cc_sys_create(cc_ctx* ctx, int o, int v, int naux, const double* fock, const double* B, cc_sys** out) {
  if (!ctx || !out) return CC_ERR_INVALID;
  *out = nullptr;
  return guarded(ctx, [&]() {
    CC_REQUIRE(o >= 1 && v >= 1 && naux >= 1, CC_ERR_INVALID, "need o >= 1, v >= 1, naux >= 1");
    CC_REQUIRE(fock && B, CC_ERR_INVALID, "NULL fock or B");
    const int n = o + v;
    Exec ex = ctx->ex();
    DBuf<double> f(ex.pool, (size_t)n * n), b(ex.pool, (size_t)naux * n * n), chk(ex.pool, 4096);
    copy_in(ctx, f.p, fock, (size_t)n * n);
    copy_in(ctx, b.p, B, (size_t)naux * n * n);
    k_asym(ex, naux, n, b.p, chk.p, chk.p + 2);
    k_asym(ex, 1, n, f.p, chk.p + 4, chk.p + 8);
    double h[6];
    CC_CUDA(cudaMemcpyAsync(h, chk.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    CC_REQUIRE(std::isfinite(h[0]) && std::isfinite(h[1]), CC_ERR_INVALID, "B holds non-finite values");
    CC_REQUIRE(h[0] <= 1e-12 * std::max(h[1], 1e-300), CC_ERR_INVALID, "B[P] is not symmetric in its orbital indices");
    CC_REQUIRE(std::isfinite(h[4]) && std::isfinite(h[5]), CC_ERR_INVALID, "fock holds non-finite values");
    std::unique_ptr<cc_sys> s(new cc_sys);
    s->ctx = ctx;
    system_init(ex, s->s, o, v, naux, f.p, b.p);
    // the allocation-free energy entry point loads its module and looks up its scratch array
    // here, so that its own first call on this device has nothing left to load
    noalloc_prepare(ex, s->s);
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = s.release();
    return CC_OK;
  });
}

void cc_sys_destroy(cc_sys* sys) {
  if (!sys) return;
  cudaSetDevice(sys->ctx->device);
  cudaStreamSynchronize(sys->ctx->stream);
  delete sys;
}

int cc_residual(cc_ctx* ctx, cc_sys* sys, const double* t1, const double* t2, double* r1, double* r2,
                double* energy, cc_precision prec) {
  if (!ctx || !sys) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    check_prec(prec);
    const System& s = sys->s;
    Engine& eng = engine(sys);
    Exec ex = ctx->ex();
    DBuf<double> t(ex.pool, s.namp()), r(ex.pool, s.namp()), e(ex.pool, 1);
    load_amplitudes(ctx, s, t1, t2, t.p);
    eng.value(t.p, r.p, e.p, prec);
    const size_t ov = (size_t)s.o * s.v;
    copy_out(ctx, r1, r.p, ov);
    copy_out(ctx, r2, r.p + ov, s.namp() - ov);
    double eh = 0.0;
    CC_CUDA(cudaMemcpyAsync(&eh, e.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    if (energy) *energy = eh;
    return CC_OK;
  });
}

int cc_jvp(cc_ctx* ctx, cc_sys* sys, const double* t1, const double* t2, const double* d1, const double* d2,
           double* j1, double* j2, cc_precision prec) {
  if (!ctx || !sys) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    check_prec(prec);
    const System& s = sys->s;
    Engine& eng = engine(sys);
    Exec ex = ctx->ex();
    DBuf<double> t(ex.pool, s.namp()), d(ex.pool, s.namp()), r(ex.pool, s.namp());
    load_amplitudes(ctx, s, t1, t2, t.p);
    load_amplitudes(ctx, s, d1, d2, d.p);
    eng.value(t.p, r.p, nullptr, value_prec(prec));
    eng.tangent(d.p, r.p, prec);
    const size_t ov = (size_t)s.o * s.v;
    copy_out(ctx, j1, r.p, ov);
    copy_out(ctx, j2, r.p + ov, s.namp() - ov);
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    return CC_OK;
  });
}

int cc_jvp_multi(cc_ctx* ctx, cc_sys* sys, const double* t1, const double* t2, int ndir, const double* d1s,
                 const double* d2s, double* j1s, double* j2s, cc_precision prec) {
  if (!ctx || !sys || ndir < 0) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    check_prec(prec);
    if (ndir == 0) return CC_OK;
    CC_REQUIRE(d1s && d2s, CC_ERR_INVALID, "NULL direction");
    const System& s = sys->s;
    Engine& eng = engine(sys);
    Exec ex = ctx->ex();
    const size_t ov = (size_t)s.o * s.v, oovv = s.namp() - ov;
    DBuf<double> t(ex.pool, s.namp()), d(ex.pool, s.namp()), r(ex.pool, s.namp());
    load_amplitudes(ctx, s, t1, t2, t.p);
    eng.value(t.p, r.p, nullptr, value_prec(prec));
    for (int k = 0; k < ndir; ++k) {
      load_amplitudes(ctx, s, d1s + k * ov, d2s + k * oovv, d.p);
      eng.tangent(d.p, r.p, prec);
      if (j1s) copy_out(ctx, j1s + k * ov, r.p, ov);
      if (j2s) copy_out(ctx, j2s + k * oovv, r.p + ov, oovv);
    }
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    return CC_OK;
  });
}

int cc_apply_AF(cc_ctx* ctx, cc_sys* sys, const double* x1, const double* x2, double* y1, double* y2, int inverse,
                cc_precision prec) {
  if (!ctx || !sys) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    check_prec(prec);
    System& s = sys->s;
    Exec ex = ctx->ex();
    DBuf<double> x(ex.pool, s.namp()), y(ex.pool, s.namp());
    const size_t ov = (size_t)s.o * s.v;
    copy_in(ctx, x.p, x1, ov);
    copy_in(ctx, x.p + ov, x2, s.namp() - ov);
    if (inverse == 0) apply_AF(ex, s, x.p, y.p, prec);
    else if (inverse == 1) solve_AF(ex, s, x.p, y.p, prec, prec == CC_FP64 ? 1e-12 : 1e-6, 50, false, nullptr);
    else solve_AF(ex, s, x.p, y.p, prec, 0.0, 0, true, nullptr);  // inverse == 2: eigenbasis inverse
    copy_out(ctx, y1, y.p, ov);
    copy_out(ctx, y2, y.p + ov, s.namp() - ov);
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    return CC_OK;
  });
}

int cc_solve(cc_ctx* ctx, cc_sys* sys, const cc_solve_opts* opts, double* t1, double* t2, int use_guess,
             cc_report* report) {
  return ccpnk::solve_cancellable(ctx, sys, opts, t1, t2, use_guess, report, nullptr);
}

int cc_solve_batch(cc_ctx* ctx, int nsys, cc_sys* const* sys, const cc_solve_opts* opts, double* const* t1s,
                   double* const* t2s, cc_report* reports) {
  return ccpnk::solve_batch_notify(ctx, nsys, sys, opts, t1s, t2s, reports, nullptr, nullptr);
}

}  // extern "C"

namespace ccpnk {

int solve_batch_notify(cc_ctx* ctx, int nsys, cc_sys* const* sys, const cc_solve_opts* opts, double* const* t1s,
                       double* const* t2s, cc_report* reports, const std::function<void(int, int)>& notify,
                       const std::vector<const std::atomic<int>*>* cancel) {
  if (!ctx || !sys || !opts || nsys < 0 || (nsys > 0 && !reports)) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    check_prec(opts->prec);
    CC_REQUIRE(opts->method >= CC_FP_DIIS && opts->method <= CC_INK, CC_ERR_INVALID, "unknown method");
    if (nsys == 0) return CC_OK;
    Exec ex = ctx->ex();
    std::vector<System*> ss;
    std::vector<Engine*> es;
    std::vector<DBuf<double>> tb(nsys);
    std::vector<double*> ts;
    for (int k = 0; k < nsys; ++k) {
      CC_REQUIRE(sys[k] && sys[k]->ctx == ctx, CC_ERR_INVALID, "every problem must belong to the context");
      for (int j = 0; j < k; ++j) CC_REQUIRE(sys[j] != sys[k], CC_ERR_INVALID, "a problem appears twice");
      ss.push_back(&sys[k]->s);
      es.push_back(&engine(sys[k]));
      tb[k].alloc(ex.pool, sys[k]->s.namp());
      ts.push_back(tb[k].p);
    }
    std::vector<cc_report> reps;
    // each problem's amplitudes and report are handed out as soon as it has finished
    auto done = [&](int k, int st) {
      const System& s = *ss[k];
      const size_t ov = (size_t)s.o * s.v;
      if (t1s) copy_out(ctx, t1s[k], ts[k], ov);
      if (t2s) copy_out(ctx, t2s[k], ts[k] + ov, s.namp() - ov);
      CC_CUDA(cudaStreamSynchronize(ctx->stream));
      reports[k] = reps[k];
      if (notify) notify(k, st);
    };
    solve_batch(ex, ss, es, *opts, ts, reps, done, cancel);
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    return CC_OK;
  });
}

int solve_cancellable(cc_ctx* ctx, cc_sys* sys, const cc_solve_opts* opts, double* t1, double* t2, int use_guess,
                      cc_report* report, const std::atomic<int>* cancel) {
  if (!ctx || !sys || !opts) return CC_ERR_INVALID;
  return guarded(ctx, [&]() {
    check_prec(opts->prec);
    CC_REQUIRE(opts->method >= CC_FP_DIIS && opts->method <= CC_INK, CC_ERR_INVALID, "unknown method");
    System& s = sys->s;
    Engine& eng = engine(sys);
    Exec ex = ctx->ex();
    DBuf<double> t(ex.pool, s.namp());
    if (use_guess) load_amplitudes(ctx, s, t1, t2, t.p);
    int st = solve(ex, s, eng, *opts, t.p, report, use_guess != 0, cancel);
    const size_t ov = (size_t)s.o * s.v;
    copy_out(ctx, t1, t.p, ov);
    copy_out(ctx, t2, t.p + ov, s.namp() - ov);
    CC_CUDA(cudaStreamSynchronize(ctx->stream));
    return st;
  });
}

}  // namespace ccpnk

