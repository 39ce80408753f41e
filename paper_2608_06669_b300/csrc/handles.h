// The opaque handles of the C ABI (cc_ctx, cc_sys), shared by the sources that implement it.
#pragma once

#include <atomic>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "solver.h"

struct cc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::unique_ptr<ccpnk::Pool> pool;
  uint64_t launches = 0;
  uint64_t launch_calls = 0;
  int sm_count = 148;
  int* dflag = nullptr;  // device error flag written by bounded waits
  std::string err;
  ccpnk::Prof prof;
  unsigned long long wait_ns = 4000000000ull;  // CC_OPT_WAIT_LIMIT_NS
  long long stage_cap = -1;                    // CC_OPT_STAGE_CACHE_BYTES (-1: the default)
  int graphs = 1;                              // CC_OPT_GRAPHS
  int emu_chunk = 64;                          // CC_OPT_EMU_CHUNK
  int ladder_pack = -1;                        // CC_OPT_LADDER_PACK
  int emu_onchip = -1;                         // CC_OPT_EMU_ONCHIP
  ccpnk::Exec ex() {
    ccpnk::Exec e;
    e.stream = stream;
    e.pool = pool.get();
    e.launches = &launches;
    e.calls = &launch_calls;
    e.sm_count = sm_count;
    e.dev_flag = dflag;
    e.prof = &prof;
    e.wait_ns = wait_ns;
    e.stage_cap = stage_cap;
    e.graphs = graphs;
    e.emu_chunk = emu_chunk;
    e.ladder_pack = ladder_pack;
    e.emu_onchip = emu_onchip;
    return e;
  }
};

struct cc_sys {
  cc_ctx* ctx = nullptr;
  ccpnk::System s;
  std::unique_ptr<ccpnk::Engine> eng;
};

namespace ccpnk {
// cc_solve_batch with a callback notify(k, status), called once problem k's amplitudes are in
// t1s[k] / t2s[k] and its report in reports[k], and per-problem cancellation flags.
int solve_batch_notify(cc_ctx* ctx, int nsys, cc_sys* const* sys, const cc_solve_opts* opts, double* const* t1s,
                       double* const* t2s, cc_report* reports, const std::function<void(int, int)>& notify,
                       const std::vector<const std::atomic<int>*>* cancel);
// cc_solve with a cancellation flag that another thread may set (the server's cancel).
int solve_cancellable(cc_ctx* ctx, cc_sys* sys, const cc_solve_opts* opts, double* t1, double* t2, int use_guess,
                      cc_report* report, const std::atomic<int>* cancel);
}  // namespace ccpnk
