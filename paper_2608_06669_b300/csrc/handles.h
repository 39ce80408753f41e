// The opaque handles of the C ABI (cc_ctx, cc_sys), shared by the sources that implement it.
#pragma once

#include <memory>
#include <string>

#include "solver.h"

struct cc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::unique_ptr<ccpnk::Pool> pool;
  uint64_t launches = 0;
  int sm_count = 148;
  int* dflag = nullptr;  // device error flag written by bounded waits
  std::string err;
  ccpnk::Prof prof;
  ccpnk::Exec ex() {
    ccpnk::Exec e;
    e.stream = stream;
    e.pool = pool.get();
    e.launches = &launches;
    e.sm_count = sm_count;
    e.dev_flag = dflag;
    e.prof = &prof;
    return e;
  }
};

struct cc_sys {
  cc_ctx* ctx = nullptr;
  ccpnk::System s;
  std::unique_ptr<ccpnk::Engine> eng;
};
