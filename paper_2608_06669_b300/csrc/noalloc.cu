// The correlation energy without any device allocation.
//
// Some callers cannot call cudaMalloc when they need a result: code running inside another
// framework's memory arena that forbids foreign allocations, real-time loops that must not
// enter the driver's allocator (it can synchronise the device), or processes whose device
// memory is fully reserved up front. cc_energy_noalloc serves them: it runs the same
// two-pass energy reduction as cc_residual, but its scratch (one partial sum per block) is a
// file-scope device array instead of memory from the context's pool, and it touches only the
// caller's buffers and that array.
#include <mutex>

#include "handles.h"

namespace {

// Partial sums of the energy reduction. Every GPU that loads the library holds these
// 8 KB until the process exits.
constexpr int kMaxPartials = 1024;
static __device__ __align__(256) double g_energy_partials[kMaxPartials];

constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// Device address of the array on the current device (looked up once per device). In host
// code the array's name only stands in for the symbol; a kernel must be given this address.
cudaError_t partials_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return cudaSuccess;
}

}  // namespace

namespace ccpnk {

// With lazy module loading (the CUDA default) the first use of this file's array or of the
// energy kernels loads their modules, and loading allocates device memory inside the driver.
// cc_sys_create calls this, so that path is taken there and not in cc_energy_noalloc.
void noalloc_prepare(const Exec& ex, const System& s) {
  double* partials = nullptr;
  CC_CUDA(partials_on_current_device(&partials));
  // the kernels run once on scratch of the pool, so this never touches the shared array
  DBuf<double> t(ex.pool, s.namp()), e(ex.pool, 1), scratch(ex.pool, (size_t)k_energy_partials(ex, s.o, s.v));
  k_fill(ex, s.namp(), 0.0, t.p);
  k_energy(ex, s.o, s.v, s.Govov.p, t.p, t.p + (size_t)s.o * s.v, s.f.p + s.o, s.n, e.p, scratch.p);
}

}  // namespace ccpnk

extern "C" int cc_energy_noalloc(const cc_sys* sys, const double* t1, const double* t2, double* energy,
                                 void* stream) {
  if (!sys || !t1 || !t2 || !energy) return CC_ERR_INVALID;
  const ccpnk::System& s = sys->s;
  if (s.o < 1 || s.v < 1) return CC_ERR_INVALID;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  const int dev = sys->ctx->device;
  if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  int status = CC_OK;
  try {
    ccpnk::Exec ex;  // no pool: nothing here may allocate
    ex.stream = static_cast<cudaStream_t>(stream);
    ex.sm_count = sys->ctx->sm_count;
    double* partials = nullptr;
    CC_CUDA(partials_on_current_device(&partials));
    if (ccpnk::k_energy_partials(ex, s.o, s.v) > kMaxPartials)
      ccpnk::fail(CC_ERR_INVALID, "cc_energy_noalloc: the reduction needs more than 1024 partial sums");
    // every partial the final pass reads is written first by the same call: nothing to clear
    ccpnk::k_energy(ex, s.o, s.v, s.Govov.p, t1, t2, s.f.p + s.o, s.n, energy, partials);
  } catch (const ccpnk::Error& e) {
    status = e.status;
  }
  if (prev != dev) cudaSetDevice(prev);
  return status;
}
