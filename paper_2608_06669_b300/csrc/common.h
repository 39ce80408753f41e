// Shared declarations of the libccpnk CUDA sources (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/ccpnk.h"

namespace ccpnk {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
  int status;
  std::string msg;
};

[[noreturn]] void fail(int status, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
#define CC_CUDA(x) ::ccpnk::cuda_check((x), #x)
#define CC_REQUIRE(cond, status, msg) \
  do {                                \
    if (!(cond)) ::ccpnk::fail((status), (msg)); \
  } while (0)

// ---------------------------------------------------------------------------
// device memory: a budgeted pool of cudaMalloc'd blocks, reused by size class
// ---------------------------------------------------------------------------
class Pool {
 public:
  explicit Pool(size_t budget) : budget_(budget) {}
  ~Pool();
  void* get(size_t bytes);
  void put(void* p);
  void release_free();  // frees cached blocks
  size_t held() const { return held_; }
  size_t budget() const { return budget_; }
  // CUDA-graph support: while record is set, every block handed out is appended to it; a pinned
  // block is never handed out again (nor freed) until it is unpinned, so a captured graph keeps
  // exclusive use of the scratch blocks its kernels were recorded with.
  std::vector<void*>* record = nullptr;
  void pin(void* p);
  void unpin(void* p);

 private:
  struct Block {
    void* p;
    size_t bytes;
    bool used;
    int pins = 0;
  };
  std::vector<Block> blocks_;
  size_t budget_;
  size_t held_ = 0;
};

// RAII device buffer from a pool
template <typename T>
struct DBuf {
  Pool* pool = nullptr;
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(Pool* pl, size_t count) { alloc(pl, count); }
  void alloc(Pool* pl, size_t count) {
    reset();
    pool = pl;
    n = count;
    p = count ? static_cast<T*>(pl->get(count * sizeof(T))) : nullptr;
  }
  void reset() {
    if (p && pool) pool->put(p);
    p = nullptr;
    n = 0;
  }
  ~DBuf() { reset(); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : pool(o.pool), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    reset();
    pool = o.pool; p = o.p; n = o.n;
    o.p = nullptr; o.n = 0;
    return *this;
  }
};

// ---------------------------------------------------------------------------
// kernel timer: CUDA events around tagged launches, resolved on request
// ---------------------------------------------------------------------------
struct Prof {
  struct Rec {
    std::string tag;
    cudaEvent_t a, b;
    double flops;
  };
  struct Sum {
    uint64_t launches = 0;
    double ms = 0.0, flops = 0.0;
  };
  bool on = false;
  bool all = false;  // also time every untagged contraction, named by its index labels
  std::vector<Rec> pending;
  std::vector<std::pair<std::string, Sum>> done;
  void resolve();  // waits for pending events and folds them into done
  void reset();
  ~Prof() { reset(); }
};

// ---------------------------------------------------------------------------
// launch bookkeeping
// ---------------------------------------------------------------------------
struct Exec {
  cudaStream_t stream = nullptr;
  Pool* pool = nullptr;
  uint64_t* launches = nullptr;  // kernels run: one per launch, a graph's kernel nodes per replay
  uint64_t* calls = nullptr;     // host launch calls: one per kernel launch or graph replay
  int* dev_flag = nullptr;       // device error flag (bounded waits, bad shapes)
  int sm_count = 148;
  Prof* prof = nullptr;
  unsigned long long wait_ns = 4000000000ull;  // bound on every device-side wait (global timer)
  long long stage_cap = -1;                    // bytes of kept staged operands (-1: the default)
  int graphs = 1;                              // replay the JVPs of a solve from CUDA graphs
  int emu_chunk = 64;                          // k blocks of 64 per exact chunk of the FP64 emulation
  int ladder_pack = -1;                        // (c, d) split of the tensor-core ladder: -1 by shape, 0, 1
  int emu_onchip = -1;                         // FP64 emulation summed on chip: -1 by shape, 0, 1
  void count(uint64_t k = 1) const {
    if (launches) *launches += k;
    if (calls) *calls += 1;
  }
  // brackets a launch with events when the timer is on and the launch is tagged
  bool timing(const char* tag) const { return prof && prof->on && tag; }
  void mark_begin(cudaEvent_t* a) const;
  void mark_end(const char* tag, cudaEvent_t a, double flops) const;
};

// Digit slices per operand of the FP64 emulation (CC_FP64_EMU): 9 slices of 6 bits keep 54
// significant bits below each row's largest element, one more than FP64's significand; the
// S (S + 1) / 2 slice products of levels 2..S + 1 run on the tensor cores.
constexpr int kOzSlices = 9;
constexpr int kOzProducts = kOzSlices * (kOzSlices + 1) / 2;

// Pair indices, row-major over the upper triangle: c <= d (with the diagonal) and c < d.
__host__ __device__ __forceinline__ size_t pair_le(int c, int d, int n) {
  return (size_t)c * (2 * n - c + 1) / 2 + (d - c);
}
__host__ __device__ __forceinline__ size_t pair_lt(int c, int d, int n) {
  return (size_t)c * (2 * n - c - 1) / 2 + (d - c - 1);
}

// ---------------------------------------------------------------------------
// GEMM with compound indices of up to three strided modes:
//   x = (i0 * e1 + i1) * e2 + i2  ->  offset i0 * s0 + i1 * s1 + i2 * s2
// ---------------------------------------------------------------------------
struct CIdx {
  int e1 = 1, e2 = 1;
  long long s0 = 0, s1 = 0, s2 = 0;
};

// Offsets of a compound index walked in steps of a fixed size: the mixed-radix digits are
// carried forward instead of divided out for every element (a division only on a carry).
struct CWalk {
  long long off;
  int i0, i1, i2;
  __device__ __forceinline__ void init(const CIdx& c, int x) {
    if (c.e1 == 1 && c.e2 == 1) {
      i0 = x;
      i1 = i2 = 0;
    } else {
      i2 = x % c.e2;
      const int r = x / c.e2;
      i1 = r % c.e1;
      i0 = r / c.e1;
    }
    off = (long long)i0 * c.s0 + (long long)i1 * c.s1 + (long long)i2 * c.s2;
  }
  __device__ __forceinline__ void step(const CIdx& c, int d) {
    if (c.e1 == 1 && c.e2 == 1) {
      i0 += d;
      off += (long long)d * c.s0;
      return;
    }
    i2 += d;
    if (i2 >= c.e2) {
      const int q = i2 / c.e2;
      i2 -= q * c.e2;
      i1 += q;
      if (i1 >= c.e1) {
        const int q1 = i1 / c.e1;
        i1 -= q1 * c.e1;
        i0 += q1;
      }
    }
    off = (long long)i0 * c.s0 + (long long)i1 * c.s1 + (long long)i2 * c.s2;
  }
};

// Tensor-core operands kept in staging layout between two contractions: a K-major TF32 (FP32
// words) or BF16 [rows][nseg * kpad] array whose nseg segments hold the high or the low part.
struct StagedOut {  // C written in that layout (C's strides count elements), beta must be 0
  void* base;
  long long kpad;
  int nseg, seg_lo;  // seg_lo: bit mask of the segments that hold the low part; nseg = 0: C as
                     // plain FP32 words
};
struct StagedIn {  // the B operand already staged (rows padded to the tile, zero k padding)
  const void* base;
  int rows_pad, kk;  // kk = nseg * kpad elements per row
};

// Tensor-core staging copies of operands that stay fixed across calls: in the tangent program
// the value-side operands do not change between the JVPs of one Newton step, so their staged
// copies are kept (up to cap bytes) instead of being gathered again for every JVP. An Engine
// owns one and clears it whenever its values change.
struct StageKey {
  const double* src;
  CIdx rix, kix, bix;
  int rows, K, batch, rows_pad, k_pad, nseg, seg_lo, bf;
};
bool operator==(const StageKey& a, const StageKey& b);
struct StageCache {
  struct Ent {
    StageKey key;
    DBuf<double> buf;
    bool fresh = true;  // false: the source changed since the copy was staged (re-stage in place)
  };
  std::vector<Ent> ents;
  size_t bytes = 0, cap = 0;
  void clear() {
    ents.clear();
    bytes = 0;
  }
  // keeps the buffers (and so their addresses, which a captured graph may hold) but marks every
  // copy out of date
  void mark_stale() {
    for (auto& e : ents) e.fresh = false;
  }
};

struct GemmArgs {
  const double* A;
  const double* B;
  double* C;
  int M, N, K, batch;
  CIdx am, ak, ab;  // A(m, k) of batch b at A + am(m) + ak(k) + ab(b)
  CIdx bk, bn, bb;  // B(k, n)
  CIdx cm, cn, cb;  // C(m, n)
  double alpha, beta;
  int a_kfast, b_kfast;  // unit stride along k in A / B (picks the coalesced load order)
  int splits;            // split-K factor (1: write C directly)
  int kchunk;            // k range per split (multiple of the k slice)
  double* part;          // split-K partials [splits][batch][M][N]
  const StagedOut* so;   // tensor-core only: C in staging layout
  const StagedIn* sb;    // tensor-core only: B already staged
  StageCache* cache;     // tensor-core only: where fixed operands' staged copies are kept
  int cache_mask;        // bit 0: A is fixed across calls (cacheable), bit 1: B
};

// Tensor-core GEMM (gemm_tc.cu): same contract as the FP64 kernel, run on tcgen05.
void gemm_tc(const Exec& ex, cc_precision prec, const GemmArgs& g, const char* tag = nullptr);
// Independent tensor-core GEMMs (no output shared, single-precision kinds) in grouped launches:
// every problem's tiles in one persistent launch of up to 16 problems per output mode.
void gemm_tc_group(const Exec& ex, cc_precision prec, const std::vector<GemmArgs>& gs, const char* tag = nullptr);
// One kernel whose bounded wait on an mbarrier that nothing arrives at gives up after
// ex.wait_ns and sets the device error flag (the self-test of the bounded waits).
void k_wait_selftest(const Exec& ex);

// ---------------------------------------------------------------------------
// tensors and contractions
// ---------------------------------------------------------------------------
constexpr int kMaxModes = 6;

// A strided view of an FP64 device array with one label per mode.
struct TView {
  double* p = nullptr;
  int nd = 0;
  int ext[kMaxModes] = {0};
  long long st[kMaxModes] = {0};
  char lab[kMaxModes + 1] = {0};
};

// Row-major view: labels like "Pac" and extents.
TView view(double* p, const char* labels, std::initializer_list<int> ext);
// View with explicit strides (elements).
TView view_strided(double* p, const char* labels, std::initializer_list<int> ext,
                   std::initializer_list<long long> strides);

// C = alpha * contract(A, B) + beta * C over the labels: labels of C present in both A and B
// are batch modes, labels in A and C the row modes, in B and C the column modes, labels in
// A and B only are summed. prec selects the FP64 FMA kernel or the tensor-core kernel.
// cache / cache_mask: operands (bit 0 for A, bit 1 for B) whose contents stay fixed until the
// cache is cleared may have their tensor-core staging kept there.
void contract(const Exec& ex, cc_precision prec, double alpha, const TView& A, const TView& B,
              double beta, const TView& C, const char* tag = nullptr, const StagedOut* so = nullptr,
              const StagedIn* sb = nullptr, StageCache* cache = nullptr, int cache_mask = 0);

// One contraction of a group (contract_group): independent of the others of its group (no
// output shared, nothing read that another writes).
struct ContractSpec {
  double alpha = 1.0, beta = 0.0;
  TView A, B, C;
  StageCache* cache = nullptr;
  int cache_mask = 0;
  const StagedOut* so = nullptr;  // tensor-core only: C written in staging layout
  const StagedIn* sb = nullptr;   // tensor-core only: B already staged
};
// Independent contractions at one precision: those the tensor cores run best share grouped
// launches (one persistent launch over all their tiles), the rest run one by one. Specs with a
// staged operand always run on the tensor cores. tag: kernel-timer tag of the whole group.
void contract_group(const Exec& ex, cc_precision prec, const std::vector<ContractSpec>& specs,
                    const char* tag = nullptr);

// ---------------------------------------------------------------------------
// kernels with host launchers (elementwise.cu)
// ---------------------------------------------------------------------------
void k_axpby(const Exec& ex, size_t n, double a, const double* x, double b, double* y);  // y = a x + b y
void k_scale(const Exec& ex, size_t n, double a, double* y);
void k_fill(const Exec& ex, size_t n, double val, double* y);
void k_copy(const Exec& ex, size_t n, const double* x, double* y);
// out[i][j][a][b] (+)= X[i][j][a][b] + X[j][i][b][a]
void k_sym_add(const Exec& ex, int o, int v, const double* X, double* out, double beta);
// u[i][j][a][b] = 2 t[i][j][a][b] - t[j][i][a][b]
void k_make_u(const Exec& ex, int o, int v, const double* t, double* u);
// R[i][j][a][b] += L[i][j][a][b] if b >= (a / blk) * blk, else L[j][i][b][a] (the ladder's mirror)
void k_ladder_mirror_add(const Exec& ex, int o, int v, int blk, const double* L, double* R);
// The ladder's symmetric/antisymmetric split over (c, d): pair-packed T+, T- (rows i <= j and
// i < j), W+, W- (per slab row), and the block of L rebuilt from L+ and L-
void k_ladder_pm_T(const Exec& ex, int o, int v, const double* T, double* Tp, double* Tm);
// the tensor-core ladder's (c, d) split: W+ and W- of FP32 slab rows, written staged
void k_ladder_pm_stage(const Exec& ex, bool bf, int nseg, long long rows, int v, const float* W, void* Wp,
                       long long kpP, void* Wm, long long kpQ);
void k_ladder_pm_W(const Exec& ex, size_t rows, int v, const double* W, double* Wp, double* Wm);
void k_ladder_pm_unpack(const Exec& ex, int o, int v, int a0, int al, int bl, const double* Lp, const double* Lm,
                        double* L, size_t ld = 0);  // ld: row stride of L+ and L- (0: al bl)
// L[p][q][r][s] = 2 g[p][q][r][s] - g[p][s][r][q] over an (o v o v) block
void k_make_L_ovov(const Exec& ex, int o, int v, const double* g, double* L);
// gamma[P] = sum_k A[P][k][k]
void k_trace_batched(const Exec& ex, int P, int m, const double* A, double* gamma);
// Deterministic reductions: result written to a device scalar.
void k_dot(const Exec& ex, size_t n, const double* x, const double* y, double* out, double* scratch);
// out[k] = dot(Q[k], w) for k < m (rows of length n), deterministic.
void k_multi_dot(const Exec& ex, int m, size_t n, const double* Q, size_t ldq, const double* w,
                 double* out, double* scratch);
// w -= sum_k h[k] Q[k]  (h on device)
void k_multi_axpy(const Exec& ex, int m, size_t n, const double* Q, size_t ldq, const double* h,
                  double* w);
// energy terms: E = sum (2 g_iajb - g_ibja)(t2_ijab + t1_ia t1_jb) + 2 sum f_ia t1_ia
void k_energy(const Exec& ex, int o, int v, const double* govov, const double* t1, const double* t2,
              const double* fov, int ldf, double* out, double* scratch);
// number of per-block partial sums (scratch doubles) k_energy uses for an (o, v) problem
int k_energy_partials(const Exec& ex, int o, int v);
// scaled elementwise divide: y = x / (D + shift) with D built from diagonal Fock entries
void k_denom_divide(const Exec& ex, int o, int v, const double* fdiag, double shift,
                    const double* x1, const double* x2, double* y1, double* y2, double scale);
// out[i][j][a][b] = scale * g[i][a][j][b]
void k_ovov_to_oovv(const Exec& ex, int o, int v, const double* g, double* out, double scale);
// copy a (rows x cols) block with strides
void k_copy2d(const Exec& ex, int rows, int cols, const double* src, long long lds, double* dst,
              long long ldd);
// checks |B[P][p][q] - B[P][q][p]| <= tol * max|B|; writes the max asymmetry to out
void k_asym(const Exec& ex, int P, int n, const double* B, double* out, double* scratch);

// FP32 staging for tensor-core contractions (elementwise.cu)
void k_to_f32(const Exec& ex, size_t n, const double* x, float* y);

}  // namespace ccpnk
