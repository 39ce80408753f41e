// Closed-shell DF-CCSD residual engine (value and tangent programs).
#pragma once

#include <functional>

#include "common.h"

namespace ccpnk {

// A problem resident on the device (the public cc_sys).
struct System {
  int o = 0, v = 0, n = 0, P = 0;
  DBuf<double> f;      // n x n Fock matrix
  DBuf<double> h;      // n x n one-electron part h = f - (2J - K)[reference density]
  DBuf<double> fdiag;  // n
  DBuf<double> Boo, Bov, Bvv;  // [P][o][o], [P][o][v], [P][v][v]
  DBuf<double> Govov;  // (kc|ld) stored [k][c][l][d]
  DBuf<double> Lovov;  // 2 (ld|kc) - (lc|kd) stored [l][d][k][c]
  // eigenbases of the occupied and virtual Fock blocks (filled on demand for A_F^{-1})
  bool eig_ready = false;
  std::vector<double> eo, ev;
  DBuf<double> Uo, Uv;  // column eigenvectors, o x o and v x v
  DBuf<double> eig_d;   // [eo | ev] on the device
  size_t namp() const { return (size_t)o * v + (size_t)o * o * v * v; }
};

void system_init(const Exec& ex, System& s, int o, int v, int P, const double* fock_dev, const double* B_dev);

// Values of a per ladder block: about v/8 (so the half-triangle saving applies) with an FP64
// (a, b, c, d) slab of at most 2 GiB; larger blocks give the tensor-core GEMMs more tiles.
int ladder_block_for(int v);

// Bytes the tangent program may keep in staged copies of its value-side operands: room for
// about 32 staged copies (4-byte words) of the largest tensors, at most 1 GiB.
size_t stage_cache_cap(int o, int v, int P);

// One step of a recorded program: a kernel-launch closure or a contraction (see
// Engine::value_batch).
struct Op {
  enum { KERNEL = 0, CONTRACT = 1 };
  int kind = KERNEL;
  ContractSpec c;
  std::function<void(const Exec&)> fn;
};
using OpList = std::vector<Op>;
// Runs the recorded programs of several engines (one stream) step by step: the i-th steps of
// all of them together, their contractions as one group (contract_group: the tensor-core ones in
// grouped launches). Programs whose steps do not line up run one after the other.
void run_lockstep(const Exec& ex, cc_precision prec, std::vector<OpList>& lists);

// Intermediates of one residual evaluation; the tangent program reuses the values.
class Engine {
 public:
  Engine(const Exec& ex, const System& s);
  ~Engine();
  // R(t), E(t): t = [t1 | t2] on the device (namp doubles), r = [r1 | r2].
  // Leaves the intermediates of t in place for later tangent() calls.
  void value(const double* t, double* r, double* energy_dev, cc_precision prec);
  // J(t) d at the t of the last value() call.
  void tangent(const double* d, double* jd, cc_precision prec);
  // value() and tangent() for several engines of one context at once, in lockstep: the same
  // contraction of every engine in one group (results equal the one-by-one calls).
  static void value_batch(const std::vector<Engine*>& engs, const std::vector<const double*>& t,
                          const std::vector<double*>& r, const std::vector<double*>& energy_dev, cc_precision prec);
  static void tangent_batch(const std::vector<Engine*>& engs, const std::vector<const double*>& d,
                            const std::vector<double*>& jd, cc_precision prec);
  const Exec& exec() const { return ex_; }
  // Takes the context's current settings (wait limit, staged-operand cache size); a smaller
  // cache drops what it kept.
  void rebind(const Exec& ex);
  // CUDA graphs for the JVPs of one solve: between begin_graphs and end_graphs, the tangent
  // program at prec is captured once as it runs right after a residual evaluation (when it
  // re-stages the value-side operands it keeps) and once as it runs later (when it reuses them),
  // and every further JVP replays the matching graph. The graphs read and write the engine's
  // own buffers at fixed addresses; their scratch blocks stay pinned in the pool until
  // end_graphs. Profiled runs (the kernel timer on) stay eager.
  void begin_graphs(cc_precision prec);
  void end_graphs() noexcept;
  double* scratch() { return scratch_.p; }
  size_t scratch_count() const { return scratch_.n; }

 private:
  struct Pair {
    DBuf<double> val, tan;
  };
  void alloc(Pair& x, size_t n);
  // fixed_xy / fixed_t: X, Y / T stay fixed until the next value() (their staging may be kept)
  void ladder(const double* Xv, const double* Yv, int Paux, const double* T, double* R, cc_precision prec,
              bool fixed_xy = false, bool fixed_t = false);
  void program(bool tan, cc_precision prec, double* r_out);
  Exec ex_;
  const System& s_;
  int ladder_block_ = 1;
  Pair t_, u_, Btoo_, Btvv_, Btvo_, gam_, hY_, Ft_, Z_, Wk_, Woo_, Cint_, Dint_, Gv_, Go_, X_, Y2_;
  DBuf<double> W_;        // ladder workspace, ladder_block_ * v^3
  DBuf<double> pmT_, pmW_, pmL_;  // the FP64 ladder's (c, d)-split operands and results
  DBuf<double> XsYs_;     // stacked factors of the tangent ladder
  DBuf<double> W2_;       // tensor-core ladder slab in staging layout (TF32 or BF16 words)
  int w2_mode_ = -1;      // precision whose layout W2_ holds
  StageCache stage_;      // staged value-side operands of the tangent program (cleared by value())
  DBuf<double> scratch_;  // reduction partials
  struct TanGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> pinned;  // pool blocks the captured kernels use as scratch
    uint64_t launches = 0;      // kernel nodes (counted as launches at every replay)
    int eager = 0;              // eager runs before the capture (they warm the pool and the cache)
  };
  void capture(TanGraph& G, cc_precision prec);
  TanGraph graphs_[2];          // [0]: first JVP after a residual evaluation, [1]: the others
  bool graphs_on_ = false, first_since_value_ = true;
  cc_precision graph_prec_ = CC_FP64;
  cudaStream_t cap_stream_ = nullptr;
  DBuf<double> jout_;           // the captured program's output
  OpList* rec_ = nullptr;       // set: program() records its steps here instead of launching them
  void record(OpList& list, bool tan, cc_precision prec, double* out);
};

// Readies cc_energy_noalloc on the current device for this problem: loads its module, looks up
// its scratch array and runs its kernels once (so its own calls have nothing left to load).
void noalloc_prepare(const Exec& ex, const System& s);

// y = A_F x on [x1 | x2] vectors (Eq. Preconditioner, App. C)
void apply_AF(const Exec& ex, const System& s, const double* x, double* y, cc_precision prec);
// y = (A_F + shift)^{-1} x in the eigenbases of the Fock blocks (exact Sylvester inverse); the
// four basis rotations run at prec, the division by the eigenvalue differences in FP64
void solve_AF_direct(const Exec& ex, System& s, const double* x, double* y, double shift, double* work,
                     cc_precision prec = CC_FP64);

}  // namespace ccpnk
