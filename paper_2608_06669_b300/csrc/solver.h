// Linear and nonlinear solvers of the Newton-Krylov family (host control, device vectors).
#pragma once

#include <atomic>
#include <functional>
#include <memory>
#include <vector>

#include "ccsd.h"

namespace ccpnk {

struct SolveStats {
  int residual_evals = 0, jvps = 0, af_applies = 0, krylov_iters = 0, newton_iters = 0;
};

// y = Op(x) on amplitude-length device vectors
using LinOp = std::function<void(const double* x, double* y)>;

// GMRES with CGS2 Arnoldi as a state machine, so that several systems can advance in lockstep
// (their operator applications done together): start from x = 0 for Op x = b; apply Op to in()
// into out(); step() orthogonalises and updates the Givens-rotated least-squares problem and
// says whether to go on (residual estimate above rtol ||b||, fewer than m_max steps);
// finish() forms x = V y. vecs: (m_max + 1) * n doubles of basis storage.
class Gmres {
 public:
  Gmres(const Exec& ex, size_t n, int m_max, double* V, double* small, double* scratch);
  bool start(const double* b, double* x, double rtol);  // false: nothing to iterate (b = 0)
  const double* in() const { return V_ + (size_t)j_ * n_; }
  double* out() { return V_ + (size_t)(j_ + 1) * n_; }
  bool step();
  int finish();
  double est() const { return est_; }
  int steps() const { return j_; }

 private:
  Exec ex_;
  size_t n_;
  int m_;
  double *V_, *small_, *scratch_, *x_ = nullptr;
  double rtol_ = 0, beta_ = 0, est_ = 0;
  int j_ = 0;
  std::vector<double> H_, cs_, sn_, g_, hh_;
};

// GMRES with CGS2 Arnoldi (Algorithm 1's Krylov loop, with classical Gram-Schmidt applied
// twice): approximately solves Op x = b from x = 0 until the residual estimate from the
// Givens-rotated Hessenberg system is <= rtol * ||b||, or m_max steps. Returns the steps taken.
// vecs: (m_max + 1) * n doubles of basis storage.
int gmres(const Exec& ex, size_t n, const LinOp& op, const double* b, double* x, double rtol, int m_max,
          double* vecs, double* small_dev, double* scratch, double* est_out = nullptr);

// x = A_F^{-1} b by inner GMRES (prec applies to the A_F contractions) or directly in the
// Fock eigenbasis (direct = true).
void solve_AF(const Exec& ex, System& s, const double* b, double* x, cc_precision prec, double rtol,
              int m_max, bool direct, SolveStats* st);

// The nonlinear solve behind cc_solve; t holds [t1 | t2] (guess in, solution out).
// cancel (may be null): a flag another thread sets to stop the solve between outer iterations.
int solve(const Exec& ex, System& s, Engine& eng, const cc_solve_opts& o, double* t, cc_report* rep,
          bool use_guess, const std::atomic<int>* cancel = nullptr);

// Several NK or PNK solves of one context in lockstep (other methods: one after the other):
// each residual and JVP is evaluated for every unfinished problem at once (Engine::value_batch,
// tangent_batch), the same contraction of all problems in one group, and each Newton step's
// Krylov iterations advance together until every problem's forcing condition holds. Every
// problem starts from the generalised MP2 guess; on_done(k, status) is called as problem k
// finishes, with t[k] holding its amplitudes and reps[k] its report. The arithmetic of each
// problem is that of solve(), so the results are the same. cancel (may be null): per-problem
// flags another thread may set; a cancelled problem stops at its next Newton iteration.
int solve_batch(const Exec& ex, const std::vector<System*>& sys, const std::vector<Engine*>& eng,
                const cc_solve_opts& opt, const std::vector<double*>& t, std::vector<cc_report>& reps,
                const std::function<void(int, int)>& on_done,
                const std::vector<const std::atomic<int>*>* cancel = nullptr);

// Host helpers
double host_dot(const Exec& ex, size_t n, const double* x, const double* y, double* dev_tmp, double* scratch);

}  // namespace ccpnk
