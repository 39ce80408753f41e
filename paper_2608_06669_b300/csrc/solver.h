// Linear and nonlinear solvers of the Newton-Krylov family (host control, device vectors).
#pragma once

#include <atomic>
#include <functional>

#include "ccsd.h"

namespace ccpnk {

struct SolveStats {
  int residual_evals = 0, jvps = 0, af_applies = 0, krylov_iters = 0, newton_iters = 0;
};

// y = Op(x) on amplitude-length device vectors
using LinOp = std::function<void(const double* x, double* y)>;

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

// Host helpers
double host_dot(const Exec& ex, size_t n, const double* x, const double* y, double* dev_tmp, double* scratch);

}  // namespace ccpnk
