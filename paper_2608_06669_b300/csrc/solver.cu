// Solvers for the CC equations: inner GMRES on A_F, Newton-Krylov (NK, PNK, INK) with
// Eisenstat-Walker forcing (Algorithm 1, App. F.1), and the fixed-point + level shift + DIIS
// baseline (Eq. mo_fixed-point_update, App. D). Control flow and the small Hessenberg / DIIS
// systems live on the host; every vector operation and operator application runs on the
// device. One device->host copy of a few scalars per Krylov step is the only synchronisation.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "solver.h"

namespace ccpnk {

namespace {

void d2h(const Exec& ex, double* host, const double* dev, size_t n) {
  CC_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
  CC_CUDA(cudaStreamSynchronize(ex.stream));
}

// Symmetric eigendecomposition by cyclic Jacobi rotations (host, small matrices):
// A = V diag(w) V^T, V column eigenvectors stored row-major V[r * n + c].
void jacobi_eigh(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int r, int c) -> double& { return A[(size_t)r * n + c]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        tot += a(p, q) * a(p, q);
        if (p != q) off += a(p, q) * a(p, q);
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a(i, i);
}

}  // namespace

double host_dot(const Exec& ex, size_t n, const double* x, const double* y, double* dev_tmp, double* scratch) {
  k_dot(ex, n, x, y, dev_tmp, scratch);
  double h;
  d2h(ex, &h, dev_tmp, 1);
  return h;
}

Gmres::Gmres(const Exec& ex, size_t n, int m_max, double* V, double* small, double* scratch)
    : ex_(ex), n_(n), m_(m_max), V_(V), small_(small), scratch_(scratch) {}

bool Gmres::start(const double* b, double* x, double rtol) {
  // small: device array of >= 2 * (m_max + 1) + 2 doubles
  x_ = x;
  rtol_ = rtol;
  j_ = 0;
  k_dot(ex_, n_, b, b, small_, scratch_);
  double beta2;
  d2h(ex_, &beta2, small_, 1);
  beta_ = std::sqrt(beta2);
  est_ = beta_;
  k_fill(ex_, n_, 0.0, x);
  if (beta_ == 0.0 || m_ <= 0) return false;
  k_axpby(ex_, n_, 1.0 / beta_, b, 0.0, V_);
  H_.assign((size_t)(m_ + 1) * m_, 0.0);
  cs_.assign(m_, 0.0);
  sn_.assign(m_, 0.0);
  g_.assign(m_ + 1, 0.0);
  g_[0] = beta_;
  hh_.assign(2 * (m_ + 1) + 1, 0.0);
  return true;
}

bool Gmres::step() {
  auto Hc = [&](int r, int c) -> double& { return H_[(size_t)c * (m_ + 1) + r]; };
  const int j = j_;
  double* w = V_ + (size_t)(j + 1) * n_;
  // CGS2: two passes of classical Gram-Schmidt against V[0..j]
  double* h1 = small_;
  double* h2 = small_ + (m_ + 1);
  double* nn = small_ + 2 * (m_ + 1);
  k_multi_dot(ex_, j + 1, n_, V_, n_, w, h1, scratch_);
  k_multi_axpy(ex_, j + 1, n_, V_, n_, h1, w);
  k_multi_dot(ex_, j + 1, n_, V_, n_, w, h2, scratch_);
  k_multi_axpy(ex_, j + 1, n_, V_, n_, h2, w);
  k_dot(ex_, n_, w, w, nn, scratch_);
  d2h(ex_, hh_.data(), small_, 2 * (m_ + 1) + 1);
  for (int i = 0; i <= j; ++i) Hc(i, j) = hh_[i] + hh_[(m_ + 1) + i];
  const double hn = std::sqrt(std::max(hh_[2 * (m_ + 1)], 0.0));
  Hc(j + 1, j) = hn;
  // previous Givens rotations on the new column, then a new one for H[j+1][j]
  for (int i = 0; i < j; ++i) {
    const double a = Hc(i, j), c = Hc(i + 1, j);
    Hc(i, j) = cs_[i] * a + sn_[i] * c;
    Hc(i + 1, j) = -sn_[i] * a + cs_[i] * c;
  }
  const double a = Hc(j, j), c = Hc(j + 1, j);
  const double r = std::hypot(a, c);
  cs_[j] = r > 0 ? a / r : 1.0;
  sn_[j] = r > 0 ? c / r : 0.0;
  Hc(j, j) = r;
  Hc(j + 1, j) = 0.0;
  g_[j + 1] = -sn_[j] * g_[j];
  g_[j] = cs_[j] * g_[j];
  est_ = std::fabs(g_[j + 1]);
  j_ = j + 1;
  if (hn > 0.0) k_scale(ex_, n_, 1.0 / hn, w);
  return j_ < m_ && est_ > rtol_ * beta_ && hn != 0.0 && std::isfinite(est_);
}

int Gmres::finish() {
  auto Hc = [&](int r, int c) -> double& { return H_[(size_t)c * (m_ + 1) + r]; };
  const int steps = j_;
  if (steps == 0) return 0;
  // back substitution for y, then x = V y
  std::vector<double> y(steps, 0.0);
  for (int i = steps - 1; i >= 0; --i) {
    double sum = g_[i];
    for (int k = i + 1; k < steps; ++k) sum -= Hc(i, k) * y[k];
    y[i] = Hc(i, i) != 0.0 ? sum / Hc(i, i) : 0.0;
  }
  for (int i = 0; i < steps; ++i) y[i] = -y[i];  // multi_axpy subtracts
  CC_CUDA(cudaMemcpyAsync(small_, y.data(), steps * sizeof(double), cudaMemcpyHostToDevice, ex_.stream));
  k_multi_axpy(ex_, steps, n_, V_, n_, small_, x_);
  CC_CUDA(cudaStreamSynchronize(ex_.stream));  // y lives on the host stack
  return steps;
}

int gmres(const Exec& ex, size_t n, const LinOp& op, const double* b, double* x, double rtol, int m_max,
          double* V, double* small, double* scratch, double* est_out) {
  Gmres gm(ex, n, m_max, V, small, scratch);
  if (gm.start(b, x, rtol)) {
    do {
      op(gm.in(), gm.out());
    } while (gm.step());
  }
  const int steps = gm.finish();
  if (est_out) *est_out = gm.est();
  return steps;
}

// ---------------------------------------------------------------------------
// A_F^{-1}
// ---------------------------------------------------------------------------
namespace {

void ensure_eig(const Exec& ex, System& s) {
  if (s.eig_ready) return;
  const int o = s.o, v = s.v, n = s.n;
  std::vector<double> f((size_t)n * n);
  d2h(ex, f.data(), s.f.p, f.size());
  std::vector<double> Ao((size_t)o * o), Av((size_t)v * v), Vo, Vv;
  for (int i = 0; i < o; ++i)
    for (int j = 0; j < o; ++j) Ao[(size_t)i * o + j] = 0.5 * (f[(size_t)i * n + j] + f[(size_t)j * n + i]);
  for (int a = 0; a < v; ++a)
    for (int b = 0; b < v; ++b)
      Av[(size_t)a * v + b] = 0.5 * (f[(size_t)(o + a) * n + o + b] + f[(size_t)(o + b) * n + o + a]);
  jacobi_eigh(o, Ao, s.eo, Vo);
  jacobi_eigh(v, Av, s.ev, Vv);
  s.Uo.alloc(ex.pool, (size_t)o * o);
  s.Uv.alloc(ex.pool, (size_t)v * v);
  CC_CUDA(cudaMemcpyAsync(s.Uo.p, Vo.data(), Vo.size() * sizeof(double), cudaMemcpyHostToDevice, ex.stream));
  CC_CUDA(cudaMemcpyAsync(s.Uv.p, Vv.data(), Vv.size() * sizeof(double), cudaMemcpyHostToDevice, ex.stream));
  std::vector<double> e(s.eo);
  e.insert(e.end(), s.ev.begin(), s.ev.end());
  s.eig_d.alloc(ex.pool, e.size());
  CC_CUDA(cudaMemcpyAsync(s.eig_d.p, e.data(), e.size() * sizeof(double), cudaMemcpyHostToDevice, ex.stream));
  CC_CUDA(cudaStreamSynchronize(ex.stream));
  s.eig_ready = true;
}

__global__ void eig_divide_kernel(int o, int v, const double* __restrict__ eo, const double* __restrict__ ev,
                                  double shift, double* __restrict__ x) {
  size_t n1 = (size_t)o * v, n2 = (size_t)o * o * v * v;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n1 + n2; e += (size_t)gridDim.x * blockDim.x) {
    if (e < n1) {
      int a = (int)(e % v), i = (int)(e / v);
      x[e] /= (ev[a] - eo[i] + shift);
    } else {
      size_t q = e - n1;
      int b = (int)(q % v);
      size_t r = q / v;
      int a = (int)(r % v);
      r /= v;
      int j = (int)(r % o), i = (int)(r / o);
      x[e] /= (ev[a] + ev[b] - eo[i] - eo[j] + shift);
    }
  }
}

}  // namespace

// x = (A_F + shift)^{-1} b: A_F is a sum of commuting Kronecker terms of the occupied and
// virtual Fock blocks, so it is diagonal in their eigenbases.
void solve_AF_direct(const Exec& ex, System& s, const double* bin, double* x, double shift, double* work,
                     cc_precision prec) {
  ensure_eig(ex, s);
  const int o = s.o, v = s.v;
  const size_t ov = (size_t)o * v;
  double* b = const_cast<double*>(bin);
  auto Uo = [&](const char* l) { return view(s.Uo.p, l, {o, o}); };
  auto Uv = [&](const char* l) { return view(s.Uv.p, l, {v, v}); };
  const cc_precision rp = prec;
  // rotate in: c = Uo^T b Uv (singles), Uo^T Uo^T b Uv Uv (doubles)
  double* w1 = work;
  double* w2 = work + s.namp();
  contract(ex, rp, 1.0, view(b, "kc", {o, v}), Uv("ca"), 0.0, view(w1, "ka", {o, v}));
  contract(ex, rp, 1.0, Uo("ki"), view(w1, "ka", {o, v}), 0.0, view(x, "ia", {o, v}));
  contract(ex, rp, 1.0, view(b + ov, "klcd", {o, o, v, v}), Uv("db"), 0.0, view(w2, "klcb", {o, o, v, v}));
  contract(ex, rp, 1.0, Uv("ca"), view(w2, "klcb", {o, o, v, v}), 0.0, view(w1 + ov, "klab", {o, o, v, v}));
  contract(ex, rp, 1.0, view(w1 + ov, "klab", {o, o, v, v}), Uo("lj"), 0.0, view(w2, "kjab", {o, o, v, v}));
  contract(ex, rp, 1.0, Uo("ki"), view(w2, "kjab", {o, o, v, v}), 0.0, view(x + ov, "ijab", {o, o, v, v}));
  // divide by the eigenvalue differences
  const double* ed = s.eig_d.p;
  int blocks = std::min<size_t>((s.namp() + 255) / 256, (size_t)ex.sm_count * 8);
  eig_divide_kernel<<<blocks, 256, 0, ex.stream>>>(o, v, ed, ed + o, shift, x);
  ex.count();
  CC_CUDA(cudaGetLastError());
  // rotate back: b' = Uo c Uv^T
  contract(ex, rp, 1.0, view(x, "ia", {o, v}), Uv("ca"), 0.0, view(w1, "ic", {o, v}));
  contract(ex, rp, 1.0, Uo("ki"), view(w1, "ic", {o, v}), 0.0, view(x, "kc", {o, v}));
  contract(ex, rp, 1.0, view(x + ov, "ijab", {o, o, v, v}), Uv("db"), 0.0, view(w2, "ijad", {o, o, v, v}));
  contract(ex, rp, 1.0, Uv("ca"), view(w2, "ijad", {o, o, v, v}), 0.0, view(w1 + ov, "ijcd", {o, o, v, v}));
  contract(ex, rp, 1.0, view(w1 + ov, "ijcd", {o, o, v, v}), Uo("lj"), 0.0, view(w2, "ilcd", {o, o, v, v}));
  contract(ex, rp, 1.0, Uo("ki"), view(w2, "ilcd", {o, o, v, v}), 0.0, view(x + ov, "klcd", {o, o, v, v}));
  if (rp != CC_FP64) {
    // A_F maps amplitudes with t_ij^ab = t_ji^ba to such amplitudes, and so does its exact
    // inverse; rotations rounded on the tensor cores do not quite, so restore the symmetry
    const size_t n2 = (size_t)o * o * v * v;
    k_sym_add(ex, o, v, x + ov, w2, 0.0);
    k_axpby(ex, n2, 0.5, w2, 0.0, x + ov);
  }
}

void solve_AF(const Exec& ex, System& s, const double* b, double* x, cc_precision prec, double rtol, int m_max,
              bool direct, SolveStats* st) {
  const size_t n = s.namp();
  if (direct) {
    DBuf<double> work(ex.pool, 2 * n);
    solve_AF_direct(ex, s, b, x, 0.0, work.p, prec);
    if (st) st->af_applies += 1;
    return;
  }
  DBuf<double> V(ex.pool, (size_t)(m_max + 1) * n);
  DBuf<double> small(ex.pool, 2 * (size_t)(m_max + 1) + 8);
  DBuf<double> scratch(ex.pool, (size_t)(m_max + 1) * 1024 + 1024);
  int applies = 0;
  LinOp op = [&](const double* xi, double* yo) {
    apply_AF(ex, s, xi, yo, prec);
    ++applies;
  };
  gmres(ex, n, op, b, x, rtol, m_max, V.p, small.p, scratch.p);
  if (st) st->af_applies += applies;
}

// ---------------------------------------------------------------------------
// nonlinear solvers
// ---------------------------------------------------------------------------
int solve(const Exec& ex, System& s, Engine& eng, const cc_solve_opts& opt, double* t, cc_report* rep,
          bool use_guess, const std::atomic<int>* cancel) {
  auto t_start = std::chrono::steady_clock::now();
  const size_t n = s.namp();
  const int o = s.o, v = s.v;
  SolveStats st;
  DBuf<double> r(ex.pool, n), tmp(ex.pool, n), dev(ex.pool, 16);
  DBuf<double> red(ex.pool, 64 * 1024);
  double* scratch = red.p;
  double inner_rtol = opt.inner_rtol > 0 ? opt.inner_rtol
                                         : (opt.prec == CC_MIXED_TF32 ? 1e-6 : opt.prec == CC_MIXED_BF16X3 ? 1e-7 : opt.prec == CC_MIXED_TF32X3 ? 1e-8 : 1e-12);
  int inner_max = opt.inner_max > 0 ? opt.inner_max : 50;
  const size_t n1 = (size_t)o * v;  // the singles block, dropped in CCD mode
  // Every vector the Newton-Krylov iteration builds keeps t_ij^ab = t_ji^ba: R and J produce
  // such vectors exactly (their doubles are symmetrised sums), and so would an exact A_F^{-1}.
  // Inverses rounded on the tensor cores (mirror elements split or paired differently) are
  // projected back, so the Krylov space never gains a spurious antisymmetric direction. FP64
  // runs are left bit for bit as they are.
  DBuf<double> symw(ex.pool, opt.prec == CC_FP64 ? 0 : n - n1);
  auto AFinv = [&](const double* b, double* x) {
    solve_AF(ex, s, b, x, opt.prec, inner_rtol, inner_max, opt.af_direct != 0, &st);
    if (opt.prec != CC_FP64) {
      k_sym_add(ex, o, v, x + n1, symw.p, 0.0);
      k_axpby(ex, n - n1, 0.5, symw.p, 0.0, x + n1);
    }
  };
  const cc_precision outer = opt.outer_prec == CC_DF64 ? CC_DF64 : opt.outer_prec == CC_FP64_EMU ? CC_FP64_EMU : CC_FP64;
  auto out_of_time = [&]() {
    return opt.max_seconds > 0 &&
           std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() > opt.max_seconds;
  };
  // a cancelled solve stops between outer iterations, like one out of time
  auto cancelled = [&]() { return cancel && cancel->load() != 0; };
  auto residual = [&](const double* tt, double* rr, double* e_host) -> double {
    eng.value(tt, rr, dev.p + 1, outer);
    if (opt.ccd) k_fill(ex, n1, 0.0, rr);
    st.residual_evals++;
    k_dot(ex, n, rr, rr, dev.p, scratch);
    double hv[2];
    d2h(ex, hv, dev.p, 2);
    if (e_host) *e_host = hv[1];
    return std::sqrt(std::max(hv[0], 0.0));
  };

  // generalised MP2 start (Eq. inexact_newton_update at t = 0): t = A_F^{-1}(-R(0)). At t = 0
  // every amplitude term of the residual vanishes: R1(0)_i^a = f_ia and R2(0)_ij^ab = (ia|jb),
  // so the start needs no residual evaluation (t1 stays 0 in CCD mode and whenever f_ov = 0).
  if (!use_guess) {
    k_fill(ex, n, 0.0, t);
    if (opt.ccd) {
      k_fill(ex, n1, 0.0, r.p);
    } else {
      k_copy2d(ex, o, v, s.f.p + o, s.n, r.p, v);
      k_scale(ex, n1, -1.0, r.p);
    }
    k_ovov_to_oovv(ex, o, v, s.Govov.p, r.p + n1, -1.0);
    AFinv(r.p, t);
  } else if (opt.ccd) {
    k_fill(ex, n1, 0.0, t);
  }

  // the JVPs of the Newton family replay CUDA graphs of the tangent program (released on return)
  struct GraphWindow {
    Engine& e;
    ~GraphWindow() { e.end_graphs(); }
  } window{eng};
  if (ex.graphs && !opt.jvp_fd && (opt.method == CC_NK || opt.method == CC_PNK)) eng.begin_graphs(opt.prec);

  double energy = 0.0, rn = 0.0, rn_prev = 0.0, eta_prev = opt.eta_max;
  int status = CC_ERR_NOT_CONVERGED;
  // no point asking the linear solve for more than its operator's precision delivers
  const double eta_min = opt.prec == CC_MIXED_TF32 ? 1e-4 : opt.prec == CC_MIXED_BF16X3 ? 1e-5 : opt.prec == CC_MIXED_TF32X3 ? 1e-7 : 1e-10;
  const int m_max = std::max(1, opt.m_max);

  if (opt.method == CC_FP_DIIS) {
    const int nd = std::max(0, opt.diis_size);
    DBuf<double> vecs(ex.pool, (size_t)std::max(nd, 1) * n), errs(ex.pool, (size_t)std::max(nd, 1) * n);
    DBuf<double> fdiag(ex.pool, s.n);
    k_copy(ex, s.n, s.fdiag.p, fdiag.p);
    std::vector<double> Bm((size_t)std::max(nd, 1) * std::max(nd, 1), 0.0);
    DBuf<double> rowdev(ex.pool, std::max(nd, 1));
    int count = 0, head = 0;
    for (int it = 0; it < opt.max_outer; ++it) {
      rn = residual(t, r.p, &energy);
      if (opt.verbose) fprintf(stderr, "[ccpnk] fp+diis it %3d  |R| %.3e  E %.12f\n", it, rn, energy);
      if (!std::isfinite(rn) || rn > 1e8) { status = CC_ERR_DIVERGED; break; }
      if (rn < opt.tol) { status = CC_OK; break; }
      if (out_of_time()) break;
      if (cancelled()) { status = CC_ERR_CANCELLED; break; }
      st.newton_iters++;
      // e = -R / (D + shift), t_new = t + e
      k_denom_divide(ex, o, v, fdiag.p, opt.level_shift, r.p, r.p + (size_t)o * v, tmp.p, tmp.p + (size_t)o * v, -1.0);
      if (nd < 1) {
        k_axpby(ex, n, 1.0, tmp.p, 1.0, t);
        continue;
      }
      double* vslot = vecs.p + (size_t)head * n;
      double* eslot = errs.p + (size_t)head * n;
      k_copy(ex, n, tmp.p, eslot);
      k_copy(ex, n, t, vslot);
      k_axpby(ex, n, 1.0, tmp.p, 1.0, vslot);
      count = std::min(count + 1, nd);
      // new row of the error overlap matrix
      std::vector<double> row(nd);
      k_multi_dot(ex, count, n, errs.p, n, eslot, rowdev.p, scratch);
      d2h(ex, row.data(), rowdev.p, count);
      for (int k = 0; k < count; ++k) {
        Bm[(size_t)head * nd + k] = row[k];
        Bm[(size_t)k * nd + head] = row[k];
      }
      head = (head + 1) % nd;
      if (it < 2 || count < 2) {
        k_copy(ex, n, vslot, t);
        continue;
      }
      // Pulay: minimise |sum c_k e_k| with sum c_k = 1 (Lagrange row), solved by Gaussian elimination
      std::vector<int> slots;
      for (int k = 0; k < count; ++k) slots.push_back(k);
      int m = count + 1;
      std::vector<double> A((size_t)m * m, 0.0), rhs(m, 0.0);
      double scale = 0.0;
      for (int a = 0; a < count; ++a) scale = std::max(scale, std::fabs(Bm[(size_t)slots[a] * nd + slots[a]]));
      if (scale == 0.0) scale = 1.0;
      for (int a = 0; a < count; ++a) {
        for (int b = 0; b < count; ++b) A[(size_t)a * m + b] = Bm[(size_t)slots[a] * nd + slots[b]] / scale;
        A[(size_t)a * m + count] = -1.0;
        A[(size_t)count * m + a] = -1.0;
      }
      rhs[count] = -1.0;
      // partial-pivot elimination
      bool ok = true;
      for (int c = 0; c < m && ok; ++c) {
        int p = c;
        for (int rr = c + 1; rr < m; ++rr)
          if (std::fabs(A[(size_t)rr * m + c]) > std::fabs(A[(size_t)p * m + c])) p = rr;
        if (std::fabs(A[(size_t)p * m + c]) < 1e-300) { ok = false; break; }
        if (p != c) {
          for (int k = 0; k < m; ++k) std::swap(A[(size_t)p * m + k], A[(size_t)c * m + k]);
          std::swap(rhs[p], rhs[c]);
        }
        for (int rr = c + 1; rr < m; ++rr) {
          double f = A[(size_t)rr * m + c] / A[(size_t)c * m + c];
          for (int k = c; k < m; ++k) A[(size_t)rr * m + k] -= f * A[(size_t)c * m + k];
          rhs[rr] -= f * rhs[c];
        }
      }
      if (!ok) {
        k_copy(ex, n, vslot, t);
        continue;
      }
      std::vector<double> c(m, 0.0);
      for (int i = m - 1; i >= 0; --i) {
        double sum = rhs[i];
        for (int k = i + 1; k < m; ++k) sum -= A[(size_t)i * m + k] * c[k];
        c[i] = sum / A[(size_t)i * m + i];
      }
      // t = sum_k c_k vecs_k (multi_axpy subtracts, so pass -c)
      std::vector<double> negc(nd, 0.0);
      for (int a = 0; a < count; ++a) negc[slots[a]] = -c[a];
      DBuf<double> cd(ex.pool, nd);
      CC_CUDA(cudaMemcpyAsync(cd.p, negc.data(), nd * sizeof(double), cudaMemcpyHostToDevice, ex.stream));
      k_fill(ex, n, 0.0, t);
      k_multi_axpy(ex, count, n, vecs.p, n, cd.p, t);
      CC_CUDA(cudaStreamSynchronize(ex.stream));
    }
  } else {
    // Newton family
    for (int k = 0; k < opt.max_outer; ++k) {
      rn = residual(t, r.p, &energy);
      if (opt.verbose) fprintf(stderr, "[ccpnk] newton %3d  |R| %.3e  E %.12f  eta %.2e\n", k, rn, energy, eta_prev);
      if (!std::isfinite(rn) || rn > 1e8) { status = CC_ERR_DIVERGED; break; }
      if (rn < opt.tol) { status = CC_OK; break; }
      if (out_of_time()) break;
      if (cancelled()) { status = CC_ERR_CANCELLED; break; }
      st.newton_iters++;
      if (opt.method == CC_INK) {
        // t <- t + A_F^{-1}(-r)
        k_scale(ex, n, -1.0, r.p);
        AFinv(r.p, tmp.p);
        k_axpby(ex, n, 1.0, tmp.p, 1.0, t);
        rn_prev = rn;
        continue;
      }
      // Eisenstat-Walker forcing (App. F.1) with the usual safeguard
      double eta = opt.eta_max;
      if (k > 0 && rn_prev > 0) {
        eta = opt.gamma * std::pow(rn / rn_prev, opt.alpha);
        double sg = opt.gamma * std::pow(eta_prev, opt.alpha);
        if (sg > 0.1) eta = std::max(eta, sg);
      }
      eta = std::min(std::max(eta, eta_min), opt.eta_max);
      eta_prev = eta;
      rn_prev = rn;
      const bool pre = opt.method == CC_PNK;
      DBuf<double> z(ex.pool, n);
      if (pre) AFinv(r.p, z.p);
      else k_copy(ex, n, r.p, z.p);
      DBuf<double> V(ex.pool, (size_t)(m_max + 1) * n), small(ex.pool, 2 * (size_t)(m_max + 1) + 8);
      DBuf<double> sc(ex.pool, (size_t)(m_max + 1) * 1024 + 1024);
      DBuf<double> jq(ex.pool, n), tp(ex.pool, n);
      double tnorm = 0.0;
      if (opt.jvp_fd) tnorm = std::sqrt(host_dot(ex, n, t, t, dev.p, scratch));
      LinOp op = [&](const double* q, double* w) {
        double* target = pre ? jq.p : w;
        if (opt.jvp_fd) {
          // J q ~ (R(t + delta q) - R(t)) / delta, delta = sqrt(eps)(1 + |t|) for unit q
          double delta = 1.4901161193847656e-08 * (1.0 + tnorm);
          k_copy(ex, n, t, tp.p);
          k_axpby(ex, n, delta, q, 1.0, tp.p);
          eng.value(tp.p, target, nullptr, outer);
          st.residual_evals++;
          k_axpby(ex, n, -1.0 / delta, r.p, 1.0 / delta, target);
        } else {
          eng.tangent(q, target, opt.prec);
        }
        st.jvps++;
        if (opt.ccd) k_fill(ex, n1, 0.0, target);
        if (pre) AFinv(jq.p, w);
      };
      DBuf<double> delta(ex.pool, n);
      int steps = gmres(ex, n, op, z.p, delta.p, eta, m_max, V.p, small.p, sc.p);
      st.krylov_iters += steps;
      // t <- t - sum_i q_i y_i (Algorithm 1)
      k_axpby(ex, n, -1.0, delta.p, 1.0, t);
    }
  }

  auto t_end = std::chrono::steady_clock::now();
  if (rep) {
    rep->energy = energy;
    rep->res_norm = rn;
    rep->newton_iters = st.newton_iters;
    rep->residual_evals = st.residual_evals;
    rep->jvps = st.jvps;
    rep->af_applies = st.af_applies;
    rep->krylov_iters = st.krylov_iters;
    rep->status = status;
    rep->seconds = std::chrono::duration<double>(t_end - t_start).count();
  }
  return status;
}

// ---------------------------------------------------------------------------
// several NK / PNK solves in lockstep
// ---------------------------------------------------------------------------
int solve_batch(const Exec& ex, const std::vector<System*>& sys, const std::vector<Engine*>& eng,
                const cc_solve_opts& opt, const std::vector<double*>& t, std::vector<cc_report>& reps,
                const std::function<void(int, int)>& on_done, const std::vector<const std::atomic<int>*>* cancel) {
  const int K = (int)sys.size();
  reps.assign(K, cc_report{});
  auto cancel_of = [&](int k) -> const std::atomic<int>* { return cancel && (int)cancel->size() > k ? (*cancel)[k] : nullptr; };
  if ((opt.method != CC_NK && opt.method != CC_PNK) || opt.jvp_fd || K <= 1) {
    for (int k = 0; k < K; ++k) {
      const int st = solve(ex, *sys[k], *eng[k], opt, t[k], &reps[k], false, cancel_of(k));
      if (on_done) on_done(k, st);
    }
    return CC_OK;
  }
  auto t_start = std::chrono::steady_clock::now();
  const double inner_rtol = opt.inner_rtol > 0 ? opt.inner_rtol
                            : (opt.prec == CC_MIXED_TF32 ? 1e-6 : opt.prec == CC_MIXED_BF16X3 ? 1e-7
                               : opt.prec == CC_MIXED_TF32X3 ? 1e-8 : 1e-12);
  const int inner_max = opt.inner_max > 0 ? opt.inner_max : 50;
  const double eta_min = opt.prec == CC_MIXED_TF32 ? 1e-4 : opt.prec == CC_MIXED_BF16X3 ? 1e-5
                         : opt.prec == CC_MIXED_TF32X3 ? 1e-7 : 1e-10;
  const int m_max = std::max(1, opt.m_max);
  const cc_precision outer = opt.outer_prec == CC_DF64 ? CC_DF64 : opt.outer_prec == CC_FP64_EMU ? CC_FP64_EMU : CC_FP64;
  const bool pre = opt.method == CC_PNK;
  struct Slot {
    System* s;
    Engine* e;
    double* t;
    size_t n = 0, n1 = 0;
    DBuf<double> r, dev, red, symw, z, V, small, sc, jq, delta;
    SolveStats st;
    double energy = 0, rn = 0, rn_prev = 0, eta_prev = 0;
    int status = CC_ERR_NOT_CONVERGED;
    bool done = false, running = false;
    std::unique_ptr<Gmres> gm;
  };
  std::vector<std::unique_ptr<Slot>> slots;
  for (int k = 0; k < K; ++k) {
    std::unique_ptr<Slot> q(new Slot);
    q->s = sys[k];
    q->e = eng[k];
    q->t = t[k];
    q->n = q->s->namp();
    q->n1 = (size_t)q->s->o * q->s->v;
    q->r.alloc(ex.pool, q->n);
    q->dev.alloc(ex.pool, 16);
    q->red.alloc(ex.pool, 64 * 1024);
    q->symw.alloc(ex.pool, opt.prec == CC_FP64 ? 0 : q->n - q->n1);
    q->z.alloc(ex.pool, q->n);
    q->V.alloc(ex.pool, (size_t)(m_max + 1) * q->n);
    q->small.alloc(ex.pool, 2 * (size_t)(m_max + 1) + 8);
    q->sc.alloc(ex.pool, (size_t)(m_max + 1) * 1024 + 1024);
    q->jq.alloc(ex.pool, q->n);
    q->delta.alloc(ex.pool, q->n);
    q->eta_prev = opt.eta_max;
    slots.push_back(std::move(q));
  }
  // A_F^{-1} of one slot, projected back onto t_ij^ab = t_ji^ba at the tensor-core precisions
  auto AFinv = [&](Slot& q, const double* b, double* x) {
    solve_AF(ex, *q.s, b, x, opt.prec, inner_rtol, inner_max, opt.af_direct != 0, &q.st);
    if (opt.prec != CC_FP64) {
      const int o = q.s->o, v = q.s->v;
      k_sym_add(ex, o, v, x + q.n1, q.symw.p, 0.0);
      k_axpby(ex, q.n - q.n1, 0.5, q.symw.p, 0.0, x + q.n1);
    }
  };
  auto finish = [&](Slot& q, int k) {
    cc_report& rep = reps[k];
    rep.energy = q.energy;
    rep.res_norm = q.rn;
    rep.newton_iters = q.st.newton_iters;
    rep.residual_evals = q.st.residual_evals;
    rep.jvps = q.st.jvps;
    rep.af_applies = q.st.af_applies;
    rep.krylov_iters = q.st.krylov_iters;
    rep.status = q.status;
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    q.done = true;
    if (on_done) on_done(k, q.status);
  };
  // the generalised MP2 start of every problem (as in solve)
  for (auto& qp : slots) {
    Slot& q = *qp;
    const int o = q.s->o, v = q.s->v;
    k_fill(ex, q.n, 0.0, q.t);
    if (opt.ccd) {
      k_fill(ex, q.n1, 0.0, q.r.p);
    } else {
      k_copy2d(ex, o, v, q.s->f.p + o, q.s->n, q.r.p, v);
      k_scale(ex, q.n1, -1.0, q.r.p);
    }
    k_ovov_to_oovv(ex, o, v, q.s->Govov.p, q.r.p + q.n1, -1.0);
    AFinv(q, q.r.p, q.t);
  }
  for (int it = 0; it < opt.max_outer; ++it) {
    std::vector<int> act;
    for (int k = 0; k < K; ++k)
      if (!slots[k]->done) act.push_back(k);
    if (act.empty()) break;
    // the residuals of every unfinished problem, evaluated together
    std::vector<Engine*> es;
    std::vector<const double*> ts;
    std::vector<double*> rs, eds;
    for (int k : act) {
      es.push_back(slots[k]->e);
      ts.push_back(slots[k]->t);
      rs.push_back(slots[k]->r.p);
      eds.push_back(slots[k]->dev.p + 1);
    }
    Engine::value_batch(es, ts, rs, eds, outer);
    const bool late = opt.max_seconds > 0 &&
                      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count() > opt.max_seconds;
    std::vector<int> go;
    for (int k : act) {
      Slot& q = *slots[k];
      if (opt.ccd) k_fill(ex, q.n1, 0.0, q.r.p);
      q.st.residual_evals++;
      k_dot(ex, q.n, q.r.p, q.r.p, q.dev.p, q.red.p);
      double hv[2];
      d2h(ex, hv, q.dev.p, 2);
      q.energy = hv[1];
      q.rn = std::sqrt(std::max(hv[0], 0.0));
      if (opt.verbose) fprintf(stderr, "[ccpnk] batch %d newton %3d  |R| %.3e  E %.12f\n", k, it, q.rn, q.energy);
      if (!std::isfinite(q.rn) || q.rn > 1e8) {
        q.status = CC_ERR_DIVERGED;
        finish(q, k);
      } else if (q.rn < opt.tol) {
        q.status = CC_OK;
        finish(q, k);
      } else if (late) {
        finish(q, k);
      } else if (cancel_of(k) && cancel_of(k)->load() != 0) {
        q.status = CC_ERR_CANCELLED;
        finish(q, k);
      } else {
        go.push_back(k);
      }
    }
    // one Newton step for each of the others, their Krylov iterations in lockstep
    for (int k : go) {
      Slot& q = *slots[k];
      q.st.newton_iters++;
      double eta = opt.eta_max;
      if (it > 0 && q.rn_prev > 0) {
        eta = opt.gamma * std::pow(q.rn / q.rn_prev, opt.alpha);
        const double sg = opt.gamma * std::pow(q.eta_prev, opt.alpha);
        if (sg > 0.1) eta = std::max(eta, sg);
      }
      eta = std::min(std::max(eta, eta_min), opt.eta_max);
      q.eta_prev = eta;
      q.rn_prev = q.rn;
      if (pre) AFinv(q, q.r.p, q.z.p);
      else k_copy(ex, q.n, q.r.p, q.z.p);
      q.gm.reset(new Gmres(ex, q.n, m_max, q.V.p, q.small.p, q.sc.p));
      q.running = q.gm->start(q.z.p, q.delta.p, eta);
    }
    while (true) {
      std::vector<int> run;
      for (int k : go)
        if (slots[k]->running) run.push_back(k);
      if (run.empty()) break;
      std::vector<Engine*> je;
      std::vector<const double*> jin;
      std::vector<double*> jout;
      for (int k : run) {
        Slot& q = *slots[k];
        je.push_back(q.e);
        jin.push_back(q.gm->in());
        jout.push_back(pre ? q.jq.p : q.gm->out());
      }
      Engine::tangent_batch(je, jin, jout, opt.prec);
      for (int k : run) {
        Slot& q = *slots[k];
        q.st.jvps++;
        if (opt.ccd) k_fill(ex, q.n1, 0.0, pre ? q.jq.p : q.gm->out());
        if (pre) AFinv(q, q.jq.p, q.gm->out());
        q.running = q.gm->step();
      }
    }
    for (int k : go) {
      Slot& q = *slots[k];
      q.st.krylov_iters += q.gm->finish();
      // t <- t - sum_i q_i y_i (Algorithm 1)
      k_axpby(ex, q.n, -1.0, q.delta.p, 1.0, q.t);
    }
  }
  for (int k = 0; k < K; ++k)
    if (!slots[k]->done) finish(*slots[k], k);
  CC_CUDA(cudaStreamSynchronize(ex.stream));
  return CC_OK;
}

}  // namespace ccpnk
