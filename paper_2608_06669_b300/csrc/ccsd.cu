// Closed-shell CCSD residual over density-fitted integrals, and its exact linearisation.
//
// The residual (Eq. CC_ampl projected on singles and doubles) is evaluated in the
// T1-similarity-transformed form: the DF factor is dressed, Bt[P] = X B[P] Y with
// X = 1 - t1, Y = 1 + t1 acting on the virtual-occupied block, which turns every singles
// contribution into dressed integrals; the doubles residual is then the CCD residual of the
// paper's App. A (ladders, rings, Fock-like intermediates, the Omega permutation) over the
// dressed Hamiltonian, and the singles residual has four terms. Integrals are never formed
// beyond o^2 v^2 blocks: the particle-particle ladder builds (ac|bd) for a block of a at a
// time from Bt and contracts it at once.
//
// One program serves both the residual and the Jacobian-vector product: run in value mode it
// computes R(t) and keeps every intermediate; run in tangent mode it computes the directional
// derivative of each step, where a bilinear contraction C = A B becomes dA B + A dB
// (App. B, Eq. AnalyticJVP) and the values of A and B are those kept from the residual at t.
#include <algorithm>
#include <cmath>
#include <functional>

#include "ccsd.h"

namespace ccpnk {

void k_transpose(const Exec& ex, int batch, int rows, int cols, const double* in, long long in_bs,
                 long long in_ld, double* out, long long out_bs, long long out_ld);
void k_copy3d(const Exec& ex, int batch, int rows, int cols, const double* src, long long sbs, long long sld,
              double* dst, long long dbs, long long dld);

void system_init(const Exec& ex, System& s, int o, int v, int P, const double* f, const double* B) {
  s.o = o;
  s.v = v;
  s.n = o + v;
  s.P = P;
  const int n = s.n;
  Pool* pl = ex.pool;
  s.f.alloc(pl, (size_t)n * n);
  s.h.alloc(pl, (size_t)n * n);
  s.fdiag.alloc(pl, n);
  s.Boo.alloc(pl, (size_t)P * o * o);
  s.Bov.alloc(pl, (size_t)P * o * v);
  s.Bvv.alloc(pl, (size_t)P * v * v);
  s.Govov.alloc(pl, (size_t)o * v * o * v);
  s.Lovov.alloc(pl, (size_t)o * v * o * v);
  k_copy(ex, (size_t)n * n, f, s.f.p);
  k_copy3d(ex, 1, n, 1, f, 0, n + 1, s.fdiag.p, 0, 1);  // the diagonal
  k_copy3d(ex, P, o, o, B, (long long)n * n, n, s.Boo.p, (long long)o * o, o);
  k_copy3d(ex, P, o, v, B + o, (long long)n * n, n, s.Bov.p, (long long)o * v, v);
  k_copy3d(ex, P, v, v, B + (size_t)o * n + o, (long long)n * n, n, s.Bvv.p, (long long)v * v, v);
  // h = f - sum_k [2 (pq|kk) - (pk|kq)]
  DBuf<double> gam(pl, P);
  k_trace_batched(ex, P, o, s.Boo.p, gam.p);
  k_copy(ex, (size_t)n * n, f, s.h.p);
  double* Bm = const_cast<double*>(B);
  contract(ex, CC_FP64, -2.0, view(Bm, "Xpq", {P, n, n}), view(gam.p, "X", {P}), 1.0, view(s.h.p, "pq", {n, n}));
  contract(ex, CC_FP64, 1.0, view_strided(Bm, "Xpk", {P, n, o}, {(long long)n * n, n, 1}),
           view_strided(Bm, "Xkq", {P, o, n}, {(long long)n * n, n, 1}), 1.0, view(s.h.p, "pq", {n, n}));
  // (kc|ld) and its exchange combination, constant for the problem
  contract(ex, CC_FP64, 1.0, view(s.Bov.p, "Xkc", {P, o, v}), view(s.Bov.p, "Xld", {P, o, v}), 0.0,
           view(s.Govov.p, "kcld", {o, v, o, v}));
  k_make_L_ovov(ex, o, v, s.Govov.p, s.Lovov.p);
}

size_t stage_cache_cap(int o, int v, int P) {
  const double big = (double)P * v * v + (double)o * o * v * v;
  return (size_t)std::min(1073741824.0, 32.0 * 4.0 * big);
}

// Whether the tensor-core ladder contracts over pairs c <= d (see Engine::ladder): per slab row,
// the MMA time of the plain contraction (o^2 rows, padded to 128-row tiles, against v^2) against
// that of the two pair contractions (i <= j rows against c <= d pairs, i < j against c < d)
// plus the HBM time of the extra pass (the build's FP32 words written and read back, L+- written
// and unpacked).
bool ladder_pack_pays(int o, int v, cc_precision prec) {
  const double rate = prec == CC_MIXED_BF16X3 ? 8e14 : 4e14;  // sustained MMA flop/s of one pass
  const double passes = prec == CC_MIXED_TF32 ? 1.0 : 3.0, hbm = 6e12;
  auto tiles = [](double rows) { return std::ceil(rows / 128.0) * 128.0; };
  const double vv = (double)v * v, Pv = v * (v + 1) / 2.0, Qv = v * (v - 1) / 2.0;
  const double o2 = (double)o * o, Po = o * (o + 1) / 2.0, Qo = o * (o - 1) / 2.0;
  const double plain = 2.0 * tiles(o2) * vv * passes / rate;
  const double packed = 2.0 * (tiles(Po) * Pv + (Qo > 0 ? tiles(Qo) * Qv : 0.0)) * passes / rate +
                        (8.0 * vv + 16.0 * o2) / hbm;
  return packed < plain;
}

constexpr size_t kLadderGroupBytes = (size_t)3 << 29;  // 1.5 GiB of staged slabs at once

int ladder_block_for(int v) {
  const double cap = 2.0 * 1024 * 1024 * 1024;
  const double per_a = 8.0 * (double)v * v * v;
  return std::max(1, std::min((v + 7) / 8, (int)(cap / std::max(per_a, 1.0))));
}

Engine::Engine(const Exec& ex, const System& s) : ex_(ex), s_(s) {
  const int o = s.o, v = s.v, n = s.n, P = s.P;
  const size_t oovv = (size_t)o * o * v * v;
  alloc(t_, s.namp());
  alloc(u_, oovv);
  alloc(Btoo_, (size_t)P * o * o);
  alloc(Btvv_, (size_t)P * v * v);
  alloc(Btvo_, (size_t)P * v * o);
  alloc(gam_, P);
  alloc(hY_, (size_t)n * n);
  alloc(Ft_, (size_t)n * n);
  alloc(Z_, (size_t)P * o * v);
  alloc(Wk_, (size_t)P * o * v);
  alloc(Woo_, (size_t)o * o * o * o);
  alloc(Cint_, oovv);
  alloc(Dint_, oovv);
  alloc(Gv_, (size_t)v * v);
  alloc(Go_, (size_t)o * o);
  alloc(X_, oovv);
  alloc(Y2_, oovv);
  ladder_block_ = ladder_block_for(v);
  rebind(ex);
  W_.alloc(ex.pool, (size_t)ladder_block_ * v * v * v);
  // the tangent's stacked factors [dBt_vv ; Bt_vv] and [Bt_vv ; dBt_vv]
  XsYs_.alloc(ex.pool, 4 * (size_t)P * v * v);
  scratch_.alloc(ex.pool, 64 * 1024);
}

void Engine::rebind(const Exec& ex) {
  ex_ = ex;
  size_t cap = stage_cache_cap(s_.o, s_.v, s_.P);
  if (ex.pool->budget()) cap = std::min(cap, ex.pool->budget() / 8);
  if (ex.stage_cap >= 0) cap = (size_t)ex.stage_cap;
  if (cap < stage_.bytes) stage_.clear();
  stage_.cap = cap;
}

void Engine::alloc(Pair& x, size_t n) {
  x.val.alloc(ex_.pool, n);
  x.tan.alloc(ex_.pool, n);
}

namespace {

// A tensor of the program: its value view and, if it depends on the amplitudes, its tangent view.
struct TP {
  TView v, t;
  bool dyn = false;
};

}  // namespace

void Engine::ladder(const double* Xv, const double* Yv, int Paux, const double* T, double* R, cc_precision prec,
                    bool fixed_xy, bool fixed_t) {
  // R[i][j][a][b] += L[i][j][a][b] = sum_{P,c,d} X[P][a][c] Y[P][b][d] T[i][j][c][d].
  // The caller guarantees that V_{ac,bd} = sum_P X[P][a][c] Y[P][b][d] is symmetric under
  // (a,c) <-> (b,d); with T[i][j][c][d] = T[j][i][d][c] that makes L[i][j][a][b] = L[j][i][b][a].
  // So for a block of a only the b >= (start of that block) part of V is built and contracted,
  // about half of both GEMMs, and the rest of R is read off the mirror.
  const int o = s_.o, v = s_.v;
  double* X = const_cast<double*>(Xv);
  double* Y = const_cast<double*>(Yv);
  double* Tm = const_cast<double*>(T);
  double* L = Y2_.val.p;
  const char* tb = prec == CC_FP64 ? "ladder_build.fp64"
                   : prec == CC_DF64 ? "ladder_build.df64"
                   : prec == CC_FP64_EMU ? "ladder_build.emu"
                   : prec == CC_MIXED_BF16X3 ? "ladder_build.bf16" : "ladder_build.tf32";
  const char* tc = prec == CC_FP64 ? "ladder_contract.fp64"
                   : prec == CC_DF64 ? "ladder_contract.df64"
                   : prec == CC_FP64_EMU ? "ladder_contract.emu"
                   : prec == CC_MIXED_BF16X3 ? "ladder_contract.bf16" : "ladder_contract.tf32";
  const bool tensor = prec == CC_MIXED_TF32 || prec == CC_MIXED_TF32X3 || prec == CC_MIXED_BF16X3;
  // tensor cores: the slab goes straight from the first GEMM's epilogue, as TF32 or BF16
  // segments in the K-major layout the second GEMM loads, to the second GEMM (no FP64 round
  // trip). A stage row is 128 bytes: k pads to 32 TF32 or 64 BF16 elements.
  const bool bf = prec == CC_MIXED_BF16X3;
  const int nseg = prec == CC_MIXED_TF32 ? 1 : 3;
  const long long align = bf ? 64 : 32;
  const long long kpad = ((long long)v * v + align - 1) / align * align, kk = nseg * kpad;
  const int rows_pad = (ladder_block_ * v + 255) / 256 * 256;
  // (c, d) split into the parts symmetric (+) and antisymmetric (-) under c <-> d. Since
  // T_ij^cd = T_ji^dc, T+ is symmetric and T- antisymmetric in (i, j), so
  // L = sum_{c<=d} W+ T+ + sum_{c<d} W- T- is contracted over pairs i <= j and c <= d only:
  // half the flops of the (c, d) contraction. Always in FP64 and double-float (from the FP64
  // slab); on the tensor cores when it pays (ladder_pack_pays) or is asked for, from a plain
  // FP32 slab that one pass turns into staged W+ and W-.
  const bool pack = tensor && (ex_.ladder_pack > 0 || (ex_.ladder_pack < 0 && ladder_pack_pays(o, v, prec)));
  const int Po = o * (o + 1) / 2, Qo = o * (o - 1) / 2, Pv = v * (v + 1) / 2, Qv = v * (v - 1) / 2;
  const long long kpP = ((long long)Pv + align - 1) / align * align, kpQ = ((long long)Qv + align - 1) / align * align;
  const size_t esz = bf ? 2 : 4;
  // Tensor cores without the split: when the slabs of all blocks of a fit side by side in the
  // staging budget, one grouped launch builds them all and one more contracts them all (the
  // contractions of a small problem fill the SMs together, not one by one)
  const int blk = ladder_block_;
  size_t group_rows = 0;
  for (int a0 = 0; a0 < v; a0 += blk) group_rows += ((size_t)std::min(blk, v - a0) * (v - a0) + 255) / 256 * 256;
  const bool grouped = tensor && !pack && group_rows * (size_t)kk * esz <= kLadderGroupBytes;
  if (tensor) {
    // the larger of the two paddings, and room for the two pair layouts (each padded)
    const long long kmax = ((long long)v * v + 63) / 64 * 64 + 128;
    size_t need = (size_t)rows_pad * 3 * kmax * 4;
    if (grouped) need = std::max(need, group_rows * (size_t)kk * esz);
    if (W2_.n * sizeof(double) < need) {
      W2_.alloc(ex_.pool, (need + 7) / 8);
      w2_mode_ = -1;
    }
    const int mode = (int)prec + (pack ? 16 : 0) + (grouped ? 32 : 0);
    if (w2_mode_ != mode) {  // the k padding of the plain layout must read as zeros
      CC_CUDA(cudaMemsetAsync(W2_.p, 0, W2_.n * sizeof(double), ex_.stream));
      w2_mode_ = mode;
    }
  }
  void* W2 = W2_.p;
  double* Tp = nullptr;
  double* Tmn = nullptr;
  // FP64 (native or emulated) and double-float: when the split slabs of all blocks fit side by
  // side in the same budget, every block's W+- goes into one array and the pair contractions
  // run once over all blocks' rows (two contractions per ladder instead of two per block)
  size_t all_rows = 0;
  for (int a0 = 0; a0 < v; a0 += blk) all_rows += (size_t)std::min(blk, v - a0) * (v - a0);
  const bool fused = !tensor && all_rows * (size_t)(Pv + Qv) * sizeof(double) <= kLadderGroupBytes;
  if (!tensor || pack) {
    const size_t nbmax = fused ? all_rows : (size_t)ladder_block_ * v;
    if (!pmT_.p) pmT_.alloc(ex_.pool, (size_t)Po * Pv + (size_t)Qo * Qv + 1);
    if (pmL_.n < (size_t)(Po + Qo) * nbmax + 1) pmL_.alloc(ex_.pool, (size_t)(Po + Qo) * nbmax + 1);
    if (!tensor && pmW_.n < nbmax * (size_t)(Pv + Qv) + 1) pmW_.alloc(ex_.pool, nbmax * (size_t)(Pv + Qv) + 1);
    Tp = pmT_.p;
    Tmn = Tp + (size_t)Po * Pv;
    k_ladder_pm_T(ex_, o, v, T, Tp, Tmn);
  }
  if (fused) {
    const size_t ld = all_rows;
    double* Wp = pmW_.p;
    double* Wm = Wp + ld * Pv;
    double* Lp = pmL_.p;
    double* Lm = Lp + (size_t)Po * ld;
    size_t r0 = 0;
    for (int a0 = 0; a0 < v; a0 += blk) {
      const int al = std::min(blk, v - a0), bl = v - a0;
      TView Xa = view_strided(X + (size_t)a0 * v, "Pac", {Paux, al, v}, {(long long)v * v, v, 1});
      TView Yb = view_strided(Y + (size_t)a0 * v, "Pbd", {Paux, bl, v}, {(long long)v * v, v, 1});
      contract(ex_, prec, 1.0, Xa, Yb, 0.0, view(W_.p, "abcd", {al, bl, v, v}), tb);
      k_ladder_pm_W(ex_, (size_t)al * bl, v, W_.p, Wp + r0 * Pv, Wm + r0 * Qv);
      r0 += (size_t)al * bl;
    }
    const int nall = (int)ld;
    contract(ex_, prec, 1.0, view(Tp, "xq", {Po, Pv}), view(Wp, "nq", {nall, Pv}), 0.0, view(Lp, "xn", {Po, nall}), tc);
    if (Qo > 0 && Qv > 0)
      contract(ex_, prec, 1.0, view(Tmn, "xq", {Qo, Qv}), view(Wm, "nq", {nall, Qv}), 0.0, view(Lm, "xn", {Qo, nall}),
               tc);
    else if (Qo > 0)
      k_fill(ex_, (size_t)Qo * ld, 0.0, Lm);
    r0 = 0;
    for (int a0 = 0; a0 < v; a0 += blk) {
      const int al = std::min(blk, v - a0), bl = v - a0;
      k_ladder_pm_unpack(ex_, o, v, a0, al, bl, Lp + r0, Lm + r0, L, ld);
      r0 += (size_t)al * bl;
    }
    k_ladder_mirror_add(ex_, o, v, blk, L, R);
    return;
  }
  if (grouped) {
    std::vector<StagedOut> sos;
    std::vector<StagedIn> sbs;
    sos.reserve((v + blk - 1) / blk);
    sbs.reserve((v + blk - 1) / blk);
    std::vector<ContractSpec> builds, cons;
    StageCache tcache;  // the amplitudes staged once for all blocks when they are not kept across calls
    tcache.cap = ~(size_t)0 >> 1;
    size_t row0 = 0;
    for (int a0 = 0; a0 < v; a0 += blk) {
      const int al = std::min(blk, v - a0), bl = v - a0;
      const int rp = (al * bl + 255) / 256 * 256;
      void* base = static_cast<char*>(W2) + row0 * (size_t)kk * esz;
      row0 += rp;
      sos.push_back(StagedOut{base, kpad, nseg, nseg == 3 ? 0b010 : 0});
      sbs.push_back(StagedIn{base, rp, (int)kk});
      ContractSpec b;
      b.A = view_strided(X + (size_t)a0 * v, "Pac", {Paux, al, v}, {(long long)v * v, v, 1});
      b.B = view_strided(Y + (size_t)a0 * v, "Pbd", {Paux, bl, v}, {(long long)v * v, v, 1});
      b.C = view_strided(nullptr, "abcd", {al, bl, v, v}, {(long long)bl * kk, kk, v, 1});
      b.cache = &stage_;
      b.cache_mask = fixed_xy ? 3 : 0;
      b.so = &sos.back();
      builds.push_back(b);
      ContractSpec c;
      c.A = view(Tm, "ijcd", {o, o, v, v});
      c.B = view(W_.p, "abcd", {al, bl, v, v});
      c.C = view_strided(L + (size_t)a0 * v + a0, "ijab", {o, o, al, bl}, {(long long)o * v * v, (long long)v * v, v, 1});
      c.cache = fixed_t ? &stage_ : &tcache;
      c.cache_mask = 1;
      c.sb = &sbs.back();
      cons.push_back(c);
    }
    contract_group(ex_, prec, builds, tb);
    contract_group(ex_, prec, cons, tc);
    k_ladder_mirror_add(ex_, o, v, blk, L, R);
    return;
  }
  for (int a0 = 0; a0 < v; a0 += blk) {
    const int al = std::min(blk, v - a0);
    const int bl = v - a0;  // b in [a0, v)
    TView Xa = view_strided(X + (size_t)a0 * v, "Pac", {Paux, al, v}, {(long long)v * v, v, 1});
    TView Yb = view_strided(Y + (size_t)a0 * v, "Pbd", {Paux, bl, v}, {(long long)v * v, v, 1});
    TView Lv = view_strided(L + (size_t)a0 * v + a0, "ijab", {o, o, al, bl},
                            {(long long)o * v * v, (long long)v * v, v, 1});
    TView W = view(W_.p, "abcd", {al, bl, v, v});
    if (!tensor) {
      contract(ex_, prec, 1.0, Xa, Yb, 0.0, W, tb);
      const int nb = al * bl;
      double* Wp = pmW_.p;
      double* Wm = Wp + (size_t)nb * Pv;
      k_ladder_pm_W(ex_, nb, v, W_.p, Wp, Wm);
      double* Lp = pmL_.p;
      double* Lm = Lp + (size_t)Po * nb;
      contract(ex_, prec, 1.0, view(Tp, "xq", {Po, Pv}), view(Wp, "nq", {nb, Pv}), 0.0, view(Lp, "xn", {Po, nb}), tc);
      if (Qo > 0 && Qv > 0)
        contract(ex_, prec, 1.0, view(Tmn, "xq", {Qo, Qv}), view(Wm, "nq", {nb, Qv}), 0.0, view(Lm, "xn", {Qo, nb}),
                 tc);
      else if (Qo > 0)
        k_fill(ex_, (size_t)Qo * nb, 0.0, Lm);
      k_ladder_pm_unpack(ex_, o, v, a0, al, bl, Lp, Lm, L);
      continue;
    }
    if (pack) {
      // the slab as FP32 words in W_ (row (a, b), column c v + d), split into staged W+ and W-
      // (rows padded to rows_pad) in W2, contracted with T+ and T- over pairs, unpacked into L
      float* Wf = reinterpret_cast<float*>(W_.p);
      StagedOut sf{Wf, 0, 0, 0};
      TView Wfv = view_strided(nullptr, "abcd", {al, bl, v, v}, {(long long)bl * v * v, (long long)v * v, v, 1});
      contract(ex_, prec, 1.0, Xa, Yb, 0.0, Wfv, tb, &sf, nullptr, &stage_, fixed_xy ? 3 : 0);
      const int nb = al * bl;
      void* Wp2 = W2;
      void* Wm2 = static_cast<char*>(W2) + (size_t)rows_pad * nseg * kpP * esz;
      k_ladder_pm_stage(ex_, bf, nseg, nb, v, Wf, Wp2, kpP, Qv > 0 ? Wm2 : nullptr, kpQ);
      double* Lp = pmL_.p;
      double* Lm = Lp + (size_t)Po * nb;
      StagedIn sbp{Wp2, rows_pad, (int)(nseg * kpP)};
      contract(ex_, prec, 1.0, view(Tp, "xq", {Po, Pv}), view(W_.p, "nq", {nb, Pv}), 0.0, view(Lp, "xn", {Po, nb}), tc,
               nullptr, &sbp);
      if (Qo > 0 && Qv > 0) {
        StagedIn sbm{Wm2, rows_pad, (int)(nseg * kpQ)};
        contract(ex_, prec, 1.0, view(Tmn, "xq", {Qo, Qv}), view(W_.p, "nq", {nb, Qv}), 0.0,
                 view(Lm, "xn", {Qo, nb}), tc, nullptr, &sbm);
      } else if (Qo > 0) {
        k_fill(ex_, (size_t)Qo * nb, 0.0, Lm);
      }
      k_ladder_pm_unpack(ex_, o, v, a0, al, bl, Lp, Lm, L);
      continue;
    }
    // W2[(a,b)][s * kpad + c v + d]: the strides below count floats of W2
    StagedOut so{W2, kpad, nseg, nseg == 3 ? 0b010 : 0};
    TView Ws = view_strided(nullptr, "abcd", {al, bl, v, v}, {(long long)bl * kk, kk, v, 1});
    contract(ex_, prec, 1.0, Xa, Yb, 0.0, Ws, tb, &so, nullptr, &stage_, fixed_xy ? 3 : 0);
    StagedIn sb{W2, rows_pad, (int)kk};
    contract(ex_, prec, 1.0, view(Tm, "ijcd", {o, o, v, v}), W, 0.0, Lv, tc, nullptr, &sb, &stage_, fixed_t ? 1 : 0);
  }
  k_ladder_mirror_add(ex_, o, v, blk, L, R);
}

void Engine::program(bool tan, cc_precision prec, double* rout) {
  const int o = s_.o, v = s_.v, n = s_.n, P = s_.P;
  const size_t ov = (size_t)o * v, oovv = (size_t)o * o * v * v;
  // Every launch of the program goes through run (kernels) or con (contractions): executed at
  // once, or, while rec_ is set, recorded for a lockstep run over several engines. A recorded
  // kernel closure holds the pointers it needs by value.
  auto run = [&](std::function<void(const Exec&)> f) {
    if (rec_) rec_->push_back(Op{Op::KERNEL, ContractSpec{}, std::move(f)});
    else f(ex_);
  };
  auto con = [&](double alpha, const TView& A, const TView& B, double beta, const TView& C, int mask) {
    StageCache* cache = mask ? &stage_ : nullptr;
    if (rec_) {
      Op op;
      op.kind = Op::CONTRACT;
      op.c.alpha = alpha;
      op.c.beta = beta;
      op.c.A = A;
      op.c.B = B;
      op.c.C = C;
      op.c.cache = cache;
      op.c.cache_mask = mask;
      rec_->push_back(std::move(op));
    } else {
      contract(ex_, prec, alpha, A, B, beta, C, nullptr, nullptr, nullptr, cache, mask);
    }
  };

  auto dyn = [&](Pair& x, size_t off, const char* lab, std::initializer_list<int> ext) {
    TP r;
    r.v = view(x.val.p + off, lab, ext);
    r.t = view(x.tan.p + off, lab, ext);
    r.dyn = true;
    return r;
  };
  auto dyns = [&](Pair& x, size_t off, const char* lab, std::initializer_list<int> ext,
                  std::initializer_list<long long> st) {
    TP r;
    r.v = view_strided(x.val.p + off, lab, ext, st);
    r.t = view_strided(x.tan.p + off, lab, ext, st);
    r.dyn = true;
    return r;
  };
  auto cst = [&](const double* p, const char* lab, std::initializer_list<int> ext) {
    TP r;
    r.v = view(const_cast<double*>(p), lab, ext);
    r.t = r.v;
    return r;
  };
  auto csts = [&](const double* p, const char* lab, std::initializer_list<int> ext,
                  std::initializer_list<long long> st) {
    TP r;
    r.v = view_strided(const_cast<double*>(p), lab, ext, st);
    r.t = r.v;
    return r;
  };
  // the output vector is the value in value mode and the tangent in tangent mode
  auto out = [&](size_t off, const char* lab, std::initializer_list<int> ext) {
    TP r;
    r.v = view(rout + off, lab, ext);
    r.t = r.v;
    r.dyn = true;
    return r;
  };
  // C = alpha A B + beta C, linearised in tangent mode. There the value-side factor is fixed
  // until the next value() call, so its tensor-core staging may be kept across JVPs.
  auto bil = [&](double alpha, const TP& A, const TP& B, double beta, const TP& C) {
    if (!tan) {
      con(alpha, A.v, B.v, beta, C.v, 0);
      return;
    }
    double b = beta;
    if (A.dyn) {
      con(alpha, A.t, B.v, b, C.t, 2);
      b = 1.0;
    }
    if (B.dyn) {
      con(alpha, A.v, B.t, b, C.t, 1);
      b = 1.0;
    }
  };
  auto cur = [&](Pair& x) { return tan ? x.tan.p : x.val.p; };

  TP T1 = dyn(t_, 0, "ia", {o, v});
  auto t1l = [&](const char* l) { return dyn(t_, 0, l, {o, v}); };
  auto t2l = [&](const char* l) { return dyn(t_, ov, l, {o, o, v, v}); };
  auto ul = [&](const char* l) { return dyn(u_, 0, l, {o, o, v, v}); };
  auto Boo = [&](const char* l) { return dyn(Btoo_, 0, l, {P, o, o}); };
  auto Bvv = [&](const char* l) { return dyn(Btvv_, 0, l, {P, v, v}); };
  auto Bvo = [&](const char* l) { return dyn(Btvo_, 0, l, {P, v, o}); };
  auto Bov = [&](const char* l) { return cst(s_.Bov.p, l, {P, o, v}); };
  auto Gl = [&](const char* l) { return cst(s_.Govov.p, l, {o, v, o, v}); };
  (void)T1;

  // amplitudes u = 2 t - t(i<->j)
  {
    double *tt = cur(t_) + ov, *uu = cur(u_);
    run([=](const Exec& e) { k_make_u(e, o, v, tt, uu); });
  }

  // ---- a1: T1 dressing of the DF factor -------------------------------------------------
  // Bt_oo = B_oo + B_ov t1^T
  if (!tan) {
    const double* src = s_.Boo.p;
    double* dst = Btoo_.val.p;
    run([=](const Exec& e) { k_copy(e, (size_t)P * o * o, src, dst); });
  }
  bil(1.0, Bov("Pic"), t1l("jc"), tan ? 0.0 : 1.0, Boo("Pij"));
  // Bt_vv = B_vv - t1^T B_ov
  if (!tan) {
    const double* src = s_.Bvv.p;
    double* dst = Btvv_.val.p;
    run([=](const Exec& e) { k_copy(e, (size_t)P * v * v, src, dst); });
  }
  bil(-1.0, t1l("ka"), Bov("Pkb"), tan ? 0.0 : 1.0, Bvv("Pab"));
  // Bt_vo = B_vo + B_vv t1^T - t1^T Bt_oo
  if (!tan) {
    const double* src = s_.Bov.p;
    double* dst = Btvo_.val.p;
    run([=](const Exec& e) { k_transpose(e, P, o, v, src, (long long)o * v, v, dst, (long long)v * o, o); });
  }
  bil(1.0, cst(s_.Bvv.p, "Pac", {P, v, v}), t1l("ic"), tan ? 0.0 : 1.0, Bvo("Pai"));
  bil(-1.0, t1l("ka"), Boo("Pki"), 1.0, Bvo("Pai"));
  {
    double *bo = cur(Btoo_), *gm = cur(gam_);
    run([=](const Exec& e) { k_trace_batched(e, P, o, bo, gm); });
  }

  // ---- dressed Fock matrix Ft = X h Y + 2 sum_P Bt gamma - sum_Pk Bt_pk Bt_kq -----------
  if (!tan) {
    const double* src = s_.h.p;
    double* dst = hY_.val.p;
    run([=](const Exec& e) { k_copy(e, (size_t)n * n, src, dst); });
  } else {
    double* dst = hY_.tan.p;
    run([=](const Exec& e) { k_fill(e, (size_t)n * n, 0.0, dst); });
  }
  bil(1.0, csts(s_.h.p + o, "pc", {n, v}, {n, 1}), t1l("jc"), 1.0, dyns(hY_, 0, "pj", {n, o}, {n, 1}));
  {
    double *src = cur(hY_), *dst = cur(Ft_);
    run([=](const Exec& e) { k_copy(e, (size_t)n * n, src, dst); });
  }
  bil(-1.0, t1l("ka"), dyns(hY_, 0, "kq", {o, n}, {n, 1}), 1.0, dyns(Ft_, (size_t)o * n, "aq", {v, n}, {n, 1}));
  TP Foo = dyns(Ft_, 0, "ij", {o, o}, {n, 1});
  TP Fov = dyns(Ft_, o, "kc", {o, v}, {n, 1});
  TP Fvo = dyns(Ft_, (size_t)o * n, "ai", {v, o}, {n, 1});
  TP Fvv = dyns(Ft_, (size_t)o * n + o, "ab", {v, v}, {n, 1});
  TP gam = dyn(gam_, 0, "P", {P});
  bil(2.0, Boo("Pij"), gam, 1.0, Foo);
  bil(2.0, Bov("Pkc"), gam, 1.0, Fov);
  bil(2.0, Bvo("Pai"), gam, 1.0, Fvo);
  bil(2.0, Bvv("Pab"), gam, 1.0, Fvv);
  bil(-1.0, Boo("Pik"), Boo("Pkj"), 1.0, Foo);
  bil(-1.0, Boo("Pkl"), Bov("Plc"), 1.0, Fov);
  bil(-1.0, Bvo("Pak"), Boo("Pki"), 1.0, Fvo);
  bil(-1.0, Bvo("Pak"), Bov("Pkb"), 1.0, Fvv);

  // ---- singles residual -----------------------------------------------------------------
  TP R1 = out(0, "ia", {o, v});
  {
    double* src = cur(Ft_) + (size_t)o * n;
    run([=](const Exec& e) { k_transpose(e, 1, v, o, src, 0, n, rout, 0, v); });  // Ft_vo^T
  }
  bil(1.0, Bov("Pkc"), ul("kicd"), 0.0, dyn(Z_, 0, "Pid", {P, o, v}));
  bil(1.0, dyn(Z_, 0, "Pid", {P, o, v}), Bvv("Pad"), 1.0, R1);
  bil(1.0, Bov("Plc"), ul("klac"), 0.0, dyn(Wk_, 0, "Pka", {P, o, v}));
  bil(-1.0, Boo("Pki"), dyn(Wk_, 0, "Pka", {P, o, v}), 1.0, R1);
  bil(1.0, ul("ikac"), dyns(Ft_, o, "kc", {o, v}, {n, 1}), 1.0, R1);

  // ---- doubles residual -----------------------------------------------------------------
  TP R2 = out(ov, "ijab", {o, o, v, v});
  double* r2 = rout + ov;
  // (ai|bj)~
  bil(1.0, Bvo("Pai"), Bvo("Pbj"), 0.0, R2);
  // particle-particle ladder sum_cd (ac|bd)~ t_ij^cd
  // (the ladder runs as one step of its own engine in a lockstep run; its GEMMs are large)
  if (!tan) {
    run([=](const Exec&) { ladder(Btvv_.val.p, Btvv_.val.p, P, t_.val.p + ov, r2, prec); });
  } else {
    // d[(ac|bd)~ t] = (ac|bd)~ dt + sum_P (dBt_ac Bt_bd + Bt_ac dBt_bd) t; the second factor
    // pair, stacked along the auxiliary index, is again symmetric under (a,c) <-> (b,d)
    run([=](const Exec& e) {
      ladder(Btvv_.val.p, Btvv_.val.p, P, t_.tan.p + ov, r2, prec, true, false);
      const size_t pvv = (size_t)P * v * v;
      double* Xs = XsYs_.p;
      double* Ys = XsYs_.p + 2 * pvv;
      k_copy(e, pvv, Btvv_.tan.p, Xs);
      k_copy(e, pvv, Btvv_.val.p, Xs + pvv);
      k_copy(e, pvv, Btvv_.val.p, Ys);
      k_copy(e, pvv, Btvv_.tan.p, Ys + pvv);
      ladder(Xs, Ys, 2 * P, t_.val.p + ov, r2, prec, false, true);
    });
  }
  // hole ladder with its quadratic part: W_klij = (ki|lj)~ + sum_cd (kc|ld) t_ij^cd
  TP Woo = dyn(Woo_, 0, "klij", {o, o, o, o});
  bil(1.0, Boo("Pki"), Boo("Plj"), 0.0, Woo);
  bil(1.0, Gl("kcld"), t2l("ijcd"), 1.0, Woo);
  bil(1.0, Woo, t2l("klab"), 1.0, R2);
  // C_kiac = (ki|ac)~ - 1/2 sum_ld t_li^ad (kd|lc), stored [k][c][i][a]
  auto Cl = [&](const char* l) { return dyn(Cint_, 0, l, {o, v, o, v}); };
  bil(1.0, Boo("Pki"), Bvv("Pac"), 0.0, Cl("kcia"));
  bil(-0.5, t2l("liad"), Gl("kdlc"), 1.0, Cl("kcia"));
  TP X = dyn(X_, 0, "ijab", {o, o, v, v});
  bil(-0.5, Cl("kcia"), t2l("kjbc"), 0.0, X);
  bil(-1.0, Cl("kcja"), t2l("kibc"), 1.0, X);
  // D_aikc = 2 (ai|kc)~ - (ac|ki)~ + 1/2 sum_ld u_il^ad L_ldkc, stored [k][c][i][a]
  auto Dl = [&](const char* l) { return dyn(Dint_, 0, l, {o, v, o, v}); };
  bil(2.0, Bvo("Pai"), Bov("Pkc"), 0.0, Dl("kcia"));
  bil(-1.0, Bvv("Pac"), Boo("Pki"), 1.0, Dl("kcia"));
  bil(0.5, ul("ilad"), cst(s_.Lovov.p, "ldkc", {o, v, o, v}), 1.0, Dl("kcia"));
  bil(0.5, Dl("kcia"), ul("jkbc"), 1.0, X);
  // Fock-like intermediates
  {
    double *src = cur(Ft_) + (size_t)o * n + o, *dst = cur(Gv_);
    run([=](const Exec& e) { k_copy3d(e, 1, v, v, src, 0, n, dst, 0, v); });
  }
  bil(-1.0, ul("klbd"), Gl("ldkc"), 1.0, dyn(Gv_, 0, "bc", {v, v}));
  {
    double *src = cur(Ft_), *dst = cur(Go_);
    run([=](const Exec& e) { k_copy3d(e, 1, o, o, src, 0, n, dst, 0, o); });
  }
  bil(1.0, ul("ljcd"), Gl("kdlc"), 1.0, dyn(Go_, 0, "kj", {o, o}));
  bil(1.0, t2l("ijac"), dyn(Gv_, 0, "bc", {v, v}), 1.0, X);
  bil(-1.0, t2l("ikab"), dyn(Go_, 0, "kj", {o, o}), 1.0, X);
  // Omega permutation: R_ij^ab += X_ij^ab + X_ji^ba
  {
    double* xx = cur(X_);
    run([=](const Exec& e) { k_sym_add(e, o, v, xx, r2, 1.0); });
  }
  (void)Fvo;
  (void)Fvv;
}

void Engine::value(const double* t, double* r, double* energy_dev, cc_precision prec) {
  const int o = s_.o, v = s_.v, n = s_.n;
  // the values change: staged copies of the old ones are stale (kept in place for the graphs)
  if (graphs_on_) stage_.mark_stale();
  else stage_.clear();
  first_since_value_ = true;
  if (t != t_.val.p) k_copy(ex_, s_.namp(), t, t_.val.p);
  program(false, prec, r);
  if (energy_dev)
    k_energy(ex_, o, v, s_.Govov.p, t_.val.p, t_.val.p + (size_t)o * v, s_.f.p + o, n, energy_dev, scratch_.p);
}

void Engine::record(OpList& list, bool tan, cc_precision prec, double* out) {
  rec_ = &list;
  try {
    program(tan, prec, out);
  } catch (...) {
    rec_ = nullptr;
    throw;
  }
  rec_ = nullptr;
}

void run_lockstep(const Exec& ex, cc_precision prec, std::vector<OpList>& lists) {
  bool aligned = true;
  for (const OpList& l : lists) {
    if (l.size() != lists[0].size()) aligned = false;
    for (size_t i = 0; aligned && i < l.size(); ++i)
      if (l[i].kind != lists[0][i].kind) aligned = false;
  }
  if (!aligned) {
    for (OpList& l : lists)
      for (Op& op : l) {
        if (op.kind == Op::KERNEL) op.fn(ex);
        else contract_group(ex, prec, {op.c});
      }
    return;
  }
  std::vector<ContractSpec> specs;
  for (size_t i = 0; i < lists[0].size(); ++i) {
    if (lists[0][i].kind == Op::KERNEL) {
      for (OpList& l : lists) l[i].fn(ex);
      continue;
    }
    specs.clear();
    for (OpList& l : lists) specs.push_back(l[i].c);
    contract_group(ex, prec, specs);
  }
}

void Engine::value_batch(const std::vector<Engine*>& engs, const std::vector<const double*>& t,
                         const std::vector<double*>& r, const std::vector<double*>& energy_dev, cc_precision prec) {
  if (engs.empty()) return;
  std::vector<OpList> lists(engs.size());
  for (size_t i = 0; i < engs.size(); ++i) {
    Engine& E = *engs[i];
    if (E.graphs_on_) E.stage_.mark_stale();
    else E.stage_.clear();
    E.first_since_value_ = true;
    if (t[i] != E.t_.val.p) k_copy(E.ex_, E.s_.namp(), t[i], E.t_.val.p);
    E.record(lists[i], false, prec, r[i]);
  }
  run_lockstep(engs[0]->ex_, prec, lists);
  for (size_t i = 0; i < engs.size(); ++i) {
    Engine& E = *engs[i];
    const int o = E.s_.o, v = E.s_.v;
    if (energy_dev[i])
      k_energy(E.ex_, o, v, E.s_.Govov.p, E.t_.val.p, E.t_.val.p + (size_t)o * v, E.s_.f.p + o, E.s_.n, energy_dev[i],
               E.scratch_.p);
  }
}

void Engine::tangent_batch(const std::vector<Engine*>& engs, const std::vector<const double*>& d,
                           const std::vector<double*>& jd, cc_precision prec) {
  if (engs.empty()) return;
  std::vector<OpList> lists(engs.size());
  for (size_t i = 0; i < engs.size(); ++i) {
    Engine& E = *engs[i];
    if (d[i] != E.t_.tan.p) k_copy(E.ex_, E.s_.namp(), d[i], E.t_.tan.p);
    E.first_since_value_ = false;
    E.record(lists[i], true, prec, jd[i]);
  }
  run_lockstep(engs[0]->ex_, prec, lists);
}

void Engine::tangent(const double* d, double* jd, cc_precision prec) {
  if (d != t_.tan.p) k_copy(ex_, s_.namp(), d, t_.tan.p);
  const bool graph = graphs_on_ && prec == graph_prec_ && !(ex_.prof && ex_.prof->on);
  TanGraph& G = graphs_[first_since_value_ ? 0 : 1];
  first_since_value_ = false;
  if (!graph) {
    program(true, prec, jd);
    return;
  }
  if (!G.exec) {
    if (G.eager < 1) {
      ++G.eager;
      program(true, prec, jd);
      return;
    }
    capture(G, prec);
  }
  CC_CUDA(cudaGraphLaunch(G.exec, ex_.stream));
  ex_.count(G.launches);
  k_copy(ex_, s_.namp(), jout_.p, jd);
}

void Engine::capture(TanGraph& G, cc_precision prec) {
  if (!cap_stream_) CC_CUDA(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
  const Exec saved = ex_;
  uint64_t nodes = 0, calls = 0;
  std::vector<void*> rec;
  ex_.stream = cap_stream_;  // captured on a private stream, launched on the context's
  ex_.launches = &nodes;
  ex_.calls = &calls;
  ex_.pool->record = &rec;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    try {
      program(true, prec, jout_.p);
    } catch (...) {
      cudaStreamEndCapture(cap_stream_, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      ex_ = saved;
      ex_.pool->record = nullptr;
      throw;
    }
    e = cudaStreamEndCapture(cap_stream_, &graph);
  }
  ex_ = saved;
  ex_.pool->record = nullptr;
  CC_CUDA(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CC_CUDA(e);
  std::sort(rec.begin(), rec.end());
  rec.erase(std::unique(rec.begin(), rec.end()), rec.end());
  for (void* p : rec) ex_.pool->pin(p);
  G.pinned = std::move(rec);
  G.exec = exec;
  G.launches = nodes;
}

void Engine::begin_graphs(cc_precision prec) {
  end_graphs();
  if (!jout_.p) jout_.alloc(ex_.pool, s_.namp());
  graphs_on_ = true;
  graph_prec_ = prec;
  first_since_value_ = true;
}

void Engine::end_graphs() noexcept {
  if (!graphs_on_) return;
  cudaStreamSynchronize(ex_.stream);  // no replay may still be running when its scratch is released
  for (auto& G : graphs_) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    for (void* p : G.pinned) ex_.pool->unpin(p);
    G = TanGraph{};
  }
  graphs_on_ = false;
  stage_.clear();
  cudaGetLastError();
}

Engine::~Engine() {
  end_graphs();
  if (cap_stream_) cudaStreamDestroy(cap_stream_);
}

// ---------------------------------------------------------------------------
// A_F (Eq. Preconditioner, App. C): the occupied and virtual Fock blocks on every index
// ---------------------------------------------------------------------------
void apply_AF(const Exec& ex, const System& s, const double* xin, double* y, cc_precision prec) {
  const int o = s.o, v = s.v, n = s.n;
  const size_t ov = (size_t)o * v;
  double* x = const_cast<double*>(xin);
  TView foo = view_strided(s.f.p, "ki", {o, o}, {n, 1});
  auto fvv = [&](const char* l) { return view_strided(s.f.p + (size_t)o * n + o, l, {v, v}, {n, 1}); };
  auto fo = [&](const char* l) { return view_strided(s.f.p, l, {o, o}, {n, 1}); };
  (void)foo;
  // singles: y_i^a = sum_c f_ac x_i^c - sum_k f_ki x_k^a
  contract(ex, prec, 1.0, view(x, "ic", {o, v}), fvv("ac"), 0.0, view(y, "ia", {o, v}));
  contract(ex, prec, -1.0, fo("ki"), view(x, "ka", {o, v}), 1.0, view(y, "ia", {o, v}));
  // doubles
  double* x2 = x + ov;
  double* y2 = y + ov;
  TView Y = view(y2, "ijab", {o, o, v, v});
  contract(ex, prec, 1.0, fvv("ac"), view(x2, "ijcb", {o, o, v, v}), 0.0, Y);
  contract(ex, prec, 1.0, view(x2, "ijac", {o, o, v, v}), fvv("bc"), 1.0, Y);
  contract(ex, prec, -1.0, fo("ki"), view(x2, "kjab", {o, o, v, v}), 1.0, Y);
  contract(ex, prec, -1.0, view(x2, "ikab", {o, o, v, v}), fo("kj"), 1.0, Y);
}

}  // namespace ccpnk
