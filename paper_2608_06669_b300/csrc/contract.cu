// Tensor contractions as compound-index GEMMs.
//
// Every term of the CCSD residual, of its linearisation and of the A_F operator is a
// contraction of two tensors over shared labels. The planner below maps a contraction onto
// one GEMM whose row, column, sum and batch indices are each a compound of at most two
// strided modes (after merging modes that are contiguous in every operand), so permuted
// layouts are read in place with no transpose copies. Groups with more modes are split into
// a host loop. The FP64 kernel runs on the FMA pipe (there is no FP64 tensor-core kind of
// tcgen05.mma); tensor-core precisions gather their operands into K-major FP32 staging
// buffers and run the tcgen05 kernel (gemm_tc.cu).
#include <algorithm>
#include <cstring>

#include "common.h"

namespace ccpnk {

TView view(double* p, const char* labels, std::initializer_list<int> ext) {
  TView t;
  t.p = p;
  t.nd = (int)strlen(labels);
  CC_REQUIRE(t.nd == (int)ext.size() && t.nd <= kMaxModes, CC_ERR_INVALID, "view: label/extent mismatch");
  int i = 0;
  for (int e : ext) t.ext[i++] = e;
  long long s = 1;
  for (int d = t.nd - 1; d >= 0; --d) {
    t.st[d] = s;
    s *= t.ext[d];
  }
  memcpy(t.lab, labels, t.nd);
  t.lab[t.nd] = 0;
  return t;
}

TView view_strided(double* p, const char* labels, std::initializer_list<int> ext,
                   std::initializer_list<long long> strides) {
  TView t = view(p, labels, ext);
  CC_REQUIRE((int)strides.size() == t.nd, CC_ERR_INVALID, "view_strided: stride count");
  int i = 0;
  for (long long s : strides) t.st[i++] = s;
  return t;
}

// ---------------------------------------------------------------------------
// FP64 kernel: 64 x 64 output tile, 16-deep k slices staged in shared memory,
// 256 threads each holding a 4 x 4 accumulator block.
// ---------------------------------------------------------------------------
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ long long cidx(const CIdx& c, int x) {
  if (c.inner == 1) return (long long)x * c.s1;
  int q = x / c.inner;
  int r = x - q * c.inner;
  return (long long)q * c.s1 + (long long)r * c.s2;
}

__global__ void __launch_bounds__(NT) gemm_f64_kernel(GemmArgs g) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  // per-thread load coordinates (fixed across k slices)
  int a_mm[4], a_kk[4], b_nn[4], b_kk[4];
  long long a_moff[4], b_noff[4];
  bool a_mok[4], b_nok[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int e = tid + NT * r;
    if (g.a_kfast) { a_kk[r] = e % BK; a_mm[r] = e / BK; }
    else           { a_mm[r] = e % BM; a_kk[r] = e / BM; }
    if (g.b_kfast) { b_kk[r] = e % BK; b_nn[r] = e / BK; }
    else           { b_nn[r] = e % BN; b_kk[r] = e / BN; }
    int m = m0 + a_mm[r], n = n0 + b_nn[r];
    a_mok[r] = m < g.M;
    b_nok[r] = n < g.N;
    a_moff[r] = a_mok[r] ? cidx(g.am, m) : 0;
    b_noff[r] = b_nok[r] ? cidx(g.bn, n) : 0;
  }

  for (int bz = blockIdx.z; bz < g.batch; bz += gridDim.z) {
    const double* A = g.A + cidx(g.ab, bz);
    const double* B = g.B + cidx(g.bb, bz);
    double* C = g.C + cidx(g.cb, bz);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int k = k0 + a_kk[r];
        As[a_kk[r]][a_mm[r]] = (a_mok[r] && k < g.K) ? A[a_moff[r] + cidx(g.ak, k)] : 0.0;
        int kb = k0 + b_kk[r];
        Bs[b_kk[r]][b_nn[r]] = (b_nok[r] && kb < g.K) ? B[b_noff[r] + cidx(g.bk, kb)] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
      long long cm = cidx(g.cm, m);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int n = n0 + tx + 16 * j;
        if (n >= g.N) continue;
        double* c = C + cm + cidx(g.cn, n);
        double val = g.alpha * acc[i][j];
        if (g.beta != 0.0) val = fma(g.beta, *c, val);
        *c = val;
      }
    }
  }
}

struct Mode {
  char l;
  int ext;
  long long sa, sb, sc;  // strides in A, B, C (0 if absent)
};

// Merges adjacent modes of a group that are contiguous in every operand that carries them.
void merge_modes(std::vector<Mode>& g, bool inA, bool inB, bool inC) {
  bool changed = true;
  while (changed && g.size() > 1) {
    changed = false;
    for (size_t i = 0; i + 1 < g.size(); ++i) {
      Mode& o = g[i];
      Mode& in = g[i + 1];
      bool ok = true;
      if (inA && o.sa != in.sa * in.ext) ok = false;
      if (inB && o.sb != in.sb * in.ext) ok = false;
      if (inC && o.sc != in.sc * in.ext) ok = false;
      if (ok) {
        Mode mrg{o.l, o.ext * in.ext, in.sa, in.sb, in.sc};
        g[i] = mrg;
        g.erase(g.begin() + i + 1);
        changed = true;
        break;
      }
    }
  }
}

CIdx make_cidx(const std::vector<Mode>& g, int which) {
  CIdx c{1, 0, 0};
  auto s = [&](const Mode& m) { return which == 0 ? m.sa : which == 1 ? m.sb : m.sc; };
  if (g.empty()) return c;
  if (g.size() == 1) {
    c.inner = 1;
    c.s1 = s(g[0]);
    return c;
  }
  c.inner = g[1].ext;
  c.s1 = s(g[0]);
  c.s2 = s(g[1]);
  return c;
}

long long group_size(const std::vector<Mode>& g) {
  long long n = 1;
  for (auto& m : g) n *= m.ext;
  return n;
}

void launch_gemm(const Exec& ex, cc_precision prec, const GemmArgs& g) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  if (prec == CC_FP64) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, std::min(g.batch, 65535));
    CC_REQUIRE(grid.y <= 65535, CC_ERR_INVALID, "gemm: M too large for the grid");
    gemm_f64_kernel<<<grid, NT, 0, ex.stream>>>(g);
    ex.count();
    CC_CUDA(cudaGetLastError());
  } else {
    gemm_tc(ex, prec, g);
  }
}

}  // namespace

void contract(const Exec& ex, cc_precision prec, double alpha, const TView& A, const TView& B,
              double beta, const TView& C) {
  auto find = [](const TView& t, char l) {
    for (int d = 0; d < t.nd; ++d)
      if (t.lab[d] == l) return d;
    return -1;
  };
  std::vector<Mode> gb, gm, gn, gk;
  for (int d = 0; d < C.nd; ++d) {
    char l = C.lab[d];
    int ia = find(A, l), ib = find(B, l);
    Mode m{l, C.ext[d], ia >= 0 ? A.st[ia] : 0, ib >= 0 ? B.st[ib] : 0, C.st[d]};
    if (ia >= 0) CC_REQUIRE(A.ext[ia] == C.ext[d], CC_ERR_INVALID, std::string("contract: extent of ") + l);
    if (ib >= 0) CC_REQUIRE(B.ext[ib] == C.ext[d], CC_ERR_INVALID, std::string("contract: extent of ") + l);
    if (ia >= 0 && ib >= 0) gb.push_back(m);
    else if (ia >= 0) gm.push_back(m);
    else if (ib >= 0) gn.push_back(m);
    else fail(CC_ERR_INVALID, std::string("contract: output label only in C: ") + l);
  }
  for (int d = 0; d < A.nd; ++d) {
    char l = A.lab[d];
    if (find(C, l) >= 0) continue;
    int ib = find(B, l);
    CC_REQUIRE(ib >= 0, CC_ERR_INVALID, std::string("contract: label summed in A only: ") + l);
    CC_REQUIRE(B.ext[ib] == A.ext[d], CC_ERR_INVALID, std::string("contract: extent of ") + l);
    gk.push_back(Mode{l, A.ext[d], A.st[d], B.st[ib], 0});
  }
  for (int d = 0; d < B.nd; ++d) {
    char l = B.lab[d];
    CC_REQUIRE(find(C, l) >= 0 || find(A, l) >= 0, CC_ERR_INVALID,
               std::string("contract: label summed in B only: ") + l);
  }
  merge_modes(gb, true, true, true);
  merge_modes(gm, true, false, true);
  merge_modes(gn, false, true, true);
  merge_modes(gk, true, true, false);

  // modes beyond two per group go to a host loop (outermost first)
  std::vector<Mode> loops;
  auto spill = [&](std::vector<Mode>& g) {
    while (g.size() > 2) {
      loops.push_back(g.front());
      g.erase(g.begin());
    }
  };
  spill(gb);
  spill(gm);
  spill(gn);
  spill(gk);
  for (auto* g : {&gm, &gn, &gk, &gb})
    for (auto& m : *g) if (m.ext == 0) return;  // empty contraction output or sum
  for (auto& m : loops)
    if (m.ext == 0) return;

  GemmArgs g{};
  g.M = (int)group_size(gm);
  g.N = (int)group_size(gn);
  g.K = (int)group_size(gk);
  g.batch = (int)group_size(gb);
  g.am = make_cidx(gm, 0);
  g.ak = make_cidx(gk, 0);
  g.ab = make_cidx(gb, 0);
  g.bk = make_cidx(gk, 1);
  g.bn = make_cidx(gn, 1);
  g.bb = make_cidx(gb, 1);
  g.cm = make_cidx(gm, 2);
  g.cn = make_cidx(gn, 2);
  g.cb = make_cidx(gb, 2);
  g.alpha = alpha;
  g.beta = beta;
  auto inner_stride = [](const CIdx& c) { return c.inner == 1 ? c.s1 : c.s2; };
  g.a_kfast = gk.empty() ? 1 : (inner_stride(g.ak) == 1);
  g.b_kfast = gk.empty() ? 1 : (inner_stride(g.bk) == 1 && inner_stride(g.bn) != 1);

  // host loop over spilled modes
  const int nl = (int)loops.size();
  std::vector<int> idx(nl, 0);
  while (true) {
    GemmArgs gi = g;
    long long oa = 0, ob = 0, oc = 0;
    bool first_k = true;  // a spilled sum mode accumulates: later slices add to C
    for (int q = 0; q < nl; ++q) {
      oa += idx[q] * loops[q].sa;
      ob += idx[q] * loops[q].sb;
      oc += idx[q] * loops[q].sc;
      if (loops[q].sc == 0 && idx[q] != 0) first_k = false;
    }
    gi.A = A.p + oa;
    gi.B = B.p + ob;
    gi.C = C.p + oc;
    if (!first_k) gi.beta = 1.0;
    launch_gemm(ex, prec, gi);
    int q = nl - 1;
    while (q >= 0) {
      if (++idx[q] < loops[q].ext) break;
      idx[q] = 0;
      --q;
    }
    if (q < 0) break;
  }
}

}  // namespace ccpnk
