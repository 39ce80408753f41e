// Tensor contractions as compound-index GEMMs.
//
// Every term of the CCSD residual, of its linearisation and of the A_F operator is a
// contraction of two tensors over shared labels. The planner below maps a contraction onto
// one GEMM whose row, column, sum and batch indices are each a compound of up to three
// strided modes (after merging modes that are contiguous in every operand), so permuted
// layouts are read in place with no transpose copies. Contractions with few output tiles and
// a long sum are split along k over extra blocks whose partial sums are added in a fixed
// order afterwards (deterministic results). The FP64 kernel runs on the FMA pipe (tcgen05.mma
// has no FP64 kind); tensor-core precisions go to gemm_tc.cu.
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
// 256 threads each holding a 4 x 4 accumulator block, two blocks per SM.
// ---------------------------------------------------------------------------
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ long long cidx(const CIdx& c, int x) {
  if (c.e1 == 1 && c.e2 == 1) return (long long)x * c.s0;
  int i2 = x % c.e2;
  int r = x / c.e2;
  int i1 = r % c.e1;
  int i0 = r / c.e1;
  return (long long)i0 * c.s0 + (long long)i1 * c.s1 + (long long)i2 * c.s2;
}

// TMR x TNR outputs per thread on a 16 x 16 thread grid: a (16 TMR) x (16 TNR) tile. FP64 on
// this part is so much slower than its loads and shared memory that even the smallest tile is
// bound by the FMA pipe, so the host picks the tile that wastes the least on padding and
// spreads the work most evenly over the SMs. Acc = float is the same kernel on the FP32 pipe
// (FP64 operands rounded to FP32 as they are staged, FP64 output and split-k partials): the
// thin contractions of the tensor-core precisions, whose tiles the tensor cores would mostly
// pad, with at most 512 terms summed in FP32 per split.
__device__ __forceinline__ double fma_acc(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_acc(float a, float b, float c) { return fmaf(a, b, c); }

template <int TMR, int TNR, typename Acc>
__device__ __forceinline__ void gemm_fma_body(const GemmArgs& g) {
  constexpr int TBM = 16 * TMR, TBN = 16 * TNR;
  __shared__ Acc As[BK][TBM + 1];
  __shared__ Acc Bs[BK][TBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int split = blockIdx.z % g.splits;
  const int kbeg = split * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);

  // per-thread load coordinates (fixed across k slices)
  // (TBM x BK = 256 TMR elements of A and 256 TNR of B per k slice)
  int a_mm[TMR], a_kk[TMR], b_nn[TNR], b_kk[TNR];
  long long a_moff[TMR], b_noff[TNR];
#pragma unroll
  for (int r = 0; r < TMR; ++r) {
    int e = tid + NT * r;
    if (g.a_kfast) { a_kk[r] = e % BK; a_mm[r] = e / BK; }
    else           { a_mm[r] = e % TBM; a_kk[r] = e / TBM; }
    int m = m0 + a_mm[r];
    a_moff[r] = m < g.M ? cidx(g.am, m) : -1;
  }
#pragma unroll
  for (int r = 0; r < TNR; ++r) {
    int e = tid + NT * r;
    if (g.b_kfast) { b_kk[r] = e % BK; b_nn[r] = e / BK; }
    else           { b_nn[r] = e % TBN; b_kk[r] = e / TBN; }
    int n = n0 + b_nn[r];
    b_noff[r] = n < g.N ? cidx(g.bn, n) : -1;
  }

  for (int bz = blockIdx.z / g.splits; bz < g.batch; bz += gridDim.z / g.splits) {
    const double* A = g.A + cidx(g.ab, bz);
    const double* B = g.B + cidx(g.bb, bz);
    Acc acc[TMR][TNR];
#pragma unroll
    for (int i = 0; i < TMR; ++i)
#pragma unroll
      for (int j = 0; j < TNR; ++j) acc[i][j] = Acc(0);

    // the next k slice is loaded into registers while the current one is multiplied, so the
    // loads' latency hides behind the FMAs
    Acc ra[TMR], rb[TNR];
    auto load_slice = [&](int k0) {
#pragma unroll
      for (int r = 0; r < TMR; ++r) {
        const int k = k0 + a_kk[r];
        ra[r] = (Acc)((a_moff[r] >= 0 && k < kend) ? A[a_moff[r] + cidx(g.ak, k)] : 0.0);
      }
#pragma unroll
      for (int r = 0; r < TNR; ++r) {
        const int kb = k0 + b_kk[r];
        rb[r] = (Acc)((b_noff[r] >= 0 && kb < kend) ? B[b_noff[r] + cidx(g.bk, kb)] : 0.0);
      }
    };
    if (kbeg < kend) load_slice(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
      for (int r = 0; r < TMR; ++r) As[a_kk[r]][a_mm[r]] = ra[r];
#pragma unroll
      for (int r = 0; r < TNR; ++r) Bs[b_kk[r]][b_nn[r]] = rb[r];
      __syncthreads();
      if (k0 + BK < kend) load_slice(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        Acc a[TMR], b[TNR];
#pragma unroll
        for (int i = 0; i < TMR; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < TNR; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < TMR; ++i)
#pragma unroll
          for (int j = 0; j < TNR; ++j) acc[i][j] = fma_acc(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
    if (g.splits > 1) {
      // partials [split][batch][M][N]
      double* P = g.part + ((size_t)split * g.batch + bz) * (size_t)g.M * g.N;
#pragma unroll
      for (int i = 0; i < TMR; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TNR; ++j) {
          int n = n0 + tx + 16 * j;
          if (n < g.N) P[(size_t)m * g.N + n] = (double)acc[i][j];
        }
      }
      continue;
    }
    double* C = g.C + cidx(g.cb, bz);
#pragma unroll
    for (int i = 0; i < TMR; ++i) {
      int m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
      long long cm = cidx(g.cm, m);
#pragma unroll
      for (int j = 0; j < TNR; ++j) {
        int n = n0 + tx + 16 * j;
        if (n >= g.N) continue;
        double* c = C + cm + cidx(g.cn, n);
        double val = g.alpha * (double)acc[i][j];
        if (g.beta != 0.0) val = fma(g.beta, *c, val);
        *c = val;
      }
    }
  }
}

template <int TMR, int TNR>
__global__ void __launch_bounds__(NT, 2) gemm_f64_kernel(GemmArgs g) {
  gemm_fma_body<TMR, TNR, double>(g);
}
template <int TMR, int TNR>
__global__ void __launch_bounds__(NT, 2) gemm_f32_kernel(GemmArgs g) {
  gemm_fma_body<TMR, TNR, float>(g);
}

// ---------------------------------------------------------------------------
// Double-float variant: the same tiles, with every FP64 operand split into an FP32 pair
// x = hi + lo (hi = fl(x), lo = fl(x - hi), about 48 significant bits) and every
// multiply-add done on the FP32 pipe, which a B300 runs about 60x faster than FP64:
//   product   a b = p + e exactly up to the dropped lo*lo term: p = fl(ah bh),
//             e = fma(ah, bh, -p) + ah bl + al bh   (Dekker's error-free product via FMA)
//   sum       (sh, sl) += (p, e) with Knuth's two-sum on the high parts, lows added
// The explicit __fadd_rn / __fmul_rn keep the compiler from fusing the two-sum steps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_mac(float2 a, float2 b, float& sh, float& sl) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = __fadd_rn(sh, p);
  const float bv = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = s;
}

__device__ __forceinline__ float2 df_split(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

__global__ void __launch_bounds__(NT, 2) gemm_df64_kernel(GemmArgs g) {
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int split = blockIdx.z % g.splits;
  const int kbeg = split * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  int a_mm[4], a_kk[4], b_nn[4], b_kk[4];
  long long a_moff[4], b_noff[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int e = tid + NT * r;
    if (g.a_kfast) { a_kk[r] = e % BK; a_mm[r] = e / BK; }
    else           { a_mm[r] = e % BM; a_kk[r] = e / BM; }
    if (g.b_kfast) { b_kk[r] = e % BK; b_nn[r] = e / BK; }
    else           { b_nn[r] = e % BN; b_kk[r] = e / BN; }
    int m = m0 + a_mm[r], n = n0 + b_nn[r];
    a_moff[r] = m < g.M ? cidx(g.am, m) : -1;
    b_noff[r] = n < g.N ? cidx(g.bn, n) : -1;
  }
  for (int bz = blockIdx.z / g.splits; bz < g.batch; bz += gridDim.z / g.splits) {
    const double* A = g.A + cidx(g.ab, bz);
    const double* B = g.B + cidx(g.bb, bz);
    float sh[4][4], sl[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.0f;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int k = k0 + a_kk[r];
        As[a_kk[r]][a_mm[r]] = df_split((a_moff[r] >= 0 && k < kend) ? A[a_moff[r] + cidx(g.ak, k)] : 0.0);
        int kb = k0 + b_kk[r];
        Bs[b_kk[r]][b_nn[r]] = df_split((b_noff[r] >= 0 && kb < kend) ? B[b_noff[r] + cidx(g.bk, kb)] : 0.0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) df_mac(a[i], b[j], sh[i][j], sl[i][j]);
      }
      __syncthreads();
    }
    if (g.splits > 1) {
      double* P = g.part + ((size_t)split * g.batch + bz) * (size_t)g.M * g.N;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int n = n0 + tx + 16 * j;
          if (n < g.N) P[(size_t)m * g.N + n] = (double)sh[i][j] + (double)sl[i][j];
        }
      }
      continue;
    }
    double* C = g.C + cidx(g.cb, bz);
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
        double val = g.alpha * ((double)sh[i][j] + (double)sl[i][j]);
        if (g.beta != 0.0) val = fma(g.beta, *c, val);
        *c = val;
      }
    }
  }
}

// Matrix-vector contractions (N == 1, or M == 1 with the operands' roles swapped): bound by
// reading the matrix once, so the GEMM tiles (15/16 of them idle on the unit dimension) are
// the wrong shape. One warp per output element: lanes walk k (32 loads in flight per output;
// coalesced when the matrix is contiguous along k), then a fixed shuffle tree, so the sum
// order is fixed and results are reproducible.
__global__ void gemv_f64_kernel(GemmArgs g, int trans) {
  const int rows = trans ? g.N : g.M;
  const long long nout = (long long)rows * g.batch;
  // the matrix operand (indexed by row and k) and the vector operand (by k)
  const double* Mx = trans ? g.B : g.A;
  const double* Vx = trans ? g.A : g.B;
  const CIdx& mr = trans ? g.bn : g.am;  // row index of the matrix
  const CIdx& mk = trans ? g.bk : g.ak;
  const CIdx& mb = trans ? g.bb : g.ab;
  const CIdx& vk = trans ? g.ak : g.bk;
  const CIdx& vb = trans ? g.ab : g.bb;
  const CIdx& cr = trans ? g.cn : g.cm;
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long e = w0; e < nout; e += nw) {
    const int b = (int)(e / rows), r = (int)(e - (long long)b * rows);
    const double* mrow = Mx + cidx(mb, b) + cidx(mr, r);
    const double* vrow = Vx + cidx(vb, b);  // the unit dimension's index is 0
    double s = 0.0;
    CWalk wm, wv;
    wm.init(mk, lane);
    wv.init(vk, lane);
#pragma unroll 4
    for (int k = lane; k < g.K; k += 32) {
      s = fma(mrow[wm.off], vrow[wv.off], s);
      wm.step(mk, 32);
      wv.step(vk, 32);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      double* c = g.C + cidx(g.cb, b) + cidx(cr, r);
      const double val = g.alpha * s;
      *c = g.beta == 0.0 ? val : fma(g.beta, *c, val);
    }
  }
}

// C = alpha * sum_s part[s] + beta * C, the splits added in order. One warp per piece of
// 256 elements of an output row: the row offset is located once and the column digits are
// carried, not divided out per element.
// the same with few outputs and many splits: 32 consecutive outputs per block of eight warps,
// warp w adding the splits w, w + 8, ... in order, warp 0 adding the eight sums in order
__global__ void __launch_bounds__(256) splitk_reduce_small_kernel(GemmArgs g) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t tot = (size_t)g.M * g.N * g.batch;
  for (size_t o0 = (size_t)blockIdx.x * 32; o0 < tot; o0 += (size_t)gridDim.x * 32) {
    const size_t o = o0 + lane;
    double s = 0.0;
    if (o < tot)
      for (int p = w; p < g.splits; p += 8) s += g.part[(size_t)p * tot + o];
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && o < tot) {
      double t = red[0][lane];
#pragma unroll
      for (int j = 1; j < 8; ++j) t += red[j][lane];
      const size_t q = o / g.N;  // output row b * M + m
      const int n = (int)(o - q * g.N);
      const int b = (int)(q / g.M), m = (int)(q - (size_t)b * g.M);
      double* c = g.C + cidx(g.cb, b) + cidx(g.cm, m) + cidx(g.cn, n);
      const double val = g.alpha * t;
      *c = g.beta == 0.0 ? val : fma(g.beta, *c, val);
    }
    __syncthreads();
  }
}

__global__ void splitk_reduce_kernel(GemmArgs g) {
  const int lane = threadIdx.x & 31;
  const size_t tot = (size_t)g.M * g.N * g.batch;
  const int pieces = (g.N + 255) / 256;
  const long long items = (long long)g.batch * g.M * pieces;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = w0; it < items; it += nw) {
    const long long q = it / pieces;  // output row b * M + m
    const int n0 = (int)(it - q * pieces) * 256, n1 = min(g.N, n0 + 256);
    const int b = (int)(q / g.M), m = (int)(q - (long long)b * g.M);
    const long long rowoff = cidx(g.cb, b) + cidx(g.cm, m);
    const double* pr = g.part + (size_t)q * g.N;
    CWalk cw;
    cw.init(g.cn, n0 + lane);
    for (int n = n0 + lane; n < n1; n += 32) {
      double s = 0.0;
#pragma unroll 8
      for (int p = 0; p < g.splits; ++p) s += pr[(size_t)p * tot + n];
      double* c = g.C + rowoff + cw.off;
      const double val = g.alpha * s;
      *c = g.beta == 0.0 ? val : fma(g.beta, *c, val);
      cw.step(g.cn, 32);
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

// compound index of up to three modes (outermost first)
CIdx make_cidx(const std::vector<Mode>& g, int which) {
  CIdx c;
  auto s = [&](const Mode& m) { return which == 0 ? m.sa : which == 1 ? m.sb : m.sc; };
  if (g.empty()) return c;
  if (g.size() == 1) {
    c.s0 = s(g[0]);
  } else if (g.size() == 2) {
    c.e1 = 1;
    c.e2 = g[1].ext;
    c.s0 = s(g[0]);
    c.s2 = s(g[1]);
  } else {
    c.e1 = g[1].ext;
    c.e2 = g[2].ext;
    c.s0 = s(g[0]);
    c.s1 = s(g[1]);
    c.s2 = s(g[2]);
  }
  return c;
}

long long group_size(const std::vector<Mode>& g) {
  long long n = 1;
  for (auto& m : g) n *= m.ext;
  return n;
}

long long inner_stride(const CIdx& c) { return (c.e1 == 1 && c.e2 == 1) ? c.s0 : c.s2; }

// A contraction too thin for 128 x 256 tensor-core tiles (a short k, or a narrow M or N) costs
// more in staging, padding and launch latency than it saves: true when the tensor-core run is
// estimated to be faster than the CUDA-core kernel (FP32 pipe for the single-precision kinds,
// FP64 pipe for the FP64 emulation; either is at least as accurate).
bool tc_faster(const Exec& ex, cc_precision prec, const GemmArgs& g) {
  const int nseg = prec == CC_MIXED_TF32 ? 1 : 3;
  const int tk = prec == CC_MIXED_BF16X3 || prec == CC_FP64_EMU ? 64 : 32;
  const double padded = 2.0 * ((g.M + 127) / 128 * 128.0) * ((g.N + 255) / 256 * 256.0) *
                        ((g.K + tk - 1) / tk * (double)tk) * nseg * g.batch;
  double t_tc = 12e-6 + padded / 4.5e14 + 8.0 * g.M * (double)g.N * g.batch / 1e12;
  if (prec == CC_FP64_EMU) {
    // the slice products on kind::f16, the exact partial sums (one per chunk of up to 4096 k,
    // written and read once in FP32; none when they are summed on chip, so this is an upper
    // bound), the digit staging of both operands
    const double kp = (g.K + 63) / 64 * 64.0, chunks = kOzProducts * kp / 4096.0 + kOzSlices;
    t_tc = 20e-6 + kOzProducts * padded / 1.2e15 + chunks * 8.0 * g.M * (double)g.N * g.batch / 5e12 +
           ((double)g.M + g.N) * kp * g.batch * (8.0 + 2.0 * kOzSlices) / 5e12;
  }
  // the CUDA-core kernel's parallelism: 16 x 16 tiles, k split at most 1024 ways
  const double blocks = (double)((g.M + 15) / 16) * ((g.N + 15) / 16) * g.batch * std::min(1024, std::max(1, g.K / 32));
  const double flops16 = 2.0 * ((g.M + 15) / 16 * 16.0) * ((g.N + 15) / 16 * 16.0) * g.K * g.batch;
  // FP64 pipe, or the FP32 kernel as measured on these shapes (its staging loads and compound
  // indices, not the FP32 pipe's 75 TFLOP/s, set its pace)
  const double cuda_rate = prec == CC_FP64_EMU ? 1.0e12 : 5.0e12;
  double t_f64 = 4e-6 + flops16 / (cuda_rate * std::min(1.0, blocks / ex.sm_count));
  if ((g.N == 1 || g.M == 1) && (long long)(g.N == 1 ? g.M : g.N) * g.batch >= 256)
    t_f64 = 4e-6 + 8.0 * (g.N == 1 ? g.M : g.N) * (double)g.K * g.batch / 2e12;  // the FP64 GEMV reads the matrix once
  return t_tc <= t_f64;
}

void launch_gemm(const Exec& ex, cc_precision prec, GemmArgs g, const char* tag) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  CC_REQUIRE(!((g.so || g.sb) && (prec == CC_FP64 || prec == CC_DF64)), CC_ERR_INVALID, "staged operands need a tensor-core precision");
  // thin contractions of the single-precision tensor-core kinds run on the FP32 pipe (more
  // accurate than their tensor-core passes); those of the FP64 emulation on the FP64 pipe
  bool f32 = false;
  if (prec != CC_FP64 && prec != CC_DF64) {
    if (g.so || g.sb || tc_faster(ex, prec, g)) {
      gemm_tc(ex, prec, g, tag);
      return;
    }
    f32 = prec != CC_FP64_EMU;
    prec = CC_FP64;
  }
  // (a few outputs over a long k stay on the split-k GEMM path, which spreads k over SMs)
  if (prec == CC_FP64 && (g.N == 1 || g.M == 1) && g.K > 0 &&
      (long long)(g.N == 1 ? g.M : g.N) * g.batch >= 256) {
    const int trans = g.N == 1 ? 0 : 1;
    const long long nout = (long long)(trans ? g.N : g.M) * g.batch;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((nout * 32 + 255) / 256, (long long)ex.sm_count * 16));
    cudaEvent_t ev = nullptr;
    if (ex.timing(tag)) ex.mark_begin(&ev);
    gemv_f64_kernel<<<blocks, 256, 0, ex.stream>>>(g, trans);
    ex.count();
    CC_CUDA(cudaGetLastError());
    if (ev) ex.mark_end(tag, ev, 2.0 * g.M * (double)g.N * g.K * g.batch);
    return;
  }
  // The kernel's lanes run along the columns of C; when C is contiguous along its rows instead
  // (and strided along its columns), the transposed product C^T = B A^T writes the same memory
  // with coalesced stores. Each output is the same k-ordered sum either way.
  if (inner_stride(g.cn) != 1 && inner_stride(g.cm) == 1) {
    std::swap(g.M, g.N);
    std::swap(g.A, g.B);
    std::swap(g.am, g.bn);
    std::swap(g.ak, g.bk);
    std::swap(g.ab, g.bb);
    std::swap(g.cm, g.cn);
    g.a_kfast = g.K <= 0 || inner_stride(g.ak) == 1;
    g.b_kfast = g.K <= 0 || (inner_stride(g.bk) == 1 && inner_stride(g.bn) != 1);
  }
  const int ksteps = (g.K + BK - 1) / BK;
  // FP64: tile (16 TMR) x (16 TNR) and split-K factor from a model of the FMA-bound kernel:
  // blocks are spread evenly over the SMs, so the time is ceil(blocks / SMs) blocks' FMA
  // work (padding included) plus a small per-block cost, plus the split-K reduce (partial
  // sums written and read, and a launch). Ties go to the larger tile and the fewer splits.
  // The double-float kernel keeps its 64 x 64 tile and the occupancy-based split.
  int tmr = 4, tnr = 4, splits = 1;
  if (prec == CC_FP64) {
    // FP64 FMAs per second of one SM; the FP32 kernel runs about 4x that (measured), bound by
    // its staging loads rather than by the FP32 pipe
    const double fma_rate = 2.0 * 2.0e9 * (f32 ? 4.0 : 1.0);
    const double blk_cost = 2e-6, hbm = 6.0e12;
    double best = 1e300;
    // in FP32 at most 32 k steps of 16 (512 terms) per split
    const int smin = f32 ? (ksteps + 31) / 32 : 1;
    const int smax = std::max(smin, std::min(1024, ksteps / 2));
    for (int r : {4, 2, 1})
      for (int c : {4, 2, 1}) {
        const long long bm = 16 * r, bn = 16 * c;
        const long long tiles = ((g.M + bm - 1) / bm) * ((g.N + bn - 1) / bn) * g.batch;
        if ((g.M + bm - 1) / bm > 65535) continue;
        for (int sp = smin; sp <= smax; ++sp) {
          if (sp > smin && tiles * sp > 16LL * ex.sm_count * 8) break;  // enough blocks already
          const long long kst = (ksteps + sp - 1) / sp;
          const double per_sm = (double)((tiles * sp + ex.sm_count - 1) / ex.sm_count);
          double t = per_sm * ((double)bm * bn * BK * kst / fma_rate + blk_cost);
          if (sp > 1) t += 16.0 * sp * (double)g.M * g.N * g.batch / hbm + 5e-6;
          if (t < best * (1.0 - 1e-6)) {
            best = t;
            tmr = r;
            tnr = c;
            splits = sp;
          }
        }
      }
  } else {
    const long long tiles = (long long)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * g.batch;
    const long long target = 4LL * ex.sm_count;  // two resident blocks per SM, two waves
    if (tiles < target && ksteps >= 8) splits = (int)std::max<long long>(1, std::min<long long>((target + tiles - 1) / tiles, ksteps / 4));
  }
  const long long tm = (g.M + 16 * tmr - 1) / (16 * tmr), tn = (g.N + 16 * tnr - 1) / (16 * tnr);
  CC_REQUIRE(tm <= 65535, CC_ERR_INVALID, "gemm: M too large for the grid");
  DBuf<double> part;
  g.splits = splits;
  g.kchunk = ((ksteps + splits - 1) / splits) * BK;
  if (splits > 1) {
    part.alloc(ex.pool, (size_t)splits * g.batch * g.M * g.N);
    g.part = part.p;
  }
  long long zb = std::min<long long>(g.batch, std::max<long long>(1, 65535 / splits));
  dim3 grid((unsigned)tn, (unsigned)tm, (unsigned)(zb * splits));
  cudaEvent_t ev = nullptr;
  if (ex.timing(tag)) ex.mark_begin(&ev);
  if (prec == CC_DF64) {
    gemm_df64_kernel<<<grid, NT, 0, ex.stream>>>(g);
  } else if (f32) {
    auto k = gemm_f32_kernel<4, 4>;
    if (tmr == 4) k = tnr == 4 ? gemm_f32_kernel<4, 4> : tnr == 2 ? gemm_f32_kernel<4, 2> : gemm_f32_kernel<4, 1>;
    else if (tmr == 2) k = tnr == 4 ? gemm_f32_kernel<2, 4> : tnr == 2 ? gemm_f32_kernel<2, 2> : gemm_f32_kernel<2, 1>;
    else k = tnr == 4 ? gemm_f32_kernel<1, 4> : tnr == 2 ? gemm_f32_kernel<1, 2> : gemm_f32_kernel<1, 1>;
    k<<<grid, NT, 0, ex.stream>>>(g);
  } else {
    auto k = gemm_f64_kernel<4, 4>;
    if (tmr == 4) k = tnr == 4 ? gemm_f64_kernel<4, 4> : tnr == 2 ? gemm_f64_kernel<4, 2> : gemm_f64_kernel<4, 1>;
    else if (tmr == 2) k = tnr == 4 ? gemm_f64_kernel<2, 4> : tnr == 2 ? gemm_f64_kernel<2, 2> : gemm_f64_kernel<2, 1>;
    else k = tnr == 4 ? gemm_f64_kernel<1, 4> : tnr == 2 ? gemm_f64_kernel<1, 2> : gemm_f64_kernel<1, 1>;
    k<<<grid, NT, 0, ex.stream>>>(g);
  }
  ex.count();
  CC_CUDA(cudaGetLastError());
  if (splits > 1) {
    const size_t items = (size_t)g.batch * g.M * ((g.N + 255) / 256);
    int blocks = (int)std::max<size_t>(1, std::min<size_t>((items + 7) / 8, (size_t)ex.sm_count * 16));
    const size_t outs = (size_t)g.batch * g.M * g.N;
    if (outs < 65536 && splits >= 16) {  // few outputs, many splits: spread the splits
      const int sblocks = (int)std::max<size_t>(1, std::min<size_t>((outs + 31) / 32, (size_t)ex.sm_count * 16));
      splitk_reduce_small_kernel<<<sblocks, 256, 0, ex.stream>>>(g);
    } else {
      splitk_reduce_kernel<<<blocks, 256, 0, ex.stream>>>(g);
    }
    ex.count();
    CC_CUDA(cudaGetLastError());
  }
  if (ev) ex.mark_end(tag, ev, 2.0 * g.M * (double)g.N * g.K * g.batch);
  // part returns to the pool here; later launches on the same stream are ordered after the reduce
}

}  // namespace

static bool same_cidx(const CIdx& a, const CIdx& b) {
  return a.e1 == b.e1 && a.e2 == b.e2 && a.s0 == b.s0 && a.s1 == b.s1 && a.s2 == b.s2;
}

bool operator==(const StageKey& a, const StageKey& b) {
  return a.src == b.src && same_cidx(a.rix, b.rix) && same_cidx(a.kix, b.kix) && same_cidx(a.bix, b.bix) &&
         a.rows == b.rows && a.K == b.K && a.batch == b.batch && a.rows_pad == b.rows_pad && a.k_pad == b.k_pad &&
         a.nseg == b.nseg && a.seg_lo == b.seg_lo && a.bf == b.bf;
}

namespace {

// The GEMMs of C = alpha contract(A, B) + beta C: one, or several when modes beyond three
// spill to a host loop (run in order: later slices of a spilled sum accumulate into C), or
// none when the output is empty.
std::vector<GemmArgs> plan_contract(double alpha, const TView& A, const TView& B, double beta, const TView& C,
                                    const StagedOut* so, const StagedIn* sb, StageCache* cache, int cache_mask) {
  std::vector<GemmArgs> out;
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
    if (ia < 0 && ib < 0) fail(CC_ERR_INVALID, std::string("contract: output label only in C: ") + l);
    if (C.ext[d] == 1) continue;
    if (ia >= 0 && ib >= 0) gb.push_back(m);
    else if (ia >= 0) gm.push_back(m);
    else gn.push_back(m);
  }
  for (int d = 0; d < A.nd; ++d) {
    char l = A.lab[d];
    if (find(C, l) >= 0) continue;
    int ib = find(B, l);
    CC_REQUIRE(ib >= 0, CC_ERR_INVALID, std::string("contract: label summed in A only: ") + l);
    CC_REQUIRE(B.ext[ib] == A.ext[d], CC_ERR_INVALID, std::string("contract: extent of ") + l);
    if (A.ext[d] == 1) continue;
    gk.push_back(Mode{l, A.ext[d], A.st[d], B.st[ib], 0});
  }
  for (int d = 0; d < B.nd; ++d) {
    char l = B.lab[d];
    CC_REQUIRE(find(C, l) >= 0 || find(A, l) >= 0, CC_ERR_INVALID,
               std::string("contract: label summed in B only: ") + l);
  }
  for (auto* g : {&gb, &gm, &gn})
    for (auto& m : *g)
      if (m.ext == 0) return out;  // empty output
  bool empty_sum = false;
  for (auto& m : gk)
    if (m.ext == 0) empty_sum = true;
  if (empty_sum) gk.clear();  // C = beta C (K = 0 below)

  merge_modes(gb, true, true, true);
  merge_modes(gm, true, false, true);
  merge_modes(gn, false, true, true);
  merge_modes(gk, true, true, false);
  // row or column modes beyond three become batch modes (offsets in their operands only)
  while (gm.size() > 3) { gb.insert(gb.begin(), gm.front()); gm.erase(gm.begin()); }
  while (gn.size() > 3) { gb.insert(gb.begin(), gn.front()); gn.erase(gn.begin()); }
  // modes beyond three per group go to a host loop (outermost first)
  std::vector<Mode> loops;
  auto spill = [&](std::vector<Mode>& g) {
    while (g.size() > 3) {
      loops.push_back(g.front());
      g.erase(g.begin());
    }
  };
  spill(gb);
  spill(gk);

  GemmArgs g{};
  g.M = (int)group_size(gm);
  g.N = (int)group_size(gn);
  g.K = empty_sum ? 0 : (int)group_size(gk);
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
  g.splits = 1;
  g.so = so;
  g.sb = sb;
  g.cache = cache;
  g.cache_mask = cache ? cache_mask : 0;
  g.a_kfast = gk.empty() ? 1 : (inner_stride(g.ak) == 1);
  g.b_kfast = gk.empty() ? 1 : (inner_stride(g.bk) == 1 && inner_stride(g.bn) != 1);

  const int nl = (int)loops.size();
  CC_REQUIRE(nl == 0 || (!so && !sb), CC_ERR_INVALID, "staged operands need a contraction without spilled modes");
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
    out.push_back(gi);
    int q = nl - 1;
    while (q >= 0) {
      if (++idx[q] < loops[q].ext) break;
      idx[q] = 0;
      --q;
    }
    if (q < 0) break;
  }
  return out;
}

}  // namespace

void contract(const Exec& ex, cc_precision prec, double alpha, const TView& A, const TView& B,
              double beta, const TView& C, const char* tag, const StagedOut* so, const StagedIn* sb,
              StageCache* cache, int cache_mask) {
  std::string auto_tag;  // with the timer on, an untagged contraction is named by its labels
  if (!tag && ex.prof && ex.prof->on && ex.prof->all) {
    auto_tag = std::string(A.lab) + "*" + B.lab + ">" + C.lab +
               (prec == CC_FP64 ? ".f64" : prec == CC_DF64 ? ".df64" : ".tc");
    tag = auto_tag.c_str();
  }
  for (const GemmArgs& g : plan_contract(alpha, A, B, beta, C, so, sb, cache, cache_mask)) launch_gemm(ex, prec, g, tag);
}

void contract_group(const Exec& ex, cc_precision prec, const std::vector<ContractSpec>& specs, const char* tag) {
  const bool tc = prec == CC_MIXED_TF32 || prec == CC_MIXED_TF32X3 || prec == CC_MIXED_BF16X3;
  std::vector<GemmArgs> grouped;
  for (const ContractSpec& c : specs) {
    CC_REQUIRE(tc || (!c.so && !c.sb), CC_ERR_INVALID, "staged operands need a tensor-core precision");
    std::vector<GemmArgs> gs = plan_contract(c.alpha, c.A, c.B, c.beta, c.C, c.so, c.sb, c.cache, c.cache_mask);
    if (tc && gs.size() == 1 && gs[0].M > 0 && gs[0].N > 0 && gs[0].batch > 0 && gs[0].K > 0 &&
        (c.so || c.sb || tc_faster(ex, prec, gs[0]))) {
      grouped.push_back(gs[0]);
    } else {
      for (const GemmArgs& g : gs) launch_gemm(ex, prec, g, tag);
    }
  }
  if (!grouped.empty()) gemm_tc_group(ex, prec, grouped, tag);
}

}  // namespace ccpnk
