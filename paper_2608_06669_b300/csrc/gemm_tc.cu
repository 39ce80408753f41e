// Tensor-core contractions on sm_103a: tcgen05.mma (kind::tf32, FP32 accumulation in TMEM),
// operands brought into 128-byte-swizzled shared memory by TMA through a multi-stage mbarrier
// pipeline, one elected thread issuing the MMAs, and an epilogue that reads the accumulator
// with tcgen05.ld and applies C = alpha * acc + beta * C in FP64.
//
// The compound-index operands of a contraction are first gathered into K-major FP32 staging
// buffers (rounded to TF32 to nearest, padded to whole tiles with zeros), so the tensor-core
// kernel sees plain [batch][rows][k] arrays that TMA can tile. Every wait on an mbarrier is
// bounded by the global timer; a timeout sets the context's error flag and the kernel leaves
// after releasing its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>

#include "common.h"

namespace ccpnk {
namespace {

constexpr int TM = 128;         // tile rows = UMMA M
constexpr int TN = 256;         // tile columns = UMMA N
// Operand element types: TF32 (kind::tf32, 32 per 128-byte row, 8 per MMA) and BF16
// (kind::f16 with BF16 operands, 64 per row, 16 per MMA). A pipeline stage is 128 bytes of
// k for every row in both cases, so the shared-memory layout does not depend on the type.
template <bool BF>
struct Elt;
template <>
struct Elt<false> {
  using T = float;
  static constexpr int TK = 32, UK = 8;
  static constexpr uint32_t FMT = 2;  // TF32 in the instruction descriptor
};
template <>
struct Elt<true> {
  using T = __nv_bfloat16;
  static constexpr int TK = 64, UK = 16;
  static constexpr uint32_t FMT = 1;  // BF16
};
constexpr int STAGES = 4;
constexpr int EPI_WARPS = 8;    // two per TMEM lane quadrant, each on half of the tile's columns
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // TMA producer, MMA issuer, epilogue warps
constexpr uint32_t A_BYTES = TM * 128;
constexpr uint32_t B_BYTES = TN * 128;
constexpr uint32_t TMEM_COLS = 2 * TN;  // two FP32 accumulators of TN columns (all 512)

__device__ __forceinline__ long long cidx(const CIdx& c, int x) {
  if (c.e1 == 1 && c.e2 == 1) return (long long)x * c.s0;
  int i2 = x % c.e2;
  int r = x / c.e2;
  int i1 = r % c.e1;
  int i0 = r / c.e1;
  return (long long)i0 * c.s0 + (long long)i1 * c.s1 + (long long)i2 * c.s2;
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// writes x into the staging segments of one element: the TF32 high part, or the low part.
// All in FP32: x - tf32(x) is exact in FP32, and nothing here touches the FP64 pipe.
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = to_tf32(x);
  lo = to_tf32(__fsub_rn(x, hi));
}
__device__ __forceinline__ void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(__fsub_rn(x, __bfloat162float(hi)));
}
// the epilogue's fixed-layout versions: one segment (hi), or three as [hi|lo|hi]
template <int NSEG, typename T>
__device__ __forceinline__ void store_staged_fixed(T* p, long long kpad, float x) {
  T hi, lo;
  split(x, hi, lo);
  p[0] = hi;
  if constexpr (NSEG == 3) {
    p[kpad] = lo;
    p[2 * kpad] = hi;
  }
}
template <typename T>
__device__ __forceinline__ void store_staged(T* p, long long kpad, int nseg, int seglo, float x) {
  T hi, lo;
  split(x, hi, lo);
  for (int s = 0; s < nseg; ++s) p[(long long)s * kpad] = ((seglo >> s) & 1) ? lo : hi;
}


// The warp-per-row kernels below cut a row into pieces of ROW_PIECE elements, so that short
// and long rows alike give enough warps to fill the GPU.
constexpr int ROW_PIECE = 256;

// out[b][r][s * k_pad + k] for r < rows_pad, k < k_pad and the nseg segments s of a row
// (TF32 words or BF16, zero outside rows x K). seg_lo is a bit mask of the segments that hold
// the low part lo = x - hi instead of the high part hi; one segment with mask 0 is the plain
// operand, three segments [hi|hi|lo] and [hi|lo|hi] on the two operands give the three-pass
// split product hi hi + hi lo + lo hi along one long k. One warp per piece of a staged row:
// the row's source offset is located once, and the lanes walk k.
// An operand whose rows are contiguous in the source and whose k is strided (tr = 1) is staged
// by 32 x 32 tiles instead: a warp reads the tile down its rows, one k per step (coalesced),
// and writes it along k through shared memory.
// Several operands staged by one launch: their descriptors and the prefix sums of their work
// items (batch x rows_pad x row pieces each, or batch x row tiles x k tiles) are a grid-constant
// parameter, and every warp walks the combined item list, finding its operand by the prefix sums.
struct GatherDesc {
  const double* src;
  void* out;
  CIdx rix, kix, bix;
  int rows, K, batch, rows_pad, k_pad, nseg, seg_lo, tr;
};
constexpr int GATHER_MAX = 24;
constexpr int GATHER_THREADS = 256;
struct GatherList {
  GatherDesc d[GATHER_MAX];
  long long item0[GATHER_MAX + 1];
  int n;
};

template <typename T>
__global__ void __launch_bounds__(GATHER_THREADS) gather_kernel(const __grid_constant__ GatherList L) {
  __shared__ float tiles[GATHER_THREADS / 32][32 * 33];
  const int lane = threadIdx.x & 31;
  float* tile = tiles[threadIdx.x >> 5];
  const long long total = L.item0[L.n];
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  int gi = 0;
  for (long long it = w0; it < total; it += nw) {
    while (it >= L.item0[gi + 1]) ++gi;  // a warp's items only grow
    const GatherDesc& d = L.d[gi];
    if (d.tr) {
      const int rtiles = (d.rows_pad + 31) >> 5, ktiles = (d.k_pad + 31) >> 5;
      const long long li = it - L.item0[gi];
      const long long q = li / ktiles;  // row tile b * rtiles + rt
      const int k0 = (int)(li - q * ktiles) << 5;
      const int b = (int)(q / rtiles), r0 = (int)(q - (long long)b * rtiles) << 5;
      const bool rv = r0 + lane < d.rows;
      const double* src = d.src + cidx(d.bix, b) + (rv ? cidx(d.rix, r0 + lane) : 0);
      CWalk kw;
      kw.init(d.kix, k0 + lane);
      const long long koff = kw.off;  // lane j holds the offset of k0 + j
      const int kn = min(32, d.K - k0);
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const long long o = __shfl_sync(0xffffffffu, koff, j);
        tile[lane * 33 + j] = (rv && j < kn) ? (float)src[o] : 0.0f;
      }
      __syncwarp();
      const int k = k0 + lane;
      const int rn = min(32, d.rows_pad - r0);
      const size_t row_len = (size_t)d.nseg * d.k_pad;
      if (k < d.k_pad) {
        for (int j = 0; j < rn; ++j) {
          T hi, lo;
          split(tile[j * 33 + lane], hi, lo);
          T* row = static_cast<T*>(d.out) + ((size_t)b * d.rows_pad + r0 + j) * row_len;
          for (int s = 0; s < d.nseg; ++s) row[(size_t)s * d.k_pad + k] = ((d.seg_lo >> s) & 1) ? lo : hi;
        }
      }
      __syncwarp();
      continue;
    }
    const int pieces = (d.k_pad + ROW_PIECE - 1) / ROW_PIECE;
    const size_t row_len = (size_t)d.nseg * d.k_pad;
    const long long li = it - L.item0[gi];
    const long long q = li / pieces;  // staged row b * rows_pad + r
    const int k0 = (int)(li - q * pieces) * ROW_PIECE, k1 = min(d.k_pad, k0 + ROW_PIECE);
    const int b = (int)(q / d.rows_pad), r = (int)(q - (long long)b * d.rows_pad);
    T* row = static_cast<T*>(d.out) + (size_t)q * row_len;
    if (r >= d.rows) {
      T z, zl;
      split(0.0f, z, zl);
      for (int k = k0 + lane; k < k1; k += 32)
        for (int s = 0; s < d.nseg; ++s) row[(size_t)s * d.k_pad + k] = z;
      continue;
    }
    const double* srow = d.src + cidx(d.bix, b) + cidx(d.rix, r);
    CWalk kw;
    kw.init(d.kix, k0 + lane);
    for (int k = k0 + lane; k < k1; k += 32) {
      T hi, lo;
      split(k < d.K ? (float)srow[kw.off] : 0.0f, hi, lo);
      for (int s = 0; s < d.nseg; ++s) row[(size_t)s * d.k_pad + k] = ((d.seg_lo >> s) & 1) ? lo : hi;
      kw.step(d.kix, 32);
    }
  }
}

// split-k: C = alpha * sum_s part[s] + beta * C, the splits added in a fixed order (or, with
// a staged output, alpha * sum written as TF32 or BF16 segments). One warp per piece of an
// output row.
template <typename T>
__global__ void tc_splitk_reduce_kernel(GemmArgs g, const float* __restrict__ part, int splits, T* Cs,
                                        long long kpad, int nseg, int seglo, int piece) {
  const int lane = threadIdx.x & 31;
  const size_t tot = (size_t)g.batch * g.M * g.N;
  const int pieces = (g.N + piece - 1) / piece;
  const long long items = (long long)g.batch * g.M * pieces;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = w0; it < items; it += nw) {
    const long long q = it / pieces;  // output row b * M + m
    const int n0 = (int)(it - q * pieces) * piece, n1 = min(g.N, n0 + piece);
    const int b = (int)(q / g.M), m = (int)(q - (long long)b * g.M);
    const long long rowoff = cidx(g.cb, b) + cidx(g.cm, m);
    const float* pr = part + (size_t)q * g.N;
    CWalk cw;
    cw.init(g.cn, n0 + lane);
    for (int n = n0 + lane; n < n1; n += 32) {
      double s = 0.0;
#pragma unroll 8
      for (int p = 0; p < splits; ++p) s += (double)pr[(size_t)p * tot + n];
      const long long off = rowoff + cw.off;
      if (Cs && nseg == 0) {  // plain FP32 words
        reinterpret_cast<float*>(Cs)[off] = (float)(g.alpha * s);
      } else if (Cs) {
        store_staged(Cs + off, kpad, nseg, seglo, (float)(g.alpha * s));
      } else {
        double* c = g.C + off;
        *c = g.beta == 0.0 ? g.alpha * s : fma(g.beta, *c, g.alpha * s);
      }
      cw.step(g.cn, 32);
    }
  }
}

// The (c, d) split of the tensor-core ladder's slab. W holds rows r of v x v FP32 values
// (column c v + d) as the build GEMM wrote them; W+[r][pair_le(c, d)] = W_r^cd + W_r^dc (W_r^cc
// on the diagonal) and W-[r][pair_lt(c, d)] = W_r^cd - W_r^dc are written in staging layout:
// nseg segments of kpP (kpQ) elements per row ([hi|lo|hi] for three), zero past the last pair.
// One 256-thread block per (row, 32 x 32 block pair with c-block <= d-block) at a time: the
// blocks W^(c0.., d0..) and W^(d0.., c0..) are both read along rows into shared memory, so the
// loads and the stores (consecutive d for one c) are coalesced.
template <typename T>
__global__ void __launch_bounds__(256) ladder_pm_stage_kernel(long long rows, int v, const float* __restrict__ W,
                                                              T* __restrict__ Wp, long long kpP, T* __restrict__ Wm,
                                                              long long kpQ, int nseg) {
  __shared__ float xs[32][33], ys[32][33];
  const int nt = (v + 31) / 32, npairs = nt * (nt + 1) / 2;
  const long long Pv = (long long)v * (v + 1) / 2, Qv = (long long)v * (v - 1) / 2;
  const int seglo = nseg == 3 ? 0b010 : 0;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long vv = (long long)v * v, items = rows * npairs;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const long long r = it / npairs;
    const int q0 = (int)(it - r * npairs);
    int q = q0, cb = 0;
    while (q >= nt - cb) {  // q -> (cb <= db), row-major over the block pairs
      q -= nt - cb;
      ++cb;
    }
    const int c0 = cb * 32, d0 = (cb + q) * 32;
    const float* Wr = W + r * vv;
    __syncthreads();  // the previous item's reads of xs and ys are done
    for (int i = ty; i < 32; i += 8) {
      const int c = c0 + i, d = d0 + tx;
      xs[i][tx] = (c < v && d < v) ? Wr[(long long)c * v + d] : 0.f;  // W^(c0 + i, d0 + tx)
      const int d1 = d0 + i, c1 = c0 + tx;
      ys[i][tx] = (d1 < v && c1 < v) ? Wr[(long long)d1 * v + c1] : 0.f;  // W^(d0 + i, c0 + tx)
    }
    __syncthreads();
    T* wp = Wp + r * nseg * kpP;
    T* wm = Wm ? Wm + r * nseg * kpQ : nullptr;
    for (int i = ty; i < 32; i += 8) {
      const int c = c0 + i, d = d0 + tx;
      if (c >= v || d >= v || d < c) continue;
      const float x = xs[i][tx], y = ys[tx][i];  // W^cd and W^dc
      store_staged(wp + pair_le(c, d, v), kpP, nseg, seglo, c < d ? __fadd_rn(x, y) : x);
      if (wm && c < d) store_staged(wm + pair_lt(c, d, v), kpQ, nseg, seglo, __fsub_rn(x, y));
    }
    if (q0 == 0) {  // the row's k padding (fewer than 64 elements per segment)
      T zero, zlo;
      split(0.f, zero, zlo);
      const int padP = (int)(kpP - Pv), padQ = (int)(kpQ - Qv);
      for (int e = threadIdx.x; e < nseg * padP; e += blockDim.x) wp[(e / padP) * kpP + Pv + e % padP] = zero;
      if (wm)
        for (int e = threadIdx.x; e < nseg * padQ; e += blockDim.x) wm[(e / padQ) * kpQ + Qv + e % padQ] = zero;
    }
  }
}

// split-k for few outputs and many splits: a block of eight warps takes 32 consecutive outputs
// (lanes along the outputs, so the reads coalesce), warp w adds the splits w, w + 8, ... in
// order, and warp 0 adds the eight warp sums in order: a fixed summation order for a given
// split count, with the splits instead of the outputs spread over the warps.
template <typename T>
__global__ void __launch_bounds__(256) tc_splitk_reduce_small_kernel(GemmArgs g, const float* __restrict__ part,
                                                                     int splits, T* Cs, long long kpad, int nseg,
                                                                     int seglo) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t tot = (size_t)g.batch * g.M * g.N;
  for (size_t o0 = (size_t)blockIdx.x * 32; o0 < tot; o0 += (size_t)gridDim.x * 32) {
    const size_t o = o0 + lane;
    double s = 0.0;
    if (o < tot)
      for (int p = w; p < splits; p += 8) s += (double)part[(size_t)p * tot + o];
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && o < tot) {
      double t = red[0][lane];
#pragma unroll
      for (int j = 1; j < 8; ++j) t += red[j][lane];
      const size_t q = o / g.N;  // output row b * M + m
      const int n = (int)(o - q * g.N);
      const int b = (int)(q / g.M), m = (int)(q - (size_t)b * g.M);
      const long long off = cidx(g.cb, b) + cidx(g.cm, m) + cidx(g.cn, n);
      if (Cs && nseg == 0) {
        reinterpret_cast<float*>(Cs)[off] = (float)(g.alpha * t);
      } else if (Cs) {
        store_staged(Cs + off, kpad, nseg, seglo, (float)(g.alpha * t));
      } else {
        double* c = g.C + off;
        *c = g.beta == 0.0 ? g.alpha * t : fma(g.beta, *c, g.alpha * t);
      }
    }
    __syncthreads();
  }
}

__global__ void scale_c_kernel(GemmArgs g) {  // K == 0: C = beta C
  const size_t tot = (size_t)g.batch * g.M * g.N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    int n = (int)(e % g.N);
    size_t r = e / g.N;
    int m = (int)(r % g.M);
    int b = (int)(r / g.M);
    double* c = g.C + cidx(g.cb, b) + cidx(g.cm, m) + cidx(g.cn, n);
    *c = g.beta == 0.0 ? 0.0 : g.beta * *c;
  }
}

// ---------------------------------------------------------------------------
// FP64-accurate products on the tensor cores: Ozaki's error-free splitting (Ozaki, Ogita,
// Oishi and Rump, Numer. Algorithms 59 (2012) 95; on tensor cores: Mukunoki, Ozaki, Ogita and
// Imamura, ICCS 2020). Every row x of an operand (a row of A, a column of B) is written as
//   x_k = sign(x_k) sum_{s=1..S} d_s(x_k) 2^(sigma - OZ_BETA s) + (error <= 2^(sigma - OZ_BETA S - 1)),
// with sigma the row's exponent (|x_k| < 2^sigma): |x_k| is rounded to the nearest multiple of
// 2^(sigma - OZ_BETA S), so the representation error has no sign bias and sums of many products
// grow like their square root, not like their count. The digits are integers 0 <= d_s < 2^OZ_BETA
// (d_1 <= 2^OZ_BETA when the rounding carries into it), which BF16 holds exactly. A product of
// two digit slices is then a sum of integers: each MMA chunk of at most nk k blocks sums at most
// nk * 64 products of at most 2^(2 OZ_BETA), an integer of at most 2^24 up to nk = 64, which the
// FP32 accumulator represents exactly. The slice products of one level L = s + t share the
// scale 2^(sigma_i + tau_j - OZ_BETA L); levels up to S + 1 are kept (the first term dropped is
// below 2^(-OZ_BETA S) of the leading one) and added exactly in two 64-bit integer fixed-point
// sums (oz_fixed_value), so the only rounding is the final conversion to FP64.
// ---------------------------------------------------------------------------
constexpr int OZ_S = kOzSlices;  // slices per operand: 54 significant bits
constexpr int OZ_BETA = 6;   // bits per slice digit
constexpr int OZ_NK = 64;    // default k blocks (of 64) per exact FP32 chunk: 64 * 64 * 64^2 = 2^24

// |x| of an FP64 bit pattern in units of 2^(sigma - OZ_BETA S), rounded to nearest (ties away
// from zero), for a row whose largest biased exponent is em (sigma = em - 1022): the digits of
// the result are the slices. Integer shifts only; at most 2^(OZ_BETA S).
__device__ __forceinline__ unsigned long long oz_quantize(unsigned long long bits, unsigned em) {
  unsigned e = (unsigned)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & ((1ull << 52) - 1);
  if (e) m |= 1ull << 52;
  else e = 1;
  // |x| = m 2^(e - 1075) = m 2^-sh units, sh = em - e + 53 - beta S (at least 53 - beta S = -1:
  // then the shift is exact)
  const int sh = (int)em - (int)e + 53 - OZ_BETA * OZ_S;
  if (sh <= 0) return m << (-sh);
  return sh >= 64 ? 0ull : ((m + (1ull << (sh - 1))) >> sh);
}
// slice sl (1 = leading) of a quantised magnitude; the leading digit keeps a rounding carry
__device__ __forceinline__ int oz_digit(unsigned long long qv, int sl) {
  const unsigned long long d = qv >> (OZ_BETA * (OZ_S - sl));
  return sl == 1 ? (int)d : (int)(d & ((1u << OZ_BETA) - 1));
}

// Pass 1 of the digit staging: the largest biased exponent of every staged row (a row of A or
// a column of B), one warp per piece of ROW_PIECE elements of a row, combined by an integer
// atomicMax (order-independent). emax must start at 0; a row of zeros keeps 0.
__global__ void oz_rowexp_kernel(const double* __restrict__ src, CIdx rix, CIdx kix, CIdx bix, int rows, int K,
                                 int batch, int rows_pad, unsigned* __restrict__ emax) {
  const int lane = threadIdx.x & 31;
  const int pieces = (K + ROW_PIECE - 1) / ROW_PIECE;
  const long long items = (long long)batch * rows * pieces;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = w0; it < items; it += nw) {
    const long long q = it / pieces;  // real row b * rows + r
    const int k0 = (int)(it - q * pieces) * ROW_PIECE, k1 = min(K, k0 + ROW_PIECE);
    const int b = (int)(q / rows), r = (int)(q - (long long)b * rows);
    const double* srow = src + cidx(bix, b) + cidx(rix, r);
    unsigned e = 0;
    CWalk kw;
    kw.init(kix, k0 + lane);
    for (int k = k0 + lane; k < k1; k += 32) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(srow[kw.off]);
      e = max(e, (unsigned)((bits >> 52) & 0x7FF));
      kw.step(kix, 32);
    }
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0 && e) atomicMax(emax + (size_t)b * rows_pad + r, e);
  }
}

// Pass 2: the S digit slices of every element as BF16 in the K-major staging layout
// out[b][r][seg * k_pad + k] (segment s - 1 holds slice s for A; B holds slice t in segment
// S - t), zeros outside rows x K; one warp per piece of a staged row. With the row's exponent
// sigma = max(emax, 1) - 1022 (every |x| of the row is below 2^sigma), the digits come from the
// FP64 bit pattern by integer shifts (no FP64 arithmetic).
__global__ void oz_digits_kernel(const double* __restrict__ src, CIdx rix, CIdx kix, CIdx bix, int rows, int K,
                                 int batch, int rows_pad, int k_pad, int rev, const unsigned* __restrict__ emax,
                                 __nv_bfloat16* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int pieces = (k_pad + ROW_PIECE - 1) / ROW_PIECE;
  const long long items = (long long)batch * rows_pad * pieces;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const size_t row_len = (size_t)OZ_S * k_pad;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (long long it = w0; it < items; it += nw) {
    const long long q = it / pieces;  // staged row b * rows_pad + r
    const int k0 = (int)(it - q * pieces) * ROW_PIECE, k1 = min(k_pad, k0 + ROW_PIECE);
    const int b = (int)(q / rows_pad), r = (int)(q - (long long)b * rows_pad);
    __nv_bfloat16* row = out + (size_t)q * row_len;
    if (r >= rows) {
      for (int k = k0 + lane; k < k1; k += 32)
#pragma unroll
        for (int sl = 0; sl < OZ_S; ++sl) row[(size_t)sl * k_pad + k] = zero;
      continue;
    }
    const unsigned em = max(emax[q], 1u);
    const double* srow = src + cidx(bix, b) + cidx(rix, r);
    CWalk kw;
    kw.init(kix, k0 + lane);
    for (int k = k0 + lane; k < k1; k += 32) {
      unsigned long long qv = 0, neg = 0;
      if (k < K) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(srow[kw.off]);
        neg = bits >> 63;
        qv = oz_quantize(bits, em);
      }
#pragma unroll
      for (int sl = 1; sl <= OZ_S; ++sl) {
        const int d = oz_digit(qv, sl);
        const float f = neg ? -(float)d : (float)d;
        const int seg = rev ? OZ_S - sl : sl - 1;
        row[(size_t)seg * k_pad + k] = __float2bfloat16_rn(f);
      }
      kw.step(kix, 32);
    }
  }
}

// Both passes in one kernel for rows of at most a few thousand elements: one warp per staged
// row finds the row's exponent (warp maximum, no atomics) and then writes its digits (the second
// read of the row comes from L1/L2). Writes emax like the two-pass version.
// The two operands of a product staged by one launch: their descriptors, and the warps' rows
// numbered across both (rows of A first).
struct OzStageDesc {
  const double* src;
  CIdx rix, kix, bix;
  int rows, batch, rows_pad, rev;
  unsigned* emax;
  __nv_bfloat16* out;
};
struct OzStagePair {
  OzStageDesc d[2];
  long long row0[3];
  int K, k_pad;
};

__global__ void oz_stage_rows_kernel(const __grid_constant__ OzStagePair P) {
  const int lane = threadIdx.x & 31;
  const long long items = P.row0[2];
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int K = P.K, k_pad = P.k_pad;
  const size_t row_len = (size_t)OZ_S * k_pad;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (long long it = w0; it < items; it += nw) {
    const int which = it >= P.row0[1] ? 1 : 0;
    const OzStageDesc& D = P.d[which];
    const double* src = D.src;
    const CIdx& rix = D.rix;
    const CIdx& kix = D.kix;
    const CIdx& bix = D.bix;
    const int rows = D.rows, rows_pad = D.rows_pad, rev = D.rev;
    unsigned* emax = D.emax;
    __nv_bfloat16* out = D.out;
    const long long q = it - P.row0[which];  // staged row b * rows_pad + r of this operand
    const int b = (int)(q / rows_pad), r = (int)(q - (long long)b * rows_pad);
    __nv_bfloat16* row = out + (size_t)q * row_len;
    if (r >= rows) {
      for (size_t k = lane; k < row_len; k += 32) row[k] = zero;
      if (lane == 0) emax[q] = 0;
      continue;
    }
    const double* srow = src + cidx(bix, b) + cidx(rix, r);
    unsigned e = 0;
    CWalk kw;
    kw.init(kix, lane);
    for (int k = lane; k < K; k += 32) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(srow[kw.off]);
      e = max(e, (unsigned)((bits >> 52) & 0x7FF));
      kw.step(kix, 32);
    }
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) emax[q] = e;
    const unsigned em = max(e, 1u);
    kw.init(kix, lane);
    for (int k = lane; k < k_pad; k += 32) {
      unsigned long long qv = 0, neg = 0;
      if (k < K) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(srow[kw.off]);
        neg = bits >> 63;
        qv = oz_quantize(bits, em);
      }
#pragma unroll
      for (int sl = 1; sl <= OZ_S; ++sl) {
        const int d = oz_digit(qv, sl);
        const float f = neg ? -(float)d : (float)d;
        const int seg = rev ? OZ_S - sl : sl - 1;
        row[(size_t)seg * k_pad + k] = __float2bfloat16_rn(f);
      }
      kw.step(kix, 32);
    }
  }
}

// 2^e as a double from its exponent bits (callers keep e inside the normal range)
__device__ __forceinline__ double pow2(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// The levels' exact sums in fixed point without any rounding: levels 2..OZ_LH go into acc_h in
// units of level OZ_LH, the rest into acc_l in units of level S + 1, each level's sum shifted by
// OZ_BETA bits per level below its group's unit. With products of at most 2^12 and level L
// holding (L - 1) k_pad of them, |acc_h| <= k_pad 2^30.1 and |acc_l| <= k_pad 2^38.3, inside
// int64 for k_pad < 2^24. The value in units of level S + 1 is acc_h 2^OZ_HSH + acc_l.
constexpr int OZ_LH = 5;
constexpr int OZ_HSH = OZ_BETA * (OZ_S + 1 - OZ_LH);
__device__ __forceinline__ int oz_level_shift(int L) {
  return L <= OZ_LH ? OZ_BETA * (OZ_LH - L) : OZ_BETA * (OZ_S + 1 - L);
}
// acc_h 2^OZ_HSH + acc_l as a double: the exact sum is hi 2^OZ_HSH + lo with 0 <= lo < 2^OZ_HSH;
// hi is exact in FP64 for k_pad < 2^22 (|hi| < 2^53), so the one rounding is the fma's (beyond
// that, up to the 2^24 the callers allow, hi is rounded first: within an ulp, no longer one
// rounding).
__device__ __forceinline__ double oz_fixed_value(long long acc_h, long long acc_l) {
  const long long hi = acc_h + (acc_l >> OZ_HSH);
  const long long lo = acc_l & ((1ll << OZ_HSH) - 1);
  return fma((double)hi, (double)(1ll << OZ_HSH), (double)lo);
}

// C = alpha * sum over levels of the exact chunk sums (scaled per level) + beta * C. One warp
// per piece of an output row; the chunk sums are integers of at most 2^24, added per level and
// into the two fixed-point accumulators above, converted once to FP64.
__global__ void oz_combine_kernel(GemmArgs g, const float* __restrict__ part, int kseg, int nk,
                                  const unsigned* __restrict__ expA, int rowsA_pad, const unsigned* __restrict__ expB,
                                  int rowsB_pad, int piece) {
  const int lane = threadIdx.x & 31;
  const size_t tot = (size_t)g.batch * g.M * g.N;
  const int pieces = (g.N + piece - 1) / piece;
  const long long items = (long long)g.batch * g.M * pieces;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = w0; it < items; it += nw) {
    const long long qrow = it / pieces;
    const int n0 = (int)(it - qrow * pieces) * piece, n1 = min(g.N, n0 + piece);
    const int b = (int)(qrow / g.M), m = (int)(qrow - (long long)b * g.M);
    const long long rowoff = cidx(g.cb, b) + cidx(g.cm, m);
    const float* pr = part + (size_t)qrow * g.N;
    const int ea = (int)max(expA[(size_t)b * rowsA_pad + m], 1u) - 1022;  // sigma of row m
    // alpha 2^(sigma_m - beta (S + 1)) for the row, 2^tau_n per column: the scaling is two
    // multiplications by exact powers of two while their exponents are inside the normal range
    const int er = ea - OZ_BETA * (OZ_S + 1);
    const double row_scale = g.alpha * pow2(er);
    CWalk cw;
    cw.init(g.cn, n0 + lane);
    for (int n = n0 + lane; n < n1; n += 32) {
      long long acc_h = 0, acc_l = 0;
      int v = 0;
      for (int L = 2; L <= OZ_S + 1; ++L) {
        const int nch = ((L - 1) * kseg + nk - 1) / nk;
        long long lv = 0;
        for (int c = 0; c < nch; ++c, ++v) lv += (long long)__float2int_rn(pr[(size_t)v * tot + n]);
        if (L <= OZ_LH) acc_h += lv << oz_level_shift(L);
        else acc_l += lv << oz_level_shift(L);
      }
      const double x = oz_fixed_value(acc_h, acc_l);
      const int eb = (int)max(expB[(size_t)b * rowsB_pad + n], 1u) - 1022;
      const double val = (er > -960 && er < 960 && eb > -960 && eb < 960 && er + eb > -960 && er + eb < 960)
                             ? x * row_scale * pow2(eb)
                             : g.alpha * ldexp(x, er + eb);
      double* c = g.C + rowoff + cw.off;
      *c = g.beta == 0.0 ? val : fma(g.beta, *c, val);
      cw.step(g.cn, 32);
    }
  }
}

struct TcArgs {
  int M, N, kblocks, num_m, num_n, tiles;  // tiles counts splits x batch x num_m x num_n
  int m_fast;                             // 1: consecutive tiles walk down m (they share a B tile)
  int splits, kchunk;                     // split-k: k blocks [s * kchunk, (s + 1) * kchunk)
  // Ozaki slices (oz_S > 0): the operands hold oz_S slices of oz_kseg k blocks each, and the
  // splits enumerate the (level, chunk) pairs of the slice products (see oz_split_range)
  int oz_S, oz_kseg, oz_nk;
  int batch;
  CIdx cm, cn, cb;
  double alpha, beta;
  double* C;
  float* part;  // split-k partial sums [splits][batch][M][N] (splits > 1)
  int* err;
  unsigned long long wait_ns;  // bound on every mbarrier wait (global timer)
  void* Cs;     // non-null: C in staging layout (offsets from cm/cn/cb count elements)
  long long cs_kpad;
  int cs_nseg, cs_seglo;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// waits for the phase of the given parity to complete; false after limit_ns of global time
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it >= 32) __nanosleep(64);  // back off so idle roles do not take issue slots
    if ((it & 63) == 0) {
      unsigned long long t = gtime();
      if (t0 == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// instruction descriptor: D = F32, A = B = TF32 or BF16, both K-major, N = TNT, M = TM
template <bool BF, int TNT>
constexpr uint32_t idesc() {
  return (1u << 4) | (Elt<BF>::FMT << 7) | (Elt<BF>::FMT << 10) | ((uint32_t)(TNT >> 3) << 17) |
         ((uint32_t)(TM >> 4) << 24);
}

// Split sp of an Ozaki product -> its level L and k-block ranges. Level L = s + t collects the
// slice products A_s B_t (s, t >= 1): A's slices 1..L-1 are its segments 0..L-2, B holds its
// slices in reverse order (slice t in segment S - t), so the partners L-1..1 are B's segments
// S-L+1..S-1 and one level is a single run of (L-1) kseg k blocks in both operands. A level is
// cut into chunks of at most nk k blocks, each one split (its own FP32 partial sum).
__host__ __device__ __forceinline__ int oz_split_range(int S, int kseg, int nk, int sp, int& kA0, int& kB0,
                                                      int& nkb) {
  for (int L = 2; L <= S + 1; ++L) {
    const int len = (L - 1) * kseg, nch = (len + nk - 1) / nk;
    if (sp < nch) {
      kA0 = sp * nk;
      kB0 = (S - L + 1) * kseg + sp * nk;
      nkb = min(nk, len - sp * nk);
      return L;
    }
    sp -= nch;
  }
  kA0 = kB0 = nkb = 0;
  return 0;
}

// tile t -> (split, batch entry, first row, first column, k blocks of A and of B, their count)
template <int TNT>
__device__ __forceinline__ void tile_coords(const TcArgs& g, int t, int& sp, int& bz, int& m0, int& n0, int& kA0,
                                            int& kB0, int& nkb) {
  const int per = g.num_m * g.num_n;
  const int outer = t / per;
  sp = outer / g.batch;
  bz = outer - sp * g.batch;
  const int r = t - outer * per;
  if (g.m_fast) {
    m0 = (r % g.num_m) * TM;
    n0 = (r / g.num_m) * TNT;
  } else {
    m0 = (r / g.num_n) * TM;
    n0 = (r % g.num_n) * TNT;
  }
  if (g.oz_S > 0) {
    oz_split_range(g.oz_S, g.oz_kseg, g.oz_nk, sp, kA0, kB0, nkb);
  } else {
    kA0 = kB0 = sp * g.kchunk;
    nkb = min(g.kblocks, kA0 + g.kchunk) - kA0;
  }
}

// The problems of one launch: one contraction, or several independent contractions (a
// grouped launch) that share the tile shape, the operand type and the output mode. Their tiles
// are numbered consecutively (tile0 holds the prefix sums), and every CTA walks the combined
// tile list. Passed by value as a __grid_constant__ parameter, so the tensor maps live in the
// parameter space that TMA reads.
template <int MAXP>
struct TcGroup {
  CUtensorMap tmA[MAXP];
  CUtensorMap tmB[MAXP];
  TcArgs args[MAXP];
  int tile0[MAXP + 1];
  int nprob;
};
constexpr int GROUP_MAX = 16;  // problems of a grouped launch (about 7 KB of parameters)

// the problem that owns global tile t, searched onward from the previous one (t only grows)
template <int MAXP>
__device__ __forceinline__ int group_problem(const TcGroup<MAXP>& G, int t, int p) {
  while (p + 1 < G.nprob && t >= G.tile0[p + 1]) ++p;
  return p;
}

// shared memory: STAGES x (A tile, B tile), the epilogue's turn-around tiles, barriers
constexpr uint32_t EP_FLOATS = 32 * 33;
constexpr size_t SMEM_USED =
    (size_t)STAGES * (A_BYTES + B_BYTES) + EPI_WARPS * EP_FLOATS * 4 + (2 * STAGES + 4) * 8 + 16;
static_assert(1024 + SMEM_USED <= 232448, "shared memory beyond 227 KB");

// What the epilogue writes: C in FP64 (alpha acc + beta C), split-k FP32 partial sums, the
// staging layout of a later contraction with one segment or three ([hi|lo|hi]), or C as plain
// FP32 words (alpha acc) at the compound offsets of C.
enum { EPI_F64 = 0, EPI_PART = 1, EPI_STAGED1 = 2, EPI_STAGED3 = 3, EPI_F32 = 4, EPI_COUNT = 5 };
constexpr size_t SMEM_BYTES = 1024 + SMEM_USED;

// Persistent, warp-specialised GEMM: each CTA walks tiles blockIdx.x, +gridDim.x, ...
//   warp 0: TMA producer through the STAGES-deep full/empty ring
//   warp 1: TMEM allocator and the single MMA-issuing thread; alternates two accumulators
//   warps 2-9: epilogue (TMEM lane quadrant = warp % 4, two warps per quadrant on the two
//              column halves), releasing an accumulator as soon as it has been read, so the
//              next tile's MMAs overlap this tile's stores
// Tiles are TM x TNT, TNT = 256 or 128 (the narrower tile for outputs with fewer tiles than SMs:
// twice the tiles for the same output); the shared-memory ring keeps its 256-row B stages.
template <bool BF, int EPI, int MAXP, int TNT>
__global__ void __launch_bounds__(THREADS, 1) gemm_tc_kernel(const __grid_constant__ TcGroup<MAXP> G) {
  static_assert(TNT == 256 || TNT == 128, "tile width");
  constexpr int TK = Elt<BF>::TK, UK = Elt<BF>::UK;
  using T = typename Elt<BF>::T;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  float* ep = reinterpret_cast<float*>(sB + STAGES * B_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ep + EPI_WARPS * EP_FLOATS);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, EPI_WARPS);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TNT)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  const int total = G.tile0[G.nprob];
  const unsigned long long wait_ns = G.args[0].wait_ns;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t q = 0;  // pipeline slot counter, continued across tiles
      int p = 0;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        p = group_problem(G, t, p);
        const TcArgs& g = G.args[p];
        int sp, bz, m0, n0, kA0, kB0, nkb;
        tile_coords<TNT>(g, t - G.tile0[p], sp, bz, m0, n0, kA0, kB0, nkb);
        for (int kb = 0; kb < nkb; ++kb, ++q) {
          const int s = q % STAGES;
          const uint32_t ph = (q / STAGES) & 1;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1, wait_ns)) { ok = false; break; }
          mbar_expect_tx(full0 + 8 * s, A_BYTES + TNT * 128);
          tma_load_3d(smem_u32(sA + s * A_BYTES), &G.tmA[p], full0 + 8 * s, (kA0 + kb) * TK, m0, bz);
          tma_load_3d(smem_u32(sB + s * B_BYTES), &G.tmB[p], full0 + 8 * s, (kB0 + kb) * TK, n0, bz);
        }
      }
      // never leave with copies in flight: the last loads issued must have landed (bounded)
      for (uint32_t r = q > (uint32_t)STAGES ? q - STAGES : 0; r < q; ++r)
        if (!mbar_wait(full0 + 8 * (r % STAGES), (r / STAGES) & 1, wait_ns)) ok = false;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t q = 0;
      int it = 0, p = 0;
      const uint64_t descA = sdesc(smem_u32(sA)), descB = sdesc(smem_u32(sB));
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
        const int acc = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(tempty0 + 8 * acc, (use & 1) ^ 1, wait_ns)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(acc * TNT);
        p = group_problem(G, t, p);
        int sp, bz, m0, n0, kA0, kB0, nkb;
        tile_coords<TNT>(G.args[p], t - G.tile0[p], sp, bz, m0, n0, kA0, kB0, nkb);
        for (int kb = 0; kb < nkb; ++kb, ++q) {
          const int s = q % STAGES;
          const uint32_t ph = (q / STAGES) & 1;
          if (!mbar_wait(full0 + 8 * s, ph, wait_ns)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // the descriptors' address field counts 16 bytes: stage s and step j (UK elements = 32
          // bytes) are offsets from the first stage's descriptors
          const uint64_t da0 = descA + (uint64_t)(s * (A_BYTES >> 4)), db0 = descB + (uint64_t)(s * (B_BYTES >> 4));
#pragma unroll
          for (int j = 0; j < TK / UK; ++j) {
            const uint64_t da = da0 + 2 * j, db = db0 + 2 * j;
            const uint32_t accum = (kb > 0 || j > 0) ? 1u : 0u;
            if constexpr (BF) {
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                  "l"(da), "l"(db), "r"(idesc<BF, TNT>()), "r"(accum)
                  : "memory");
            } else {
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                  "l"(da), "l"(db), "r"(idesc<BF, TNT>()), "r"(accum)
                  : "memory");
            }
          }
          // frees the stage once these MMAs have read it
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * s)
                       : "memory");
        }
        if (!ok) break;
        // the accumulator is complete once every MMA issued so far has finished
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tfull0 + 8 * acc)
                     : "memory");
      }
    }
    __syncwarp();
  } else {
    const int quad = warp & 3;          // the TMEM lanes (tile rows) this warp may read
    const int half = (warp - 2) >> 2;   // the half of the tile's columns it stores
    float* tile = ep + (warp - 2) * EP_FLOATS;
    int it = 0, p = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
      const int acc = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      bool got = mbar_wait(tfull0 + 8 * acc, use & 1, wait_ns);
      got = __all_sync(0xffffffffu, got);
      if (!got) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      p = group_problem(G, t, p);
      const TcArgs& g = G.args[p];
      const float alpha_f = (float)g.alpha;
      int sp, bz, m0, n0, kA0, kB0, nkb;
      tile_coords<TNT>(g, t - G.tile0[p], sp, bz, m0, n0, kA0, kB0, nkb);
      // each lane locates one of the warp's 32 rows once; the store loop broadcasts them
      const int my_row = m0 + quad * 32 + lane;
      long long my_off = -1;
      if (my_row < g.M)
        my_off = EPI == EPI_PART ? (((long long)sp * g.batch + bz) * g.M + my_row) * (long long)g.N
                                 : cidx(g.cb, bz) + cidx(g.cm, my_row);
#pragma unroll 1
      for (int c0 = half * (TNT / 2); c0 < (half + 1) * (TNT / 2); c0 += 32) {
        // the rest of the tile lies past the last column, or this warp's 32 rows past the last
        // row (both warp-uniform)
        if (n0 + c0 >= g.N || m0 + quad * 32 >= g.M) break;
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * TNT + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%"
            "22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
              "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
              "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        // a warp's stores run along a row of C
        const int n = n0 + c0 + lane;
        const bool n_ok = n < g.N;
        if constexpr (EPI == EPI_PART) {
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) {
            const long long ro = __shfl_sync(0xffffffffu, my_off, rr);
            if (ro >= 0 && n_ok) g.part[ro + n] = tile[rr * 33 + lane];
          }
        } else if constexpr (EPI == EPI_F32) {
          float* cs = static_cast<float*>(g.Cs) + (n_ok ? cidx(g.cn, n) : 0);
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) {
            const long long ro = __shfl_sync(0xffffffffu, my_off, rr);
            if (ro >= 0 && n_ok) cs[ro] = alpha_f * tile[rr * 33 + lane];
          }
        } else if constexpr (EPI == EPI_STAGED1 || EPI == EPI_STAGED3) {
          T* cs = static_cast<T*>(g.Cs) + (n_ok ? cidx(g.cn, n) : 0);
          const long long kpad = g.cs_kpad;
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) {
            const long long ro = __shfl_sync(0xffffffffu, my_off, rr);
            if (ro >= 0 && n_ok)
              store_staged_fixed<EPI == EPI_STAGED3 ? 3 : 1>(cs + ro, kpad, alpha_f * tile[rr * 33 + lane]);
          }
        } else {
          double* cc = g.C + (n_ok ? cidx(g.cn, n) : 0);
          if (g.beta == 0.0) {
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) {
              const long long ro = __shfl_sync(0xffffffffu, my_off, rr);
              if (ro >= 0 && n_ok) cc[ro] = g.alpha * (double)tile[rr * 33 + lane];
            }
          } else {
            // the 32 rows' old values are read first, so that all their loads are in flight at
            // once (an accumulating epilogue otherwise waits for one load latency per few rows)
            double old[32];
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
              const long long ro = __shfl_sync(0xffffffffu, my_off, rr);
              old[rr] = (ro >= 0 && n_ok) ? cc[ro] : 0.0;
            }
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
              const long long ro = __shfl_sync(0xffffffffu, my_off, rr);
              if (ro >= 0 && n_ok) cc[ro] = fma(g.beta, old[rr], g.alpha * (double)tile[rr * 33 + lane]);
            }
          }
        }
        __syncwarp();
      }
      // hand the accumulator back to the MMA thread
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
    }
  }
  if (!ok) atomicExch(G.args[0].err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TNT) : "memory");
}

// ---------------------------------------------------------------------------
// On-chip recombination of the FP64 emulation: one persistent launch whose tile is a 128 x 128
// block of C and whose work per tile is every (level, chunk) slice product in turn, level by
// level. The MMA thread alternates two FP32 accumulators over a tile's slice products; the
// epilogue warps read each exact chunk sum once and add it, shifted for its level, into a 64-bit
// fixed-point sum in registers (64 columns of one row per thread), so no partial sum leaves the
// SM. A tile's slice products run from the highest level down: the longest ones come first, so
// while the epilogue finishes one tile (conversion and stores) the MMA thread works through the
// next tile's two longest products. After the levels above OZ_LH (oz_fixed_value) the register
// sums are parked in TMEM and the levels up to OZ_LH start from zero; the two are joined at the
// end. Same integers, same single rounding as oz_combine_kernel: the result is the same bits.
// ---------------------------------------------------------------------------
constexpr int OZ_TN = 128;
constexpr int OZ_STAGES = 5;
constexpr uint32_t OZ_B_BYTES = OZ_TN * 128;
constexpr uint32_t OZ_EP_DOUBLES = 32 * 17;  // per epilogue warp: 32 rows x 16 columns (+1 pad)
constexpr size_t OZ_SMEM_BYTES = 1024 + (size_t)OZ_STAGES * (A_BYTES + OZ_B_BYTES) +
                                 EPI_WARPS * OZ_EP_DOUBLES * 8 + (2 * OZ_STAGES + 4) * 8 + 16;
static_assert(OZ_SMEM_BYTES <= 232448, "shared memory beyond 227 KB");
constexpr uint32_t OZ_TMEM_COLS = 512;  // two accumulators of 128 columns; the first group's int64 sums

struct OzArgs {
  int M, N, num_m, num_n, tiles, batch, m_fast;
  int kseg, nk, nsplit;
  CIdx cm, cn, cb;
  double alpha, beta;
  double* C;
  const unsigned* expA;  // biased exponent maxima of A's rows and B's columns
  const unsigned* expB;
  int rowsA_pad, rowsB_pad;
  int* err;
  unsigned long long wait_ns;
};

// instruction descriptor: D = F32, A = B = BF16, both K-major, N = OZ_TN, M = TM
constexpr uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void oz_tile(const OzArgs& a, int t, int& bz, int& m0, int& n0) {
  const int per = a.num_m * a.num_n;
  bz = t / per;
  const int r = t - bz * per;
  if (a.m_fast) {
    m0 = (r % a.num_m) * TM;
    n0 = (r / a.num_m) * OZ_TN;
  } else {
    m0 = (r / a.num_n) * TM;
    n0 = (r % a.num_n) * OZ_TN;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// waits for this thread's TMEM loads; the registers are operands, so no use of them moves above
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16], uint32_t (&s)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]), "+r"(s[7]), "+r"(s[8]), "+r"(s[9]), "+r"(s[10]), "+r"(s[11]), "+r"(s[12]), "+r"(s[13]), "+r"(s[14]), "+r"(s[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ OzArgs a) {
  constexpr int TK = Elt<true>::TK, UK = Elt<true>::UK;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + OZ_STAGES * A_BYTES;
  double* ep = reinterpret_cast<double*>(sB + OZ_STAGES * OZ_B_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ep + EPI_WARPS * OZ_EP_DOUBLES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_STAGES + 4);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + OZ_STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * OZ_STAGES), tempty0 = smem_u32(bars + 2 * OZ_STAGES + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  const unsigned long long wait_ns = a.wait_ns;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t q = 0;
      for (int t = blockIdx.x; t < a.tiles && ok; t += gridDim.x) {
        int bz, m0, n0;
        oz_tile(a, t, bz, m0, n0);
        for (int i = 0; i < a.nsplit && ok; ++i) {
          int kA0, kB0, nkb;
          oz_split_range(OZ_S, a.kseg, a.nk, a.nsplit - 1 - i, kA0, kB0, nkb);
          for (int kb = 0; kb < nkb; ++kb, ++q) {
            const int s = q % OZ_STAGES;
            const uint32_t ph = (q / OZ_STAGES) & 1;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1, wait_ns)) { ok = false; break; }
            mbar_expect_tx(full0 + 8 * s, A_BYTES + OZ_B_BYTES);
            tma_load_3d(smem_u32(sA + s * A_BYTES), &tmA, full0 + 8 * s, (kA0 + kb) * TK, m0, bz);
            tma_load_3d(smem_u32(sB + s * OZ_B_BYTES), &tmB, full0 + 8 * s, (kB0 + kb) * TK, n0, bz);
          }
        }
      }
      for (uint32_t r = q > (uint32_t)OZ_STAGES ? q - OZ_STAGES : 0; r < q; ++r)
        if (!mbar_wait(full0 + 8 * (r % OZ_STAGES), (r / OZ_STAGES) & 1, wait_ns)) ok = false;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t q = 0, u = 0;  // pipeline slots; slice products (accumulator uses)
      const uint64_t descA = sdesc(smem_u32(sA)), descB = sdesc(smem_u32(sB));
      for (int t = blockIdx.x; t < a.tiles && ok; t += gridDim.x) {
        for (int i = 0; i < a.nsplit; ++i, ++u) {
          const int acc = u & 1;
          if (!mbar_wait(tempty0 + 8 * acc, ((u >> 1) & 1) ^ 1, wait_ns)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(acc * OZ_TN);
          int kA0, kB0, nkb;
          oz_split_range(OZ_S, a.kseg, a.nk, a.nsplit - 1 - i, kA0, kB0, nkb);
          for (int kb = 0; kb < nkb; ++kb, ++q) {
            const int s = q % OZ_STAGES;
            if (!mbar_wait(full0 + 8 * s, (q / OZ_STAGES) & 1, wait_ns)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da0 = descA + (uint64_t)(s * (A_BYTES >> 4)), db0 = descB + (uint64_t)(s * (OZ_B_BYTES >> 4));
#pragma unroll
            for (int j = 0; j < TK / UK; ++j) {
              const uint64_t da = da0 + 2 * j, db = db0 + 2 * j;
              const uint32_t accum = (kb > 0 || j > 0) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                  "l"(da), "l"(db), "r"(oz_idesc()), "r"(accum)
                  : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty0 + 8 * s)
                         : "memory");
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tfull0 + 8 * acc)
                       : "memory");
        }
      }
    }
    __syncwarp();
  } else {
    const int quad = warp & 3;         // TMEM lanes = tile rows quad * 32 .. + 31
    const int half = (warp - 2) >> 2;  // columns half * 64 .. + 63 of the tile
    double* tile = ep + (warp - 2) * OZ_EP_DOUBLES;
    const uint32_t lanes = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t tpark = lanes + 2 * OZ_TN + half * 128;  // the first group's sums: 64 int64
    uint32_t u = 0;
    for (int t = blockIdx.x; t < a.tiles && ok; t += gridDim.x) {
      int bz, m0, n0;
      oz_tile(a, t, bz, m0, n0);
      long long acc[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) acc[j] = 0;
      bool low = true;  // summing the levels above OZ_LH (they come first)
      for (int i = 0; i < a.nsplit; ++i, ++u) {
        int kA0, kB0, nkb;
        const int L = oz_split_range(OZ_S, a.kseg, a.nk, a.nsplit - 1 - i, kA0, kB0, nkb);
        if (low && L <= OZ_LH) {  // first group done: park its sums in TMEM, start the second
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            uint32_t w[16];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              w[2 * j] = (uint32_t)(unsigned long long)acc[p * 8 + j];
              w[2 * j + 1] = (uint32_t)((unsigned long long)acc[p * 8 + j] >> 32);
            }
            tmem_st16(tpark + p * 16, w);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 64; ++j) acc[j] = 0;
          low = false;
        }
        const int sh = oz_level_shift(L);
        const int buf = u & 1;
        bool got = mbar_wait(tfull0 + 8 * buf, (u >> 1) & 1, wait_ns);
        got = __all_sync(0xffffffffu, got);
        if (!got) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tacc = lanes + buf * OZ_TN + half * 64;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          uint32_t r[16];
          tmem_ld16(tacc + p * 16, r);
          tmem_wait_ld(r);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[p * 16 + j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
        }
        // the accumulator goes back to the MMA thread
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
      }
      if (!ok) break;
      // C = alpha 2^(sigma_m + tau_n - beta (S + 1)) (acc_h 2^OZ_HSH + acc_l) + beta C, as in
      // oz_combine_kernel. A thread holds one row: 16 columns at a time go through shared memory
      // so that a warp's stores run along rows of C (two rows of 16 columns per store).
      const int my_row = m0 + quad * 32 + lane;
      long long my_off = -1;
      int my_er = 0;
      if (my_row < a.M) {
        my_off = cidx(a.cb, bz) + cidx(a.cm, my_row);
        my_er = (int)max(a.expA[(size_t)bz * a.rowsA_pad + my_row], 1u) - 1022 - OZ_BETA * (OZ_S + 1);
      }
      const bool rows_left = m0 + quad * 32 < a.M;  // warp-uniform
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int c0 = n0 + half * 64 + p * 16;
        if (!rows_left || c0 >= a.N) break;  // warp-uniform
        uint32_t w0[16], w1[16];
        tmem_ld16(tpark + p * 32, w0);
        tmem_ld16(tpark + p * 32 + 16, w1);
        tmem_wait_ld(w0, w1);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t lo32 = j < 8 ? w0[2 * j] : w1[2 * (j - 8)];
          const uint32_t hi32 = j < 8 ? w0[2 * j + 1] : w1[2 * (j - 8) + 1];
          const long long acc_l = (long long)(((unsigned long long)hi32 << 32) | lo32);  // parked
          tile[lane * 17 + j] = oz_fixed_value(acc[p * 16 + j], acc_l);
        }
        __syncwarp();
        const int col = c0 + (lane & 15);
        const bool n_ok = col < a.N;
        int eb = 0;
        long long coff = 0;
        if (n_ok) {
          eb = (int)max(a.expB[(size_t)bz * a.rowsB_pad + col], 1u) - 1022;
          coff = cidx(a.cn, col);
        }
#pragma unroll 4
        for (int r0 = 0; r0 < 32; r0 += 2) {
          const int row = r0 + (lane >> 4);
          const long long ro = __shfl_sync(0xffffffffu, my_off, row);
          const int er = __shfl_sync(0xffffffffu, my_er, row);
          if (ro >= 0 && n_ok) {
            const double x = tile[row * 17 + (lane & 15)];
            const double row_scale = a.alpha * pow2(er);
            const double val = (er > -960 && er < 960 && eb > -960 && eb < 960 && er + eb > -960 && er + eb < 960)
                                   ? x * row_scale * pow2(eb)
                                   : a.alpha * ldexp(x, er + eb);
            double* c = a.C + ro + coff;
            *c = a.beta == 0.0 ? val : fma(a.beta, *c, val);
          }
        }
        __syncwarp();
      }
    }
  }
  if (!ok) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
}

// Self-test of the bounded waits: one thread waits on an mbarrier that expects one arrival
// which never comes, with the same bounded wait as the GEMM's pipeline. After limit_ns it
// gives up, records the failure in the error flag and the kernel returns normally.
__global__ void wait_selftest_kernel(int* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(b, 0, limit_ns)) atomicExch(err, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // looked up once per process (thread-safe static initialisation; retried if it threw)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    CC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    CC_REQUIRE(p && q == cudaDriverEntryPointSuccess, CC_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

// 3-D map over a [batch][rows][k_pad] array of FP32 or BF16, box = 128 bytes of k x box_rows x 1
CUtensorMap make_map(const void* base, int k_pad, int rows_pad, int batch, int box_rows, bool bf) {
  CUtensorMap m;
  const cuuint64_t es = bf ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)k_pad, (cuuint64_t)rows_pad, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)k_pad * es, (cuuint64_t)k_pad * rows_pad * es};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                           const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CC_REQUIRE(r == CUDA_SUCCESS, CC_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

}  // namespace

namespace {

// The dynamic shared-memory opt-in is per device and per kernel instance; server threads may
// race here, so the per-device bits are atomic.
template <typename K>
void ensure_smem_attr(K kern, std::atomic<uint64_t>& done, size_t bytes = SMEM_BYTES) {
  int dev = 0;
  CC_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (!(done.load() & bit)) {
    CC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.fetch_or(bit);
  }
}

// A tensor-core contraction made ready to launch: operands staged, tensor maps and tile
// arguments set, split-k partial buffer allocated. It is launched alone or in a group with
// other jobs of the same operand type and output mode.
template <bool BF>
struct TcJob {
  GemmArgs g{};
  CUtensorMap mA, mB;
  TcArgs a{};
  int epi = EPI_F64;
  int tn = TN;  // tile width: TN, or 128 when the output has fewer TN-wide tiles than SMs
  DBuf<double> stA, stB, part;
};

// Operands waiting to be staged: collected while contractions are prepared, then staged by as
// few launches as possible (GATHER_MAX operands each) before the GEMMs that read them.
template <typename T>
struct GatherBatch {
  std::vector<GatherDesc> pend;
  void flush(const Exec& ex) {
    for (size_t i = 0; i < pend.size(); i += GATHER_MAX) {
      GatherList L;
      memset(&L, 0, sizeof(L));
      L.n = (int)std::min<size_t>(GATHER_MAX, pend.size() - i);
      L.item0[0] = 0;
      for (int j = 0; j < L.n; ++j) {
        const GatherDesc& d = pend[i + j];
        L.d[j] = d;
        const long long per_b = d.tr ? (long long)((d.rows_pad + 31) / 32) * ((d.k_pad + 31) / 32)
                                     : (long long)d.rows_pad * ((d.k_pad + ROW_PIECE - 1) / ROW_PIECE);
        L.item0[j + 1] = L.item0[j] + (long long)d.batch * per_b;
      }
      const long long items = L.item0[L.n];
      const int blocks = (int)std::max<long long>(1, std::min<long long>((items + 7) / 8, (long long)ex.sm_count * 16));
      gather_kernel<T><<<blocks, GATHER_THREADS, 0, ex.stream>>>(L);
      ex.count();
    }
    pend.clear();
    CC_CUDA(cudaGetLastError());
  }
};

template <bool BF>
void tc_prepare(const Exec& ex, cc_precision prec, const GemmArgs& g, TcJob<BF>& job,
                GatherBatch<typename Elt<BF>::T>& gb) {
  using T = typename Elt<BF>::T;
  constexpr int TK = Elt<BF>::TK;
  job.g = g;
  // outputs with fewer TN-wide tiles than SMs take 128-wide tiles: twice the tiles (and CTAs
  // writing the output) before any split of k
  const long long tiles_wide = (long long)((g.M + TM - 1) / TM) * ((g.N + TN - 1) / TN) * g.batch;
  const int tn = tiles_wide < ex.sm_count ? 128 : TN;
  job.tn = tn;
  const int rowsA = (g.M + TM - 1) / TM * TM, rowsB = (g.N + tn - 1) / tn * tn;
  const int k_pad = (g.K + TK - 1) / TK * TK;
  // the split precisions stage [hi|hi|lo] against [hi|lo|hi] along a three times longer k
  const int nseg = prec == CC_MIXED_TF32 ? 1 : 3;
  const int kk = nseg * k_pad;
  // Staged copy of one operand: taken from the cache when the caller marked the operand as
  // fixed and it was staged before with the same layout, else gathered (into the cache when
  // it is marked and fits, into a temporary otherwise) by the batch's next launch.
  auto stage = [&](int which, const double* src, const CIdx& rix, const CIdx& kix, const CIdx& bix, int rows,
                   int rows_pad, int seg_lo, DBuf<double>& tmp) -> T* {
    const size_t dbl = ((size_t)g.batch * rows_pad * kk * sizeof(T) + 7) / 8;
    double* dst = nullptr;
    if (g.cache && (g.cache_mask & which)) {
      const StageKey key{src, rix, kix, bix, rows, g.K, g.batch, rows_pad, k_pad, nseg, seg_lo, BF ? 1 : 0};
      for (auto& e : g.cache->ents)
        if (e.key == key) {
          if (e.fresh) return reinterpret_cast<T*>(e.buf.p);
          dst = e.buf.p;  // out of date: staged again in place (same address)
          e.fresh = true;
          break;
        }
      if (!dst && g.cache->bytes + dbl * 8 <= g.cache->cap) {
        // allocate first: if the pool throws, no entry is left keyed to a missing buffer
        DBuf<double> buf(ex.pool, dbl);
        g.cache->ents.emplace_back();
        StageCache::Ent& e = g.cache->ents.back();
        e.key = key;
        e.buf = std::move(buf);
        g.cache->bytes += dbl * 8;
        dst = e.buf.p;
      }
    }
    if (!dst) {
      tmp.alloc(ex.pool, dbl);
      dst = tmp.p;
    }
    GatherDesc d;
    d.src = src;
    d.out = dst;
    d.rix = rix;
    d.kix = kix;
    d.bix = bix;
    d.rows = rows;
    d.K = g.K;
    d.batch = g.batch;
    d.rows_pad = rows_pad;
    d.k_pad = k_pad;
    d.nseg = nseg;
    d.seg_lo = seg_lo;
    // the stride of a compound index's innermost mode of extent > 1
    auto inner = [](const CIdx& c) { return c.e2 > 1 ? c.s2 : c.e1 > 1 ? c.s1 : c.s0; };
    d.tr = (g.K > 1 && inner(kix) != 1 && rows > 1 && inner(rix) == 1) ? 1 : 0;
    gb.pend.push_back(d);
    return reinterpret_cast<T*>(dst);
  };
  T* fA = stage(1, g.A, g.am, g.ak, g.ab, g.M, rowsA, nseg == 3 ? 0b100 : 0, job.stA);
  T* fB = nullptr;
  int rowsBmap = rowsB;
  if (g.sb) {
    // B was written in staging layout by an earlier contraction
    CC_REQUIRE(g.batch == 1 && g.sb->kk == kk && g.sb->rows_pad >= rowsB && g.sb->rows_pad % tn == 0,
               CC_ERR_INVALID, "staged operand does not match the contraction");
    fB = static_cast<T*>(const_cast<void*>(g.sb->base));
    rowsBmap = g.sb->rows_pad;
  } else {
    fB = stage(2, g.B, g.bn, g.bk, g.bb, g.N, rowsB, nseg == 3 ? 0b010 : 0, job.stB);
  }
  CC_REQUIRE(!g.so || g.beta == 0.0, CC_ERR_INVALID, "a staged output cannot accumulate");
  job.mA = make_map(fA, kk, rowsA, g.batch, TM, BF);
  job.mB = make_map(fB, kk, rowsBmap, g.batch, tn, BF);
  TcArgs& a = job.a;
  a.M = g.M;
  a.N = g.N;
  a.kblocks = kk / TK;
  a.num_m = rowsA / TM;
  a.num_n = rowsB / tn;
  a.batch = g.batch;
  // Tiles that run at the same time share operand tiles through L2: the shorter of the two
  // tile dimensions runs fastest, so a wave of CTAs covers whole columns (or rows) of tiles
  // and the long operand is read from HBM about once instead of once per tile row.
  a.m_fast = a.num_m <= a.num_n ? 1 : 0;
  // split k when the output has fewer tiles than SMs and the sum is long: every split is a
  // tile of its own that writes FP32 partial sums, added in order by a second kernel. The
  // factor s minimises a time model of the persistent grid: waves(s) = ceil(tiles s / SMs)
  // passes of (a tile's MMA time / s + a fixed per-tile cost for the pipeline fill and the
  // epilogue), plus the HBM time of writing and re-reading the s partial sums.
  const long long base_tiles = (long long)a.num_m * a.num_n * g.batch;
  int splits = 1;
  if (base_tiles < ex.sm_count && a.kblocks >= 8) {
    const double sm_rate = (BF ? 2.0 : 1.0) * 5.8e12;  // dense MMA flop/s of one SM
    const double t_tile = 2.0 * TM * tn * (double)a.kblocks * TK / sm_rate;
    const double t_fix = 3e-6, hbm = 6.0e12;
    const double part_bytes = 8.0 * (double)g.batch * g.M * g.N;  // FP32 written + read, per split
    auto model = [&](int sp) {
      const double waves = (double)((base_tiles * sp + ex.sm_count - 1) / ex.sm_count);
      // the reduce: launch, partial-sum traffic, and one dependent load batch per 8 splits
      return waves * (t_tile / sp + t_fix) + (sp > 1 ? (sp * part_bytes / hbm + 4e-6 + sp * 0.1e-6) : 0.0);
    };
    double best = model(1);
    const int smax = (int)std::min<long long>(256, a.kblocks / 2);
    for (int sp = 2; sp <= smax; ++sp) {
      const double t = model(sp);
      if (t < best * (1.0 - 1e-9)) {
        best = t;
        splits = sp;
      }
    }
  }
  a.kchunk = (a.kblocks + splits - 1) / splits;
  splits = (a.kblocks + a.kchunk - 1) / a.kchunk;  // no empty split
  a.oz_S = a.oz_kseg = a.oz_nk = 0;
  a.splits = splits;
  a.tiles = (int)(base_tiles * splits);
  a.cm = g.cm;
  a.cn = g.cn;
  a.cb = g.cb;
  a.alpha = g.alpha;
  a.beta = g.beta;
  a.C = g.C;
  a.err = ex.dev_flag;
  a.wait_ns = ex.wait_ns;
  a.Cs = g.so ? g.so->base : nullptr;
  a.cs_kpad = g.so ? g.so->kpad : 0;
  a.cs_nseg = g.so ? g.so->nseg : 0;
  a.cs_seglo = g.so ? g.so->seg_lo : 0;
  a.part = nullptr;
  if (splits > 1) {
    const size_t np = (size_t)splits * g.batch * g.M * g.N;
    job.part.alloc(ex.pool, (np + 1) / 2);
    a.part = reinterpret_cast<float*>(job.part.p);
  }
  // the epilogue's output mode is a template parameter, so its store loop has no run-time
  // branching on the layout
  job.epi = EPI_F64;
  if (splits > 1) {
    job.epi = EPI_PART;
  } else if (g.so) {
    CC_REQUIRE(g.so->nseg == 0 || (g.so->nseg == 1 && g.so->seg_lo == 0) || (g.so->nseg == 3 && g.so->seg_lo == 0b010),
               CC_ERR_INVALID, "staged output layout not supported by the tensor-core epilogue");
    job.epi = g.so->nseg == 0 ? EPI_F32 : g.so->nseg == 3 ? EPI_STAGED3 : EPI_STAGED1;
  }
}

// One launch over n jobs of one output mode (n <= MAXP): their tiles numbered consecutively,
// one persistent CTA per SM at most.
template <bool BF, int EPI, int MAXP, int TNT>
void tc_launch_group(const Exec& ex, TcJob<BF>* const* jobs, int n) {
  static std::atomic<uint64_t> attr_done{0};
  auto kern = gemm_tc_kernel<BF, EPI, MAXP, TNT>;
  ensure_smem_attr(kern, attr_done);
  TcGroup<MAXP> G;
  memset(&G, 0, sizeof(G));
  G.nprob = n;
  G.tile0[0] = 0;
  for (int i = 0; i < n; ++i) {
    G.tmA[i] = jobs[i]->mA;
    G.tmB[i] = jobs[i]->mB;
    G.args[i] = jobs[i]->a;
    CC_REQUIRE((long long)G.tile0[i] + jobs[i]->a.tiles < (1LL << 31), CC_ERR_INVALID, "grouped launch: too many tiles");
    G.tile0[i + 1] = G.tile0[i] + jobs[i]->a.tiles;
  }
  const int grid = std::min(G.tile0[n], ex.sm_count);
  if (grid <= 0) return;
  kern<<<grid, THREADS, SMEM_BYTES, ex.stream>>>(G);
  ex.count();
  CC_CUDA(cudaGetLastError());
}

template <bool BF, int MAXP, int TNT>
void tc_launch_tn(const Exec& ex, int epi, TcJob<BF>* const* jobs, int n) {
  switch (epi) {
    case EPI_PART: tc_launch_group<BF, EPI_PART, MAXP, TNT>(ex, jobs, n); break;
    case EPI_STAGED1: tc_launch_group<BF, EPI_STAGED1, MAXP, TNT>(ex, jobs, n); break;
    case EPI_STAGED3: tc_launch_group<BF, EPI_STAGED3, MAXP, TNT>(ex, jobs, n); break;
    case EPI_F32: tc_launch_group<BF, EPI_F32, MAXP, TNT>(ex, jobs, n); break;
    default: tc_launch_group<BF, EPI_F64, MAXP, TNT>(ex, jobs, n); break;
  }
}
template <bool BF, int MAXP>
void tc_launch(const Exec& ex, int epi, int tn, TcJob<BF>* const* jobs, int n) {
  if (tn == 128) tc_launch_tn<BF, MAXP, 128>(ex, epi, jobs, n);
  else tc_launch_tn<BF, MAXP, TN>(ex, epi, jobs, n);
}

// split-k: the partial sums of a finished job added in a fixed order into C (or its staging)
template <bool BF>
void tc_finish(const Exec& ex, TcJob<BF>& job) {
  using T = typename Elt<BF>::T;
  const GemmArgs& g = job.g;
  if (job.a.splits <= 1) return;
  const size_t outs = (size_t)g.batch * g.M * g.N;
  if (outs < 65536 && job.a.splits >= 16) {  // few outputs, many splits: spread the splits
    const int rblocks = (int)std::max<size_t>(1, std::min<size_t>((outs + 31) / 32, (size_t)ex.sm_count * 16));
    tc_splitk_reduce_small_kernel<T><<<rblocks, 256, 0, ex.stream>>>(
        g, job.a.part, job.a.splits, static_cast<T*>(job.a.Cs), job.a.cs_kpad, job.a.cs_nseg, job.a.cs_seglo);
    ex.count();
    CC_CUDA(cudaGetLastError());
    return;
  }
  // short outputs are cut into warp-sized pieces so that enough warps share the reads
  const size_t rows = (size_t)g.batch * g.M;
  const int piece = rows * ((g.N + ROW_PIECE - 1) / ROW_PIECE) >= (size_t)ex.sm_count * 64 ? ROW_PIECE : 32;
  const size_t items = rows * ((g.N + piece - 1) / piece);
  const int rblocks = (int)std::max<size_t>(1, std::min<size_t>((items + 7) / 8, (size_t)ex.sm_count * 16));
  tc_splitk_reduce_kernel<T><<<rblocks, 256, 0, ex.stream>>>(g, job.a.part, job.a.splits, static_cast<T*>(job.a.Cs),
                                                             job.a.cs_kpad, job.a.cs_nseg, job.a.cs_seglo, piece);
  ex.count();
  CC_CUDA(cudaGetLastError());
}

template <bool BF>
void run_tc(const Exec& ex, cc_precision prec, const GemmArgs& g, const char* tag) {
  TcJob<BF> job;
  GatherBatch<typename Elt<BF>::T> gb;
  tc_prepare<BF>(ex, prec, g, job, gb);
  gb.flush(ex);
  cudaEvent_t ev = nullptr;
  if (ex.timing(tag)) ex.mark_begin(&ev);
  TcJob<BF>* one = &job;
  tc_launch<BF, 1>(ex, job.epi, job.tn, &one, 1);
  tc_finish<BF>(ex, job);
  if (ev) ex.mark_end(tag, ev, 2.0 * g.M * (double)g.N * g.K * g.batch);
}

// Independent contractions of one precision in as few launches as possible: every job is
// prepared (operands staged), jobs of the same output mode share launches of up to GROUP_MAX
// problems, then the split-k reductions run.
template <bool BF>
void run_tc_group(const Exec& ex, cc_precision prec, const std::vector<GemmArgs>& gs, const char* tag) {
  std::vector<std::unique_ptr<TcJob<BF>>> jobs;
  GatherBatch<typename Elt<BF>::T> gb;
  double flops = 0.0;
  for (const auto& g : gs) {
    jobs.emplace_back(new TcJob<BF>());
    tc_prepare<BF>(ex, prec, g, *jobs.back(), gb);
    flops += 2.0 * g.M * (double)g.N * g.K * g.batch;
  }
  gb.flush(ex);
  cudaEvent_t ev = nullptr;
  if (ex.timing(tag)) ex.mark_begin(&ev);
  for (int epi = 0; epi < EPI_COUNT; ++epi)
    for (int tn : {TN, 128}) {
      std::vector<TcJob<BF>*> sel;
      for (auto& j : jobs)
        if (j->epi == epi && j->tn == tn) sel.push_back(j.get());
      for (size_t i = 0; i < sel.size(); i += GROUP_MAX) {
        const int n = (int)std::min<size_t>(GROUP_MAX, sel.size() - i);
        if (n == 1) tc_launch<BF, 1>(ex, epi, tn, &sel[i], 1);
        else tc_launch<BF, GROUP_MAX>(ex, epi, tn, &sel[i], n);
      }
    }
  for (auto& j : jobs) tc_finish<BF>(ex, *j);
  if (ev) ex.mark_end(tag, ev, flops);
}

// FP64-accurate contraction on the tensor cores (Ozaki splitting, above): stage both operands
// as OZ_S BF16 digit slices with per-row exponents, run every (level, chunk) slice product on
// kind::f16 (on chip, or as splits writing exact FP32 partial sums that a combine pass adds),
// and add the levels in integer fixed point into C = alpha A B + beta C.
int oz_splits(int kseg, int nk) {
  int n = 0;
  for (int L = 2; L <= OZ_S + 1; ++L) n += ((L - 1) * kseg + nk - 1) / nk;
  return n;
}

// Which form of the emulated product runs: on chip (oz_gemm_kernel: 128 x 128 tiles, every slice
// product of a tile on one SM, no partial sums) or through FP32 partial sums (every (level, chunk)
// slice product of a 128 x 256 tile a split of its own, then oz_combine_kernel). On chip saves 8
// bytes per output and chunk but feeds the tensor cores from L2 at twice the bytes per MMA of
// the wider tiles (measured: about 0.44 of the BF16 peak against 0.56 with partial sums on an
// 8100^3 product at o = 30, v = 270), and spreads only the output tiles over the SMs. So it
// runs where the partial sums weigh most against the MMA work, short sums: measured on the
// o = 10, 20 and 30 workloads, it wins for k up to 16 blocks of 64 (the ladder build over the
// auxiliary index, 10-20% faster) and loses beyond (the rings and the ladder contraction over
// o v and v^2), given at least one tile per SM.
bool oz_onchip(const Exec& ex, const GemmArgs& g, int kseg) {
  if (ex.emu_onchip >= 0) return ex.emu_onchip == 1;
  const double tiles128 = (double)g.batch * std::ceil(g.M / (double)TM) * std::ceil(g.N / (double)OZ_TN);
  return kseg <= 16 && tiles128 >= ex.sm_count;
}

void run_oz(const Exec& ex, const GemmArgs& g, const char* tag) {
  constexpr int TK = Elt<true>::TK;
  const int k_pad = (g.K + TK - 1) / TK * TK;
  const int kseg = k_pad / TK, kk = OZ_S * k_pad;
  const int nk = std::max(1, std::min(OZ_NK, ex.emu_chunk));
  const int nsplit = oz_splits(kseg, nk);
  CC_REQUIRE(k_pad < (1 << 24), CC_ERR_INVALID, "FP64-emulated contraction: sum longer than 2^24");
  const bool onchip = oz_onchip(ex, g, kseg);
  const int tn = onchip ? OZ_TN : TN;
  const int rowsA = (g.M + TM - 1) / TM * TM, rowsB = (g.N + tn - 1) / tn * tn;
  auto blocks_for_rows = [&](size_t rows) {
    return (int)std::max<size_t>(1, std::min<size_t>((rows + 7) / 8, (size_t)ex.sm_count * 16));
  };
  cudaEvent_t ev = nullptr;
  if (ex.timing(tag)) ex.mark_begin(&ev);
  DBuf<double> stA(ex.pool, ((size_t)g.batch * rowsA * kk * 2 + 7) / 8);
  DBuf<double> stB(ex.pool, ((size_t)g.batch * rowsB * kk * 2 + 7) / 8);
  DBuf<double> exA(ex.pool, ((size_t)g.batch * rowsA + 1) / 2), exB(ex.pool, ((size_t)g.batch * rowsB + 1) / 2);
  auto* fA = reinterpret_cast<__nv_bfloat16*>(stA.p);
  auto* fB = reinterpret_cast<__nv_bfloat16*>(stB.p);
  auto* eA = reinterpret_cast<unsigned*>(exA.p);
  auto* eB = reinterpret_cast<unsigned*>(exB.p);
  if (g.K <= 2048) {  // short rows: one warp per row, both passes and both operands in one kernel
    OzStagePair P;
    memset(&P, 0, sizeof(P));
    P.d[0] = OzStageDesc{g.A, g.am, g.ak, g.ab, g.M, g.batch, rowsA, 0, eA, fA};
    P.d[1] = OzStageDesc{g.B, g.bn, g.bk, g.bb, g.N, g.batch, rowsB, 1, eB, fB};
    P.row0[0] = 0;
    P.row0[1] = (long long)g.batch * rowsA;
    P.row0[2] = P.row0[1] + (long long)g.batch * rowsB;
    P.K = g.K;
    P.k_pad = k_pad;
    oz_stage_rows_kernel<<<blocks_for_rows((size_t)P.row0[2]), 256, 0, ex.stream>>>(P);
    ex.count();
  }
  auto stage = [&](const double* src, const CIdx& rix, const CIdx& kix, const CIdx& bix, int rows, int rows_pad,
                   int rev, unsigned* e, __nv_bfloat16* f) {
    if (g.K <= 2048) return;  // staged above
    CC_CUDA(cudaMemsetAsync(e, 0, (size_t)g.batch * rows_pad * sizeof(unsigned), ex.stream));
    const size_t pieces1 = (size_t)g.batch * rows * ((g.K + ROW_PIECE - 1) / ROW_PIECE);
    oz_rowexp_kernel<<<blocks_for_rows(pieces1), 256, 0, ex.stream>>>(src, rix, kix, bix, rows, g.K, g.batch,
                                                                        rows_pad, e);
    ex.count();
    const size_t pieces2 = (size_t)g.batch * rows_pad * ((k_pad + ROW_PIECE - 1) / ROW_PIECE);
    oz_digits_kernel<<<blocks_for_rows(pieces2), 256, 0, ex.stream>>>(src, rix, kix, bix, rows, g.K, g.batch,
                                                                        rows_pad, k_pad, rev, e, f);
    ex.count();
  };
  stage(g.A, g.am, g.ak, g.ab, g.M, rowsA, 0, eA, fA);
  stage(g.B, g.bn, g.bk, g.bb, g.N, rowsB, 1, eB, fB);
  CC_CUDA(cudaGetLastError());
  CUtensorMap mA = make_map(fA, kk, rowsA, g.batch, TM, true);
  CUtensorMap mB = make_map(fB, kk, rowsB, g.batch, tn, true);
  if (onchip) {
    OzArgs o{};
    o.M = g.M;
    o.N = g.N;
    o.num_m = rowsA / TM;
    o.num_n = rowsB / OZ_TN;
    o.batch = g.batch;
    o.m_fast = o.num_m <= o.num_n ? 1 : 0;
    const long long tiles = (long long)o.num_m * o.num_n * g.batch;
    CC_REQUIRE(tiles < (1LL << 31), CC_ERR_INVALID, "FP64-emulated contraction: too many tiles");
    o.tiles = (int)tiles;
    o.kseg = kseg;
    o.nk = nk;
    o.nsplit = nsplit;
    o.cm = g.cm;
    o.cn = g.cn;
    o.cb = g.cb;
    o.alpha = g.alpha;
    o.beta = g.beta;
    o.C = g.C;
    o.expA = eA;
    o.expB = eB;
    o.rowsA_pad = rowsA;
    o.rowsB_pad = rowsB;
    o.err = ex.dev_flag;
    o.wait_ns = ex.wait_ns;
    static std::atomic<uint64_t> attr_done{0};
    ensure_smem_attr(oz_gemm_kernel, attr_done, OZ_SMEM_BYTES);
    oz_gemm_kernel<<<(int)std::min<long long>(tiles, ex.sm_count), THREADS, OZ_SMEM_BYTES, ex.stream>>>(mA, mB, o);
    ex.count();
    CC_CUDA(cudaGetLastError());
    if (ev) ex.mark_end(tag, ev, 2.0 * g.M * (double)g.N * g.K * g.batch);
    return;
  }
  TcArgs a{};
  a.M = g.M;
  a.N = g.N;
  a.kblocks = kk / TK;
  a.num_m = rowsA / TM;
  a.num_n = rowsB / TN;
  a.batch = g.batch;
  a.m_fast = a.num_m <= a.num_n ? 1 : 0;
  a.splits = nsplit;
  a.kchunk = nk;
  a.oz_S = OZ_S;
  a.oz_kseg = kseg;
  a.oz_nk = nk;
  const long long tiles = (long long)a.num_m * a.num_n * g.batch * nsplit;
  CC_REQUIRE(tiles < (1LL << 31), CC_ERR_INVALID, "FP64-emulated contraction: too many tiles");
  a.tiles = (int)tiles;
  a.cm = g.cm;
  a.cn = g.cn;
  a.cb = g.cb;
  a.alpha = g.alpha;
  a.beta = g.beta;
  a.C = g.C;
  a.err = ex.dev_flag;
  a.wait_ns = ex.wait_ns;
  a.Cs = nullptr;
  const size_t np = (size_t)nsplit * g.batch * g.M * g.N;
  DBuf<double> part(ex.pool, (np + 1) / 2);
  a.part = reinterpret_cast<float*>(part.p);
  TcJob<true> job;
  job.mA = mA;
  job.mB = mB;
  job.a = a;
  TcJob<true>* one = &job;
  tc_launch_group<true, EPI_PART, 1, TN>(ex, &one, 1);
  const size_t rows = (size_t)g.batch * g.M;
  const int piece = rows * ((g.N + ROW_PIECE - 1) / ROW_PIECE) >= (size_t)ex.sm_count * 64 ? ROW_PIECE : 32;
  const size_t items = rows * ((g.N + piece - 1) / piece);
  const int rblocks = (int)std::max<size_t>(1, std::min<size_t>((items + 7) / 8, (size_t)ex.sm_count * 16));
  oz_combine_kernel<<<rblocks, 256, 0, ex.stream>>>(g, a.part, kseg, nk, eA, rowsA, eB, rowsB, piece);
  ex.count();
  CC_CUDA(cudaGetLastError());
  if (ev) ex.mark_end(tag, ev, 2.0 * g.M * (double)g.N * g.K * g.batch);
}

}  // namespace

void k_wait_selftest(const Exec& ex) {
  CC_REQUIRE(ex.dev_flag, CC_ERR_INVALID, "the wait self-test needs a device error flag");
  wait_selftest_kernel<<<1, 32, 0, ex.stream>>>(ex.dev_flag, ex.wait_ns);
  ex.count();
  CC_CUDA(cudaGetLastError());
}

void k_ladder_pm_stage(const Exec& ex, bool bf, int nseg, long long rows, int v, const float* W, void* Wp,
                       long long kpP, void* Wm, long long kpQ) {
  CC_REQUIRE(nseg == 1 || nseg == 3, CC_ERR_INVALID, "ladder split: one or three staging segments");
  const long long Pv = (long long)v * (v + 1) / 2, Qv = (long long)v * (v - 1) / 2;
  CC_REQUIRE(kpP >= Pv && kpP - Pv < 64 && (!Wm || (kpQ >= Qv && kpQ - Qv < 64)), CC_ERR_INVALID,
             "ladder split: k padding");
  const int nt = (v + 31) / 32;
  const long long items = rows * (long long)(nt * (nt + 1) / 2);
  if (items <= 0) return;
  const int blocks = (int)std::min<long long>(items, (long long)ex.sm_count * 8);
  if (bf)
    ladder_pm_stage_kernel<__nv_bfloat16><<<blocks, 256, 0, ex.stream>>>(
        rows, v, W, static_cast<__nv_bfloat16*>(Wp), kpP, static_cast<__nv_bfloat16*>(Wm), kpQ, nseg);
  else
    ladder_pm_stage_kernel<float><<<blocks, 256, 0, ex.stream>>>(rows, v, W, static_cast<float*>(Wp), kpP,
                                                                static_cast<float*>(Wm), kpQ, nseg);
  ex.count();
  CC_CUDA(cudaGetLastError());
}

void gemm_tc_group(const Exec& ex, cc_precision prec, const std::vector<GemmArgs>& gs, const char* tag) {
  CC_REQUIRE(prec == CC_MIXED_TF32 || prec == CC_MIXED_TF32X3 || prec == CC_MIXED_BF16X3, CC_ERR_INVALID,
             "grouped launches run the single-precision tensor-core kinds");
  CC_REQUIRE(ex.dev_flag, CC_ERR_INVALID, "tensor-core contraction needs a device error flag");
  std::vector<GemmArgs> todo;
  for (const auto& g : gs) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) continue;
    if (g.K <= 0) {
      gemm_tc(ex, prec, g);  // C = beta C
      continue;
    }
    todo.push_back(g);
  }
  if (todo.empty()) return;
  if (prec == CC_MIXED_BF16X3) run_tc_group<true>(ex, prec, todo, tag);
  else run_tc_group<false>(ex, prec, todo, tag);
}

void gemm_tc(const Exec& ex, cc_precision prec, const GemmArgs& g, const char* tag) {
  CC_REQUIRE(prec == CC_MIXED_TF32 || prec == CC_MIXED_TF32X3 || prec == CC_MIXED_BF16X3 || prec == CC_FP64_EMU,
             CC_ERR_INVALID, "tensor-core precision not available");
  CC_REQUIRE(ex.dev_flag, CC_ERR_INVALID, "tensor-core contraction needs a device error flag");
  if (g.K <= 0) {
    int blocks = (int)std::min<size_t>(((size_t)g.batch * g.M * g.N + 255) / 256, (size_t)ex.sm_count * 8);
    scale_c_kernel<<<std::max(blocks, 1), 256, 0, ex.stream>>>(g);
    ex.count();
    CC_CUDA(cudaGetLastError());
    return;
  }
  CC_REQUIRE((long long)((g.M + TM - 1) / TM) * ((g.N + TN - 1) / TN) * g.batch < (1LL << 31), CC_ERR_INVALID,
             "tensor-core contraction: too many tiles");
  if (prec == CC_FP64_EMU) {
    CC_REQUIRE(!g.so && !g.sb, CC_ERR_INVALID, "staged operands need a single-precision tensor-core path");
    run_oz(ex, g, tag);
  } else if (prec == CC_MIXED_BF16X3) {
    run_tc<true>(ex, prec, g, tag);
  } else {
    run_tc<false>(ex, prec, g, tag);
  }
}

}  // namespace ccpnk
