// Bandwidth-bound kernels: vector updates, permutation-adds, deterministic reductions.
//
// Grids are sized to a multiple of the SM count (grid-stride loops), loads are coalesced
// along the innermost index, and every reduction is two-pass (per-block partials, then one
// block) with warp-shuffle trees, so results do not depend on scheduling.
#include "common.h"

namespace ccpnk {
namespace {

constexpr int TPB = 256;

int grid_for(const Exec& ex, size_t n, int per_sm = 8) {
  size_t want = (n + TPB - 1) / TPB;
  size_t cap = (size_t)ex.sm_count * per_sm;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

__global__ void axpby_kernel(size_t n, double a, const double* __restrict__ x, double b,
                             double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

__global__ void scale_kernel(size_t n, double a, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * y[i];
}

__global__ void fill_kernel(size_t n, double val, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = val;
}

__global__ void copy_kernel(size_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = x[i];
}

__global__ void to_f32_kernel(size_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// out[i][j][a][b] = beta*out + X[i][j][a][b] + X[j][i][b][a]
__global__ void sym_add_kernel(int o, int v, const double* __restrict__ X, double* __restrict__ out,
                               double beta) {
  size_t n = (size_t)o * o * v * v;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(e % v);
    size_t r = e / v;
    int a = (int)(r % v);
    r /= v;
    int j = (int)(r % o);
    int i = (int)(r / o);
    double s = X[e] + X[(((size_t)j * o + i) * v + b) * v + a];
    out[e] = (beta == 0.0) ? s : fma(beta, out[e], s);
  }
}

// R[i][j][a][b] += L[i][j][a][b] where b >= start of a's block of size blk, else L[j][i][b][a]
__global__ void ladder_mirror_add_kernel(int o, int v, int blk, const double* __restrict__ L, double* __restrict__ R) {
  size_t n = (size_t)o * o * v * v;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(e % v);
    size_t r = e / v;
    int a = (int)(r % v);
    r /= v;
    int j = (int)(r % o), i = (int)(r / o);
    const int bs = (a / blk) * blk;
    R[e] += (b >= bs) ? L[e] : L[(((size_t)j * o + i) * v + b) * v + a];
  }
}

// T+[(i<=j)][(c<=d)] = (T_ij^cd + T_ij^dc) / 2 (T_ij^cc on the diagonal), T-[(i<j)][(c<d)] =
// (T_ij^cd - T_ij^dc) / 2, for T with T_ij^cd = T_ji^dc
__global__ void ladder_pm_T_kernel(int o, int v, const double* __restrict__ T, double* __restrict__ Tp,
                                   double* __restrict__ Tm) {
  const size_t n = (size_t)o * o * v * v;
  const size_t Pv = (size_t)v * (v + 1) / 2, Qv = (size_t)v * (v - 1) / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(e % v);
    size_t r = e / v;
    const int c = (int)(r % v);
    r /= v;
    const int j = (int)(r % o), i = (int)(r / o);
    if (i > j || c > d) continue;
    const double x = T[e], y = T[(((size_t)i * o + j) * v + d) * v + c];
    Tp[pair_le(i, j, o) * Pv + pair_le(c, d, v)] = c < d ? 0.5 * (x + y) : x;
    if (i < j && c < d) Tm[pair_lt(i, j, o) * Qv + pair_lt(c, d, v)] = 0.5 * (x - y);
  }
}

// W+[r][(c<=d)] = W_r^cd + W_r^dc (W_r^cc on the diagonal), W-[r][(c<d)] = W_r^cd - W_r^dc
__global__ void ladder_pm_W_kernel(size_t rows, int v, const double* __restrict__ W, double* __restrict__ Wp,
                                   double* __restrict__ Wm) {
  const size_t vv = (size_t)v * v, n = rows * vv;
  const size_t Pv = (size_t)v * (v + 1) / 2, Qv = (size_t)v * (v - 1) / 2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(e % v);
    const size_t q = e / v;
    const int c = (int)(q % v);
    const size_t r = q / v;
    if (c > d) continue;
    const double x = W[e], y = W[r * vv + (size_t)d * v + c];
    Wp[r * Pv + pair_le(c, d, v)] = c < d ? x + y : x;
    if (c < d) Wm[r * Qv + pair_lt(c, d, v)] = x - y;
  }
}

// L[i][j][a0 + a][a0 + b] = L+[(i<=j)][n] + L-[(i<j)][n] for i <= j and L+[(j<=i)][n] -
// L-[(j<i)][n] for i > j, n = a bl + b (L+ symmetric and L- antisymmetric in i, j); the rows of
// L+ and L- are ld apart
__global__ void ladder_pm_unpack_kernel(int o, int v, int a0, int al, int bl, size_t ld, const double* __restrict__ Lp,
                                        const double* __restrict__ Lm, double* __restrict__ L) {
  const size_t nb = (size_t)al * bl, n = (size_t)o * o * nb;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t nn = e % nb, ij = e / nb;
    const int j = (int)(ij % o), i = (int)(ij / o);
    const int a = (int)(nn / bl), b = (int)(nn % bl);
    double val;
    if (i <= j) val = Lp[pair_le(i, j, o) * ld + nn] + (i < j ? Lm[pair_lt(i, j, o) * ld + nn] : 0.0);
    else val = Lp[pair_le(j, i, o) * ld + nn] - Lm[pair_lt(j, i, o) * ld + nn];
    L[(((size_t)i * o + j) * v + a0 + a) * v + a0 + b] = val;
  }
}

// u[i][j][a][b] = 2 t[i][j][a][b] - t[j][i][a][b]
__global__ void make_u_kernel(int o, int v, const double* __restrict__ t, double* __restrict__ u) {
  size_t n = (size_t)o * o * v * v;
  size_t vv = (size_t)v * v;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    size_t ab = e % vv;
    size_t ij = e / vv;
    int j = (int)(ij % o), i = (int)(ij / o);
    u[e] = 2.0 * t[e] - t[((size_t)j * o + i) * vv + ab];
  }
}

// L[p][q][r][s] = 2 g[p][q][r][s] - g[p][s][r][q], g an (o v o v) block
__global__ void make_L_kernel(int o, int v, const double* __restrict__ g, double* __restrict__ L) {
  size_t n = (size_t)o * v * o * v;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    int s = (int)(e % v);
    size_t r1 = e / v;
    int r = (int)(r1 % o);
    r1 /= o;
    int q = (int)(r1 % v);
    int p = (int)(r1 / v);
    L[e] = 2.0 * g[e] - g[(((size_t)p * v + s) * o + r) * v + q];
  }
}

__global__ void trace_batched_kernel(int P, int m, const double* __restrict__ A, double* __restrict__ g) {
  int Pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (Pi >= P) return;
  double s = 0.0;
  for (int k = 0; k < m; ++k) s += A[((size_t)Pi * m + k) * m + k];
  g[Pi] = s;
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  return x;
}

// block-level sum of x; valid in thread 0
__device__ __forceinline__ double block_sum(double x) {
  __shared__ double sh[32];
  x = warp_sum(x);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  x = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) x = warp_sum(x);
  __syncthreads();
  return x;
}

__global__ void dot_partial_kernel(size_t n, const double* __restrict__ x, const double* __restrict__ y,
                                   double* __restrict__ part) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// final reduce of nparts partials for each of m rows: out[r] = sum_b part[r * nparts + b]
__global__ void final_reduce_kernel(int m, int nparts, const double* __restrict__ part, double* __restrict__ out) {
  int r = blockIdx.x;
  if (r >= m) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(size_t)r * nparts + b];
  s = block_sum(s);
  if (threadIdx.x == 0) out[r] = s;
}

// partial dots of w with m rows of Q: part[r][blockIdx.x]
__global__ void multi_dot_partial_kernel(int m, size_t n, const double* __restrict__ Q, size_t ldq,
                                         const double* __restrict__ w, double* __restrict__ part) {
  constexpr int RB = 8;  // rows per pass share each load of w
  for (int r0 = 0; r0 < m; r0 += RB) {
    double s[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) s[q] = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      double wi = w[i];
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (r0 + q < m) s[q] = fma(Q[(size_t)(r0 + q) * ldq + i], wi, s[q]);
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      double t = block_sum(s[q]);
      if (threadIdx.x == 0 && r0 + q < m) part[(size_t)(r0 + q) * gridDim.x + blockIdx.x] = t;
    }
  }
}

__global__ void multi_axpy_kernel(int m, size_t n, const double* __restrict__ Q, size_t ldq,
                                  const double* __restrict__ h, double* __restrict__ w) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int r = 0; r < m; ++r) acc = fma(-h[r], Q[(size_t)r * ldq + i], acc);
    w[i] = acc;
  }
}

// E partials: sum over (i,a,j,b) of (2 g_iajb - g_ibja)(t2_ijab + t1_ia t1_jb), g stored [i][a][j][b]
__global__ void energy_partial_kernel(int o, int v, const double* __restrict__ g, const double* __restrict__ t1,
                                      const double* __restrict__ t2, const double* __restrict__ fov, int ldf,
                                      double* __restrict__ part) {
  size_t n = (size_t)o * v * o * v;
  double s = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(e % v);
    size_t r = e / v;
    int j = (int)(r % o);
    r /= o;
    int a = (int)(r % v);
    int i = (int)(r / v);
    double gx = g[(((size_t)i * v + b) * o + j) * v + a];
    double tau = t2[(((size_t)i * o + j) * v + a) * v + b] + t1[(size_t)i * v + a] * t1[(size_t)j * v + b];
    s = fma(2.0 * g[e] - gx, tau, s);
  }
  // 2 sum f_ia t1_ia
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)o * v; e += (size_t)gridDim.x * blockDim.x) {
    int a = (int)(e % v), i = (int)(e / v);
    s = fma(2.0 * fov[(size_t)i * ldf + a], t1[e], s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void denom_divide_kernel(int o, int v, const double* __restrict__ fd, double shift,
                                    const double* __restrict__ x1, const double* __restrict__ x2,
                                    double* __restrict__ y1, double* __restrict__ y2, double scale) {
  size_t n2 = (size_t)o * o * v * v, n1 = (size_t)o * v;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n1 + n2; e += (size_t)gridDim.x * blockDim.x) {
    if (e < n1) {
      int a = (int)(e % v), i = (int)(e / v);
      y1[e] = scale * x1[e] / (fd[o + a] - fd[i] + shift);
    } else {
      size_t q = e - n1;
      int b = (int)(q % v);
      size_t r = q / v;
      int a = (int)(r % v);
      r /= v;
      int j = (int)(r % o), i = (int)(r / o);
      y2[q] = scale * x2[q] / (fd[o + a] + fd[o + b] - fd[i] - fd[j] + shift);
    }
  }
}

__global__ void copy2d_kernel(int rows, int cols, const double* __restrict__ s, long long lds,
                              double* __restrict__ d, long long ldd) {
  size_t n = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(e % cols), r = (int)(e / cols);
    d[(size_t)r * ldd + c] = s[(size_t)r * lds + c];
  }
}

// out[b][c][r] = in[b][r][c] through a 32 x 33 shared tile (coalesced on both sides)
__global__ void transpose_kernel(int rows, int cols, const double* __restrict__ in, long long in_bs,
                                 long long in_ld, double* __restrict__ out, long long out_bs, long long out_ld) {
  __shared__ double tile[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const double* src = in + (size_t)b * in_bs;
  double* dst = out + (size_t)b * out_bs;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = src[(size_t)r * in_ld + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[(size_t)c * out_ld + r] = tile[threadIdx.x][k];
  }
}

__global__ void copy3d_kernel(int batch, int rows, int cols, const double* __restrict__ s, long long sbs,
                              long long sld, double* __restrict__ d, long long dbs, long long dld) {
  size_t n = (size_t)batch * rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(e % cols);
    size_t q = e / cols;
    int r = (int)(q % rows);
    size_t b = q / rows;
    d[b * dbs + (size_t)r * dld + c] = s[b * sbs + (size_t)r * sld + c];
  }
}

__global__ void asym_partial_kernel(int P, int n, const double* __restrict__ B, double* __restrict__ part) {
  size_t tot = (size_t)P * n * n;
  double mx = 0.0, mb = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    int q = (int)(e % n);
    size_t r = e / n;
    int p = (int)(r % n);
    size_t Pi = r / n;
    double x = B[e];
    double y = B[(Pi * n + q) * n + p];
    mx = fmax(mx, fabs(x - y));
    mb = fmax(mb, fabs(x));
    if (!isfinite(x)) mb = INFINITY;  // fmax drops NaN operands: report a NaN as an infinite entry
  }
  __shared__ double s1[TPB], s2[TPB];
  s1[threadIdx.x] = mx;
  s2[threadIdx.x] = mb;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      s1[threadIdx.x] = fmax(s1[threadIdx.x], s1[threadIdx.x + st]);
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1[0];
    part[2 * blockIdx.x + 1] = s2[0];
  }
}

__global__ void asym_final_kernel(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) {
    a = fmax(a, part[2 * i]);
    b = fmax(b, part[2 * i + 1]);
  }
  out[0] = a;
  out[1] = b;
}

}  // namespace

#define LAUNCH_CHECK() \
  do {                 \
    ex.count();        \
    CC_CUDA(cudaGetLastError()); \
  } while (0)

void k_axpby(const Exec& ex, size_t n, double a, const double* x, double b, double* y) {
  if (!n) return;
  axpby_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(n, a, x, b, y);
  LAUNCH_CHECK();
}
void k_scale(const Exec& ex, size_t n, double a, double* y) {
  if (!n) return;
  scale_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(n, a, y);
  LAUNCH_CHECK();
}
void k_fill(const Exec& ex, size_t n, double val, double* y) {
  if (!n) return;
  fill_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(n, val, y);
  LAUNCH_CHECK();
}
void k_copy(const Exec& ex, size_t n, const double* x, double* y) {
  if (!n) return;
  copy_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(n, x, y);
  LAUNCH_CHECK();
}
void k_to_f32(const Exec& ex, size_t n, const double* x, float* y) {
  if (!n) return;
  to_f32_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(n, x, y);
  LAUNCH_CHECK();
}
void k_sym_add(const Exec& ex, int o, int v, const double* X, double* out, double beta) {
  size_t n = (size_t)o * o * v * v;
  if (!n) return;
  sym_add_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, X, out, beta);
  LAUNCH_CHECK();
}
void k_ladder_mirror_add(const Exec& ex, int o, int v, int blk, const double* L, double* R) {
  size_t n = (size_t)o * o * v * v;
  if (!n) return;
  ladder_mirror_add_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, blk, L, R);
  LAUNCH_CHECK();
}
void k_ladder_pm_T(const Exec& ex, int o, int v, const double* T, double* Tp, double* Tm) {
  const size_t n = (size_t)o * o * v * v;
  if (!n) return;
  ladder_pm_T_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, T, Tp, Tm);
  LAUNCH_CHECK();
}
void k_ladder_pm_W(const Exec& ex, size_t rows, int v, const double* W, double* Wp, double* Wm) {
  const size_t n = rows * v * v;
  if (!n) return;
  ladder_pm_W_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(rows, v, W, Wp, Wm);
  LAUNCH_CHECK();
}
void k_ladder_pm_unpack(const Exec& ex, int o, int v, int a0, int al, int bl, const double* Lp, const double* Lm,
                        double* L, size_t ld) {
  const size_t n = (size_t)o * o * al * bl;
  if (!n) return;
  ladder_pm_unpack_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, a0, al, bl, ld ? ld : (size_t)al * bl, Lp, Lm,
                                                                   L);
  LAUNCH_CHECK();
}
void k_make_u(const Exec& ex, int o, int v, const double* t, double* u) {
  size_t n = (size_t)o * o * v * v;
  if (!n) return;
  make_u_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, t, u);
  LAUNCH_CHECK();
}
void k_make_L_ovov(const Exec& ex, int o, int v, const double* g, double* L) {
  size_t n = (size_t)o * o * v * v;
  if (!n) return;
  make_L_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, g, L);
  LAUNCH_CHECK();
}
void k_trace_batched(const Exec& ex, int P, int m, const double* A, double* gamma) {
  if (P <= 0) return;
  trace_batched_kernel<<<(P + TPB - 1) / TPB, TPB, 0, ex.stream>>>(P, m, A, gamma);
  LAUNCH_CHECK();
}
void k_dot(const Exec& ex, size_t n, const double* x, const double* y, double* out, double* scratch) {
  int nb = grid_for(ex, n, 4);
  dot_partial_kernel<<<nb, TPB, 0, ex.stream>>>(n, x, y, scratch);
  LAUNCH_CHECK();
  final_reduce_kernel<<<1, TPB, 0, ex.stream>>>(1, nb, scratch, out);
  LAUNCH_CHECK();
}
void k_multi_dot(const Exec& ex, int m, size_t n, const double* Q, size_t ldq, const double* w, double* out,
                 double* scratch) {
  if (m <= 0) return;
  int nb = grid_for(ex, n, 4);
  multi_dot_partial_kernel<<<nb, TPB, 0, ex.stream>>>(m, n, Q, ldq, w, scratch);
  LAUNCH_CHECK();
  final_reduce_kernel<<<m, TPB, 0, ex.stream>>>(m, nb, scratch, out);
  LAUNCH_CHECK();
}
void k_multi_axpy(const Exec& ex, int m, size_t n, const double* Q, size_t ldq, const double* h, double* w) {
  if (m <= 0 || !n) return;
  multi_axpy_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(m, n, Q, ldq, h, w);
  LAUNCH_CHECK();
}
void k_energy(const Exec& ex, int o, int v, const double* govov, const double* t1, const double* t2,
              const double* fov, int ldf, double* out, double* scratch) {
  size_t n = (size_t)o * o * v * v;
  int nb = grid_for(ex, n, 4);
  energy_partial_kernel<<<nb, TPB, 0, ex.stream>>>(o, v, govov, t1, t2, fov, ldf, scratch);
  LAUNCH_CHECK();
  final_reduce_kernel<<<1, TPB, 0, ex.stream>>>(1, nb, scratch, out);
  LAUNCH_CHECK();
}
int k_energy_partials(const Exec& ex, int o, int v) { return grid_for(ex, (size_t)o * o * v * v, 4); }
void k_denom_divide(const Exec& ex, int o, int v, const double* fdiag, double shift, const double* x1,
                    const double* x2, double* y1, double* y2, double scale) {
  size_t n = (size_t)o * v + (size_t)o * o * v * v;
  denom_divide_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, fdiag, shift, x1, x2, y1, y2, scale);
  LAUNCH_CHECK();
}
__global__ void ovov_to_oovv_kernel(int o, int v, const double* __restrict__ g, double* __restrict__ out, double scale) {
  const size_t n = (size_t)o * o * v * v;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e % v);
    size_t q = e / v;
    const int a = (int)(q % v);
    q /= v;
    const int j = (int)(q % o), i = (int)(q / o);
    out[e] = scale * g[(((size_t)i * v + a) * o + j) * v + b];
  }
}
void k_ovov_to_oovv(const Exec& ex, int o, int v, const double* g, double* out, double scale) {
  const size_t n = (size_t)o * o * v * v;
  if (!n) return;
  ovov_to_oovv_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(o, v, g, out, scale);
  LAUNCH_CHECK();
}
void k_copy2d(const Exec& ex, int rows, int cols, const double* src, long long lds, double* dst, long long ldd) {
  size_t n = (size_t)rows * cols;
  if (!n) return;
  copy2d_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(rows, cols, src, lds, dst, ldd);
  LAUNCH_CHECK();
}
void k_transpose(const Exec& ex, int batch, int rows, int cols, const double* in, long long in_bs,
                 long long in_ld, double* out, long long out_bs, long long out_ld) {
  if (batch <= 0 || rows <= 0 || cols <= 0) return;
  CC_REQUIRE(batch <= 65535, CC_ERR_INVALID, "transpose: batch too large");
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
  transpose_kernel<<<grid, dim3(32, 8), 0, ex.stream>>>(rows, cols, in, in_bs, in_ld, out, out_bs, out_ld);
  LAUNCH_CHECK();
}
void k_copy3d(const Exec& ex, int batch, int rows, int cols, const double* src, long long sbs, long long sld,
              double* dst, long long dbs, long long dld) {
  size_t n = (size_t)batch * rows * cols;
  if (!n) return;
  copy3d_kernel<<<grid_for(ex, n), TPB, 0, ex.stream>>>(batch, rows, cols, src, sbs, sld, dst, dbs, dld);
  LAUNCH_CHECK();
}
// out[0] = max |B[P][p][q] - B[P][q][p]|, out[1] = max |B| (infinite if any entry is not finite)
void k_asym(const Exec& ex, int P, int n, const double* B, double* out, double* scratch) {
  size_t tot = (size_t)P * n * n;
  int nb = grid_for(ex, tot, 2);
  asym_partial_kernel<<<nb, TPB, 0, ex.stream>>>(P, n, B, scratch);
  LAUNCH_CHECK();
  asym_final_kernel<<<1, 32, 0, ex.stream>>>(nb, scratch, out);
  LAUNCH_CHECK();
}

}  // namespace ccpnk
