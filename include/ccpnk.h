/*
 * ccpnk.h -- C ABI of the B300 closed-shell CCSD Newton-Krylov library (libccpnk.so).
 *
 * The problem (paper Sec. "Theory"): find amplitudes t = (t1, t2) with
 *   r_mu(t) = <Phi_mu| e^{-T} H e^{T} |Phi_0> = 0  for all singles and doubles mu   (Eq. CC_ampl)
 * and report E(t) = <Phi_0| e^{-T} H e^{T} |Phi_0> - E_ref                         (Eq. CC_energy).
 * The paper works at the CCD level with 4-index integrals; this library solves
 * closed-shell CCSD with density-fitted integrals (pq|rs) = sum_P B[P][p][q] B[P][r][s].
 *
 * Layouts (all row-major, FP64 on every precision path):
 *   fock  n x n (n = o + v), occupied orbitals first; it is the Fock matrix of the
 *         closed-shell reference, so the one-electron part is h = f - sum_k [2 (pq|kk) - (pk|kq)].
 *   B     naux x n x n, B[P][p][q] == B[P][q][p] (checked to 1e-12 relative at cc_sys_create).
 *   t1    o x v,          t1[i][a]       = t_i^a
 *   t2    o x o x v x v,  t2[i][j][a][b] = t_ij^ab, with t_ij^ab = t_ji^ba.
 *   r1/r2 same layouts as t1/t2: r1 is the alpha-alpha singles projection and r2
 *         the alpha-beta doubles projection of e^{-T} H e^{T}|Phi_0>.
 *   ||R|| is the Euclidean norm over the concatenation of r1 and r2.
 *
 * Memory: every amplitude/residual pointer may be host memory or device memory of the
 * context's device; the library asks the CUDA runtime which it is. The caller owns
 * every pointer it passes; the library never frees caller memory. cc_sys_create copies
 * fock and B into device memory owned by the cc_sys handle.
 *
 * Streams: all device work of a context runs on the context's stream (the one passed to
 * cc_ctx_create, or one the context creates). Calls return after that work is complete,
 * except where stated. A context must not be used from two threads at once.
 *
 * Errors: every call returns CC_OK (0) or a negative status; cc_last_error() gives a
 * one-line description of the last failure of that context.
 */
#ifndef CCPNK_H
#define CCPNK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_OK 0
#define CC_PENDING 1             /* cc_serve_poll: the request is still running */
#define CC_ERR_INVALID (-1)      /* bad argument: NULL, o < 1, v < 1, naux < 1, B not symmetric */
#define CC_ERR_OOM (-2)          /* device memory beyond the context's budget, or not admissible */
#define CC_ERR_NOT_CONVERGED (-3) /* cc_solve hit its iteration cap; the report is filled */
#define CC_ERR_DIVERGED (-4)     /* non-finite or exploding residual */
#define CC_ERR_CUDA (-5)         /* a CUDA runtime error */
#define CC_ERR_TIMEOUT (-6)      /* a bounded device-side wait gave up */
#define CC_ERR_CANCELLED (-7)    /* cc_serve_cancel stopped the request; the report is filled */

typedef enum {
  CC_FP64 = 0,          /* every contraction in FP64 (FMA pipe) */
  CC_MIXED_TF32 = 1,    /* contractions of JVPs / inner solves on tcgen05 TF32, FP32 accumulate */
  CC_MIXED_BF16X3 = 2,  /* 3-pass BF16 split: x = hi + lo in BF16, a b ~ hi hi + hi lo + lo hi on
                           tcgen05 kind::f16, FP32 accumulate (about 16 significant bits) */
  CC_MIXED_TF32X3 = 3,  /* 3-pass TF32 split: x = hi + lo, a b ~ hi hi + hi lo + lo hi on tcgen05,
                           FP32 accumulate (about FP32 accuracy at a third of the TF32 rate).
                           In the three single-precision tensor-core kinds, contractions too thin
                           for the tensor cores' tiles run on the FP32 pipe (FP32 products, at
                           most 512 terms per FP32 sum, FP64 split-k and output) */
  CC_DF64 = 4,          /* double-float: FP64 operands as FP32 pairs on the FP32 pipe (error-free
                           products, two-sum accumulation; about 48 significant bits), for the
                           residual when FP64 FMA throughput is the limit */
  CC_FP64_EMU = 5       /* FP64-accurate contractions on the tensor cores: each FP64 row split into
                           9 BF16 slices of 6-bit integer digits under a per-row exponent (Ozaki's
                           error-free splitting), slice products summed exactly in FP32 chunks on
                           tcgen05 kind::f16 and combined in 64-bit integer fixed point; every
                           element rounded to nearest at 54 bits below its row's largest, so the
                           representation errors carry no sign bias. Thin contractions stay on the
                           FP64 pipe */
} cc_precision;

typedef enum {
  CC_FP_DIIS = 0,  /* fixed point with the diagonal-Fock denominator, level shift, DIIS (Eq. mo_fixed-point_update, App. D) */
  CC_NK = 1,       /* Jacobian-free Newton-Krylov, no preconditioner (Table 1) */
  CC_PNK = 2,      /* Newton-Krylov left-preconditioned by A_F (Eq. Preconditioner, Algorithm 1) */
  CC_INK = 3       /* inexact Newton: step = A_F^{-1}(-r) (Eq. inexact_newton_update) */
} cc_method;

typedef struct cc_ctx cc_ctx;
typedef struct cc_sys cc_sys;
typedef struct cc_server cc_server;

typedef struct {
  cc_method method;
  cc_precision prec;     /* precision of JVPs and of the inner A_F solves; the outer residual,
                            energy, Newton update and Arnoldi orthogonalisation are always FP64 */
  double tol;            /* stop when ||R|| < tol (default 1e-8) */
  int max_outer;         /* Newton steps (NK/PNK/INK) or iterations (FP+DIIS); default 100 */
  int m_max;             /* outer Arnoldi cap per Newton step (default 30) */
  double gamma, alpha;   /* Eisenstat-Walker forcing (App. F.1): 0.9, 1.5 */
  double eta_max;        /* forcing cap and eta_0 (default 0.9) */
  double level_shift;    /* FP+DIIS denominator shift, App. D (default 0) */
  int diis_size;         /* FP+DIIS subspace size (default 8; 0 disables DIIS) */
  int jvp_fd;            /* 1: forward finite-difference JVP (Eq. jacobian_vector_product_via_finite_difference) */
  double inner_rtol;     /* inner A_F GMRES relative tolerance (default 1e-12 FP64, 1e-8 TF32X3, 1e-6 TF32) */
  int inner_max;         /* inner GMRES cap (default 50) */
  int af_direct;         /* 1: invert A_F in the Fock eigenbasis instead of by inner GMRES */
  int verbose;           /* 1: one line per outer iteration on stderr */
  int ccd;               /* 1: CCD, the paper's level of theory (Sec. Numerics): t1 = 0 throughout and
                            only the doubles projections are solved */
  double max_seconds;    /* > 0: stop with CC_ERR_NOT_CONVERGED once a solve has run this long
                            (checked between outer iterations) */
  int outer_prec;        /* precision of the outer residual: CC_FP64 (default), CC_DF64 or CC_FP64_EMU */
} cc_solve_opts;

typedef struct {
  double energy;         /* correlation energy at the returned amplitudes */
  double res_norm;       /* FP64 ||R|| at the returned amplitudes */
  int newton_iters;      /* Newton steps (or FP iterations) taken */
  int residual_evals;    /* FP64 residual evaluations (the paper's cost metric) */
  int jvps;              /* Jacobian-vector products */
  int af_applies;        /* applications of A_F (inside inner solves) or of A_F^{-1} (direct) */
  int krylov_iters;      /* total outer Arnoldi steps */
  int status;            /* CC_OK, CC_ERR_NOT_CONVERGED, CC_ERR_DIVERGED or CC_ERR_CANCELLED */
  double seconds;        /* wall time of the solve */
} cc_report;

/* Fills opts with the defaults listed above for the given method and precision. */
void cc_solve_opts_default(cc_solve_opts* opts, cc_method method, cc_precision prec);

/* Context on one device. mem_budget: bytes of device memory the context may hold
 * (0 = no limit beyond the device). stream: a cudaStream_t, or NULL to create one. */
int cc_ctx_create(cc_ctx** ctx, int device, size_t mem_budget, void* stream);
void cc_ctx_destroy(cc_ctx* ctx);
const char* cc_last_error(const cc_ctx* ctx);
/* Options of a context (tuning and testing knobs of this library; the paper has no counterpart).
 * CC_OPT_STAGE_CACHE_BYTES: bytes the JVPs of a solve may keep in tensor-core staged copies of
 *   operands that stay fixed between two residual evaluations (default: room for about 32 copies
 *   of the largest tensors, at most 1 GiB or an eighth of the budget; 0 turns the cache off;
 *   -1 restores the default). Results do not depend on it, only the time does.
 * CC_OPT_WAIT_LIMIT_NS: bound, in nanoseconds of the GPU's global timer, on every wait of a
 *   device-side pipeline (default 4e9, at least 1e5); a wait that gives up makes the call
 *   return CC_ERR_TIMEOUT and leaves the context usable.
 * CC_OPT_GRAPHS: 1 (default) replays the JVPs of an NK or PNK solve from CUDA graphs of the
 *   tangent program (captured during the solve, released when it returns; the kernel timer, when
 *   on, keeps them eager); 0 launches every kernel. Results are the same bits either way.
 * CC_OPT_EMU_CHUNK: k blocks of 64 products that one exact FP32 chunk of CC_FP64_EMU sums
 *   (1..64, default 64: a chunk sum stays within 2^24, where FP32 still holds every integer
 *   exactly). Results do not depend on it (the chunk sums are exact); fewer, longer chunks move
 *   fewer partial sums.
 * CC_OPT_LADDER_PACK: the (c, d) split of the tensor-core particle-particle ladder: the slab
 *   (ac|bd) goes through one more pass that forms its parts symmetric and antisymmetric under
 *   c <-> d, and the contraction with the amplitudes runs over pairs i <= j, c <= d (half the
 *   MMA work for an extra read and write of the slab). -1 (default) decides per shape by a time
 *   model, 0 never, 1 always. Results agree within the precision's bound either way.
 * CC_OPT_EMU_ONCHIP: how CC_FP64_EMU sums its slice products: 1 on chip (each 128 x 128 tile of
 *   C runs all its slice products on one SM and adds the exact chunk sums in registers), 0
 *   through FP32 partial sums in device memory and a combine pass (the slice products of one
 *   tile spread over SMs), -1 (default) by a time model of the shape. The bits of the result
 *   are the same either way.
 * Returns CC_OK or CC_ERR_INVALID (unknown option, value out of range). */
#define CC_OPT_STAGE_CACHE_BYTES 1
#define CC_OPT_WAIT_LIMIT_NS 2
#define CC_OPT_GRAPHS 3
#define CC_OPT_EMU_CHUNK 4
#define CC_OPT_LADDER_PACK 5
#define CC_OPT_EMU_ONCHIP 6
int cc_ctx_set_option(cc_ctx* ctx, int option, long long value);
/* Self-test of the bounded device waits: runs one kernel whose wait on an mbarrier that nothing
 * arrives at gives up after CC_OPT_WAIT_LIMIT_NS, so the call returns CC_ERR_TIMEOUT; the
 * kernel returns normally and the context stays usable. A diagnostic of this library. */
int cc_ctx_selftest_wait(cc_ctx* ctx);
/* Measured FMA throughput of the device (a diagnostic of this library): fp64 = 1 the FP64 pipe,
 * 0 the FP32 pipe, in TFLOP/s (2 flops per FMA) from the fastest of three timed launches of a
 * kernel running eight independent FMA chains per thread on every SM. It is the measured
 * counterpart of the FMA-pipe peaks the rooflines divide by. Allocates and frees its own
 * output buffer. Returns CC_OK, CC_ERR_INVALID or CC_ERR_CUDA. */
int cc_probe_fma_rate(int device, int fp64, double* tflops);
/* Device bytes currently held by the context's pools. */
size_t cc_ctx_device_bytes(const cc_ctx* ctx);
/* Number of kernels the context has run since it was created (a replayed CUDA graph counts
 * its kernel nodes). */
uint64_t cc_ctx_launches(const cc_ctx* ctx);
/* Number of host launch calls the context has made: one per kernel launch and one per CUDA
 * graph replay. */
uint64_t cc_ctx_launch_calls(const cc_ctx* ctx);
/* Kernel timer (tracing): enable != 0 clears the records and brackets GEMM launches with CUDA
 * events on the context's stream; enable = 0 turns it off. enable = 1 times the two GEMMs of
 * the particle-particle ladder, tagged "ladder_build.<p>" and "ladder_contract.<p>" (<p> =
 * fp64, df64, tf32 or bf16); enable = 2 also times every other contraction under its index
 * labels and the precision asked for, e.g. "kc*Pkd>Pcd.f64" (A labels * B labels > C labels;
 * .f64, .df64 or .tc, the last also when a thin contraction ran on the FP64 kernel). The time
 * of a tensor-core launch covers the GEMM and its split-k reduce, not the operand staging. */
int cc_ctx_profile(cc_ctx* ctx, int enable);
/* Launch count, summed event time (ms) and summed algorithmic flops of one tag since the
 * last cc_ctx_profile(ctx, 1). Waits for the recorded launches to finish. */
int cc_ctx_profile_get(cc_ctx* ctx, const char* tag, uint64_t* launches, double* total_ms, double* flops);
/* Every tag recorded since the last cc_ctx_profile(ctx, 1), one line each as
 * "tag<TAB>launches<TAB>total_ms<TAB>flops<LF>", written to buf (cap bytes, NUL-terminated,
 * truncated at a line boundary). *needed (may be NULL) receives the full length + 1. A
 * diagnostic of this library: the paper has no counterpart. */
int cc_ctx_profile_list(cc_ctx* ctx, char* buf, size_t cap, size_t* needed);

/* A problem resident on the device: copies fock (n x n) and B (naux x n x n), host or device.
 * Its device memory comes from the context's pool, so every cc_sys of a context must be
 * destroyed before the context is. */
int cc_sys_create(cc_ctx* ctx, int o, int v, int naux, const double* fock, const double* B, cc_sys** out);
void cc_sys_destroy(cc_sys* sys);

/* R(t) and E(t) (Eqs. CC_ampl, CC_energy). r1/r2 may be NULL to skip the copy-out;
 * energy may be NULL. prec selects the contraction precision (CC_FP64 for the outer residual). */
int cc_residual(cc_ctx* ctx, cc_sys* sys, const double* t1, const double* t2,
                double* r1, double* r2, double* energy, cc_precision prec);

/* J(t) d, the exact directional derivative of R at t along d (App. B: every bilinear
 * contraction becomes two). Mixed precisions run the contractions on tensor cores; the
 * intermediates at t that the derivative multiplies are computed in FP64 for prec = CC_FP64 or
 * CC_DF64, and in the FP64 emulation (CC_FP64_EMU) otherwise. */
int cc_jvp(cc_ctx* ctx, cc_sys* sys, const double* t1, const double* t2,
           const double* d1, const double* d2, double* j1, double* j2, cc_precision prec);

/* J(t) d_k for ndir directions at one point t, with one residual evaluation at t (App. B): the
 * values of the intermediates are kept and each direction runs the tangent program, which keeps
 * the tensor-core staging of its fixed operands across the directions. d1s / d2s / j1s / j2s
 * hold ndir vectors back to back ([ndir][o][v] and [ndir][o][o][v][v]); host or device. */
int cc_jvp_multi(cc_ctx* ctx, cc_sys* sys, const double* t1, const double* t2, int ndir, const double* d1s,
                 const double* d2s, double* j1s, double* j2s, cc_precision prec);

/* y = A_F x (inverse = 0) or y = A_F^{-1} x (inverse = 1 or 2), where
 * (A_F x)_ij^ab = sum_c (f_ac x_ij^cb + f_bc x_ij^ac) - sum_k (f_ki x_kj^ab + f_kj x_ik^ab) and
 * (A_F x)_i^a = sum_c f_ac x_i^c - sum_k f_ki x_k^a (Eq. Preconditioner, App. C; the factor 4
 * printed there comes from an unnormalised projection and is not applied). inverse = 1 is the
 * inner GMRES of the solver (relative tolerance 1e-12 in FP64, 1e-6 otherwise); inverse = 2 is
 * exact: rotate into the eigenbases of the occupied and virtual Fock blocks, divide by
 * e_a + e_b - e_i - e_j (e_a - e_i for singles) and rotate back, the rotations at prec and,
 * for the tensor-core precisions, the doubles projected back onto y_ij^ab = y_ji^ba. */
int cc_apply_AF(cc_ctx* ctx, cc_sys* sys, const double* x1, const double* x2,
                double* y1, double* y2, int inverse, cc_precision prec);

/* Solves R(t) = 0. t1/t2: on input the initial guess if use_guess != 0 (otherwise the
 * generalised MP2 start t1 = 0, t2 = A_F^{-1}(-R2(0)) is used, with R2(0)_ij^ab = (ia|jb)); on
 * output the solution. With a tensor-core precision the JVPs and A_F^{-1} run on tensor cores
 * and every A_F^{-1} output is projected onto t_ij^ab = t_ji^ba before it enters the Krylov
 * space; the residual, energy, update and orthogonalisation stay FP64 (or double-float, by
 * outer_prec). Between two residual evaluations the JVPs keep the tensor-core staging of the
 * operands that do not change (at most about 32 copies of the largest tensors, 1 GiB, or an
 * eighth of the context's budget), so a mixed solve holds that much more device memory.
 * Returns CC_OK, CC_ERR_NOT_CONVERGED or CC_ERR_DIVERGED with the report filled. */
int cc_solve(cc_ctx* ctx, cc_sys* sys, const cc_solve_opts* opts, double* t1, double* t2,
             int use_guess, cc_report* report);

/* Solves nsys problems of one context together (the batching of the serving pattern; the paper
 * solves one problem at a time). NK and PNK run in lockstep: every residual and JVP is evaluated
 * for all unfinished problems at once, the same contraction of every problem in one group, whose
 * tensor-core contractions share persistent grouped launches (up to 16 problems per launch), and
 * the Krylov iterations of each Newton step advance together until each problem's forcing
 * condition holds. Each problem's arithmetic is that of cc_solve from the generalised MP2 start,
 * so its result is the same (bit for bit). Other methods solve the problems one after the other.
 * sys: nsys distinct problems of ctx; t1s / t2s: nsys output pointers each (host or device; the
 * arrays may be NULL), written as each problem finishes; reports: nsys entries. Returns CC_OK
 * once all have finished (each problem's own status is in its report), or an error of the call. */
int cc_solve_batch(cc_ctx* ctx, int nsys, cc_sys* const* sys, const cc_solve_opts* opts, double* const* t1s,
                   double* const* t2s, cc_report* reports);

/* The correlation energy E(t) of cc_residual, computed without allocating any device memory.
 * The paper has no counterpart: this is a service for callers that cannot call cudaMalloc at
 * this point (code inside another framework's memory arena, real-time loops that must stay
 * out of the driver's allocator, processes whose device memory is reserved up front).
 * t1 (o x v), t2 (o x o x v x v, already satisfying t_ij^ab = t_ji^ba) and energy (one double)
 * are device pointers on the problem's device; the call enqueues the work on `stream`
 * (a cudaStream_t, NULL for the default stream) and returns without waiting.
 * Scratch: up to 1024 partial sums in a fixed device array inside the library (8 KB per GPU
 * that loads it, held until exit); a launch that would need more partial sums is rejected
 * with CC_ERR_INVALID. Every call shares that array, so calls that overlap on the GPU (on
 * different streams, or from different threads) race; order them on one stream. cc_sys_create
 * readies this entry point: it loads the module that holds the array and the energy kernels
 * (lazy module loading would otherwise allocate inside the driver on the first call) and looks
 * up the array's device address, so the calls themselves load and allocate nothing.
 * Returns CC_OK, CC_ERR_INVALID (NULL pointer, bad sizes) or CC_ERR_CUDA. */
int cc_energy_noalloc(const cc_sys* sys, const double* t1, const double* t2, double* energy, void* stream);

/* Continuous-batching server on one device (the serving pattern of the solver; the paper
 * solves one problem at a time). max_slots worker slots, each with its own stream and memory
 * pool, take submitted solves in arrival order as soon as a slot is free and the request's
 * device-memory estimate fits under mem_budget (0: no budget), so the kernels of different
 * requests overlap on the device. Results are bitwise independent of what else runs. */
int cc_server_create(cc_server** srv, int device, size_t mem_budget, int max_slots);
/* Admission order: CC_SERVE_FIFO (default) takes the oldest waiting request; with
 * CC_SERVE_SHORTEST_FIRST a free slot takes the waiting request with the least estimated work
 * ((naux + o^2) v^4, the residual's ladder cost) divided by (1 + seconds it has waited), so small
 * requests do not queue behind large ones and a large one is not passed over for ever. Results
 * do not depend on the order. CC_ERR_INVALID for another value. */
#define CC_SERVE_FIFO 0
#define CC_SERVE_SHORTEST_FIRST 1
int cc_server_set_policy(cc_server* srv, int policy);
/* Grouped mode: with group_max > 1 a slot that takes a waiting request also takes up to
 * group_max - 1 later waiting requests with identical NK/PNK options whose memory estimates fit,
 * and solves them as one lockstep batch (cc_solve_batch: the same contraction of every request in
 * one grouped launch); each request is posted as soon as it has finished, with the result it
 * would have alone. 1 (the default) solves one request per slot. CC_ERR_INVALID outside 1..64. */
int cc_server_set_grouping(cc_server* srv, int group_max);
/* Finishes the running solves, drops queued ones and frees everything. */
void cc_server_destroy(cc_server* srv);
/* Copies the problem (host pointers) before returning; ticket identifies the request.
 * CC_ERR_OOM if the request's estimate exceeds the whole budget (it could never run). */
int cc_serve_submit(cc_server* srv, int o, int v, int naux, const double* fock, const double* B,
                    const cc_solve_opts* opts, uint64_t* ticket);
/* CC_PENDING while the request waits or runs; then its cc_solve status, with report filled and
 * the solution copied to t1/t2 (host, may be NULL). That call releases the amplitudes; the
 * ticket's times stay available through cc_serve_times. */
int cc_serve_poll(cc_server* srv, uint64_t ticket, cc_report* report, double* t1, double* t2);
/* Cancels a request: one still waiting is dropped, one running stops at its next outer
 * iteration. Its poll then returns CC_ERR_CANCELLED with the report of what ran (a waiting one:
 * zeros) and the amplitudes reached so far. CC_ERR_INVALID for an unknown or released ticket. */
int cc_serve_cancel(cc_server* srv, uint64_t ticket);
/* Timestamps of a request in seconds since server creation: submit, admit, finish (CC_PENDING
 * until it has finished). */
int cc_serve_times(cc_server* srv, uint64_t ticket, double* t_submit, double* t_admit, double* t_finish);
/* Requests running now, waiting now, the most that ran at once, and admitted bytes. */
int cc_server_stats(cc_server* srv, int* running, int* queued, int* max_running, size_t* bytes_admitted);

#ifdef __cplusplus
}
#endif
#endif /* CCPNK_H */
