#!/usr/bin/env python
"""Benchmark: PNK time-to-solution on the o=10, v=90, naux=300 rotated-gauge workload.

One step is one complete preconditioned Newton-Krylov solve (every step of the hot path:
T1 dressing, intermediates, the particle-particle ladder, hole ladder and rings, the
singles, the energy, the analytic JVP, A_F and its inner GMRES, the outer CGS2 Arnoldi
with Eisenstat-Walker forcing and the Newton update) from the generalised-MP2 start to
||R|| < 1e-8, in the mixed path (JVPs on tcgen05 with the three-pass BF16 split, outer
residual and energy in FP64 emulated on tcgen05, update and orthogonalisation in FP64;
A_F^{-1} applied exactly in the Fock eigenbasis, the paper's inner-GMRES inversion timed
beside it). Inputs are resident on the
device before the timed region; L2 is flushed between steps. The line also carries the FP64 PNK time, the roofline of the dominant
kernel, the CPU oracle baseline and an end-to-end time through the C ABI with host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica (no collective on the data path);
rank 0 prints the line with the maximum over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "o10v90_rotated"
METRIC = "PNK time-to-‖R‖<1e-8, mixed vs FP64; residual TFLOP/s vs peak; p50/p99 served"
# FP64 FMA pipe of a B300: 148 SMs x 2 DFMA/clk x 2 flop x 2.032 GHz (a DFMA-loop probe
# measured 1.201 TFLOP/s on this machine)
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12
# TF32 dense tensor peak: measured bf16 burst x the nominal TF32/BF16 ratio (1.1 / 2.25)
TF32_RATIO = 1.1 / 2.25
OZ_PRODUCTS = 45  # BF16 slice products per FP64-equivalent product of the emulation (9 slices)
# DRAM read + write bytes per launch of a tagged GEMM, from one ncu capture of the current build:
# (bytes, where they come from)
TRAFFIC_FROM_CAPTURE = {
    "emu": (58.4e6, "ncu launch list of one o10v90 emulated residual (profiles/oz_gemm_emu_ladder_build_o10v90.md): "
                    "mean over the ladder-build blocks summed on chip of their two digit-staging launches and the "
                    "oz_gemm_kernel launch; a constant from that capture, not measured by this run"),
}


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over the ranks of the job (x itself without a process group): the step time
    of N independent replicas is that of the slowest."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_threads():
    """Threads the oracle's BLAS runs on (threadpoolctl when installed, else the environment)."""
    try:
        from threadpoolctl import threadpool_info

        return max([i.get("num_threads", 1) for i in threadpool_info()] or [os.cpu_count()])
    except Exception:
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            if os.environ.get(var, "").isdigit():
                return int(os.environ[var])
        return os.cpu_count()


ONE_THREAD_SNIPPET = """
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth
s = synth.workload({workload!r})
f, Bc, _ = cc.to_eigenbasis(s.fock, s.B, s.o)
steps = cc.fp_diis_iterates(f, Bc, s.o, diis_size=12)
next(steps)
t0 = time.perf_counter()
next(steps)
print(json.dumps({{"s_per_iteration": time.perf_counter() - t0}}))
"""


def one_thread_iteration():
    """Seconds of one oracle FP+DIIS iteration with the BLAS held to one thread (a child process
    started with the thread-count variables set to 1)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ONE_THREAD_SNIPPET.format(root=ROOT, workload=WORKLOAD)
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return json.loads(out.stdout.strip().splitlines()[-1])["s_per_iteration"]
    except Exception:
        return None


def oracle_solve_iterations():
    """Residual evaluations the oracle's FP+DIIS solve of the bench workload takes to reach
    ||R|| < 1e-8, from a complete oracle run (tests/golden/make_golden.py)."""
    with open(os.path.join(ROOT, "tests", "golden", "energies.json")) as fh:
        rec = json.load(fh)[WORKLOAD]
    return rec.get("iterations_to_1e-8") or rec["iterations"]


class OracleSolve:
    """The oracle's own FP+DIIS solve of the bench workload from the MP2 start, run one
    iteration (a residual evaluation, the update and the DIIS extrapolation) at a time."""

    def __init__(self):
        from oracle import dfccsd as cc
        from paper_2608_06669_b300 import synth

        s = synth.workload(WORKLOAD)
        f, Bc, _ = cc.to_eigenbasis(s.fock, s.B, s.o)
        t0 = time.perf_counter()
        self.steps = cc.fp_diis_iterates(f, Bc, s.o, diis_size=12)
        self.start_s = time.perf_counter() - t0
        self.done = 0
        self.last_res = None

    def run(self, n):
        """n iterations; returns their wall time in seconds."""
        t0 = time.perf_counter()
        for _ in range(n):
            _, _, _, _, self.last_res = next(self.steps)
            self.done += 1
        return time.perf_counter() - t0


def cpu_baseline(seconds_budget=12.0):
    """The oracle as it stands on the host cores, on a bounded sample of the bench workload:
    iterations of its own FP+DIIS solve from the MP2 start on every thread the BLAS runs (about
    seconds_budget of work), and one iteration with one thread. The metric is time to
    solution, so the sample's seconds per iteration are scaled by the iterations the complete
    oracle solve takes to reach 1e-8 (tests/golden/energies.json)."""
    evals = oracle_solve_iterations()
    cores = oracle_threads()
    sol = OracleSolve()
    times = []
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < seconds_budget or len(times) < 2:
        times.append(sol.run(1))
    per = statistics.mean(times[1:]) if len(times) > 2 else statistics.mean(times)
    per1 = one_thread_iteration()
    one = f"{per1:.3f} s" if per1 else "not measured"
    return {"value": per * evals, "unit": "s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "s_per_iteration": per, "s_per_iteration_1_thread": per1, "iterations_to_solution": evals,
            "value_1_thread": per1 * evals if per1 else None,
            "sample": f"{len(times)} iterations of the oracle's FP+DIIS solve of o=10 v=90 naux=300 from the "
                      f"MP2 start ({per:.3f} s each on {cores} threads; one iteration on 1 thread {one}; the "
                      f"complete solve takes {evals} iterations, so value = s/iteration x {evals}); ||R|| after "
                      f"{sol.done} iterations {sol.last_res:.2e}"}


def run_reference(args):
    """The reference arm: the CPU oracle's own FP+DIIS solve of the bench workload. Each step
    runs a bounded sample of that one solve (--ref-iterations iterations, continuing where the
    previous step stopped, warm-up steps included), so ms_per_step is the measured time of a
    step; value is the time to solution, the measured seconds per iteration times the
    iterations the complete oracle solve takes."""
    rank, _, world = rank_info()
    if rank != 0:
        return
    evals = oracle_solve_iterations()
    cores = oracle_threads()
    sol = OracleSolve()
    for _ in range(args.warmup):
        sol.run(args.ref_iterations)
    steps = [sol.run(args.ref_iterations) for _ in range(args.steps)]
    per_step = statistics.mean(steps)
    per_it = per_step / args.ref_iterations
    val = per_it * evals
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "o": 10, "v": 90, "naux": 300, "gauge": "rotated",
                       "tol": 1e-8, "l2": "n/a (CPU)",
                       "step": f"{args.ref_iterations} iterations of the oracle FP+DIIS solve (value: time to "
                               f"solution = s/iteration x {evals})"},
            "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"{(args.warmup + args.steps) * args.ref_iterations} iterations of one oracle "
                                       f"FP+DIIS solve from the MP2 start, {per_it:.3f} s each; ||R|| {sol.last_res:.2e} "
                                       f"after {sol.done}; the complete solve takes {evals}"},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def roofline_entry(rec, kind, peaks, peak_kind):
    """Roofline of one tagged GEMM from the kernel timer's (launches, ms, flops) record. kind:
    'fp64' (FMA pipe), 'tf32x3' (three TF32 passes on tcgen05), 'emu' (Ozaki slices: 45 BF16
    slice products per FP64-equivalent product on tcgen05 kind::f16)."""
    n, ms, fl = rec
    if not n or ms <= 0:
        return None
    if kind == "fp64":
        ach, peak = fl / (ms / 1e3) / 1e12, FP64_PEAK_TFLOPS
        return {"bound": "alu", "kernel": "gemm_f64_kernel (FP64 ladder build, FMA pipe)", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "launches": n, "ms_per_launch": ms / n,
                "flops_per_launch": fl / n, "peak_source": "148 SMs x 2 DFMA/clk x 2 x 2.032 GHz (unit counts)"}
    if kind == "tf32x3":
        peak = peaks["bf16_tflops"] * TF32_RATIO
        ach = 3.0 * fl / (ms / 1e3) / 1e12
        return {"bound": "tensor", "kernel": "gemm_tc_kernel<tf32> (ladder build of the JVP, three TF32 passes)",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "launches": n,
                "ms_per_launch": ms / n, "flops_per_launch": 3.0 * fl / n, "logical_tflops": fl / (ms / 1e3) / 1e12,
                "peak_source": f"{peak_kind} bf16 burst x 1.1/2.25 (of {peak_kind})"}
    if kind == "bf16x3":
        peak = peaks["bf16_tflops"]
        ach = 3.0 * fl / (ms / 1e3) / 1e12
        return {"bound": "tensor", "kernel": "gemm_tc_kernel<bf16> (ladder build of the JVP, three BF16 passes)",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "launches": n,
                "ms_per_launch": ms / n, "flops_per_launch": 3.0 * fl / n, "logical_tflops": fl / (ms / 1e3) / 1e12,
                "peak_source": f"{peak_kind} bf16 burst (of {peak_kind})"}
    peak = peaks["bf16_tflops"]
    ach = OZ_PRODUCTS * fl / (ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "FP64-emulated ladder build: digit staging (oz_stage_rows or oz_rowexp + "
                                         "oz_digits), then oz_gemm_kernel (slice products summed on chip) or "
                                         "gemm_tc_kernel<bf16, partials> + oz_combine, by shape",
            "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "launches": n,
            "ms_per_launch": ms / n, "flops_per_launch": OZ_PRODUCTS * fl / n,
            "fp64_equivalent_tflops": fl / (ms / 1e3) / 1e12,
            "peak_source": f"{peak_kind} bf16 burst (of {peak_kind}); achieved counts the 45 BF16 slice products "
                           f"of each FP64-equivalent product, time covers staging, MMA and the recombination"}


def timed(fn):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, r


def large_block(args, peaks, peak_kind):
    """The o=30, v=270, naux=900 workload: FP64 residual natively and emulated on the tensor
    cores, the mixed JVPs, ladder rates against their peaks, and capped Newton steps of the
    mixed PNK solve (the workload is outside the range where any method converges; see the
    convergence study), one JVP of the native FP64 path for the FP64 per-step cost."""
    import numpy as np
    import torch

    from paper_2608_06669_b300 import ccpnk, synth

    s = synth.workload("o30v270_rotated")
    o, v = s.o, s.v
    ctx = ccpnk.Context(0)
    g = ccpnk.System.from_synth(ctx, s)
    rng = np.random.default_rng(0)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.01, 0.01)
    T1, T2 = torch.from_numpy(t1).cuda(), torch.from_numpy(t2).cuda()
    out = {"workload": "o30v270_rotated", "o": o, "v": v, "naux": s.naux}
    ctx.profile(True)
    out["fp64emu_residual_s"], (_, _, e_emu) = timed(lambda: g.residual(T1, T2, prec="fp64emu"))
    out["ladder_build_fp64emu"] = roofline_entry(ctx.profile_get("ladder_build.emu"), "emu", peaks, peak_kind)
    if not args.no_fp64_large:
        ctx.profile(True)
        out["fp64_residual_s"], (_, _, e64) = timed(lambda: g.residual(T1, T2, prec="fp64"))
        out["ladder_build_fp64"] = roofline_entry(ctx.profile_get("ladder_build.fp64"), "fp64", peaks, peak_kind)
        out["emu_vs_fp64_energy_diff"] = e_emu - e64
        out["fp64emu_residual_speedup"] = out["fp64_residual_s"] / out["fp64emu_residual_s"]
    for prec in ("tf32x3", "bf16x3"):
        ctx.profile(True)
        dt, _ = timed(lambda: g.jvp(T1, T2, T1, T2, prec=prec))
        out[f"{prec}_jvp_incl_fp64emu_value_s"] = dt
        sfx = "bf16" if prec == "bf16x3" else "tf32"
        n, ms, fl = ctx.profile_get(f"ladder_build.{sfx}")
        out[f"{prec}_ladder_build_logical_tflops"] = fl / (ms / 1e3) / 1e12 if ms > 0 else None
        if prec == "tf32x3":
            out["ladder_build_tf32x3"] = roofline_entry((n, ms, fl), "tf32x3", peaks, peak_kind)
    ctx.profile(False)
    steps = args.large_newton
    dt, (_, _, rep) = timed(lambda: g.solve("pnk", "tf32x3", af_direct=1, outer_prec=5, max_outer=steps))
    out["mixed_pnk_newton_steps"] = {"steps": rep["newton_iters"], "seconds": dt,
                                     "s_per_newton_step": dt / max(rep["newton_iters"], 1), "jvps": rep["jvps"],
                                     "res_norm": rep["res_norm"], "energy": rep["energy"]}
    dt, (_, _, rep) = timed(lambda: g.solve("pnk", "fp64emu", af_direct=1, outer_prec=5, max_outer=steps))
    out["fp64emu_pnk_newton_steps"] = {"steps": rep["newton_iters"], "seconds": dt,
                                       "s_per_newton_step": dt / max(rep["newton_iters"], 1), "jvps": rep["jvps"],
                                       "res_norm": rep["res_norm"]}
    if args.fp64_large_jvp:
        dt, _ = timed(lambda: g.jvp(T1, T2, T1, T2, prec="fp64"))
        out["fp64_jvp_incl_fp64_value_s"] = dt
    g.close()
    ctx.close()
    return out


def serve_pass(reqs, prec, extra, args, slots=None, group=1, policy="fifo"):
    """Submits the requests at their arrival times to a fresh server and waits for all of them;
    returns p50/p99 time to solution, solves/s and convergence. group > 1: grouped mode (a slot
    solves up to that many compatible requests together, in lockstep)."""
    import numpy as np

    from paper_2608_06669_b300 import ccpnk

    srv = ccpnk.Server(0, mem_budget=200 << 30, max_slots=slots or args.slots)
    if group > 1:
        srv.set_grouping(group)
    srv.set_policy(policy)
    t_start = time.perf_counter()
    tickets = []
    for arrival, sy in reqs:
        wait = arrival - (time.perf_counter() - t_start)
        if wait > 0:
            time.sleep(wait)
        tickets.append(srv.submit(sy.o, sy.v, sy.naux, sy.fock, sy.B, "pnk", prec, af_direct=1,
                                  max_outer=args.max_newton, max_seconds=args.solve_seconds, **extra))
    results = {}
    while len(results) < len(tickets):
        for t in tickets:
            if t not in results:
                r = srv.poll(t)
                if r is not None:
                    results[t] = r
        time.sleep(0.002)
    times = [srv.times(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    lat = np.array([f - sub for sub, _, f in times])
    span = max(f for _, _, f in times) - min(sub for sub, _, _ in times)
    conv = [results[t][2]["status_code"] == 0 for t in tickets]
    return {"requests": len(reqs), "slots": slots or args.slots, "group": group, "policy": policy,
            "solves_per_s": len(tickets) / span, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "converged": int(sum(conv)), "makespan_s": span,
            "max_concurrent": stats["max_running"],
            "not_converged": [f"o{sy.o}v{sy.v}" for (_, sy), c in zip(reqs, conv) if not c]}


def served_block(args):
    """The first --serve-default requests of the served mix (Poisson arrivals, mean 20 ms),
    each through the continuous-batching server: the mixed path (three-pass TF32 JVPs, FP64-
    emulated outer residual) on all of them; the native FP64 path and the mixed path again on
    the same subset of the requests with o <= --serve-fp64-max-o (native FP64 PNK of the larger
    requests takes minutes: all 32 took 431 s on one B300); with --serve-fp64-all the native
    FP64 path serves every request. The mixed path also runs in the server's grouped mode
    (--group-slots slots, each solving up to --serve-group requests in one lockstep batch)."""
    from paper_2608_06669_b300 import synth

    reqs = synth.served_requests(args.serve_default)
    out = {"slots": args.slots, "arrivals": "exponential, mean 20 ms", "caps": {
        "max_newton": args.max_newton, "max_seconds": args.solve_seconds}}
    mixed = {"outer_prec": 5}
    out["mixed"] = serve_pass(reqs, args.prec, mixed, args)
    # shortest first: a free slot takes the waiting request with the least estimated work
    out["mixed_shortest_first"] = serve_pass(reqs, args.prec, mixed, args, policy="shortest_first")
    # grouped mode: fewer slots, each solving up to --serve-group requests in one lockstep batch
    out["mixed_grouped"] = serve_pass(reqs, args.prec, mixed, args, slots=args.group_slots,
                                      group=args.serve_group, policy="shortest_first")
    sub = reqs if args.serve_fp64_all else [(t, sy) for t, sy in reqs if sy.o <= args.serve_fp64_max_o]
    out["subset"] = ("all" if args.serve_fp64_all else f"the {len(sub)} requests with o <= {args.serve_fp64_max_o}")
    out["fp64_on_subset"] = serve_pass(sub, "fp64", {}, args)
    out["mixed_on_subset"] = serve_pass(sub, args.prec, mixed, args)
    return out


def run_ours(args):
    import torch

    from paper_2608_06669_b300 import ccpnk, synth

    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()

    peaks, peak_kind = measured_peaks()
    s = synth.workload(WORKLOAD)
    ctx = ccpnk.Context(local)
    g = ccpnk.System.from_synth(ctx, s)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()
    # JVPs and A_F^{-1} in the mixed precision, the outer residual (convergence test, energy) in
    # FP64 emulated on the tensor cores, A_F^{-1} exactly in the Fock eigenbasis
    kw = dict(method="pnk", prec=args.prec, af_direct=0 if args.af_gmres else 1, outer_prec=args.outer)

    for _ in range(args.warmup):
        g.solve(**kw)
    torch.cuda.synchronize()

    launches0, calls0 = ctx.launches, ctx.launch_calls
    times, reports = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, rep = g.solve(**kw)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            reports.append(rep)
    launches = ctx.launches - launches0
    calls = ctx.launch_calls - calls0
    # the kernel timer brackets the ladder GEMMs with events, which keeps the JVPs eager (no
    # CUDA graphs), so it runs on repeats of the timed solve right after the timed region
    ctx.profile(True)
    t_prof = 0.0
    for _ in range(max(1, min(args.steps, 3))):
        dt, _ = timed(lambda: g.solve(**kw))
        t_prof += dt
    tags = {"fp64": ctx.profile_get("ladder_build.fp64"), "emu": ctx.profile_get("ladder_build.emu"),
            "tf32x3": ctx.profile_get("ladder_build.tf32"), "bf16x3": ctx.profile_get("ladder_build.bf16")}
    ctx.profile(False)
    t_mean = statistics.mean(times)
    t_max = max_over_ranks(t_mean, dist, device="cuda")

    # the same mixed solve with a native FP64 outer residual, the native FP64 PNK (the mixed
    # path must beat it), PNK with every contraction FP64-emulated, the inner-GMRES A_F^{-1}
    # (the paper's protocol), and the double-float variants
    variants = {
        "mixed_pnk_fp64_outer": dict(method="pnk", prec=args.prec, af_direct=1),
        "fp64_pnk": dict(method="pnk", prec="fp64", af_direct=1),
        "fp64emu_pnk": dict(method="pnk", prec="fp64emu", af_direct=1, outer_prec=5),
        "mixed_pnk_af_gmres": dict(method="pnk", prec=args.prec, af_direct=0, outer_prec=args.outer),
        "mixed_pnk_tf32x3": dict(method="pnk", prec="tf32x3", af_direct=1, outer_prec=args.outer),
        "mixed_pnk_df64_outer": dict(method="pnk", prec=args.prec, af_direct=1, outer_prec=4),
        "df64_pnk": dict(method="pnk", prec="df64", af_direct=1, outer_prec=4),
    }
    if args.only_headline:
        variants = {}
    var_out = {}
    for name, vkw in variants.items():
        dt, (_, _, rep) = timed(lambda: g.solve(**vkw))
        var_out[name] = {"s": dt, **{k: rep[k] for k in ("energy", "res_norm", "newton_iters", "jvps", "status_code")}}

    # end to end through the C ABI with host buffers: upload the problem, solve, read back
    n = s.o + s.v
    e2e_times = []
    for _ in range(0 if args.only_headline else max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gh = ccpnk.System(ctx, s.o, s.v, s.naux, s.fock, s.B)
        t1h, t2h, reph = gh.solve(**kw)  # host outputs (numpy)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        gh.close()
    h2d = 8 * (n * n + s.naux * n * n)
    d2h = 8 * (s.o * s.v + s.o ** 2 * s.v ** 2)
    g.close()
    ctx.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # rooflines of the timed solve's ladder GEMMs; the dominant one (most event time) is the line's
    roofs = {k: roofline_entry(tags[k], k, peaks, peak_kind) for k in tags}
    roofs = {k: r for k, r in roofs.items() if r}
    dom = max(roofs, key=lambda k: tags[k][1]) if roofs else None
    roof = dict(roofs[dom]) if dom else None
    if roof:
        # DRAM bytes per launch from one ncu capture of the same kernels (a constant, labelled as
        # such; null for a kernel without a capture of the current build)
        cap = TRAFFIC_FROM_CAPTURE.get(dom)
        roof["traffic"] = cap[0] if cap else None
        if cap:
            roof["traffic_source"] = cap[1]
        roof["share_of_profiled_solves"] = tags[dom][1] / 1e3 / t_prof
        roof["measured_on"] = "repeats of the timed solve with the kernel timer on (eager JVPs), right after it"
    cpu = None
    if world == 1 and not args.no_cpu and not args.only_headline:
        cpu = cpu_baseline()
    extra = world == 1 and not args.only_headline
    large = large_block(args, peaks, peak_kind) if (extra and not args.no_large) else None
    served = served_block(args) if (extra and args.serve_default > 0) else None
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": f"{args.prec} JVPs + {'fp64emu' if args.outer == 5 else 'f64'} outer residual", "data": "synthetic",
        "config": {"workload": WORKLOAD, "o": s.o, "v": s.v, "naux": s.naux, "gauge": "rotated (off-diagonal f up to 0.1 Eh)",
                   "method": "pnk", "prec": args.prec, "outer_residual": "fp64emu" if args.outer == 5 else "fp64",
                   "tol": 1e-8, "start": "generalised MP2", "af_inverse": "gmres" if args.af_gmres else "eigenbasis",
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": roof, "rooflines": roofs,
        "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(e2e_times) if e2e_times else None, "unit": "s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches // max(args.steps, 1),
        "host_launch_calls": calls // max(args.steps, 1),
        "clocks": clk.summary(),
        "fp64_pnk_s": var_out["fp64_pnk"]["s"] if var_out else None,
        "speedup_mixed_vs_fp64": var_out["fp64_pnk"]["s"] / t_max if var_out else None,
        "variants": var_out,
        "solve": {k: reports[-1][k] for k in ("energy", "res_norm", "newton_iters", "residual_evals", "jvps",
                                               "af_applies", "krylov_iters")},
        "large": large,
        "served": served,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_serve(args):
    """The served mix: requests of uneven (o, v) (o ~ U{4..16}, v = round(o U[6,9]),
    naux = 3(o+v), half canonical, half Haar-rotated) arriving with exponential gaps
    (mean 20 ms), submitted to the continuous-batching server at their arrival times;
    reports solves/s and p50/p99 time-to-solution for the mixed path and the FP64 path."""
    import numpy as np

    from paper_2608_06669_b300 import ccpnk, synth

    reqs_all = synth.served_requests(args.serve)
    out = {}
    # the FP64 path is ~4-12x slower per solve, so it serves the first requests of the same
    # stream only (the mixed path serves all of them); both cap a solve at max_newton steps
    # the mixed path also serves that same prefix alone, so p50/p99 compare like with like
    passes = (("tf32x3", "tf32x3", reqs_all), ("tf32x3_fp64_set", "tf32x3", reqs_all[: args.serve_fp64]),
              ("fp64", "fp64", reqs_all[: args.serve_fp64]))
    for key, prec, reqs in passes:
        srv = ccpnk.Server(0, mem_budget=200 << 30, max_slots=args.slots)
        t_start = time.perf_counter()
        tickets = []
        for arrival, s in reqs:
            wait = arrival - (time.perf_counter() - t_start)
            if wait > 0:
                time.sleep(wait)
            tickets.append(srv.submit(s.o, s.v, s.naux, s.fock, s.B, "pnk", prec, af_direct=1,
                                      max_outer=args.max_newton, max_seconds=args.solve_seconds))
        results = {}
        while len(results) < len(tickets):
            for t in tickets:
                if t not in results:
                    r = srv.poll(t)
                    if r is not None:
                        results[t] = r
            time.sleep(0.005)
        times = [srv.times(t) for t in tickets]
        stats = srv.stats()
        srv.close()
        lat = np.array([f - sub for sub, _, f in times])
        span = max(f for _, _, f in times) - min(sub for sub, _, _ in times)
        conv = [results[t][2]["status_code"] == 0 for t in tickets]
        out[key] = {"solves_per_s": len(tickets) / span, "p50_s": float(np.percentile(lat, 50)),
                     "p99_s": float(np.percentile(lat, 99)), "converged": int(sum(conv)), "requests": len(tickets),
                     "max_concurrent": stats["max_running"], "makespan_s": span,
                     "not_converged": [f"o{s.o}v{s.v}" for (_, s), c in zip(reqs, conv) if not c]}
    line = {"metric": METRIC, "mode": "served", "value": out["tf32x3"]["p99_s"], "unit": "s (p99 time-to-solution)",
            "higher_is_better": False, "n_gpus": 1, "dtype": "tf32x3+f64", "data": "synthetic",
            "config": {"workload": "served mix", "requests": args.serve, "arrivals": "exponential, mean 20 ms",
                       "o": "U{4..16}", "v": "round(o U[6,9])", "naux": "3(o+v)", "gauges": "canonical / Haar",
                       "slots": args.slots, "af_inverse": "eigenbasis"},
            "mixed": out["tf32x3"], "mixed_on_fp64_requests": out["tf32x3_fp64_set"], "fp64": out["fp64"]}
    print(json.dumps(line), flush=True)


def run_kernels(args):
    """Per-kernel rates on one workload: an FP64 residual and the tangent programs in the
    tensor-core precisions, timed by the library's tagged kernel timer (CUDA events on the
    context's stream), then capped solves with several methods. Used for the large and the
    near-degenerate workloads, where the default bench line would take too long."""
    import numpy as np
    import torch

    from paper_2608_06669_b300 import ccpnk, synth

    s = synth.workload(args.kernels)
    o, v, P = s.o, s.v, s.naux
    ctx = ccpnk.Context(0)
    g = ccpnk.System.from_synth(ctx, s)
    rng = np.random.default_rng(0)
    t1 = torch.zeros((o, v), dtype=torch.float64, device="cuda")
    t2 = torch.from_numpy(synth.random_amplitudes(rng, o, v, 0.02, 0.02)[1]).cuda()
    peaks, _ = measured_peaks()
    tf32_peak = peaks["bf16_tflops"] * TF32_RATIO
    out = {"workload": args.kernels, "o": o, "v": v, "naux": P}

    def rate(tag):
        n, ms, fl = ctx.profile_get(tag)
        return {"launches": n, "ms": ms, "tflops": fl / (ms / 1e3) / 1e12 if ms > 0 else None}

    ctx.profile(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.residual(t1, t2, prec="fp64")
    torch.cuda.synchronize()
    t_res = time.perf_counter() - t0
    out["fp64_residual_s"] = t_res
    out["fp64_ladder_build"] = rate("ladder_build.fp64")
    out["fp64_ladder_contract"] = rate("ladder_contract.fp64")
    full = (2 * P + 2 * o * o) * v ** 4
    out["fp64_residual_ladder_equiv_tflops"] = full / t_res / 1e12
    out["fp64_peak_tflops"] = FP64_PEAK_TFLOPS
    for prec in ("tf32x3", "bf16x3", "tf32"):
        ctx.profile(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.jvp(t1, t2, t1, t2, prec=prec)
        torch.cuda.synchronize()
        out[f"{prec}_jvp_incl_fp64_value_s"] = time.perf_counter() - t0
        sfx = "bf16" if prec == "bf16x3" else "tf32"
        out[f"{prec}_ladder_build"] = rate(f"ladder_build.{sfx}")
        out[f"{prec}_ladder_contract"] = rate(f"ladder_contract.{sfx}")
    ctx.profile(False)
    out["tf32_peak_tflops"] = tf32_peak
    print(json.dumps({"metric": METRIC, "mode": "kernels", **out}), flush=True)
    if args.kernels_only:
        return
    # capped solves, one line each so that a partial run still reports
    for meth, prec, extra in (("pnk", "tf32x3", {}), ("nk", "tf32x3", {}),
                              ("fp_diis", "fp64", {"level_shift": args.shift}), ("pnk", "fp64", {})):
        if prec == "fp64" and meth == "pnk" and args.no_fp64_solve:
            continue
        t0 = time.perf_counter()
        _, _, rep = g.solve(meth, prec, af_direct=1, max_seconds=args.solve_seconds,
                            max_outer=args.max_newton if meth != "fp_diis" else 10 * args.max_newton, **extra)
        rep["wall_s"] = time.perf_counter() - t0
        rep["jvps_per_newton"] = rep["jvps"] / max(rep["newton_iters"], 1)
        keep = ("energy", "res_norm", "newton_iters", "residual_evals", "jvps", "jvps_per_newton", "status_code",
                "wall_s")
        print(json.dumps({"mode": "kernels.solve", "workload": args.kernels, "method": meth, "prec": prec,
                          **extra, **{k: rep[k] for k in keep}}), flush=True)


CPU_TABLE_SNIPPET = """
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth
s = synth.workload({workload!r})
t1, t2 = synth.random_amplitudes(np.random.default_rng(0), s.o, s.v, 0.01, 0.01)
t0 = time.perf_counter()
cc.residual(s.fock, s.B, s.o, t1, t2)
print(json.dumps({{"residual_s": time.perf_counter() - t0}}))
"""


def run_cpu_table(args):
    """The CPU oracle as it stands on this host: one residual evaluation of each workload on
    every BLAS thread and on one thread (child processes with the thread variables set), and the
    oracle's complete FP+DIIS solve where it converges."""
    from oracle import dfccsd as cc
    from paper_2608_06669_b300 import synth

    def child(workload, threads):
        env = dict(os.environ)
        if threads:
            env.update(OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads), MKL_NUM_THREADS=str(threads))
        code = CPU_TABLE_SNIPPET.format(root=ROOT, workload=workload)
        try:
            out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1800)
            return json.loads(out.stdout.strip().splitlines()[-1])["residual_s"]
        except Exception as e:  # report, do not fail the table
            return f"failed: {type(e).__name__}"

    table = {"cpu": cpu_model(), "threads": oracle_threads(), "nproc": os.cpu_count(), "rows": {}}
    for workload, one_thread in (("o5v20_canonical", True), ("o10v90_rotated", True),
                                 ("o20v180_neardegenerate", True), ("o30v270_rotated", False)):
        row = {"residual_all_threads_s": child(workload, None)}
        row["residual_1_thread_s"] = child(workload, 1) if one_thread else "not run (minutes on one thread)"
        table["rows"][workload] = row
        print(json.dumps({"mode": "cpu_table.partial", workload: row}), flush=True)
    for workload in ("o5v20_canonical", "o10v90_rotated"):
        s = synth.workload(workload)
        f, Bc, _ = cc.to_eigenbasis(s.fock, s.B, s.o)
        t0 = time.perf_counter()
        _, _, e, hist = cc.solve_fp_diis(f, Bc, s.o, tol=1e-8, maxiter=400, diis_size=12)
        table["rows"][workload]["fp_diis_solve_all_threads_s"] = time.perf_counter() - t0
        table["rows"][workload]["fp_diis_iterations"] = len(hist)
        table["rows"][workload]["fp_diis_energy"] = e
    print(json.dumps({"mode": "cpu_table", **table}), flush=True)


def run_peaks(args):
    """Measured arithmetic rates on this GPU: the FP64 and FP32 FMA pipes (the library's FMA-chain
    probe) and torch's FP64, TF32 and BF16 matmuls (best of five, CUDA events)."""
    import torch

    from paper_2608_06669_b300 import ccpnk

    out = {"mode": "peaks", "fp64_fma_tflops": ccpnk.probe_fma_rate(0, True),
           "fp32_fma_tflops": ccpnk.probe_fma_rate(0, False),
           "fp64_fma_nominal_tflops": FP64_PEAK_TFLOPS}

    def mm(dtype, n, tf32=False):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        best = 1e30
        for rep in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            if rep:
                best = min(best, e0.elapsed_time(e1) / 1e3)
        torch.backends.cuda.matmul.allow_tf32 = False
        return 2.0 * n ** 3 / best / 1e12

    out["torch_fp64_matmul_4096_tflops"] = mm(torch.float64, 4096)
    out["torch_tf32_matmul_8192_tflops"] = mm(torch.float32, 8192, tf32=True)
    out["torch_bf16_matmul_8192_tflops"] = mm(torch.bfloat16, 8192)
    print(json.dumps(out), flush=True)


def run_case(args):
    """One residual or JVP evaluation on a named workload or an (o, v, naux) system: the small,
    single-call cases that kernel profiles are taken on."""
    import torch

    from paper_2608_06669_b300 import ccpnk, synth

    import numpy as np

    spec = args.case
    if "," in spec:
        o, v, P = (int(x) for x in spec.split(","))
        s = synth.make_system(o, v, P, seed=4, gauge="small")
    else:
        s = synth.workload(spec)
    o, v = s.o, s.v
    ctx = ccpnk.Context(0)
    g = ccpnk.System.from_synth(ctx, s)
    t1, t2 = synth.random_amplitudes(np.random.default_rng(0), o, v, 0.02, 0.02)
    T1, T2 = torch.from_numpy(t1).cuda(), torch.from_numpy(t2).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.case_op == "jvp":
        _, out = g.jvp(T1, T2, T1, T2, prec=args.case_prec)
    else:
        _, out, _ = g.residual(T1, T2, prec=args.case_prec)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({"mode": "case", "case": spec, "op": args.case_op, "prec": args.case_prec, "o": o, "v": v,
                      "naux": s.naux, "seconds": dt, "max_abs": float(out.abs().max()),
                      "device_bytes": ctx.device_bytes}), flush=True)
    g.close()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="", help="one evaluation on a workload name or 'o,v,naux' instead")
    ap.add_argument("--case-op", default="jvp", choices=["jvp", "residual"])
    ap.add_argument("--case-prec", default="tf32x3", choices=["fp64", "tf32", "tf32x3", "bf16x3", "df64", "fp64emu"])
    ap.add_argument("--peaks", action="store_true", help="measure the FMA-pipe and matmul rates instead")
    ap.add_argument("--cpu-table", action="store_true", help="time the CPU oracle on every workload instead")
    ap.add_argument("--kernels", default="", help="per-kernel rates and capped solves on this workload instead")
    ap.add_argument("--shift", type=float, default=0.2, help="FP+DIIS level shift in --kernels")
    ap.add_argument("--no-fp64-solve", action="store_true")
    ap.add_argument("--kernels-only", action="store_true", help="--kernels without the capped solves")
    ap.add_argument("--solve-seconds", type=float, default=120.0, help="wall-time cap of each solve in --kernels")
    ap.add_argument("--serve", type=int, default=0, help="run the served mix with this many requests instead")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-fp64", type=int, default=8, help="requests the FP64 pass of --serve runs")
    ap.add_argument("--max-newton", type=int, default=30, help="Newton-step cap of a served solve")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["tf32x3", "bf16x3", "tf32", "fp64", "fp64emu"])
    ap.add_argument("--outer", type=int, default=5, help="outer-residual precision code (0 FP64, 4 DF64, 5 FP64-emulated)")
    ap.add_argument("--no-large", action="store_true", help="skip the o=30 v=270 block of the main line")
    ap.add_argument("--no-fp64-large", action="store_true", help="skip the native FP64 residual/JVP at o=30 v=270")
    ap.add_argument("--large-newton", type=int, default=2, help="capped Newton steps at o=30 v=270")
    ap.add_argument("--fp64-large-jvp", action="store_true", help="also time one native FP64 JVP at o=30 v=270")
    ap.add_argument("--serve-default", type=int, default=32, help="requests of the served block (0: skip)")
    ap.add_argument("--serve-fp64-max-o", type=int, default=8, help="native FP64 serves the requests with o <= this")
    ap.add_argument("--serve-fp64-all", action="store_true", help="native FP64 serves every request of the block")
    ap.add_argument("--serve-group", type=int, default=8, help="requests per lockstep batch in the grouped pass")
    ap.add_argument("--group-slots", type=int, default=2, help="slots of the grouped pass")
    ap.add_argument("--only-headline", action="store_true",
                    help="only the timed solves (the launch-list and profile captures run this)")
    ap.add_argument("--af-gmres", action="store_true", help="invert A_F by inner GMRES in the timed solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ref-iterations", type=int, default=3, help="oracle iterations per reference step")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.peaks:
        run_peaks(args)
    elif args.cpu_table:
        run_cpu_table(args)
    elif args.serve:
        run_serve(args)
    elif args.kernels:
        run_kernels(args)
    elif args.case:
        run_case(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
