"""Mixed precision: tcgen05 TF32 contractions (FP32 accumulation) against the FP64 oracle.

TF32 keeps 10 explicit mantissa bits, so each product carries a relative error near 2^-11
and a contraction of K terms an error near 2^-11 * sum|a b|. The tests bound the error
normwise (max element error over the largest oracle element); the solver keeps its outer
residual, energy and update in FP64, so a mixed-precision solve still lands on the FP64 root
to 1e-8 Eh.
"""
import json
import os

import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energies.json")
TF32_TOL = 5e-3


def nrel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def ctx(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    c = ccpnk.Context(0)
    yield c
    c.close()


def gsys(ctx, s):
    from paper_2608_06669_b300 import ccpnk

    return ccpnk.System.from_synth(ctx, s)


@pytest.mark.parametrize("o,v,gauge", [(1, 1, "canonical"), (3, 7, "haar"), (6, 40, "small"), (10, 90, "small")])
def test_tf32_AF_apply(ctx, o, v, gauge):
    s = synth.make_system(o, v, 4, seed=3, gauge=gauge)
    x1, x2 = synth.random_amplitudes(np.random.default_rng(1), o, v, 1.0, 1.0)
    y1, y2 = gsys(ctx, s).apply_AF(x1, x2, 0, prec="tf32")
    q1, q2 = cc.apply_AF(s.fock, o, x1, x2)
    assert nrel(y1, q1) < 2e-3 and nrel(y2, q2) < 2e-3


@pytest.mark.parametrize("o,v,naux,gauge", [(2, 4, 5, "haar"), (4, 9, 11, "small"), (7, 33, 20, "haar")])
def test_tf32_residual_and_jvp(ctx, o, v, naux, gauge):
    s = synth.make_system(o, v, naux, seed=7 + o, gauge=gauge)
    rng = np.random.default_rng(o * v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    g = gsys(ctx, s)
    r1, r2, e = g.residual(t1, t2, prec="tf32")
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r2 - q2).max() < TF32_TOL * scale and np.abs(r1 - q1).max() < TF32_TOL * scale
    j1, j2 = g.jvp(t1, t2, d1, d2, prec="tf32")
    p1, p2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    scale = max(np.abs(p1).max(), np.abs(p2).max())
    assert np.abs(j2 - p2).max() < TF32_TOL * scale and np.abs(j1 - p1).max() < TF32_TOL * scale


@pytest.mark.parametrize("o,v,naux,gauge", [(2, 4, 5, "haar"), (7, 33, 20, "haar")])
def test_tf32x3_residual_and_jvp(ctx, o, v, naux, gauge):
    """The three-pass split keeps about FP32 accuracy: 1e-6 normwise."""
    s = synth.make_system(o, v, naux, seed=9 + o, gauge=gauge)
    rng = np.random.default_rng(o + 3 * v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    g = gsys(ctx, s)
    r1, r2, _ = g.residual(t1, t2, prec="tf32x3")
    q1, q2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r2 - q2).max() < 1e-6 * scale and np.abs(r1 - q1).max() < 1e-6 * scale
    j1, j2 = g.jvp(t1, t2, d1, d2, prec="tf32x3")
    p1, p2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    scale = max(np.abs(p1).max(), np.abs(p2).max())
    assert np.abs(j2 - p2).max() < 1e-6 * scale and np.abs(j1 - p1).max() < 1e-6 * scale


@pytest.mark.parametrize("o,v,naux,gauge", [(2, 4, 5, "haar"), (5, 21, 13, "small"), (7, 33, 20, "haar")])
def test_bf16x3_residual_and_jvp(ctx, o, v, naux, gauge):
    """BF16 keeps 8 significant bits, so hi + lo holds 16 and each split product is off by
    about 3 * 2^-18 relative; the bound is 2e-5 normwise."""
    s = synth.make_system(o, v, naux, seed=11 + o, gauge=gauge)
    rng = np.random.default_rng(5 * o + v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    g = gsys(ctx, s)
    r1, r2, _ = g.residual(t1, t2, prec="bf16x3")
    q1, q2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r2 - q2).max() < 2e-5 * scale and np.abs(r1 - q1).max() < 2e-5 * scale
    j1, j2 = g.jvp(t1, t2, d1, d2, prec="bf16x3")
    p1, p2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    scale = max(np.abs(p1).max(), np.abs(p2).max())
    assert np.abs(j2 - p2).max() < 2e-5 * scale and np.abs(j1 - p1).max() < 2e-5 * scale
    # and it is a real improvement over one TF32 pass
    k1, k2 = g.jvp(t1, t2, d1, d2, prec="tf32")
    assert np.abs(j2 - p2).max() < np.abs(k2 - p2).max()


def test_tf32_jvp_workload_error(ctx):
    """The error of the TF32 JVP on the o=10, v=90 workload, stated against the FP64 oracle."""
    s = synth.workload("o10v90_rotated")
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    d1, d2 = synth.random_amplitudes(np.random.default_rng(4), o, v, 0.01, 0.01)
    j1, j2 = gsys(ctx, s).jvp(t1, t2, d1, d2, prec="tf32")
    p1, p2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    err = max(nrel(j1, p1) * np.abs(p1).max(), np.abs(j2 - p2).max()) / max(np.abs(p1).max(), np.abs(p2).max())
    assert err < TF32_TOL


@pytest.mark.parametrize("method,prec", [("pnk", "tf32"), ("nk", "tf32"), ("pnk", "tf32x3"), ("pnk", "bf16x3")])
def test_mixed_solve_reaches_fp64_root(ctx, method, prec):
    s = synth.workload("o5v20_canonical")
    ref = json.load(open(GOLDEN))["o5v20_canonical"]["e_corr"]
    _, _, rep = gsys(ctx, s).solve(method, prec)
    assert rep["status_code"] == 0, rep
    assert rep["res_norm"] < 1e-8 and abs(rep["energy"] - ref) < 1e-8


def test_mixed_pnk_workload(ctx):
    s = synth.workload("o10v90_rotated")
    ref = json.load(open(GOLDEN))["o10v90_rotated"]["e_corr"]
    _, _, rep = gsys(ctx, s).solve("pnk", "tf32")
    assert rep["status_code"] == 0, rep
    assert abs(rep["energy"] - ref) < 1e-8


def test_jvp_directions_share_the_kept_staging(ctx):
    """Several JVPs at one point (cc_jvp_multi) keep the tensor-core staging of the fixed,
    value-side operands between directions; each result equals a JVP computed on its own
    (where every staged operand is gathered afresh) bit for bit, and the oracle's JVP within
    the three-pass bound. With the cache turned off the results are the same bits again."""
    o, v, naux = 4, 40, 24
    s = synth.make_system(o, v, naux, seed=33, gauge="haar")
    rng = np.random.default_rng(6)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    dirs = [synth.random_amplitudes(rng, o, v, 0.05, 0.05) for _ in range(3)]
    D1 = np.stack([d[0] for d in dirs])
    D2 = np.stack([d[1] for d in dirs])
    g = gsys(ctx, s)
    J1, J2 = g.jvp_multi(t1, t2, D1, D2, prec="tf32x3")
    for k, (d1, d2) in enumerate(dirs):
        j1, j2 = g.jvp(t1, t2, d1, d2, prec="tf32x3")
        assert np.array_equal(j1, J1[k]) and np.array_equal(j2, J2[k]), k
        p1, p2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
        scale = max(np.abs(p1).max(), np.abs(p2).max())
        assert max(np.abs(J1[k] - p1).max(), np.abs(J2[k] - p2).max()) < 1e-6 * scale
    ctx.set_option("stage_cache_bytes", 0)
    try:
        K1, K2 = g.jvp_multi(t1, t2, D1, D2, prec="tf32x3")
    finally:
        ctx.set_option("stage_cache_bytes", -1)
    assert np.array_equal(K1, J1) and np.array_equal(K2, J2)


def test_mixed_solve_is_the_same_with_and_without_kept_staging(ctx):
    s = synth.workload("o10v90_rotated")
    g = gsys(ctx, s)
    a1, a2, with_cache = g.solve("pnk", "tf32x3", af_direct=1)
    ctx.set_option("stage_cache_bytes", 0)
    try:
        b1, b2, without = g.solve("pnk", "tf32x3", af_direct=1)
    finally:
        ctx.set_option("stage_cache_bytes", -1)
    assert with_cache["status_code"] == 0 == without["status_code"]
    for k in ("newton_iters", "jvps", "krylov_iters", "residual_evals"):
        assert with_cache[k] == without[k], k
    assert with_cache["energy"] == without["energy"] and np.array_equal(a2, b2)


def test_mixed_jvp_error_table(ctx):
    """The error of each tensor-core precision's JVP against the FP64 oracle on the o=10, v=90
    workload at its MP2 start (normwise: max element error over max element). The table is
    written to $CCPNK_REPORT_DIR/jvp_error_table.json when that variable is set."""
    import os

    s = synth.workload("o10v90_rotated")
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    d1, d2 = synth.random_amplitudes(np.random.default_rng(4), o, v, 0.01, 0.01)
    p1, p2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    scale = max(np.abs(p1).max(), np.abs(p2).max())
    g = gsys(ctx, s)
    table = {}
    for prec, bound in (("tf32", 5e-3), ("bf16x3", 2e-5), ("tf32x3", 5e-6), ("df64", 1e-10), ("fp64emu", 1e-10),
                        ("fp64", 1e-10)):
        j1, j2 = g.jvp(t1, t2, d1, d2, prec=prec)
        err = max(np.abs(j1 - p1).max(), np.abs(j2 - p2).max()) / scale
        table[prec] = err
        assert err < bound, (prec, err)
    assert table["fp64"] < table["tf32x3"] < table["bf16x3"] < table["tf32"]
    out = os.environ.get("CCPNK_REPORT_DIR")
    if out:
        with open(os.path.join(out, "jvp_error_table.json"), "w") as fh:
            json.dump({"workload": "o10v90_rotated, MP2 start, random direction (scale 0.01)",
                       "normwise_error_vs_oracle": table}, fh, indent=1)


@pytest.mark.parametrize("prec", ["tf32x3", "fp64"])
def test_graph_replayed_jvps_give_the_same_solve(ctx, prec):
    """The JVPs of a PNK solve replayed from CUDA graphs of the tangent program (the default)
    give the same solve, bit for bit, as launching every kernel."""
    s = synth.workload("o10v90_rotated" if prec == "tf32x3" else "o5v20_canonical")
    g = gsys(ctx, s)
    runs = {}
    for graphs in (1, 0):
        ctx.set_option("graphs", graphs)
        n0 = ctx.launches
        t1, t2, rep = g.solve("pnk", prec, af_direct=1, outer_prec=5 if prec == "tf32x3" else 0)
        runs[graphs] = (t1, t2, rep, ctx.launches - n0)
    ctx.set_option("graphs", 1)
    (a1, a2, ra, na), (b1, b2, rb, nb) = runs[1], runs[0]
    assert ra["status_code"] == 0 == rb["status_code"]
    for k in ("newton_iters", "jvps", "krylov_iters", "residual_evals"):
        assert ra[k] == rb[k], k
    assert ra["energy"] == rb["energy"] and np.array_equal(a2, b2) and np.array_equal(a1, b1)
    assert na >= nb  # a replay counts every kernel node it runs
