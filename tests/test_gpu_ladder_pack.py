"""The (c, d) split of the tensor-core particle-particle ladder (CC_OPT_LADDER_PACK).

With the split, the ladder's slab (ac|bd) leaves the build GEMM as plain FP32 words; one pass
forms W+ = W^cd + W^dc (c <= d) and W- = W^cd - W^dc (c < d) in staging layout, and the
contraction runs T+ (i <= j, c <= d) and T- (i < j, c < d) against them: half the MMA work of
the (c, d) contraction. The identity itself is checked in numpy on the CPU
(tests/test_ladder_algebra.py); here the GPU path with the split forced on is compared with
the oracle at the bounds of each precision, on shapes from the degenerate (v = 1: no c < d
pair; o = 1: no i < j pair) to the o=10 v=90 workload and the slab-capped v = 270, and a mixed
PNK solve with the split reaches the FP64 root.

Tolerances are those of the unsplit path: 5e-3 (TF32), 5e-6 (TF32x3), 2e-5 (BF16x3),
normwise. The split adds one FP32 rounding of W^cd + W^dc (2^-24 relative) before the
staging split, below the 2^-22 the three-pass splits keep.
"""
import json
import os

import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energies.json")
TOL = {"tf32": 5e-3, "tf32x3": 5e-6, "bf16x3": 2e-5}


def nerr(got, ref):
    scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
    return max(np.abs(got[0] - ref[0]).max(), np.abs(got[1] - ref[1]).max()) / scale


@pytest.fixture(scope="module")
def ctx(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    c = ccpnk.Context(0)
    c.set_option("ladder_pack", 1)
    yield c
    c.close()


def gsys(ctx, s):
    from paper_2608_06669_b300 import ccpnk

    return ccpnk.System.from_synth(ctx, s)


@pytest.mark.parametrize("prec", ["tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("o,v,naux,gauge", [(1, 1, 3, "canonical"), (3, 7, 5, "haar"), (1, 33, 9, "small"),
                                            (7, 33, 20, "haar"), (5, 70, 11, "small")])
def test_split_ladder_residual_and_jvp(ctx, prec, o, v, naux, gauge):
    s = synth.make_system(o, v, naux, seed=40 + o + v, gauge=gauge)
    rng = np.random.default_rng(o * 100 + v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    g = gsys(ctx, s)
    r1, r2, _ = g.residual(t1, t2, prec=prec)
    q1, q2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    assert nerr((r1, r2), (q1, q2)) < TOL[prec]
    j = g.jvp(t1, t2, d1, d2, prec=prec)
    p = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    assert nerr(j, p) < TOL[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_split_ladder_at_the_workload(ctx, prec):
    """The o=10 v=90 naux=300 workload at its MP2 start, a random direction."""
    s = synth.workload("o10v90_rotated")
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    d1, d2 = synth.random_amplitudes(np.random.default_rng(8), o, v, 0.01, 0.01)
    g = gsys(ctx, s)
    r1, r2, _ = g.residual(t1, t2, prec=prec)
    q1, q2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    assert nerr((r1, r2), (q1, q2)) < TOL[prec]
    j = g.jvp(t1, t2, d1, d2, prec=prec)
    p = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    assert nerr(j, p) < TOL[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("v", [180, 270])
def test_split_ladder_large_v(ctx, prec, v):
    """v = 270 runs the slab-capped blocking (13 values of a per block)."""
    o, naux = 3, 6
    s = synth.make_system(o, v, naux, seed=330 + v, gauge="haar")
    rng = np.random.default_rng(5 * v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    g = gsys(ctx, s)
    r1, r2, _ = g.residual(t1, t2, prec=prec)
    q1, q2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    assert nerr((r1, r2), (q1, q2)) < TOL[prec]
    j = g.jvp(t1, t2, d1, d2, prec=prec)
    p = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    assert nerr(j, p) < TOL[prec]


def test_split_and_unsplit_agree(ctx):
    """Same JVP with the split on and off, within the three-pass TF32 bound of each other."""
    o, v, naux = 6, 48, 14
    s = synth.make_system(o, v, naux, seed=61, gauge="haar")
    rng = np.random.default_rng(61)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    g = gsys(ctx, s)
    a = g.jvp(t1, t2, d1, d2, prec="tf32x3")
    ctx.set_option("ladder_pack", 0)
    try:
        b = g.jvp(t1, t2, d1, d2, prec="tf32x3")
    finally:
        ctx.set_option("ladder_pack", 1)
    assert nerr(a, b) < 2 * TOL["tf32x3"]
    assert not (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]))  # the split path ran


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_split_ladder_pnk_reaches_the_fp64_root(ctx, prec):
    """A mixed PNK solve of the o=10 v=90 workload with the split (JVPs replayed from graphs,
    FP64-emulated outer residual) lands on the oracle's root energy to 1e-8 Eh."""
    s = synth.workload("o10v90_rotated")
    ref = json.load(open(GOLDEN))["o10v90_rotated"]["e_corr"]
    _, _, rep = gsys(ctx, s).solve("pnk", prec, af_direct=1, outer_prec=5)
    assert rep["status_code"] == 0, rep
    assert rep["res_norm"] < 1e-8 and abs(rep["energy"] - ref) < 1e-8


def test_option_range(ctx):
    from paper_2608_06669_b300 import ccpnk

    for bad in (-2, 2):
        with pytest.raises(ccpnk.CCError):
            ctx.set_option("ladder_pack", bad)
    ctx.set_option("ladder_pack", 1)
