"""Parity at the large virtual spaces of the o=20 v=180 and o=30 v=270 workloads.

The particle-particle ladder works on blocks of a whose (a, b, c, d) slab is capped at 2 GiB;
the cap binds for v above about 230 (19 values of a per block at v = 240 and 13 at v = 270,
against ceil(v / 8)), and the tensor-core contractions there run at tile and split-k shapes
that smaller cases never reach. Small o and naux keep the oracle's cost at seconds while the
v-dependent paths run at full size. The o=20 v=180 naux=600 workload itself is compared in
full (FP64 residual and energy per element), once.

Tolerances: 1e-10 normwise-elementwise for FP64 (and its tensor-core emulation), 2e-5 for the
three-pass BF16 split, and 5e-6 for the three-pass TF32 split: each product keeps all but about
3 * 2^-22 of its value (the dropped lo * lo term and the two splitting remainders), and the FP32
accumulation over the ladder's v^2 (about 3e4 to 7e4) terms adds to that; up to 1.9e-6 is
observed at v = 180.
"""
import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def nerr(got, ref):
    """max |got - ref| over max |ref| across the singles and doubles blocks together."""
    scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
    return max(np.abs(got[0] - ref[0]).max(), np.abs(got[1] - ref[1]).max()) / scale


@pytest.fixture(scope="module")
def ctx(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    c = ccpnk.Context(0)
    yield c
    c.close()


def gsys(ctx, s):
    from paper_2608_06669_b300 import ccpnk

    return ccpnk.System.from_synth(ctx, s)


def test_ladder_block_sizes_cover_the_capped_branch():
    """The shapes below exercise both branches of the ladder blocking: ceil(v / 8) values of a
    per block while the FP64 slab fits in 2 GiB, fewer once it does not."""
    cap = 2 * 1024 ** 3

    def block(v):
        return max(1, min((v + 7) // 8, cap // (8 * v ** 3)))

    assert block(180) == 23 == (180 + 7) // 8
    assert block(240) == 19 < (240 + 7) // 8
    assert block(270) == 13 < (270 + 7) // 8


@pytest.mark.parametrize("o,v,naux", [(2, 180, 8), (2, 240, 6), (2, 270, 6)])
def test_fp64_residual_large_v(ctx, o, v, naux):
    """FP64 and its tensor-core emulation (CC_FP64_EMU) at the FP64 bound."""
    s = synth.make_system(o, v, naux, seed=300 + v, gauge="haar")
    t1, t2 = synth.random_amplitudes(np.random.default_rng(v), o, v, 0.05, 0.05)
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    g = gsys(ctx, s)
    for prec in ("fp64", "fp64emu"):
        r1, r2, e = g.residual(t1, t2, prec=prec)
        assert nerr((r1, r2), (q1, q2)) <= TOL64, prec
        assert abs(e - eq) <= TOL64 * max(1.0, abs(eq))


@pytest.mark.parametrize("o,v,naux", [(1, 240, 4), (2, 270, 4)])
def test_fp64_jvp_large_v(ctx, o, v, naux):
    s = synth.make_system(o, v, naux, seed=310 + v, gauge="small")
    rng = np.random.default_rng(2 * v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    j = gsys(ctx, s).jvp(t1, t2, d1, d2)
    q = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    assert nerr(j, q) <= TOL64


@pytest.mark.parametrize("prec,tol", [("tf32x3", 5e-6), ("bf16x3", 2e-5)])
@pytest.mark.parametrize("v", [180, 270])
def test_mixed_residual_and_jvp_large_v(ctx, prec, tol, v):
    o, naux = 2, 6
    s = synth.make_system(o, v, naux, seed=320 + v, gauge="haar")
    rng = np.random.default_rng(3 * v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    g = gsys(ctx, s)
    r1, r2, _ = g.residual(t1, t2, prec=prec)
    q1, q2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    assert nerr((r1, r2), (q1, q2)) < tol
    j = g.jvp(t1, t2, d1, d2, prec=prec)
    p = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    assert nerr(j, p) < tol


def test_fp64_residual_near_degenerate_workload(ctx):
    """The o=20 v=180 naux=600 workload (gap 0.02 Eh, Haar gauge), full size, at random
    amplitudes of the size of its MP2 doubles, singles included: every element and the energy."""
    s = synth.workload("o20v180_neardegenerate")
    o, v = s.o, s.v
    t1, t2 = synth.random_amplitudes(np.random.default_rng(17), o, v, 0.01, 0.01)
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    g = gsys(ctx, s)
    for prec in ("fp64", "fp64emu"):
        r1, r2, e = g.residual(t1, t2, prec=prec)
        assert nerr((r1, r2), (q1, q2)) <= TOL64, prec
        assert abs(e - eq) <= TOL64 * max(1.0, abs(eq))


def test_spot_check_at_the_large_workload(ctx):
    """The o=30 v=270 naux=900 workload, full size: two capped PNK steps (mixed JVPs, FP64-emulated
    outer residual), then the oracle's residual and energy at the GPU's last iterate against the
    GPU's own residual there, native FP64 and emulated, element by element. (The workload has
    no root the reference solver reaches, so the check is made at the iterate.)"""
    s = synth.workload("o30v270_rotated")
    g = gsys(ctx, s)
    t1, t2, rep = g.solve("pnk", "tf32x3", af_direct=1, outer_prec=5, max_outer=2)
    assert rep["newton_iters"] == 2 and np.isfinite(rep["res_norm"])
    q1, q2, eq = cc.residual(s.fock, s.B, s.o, t1, t2)
    for prec in ("fp64emu", "fp64"):
        r1, r2, e = g.residual(t1, t2, prec=prec)
        assert nerr((r1, r2), (q1, q2)) <= TOL64, prec
        assert abs(e - eq) <= TOL64 * max(1.0, abs(eq)), prec
