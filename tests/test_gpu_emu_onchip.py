"""The two forms of the FP64 emulation's recombination (CC_OPT_EMU_ONCHIP) give the same bits.

On chip, each 128 x 128 tile of C runs all its (level, chunk) slice products on one SM and the
epilogue adds the exact chunk sums into 64-bit fixed-point sums in registers (the first group of
levels parked in TMEM while the second is summed). Through partial sums, every slice product is
written as FP32 and a combine pass adds the levels. Both form the same exact integers and round
once, at the conversion to FP64, so residuals and JVPs must agree bit for bit, at shapes where
levels span several chunks (long k: the ladder contraction over v^2) and where tiles are ragged,
and both meet the FP64 bound against the oracle.
"""
import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def ctx(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    c = ccpnk.Context(0)
    yield c
    c.close()


def run_both(ctx, fn):
    out = {}
    for mode in (1, 0):
        ctx.set_option("emu_onchip", mode)
        try:
            out[mode] = fn()
        finally:
            ctx.set_option("emu_onchip", -1)
    return out[1], out[0]


def same(a, b):
    return all(np.array_equal(np.asarray(x), np.asarray(y)) for x, y in zip(a, b))


@pytest.mark.parametrize("chunk", [64, 16])
def test_onchip_equals_partials_at_the_workload(ctx, chunk):
    """o=10 v=90 naux=300 near its MP2 start: the ladder contraction's k = 8100 makes level L
    span about 2 (L - 1) chunks of 64 k blocks (8 (L - 1) of 16)."""
    from paper_2608_06669_b300 import ccpnk

    s = synth.workload("o10v90_rotated")
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    rng = np.random.default_rng(12)
    p1, p2 = synth.random_amplitudes(rng, o, v, 0.01, 0.01)
    t1, t2 = t1 + p1, t2 + p2
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.01, 0.01)
    g = ccpnk.System.from_synth(ctx, s)
    ctx.set_option("emu_chunk", chunk)
    try:
        ra, rb = run_both(ctx, lambda: g.residual(t1, t2, prec="fp64emu"))
        ja, jb = run_both(ctx, lambda: g.jvp(t1, t2, d1, d2, prec="fp64emu"))
    finally:
        ctx.set_option("emu_chunk", 64)
    assert same(ra, rb) and same(ja, jb)
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert max(np.abs(ra[0] - q1).max(), np.abs(ra[1] - q2).max()) <= TOL64 * scale
    assert abs(ra[2] - eq) <= TOL64 * max(1.0, abs(eq))


@pytest.mark.parametrize("o,v,naux", [(3, 37, 7), (2, 270, 6)])
def test_onchip_equals_partials_ragged_and_large_v(ctx, o, v, naux):
    from paper_2608_06669_b300 import ccpnk

    s = synth.make_system(o, v, naux, seed=500 + v, gauge="haar")
    rng = np.random.default_rng(v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.05, 0.05)
    g = ccpnk.System.from_synth(ctx, s)
    ra, rb = run_both(ctx, lambda: g.residual(t1, t2, prec="fp64emu"))
    assert same(ra, rb)
    q1, q2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert max(np.abs(ra[0] - q1).max(), np.abs(ra[1] - q2).max()) <= TOL64 * scale


@pytest.mark.parametrize("bits", [54, 56])
def test_onchip_chunk_sums_at_their_bound(ctx, bits):
    """Every digit at its largest (63), or the leading one carried to 64 by the rounding: the
    on-chip sums stay exact and equal the native FP64 residual."""
    from paper_2608_06669_b300 import ccpnk

    o, v, naux = 1, 40, 640
    n = o + v
    fock = np.diag(np.concatenate([[-1.0], np.linspace(0.5, 2.0, v)]))
    B = np.full((naux, n, n), 1.0 - 2.0 ** -bits)
    g = ccpnk.System(ctx, o, v, naux, fock, B)
    _, t2 = synth.random_amplitudes(np.random.default_rng(5), o, v, 0.01, 0.01)
    t1 = np.zeros((o, v))
    ea, eb = run_both(ctx, lambda: g.residual(t1, t2, prec="fp64emu"))
    assert same(ea, eb)
    f1, f2, ef = g.residual(t1, t2, prec="fp64")
    scale = max(np.abs(f1).max(), np.abs(f2).max())
    assert max(np.abs(ea[0] - f1).max(), np.abs(ea[1] - f2).max()) <= 1e-12 * scale


def test_option_range(ctx):
    from paper_2608_06669_b300 import ccpnk

    for bad in (-2, 2):
        with pytest.raises(ccpnk.CCError):
            ctx.set_option("emu_onchip", bad)
