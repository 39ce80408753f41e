"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the FP64 path must match the oracle per element to 1e-10 relative to the
largest oracle element (normwise-elementwise, since relative errors of elements near zero
mean nothing); converged correlation energies to 1e-8 Eh on every path.
"""
import json
import os

import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energies.json")
TOL64 = 1e-10


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def ctx(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    c = ccpnk.Context(0)
    yield c
    c.close()


def gpu_system(ctx, s):
    from paper_2608_06669_b300 import ccpnk

    return ccpnk.System.from_synth(ctx, s)


SHAPES = [
    (1, 1, 1, "canonical"),
    (1, 3, 2, "haar"),
    (2, 3, 4, "haar"),
    (3, 5, 7, "small"),
    (4, 9, 11, "haar"),
    (7, 33, 20, "haar"),   # ragged against the 64-wide tiles
    (5, 70, 40, "small"),  # v^2 spans several tiles with a tail
]


@pytest.mark.parametrize("o,v,naux,gauge", SHAPES)
def test_residual_parity(ctx, o, v, naux, gauge):
    s = synth.make_system(o, v, naux, seed=100 + o * v, gauge=gauge)
    t1, t2 = synth.random_amplitudes(np.random.default_rng(o + v), o, v, 0.1, 0.1)
    g = gpu_system(ctx, s)
    r1, r2, e = g.residual(t1, t2)
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r1 - q1).max() <= TOL64 * scale
    assert np.abs(r2 - q2).max() <= TOL64 * scale
    assert abs(e - eq) <= TOL64 * max(1.0, abs(eq))


def test_residual_parity_general_fock(ctx):
    """A non-Hartree-Fock reference (f_ov != 0) exercises every dressed-Fock term."""
    o, v, naux = 3, 6, 5
    s = synth.make_system(o, v, naux, seed=5, gauge="haar")
    rng = np.random.default_rng(2)
    fov = rng.normal(0, 0.05, size=(o, v))
    s.fock[:o, o:] = fov
    s.fock[o:, :o] = fov.T
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.2, 0.2)
    r1, r2, e = gpu_system(ctx, s).residual(t1, t2)
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r1 - q1).max() <= TOL64 * scale
    assert np.abs(r2 - q2).max() <= TOL64 * scale
    assert abs(e - eq) <= TOL64


@pytest.mark.parametrize("name", ["o5v20_canonical", "o10v90_rotated"])
def test_residual_parity_workload(ctx, name):
    """Full workload size at the MP2 start plus a random perturbation (singles included)."""
    s = synth.workload(name)
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    p1, p2 = synth.random_amplitudes(np.random.default_rng(3), o, v, 0.01, 0.01)
    t1, t2 = t1 + p1, t2 + p2
    r1, r2, e = gpu_system(ctx, s).residual(t1, t2)
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert rel_err(r1, q1) * np.abs(q1).max() <= TOL64 * scale
    assert np.abs(r2 - q2).max() <= TOL64 * scale
    assert abs(e - eq) <= TOL64 * max(1.0, abs(eq))


@pytest.mark.parametrize("name", ["o5v20_canonical", "o10v90_rotated"])
def test_double_float_residual_and_jvp_parity(ctx, name):
    """CC_DF64 (FP64 operands as FP32 pairs on the FP32 pipe) meets the FP64 bound."""
    s = synth.workload(name)
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    p1, p2 = synth.random_amplitudes(np.random.default_rng(8), o, v, 0.01, 0.01)
    t1, t2 = t1 + p1, t2 + p2
    g = gpu_system(ctx, s)
    r1, r2, e = g.residual(t1, t2, prec="df64")
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r1 - q1).max() <= TOL64 * scale and np.abs(r2 - q2).max() <= TOL64 * scale
    assert abs(e - eq) <= TOL64 * max(1.0, abs(eq))
    if name == "o5v20_canonical":
        d1, d2 = synth.random_amplitudes(np.random.default_rng(9), o, v, 0.01, 0.01)
        j1, j2 = g.jvp(t1, t2, d1, d2, prec="df64")
        k1, k2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
        scale = max(np.abs(k1).max(), np.abs(k2).max())
        assert np.abs(j1 - k1).max() <= TOL64 * scale and np.abs(j2 - k2).max() <= TOL64 * scale


def test_double_float_outer_residual_solve(ctx):
    s = synth.workload("o10v90_rotated")
    ref = _golden()["o10v90_rotated"]["e_corr"]
    _, _, rep = gpu_system(ctx, s).solve("pnk", "tf32x3", af_direct=1, outer_prec=4)
    assert rep["status_code"] == 0, rep
    assert abs(rep["energy"] - ref) < 1e-8


@pytest.mark.parametrize("o,v,naux,gauge", [(1, 2, 2, "haar"), (2, 4, 5, "haar"), (4, 9, 11, "small"),
                                             (7, 33, 20, "haar")])
def test_jvp_parity(ctx, o, v, naux, gauge):
    """The analytic JVP equals the exact stencil derivative of the oracle residual."""
    s = synth.make_system(o, v, naux, seed=7 + o, gauge=gauge)
    rng = np.random.default_rng(o * v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    j1, j2 = gpu_system(ctx, s).jvp(t1, t2, d1, d2)
    q1, q2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(j1 - q1).max() <= TOL64 * scale
    assert np.abs(j2 - q2).max() <= TOL64 * scale


def test_jvp_parity_workload(ctx):
    s = synth.workload("o10v90_rotated")
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    rng = np.random.default_rng(11)
    p1, _ = synth.random_amplitudes(rng, o, v, 0.01, 0.01)
    t1 = t1 + p1
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.01, 0.01)
    j1, j2 = gpu_system(ctx, s).jvp(t1, t2, d1, d2)
    q1, q2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(j1 - q1).max() <= TOL64 * scale
    assert np.abs(j2 - q2).max() <= TOL64 * scale


@pytest.mark.parametrize("o,v,gauge", [(1, 1, "canonical"), (3, 7, "haar"), (6, 40, "small")])
def test_AF_apply_and_inverse(ctx, o, v, gauge):
    s = synth.make_system(o, v, 4, seed=3, gauge=gauge)
    rng = np.random.default_rng(1)
    x1, x2 = synth.random_amplitudes(rng, o, v, 1.0, 1.0)
    g = gpu_system(ctx, s)
    y1, y2 = g.apply_AF(x1, x2, 0)
    q1, q2 = cc.apply_AF(s.fock, o, x1, x2)
    assert rel_err(y1, q1) <= TOL64 and rel_err(y2, q2) <= TOL64
    e1, e2 = cc.solve_AF(s.fock, o, x1, x2)
    for mode, tol in ((1, 1e-9), (2, 1e-10)):  # inner GMRES to 1e-12 relative; eigenbasis
        z1, z2 = g.apply_AF(x1, x2, mode)
        assert rel_err(z2, e2) <= tol and rel_err(z1, e1) <= tol


def test_host_and_device_pointers_agree(ctx):
    import torch

    s = synth.make_system(3, 8, 6, seed=9, gauge="haar")
    t1, t2 = synth.random_amplitudes(np.random.default_rng(0), 3, 8, 0.1, 0.1)
    g = gpu_system(ctx, s)
    r1, r2, e = g.residual(t1, t2)
    d1, d2, ed = g.residual(torch.from_numpy(t1).cuda(), torch.from_numpy(t2).cuda())
    assert d2.is_cuda
    assert np.array_equal(r2, d2.cpu().numpy()) and np.array_equal(r1, d1.cpu().numpy()) and e == ed


def test_invalid_inputs_are_rejected(ctx):
    from paper_2608_06669_b300 import ccpnk

    s = synth.make_system(2, 3, 2, seed=1)
    B = s.B.copy()
    B[0, 0, 1] += 1e-3
    with pytest.raises(ccpnk.CCError) as ei:
        ccpnk.System(ctx, 2, 3, 2, s.fock, B)
    assert ei.value.status == -1
    with pytest.raises(ccpnk.CCError):
        ccpnk.System(ctx, 0, 3, 2, s.fock, s.B)
    g = gpu_system(ctx, s)
    with pytest.raises(ccpnk.CCError):
        g.residual(np.zeros((2, 3)), np.zeros((2, 2, 3, 3)), prec=9)


def _golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


@pytest.mark.parametrize("method", ["fp_diis", "pnk", "nk", "ink"])
def test_solvers_reach_the_oracle_root(ctx, method):
    s = synth.workload("o5v20_canonical")
    ref = _golden()["o5v20_canonical"]["e_corr"]
    g = gpu_system(ctx, s)
    kw = {"max_outer": 400} if method == "fp_diis" else {}
    t1, t2, rep = g.solve(method, "fp64", **kw)
    assert rep["status_code"] == 0, rep
    assert rep["res_norm"] < 1e-8
    assert abs(rep["energy"] - ref) < 1e-8
    # the returned amplitudes are the root: the oracle residual vanishes there
    q1, q2, eq = cc.residual(s.fock, s.B, s.o, t1, t2)
    assert np.sqrt((q1 ** 2).sum() + (q2 ** 2).sum()) < 1e-8
    assert abs(eq - rep["energy"]) < 1e-10


@pytest.mark.parametrize("method", ["pnk", "fp_diis"])
def test_ccd_mode_reaches_the_paper_ccd_root(ctx, method):
    """CCD (the paper's level of theory): the GPU root is a root of the paper's own CCD
    working equations (App. A.1, with the readings of its misprints) and its energy equals
    the oracle's CCD solve."""
    from oracle import ccd_paper

    s = synth.workload("o5v20_canonical")
    _, q2, e_ref, hist = cc.solve_fp_diis(s.fock, s.B, s.o, tol=1e-11, maxiter=300, ccd=True)
    assert hist[-1] < 1e-11
    t1, t2, rep = gpu_system(ctx, s).solve(method, "fp64", ccd=1, max_outer=400)
    assert rep["status_code"] == 0, rep
    assert np.all(t1 == 0.0)
    assert abs(rep["energy"] - e_ref) < 1e-8
    r = ccd_paper.ccd_residual(s.fock, s.B, s.o, t2)
    assert np.sqrt((r ** 2).sum()) < 1e-8


def test_pnk_is_gauge_invariant(ctx):
    """The same problem in a Haar-rotated gauge: PNK lands on the same energy (App. A.2)."""
    s = synth.workload("o5v20_canonical")
    rng = np.random.default_rng(5)
    U = synth.block_rotation(s.o, s.v, synth.haar_orthogonal(rng, s.o), synth.haar_orthogonal(rng, s.v))
    sr = synth.rotate_system(s, U)
    ref = _golden()["o5v20_canonical"]["e_corr"]
    _, _, rep = gpu_system(ctx, sr).solve("pnk", "fp64")
    assert rep["status_code"] == 0 and abs(rep["energy"] - ref) < 1e-8


def test_pnk_fp64_workload(ctx):
    s = synth.workload("o10v90_rotated")
    ref = _golden()["o10v90_rotated"]["e_corr"]
    t1, t2, rep = gpu_system(ctx, s).solve("pnk", "fp64")
    assert rep["status_code"] == 0, rep
    assert abs(rep["energy"] - ref) < 1e-8


def test_kernel_timer_levels(ctx):
    """Level 1 times only the ladder GEMMs; level 2 also names every other contraction by its
    index labels. Timing does not change the result."""
    s = synth.make_system(3, 9, 10, seed=21, gauge="haar")
    g = gpu_system(ctx, s)
    t1, t2 = synth.random_amplitudes(np.random.default_rng(2), 3, 9, 0.1, 0.1)
    r1, r2, e = g.residual(t1, t2)
    ctx.profile(True)
    g.residual(t1, t2)
    lvl1 = ctx.profile_list()
    ctx.profile(True, all_contractions=True)
    q1, q2, eq = g.residual(t1, t2)
    lvl2 = ctx.profile_list()
    ctx.profile(False)
    assert set(lvl1) == {"ladder_build.fp64", "ladder_contract.fp64"}
    assert set(lvl1) < set(lvl2) and any(k.endswith(".f64") and ">" in k for k in lvl2)
    assert all(n >= 1 and ms >= 0.0 for n, ms, _ in lvl2.values())
    assert np.array_equal(r2, q2) and np.array_equal(r1, q1) and e == eq


@pytest.mark.parametrize("name,shift", [("o5v20_canonical", 0.2), ("o10v90_rotated", 0.2)])
def test_level_shifted_fp_diis_reaches_the_oracle_root(ctx, name, shift):
    """FP + DIIS with the level shift of App. D (every denominator D + shift) lands on the
    oracle's root, and its amplitudes zero the oracle residual."""
    s = synth.workload(name)
    ref = _golden()[name]["e_corr"]
    t1, t2, rep = gpu_system(ctx, s).solve("fp_diis", "fp64", level_shift=shift, max_outer=500)
    assert rep["status_code"] == 0, rep
    assert abs(rep["energy"] - ref) < 1e-8
    if name == "o5v20_canonical":
        q1, q2, eq = cc.residual(s.fock, s.B, s.o, t1, t2)
        assert np.sqrt((q1 ** 2).sum() + (q2 ** 2).sum()) < 1e-8 and abs(eq - rep["energy"]) < 1e-10


def test_mp2_start_with_singles_driving_term(ctx):
    """A non-Hartree-Fock reference (f_ov != 0): the generalised MP2 start is the inexact
    Newton step at t = 0 (Eq. inexact_newton_update), t = A_F^{-1}(-R(0)) with R1(0) = f_ov,
    singles included. max_outer = 0 returns the start itself."""
    o, v, naux = 3, 9, 8
    s = synth.make_system(o, v, naux, seed=12, gauge="haar")
    fov = np.random.default_rng(4).normal(0, 0.05, size=(o, v))
    s.fock[:o, o:] = fov
    s.fock[o:, :o] = fov.T
    t1, t2, rep = gpu_system(ctx, s).solve("pnk", "fp64", af_direct=1, max_outer=0)
    q1, q2 = cc.mp2_guess(s.fock, s.B, o)
    assert np.abs(q1).max() > 1e-3
    assert rel_err(t1, q1) <= TOL64 and rel_err(t2, q2) <= TOL64


@pytest.mark.parametrize("o,v,naux,gauge", [(1, 1, 1, "canonical"), (2, 3, 4, "haar"), (4, 9, 11, "haar"),
                                             (7, 33, 20, "haar"), (5, 70, 40, "small")])
def test_fp64_emulated_residual_and_jvp_parity(ctx, o, v, naux, gauge):
    """CC_FP64_EMU (Ozaki slices on the tensor cores, exact FP32 chunk sums, integer recombination)
    meets the FP64 bound element by element, on the residual and on the JVP."""
    s = synth.make_system(o, v, naux, seed=200 + o * v, gauge=gauge)
    rng = np.random.default_rng(o + 2 * v)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    g = gpu_system(ctx, s)
    r1, r2, e = g.residual(t1, t2, prec="fp64emu")
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r1 - q1).max() <= TOL64 * scale and np.abs(r2 - q2).max() <= TOL64 * scale
    assert abs(e - eq) <= TOL64 * max(1.0, abs(eq))
    j1, j2 = g.jvp(t1, t2, d1, d2, prec="fp64emu")
    p1, p2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2)
    scale = max(np.abs(p1).max(), np.abs(p2).max())
    assert np.abs(j1 - p1).max() <= TOL64 * scale and np.abs(j2 - p2).max() <= TOL64 * scale


@pytest.mark.parametrize("chunk", [16, 64, 1])
def test_fp64_emulated_workload_residual(ctx, chunk):
    """The o=10 v=90 workload; the exact chunks of the emulation summing 64 (the default: sums up
    to just below 2^24), 16 or 1 k block of 64 products each."""
    s = synth.workload("o10v90_rotated")
    o, v = s.o, s.v
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    p1, p2 = synth.random_amplitudes(np.random.default_rng(3), o, v, 0.01, 0.01)
    t1, t2 = t1 + p1, t2 + p2
    ctx.set_option("emu_chunk", chunk)
    try:
        r1, r2, e = gpu_system(ctx, s).residual(t1, t2, prec="fp64emu")
    finally:
        ctx.set_option("emu_chunk", 64)
    q1, q2, eq = cc.residual(s.fock, s.B, o, t1, t2)
    scale = max(np.abs(q1).max(), np.abs(q2).max())
    assert np.abs(r1 - q1).max() <= TOL64 * scale and np.abs(r2 - q2).max() <= TOL64 * scale
    assert abs(e - eq) <= TOL64 * max(1.0, abs(eq))


@pytest.mark.parametrize("prec", ["fp64emu", "tf32x3"])
def test_pnk_with_emulated_outer_residual(ctx, prec):
    """PNK with the outer residual (convergence test, energy) in CC_FP64_EMU lands on the oracle
    root within 1e-8 Eh, and its amplitudes zero the oracle residual."""
    for name in ("o5v20_canonical", "o10v90_rotated"):
        s = synth.workload(name)
        ref = _golden()[name]["e_corr"]
        t1, t2, rep = gpu_system(ctx, s).solve("pnk", prec, af_direct=1, outer_prec=5)
        assert rep["status_code"] == 0, (name, rep)
        assert abs(rep["energy"] - ref) < 1e-8, name
        if name == "o5v20_canonical":
            q1, q2, eq = cc.residual(s.fock, s.B, s.o, t1, t2)
            assert np.sqrt((q1 ** 2).sum() + (q2 ** 2).sum()) < 1e-8 and abs(eq - rep["energy"]) < 1e-10



@pytest.mark.parametrize("chunk", [16, 64])
@pytest.mark.parametrize("bits", [54, 56])
def test_fp64_emulation_chunk_sums_at_their_bound(ctx, chunk, bits):
    """Worst cases for the exactness of the emulation's FP32 chunk sums. With every entry of B
    equal to 1 - 2^-54, every digit slice of the ladder build's operands holds the largest digit
    (63: nine slices of six bits) and a chunk of 64 (or 16) k blocks sums 4096 (1024) products
    63 * 63 = 16,257,024 (4,064,256), just below 2^24 (2^22). With 1 - 2^-56 the rounding to 54
    bits carries into the leading digit (64, the rest 0): the leading level's chunk sums reach
    4096 * 64 * 64 = 2^24 exactly. The emulated residual must still equal the native FP64 one."""
    from paper_2608_06669_b300 import ccpnk

    o, v, naux = 1, 40, 640
    n = o + v
    fock = np.diag(np.concatenate([[-1.0], np.linspace(0.5, 2.0, v)]))
    B = np.full((naux, n, n), 1.0 - 2.0 ** -bits)
    g = ccpnk.System(ctx, o, v, naux, fock, B)
    # t1 = 0 leaves the dressed factor equal to B, so the ladder build's operands keep the digits
    _, t2 = synth.random_amplitudes(np.random.default_rng(5), o, v, 0.01, 0.01)
    t1 = np.zeros((o, v))
    ctx.set_option("emu_chunk", chunk)
    try:
        e1, e2, ee = g.residual(t1, t2, prec="fp64emu")
    finally:
        ctx.set_option("emu_chunk", 64)
    f1, f2, ef = g.residual(t1, t2, prec="fp64")
    scale = max(np.abs(f1).max(), np.abs(f2).max())
    assert max(np.abs(e1 - f1).max(), np.abs(e2 - f2).max()) <= 1e-12 * scale
    assert abs(ee - ef) <= 1e-12 * max(1.0, abs(ef))
