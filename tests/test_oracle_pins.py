"""Pins of the CPU oracle to things other than itself.

O1 (oracle/dfccsd.py) is checked against the definition written out in
determinant space (O0, oracle/fock_space.py), against FCI, against the closed
form of the MP2 energy, against the gauge covariance of the CC equations
(App. A.2 with orthogonal U), against the exactness of A_F when the
two-electron part vanishes (Eq. Commutator_AR), and against the polynomial
degree of the residual (the JVP stencil).  A dropped term, a wrong sign, a
swapped index pair or a transposed operand in O1 fails at least one of them.
"""
import numpy as np
import pytest

from oracle import dfccsd as cc
from oracle import fock_space as fs
from paper_2608_06669_b300 import synth

CASES = [
    (1, 3, 3, "canonical"),
    (2, 3, 4, "canonical"),
    (2, 3, 5, "haar"),
    (2, 4, 7, "small"),
    (3, 2, 3, "haar"),
    (3, 3, 1, "haar"),
]


def _norm(x):
    return float(np.max(np.abs(x)))


@pytest.mark.parametrize("o,v,naux,gauge", CASES)
def test_residual_matches_determinant_space(o, v, naux, gauge):
    """P1: every CCSD residual element and the energy equal the literal
    projection <Phi_mu| e^{-T} H e^{T} |Phi_0> (Eq. CC_ampl, Eq. CC_energy)."""
    s = synth.make_system(o, v, naux, seed=11 * o + v, gauge=gauge)
    rng = np.random.default_rng(5 + o + v)
    h, g = fs.integrals_from_df(s.fock, s.B, o)
    for scale in (0.05, 0.3):
        t1, t2 = synth.random_amplitudes(rng, o, v, scale, scale)
        r1a, r2a, ea = fs.cc_residual(h, g, o, t1, t2)
        r1b, r2b, eb = cc.residual(s.fock, s.B, o, t1, t2)
        ref = max(_norm(r1a), _norm(r2a), 1.0)
        assert _norm(r1a - r1b) <= 1e-12 * ref
        assert _norm(r2a - r2b) <= 1e-12 * ref
        assert abs(ea - eb) <= 1e-12 * max(1.0, abs(ea))


def test_residual_general_fock_with_ov_block():
    """P1 with a non-Hartree-Fock reference (f_ov != 0): the dressed Fock
    matrix carries every one-electron term."""
    o, v, naux = 2, 3, 4
    s = synth.make_system(o, v, naux, seed=3, gauge="haar")
    rng = np.random.default_rng(9)
    f = s.fock.copy()
    fov = rng.normal(0, 0.05, size=(o, v))
    f[:o, o:] = fov
    f[o:, :o] = fov.T
    h, g = fs.integrals_from_df(f, s.B, o)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.2, 0.2)
    r1a, r2a, ea = fs.cc_residual(h, g, o, t1, t2)
    r1b, r2b, eb = cc.residual(f, s.B, o, t1, t2)
    assert _norm(r1a - r1b) <= 1e-12
    assert _norm(r2a - r2b) <= 1e-12
    assert abs(ea - eb) <= 1e-12


def test_t1_dressing_is_the_similarity_transform():
    """e^{-T1} H e^{T1} has the integrals X h Y and (X B Y)(X B Y): the CCD
    projection with dressed integrals equals the CCSD projection (O0 on both
    sides, so the dressing formula is pinned independently of O1's terms)."""
    o, v, naux = 2, 3, 4
    s = synth.make_system(o, v, naux, seed=21, gauge="haar")
    rng = np.random.default_rng(2)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.2, 0.2)
    h, g = fs.integrals_from_df(s.fock, s.B, o)
    X, Y = cc.dressing_matrices(o, t1)
    Bt = np.einsum("pr,Xrs,sq->Xpq", X, s.B, Y)
    gt = np.einsum("Xpq,Xrs->pqrs", Bt, Bt)
    ht = X @ h @ Y
    r1a, r2a, ea = fs.cc_residual(h, g, o, t1, t2)
    r1b, r2b, _ = fs.cc_residual(ht, gt, o, np.zeros_like(t1), t2)
    assert _norm(r1a - r1b) <= 1e-12
    assert _norm(r2a - r2b) <= 1e-12


def test_ccsd_is_fci_for_two_electrons():
    """P2: with o = 1 CCSD is exact: E_ref + E_corr equals the lowest singlet
    eigenvalue of H in the full two-electron space."""
    o, v, naux = 1, 5, 6
    s = synth.make_system(o, v, naux, seed=4, gauge="haar")
    t1, t2, e, hist = cc.solve_fp_diis(s.fock, s.B, o, tol=1e-12, maxiter=300)
    assert hist[-1] < 1e-12
    h, g = fs.integrals_from_df(s.fock, s.B, o)
    e_ref = fs.reference_energy(h, g, o)
    evals = fs.fci_singlet_energies(h, g, o)
    assert abs((e_ref + e) - evals[0]) < 1e-10
    # and the reference energy is sum_k (h_kk + f_kk) for a closed shell
    assert abs(e_ref - (np.trace(h[:o, :o]) + np.trace(s.fock[:o, :o]))) < 1e-12


@pytest.mark.parametrize("gauge", ["canonical", "haar"])
def test_mp2_closed_form(gauge):
    """P3: R(0) = (ai|bj) with R1(0) = 0 (f_ov = 0), and the generalised MP2
    start A_F^{-1}(-R(0)) reproduces the closed-form MP2 energy
    sum (ia|jb)[2(ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b) in every gauge
    (Eq. inexact_newton_update at t = 0)."""
    o, v, naux = 3, 7, 9
    s = synth.make_system(o, v, naux, seed=8, gauge=gauge)
    r1, r2, e0 = cc.residual(s.fock, s.B, o, np.zeros((o, v)), np.zeros((o, o, v, v)))
    assert e0 == 0.0
    assert _norm(r1) < 1e-14
    # canonical integrals from the generator's own canonical factor
    U = s.U
    Bc = np.einsum("rp,Xrs,sq->Xpq", U, s.B, U)
    Bov = Bc[:, :o, o:]
    iajb = np.einsum("Xia,Xjb->iajb", Bov, Bov)
    e = s.eps
    den = e[:o, None, None, None] - e[None, o:, None, None] + e[None, None, :o, None] - e[None, None, None, o:]
    e_mp2 = float(np.sum(iajb * (2.0 * iajb - iajb.transpose(0, 3, 2, 1)) / den))
    t1, t2 = cc.mp2_guess(s.fock, s.B, o)
    assert abs(cc.energy(s.fock, s.B, o, t1, t2) - e_mp2) < 1e-12


def test_mp2_start_singles_closed_form():
    """P3 with a singles driving term: for a reference with f_ov != 0 the generalised MP2
    start's singles are the first-order amplitudes t_i^a = -f_ia / (eps_a - eps_i) in the
    canonical gauge (the closed form of A_F^{-1}(-R1(0)) with R1(0) = f_ov)."""
    o, v, naux = 3, 5, 6
    s = synth.make_system(o, v, naux, seed=41, gauge="canonical")
    fov = np.random.default_rng(2).normal(0, 0.05, size=(o, v))
    f = s.fock.copy()
    f[:o, o:] = fov
    f[o:, :o] = fov.T
    t1, t2 = cc.mp2_guess(f, s.B, o)
    e = np.diag(f)
    assert _norm(t1 + fov / (e[None, o:] - e[:o, None])) < 1e-15
    # the doubles are the closed-form first-order doubles, untouched by f_ov
    Bov = s.B[:, :o, o:]
    iajb = np.einsum("Xia,Xjb->iajb", Bov, Bov)
    D = e[None, None, o:, None] + e[None, None, None, o:] - e[:o, None, None, None] - e[None, :o, None, None]
    assert _norm(t2 + iajb.transpose(0, 2, 1, 3) / D) < 1e-14


def test_gauge_covariance():
    """P4: rotating the problem by U = diag(U_o, U_v) rotates the residual the
    same way, R(U t) = U R(t), and leaves the energy unchanged (the gauge
    invariance the NK family relies on)."""
    o, v, naux = 3, 6, 8
    s = synth.make_system(o, v, naux, seed=31, gauge="canonical")
    rng = np.random.default_rng(4)
    Uo, Uv = synth.haar_orthogonal(rng, o), synth.haar_orthogonal(rng, v)
    U = synth.block_rotation(o, v, Uo, Uv)
    sr = synth.rotate_system(s, U)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    r1, r2, e = cc.residual(s.fock, s.B, o, t1, t2)
    q1, q2 = cc.rotate_amplitudes(t1, t2, Uo, Uv)
    s1, s2, es = cc.residual(sr.fock, sr.B, o, q1, q2)
    p1, p2 = cc.rotate_amplitudes(r1, r2, Uo, Uv)
    assert _norm(s1 - p1) < 1e-12
    assert _norm(s2 - p2) < 1e-12
    assert abs(es - e) < 1e-12


def test_AF_is_the_jacobian_without_two_electron_part():
    """P5: with B = 0 and f_ov = 0, [[F,T],T] = 0, so R(t) = A_F t exactly
    (Eq. Commutator_AR); in the canonical gauge A_F is the diagonal
    denominator (Eq. Commutator_MO); and the eigenbasis inverse inverts A_F."""
    o, v, naux = 2, 4, 3
    s = synth.make_system(o, v, naux, seed=13, gauge="haar")
    rng = np.random.default_rng(3)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.3, 0.3)
    Bz = np.zeros_like(s.B)
    r1, r2, _ = cc.residual(s.fock, Bz, o, t1, t2)
    y1, y2 = cc.apply_AF(s.fock, o, t1, t2)
    assert _norm(r1 - y1) < 1e-14 and _norm(r2 - y2) < 1e-14
    # and O0 agrees for this one-body Hamiltonian
    h, g = fs.integrals_from_df(s.fock, Bz, o)
    q1, q2, _ = fs.cc_residual(h, g, o, t1, t2)
    assert _norm(q1 - y1) < 1e-13 and _norm(q2 - y2) < 1e-13
    # canonical: diagonal
    sc = synth.make_system(o, v, naux, seed=13, gauge="canonical")
    d = np.diag(sc.fock)
    D1 = d[None, o:] - d[:o, None]
    D2 = d[None, None, o:, None] + d[None, None, None, o:] - d[:o, None, None, None] - d[None, :o, None, None]
    z1, z2 = cc.apply_AF(sc.fock, o, t1, t2)
    assert _norm(z1 - D1 * t1) < 1e-14 and _norm(z2 - D2 * t2) < 1e-14
    # inverse (with and without a level shift, App. D)
    for shift in (0.0, 0.3):
        x1, x2 = cc.solve_AF(s.fock, o, t1, t2, shift)
        b1, b2 = cc.apply_AF(s.fock, o, x1, x2)
        assert _norm(b1 + shift * x1 - t1) < 1e-12 and _norm(b2 + shift * x2 - t2) < 1e-12


def test_jvp_stencil_is_exact():
    """P6: the residual is a polynomial of degree <= 4, so the five-point
    stencil gives J d for any step (two steps agree to rounding); with
    t1 = 0 and no singles direction the residual is quadratic along the line
    and the central difference is exact too; the forward difference of
    Eq. jacobian_vector_product_via_finite_difference converges at O(delta)."""
    o, v, naux = 2, 5, 6
    s = synth.make_system(o, v, naux, seed=17, gauge="haar")
    rng = np.random.default_rng(6)
    t1, t2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    d1, d2 = synth.random_amplitudes(rng, o, v, 0.1, 0.1)
    a1, a2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2, h=1.0)
    b1, b2 = cc.jvp(s.fock, s.B, o, t1, t2, d1, d2, h=0.1)
    scale = max(_norm(a1), _norm(a2))
    assert _norm(a1 - b1) < 1e-12 * scale and _norm(a2 - b2) < 1e-12 * scale
    # a quintic test function would break the stencil: check the residual's
    # degree directly by the fifth finite difference along the line
    vals = [cc.residual(s.fock, s.B, o, t1 + k * d1, t2 + k * d2)[1] for k in range(6)]
    fifth = vals[5] - 5 * vals[4] + 10 * vals[3] - 10 * vals[2] + 5 * vals[1] - vals[0]
    assert _norm(fifth) < 1e-11 * max(_norm(x) for x in vals)
    # central difference exact on the doubles-only line through t1 = 0
    z1 = np.zeros_like(t1)
    c1, c2 = cc.jvp(s.fock, s.B, o, z1, t2, z1, d2, h=1.0)
    h = 0.7
    rp = cc.residual(s.fock, s.B, o, z1, t2 + h * d2)
    rm = cc.residual(s.fock, s.B, o, z1, t2 - h * d2)
    assert _norm((rp[1] - rm[1]) / (2 * h) - c2) < 1e-12 * _norm(c2)
    # forward difference: error shrinks linearly with delta
    r0 = cc.residual(s.fock, s.B, o, t1, t2)
    errs = []
    for delta in (1e-3, 1e-4):
        rd = cc.residual(s.fock, s.B, o, t1 + delta * d1, t2 + delta * d2)
        errs.append(_norm((rd[1] - r0[1]) / delta - a2))
    assert errs[1] < 0.2 * errs[0]


@pytest.mark.parametrize("gauge", ["canonical", "haar"])
def test_paper_ccd_equations(gauge):
    """The paper's own CCD working equations (App. A.1), with the readings of its three
    misprints, equal the oracle's doubles residual at t1 = 0 in any gauge; the equations as
    printed do not (which is what makes the readings necessary)."""
    from oracle import ccd_paper

    o, v, naux = 3, 5, 6
    s = synth.make_system(o, v, naux, seed=4, gauge=gauge)
    _, t2 = synth.random_amplitudes(np.random.default_rng(1), o, v, 0.1, 0.1)
    _, r2, _ = cc.residual(s.fock, s.B, o, np.zeros((o, v)), t2)
    read = ccd_paper.ccd_residual(s.fock, s.B, o, t2)
    assert _norm(read - r2) < 1e-13 * _norm(r2)
    printed = ccd_paper.ccd_residual(s.fock, s.B, o, t2, literal=True)
    assert _norm(printed - r2) > 1e-4 * _norm(r2)


def test_residual_symmetry():
    """P7: R_ij^ab = R_ji^ba for symmetric amplitudes."""
    o, v, naux = 3, 5, 7
    s = synth.make_system(o, v, naux, seed=2, gauge="haar")
    t1, t2 = synth.random_amplitudes(np.random.default_rng(1), o, v, 0.2, 0.2)
    _, r2, _ = cc.residual(s.fock, s.B, o, t1, t2)
    assert _norm(r2 - r2.transpose(1, 0, 3, 2)) < 1e-14


def test_spectral_toy():
    """P8: the 2x2 example of the conclusion: diagonal entries 0.001 apart,
    eigenvalues about 20 apart (-8.9995, 11.0005), so a diagonal
    preconditioner misses the spectrum."""
    M = np.array([[1.0, 10.0], [10.0, 1.001]])
    w = np.linalg.eigvalsh(M)
    assert abs(w[0] - (-8.9995)) < 1e-4 and abs(w[1] - 11.0005) < 1e-4
    assert abs(M[0, 0] - M[1, 1]) == pytest.approx(0.001)


def test_fp_diis_reaches_root_of_small_workload():
    """The reference solver converges on the smallest workload, and the root
    is gauge invariant: the same problem solved in its eigenbasis gives the
    same energy."""
    s = synth.workload("o5v20_canonical")
    t1, t2, e, hist = cc.solve_fp_diis(s.fock, s.B, s.o, tol=1e-10, maxiter=100)
    assert hist[-1] < 1e-10
    rng = np.random.default_rng(12)
    U = synth.block_rotation(s.o, s.v, synth.haar_orthogonal(rng, s.o), synth.haar_orthogonal(rng, s.v))
    sr = synth.rotate_system(s, U)
    f, Bc, _ = cc.to_eigenbasis(sr.fock, sr.B, s.o)
    _, _, e2, hist2 = cc.solve_fp_diis(f, Bc, s.o, tol=1e-10, maxiter=100)
    assert hist2[-1] < 1e-10
    assert abs(e - e2) < 1e-10


@pytest.mark.parametrize("gauge", ["canonical", "haar"])
def test_residual_at_zero_amplitudes_is_the_driving_term(gauge):
    """At t = 0 every amplitude term of the projected equations vanishes: <Phi_i^a|H|Phi_0> =
    f_ia and <Phi_ij^ab|H|Phi_0> = (ia|jb), checked in determinant space (O0) and against the
    integrals built directly from B. The generalised MP2 start of the solvers relies on it."""
    o, v, naux = 2, 3, 4
    s = synth.make_system(o, v, naux, seed=31, gauge=gauge)
    z1, z2 = np.zeros((o, v)), np.zeros((o, o, v, v))
    r1, r2, e = cc.residual(s.fock, s.B, o, z1, z2)
    B = s.B
    g = np.einsum("Pia,Pjb->ijab", B[:, :o, o:], B[:, :o, o:])
    assert _norm(r1 - s.fock[:o, o:]) < 1e-14 and _norm(r2 - g) < 1e-14 and e == 0.0
    h, gi = fs.integrals_from_df(s.fock, s.B, o)
    q1, q2, _ = fs.cc_residual(h, gi, o, z1, z2)
    assert _norm(q2 - g) < 1e-12 and _norm(q1 - s.fock[:o, o:]) < 1e-12
