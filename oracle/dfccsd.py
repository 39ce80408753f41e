"""O1: closed-shell CCSD over density-fitted integrals, plain FP64 numpy.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module;
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use the oracle.

What it computes (the paper states the problem, Eqs. CC_ampl / CC_energy, and
works at the CCD level in its App. A; singles, the T1 dressing and density
fitting are not in the paper and follow the published closed-shell CCSD
equations in T1-similarity-transformed form: Koch, Sanchez de Meras, Helgaker
et al. 1994; Helgaker, Jorgensen, Olsen, "Molecular Electronic-Structure
Theory", ch. 13):

* integrals (pq|rs) = sum_P B[P,p,q] B[P,r,s]; f is the Fock matrix of the
  closed-shell reference, so h = f - sum_k [2 (pq|kk) - (pk|kq)];
* T1 dressing: with tt[a,i] = t1[i,a] (n x n, virtual-occupied block only),
  X = 1 - tt and Y = 1 + tt, every integral index is transformed as
  Bt[P] = X B[P] Y and ht = X h Y (this is e^{-T1} H e^{T1});
* the dressed Fock matrix Ft = ht + sum_k [2 gt_pqkk - gt_pkkq];
* the doubles residual is the CCD residual of the dressed Hamiltonian (terms
  A2..E2 below), the singles residual terms A1..D1;
* residual normalisation: R1[i,a] is the alpha-alpha singles projection and
  R2[i,j,a,b] the alpha-beta doubles projection of e^{-T} H e^{T}|Phi_0>
  (the coefficient of v_ij^ab in the paper's CCD residual of App. A.1 is 1,
  which is this projection); the brute-force module pins every term.

Array conventions: t1[i,a], t2[i,j,a,b] = t_ij^ab with t2[i,j,a,b] = t2[j,i,b,a];
u = 2 t2 - t2 with i,j swapped; the same layout for the residuals.

The Jacobian-vector product here is the exact directional derivative obtained
from the five-point central stencil: every CCSD residual is a polynomial of
degree <= 4 in the amplitudes, and that stencil differentiates such
polynomials exactly, so for any step h the only error is rounding.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# integrals and dressing
# --------------------------------------------------------------------------
def core_hamiltonian(fock: np.ndarray, B: np.ndarray, o: int) -> np.ndarray:
    """h = f - sum_k [2 (pq|kk) - (pk|kq)] from the DF factor."""
    gam = np.einsum("Xkk->X", B[:, :o, :o])
    J = np.einsum("Xpq,X->pq", B, gam)
    K = np.einsum("Xpk,Xkq->pq", B[:, :, :o], B[:, :o, :])
    return fock - (2.0 * J - K)


def dressing_matrices(o: int, t1: np.ndarray):
    """X = 1 - tt, Y = 1 + tt with tt[o+a, i] = t1[i, a]."""
    v = t1.shape[1]
    n = o + v
    tt = np.zeros((n, n))
    tt[o:, :o] = t1.T
    return np.eye(n) - tt, np.eye(n) + tt


def dressed(fock: np.ndarray, B: np.ndarray, o: int, t1: np.ndarray):
    """(Bt, Ft): T1-dressed DF factor and T1-dressed Fock matrix."""
    X, Y = dressing_matrices(o, t1)
    Bt = np.einsum("pr,Xrs,sq->Xpq", X, B, Y, optimize=True)
    ht = X @ core_hamiltonian(fock, B, o) @ Y
    gam = np.einsum("Xkk->X", Bt[:, :o, :o])
    Ft = ht + 2.0 * np.einsum("Xpq,X->pq", Bt, gam) - np.einsum("Xpk,Xkq->pq", Bt[:, :, :o], Bt[:, :o, :])
    return Bt, Ft


def _blk(Bt: np.ndarray, o: int, a: str, b: str) -> np.ndarray:
    sa = slice(0, o) if a == "o" else slice(o, None)
    sb = slice(0, o) if b == "o" else slice(o, None)
    return Bt[:, sa, sb]


def eri(Bt: np.ndarray, o: int, spec: str) -> np.ndarray:
    """A block of (pq|rs)~ = sum_P Bt[P,p,q] Bt[P,r,s]; spec like 'vovo'."""
    return np.einsum("Xpq,Xrs->pqrs", _blk(Bt, o, spec[0], spec[1]), _blk(Bt, o, spec[2], spec[3]),
                     optimize=True)


# --------------------------------------------------------------------------
# energy and residual
# --------------------------------------------------------------------------
def energy(fock: np.ndarray, B: np.ndarray, o: int, t1: np.ndarray, t2: np.ndarray) -> float:
    """Correlation energy, Eq. CC_energy minus the reference energy:
    E = sum (2 (ia|jb) - (ib|ja)) (t_ij^ab + t_i^a t_j^b) + 2 sum f_ia t_i^a."""
    g = eri(B, o, "ovov")  # g[i,a,j,b] = (ia|jb)
    tau = t2 + np.einsum("ia,jb->ijab", t1, t1)
    L = 2.0 * g - g.transpose(0, 3, 2, 1)
    return float(np.einsum("iajb,ijab->", L, tau) + 2.0 * np.einsum("ia,ia->", fock[:o, o:], t1))


def residual(fock: np.ndarray, B: np.ndarray, o: int, t1: np.ndarray, t2: np.ndarray):
    """(R1, R2, E) of closed-shell CCSD (Eq. CC_ampl projected on singles and
    doubles; Eq. CC_energy)."""
    Bt, Ft = dressed(fock, B, o, t1)
    Fov, Fvo, Foo, Fvv = Ft[:o, o:], Ft[o:, :o], Ft[:o, :o], Ft[o:, o:]
    u = 2.0 * t2 - t2.transpose(1, 0, 2, 3)

    g_vovo = eri(Bt, o, "vovo")
    g_oooo = eri(Bt, o, "oooo")
    g_ovov = eri(Bt, o, "ovov")  # undressed: the ov block of Bt equals that of B
    g_oovv = eri(Bt, o, "oovv")
    g_voov = eri(Bt, o, "voov")
    g_vvoo = eri(Bt, o, "vvoo")
    g_vvov = eri(Bt, o, "vvov")
    g_ooov = eri(Bt, o, "ooov")
    L_voov = 2.0 * g_voov - g_vvoo.transpose(0, 3, 2, 1)  # L_aikc = 2 g_aikc - g_acki
    L_ovov = 2.0 * g_ovov - g_ovov.transpose(0, 3, 2, 1)  # L_ldkc = 2 g_ldkc - g_lckd

    # singles
    R1 = np.einsum("kicd,adkc->ia", u, g_vvov, optimize=True)
    R1 -= np.einsum("klac,kilc->ia", u, g_ooov, optimize=True)
    R1 += np.einsum("ikac,kc->ia", u, Fov)
    R1 += Fvo.T

    # doubles: A2 (constant + particle-particle ladder)
    R2 = g_vovo.transpose(1, 3, 0, 2).copy()
    # sum_cd (ac|bd)~ t_ij^cd, one a at a time: with G_a[b, d, c] = (ac|bd)~ = sum_X Bt[X,b,d] Bt[X,a,c]
    # and t2 read as [ij, (d, c)], the sum over (d, c) is one matrix product (no permuted copies)
    Bvv = _blk(Bt, o, "v", "v")
    nv = Bvv.shape[1]
    Bflat = Bvv.reshape(Bvv.shape[0], nv * nv)                          # [X, (b, d)]
    t2_dc = np.ascontiguousarray(t2.transpose(0, 1, 3, 2)).reshape(o * o, nv * nv)  # [ij, (d, c)]
    for a in range(nv):
        G_a = (Bflat.T @ Bvv[:, a, :]).reshape(nv, nv * nv)           # [b, (d, c)] = (ac|bd)~
        R2[:, :, a, :] += (t2_dc @ G_a.T).reshape(o, o, nv)
    # B2 (hole ladder with its quadratic part)
    W = g_oooo + np.einsum("ijcd,kcld->kilj", t2, g_ovov, optimize=True)
    R2 += np.einsum("klab,kilj->ijab", t2, W, optimize=True)

    # C2, D2, E2, then the permutation P: X_ij^ab + X_ji^ba
    C = g_oovv - 0.5 * np.einsum("liad,kdlc->kiac", t2, g_ovov, optimize=True)  # C_kiac
    X = -0.5 * np.einsum("kjbc,kiac->ijab", t2, C, optimize=True)
    X -= np.einsum("kibc,kjac->ijab", t2, C, optimize=True)
    D = L_voov + 0.5 * np.einsum("ilad,ldkc->aikc", u, L_ovov, optimize=True)  # D_aikc
    X += 0.5 * np.einsum("jkbc,aikc->ijab", u, D, optimize=True)
    Gv = Fvv - np.einsum("klbd,ldkc->bc", u, g_ovov, optimize=True)
    Go = Foo + np.einsum("ljcd,kdlc->kj", u, g_ovov, optimize=True)
    X += np.einsum("ijac,bc->ijab", t2, Gv, optimize=True)
    X -= np.einsum("ikab,kj->ijab", t2, Go, optimize=True)
    R2 += X + X.transpose(1, 0, 3, 2)

    return R1, R2, energy(fock, B, o, t1, t2)


def jvp(fock, B, o, t1, t2, d1, d2, h: float = 1.0):
    """J(t) d exactly: [R(t-2hd) - 8R(t-hd) + 8R(t+hd) - R(t+2hd)] / (12h)."""
    def R(s):
        r1, r2, _ = residual(fock, B, o, t1 + s * h * d1, t2 + s * h * d2)
        return r1, r2
    m2, m1, p1, p2 = R(-2.0), R(-1.0), R(1.0), R(2.0)
    j1 = (m2[0] - 8.0 * m1[0] + 8.0 * p1[0] - p2[0]) / (12.0 * h)
    j2 = (m2[1] - 8.0 * m1[1] + 8.0 * p1[1] - p2[1]) / (12.0 * h)
    return j1, j2


# --------------------------------------------------------------------------
# the gauge-invariant Fock preconditioner A_F (Eq. Preconditioner, App. C)
# --------------------------------------------------------------------------
def apply_AF(fock: np.ndarray, o: int, x1: np.ndarray, x2: np.ndarray):
    """(A_F x): the occupied and virtual Fock blocks acting on every index,
    (A_F x)_ij^ab = sum_c (f_ac x_ij^cb + f_bc x_ij^ac) - sum_k (f_ki x_kj^ab + f_kj x_ik^ab),
    (A_F x)_i^a   = sum_c f_ac x_i^c - sum_k f_ki x_k^a.
    (App. C prints an overall factor 4 from an unnormalised projection; with the
    alpha-beta normalisation of the residual the factor is 1.)"""
    Foo, Fvv = fock[:o, :o], fock[o:, o:]
    y1 = x1 @ Fvv.T - Foo.T @ x1
    y2 = (np.einsum("ac,ijcb->ijab", Fvv, x2) + np.einsum("bc,ijac->ijab", Fvv, x2)
          - np.einsum("ki,kjab->ijab", Foo, x2) - np.einsum("kj,ikab->ijab", Foo, x2))
    return y1, y2


def solve_AF(fock: np.ndarray, o: int, b1: np.ndarray, b2: np.ndarray, shift: float = 0.0):
    """(A_F + shift I)^{-1} b exactly: rotate to the eigenbases of the occupied
    and virtual Fock blocks, divide by eps_a (+ eps_b) - eps_i (- eps_j) + shift,
    rotate back (A_F is a sum of commuting Kronecker terms)."""
    eo, Uo = np.linalg.eigh(fock[:o, :o])
    ev, Uv = np.linalg.eigh(fock[o:, o:])
    c1 = Uo.T @ b1 @ Uv
    c1 = c1 / (ev[None, :] - eo[:, None] + shift)
    c2 = np.einsum("ki,lj,klcd,ca,db->ijab", Uo, Uo, b2, Uv, Uv, optimize=True)
    D = ev[None, None, :, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, :, None, None]
    c2 = c2 / (D + shift)
    x1 = Uo @ c1 @ Uv.T
    x2 = np.einsum("ik,jl,klcd,ac,bd->ijab", Uo, Uo, c2, Uv, Uv, optimize=True)
    return x1, x2


def mp2_guess(fock, B, o):
    """Generalised MP2 start (Eq. inexact_newton_update at t = 0): t = A_F^{-1}(-R(0)), where
    R1(0)_i^a = f_ia (zero for a Hartree-Fock reference) and R2(0)_ij^ab = (ai|bj)."""
    v = fock.shape[0] - o
    r1, r2, _ = residual(fock, B, o, np.zeros((o, v)), np.zeros((o, o, v, v)))
    return solve_AF(fock, o, -r1, -r2)


# --------------------------------------------------------------------------
# the reference solver: fixed point with the diagonal denominator + DIIS
# --------------------------------------------------------------------------
def fp_diis_iterates(fock, B, o, t1=None, t2=None, shift=0.0, diis_size=8, diis_start=2, ccd=False):
    """The fixed-point + DIIS iteration one step at a time: t <- t - R(t) / (D + shift) with D
    the diagonal-Fock denominator (Eq. mo_fixed-point_update; App. D for the shift), Pulay DIIS
    on (t_new, t_new - t).  Yields (iteration, t1, t2, E, ||R||) at every iterate, before the
    update is taken; ccd=True solves CCD (t1 = 0, doubles projections only)."""
    v = fock.shape[0] - o
    if t1 is None:
        t1, t2 = mp2_guess(fock, B, o)
    fd = np.diag(fock)
    D1 = fd[None, o:] - fd[:o, None] + shift
    D2 = (fd[None, None, o:, None] + fd[None, None, None, o:] - fd[:o, None, None, None]
          - fd[None, :o, None, None] + shift)
    vecs, errs = [], []
    if ccd:
        t1 = np.zeros_like(t1)
    it = 0
    while True:
        r1, r2, e = residual(fock, B, o, t1, t2)
        if ccd:
            r1 = np.zeros_like(r1)
        rn = float(np.sqrt(np.sum(r1 * r1) + np.sum(r2 * r2)))
        yield it, t1, t2, e, rn
        n1 = t1 - r1 / D1
        n2 = t2 - r2 / D2
        vec = np.concatenate([n1.ravel(), n2.ravel()])
        err = vec - np.concatenate([t1.ravel(), t2.ravel()])
        vecs.append(vec)
        errs.append(err)
        if len(vecs) > diis_size:
            vecs.pop(0)
            errs.pop(0)
        if it >= diis_start and len(vecs) >= 2:
            m = len(vecs)
            Bm = -np.ones((m + 1, m + 1))
            Bm[m, m] = 0.0
            for a in range(m):
                for b in range(m):
                    Bm[a, b] = errs[a] @ errs[b]
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            c = np.linalg.lstsq(Bm, rhs, rcond=None)[0][:m]
            vec = sum(ci * vi for ci, vi in zip(c, vecs))
        t1 = vec[: o * v].reshape(o, v)
        t2 = vec[o * v:].reshape(o, o, v, v)
        t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
        it += 1


def solve_fp_diis(fock, B, o, t1=None, t2=None, tol=1e-10, maxiter=200, shift=0.0, diis_size=8,
                  diis_start=2, verbose=False, ccd=False, diverge_at=None, energies=None):
    """The reference solver: fp_diis_iterates until ||R|| < tol, at most maxiter residual
    evaluations (then one more at the last update).  diverge_at: stop as soon as ||R||
    exceeds it (or is not finite); energies: a list that receives E at every iterate.
    Returns (t1, t2, E, history of ||R||)."""
    hist = []
    steps = fp_diis_iterates(fock, B, o, t1, t2, shift=shift, diis_size=diis_size, diis_start=diis_start,
                             ccd=ccd)
    for it, t1, t2, e, rn in steps:
        hist.append(rn)
        if energies is not None:
            energies.append(e)
        if verbose:
            print(f"  fp+diis it {it:3d}  |R| {rn:.3e}  E {e:.12f}", flush=True)
        if rn < tol:
            return t1, t2, e, hist
        if diverge_at is not None and not (rn <= diverge_at):
            return t1, t2, e, hist
        if it + 1 >= maxiter:
            break
    _, t1, t2, e, _ = next(steps)
    return t1, t2, e, hist


def to_eigenbasis(fock, B, o):
    """The canonical gauge of the same problem: U = diag(U_o, U_v) from the
    eigenvectors of the occupied and virtual Fock blocks (f_ov = 0)."""
    n = fock.shape[0]
    _, Uo = np.linalg.eigh(fock[:o, :o])
    _, Uv = np.linalg.eigh(fock[o:, o:])
    U = np.zeros((n, n))
    U[:o, :o] = Uo
    U[o:, o:] = Uv
    f = U.T @ fock @ U
    Bc = np.einsum("rp,Xrs,sq->Xpq", U, B, U, optimize=True)
    return f, Bc, U


def rotate_amplitudes(t1, t2, Uo, Uv):
    """Amplitudes of the rotated problem: every occupied index by U_o, every
    virtual index by U_v (the covariance of App. A.2 with orthogonal U)."""
    r1 = Uo @ t1 @ Uv.T
    r2 = np.einsum("ik,jl,klcd,ac,bd->ijab", Uo, Uo, t2, Uv, Uv, optimize=True)
    return r1, r2
