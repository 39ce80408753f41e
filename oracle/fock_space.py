"""O0: coupled-cluster quantities by brute force in determinant space.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module;
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use the oracle.

This is the definition of the projective CC equations written out literally:
r_mu(t) = <Phi_mu| e^{-T} H e^{T} |Phi_0> (Eq. CC_ampl) and
E(t) = <Phi_0| e^{-T} H e^{T} |Phi_0> (Eq. CC_energy).  The N = 2o electron,
S_z = 0 sector of Fock space is enumerated explicitly (alpha string x beta string),
H = sum_pq h_pq E_pq + 1/2 sum_pqrs g_pqrs (E_pq E_rs - delta_qr E_ps) is applied as
sparse matrices, e^{+-T} by the terminating power series, and the result is
projected on the excited determinants.

Closed-shell conventions (the reading used throughout this project):
  T1 = sum_ai t1[i,a] E_ai,  T2 = 1/2 sum_aibj t2[i,j,a,b] E_ai E_bj,
  E_pq = a+_{p alpha} a_{q alpha} + a+_{p beta} a_{q beta};
  R1[i,a]     = < E^alpha_ai Phi_0 | e^{-T} H e^{T} Phi_0 >          (alpha-alpha singles)
  R2[i,j,a,b] = < E^alpha_ai E^beta_bj Phi_0 | e^{-T} H e^{T} Phi_0 > (alpha-beta doubles)
  E_corr      = < Phi_0 | e^{-T} H e^{T} Phi_0 > - < Phi_0 | H | Phi_0 >.

Sizes: C(n,o)^2 determinants (225 at o=2,v=4; 3136 at o=3,v=5), so this is for
tiny systems only.  The integrals h, g may be any real arrays: no permutational
symmetry is assumed beyond what the operator form above implies, which lets the
same code act on T1-similarity-transformed (non-Hermitian) integrals.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


class Sector:
    """The N = 2o, S_z = 0 determinant basis for n spatial orbitals."""

    def __init__(self, n: int, o: int):
        self.n, self.o = n, o
        self.strings = [sum(1 << p for p in occ) for occ in itertools.combinations(range(n), o)]
        self.index = {s: k for k, s in enumerate(self.strings)}
        self.ns = len(self.strings)
        self.dim = self.ns * self.ns
        self._E = {}

    def _string_excitation(self, p: int, q: int):
        """a+_p a_q on single-spin strings: (dst, src, sign) triples."""
        rows, cols, vals = [], [], []
        for k, s in enumerate(self.strings):
            if not (s >> q) & 1:
                continue
            s1 = s & ~(1 << q)
            if (s1 >> p) & 1:
                continue
            # sign: electrons passed by a_q, then by a+_p
            sgn = (-1) ** bin(s & ((1 << q) - 1)).count("1")
            sgn *= (-1) ** bin(s1 & ((1 << p) - 1)).count("1")
            s2 = s1 | (1 << p)
            rows.append(self.index[s2])
            cols.append(k)
            vals.append(float(sgn))
        return rows, cols, vals

    def E_spin(self, p: int, q: int, spin: str) -> sp.csr_matrix:
        """a+_{p sigma} a_{q sigma} on the sector.  Beta operators pass all o alpha
        electrons twice, so only the beta string decides the sign."""
        key = (p, q, spin)
        if key not in self._E:
            rows, cols, vals = self._string_excitation(p, q)
            ns = self.ns
            I = np.arange(ns)
            R, C, V = [], [], []
            for r, c, x in zip(rows, cols, vals):
                if spin == "a":
                    R.append(r * ns + I)
                    C.append(c * ns + I)
                else:
                    R.append(I * ns + r)
                    C.append(I * ns + c)
                V.append(np.full(ns, x))
            if R:
                M = sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                                  shape=(self.dim, self.dim))
            else:
                M = sp.csr_matrix((self.dim, self.dim))
            self._E[key] = M
        return self._E[key]

    def E(self, p: int, q: int) -> sp.csr_matrix:
        key = (p, q, "s")
        if key not in self._E:
            self._E[key] = (self.E_spin(p, q, "a") + self.E_spin(p, q, "b")).tocsr()
        return self._E[key]

    def reference(self) -> np.ndarray:
        ref = self.index[(1 << self.o) - 1]
        v = np.zeros(self.dim)
        v[ref * self.ns + ref] = 1.0
        return v


def apply_H(sec: Sector, h: np.ndarray, g: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """H psi with H = sum h_pq E_pq + 1/2 sum g_pqrs (E_pq E_rs - delta_qr E_ps)."""
    n = sec.n
    Epsi = np.stack([sec.E(p, q) @ psi for p in range(n) for q in range(n)])  # (n^2, dim)
    k = h - 0.5 * np.einsum("prrq->pq", g)
    out = k.reshape(-1) @ Epsi
    phi = g.reshape(n * n, n * n) @ Epsi  # phi[pq] = sum_rs g_pqrs E_rs psi
    for idx, (p, q) in enumerate(itertools.product(range(n), range(n))):
        out = out + 0.5 * (sec.E(p, q) @ phi[idx])
    return out


def hamiltonian_matrix(sec: Sector, h: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Dense H on the sector (small sectors only; used for FCI)."""
    cols = [apply_H(sec, h, g, e) for e in np.eye(sec.dim)]
    return np.array(cols).T


def apply_T(sec: Sector, o: int, t1: np.ndarray, t2: np.ndarray, psi: np.ndarray) -> np.ndarray:
    v = t1.shape[1]
    out = np.zeros_like(psi)
    for i in range(o):
        for a in range(v):
            if t1[i, a] != 0.0:
                out += t1[i, a] * (sec.E(o + a, i) @ psi)
    for j in range(o):
        for b in range(v):
            Ebj = sec.E(o + b, j) @ psi
            for i in range(o):
                for a in range(v):
                    c = t2[i, j, a, b]
                    if c != 0.0:
                        out += 0.5 * c * (sec.E(o + a, i) @ Ebj)
    return out


def apply_expT(sec: Sector, o: int, t1, t2, psi, sign: float = 1.0) -> np.ndarray:
    """e^{sign T} psi by the power series; T raises the excitation level, so the
    series ends after at most 2o + 1 terms."""
    out = psi.copy()
    term = psi.copy()
    for k in range(1, 2 * o + 2):
        term = sign * apply_T(sec, o, t1, t2, term) / k
        if not np.any(term):
            break
        out += term
    return out


def projections(sec: Sector, o: int, v: int, chi: np.ndarray):
    """(r1, r2, <Phi_0|chi>) of a sector vector chi."""
    ref = sec.reference()
    r1 = np.zeros((o, v))
    r2 = np.zeros((o, o, v, v))
    for i in range(o):
        for a in range(v):
            r1[i, a] = (sec.E_spin(o + a, i, "a") @ ref) @ chi
    for i in range(o):
        for a in range(v):
            ai = sec.E_spin(o + a, i, "a") @ ref
            for j in range(o):
                for b in range(v):
                    r2[i, j, a, b] = (sec.E_spin(o + b, j, "b") @ ai) @ chi
    return r1, r2, ref @ chi


def similarity_transformed(h, g, o, t1, t2, sec: Sector | None = None):
    """e^{-T} H e^{T} |Phi_0> as a sector vector."""
    n = h.shape[0]
    sec = sec or Sector(n, o)
    psi = apply_expT(sec, o, t1, t2, sec.reference(), +1.0)
    Hpsi = apply_H(sec, h, g, psi)
    return apply_expT(sec, o, t1, t2, Hpsi, -1.0), sec


def cc_residual(h, g, o, t1, t2):
    """(r1, r2, E_corr) of the projective CC equations (Eqs. CC_ampl, CC_energy)
    restricted to singles and doubles, for integrals h (n x n), g (n^4)."""
    n = h.shape[0]
    v = n - o
    chi, sec = similarity_transformed(h, g, o, t1, t2)
    r1, r2, e = projections(sec, o, v, chi)
    eref = sec.reference() @ apply_H(sec, h, g, sec.reference())
    return r1, r2, e - eref


def reference_energy(h, g, o):
    n = h.shape[0]
    sec = Sector(n, o)
    return sec.reference() @ apply_H(sec, h, g, sec.reference())


def integrals_from_df(fock: np.ndarray, B: np.ndarray, o: int):
    """h and g from the Fock matrix and the density-fitting factor:
    g_pqrs = sum_P B_pq^P B_rs^P and h = f - sum_k (2 g_pqkk - g_pkkq), so that f
    is the Fock matrix of the closed-shell reference determinant."""
    g = np.einsum("Xpq,Xrs->pqrs", B, B)
    occ = np.arange(o)
    G = 2.0 * np.einsum("pqkk->pq", g[:, :, occ][:, :, :, occ]) - np.einsum("pkkq->pq", g[:, occ][:, :, occ])
    return fock - G, g


def fci_singlet_energies(h, g, o):
    """Eigenvalues of H on the spin-flip-symmetric part of the sector (the
    singlets, for two electrons), ascending."""
    n = h.shape[0]
    sec = Sector(n, o)
    H = hamiltonian_matrix(sec, h, g)
    ns = sec.ns
    # string swap |A, B> -> |B, A>: the spin flip up to the global phase
    # (-1)^{o*o}; its +1 eigenspace holds the closed-shell reference, i.e. the
    # states whose total spin has the parity of S = 0 (for two electrons, the
    # singlets)
    perm = np.array([(k % ns) * ns + (k // ns) for k in range(sec.dim)])
    Pm = np.zeros((sec.dim, sec.dim))
    Pm[perm, np.arange(sec.dim)] = 1.0
    S = 0.5 * (np.eye(sec.dim) + Pm)
    w, V = np.linalg.eigh(S)
    basis = V[:, w > 0.5]
    Hs = basis.T @ H @ basis
    return np.sort(np.linalg.eigvals(Hs).real)


__all__ = ["Sector", "apply_H", "hamiltonian_matrix", "cc_residual", "reference_energy",
           "integrals_from_df", "fci_singlet_energies", "similarity_transformed"]
