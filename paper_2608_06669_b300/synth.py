"""Seeded synthetic closed-shell Hamiltonians (inputs only).

This module builds the inputs that both the CUDA path and the CPU oracle consume:
a Fock matrix ``f`` (n x n, occupied orbitals first) and a density-fitting factor
``B`` (naux x n x n, symmetric in its two orbital indices) such that the
two-electron integrals are (pq|rs) = sum_P B[P,p,q] B[P,r,s].  It holds none of
the coupled-cluster arithmetic: no residual, energy, preconditioner or solver.

The value distributions follow the workloads the solver is benchmarked on:
orbital energies uniform in [-1.5, -0.5] Eh (occupied) and [0.3, 3.0] Eh
(virtual), B Gaussian with sigma = 0.05 scaled by exp(-0.1 |p - q|), naux = 3 n
where the workload says so.  Non-canonical gauges are produced by rotating f and
B with the same block-orthogonal U = diag(U_o, U_v), which changes the gauge of
one physical problem (the paper's "random gauge", App. A.2, restricted to
orthogonal U so that the overlap is the identity).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class System:
    """One closed-shell problem: o occupied and v virtual spatial orbitals."""

    o: int
    v: int
    naux: int
    fock: np.ndarray  # (n, n) float64, occupied first
    B: np.ndarray  # (naux, n, n) float64, B[P] symmetric
    eps: np.ndarray  # canonical orbital energies before any rotation
    U: np.ndarray  # (n, n) block-orthogonal rotation applied (identity if canonical)
    label: str = ""

    @property
    def n(self) -> int:
        return self.o + self.v


def orbital_energies(rng: np.random.Generator, o: int, v: int, gap: float | None = None) -> np.ndarray:
    """Occupied energies U[-1.5,-0.5], virtual U[0.3,3.0]; optionally shift the
    virtual block so that the HOMO-LUMO gap is exactly ``gap``."""
    eo = np.sort(rng.uniform(-1.5, -0.5, size=o))
    ev = np.sort(rng.uniform(0.3, 3.0, size=v))
    if gap is not None:
        ev = ev + (eo.max() + gap - ev.min())
    return np.concatenate([eo, ev])


def df_factor(rng: np.random.Generator, naux: int, n: int, sigma: float = 0.05, decay: float = 0.1) -> np.ndarray:
    """B[P,p,q]: Gaussian entries (sigma) times exp(-decay |p-q|); the upper
    triangle (p <= q) is drawn and mirrored, over the global orbital index."""
    B = np.zeros((naux, n, n))
    iu = np.triu_indices(n)
    scale = np.exp(-decay * np.abs(iu[0] - iu[1]))
    B[:, iu[0], iu[1]] = rng.normal(0.0, sigma, size=(naux, iu[0].size)) * scale
    B[:, iu[1], iu[0]] = B[:, iu[0], iu[1]]
    return B


def haar_orthogonal(rng: np.random.Generator, m: int) -> np.ndarray:
    """Haar-random orthogonal matrix: QR of a Gaussian with the sign fix."""
    if m == 0:
        return np.zeros((0, 0))
    Z = rng.normal(size=(m, m))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))


def _expm_antisym(K: np.ndarray) -> np.ndarray:
    """exp(K) for antisymmetric K via the eigendecomposition of the Hermitian iK."""
    if K.shape[0] == 0:
        return K.copy()
    w, V = np.linalg.eigh(1j * K)
    return (V @ np.diag(np.exp(-1j * w)) @ V.conj().T).real


def _rotate(eps: np.ndarray, B: np.ndarray, U: np.ndarray):
    f = U @ np.diag(eps) @ U.T
    Br = np.einsum("pr,Xrs,qs->Xpq", U, B, U, optimize=True)
    Br = 0.5 * (Br + Br.transpose(0, 2, 1))
    f = 0.5 * (f + f.T)
    return f, Br


def block_rotation(o: int, v: int, Uo: np.ndarray, Uv: np.ndarray) -> np.ndarray:
    n = o + v
    U = np.zeros((n, n))
    U[:o, :o] = Uo
    U[o:, o:] = Uv
    return U


def small_rotation(rng: np.random.Generator, o: int, v: int, eps: np.ndarray, max_offdiag: float) -> np.ndarray:
    """U_o = exp(s K_o), U_v = exp(s K_v) with K antisymmetric Gaussian; s is found
    by bisection so that the largest off-diagonal |f| after rotation is
    ``max_offdiag``."""
    Ko = rng.normal(size=(o, o))
    Ko = Ko - Ko.T
    Kv = rng.normal(size=(v, v))
    Kv = Kv - Kv.T
    F = np.diag(eps)

    def offdiag(s: float) -> float:
        U = block_rotation(o, v, _expm_antisym(s * Ko), _expm_antisym(s * Kv))
        fr = U @ F @ U.T
        return float(np.max(np.abs(fr - np.diag(np.diag(fr)))))

    lo, hi = 0.0, 1.0
    while offdiag(hi) < max_offdiag and hi < 1e3:
        hi *= 2.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if offdiag(mid) < max_offdiag:
            lo = mid
        else:
            hi = mid
    s = 0.5 * (lo + hi)
    return block_rotation(o, v, _expm_antisym(s * Ko), _expm_antisym(s * Kv))


def make_system(o: int, v: int, naux: int, seed: int, gauge: str = "canonical",
                max_offdiag: float = 0.1, gap: float | None = None, label: str = "") -> System:
    """gauge: 'canonical' (diagonal f), 'small' (exp of scaled antisymmetric
    generators, off-diagonal |f| up to ``max_offdiag``) or 'haar' (Haar-random
    orthogonal U_o, U_v mixing every occupied and every virtual orbital)."""
    rng = np.random.default_rng(seed)
    n = o + v
    eps = orbital_energies(rng, o, v, gap)
    B = df_factor(rng, naux, n)
    if gauge == "canonical":
        U = np.eye(n)
    elif gauge == "small":
        U = small_rotation(rng, o, v, eps, max_offdiag)
    elif gauge == "haar":
        U = block_rotation(o, v, haar_orthogonal(rng, o), haar_orthogonal(rng, v))
    else:
        raise ValueError(f"unknown gauge {gauge!r}")
    f, Br = _rotate(eps, B, U)
    return System(o=o, v=v, naux=naux, fock=f, B=Br, eps=eps, U=U, label=label)


def rotate_system(sys: System, U: np.ndarray) -> System:
    """The same physical problem in another orthogonal gauge: f -> U f U^T, B[P] -> U B[P] U^T."""
    f = U @ sys.fock @ U.T
    Br = np.einsum("pr,Xrs,qs->Xpq", U, sys.B, U, optimize=True)
    return System(o=sys.o, v=sys.v, naux=sys.naux, fock=0.5 * (f + f.T),
                  B=0.5 * (Br + Br.transpose(0, 2, 1)), eps=sys.eps, U=U @ sys.U, label=sys.label)


def random_amplitudes(rng: np.random.Generator, o: int, v: int, scale1: float = 0.05, scale2: float = 0.05):
    """Random (t1, t2) with the closed-shell symmetry t2[i,j,a,b] = t2[j,i,b,a]."""
    t1 = rng.normal(0.0, scale1, size=(o, v))
    t2 = rng.normal(0.0, scale2, size=(o, o, v, v))
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    return t1, t2


# ---------------------------------------------------------------------------
# The benchmark workloads (sizes, gauges and seeds fixed per workload).
# ---------------------------------------------------------------------------
WORKLOADS = {
    "o5v20_canonical": dict(o=5, v=20, naux=75, seed=1, gauge="canonical"),
    "o10v90_rotated": dict(o=10, v=90, naux=300, seed=2, gauge="small", max_offdiag=0.1),
    "o30v270_rotated": dict(o=30, v=270, naux=900, seed=3, gauge="small", max_offdiag=0.1),
    "o20v180_neardegenerate": dict(o=20, v=180, naux=600, seed=5, gauge="haar", gap=0.02),
}


def workload(name: str) -> System:
    kw = dict(WORKLOADS[name])
    return make_system(label=name, **kw)


def served_requests(n_requests: int = 256, seed: int = 4, mean_interval_s: float = 0.020):
    """The served mix: o ~ U{4..16}, v = round(o u) with u ~ U[6,9], naux = 3 (o + v);
    even requests canonical, odd ones Haar-rotated; exponential inter-arrival times.
    Returns a list of (arrival_time_s, System)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for r in range(n_requests):
        o = int(rng.integers(4, 17))
        v = int(round(o * rng.uniform(6.0, 9.0)))
        naux = 3 * (o + v)
        gauge = "canonical" if r % 2 == 0 else "haar"
        sys = make_system(o, v, naux, seed=1000 + r, gauge=gauge, label=f"req{r}")
        out.append((t, sys))
        t += float(rng.exponential(mean_interval_s))
    return out


def mixed_sizes(count: int, seed: int, o_range=(1, 4), v_range=(2, 9)):
    """Small ragged shapes for parity sweeps: (o, v, naux) triples."""
    rng = np.random.default_rng(seed)
    res = []
    for _ in range(count):
        o = int(rng.integers(o_range[0], o_range[1] + 1))
        v = int(rng.integers(v_range[0], v_range[1] + 1))
        res.append((o, v, int(rng.integers(1, 3 * (o + v) + 1))))
    return res


def fmt_bytes(x: float) -> str:
    for unit in ("B", "KB", "MB", "GB", "TB"):
        if abs(x) < 1024.0:
            return f"{x:.1f} {unit}"
        x /= 1024.0
    return f"{x:.1f} PB"


__all__ = ["System", "make_system", "rotate_system", "random_amplitudes", "workload", "WORKLOADS",
           "served_requests", "mixed_sizes", "haar_orthogonal", "block_rotation"]
