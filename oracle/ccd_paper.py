"""The paper's closed-shell CCD working equations (App. A.1, molecular-orbital form).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Written term by term from App. A.1 in its notation: v_pq^rs = <pq|rs> = (pr|qs), the
antisymmetrised w_ij^ab = 2 v_ij^ab - v_ij^ba, the intermediates g_i^k, g_c^a, J_ic^ak,
K_ic^ka and the permutation Omega_ij^ab(Z_ij^ab) = Z_ji^ba. Three places of the printed
text are read differently (the determinant-space definition decides; the pin tests show
that the printed forms disagree with it):
  * g_c^a = f_c^a - w_cd^kl t_kl^ad   (printed with +; the random-gauge form of App. A.2 has -)
  * K_ic^ka = v_ic^ka - 1/2 v_dc^kl t_il^da   (printed with +; App. A.2 has -)
  * the two K terms of the residual are K_ic^ka t_kj^cb and K_ic^kb t_kj^ac   (printed
    K_kc^ka and K_kc^kb, where the free index i is lost)
Integrals come from the DF factor, (pq|rs) = sum_P B_pq B_rs; t is t2[i,j,a,b] = t_ij^ab.
"""
from __future__ import annotations

import numpy as np


def physicist_integrals(B: np.ndarray) -> np.ndarray:
    """v[p,q,r,s] = <pq|rs> = (pr|qs)."""
    g = np.einsum("Xpq,Xrs->pqrs", B, B)
    return g.transpose(0, 2, 1, 3)


def ccd_residual(fock: np.ndarray, B: np.ndarray, o: int, t: np.ndarray, literal: bool = False) -> np.ndarray:
    """r_ij^ab(t) of App. A.1. literal=True uses the signs and indices exactly as printed."""
    v = physicist_integrals(B)
    w = 2.0 * v - v.transpose(0, 1, 3, 2)
    O, V = slice(0, o), slice(o, None)
    s_g = 1.0 if literal else -1.0
    s_k = 1.0 if literal else -1.0
    g_ik = fock[O, O] + np.einsum("klcd,ilcd->ik", w[O, O, V, V], t)
    g_ca = fock[V, V] + s_g * np.einsum("klcd,klad->ca", w[O, O, V, V], t)
    J = (v[O, V, V, O] - 0.5 * np.einsum("klcd,ilda->icak", v[O, O, V, V], t)
         + 0.5 * np.einsum("klcd,ilad->icak", w[O, O, V, V], t))
    K = v[O, V, O, V] + s_k * 0.5 * np.einsum("kldc,ilda->icka", v[O, O, V, V], t)
    r = v[O, O, V, V].copy()
    r += np.einsum("klij,klab->ijab", v[O, O, O, O], t)
    r += np.einsum("abcd,ijcd->ijab", v[V, V, V, V], t)
    r += np.einsum("klcd,ijcd,klab->ijab", v[O, O, V, V], t, t)
    X = np.einsum("ca,ijcb->ijab", g_ca, t) - np.einsum("ik,kjab->ijab", g_ik, t)
    X += np.einsum("icak,kjcb->ijab", J, 2.0 * t - t.transpose(0, 1, 3, 2))
    if literal:
        # K_kc^ka t_kj^cb and K_kc^kb t_kj^ac as printed: k repeated, nothing depends on i
        Kd = np.einsum("kcka->kca", K)
        X -= np.einsum("kca,kjcb->jab", Kd, t)[None]
        X -= np.einsum("kcb,kjac->jab", Kd, t)[None]
    else:
        X -= np.einsum("icka,kjcb->ijab", K, t)
        X -= np.einsum("ickb,kjac->ijab", K, t)
    return r + X + X.transpose(1, 0, 3, 2)
