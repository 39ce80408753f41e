"""The identities the particle-particle ladder kernels rely on, checked in numpy (CPU).

L_ij^ab = sum_cd V_{ac,bd} T_ij^cd with V_{ac,bd} = sum_P X_P,ac Y_P,bd, for V symmetric under
(a,c) <-> (b,d) and T_ij^cd = T_ji^dc:
- the half-triangle scheme: for a block of a, build and contract only b >= the block's first
  a; every other L_ij^ab is L_ji^ba (the mirror);
- the (c,d) split: L = sum_{c<=d} W+ T+ + sum_{c<d} W- T- with W+- = W^cd +- W^dc,
  T+- = (T^cd +- T^dc)/2 (diagonal: W^cc, T^cc), T+ symmetric and T- antisymmetric in (i,j),
  so the contraction runs over pairs i <= j only;
- the tangent's stacked factors: dV = sum_P (dX_ac X_bd + X_ac dX_bd) is the product of
  [dX; X] and [X; dX] stacked along P, and is again symmetric under (a,c) <-> (b,d).
"""
import numpy as np


def _sym_T(rng, o, v):
    t = rng.normal(size=(o, o, v, v))
    return 0.5 * (t + t.transpose(1, 0, 3, 2))


def _ladder(X, Y, T):
    V = np.einsum("Pac,Pbd->acbd", X, Y)
    return np.einsum("acbd,ijcd->ijab", V, T)


def test_half_triangle_with_mirror():
    rng = np.random.default_rng(0)
    o, v, P, blk = 3, 11, 5, 4
    X = rng.normal(size=(P, v, v))
    T = _sym_T(rng, o, v)
    full = _ladder(X, X, T)
    L = np.zeros_like(full)
    for a0 in range(0, v, blk):
        al = min(blk, v - a0)
        W = np.einsum("Pac,Pbd->abcd", X[:, a0:a0 + al], X[:, a0:])  # b >= a0 only
        L[:, :, a0:a0 + al, a0:] = np.einsum("abcd,ijcd->ijab", W, T)
    R = np.empty_like(full)
    for a in range(v):
        bs = (a // blk) * blk
        R[:, :, a, bs:] = L[:, :, a, bs:]
        R[:, :, a, :bs] = L.transpose(1, 0, 3, 2)[:, :, a, :bs]
    assert np.abs(R - full).max() < 1e-12 * np.abs(full).max()


def test_cd_split_over_pairs():
    rng = np.random.default_rng(1)
    o, v, P = 4, 7, 6
    X = rng.normal(size=(P, v, v))
    T = _sym_T(rng, o, v)
    full = _ladder(X, X, T)
    W = np.einsum("Pac,Pbd->abcd", X, X)
    iu_le, iu_lt = np.triu_indices(v), np.triu_indices(v, 1)
    io_le, io_lt = np.triu_indices(o), np.triu_indices(o, 1)
    Wd = W.transpose(0, 1, 3, 2)
    Wp = (W + Wd)[:, :, iu_le[0], iu_le[1]]
    diag = iu_le[0] == iu_le[1]
    Wp[:, :, diag] = W[:, :, iu_le[0][diag], iu_le[1][diag]]
    Wm = (W - Wd)[:, :, iu_lt[0], iu_lt[1]]
    Td = T.transpose(0, 1, 3, 2)
    Tp = (0.5 * (T + Td))[:, :, iu_le[0], iu_le[1]]
    Tp[:, :, diag] = T[:, :, iu_le[0][diag], iu_le[1][diag]]
    Tm = (0.5 * (T - Td))[:, :, iu_lt[0], iu_lt[1]]
    # symmetric / antisymmetric in (i, j): only i <= j (i < j) are contracted
    assert np.allclose(Tp, Tp.transpose(1, 0, 2)) and np.allclose(Tm, -Tm.transpose(1, 0, 2))
    Lp = np.einsum("abq,xq->xab", Wp, Tp[io_le[0], io_le[1]])
    Lm = np.einsum("abq,xq->xab", Wm, Tm[io_lt[0], io_lt[1]])
    L = np.zeros_like(full)
    for x, (i, j) in enumerate(zip(*io_le)):
        L[i, j] += Lp[x]
        if i != j:
            L[j, i] += Lp[x]
    for x, (i, j) in enumerate(zip(*io_lt)):
        L[i, j] += Lm[x]
        L[j, i] -= Lm[x]
    assert np.abs(L - full).max() < 1e-12 * np.abs(full).max()
    # half the multiply-adds of the unsplit (c, d) contraction, to leading order
    split = len(io_le[0]) * len(iu_le[0]) + len(io_lt[0]) * len(iu_lt[0])
    assert split < 0.75 * (o * o * v * v)


def test_tangent_factors_stack_symmetrically():
    rng = np.random.default_rng(2)
    o, v, P = 2, 6, 4
    X, dX = rng.normal(size=(P, v, v)), rng.normal(size=(P, v, v))
    T = _sym_T(rng, o, v)
    dV = np.einsum("Pac,Pbd->acbd", dX, X) + np.einsum("Pac,Pbd->acbd", X, dX)
    Xs, Ys = np.concatenate([dX, X]), np.concatenate([X, dX])
    Vs = np.einsum("Pac,Pbd->acbd", Xs, Ys)
    assert np.allclose(Vs, dV) and np.allclose(Vs, Vs.transpose(2, 3, 0, 1))
    # so the stacked pair goes through the same half-triangle ladder
    assert np.allclose(_ladder(Xs, Ys, T), np.einsum("acbd,ijcd->ijab", dV, T))
    # and the directional derivative of the ladder in X is exactly that term
    h = 1e-6
    fd = (_ladder(X + h * dX, X + h * dX, T) - _ladder(X - h * dX, X - h * dX, T)) / (2 * h)
    assert np.abs(fd - _ladder(Xs, Ys, T)).max() < 1e-6 * np.abs(fd).max()
