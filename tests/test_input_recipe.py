"""The seeded synthetic inputs follow their stated recipe (CPU).

The workloads stand in for the paper's molecules, so their construction is checked directly:
orbital-energy ranges, the symmetric density-fitting factor with its exp(-0.1|p-q|) envelope,
gauges that are block-orthogonal changes of one problem (the Fock spectrum per block is kept),
the 0.1 Eh bound on off-diagonal Fock elements of the 'small' gauge, the 0.02 Eh gap of the
near-degenerate workload, the sizes of the named workloads and of the served mix, and seeding.
"""
import numpy as np
import pytest

from paper_2608_06669_b300 import synth


def test_orbital_energy_ranges_and_gap():
    e = synth.orbital_energies(np.random.default_rng(0), 7, 30)
    assert np.all((e[:7] >= -1.5) & (e[:7] <= -0.5)) and np.all((e[7:] >= 0.3) & (e[7:] <= 3.0))
    g = synth.orbital_energies(np.random.default_rng(0), 7, 30, gap=0.02)
    assert abs(g[7:].min() - g[:7].max() - 0.02) < 1e-14
    assert np.array_equal(g[:7], e[:7])


def test_df_factor_symmetry_and_envelope():
    n, naux = 40, 400
    B = synth.df_factor(np.random.default_rng(1), naux, n)
    assert np.array_equal(B, B.transpose(0, 2, 1))
    p, q = np.indices((n, n))
    # per-pair standard deviation over P against sigma exp(-0.1 |p - q|), for |p - q| <= 10
    sd = B.std(axis=0)
    env = 0.05 * np.exp(-0.1 * np.abs(p - q))
    near = np.abs(p - q) <= 10
    ratio = sd[near] / env[near]
    assert 0.85 < ratio.mean() < 1.15


@pytest.mark.parametrize("gauge", ["canonical", "small", "haar"])
def test_gauges_are_block_orthogonal_changes_of_one_problem(gauge):
    o, v, naux = 4, 11, 12
    s = synth.make_system(o, v, naux, seed=3, gauge=gauge)
    U = s.U
    assert np.allclose(U @ U.T, np.eye(o + v), atol=1e-12)
    assert np.abs(U[:o, o:]).max() == 0.0 and np.abs(U[o:, :o]).max() == 0.0
    f = s.fock
    assert np.allclose(f, f.T, atol=1e-14) and np.abs(f[:o, o:]).max() < 1e-12
    assert np.allclose(np.linalg.eigvalsh(f[:o, :o]), np.sort(s.eps[:o]), atol=1e-12)
    assert np.allclose(np.linalg.eigvalsh(f[o:, o:]), np.sort(s.eps[o:]), atol=1e-12)
    assert np.allclose(s.B, s.B.transpose(0, 2, 1), atol=1e-15)
    # (pq|rs) of the rotated problem is the rotated (pq|rs) of the canonical one
    c = synth.make_system(o, v, naux, seed=3, gauge="canonical")
    if gauge != "canonical":
        back = synth.rotate_system(s, s.U.T @ np.eye(o + v))
        assert np.allclose(back.fock, np.diag(c.eps), atol=1e-12)


def test_small_gauge_offdiagonal_bound():
    s = synth.make_system(6, 30, 20, seed=4, gauge="small", max_offdiag=0.1)
    off = s.fock - np.diag(np.diag(s.fock))
    assert abs(np.abs(off).max() - 0.1) < 1e-6


def test_named_workload_shapes():
    shapes = {k: (w["o"], w["v"], w["naux"]) for k, w in synth.WORKLOADS.items()}
    assert shapes == {"o5v20_canonical": (5, 20, 75), "o10v90_rotated": (10, 90, 300),
                      "o30v270_rotated": (30, 270, 900), "o20v180_neardegenerate": (20, 180, 600)}
    for k, (o, v, naux) in shapes.items():
        assert naux == 3 * (o + v)
    s = synth.workload("o5v20_canonical")
    assert np.allclose(s.fock, np.diag(np.diag(s.fock)))


def test_served_mix_recipe_and_seeding():
    reqs = synth.served_requests(16)
    times = np.array([t for t, _ in reqs])
    assert times[0] == 0.0 and np.all(np.diff(times) >= 0.0)
    assert 0.005 < np.diff(times).mean() < 0.060  # exponential gaps, mean 20 ms (15 draws)
    for r, (_, s) in enumerate(reqs):
        assert 4 <= s.o <= 16 and 6 * s.o - 0.5 <= s.v <= 9 * s.o + 0.5 and s.naux == 3 * (s.o + s.v)
        assert (np.abs(s.fock - np.diag(np.diag(s.fock))).max() == 0.0) == (r % 2 == 0)
    again = synth.served_requests(16)
    assert all(a[0] == b[0] and np.array_equal(a[1].B, b[1].B) for a, b in zip(reqs, again))
