"""Failure detection, made on the host: bad inputs, a diverging start, a time cap, an
allocation beyond the budget, cancelled requests, and the bounded device waits.

Nothing here faults, traps or hangs the GPU. The one device-side failure is the self-test of
the bounded waits: a kernel waits on an mbarrier that nothing arrives at, gives up after the
context's wait limit (set to a few milliseconds), records that in the context's error flag and
returns; the call reports CC_ERR_TIMEOUT and the context keeps working.
"""
import time

import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu

INVALID, OOM, NOT_CONVERGED, DIVERGED, TIMEOUT, CANCELLED = -1, -2, -3, -4, -6, -7


@pytest.fixture(scope="module")
def ctx(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    c = ccpnk.Context(0)
    yield c
    c.close()


def test_non_finite_inputs_are_rejected(ctx):
    from paper_2608_06669_b300 import ccpnk

    s = synth.make_system(3, 8, 6, seed=2, gauge="haar")
    for which, bad in (("B", np.nan), ("B", np.inf), ("fock", np.nan), ("fock", -np.inf)):
        f, B = s.fock.copy(), s.B.copy()
        if which == "B":
            B[1, 2, 5] = B[1, 5, 2] = bad
        else:
            f[4, 4] = bad
        with pytest.raises(ccpnk.CCError) as ei:
            ccpnk.System(ctx, s.o, s.v, s.naux, f, B)
        assert ei.value.status == INVALID, (which, bad)


def test_non_finite_start_reports_divergence(ctx):
    from paper_2608_06669_b300 import ccpnk

    s = synth.make_system(3, 8, 6, seed=3, gauge="canonical")
    g = ccpnk.System.from_synth(ctx, s)
    t1, t2 = synth.random_amplitudes(np.random.default_rng(1), 3, 8, 0.01, 0.01)
    t2[0, 1, 2, 3] = t2[1, 0, 3, 2] = np.nan
    for method in ("pnk", "fp_diis"):
        _, _, rep = g.solve(method, "fp64", t1=t1, t2=t2)
        assert rep["status_code"] == DIVERGED and rep["status"] == DIVERGED, rep
        assert rep["residual_evals"] == 1 and not np.isfinite(rep["res_norm"])


def test_time_cap_stops_with_a_filled_report(ctx):
    from paper_2608_06669_b300 import ccpnk

    s = synth.workload("o10v90_rotated")
    g = ccpnk.System.from_synth(ctx, s)
    t0 = time.perf_counter()
    _, _, rep = g.solve("pnk", "fp64", max_seconds=1e-6)
    assert time.perf_counter() - t0 < 30.0
    assert rep["status_code"] == NOT_CONVERGED and rep["status"] == NOT_CONVERGED
    # the first residual is evaluated before the cap is checked; its norm and energy are reported
    assert rep["residual_evals"] == 1 and rep["newton_iters"] == 0
    assert np.isfinite(rep["res_norm"]) and rep["res_norm"] > 1e-8 and rep["energy"] < 0.0


def test_allocation_beyond_the_budget_is_reported(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    small = ccpnk.Context(0, mem_budget=8 << 20)
    s = synth.workload("o10v90_rotated")  # its DF factor alone is 24 MB
    with pytest.raises(ccpnk.CCError) as ei:
        ccpnk.System.from_synth(small, s)
    assert ei.value.status == OOM
    # the context stays usable for what fits
    t = synth.make_system(2, 5, 4, seed=1)
    r1, r2, e = ccpnk.System.from_synth(small, t).residual(np.zeros((2, 5)), np.zeros((2, 2, 5, 5)))
    q1, q2, eq = cc.residual(t.fock, t.B, 2, np.zeros((2, 5)), np.zeros((2, 2, 5, 5)))
    assert np.abs(r2 - q2).max() <= 1e-12 and e == 0.0 == eq
    small.close()


def test_bounded_wait_gives_up_and_the_context_survives(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    c = ccpnk.Context(0)
    c.set_option("wait_limit_ns", 5_000_000)  # 5 ms
    t0 = time.perf_counter()
    assert c.selftest_wait() == TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the error flag was cleared: the tensor-core pipeline works again on the same context
    c.set_option("wait_limit_ns", 1_000_000_000)
    s = synth.make_system(3, 20, 10, seed=8, gauge="haar")
    t1, t2 = synth.random_amplitudes(np.random.default_rng(3), 3, 20, 0.05, 0.05)
    r1, r2, _ = ccpnk.System.from_synth(c, s).residual(t1, t2, prec="tf32x3")
    q1, q2, _ = cc.residual(s.fock, s.B, 3, t1, t2)
    assert np.abs(r2 - q2).max() < 1e-6 * np.abs(q2).max()
    with pytest.raises(ccpnk.CCError):
        c.set_option("wait_limit_ns", 10)  # below the 1e5 ns floor
    with pytest.raises(ccpnk.CCError):
        c.set_option("stage_cache_bytes", -5)
    c.close()


def _wait(srv, ticket, limit_s=300.0):
    t0 = time.time()
    while True:
        r = srv.poll(ticket)
        if r is not None:
            return r
        assert time.time() - t0 < limit_s
        time.sleep(0.01)


def test_server_cancels_waiting_and_running_requests(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    s = synth.workload("o10v90_rotated")
    srv = ccpnk.Server(0, 0, max_slots=1)
    # FP64 PNK at this size runs for seconds: the first request is running when it is cancelled,
    # the second is still waiting behind it
    a = srv.submit(s.o, s.v, s.naux, s.fock, s.B, "pnk", "fp64", af_direct=1)
    b = srv.submit(s.o, s.v, s.naux, s.fock, s.B, "pnk", "fp64", af_direct=1)
    t0 = time.time()
    while srv.stats()["running"] < 1:
        assert time.time() - t0 < 60.0
        time.sleep(0.005)
    time.sleep(0.3)
    assert srv.cancel(b) == 0
    assert srv.cancel(a) == 0
    t1b, t2b, repb = _wait(srv, b)
    t1a, t2a, repa = _wait(srv, a)
    assert repb["status_code"] == CANCELLED and repb["residual_evals"] == 0 and not t2b.any()
    assert repa["status_code"] == CANCELLED and repa["status"] == CANCELLED
    assert 1 <= repa["residual_evals"] and np.isfinite(repa["res_norm"])
    # a request with non-finite input fails on its own and leaves the server working
    B = s.B.copy()
    B[0, 0, 0] = np.nan
    c = srv.submit(s.o, s.v, s.naux, s.fock, B, "pnk", "fp64")
    assert _wait(srv, c)[2]["status_code"] == INVALID
    small = synth.make_system(3, 12, 9, seed=4, gauge="haar")
    d = srv.submit(small.o, small.v, small.naux, small.fock, small.B, "pnk", "fp64", af_direct=1)
    assert _wait(srv, d)[2]["status_code"] == 0
    assert srv.cancel(d) == -1  # released by its poll
    srv.close()
