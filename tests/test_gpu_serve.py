"""The continuous-batching server: each request's result is the same alone and in the mix.

Requests of uneven (o, v) and gauge are submitted together to a server with several slots,
so several solves run on the device at once; each result must equal the same request solved
alone through cc_solve (1e-10 Eh in FP64, 1e-8 Eh in the mixed precisions; the kernels are
deterministic, so the amplitudes agree to rounding), and the served amplitudes must be a root
of the CPU oracle's residual.
"""
import time

import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu


def _requests():
    shapes = [(4, 24, "canonical"), (5, 31, "haar"), (4, 30, "haar"), (6, 37, "canonical"), (5, 28, "haar"),
              (4, 26, "canonical")]
    return [synth.make_system(o, v, 3 * (o + v), seed=500 + k, gauge=g) for k, (o, v, g) in enumerate(shapes)]


def _wait_all(srv, tickets, limit_s=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        assert time.time() - t0 < limit_s, "served requests did not finish in time"
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        time.sleep(0.01)
    return out


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32x3", 1e-8)])
def test_served_results_equal_solo_results(cuda_device, prec, tol):
    from paper_2608_06669_b300 import ccpnk

    systems = _requests()
    srv = ccpnk.Server(0, 0, max_slots=3)
    tickets = [srv.submit(s.o, s.v, s.naux, s.fock, s.B, "pnk", prec, af_direct=1) for s in systems]
    served = _wait_all(srv, tickets)
    stats = srv.stats()
    times = [srv.times(t) for t in tickets]
    srv.close()
    assert stats["max_running"] >= 2, stats  # the solves overlapped on the device
    # some request was admitted while another was still running
    assert any(times[i][1] < times[j][2] and times[j][1] < times[i][2] for i in range(len(times))
               for j in range(len(times)) if i != j)
    ctx = ccpnk.Context(0)
    for s, t in zip(systems, tickets):
        t1, t2, rep = served[t]
        assert rep["status_code"] == 0, rep
        a1, a2, alone = ccpnk.System.from_synth(ctx, s).solve("pnk", prec, af_direct=1)
        assert abs(rep["energy"] - alone["energy"]) <= tol
        assert np.max(np.abs(t2 - a2)) <= 1e-8
    ctx.close()
    # the served amplitudes are a root of the oracle's residual
    s = systems[1]
    t1, t2, rep = served[tickets[1]]
    q1, q2, eq = cc.residual(s.fock, s.B, s.o, t1, t2)
    assert np.sqrt((q1 ** 2).sum() + (q2 ** 2).sum()) < 1e-8 and abs(eq - rep["energy"]) < 1e-10


def test_server_rejects_what_can_never_fit(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    s = synth.workload("o10v90_rotated")
    srv = ccpnk.Server(0, mem_budget=64 << 20, max_slots=1)
    with pytest.raises(ccpnk.CCError) as ei:
        srv.submit(s.o, s.v, s.naux, s.fock, s.B, "pnk", "fp64")
    assert ei.value.status == -2
    srv.close()
