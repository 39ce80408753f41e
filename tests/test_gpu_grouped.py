"""Grouped, lockstep solves of several problems (cc_solve_batch and the server's grouped mode).

Problems of uneven (o, v) and gauge are solved together: every residual and JVP is evaluated for
all unfinished problems at once, the same contraction of every problem in one group whose
tensor-core contractions share persistent grouped launches. Each problem's arithmetic is that
of a solve on its own, so the result is the same bit for bit (asserted), and the roots zero the
oracle residual.
"""
import time

import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu


def _systems():
    shapes = [(4, 24, "canonical"), (5, 31, "haar"), (3, 20, "haar"), (6, 37, "canonical"), (5, 28, "haar")]
    return [synth.make_system(o, v, 3 * (o + v), seed=700 + k, gauge=g) for k, (o, v, g) in enumerate(shapes)]


@pytest.mark.parametrize("prec,outer", [("tf32x3", 5), ("fp64", 0), ("bf16x3", 5)])
def test_batch_equals_solo(cuda_device, prec, outer):
    from paper_2608_06669_b300 import ccpnk

    systems = _systems()
    ctx = ccpnk.Context(0)
    gs = [ccpnk.System.from_synth(ctx, s) for s in systems]
    batch = ccpnk.solve_batch(ctx, gs, "pnk", prec, af_direct=1, outer_prec=outer)
    for s, g, (b1, b2, rb) in zip(systems, gs, batch):
        a1, a2, ra = g.solve("pnk", prec, af_direct=1, outer_prec=outer)
        assert rb["status_code"] == 0 == ra["status_code"], (rb, ra)
        for k in ("newton_iters", "jvps", "krylov_iters", "residual_evals"):
            assert rb[k] == ra[k], k
        assert rb["energy"] == ra["energy"]
        assert np.array_equal(b2, a2) and np.array_equal(b1, a1)
    s, (t1, t2, rep) = systems[1], batch[1]
    q1, q2, eq = cc.residual(s.fock, s.B, s.o, t1, t2)
    assert np.sqrt((q1 ** 2).sum() + (q2 ** 2).sum()) < 1e-8 and abs(eq - rep["energy"]) < 1e-10
    for g in gs:
        g.close()
    ctx.close()


def test_batch_of_other_methods_runs_them_one_by_one(cuda_device):
    from paper_2608_06669_b300 import ccpnk

    systems = _systems()[:2]
    ctx = ccpnk.Context(0)
    gs = [ccpnk.System.from_synth(ctx, s) for s in systems]
    batch = ccpnk.solve_batch(ctx, gs, "fp_diis", "fp64", max_outer=400)
    for g, (b1, b2, rb) in zip(gs, batch):
        a1, a2, ra = g.solve("fp_diis", "fp64", max_outer=400)
        assert rb["status_code"] == 0 and rb["energy"] == ra["energy"] and np.array_equal(b2, a2)
    ctx.close()


def _wait_all(srv, tickets, limit_s=300.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        assert time.time() - t0 < limit_s
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        time.sleep(0.005)
    return out


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32x3", 1e-8)])
def test_grouped_server_results_equal_solo(cuda_device, prec, tol):
    from paper_2608_06669_b300 import ccpnk

    systems = _systems() + [synth.make_system(4, 26, 90, seed=799, gauge="canonical")]
    srv = ccpnk.Server(0, 0, max_slots=1)
    srv.set_grouping(4)
    extra = {"outer_prec": 5} if prec == "tf32x3" else {}
    tickets = [srv.submit(s.o, s.v, s.naux, s.fock, s.B, "pnk", prec, af_direct=1, **extra) for s in systems]
    served = _wait_all(srv, tickets)
    times = [srv.times(t) for t in tickets]
    srv.close()
    # one slot, so several requests ran at once only as members of one batch
    assert sum(1 for i in range(len(times)) for j in range(len(times))
               if i < j and times[i][1] < times[j][2] and times[j][1] < times[i][2]) >= 1
    ctx = ccpnk.Context(0)
    for s, t in zip(systems, tickets):
        t1, t2, rep = served[t]
        assert rep["status_code"] == 0, rep
        a1, a2, alone = ccpnk.System.from_synth(ctx, s).solve("pnk", prec, af_direct=1, **extra)
        assert abs(rep["energy"] - alone["energy"]) <= tol
        assert np.max(np.abs(t2 - a2)) <= 1e-8
    ctx.close()
    with pytest.raises(ccpnk.CCError):
        ccpnk.Server(0, 0, max_slots=1).set_grouping(0)
