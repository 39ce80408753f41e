"""cc_energy_noalloc: the correlation energy without device allocation.

For callers that cannot call cudaMalloc at the point where they need the energy (another
framework's arena, a real-time loop, memory reserved up front). The entry point is called
through the C ABI with device buffers the test owns, twice in a row on different amplitudes,
and each result must equal the oracle's energy and the energy cc_residual returns for the
same amplitudes, to the FP64 parity tolerance. This file sorts last so that a run stopping at
its first failure has already run every other test; it also passes on its own in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

from oracle import dfccsd as cc
from paper_2608_06669_b300 import synth

pytestmark = pytest.mark.gpu


def test_energy_without_allocation_matches_cc_residual(cuda_device):
    import torch

    from paper_2608_06669_b300 import ccpnk

    L = ccpnk.lib()
    ctx = ccpnk.Context(0)
    s = synth.workload("o10v90_rotated")
    g = ccpnk.System.from_synth(ctx, s)
    rng = np.random.default_rng(21)
    stream = torch.cuda.current_stream()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        t1, t2 = synth.random_amplitudes(rng, s.o, s.v, 0.05 * (call + 1), 0.05 * (call + 1))
        T1 = torch.from_numpy(t1).cuda()
        T2 = torch.from_numpy(t2).cuda()
        _, _, e_ref = g.residual(T1, T2)  # the allocating entry point
        torch.cuda.synchronize()
        st = L.cc_energy_noalloc(g.h, ctypes.c_void_p(T1.data_ptr()), ctypes.c_void_p(T2.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        e = float(out.item())
        assert abs(e - e_ref) <= 1e-10 * max(1.0, abs(e_ref)), (call, e, e_ref)
        e_or = cc.energy(s.fock, s.B, s.o, t1, t2)
        assert abs(e - e_or) <= 1e-10 * max(1.0, abs(e_or)), (call, e, e_or)
    # NULL arguments are rejected before any launch
    assert L.cc_energy_noalloc(g.h, None, None, None, None) == -1
    g.close()
    ctx.close()
