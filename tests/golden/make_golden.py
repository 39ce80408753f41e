"""Writes tests/golden/energies.json: converged CCSD correlation energies of the
benchmark workloads, computed by the CPU oracle alone.

The reference root is the one the oracle's fixed-point + DIIS solver reaches
from the generalised MP2 start after the problem is rotated to the eigenbasis
of its occupied and virtual Fock blocks (the gauge invariance of the energy,
App. A.2, makes that the root of every gauge).

    python tests/golden/make_golden.py [workload ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import dfccsd as cc  # noqa: E402
from paper_2608_06669_b300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "energies.json")


def solve(name: str, tol: float = 1e-10, maxiter: int = 400):
    s = synth.workload(name)
    f, Bc, _ = cc.to_eigenbasis(s.fock, s.B, s.o)
    t0 = time.time()
    t1, t2, e, hist = cc.solve_fp_diis(f, Bc, s.o, tol=tol, maxiter=maxiter, diis_size=12)
    to_1e8 = next((i + 1 for i, r in enumerate(hist) if r < 1e-8), None)
    return {"o": s.o, "v": s.v, "naux": s.naux, "e_corr": e, "res_norm": hist[-1],
            "iterations": len(hist), "iterations_to_1e-8": to_1e8, "seconds": round(time.time() - t0, 1),
            "solver": "oracle fp+diis(12), eigenbasis, generalised MP2 start"}


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    for name in names:
        data[name] = solve(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["o5v20_canonical", "o10v90_rotated"])
