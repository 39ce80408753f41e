"""Writes tests/golden/convergence.json: what the oracle's own reference solver does on the
large and near-degenerate synthetic workloads and on reduced copies with their integral
strength.

The question it answers: when a GPU solve of such a workload does not reach ||R|| < 1e-8,
is that the input or the GPU path?  The reference root of a workload is the one the
oracle's fixed-point + DIIS solver reaches from the generalised MP2 start in the eigenbasis
of the occupied and virtual Fock blocks (the canonical gauge; the energy is gauge
invariant, App. A.2).  This script runs that solver, with and without the level shift of
App. D, and records for every case whether it converges, diverges or stalls, together with
the size of the integrals against the orbital-energy denominators, which decides whether
the problem is in the perturbative regime the MP2 start and the diagonal denominator rely
on.  A scan of the integral strength (B -> lambda B, i.e. every (pq|rs) times lambda^2) on
the reduced copy of the o=30, v=270, naux=900 workload locates where the solver stops
converging.  It calls only oracle/ and the input generator.

    OMP_NUM_THREADS=6 python tests/golden/convergence_study.py [case ...]
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "convergence.json")

# name -> (system recipe, solver settings)
CASES = {
    # the o=10 v=90 naux=300 workload (converges; the reference point)
    "o10v90n300_rotated": dict(sys=dict(o=10, v=90, naux=300, seed=2, gauge="small"), shift=0.0, maxiter=200),
    # the o=30 v=270 naux=900 workload's integral strength (naux = 9 (o + v) at sigma = 0.05) at o=10 v=90
    "o10v90n900_rotated": dict(sys=dict(o=10, v=90, naux=900, seed=3, gauge="small"), shift=0.0, maxiter=150),
    "o10v90n900_rotated_shift0.2": dict(sys=dict(o=10, v=90, naux=900, seed=3, gauge="small"), shift=0.2,
                                        maxiter=150),
    # the near-degenerate workload's regime (gap 0.02 Eh, naux = 3 (o + v), Haar gauge) at o=10 v=90
    "o10v90n300_gap0.02": dict(sys=dict(o=10, v=90, naux=300, seed=5, gauge="haar", gap=0.02), shift=0.0,
                               maxiter=150),
    "o10v90n300_gap0.02_shift0.2": dict(sys=dict(o=10, v=90, naux=300, seed=5, gauge="haar", gap=0.02),
                                        shift=0.2, maxiter=150),
    # the near-degenerate workload itself (o=20 v=180 naux=600, gap 0.02 Eh)
    "o20v180n600_gap0.02": dict(workload="o20v180_neardegenerate", shift=0.0, maxiter=40),
    "o20v180n600_gap0.02_shift0.2": dict(workload="o20v180_neardegenerate", shift=0.2, maxiter=40),
}
for lam in (0.5, 0.6, 0.7, 0.8, 0.9):
    CASES[f"o10v90n900_rotated_lambda{lam}"] = dict(sys=dict(o=10, v=90, naux=900, seed=3, gauge="small"),
                                                    shift=0.0, maxiter=150, lam=lam)


def regime(f, B, o):
    """Integral sizes against the denominators, in the canonical gauge."""
    eo, ev = np.diag(f)[:o], np.diag(f)[o:]
    Bov = B[:, :o, o:]
    ovov_diag = np.einsum("Xia,Xia->ia", Bov, Bov)  # (ia|ia)
    den = ev[None, :] - eo[:, None]
    vv_diag = np.einsum("Xab,Xab->ab", B[:, o:, o:], B[:, o:, o:])  # (ab|ab)
    return {"max_(ia|ia)": float(ovov_diag.max()), "max_(ab|ab)": float(vv_diag.max()),
            "min_eps_a-eps_i": float(den.min()),
            "max_(ia|ia)/(eps_a-eps_i)": float((ovov_diag / den).max()),
            "mean_(ia|ia)/(eps_a-eps_i)": float((ovov_diag / den).mean())}


def run(name, spec):
    if "workload" in spec:
        s = synth.workload(spec["workload"])
    else:
        s = synth.make_system(**spec["sys"])
    B = s.B * spec.get("lam", 1.0)
    f, Bc, _ = cc.to_eigenbasis(s.fock, B, s.o)
    energies, hist = [], []
    t0 = time.time()
    outcome = "not converged within the iteration cap"
    e = None
    for it, _, _, e, rn in cc.fp_diis_iterates(f, Bc, s.o, shift=spec["shift"], diis_size=8):
        hist.append(rn)
        energies.append(e)
        print(f"  {name} it {it:3d}  |R| {rn:.3e}  E {e:.12f}", flush=True)
        if rn < 1e-8:
            outcome = "converged"
            break
        if not np.isfinite(rn) or rn > 1e3 * hist[0]:
            outcome = "diverged"
            break
        if len(hist) >= spec["maxiter"]:
            break
    rn = hist[-1]
    return {"o": s.o, "v": s.v, "naux": s.naux, "lambda": spec.get("lam", 1.0), "shift": spec["shift"],
            "outcome": outcome, "iterations": len(hist), "final_res_norm": rn, "final_energy": e,
            "mp2_energy": energies[0] if energies else None, "min_res_norm": float(np.nanmin(hist)),
            "seconds": round(time.time() - t0, 1), "regime": regime(f, Bc, s.o),
            "res_norm_history": [float(f"{x:.3e}") for x in hist],
            "energy_history": [float(f"{x:.10f}") for x in energies],
            "solver": "oracle fp+diis(8), eigenbasis, generalised MP2 start; diverged: ||R|| above 1e3 times "
                      "its value at the start"}


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    for name in names:
        print("==", name, flush=True)
        data[name] = run(name, CASES[name])
        print(name, {k: v for k, v in data[name].items() if not k.endswith("history")}, flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
