"""CPU oracle for the closed-shell CCSD / Newton-Krylov hot path.

TEST INFRASTRUCTURE ONLY: plain, slow, obviously correct FP64 code that the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
compare the CUDA path against.  The product path never imports, links or runs
anything here, and nothing here imports the CUDA path.

fock_space  O0: the CC equations by brute force in determinant space (the
            definition, Eqs. CC_ampl and CC_energy), plus FCI.
dfccsd      O1: closed-shell DF-CCSD residual and energy, the exact JVP, the
            gauge-invariant preconditioner A_F and its exact inverse, the
            generalised-MP2 start and the fixed-point + DIIS reference solver.

Parity status: every function is pinned by tests/test_oracle_pins.py except
the iteration counts of the solvers, which are not compared (parity unpinned:
the paper's convergence curves are figures that are not available).
"""
