"""B300-native preconditioned Newton-Krylov solver for closed-shell CCSD.

Importing the package loads nothing; the CUDA library is opened by
``paper_2608_06669_b300.ccpnk`` on first use.
"""
