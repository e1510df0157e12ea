"""FP64 oracle of the scattering problem (paper Sect. 5.3.2: in strongly
scattering media the source function depends on the intensity). Per band b
and point: S_b = (1 - eps_b) J_b[S] + eps_b B_b, J_b[S] the mean intensity of
the formal solution (the oracle's orc_solve) with source S_b.

TEST INFRASTRUCTURE ONLY: used by tests/ and nothing else.

The fixed point is found by the plain Lambda iteration, in the order the
definition reads: S <- (1 - eps) J[S] + eps B, from S = B, until the largest
change is <= tol times the largest S. The solve's bottom boundary (I = S)
takes the current S, so it scatters too.
"""
from __future__ import annotations

import numpy as np


def scatter_solve(problem, chi, B, eps, tol=1e-13, max_iter=20000, nthreads=1):
    """Returns (S, outputs of the solve with S, iterations)."""
    chi = np.asarray(chi, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    S = B.copy()
    for it in range(1, max_iter + 1):
        Jb = problem.solve(chi, S, debug=True, nthreads=nthreads)["Jb"]
        S_new = (1.0 - eps) * Jb + eps * B
        change = np.abs(S_new - S).max()
        S = S_new
        if change <= tol * np.abs(S).max():
            break
    else:
        raise RuntimeError("Lambda iteration did not converge")
    return S, problem.solve(chi, S, nthreads=nthreads), it
