"""Oracle: critical mass of a gauge field from the spectrum of D.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper sets its bare masses relative to the critical mass m_c (Sec. 5 and
its critical-mass table).  For a synthetic field it is read here as
m_crit = -min_k Re lambda_k(D at m0 = 0): D(m0) = m0 I + D(0), so at
m0 = m_crit + delta every eigenvalue of D has real part >= delta.
Small lattices use dense eigenvalues; larger ones ARPACK ("smallest real part").
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .wilson import dirac_matrix

DENSE_MAX_DOF = 2 * 32 * 32


def critical_mass(U: np.ndarray, tol: float = 1e-10) -> float:
    D0 = dirac_matrix(U, 0.0)
    n = D0.shape[0]
    if n <= DENSE_MAX_DOF:
        lam = np.linalg.eigvals(D0.toarray())
    else:
        lam = spla.eigs(D0, k=6, which="SR", tol=tol, maxiter=200000, ncv=64,
                        return_eigenvectors=False)
    return float(-np.min(lam.real))
