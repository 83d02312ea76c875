"""Oracle: critical mass of a gauge field from the spectrum of D.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper sets its bare masses relative to the critical mass m_c (Sec. 5 and
its critical-mass table).  For a synthetic field it is read here as
m_crit = -min_k Re lambda_k(D at m0 = 0): D(m0) = m0 I + D(0), so at
m0 = m_crit + delta every eigenvalue of D has real part >= delta.
Small lattices use dense eigenvalues.  Larger ones use ARPACK's implicitly
restarted Arnoldi for the eigenvalues of smallest real part (k = 4, 128 Arnoldi
vectors, relative tolerance 1e-6 by default, which fixes m_crit far better
than the mass offsets it is used for; the fields of 256^2 and more at weak
coupling, whose lowest eigenvalues are dense, use 1e-4, which reproduced the
1e-6 value of the 256^2 benchmark field to 1e-14).  Shift-invert around a real shift is not used: on
quenched fields the leftmost eigenvalue can carry a sizeable imaginary part
and then is not among the eigenvalues nearest a real shift.  The tests compare
this route with dense eigenvalues on 32^2 and 40^2 fields.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .wilson import dirac_matrix

DENSE_MAX_DOF = 2 * 32 * 32


def critical_mass(U: np.ndarray, dense: bool = None, tol: float = 1e-6) -> float:
    """m_crit = -min Re lambda(D at m0 = 0); tol is ARPACK's relative tolerance
    (the Arnoldi route only)."""
    D0 = dirac_matrix(U, 0.0)
    n = D0.shape[0]
    if dense is None:
        dense = n <= DENSE_MAX_DOF
    if dense:
        lam = np.linalg.eigvals(D0.toarray())
    else:
        lam = spla.eigs(D0.tocsr(), k=4, which="SR", ncv=128, tol=tol, maxiter=100000,
                        return_eigenvectors=False)
    return float(-np.min(lam.real))
