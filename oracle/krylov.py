"""Oracle: flexible GMRES, the outer solver (Sec. 1 and Sec. 5: "preconditioners
for FGMRES ... relative convergence tolerance 1e-10").

TEST INFRASTRUCTURE ONLY (see the package docstring).

Right-preconditioned flexible GMRES with restart length m (Saad's FGMRES):
the preconditioned directions z_j = M(v_j) are kept in a second basis Z so that
M may change between steps (the V-cycle is not a fixed linear operator once it
runs in reduced precision).  Arnoldi uses modified Gram-Schmidt (gs="mgs",
default), or classical Gram-Schmidt with a second pass where the first one
cancelled much of w (gs="cgs2": the criterion of Daniel, Gragg, Kaufman and
Stewart, 1976, ||w after|| < ||w before|| / sqrt(2)); the small least-squares
problem is solved with complex Givens rotations.

Readings (the paper fixes none of them): start vector x0 = 0; residual measured
as ||b - A x||_2 / ||b||_2; the iteration count is the total number of Arnoldi
steps; the recursive residual estimate only ends a cycle early, and the solve
stops only when the true residual, recomputed at every restart and at a claimed
convergence, is below the tolerance.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np


@dataclass
class FgmresResult:
    x: np.ndarray
    iterations: int
    true_relres: float
    converged: bool
    estimates: List[float] = field(default_factory=list)   # |g_{j+1}| / ||b|| after each step
    restarts: int = 0
    second_passes: int = 0                                   # gs="cgs2": steps that reorthogonalised


def givens(a: complex, b: complex):
    """(c, s) with c real such that [[c, s], [-conj(s), c]] @ [a, b] = [r, 0]."""
    if b == 0:
        return 1.0, 0.0 + 0j
    if a == 0:
        return 0.0, 1.0 + 0j
    r = np.hypot(abs(a), abs(b))
    c = abs(a) / r
    s = (a / abs(a)) * np.conj(b) / r
    return c, s


def fgmres(apply_A: Callable[[np.ndarray], np.ndarray],
           precond: Callable[[np.ndarray], np.ndarray],
           b: np.ndarray, m: int, tol: float, max_iter: int, gs: str = "mgs") -> FgmresResult:
    if gs not in ("mgs", "cgs2"):
        raise ValueError(f"gs must be 'mgs' or 'cgs2', got {gs!r}")
    n = b.shape[0]
    second = 0
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return FgmresResult(x, 0, 0.0, True)
    iters = 0
    restarts = 0
    estimates: List[float] = []
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            return FgmresResult(x, iters, beta / bnorm, True, estimates, restarts, second)
        if iters >= max_iter:
            return FgmresResult(x, iters, beta / bnorm, False, estimates, restarts, second)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            if gs == "mgs":
                for i in range(j + 1):                   # modified Gram-Schmidt
                    H[i, j] = np.vdot(V[i], w)
                    w = w - H[i, j] * V[i]
            else:
                # classical Gram-Schmidt: all projections from the same w, then
                # once more if the pass removed more than 1 - 1/sqrt(2) of ||w||
                w0 = np.linalg.norm(w)
                h = V[:j + 1].conj() @ w
                w = w - V[:j + 1].T @ h
                if np.linalg.norm(w) < w0 / np.sqrt(2.0):
                    h2 = V[:j + 1].conj() @ w
                    w = w - V[:j + 1].T @ h2
                    h = h + h2
                    second += 1
                H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # earlier rotations
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            estimates.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or iters >= max_iter or breakdown:
                break
        # least squares: upper triangular H[:k, :k] y = g[:k]
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        restarts += 1


@dataclass
class CgnrResult:
    x: np.ndarray
    iterations: int
    true_relres: float
    converged: bool


def cgnr(apply_A: Callable[[np.ndarray], np.ndarray],
         apply_AH: Callable[[np.ndarray], np.ndarray],
         b: np.ndarray, tol: float, max_iter: int) -> CgnrResult:
    """Conjugate gradients on the normal equations A^H A x = A^H b (CGNR, Saad's
    "Iterative Methods for Sparse Linear Systems", Sec. 8.3), the paper's
    unpreconditioned comparison solver (Sec. 5), with A^H = sigma_3 A sigma_3 for
    the Wilson operator (Eq. (6)).

    x0 = 0; r = b - A x is the residual of the original system, carried by the
    recurrence; z = A^H r is the normal-equation residual.  One iteration:
        w = A p,  alpha = ||z||^2 / ||w||^2,  x += alpha p,  r -= alpha w,
        z' = A^H r,  beta = ||z'||^2 / ||z||^2,  p = z' + beta p.
    The iteration count is the number of such steps; a step whose recursive
    ||r|| / ||b|| reaches tol ends the loop, and the solve stops only when the
    true residual ||b - A x|| / ||b|| is below tol (else it restarts the
    recurrence from the true residual)."""
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return CgnrResult(x, 0, 0.0, True)
    iters = 0
    while True:
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return CgnrResult(x, iters, rel, True)
        if iters >= max_iter:
            return CgnrResult(x, iters, rel, False)
        z = apply_AH(r)
        p = z.copy()
        zz = np.vdot(z, z).real
        while iters < max_iter:
            w = apply_A(p)
            ww = np.vdot(w, w).real
            if ww == 0.0:
                break
            alpha = zz / ww
            x = x + alpha * p
            r = r - alpha * w
            iters += 1
            if np.linalg.norm(r) <= tol * bnorm:
                break
            z = apply_AH(r)
            zz_new = np.vdot(z, z).real
            p = z + (zz_new / zz) * p
            zz = zz_new
