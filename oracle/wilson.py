"""Oracle: the Wilson-Dirac operator of the two-dimensional Schwinger model.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 1.1, Eq. (3):
    D[n, m] = (m0 + 2) delta_{n,m}
              - 1/2 sum_mu [ (1 - sigma_mu) U_mu(n) delta_{n+mu, m}
                             + (1 + sigma_mu) U_mu(n - mu)^* delta_{n-mu, m} ]
with sigma_0, sigma_1 of Eq. (4), sigma_3 = i sigma_0 sigma_1 of Eq. (5) and
the boundary conditions of Eq. (7): periodic in x, antiperiodic in t.

Readings (the paper does not fix them):
  * direction mu = 0 is t and mu = 1 is x (Lambda is written (n_t, n_x) and
    sigma_0 is the first Pauli matrix);
  * the antiperiodic sign sits on every fermion hop that crosses the t boundary,
    in both directions; the links themselves are periodic.

Index conventions: site s = t * Nx + x, degree of freedom (s, alpha) -> 2 s + alpha.
Gauge links U[mu, t, x] complex128; vectors as [2, Nt, Nx] complex128 or flat
length 2 * Nt * Nx in DOF order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA0 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA1 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SIGMA3 = 1j * SIGMA0 @ SIGMA1          # Eq. (5): diag(-1, 1)
IDENT2 = np.eye(2, dtype=np.complex128)
SIGMAS = (SIGMA0, SIGMA1)


def site_index(t, x, Nx):
    return t * Nx + x


def _add_site_row(U: np.ndarray, m0: float, t: int, x: int, t_sign: float, rows, cols, vals) -> None:
    """Entries of D's two rows of site (t, x) (Eq. (3)), appended to rows/cols/vals."""
    _, Nt, Nx = U.shape

    def add_block(s_row, s_col, block):
        for a in range(2):
            for b in range(2):
                if block[a, b] != 0:
                    rows.append(2 * s_row + a)
                    cols.append(2 * s_col + b)
                    vals.append(block[a, b])

    n = site_index(t, x, Nx)
    add_block(n, n, (m0 + 2.0) * IDENT2)
    for mu in (0, 1):
        # forward neighbour n + mu_hat, with the Eq. (7) sign when it wraps in t
        if mu == 0:
            tf, xf = (t + 1) % Nt, x
            sign_f = t_sign if t == Nt - 1 else 1.0
            tb, xb = (t - 1) % Nt, x
            sign_b = t_sign if t == 0 else 1.0
        else:
            tf, xf = t, (x + 1) % Nx
            sign_f = 1.0
            tb, xb = t, (x - 1) % Nx
            sign_b = 1.0
        m_f = site_index(tf, xf, Nx)
        m_b = site_index(tb, xb, Nx)
        u_f = U[mu, t, x]                 # U_mu(n)
        u_b = np.conj(U[mu, tb, xb])      # U_mu(n - mu)^dagger
        add_block(n, m_f, -0.5 * sign_f * u_f * (IDENT2 - SIGMAS[mu]))
        add_block(n, m_b, -0.5 * sign_b * u_b * (IDENT2 + SIGMAS[mu]))


def dirac_matrix(U: np.ndarray, m0: float, t_sign: float = -1.0) -> sp.csr_matrix:
    """Assemble D of Eq. (3) as a sparse (2 V) x (2 V) complex matrix, one entry at a time.

    t_sign is the factor on hops across the t boundary: -1 (antiperiodic, Eq. (7);
    the method's case) or +1 (periodic, used only by the normalisation pin)."""
    _, Nt, Nx = U.shape
    V = Nt * Nx
    rows, cols, vals = [], [], []
    for t in range(Nt):
        for x in range(Nx):
            _add_site_row(U, m0, t, x, t_sign, rows, cols, vals)
    D = sp.coo_matrix((vals, (rows, cols)), shape=(2 * V, 2 * V)).tocsr()
    D.sum_duplicates()
    return D


def dirac_rows(U: np.ndarray, m0: float, sites, t_sign: float = -1.0) -> sp.csr_matrix:
    """D of Eq. (3) restricted to the rows of the given (t, x) sites (other rows
    zero), same shape as dirac_matrix: for local work on lattices too large to
    assemble whole."""
    _, Nt, Nx = U.shape
    V = Nt * Nx
    rows, cols, vals = [], [], []
    for (t, x) in sorted(set((int(t), int(x)) for t, x in sites)):
        _add_site_row(U, m0, t, x, t_sign, rows, cols, vals)
    D = sp.coo_matrix((vals, (rows, cols)), shape=(2 * V, 2 * V)).tocsr()
    D.sum_duplicates()
    return D


def apply_dirac(U: np.ndarray, m0: float, psi: np.ndarray) -> np.ndarray:
    """Matrix-free D psi for psi[2, Nt, Nx] (a second, independent route to Eq. (3))."""
    _, Nt, Nx = U.shape
    out = (m0 + 2.0) * psi.astype(np.complex128)
    tsign_fwd = np.ones((Nt, 1)); tsign_fwd[Nt - 1, 0] = -1.0
    tsign_bwd = np.ones((Nt, 1)); tsign_bwd[0, 0] = -1.0
    for mu in (0, 1):
        axis = mu  # arrays are [t, x]; mu = 0 -> axis 0 (t), mu = 1 -> axis 1 (x)
        fwd = np.roll(psi, -1, axis=1 + axis)           # psi(n + mu)
        bwd = np.roll(psi, 1, axis=1 + axis)            # psi(n - mu)
        if mu == 0:
            fwd = fwd * tsign_fwd
            bwd = bwd * tsign_bwd
        u_f = U[mu]
        u_b = np.conj(np.roll(U[mu], 1, axis=axis))    # U_mu(n - mu)^*
        pm = IDENT2 - SIGMAS[mu]
        pp = IDENT2 + SIGMAS[mu]
        hop_f = np.einsum("ab,bij->aij", pm, fwd) * u_f
        hop_b = np.einsum("ab,bij->aij", pp, bwd) * u_b
        out = out - 0.5 * (hop_f + hop_b)
    return out


def to_flat(psi: np.ndarray) -> np.ndarray:
    """[2, Nt, Nx] -> DOF order 2 s + alpha."""
    return np.ascontiguousarray(np.moveaxis(psi, 0, -1)).reshape(-1)


def from_flat(v: np.ndarray, Nt: int, Nx: int) -> np.ndarray:
    """DOF order -> [2, Nt, Nx]."""
    return np.moveaxis(v.reshape(Nt, Nx, 2), -1, 0).copy()


def sigma3_full(V: int) -> sp.csr_matrix:
    """sigma_3 acting on every site (block diagonal)."""
    return sp.kron(sp.identity(V, format="csr"), sp.csr_matrix(SIGMA3), format="csr")


def gauge_transform_links(U: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """U_mu(n) -> Omega(n) U_mu(n) Omega(n + mu)^* with omega[t, x] a U(1) phase field.
    Omega is periodic in both directions (the antiperiodic sign belongs to fermions)."""
    U2 = U.copy()
    U2[0] = omega * U[0] * np.conj(np.roll(omega, -1, axis=0))
    U2[1] = omega * U[1] * np.conj(np.roll(omega, -1, axis=1))
    return U2


def k_formulation(A: sp.spmatrix) -> sp.csr_matrix:
    """Real form of Sec. 4.2: each complex entry a + ib becomes [[a, -b], [b, a]]."""
    A = sp.coo_matrix(A)
    r, c, v = A.row, A.col, A.data
    rows = np.concatenate([2 * r, 2 * r, 2 * r + 1, 2 * r + 1])
    cols = np.concatenate([2 * c, 2 * c + 1, 2 * c, 2 * c + 1])
    vals = np.concatenate([v.real, -v.imag, v.imag, v.real])
    n = A.shape[0]
    return sp.coo_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n)).tocsr()
