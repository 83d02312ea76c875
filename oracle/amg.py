"""Oracle: SM-AMG hierarchy (wirebaskets, interpolation, Galerkin product), block
Gauss-Seidel smoother, coarsest direct solve and the V-cycle of Algorithm 1.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Structured wirebaskets (Sec. 4.1).  On a level whose sites form an Nt x Nx
periodic lattice and with tile side a (a | Nt, a | Nx, Nt/a >= 2, Nx/a >= 2):
  * vertices V are the sites with t = 0 and x = 0 (mod a); they span the next level;
  * wirebasket W(p, q) = {(p a + i, q a + j) mod (Nt, Nx) : 0 <= i, j <= a},
    (a+1)^2 sites whose borders overlap their neighbours' by one row/column;
    a = 2 gives the nine-point basket drawn in the paper's wirebasket figure;
  * role of a site: vertex if t = x = 0 (mod a), edge if exactly one of them is,
    interior otherwise (both spin components share the role of their site);
  * ownership: a non-vertex site (t, x) takes its interpolation formula from the
    single basket W(t // a, x // a) ("the first aggregate it was assigned to"
    read as the basket of the tile that contains it; each basket owns its
    lower and left borders).  The alternative reading, the basket of smallest
    index among those containing the site ("first_lex"), is available for
    comparison.

Local interpolation (Eqs. (14)-(16)): with A_W = A[W, W] (couplings inside the
basket only) and F = W minus its four corner vertices, the ideal-smoothing system
of Eq. (15) gives u_F = -A_FF^{-1} A_FV u_V.  Route A solves that system as one
block; route B applies the two Schur-complement formulas printed after Eq. (15)
(interior and edge rows separately).  Both routes must agree.  The normalisation
N of Eq. (16) is read as the identity (exact ideal interpolation); a row-sum
normalisation (each non-vertex row divided by its complex row sum) and a
spin-split interpolation (spin-diagonal weights only) are available for
comparison.

Global interpolator (Sec. 4.1, last paragraph): rows of owned non-vertex sites
come from their basket's local formula, vertex rows are the identity onto their
own coarse variable.  Coarse variable index: 2 * (p * Nx/a + q) + alpha.

Galerkin product (Sec. 2): A_H = P^H A_h P; restriction is P^H.

Smoother: "block solver as smoother, 2 post-smoothing steps" (Sec. 5).  Block =
one site (its 2 x 2 diagonal block).  The colouring is red-black (t + x parity)
on the fine Wilson level; on coarse levels it is c = (t + 3 x) mod 8 when that
separates every coupled pair (extents multiples of 8; true for the 21-offset
operator of a first coarse level), else 16 colours (t mod 4, x mod 4).  Colours
are visited in increasing number; sites of one colour never couple, so each
colour is a simultaneous block update.

V-cycle (Algorithm 1 used as a preconditioner, start vector 0, no
pre-smoothing): e = P M_{l+1}(P^H r), then post-smoothing sweeps on A_l e = r;
the coarsest level is solved exactly by LU (scipy.linalg.lu_factor).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .wilson import dirac_rows

ROLE_VERTEX, ROLE_EDGE, ROLE_INTERIOR = 0, 1, 2


# --------------------------------------------------------------------------- structure

def check_tiling(Nt: int, Nx: int, a: int) -> None:
    if a < 2 or Nt % a or Nx % a or Nt // a < 2 or Nx // a < 2:
        raise ValueError(f"tile side {a} does not tile a {Nt}x{Nx} lattice with >= 2 tiles per side")


def site_roles(Nt: int, Nx: int, a: int) -> np.ndarray:
    """role[t, x]: 0 vertex, 1 edge, 2 interior."""
    check_tiling(Nt, Nx, a)
    t0 = (np.arange(Nt) % a == 0)[:, None]
    x0 = (np.arange(Nx) % a == 0)[None, :]
    role = np.full((Nt, Nx), ROLE_INTERIOR, dtype=np.int32)
    role[np.logical_xor(t0, x0)] = ROLE_EDGE
    role[t0 & x0] = ROLE_VERTEX
    return role


OWNERSHIP_RULES = ("tile", "first_lex")


def owner_basket(t: int, x: int, Nt: int, Nx: int, a: int, rule: str = "tile") -> int:
    """Index p * (Nx/a) + q of the basket whose formula site (t, x) uses.

    "tile" (the method's reading): the basket of the tile that contains the
    site, W(t // a, x // a).  "first_lex" (the alternative reading of "the first
    aggregate it was assigned to", Sec. 4.1): among the baskets that contain the
    site, the one with the smallest index p * (Nx/a) + q.  An interior site lies
    in one basket only, so the rules differ on edge sites; a vertex gets the tile
    whose corner (0, 0) it is under both."""
    Np, Nq = Nt // a, Nx // a
    p, q = t // a, x // a
    if rule == "tile" or (t % a == 0 and x % a == 0):
        return p * Nq + q
    if rule != "first_lex":
        raise ValueError(f"unknown ownership rule {rule!r}")
    if t % a == 0:                       # bottom border of W(p, q), top border of W(p-1, q)
        return min(p * Nq + q, ((p - 1) % Np) * Nq + q)
    if x % a == 0:                       # left border of W(p, q), right border of W(p, q-1)
        return min(p * Nq + q, p * Nq + (q - 1) % Nq)
    return p * Nq + q


def owner_tiles(Nt: int, Nx: int, a: int, rule: str = "tile") -> np.ndarray:
    """owner[t, x] = owner_basket(t, x) for every site."""
    check_tiling(Nt, Nx, a)
    if rule == "tile":
        p = (np.arange(Nt) // a)[:, None]
        q = (np.arange(Nx) // a)[None, :]
        return (p * (Nx // a) + q).astype(np.int32)
    out = np.empty((Nt, Nx), dtype=np.int32)
    for t in range(Nt):
        for x in range(Nx):
            out[t, x] = owner_basket(t, x, Nt, Nx, a, rule)
    return out


def basket_sites(Nt: int, Nx: int, a: int, p: int, q: int):
    """Sites of W(p, q) as (t, x) pairs, i-major, with their in-basket (i, j)."""
    out = []
    for i in range(a + 1):
        for j in range(a + 1):
            out.append(((p * a + i) % Nt, (q * a + j) % Nx, i, j))
    return out


def corner_vertex(Nt: int, Nx: int, a: int, p: int, q: int, c: int) -> int:
    """Coarse site index of corner c of W(p, q); c = 2 di + dj, corner (p + di, q + dj)."""
    Np, Nq = Nt // a, Nx // a
    di, dj = c >> 1, c & 1
    return ((p + di) % Np) * Nq + (q + dj) % Nq


# --------------------------------------------------------------------------- interpolation

def _dense_block(A: sp.csr_matrix, dofs: np.ndarray) -> np.ndarray:
    return A[dofs][:, dofs].toarray()


def local_interpolation(A: sp.csr_matrix, Nt: int, Nx: int, a: int, p: int, q: int,
                        route: str = "A"):
    """Local interpolation of basket W(p, q), Eq. (16) with G and N the identity.

    Returns (F_sites, P_F) where F_sites lists the basket's non-vertex sites
    (t, x, i, j) in basket order and P_F[2k + alpha, 2c + beta] is the weight of
    corner c, spin beta for F-site k, spin alpha.
    """
    sites = basket_sites(Nt, Nx, a, p, q)
    is_corner = [(i in (0, a)) and (j in (0, a)) for (_, _, i, j) in sites]
    is_edge = [((i in (0, a)) != (j in (0, a))) for (_, _, i, j) in sites]
    dof = lambda t, x: np.array([2 * (t * Nx + x), 2 * (t * Nx + x) + 1])
    F_sites = [s for s, c in zip(sites, is_corner) if not c]
    # corner DOFs ordered by corner number c = 2 di + dj
    corner_order = sorted([s for s, c in zip(sites, is_corner) if c], key=lambda s: 2 * (s[2] // a) + (s[3] // a))
    F_dofs = np.concatenate([dof(t, x) for (t, x, _, _) in F_sites])
    V_dofs = np.concatenate([dof(t, x) for (t, x, _, _) in corner_order])
    if route == "A":
        A_FF = _dense_block(A, F_dofs)
        A_FV = A[F_dofs][:, V_dofs].toarray()
        P_F = -np.linalg.solve(A_FF, A_FV)
        return F_sites, P_F
    if route != "B":
        raise ValueError(route)
    # Route B: the two Schur-complement formulas after Eq. (15).
    E_mask = np.array([is_edge[k] for k, c in enumerate(is_corner) if not c])
    E_rows = np.concatenate([[2 * k, 2 * k + 1] for k in np.nonzero(E_mask)[0]])
    I_rows = np.concatenate([[2 * k, 2 * k + 1] for k in np.nonzero(~E_mask)[0]])
    E_dofs, I_dofs = F_dofs[E_rows], F_dofs[I_rows]
    blk = lambda r, c: A[r][:, c].toarray()
    A_II, A_IE, A_IV = blk(I_dofs, I_dofs), blk(I_dofs, E_dofs), blk(I_dofs, V_dofs)
    A_EI, A_EE, A_EV = blk(E_dofs, I_dofs), blk(E_dofs, E_dofs), blk(E_dofs, V_dofs)
    A_II_inv = np.linalg.inv(A_II)
    A_EE_inv = np.linalg.inv(A_EE)
    hat_EE = A_EE - A_EI @ A_II_inv @ A_IE
    u_E = -np.linalg.solve(hat_EE, A_EV - A_EI @ A_II_inv @ A_IV)
    hat_II = A_II - A_IE @ A_EE_inv @ A_EI
    u_I = -np.linalg.solve(hat_II, A_IV - A_IE @ A_EE_inv @ A_EV)
    P_F = np.zeros((len(F_dofs), len(V_dofs)), dtype=np.complex128)
    P_F[E_rows] = u_E
    P_F[I_rows] = u_I
    return F_sites, P_F


NORMALIZATIONS = ("none", "rowsum")
ROWSUM_FLOOR = 1e-12


def build_interpolator(A: sp.csr_matrix, Nt: int, Nx: int, a: int, route: str = "A",
                       ownership: str = "tile", normalization: str = "none", stats: dict = None,
                       spin_split: bool = False):
    """Global interpolator P (2 Nt Nx) x (2 Nt Nx / a^2) and its structural pattern.

    Every owned row stores all 8 corner weights, so the structural pattern does
    not depend on numeric zeros.  ownership picks the basket whose formula a
    border site takes (owner_basket).  normalization "none" keeps the exact
    ideal interpolation (the method's reading of N in Eq. (16)); "rowsum"
    divides every non-vertex scalar row by its complex row sum, leaving rows
    whose |sum| is below ROWSUM_FLOOR times the largest |sum| unnormalised
    (their number goes to stats["rowsum_skipped"] when stats is given).
    spin_split keeps only the spin-diagonal weights, P -> (P + s3 P s3) / 2 with
    s3 = sigma_3 on every site (fine and coarse): P then commutes with sigma_3
    and the Galerkin operator inherits sigma_3-hermiticity (the direction the
    paper proposes for future work, Sec. 6; comparison only)."""
    check_tiling(Nt, Nx, a)
    if normalization not in NORMALIZATIONS:
        raise ValueError(f"unknown normalisation {normalization!r}")
    Np, Nq = Nt // a, Nx // a
    rows, cols, vals = [], [], []
    for p in range(Np):
        for q in range(Nq):
            F_sites, P_F = local_interpolation(A, Nt, Nx, a, p, q, route)
            for k, (t, x, i, j) in enumerate(F_sites):
                if owner_basket(t, x, Nt, Nx, a, ownership) != p * Nq + q:   # another basket's row
                    continue
                for alpha in range(2):
                    r = 2 * (t * Nx + x) + alpha
                    for c in range(4):
                        v = corner_vertex(Nt, Nx, a, p, q, c)
                        for beta in range(2):
                            rows.append(r)
                            cols.append(2 * v + beta)
                            vals.append(P_F[2 * k + alpha, 2 * c + beta])
            # the basket's own vertex (i = j = 0): identity onto its coarse variable
            t, x = p * a, q * a
            v = p * Nq + q
            for alpha in range(2):
                rows.append(2 * (t * Nx + x) + alpha)
                cols.append(2 * v + alpha)
                vals.append(1.0 + 0j)
    shape = (2 * Nt * Nx, 2 * Np * Nq)
    P = sp.csr_matrix((vals, (rows, cols)), shape=shape)
    pattern = sp.csr_matrix((np.ones(len(rows), dtype=np.int64), (rows, cols)), shape=shape)
    if normalization == "rowsum":
        role = site_roles(Nt, Nx, a).reshape(-1)
        sums = np.asarray(P.sum(axis=1)).reshape(-1)
        vertex_row = np.repeat(role == ROLE_VERTEX, 2)
        floor = ROWSUM_FLOOR * np.max(np.abs(sums[~vertex_row]))
        ok = (~vertex_row) & (np.abs(sums) >= floor)
        scale = np.ones(P.shape[0], dtype=complex)
        scale[ok] = 1.0 / sums[ok]
        P = (sp.diags(scale) @ P).tocsr()
        if stats is not None:
            stats["rowsum_skipped"] = int(np.sum((~vertex_row) & ~ok))
    if spin_split:
        s3f = sp.diags(np.tile([1.0, -1.0], Nt * Nx))
        s3c = sp.diags(np.tile([1.0, -1.0], Np * Nq))
        P = (0.5 * (P + s3f @ P @ s3c)).tocsr()
        P.eliminate_zeros()
    return P, pattern


def galerkin_rows(U: np.ndarray, m0: float, a: int, vertices):
    """Rows of the first coarse operator A_1 = P^H D P (Sec. 2; tile edge
    ownership, N the identity) for the coarse sites `vertices` ((p, q) pairs),
    from the baskets near them only: row v of A_1 involves P's column v (the
    owned rows of the four tiles around v and v's own site) and, through the
    nearest-neighbour D, the columns of every coarse site whose tiles reach a
    neighbour of those rows, all within three tiles of v.  Returns
    {(p, q): {w: 2x2 block A_1[(v, alpha), (w, beta)]}} with w the coarse site
    index p_w (Nx / a) + q_w.  For lattices too large to assemble D and P whole;
    equal to the rows of galerkin(P, D) (pinned)."""
    _, Nt, Nx = U.shape
    check_tiling(Nt, Nx, a)
    Np, Nq = Nt // a, Nx // a
    vertices = [(int(p) % Np, int(q) % Nq) for p, q in vertices]
    tiles = sorted({((p + dp) % Np, (q + dq) % Nq) for (p, q) in vertices
                    for dp in range(-3, 3) for dq in range(-3, 3)})
    sites = {(t, x) for (tp, tq) in tiles for (t, x, _, _) in basket_sites(Nt, Nx, a, tp, tq)}
    D = dirac_rows(U, m0, sites)
    # rows of P owned by the tiles in reach: fine DOF -> {coarse DOF: weight}
    Prow = {}
    for (tp, tq) in tiles:
        F_sites, P_F = local_interpolation(D, Nt, Nx, a, tp, tq)
        for k, (t, x, i, j) in enumerate(F_sites):
            if owner_basket(t, x, Nt, Nx, a, "tile") != tp * Nq + tq:
                continue
            for alpha in range(2):
                row = Prow.setdefault(2 * (t * Nx + x) + alpha, {})
                for c in range(4):
                    v = corner_vertex(Nt, Nx, a, tp, tq, c)
                    for beta in range(2):
                        row[2 * v + beta] = row.get(2 * v + beta, 0) + P_F[2 * k + alpha, 2 * c + beta]
        for alpha in range(2):
            Prow[2 * ((tp * a) * Nx + tq * a) + alpha] = {2 * (tp * Nq + tq) + alpha: 1.0 + 0j}
    out = {}
    for (p, q) in vertices:
        v = p * Nq + q
        blocks = {}
        for alpha in range(2):
            col = 2 * v + alpha
            # column v of P: the fine rows that reference it
            supp = [(i, r[col]) for i, r in Prow.items() if col in r]
            # (P_v)^H D: a sparse fine row vector
            acc = {}
            for i, pv in supp:
                lo, hi = D.indptr[i], D.indptr[i + 1]
                if lo == hi:
                    raise ValueError("row of D outside the window")
                for jj, dij in zip(D.indices[lo:hi], D.data[lo:hi]):
                    acc[jj] = acc.get(jj, 0) + np.conj(pv) * dij
            # times P
            for j, val in acc.items():
                if j not in Prow:
                    raise ValueError("row of P outside the window")
                for cdof, pw in Prow[j].items():
                    w, beta = divmod(cdof, 2)
                    blocks.setdefault(w, np.zeros((2, 2), dtype=np.complex128))[alpha, beta] += val * pw
        out[(p, q)] = blocks
    return out


# --------------------------------------------------------------------------- Galerkin / sparsity

def canonical_offsets(pairs, Nt: int, Nx: int):
    """Offsets reduced mod the lattice, duplicates merged, sorted lexicographically."""
    return sorted({(int(dt) % Nt, int(dx) % Nx) for dt, dx in pairs})


def site_pattern(pattern_dof: sp.spmatrix) -> sp.csr_matrix:
    """Collapse a DOF-level (2 per site) boolean pattern to the site level."""
    P = sp.coo_matrix(pattern_dof)
    n_r, n_c = P.shape[0] // 2, P.shape[1] // 2
    return sp.csr_matrix((np.ones_like(P.row), (P.row // 2, P.col // 2)), shape=(n_r, n_c))


def coarse_offsets(P_pattern: sp.spmatrix, A_pattern: sp.spmatrix, Nt: int, Nx: int, a: int,
                   union: bool = False):
    """Block-neighbour offsets of P^H A P from the boolean product of structural patterns.

    Returns the canonical offset list shared by every coarse site, after checking
    that the pattern is the same for all sites (translation invariance).  The
    first-lex ownership reading of Sec. 4.1 gives the first tile row and column
    other baskets than the rest, so its pattern can differ between coarse sites:
    with union=True the list is the union over all sites (a site's blocks at
    offsets it does not couple through are zero)."""
    Ps = site_pattern(P_pattern)
    As = site_pattern(A_pattern)
    C = (Ps.T @ As @ Ps).tocsr()
    Np, Nq = Nt // a, Nx // a
    ref = None
    seen = set()
    for v in range(Np * Nq):
        pv, qv = divmod(v, Nq)
        nbrs = C.indices[C.indptr[v]:C.indptr[v + 1]]
        offs = canonical_offsets([((w // Nq) - pv, (w % Nq) - qv) for w in nbrs], Np, Nq)
        seen.update(offs)
        if ref is None:
            ref = offs
        elif offs != ref and not union:
            raise AssertionError("coarse sparsity is not translation invariant")
    return sorted(seen) if union else ref


def galerkin(P: sp.csr_matrix, A: sp.csr_matrix) -> sp.csr_matrix:
    """A_H = P^H A P (Sec. 2), exact sparse products."""
    return (P.conj().T @ A @ P).tocsr()


def pattern_from_offsets(offsets, Nt: int, Nx: int) -> sp.csr_matrix:
    """DOF-level structural pattern of an operator with full 2x2 blocks on the given site offsets."""
    rows, cols = [], []
    for t in range(Nt):
        for x in range(Nx):
            s = t * Nx + x
            for dt, dx in offsets:
                s2 = ((t + dt) % Nt) * Nx + (x + dx) % Nx
                for aa in range(2):
                    for bb in range(2):
                        rows.append(2 * s + aa)
                        cols.append(2 * s2 + bb)
    n = 2 * Nt * Nx
    M = sp.csr_matrix((np.ones(len(rows), dtype=np.int64), (rows, cols)), shape=(n, n))
    M.data[:] = 1
    return M


WILSON_OFFSETS_RAW = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]


def block_stencil(A: sp.csr_matrix, offsets, Nt: int, Nx: int) -> np.ndarray:
    """blocks[k, s, alpha, beta] = A[(s, alpha), (s + offset_k, beta)] (0 where absent)."""
    n = Nt * Nx
    A = A.tocsr()
    t, x = np.divmod(np.arange(n), Nx)
    B = np.zeros((len(offsets), n, 2, 2), dtype=np.complex128)
    for k, (dt, dx) in enumerate(offsets):
        s2 = ((t + dt) % Nt) * Nx + (x + dx) % Nx
        for aa in range(2):
            for bb in range(2):
                B[k, :, aa, bb] = np.asarray(A[2 * np.arange(n) + aa, 2 * s2 + bb]).ravel()
    return B


# --------------------------------------------------------------------------- smoother

def eight_colour_valid(Nt: int, Nx: int, offsets) -> bool:
    """The colouring c = (t + 3 x) mod 8 separates every pair of coupled sites
    when both extents are multiples of 8 and no off-diagonal offset has
    dt + 3 dx = 0 (mod 8)."""
    if Nt % 8 or Nx % 8:
        return False
    return all((dt + 3 * dx) % 8 != 0 for dt, dx in offsets if (dt % Nt, dx % Nx) != (0, 0))


def colouring(Nt: int, Nx: int, fine: bool, offsets=None) -> np.ndarray:
    """Gauss-Seidel colours: red-black on the fine level; on coarse levels
    c = (t + 3 x) mod 8 where that separates all couplings (8 colours), else
    c = 4 (t mod 4) + (x mod 4) (16 colours)."""
    t = np.arange(Nt)[:, None]
    x = np.arange(Nx)[None, :]
    if fine:
        if Nt % 2 or Nx % 2:
            raise ValueError("red-black colouring needs even extents")
        return ((t + x) % 2).astype(np.int32)
    if offsets is not None and eight_colour_valid(Nt, Nx, offsets):
        return ((t + 3 * x) % 8).astype(np.int32)
    if Nt % 4 or Nx % 4:
        raise ValueError("16-colour Gauss-Seidel needs extents divisible by 4")
    return ((t % 4) * 4 + (x % 4)).astype(np.int32)


def check_colouring(colour: np.ndarray, offsets) -> None:
    """Sites of one colour never couple (required for a simultaneous colour update)."""
    Nt, Nx = colour.shape
    for dt, dx in offsets:
        if (dt % Nt, dx % Nx) == (0, 0):
            continue
        shifted = np.roll(np.roll(colour, -dt, axis=0), -dx, axis=1)
        if np.any(shifted == colour):
            raise AssertionError(f"offset {(dt, dx)} couples sites of one colour")


def diag_block_inverses(A: sp.csr_matrix, n_sites: int) -> np.ndarray:
    inv = np.zeros((n_sites, 2, 2), dtype=np.complex128)
    for s in range(n_sites):
        inv[s] = np.linalg.inv(A[2 * s:2 * s + 2, 2 * s:2 * s + 2].toarray())
    return inv


def gs_sweep(A: sp.csr_matrix, dinv: np.ndarray, colour: np.ndarray, e: np.ndarray, r: np.ndarray) -> np.ndarray:
    """One block Gauss-Seidel sweep on A e = r, colours in increasing order:
    e_s <- e_s + A_ss^{-1} (r - A e)_s for every site s of the current colour."""
    e = e.copy()
    col = colour.reshape(-1)
    for c in range(int(col.max()) + 1):
        sites = np.nonzero(col == c)[0]
        dofs = np.stack([2 * sites, 2 * sites + 1], axis=1).reshape(-1)
        res = r[dofs] - A[dofs] @ e
        corr = np.einsum("sab,sb->sa", dinv[sites], res.reshape(-1, 2))
        e[dofs] += corr.reshape(-1)
    return e


# --------------------------------------------------------------------------- hierarchy and V-cycle

@dataclass
class Level:
    Nt: int
    Nx: int
    A: sp.csr_matrix
    offsets: list                       # canonical site offsets of A's structural pattern
    a: Optional[int] = None             # tile side used to coarsen this level
    P: Optional[sp.csr_matrix] = None
    P_pattern: Optional[sp.csr_matrix] = None
    colour: Optional[np.ndarray] = None
    dinv: Optional[np.ndarray] = None
    lu: object = None                   # coarsest only


def build_hierarchy(D: sp.csr_matrix, Nt: int, Nx: int, aggs: List[int], route: str = "A",
                    smooth: bool = True, ownership: str = "tile", normalization: str = "none",
                    spin_split: bool = False) -> List[Level]:
    """Setup phase (Sec. 2): coarsening, interpolation, Galerkin, recursively;
    the last level is factorised for the exact coarsest solve.  ownership and
    normalization select the readings of build_interpolator (defaults: the
    method's)."""
    levels = [Level(Nt, Nx, D.tocsr(), canonical_offsets(WILSON_OFFSETS_RAW, Nt, Nx))]
    A_pat = pattern_from_offsets(levels[0].offsets, Nt, Nx)
    for li, a in enumerate(aggs):
        L = levels[-1]
        L.a = a
        L.P, L.P_pattern = build_interpolator(L.A, L.Nt, L.Nx, a, route, ownership, normalization,
                                              spin_split=spin_split)
        offs = coarse_offsets(L.P_pattern, A_pat, L.Nt, L.Nx, a, union=(ownership != "tile"))
        Ac = galerkin(L.P, L.A)
        nxt = Level(L.Nt // a, L.Nx // a, Ac, offs)
        A_pat = pattern_from_offsets(offs, nxt.Nt, nxt.Nx)
        levels.append(nxt)
    if smooth:
        for li, L in enumerate(levels[:-1]):
            L.colour = colouring(L.Nt, L.Nx, fine=(li == 0), offsets=L.offsets)
            check_colouring(L.colour, L.offsets)
            L.dinv = diag_block_inverses(L.A, L.Nt * L.Nx)
    last = levels[-1]
    last.lu = sla.lu_factor(last.A.toarray())
    return levels


COARSEST_SOLVERS = ("lu", "gmres")


def coarsest_gmres(L: "Level", r: np.ndarray, tol: float = 0.1, restart: int = 30) -> np.ndarray:
    """The paper's coarsest-level solver (Sec. 5): unpreconditioned GMRES from a
    zero start to a relative residual of tol (the oracle's FGMRES with the
    identity as preconditioner, which is plain restarted GMRES)."""
    from . import krylov
    return krylov.fgmres(lambda v: L.A @ v, lambda v: v, r, restart, tol, 100000).x


def vcycle(levels: List[Level], r: np.ndarray, level: int = 0, post_smooth: int = 2,
           coarsest: str = "lu") -> np.ndarray:
    """Preconditioner M(r) of Algorithm 1 with start vector 0 and no pre-smoothing.
    coarsest: "lu" (the method's reading: exact solve) or "gmres" (the paper's
    setting: GMRES to 0.1, for comparison)."""
    L = levels[level]
    if level == len(levels) - 1:
        if coarsest == "gmres":
            return coarsest_gmres(L, r)
        if coarsest != "lu":
            raise ValueError(f"unknown coarsest solver {coarsest!r}")
        return sla.lu_solve(L.lu, r)
    rc = L.P.conj().T @ r                       # restrict: d^H = I_h^H d^h
    ec = vcycle(levels, rc, level + 1, post_smooth, coarsest)
    e = L.P @ ec                                # interpolate the coarse correction
    for _ in range(post_smooth):
        e = gs_sweep(L.A, L.dinv, L.colour, e, r)
    return e
