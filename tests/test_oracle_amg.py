"""Pins of the oracle's SM-AMG hierarchy, smoother and V-cycle (Sec. 2, Sec. 4.1,
Eqs. (14)-(16), Algorithm 1) to exact properties, dense linear algebra and brute force."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg
from oracle import wilson as W
from paper_2608_03515_b300 import fixtures as fx


def random_links(Nt, Nx, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))


CASES = [(4, 4, 2), (8, 8, 2), (8, 8, 4), (8, 12, 4)]


@pytest.mark.parametrize("Nt,Nx,a", CASES)
def test_roles_and_ownership_partition(Nt, Nx, a):
    role = amg.site_roles(Nt, Nx, a)
    owner = amg.owner_tiles(Nt, Nx, a)
    Np, Nq = Nt // a, Nx // a
    # every basket contains 4 vertices, 4(a-1) edge and (a-1)^2 interior sites
    count = np.zeros(Nt * Nx, dtype=int)
    for p in range(Np):
        for q in range(Nq):
            sites = amg.basket_sites(Nt, Nx, a, p, q)
            roles = [role[t, x] for (t, x, _, _) in sites]
            assert roles.count(amg.ROLE_VERTEX) == 4
            assert roles.count(amg.ROLE_EDGE) == 4 * (a - 1)
            assert roles.count(amg.ROLE_INTERIOR) == (a - 1) ** 2
            for (t, x, i, j) in sites:
                if role[t, x] != amg.ROLE_VERTEX and owner[t, x] == p * Nq + q:
                    count[t * Nx + x] += 1
                    assert i < a and j < a
    # each non-vertex site is owned by exactly one basket that contains it
    nonvertex = (role.reshape(-1) != amg.ROLE_VERTEX)
    assert np.all(count[nonvertex] == 1)
    assert np.all(count[~nonvertex] == 0)
    # interior sites belong to exactly one basket, edges to two, vertices to four
    member = np.zeros(Nt * Nx, dtype=int)
    for p in range(Np):
        for q in range(Nq):
            for (t, x, _, _) in amg.basket_sites(Nt, Nx, a, p, q):
                member[t * Nx + x] += 1
    expect = {amg.ROLE_VERTEX: 4, amg.ROLE_EDGE: 2, amg.ROLE_INTERIOR: 1}
    for s in range(Nt * Nx):
        assert member[s] == expect[role.reshape(-1)[s]]


def test_nine_point_basket_matches_the_figure():
    """a = 2: four vertices (corners), four edges (mid-sides), one interior point (centre)."""
    role = amg.site_roles(4, 4, 2)
    sites = amg.basket_sites(4, 4, 2, 0, 0)
    grid = np.array([role[t, x] for (t, x, _, _) in sites]).reshape(3, 3)
    V, E, I = amg.ROLE_VERTEX, amg.ROLE_EDGE, amg.ROLE_INTERIOR
    assert grid.tolist() == [[V, E, V], [E, I, E], [V, E, V]]


@pytest.mark.parametrize("Nt,Nx,a", CASES)
def test_routes_agree_and_ideal_interpolation(Nt, Nx, a):
    U = random_links(Nt, Nx, 7)
    D = W.dirac_matrix(U, 0.3)
    for p in range(Nt // a):
        for q in range(Nx // a):
            F_sites, PA = amg.local_interpolation(D, Nt, Nx, a, p, q, "A")
            _, PB = amg.local_interpolation(D, Nt, Nx, a, p, q, "B")
            assert np.max(np.abs(PA - PB)) <= 1e-12 * np.max(np.abs(PA))
            # Eq. (15): F rows of A_W [P_F; I] vanish (zero interior/edge residual)
            sites = amg.basket_sites(Nt, Nx, a, p, q)
            corners = sorted([s for s in sites if s[2] in (0, a) and s[3] in (0, a)],
                             key=lambda s: 2 * (s[2] // a) + (s[3] // a))
            dof = lambda s: [2 * (s[0] * Nx + s[1]), 2 * (s[0] * Nx + s[1]) + 1]
            Fd = np.concatenate([dof(s) for s in F_sites])
            Vd = np.concatenate([dof(s) for s in corners])
            res = D[Fd][:, Fd].toarray() @ PA + D[Fd][:, Vd].toarray()
            assert np.max(np.abs(res)) < 1e-12


@pytest.mark.parametrize("Nt,Nx,a", CASES)
def test_interpolator_identity_on_vertices(Nt, Nx, a):
    U = random_links(Nt, Nx, 8)
    D = W.dirac_matrix(U, 0.3)
    P, pat = amg.build_interpolator(D, Nt, Nx, a)
    role = amg.site_roles(Nt, Nx, a).reshape(-1)
    Nq = Nx // a
    Pd = P.toarray()
    for s in range(Nt * Nx):
        t, x = divmod(s, Nx)
        rows = Pd[2 * s:2 * s + 2]
        if role[s] == amg.ROLE_VERTEX:
            v = (t // a) * Nq + x // a
            expect = np.zeros_like(rows)
            expect[0, 2 * v] = expect[1, 2 * v + 1] = 1.0
            assert np.array_equal(rows, expect)
        else:
            assert pat[2 * s].nnz == 8 and pat[2 * s + 1].nnz == 8
            assert np.all(np.abs(rows).sum(axis=1) > 0)


def test_level1_sparsity_is_21_offsets():
    """Galerkin sparsity from the boolean product: |dp|, |dq| <= 2 minus the four corners."""
    Nt = Nx = 32
    a = 4
    U = random_links(Nt, Nx, 9)
    D = W.dirac_matrix(U, 0.3)
    P, pat = amg.build_interpolator(D, Nt, Nx, a)
    A_pat = amg.pattern_from_offsets(amg.canonical_offsets(amg.WILSON_OFFSETS_RAW, Nt, Nx), Nt, Nx)
    offs = amg.coarse_offsets(pat, A_pat, Nt, Nx, a)
    expect = amg.canonical_offsets([(dp, dq) for dp in range(-2, 3) for dq in range(-2, 3)
                                    if not (abs(dp) == 2 and abs(dq) == 2)], 8, 8)
    assert offs == expect and len(offs) == 21


@pytest.mark.parametrize("Nt,Nx,a", CASES)
def test_galerkin_equals_dense_product_and_pattern(Nt, Nx, a):
    U = random_links(Nt, Nx, 10)
    D = W.dirac_matrix(U, 0.3)
    P, pat = amg.build_interpolator(D, Nt, Nx, a)
    Dc = amg.galerkin(P, D)
    dense = P.toarray().conj().T @ D.toarray() @ P.toarray()
    assert np.max(np.abs(Dc.toarray() - dense)) < 1e-13 * np.max(np.abs(dense))
    A_pat = amg.pattern_from_offsets(amg.canonical_offsets(amg.WILSON_OFFSETS_RAW, Nt, Nx), Nt, Nx)
    offs = amg.coarse_offsets(pat, A_pat, Nt, Nx, a)
    sym = amg.pattern_from_offsets(offs, Nt // a, Nx // a).toarray() > 0
    assert np.all(sym[np.abs(dense) > 1e-14])          # numeric nonzeros inside the symbolic pattern
    # blocks read back from the stencil layout reproduce the matrix
    B = amg.block_stencil(Dc, offs, Nt // a, Nx // a)
    rebuilt = np.zeros_like(dense)
    Np, Nq = Nt // a, Nx // a
    for k, (dp, dq) in enumerate(offs):
        for v in range(Np * Nq):
            pv, qv = divmod(v, Nq)
            w = ((pv + dp) % Np) * Nq + (qv + dq) % Nq
            rebuilt[2 * v:2 * v + 2, 2 * w:2 * w + 2] += B[k, v]
    assert np.max(np.abs(rebuilt - dense)) < 1e-13 * np.max(np.abs(dense))


@pytest.mark.parametrize("Nt,Nx,a", [(8, 8, 2), (8, 8, 4)])
def test_coarse_grid_correction_is_a_projection(Nt, Nx, a):
    U = random_links(Nt, Nx, 11)
    Dd = W.dirac_matrix(U, 0.3).toarray()
    P, _ = amg.build_interpolator(W.dirac_matrix(U, 0.3), Nt, Nx, a)
    Pd = P.toarray()
    Dc = Pd.conj().T @ Dd @ Pd
    K = np.eye(Dd.shape[0]) - Pd @ np.linalg.solve(Dc, Pd.conj().T @ Dd)
    assert np.max(np.abs(K @ K - K)) < 1e-12
    assert np.max(np.abs(Pd.conj().T @ Dd @ K)) < 1e-12


@pytest.mark.parametrize("Nt,Nx,a", [(8, 8, 2), (8, 8, 4)])
def test_interpolator_and_coarse_operator_gauge_covariance(Nt, Nx, a):
    U = random_links(Nt, Nx, 12)
    rng = np.random.Generator(np.random.PCG64(13))
    omega = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(Nt, Nx)))
    U2 = W.gauge_transform_links(U, omega)
    D1, D2 = W.dirac_matrix(U, 0.3), W.dirac_matrix(U2, 0.3)
    P1, _ = amg.build_interpolator(D1, Nt, Nx, a)
    P2, _ = amg.build_interpolator(D2, Nt, Nx, a)
    Om = np.diag(np.repeat(omega.reshape(-1), 2))
    omV = omega[::a, ::a].reshape(-1)
    OmV = np.diag(np.repeat(omV, 2))
    assert np.max(np.abs(P2.toarray() - Om @ P1.toarray() @ OmV.conj().T)) < 1e-12
    Dc1, Dc2 = amg.galerkin(P1, D1).toarray(), amg.galerkin(P2, D2).toarray()
    assert np.max(np.abs(Dc2 - OmV @ Dc1 @ OmV.conj().T)) < 1e-12


def sequential_gs(A, e, r, order):
    """Brute force: point-block Gauss-Seidel, one site at a time in the given order."""
    e = e.copy()
    Ad = A.toarray()
    for s in order:
        d = slice(2 * s, 2 * s + 2)
        res = r[d] - Ad[d] @ e
        e[d] = e[d] + np.linalg.solve(Ad[d, d], res)
    return e


def test_red_black_sweep_equals_sequential_gs():
    Nt = Nx = 4
    U = random_links(Nt, Nx, 14)
    D = W.dirac_matrix(U, 0.1)
    colour = amg.colouring(Nt, Nx, fine=True)
    dinv = amg.diag_block_inverses(D, Nt * Nx)
    rng = np.random.Generator(np.random.PCG64(15))
    r = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    e0 = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    order = [s for c in (0, 1) for s in range(16) if colour.reshape(-1)[s] == c]
    assert np.max(np.abs(amg.gs_sweep(D, dinv, colour, e0, r) - sequential_gs(D, e0, r, order))) < 1e-13


@pytest.mark.parametrize("Nt,ncol", [(16, 8), (24, 16)])
def test_coarse_colour_sweep_equals_sequential_gs(Nt, ncol):
    """Level 1 of a [2, 2] hierarchy: 8 x 8 takes the 8-colour ordering
    (t + 3x) mod 8, 12 x 12 (not a multiple of 8) the 16-colour one; either
    way one sweep equals point-block GS visiting the sites in colour order."""
    Nx = Nt
    U = random_links(Nt, Nx, 16)
    D = W.dirac_matrix(U, 0.2)
    levels = amg.build_hierarchy(D, Nt, Nx, [2, 2])
    L1 = levels[1]
    assert int(L1.colour.max()) + 1 == ncol
    rng = np.random.Generator(np.random.PCG64(17))
    n = 2 * L1.Nt * L1.Nx
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    e0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    col = L1.colour.reshape(-1)
    order = [s for c in range(ncol) for s in range(L1.Nt * L1.Nx) if col[s] == c]
    got = amg.gs_sweep(L1.A, L1.dinv, L1.colour, e0, r)
    assert np.max(np.abs(got - sequential_gs(L1.A, e0, r, order))) < 1e-12 * np.max(np.abs(got))


def test_eight_colouring_separates_level1_couplings():
    """(t + 3x) mod 8 separates the 21 level-1 offsets (|dp|, |dq| <= 2 without
    the corners) but not the full 5 x 5 block of offsets."""
    offs21 = [(dp, dq) for dp in range(-2, 3) for dq in range(-2, 3) if not (abs(dp) == 2 and abs(dq) == 2)]
    offs25 = [(dp, dq) for dp in range(-2, 3) for dq in range(-2, 3)]
    assert amg.eight_colour_valid(16, 16, amg.canonical_offsets(offs21, 16, 16))
    assert not amg.eight_colour_valid(16, 16, amg.canonical_offsets(offs25, 16, 16))
    assert not amg.eight_colour_valid(12, 12, amg.canonical_offsets(offs21, 12, 12))
    col = amg.colouring(16, 16, fine=False, offsets=amg.canonical_offsets(offs21, 16, 16))
    amg.check_colouring(col, amg.canonical_offsets(offs21, 16, 16))


def test_gauss_seidel_converges_when_diagonally_dominant():
    Nt = Nx = 8
    U = random_links(Nt, Nx, 18)
    D = W.dirac_matrix(U, 2.0)
    colour = amg.colouring(Nt, Nx, fine=True)
    dinv = amg.diag_block_inverses(D, Nt * Nx)
    rng = np.random.Generator(np.random.PCG64(19))
    b = rng.standard_normal(128) + 1j * rng.standard_normal(128)
    e = np.zeros(128, dtype=complex)
    for _ in range(200):
        e = amg.gs_sweep(D, dinv, colour, e, b)
    x = np.linalg.solve(D.toarray(), b)
    assert np.max(np.abs(e - x)) < 1e-12 * np.max(np.abs(x))


def test_coarsest_lu_matches_dense_solve():
    Nt = Nx = 8
    U = random_links(Nt, Nx, 20)
    D = W.dirac_matrix(U, 0.2)
    levels = amg.build_hierarchy(D, Nt, Nx, [2])
    rng = np.random.Generator(np.random.PCG64(21))
    n = levels[-1].A.shape[0]
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    import scipy.linalg as sla
    got = sla.lu_solve(levels[-1].lu, r)
    want = np.linalg.solve(levels[-1].A.toarray(), r)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_vcycle_two_level_on_exact_coarse_space_is_exact_for_coarse_vectors():
    """With no smoothing, M(D P y) = P y for every coarse vector y (P D_c^{-1} P^H D P = P)."""
    Nt = Nx = 8
    U = random_links(Nt, Nx, 22)
    D = W.dirac_matrix(U, 0.2)
    levels = amg.build_hierarchy(D, Nt, Nx, [4])
    rng = np.random.Generator(np.random.PCG64(23))
    y = rng.standard_normal(levels[1].A.shape[0]) + 1j * rng.standard_normal(levels[1].A.shape[0])
    Py = levels[0].P @ y
    got = amg.vcycle(levels, D @ Py, post_smooth=0)
    assert np.max(np.abs(got - Py)) < 1e-11 * np.max(np.abs(Py))


def test_stationary_vcycle_reduces_residual_c1_field():
    """x <- x + M(b - D x) reduces ||r|| every cycle on the 32^2, beta = 3 field
    (empirical check of the preconditioner, not a theorem)."""
    theta = fx.metropolis_u1(32, 32, 3.0, 500, 0)
    U = fx.links_from_angles(theta)
    m0 = -0.1383495190759743 + 0.05        # m_crit of this field from the oracle's spectrum
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, 32, 32, [4])
    b = W.to_flat(fx.gaussian_rhs(1, 32, 32, 1)[0])
    x = np.zeros_like(b)
    prev = np.linalg.norm(b)
    for _ in range(8):
        x = x + amg.vcycle(levels, b - D @ x)
        now = np.linalg.norm(b - D @ x)
        assert now < prev
        prev = now


# ------------------------------------------------------------------ alternative readings (comparison only)

@pytest.mark.parametrize("Nt,Nx,a", [(8, 8, 2), (8, 12, 4), (12, 8, 2)])
def test_first_lex_ownership_by_enumeration(Nt, Nx, a):
    """The first_lex owner of every non-vertex site is the smallest-index basket
    among all baskets listing it (brute force over basket_sites); the tile rule
    is the basket of the containing tile; the two agree off the borders."""
    Np, Nq = Nt // a, Nx // a
    containing = {}
    for p in range(Np):
        for q in range(Nq):
            for (t, x, _, _) in amg.basket_sites(Nt, Nx, a, p, q):
                containing.setdefault((t, x), []).append(p * Nq + q)
    lex = amg.owner_tiles(Nt, Nx, a, "first_lex")
    tile = amg.owner_tiles(Nt, Nx, a, "tile")
    role = amg.site_roles(Nt, Nx, a)
    for (t, x), bs in containing.items():
        if role[t, x] == amg.ROLE_VERTEX:
            continue
        assert lex[t, x] == min(bs)
        assert tile[t, x] == (t // a) * Nq + x // a and tile[t, x] in bs
        if role[t, x] == amg.ROLE_INTERIOR:
            assert len(bs) == 1 and lex[t, x] == tile[t, x]
        else:
            assert len(bs) == 2
    # the interpolator takes each non-vertex row from its owner's corners
    P, _ = amg.build_interpolator(W.dirac_matrix(random_links(Nt, Nx, 5), 0.2), Nt, Nx, a, ownership="first_lex")
    Pc = P.tocsr()
    for t in range(Nt):
        for x in range(Nx):
            if role[t, x] == amg.ROLE_VERTEX:
                continue
            ob = lex[t, x]
            corners = {amg.corner_vertex(Nt, Nx, a, ob // Nq, ob % Nq, c) for c in range(4)}
            for alpha in range(2):
                r = 2 * (t * Nx + x) + alpha
                cols = Pc.indices[Pc.indptr[r]:Pc.indptr[r + 1]]
                assert len(cols) == 8 and {c // 2 for c in cols} == corners


def test_first_lex_ownership_is_not_translation_invariant_but_still_solves():
    """Under first_lex a border site goes to the neighbouring basket except on
    the first tile row / column, where the periodic wrap makes its own basket
    the smaller index: the ownership map does not commute with a one-tile shift
    (the tile rule's does; the per-tile interpolator storage of the CUDA path
    relies on that).  The coarse neighbour pattern is still the 21 offsets, and
    the hierarchy gives a convergent preconditioner."""
    from oracle import krylov
    Nt = Nx = 16
    a = 2
    Np, Nq = Nt // a, Nx // a

    def shifted_by_one_tile(own):
        # owner map of the lattice shifted by one tile in t, as basket indices shifted back
        sh = np.roll(own, -a, axis=0)
        p, q = sh // Nq, sh % Nq
        return ((p - 1) % Np) * Nq + q

    tile = amg.owner_tiles(Nt, Nx, a, "tile")
    lex = amg.owner_tiles(Nt, Nx, a, "first_lex")
    assert np.array_equal(shifted_by_one_tile(tile), tile)
    assert not np.array_equal(shifted_by_one_tile(lex), lex)
    U = fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 100, 7))
    D = W.dirac_matrix(U, 0.05)
    levels = amg.build_hierarchy(D, Nt, Nx, [2, 2], ownership="first_lex")
    assert len(levels[1].offsets) == 21
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 8)[0])
    res = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 2000)
    x = np.linalg.solve(D.toarray(), b)
    assert np.linalg.norm(b - D @ res.x) / np.linalg.norm(b) <= 1e-10
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= 1e-7


@pytest.mark.parametrize("a", [2, 4])
def test_rowsum_normalisation_maps_constants_to_constants(a):
    """Row-sum normalisation: on the free field with periodic boundaries at
    m0 = 0 (where constants solve D u = 0) P 1 = 1, vertex rows stay the
    identity, no row is left unnormalised; the exact (none) interpolation does
    not map constants to constants there, because a basket drops its couplings
    to outside sites."""
    Nt = Nx = 8
    U = np.ones((2, Nt, Nx), dtype=complex)
    D = W.dirac_matrix(U, 0.0, t_sign=1.0)
    assert np.max(np.abs(D @ np.ones(2 * Nt * Nx))) < 1e-14
    stats = {}
    P, _ = amg.build_interpolator(D, Nt, Nx, a, normalization="rowsum", stats=stats)
    P0, _ = amg.build_interpolator(D, Nt, Nx, a)
    ones_c = np.ones(P.shape[1])
    assert stats["rowsum_skipped"] == 0
    assert np.max(np.abs(P @ ones_c - 1.0)) < 1e-12
    assert np.max(np.abs(P0 @ ones_c - 1.0)) > 1e-3
    role = amg.site_roles(Nt, Nx, a).reshape(-1)
    vrows = np.repeat(role == amg.ROLE_VERTEX, 2)
    assert np.array_equal(P.toarray()[vrows], P0.toarray()[vrows])


def test_rowsum_normalisation_is_not_gauge_covariant_and_still_solves():
    """With U(1) phases the row sum changes under a gauge transformation, so the
    row-sum normalised P is not covariant (the reason the method keeps the exact
    interpolation, whose covariance is pinned above); the preconditioner built
    from it still converges."""
    from oracle import krylov
    Nt = Nx = 8
    a = 2
    U = random_links(Nt, Nx, 21)
    rng = np.random.Generator(np.random.PCG64(22))
    omega = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(Nt, Nx)))
    D1, D2 = W.dirac_matrix(U, 0.3), W.dirac_matrix(W.gauge_transform_links(U, omega), 0.3)
    P1, _ = amg.build_interpolator(D1, Nt, Nx, a, normalization="rowsum")
    P2, _ = amg.build_interpolator(D2, Nt, Nx, a, normalization="rowsum")
    Om = np.diag(np.repeat(omega.reshape(-1), 2))
    OmV = np.diag(np.repeat(omega[::a, ::a].reshape(-1), 2))
    assert np.max(np.abs(P2.toarray() - Om @ P1.toarray() @ OmV.conj().T)) > 1e-3
    levels = amg.build_hierarchy(D1, Nt, Nx, [2], normalization="rowsum")
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 23)[0])
    res = krylov.fgmres(lambda v: D1 @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 2000)
    x = np.linalg.solve(D1.toarray(), b)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= 1e-7


def test_coarsest_gmres_setting_meets_its_tolerance_and_the_solve_converges():
    """The paper's coarsest solver (unpreconditioned GMRES to a relative residual
    of 0.1) as an oracle option: each coarse solve meets its tolerance, a tight
    tolerance reproduces the LU solve, and the flexible outer solve still
    reaches 1e-10 and the dense solution on the 32^2 beta = 3 field."""
    import json
    import os
    from oracle import krylov
    Nt = Nx = 32
    U = fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 500, 0))
    here = os.path.dirname(os.path.abspath(__file__))
    mc = json.load(open(os.path.join(here, "golden", "mcrit.json")))["L32_b3_s0"]["m_crit"]
    D = W.dirac_matrix(U, mc + 0.05)
    levels = amg.build_hierarchy(D, Nt, Nx, [4, 2])
    C = levels[-1]
    rng = np.random.Generator(np.random.PCG64(31))
    rc = rng.standard_normal(C.A.shape[0]) + 1j * rng.standard_normal(C.A.shape[0])
    e = amg.coarsest_gmres(C, rc)
    assert np.linalg.norm(rc - C.A @ e) <= 0.1 * np.linalg.norm(rc)
    e_tight = amg.coarsest_gmres(C, rc, tol=1e-13)
    e_lu = amg.sla.lu_solve(C.lu, rc)
    assert np.linalg.norm(e_tight - e_lu) <= 1e-10 * np.linalg.norm(e_lu)
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 1)[0])
    res = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r, coarsest="gmres"), b, 30, 1e-10, 5000)
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 5000)
    x = np.linalg.solve(D.toarray(), b)
    assert np.linalg.norm(b - D @ res.x) / np.linalg.norm(b) <= 1e-10
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= 1e-7
    assert res.iterations <= 1.5 * ref.iterations


def test_spin_split_interpolation_restores_sigma3_hermiticity():
    """Spin-split interpolation (spin-diagonal weights only): P commutes with
    sigma_3, so P^H D P inherits sigma_3 D sigma_3 = D^H (Eq. (5)); the full
    interpolation of reading 3 mixes spins and its coarse operator lacks the
    property.  The spin-split hierarchy still solves to the dense solution."""
    from oracle import krylov
    Nt = Nx = 16
    U = fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 100, 9))
    D = W.dirac_matrix(U, 0.1)
    a = 2
    s3f = sp.diags(np.tile([1.0, -1.0], Nt * Nx))
    s3c = sp.diags(np.tile([1.0, -1.0], (Nt // a) * (Nx // a)))
    P, _ = amg.build_interpolator(D, Nt, Nx, a, spin_split=True)
    Pf, _ = amg.build_interpolator(D, Nt, Nx, a)
    assert abs(s3f @ P @ s3c - P).max() < 1e-15
    Dc = amg.galerkin(P, D).toarray()
    Dcf = amg.galerkin(Pf, D).toarray()
    S = s3c.toarray()
    assert np.max(np.abs(S @ Dc @ S - Dc.conj().T)) < 1e-12 * np.max(np.abs(Dc))
    assert np.max(np.abs(S @ Dcf @ S - Dcf.conj().T)) > 1e-3 * np.max(np.abs(Dcf))
    # vertex rows stay the identity; a site's weights keep its spin
    role = amg.site_roles(Nt, Nx, a).reshape(-1)
    vrows = np.repeat(role == amg.ROLE_VERTEX, 2)
    assert np.array_equal(P.toarray()[vrows], Pf.toarray()[vrows])
    levels = amg.build_hierarchy(D, Nt, Nx, [2, 2], spin_split=True)
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 10)[0])
    res = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 2000)
    x = np.linalg.solve(D.toarray(), b)
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= 1e-7


def test_vcycle_post_smoothing_placement_two_level_formula():
    """Algorithm 1 with no pre-smoothing and two post-smoothing sweeps,
    assembled by hand from dense matrices on a 4^2 lattice (a = 2, two
    levels): e0 = P A_c^{-1} P^H r, then two red-black block Gauss-Seidel
    sweeps on A e = r, each e_R <- A_RR^{-1} (r_R - A_RB e_B) followed by
    e_B <- A_BB^{-1} (r_B - A_BR e_R) (red = even t + x).  The oracle's V-cycle
    equals it, and differs from the same two sweeps placed before the coarse
    correction (pre-smoothing) or left out."""
    Nt = Nx = 4
    rng = np.random.Generator(np.random.PCG64(77))
    U = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))
    m0 = 0.3
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, Nt, Nx, [2])
    A = D.toarray()
    P = levels[0].P.toarray()
    Ac = P.conj().T @ A @ P
    r = rng.standard_normal(2 * Nt * Nx) + 1j * rng.standard_normal(2 * Nt * Nx)
    t, x = np.divmod(np.arange(Nt * Nx), Nx)
    red_sites = np.nonzero((t + x) % 2 == 0)[0]
    black_sites = np.nonzero((t + x) % 2 == 1)[0]
    Rd = np.concatenate([[2 * s, 2 * s + 1] for s in red_sites])
    Bd = np.concatenate([[2 * s, 2 * s + 1] for s in black_sites])

    def sweep(e):
        e = e.copy()
        e[Rd] = np.linalg.solve(A[np.ix_(Rd, Rd)], r[Rd] - A[np.ix_(Rd, Bd)] @ e[Bd])
        e[Bd] = np.linalg.solve(A[np.ix_(Bd, Bd)], r[Bd] - A[np.ix_(Bd, Rd)] @ e[Rd])
        return e

    coarse = lambda v: P @ np.linalg.solve(Ac, P.conj().T @ v)
    post = sweep(sweep(coarse(r)))
    got = amg.vcycle(levels, r, post_smooth=2)
    assert np.linalg.norm(got - post) <= 1e-12 * np.linalg.norm(post)
    x1 = sweep(sweep(np.zeros_like(r)))
    pre = x1 + coarse(r - A @ x1)
    assert np.linalg.norm(got - pre) > 1e-3 * np.linalg.norm(post)
    assert np.linalg.norm(got - coarse(r)) > 1e-3 * np.linalg.norm(post)
    assert np.linalg.norm(amg.vcycle(levels, r, post_smooth=0) - coarse(r)) <= 1e-12 * np.linalg.norm(post)


@pytest.mark.parametrize("Nt,Nx", [(16, 16), (24, 32), (40, 24)])
def test_local_galerkin_rows_equal_the_global_product(Nt, Nx):
    """galerkin_rows builds rows of the first coarse operator from the baskets
    near each coarse site and the rows of D at their sites only; they equal the
    rows of the global Galerkin product P^H D P (16 x 16: the three-tile reach
    wraps around the 4 x 4 coarse lattice)."""
    rng = np.random.Generator(np.random.PCG64(90 + Nt))
    U = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))
    m0 = 0.13
    a = 4
    D = W.dirac_matrix(U, m0)
    P, _ = amg.build_interpolator(D, Nt, Nx, a)
    Ac = amg.galerkin(P, D).tocsr()
    Nq = Nx // a
    verts = [(0, 0), (Nt // a - 1, Nq - 1), (1, Nq // 2), (Nt // a // 2, 0)]
    rows = amg.galerkin_rows(U, m0, a, verts)
    scale = np.max(np.abs(Ac.data))
    for (p, q) in verts:
        v = p * Nq + q
        blocks = rows[(p, q)]
        dense = Ac[[2 * v, 2 * v + 1]].toarray()
        got = np.zeros_like(dense)
        for w, blk in blocks.items():
            got[:, 2 * w:2 * w + 2] += blk
        assert np.max(np.abs(got - dense)) <= 1e-13 * scale, (p, q)
        # and only sites within two coarse sites carry blocks (21 offsets)
        nz = [w for w, blk in blocks.items() if np.max(np.abs(blk)) > 1e-14 * scale]
        assert len(nz) <= 21


def test_dirac_rows_are_rows_of_the_matrix():
    rng = np.random.Generator(np.random.PCG64(95))
    U = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, 8, 12)))
    D = W.dirac_matrix(U, 0.2)
    sites = [(0, 0), (7, 11), (3, 5), (0, 11)]
    Dr = W.dirac_rows(U, 0.2, sites)
    for (t, x) in sites:
        for alpha in range(2):
            r = 2 * (t * 12 + x) + alpha
            assert (Dr[r] != D[r]).nnz == 0
    assert Dr.nnz == sum(D[2 * (t * 12 + x) + al].nnz for (t, x) in sites for al in range(2))
