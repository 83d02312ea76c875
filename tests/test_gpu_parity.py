"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances: FP64 kernels 1e-13 relative (max-norm over the output), setup
products (P, coarse blocks) 1e-12, FP32 stencil 2e-6; whole solves reach the
1e-10 true relative residual with iteration counts within 10 % of the oracle's.
"""
import numpy as np
import pytest

from oracle import amg, krylov
from oracle import wilson as W
from paper_2608_03515_b300 import fixtures as fx

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2608_03515_b300 import build  # noqa: E402

build.build()
from paper_2608_03515_b300 import amamg as A  # noqa: E402

DEV = torch.device("cuda:0")


def canary(*shape_and_dtype):
    """canary(d0, d1, ..., dtype) or canary(shape, dtype): an output buffer
    filled with NaN (a canary): an element the kernel does not write stays NaN
    and fails the element-wise comparison."""
    *shape, dtype = shape_and_dtype
    if len(shape) == 1 and not isinstance(shape[0], int):
        shape = tuple(shape[0])
    return torch.full(tuple(shape), complex(float("nan"), float("nan")), dtype=dtype, device=DEV)


def canary_like(t):
    return canary(t.shape, t.dtype)


def random_links(Nt, Nx, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(got, want):
    return np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)


def lattice_vec(flat, Nt, Nx):
    return W.from_flat(flat, Nt, Nx)


def oracle_P_tiles(P, Nt, Nx, a):
    """Oracle interpolator in the library's per-tile [8][nrows] layout."""
    Np, Nq = Nt // a, Nx // a
    nrows = 2 * (a * a - 1)
    Pd = P.tocsr()
    out = np.zeros((Np * Nq, 8, nrows), dtype=complex)
    for p in range(Np):
        for q in range(Nq):
            tile = p * Nq + q
            for lr in range(nrows):
                l, alpha = lr // 2 + 1, lr % 2
                t, x = p * a + l // a, q * a + l % a
                row = 2 * (t * Nx + x) + alpha
                for c in range(4):
                    v = amg.corner_vertex(Nt, Nx, a, p, q, c)
                    for beta in range(2):
                        out[tile, 2 * c + beta, lr] = Pd[row, 2 * v + beta]
    return out


def make(Nt, Nx, aggs, m0=0.1, seed=1, U=None, precision=0, restart=30):
    U = random_links(Nt, Nx, seed) if U is None else U
    params = A.make_params(aggs, precision=precision, restart=restart)
    hier = A.setup(dev(U), m0, params)
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, Nt, Nx, aggs)
    return U, D, hier, levels


# ------------------------------------------------------------------ Wilson stencil

@pytest.mark.parametrize("Nt,Nx,R", [(8, 8, 1), (16, 32, 3), (34, 18, 2)])
def test_apply_D_fp64_and_fp32(Nt, Nx, R):
    U = random_links(Nt, Nx, 3)
    hier = A.setup(dev(U), 0.07, A.make_params([2]))
    psi = fx.gaussian_rhs(R, Nt, Nx, 4)
    out = canary(R, 2, Nt, Nx, torch.complex128)
    A.apply_D(hier, dev(psi), out)
    got = host(out)
    want = np.stack([W.apply_dirac(U, 0.07, psi[r]) for r in range(R)])
    assert relerr(got, want) <= 1e-13
    D = W.dirac_matrix(U, 0.07)
    for r in range(R):
        assert relerr(got[r], lattice_vec(D @ W.to_flat(psi[r]), Nt, Nx)) <= 1e-13
    # FP32: inputs rounded to complex64, reference in FP64 on the rounded inputs
    psi32 = psi.astype(np.complex64)
    out32 = canary(R, 2, Nt, Nx, torch.complex64)
    A.apply_D(hier, dev(psi32, torch.complex64), out32)
    U32 = U.astype(np.complex64).astype(np.complex128)
    want32 = np.stack([W.apply_dirac(U32, 0.07, psi32[r].astype(np.complex128)) for r in range(R)])
    assert relerr(host(out32), want32) <= 2e-6


def test_apply_D_full_size_256_properties():
    """256^2 (the benchmark lattice): full comparison with the matrix-free oracle."""
    Nt = Nx = 256
    theta = fx.metropolis_u1(Nt, Nx, 6.0, 20, 2)
    U = fx.links_from_angles(theta)
    hier = A.setup(dev(U), 0.03, A.make_params([4, 2]))
    psi = fx.gaussian_rhs(1, Nt, Nx, 3)
    out = canary(1, 2, Nt, Nx, torch.complex128)
    A.apply_D(hier, dev(psi), out)
    assert relerr(host(out)[0], W.apply_dirac(U, 0.03, psi[0])) <= 1e-13


# ------------------------------------------------------------------ structure and setup

@pytest.mark.parametrize("Nt,Nx,aggs", [(8, 8, [4]), (16, 16, [2, 2]), (32, 32, [4, 2]), (16, 24, [4])])
def test_structure_bit_exact(Nt, Nx, aggs):
    U, D, hier, levels = make(Nt, Nx, aggs)
    for l in range(len(aggs)):
        role, owner, offs = A.export_structure(hier, l)
        L = levels[l]
        assert np.array_equal(role, amg.site_roles(L.Nt, L.Nx, aggs[l]))
        assert np.array_equal(owner, amg.owner_tiles(L.Nt, L.Nx, aggs[l]))
        assert offs == [tuple(o) for o in levels[l + 1].offsets]
        assert hier.level_info(l + 1)[:2] == (levels[l + 1].Nt, levels[l + 1].Nx)


@pytest.mark.parametrize("Nt,Nx,aggs", [(8, 8, [4]), (8, 8, [2]), (16, 16, [2, 2]), (32, 32, [4, 2]),
                                        (32, 16, [4, 2])])
def test_interpolator_and_galerkin_fp64(Nt, Nx, aggs):
    U, D, hier, levels = make(Nt, Nx, aggs, m0=0.05, seed=5)
    for l, a in enumerate(aggs):
        L = levels[l]
        want = oracle_P_tiles(L.P, L.Nt, L.Nx, a)
        got = canary(want.shape, torch.complex128)
        A.export_P(hier, l, got)
        assert relerr(host(got), want) <= 1e-12
        C = levels[l + 1]
        Bw = amg.block_stencil(C.A, C.offsets, C.Nt, C.Nx)            # [K, n, 2, 2]
        Bw = np.transpose(Bw.reshape(len(C.offsets), C.Nt * C.Nx, 4), (0, 2, 1))
        Bg = canary(Bw.shape, torch.complex128)
        A.export_coarse(hier, l + 1, Bg)
        assert relerr(host(Bg), Bw) <= 1e-12


def test_spin_split_hierarchy_matches_oracle():
    """The opt-in spin-split hierarchy (spin-diagonal interpolation weights,
    amamg_params.spin_split = 1) against the oracle's: interpolator tiles and
    coarse blocks to 1e-12, and the FP64 solve on the 32^2 beta = 3 field to
    1e-10 with an iteration count within 10 % of the oracle's."""
    import json
    import os
    Nt = Nx = 32
    aggs = [4, 2]
    U = fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 500, 0))
    here = os.path.dirname(os.path.abspath(__file__))
    m0 = json.load(open(os.path.join(here, "golden", "mcrit.json")))["L32_b3_s0"]["m_crit"] + 0.05
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, Nt, Nx, aggs, spin_split=True)
    hier = A.setup(dev(U), m0, A.make_params(aggs, spin_split=True))
    for l, a in enumerate(aggs):
        L = levels[l]
        want = oracle_P_tiles(L.P, L.Nt, L.Nx, a)
        got = canary(want.shape, torch.complex128)
        A.export_P(hier, l, got)
        assert relerr(host(got), want) <= 1e-12
        C = levels[l + 1]
        Bw = amg.block_stencil(C.A, C.offsets, C.Nt, C.Nx)
        Bw = np.transpose(Bw.reshape(len(C.offsets), C.Nt * C.Nx, 4), (0, 2, 1))
        Bg = canary(Bw.shape, torch.complex128)
        A.export_coarse(hier, l + 1, Bg)
        assert relerr(host(Bg), Bw) <= 1e-12
    psi = fx.gaussian_rhs(1, Nt, Nx, 1)
    x = canary(psi.shape, torch.complex128)
    info = A.solve(hier, dev(psi), x)
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), W.to_flat(psi[0]), 30, 1e-10, 5000)
    b = W.to_flat(psi[0])
    res = np.linalg.norm(b - D @ W.to_flat(host(x)[0])) / np.linalg.norm(b)
    assert info[0].status == A.OK and res <= 1e-10
    assert abs(info[0].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations)


# ------------------------------------------------------------------ transfers, coarse operator

@pytest.mark.parametrize("Nt,Nx,aggs,R", [(16, 16, [4], 2), (32, 32, [4, 2], 1), (16, 24, [2, 2], 3)])
def test_transfers_and_coarse_apply_fp64(Nt, Nx, aggs, R):
    U, D, hier, levels = make(Nt, Nx, aggs, m0=0.2, seed=6)
    rng = np.random.Generator(np.random.PCG64(7))
    for l in range(len(aggs)):
        F, C = levels[l], levels[l + 1]
        ec = rng.standard_normal((R, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((R, 2, C.Nt, C.Nx))
        ef = rng.standard_normal((R, 2, F.Nt, F.Nx)) + 1j * rng.standard_normal((R, 2, F.Nt, F.Nx))
        out_f = canary(R, 2, F.Nt, F.Nx, torch.complex128)
        out_c = canary(R, 2, C.Nt, C.Nx, torch.complex128)
        A.apply_P(hier, l, dev(ec), out_f)
        A.apply_PH(hier, l, dev(ef), out_c)
        gf, gc = host(out_f), host(out_c)
        for r in range(R):
            wf = lattice_vec(F.P @ W.to_flat(ec[r]), F.Nt, F.Nx)
            wc = lattice_vec(F.P.conj().T @ W.to_flat(ef[r]), C.Nt, C.Nx)
            assert relerr(gf[r], wf) <= 1e-13
            assert relerr(gc[r], wc) <= 1e-13
        A.apply_coarse(hier, l + 1, dev(ec), out_c)
        gc = host(out_c)
        for r in range(R):
            assert relerr(gc[r], lattice_vec(C.A @ W.to_flat(ec[r]), C.Nt, C.Nx)) <= 1e-12


# ------------------------------------------------------------------ smoother, coarsest, V-cycle

@pytest.mark.parametrize("sweeps,Nt", [(1, 32), (2, 32), (2, 128)])
def test_smoothers_fp64(sweeps, Nt):
    """Level 1 (21 offsets, 8 colours) is 16^2 at Nt = 32 and 64^2 at Nt = 128:
    the default FP64 coarse kernel (cooperative grid sweep) at 32 and 512 sites
    per colour."""
    Nx = Nt
    U, D, hier, levels = make(Nt, Nx, [2, 2], m0=0.1, seed=8)
    rng = np.random.Generator(np.random.PCG64(9))
    for l in range(2):
        L = levels[l]
        r = rng.standard_normal((1, 2, L.Nt, L.Nx)) + 1j * rng.standard_normal((1, 2, L.Nt, L.Nx))
        e0 = rng.standard_normal((1, 2, L.Nt, L.Nx)) + 1j * rng.standard_normal((1, 2, L.Nt, L.Nx))
        e = dev(e0)
        A.smooth(hier, l, dev(r), e, sweeps)
        want = W.to_flat(e0[0])
        for _ in range(sweeps):
            want = amg.gs_sweep(L.A, L.dinv, L.colour, want, W.to_flat(r[0]))
        assert relerr(host(e)[0], lattice_vec(want, L.Nt, L.Nx)) <= 1e-12


def quantised_operator(L):
    """Level operator as the FP32 Gauss-Seidel kernels hold it: off-diagonal
    blocks in FP16 + per-block scale (oracle.mixed), diagonal blocks exact."""
    import scipy.sparse as sp
    from oracle import mixed
    Bq = mixed.quantise_blocks(amg.block_stencil(L.A, L.offsets, L.Nt, L.Nx))
    Bq[0] = amg.block_stencil(L.A, L.offsets, L.Nt, L.Nx)[0]
    n = L.Nt * L.Nx
    rows, cols, vals = [], [], []
    for k, (dt, dx) in enumerate(L.offsets):
        for v in range(n):
            tv, xv = divmod(v, L.Nx)
            w = ((tv + dt) % L.Nt) * L.Nx + (xv + dx) % L.Nx
            for al in range(2):
                for be in range(2):
                    rows.append(2 * v + al); cols.append(2 * w + be); vals.append(Bq[k, v, al, be])
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n))


def test_coarse_gs_kernels_agree_with_oracle(monkeypatch):
    """Every coarse Gauss-Seidel kernel (one launch per colour, L2 cluster,
    distributed-shared-memory cluster, cooperative grid, site-owning blocks with
    neighbour waits) on a 32^2 level with 21
    offsets (8 colours) and a 16^2 level with 25 offsets (16 colours), two
    right-hand sides, FP64 and FP32 (FP16 + scale blocks)."""
    from oracle import mixed
    Nt = Nx = 64
    aggs = [2, 2, 2]
    U = random_links(Nt, Nx, 31)
    levels = amg.build_hierarchy(W.dirac_matrix(U, 0.1), Nt, Nx, aggs)
    assert levels[1].colour.max() + 1 == 8 and levels[2].colour.max() + 1 == 16
    rng = np.random.Generator(np.random.PCG64(32))
    R = 2
    inputs = {}
    for l in (1, 2):
        L = levels[l]
        shape = (R, 2, L.Nt, L.Nx)
        inputs[l] = [mixed.round32(rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) for _ in range(2)]
    got64 = {}
    for kind in ("colour", "cluster", "dsmem", "grid", "owner"):
        monkeypatch.setenv("AMAMG_COARSE_GS", kind)
        hier = A.setup(dev(U), 0.1, A.make_params(aggs))
        for l in (1, 2):
            L = levels[l]
            r, e0 = inputs[l]
            e = dev(e0)
            A.smooth(hier, l, dev(r), e, 2)
            g = host(e)
            Aq = quantised_operator(L)
            dinv32 = mixed.round32(L.dinv)
            e32 = dev(e0, torch.complex64)
            A.smooth(hier, l, dev(r, torch.complex64), e32, 2)
            g32 = host(e32)
            for q in range(R):
                want = W.to_flat(e0[q])
                want32 = W.to_flat(e0[q])
                for _ in range(2):
                    want = amg.gs_sweep(L.A, L.dinv, L.colour, want, W.to_flat(r[q]))
                    want32 = amg.gs_sweep(Aq, dinv32, L.colour, want32, W.to_flat(r[q]))
                assert relerr(g[q], lattice_vec(want, L.Nt, L.Nx)) <= 1e-12, (kind, l, q)
                assert relerr(g32[q], lattice_vec(want32, L.Nt, L.Nx)) <= 1e-5, (kind, l, q)
            got64.setdefault(l, []).append(g)
        hier.destroy()
    for l in (1, 2):
        for g in got64[l][1:]:
            assert relerr(g, got64[l][0]) <= 1e-14


@pytest.mark.parametrize("R", [1, 3])
def test_fused_fine_post_smoother_equals_separate_launches(monkeypatch, R):
    """The fine-level end of the V-cycle (prolongation + two red-black sweeps)
    as one cooperative launch gives the result of the separate kernels (same
    arithmetic per site), in FP64 and FP32, and the FP64 V-cycle matches the
    oracle's."""
    Nt, Nx = 64, 32
    aggs = [4, 2]
    U = random_links(Nt, Nx, 41)
    levels = amg.build_hierarchy(W.dirac_matrix(U, 0.1), Nt, Nx, aggs)
    psi = fx.gaussian_rhs(R, Nt, Nx, 42)
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("AMAMG_FINE_FUSED", fused)
        hier = A.setup(dev(U), 0.1, A.make_params(aggs))
        e64 = canary(psi.shape, torch.complex128)
        e32 = canary(psi.shape, torch.complex64)
        A.vcycle(hier, dev(psi), e64)
        A.vcycle(hier, dev(psi, torch.complex64), e32)
        out[fused] = (host(e64), host(e32))
        hier.destroy()
    assert relerr(out["1"][0], out["0"][0]) <= 1e-15
    assert relerr(out["1"][1], out["0"][1]) <= 1e-6
    for r in range(R):
        want = lattice_vec(amg.vcycle(levels, W.to_flat(psi[r])), Nt, Nx)
        assert relerr(out["1"][0][r], want) <= 1e-11


def test_owner_sweep_wait_time_out_is_reported_and_handle_recovers():
    """A block of the owner sweep that never publishes makes its neighbours'
    bounded waits run out: the library reports AMAMG_ERR_TIMEOUT (no fault, no
    hang), re-arms its counters, and the next smoothing is correct again."""
    import time
    Nt = Nx = 64
    aggs = [2, 2, 2]
    U, D, hier, levels = make(Nt, Nx, aggs, m0=0.1, seed=33)
    L = levels[1]
    rng = np.random.Generator(np.random.PCG64(34))
    for prec in (A.F64, A.F32):
        t0 = time.time()
        assert A.selftest_sync_timeout(hier, 1, prec) == A.OK      # enqueued; not reported by itself
        assert A.sync_status(hier) == A.ERR_TIMEOUT
        assert time.time() - t0 < 60.0
        assert A.sync_status(hier) == A.OK                          # re-armed
        r = rng.standard_normal((1, 2, L.Nt, L.Nx)) + 1j * rng.standard_normal((1, 2, L.Nt, L.Nx))
        e0 = rng.standard_normal((1, 2, L.Nt, L.Nx)) + 1j * rng.standard_normal((1, 2, L.Nt, L.Nx))
        e = dev(e0)
        A.smooth(hier, 1, dev(r), e, 2)
        want = W.to_flat(e0[0])
        for _ in range(2):
            want = amg.gs_sweep(L.A, L.dinv, L.colour, want, W.to_flat(r[0]))
        assert relerr(host(e)[0], lattice_vec(want, L.Nt, L.Nx)) <= 1e-12


def test_coarsest_solve_and_vcycle_fp64():
    Nt = Nx = 32
    U, D, hier, levels = make(Nt, Nx, [4, 2], m0=0.05, seed=10)
    C = levels[-1]
    rng = np.random.Generator(np.random.PCG64(11))
    rc = rng.standard_normal((2, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((2, 2, C.Nt, C.Nx))
    ec = canary(rc.shape, torch.complex128)
    A.coarsest_solve(hier, dev(rc), ec)
    import scipy.linalg as sla
    got = host(ec)
    cond = np.linalg.cond(C.A.toarray())
    for r in range(2):
        want = lattice_vec(sla.lu_solve(C.lu, W.to_flat(rc[r])), C.Nt, C.Nx)
        assert relerr(got[r], want) <= 1e-15 * cond * 10
    psi = fx.gaussian_rhs(2, Nt, Nx, 12)
    e = canary(psi.shape, torch.complex128)
    A.vcycle(hier, dev(psi), e)
    got = host(e)
    for r in range(2):
        want = lattice_vec(amg.vcycle(levels, W.to_flat(psi[r])), Nt, Nx)
        assert relerr(got[r], want) <= 1e-11


# ------------------------------------------------------------------ whole solves

def oracle_solve(D, levels, b, m, tol=1e-10):
    return krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, m, tol, 5000)


@pytest.mark.parametrize("aggs", [[4], [4, 2]])
def test_solve_fp64_matches_oracle_c1_field(aggs):
    """32^2, beta = 3 quenched field, m0 = m_crit + 0.05 (m_crit from the oracle's spectrum)."""
    Nt = Nx = 32
    theta = fx.metropolis_u1(Nt, Nx, 3.0, 500, 0)
    U = fx.links_from_angles(theta)
    m0 = -0.1383495190759743 + 0.05
    U_, D, hier, levels = make(Nt, Nx, aggs, m0=m0, U=U)
    psi = fx.gaussian_rhs(1, Nt, Nx, 1)
    x = canary(psi.shape, torch.complex128)
    info = A.solve(hier, dev(psi), x)
    ref = oracle_solve(D, levels, W.to_flat(psi[0]), 30)
    assert info[0].status == A.OK
    xg = host(x)[0]
    # independent FP64 check of the returned solution
    res = np.linalg.norm(W.to_flat(psi[0]) - D @ W.to_flat(xg)) / np.linalg.norm(psi[0])
    assert res <= 1e-10 and info[0].true_relres <= 1e-10
    assert abs(info[0].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations)
    assert relerr(xg, lattice_vec(ref.x, Nt, Nx)) <= 1e-7


def test_solve_multi_rhs_each_equals_single():
    Nt = Nx = 16
    U, D, hier, levels = make(Nt, Nx, [2, 2], m0=0.05, seed=13)
    psi = fx.gaussian_rhs(3, Nt, Nx, 14)
    x = canary(psi.shape, torch.complex128)
    info = A.solve(hier, dev(psi), x)
    xb = host(x)
    for r in range(3):
        x1 = canary((1,) + psi.shape[1:], torch.complex128)
        i1 = A.solve(hier, dev(psi[r:r + 1]), x1)
        assert i1[0].iterations == info[r].iterations
        assert relerr(host(x1)[0], xb[r]) <= 1e-12
        assert info[r].true_relres <= 1e-10


def test_solve_mixed_precision_reaches_tolerance():
    Nt = Nx = 32
    theta = fx.metropolis_u1(Nt, Nx, 3.0, 500, 0)
    U = fx.links_from_angles(theta)
    m0 = -0.1383495190759743 + 0.05
    hier64 = A.setup(dev(U), m0, A.make_params([4, 2]))
    hier32 = A.setup(dev(U), m0, A.make_params([4, 2], precision=A.SOLVE_MIXED))
    psi = fx.gaussian_rhs(1, Nt, Nx, 1)
    x64 = canary(psi.shape, torch.complex128)
    x32 = canary(psi.shape, torch.complex128)
    i64 = A.solve(hier64, dev(psi), x64)
    i32 = A.solve(hier32, dev(psi), x32)
    assert i32[0].status == A.OK and i32[0].true_relres <= 1e-10
    D = W.dirac_matrix(U, m0)
    res = np.linalg.norm(W.to_flat(psi[0]) - D @ W.to_flat(host(x32)[0])) / np.linalg.norm(psi[0])
    assert res <= 1e-10
    assert i32[0].iterations <= 1.1 * i64[0].iterations + 1


# ------------------------------------------------------------------ edge cases

def test_zero_and_nonfinite_rhs():
    Nt = Nx = 16
    U, D, hier, levels = make(Nt, Nx, [4], m0=0.1, seed=15)
    psi = np.zeros((2, 2, Nt, Nx), dtype=complex)
    psi[1] = fx.gaussian_rhs(1, Nt, Nx, 16)[0]
    x = torch.full(psi.shape, 7.0, dtype=torch.complex128, device=DEV)
    info = A.solve(hier, dev(psi), x)
    assert info[0].status == A.OK and info[0].iterations == 0
    assert np.all(host(x)[0] == 0)
    assert info[1].status == A.OK and info[1].true_relres <= 1e-10
    psi[1, 0, 3, 3] = np.nan
    with pytest.raises(A.AmamgError) as ei:
        A.solve(hier, dev(psi), x)
    assert ei.value.status == A.ERR_NONFINITE


def test_invalid_arguments_rejected():
    Nt = Nx = 16
    U, D, hier, levels = make(Nt, Nx, [4], m0=0.1, seed=17)
    v = torch.zeros(1, 2, Nt, Nx, dtype=torch.complex128, device=DEV)
    with pytest.raises(A.AmamgError):
        A.apply_P(hier, 1, v, v)          # level 1 is the coarsest: nothing below it
    with pytest.raises(A.AmamgError):
        A.apply_coarse(hier, 0, v, v)     # level 0 is the Wilson operator
    L = A.lib()
    assert L.amamg_apply_D(hier.h, None, None, 1, 0, None) == A.ERR_INVALID_ARG


# ------------------------------------------------------------------ FP32 path (FP16 + scale storage)

@pytest.mark.parametrize("Nt", [32, 64])
def test_fp32_transfers_coarse_and_smoothers_match_emulated_storage(Nt):
    """FP32 kernels against FP64 arithmetic on the emulated FP16+scale operators
    and complex64-rounded inputs (oracle.mixed): FP32 rounding only.  The
    coarse level (8 colours) is 8^2 at Nt = 32 (cooperative grid sweep) and
    16^2 at Nt = 64 (cluster sweep with the level in distributed shared memory)."""
    from oracle import mixed
    Nx = Nt
    aggs = [4, 2]
    U, D, hier, levels = make(Nt, Nx, aggs, m0=0.2, seed=21)
    rng = np.random.Generator(np.random.PCG64(22))
    R = 2
    for l, a in enumerate(aggs):
        F, C = levels[l], levels[l + 1]
        Pq = mixed.quantise_tiles(oracle_P_tiles(F.P, F.Nt, F.Nx, a))
        ec = mixed.round32(rng.standard_normal((R, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((R, 2, C.Nt, C.Nx)))
        ef = mixed.round32(rng.standard_normal((R, 2, F.Nt, F.Nx)) + 1j * rng.standard_normal((R, 2, F.Nt, F.Nx)))
        out_f = canary(R, 2, F.Nt, F.Nx, torch.complex64)
        out_c = canary(R, 2, C.Nt, C.Nx, torch.complex64)
        A.apply_P(hier, l, dev(ec, torch.complex64), out_f)
        A.apply_PH(hier, l, dev(ef, torch.complex64), out_c)
        gf, gc = host(out_f), host(out_c)
        Np, Nq = F.Nt // a, F.Nx // a
        nrows = 2 * (a * a - 1)
        for r in range(R):
            wf = np.zeros((2, F.Nt, F.Nx), dtype=complex)
            wc = np.zeros((2, C.Nt, C.Nx), dtype=complex)
            for p in range(Np):
                for q in range(Nq):
                    tile = p * Nq + q
                    corners = [amg.corner_vertex(F.Nt, F.Nx, a, p, q, c) for c in range(4)]
                    ecv = np.array([ec[r, beta].reshape(-1)[corners[c]] for c in range(4) for beta in range(2)])
                    vals = Pq[tile].T @ ecv                                   # [nrows]
                    for lr in range(nrows):
                        l_, alpha = lr // 2 + 1, lr % 2
                        t, x = p * a + l_ // a, q * a + l_ % a
                        wf[alpha, t, x] = vals[lr]
                        for c in range(4):
                            for beta in range(2):
                                wc[beta].reshape(-1)[corners[c]] += np.conj(Pq[tile, 2 * c + beta, lr]) * ef[r, alpha, t, x]
                    wf[:, p * a, q * a] = ec[r, :, p, q]
                    wc[:, p, q] += ef[r, :, p * a, q * a]
            assert relerr(gf[r], wf) <= 2e-6
            assert relerr(gc[r], wc) <= 2e-6
        # coarse operator with FP16 blocks
        Bq = mixed.quantise_blocks(amg.block_stencil(C.A, C.offsets, C.Nt, C.Nx))
        A.apply_coarse(hier, l + 1, dev(ec, torch.complex64), out_c)
        gc = host(out_c)
        for r in range(R):
            want = np.zeros((2, C.Nt * C.Nx), dtype=complex)
            x0 = ec[r].reshape(2, -1)
            for k, (dt, dx) in enumerate(C.offsets):
                for v in range(C.Nt * C.Nx):
                    tv, xv = divmod(v, C.Nx)
                    w = ((tv + dt) % C.Nt) * C.Nx + (xv + dx) % C.Nx
                    want[:, v] += Bq[k, v] @ x0[:, w]
            assert relerr(gc[r], want.reshape(2, C.Nt, C.Nx)) <= 2e-6
    # fine red-black sweep with FP32 links and (m0 + 2) in FP32
    L0 = levels[0]
    r0 = mixed.round32(fx.gaussian_rhs(1, Nt, Nx, 23))
    e0 = mixed.round32(fx.gaussian_rhs(1, Nt, Nx, 24))
    e = dev(e0, torch.complex64)
    A.smooth(hier, 0, dev(r0, torch.complex64), e, 2)
    D32 = W.dirac_matrix(mixed.round32(U), 0.2)
    want = W.to_flat(e0[0])
    for _ in range(2):
        want = amg.gs_sweep(D32, L0.dinv, L0.colour, want, W.to_flat(r0[0]))
    assert relerr(host(e)[0], lattice_vec(want, Nt, Nx)) <= 1e-5
    # coarse multicolour sweep: FP16 off-diagonal blocks, FP32-rounded diagonal inverses
    L1 = levels[1]
    Bq = mixed.quantise_blocks(amg.block_stencil(L1.A, L1.offsets, L1.Nt, L1.Nx))
    Bex = amg.block_stencil(L1.A, L1.offsets, L1.Nt, L1.Nx)
    Bq[0] = Bex[0]                                                  # diagonal blocks stay exact
    n1 = L1.Nt * L1.Nx
    rows, cols, vals = [], [], []
    for k, (dt, dx) in enumerate(L1.offsets):
        for v in range(n1):
            tv, xv = divmod(v, L1.Nx)
            w = ((tv + dt) % L1.Nt) * L1.Nx + (xv + dx) % L1.Nx
            for al in range(2):
                for be in range(2):
                    rows.append(2 * v + al); cols.append(2 * w + be); vals.append(Bq[k, v, al, be])
    import scipy.sparse as sp
    Aq = sp.csr_matrix((vals, (rows, cols)), shape=(2 * n1, 2 * n1))
    dinv32 = mixed.round32(L1.dinv)
    r1 = mixed.round32(rng.standard_normal((1, 2, L1.Nt, L1.Nx)) + 1j * rng.standard_normal((1, 2, L1.Nt, L1.Nx)))
    e1 = mixed.round32(rng.standard_normal((1, 2, L1.Nt, L1.Nx)) + 1j * rng.standard_normal((1, 2, L1.Nt, L1.Nx)))
    eg = dev(e1, torch.complex64)
    A.smooth(hier, 1, dev(r1, torch.complex64), eg, 2)
    want = W.to_flat(e1[0])
    for _ in range(2):
        want = amg.gs_sweep(Aq, dinv32, L1.colour, want, W.to_flat(r1[0]))
    assert relerr(host(eg)[0], lattice_vec(want, L1.Nt, L1.Nx)) <= 1e-5


def test_graph_replay_matches_eager_profiled_solve():
    """The captured-graph Arnoldi steps and the eager (profiled) path give the same solve."""
    Nt = Nx = 32
    U, D, hier, levels = make(Nt, Nx, [4, 2], m0=0.05, seed=25)
    psi = fx.gaussian_rhs(2, Nt, Nx, 26)
    x1 = canary(psi.shape, torch.complex128)
    x2 = canary(psi.shape, torch.complex128)
    i1 = A.solve(hier, dev(psi), x1)
    A.profile_enable(hier, True)
    i2 = A.solve(hier, dev(psi), x2)
    A.profile_enable(hier, False)
    prof = A.profile_get(hier)
    assert any(name.startswith("dslash") for name, *_ in prof)
    assert [i.iterations for i in i1] == [i.iterations for i in i2]
    assert relerr(host(x1), host(x2)) <= 1e-13
    n0 = A.launch_count(hier)
    A.solve(hier, dev(psi), x1)
    assert A.launch_count(hier) > n0


@pytest.mark.parametrize("R", [4, 9, 17])
def test_coarse_apply_many_rhs_loads_blocks_once_same_result(R):
    """The right-hand-side-blocked coarse apply (R >= 4) gives every right-hand
    side bit for bit the result of the one-right-hand-side kernel, and the
    oracle's Galerkin operator to 1e-12 (FP64); FP32 likewise against R = 1."""
    U, D, hier, levels = make(32, 32, [4, 2], m0=0.2, seed=6)
    rng = np.random.Generator(np.random.PCG64(8))
    for l in (1, 2):
        C = levels[l]
        for dt in (torch.complex128, torch.complex64):
            xin = rng.standard_normal((R, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((R, 2, C.Nt, C.Nx))
            xd = dev(xin, dt)
            out = canary_like(xd)
            A.apply_coarse(hier, l, xd, out)
            got = host(out)
            for r in range(R):
                one = canary_like(xd[r:r + 1])
                A.apply_coarse(hier, l, xd[r:r + 1].contiguous(), one)
                assert np.array_equal(host(one)[0], got[r])
                if dt == torch.complex128:
                    want = lattice_vec(C.A @ W.to_flat(xin[r]), C.Nt, C.Nx)
                    assert relerr(got[r], want) <= 1e-12


@pytest.mark.parametrize("R", [4, 9, 17])
def test_transfers_many_rhs_load_P_once_same_result(R):
    """The right-hand-side-blocked prolongation and restriction (R >= 4: each
    entry of P loaded once per group of right-hand sides) give every
    right-hand side bit for bit the one-right-hand-side kernels' result, and
    the oracle's P and P^H to 1e-13 (FP64)."""
    U, D, hier, levels = make(32, 32, [4, 2], m0=0.2, seed=7)
    rng = np.random.Generator(np.random.PCG64(9))
    for l in (0, 1):
        F, C = levels[l], levels[l + 1]
        for dt in (torch.complex128, torch.complex64):
            ec = rng.standard_normal((R, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((R, 2, C.Nt, C.Nx))
            ef = rng.standard_normal((R, 2, F.Nt, F.Nx)) + 1j * rng.standard_normal((R, 2, F.Nt, F.Nx))
            ecd, efd = dev(ec, dt), dev(ef, dt)
            out_f, out_c = canary_like(efd), canary_like(ecd)
            A.apply_P(hier, l, ecd, out_f)
            A.apply_PH(hier, l, efd, out_c)
            gf, gc = host(out_f), host(out_c)
            for r in range(R):
                one_f, one_c = canary_like(efd[r:r + 1]), canary_like(ecd[r:r + 1])
                A.apply_P(hier, l, ecd[r:r + 1].contiguous(), one_f)
                A.apply_PH(hier, l, efd[r:r + 1].contiguous(), one_c)
                assert np.array_equal(host(one_f)[0], gf[r])
                assert np.array_equal(host(one_c)[0], gc[r])
                if dt == torch.complex128:
                    wf = lattice_vec(F.P @ W.to_flat(ec[r]), F.Nt, F.Nx)
                    wc = lattice_vec(F.P.conj().T @ W.to_flat(ef[r]), C.Nt, C.Nx)
                    assert relerr(gf[r], wf) <= 1e-13
                    assert relerr(gc[r], wc) <= 1e-13


@pytest.mark.parametrize("R", [4, 6])
def test_grid_sweep_groups_of_right_hand_sides_same_result(monkeypatch, R):
    """The cooperative grid sweep with R >= 4 takes a site and a group of 4
    right-hand sides per work unit (the site's blocks loaded once per group; a
    ragged last group at R = 6); every right-hand side gets the one-at-a-time
    sweep's result bit for bit, and the oracle's sequential Gauss-Seidel to
    1e-12 (FP64)."""
    monkeypatch.setenv("AMAMG_COARSE_GS", "grid")
    Nt = Nx = 64
    aggs = [2, 2, 2]
    U = random_links(Nt, Nx, 33)
    levels = amg.build_hierarchy(W.dirac_matrix(U, 0.1), Nt, Nx, aggs)
    hier = A.setup(dev(U), 0.1, A.make_params(aggs))
    rng = np.random.Generator(np.random.PCG64(34))
    for l in (1, 2):
        L = levels[l]
        shape = (R, 2, L.Nt, L.Nx)
        r = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        e0 = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        for dt in (torch.complex128, torch.complex64):
            e = dev(e0, dt)
            A.smooth(hier, l, dev(r, dt), e, 2)
            g = host(e)
            for q in range(R):
                e1 = dev(e0[q:q + 1], dt)
                A.smooth(hier, l, dev(r[q:q + 1], dt), e1, 2)
                assert np.array_equal(host(e1)[0], g[q]), (l, q, dt)
                if dt == torch.complex128:
                    want = W.to_flat(e0[q])
                    for _ in range(2):
                        want = amg.gs_sweep(L.A, L.dinv, L.colour, want, W.to_flat(r[q]))
                    assert relerr(g[q], lattice_vec(want, L.Nt, L.Nx)) <= 1e-12
    hier.destroy()


def test_apply_D_fp32_input_fp64_output_equals_fp64_on_widened_input():
    """AMAMG_F32_F64 (the product w = D z of the mixed solve) widens its
    complex64 input exactly, so it equals the FP64 stencil of the widened input
    bit for bit, here with zeros, subnormals and entries from 1e-30 to 1e30
    among Gaussian ones."""
    Nt, Nx, R = 16, 32, 3
    U = random_links(Nt, Nx, 61)
    hier = A.setup(dev(U), 0.07, A.make_params([4]))
    rng = np.random.Generator(np.random.PCG64(62))
    z = (rng.standard_normal((R, 2, Nt, Nx)) + 1j * rng.standard_normal((R, 2, Nt, Nx))).astype(np.complex64)
    flat = z.reshape(-1)
    flat[:40] = 0
    flat[40:80] = np.float32(1e-41) * (1 + 1j)                       # subnormal in FP32
    flat[80:120] *= np.float32(1e30)
    flat[120:160] *= np.float32(1e-30)
    flat[160:170] = -0.0 + 0j
    zd = torch.from_numpy(z).to(DEV)
    out_mixed = canary(R, 2, Nt, Nx, torch.complex128)
    A.apply_D(hier, zd, out_mixed)
    out64 = canary(R, 2, Nt, Nx, torch.complex128)
    A.apply_D(hier, zd.to(torch.complex128), out64)
    assert np.array_equal(host(out_mixed), host(out64))
    for r in range(R):
        ref = W.apply_dirac(U, 0.07, z[r].astype(np.complex128))
        assert relerr(host(out_mixed)[r], ref) <= 1e-13
    hier.destroy()
