"""The two alternative readings of the interpolator on the GPU (amamg_params
edge_owner and normalization) against the oracle's build_hierarchy with the
same readings: structure bit-exact, interpolator and coarse blocks to 1e-12,
transfers to 1e-13, whole solves to 1e-10 with iteration counts within 10 %.

Sec. 4.1: a border site takes its formula from "the first aggregate it was
assigned to" (tile rule or lexicographic first basket); Eq. (16): the
normalisation N (identity, or division by the complex row sum)."""
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
READINGS = [("first_lex", "none"), ("tile", "rowsum"), ("first_lex", "rowsum")]


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(got, want):
    return np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)


def oracle_P_tiles(P, Nt, Nx, a, rule):
    """The oracle's interpolator in the library's per-tile layout: rows of the
    tile's in-tile sites, columns 2c + beta = corner c of the basket whose
    formula the row takes (the oracle's owner_basket)."""
    Np, Nq = Nt // a, Nx // a
    nrows = 2 * (a * a - 1)
    Pd = P.tocsr()
    out = np.zeros((Np * Nq, 8, nrows), dtype=complex)
    for p in range(Np):
        for q in range(Nq):
            for lr in range(nrows):
                l, alpha = lr // 2 + 1, lr % 2
                t, x = p * a + l // a, q * a + l % a
                pb, qb = divmod(amg.owner_basket(t, x, Nt, Nx, a, rule), Nq)
                row = 2 * (t * Nx + x) + alpha
                for c in range(4):
                    v = amg.corner_vertex(Nt, Nx, a, pb, qb, c)
                    for beta in range(2):
                        out[p * Nq + q, 2 * c + beta, lr] = Pd[row, 2 * v + beta]
    return out


def links(Nt, Nx, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))


@pytest.mark.parametrize("ownership,normalization", READINGS)
@pytest.mark.parametrize("Nt,Nx,aggs", [(8, 8, [2]), (16, 16, [4]), (32, 32, [4, 2]), (16, 24, [2, 2]),
                                        (64, 64, [4, 2])])
def test_setup_matches_oracle(Nt, Nx, aggs, ownership, normalization):
    U = links(Nt, Nx, 41)
    m0 = 0.07
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, Nt, Nx, aggs, ownership=ownership, normalization=normalization)
    hier = A.setup(dev(U), m0, A.make_params(aggs, ownership=ownership, normalization=normalization))
    rng = np.random.Generator(np.random.PCG64(42))
    for l, a in enumerate(aggs):
        L, C = levels[l], levels[l + 1]
        role, owner, offs = A.export_structure(hier, l)
        assert np.array_equal(role, amg.site_roles(L.Nt, L.Nx, a))
        assert np.array_equal(owner, amg.owner_tiles(L.Nt, L.Nx, a, ownership))
        assert offs == [tuple(o) for o in C.offsets]
        want = oracle_P_tiles(L.P, L.Nt, L.Nx, a, ownership)
        got = torch.empty(want.shape, dtype=torch.complex128, device=DEV)
        A.export_P(hier, l, got)
        assert relerr(host(got), want) <= 1e-12
        Bw = amg.block_stencil(C.A, C.offsets, C.Nt, C.Nx)
        Bw = np.transpose(Bw.reshape(len(C.offsets), C.Nt * C.Nx, 4), (0, 2, 1))
        Bg = torch.empty(Bw.shape, dtype=torch.complex128, device=DEV)
        A.export_coarse(hier, l + 1, Bg)
        assert relerr(host(Bg), Bw) <= 1e-12
        # transfers with the stored rows, two right-hand sides
        ec = rng.standard_normal((2, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((2, 2, C.Nt, C.Nx))
        ef = rng.standard_normal((2, 2, L.Nt, L.Nx)) + 1j * rng.standard_normal((2, 2, L.Nt, L.Nx))
        out_f = torch.empty(2, 2, L.Nt, L.Nx, dtype=torch.complex128, device=DEV)
        out_c = torch.empty(2, 2, C.Nt, C.Nx, dtype=torch.complex128, device=DEV)
        A.apply_P(hier, l, dev(ec), out_f)
        A.apply_PH(hier, l, dev(ef), out_c)
        gf, gc = host(out_f), host(out_c)
        # row sums near the floor make some normalised weights large: their
        # rounding sets the relative error of the transfers
        tol = 1e-13 if normalization == "none" else 1e-12
        for r in range(2):
            assert relerr(gf[r], W.from_flat(L.P @ W.to_flat(ec[r]), L.Nt, L.Nx)) <= tol
            assert relerr(gc[r], W.from_flat(L.P.conj().T @ W.to_flat(ef[r]), C.Nt, C.Nx)) <= tol
    hier.destroy()


@pytest.mark.parametrize("ownership,normalization", READINGS)
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_matches_oracle(ownership, normalization, precision):
    """FP64 and mixed-precision solves on the 32^2 beta = 3 field (m_crit + 0.05)
    reach 1e-10 with the oracle's outer iteration count within 10 %."""
    import json
    import os
    Nt = Nx = 32
    aggs = [4, 2]
    U = fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 500, 0))
    here = os.path.dirname(os.path.abspath(__file__))
    m0 = json.load(open(os.path.join(here, "golden", "mcrit.json")))["L32_b3_s0"]["m_crit"] + 0.05
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, Nt, Nx, aggs, ownership=ownership, normalization=normalization)
    hier = A.setup(dev(U), m0, A.make_params(aggs, precision=precision, ownership=ownership,
                                             normalization=normalization))
    psi = fx.gaussian_rhs(1, Nt, Nx, 1)
    x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    info = A.solve(hier, dev(psi), x)
    b = W.to_flat(psi[0])
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 5000)
    res = np.linalg.norm(b - D @ W.to_flat(host(x)[0])) / np.linalg.norm(b)
    assert info[0].status == A.OK and res <= 1e-10
    assert abs(info[0].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info[0].iterations,
                                                                                       ref.iterations)
    hier.destroy()


def test_first_lex_smoothed_level_beyond_the_smoother_is_rejected():
    """Under first-lex ownership the second coarse level of a 32^2 lattice with
    tile sides 2, 2, 2 couples 37 block offsets (the union over its sites); it
    is a smoothed level, so setup rejects it with a clear error instead of
    building a smoother it cannot run."""
    U = links(32, 32, 43)
    with pytest.raises(A.AmamgError) as ei:
        A.setup(dev(U), 0.1, A.make_params([2, 2, 2], ownership="first_lex"))
    assert ei.value.status == A.ERR_INVALID_ARG
