"""The paper's coarsest-level solver on the GPU (amamg_params.coarsest =
AMAMG_COARSEST_GMRES: unpreconditioned GMRES(30) from a zero start to relative
residual 0.1, Sec. 5) against the oracle's coarsest_gmres, and whole solves
with it against the oracle's FGMRES with vcycle(coarsest="gmres")."""
import json
import os

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
MCRIT = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mcrit.json")))


def links(L, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, L, L)))


@pytest.mark.parametrize("L,aggs,R", [(32, [4, 2], 3), (64, [4, 2], 2), (128, [4, 2], 1), (64, [2, 2], 40)])
def test_coarsest_gmres_matches_oracle(L, aggs, R):
    """Both run the same GMRES(30) to 0.1 in FP64, so they stop after the same
    step with the same Krylov space: e agrees to rounding; and the residual of
    the returned e is at most 0.1 of the right-hand side's norm.  R = 40 takes
    two launches (32 right-hand sides per launch)."""
    U = links(L, 91)
    m0 = 0.05
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, L, L, aggs, smooth=False)
    C = levels[-1]
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params(aggs, coarsest="gmres"))
    assert hier.level_info(len(aggs))[:2] == (C.Nt, C.Nx)
    rng = np.random.Generator(np.random.PCG64(92))
    r = rng.standard_normal((R, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((R, 2, C.Nt, C.Nx))
    e = torch.empty(R, 2, C.Nt, C.Nx, dtype=torch.complex128, device=DEV)
    A.coarsest_solve(hier, torch.from_numpy(r).to(DEV), e)
    assert A.sync_status(hier) == A.OK
    got = e.cpu().numpy()
    for k in range(R):
        rf = W.to_flat(r[k])
        want = amg.coarsest_gmres(C, rf)
        gf = W.to_flat(got[k])
        assert np.linalg.norm(rf - C.A @ gf) <= 0.1 * np.linalg.norm(rf)
        assert np.linalg.norm(gf - want) <= 1e-9 * np.linalg.norm(want), k
    hier.destroy()


@pytest.mark.parametrize("precision", [A.SOLVE_FP64, A.SOLVE_MIXED])
def test_solve_with_coarsest_gmres_matches_oracle(precision):
    """32^2 beta = 3 field at m_crit + 0.05, tiles 4 then 2: iterations within
    10 % of the oracle's FGMRES with the same coarsest solver, residual 1e-10."""
    L = 32
    U = fx.links_from_angles(fx.metropolis_u1(L, L, 3.0, 500, 0))
    m0 = MCRIT["L32_b3_s0"]["m_crit"] + 0.05
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, L, L, [4, 2])
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params([4, 2], precision=precision, coarsest="gmres"))
    psi = fx.gaussian_rhs(1, L, L, 1)
    x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    info = A.solve(hier, torch.from_numpy(psi).to(DEV), x)
    b = W.to_flat(psi[0])
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r, coarsest="gmres"), b, 30, 1e-10, 5000)
    res = np.linalg.norm(b - D @ W.to_flat(x.cpu().numpy()[0])) / np.linalg.norm(b)
    assert info[0].status == A.OK and res <= 1e-10
    assert abs(info[0].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info[0].iterations,
                                                                                      ref.iterations)
    hier.destroy()


def test_benchmark_field_256_with_coarsest_gmres():
    """The 256^2 beta = 6 benchmark field at m_crit + 0.1 (coarsest 32^2, 2048
    unknowns) with the paper's coarsest setting: FP64 iterations within 10 % of
    the oracle's."""
    L = 256
    U = fx.links_from_angles(fx.metropolis_u1(L, L, 6.0, 500, 2))
    m0 = MCRIT["L256_b6_s2"]["m_crit"] + 0.1
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, L, L, [4, 2])
    psi = fx.gaussian_rhs(1, L, L, 1000)
    b = W.to_flat(psi[0])
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r, coarsest="gmres"), b, 30, 1e-10, 3000)
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params([4, 2], coarsest="gmres"))
    x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    info = A.solve(hier, torch.from_numpy(psi).to(DEV), x)
    res = np.linalg.norm(b - D @ W.to_flat(x.cpu().numpy()[0])) / np.linalg.norm(b)
    assert info[0].status == A.OK and res <= 1e-10
    assert abs(info[0].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info[0].iterations,
                                                                                      ref.iterations)
    print(f"256^2 m_crit+0.1, coarsest GMRES: {info[0].iterations} iterations (oracle {ref.iterations})")
    hier.destroy()
