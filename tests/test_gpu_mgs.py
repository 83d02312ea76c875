"""Modified Gram-Schmidt in the outer FGMRES (amamg_params.gs_method = MGS, the
oracle's own variant): the solve reaches the tolerance with the oracle's
iteration counts (within 10 %) and the solutions agree with a dense solve and
with the oracle's; several right-hand sides in one call give each one's own
result; MGS with double-float arithmetic is rejected."""
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


def setup(U, m0, aggs, precision=A.SOLVE_FP64, restart=30, **kw):
    return A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params(aggs, precision=precision, restart=restart,
                                                                  gs_method="mgs", **kw))


@pytest.mark.parametrize("precision", [A.SOLVE_FP64, A.SOLVE_MIXED])
def test_mgs_solve_matches_oracle_and_dense_solve_32(precision):
    Nt = Nx = 32
    U = fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 500, 0))
    m0 = MCRIT["L32_b3_s0"]["m_crit"] + 0.05
    psi = fx.gaussian_rhs(1, Nt, Nx, 1)
    hier = setup(U, m0, [4], precision)
    x = torch.full(psi.shape, complex(float("nan"), float("nan")), dtype=torch.complex128, device=DEV)
    info = A.solve(hier, torch.from_numpy(psi).to(DEV), x)[0]
    assert info.status == A.OK and info.true_relres <= 1e-10
    D = W.dirac_matrix(U, m0)
    b = W.to_flat(psi[0])
    xs = W.to_flat(x.cpu().numpy()[0])
    x_dense = np.linalg.solve(D.toarray(), b)
    assert np.linalg.norm(xs - x_dense) <= 1e-8 * np.linalg.norm(x_dense)
    levels = amg.build_hierarchy(D, Nt, Nx, [4])
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 3000)
    assert abs(info.iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info.iterations, ref.iterations)
    hier.destroy()


def test_mgs_multi_rhs_each_equals_single():
    Nt = Nx = 32
    U = fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 500, 0))
    m0 = MCRIT["L32_b3_s0"]["m_crit"] + 0.05
    psi = fx.gaussian_rhs(3, Nt, Nx, 11)
    hier = setup(U, m0, [4, 2])
    xb = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    ib = A.solve(hier, torch.from_numpy(psi).to(DEV), xb)
    for r in range(3):
        x1 = torch.empty((1,) + psi.shape[1:], dtype=torch.complex128, device=DEV)
        i1 = A.solve(hier, torch.from_numpy(psi[r:r + 1]).to(DEV), x1)[0]
        assert i1.iterations == ib[r].iterations
        assert np.array_equal(x1.cpu().numpy()[0], xb.cpu().numpy()[r])
    hier.destroy()


def test_mgs_benchmark_field_256_against_oracle():
    """The 256^2 benchmark field at m_crit + 0.1 (tiles 4, 2): FP64 and mixed
    MGS solves against the oracle's (MGS) FGMRES."""
    U = fx.links_from_angles(fx.metropolis_u1(256, 256, 6.0, 500, 2))
    m0 = MCRIT["L256_b6_s2"]["m_crit"] + 0.1
    psi = fx.gaussian_rhs(1, 256, 256, 1000)
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, 256, 256, [4, 2])
    b = W.to_flat(psi[0])
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 3000)
    assert ref.converged
    for precision in (A.SOLVE_FP64, A.SOLVE_MIXED):
        hier = setup(U, m0, [4, 2], precision)
        x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
        info = A.solve(hier, torch.from_numpy(psi).to(DEV), x)[0]
        assert info.status == A.OK and info.true_relres <= 1e-10
        assert abs(info.iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info.iterations,
                                                                                        ref.iterations)
        err = np.linalg.norm(W.to_flat(x.cpu().numpy()[0]) - ref.x)
        assert err <= 2e-9 * np.linalg.norm(b) / 0.1
        print(f"MGS precision {precision}: {info.iterations} iterations (oracle {ref.iterations}), "
              f"||x - x_oracle|| / ||x_oracle|| = {err / np.linalg.norm(ref.x):.2e}")
        hier.destroy()


def test_mgs_with_double_float_arithmetic_is_rejected():
    U = fx.links_from_angles(fx.metropolis_u1(16, 16, 3.0, 50, 0))
    with pytest.raises(A.AmamgError):
        setup(U, 0.1, [2], A.SOLVE_MIXED, gs="df64")
