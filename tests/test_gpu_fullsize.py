"""Full-size workloads (the benchmark lattice and the mixed-precision 512^2 case):
properties that hold at any size, checked with the oracle's FP64 operator --
true relative residual of every solution, iteration counts of the mixed form
against the FP64 form, and the oracle's own iteration count where it is cheap."""
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


def true_relres(U, m0, psi, x):
    r = psi - W.apply_dirac(U, m0, x)
    return np.linalg.norm(r) / np.linalg.norm(psi)


def solve(U, m0, aggs, precision, restart, psi):
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params(aggs, precision=precision, restart=restart))
    x = torch.empty((1,) + psi.shape, dtype=torch.complex128, device=DEV)
    info = A.solve(hier, torch.from_numpy(psi[None]).to(DEV), x)[0]
    return info, x.cpu().numpy()[0]


@pytest.fixture(scope="module")
def field256():
    return fx.links_from_angles(fx.metropolis_u1(256, 256, 6.0, 500, 2))


@pytest.mark.parametrize("dm", [0.1, 0.02, 0.005])
def test_benchmark_workload_256(field256, dm):
    """256^2, beta = 6, m0 = m_crit + dm, tiles 4 then 2, FGMRES(30): FP64 and
    mixed against the oracle's FP64 solve of the same system: iteration counts
    within 10 %, solutions within the conditioning bound of two 1e-10 solves,
    ||x - x_oracle|| <= 2e-10 ||psi|| ||D^-1|| with ||D^-1|| taken as 10 / dm
    (1 / dm bounds the inverse eigenvalues; the factor 10 allows for D not
    being normal)."""
    U = field256
    m0 = MCRIT["L256_b6_s2"]["m_crit"] + dm
    psi = fx.gaussian_rhs(1, 256, 256, 1000)[0]
    i64, x64 = solve(U, m0, [4, 2], A.SOLVE_FP64, 30, psi)
    i32, x32 = solve(U, m0, [4, 2], A.SOLVE_MIXED, 30, psi)
    assert i64.status == A.OK and i32.status == A.OK
    assert true_relres(U, m0, psi, x64) <= 1e-10
    assert true_relres(U, m0, psi, x32) <= 1e-10
    assert abs(i32.iterations - i64.iterations) <= max(1, 0.1 * i64.iterations)
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, 256, 256, [4, 2])
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), W.to_flat(psi), 30, 1e-10, 3000)
    assert ref.converged
    assert abs(i64.iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (i64.iterations, ref.iterations)
    assert abs(i32.iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (i32.iterations, ref.iterations)
    bound = 2e-9 * np.linalg.norm(psi) / dm
    for x in (x64, x32):
        err = np.linalg.norm(W.to_flat(x) - ref.x)
        print(f"256^2 m_crit+{dm}: ||x - x_oracle|| / ||x_oracle|| = {err / np.linalg.norm(ref.x):.2e}")
        assert err <= bound


def test_mixed_precision_workload_512():
    """512^2, beta = 10, m0 = m_crit + 0.01, tiles 4 then 4, FGMRES(40), mixed vs FP64."""
    U = fx.links_from_angles(fx.metropolis_u1(512, 512, 10.0, 500, 4))
    m0 = MCRIT["L512_b10_s4"]["m_crit"] + 0.01
    psi = fx.gaussian_rhs(1, 512, 512, 4000)[0]
    i32, x32 = solve(U, m0, [4, 4], A.SOLVE_MIXED, 40, psi)
    i64, x64 = solve(U, m0, [4, 4], A.SOLVE_FP64, 40, psi)
    assert i32.status == A.OK and true_relres(U, m0, psi, x32) <= 1e-10
    assert i64.status == A.OK and true_relres(U, m0, psi, x64) <= 1e-10
    assert abs(i32.iterations - i64.iterations) <= max(1, 0.1 * i64.iterations)
    # both solve the same system to 1e-10: their difference is bounded by the
    # conditioning (m0 - m_crit = 0.01 -> ||D^-1|| <= ~100)
    assert np.linalg.norm(x32 - x64) <= 1e-7 * np.linalg.norm(x64)
    # the oracle's FP64 solve of the same system (its iteration count, and the
    # mixed result's error against it, stated per result)
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, 512, 512, [4, 4])
    ref = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), W.to_flat(psi), 40, 1e-10, 3000)
    assert ref.converged
    assert abs(i32.iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (i32.iterations, ref.iterations)
    bound = 2e-9 * np.linalg.norm(psi) / 0.01
    for name, x in (("mixed", x32), ("fp64", x64)):
        err = np.linalg.norm(W.to_flat(x) - ref.x)
        print(f"512^2 {name}: ||x - x_oracle|| / ||x_oracle|| = {err / np.linalg.norm(ref.x):.2e}, "
              f"iterations {i32.iterations if name == 'mixed' else i64.iterations} (oracle {ref.iterations})")
        assert err <= bound
