"""CG on the normal equations on the GPU (amamg_cgnr; the paper's
unpreconditioned comparison solver, Sec. 5) against the oracle's CGNR, with
D^H = sigma_3 D sigma_3 (Eq. (6)) checked against the oracle's adjoint."""
import json
import os

import numpy as np
import pytest

from oracle import krylov
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


def relerr(got, want):
    return np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)


def test_apply_Ddag_is_the_adjoint():
    Nt, Nx, R = 16, 24, 2
    rng = np.random.Generator(np.random.PCG64(81))
    U = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))
    m0 = 0.13
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params([2]))
    psi = rng.standard_normal((R, 2, Nt, Nx)) + 1j * rng.standard_normal((R, 2, Nt, Nx))
    out = torch.empty(R, 2, Nt, Nx, dtype=torch.complex128, device=DEV)
    A.apply_Ddag(hier, torch.from_numpy(psi).to(DEV), out)
    DH = W.dirac_matrix(U, m0).conj().T.tocsr()
    got = out.cpu().numpy()
    for r in range(R):
        assert relerr(got[r], W.from_flat(DH @ W.to_flat(psi[r]), Nt, Nx)) <= 1e-13
    hier.destroy()


def cgnr_case(L, beta, seed, key, dm, R=1, max_iter=200000):
    U = fx.links_from_angles(fx.metropolis_u1(L, L, beta, 500, seed))
    m0 = MCRIT[key]["m_crit"] + dm
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params([4] if L <= 64 else [4, 2]))
    psi = fx.gaussian_rhs(R, L, L, 7)
    x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    info = A.cgnr(hier, torch.from_numpy(psi).to(DEV), x, max_iter=max_iter, tol=1e-10)
    D = W.dirac_matrix(U, m0)
    hier.destroy()
    return U, D, psi, info, x.cpu().numpy()


def test_cgnr_matches_oracle_c1_field():
    """32^2, beta = 3, m0 = m_crit + 0.05: iteration count within 10 % of the
    oracle's CGNR, true residual <= 1e-10, solution within the conditioning
    bound of two 1e-10 solves; three right-hand sides each as if alone."""
    U, D, psi, info, x = cgnr_case(32, 3.0, 0, "L32_b3_s0", 0.05, R=3)
    for r in range(3):
        b = W.to_flat(psi[r])
        ref = krylov.cgnr(lambda v: D @ v, lambda v: D.conj().T @ v, b, 1e-10, 200000)
        assert ref.converged
        assert info[r].status == A.OK
        res = np.linalg.norm(b - D @ W.to_flat(x[r])) / np.linalg.norm(b)
        assert res <= 1e-10 and abs(res - info[r].true_relres) <= 1e-3 * res
        assert abs(info[r].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info[r].iterations,
                                                                                          ref.iterations)
        assert np.linalg.norm(W.to_flat(x[r]) - ref.x) <= 2e-9 * np.linalg.norm(b) / 0.05


def test_cgnr_budget_reports_not_converged():
    U, D, psi, info, x = cgnr_case(32, 3.0, 0, "L32_b3_s0", 0.05, R=1, max_iter=30)
    assert info[0].status == A.NOT_CONVERGED and info[0].iterations == 30
    b = W.to_flat(psi[0])
    res = np.linalg.norm(b - D @ W.to_flat(x[0])) / np.linalg.norm(b)
    assert res < 1.0 and abs(res - info[0].true_relres) <= 1e-6 * res


def test_cgnr_benchmark_field_256():
    """The 256^2 beta = 6 benchmark field at m_crit + 0.1 against the oracle's CGNR."""
    U, D, psi, info, x = cgnr_case(256, 6.0, 2, "L256_b6_s2", 0.1)
    b = W.to_flat(psi[0])
    ref = krylov.cgnr(lambda v: D @ v, lambda v: D.conj().T @ v, b, 1e-10, 200000)
    assert ref.converged and info[0].status == A.OK
    assert abs(info[0].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info[0].iterations,
                                                                                      ref.iterations)
    res = np.linalg.norm(b - D @ W.to_flat(x[0])) / np.linalg.norm(b)
    assert res <= 1e-10
    print(f"CGNR 256^2 m_crit+0.1: {info[0].iterations} iterations (oracle {ref.iterations})")
