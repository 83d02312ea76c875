"""The opt-in double-float Gram-Schmidt of the mixed-precision outer solver
(amamg_params.gs_arith = AMAMG_GS_DF64): solves reach the 1e-10 true residual
with the oracle's FP64 iteration count within 10 %, and their solutions agree
with the oracle's within the conditioning bound."""
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


def test_df64_gs_requires_mixed_precision():
    U = torch.ones(2, 16, 16, dtype=torch.complex128, device=DEV)
    with pytest.raises(A.AmamgError) as ei:
        A.setup(U, 0.1, A.make_params([2], precision=A.SOLVE_FP64, gs="df64"))
    assert ei.value.status == A.ERR_INVALID_ARG


@pytest.mark.parametrize("L,beta,seed,key,aggs,dm,R", [(32, 3.0, 0, "L32_b3_s0", [4, 2], 0.05, 3),
                                                      (256, 6.0, 2, "L256_b6_s2", [4, 2], 0.02, 1)])
def test_df64_gs_solve_matches_oracle(L, beta, seed, key, aggs, dm, R):
    Uh = fx.links_from_angles(fx.metropolis_u1(L, L, beta, 500, seed))
    m0 = MCRIT[key]["m_crit"] + dm
    D = W.dirac_matrix(Uh, m0)
    levels = amg.build_hierarchy(D, L, L, aggs)
    hier = A.setup(torch.from_numpy(Uh).to(DEV), m0, A.make_params(aggs, precision=A.SOLVE_MIXED, gs="df64"))
    psi = fx.gaussian_rhs(R, L, L, 1000)
    x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    info = A.solve(hier, torch.from_numpy(psi).to(DEV), x)
    xs = x.cpu().numpy()
    for r in range(R):
        b = W.to_flat(psi[r])
        ref = krylov.fgmres(lambda v: D @ v, lambda v: amg.vcycle(levels, v), b, 30, 1e-10, 3000)
        res = np.linalg.norm(b - D @ W.to_flat(xs[r])) / np.linalg.norm(b)
        assert info[r].status == A.OK and res <= 1e-10
        assert abs(info[r].iterations - ref.iterations) <= max(1, 0.1 * ref.iterations), (info[r].iterations,
                                                                                          ref.iterations)
        err = np.linalg.norm(W.to_flat(xs[r]) - ref.x)
        assert err <= 2e-9 * np.linalg.norm(b) / dm
        print(f"{L}^2 m_crit+{dm} df64 GS: {info[r].iterations} iterations (oracle {ref.iterations}), "
              f"||x - x_oracle|| / ||x_oracle|| = {err / np.linalg.norm(ref.x):.2e}")
    hier.destroy()
