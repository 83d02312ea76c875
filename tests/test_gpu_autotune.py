"""The coarse-smoother autotuner (amamg_params.autotune): before the first
solve the fixed rule stands; the first solve of each right-hand-side count
times the candidate kernels and shapes and keeps one; solves with the tuned
hierarchy reach the tolerance with the untuned hierarchy's iteration counts
(within 10 %) on the benchmark field."""
import json
import os

import numpy as np
import pytest

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
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("precision,R", [(A.SOLVE_FP64, 1), (A.SOLVE_MIXED, 1), (A.SOLVE_MIXED, 4)])
def test_autotuned_solve_matches_untuned(precision, R):
    L = 256
    Uh = fx.links_from_angles(fx.metropolis_u1(L, L, 6.0, 500, 2))
    m0 = json.load(open(os.path.join(HERE, "golden", "mcrit.json")))["L256_b6_s2"]["m_crit"] + 0.02
    U = torch.from_numpy(Uh).to(DEV)
    psi = torch.from_numpy(fx.gaussian_rhs(R, L, L, 41)).to(DEV)
    prec = A.F64 if precision == A.SOLVE_FP64 else A.F32
    h0 = A.setup(U, m0, A.make_params([4, 2], precision=precision))
    ht = A.setup(U, m0, A.make_params([4, 2], precision=precision, autotune=True))
    fixed = A.query_smoother(h0, 1, prec, R)
    assert A.query_smoother(ht, 1, prec, R) == fixed                 # nothing tuned yet
    x0 = torch.empty_like(psi)
    xt = torch.empty_like(psi)
    i0 = A.solve(h0, psi, x0)
    it = A.solve(ht, psi, xt)
    kind, variant = A.query_smoother(ht, 1, prec, R)
    assert kind in ("owner", "grid", "dsmem") and 0 <= variant <= 6
    assert A.query_smoother(h0, 1, prec, R) == fixed                 # the untuned handle keeps its rule
    D = W.dirac_matrix(Uh, m0)
    xs = xt.cpu().numpy()
    for k in range(R):
        assert it[k].status == A.OK and it[k].true_relres <= 1e-10
        b = W.to_flat(psi[k].cpu().numpy())
        assert np.linalg.norm(b - D @ W.to_flat(xs[k])) / np.linalg.norm(b) <= 1e-10
        assert abs(it[k].iterations - i0[k].iterations) <= max(1, 0.1 * i0[k].iterations)
    print(f"precision {precision} R {R}: fixed {fixed}, tuned {(kind, variant)}, "
          f"iterations {[i.iterations for i in i0]} / {[i.iterations for i in it]}")
    A.destroy(h0)
    A.destroy(ht)
