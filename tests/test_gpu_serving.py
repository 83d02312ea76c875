"""Serving loop: a small Poisson request stream over resident hierarchies of
several fields and lattice sizes; every request converges, and a right-hand
side gives the same result alone and inside the mixed-precision batch mix."""
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
from paper_2608_03515_b300 import serving  # noqa: E402

DEV = torch.device("cuda:0")


def test_aggregate_rule():
    assert serving.aggregates_for(64) == [2]
    assert serving.aggregates_for(128) == [4]
    assert serving.aggregates_for(256) == [4, 2]
    assert serving.aggregates_for(512) == [4, 4]
    assert serving.aggregates_for(1024) == [4, 4, 2]


def test_mixed_precision_slot_alone_equals_in_mix():
    L = 64
    U = fx.links_from_angles(fx.metropolis_u1(L, L, 4.0, 200, 11))
    m_setup = 0.0
    hier = A.setup(torch.from_numpy(U).to(DEV), m_setup, A.make_params([2], precision=A.SOLVE_MIXED))
    psi = fx.gaussian_rhs_device(L, L, 123, DEV)

    def run(extra):
        b = A.Batch(hier, 4)
        b.admit(0, psi, m_setup + 0.02)
        for i, m in enumerate(extra):
            b.admit(1 + i, fx.gaussian_rhs_device(L, L, 500 + i, DEV), m)
        for _ in range(200):
            info = b.cycle()
            if all(info[s][1] for s in range(1 + len(extra))):
                break
        x = torch.empty(2, L, L, dtype=torch.complex128, device=DEV)
        b.retire(0, x)
        b.destroy()
        return info[0], x.cpu().numpy()

    (a0, d0, s0, it0, rr0), x0 = run([])
    (a1, d1, s1, it1, rr1), x1 = run([m_setup + 0.05, m_setup + 0.08])
    assert s0 == A.OK and rr0 <= 1e-10
    assert it0 == it1
    assert np.max(np.abs(x0 - x1)) <= 1e-12 * np.max(np.abs(x0))
    D = W.dirac_matrix(U, m_setup + 0.02)
    b = W.to_flat(psi.cpu().numpy())
    assert np.linalg.norm(b - D @ W.to_flat(x0)) / np.linalg.norm(b) <= 1e-10


def test_server_stream_converges_and_reports_latency():
    fields = {}
    mcrit = {}
    for L in (32, 64):
        for k in range(2):
            U = fx.links_from_angles(fx.metropolis_u1(L, L, 4.0 + 2 * k, 200, 20 + k))
            mcrit[(L, k)] = -0.05          # a safe lower bound for these fields: masses sit well above it
            fields[(L, k)] = (torch.from_numpy(U).to(DEV), mcrit[(L, k)] + 0.05)
    srv = serving.Server(fields, mem_budget_bytes=8 << 30, max_slots=4)
    reqs = serving.poisson_requests(12, rate=200.0, pairs=list(fields), mcrit=mcrit, seed=7, max_rhs=3,
                                    dm=(0.05, 0.1))
    out = serving.serve(srv, reqs)
    assert out["requests"] == 12 and out["not_converged"] == 0
    assert out["max_true_relres"] <= 1e-10
    assert out["latency_p99_ms"] >= out["latency_p50_ms"] > 0
    assert all(r.done_units == r.R for r in reqs)
    # a second stream on the same resident hierarchies (the server restarts its workers)
    reqs2 = serving.poisson_requests(6, rate=200.0, pairs=list(fields), mcrit=mcrit, seed=8, max_rhs=2,
                                     dm=(0.05, 0.1))
    out2 = serving.serve(srv, reqs2)
    assert out2["requests"] == 6 and out2["not_converged"] == 0 and out2["max_true_relres"] <= 1e-10
    assert all(r.done_units == r.R for r in reqs2)
