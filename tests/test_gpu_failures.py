"""Failure paths of the C ABI, all made on the host or by the inputs (nothing
here faults, traps or hangs the GPU): injected allocation failures report
AMAMG_ERR_OOM and free what was allocated; a singular local operator reports
AMAMG_ERR_SINGULAR; an iteration budget too small reports AMAMG_NOT_CONVERGED
with the best iterate in x; a cancelled serving request frees its slots."""
import os
import time

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


def links(L, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return torch.from_numpy(np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, L, L)))).to(DEV)


def test_injected_allocation_failures_report_oom_and_release_memory(monkeypatch):
    L = 64
    U = links(L, 51)
    psi = torch.from_numpy(fx.gaussian_rhs(2, L, L, 52)).to(DEV)
    x = torch.empty_like(psi)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen = {"setup": 0, "solve": 0, "ok": 0}
    for n in list(range(0, 40, 3)) + [60, 100, 1000]:
        monkeypatch.setenv("AMAMG_FAIL_ALLOC_AFTER", str(n))
        try:
            hier = A.setup(U, 0.1, A.make_params([4, 2]))
        except A.AmamgError as e:
            assert e.status == A.ERR_OOM
            seen["setup"] += 1
            continue
        try:
            info = A.solve(hier, psi, x)
            assert all(i.status == A.OK for i in info)
            seen["ok"] += 1
        except A.AmamgError as e:
            assert e.status == A.ERR_OOM
            assert "AMAMG_FAIL_ALLOC_AFTER" in A.lib().amamg_last_error(hier.h).decode()
            seen["solve"] += 1
        hier.destroy()
    assert seen["setup"] > 0 and seen["solve"] > 0 and seen["ok"] > 0, seen
    monkeypatch.delenv("AMAMG_FAIL_ALLOC_AFTER")
    hier = A.setup(U, 0.1, A.make_params([4, 2]))
    info = A.solve(hier, psi, x)
    assert all(i.status == A.OK and i.true_relres <= 1e-10 for i in info)
    hier.destroy()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (64 << 20)          # failed setups and solves left nothing behind


def test_singular_local_operator_reports_singular():
    """Zero links and m0 = -2 make D = 0: every local basket solve meets a
    vanishing pivot, which setup reports (the kernel keeps its arithmetic
    finite and only raises the status flag)."""
    L = 16
    U = torch.zeros(2, L, L, dtype=torch.complex128, device=DEV)
    with pytest.raises(A.AmamgError) as ei:
        A.setup(U, -2.0, A.make_params([2]))
    assert ei.value.status == A.ERR_SINGULAR


def test_iteration_budget_reports_not_converged_with_best_iterate():
    import json
    L = 32
    U = fx.links_from_angles(fx.metropolis_u1(L, L, 3.0, 500, 0))
    here = os.path.dirname(os.path.abspath(__file__))
    m0 = json.load(open(os.path.join(here, "golden", "mcrit.json")))["L32_b3_s0"]["m_crit"] + 0.05
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params([4, 2], max_iter=4))
    psi = fx.gaussian_rhs(1, L, L, 1)
    x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    info = A.solve(hier, torch.from_numpy(psi).to(DEV), x)       # positive status: no exception
    assert info[0].status == A.NOT_CONVERGED and info[0].iterations == 4
    D = W.dirac_matrix(U, m0)
    b = W.to_flat(psi[0])
    res = np.linalg.norm(b - D @ W.to_flat(x.cpu().numpy()[0])) / np.linalg.norm(b)
    assert np.isfinite(res) and res < 1.0                         # the iterate after 4 steps, not x0 = 0
    assert abs(res - info[0].true_relres) <= 1e-6 * res
    hier.destroy()


def test_cancelled_request_frees_its_slots_and_others_finish():
    L = 64
    U = fx.links_from_angles(fx.metropolis_u1(L, L, 4.0, 200, 21))
    fields = {(L, 0): (torch.from_numpy(U).to(DEV), -0.05)}
    srv = serving.Server(fields, mem_budget_bytes=8 << 30, max_slots=4)
    g = srv.groups[(L, 0)]
    big = serving.Request(0, L, 0, m0=-0.09, R=6, arrival=0.0, rhs_seed=900)     # far below the setup mass: slow
    small = serving.Request(1, L, 0, m0=0.05, R=2, arrival=0.0, rhs_seed=950)
    srv.start()
    srv.submit(big)
    t0 = time.time()
    while g.cycles < 2 and time.time() - t0 < 60:
        time.sleep(0.002)
    assert g.cycles >= 2 and big.finish is None                  # in flight, holding slots
    srv.cancel(big)
    srv.submit(small)
    t0 = time.time()
    while (big.finish is None or small.finish is None) and time.time() - t0 < 120:
        time.sleep(0.005)
    srv.close()
    assert big.status == serving.CANCELLED
    assert small.status == A.OK and small.done_units == 2 and max(small.relres) <= 1e-10
    assert sorted(g.free) == list(range(g.slots)) and not g.where and not g.queue
