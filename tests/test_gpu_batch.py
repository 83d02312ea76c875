"""Slot batches (continuous batching): right-hand sides with their own masses
admitted while others are in flight give the same result as when solved alone,
and match the oracle's FGMRES with the same mass-shifted preconditioner."""
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
NT = NX = 32
M_SETUP = -0.1383495190759743 + 0.05          # 32^2 beta = 3 field: m_crit from the oracle + 0.05


@pytest.fixture(scope="module")
def field():
    return fx.links_from_angles(fx.metropolis_u1(NT, NX, 3.0, 500, 0))


def run_batch(hier, psis, masses, admit_at, slots=4, max_cycles=200):
    """Admit psis[i] (mass masses[i]) before cycle admit_at[i]; retire when done."""
    b = A.Batch(hier, slots)
    out = [None] * len(psis)
    info = [None] * len(psis)
    where = {}
    free = list(range(slots))
    pending = list(range(len(psis)))
    for cyc in range(max_cycles):
        for i in [p for p in pending if admit_at[p] <= cyc]:
            if not free:
                break
            s = free.pop(0)
            b.admit(s, torch.from_numpy(psis[i]).to(DEV), masses[i])
            where[s] = i
            pending.remove(i)
        if not where and not pending:
            break
        res = b.cycle()
        for s, i in list(where.items()):
            active, done, status, iters, relres = res[s]
            if done:
                x = torch.empty(2, NT, NX, dtype=torch.complex128, device=DEV)
                b.retire(s, x)
                out[i] = x.cpu().numpy()
                info[i] = (status, iters, relres)
                del where[s]
                free.append(s)
    b.destroy()
    return out, info


def test_batch_results_equal_single_solves_and_meet_tolerance(field):
    U = field
    hier = A.setup(torch.from_numpy(U).to(DEV), M_SETUP, A.make_params([4, 2]))
    psis = [fx.gaussian_rhs(1, NT, NX, 70 + i)[0] for i in range(5)]
    masses = [M_SETUP, M_SETUP + 0.03, M_SETUP + 0.1, M_SETUP, M_SETUP + 0.01]
    admit_at = [0, 0, 1, 2, 3]                     # later requests join while others run
    xs, infos = run_batch(hier, psis, masses, admit_at, slots=3)
    for i, (psi, m0) in enumerate(zip(psis, masses)):
        status, iters, relres = infos[i]
        assert status == A.OK and relres <= 1e-10
        D = W.dirac_matrix(U, m0)
        res = np.linalg.norm(W.to_flat(psi) - D @ W.to_flat(xs[i])) / np.linalg.norm(psi)
        assert res <= 1e-10
        if m0 == M_SETUP:
            # alone (amamg_solve, R = 1) and in the mix: same steps, same solution
            x1 = torch.empty(1, 2, NT, NX, dtype=torch.complex128, device=DEV)
            i1 = A.solve(hier, torch.from_numpy(psi[None]).to(DEV), x1)
            assert i1[0].iterations == iters
            got = x1.cpu().numpy()[0]
            assert np.max(np.abs(got - xs[i])) <= 1e-12 * np.max(np.abs(got))


def test_batch_mass_shift_matches_oracle_iterations(field):
    """A slot at m0 != m_setup: outer operator D(m0), fine smoother with m0, P and
    coarse levels from m_setup; the oracle builds the same preconditioner."""
    U = field
    hier = A.setup(torch.from_numpy(U).to(DEV), M_SETUP, A.make_params([4, 2]))
    m0 = M_SETUP + 0.04
    psi = fx.gaussian_rhs(1, NT, NX, 80)[0]
    xs, infos = run_batch(hier, [psi], [m0], [0], slots=2)
    levels = amg.build_hierarchy(W.dirac_matrix(U, M_SETUP), NT, NX, [4, 2])
    Dm = W.dirac_matrix(U, m0)
    levels[0].A = Dm
    levels[0].dinv = amg.diag_block_inverses(Dm, NT * NX)
    ref = krylov.fgmres(lambda v: Dm @ v, lambda r: amg.vcycle(levels, r), W.to_flat(psi), 30, 1e-10, 3000)
    status, iters, relres = infos[0]
    assert status == A.OK
    assert abs(iters - ref.iterations) <= max(1, 0.1 * ref.iterations)
    assert np.linalg.norm(W.to_flat(xs[0]) - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_batch_rejects_occupied_slot(field):
    hier = A.setup(torch.from_numpy(field).to(DEV), M_SETUP, A.make_params([4]))
    b = A.Batch(hier, 2)
    psi = torch.from_numpy(fx.gaussian_rhs(1, NT, NX, 90)[0]).to(DEV)
    b.admit(0, psi, M_SETUP)
    with pytest.raises(A.AmamgError):
        b.admit(0, psi, M_SETUP)
    b.destroy()
