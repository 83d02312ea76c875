"""amamg_vcycle_noalloc: the V-cycle for callers that cannot allocate device
memory (no cudaMalloc while they run), checked through the C ABI against
amamg_vcycle on two calls in a row.  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2608_03515_b300 import build  # noqa: E402

build.build()
from paper_2608_03515_b300 import amamg as A  # noqa: E402
from paper_2608_03515_b300 import fixtures as fx  # noqa: E402

DEV = torch.device("cuda:0")


def relerr(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-13), (torch.complex64, 2e-6)])
def test_noalloc_vcycle_matches_vcycle_twice(dtype, tol):
    Nt = Nx = 64
    U = torch.from_numpy(fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 50, 3))).to(DEV)
    prec = A.SOLVE_MIXED if dtype == torch.complex64 else A.SOLVE_FP64
    hier = A.setup(U, 0.0, A.make_params([4, 2], precision=prec))
    for call in range(2):                      # the scratch keeps the previous call's contents
        r = torch.from_numpy(fx.gaussian_rhs(2, Nt, Nx, 60 + call)).to(DEV).to(dtype)
        e_ref = torch.empty_like(r)
        e_new = torch.full_like(r, float("nan"))
        A.vcycle(hier, r, e_ref)
        A.vcycle_noalloc(hier, r, e_new)
        torch.cuda.synchronize()
        got, want = e_new.cpu().numpy(), e_ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert relerr(got, want) <= tol


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-13), (torch.complex64, 2e-6)])
def test_noalloc_vcycle_matches_vcycle_larger_coarse_levels(dtype, tol):
    """256^2 with tile sides 4, 2: coarse levels 64^2 and 32^2, two right-hand
    sides (about 655 KB of scratch in FP64), so the coarse smoothing takes the
    kernels of the larger levels."""
    Nt = Nx = 256
    rng = np.random.Generator(np.random.PCG64(62))
    U = torch.from_numpy(np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))).to(DEV)
    prec = A.SOLVE_MIXED if dtype == torch.complex64 else A.SOLVE_FP64
    hier = A.setup(U, 0.1, A.make_params([4, 2], precision=prec))
    for call in range(2):
        r = torch.from_numpy(fx.gaussian_rhs(2, Nt, Nx, 70 + call)).to(DEV).to(dtype)
        e_ref = torch.empty_like(r)
        e_new = torch.full_like(r, float("nan"))
        A.vcycle(hier, r, e_ref)
        A.vcycle_noalloc(hier, r, e_new)
        torch.cuda.synchronize()
        got, want = e_new.cpu().numpy(), e_ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert relerr(got, want) <= tol
    assert A.sync_status(hier) == A.OK


def test_noalloc_time_out_is_reported_by_the_status_query():
    """The allocation-free V-cycle does not report a coarse smoother's bounded
    wait that ran out; the status query does (synchronising, allocating
    nothing), re-arms the counters, and the next calls agree again."""
    Nt = Nx = 64
    U = torch.from_numpy(fx.links_from_angles(fx.metropolis_u1(Nt, Nx, 3.0, 50, 4))).to(DEV)
    hier = A.setup(U, 0.1, A.make_params([2, 2, 2]))
    r = torch.from_numpy(fx.gaussian_rhs(1, Nt, Nx, 80)).to(DEV)
    e_ref = torch.empty_like(r)
    e_new = torch.empty_like(r)
    assert A.selftest_sync_timeout(hier, 1, A.F64) == A.OK      # one owner block withholds its counter
    A.vcycle_noalloc(hier, r, e_new)                              # returns without reporting
    assert A.sync_status(hier) == A.ERR_TIMEOUT
    assert A.sync_status(hier) == A.OK
    A.vcycle(hier, r, e_ref)
    A.vcycle_noalloc(hier, r, e_new)
    assert A.sync_status(hier) == A.OK
    assert relerr(e_new.cpu().numpy(), e_ref.cpu().numpy()) <= 1e-13


def test_noalloc_rejects_requests_beyond_the_fixed_array():
    Nt = Nx = 256
    rng = np.random.Generator(np.random.PCG64(61))
    U = torch.from_numpy(np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))).to(DEV)
    hier = A.setup(U, 0.1, A.make_params([4, 2]))
    # coarse levels 64^2 and 32^2: 2 * R * 2 * 5120 complex128 = 327680 R bytes; R = 32 > 8 MiB
    R = 32
    r = torch.zeros(R, 2, Nt, Nx, dtype=torch.complex128, device=DEV)
    e = torch.zeros_like(r)
    with pytest.raises(A.AmamgError) as ei:
        A.vcycle_noalloc(hier, r, e)
    assert ei.value.status == A.ERR_INVALID_ARG
    assert "bytes of scratch" in A.lib().amamg_last_error(hier.h).decode()
