"""The coarsest apply of the mixed-precision V-cycle on the tensor cores
(tcgen05.mma, TF32 inputs, FP32 accumulation in tensor memory), used for eight
or more right-hand sides: against the FP64 inverse and the FP32 CUDA-core path
(norm-wise, within the TF32 rounding of the inputs), column-wise independent
of the batch it runs in, and inside whole mixed-precision batched solves."""
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
# TF32 keeps 10 explicit mantissa bits (relative rounding 2^-11 per input):
# the norm-wise error of a product with FP32 accumulation stays far below this
TF32_TOL = 4e-3


def hierarchy(L, aggs, seed, tc=True, monkeypatch=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    U = torch.from_numpy(np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, L, L)))).to(DEV)
    if monkeypatch is not None:
        monkeypatch.setenv("AMAMG_COARSEST_TC", "1" if tc else "0")
    return A.setup(U, 0.1, A.make_params(aggs, precision=A.SOLVE_MIXED))


def nrm_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L,aggs,R", [(128, [4, 2], 8), (256, [4, 2], 16), (256, [4, 2], 40), (256, [4, 4], 64)])
def test_tensor_core_coarsest_apply(monkeypatch, L, aggs, R):
    h_tc = hierarchy(L, aggs, 95, True, monkeypatch)
    h_ref = hierarchy(L, aggs, 95, False, monkeypatch)
    nt, nx, _ = h_tc.level_info(len(aggs))
    assert (2 * nt * nx) % 128 == 0
    rng = np.random.Generator(np.random.PCG64(96))
    r = rng.standard_normal((R, 2, nt, nx)) + 1j * rng.standard_normal((R, 2, nt, nx))
    r64 = torch.from_numpy(r).to(DEV)
    r32 = r64.to(torch.complex64)
    e64 = torch.empty_like(r64)
    e_tc = torch.empty_like(r32)
    e_cc = torch.empty_like(r32)
    A.coarsest_apply(h_tc, r64, e64)            # FP64 inverse
    A.coarsest_apply(h_tc, r32, e_tc)           # tensor cores
    A.coarsest_apply(h_ref, r32, e_cc)          # FP32 CUDA cores
    assert A.sync_status(h_tc) == A.OK
    y64, ytc, ycc = e64.cpu().numpy(), e_tc.cpu().numpy(), e_cc.cpu().numpy()
    assert np.all(np.isfinite(ytc))
    for k in range(R):
        assert nrm_err(ycc[k], y64[k]) <= 1e-5
        assert nrm_err(ytc[k], y64[k]) <= TF32_TOL, k
    # each output column depends only on its own right-hand side: the first
    # eight of the batch equal the same eight run alone, bit for bit
    e8 = torch.empty_like(r32[:8])
    A.coarsest_apply(h_tc, r32[:8].contiguous(), e8)
    assert np.array_equal(e8.cpu().numpy(), ytc[:8])
    h_tc.destroy()
    h_ref.destroy()


def test_mixed_batched_solve_with_tensor_core_coarsest():
    """16 right-hand sides on the 256^2 benchmark field at m_crit + 0.1, mixed
    precision (the coarsest apply on the tensor cores): all reach 1e-10 with the
    FP64 form's iteration count within 10 %."""
    import json
    import os
    L = 256
    Uh = fx.links_from_angles(fx.metropolis_u1(L, L, 6.0, 500, 2))
    here = os.path.dirname(os.path.abspath(__file__))
    m0 = json.load(open(os.path.join(here, "golden", "mcrit.json")))["L256_b6_s2"]["m_crit"] + 0.1
    U = torch.from_numpy(Uh).to(DEV)
    psi = fx.gaussian_rhs(16, L, L, 97)
    x = torch.empty(psi.shape, dtype=torch.complex128, device=DEV)
    h32 = A.setup(U, m0, A.make_params([4, 2], precision=A.SOLVE_MIXED))
    info = A.solve(h32, torch.from_numpy(psi).to(DEV), x)
    h64 = A.setup(U, m0, A.make_params([4, 2]))
    x64 = torch.empty_like(x[:1])
    i64 = A.solve(h64, torch.from_numpy(psi[:1]).to(DEV), x64)[0]
    D = W.dirac_matrix(Uh, m0)
    xs = x.cpu().numpy()
    for k in range(16):
        b = W.to_flat(psi[k])
        assert info[k].status == A.OK
        assert np.linalg.norm(b - D @ W.to_flat(xs[k])) / np.linalg.norm(b) <= 1e-10
    assert abs(info[0].iterations - i64.iterations) <= max(1, 0.1 * i64.iterations)
