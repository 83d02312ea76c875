"""Tensor-core coarse apply (FP32 vectors, 32 or more right-hand sides):
y = A_l x over 2 x 4-site super-blocks with FP16 operands and FP32 accumulation.

Against the oracle: the oracle's Galerkin operator stored as the kernel stores
it (FP16 with one scale per operator row, oracle.mixed.quantise_rows) applied in
FP64 to the right-hand sides rounded as the kernel rounds them (FP16 with one
power-of-two scale per right-hand side, oracle.mixed.quantise_rhs_pow2): equal
up to FP32 accumulation, 1e-5 of the output's largest entry.  Against the
exact FP64 product: the FP16 rounding of both operands, 2e-3.  Sizes: coarse
levels of 8 x 8 (the box wraps the whole x extent) to 32 x 16, one to two
groups of 64 right-hand sides with a ragged last group, and the benchmark's
256^2 x 64 on sampled sites (oracle rows built locally)."""
import numpy as np
import pytest

from oracle import amg, mixed
from oracle import wilson as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2608_03515_b300 import build  # noqa: E402

build.build()
from paper_2608_03515_b300 import amamg as A  # noqa: E402

DEV = torch.device("cuda:0")


def random_links(Nt, Nx, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))


def stencil_apply(B, offsets, x, Nt, Nx):
    """y[:, v] = sum_k B[k, v] x[:, v + offset_k] for one right-hand side [2][Nt][Nx]."""
    n = Nt * Nx
    t, xx = np.divmod(np.arange(n), Nx)
    xf = x.reshape(2, n)
    y = np.zeros((2, n), dtype=complex)
    for k, (dt, dx) in enumerate(offsets):
        w = ((t + dt) % Nt) * Nx + (xx + dx) % Nx
        y += np.einsum("vab,bv->av", B[k], xf[:, w])
    return y.reshape(2, Nt, Nx)


def relerr(got, want):
    return np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)


@pytest.mark.parametrize("Nt,Nx,R", [(64, 64, 64), (64, 128, 100), (128, 64, 32)])
def test_tensor_core_coarse_apply_matches_emulated_fp16_operands(Nt, Nx, R):
    U = random_links(Nt, Nx, 40 + R)
    m0 = 0.15
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params([4, 2], precision=A.SOLVE_MIXED))
    D = W.dirac_matrix(U, m0)
    levels = amg.build_hierarchy(D, Nt, Nx, [4, 2])
    rng = np.random.Generator(np.random.PCG64(41))
    for l in (1, 2):
        C = levels[l]
        x = (rng.standard_normal((R, 2, C.Nt, C.Nx)) + 1j * rng.standard_normal((R, 2, C.Nt, C.Nx)))
        x *= np.exp(rng.uniform(-3, 3, size=(R, 1, 1, 1)))          # right-hand sides of unequal size
        x = x.astype(np.complex64)
        xd = torch.from_numpy(x).to(DEV)
        out = torch.full(x.shape, complex(float("nan"), float("nan")), dtype=torch.complex64, device=DEV)
        A.profile_enable(hier, True)
        A.apply_coarse(hier, l, xd, out)
        A.profile_enable(hier, False)
        assert any(name == "coarse_apply_tc" for name, *_ in A.profile_get(hier))
        got = out.cpu().numpy()
        B = amg.block_stencil(C.A, C.offsets, C.Nt, C.Nx)
        Bq = mixed.quantise_rows(B)
        xq = mixed.quantise_rhs_pow2(x)
        worst_emul = worst_exact = 0.0
        for r in range(R):
            want_q = stencil_apply(Bq, C.offsets, xq[r], C.Nt, C.Nx)
            want = stencil_apply(B, C.offsets, x[r].astype(np.complex128), C.Nt, C.Nx)
            worst_emul = max(worst_emul, relerr(got[r], want_q))
            worst_exact = max(worst_exact, relerr(got[r], want))
        assert worst_emul <= 1e-5, (l, worst_emul)
        assert worst_exact <= 2e-3, (l, worst_exact)
        print(f"level {l} ({C.Nt}x{C.Nx}), R = {R}: vs emulated FP16 operands {worst_emul:.2e}, "
              f"vs exact {worst_exact:.2e}")
    hier.destroy()


def test_tensor_core_coarse_apply_agrees_with_cuda_core_kernels_and_repeats():
    """Same level, same inputs: the tensor-core result (R = 48) against the
    CUDA-core FP32 kernel (one right-hand side per call, FP16 blocks with
    per-block scales) within the FP16 rounding of the operators, against the
    FP64 kernel within 2e-3, and bit for bit the same on a second call."""
    Nt = Nx = 128
    U = random_links(Nt, Nx, 44)
    hier = A.setup(torch.from_numpy(U).to(DEV), 0.1, A.make_params([4, 2], precision=A.SOLVE_MIXED))
    rng = np.random.Generator(np.random.PCG64(45))
    R, l = 48, 1
    n1 = Nt // 4
    x = (rng.standard_normal((R, 2, n1, n1)) + 1j * rng.standard_normal((R, 2, n1, n1))).astype(np.complex64)
    xd = torch.from_numpy(x).to(DEV)
    y_tc = torch.empty_like(xd)
    A.apply_coarse(hier, l, xd, y_tc)
    y_tc2 = torch.empty_like(xd)
    A.apply_coarse(hier, l, xd, y_tc2)
    y64 = torch.empty(x.shape, dtype=torch.complex128, device=DEV)
    A.apply_coarse(hier, l, xd.to(torch.complex128), y64)
    g, g2, g64 = y_tc.cpu().numpy(), y_tc2.cpu().numpy(), y64.cpu().numpy()
    assert np.array_equal(g, g2)
    for r in range(R):
        one = torch.empty_like(xd[r:r + 1])
        A.apply_coarse(hier, l, xd[r:r + 1].contiguous(), one)
        assert relerr(g[r], one.cpu().numpy()[0]) <= 2e-3
        assert relerr(g[r], g64[r]) <= 2e-3
    hier.destroy()


def test_tensor_core_coarse_apply_full_size_sampled_rows_against_oracle():
    """At the benchmark's size and launch (level 1 of a 1024^2 lattice: 256^2
    coarse sites, 64 right-hand sides in one group): sampled output sites,
    including both periodic edges, against the oracle's Galerkin rows built
    locally (oracle.amg.galerkin_rows) -- with the kernel's FP16 operands
    emulated (row-scaled operator, power-of-two scaled right-hand sides) to
    1e-5 of the sampled outputs' largest entry, and against exact FP64 to 2e-3."""
    L, a, R, m0 = 1024, 4, 64, 0.1
    U = random_links(L, L, 71)
    hier = A.setup(torch.from_numpy(U).to(DEV), m0, A.make_params([4, 4, 2], precision=A.SOLVE_MIXED))
    n1 = L // a
    rng = np.random.Generator(np.random.PCG64(72))
    x = (rng.standard_normal((R, 2, n1, n1)) + 1j * rng.standard_normal((R, 2, n1, n1))).astype(np.complex64)
    y = torch.full(x.shape, complex(float("nan"), float("nan")), dtype=torch.complex64, device=DEV)
    A.profile_enable(hier, True)
    A.apply_coarse(hier, 1, torch.from_numpy(x).to(DEV), y)
    A.profile_enable(hier, False)
    assert any(name == "coarse_apply_tc" for name, *_ in A.profile_get(hier))
    got = y.cpu().numpy()
    hier.destroy()
    verts = [(0, 0), (n1 - 1, n1 - 1), (1, n1 // 2), (n1 // 2, 0), (77, 200), (200, 31)]
    rows = amg.galerkin_rows(U, m0, a, verts)
    xf = x.astype(np.complex128).reshape(R, 2, -1)
    xq = mixed.quantise_rhs_pow2(x).reshape(R, 2, -1)     # one scale per whole right-hand side
    want, want_q, g = [], [], []
    for (p, q) in verts:
        ws = sorted(rows[(p, q)])
        B = np.stack([rows[(p, q)][w] for w in ws])              # [K, 2, 2]
        Bq = mixed.quantise_rows(B[:, None])[:, 0]               # the kernel's row-scaled FP16 storage
        for r in range(R):
            want.append(sum(B[k] @ xf[r][:, w] for k, w in enumerate(ws)))
            want_q.append(sum(Bq[k] @ xq[r][:, w] for k, w in enumerate(ws)))
            g.append(got[r][:, p, q])
    want, want_q, g = np.array(want), np.array(want_q), np.array(g)
    e_q, e_x = relerr(g, want_q), relerr(g, want)
    print(f"1024^2 level 1 x 64 RHS, {len(verts)} sampled sites: vs emulated FP16 operands {e_q:.2e}, "
          f"vs exact {e_x:.2e}")
    assert e_q <= 1e-5
    assert e_x <= 2e-3
