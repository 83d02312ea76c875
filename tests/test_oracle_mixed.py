"""Pins of the oracle's FP16 + scale storage emulation."""
import numpy as np

from oracle import mixed


def test_quantisation_error_bound_and_exact_cases():
    rng = np.random.Generator(np.random.PCG64(50))
    B = rng.standard_normal((3, 8, 30)) + 1j * rng.standard_normal((3, 8, 30))
    B[1] *= 1e-6
    B[2] = 0
    Q = mixed.quantise_tiles(B)
    for t in range(2):
        m = max(np.abs(B[t].real).max(), np.abs(B[t].imag).max())
        # FP16 keeps 11 significant bits: error <= 2^-11 of the block scale (+ FP32 decode)
        assert np.max(np.abs(Q[t] - B[t])) <= (2.0 ** -11) * m * (1 + 1e-6)
    assert np.all(Q[2] == 0)
    # values on the FP16 grid of their scale are exact; the largest entry maps to +-1 exactly
    grid = np.array([[1.0 + 0.5j, -0.25, 0.125j]])
    assert np.array_equal(mixed.quantise_tiles(grid[None])[0], grid)


def test_quantisation_is_idempotent():
    rng = np.random.Generator(np.random.PCG64(51))
    B = rng.standard_normal((5, 4, 2, 2)) + 1j * rng.standard_normal((5, 4, 2, 2))
    Q = mixed.quantise_blocks(B)
    assert np.array_equal(mixed.quantise_blocks(Q), Q)


def test_round_half_even_at_fp16_ties():
    # 1 + 2^-11 lies half-way between 1 and 1 + 2^-10: rounds to even (1.0)
    x = np.array([[[2.0 + 0j, 1.0 + 2.0 ** -11]]])        # block max 2 -> scale 2
    q = mixed.quantise_tiles(x)[0, 0]
    assert q[1] == 1.0


def test_row_scaled_quantisation_bound_and_exact_cases():
    rng = np.random.Generator(np.random.PCG64(52))
    B = rng.standard_normal((21, 6, 2, 2)) + 1j * rng.standard_normal((21, 6, 2, 2))
    B[:, 2, 1, :] *= 1e-5            # one row much smaller than its neighbours
    B[:, 3, 0, :] = 0                # an all-zero row
    Q = mixed.quantise_rows(B)
    for v in range(6):
        for a in range(2):
            row = B[:, v, a, :]
            m = max(np.abs(row.real).max(), np.abs(row.imag).max())
            # 11 significant bits relative to the row's own largest entry, not the level's
            for part in (np.real, np.imag):
                assert np.max(np.abs(part(Q[:, v, a, :]) - part(row))) <= (2.0 ** -12) * m * (1 + 1e-6)
    assert np.all(Q[:, 3, 0, :] == 0)
    # a row whose entries lie on the FP16 grid of its largest entry is exact;
    # the other spin row of the same site has its own scale
    G = np.zeros((2, 1, 2, 2), dtype=complex)
    G[0, 0, 0] = [4.0 + 2.0j, -1.0]
    G[1, 0, 0] = [0.5j, 0.25]
    G[0, 0, 1] = [1e-3, 3e-3j]
    Qg = mixed.quantise_rows(G)
    assert np.array_equal(Qg[:, :, 0, :], G[:, :, 0, :])
    assert np.max(np.abs(Qg[:, :, 1, :] - G[:, :, 1, :])) <= 2.0 ** -12 * 3e-3 * 1.000001
    assert np.array_equal(mixed.quantise_rows(Q), Q)      # idempotent


def test_pow2_rhs_scale_is_exact_power_above_the_largest_component():
    rng = np.random.Generator(np.random.PCG64(53))
    x = (rng.standard_normal((4, 2, 8, 8)) + 1j * rng.standard_normal((4, 2, 8, 8))).astype(np.complex64)
    x[1] *= np.float32(3e4)          # would overflow FP16 without the scale
    x[2] *= np.float32(1e-7)         # would be subnormal in FP16 without the scale
    x[3] = 0
    for r in range(3):
        s = float(mixed.pow2_scale(x[r]))
        m = max(np.abs(x[r].real).max(), np.abs(x[r].imag).max())
        assert np.log2(s) == np.round(np.log2(s))          # a power of two
        assert m < s <= 2 * m                               # just above the largest component
    assert mixed.pow2_scale(x[3]) == 1
    assert mixed.pow2_scale(np.array([1.0 + 0j], dtype=np.complex64)) == 2     # exactly 2^0 -> 2^1
    Q = mixed.quantise_rhs_pow2(x)
    for r in range(3):
        s = float(mixed.pow2_scale(x[r]))
        # FP16 rounding of x / s (|x / s| < 1): absolute error <= 2^-12 s (normal range)
        # plus the subnormal spacing 2^-24 s for the smallest entries
        for part in (np.real, np.imag):
            assert np.max(np.abs(part(Q[r]) - part(x[r]))) <= (2.0 ** -12 + 2.0 ** -24) * s
    assert np.all(Q[3] == 0)
    # entries on the FP16 grid of the scale are kept exactly
    g = np.array([[0.5 + 0.25j, -0.375, 0.0009765625j]], dtype=np.complex64)
    assert np.array_equal(mixed.quantise_rhs_pow2(g), g.astype(np.complex128))


def test_row_scale_spans_blocks_of_one_spin_row_only():
    # one scalar row (site 0, alpha 0) with entries 1 and 3e-7 in two different
    # blocks: with the row's scale 1 the small entry is an FP16 subnormal
    # (spacing 2^-24), which a per-block scale would have kept to 11 bits
    H = np.zeros((2, 1, 2, 2), dtype=complex)
    H[0, 0, 0, 0] = 1.0
    H[1, 0, 0, 1] = 3e-7
    H[0, 0, 1, 0] = 3e-7          # alone in the other spin row: its own scale keeps it
    Q = mixed.quantise_rows(H)
    assert Q[1, 0, 0, 1] == float(np.float16(3e-7))
    assert abs(Q[1, 0, 0, 1] - 3e-7) > 1e-9
    assert abs(Q[0, 0, 1, 0] - 3e-7) <= 3e-7 * 2.0 ** -23


def test_pow2_rhs_scale_is_one_per_right_hand_side():
    # a component 1e-5 beside one of 1e3 in the same right-hand side: x / s is
    # below half the smallest FP16 subnormal and rounds to zero; the other
    # right-hand side keeps its own scale
    x = np.zeros((2, 4), dtype=np.complex64)
    x[0, 0] = 1e3
    x[0, 1] = 1e-5
    x[1, 1] = 1e-5
    Q = mixed.quantise_rhs_pow2(x)
    assert Q[0, 1] == 0 and Q[0, 0] == 1e3
    assert abs(Q[1, 1] - 1e-5) <= 1e-5 * 2.0 ** -11
