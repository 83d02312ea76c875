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
