"""Oracle: emulation of the reduced-precision storage used by the mixed-precision
V-cycle (FP32 vectors, FP16 interpolator and coarse blocks with an FP32 scale).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper states no precision for its solver.  The mixed-precision form keeps
the outer FGMRES in FP64 and stores the interpolator P and the coarse operator's
2x2 blocks in FP16 with one FP32 scale per block, where a block is one tile of
P (all 8 columns x 2(a^2 - 1) rows) or one 2x2 block of the coarse operator:
    s = float32(max over the block of max(|Re|, |Im|)),   s = 1 when the block is 0,
    stored value = float16_round_to_nearest_even(v / s)   (division in FP64),
    decoded value = float32(stored) * s.
These functions produce the decoded FP64 values, so that FP64 arithmetic on them
reproduces what the FP32 kernels compute up to FP32 rounding.
"""
from __future__ import annotations

import numpy as np


def _quantise(block: np.ndarray) -> np.ndarray:
    m = max(np.max(np.abs(block.real)), np.max(np.abs(block.imag))) if block.size else 0.0
    s = np.float32(m)
    if s == 0:
        s = np.float32(1.0)
    inv = 1.0 / np.float64(s)
    re = (block.real * inv).astype(np.float16).astype(np.float32) * s
    im = (block.imag * inv).astype(np.float16).astype(np.float32) * s
    return re.astype(np.float64) + 1j * im.astype(np.float64)


def quantise_tiles(P_tiles: np.ndarray) -> np.ndarray:
    """P_tiles[tile, 8, nrows] -> decoded FP16+scale values, one scale per tile."""
    out = np.empty_like(P_tiles)
    for t in range(P_tiles.shape[0]):
        out[t] = _quantise(P_tiles[t])
    return out


def quantise_blocks(B: np.ndarray) -> np.ndarray:
    """B[K, n, 2, 2] (block stencil) -> decoded FP16+scale values, one scale per 2x2 block."""
    out = np.empty_like(B)
    for k in range(B.shape[0]):
        for v in range(B.shape[1]):
            out[k, v] = _quantise(B[k, v])
    return out


def round32(z: np.ndarray) -> np.ndarray:
    """Round a complex128 array to complex64 and back."""
    return z.astype(np.complex64).astype(np.complex128)
