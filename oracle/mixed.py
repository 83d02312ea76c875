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


# ---------------------------------------------------------------------------
# FP16 operands of the tensor-core coarse apply for many right-hand sides.
# A tensor-core product sums over the whole K dimension of a tile in one
# instruction, so a scale must not vary along K:
#   - the coarse operator is stored with one FP32 scale per scalar row
#     (coarse site v, spin alpha), s = float32(max over the row's blocks and
#     columns beta of max(|Re|, |Im|)), s = 1 for an all-zero row, entries
#     float16_rn(v / s) (division in FP64), decoded float32(stored) * s;
#   - each right-hand side (all sites and spins) is scaled by a power of two
#     above its largest component, 2^(E - 126) with E the FP32 exponent field
#     of max(|Re|, |Im|) (at least 1), so that x / s is exact and below 1 in
#     magnitude, then rounded to FP16; s = 1 for a zero right-hand side.

def quantise_rows(B: np.ndarray) -> np.ndarray:
    """B[K, n, 2, 2] (block stencil) -> decoded FP16 values with one scale per
    scalar row (site, alpha) over all K blocks and both columns."""
    out = np.empty_like(B)
    for v in range(B.shape[1]):
        for a in range(2):
            row = B[:, v, a, :]
            m = max(np.max(np.abs(row.real)), np.max(np.abs(row.imag)))
            s = np.float32(m)
            if s == 0:
                s = np.float32(1.0)
            inv = 1.0 / np.float64(s)
            re = (row.real * inv).astype(np.float16).astype(np.float32) * s
            im = (row.imag * inv).astype(np.float16).astype(np.float32) * s
            out[:, v, a, :] = re.astype(np.float64) + 1j * im.astype(np.float64)
    return out


def pow2_scale(x32: np.ndarray) -> np.float32:
    """The power-of-two scale of one FP32 right-hand side (complex64 array)."""
    m = max(np.max(np.abs(x32.real)), np.max(np.abs(x32.imag))) if x32.size else np.float32(0)
    m = np.float32(m)
    if m == 0:
        return np.float32(1.0)
    E = int(np.array([m], dtype=np.float32).view(np.uint32)[0] >> 23) & 0xFF
    E = min(max(E, 1), 252)
    return np.float32(2.0 ** (E - 126))


def quantise_rhs_pow2(x: np.ndarray) -> np.ndarray:
    """x[R, ...] complex64 right-hand sides -> decoded FP16 values, one
    power-of-two scale per right-hand side (x / s is exact, then FP16 rounding)."""
    x = np.asarray(x, dtype=np.complex64)
    out = np.empty(x.shape, dtype=np.complex128)
    for r in range(x.shape[0]):
        s = pow2_scale(x[r])
        inv = np.float32(1.0) / s
        re = (x[r].real * inv).astype(np.float16).astype(np.float64) * np.float64(s)
        im = (x[r].imag * inv).astype(np.float16).astype(np.float64) * np.float64(s)
        out[r] = re + 1j * im
    return out
