"""Core quantiser: the rate knob of the coding scheme.

The paper adjusts the bitrate "by changing the rank of core tensor and its
quantization" (abstract, Section I) but never defines the quantiser.  Reading
used here: the core Q (R_1 x R_2 x R_3 x ... x R_N) is cut into its
R_1 x R_2 planes, one per index of modes 3..N (these are the planes handed to
the video coder).  For each plane:

    m     = max |Q_plane|                      (exact)
    qmax  = 2^(bits-1) - 1
    scale = m / qmax                           (one IEEE FP32 division)
    q     = clamp(rint(x / scale), -qmax, qmax)   (FP32 division, ties to even)
    m == 0  ->  scale = 0, q = 0

Dequantisation is x ~= q * scale (FP32).  The arithmetic is FP32 by
definition so that an integer code is decided in the same precision on every
implementation.  Parity is then bit-exact for identical FP32 input.
"""
from __future__ import annotations

import numpy as np


def num_planes(ranks) -> int:
    p = 1
    for r in ranks[2:]:
        p *= int(r)
    return p


def planes_of(core: np.ndarray) -> np.ndarray:
    """Core (R_1, R_2, ...) -> planes (P, R_1, R_2) with P = prod R_3..R_N.

    Plane p holds Q(:, :, i_3, ..., i_N) with p = i_3 + R_3 * (i_4 + ...),
    i.e. the mode-3 index varies fastest, matching a first-mode-fastest
    memory layout of the core.
    """
    c = np.asarray(core)
    if c.ndim == 1:
        c = c[:, None]
    r1, r2 = c.shape[0], c.shape[1]
    P = int(np.prod(c.shape[2:], dtype=np.int64)) if c.ndim > 2 else 1
    # Fortran-order flatten of the trailing modes puts mode 3 fastest.
    flat = np.reshape(c, (r1, r2, P), order="F")
    return np.transpose(flat, (2, 0, 1))


def core_of_planes(planes: np.ndarray, ranks) -> np.ndarray:
    """Planes (P, R1, R2) -> core of shape `ranks`: the inverse of planes_of."""
    flat = np.transpose(np.asarray(planes), (1, 2, 0))
    return np.reshape(flat, tuple(int(r) for r in ranks), order="F")


def quantize_planes(planes: np.ndarray, bits: int):
    """FP32 planes (P, R1, R2) -> (int16 codes (P, R1, R2), FP32 scales (P,))."""
    if not 2 <= bits <= 16:
        raise ValueError("bits must be in 2..16")
    x = np.asarray(planes, dtype=np.float32)
    qmax = np.float32(2 ** (bits - 1) - 1)
    P = x.shape[0]
    q = np.zeros(x.shape, dtype=np.int16)
    scales = np.zeros(P, dtype=np.float32)
    for p in range(P):
        m = np.float32(np.max(np.abs(x[p]))) if x[p].size else np.float32(0)
        if m == 0:
            continue
        s = np.float32(m / qmax)
        scales[p] = s
        v = np.rint(np.divide(x[p], s, dtype=np.float32))
        q[p] = np.clip(v, -qmax, qmax).astype(np.int16)
    return q, scales


def dequantize_planes(q: np.ndarray, scales: np.ndarray) -> np.ndarray:
    return (q.astype(np.float32) * scales.astype(np.float32)[:, None, None]).astype(np.float32)
