"""Seeded synthetic multi-exposure stereo scenes.

This module only simulates a camera: it holds none of the coding scheme's
arithmetic (no colour transform, no tensor algebra).  Both the CPU oracle
tests and the CUDA path consume the same 8-bit images it produces.

The paper's own data (four natural scenes captured with a ZED stereo camera at
2208x1242, Section IV and Table "Experimental Parameters") is not available,
so these scenes stand in for it.  Recipe:

1. Irradiance.  For each colour channel c,
   E0_c(y, x) = sum_{j=1..8} a_j * p_j(y) * q_j(x) * m_jc
   with smooth positive profiles p, q = 1 + 0.9 cos(2 pi f t + phi),
   f uniform in [0.5, 3] cycles per image, tints m_jc uniform in [0.6, 1.4]
   and lognormal amplitudes a_j.  A constant offset then sets the dynamic range
   max E / min E to exactly 2^12 (the field stays of rank <= 9 per channel),
   and a global scale puts the geometric mean at 0.18.
2. Disparity.  An integer map d(y, x) in [0, d_max], constant on 16x16 blocks,
   drawn from a smoothed random field.  The right view is
   E_right(y, x) = E_left(y, clamp(x - d(y, x))).
3. Exposures.  For each exposure time t_e the 8-bit value is
   round(255 * clip((t_e * E)^(1/2.2), 0, 1)).

Layout of the result: uint8 array of shape (K, s2, s1, 3), i.e. K images,
each row-major with s1 pixels per row and interleaved R, G, B.  Image index
k = view * E + exposure (view 0 = left).  Mode 1 of the stacked tensor is the
pixel column x (length s1), mode 2 the row y (length s2).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["SceneSpec", "make_stack", "config_spec", "CONFIGS", "seed_for"]


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    s1: int                 # pixels per row (mode 1)
    s2: int                 # rows (mode 2)
    exposures: tuple        # exposure times t_e
    views: int = 2
    d_max: int = 4
    rank: int = 8
    dyn_range_log2: float = 12.0
    gamma: float = 2.2

    @property
    def K(self) -> int:
        return self.views * len(self.exposures)


# The five workloads, by their sizes.  Ranks, iterations and colour space are
# fixed here too so that tests and the benchmark agree on them.
CONFIGS = {
    # 64x48, 2 views x 3 exposures, Y'CbCr, ranks (16,12,3,6), 10 sweeps, tol 1e-8
    "small_64x48": dict(spec=SceneSpec(64, 48, (0.25, 1.0, 4.0), d_max=4),
                        space="ycbcr", ranks=(16, 12, 3, 6), iters=10, tol=1e-8),
    # 1024x768, 2 views x 3 exposures, IPT, ranks (256,192,3,6), 20 sweeps
    "xga_1024x768": dict(spec=SceneSpec(1024, 768, (0.25, 1.0, 4.0), d_max=24),
                         space="ipt", ranks=(256, 192, 3, 6), iters=20, tol=0.0),
    # 1920x1080, 2 views x 5 exposures at stops -4..+4, ranks (384,256,3,10)
    "fhd_1920x1080": dict(spec=SceneSpec(1920, 1080, (2.0 ** -4, 2.0 ** -2, 1.0, 2.0 ** 2, 2.0 ** 4),
                                         d_max=48),
                          space="ipt", ranks=(384, 256, 3, 10), iters=20, tol=0.0),
}

_CONFIG_INDEX = {"small_64x48": 1, "xga_1024x768": 2, "fhd_1920x1080": 3}


def seed_for(config: str, stack_index: int = 0) -> int:
    """Seed of stack `stack_index` of a named workload: 1000*config + index."""
    return 1000 * _CONFIG_INDEX[config] + stack_index


def config_spec(name: str) -> dict:
    return dict(CONFIGS[name])


def _profile(rng: np.random.Generator, n: int) -> np.ndarray:
    f = rng.uniform(0.5, 3.0)
    phi = rng.uniform(0.0, 2.0 * np.pi)
    t = np.arange(n, dtype=np.float64) / n
    return 1.0 + 0.9 * np.cos(2.0 * np.pi * f * t + phi)


def _irradiance(rng: np.random.Generator, spec: SceneSpec) -> np.ndarray:
    """Linear-light irradiance, shape (3, s2, s1), strictly positive."""
    a = rng.lognormal(mean=0.0, sigma=1.0, size=spec.rank)
    E0 = np.zeros((3, spec.s2, spec.s1))
    for j in range(spec.rank):
        p = _profile(rng, spec.s2)
        q = _profile(rng, spec.s1)
        m = rng.uniform(0.6, 1.4, size=3)
        base = a[j] * np.outer(p, q)
        for c in range(3):
            E0[c] += m[c] * base
    lo, hi = E0.min(), E0.max()
    ratio = 2.0 ** spec.dyn_range_log2
    offset = (hi - lo) / (ratio - 1.0)
    E = E0 - lo + offset                       # max/min == ratio exactly
    E *= 0.18 / np.exp(np.mean(np.log(E)))     # geometric mean 0.18
    return E


def _disparity(rng: np.random.Generator, spec: SceneSpec) -> np.ndarray:
    """Integer disparity, shape (s2, s1), constant on 16x16 blocks."""
    by = -(-spec.s2 // 16)
    bx = -(-spec.s1 // 16)
    field = rng.standard_normal((by + 4, bx + 4))
    # smooth with a 5x5 box filter
    sm = np.zeros((by, bx))
    for dy in range(5):
        for dx in range(5):
            sm += field[dy:dy + by, dx:dx + bx]
    sm -= sm.min()
    if sm.max() > 0:
        sm /= sm.max()
    d_blocks = np.rint(sm * spec.d_max).astype(np.int64)
    d = np.repeat(np.repeat(d_blocks, 16, axis=0), 16, axis=1)
    return d[:spec.s2, :spec.s1]


def make_stack(spec: SceneSpec, seed: int) -> np.ndarray:
    """uint8 array (K, s2, s1, 3): K = views*len(exposures) LDR images."""
    rng = np.random.Generator(np.random.PCG64(seed))
    E_left = _irradiance(rng, spec)
    d = _disparity(rng, spec)
    xs = np.arange(spec.s1)[None, :] - d
    np.clip(xs, 0, spec.s1 - 1, out=xs)
    ys = np.broadcast_to(np.arange(spec.s2)[:, None], xs.shape)
    E_right = E_left[:, ys, xs]
    views = [E_left, E_right][:spec.views]
    out = np.empty((spec.K, spec.s2, spec.s1, 3), dtype=np.uint8)
    inv_g = 1.0 / spec.gamma
    k = 0
    for E in views:
        Ehwc = np.moveaxis(E, 0, -1)
        for t in spec.exposures:
            v = np.clip(np.power(t * Ehwc, inv_g), 0.0, 1.0)
            out[k] = np.rint(255.0 * v).astype(np.uint8)
            k += 1
    return out
