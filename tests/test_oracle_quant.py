"""Pins of the oracle's core quantiser against hand-worked cases."""
import os

import numpy as np
import pytest

from oracle import quant

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cases():
    out = []
    with open(os.path.join(GOLDEN, "quant_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            bits, vals, scale, codes = [s.strip() for s in line.split("|")]
            out.append((int(bits), [float(v) for v in vals.split()], float(scale),
                        [int(c) for c in codes.split()]))
    return out


@pytest.mark.parametrize("bits,vals,scale,codes", _cases())
def test_hand_cases(bits, vals, scale, codes):
    planes = np.array(vals, dtype=np.float32).reshape(1, 1, -1)
    q, s = quant.quantize_planes(planes, bits)
    assert s[0] == np.float32(scale)
    assert q.ravel().tolist() == codes


def test_plane_order_mode3_fastest():
    core = np.zeros((2, 3, 4, 5), dtype=np.float32)
    for i3 in range(4):
        for i4 in range(5):
            core[:, :, i3, i4] = 10 * i4 + i3
    planes = quant.planes_of(core)
    assert planes.shape == (20, 2, 3)
    for p in range(20):
        assert np.all(planes[p] == 10 * (p // 4) + (p % 4))


def test_dequantised_error_bound():
    rng = np.random.default_rng(11)
    planes = (rng.standard_normal((6, 17, 13)) * np.logspace(-3, 3, 6)[:, None, None]).astype(np.float32)
    for bits in (2, 4, 8, 12, 16):
        q, s = quant.quantize_planes(planes, bits)
        back = quant.dequantize_planes(q, s)
        qmax = 2 ** (bits - 1) - 1
        assert np.abs(q).max() <= qmax
        # half a step, plus FP32 rounding of the division and the product
        err = np.abs(back - planes)
        assert np.all(err <= s[:, None, None] * 0.5 * (1 + 1e-5) + 1e-30)
        # the plane maximum is coded exactly as +-qmax
        for p in range(planes.shape[0]):
            i = np.argmax(np.abs(planes[p]))
            assert abs(int(q[p].ravel()[i])) == qmax


def test_bits_range():
    with pytest.raises(ValueError):
        quant.quantize_planes(np.zeros((1, 2, 2), np.float32), 1)
    with pytest.raises(ValueError):
        quant.quantize_planes(np.zeros((1, 2, 2), np.float32), 17)


def test_core_of_planes_inverts_planes_of():
    rng = np.random.default_rng(5)
    for ranks in ((4, 3, 2, 5), (3, 2), (2, 2, 3)):
        core = rng.standard_normal(ranks)
        planes = quant.planes_of(core)
        assert planes.shape == (quant.num_planes(ranks), ranks[0], ranks[1])
        assert np.array_equal(quant.core_of_planes(planes, ranks), core)
