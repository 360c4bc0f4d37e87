"""Pins of the oracle's colour pre-pass (Section III-A) against facts that do
not come from the oracle itself: hand-worked BT.601 values, the algebraic
inverse of BT.601, the white point and grey axis of IPT, and the opponent
axes IPT is defined by (P red-green, T yellow-blue)."""
import os

import numpy as np
import pytest

from oracle import colour

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rgb8(r, g, b):
    return np.array([r, g, b], dtype=np.uint8)


def test_bt601_primaries_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "bt601_primaries.txt"), comments="#")
    rgb8 = rows[:, :3].astype(np.uint8)
    want = rows[:, 3:]
    got = colour.ycbcr601(colour.rgb_prime(rgb8))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_bt601_algebraic_inverse_roundtrip():
    # Inverse written from the standard's definitions, solved by hand:
    # R' = Y' + 1.402 Cr, B' = Y' + 1.772 Cb, G' = (Y' - 0.299 R' - 0.114 B') / 0.587
    rng = np.random.default_rng(7)
    rgb8 = rng.integers(0, 256, size=(1000, 3), dtype=np.uint8)
    p = colour.rgb_prime(rgb8)
    ycc = colour.ycbcr601(p)
    y, cb, cr = ycc[:, 0], ycc[:, 1], ycc[:, 2]
    r = y + 1.402 * cr
    b = y + 1.772 * cb
    g = (y - 0.299 * r - 0.114 * b) / 0.587
    np.testing.assert_allclose(np.stack([r, g, b], 1), p, atol=1e-12)


def test_bt601_grey_has_no_chroma():
    v = np.arange(256, dtype=np.uint8)
    ycc = colour.ycbcr601(colour.rgb_prime(np.stack([v, v, v], 1)))
    np.testing.assert_allclose(ycc[:, 0], v / 255.0, atol=1e-12)
    assert np.abs(ycc[:, 1:]).max() < 1e-12


def test_ipt_white_point():
    # D65 white maps to LMS ~ (1,1,1) (the HPE matrix is normalised to D65),
    # and the IPT rows give I = 0.4+0.4+0.2 = 1, P = T = 0 for equal cone
    # responses.  The published matrices carry four digits, hence 1e-3.
    ipt = colour.ipt(colour.rgb_prime(_rgb8(255, 255, 255)))
    np.testing.assert_allclose(ipt, [1.0, 0.0, 0.0], atol=1e-3)


@pytest.mark.parametrize("gamma", [2.2, 1.0, 2.4])
def test_ipt_grey_axis(gamma):
    # grey level g: linear value g^gamma on all three channels, LMS = g^gamma*(1,1,1)
    # so I = (g^gamma)^0.43 and P = T = 0.
    v = np.arange(1, 256, dtype=np.uint8)
    ipt = colour.ipt(colour.rgb_prime(np.stack([v, v, v], 1)), gamma)
    g = v / 255.0
    np.testing.assert_allclose(ipt[:, 0], g ** (0.43 * gamma), rtol=2e-3)
    assert np.abs(ipt[:, 1:]).max() < 2e-3
    assert np.all(np.diff(ipt[:, 0]) > 0)


def test_ipt_opponent_axes():
    # Section III-A: I is lightness, P the red-green and T the yellow-blue
    # dimension.  Red is positive on P, green negative; yellow is positive on
    # T, blue negative.
    red = colour.ipt(colour.rgb_prime(_rgb8(255, 0, 0)))
    green = colour.ipt(colour.rgb_prime(_rgb8(0, 255, 0)))
    yellow = colour.ipt(colour.rgb_prime(_rgb8(255, 255, 0)))
    blue = colour.ipt(colour.rgb_prime(_rgb8(0, 0, 255)))
    assert red[1] > 0.2 and green[1] < -0.2
    assert yellow[2] > 0.2 and blue[2] < -0.2


def test_stack_layout():
    # T(x, y, c, k) is channel c of pixel (x, y) of image k, image row-major
    # with x along the row.
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(4, 5, 7, 3), dtype=np.uint8)   # K, s2, s1, 3
    T = colour.colour_convert(img, "ycbcr")
    assert T.shape == (7, 5, 3, 4)
    for (x, y, k) in [(0, 0, 0), (6, 4, 3), (3, 2, 1)]:
        want = colour.ycbcr601(colour.rgb_prime(img[k, y, x]))
        np.testing.assert_allclose(T[x, y, :, k], want, atol=1e-15)
