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


def test_srgb_to_xyz_matrix_from_primaries_and_d65():
    # IEC 61966-2-1 builds the matrix from the chromaticities of the sRGB
    # primaries (x, y) R (0.64, 0.33), G (0.30, 0.60), B (0.15, 0.06) and of
    # D65 (0.3127, 0.3290): the columns are the primaries' XYZ, scaled so
    # that R = G = B = 1 gives the white point with Y = 1.  Derived here from
    # those six numbers alone, it must round to the oracle's 4-digit table
    # entry by entry (a typo in any fourth digit fails).
    xyz = lambda x, y: np.array([x / y, 1.0, (1.0 - x - y) / y])
    P = np.stack([xyz(0.64, 0.33), xyz(0.30, 0.60), xyz(0.15, 0.06)], 1)
    M = P * np.linalg.solve(P, xyz(0.3127, 0.3290))
    np.testing.assert_array_equal(np.round(M, 4), colour.M_RGB2XYZ)
    assert np.abs(M - colour.M_RGB2XYZ).max() < 5e-5


def test_lms_matrix_is_normalised_to_d65():
    # Ebner-Fairchild normalise the Hunt-Pointer-Estevez cone matrix so that
    # the D65 white (CIE 1931, X = 0.95047, Y = 1, Z = 1.08883) gives equal
    # cone responses L = M = S = 1; with four published digits each row lands
    # within 1e-4 of 1 (a fourth-digit typo in a large entry moves it further).
    lms = colour.M_XYZ2LMS @ np.array([0.95047, 1.0, 1.08883])
    assert np.abs(lms - 1.0).max() < 1e-4
    assert colour.M_XYZ2LMS[2, 0] == 0.0 and colour.M_XYZ2LMS[2, 1] == 0.0


def test_ipt_matrix_rows_are_achromatic_exact():
    # The IPT matrix maps equal L'M'S' to I = 1, P = T = 0: the first row sums
    # to exactly 1, the two opponent rows to exactly 0 (4.4550 - 4.8510 +
    # 0.3960 and 0.8056 + 0.3572 - 1.1628), so a single-digit typo anywhere in
    # the matrix breaks one of the sums.
    np.testing.assert_allclose(colour.M_LMS2IPT.sum(1), [1.0, 0.0, 0.0], rtol=0, atol=1e-12)
    assert colour.IPT_EXPONENT == 0.43


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


# ---- constant-luminance BT.2020 Y'CbCr and the inverse transforms ----

_D65 = (0.3127, 0.3290)
_PRIM_709 = ((0.640, 0.330), (0.300, 0.600), (0.150, 0.060))
_PRIM_2020 = ((0.708, 0.292), (0.170, 0.797), (0.131, 0.046))


def _npm(prims, white):
    """Normalised primary matrix (linear RGB -> XYZ) from the xy
    chromaticities of the primaries and the white point: columns are the
    primaries' XYZ scaled so that RGB = (1,1,1) gives the white with Y = 1."""
    P = np.array([[x / y, 1.0, (1 - x - y) / y] for x, y in prims]).T
    wx, wy = white
    W = np.array([wx / wy, 1.0, (1 - wx - wy) / wy])
    return P * np.linalg.solve(P, W)


def test_bt2020_luminance_weights_from_the_primaries():
    # the luminance row of the BT.2020 primary matrix, derived here from the
    # chromaticities, equals the published weights (four digits)
    np.testing.assert_allclose(_npm(_PRIM_2020, _D65)[1], [colour.KR20, colour.KG20, colour.KB20], atol=5e-5)
    # and the same derivation gives the BT.601/709 weights' row for 709 primaries
    np.testing.assert_allclose(_npm(_PRIM_709, _D65)[1], [0.2126, 0.7152, 0.0722], atol=5e-5)


def test_709_to_2020_matrix_from_the_primaries():
    M = np.linalg.solve(_npm(_PRIM_2020, _D65), _npm(_PRIM_709, _D65))
    np.testing.assert_allclose(colour.M_709_TO_2020, M, atol=1e-4)
    np.testing.assert_allclose(colour.M_709_TO_2020.sum(axis=1), 1.0, atol=1e-12)


def test_bt2020_transfer_function():
    assert colour.bt2020_oetf(0.0) == 0.0
    assert abs(colour.bt2020_oetf(1.0) - 1.0) < 1e-12
    b = colour.OETF_BETA
    # the two segments meet at beta (to the four digits of the constants)
    assert abs(4.5 * b - (colour.OETF_ALPHA * b ** 0.45 - (colour.OETF_ALPHA - 1))) < 2e-5
    E = np.linspace(-0.05, 1.0, 2001)
    Ep = colour.bt2020_oetf(E)
    assert np.all(np.diff(Ep) > 0)
    np.testing.assert_allclose(colour.bt2020_oetf_inverse(Ep), E, atol=1e-12)


@pytest.mark.parametrize("rgb,chan,want", [((0, 0, 1), 1, 0.5), ((1, 1, 0), 1, -0.5),
                                           ((1, 0, 0), 2, 0.5), ((0, 1, 1), 2, -0.5)])
def test_cl_chroma_reaches_its_range_at_the_primaries(rgb, chan, want):
    # BT.2020 sizes the four chroma divisors so that the BT.2020 primaries and
    # secondaries land on +-1/2: blue and yellow on Cb, red and cyan on Cr.
    # The branch (divisor by sign) is what puts each extreme on +-1/2.
    ycc = colour.ycbcr2020cl_from_linear(np.array(rgb, dtype=np.float64))
    assert abs(ycc[chan] - want) < 3e-4


def test_cl_grey_axis():
    v = np.arange(256, dtype=np.uint8)
    g = v / 255.0
    for gamma in (2.2, 1.0):
        ycc = colour.ycbcr2020cl(colour.rgb_prime(np.stack([v, v, v], 1)), gamma)
        np.testing.assert_allclose(ycc[:, 0], colour.bt2020_oetf(g ** gamma), atol=1e-12)
        assert np.abs(ycc[:, 1:]).max() < 1e-12


@pytest.mark.parametrize("space", ["ycbcr", "ipt", "ycbcr2020cl"])
def test_inverse_transforms_recover_the_images(space):
    rng = np.random.default_rng(11)
    rgb8 = rng.integers(0, 256, size=(3, 7, 9, 3), dtype=np.uint8)
    rgb8[0, 0, :4] = [[0, 0, 0], [255, 255, 255], [255, 0, 0], [0, 0, 255]]
    T = colour.colour_convert(rgb8, space)
    back = colour.colour_invert(T, space)
    # FP64 round-off near black is raised to the power 1/gamma: 1e-6, far
    # inside the half step 0.5/255 that the 8-bit recovery needs
    np.testing.assert_allclose(back, colour.rgb_prime(rgb8), atol=1e-6)
    assert np.array_equal(colour.to_u8(back), rgb8)


def test_to_u8_rounds_half_to_even_and_clamps():
    x = np.array([-0.1, 0.0, 0.5 / 255, 1.5 / 255, 2.5 / 255, 254.5 / 255, 1.0, 1.2])
    assert colour.to_u8(x).tolist() == [0, 0, 0, 2, 2, 254, 255, 255]


def test_psnr8_definition():
    a = np.zeros((2, 3, 4, 3), dtype=np.uint8)
    b = a.copy()
    assert colour.psnr8(a, b) == float("inf")
    b[0, 0, 0, 0] = 1            # one byte off by one of n = 72: mse = 1/72
    assert abs(colour.psnr8(a, b) - 10 * np.log10(255.0 ** 2 * 72)) < 1e-12
    b[:] = 255                   # every byte off by the peak: 0 dB
    assert colour.psnr8(a, b) == 0.0
