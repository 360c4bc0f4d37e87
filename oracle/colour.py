"""Colour pre-pass of Section III-A and the stacking of Section III-B.

Readings of the paper (it gives no matrices, offsets or ranges):

* Y'CbCr: ITU-R BT.601 non-constant luminance, full range, 4:4:4, no
  offsets: Y' = 0.299 R' + 0.587 G' + 0.114 B', Cb = (B' - Y') / 1.772,
  Cr = (R' - Y') / 1.402, with R', G', B' = u8 / 255.  (Section III-A names
  BT.601 for Y'CbCr; the constant-luminance BT.2020 variant it mentions is not
  the default.)
* IPT (Ebner & Fairchild): linearise R = (R')^gamma (gamma = 2.2 matches the
  camera response of the synthetic scenes), linear sRGB (D65) -> XYZ with the
  sRGB matrix, XYZ -> LMS with the D65-normalised Hunt-Pointer-Estevez matrix,
  L' = sign(L) |L|^0.43 (same for M, S), then the published LMS'->IPT matrix.

Stacking: the images (K, s2, s1, 3) become the order-4 tensor
T(x, y, c, k) of shape (s1, s2, 3, K); mode 1 is the pixel column.
"""
from __future__ import annotations

import numpy as np

# BT.601 luma weights and chroma divisors (ITU-R BT.601).
_KR, _KG, _KB = 0.299, 0.587, 0.114
_CB_DIV, _CR_DIV = 1.772, 1.402

# Linear sRGB (D65) -> CIE XYZ (IEC 61966-2-1).
M_RGB2XYZ = np.array([[0.4124, 0.3576, 0.1805],
                      [0.2126, 0.7152, 0.0722],
                      [0.0193, 0.1192, 0.9505]])
# XYZ -> LMS, Hunt-Pointer-Estevez normalised to D65 (Ebner & Fairchild).
M_XYZ2LMS = np.array([[0.4002, 0.7075, -0.0807],
                      [-0.2280, 1.1500, 0.0612],
                      [0.0, 0.0, 0.9184]])
# Non-linear L'M'S' -> IPT (Ebner & Fairchild).
M_LMS2IPT = np.array([[0.4000, 0.4000, 0.2000],
                      [4.4550, -4.8510, 0.3960],
                      [0.8056, 0.3572, -1.1628]])
IPT_EXPONENT = 0.43


def rgb_prime(rgb8: np.ndarray) -> np.ndarray:
    """u8 -> gamma-encoded R'G'B' in [0, 1], FP64."""
    return np.asarray(rgb8, dtype=np.float64) / 255.0


def ycbcr601(rgbp: np.ndarray) -> np.ndarray:
    """R'G'B' (..., 3) -> Y'CbCr (..., 3), BT.601 full range (Section III-A)."""
    r, g, b = rgbp[..., 0], rgbp[..., 1], rgbp[..., 2]
    y = _KR * r + _KG * g + _KB * b
    cb = (b - y) / _CB_DIV
    cr = (r - y) / _CR_DIV
    return np.stack([y, cb, cr], axis=-1)


def ipt(rgbp: np.ndarray, gamma: float = 2.2) -> np.ndarray:
    """R'G'B' (..., 3) -> IPT (..., 3) (Section III-A, Ebner & Fairchild)."""
    lin = np.power(rgbp, gamma)
    xyz = lin @ M_RGB2XYZ.T
    lms = xyz @ M_XYZ2LMS.T
    lmsp = np.sign(lms) * np.power(np.abs(lms), IPT_EXPONENT)
    return lmsp @ M_LMS2IPT.T


def colour_convert(rgb8: np.ndarray, space: str, gamma: float = 2.2) -> np.ndarray:
    """Images (K, s2, s1, 3) u8 -> stacked tensor T of shape (s1, s2, 3, K).

    T(x, y, c, k) is channel c of pixel (x, y) of image k: the stack
    "T_MES^c" of Section III-B, H x W x colour x (view * exposure).
    """
    p = rgb_prime(rgb8)
    if space == "ycbcr":
        conv = ycbcr601(p)
    elif space == "ipt":
        conv = ipt(p, gamma)
    else:
        raise ValueError(f"unknown colour space {space!r}")
    # (K, s2, s1, 3) -> (s1, s2, 3, K)
    return np.ascontiguousarray(np.transpose(conv, (2, 1, 3, 0)))


def frobenius2(T: np.ndarray) -> float:
    """||T||_F^2, the squared norm used by the fit."""
    return float(np.sum(np.square(T, dtype=np.float64)))
