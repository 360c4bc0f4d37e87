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

* Constant-luminance Y'CbCr (ITU-R BT.2020, the variant Section III-A credits
  with separating intensity from chroma): linearise as for IPT, convert the
  BT.709/sRGB primaries to BT.2020 primaries (ITU-R BT.2087 matrix), form the
  linear luminance Yc = 0.2627 R + 0.6780 G + 0.0593 B, apply the BT.2020
  transfer function (12-bit constants alpha = 1.0993, beta = 0.0181) to Yc,
  B and R, and take Cbc = (B' - Yc') / 1.9404 (B' - Yc' <= 0) or / 1.5816
  (> 0), Crc = (R' - Yc') / 1.7184 (<= 0) or / 0.9936 (> 0).
* Inverse transforms (the low-rank approximated images go to the encoder as
  images, Section III-C): each space solved back to R'G'B'; a linear value
  below zero (out of gamut after the approximation) keeps its sign through
  the power functions; 8-bit output is clamp(rint(255 R'), 0, 255).

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


# BT.2020 luminance weights, transfer function and constant-luminance chroma
# divisors (ITU-R BT.2020, 12-bit system constants).
KR20, KG20, KB20 = 0.2627, 0.6780, 0.0593
OETF_ALPHA, OETF_BETA = 1.0993, 0.0181
CL_NB, CL_PB, CL_NR, CL_PR = 1.9404, 1.5816, 1.7184, 0.9936
# Linear BT.709 (sRGB) primaries -> linear BT.2020 primaries (ITU-R BT.2087).
M_709_TO_2020 = np.array([[0.6274, 0.3293, 0.0433],
                          [0.0691, 0.9195, 0.0114],
                          [0.0164, 0.0880, 0.8956]])


def bt2020_oetf(E: np.ndarray) -> np.ndarray:
    """BT.2020 transfer function E' of linear E in [0, 1]; the linear segment
    4.5 E continues below zero."""
    E = np.asarray(E, dtype=np.float64)
    hi = OETF_ALPHA * np.power(np.maximum(E, OETF_BETA), 0.45) - (OETF_ALPHA - 1.0)
    return np.where(E < OETF_BETA, 4.5 * E, hi)


def bt2020_oetf_inverse(Ep: np.ndarray) -> np.ndarray:
    Ep = np.asarray(Ep, dtype=np.float64)
    knee = 4.5 * OETF_BETA
    hi = np.power(np.maximum((Ep + OETF_ALPHA - 1.0) / OETF_ALPHA, 0.0), 1.0 / 0.45)
    return np.where(Ep < knee, Ep / 4.5, hi)


def ycbcr2020cl_from_linear(rgb2020: np.ndarray) -> np.ndarray:
    """Linear BT.2020 RGB (..., 3) -> constant-luminance Yc'Cbc'Crc'."""
    r, g, b = rgb2020[..., 0], rgb2020[..., 1], rgb2020[..., 2]
    yc = KR20 * r + KG20 * g + KB20 * b
    ycp, bp, rp = bt2020_oetf(yc), bt2020_oetf(b), bt2020_oetf(r)
    db, dr = bp - ycp, rp - ycp
    cb = np.where(db <= 0, db / CL_NB, db / CL_PB)
    cr = np.where(dr <= 0, dr / CL_NR, dr / CL_PR)
    return np.stack([ycp, cb, cr], axis=-1)


def ycbcr2020cl(rgbp: np.ndarray, gamma: float = 2.2) -> np.ndarray:
    """R'G'B' (..., 3) of BT.709 primaries -> BT.2020 constant-luminance
    Y'CbCr (..., 3)."""
    lin = np.power(rgbp, gamma)
    return ycbcr2020cl_from_linear(lin @ M_709_TO_2020.T)


def _signed_pow(v: np.ndarray, e: float) -> np.ndarray:
    return np.sign(v) * np.power(np.abs(v), e)


def ycbcr601_inverse(ycc: np.ndarray) -> np.ndarray:
    """BT.601 Y'CbCr (..., 3) -> R'G'B' (..., 3), solved from the definition."""
    y, cb, cr = ycc[..., 0], ycc[..., 1], ycc[..., 2]
    r = y + _CR_DIV * cr
    b = y + _CB_DIV * cb
    g = (y - _KR * r - _KB * b) / _KG
    return np.stack([r, g, b], axis=-1)


def ipt_inverse(ipt_: np.ndarray, gamma: float = 2.2) -> np.ndarray:
    """IPT (..., 3) -> R'G'B' (..., 3): the matrices inverted, the 0.43 power
    undone, the linearisation undone (signs kept)."""
    lmsp = ipt_ @ np.linalg.inv(M_LMS2IPT).T
    lms = _signed_pow(lmsp, 1.0 / IPT_EXPONENT)
    lin = lms @ np.linalg.inv(M_XYZ2LMS @ M_RGB2XYZ).T
    return _signed_pow(lin, 1.0 / gamma)


def ycbcr2020cl_inverse(ycc: np.ndarray, gamma: float = 2.2) -> np.ndarray:
    """Constant-luminance Y'CbCr (..., 3) -> R'G'B' (..., 3) of BT.709
    primaries: B' and R' from the chroma (divisor by its sign), linear Yc, B,
    R, then G from the luminance equation, then back to BT.709 primaries."""
    ycp, cb, cr = ycc[..., 0], ycc[..., 1], ycc[..., 2]
    bp = ycp + np.where(cb <= 0, CL_NB, CL_PB) * cb
    rp = ycp + np.where(cr <= 0, CL_NR, CL_PR) * cr
    yc, b, r = bt2020_oetf_inverse(ycp), bt2020_oetf_inverse(bp), bt2020_oetf_inverse(rp)
    g = (yc - KR20 * r - KB20 * b) / KG20
    lin = np.stack([r, g, b], axis=-1) @ np.linalg.inv(M_709_TO_2020).T
    return _signed_pow(lin, 1.0 / gamma)


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
    elif space == "ycbcr2020cl":
        conv = ycbcr2020cl(p, gamma)
    else:
        raise ValueError(f"unknown colour space {space!r}")
    # (K, s2, s1, 3) -> (s1, s2, 3, K)
    return np.ascontiguousarray(np.transpose(conv, (2, 1, 3, 0)))


def colour_invert(T: np.ndarray, space: str, gamma: float = 2.2) -> np.ndarray:
    """Tensor (s1, s2, 3, K) -> R'G'B' images (K, s2, s1, 3), FP64, the
    inverse of colour_convert before its 8-bit quantisation."""
    ycc = np.transpose(np.asarray(T, dtype=np.float64), (3, 1, 0, 2))
    if space == "ycbcr":
        return ycbcr601_inverse(ycc)
    if space == "ipt":
        return ipt_inverse(ycc, gamma)
    if space == "ycbcr2020cl":
        return ycbcr2020cl_inverse(ycc, gamma)
    raise ValueError(f"unknown colour space {space!r}")


def to_u8(rgbp: np.ndarray) -> np.ndarray:
    """R'G'B' -> 8 bits: clamp(rint(255 x), 0, 255), ties to even."""
    return np.clip(np.rint(255.0 * np.asarray(rgbp)), 0, 255).astype(np.uint8)


def psnr8(ref8: np.ndarray, out8: np.ndarray) -> float:
    """PSNR of 8-bit views over all their bytes, peak 255 (the quality
    measure of Figs. 3 and 4)."""
    d = np.asarray(ref8, dtype=np.float64) - np.asarray(out8, dtype=np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(255.0 ** 2 / mse)


def frobenius2(T: np.ndarray) -> float:
    """||T||_F^2, the squared norm used by the fit."""
    return float(np.sum(np.square(T, dtype=np.float64)))
