"""GB300 (sm_103a) Tucker-ALS library for multi-exposure stereo coding
(Sharma & Grover, arXiv 2104.04726, Section III).

Thin Python binding over the C ABI of `include/mes.h`: every function here
only marshals torch tensors (device memory) and the current CUDA stream into
the library call; all computation runs in the library's CUDA kernels.

Tensor conventions: the library stores tensors first-mode fastest.  A tensor
of paper dims (s_1, ..., s_N) is held in a C-contiguous torch tensor of shape
(s_N, ..., s_1); a factor S^(n) (s_n x r_n, column-major) is a C-contiguous
torch tensor of shape (r_n, s_n).  `paper_dims(t)` / `torch_shape(dims)`
convert between the two.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

from . import _lib

__all__ = ["colour_invert", "rate_bits", "rate_sweep", "colour_convert", "tucker_als", "reconstruct", "quantize_core", "dequantize_core",
           "version", "torch_shape", "paper_dims", "PRECISIONS", "SPACES", "MesError"]

MesError = _lib.MesError
PRECISIONS = {"fp32": 0, "bf16": 1, "tf32": 2}
SPACES = {"ycbcr": 0, "ipt": 1, "ycbcr2020cl": 2}
INITS = {"thosvd": 0, "interlaced": 1}


def _torch():
    import torch
    return torch


def version() -> str:
    return _lib.load().mes_version().decode()


def torch_shape(dims: Sequence[int]) -> tuple:
    return tuple(int(d) for d in reversed(list(dims)))


def paper_dims(t) -> tuple:
    return tuple(int(d) for d in reversed(list(t.shape)))


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _i64(vals):
    arr = (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])
    return arr


def _need(t, dtype, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")


def colour_convert(rgb8, space: str = "ycbcr", gamma: float = 2.2, out=None, norm2=None):
    """Colour pre-pass (Section III-A).  rgb8: uint8 CUDA tensor (K, s2, s1, 3).
    Returns (T, norm2): T float32 of torch shape (K, 3, s2, s1) = paper dims
    (s1, s2, 3, K); norm2 a float64 CUDA scalar tensor with ||T||_F^2."""
    torch = _torch()
    _need(rgb8, torch.uint8, "rgb8")
    K, s2, s1, c = rgb8.shape
    if c != 3:
        raise ValueError("rgb8 must have 3 channels")
    if out is None:
        out = torch.empty((K, 3, s2, s1), dtype=torch.float32, device=rgb8.device)
    if norm2 is None:
        norm2 = torch.empty((), dtype=torch.float64, device=rgb8.device)
    lib = _lib.load()
    st = lib.mes_colour_convert(_ptr(rgb8), s1, s2, K, SPACES[space], ctypes.c_float(gamma),
                                _ptr(out), _ptr(norm2), _stream())
    _lib.check(st, "mes_colour_convert")
    return out, norm2


def colour_invert(X, space: str = "ycbcr", gamma: float = 2.2, rgb8=None, rgbp=None, want_u8: bool = True,
                  want_float: bool = False, ref8=None):
    """Inverse colour transform: float32 CUDA tensor of torch shape
    (K, 3, s2, s1) (paper dims (s1, s2, 3, K)) -> images (K, s2, s1, 3):
    uint8 (clamp(rint(255 R'))) and/or float32 R'G'B'.  Returns (rgb8, rgbp),
    None for an output not asked for; with `ref8` (uint8 images of the same
    shape) returns (rgb8, rgbp, sse8), sse8 a float64 CUDA scalar with the
    exact sum of squared byte differences."""
    torch = _torch()
    _need(X, torch.float32, "X")
    K, c, s2, s1 = X.shape
    if c != 3:
        raise ValueError("X must have 3 channels")
    if want_u8 and rgb8 is None:
        rgb8 = torch.empty((K, s2, s1, 3), dtype=torch.uint8, device=X.device)
    if want_float and rgbp is None:
        rgbp = torch.empty((K, s2, s1, 3), dtype=torch.float32, device=X.device)
    sse8 = None
    if ref8 is not None:
        _need(ref8, torch.uint8, "ref8")
        if tuple(ref8.shape) != (K, s2, s1, 3):
            raise ValueError("ref8 must have shape (K, s2, s1, 3)")
        sse8 = torch.empty((), dtype=torch.float64, device=X.device)
    lib = _lib.load()
    st = lib.mes_colour_invert(_ptr(X), s1, s2, K, SPACES[space], ctypes.c_float(gamma), _ptr(rgb8),
                               _ptr(rgbp), _ptr(ref8), _ptr(sse8), _stream())
    _lib.check(st, "mes_colour_invert")
    return (rgb8, rgbp) if ref8 is None else (rgb8, rgbp, sse8)


def tucker_als(X, dims: Sequence[int], ranks: Sequence[int], max_iters: int = 20, tol: float = 0.0,
               precision: str = "fp32", init_iters: int = 0, inner_iters: int = 0, seed: int = 0,
               canonical: bool = True, init_factors=None, history: bool = False, outputs=None,
               init: str = "thosvd", reconstruction=None, wait_ns: int = 0, concurrency: int = 0):
    """Tucker-ALS / HOOI (Section III-B).  X: float32 CUDA tensor holding the
    first-mode-fastest tensor of paper dims `dims`.  Returns a dict with
    `core` (torch shape reversed(ranks)), `factors` (list of (r_n, s_n)
    tensors = column-major S^(n)), `fit` (float64 CUDA scalar), `iters`
    (int32 CUDA scalar) and, if history, `fit_history` (max_iters float64).
    init: "thosvd" (truncated HOSVD) or "interlaced" (interlaced HOSVD); a
    given `init_factors` overrides both.  reconstruction: optional float32
    CUDA tensor like X that receives T_hat (Eq. 1) from the fit's pass.
    `status` (int32 CUDA scalar) receives the device-side status (0, or
    MES_ERR_TIMEOUT / MES_ERR_NONFINITE, with a NaN fit); wait_ns bounds the
    tensor-core pipeline waits (0: the library default); concurrency: how
    many decompositions run side by side (split-K over a share of the SMs)."""
    torch = _torch()
    _need(X, torch.float32, "X")
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    N = len(dims)
    if len(ranks) != N:
        raise ValueError("dims and ranks differ in length")
    n_el = 1
    for d in dims:
        n_el *= d
    if X.numel() != n_el:
        raise ValueError("X does not hold prod(dims) elements")
    dev = X.device
    if outputs is None:
        core = torch.empty(torch_shape(ranks), dtype=torch.float32, device=dev)
        factors = [torch.empty((r, s), dtype=torch.float32, device=dev) for s, r in zip(dims, ranks)]
        fit = torch.empty((), dtype=torch.float64, device=dev)
        iters = torch.zeros((), dtype=torch.int32, device=dev)
        hist = torch.full((max_iters,), float("nan"), dtype=torch.float64, device=dev) if history else None
    else:
        core, factors, fit, iters, hist = outputs
    status = torch.zeros((), dtype=torch.int32, device=dev)
    fac_arr = (ctypes.c_void_p * N)(*[f.data_ptr() for f in factors])
    opts = _lib.MesAlsOpts()
    opts.precision = PRECISIONS[precision]
    opts.init_iters = int(init_iters)
    opts.inner_iters = int(inner_iters)
    opts.seed = int(seed)
    opts.canonical = 0 if canonical else -1
    opts.init = INITS[init]
    if reconstruction is not None:
        _need(reconstruction, torch.float32, "reconstruction")
        if reconstruction.numel() != n_el:
            raise ValueError("reconstruction does not hold prod(dims) elements")
        opts.reconstruction = reconstruction.data_ptr()
    opts.iters_done = iters.data_ptr()
    opts.fit_history = hist.data_ptr() if hist is not None else None
    opts.status = status.data_ptr()
    opts.wait_ns = int(wait_ns)
    opts.concurrency = int(concurrency)
    keep = None
    if init_factors is not None:
        keep = (ctypes.c_void_p * N)(*[f.data_ptr() for f in init_factors])
        opts.init_factors = ctypes.cast(keep, ctypes.POINTER(ctypes.c_void_p))
    lib = _lib.load()
    st = lib.mes_tucker_als(_ptr(X), N, _i64(dims), _i64(ranks), int(max_iters), float(tol), _ptr(core),
                            fac_arr, _ptr(fit), ctypes.byref(opts), _stream())
    _lib.check(st, "mes_tucker_als")
    out = {"core": core, "factors": factors, "fit": fit, "iters": iters, "status": status}
    if hist is not None:
        out["fit_history"] = hist
    return out


def tucker_als_workspace_size(dims: Sequence[int], ranks: Sequence[int], precision: str = "fp32") -> int:
    """Bytes of device workspace mes_tucker_als takes for this shape (no
    device access)."""
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    opts = _lib.MesAlsOpts()
    opts.precision = PRECISIONS[precision]
    n = ctypes.c_size_t(0)
    lib = _lib.load()
    _lib.check(lib.mes_tucker_als_workspace_size(len(dims), _i64(dims), _i64(ranks), ctypes.byref(opts),
                                                 ctypes.byref(n)), "mes_tucker_als_workspace_size")
    return int(n.value)


def reconstruct(core, factors, dims: Sequence[int], ranks: Sequence[int], out=None, ref=None,
                precision: str = "fp32"):
    """T_hat = Q x_1 S^(1) ... x_N S^(N) (Eq. 1).  With `ref`, also returns
    sum((ref - T_hat)^2) as a float64 CUDA scalar (fused).  precision "fp32":
    CUDA cores; "tf32"/"bf16": tensor cores with the three-term TF32 split
    (FP32-level accuracy)."""
    torch = _torch()
    _need(core, torch.float32, "core")
    N = len(dims)
    if out is None:
        out = torch.empty(torch_shape(dims), dtype=torch.float32, device=core.device)
    sse = torch.empty((), dtype=torch.float64, device=core.device) if ref is not None else None
    fac_arr = (ctypes.c_void_p * N)(*[f.data_ptr() for f in factors])
    lib = _lib.load()
    st = lib.mes_reconstruct(_ptr(core), fac_arr, N, _i64(dims), _i64(ranks), _ptr(out), _ptr(ref),
                             _ptr(sse), PRECISIONS[precision], _stream())
    _lib.check(st, "mes_reconstruct")
    return (out, sse) if ref is not None else out


def quantize_core(core, ranks: Sequence[int], bits: int = 16, check_finite: bool = False):
    """Per-plane quantiser of the core.  Returns (q int16 like core, scales
    float32 of prod(ranks[2:]) entries)."""
    torch = _torch()
    _need(core, torch.float32, "core")
    P = 1
    for r in ranks[2:]:
        P *= int(r)
    q = torch.empty(core.shape, dtype=torch.int16, device=core.device)
    scales = torch.empty((P,), dtype=torch.float32, device=core.device)
    lib = _lib.load()
    st = lib.mes_quantize_core(_ptr(core), len(ranks), _i64(ranks), int(bits), _ptr(q), _ptr(scales),
                               1 if check_finite else 0, _stream())
    _lib.check(st, "mes_quantize_core")
    return q, scales


def dequantize_core(q, scales, ranks: Sequence[int]):
    torch = _torch()
    core = torch.empty(q.shape, dtype=torch.float32, device=q.device)
    lib = _lib.load()
    st = lib.mes_dequantize_core(_ptr(q), _ptr(scales), len(ranks), _i64(ranks), _ptr(core), _stream())
    _lib.check(st, "mes_dequantize_core")
    return core



def rate_bits(dims: Sequence[int], ranks: Sequence[int], bits: int = 0, factor_bits: int = 16) -> int:
    """Bits of the coded representation before entropy coding: the core at
    `bits` per entry (0: FP32) plus one FP32 scale per quantiser plane, and
    the factors at `factor_bits` per entry.  The paper codes the rank and
    the quantisation of the core as the rate knob (abstract, Section I) but
    fixes no format; this is the count a fixed-length code would take."""
    n_core = 1
    for r in ranks:
        n_core *= int(r)
    planes = 1
    for r in ranks[2:]:
        planes *= int(r)
    core = n_core * (bits if bits else 32) + (planes * 32 if bits else 0)
    return core + sum(int(d) * int(r) for d, r in zip(dims, ranks)) * factor_bits


def rate_sweep(rgb8, space: str, rank_grid, bits_grid, max_iters: int = 20, tol: float = 0.0,
               precision: str = "fp32", gamma: float = 2.2, factor_bits: int = 16, **als_opts):
    """Rate-distortion sweep over core ranks x quantiser bits (the in-scope
    half of Figs. 3 and 4): one decomposition per rank tuple, then per bit
    depth quantise -> dequantise -> reconstruct -> inverse colour -> PSNR of
    the 8-bit views against the input.  rgb8: uint8 CUDA tensor (K, s2, s1,
    3); bits 0 keeps the FP32 core.  Returns a list of dicts with ranks,
    bits, bpp (rate_bits per pixel of the stack), psnr (dB, over all bytes)
    and fit (of the unquantised decomposition).  Further keyword arguments
    go to tucker_als."""
    import math
    K, s2, s1, _ = rgb8.shape
    dims = [s1, s2, 3, K]
    X, _ = colour_convert(rgb8, space, gamma)
    n_bytes = s1 * s2 * K * 3
    rows = []
    for ranks in rank_grid:
        ranks = [int(r) for r in ranks]
        res = tucker_als(X, dims, ranks, max_iters=max_iters, tol=tol, precision=precision, **als_opts)
        fit = float(res["fit"].cpu())
        for bits in bits_grid:
            core = res["core"]
            if bits:
                q, sc = quantize_core(core, ranks, bits)
                core = dequantize_core(q, sc, ranks)
            Xh = reconstruct(core, res["factors"], dims, ranks, precision=precision)
            _, _, sse8 = colour_invert(Xh, space, gamma, want_u8=False, ref8=rgb8)
            sse = float(sse8.cpu())
            psnr = math.inf if sse == 0.0 else 10.0 * math.log10(255.0 ** 2 * n_bytes / sse)
            rows.append({"ranks": ranks, "bits": int(bits), "psnr": psnr, "fit": fit,
                         "bpp": rate_bits(dims, ranks, bits, factor_bits) / (s1 * s2 * K)})
    return rows

class Problem:
    """One stack for the batched and served forms: device buffers for the
    input (8-bit images or the FP32 tensor) and every output, and the
    `mes_problem` descriptor pointing at them.  Keep the object alive until
    its work has completed."""

    def __init__(self, dims: Sequence[int], ranks: Sequence[int], X=None, rgb8=None, space: str = "ipt",
                 gamma: float = 2.2, max_iters: int = 20, tol: float = 0.0, precision: str = "fp32",
                 quant_bits: int = 0, device=None, wait_ns: int = 0, concurrency: int = 0):
        torch = _torch()
        dims = [int(d) for d in dims]
        ranks = [int(r) for r in ranks]
        N = len(dims)
        if len(ranks) != N or not 2 <= N <= 8:
            raise ValueError("dims and ranks must have the same length, 2..8")
        src = rgb8 if rgb8 is not None else X
        dev = device if device is not None else (src.device if src is not None else torch.device("cuda"))
        if rgb8 is not None:
            _need(rgb8, torch.uint8, "rgb8")
            if N != 4 or dims[2] != 3 or tuple(rgb8.shape) != (dims[3], dims[1], dims[0], 3):
                raise ValueError("rgb8 must be (K, s2, s1, 3) for dims (s1, s2, 3, K)")
            X = torch.empty(torch_shape(dims), dtype=torch.float32, device=dev) if X is None else X
        if X is None:
            raise ValueError("give X or rgb8")
        _need(X, torch.float32, "X")
        self.dims, self.ranks, self.rgb8, self.X = dims, ranks, rgb8, X
        self.core = torch.empty(torch_shape(ranks), dtype=torch.float32, device=dev)
        self.factors = [torch.empty((r, s), dtype=torch.float32, device=dev) for s, r in zip(dims, ranks)]
        self.fit = torch.empty((), dtype=torch.float64, device=dev)
        self.iters = torch.zeros((), dtype=torch.int32, device=dev)
        self.status = torch.zeros((), dtype=torch.int32, device=dev)   # device-side status of the decomposition
        P = 1
        for r in ranks[2:]:
            P *= r
        self.q = torch.empty(torch_shape(ranks), dtype=torch.int16, device=dev) if quant_bits else None
        self.scales = torch.empty((P,), dtype=torch.float32, device=dev) if quant_bits else None
        p = _lib.MesProblem()
        p.rgb8 = _ptr(rgb8)
        p.space = SPACES[space]
        p.gamma = float(gamma)
        p.X = _ptr(X)
        p.N = N
        for n in range(N):
            p.dims[n] = dims[n]
            p.ranks[n] = ranks[n]
            p.factors[n] = self.factors[n].data_ptr()
        p.max_iters = int(max_iters)
        p.tol = float(tol)
        p.opts.precision = PRECISIONS[precision]
        p.opts.iters_done = self.iters.data_ptr()
        p.opts.status = self.status.data_ptr()
        p.opts.wait_ns = int(wait_ns)
        p.opts.concurrency = int(concurrency)   # 0: the batch's streams / the server's slots
        p.core = _ptr(self.core)
        p.fit = _ptr(self.fit)
        p.quant_bits = int(quant_bits)
        p.q = _ptr(self.q)
        p.scales = _ptr(self.scales)
        self.struct = p


def _problem_array(problems):
    arr = (_lib.MesProblem * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = p.struct
    return arr


class Batch:
    """Batched form: `run` deals the problems to `max_streams` internal streams
    (longest first, balanced), forked from and joined back into the current
    stream; `capture` records the same enqueue as one CUDA graph that
    `launch` replays."""

    def __init__(self, max_streams: int = 8):
        self._lib = _lib.load()
        self._h = ctypes.c_void_p()
        _lib.check(self._lib.mes_batch_create(int(max_streams), ctypes.byref(self._h)), "mes_batch_create")
        self._keep = None

    def run(self, problems):
        arr = _problem_array(problems)
        sts = (ctypes.c_int * len(problems))()
        _lib.check(self._lib.mes_batch_run(self._h, arr, len(problems), sts, _stream()), "mes_batch_run")

    def capture(self, problems, stream=None):
        torch = _torch()
        arr = _problem_array(problems)
        self._keep = (arr, list(problems))
        st = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(self._lib.mes_batch_capture(self._h, arr, len(problems), ctypes.c_void_p(st.cuda_stream)),
                   "mes_batch_capture")

    def launch(self):
        _lib.check(self._lib.mes_batch_launch(self._h, _stream()), "mes_batch_launch")

    def close(self):
        if self._h:
            self._lib.mes_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving form: a request loop admitting problems into `max_slots` slots
    under a device-memory budget (continuous batching).  `submit` returns a
    ticket; `wait`/`poll` give (status, latency in ms)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 8):
        self._lib = _lib.load()
        self._h = ctypes.c_void_p()
        _lib.check(self._lib.mes_serve_create(ctypes.c_size_t(int(hbm_budget_bytes)), int(max_slots),
                                              ctypes.byref(self._h)), "mes_serve_create")
        self._live = {}

    def submit(self, problem: Problem) -> int:
        t = ctypes.c_uint64()
        _lib.check(self._lib.mes_serve_submit(self._h, ctypes.byref(problem.struct), ctypes.byref(t)),
                   "mes_serve_submit")
        self._live[t.value] = problem
        return t.value

    def poll(self, ticket: int):
        done, res, lat = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _lib.check(self._lib.mes_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(res),
                                            ctypes.byref(lat)), "mes_serve_poll")
        if not done.value:
            return None
        self._live.pop(ticket, None)
        return res.value, lat.value

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        res, lat = ctypes.c_int(), ctypes.c_double()
        _lib.check(self._lib.mes_serve_wait(self._h, ctypes.c_uint64(ticket), float(timeout_ms), ctypes.byref(res),
                                            ctypes.byref(lat)), "mes_serve_wait")
        self._live.pop(ticket, None)
        return res.value, lat.value

    def stats(self) -> dict:
        s = _lib.MesServeStats()
        _lib.check(self._lib.mes_serve_get_stats(self._h, ctypes.byref(s)), "mes_serve_get_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if self._h:
            self._lib.mes_serve_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
