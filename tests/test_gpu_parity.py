"""GPU path vs the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances (FP32 path): relative fit agreement <= 1e-5; factor subspaces
compared as projectors (sign and rotation are not unique) where the relative
eigengap allows; orthonormality <= 2e-6; the core quantiser bit-exact on
identical FP32 input.

When the gap allows: the FP32 operator carries a perturbation of about
u * l_1 (u = 2^-24 ~ 6e-8) and the subspace of the r leading eigenvectors
moves by sin(theta) <~ u * l_1 / (l_r - l_{r+1}) (Davis-Kahan), so a 1e-3
gate on sin(theta) is meaningful only when (l_r - l_{r+1}) / l_1 > 1e-4.
Smaller gaps are reported, not gated.
"""
GAP_GATE = 1e-4
import numpy as np
import pytest

import synth
from oracle import colour, quant, tucker

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2104_04726_gb300 as m
    return m


DEV = "cuda:0"


def to_paper(t):
    """torch (s_N, ..., s_1) C-order -> numpy (s_1, ..., s_N) FP64."""
    a = t.detach().cpu().numpy().astype(np.float64)
    return a.transpose(tuple(range(a.ndim))[::-1])


def to_torch(a, dtype=torch.float32):
    a = np.asarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.transpose(tuple(range(a.ndim))[::-1]))).to(dtype).to(DEV)


def factors_np(res):
    return [f.detach().cpu().numpy().T.astype(np.float64) for f in res["factors"]]


def gap_and_sin(T, ref_factors, n, U_gpu):
    """Relative eigengap of the mode-n Gram at the oracle's solution and the
    largest principal-angle sine between the GPU and oracle subspaces."""
    Y = tucker.multi_mode_product(T, ref_factors, skip=n, transpose=True)
    w = np.sort(np.linalg.eigvalsh(tucker.gram(tucker.unfold(Y, n))))[::-1]
    r = ref_factors[n].shape[1]
    gap = (w[r - 1] - w[r]) / w[0] if r < len(w) else 1.0
    Uo = ref_factors[n]
    s = np.linalg.svd(Uo.T @ U_gpu, compute_uv=False)
    sin_max = float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))
    return gap, sin_max


def contained_sin(T, ref_factors, n, U_gpu, gap_gate=GAP_GATE):
    """For a large mode whose full rank-r split has no usable gap: the
    leading k eigenvectors of the mode-n Gram at the oracle's solution, for
    the largest k with (l_k - l_{r+1}) / l_1 > gap_gate, must lie in the GPU's
    r-dimensional subspace.  Davis-Kahan on the split (k | beyond r) bounds
    how far an FP32 operator can move them: sin <~ u l_1 / (l_k - l_{r+1}).
    Returns (k, largest sine between span(V_k) and span(U_gpu))."""
    Y = tucker.multi_mode_product(T, ref_factors, skip=n, transpose=True)
    w, V = np.linalg.eigh(tucker.gram(tucker.unfold(Y, n)))
    w, V = w[::-1], V[:, ::-1]
    r = ref_factors[n].shape[1]
    lr1 = w[r] if r < len(w) else 0.0
    k = int(np.sum((w[:r] - lr1) / w[0] > gap_gate))
    if k == 0:
        return 0, 0.0
    Vk = V[:, :k]
    resid = Vk - U_gpu @ (U_gpu.T @ Vk)
    return k, float(np.linalg.norm(resid, 2))


# ---------------------------------------------------------------- colour
@pytest.mark.parametrize("space,tol", [("ycbcr", 2e-7), ("ipt", 2e-6), ("ycbcr2020cl", 1e-6)])
@pytest.mark.parametrize("shape", [(64, 48, 6), (37, 23, 3), (8, 1, 1)])
def test_colour_matches_oracle(mes, space, tol, shape):
    s1, s2, K = shape
    rng = np.random.default_rng(s1 * 7 + K)
    img = rng.integers(0, 256, size=(K, s2, s1, 3), dtype=np.uint8)
    img[0, 0, 0] = (255, 255, 255)
    img[-1, -1, -1] = (0, 0, 0)
    X, n2 = mes.colour_convert(torch.from_numpy(img).to(DEV), space)
    torch.cuda.synchronize()
    want = colour.colour_convert(img, space)
    got = to_paper(X)
    assert got.shape == want.shape
    assert np.abs(got - want).max() < tol
    assert abs(float(n2.cpu()) - colour.frobenius2(want)) <= 1e-5 * colour.frobenius2(want)


@pytest.mark.parametrize("space", ["ycbcr", "ipt", "ycbcr2020cl"])
@pytest.mark.parametrize("shape", [(64, 48, 6), (37, 23, 3), (7, 1, 2)])
def test_colour_invert_matches_oracle(mes, space, shape):
    """Inverse transform of a perturbed tensor (as a reconstruction gives:
    noise of 0.02 takes some pixels out of gamut) against the oracle's FP64
    inverse of the same FP32 input.  R'G'B' within 2e-5 where R' > 0.05; near
    black the power 1/gamma magnifies FP32 round-off, so there the linear
    values (R')^gamma are compared, within 1e-6.  Bytes: equal, except within
    0.2 of a rounding boundary or below 0.06, where they may differ by one."""
    s1, s2, K = shape
    rng = np.random.default_rng(s1 * 13 + K)
    img = rng.integers(0, 256, size=(K, s2, s1, 3), dtype=np.uint8)
    T = colour.colour_convert(img, space) + 0.02 * rng.standard_normal((s1, s2, 3, K))
    T32 = T.astype(np.float32)
    u8, fp = mes.colour_invert(to_torch(T32), space, want_float=True)
    torch.cuda.synchronize()
    want = colour.colour_invert(T32.astype(np.float64), space)
    got = fp.cpu().numpy().astype(np.float64)
    big = np.abs(want) > 0.05
    assert np.abs(got - want)[big].max() < 2e-5
    lin = lambda v: np.sign(v) * np.abs(v) ** 2.2 if space != "ycbcr" else v
    assert np.abs(lin(got) - lin(want))[~big].max(initial=0.0) < 1e-6
    gb, wb = u8.cpu().numpy().astype(int), colour.to_u8(want).astype(int)
    x = np.clip(255.0 * want, 0, 255)
    near = (np.abs(x - np.floor(x) - 0.5) < 0.2) | (want < 0.06)
    assert np.array_equal(gb[~near], wb[~near])
    assert np.abs(gb - wb).max() <= 1


@pytest.mark.parametrize("space", ["ycbcr", "ipt", "ycbcr2020cl"])
@pytest.mark.parametrize("shape", [(64, 48, 6), (37, 23, 3)])
def test_colour_round_trip_recovers_the_bytes(mes, space, shape):
    s1, s2, K = shape
    rng = np.random.default_rng(s2 * 5 + K)
    img = rng.integers(0, 256, size=(K, s2, s1, 3), dtype=np.uint8)
    img[0, 0, :3] = [[0, 0, 0], [255, 255, 255], [0, 0, 255]]
    t = torch.from_numpy(img).to(DEV)
    X, _ = mes.colour_convert(t, space)
    back, _ = mes.colour_invert(X, space)
    torch.cuda.synchronize()
    assert torch.equal(back, t)


def test_colour_norm_is_reproducible(mes):
    img = synth.make_stack(synth.SceneSpec(96, 40, (0.5, 2.0)), 3)
    t = torch.from_numpy(img).to(DEV)
    a = [float(mes.colour_convert(t, "ipt")[1].cpu()) for _ in range(3)]
    assert a[0] == a[1] == a[2]


# ---------------------------------------------------------------- quantiser
def _gpu_quant(mes, core_np, ranks, bits):
    q, s = mes.quantize_core(to_torch(core_np), ranks, bits)
    torch.cuda.synchronize()
    return to_paper(q).astype(np.int64), s.cpu().numpy()


@pytest.mark.parametrize("ranks", [(16, 12, 3, 6), (5, 3, 2, 3), (7, 1), (33, 17, 1, 2)])
@pytest.mark.parametrize("bits", [2, 5, 8, 16])
def test_quantiser_bit_exact(mes, ranks, bits):
    rng = np.random.default_rng(sum(ranks) * bits)
    core = (rng.standard_normal(ranks) * 10.0 ** rng.integers(-3, 4)).astype(np.float32)
    planes = quant.planes_of(core)
    if planes.shape[0] > 1:
        core_view = core.reshape(ranks[0], ranks[1] if len(ranks) > 1 else 1, -1, order="F")
        core_view[..., 1] = 0.0          # an all-zero plane
        core = core_view.reshape(ranks, order="F")
        planes = quant.planes_of(core)
    q_ref, s_ref = quant.quantize_planes(planes, bits)
    q_gpu, s_gpu = _gpu_quant(mes, core, ranks, bits)
    assert np.array_equal(s_gpu, s_ref)
    got_planes = quant.planes_of(q_gpu.astype(np.float32))
    assert np.array_equal(got_planes.astype(np.int64), q_ref.astype(np.int64))


def test_quantiser_ties_and_dequantise(mes):
    # exact .5 ties after the division, in a 2-plane core
    core = np.zeros((4, 2, 2), np.float32)
    core[:, :, 0] = [[3.0, 1.5], [-0.5, 2.5], [0.0, -1.5], [-3.0, 0.25]]
    core[:, :, 1] = 7.0
    q, s = mes.quantize_core(to_torch(core), (4, 2, 2), 3)
    back = mes.dequantize_core(q, s, (4, 2, 2))
    torch.cuda.synchronize()
    qn = to_paper(q)
    assert qn[:, :, 0].tolist() == [[3, 2], [0, 2], [0, -2], [-3, 0]]
    assert np.all(qn[:, :, 1] == 3)
    assert np.allclose(to_paper(back)[:, :, 1], 7.0)


def test_quantiser_reports_nonfinite(mes):
    core = np.ones((4, 4, 2), np.float32)
    core[1, 2, 1] = np.nan
    with pytest.raises(mes.MesError) as e:
        mes.quantize_core(to_torch(core), (4, 4, 2), 8, check_finite=True)
    assert e.value.name == "MES_ERR_NONFINITE"


# ---------------------------------------------------------------- Tucker-ALS
def _scene(name):
    cfg = synth.config_spec(name)
    img = synth.make_stack(cfg["spec"], synth.seed_for(name))
    return cfg, img


def _run(mes, T, ranks, iters, tol, **kw):
    res = mes.tucker_als(to_torch(T), T.shape, ranks, max_iters=iters, tol=tol, history=True, **kw)
    torch.cuda.synchronize()
    return res


def test_small_scene_parity(mes):
    cfg, img = _scene("small_64x48")
    X, _ = mes.colour_convert(torch.from_numpy(img).to(DEV), cfg["space"])
    dims = (cfg["spec"].s1, cfg["spec"].s2, 3, cfg["spec"].K)
    res = mes.tucker_als(X, dims, cfg["ranks"], max_iters=cfg["iters"], tol=cfg["tol"], inner_iters=4,
                         history=True)
    torch.cuda.synchronize()
    T = colour.colour_convert(img, cfg["space"])
    ref = tucker.hooi(T, cfg["ranks"], cfg["iters"], cfg["tol"])
    fit = float(res["fit"].cpu())
    assert abs(fit - ref.fit) / ref.fit < 1e-5, (fit, ref.fit)
    Us = factors_np(res)
    for n, U in enumerate(Us):
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 2e-6
        gap, sin_max = gap_and_sin(T, ref.factors, n, U)
        print(f"mode {n}: relative gap {gap:.2e}, sin(theta) {sin_max:.2e}")
        if gap > GAP_GATE:
            assert sin_max < 1e-3, (n, gap, sin_max)
    # the returned fit is the fit of the returned decomposition
    core = to_paper(res["core"])
    Xr = tucker.reconstruct(core, Us)
    assert abs((1 - tucker.relative_error(T, Xr)) - fit) < 1e-6


def test_ragged_shape_truncated_small_modes(mes):
    rng = np.random.default_rng(21)
    spec = synth.SceneSpec(17, 13, (0.5, 1.0, 2.0, 4.0, 8.0), views=1, d_max=2)
    img = synth.make_stack(spec, 4)
    T = colour.colour_convert(img, "ipt")           # 17 x 13 x 3 x 5
    ranks = (5, 4, 2, 3)
    ref = tucker.hooi(T, ranks, 15, 0.0)
    res = _run(mes, T, ranks, 15, 0.0, inner_iters=4)
    fit = float(res["fit"].cpu())
    assert abs(fit - ref.fit) / ref.fit < 1e-5, (fit, ref.fit)
    Us = factors_np(res)
    for n in range(4):
        gap, sin_max = gap_and_sin(T, ref.factors, n, Us[n])
        if gap > GAP_GATE:
            assert sin_max < 1e-3, (n, gap, sin_max)


def test_bf16_on_unaligned_rows_runs_the_tf32_form(mes):
    """BF16 rows must start on 16-byte boundaries for TMA, so image modes
    that are not multiples of 8 take the TF32 form: the same decomposition
    as asking for TF32, bit for bit, and within the TF32 tolerance of the
    oracle."""
    spec = synth.SceneSpec(100, 75, (0.5, 2.0), views=2, d_max=4)
    img = synth.make_stack(spec, 33)
    T = colour.colour_convert(img, "ipt")           # 100 x 75 x 3 x 4
    ranks = (24, 18, 3, 4)
    a = _run(mes, T, ranks, 10, 0.0, precision="bf16")
    b = _run(mes, T, ranks, 10, 0.0, precision="tf32")
    assert torch.equal(a["core"], b["core"])
    assert all(torch.equal(x, y) for x, y in zip(a["factors"], b["factors"]))
    ref = tucker.hooi(T, ranks, 10, 0.0)
    fit = float(a["fit"].cpu())
    assert abs(fit - ref.fit) / ref.fit < 1e-4, (fit, ref.fit)


def test_mid_ranks_not_multiple_of_32(mes):
    # ranks 150 and 140 (> 128, not multiples of the 32-column blocks of the
    # cluster Cholesky and the blocked triangular solve) on a 400 x 300 scene
    spec = synth.SceneSpec(400, 300, (0.5, 2.0), views=2, d_max=8)
    img = synth.make_stack(spec, 77)
    T = colour.colour_convert(img, "ipt")           # 400 x 300 x 3 x 4
    ranks = (150, 140, 3, 4)
    ref = tucker.hooi(T, ranks, 12, 0.0)
    for prec in ("fp32", "tf32"):
        res = _run(mes, T, ranks, 12, 0.0, precision=prec)
        fit = float(res["fit"].cpu())
        tol = 1e-5 if prec == "fp32" else 1e-4
        assert abs(fit - ref.fit) / ref.fit < tol, (prec, fit, ref.fit)
        for n, U in enumerate(factors_np(res)):
            assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 2e-6, (prec, n)


def test_rank_above_512_cluster_factorization(mes):
    # r_1 = 520 takes the Cholesky kernel that works through L2 across a
    # cluster (ranks above 512, e.g. 768 for 3840x2160 stacks); 600 x 200 scene
    spec = synth.SceneSpec(600, 200, (0.5, 2.0), views=1, d_max=4)
    img = synth.make_stack(spec, 91)
    T = colour.colour_convert(img, "ycbcr")           # 600 x 200 x 3 x 2
    ranks = (520, 100, 3, 2)
    ref = tucker.hooi(T, ranks, 10, 0.0)
    for prec in ("fp32", "tf32"):
        # 520 of 600 directions: the relative eigengap at r_1 is ~1e-7, so the
        # subspace iteration gets 4 steps per update to keep up with the
        # oracle's exact eigenvectors
        res = _run(mes, T, ranks, 10, 0.0, precision=prec, inner_iters=4)
        fit = float(res["fit"].cpu())
        tol = 1e-5 if prec == "fp32" else 1e-4
        print(f"r1=520 {prec}: fit {fit:.9f} oracle {ref.fit:.9f}")
        assert abs(fit - ref.fit) / ref.fit < tol, (prec, fit, ref.fit)
        for U in factors_np(res):
            assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 5e-6, prec


def test_full_multilinear_rank_is_exact(mes):
    rng = np.random.default_rng(5)
    T = rng.standard_normal((40, 24, 3, 4))
    res = _run(mes, T, T.shape, 3, 0.0)
    fit = float(res["fit"].cpu())
    assert fit > 1 - 1e-5
    Xr = tucker.reconstruct(to_paper(res["core"]), factors_np(res))
    assert tucker.relative_error(T, Xr) < 1e-5


def test_eckart_young_order2(mes):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((300, 40)) @ np.diag(np.logspace(0, -2, 40)) @ rng.standard_normal((40, 170))
    r = 12
    # the gap sigma_12 / sigma_13 is only ~1.12: give the subspace iteration
    # enough steps to reach the optimum to 1e-5
    res = _run(mes, A, (r, r), 10, 0.0, inner_iters=4, init_iters=4)
    s = np.linalg.svd(A, compute_uv=False)
    fit_ey = 1.0 - np.sqrt(np.sum(s[r:] ** 2)) / np.linalg.norm(A)
    assert abs(float(res["fit"].cpu()) - fit_ey) / fit_ey < 1e-5


def test_planted_low_rank(mes):
    rng = np.random.default_rng(9)
    shape, ranks = (130, 70, 3, 6), (9, 7, 2, 4)
    G = rng.standard_normal(ranks)
    Qs = [np.linalg.qr(rng.standard_normal((s, r)))[0] for s, r in zip(shape, ranks)]
    T = tucker.reconstruct(G, Qs)
    res = _run(mes, T, ranks, 4, 0.0)
    assert float(res["fit"].cpu()) > 1 - 2e-5
    for U, Q in zip(factors_np(res), Qs):
        assert np.abs(U @ U.T - Q @ Q.T).max() < 1e-4


def test_stopping_rule_and_history(mes):
    cfg, img = _scene("small_64x48")
    T = colour.colour_convert(img, cfg["space"])
    res = _run(mes, T, cfg["ranks"], 10, 1.0)
    assert int(res["iters"].cpu()) == 2
    h = res["fit_history"].cpu().numpy()
    assert np.isfinite(h[:2]).all() and np.isnan(h[2:]).all()
    res = _run(mes, T, cfg["ranks"], 1, 1.0)
    assert int(res["iters"].cpu()) == 1


def test_deterministic(mes):
    cfg, img = _scene("small_64x48")
    T = colour.colour_convert(img, cfg["space"])
    a = _run(mes, T, cfg["ranks"], 4, 0.0)
    b = _run(mes, T, cfg["ranks"], 4, 0.0)
    assert torch.equal(a["core"], b["core"])
    assert all(torch.equal(x, y) for x, y in zip(a["factors"], b["factors"]))
    assert float(a["fit"].cpu()) == float(b["fit"].cpu())


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fixed_sweeps_without_history_are_the_same(mes, prec):
    """With tol = 0, no history and full-rank small modes the per-sweep core
    and fit are formed in the last sweep only: nothing else reads them, so
    the result must equal, bit for bit, the run that forms them every sweep
    (asked for by the history)."""
    cfg, img = _scene("small_64x48")
    T = colour.colour_convert(img, cfg["space"])
    X = to_torch(T)
    a = mes.tucker_als(X, T.shape, cfg["ranks"], max_iters=5, tol=0.0, precision=prec, history=False)
    b = mes.tucker_als(X, T.shape, cfg["ranks"], max_iters=5, tol=0.0, precision=prec, history=True)
    torch.cuda.synchronize()
    assert int(a["iters"].cpu()) == 5 and int(b["iters"].cpu()) == 5
    assert torch.equal(a["core"], b["core"])
    assert all(torch.equal(x, y) for x, y in zip(a["factors"], b["factors"]))
    assert float(a["fit"].cpu()) == float(b["fit"].cpu())
    h = b["fit_history"].cpu().numpy()
    assert np.isfinite(h).all() and np.all(np.diff(h) > -1e-6)


def test_warm_start_from_oracle_factors(mes):
    cfg, img = _scene("small_64x48")
    T = colour.colour_convert(img, cfg["space"])
    ref = tucker.hooi(T, cfg["ranks"], 10, 0.0)
    init = [torch.from_numpy(np.ascontiguousarray(U.T)).float().to(DEV) for U in ref.factors]
    res = _run(mes, T, cfg["ranks"], 1, 0.0, init_factors=init, inner_iters=4)
    assert float(res["fit"].cpu()) > ref.fit - 2e-6


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_reconstruct_matches_oracle(mes, prec):
    # fp32: CUDA cores; tf32: tensor cores with the three-term TF32 split of
    # every operand (~3 * 2^-22 relative per product, FP32-level accuracy)
    cfg, img = _scene("small_64x48")
    T = colour.colour_convert(img, cfg["space"])
    res = _run(mes, T, cfg["ranks"], 3, 0.0)
    dims, ranks = T.shape, cfg["ranks"]
    Xh, sse = mes.reconstruct(res["core"], res["factors"], dims, ranks, ref=to_torch(T), precision=prec)
    torch.cuda.synchronize()
    core, Us = to_paper(res["core"]), factors_np(res)
    want = tucker.reconstruct(core, Us)
    assert np.abs(to_paper(Xh) - want).max() < 2e-6 * np.abs(want).max() * 10
    assert abs(float(sse.cpu()) - np.sum((T - want) ** 2)) < 1e-3 * np.sum((T - want) ** 2)
    # energy identity of the GPU decomposition: ||T||^2 - ||Q||^2 = ||T - T_hat||^2
    # (FP32 core: ||Q||^2 carries ~1e-7 relative error, i.e. ~0.2% of the residual here)
    lhs = np.sum(T ** 2) - np.sum(core ** 2)
    assert abs(lhs - float(sse.cpu())) < 0.01 * float(sse.cpu())


def test_canonical_small_rank_matches_oracle_columns(mes):
    # With r <= 128 the basis is rotated to the eigenvectors of the core's
    # mode-n Gram and sign-fixed, like the oracle's; columns agree where the
    # eigenvalues are well separated.
    rng = np.random.default_rng(31)
    shape, ranks = (60, 50, 3, 4), (6, 5, 3, 4)
    G = rng.standard_normal(ranks) * np.logspace(1, -1, 6)[:, None, None, None]
    Qs = [np.linalg.qr(rng.standard_normal((s, r)))[0] for s, r in zip(shape, ranks)]
    T = tucker.reconstruct(G, Qs) + 1e-3 * rng.standard_normal(shape)
    ref = tucker.hooi(T, ranks, 10, 0.0)
    res = _run(mes, T, ranks, 10, 0.0, inner_iters=3)
    for n in range(2):
        U = factors_np(res)[n]
        assert np.abs(U - ref.factors[n]).max() < 1e-3, n


@pytest.mark.slow
def test_xga_scene_parity(mes):
    # 1024x768x3x6, IPT, ranks (256, 192, 3, 6), 20 sweeps, default options
    cfg, img = _scene("xga_1024x768")
    X, n2 = mes.colour_convert(torch.from_numpy(img).to(DEV), cfg["space"])
    spec = cfg["spec"]
    dims = (spec.s1, spec.s2, 3, spec.K)
    res = mes.tucker_als(X, dims, cfg["ranks"], max_iters=cfg["iters"], tol=cfg["tol"])
    torch.cuda.synchronize()
    T = colour.colour_convert(img, cfg["space"])
    ref = tucker.hooi(T, cfg["ranks"], cfg["iters"], cfg["tol"])
    fit = float(res["fit"].cpu())
    print(f"xga fit gpu {fit:.9f} oracle {ref.fit:.9f} rel {abs(fit - ref.fit) / ref.fit:.2e}")
    assert abs(fit - ref.fit) / ref.fit < 1e-5
    Us = factors_np(res)
    for n, U in enumerate(Us):
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 2e-6
    for n in (2, 3):
        gap, sin_max = gap_and_sin(T, ref.factors, n, Us[n])
        if gap > GAP_GATE:
            assert sin_max < 1e-3, (n, gap, sin_max)
    # the large modes (r = 256 of 1024, 192 of 768): the gap at r is ~1e-9 of
    # l_1, below what FP32 resolves, so the gate is on the leading directions
    # with a usable gap, which must lie inside the GPU's subspace
    for n in (0, 1):
        k, sin_k = contained_sin(T, ref.factors, n, Us[n])
        print(f"xga mode {n}: leading {k} directions with gap > {GAP_GATE}, sin {sin_k:.2e}")
        assert k >= 4 and sin_k < 1e-3, (n, k, sin_k)
    # the columns themselves (Rayleigh-Ritz of the r > 128 factors, Section
    # III-B after Eq. 8: the factor is the Gram's leading eigenvectors): a
    # column whose eigenvalue is separated from both neighbours by more than
    # 1e-3 l_1 is determined to ~u l_1 / gap in FP32, and must match the
    # oracle's column under the same sign rule
    for n in (0, 1):
        Y = tucker.multi_mode_product(T, ref.factors, skip=n, transpose=True)
        w = np.sort(np.linalg.eigvalsh(tucker.gram(tucker.unfold(Y, n))))[::-1]
        r = cfg["ranks"][n]
        sep = [min(w[i - 1] - w[i] if i > 0 else np.inf, w[i] - w[i + 1]) / w[0] for i in range(r)]
        cols = [i for i in range(r) if sep[i] > 1e-3]
        dev = [float(np.abs(Us[n][:, i] - ref.factors[n][:, i]).max()) for i in cols]
        print(f"xga mode {n}: separated columns {cols}, max deviation {max(dev):.2e}")
        assert len(cols) >= 3 and max(dev) < 2e-3, (n, cols, dev)
    # the quantiser on the GPU core is bit-exact against the oracle's quantiser
    core = res["core"].cpu().numpy().transpose(3, 2, 1, 0)
    q, sc = mes.quantize_core(res["core"], cfg["ranks"], 16)
    qo, so = quant.quantize_planes(quant.planes_of(core), 16)
    assert np.array_equal(sc.cpu().numpy(), so)
    assert np.array_equal(quant.planes_of(to_paper(q).astype(np.float32)).astype(np.int64), qo.astype(np.int64))


@pytest.mark.slow
def test_fhd_full_size_properties(mes):
    """1920x1080x3x10 in the benchmark's launch configuration: the oracle
    cannot run the full decomposition in test time, so check what holds at any
    size -- orthonormal factors, the returned fit equals the FP64 fit of the
    returned decomposition, the energy identity, and sampled entries of the
    reconstruction against the element-wise model (Eq. 2)."""
    cfg, img = _scene("fhd_1920x1080")
    spec = cfg["spec"]
    dims = (spec.s1, spec.s2, 3, spec.K)
    X, n2 = mes.colour_convert(torch.from_numpy(img).to(DEV), cfg["space"])
    res = mes.tucker_als(X, dims, cfg["ranks"], max_iters=cfg["iters"], tol=0.0, history=True)
    Xh = mes.reconstruct(res["core"], res["factors"], dims, cfg["ranks"])
    torch.cuda.synchronize()
    T = colour.colour_convert(img, cfg["space"])
    Us = factors_np(res)
    core = to_paper(res["core"])
    for U in Us:
        # FP32 CholeskyQR on columns of length s: ~sqrt(s) * 2^-24 (2.6e-6 at s = 1920)
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 5e-6
    Xr = tucker.reconstruct(core, Us)
    fit64 = 1.0 - tucker.relative_error(T, Xr)
    fit = float(res["fit"].cpu())
    print(f"fhd fit gpu {fit:.9f} fp64 evaluation {fit64:.9f}")
    assert abs(fit - fit64) < 1e-6
    h = res["fit_history"].cpu().numpy()
    assert np.all(np.isfinite(h)) and abs(h[-1] - fit) < 5e-4
    rng = np.random.default_rng(0)
    Xhn = Xh.cpu().numpy()
    for _ in range(50):
        idx = tuple(int(rng.integers(d)) for d in dims)
        want = tucker.element(core, Us, idx)
        got = float(Xhn[idx[::-1]])
        assert abs(got - want) < 2e-5, (idx, got, want)
    # energy identity ||T||^2 - ||Q||^2 = ||T - T_hat||^2: with an FP32 core
    # ||Q||^2 carries ~sqrt(s_1) * 2^-24 relative error of ||T||^2 (~3e-6
    # here), which is most of the residual at fit ~0.998
    lhs = np.sum(T ** 2) - np.sum(core ** 2)
    rhs = np.sum((T - Xr) ** 2)
    assert abs(lhs - rhs) < 3e-6 * np.sum(T ** 2)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("name", ["small_64x48", pytest.param("xga_1024x768", marks=pytest.mark.slow),
                                  pytest.param("fhd_1920x1080", marks=pytest.mark.slow)])
def test_precision_form_against_fp32_path(mes, name, prec):
    """Tensor-core TF32 and BF16 forms beside the plain FP32 path on the same
    input: relative fit deviation <= 1e-4 (the precision-form target), factors
    orthonormal, and the reported fit is the fit of the returned factors."""
    cfg, img = _scene(name)
    spec = cfg["spec"]
    dims = (spec.s1, spec.s2, 3, spec.K)
    X, _ = mes.colour_convert(torch.from_numpy(img).to(DEV), cfg["space"])
    a = mes.tucker_als(X, dims, cfg["ranks"], max_iters=cfg["iters"], tol=0.0, precision="fp32")
    b = mes.tucker_als(X, dims, cfg["ranks"], max_iters=cfg["iters"], tol=0.0, precision=prec)
    torch.cuda.synchronize()
    fa, fb = float(a["fit"].cpu()), float(b["fit"].cpu())
    print(f"{name}: fit fp32 {fa:.9f} {prec} {fb:.9f} rel dev {abs(fa - fb) / fa:.2e}")
    assert abs(fa - fb) / fa <= 1e-4
    for U in factors_np(b):
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 5e-6
    if name == "small_64x48":
        T = colour.colour_convert(img, cfg["space"])
        Xr = tucker.reconstruct(to_paper(b["core"]), factors_np(b))
        assert abs((1 - tucker.relative_error(T, Xr)) - fb) < 1e-6


@pytest.mark.slow
def test_precision_forms_against_oracle_xga(mes):
    """Error of every precision form against the FP64 oracle on the 1024x768
    scene, stated per result: relative fit, relative reconstruction error and
    PSNR of the reconstructed stack.  Gate: fit within 1e-5 (FP32) or 1e-4
    (tensor-core forms) of the oracle's."""
    cfg, img = _scene("xga_1024x768")
    spec = cfg["spec"]
    dims = (spec.s1, spec.s2, 3, spec.K)
    T = colour.colour_convert(img, cfg["space"])
    ref = tucker.hooi(T, cfg["ranks"], cfg["iters"], 0.0)
    Xo = tucker.reconstruct(ref.core, ref.factors)
    psnr_o = tucker.psnr(T, Xo)
    X, _ = mes.colour_convert(torch.from_numpy(img).to(DEV), cfg["space"])
    for prec, tol in (("fp32", 1e-5), ("tf32", 1e-4), ("bf16", 1e-4)):
        res = mes.tucker_als(X, dims, cfg["ranks"], max_iters=cfg["iters"], tol=0.0, precision=prec)
        Xh = mes.reconstruct(res["core"], res["factors"], dims, cfg["ranks"], precision=prec)
        torch.cuda.synchronize()
        fit = float(res["fit"].cpu())
        Xg = to_paper(Xh)
        rel = tucker.relative_error(T, Xg)
        ps = tucker.psnr(T, Xg)
        print(f"{prec}: fit {fit:.9f} (oracle {ref.fit:.9f}, rel dev {abs(fit - ref.fit) / ref.fit:.2e}); "
              f"rel err {rel:.6e} (oracle {1 - ref.fit:.6e}); PSNR {ps:.3f} dB (oracle {psnr_o:.3f})")
        assert abs(fit - ref.fit) / ref.fit < tol, prec
        assert abs(rel - (1 - ref.fit)) / (1 - ref.fit) < 0.05, prec


def _two_block_tensor(seed):
    """40 x 32 x 3 x 6 tensor built from two blocks of a Tucker core: rows 0..7
    of mode 1 pair with columns 0..5 of mode 2, rows 8..31 with columns
    6..11.  Truncating mode 1 first (the interlaced HOSVD) removes most of the
    second block before mode 2 is chosen, so the two initialisations lead
    HOOI to different local optima (fits about 10% apart)."""
    rng = np.random.default_rng(seed)
    C = np.zeros((32, 12, 3, 6))
    C[:8, :6] = 1.5 * rng.standard_normal((8, 6, 3, 6))
    C[8:, 6:] = 1.2 * rng.standard_normal((24, 6, 3, 6))
    C *= np.array([1.0, 0.6, 0.35])[None, None, :, None]
    C *= (0.8 ** np.arange(6))[None, None, None, :]
    T = C
    for n, (s, r) in enumerate(((40, 32), (32, 12), (3, 3), (6, 6))):
        T = tucker.mode_product(T, np.linalg.qr(rng.standard_normal((s, r)))[0], n)
    return T + 1e-4 * rng.standard_normal(T.shape)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 2e-3)])
@pytest.mark.parametrize("ranks", [(8, 6, 3, 6), (8, 6, 2, 3)])
def test_interlaced_init_follows_the_oracle(mes, ranks, prec, tol):
    """The interlaced start (mode n's factor from T truncated in modes
    1..n-1) against the oracle's st_hosvd: with the subspace iterations run
    to convergence, the fit after one sweep and after ten matches HOOI
    started from the oracle's interlaced factors, on a tensor where the
    truncated-HOSVD start ends elsewhere."""
    T = _two_block_tensor(7)
    st_init = tucker.st_hosvd(T, ranks)[0]
    for iters in (1, 10):
        ref_st = tucker.hooi(T, ranks, iters, 0.0, init_factors=st_init)
        ref_t = tucker.hooi(T, ranks, iters, 0.0)
        assert abs(ref_st.fit - ref_t.fit) / ref_t.fit > 0.01      # the case discriminates
        res = _run(mes, T, ranks, iters, 0.0, init="interlaced", init_iters=200, inner_iters=60,
                   precision=prec)
        fit = float(res["fit"].cpu())
        print(f"{ranks} {prec} {iters} sweeps: fit {fit:.9f} oracle interlaced {ref_st.fit:.9f} "
              f"truncated {ref_t.fit:.9f}")
        assert abs(fit - ref_st.fit) / ref_st.fit < tol, (fit, ref_st.fit, ref_t.fit)
        for U in factors_np(res):
            assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 5e-6


def test_interlaced_init_converges_to_the_scene_fit(mes):
    """On the 64x48 scene both starts reach the oracle's converged fit."""
    cfg, img = _scene("small_64x48")
    T = colour.colour_convert(img, cfg["space"])
    ref = tucker.hooi(T, cfg["ranks"], cfg["iters"], cfg["tol"])
    for init in ("thosvd", "interlaced"):
        res = _run(mes, T, cfg["ranks"], cfg["iters"], cfg["tol"], inner_iters=4, init=init)
        fit = float(res["fit"].cpu())
        assert abs(fit - ref.fit) / ref.fit < 1e-5, (init, fit, ref.fit)



def test_rate_sweep_matches_the_oracle_pipeline(mes):
    """Ranks x bits sweep on the 64x48 scene against the oracle's own chain
    (HOOI, per-plane quantiser, dequantiser, Eq. 1, inverse colour, 8-bit
    PSNR): PSNR within 0.05 dB of the oracle's, rising with the bit depth and
    with the ranks."""
    cfg, img = _scene("small_64x48")
    space = cfg["space"]
    grid = [(8, 6, 3, 6), (16, 12, 3, 6)]
    bits = [4, 8, 0]
    rows = mes.rate_sweep(torch.from_numpy(img).to(DEV), space, grid, bits, max_iters=10, tol=1e-8,
                          inner_iters=4)
    T = colour.colour_convert(img, space)
    for row in rows:
        ref = tucker.hooi(T, row["ranks"], 10, 1e-8)
        core = ref.core
        if row["bits"]:
            q, sc = quant.quantize_planes(quant.planes_of(core.astype(np.float32)), row["bits"])
            core = quant.core_of_planes(quant.dequantize_planes(q, sc), row["ranks"]).astype(np.float64)
        Xh = tucker.reconstruct(core, ref.factors)
        want = colour.psnr8(img, colour.to_u8(colour.colour_invert(Xh, space)))
        print(row, f"oracle {want:.4f}")
        assert abs(row["psnr"] - want) < 0.05, (row, want)
    by = {(tuple(r["ranks"]), r["bits"]): r["psnr"] for r in rows}
    for g in grid:
        assert by[(g, 4)] < by[(g, 8)] <= by[(g, 0)] + 0.05
    for b in bits:
        assert by[(grid[0], b)] < by[(grid[1], b)]



@pytest.mark.parametrize("prec,rprec", [("fp32", "fp32"), ("bf16", "tf32")])
def test_reconstruction_from_the_fit_pass(mes, prec, rprec):
    """T_hat stored by the fit's pass equals mes_reconstruct of the returned
    core and factors in the same arithmetic, bit for bit."""
    cfg, img = _scene("small_64x48")
    T = colour.colour_convert(img, cfg["space"])
    X = to_torch(T)
    Xh = torch.empty_like(X)
    res = mes.tucker_als(X, T.shape, cfg["ranks"], max_iters=4, tol=0.0, precision=prec, reconstruction=Xh)
    ref = mes.reconstruct(res["core"], res["factors"], T.shape, cfg["ranks"], precision=rprec)
    torch.cuda.synchronize()
    assert torch.equal(Xh, ref)


@pytest.mark.parametrize("name", ["small_64x48", pytest.param("xga_1024x768", marks=pytest.mark.slow)])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_early_sweeps_match_exact_hooi(mes, name, sweeps):
    """One and two sweeps at DEFAULT options against the oracle's exact HOOI
    (T-HOSVD start, exact Gram eigenvectors in every update, Eq. 6 to Eq. 8)
    after the same number of sweeps: relative fit within 1e-5, and the
    leading directions inside the GPU's subspaces.  After one or two sweeps
    the two iterates are not at a fixed point, and their Grams differ by
    ~1e-7 l_1 (each update's subspace is converged to its step count, not
    exactly), so the subspace gate applies where the gap is above 1e-3 l_1
    (full-rank small modes always agree)."""
    cfg, img = _scene(name)
    spec = cfg["spec"]
    dims = (spec.s1, spec.s2, 3, spec.K)
    X, _ = mes.colour_convert(torch.from_numpy(img).to(DEV), cfg["space"])
    res = mes.tucker_als(X, dims, cfg["ranks"], max_iters=sweeps, tol=0.0)
    torch.cuda.synchronize()
    T = colour.colour_convert(img, cfg["space"])
    ref = tucker.hooi(T, cfg["ranks"], sweeps, 0.0)
    fit = float(res["fit"].cpu())
    print(f"{name} {sweeps} sweep(s): fit {fit:.9f} oracle {ref.fit:.9f} rel {abs(fit - ref.fit) / ref.fit:.2e}")
    assert int(res["iters"].cpu()) == sweeps
    assert abs(fit - ref.fit) / ref.fit < 1e-5
    Us = factors_np(res)
    for n in range(4):
        k, sin_k = contained_sin(T, ref.factors, n, Us[n], gap_gate=1e-3)
        print(f"  mode {n}: leading {k} directions, sin {sin_k:.2e}")
        assert (k >= 2 or n >= 2) and sin_k < 1e-3, (n, k, sin_k)


@pytest.fixture(scope="module")
def fhd_oracle():
    """The FP64 oracle's decomposition of the 1920x1080x3x10 stack (20 sweeps,
    T-HOSVD start): about half a minute on the host cores."""
    cfg, img = _scene("fhd_1920x1080")
    T = colour.colour_convert(img, cfg["space"])
    ref = tucker.hooi(T, cfg["ranks"], cfg["iters"], 0.0)
    Xo = tucker.reconstruct(ref.core, ref.factors)
    return cfg, img, T, ref, tucker.psnr(T, Xo)


@pytest.mark.slow
@pytest.mark.parametrize("prec,fit_tol,sin_tol,gap_gate", [
    ("fp32", 1e-5, 1e-3, GAP_GATE), ("tf32", 1e-4, 1e-2, 1e-3), ("bf16", 1e-4, 1e-2, 1e-3)])
def test_fhd_against_the_oracle(mes, fhd_oracle, prec, fit_tol, sin_tol, gap_gate):
    """The benchmark's workload, 1920x1080x3x10 (ranks 384, 256, 3, 10; 20
    sweeps; default options), in each precision form against the FP64
    oracle: relative fit, the large-mode subspaces (the oracle's leading
    directions with a usable gap inside the GPU's subspace) and the PSNR of
    the reconstructed stack.  FP32 is gated at the plain-method tolerance,
    the tensor-core forms at the precision-form target (1e-4 in fit).  The
    PSNR tolerance follows from the fit's: a relative fit change d moves the
    residual norm by d fit / (1 - fit), i.e. the PSNR by
    20 log10(1 + d fit / (1 - fit)) dB (0.04 dB for FP32, 0.4 dB for the
    tensor-core forms at fit ~0.9978)."""
    cfg, img, T, ref, psnr_o = fhd_oracle
    spec = cfg["spec"]
    dims = (spec.s1, spec.s2, 3, spec.K)
    X, _ = mes.colour_convert(torch.from_numpy(img).to(DEV), cfg["space"])
    Xh = torch.empty_like(X)
    res = mes.tucker_als(X, dims, cfg["ranks"], max_iters=cfg["iters"], tol=0.0, precision=prec, reconstruction=Xh)
    torch.cuda.synchronize()
    assert int(res["status"].cpu()) == 0
    fit = float(res["fit"].cpu())
    dev = abs(fit - ref.fit) / ref.fit
    Us = factors_np(res)
    ps = tucker.psnr(T, to_paper(Xh))
    sins = [contained_sin(T, ref.factors, n, Us[n], gap_gate) for n in (0, 1)]
    print(f"fhd {prec}: fit {fit:.9f} oracle {ref.fit:.9f} rel dev {dev:.2e}; PSNR {ps:.3f} dB "
          f"(oracle {psnr_o:.3f}); mode 1 k={sins[0][0]} sin {sins[0][1]:.2e}, mode 2 k={sins[1][0]} "
          f"sin {sins[1][1]:.2e}")
    assert dev < fit_tol
    db_tol = 20.0 * np.log10(1.0 + fit_tol * ref.fit / (1.0 - ref.fit)) + 0.005
    assert abs(ps - psnr_o) < db_tol, (ps, psnr_o, db_tol)
    for n, (k, sin_k) in enumerate(sins):
        assert k >= 4 and sin_k < sin_tol, (n, k, sin_k)
