"""Batched and served forms: every stack's result is the one the single calls
give for it alone (same kernels, same launch shapes, one stream per stack),
whether it runs in a batch, in a replayed CUDA graph or through the serving
loop next to other requests.  The problems carry an explicit concurrency
hint (3), which the single calls repeat: the hint sets how far products split
their reduction, so equal hints give bit-identical results."""

CONC = 3
import numpy as np
import pytest
import torch

import synth
from oracle import colour, tucker

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def mes():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2104_04726_gb300 as m
    return m


def _specs():
    """(dims, ranks, input kind, colour space, precision, quant bits, seed)."""
    return [
        ((64, 48, 3, 6), (16, 12, 3, 6), "rgb8", "ycbcr", "fp32", 16, 1),
        ((96, 64, 3, 4), (20, 16, 3, 4), "rgb8", "ipt", "fp32", 8, 2),
        ((50, 40, 5), (10, 8, 3), "X", None, "fp32", 0, 3),
        ((400, 300, 3, 4), (150, 140, 3, 4), "rgb8", "ipt", "tf32", 16, 4),
        ((120, 90, 3, 6), (24, 18, 2, 5), "rgb8", "ycbcr", "tf32", 12, 5),
    ]


def _inputs(spec):
    dims, ranks, kind, space, prec, bits, seed = spec
    if kind == "rgb8":
        K = dims[3]
        sc = synth.SceneSpec(dims[0], dims[1], tuple(2.0 ** e for e in range(K // 2)), views=2, d_max=4)
        assert sc.K == K, (sc.K, K)
        img = synth.make_stack(sc, 500 + seed)
        return torch.from_numpy(img).to(DEV), None
    # a planted multilinear-rank (10, 8, 3) tensor plus 5% noise: HOOI
    # converges within the problems' 8 sweeps, so the oracle comparison is
    # a comparison of the same fixed point
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(ranks) * np.logspace(0, -1, ranks[0])[:, None, None]
    Qs = [np.linalg.qr(rng.standard_normal((s, r)))[0] for s, r in zip(dims, ranks)]
    Xp = tucker.reconstruct(G, Qs)
    Xp = Xp + 0.05 * np.std(Xp) * rng.standard_normal(dims)
    X = np.ascontiguousarray(Xp.transpose(tuple(range(len(dims)))[::-1])).astype(np.float32)
    return None, torch.from_numpy(X).to(DEV)


def _problem(mes, spec):
    dims, ranks, kind, space, prec, bits, seed = spec
    rgb8, X = _inputs(spec)
    return mes.Problem(dims, ranks, X=X, rgb8=rgb8, space=space or "ipt", max_iters=8, tol=0.0,
                       precision=prec, quant_bits=bits, concurrency=CONC)


def _single(mes, p, spec):
    """The same stack through the single calls, on the current stream."""
    dims, ranks, kind, space, prec, bits, seed = spec
    X = p.X
    if p.rgb8 is not None:
        X, _ = mes.colour_convert(p.rgb8, space, 2.2)
    res = mes.tucker_als(X, dims, ranks, max_iters=8, tol=0.0, precision=prec, concurrency=CONC)
    out = {"core": res["core"], "factors": res["factors"], "fit": res["fit"], "X": X}
    if bits:
        out["q"], out["scales"] = mes.quantize_core(res["core"], ranks, bits)
    return out


def _same(p, ref, bits):
    torch.cuda.synchronize()
    assert torch.equal(p.X, ref["X"])
    assert torch.equal(p.core, ref["core"])
    for a, b in zip(p.factors, ref["factors"]):
        assert torch.equal(a, b)
    assert float(p.fit) == float(ref["fit"])
    if bits:
        assert torch.equal(p.q, ref["q"])
        assert torch.equal(p.scales, ref["scales"])


@pytest.fixture(scope="module")
def oracle_fits(cases):
    """The FP64 oracle's fit of every stack of the batch (its own colour
    pre-pass of the 8-bit images, or the FP32 tensor read back), exact HOOI
    with the problems' sweep count."""
    specs, probs, _ = cases
    fits = []
    for p, spec in zip(probs, specs):
        dims, ranks, kind, space, prec, bits, seed = spec
        if p.rgb8 is not None:
            T = colour.colour_convert(p.rgb8.cpu().numpy(), space)
        else:
            a = p.X.cpu().numpy().astype(np.float64)
            T = a.transpose(tuple(range(a.ndim))[::-1])
        fits.append(tucker.hooi(T, ranks, 8, 0.0).fit)
    return fits


def _against_oracle(probs, specs, fits, where):
    """Each stack's fit against the oracle's after the same 8 sweeps: 1e-4
    relative (the GPU's default of one warm-started subspace step per update
    trails exact HOOI's first sweeps by up to ~5e-5 on these scenes and
    reaches the same fixed point; the tensor-core target is 1e-4 as well)."""
    torch.cuda.synchronize()
    for p, spec, fo in zip(probs, specs, fits):
        f = float(p.fit)
        print(f"{where} {spec[0]} {spec[4]}: fit {f:.9f} oracle {fo:.9f} rel {abs(f - fo) / fo:.2e}")
        assert abs(f - fo) / fo < 1e-4, (spec, f, fo)


@pytest.fixture(scope="module")
def cases(mes):
    specs = _specs()
    probs = [_problem(mes, s) for s in specs]
    refs = [_single(mes, p, s) for p, s in zip(probs, specs)]
    torch.cuda.synchronize()
    return specs, probs, refs


def _clear(p):
    for t in [p.core, p.fit, *p.factors] + ([p.q, p.scales] if p.q is not None else []):
        t.zero_()
    if p.rgb8 is not None:
        p.X.zero_()


def test_batch_matches_single_calls(mes, cases):
    specs, probs, refs = cases
    for p in probs:
        _clear(p)
    b = mes.Batch(3)
    b.run(probs)
    for p, r, s in zip(probs, refs, specs):
        _same(p, r, s[5])
    b.close()


def test_batch_stacks_against_the_oracle(mes, cases, oracle_fits):
    specs, probs, refs = cases
    for p in probs:
        _clear(p)
    b = mes.Batch(3)
    b.run(probs)
    _against_oracle(probs, specs, oracle_fits, "batch")
    b.close()


def test_batch_graph_replay(mes, cases):
    specs, probs, refs = cases
    b = mes.Batch(4)
    b.run(probs)                      # one-time setup outside the capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream(device=DEV)
    with torch.cuda.stream(side):
        b.capture(probs, side)
    torch.cuda.synchronize()
    for rep in range(2):
        for p in probs:
            _clear(p)
        torch.cuda.synchronize()
        b.launch()
        for p, r, s in zip(probs, refs, specs):
            _same(p, r, s[5])
    b.close()


def test_server_results_alone_and_in_mix(mes, cases, oracle_fits):
    specs, probs, refs = cases
    for p in probs:
        _clear(p)
    torch.cuda.synchronize()
    srv = mes.Server(8 << 30, 3)
    tickets = [srv.submit(p) for p in probs]
    for t in tickets:
        status, lat = srv.wait(t, 60000.0)
        assert status == 0 and lat > 0
    for p, r, s in zip(probs, refs, specs):
        _same(p, r, s[5])
    _against_oracle(probs, specs, oracle_fits, "served")
    st = srv.stats()
    assert st["completed"] == len(probs) and st["failed"] == 0 and st["queued"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["hbm_in_use"] == 0 and 0 < st["hbm_peak"] <= 8 << 30
    srv.close()


def test_server_budget_admission(mes, cases):
    specs, probs, refs = cases
    big = max(mes.tucker_als_workspace_size(s[0], s[1], s[4]) for s in specs)
    # room for the largest request alone, plus its buffers: at most one or two run at once
    budget = big + (64 << 20)
    srv = mes.Server(budget, 4)
    for p in probs:
        _clear(p)
    torch.cuda.synchronize()
    tickets = [srv.submit(p) for p in probs]
    for t in tickets:
        assert srv.wait(t, 60000.0)[0] == 0
    for p, r, s in zip(probs, refs, specs):
        _same(p, r, s[5])
    st = srv.stats()
    assert st["hbm_peak"] <= budget
    srv.close()
    # a request that can never fit is refused at submission
    small = mes.Server(1 << 20, 2)
    with pytest.raises(mes._lib.MesError) as e:
        small.submit(probs[3])
    assert e.value.name == "MES_ERR_OOM"
    small.close()


def test_server_poll_and_timeout(mes, cases):
    specs, probs, refs = cases
    srv = mes.Server(8 << 30, 1)
    t1 = srv.submit(probs[3])
    t2 = srv.submit(probs[0])          # queued behind the first (one slot)
    assert srv.poll(t2) is None
    with pytest.raises(mes._lib.MesError) as e:
        srv.wait(t2, 0.001)
    assert e.value.name == "MES_ERR_TIMEOUT"
    assert srv.wait(t1, 60000.0)[0] == 0
    assert srv.wait(t2, 60000.0)[0] == 0
    assert srv.poll(t2) is not None
    srv.close()
