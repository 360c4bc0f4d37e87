"""Failure paths, made without faulting the GPU: a bounded tensor-core
pipeline wait that runs out (a bound of 1 ns, set through the options), NaN
in the input tensor, and host-side injection (MES_FAULT) of a failed
allocation and of a refused admission.  Each failure must reach the caller as
a status (and a NaN fit), never as a finite-looking result, and the context
must stay usable: the same call without the fault succeeds afterwards."""
import os

import numpy as np
import pytest

import synth
from oracle import colour

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DEV = "cuda:0"
MES_ERR_OOM, MES_ERR_TIMEOUT, MES_ERR_NONFINITE = 3, 5, 6


@pytest.fixture(scope="module")
def mes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2104_04726_gb300 as m
    return m


@pytest.fixture(scope="module")
def scene():
    cfg = synth.config_spec("small_64x48")
    img = synth.make_stack(cfg["spec"], synth.seed_for("small_64x48"))
    T = colour.colour_convert(img, cfg["space"])
    X = torch.from_numpy(np.ascontiguousarray(T.transpose(3, 2, 1, 0))).float().to(DEV)
    return X, T.shape, cfg["ranks"]


@pytest.fixture
def fault_env():
    old = os.environ.get("MES_FAULT")
    yield
    if old is None:
        os.environ.pop("MES_FAULT", None)
    else:
        os.environ["MES_FAULT"] = old


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_pipeline_wait_that_runs_out_is_reported(mes, scene, prec):
    X, dims, ranks = scene
    res = mes.tucker_als(X, dims, ranks, max_iters=3, tol=0.0, precision=prec, wait_ns=1)
    torch.cuda.synchronize()
    assert int(res["status"].cpu()) == MES_ERR_TIMEOUT
    assert np.isnan(float(res["fit"].cpu()))
    # the context is intact: the same call with the default bound succeeds
    ok = mes.tucker_als(X, dims, ranks, max_iters=3, tol=0.0, precision=prec)
    torch.cuda.synchronize()
    assert int(ok["status"].cpu()) == 0
    assert 0.9 < float(ok["fit"].cpu()) <= 1.0


def test_fp32_form_has_no_pipeline_wait(mes, scene):
    # the bound only applies to tensor-core products: the CUDA-core form is unaffected
    X, dims, ranks = scene
    res = mes.tucker_als(X, dims, ranks, max_iters=3, tol=0.0, precision="fp32", wait_ns=1)
    torch.cuda.synchronize()
    assert int(res["status"].cpu()) == 0 and np.isfinite(float(res["fit"].cpu()))


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_nan_in_the_tensor_is_reported(mes, scene, prec):
    X, dims, ranks = scene
    Xn = X.clone()
    Xn.view(-1)[1234] = float("nan")
    res = mes.tucker_als(Xn, dims, ranks, max_iters=3, tol=0.0, precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].cpu()) == MES_ERR_NONFINITE
    assert np.isnan(float(res["fit"].cpu()))


def test_injected_allocation_failure(mes, scene, fault_env):
    X, dims, ranks = scene
    for k in (0, 5):
        os.environ["MES_FAULT"] = f"alloc:{k}"
        with pytest.raises(mes.MesError) as e:
            mes.tucker_als(X, dims, ranks, max_iters=2, tol=0.0)
        assert e.value.name == "MES_ERR_OOM"
        assert "MES_FAULT" in str(e.value)
    os.environ.pop("MES_FAULT")
    res = mes.tucker_als(X, dims, ranks, max_iters=2, tol=0.0)
    torch.cuda.synchronize()
    assert int(res["status"].cpu()) == 0


def test_injected_admission_refusal_and_device_failure_in_the_server(mes, scene, fault_env):
    X, dims, ranks = scene
    srv = mes.Server(4 << 30, 2)
    try:
        os.environ["MES_FAULT"] = "admit"
        p = mes.Problem(dims, ranks, X=X, max_iters=2, tol=0.0)
        st, _ = srv.wait(srv.submit(p))
        assert st == MES_ERR_OOM
        os.environ.pop("MES_FAULT")
        good = mes.Problem(dims, ranks, X=X, max_iters=2, tol=0.0)
        bad = mes.Problem(dims, ranks, X=X, max_iters=2, tol=0.0, precision="tf32", wait_ns=1)
        tg, tb = srv.submit(good), srv.submit(bad)
        assert srv.wait(tg)[0] == 0
        assert srv.wait(tb)[0] == MES_ERR_TIMEOUT
        torch.cuda.synchronize()
        assert np.isnan(float(bad.fit)) and np.isfinite(float(good.fit))
        s = srv.stats()
        assert s["failed"] == 2 and s["completed"] == 1
    finally:
        srv.close()


def test_batch_problem_status(mes, scene):
    X, dims, ranks = scene
    good = mes.Problem(dims, ranks, X=X, max_iters=2, tol=0.0, precision="tf32")
    bad = mes.Problem(dims, ranks, X=X, max_iters=2, tol=0.0, precision="tf32", wait_ns=1)
    b = mes.Batch(2)
    b.run([good, bad])
    torch.cuda.synchronize()
    b.close()
    assert int(good.status.cpu()) == 0 and np.isfinite(float(good.fit))
    assert int(bad.status.cpu()) == MES_ERR_TIMEOUT and np.isnan(float(bad.fit))



def test_phase_trace(mes, scene, tmp_path, monkeypatch):
    """MES_TRACE=<file>: one JSON line per traced call with its phases timed
    on the call's stream; a call without the variable writes nothing."""
    import json
    X, dims, ranks = scene
    path = tmp_path / "trace.jsonl"
    monkeypatch.setenv("MES_TRACE", str(path))
    res = mes.tucker_als(X, dims, ranks, max_iters=3, tol=0.0)
    assert int(res["status"].cpu()) == 0
    monkeypatch.delenv("MES_TRACE")
    mes.tucker_als(X, dims, ranks, max_iters=3, tol=0.0)
    torch.cuda.synchronize()
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["call"] == "mes_tucker_als"
    names = [p[0] for p in rec["phases"]]
    assert names[:3] == ["setup", "layout", "init"]
    assert [n for n in names if n.startswith("sweep")] == ["sweep 1", "sweep 2", "sweep 3"]
    assert names[-1] == "fit" and "orthonormalise" in names
    ms = [p[1] for p in rec["phases"]]
    assert all(m >= 0.0 for m in ms) and abs(sum(ms) - rec["total_ms"]) < 1e-2 * max(1.0, rec["total_ms"])
    assert rec["total_ms"] > 0.0
