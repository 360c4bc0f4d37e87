"""Benchmark of the Tucker-ALS coding path on GB300.

One step = the whole path on a batch of 1920x1080, 2-view x 5-exposure stacks
(dims 1920 x 1080 x 3 x 10, IPT, ranks (384, 256, 3, 10), 20 sweeps each):
colour pre-pass of the resident 8-bit images, Tucker-ALS / HOOI, core
quantiser (16 bits) and reconstruction with the fused residual.  The metric
is stacks per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--precision bf16|tf32|fp32] [--stacks S] [--no-fp32-path]
                  [--batch-stacks B] [--serve-seconds S] [--serve-rate RATE]

The default times the BF16 form over 16 concurrent stacks per step and,
beside it, the plain FP32 path on the same stacks (its stacks/s and the
largest relative fit deviation between the two), then the batched form (64
mixed stacks as one CUDA graph) and the served form (a Poisson request
stream through the serving loop, p50/p99 latency).

Multi-GPU (torchrun, one rank per GPU): every rank decomposes its own stacks
(independent problems, weak scaling, no collective on the data path); the
value is all stacks over the slowest rank's time.

--impl reference times the FP64 CPU oracle (the reference of this build) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "fhd_1920x1080"
METRIC = "Tucker-ALS stacks/s (1080p, 2x5 exp)"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def stack_seeds(workload: str, rank: int, stacks: int):
    """Seeds of the stacks rank `rank` decomposes in every step: each rank has
    its own stacks (independent problems, no collective on the data path)."""
    import synth
    return [synth.seed_for(workload, rank * stacks + i) for i in range(stacks)]


def slowest_rank_ms(ms: float, dist, device):
    """The timed region's length on the slowest rank (every rank calls it)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(stacks_per_rank: int, steps: int, world: int, ms: float) -> float:
    """Stacks per second of the whole job: every rank's stacks over the
    slowest rank's time (weak scaling: the work per rank is fixed)."""
    return stacks_per_rank * steps * world / (ms / 1e3)


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", "0")) or (os.cpu_count() or 1)


def cpu_baseline(sample_sweeps: int = 1, workload: str = WORKLOAD):
    """The FP64 oracle as it stands on this host's cores, on a bounded sample
    of the workload: colour pre-pass, T-HOSVD initialisation and
    `sample_sweeps` HOOI sweeps of one stack, plus the quantiser.  `seconds`
    is the sample's measured wall time; `stack_seconds` scales the sweep
    time to the workload's full sweep count (an extrapolation, declared)."""
    import numpy as np
    import synth
    from oracle import colour, quant, tucker
    cfg = synth.config_spec(workload)
    spec = cfg["spec"]
    img = synth.make_stack(spec, synth.seed_for(workload))
    t0 = time.perf_counter()
    T = colour.colour_convert(img, cfg["space"])
    t1 = time.perf_counter()
    U = tucker.thosvd(T, cfg["ranks"])
    t2 = time.perf_counter()
    res = tucker.hooi(T, cfg["ranks"], sample_sweeps, 0.0, init_factors=U)
    t3 = time.perf_counter()
    quant.quantize_planes(quant.planes_of(res.core.astype(np.float32)), 16)
    t4 = time.perf_counter()
    per_stack = (t1 - t0) + (t2 - t1) + (t3 - t2) * cfg["iters"] / sample_sweeps + (t4 - t3)
    return {"value": 1.0 / per_stack, "unit": "stacks/s", "cores": int(_blas_threads()), "kind": "oracle",
            "sample": (f"1 stack {spec.s1}x{spec.s2}x3x{spec.K}: colour + T-HOSVD + {sample_sweeps} "
                       f"HOOI sweep(s) + quantiser, the sweep time scaled to {cfg['iters']} sweeps"),
            "seconds": t4 - t0, "stack_seconds": per_stack, "extrapolated_from_sweeps": sample_sweeps}


def oracle_thread_scaling(workload: str = "xga_1024x768"):
    """Wall time of one oracle sample (colour, T-HOSVD, one sweep,
    quantiser) on all host cores and on one thread (a child process with
    the BLAS thread pools limited to 1)."""
    allc = cpu_baseline(1, workload)["seconds"]
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", workload],
                       capture_output=True, text=True, env=env, timeout=600)
    one = float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 and r.stdout.strip() else None
    return {"sample": f"{workload}: colour + T-HOSVD + 1 HOOI sweep + quantiser", "all_cores_s": allc,
            "all_cores_threads": int(_blas_threads()), "one_thread_s": one, "host_cores": os.cpu_count()}


def _config(name, cfg, dims, ranks, precision, stacks, world):
    return {"workload": name, "dims": dims, "ranks": ranks, "sweeps": cfg["iters"], "colour": cfg["space"],
            "precision": precision, "quant_bits": 16, "stacks_per_step": stacks,
            "l2": "inputs larger than L2: each stack's tensor is 249 MB in FP32 (124 MB per BF16 layout), "
                  "read twice per sweep",
            "parallelism": f"stack-parallel x{world}"}


def run_reference(args):
    """The oracle timed on the host cores (rank 0 only): every step is one
    bounded sample of the workload (colour, T-HOSVD, one HOOI sweep and the
    quantiser of one stack).  ms_per_step is the measured time of a sample;
    the value is stacks/s of the full 20-sweep decomposition, the sample's
    sweep scaled to 20 sweeps (declared in the line)."""
    import synth
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_baseline(1, args.workload)
    samples = [cpu_baseline(1, args.workload) for _ in range(args.steps)]
    step_s = statistics.mean(c["seconds"] for c in samples)
    stack_s = statistics.mean(c["stack_seconds"] for c in samples)
    val = 1.0 / stack_s
    cfg = synth.config_spec(args.workload)
    spec = cfg["spec"]
    conf = _config(args.workload, cfg, [spec.s1, spec.s2, 3, spec.K], list(cfg["ranks"]), "f64", 1, world)
    conf["stacks_per_step"] = step_s / stack_s
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "stacks/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": conf,
            "sample_per_step": samples[-1]["sample"],
            "extrapolated_from_sweeps": 1,
            "value_note": (f"each step times one sample (one sweep of the {cfg['iters']}); value = stacks_per_step "
                           f"/ seconds per step, i.e. the sample's sweep time scaled to {cfg['iters']} sweeps"),
            "cpu_baseline": {"value": val, "unit": "stacks/s", "cores": samples[-1]["cores"], "kind": "oracle",
                             "sample": samples[-1]["sample"]},
            "thread_scaling": oracle_thread_scaling(),
            "e2e": {"value": val, "unit": "stacks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _traffic(family):
    """DRAM bytes per launch of a kernel family from the committed ncu
    summary, or None when the kernel's source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            parts = ln.split()
            if len(parts) < 4 or parts[0] != family:
                continue
            src = os.path.join(ROOT, parts[1])
            if not os.path.exists(src):
                return None, "source missing"
            with open(src, "rb") as g:
                digest = hashlib.sha256(g.read()).hexdigest()[:12]
            if digest != parts[2]:
                return None, f"{parts[1]} changed since the capture"
            return float(parts[3]), " ".join(parts[4:])
    return None, None


def _family_roof(f, peaks, peak_src, sms):
    """Roofline of one kernel family from its profiled launches: tensor-core
    products against the measured BF16 peak (x 0.5 for the TF32 kinds,
    nominal ratio; sustained figure, as they run inside a long step), FP32
    CUDA-core arithmetic against SMs x 128 lanes x 2 x max clock, everything
    else against the measured HBM copy bandwidth."""
    name = f["name"]
    if "_tc" in name:
        peak = peaks.get("bf16_tflops_sustained", 1700.0) * (1.0 if name.startswith("gemm_bf16") else 0.5)
        achieved = f["flops"] / (f["ms"] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"{peak_src} bf16_tflops_sustained x {'1' if name.startswith('gemm_bf16') else '0.5 (tf32)'}"}
    elif f["flops"] > 0 and f["bytes"] / max(f["flops"], 1) < 0.1:
        peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        achieved = f["flops"] / (f["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"derived: {sms} SMs x 128 FP32 FMA lanes x 2 x {peaks.get('sm_max_mhz')} MHz"}
    else:
        achieved = f["bytes"] / (f["ms"] / 1e3) / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "peak_source": f"{peak_src} hbm_gbs"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    return roof


def algorithmic_flops_per_stack(dims, ranks, sweeps):
    """Algorithmic flops of the paper's method on one stack: per sweep the
    two mode products with T (2 N_el (r1 + r2)), the Gram products of the
    two large unfoldings as symmetric rank-k updates (s1^2 r2 L + s2^2 r1 L)
    and the core (2 r1 s2 L r2); once, the Gram products of the T-HOSVD
    start (s1^2 s2 L + s2^2 s1 L).  Small modes at full rank add nothing.
    The eigen-solver's own iterations are not counted (the paper does not
    fix one)."""
    s1, s2 = dims[0], dims[1]
    r1, r2 = ranks[0], ranks[1]
    L = 1
    for d in dims[2:]:
        L *= d
    nel = s1 * s2 * L
    sweep = 2.0 * nel * (r1 + r2) + s1 * s1 * r2 * L + s2 * s2 * r1 * L + 2.0 * r1 * s2 * L * r2
    init = float(s1) * s1 * s2 * L + float(s2) * s2 * s1 * L
    return sweeps * sweep + init


def _roofline(fams, peaks, peak_src, sms):
    total_ms = sum(f["ms"] for f in fams) or 1.0
    top = fams[0]
    traffic, note = _traffic(top["name"])
    per_launch = lambda x: x / max(top["launches"], 1)
    roof = _family_roof(top, peaks, peak_src, sms)
    roof.update({"traffic": traffic, "kernel": top["name"],
                 "share": top["ms"] / total_ms, "launches": top["launches"],
                 "avg_launch_us": 1e3 * top["ms"] / max(top["launches"], 1),
                 "algorithmic_bytes_per_launch": per_launch(top["bytes"]),
                 "algorithmic_flops_per_launch": per_launch(top["flops"])})
    if note:
        roof["traffic_note"] = note
    return roof


def _family_rooflines(fams, peaks, peak_src, sms, n=6):
    """The same roofline for the n families with the largest time share."""
    total_ms = sum(f["ms"] for f in fams) or 1.0
    out = []
    for f in fams[:n]:
        r = _family_roof(f, peaks, peak_src, sms)
        t, _ = _traffic(f["name"])
        out.append({"kernel": f["name"], "share": round(f["ms"] / total_ms, 4), "bound": r["bound"],
                    "achieved": round(r["achieved"], 3), "peak": r["peak"], "unit": r["unit"],
                    "frac": round(r["frac"], 5), "traffic": t})
    return out


SERVE_SIZES = ((640, 480), (1280, 720), (1920, 1080))


def _serve_mix(mes, dev, seed_base):
    """The mixed request workload of the serving form: 640x480, 1280x720 or
    1920x1080 with 3..7 exposures per view, or (5%) 3840x2160 with 3 per
    view; ranks 20% of the two image modes, full rank for colour and
    view x exposure; IPT or Y'CbCr.  Returns (scenes, draw(rng))."""
    import torch
    import synth
    stops = tuple(2.0 ** e for e in (-3, -2, -1, 0, 1, 2, 3))
    scenes = {}
    for s1, s2 in SERVE_SIZES:
        spec = synth.SceneSpec(s1, s2, stops, views=2, d_max=max(4, s1 // 40))
        scenes[(s1, s2)] = torch.from_numpy(synth.make_stack(spec, seed_base + s1)).to(dev)
    spec4k = synth.SceneSpec(3840, 2160, (0.25, 1.0, 4.0), views=2, d_max=96)
    scenes[(3840, 2160)] = torch.from_numpy(synth.make_stack(spec4k, seed_base + 999)).to(dev)
    inputs = {}

    def draw(rng):
        if rng.random() < 0.05:
            s1, s2, E = 3840, 2160, 3
        else:
            s1, s2 = SERVE_SIZES[int(rng.integers(3))]
            E = int(rng.integers(3, 8))
        key = (s1, s2, E)
        if key not in inputs:   # view-major: the first E exposures of each view
            base = scenes[(s1, s2)]
            Eb = base.shape[0] // 2
            inputs[key] = torch.cat([base[:E], base[Eb:Eb + E]]).contiguous()
        space = "ipt" if rng.random() < 0.5 else "ycbcr"
        return key, space

    return inputs, draw


def _serve_run(mes, srv, precision, inputs, draws, arrivals, window, pool):
    """Submits draws[i] at arrivals[i] seconds (host clock) and collects the
    latency of every request; completed requests give their buffers back to
    the pool (keyed by size and exposure count), so memory follows the
    number of requests outstanding.  Returns per-request latencies (ms),
    statuses and the wall time."""
    import time as _t
    out = {}
    pending = {}

    def recycle():
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                key, p, i = pending.pop(t)
                out[i] = r
                pool.setdefault((key, precision), []).append(p)

    t0 = _t.perf_counter()
    for i, ((key, space), a) in enumerate(zip(draws, arrivals)):
        while True:
            recycle()
            dt = t0 + a - _t.perf_counter()
            if dt <= 0:
                break
            _t.sleep(min(dt, 0.002))
        free = pool.get((key, precision))
        if free:
            p = free.pop()
        else:
            s1, s2, E = key
            p = mes.Problem((s1, s2, 3, 2 * E), (round(0.2 * s1), round(0.2 * s2), 3, 2 * E), rgb8=inputs[key],
                            space=space, max_iters=20, tol=0.0, precision=precision, quant_bits=16)
        p.struct.space = mes.SPACES[space]
        pending[srv.submit(p)] = (key, p, i)
    while pending:
        recycle()
        _t.sleep(0.0005)
    wall = _t.perf_counter() - t0
    lat = [out[i][1] for i in range(len(draws))]
    st = [out[i][0] for i in range(len(draws))]
    return lat, st, wall


def measure_serving(mes, dev, precision, rate_cap, seconds, warm_s, fp32_seconds, seed, slots, budget_gb):
    """Serving form as the serving workload defines it: Poisson arrivals of
    the mixed requests (20 sweeps, 16-bit quantised core) into the library's
    serving loop (continuous batching under a device-memory budget), warm_s
    seconds of warm-up then `seconds` measured; latency is submission to
    observed completion.  The arrival rate is rate_cap (200/s) or 80% of the
    measured capacity when that is lower (above capacity the queue, and with
    it every latency, grows without bound).  Capacity = a burst of requests
    submitted at once, completions per second.  Beside it the plain
    per-request FP32 path served the same way: FP32 precision, one slot (one
    request at a time on one stream), at 80% of its own capacity."""
    import numpy as np
    import torch

    inputs, draw = _serve_mix(mes, dev, 5000)
    pool = {}

    def arm(prec, nslots, secs):
        rng = np.random.default_rng(seed)
        srv = mes.Server(int(budget_gb * 2 ** 30), nslots)
        try:
            # one request of every size first: one-time setup outside the measurement
            seen = set()
            warm = []
            for _ in range(200):
                d = draw(rng)
                if d[0] not in seen:
                    seen.add(d[0])
                    warm.append(d)
            _serve_run(mes, srv, prec, inputs, warm, [0.0] * len(warm), None, pool)
            burst = [draw(rng) for _ in range(6 * nslots + 8)]
            lat, st, wall = _serve_run(mes, srv, prec, inputs, burst, [0.0] * len(burst), None, pool)
            capacity = len(burst) / wall
            rate = min(rate_cap, 0.8 * capacity)
            n = int(rate * (warm_s + secs)) + 1
            draws = [draw(rng) for _ in range(n)]
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
            lat, st, wall = _serve_run(mes, srv, prec, inputs, draws, arrivals, None, pool)
            meas = [i for i in range(n) if warm_s <= arrivals[i] < warm_s + secs]
            lm = np.array([lat[i] for i in meas if st[i] == 0]) if meas else np.array([float("nan")])
            eq = sum(draws[i][0][0] * draws[i][0][1] * 2 * draws[i][0][2] for i in meas) / (1920 * 1080 * 10)
            stats = srv.stats()
        finally:
            srv.close()
        return {"precision": prec, "slots": nslots, "capacity_req_per_s": capacity, "rate_per_s": rate,
                "warmup_s": warm_s, "measured_s": secs, "requests_measured": len(meas),
                "failed": int(sum(1 for i in meas if st[i] != 0)),
                "p50_ms": float(np.percentile(lm, 50)), "p99_ms": float(np.percentile(lm, 99)),
                "max_ms": float(lm.max()), "stacks_per_s": len(meas) / secs,
                "fhd_equiv_stacks_per_s": eq / secs, "hbm_peak_gib": stats["hbm_peak"] / 2 ** 30}

    served = arm(precision, slots, seconds)
    torch.cuda.synchronize()
    plain = arm("fp32", 1, fp32_seconds) if fp32_seconds > 0 else None
    pool.clear()
    torch.cuda.synchronize()
    out = dict(served)
    out.update({"hbm_budget_gib": budget_gb, "rate_cap_per_s": rate_cap,
                "rate_note": ("the workload's 200/s exceeds the measured capacity: run at 80% of capacity"
                              if served["rate_per_s"] < rate_cap else "run at the workload's rate"),
                "fp32_per_request_arm": plain})
    return out


def measure_batch(mes, dev, precision, n_stacks, seed, streams=16):
    """Batched form: n_stacks stacks of the mixed workload (640x480, 1280x720
    or 1920x1080; 3..7 exposures per view; ranks 20% of the two image modes,
    full rank for colour and view x exposure; IPT or Y'CbCr; 20 sweeps;
    16-bit quantiser) submitted as one captured CUDA graph and replayed,
    beside the same stacks as sequential calls of the plain FP32 path on one
    stream.  Reports both rates and the largest relative fit deviation of a
    batched stack from its FP32 result."""
    import numpy as np
    import torch
    import synth

    rng = np.random.default_rng(seed)
    stops = tuple(2.0 ** e for e in (-3, -2, -1, 0, 1, 2, 3))
    scenes = {}
    for s1, s2 in SERVE_SIZES:
        spec = synth.SceneSpec(s1, s2, stops, views=2, d_max=max(4, s1 // 40))
        scenes[(s1, s2)] = torch.from_numpy(synth.make_stack(spec, 6000 + s1)).to(dev)
    draws = []
    for _ in range(n_stacks):
        s1, s2 = SERVE_SIZES[int(rng.integers(3))]
        E = int(rng.integers(3, 8))
        base = scenes[(s1, s2)]
        Eb = base.shape[0] // 2
        rgb = torch.cat([base[:E], base[Eb:Eb + E]]).contiguous()
        draws.append(((s1, s2, 3, 2 * E), (round(0.2 * s1), round(0.2 * s2), 3, 2 * E), rgb,
                      "ipt" if rng.random() < 0.5 else "ycbcr"))

    def problems(prec):
        return [mes.Problem(d, r, rgb8=rgb, space=sp, max_iters=20, tol=0.0, precision=prec, quant_bits=16)
                for d, r, rgb, sp in draws]

    probs = problems(precision)
    st = torch.cuda.Stream(device=dev)   # graph capture needs a stream other than the legacy one
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    with torch.cuda.stream(st):
        b = mes.Batch(streams)
        b.run(probs)                  # one-time setup outside the capture
        st.synchronize()
        b.capture(probs, stream=st)
        b.launch()
        st.synchronize()
        e0.record(st)
        for _ in range(reps):
            b.launch()
        e1.record(st)
        st.synchronize()
        t_batch = e0.elapsed_time(e1) / 1e3 / reps
        fits = [float(p.fit) for p in probs]
        b.close()
        p32 = problems("fp32")
        b1 = mes.Batch(1)
        b1.run(p32[:1])
        st.synchronize()
        e0.record(st)
        for p in p32:
            b1.run([p])
        e1.record(st)
        st.synchronize()
        t_seq = e0.elapsed_time(e1) / 1e3
        b1.close()
    f32 = [float(p.fit) for p in p32]
    dev_rel = max(abs(a - c) / abs(c) for a, c in zip(fits, f32))
    return {"stacks": n_stacks, "precision": precision, "graph": True, "internal_streams": streams,
            "stacks_per_s": n_stacks / t_batch, "ms_per_batch": 1e3 * t_batch,
            "fp32_sequential_stacks_per_s": n_stacks / t_seq, "speedup_vs_fp32_sequential": t_seq / t_batch,
            "max_rel_fit_dev_vs_fp32": dev_rel,
            "fhd_equiv_stacks": sum(d[0][0] * d[0][1] * d[0][3] for d in draws) / (1920 * 1080 * 10)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mes", choices=["mes", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "tf32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-path", action="store_true",
                    help="skip timing the plain FP32 path beside the chosen precision form")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--stacks", type=int, default=16, help="independent stacks per step, one CUDA stream each")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="measured seconds of the serving form (0 = skip it)")
    ap.add_argument("--serve-warmup", type=float, default=10.0, help="warm-up seconds before the measured window")
    ap.add_argument("--serve-fp32-seconds", type=float, default=30.0,
                    help="measured seconds of the plain per-request FP32 served arm (0 = skip it)")
    ap.add_argument("--serve-rate", type=float, default=200.0,
                    help="Poisson arrival rate of the serving form (capped at 80%% of the measured capacity)")
    ap.add_argument("--batch-stacks", type=int, default=64,
                    help="stacks of the batched-form measurement (0 = skip it)")
    ap.add_argument("--batch-streams", type=int, default=16, help="internal streams of the batched form")
    ap.add_argument("--enqueue-threads", type=int, default=8,
                    help="host threads enqueueing the stacks of an eager (e2e) step")
    ap.add_argument("--concurrency", type=int, default=None,
                    help="concurrency hint of every decomposition (default: --stacks, the stacks run side by "
                         "side; 1: each as if alone, split-K fills all SMs)")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        print(cpu_baseline(1, args.oracle_sample)["seconds"])
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_2104_04726_gb300 as mes
    import synth
    from paper_2104_04726_gb300 import _lib

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if dist is not None:
        dist.barrier()
    lib = _lib.load()

    name = args.workload
    cfg = synth.config_spec(name)
    spec = cfg["spec"]
    dims = [spec.s1, spec.s2, 3, spec.K]
    ranks = list(cfg["ranks"])
    iters = cfg["iters"]
    S = args.stacks
    conc = S if args.concurrency is None else args.concurrency
    P = 1
    for r in ranks[2:]:
        P *= r

    seeds = stack_seeds(name, rank, S)

    class Stack:
        """Device-resident inputs and outputs of one stack, and its stream."""

        def __init__(self, idx):
            img = synth.make_stack(spec, seeds[idx])
            self.rgb_host = torch.from_numpy(img).pin_memory()
            self.rgb = self.rgb_host.to(dev)
            self.X = torch.empty((spec.K, 3, spec.s2, spec.s1), dtype=torch.float32, device=dev)
            self.n2 = torch.empty((), dtype=torch.float64, device=dev)
            self.core = torch.empty(mes.torch_shape(ranks), dtype=torch.float32, device=dev)
            self.facs = [torch.empty((r, s), dtype=torch.float32, device=dev) for s, r in zip(dims, ranks)]
            self.fit = torch.empty((), dtype=torch.float64, device=dev)
            self.Xh = torch.empty_like(self.X)
            self.itd = torch.zeros((), dtype=torch.int32, device=dev)
            self.stream = torch.cuda.Stream(device=dev)
            self.q_host = torch.empty(mes.torch_shape(ranks), dtype=torch.int16, pin_memory=True)
            self.s_host = torch.empty((P,), dtype=torch.float32, pin_memory=True)
            self.f_host = [torch.empty((r, s), dtype=torch.float32, pin_memory=True) for s, r in zip(dims, ranks)]
            self.fit_host = torch.empty((), dtype=torch.float64, pin_memory=True)

        def run(self, precision, e2e=False):
            with torch.cuda.stream(self.stream):
                if e2e:
                    self.rgb.copy_(self.rgb_host, non_blocking=True)
                mes.colour_convert(self.rgb, cfg["space"], out=self.X, norm2=self.n2)
                # the fit's reconstruction pass (fused residual) also stores T_hat
                # S decompositions run side by side: each splits its products'
                # reductions over its share of the SMs (the concurrency hint)
                mes.tucker_als(self.X, dims, ranks, max_iters=iters, tol=0.0, precision=precision,
                               outputs=(self.core, self.facs, self.fit, self.itd, None), reconstruction=self.Xh,
                               concurrency=conc)
                q, sc = mes.quantize_core(self.core, ranks, 16)
                if e2e:
                    self.q_host.copy_(q, non_blocking=True)
                    self.s_host.copy_(sc, non_blocking=True)
                    for a, b in zip(self.f_host, self.facs):
                        a.copy_(b, non_blocking=True)
                    self.fit_host.copy_(self.fit, non_blocking=True)

    stacks = [Stack(i) for i in range(S)]
    main_stream = torch.cuda.current_stream()

    # host threads that enqueue the stacks of an eager step side by side (the
    # library's calls are thread-safe on separate streams and release the
    # GIL): ~1100 launches per stack are too many for one enqueueing thread
    enqueue_threads = max(1, min(S, args.enqueue_threads))
    pool = None
    if enqueue_threads > 1:
        from concurrent.futures import ThreadPoolExecutor
        pool = ThreadPoolExecutor(max_workers=enqueue_threads, initializer=lambda: torch.cuda.set_device(dev))

    def step(precision, e2e=False, main=None, threaded=False):
        main = main_stream if main is None else main
        start = torch.cuda.Event()
        start.record(main)
        for st_ in stacks:
            st_.stream.wait_event(start)
        if threaded and pool is not None:
            def work(i0):
                for st_ in stacks[i0::enqueue_threads]:
                    st_.run(precision, e2e)
            for f in [pool.submit(work, i) for i in range(enqueue_threads)]:
                f.result()
        else:
            for st_ in stacks:
                st_.run(precision, e2e)
        for st_ in stacks:
            main.wait_stream(st_.stream)

    def capture(precision):
        """One step as a CUDA graph: every stack's stream forks from and joins
        the capturing stream, the library's stream-ordered allocations become
        graph memory nodes.  Replaying it issues the same kernels without the
        host enqueue of ~1100 launches per stack (measured: enqueueing 16
        stacks took 200 ms of a 279 ms step)."""
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=dev)
        cap.wait_stream(main_stream)
        with torch.cuda.graph(g, stream=cap):
            step(precision, main=torch.cuda.current_stream())
        main_stream.wait_stream(cap)
        return g

    def timed(n, precision, e2e=False, graph=None):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main_stream)
        for _ in range(n):
            if graph is not None:
                graph.replay()
            else:
                step(precision, e2e, threaded=True)
        b.record(main_stream)
        torch.cuda.synchronize()
        return slowest_rank_ms(a.elapsed_time(b), dist, dev)

    def measure(precision, detail):
        for _ in range(args.warmup):
            step(precision)
        torch.cuda.synchronize()
        graph = capture(precision)
        graph.replay()
        torch.cuda.synchronize()
        # timed region: K steps of S stacks, device events, barrier + sync
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        ms_max = timed(args.steps, precision, graph=graph)
        clocks = sampler.stop()
        del graph
        fits = [float(s_.fit.item()) for s_ in stacks]
        out = {"value": whole_job_rate(S, args.steps, world, ms_max), "ms_per_step": ms_max / args.steps, "clocks": clocks,
               "fit": fits[0], "fits": fits}
        if not detail:
            return out
        # per-kernel profile: two stacks one after the other (events on the
        # launch stream, nothing else running), so every interval is the
        # kernel's own serialised duration, as in an ncu launch list
        prof_stacks = min(2, S)
        lib.mes_profile_enable(1)
        for st_ in stacks[:prof_stacks]:
            st_.run(precision)
            torch.cuda.synchronize()
        fams = []
        for i in range(lib.mes_profile_count()):
            nm = ctypes.create_string_buffer(64)
            n = ctypes.c_int64()
            t_ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _lib.check(lib.mes_profile_get(i, nm, 64, ctypes.byref(n), ctypes.byref(t_ms), ctypes.byref(fl),
                                           ctypes.byref(by)), "mes_profile_get")
            fams.append({"name": nm.value.decode(), "launches": n.value, "ms": t_ms.value, "flops": fl.value,
                         "bytes": by.value})
        lib.mes_profile_enable(0)
        fams.sort(key=lambda f: -f["ms"])
        out["fams"] = fams
        out["launches_per_step"] = S * sum(f["launches"] for f in fams) // prof_stacks
        out["prof_stacks"] = prof_stacks
        # end to end through the public API with host buffers, the stacks
        # enqueued by several host threads
        step(precision, True, threaded=True)
        torch.cuda.synchronize()
        e2e_ms = timed(args.steps, precision, e2e=True)
        out["e2e"] = whole_job_rate(S, args.steps, world, e2e_ms)
        return out

    res = measure(args.precision, True)
    fp32 = None
    if args.precision != "fp32" and not args.no_fp32_path:
        fp32 = measure("fp32", False)

    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = _roofline(res["fams"], peaks, peak_src, sms)
    flops_stack = algorithmic_flops_per_stack(dims, ranks, iters)
    step_tf = flops_stack * S / (res["ms_per_step"] / 1e3) / 1e12
    step_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    step_roof = {"bound": "tensor", "achieved": step_tf, "peak": step_peak, "unit": "TFLOP/s",
                 "frac": step_tf / step_peak, "algorithmic_flops_per_stack": flops_stack,
                 "note": (f"whole step: algorithmic flops of the method per stack x {S} stacks / ms_per_step, "
                          f"against the {peak_src} sustained BF16 peak")}
    h2d = S * stacks[0].rgb_host.numel()
    d2h = S * (stacks[0].q_host.numel() * 2 + P * 4 + sum(f.numel() * 4 for f in stacks[0].f_host) + 8)
    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": "stacks/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
                "data": "synthetic",
                "config": dict(_config(name, cfg, dims, ranks, args.precision, S, world), concurrency_hint=conc,
                               launch="value: the step captured once as a CUDA graph and replayed; "
                                      f"e2e: eager API calls from {enqueue_threads} host threads"),
                "roofline": roof, "rooflines": _family_rooflines(res["fams"], peaks, peak_src, sms),
                "rooflines_note": (f"per kernel family from a profiled pass of {res['prof_stacks']} stacks run one "
                                   "after another (CUDA events on the launch stream, no other work on the GPU): "
                                   "serialised durations and shares, as in an ncu launch list"),
                "step_roofline": step_roof,
                "gpu_launches": int(res["launches_per_step"] * args.steps),
                "clocks": res["clocks"],
                "e2e": {"value": res["e2e"], "unit": "stacks/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "fit": res["fit"],
                "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in f.items()}
                            for f in res["fams"][:8]]}
        if fp32 is not None:
            dev_rel = max(abs(a - b) / abs(b) for a, b in zip(res["fits"], fp32["fits"]))
            line["fp32_path"] = {"value": fp32["value"], "ms_per_step": fp32["ms_per_step"], "fit": fp32["fit"],
                                 "speedup": res["value"] / fp32["value"], "max_rel_fit_dev": dev_rel,
                                 "clocks": fp32["clocks"]}
        if args.batch_stacks > 0 and world == 1:
            line["batch"] = measure_batch(mes, dev, args.precision, args.batch_stacks, seed=11,
                                          streams=args.batch_streams)
        if args.serve_seconds > 0 and world == 1:
            line["serve"] = measure_serving(mes, dev, args.precision, args.serve_rate, args.serve_seconds,
                                            args.serve_warmup, args.serve_fp32_seconds, seed=7, slots=8,
                                            budget_gb=96)
        if not args.no_cpu_baseline and world == 1:
            cb = cpu_baseline(1)
            line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.shutdown()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
