"""Benchmark of the H / H^T pair on the 256^3 spherical-aperture scan.

A step is one projection u = H alpha and one backprojection alpha' = H^T y over the 256^3 @ 0.2 mm
grid, 128 rings x 180 views (23,040 point transducers on a 65 mm sphere), 1536 samples at 20 MHz.
The metric counts G interpolations: the lattice points whose trilinear stencil touches the grid,
once for H and once for H^T per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  With torchrun (N > 1) every rank runs an independent replica of the
problem (the operator needs no exchange); the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H+H^T G interp-samples/s and % HBM/L2 roofline; PLS-TV time to 1e-3 residual"
UNIT = "interp-samples/s"
WORKLOAD = "256^3 @ 0.2 mm, 200 ellipsoids, 128 rings x 180 views (23040 transducers) on 65 mm, K=1536 @ 20 MHz, c=1.5"
# FP32 operations charged to one interpolated sample: lattice point
# 6 FMA (12), floor 3, fraction 3, 7 lerps (7 sub + 7 FMA = 21), accumulate 1.
FLOP_PER_SAMPLE = 40.0
# kernels of this library per step: k_absmax, k_brick_gather, k_apply_d_fix (H); k_absmax,
# k_brick_gather_t, k_finish_t (H^T)
LAUNCHES_PER_STEP = 6
FP32_LANES_PER_SM = 128


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return mp, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def _sm_count(dev=0):
    """SM count of the device (the FP32 peak's unit count)."""
    import torch
    return torch.cuda.get_device_properties(dev).multi_processor_count


def _config(geom, world=1):
    """The workload's identity, the same dict in both arms."""
    return {"workload": WORKLOAD, "grid": [geom.nx, geom.ny, geom.nz], "transducers": geom.n_transducers,
            "samples": geom.n_samples, "l2": "inputs larger than L2 (volume 67 MB + data 142 MB per step)",
            "parallelism": f"replicas x{world}"}


KERNEL_SOURCES = ["forward.cu", "adjoint.cu", "brick.cuh", "oat_internal.h", "plan.cpp"]


def kernel_source_hash():
    """SHA-256 (first 16 hex digits) of the sources of the H / H^T kernels and their plan tables."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1304_2017_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _counters():
    """Per-kernel ncu counters committed under profiles/ (None where not measured).  They count
    only while the kernels are the ones profiled: counters.json records the hash of their sources,
    and a different hash here discards the counters."""
    try:
        with open(os.path.join(ROOT, "profiles", "counters.json")) as f:
            c = json.load(f)
    except (OSError, ValueError):
        return {}
    if c.get("_kernel_source_hash") != kernel_source_hash():
        return {}
    out = {k: v for k, v in c.items() if not k.startswith("_")}
    out["source"] = c.get("_about")
    return out


def l2_read_gbs(dev, mb=48, reps=100):
    """L2 read bandwidth: oat_probe_read over a 48 MB buffer (resident in the 129 MB L2 after a
    warm-up pass), 16-byte loads cached in L2 only, timed with CUDA events."""
    import torch
    from paper_1304_2017_gb300 import oat
    n = mb * (1 << 20)
    buf = torch.ones(n // 4, device=dev)
    sink = torch.zeros(1, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    oat.oat_probe_read(buf.data_ptr(), n, 2, sink.data_ptr(), s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    oat.oat_probe_read(buf.data_ptr(), n, reps, sink.data_ptr(), s)
    e1.record()
    torch.cuda.synchronize(dev)
    return n * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_throughput(ms, pts, world, device):
    """Whole-job interp-samples/s of `world` replicas that each ran one H + one H^T of `pts`
    samples per step in `ms` milliseconds: the slowest replica's time counts (max over ranks).
    Returns (value, ms_max)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * 2.0 * pts / (ms_max * 1e-3), ms_max


def cpu_baseline(geom, alpha, y, n_xdcr=32, points_per_xdcr=None):
    """Time the FP64 oracle (as it stands) for H and H^T on a transducer subset of the workload."""
    import oracle
    qs = np.linspace(0, geom.n_transducers - 1, n_xdcr).round().astype(int)
    sub = geom.subset(qs)
    ys = np.ascontiguousarray(y[qs], dtype=np.float64)
    a64 = alpha.astype(np.float64)
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.H(sub, a64)
    oracle.Ht(sub, ys)
    dt = time.perf_counter() - t0
    pts = points_per_xdcr * n_xdcr if points_per_xdcr is not None else oracle.count_points(sub)[1]
    # one thread, one transducer
    one = geom.subset(qs[:1])
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.H(one, a64)
        oracle.Ht(one, ys[:1])
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(threads)
    pts1 = oracle.count_points(one)[1]
    return {"value": 2.0 * pts / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_xdcr} of {geom.n_transducers} transducers (evenly spaced), full grid and time window; "
                      f"one H + one H^T in FP64, {dt:.1f} s",
            "single_thread": {"value": 2.0 * pts1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"transducer {int(qs[0])}, one H + one H^T in FP64, {dt1:.1f} s"}}


def run_reference(args):
    """The oracle on the host cores, on the same workload, metric and unit (bounded sample per step)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1304_2017_gb300 import workloads as W
    import oracle
    geom = W.config("c2")
    alpha = W.phantom("c2", geom)
    y = W.random_data(geom, seed=7)
    # one transducer per host thread at least, so that every core works (H parallelises over
    # transducers, H^T over transducers too, capped at their number)
    threads = oracle.max_threads()
    n_x = int(os.environ.get("OAT_REF_XDCR", str(max(16, threads))))
    qs = np.linspace(0, geom.n_transducers - 1, n_x).round().astype(int)
    sub = geom.subset(qs)
    pts = oracle.count_points(sub)[1]
    a64 = alpha.astype(np.float64)
    ys = np.ascontiguousarray(y[qs], dtype=np.float64)
    for _ in range(args.warmup):
        oracle.H(sub, a64)
        oracle.Ht(sub, ys)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.H(sub, a64)
        oracle.Ht(sub, ys)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = 2.0 * pts / dt
    cores = min(threads, n_x)
    sample = (f"{n_x} of {geom.n_transducers} transducers (evenly spaced) per step, full grid and time window, "
              f"one H + one H^T in FP64 on {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(geom),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def pls_small(dev):
    """The metric's third part on a workload that fits the default run: PLS-TV (FISTA-TV, x >= 0,
    5 FGP iterations, mu = 1e-6 L) from zero to a 1e-3 relative data residual, noise-free data
    u = H alpha of a seeded ellipsoid/sphere phantom, on the 64^3 @ 0.25 mm grid with 32 rings x
    45 views (1440 transducers) on 50 mm and K = 384; GPU seconds by CUDA events (the step-size
    estimate, 40 power iterations, reported apart)."""
    import torch
    from paper_1304_2017_gb300 import oat, warmstart
    from paper_1304_2017_gb300.fista import FistaTV
    geom = warmstart.geometry(n=64)
    plan = oat.Plan(geom, device=dev.index or 0)
    alpha = torch.from_numpy(warmstart.phantom(geom, 20_000)).to(dev)
    u = plan.project(alpha).clone()
    solver = FistaTV(plan, mu=0.0, inner=5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    L = solver.lipschitz(iters=40)
    e1.record()
    torch.cuda.synchronize(dev)
    solver.mu = 1e-6 * L
    _, info = solver.solve(u, iters=400, tol=1e-3)
    r = info["residual"]
    k = next((i for i, v in enumerate(r) if v <= 1e-3), None)
    plan.close()
    return {"value": info["gpu_seconds"][k] if k is not None else None, "unit": "s", "higher_is_better": False,
            "metric": "PLS-TV GPU seconds to a 1e-3 relative data residual (zero start)",
            "iterations": (k + 1) if k is not None else None, "final_residual": r[-1],
            "step_size_estimate_s": e0.elapsed_time(e1) * 1e-3, "mu": solver.mu,
            "workload": "64^3 @ 0.25 mm, 32 rings x 45 views (1440 transducers) on 50 mm, K=384 @ 20 MHz, c=1.5, "
                        "noise-free, held-out phantom seed 20000"}


def run_pls(args):
    """PLS-TV (FISTA-TV, x >= 0) from zero to a 1e-3 relative data residual on the 160^3
    workload: 96 rings x 90 views on 50 mm, K = 1024, 120 ellipsoids, noise-free data u = H alpha.
    mu = 1e-6 L; the TV prox takes 5 FGP iterations.  GPU time by CUDA events (the step-size
    estimate, 20 power iterations, is reported separately)."""
    import torch
    from paper_1304_2017_gb300 import oat
    from paper_1304_2017_gb300 import workloads as W
    from paper_1304_2017_gb300.fista import FistaTV
    torch.cuda.set_device(0)
    geom = W.config("c3")
    plan = oat.Plan(geom)
    alpha = torch.from_numpy(W.phantom("c3", geom)).cuda()
    u = plan.project(alpha).clone()
    solver = FistaTV(plan, mu=0.0, inner=5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    L = solver.lipschitz(iters=20)
    e1.record()
    torch.cuda.synchronize()
    l_s = e0.elapsed_time(e1) * 1e-3
    solver.mu = 1e-6 * L
    _, info = solver.solve(u, iters=args.pls_iters, tol=1e-3)
    r = info["residual"]
    k = next((i for i, v in enumerate(r) if v <= 1e-3), None)
    t = info["gpu_seconds"][k] if k is not None else None
    st = plan.stats(count_grid_points=True)
    line = {"metric": "PLS-TV GPU seconds to a 1e-3 relative data residual (zero start)", "value": t, "unit": "s",
            "higher_is_better": False, "iterations": (k + 1) if k is not None else None,
            "final_residual": r[-1], "seconds_per_iteration": info["gpu_seconds"][-1] / len(r),
            "step_size_estimate_s": l_s, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "160^3 @ 0.25 mm, 120 ellipsoids, 96 rings x 90 views (8640 transducers) on 50 mm, "
                                   "K=1024 @ 20 MHz, c=1.5, noise-free", "mu": solver.mu, "L": L, "inner": 5,
                       "points_per_operator": st["points_grid"]}}
    plan.close()
    print(json.dumps(line), flush=True)


def run_fbp(args):
    """Filtered backprojection (Eq. disfbp) on a workload (default the 256^3 / 23,040-transducer /
    K = 1536 one): seconds per reconstruction and voxel-transducer pairs per second, CUDA events
    around W untimed and K timed calls; the FP64 reference timed on a 16-transducer sample."""
    import torch
    from paper_1304_2017_gb300 import oat
    from paper_1304_2017_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    geom = W.config(args.config)
    scans = {"c1": (16, 16), "c2": (128, 180), "c3": (96, 90), "c5": (128, 60)}
    if args.config not in scans:
        raise SystemExit(f"--fbp: no rings x views scan known for --config {args.config}")
    n_r, n_v = scans[args.config]
    pos = geom.positions_mm
    rs = np.linalg.norm(pos, axis=1)
    theta = np.arccos(np.clip(pos[:, 2] / rs, -1.0, 1.0))
    w = rs * (np.pi / n_r) * (2.0 * np.pi / n_v) * np.sin(theta)      # patch area / R^s
    plan = oat.Plan(geom)
    plan.set_fbp_weights(w)
    p = torch.from_numpy(W.random_data(geom, seed=7)).to(dev)
    out = torch.empty(plan.vol_shape, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        plan.fbp(p, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(args.steps):
        plan.fbp(p, out=out)
    e1.record()
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) * 1e-3 / args.steps
    pairs = float(geom.n_voxels) * geom.n_transducers
    line = {"metric": "FBP voxel-transducer pairs/s (filtered backprojection, Eq. disfbp)", "value": pairs / sec,
            "unit": "pairs/s", "seconds_per_fbp": sec, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": W.DESCRIPTIONS.get(args.config, args.config), "pairs": pairs}}
    if not args.no_cpu_baseline:
        import oracle.fbp as F
        qs = np.linspace(0, geom.n_transducers - 1, 16).round().astype(int)
        sub = geom.subset(qs)
        t0 = time.perf_counter()
        F.fbp(sub, p[qs].cpu().numpy(), w[qs])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": float(geom.n_voxels) * len(qs) / dt, "unit": "pairs/s", "cores": 1,
                                "kind": "oracle", "sample": f"16 of {geom.n_transducers} transducers, full grid, "
                                                            f"numpy FP64, {dt:.1f} s"}
    plan.close()
    print(json.dumps(line), flush=True)


def run_sph(args):
    """Spherical-voxel model H_sph + H_sph^T (Eqs. dis_sph, sphbwd) on the paper's simulation grid
    (210 x 210 x 440 at 0.14 mm), its 64 x 90 scan on 65 mm and 511 frequencies in (0, 5] MHz:
    complex voxel-transducer-frequency terms per second, CUDA events around W untimed and K timed
    steps (one H_sph and one H_sph^T each); the FP64 reference timed on one transducer x 8
    frequencies.  --sph-transducers n keeps n transducers spread over the scan (small captures)."""
    import torch
    from paper_1304_2017_gb300 import oat
    from paper_1304_2017_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    geom = W.sph_config()
    if args.sph_transducers:
        geom = geom.subset(np.linspace(0, geom.n_transducers - 1, args.sph_transducers).round().astype(int))
    L, f0, df = 511, 5.0 / 511, 5.0 / 511
    alpha = torch.from_numpy(W.phantom_sph(geom)).to(dev)
    op = oat.SphOp(geom, L, f0, df)
    u = torch.empty(op.data_shape, dtype=torch.complex64, device=dev)
    a = torch.empty(op.vol_shape, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        op.project(alpha, out=u)
        op.backproject(u, out=a)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    clk = ClockSampler(0)
    torch.cuda.synchronize(dev)
    clk.start()
    for i in range(args.steps):
        ev[3 * i].record()
        op.project(alpha, out=u)
        ev[3 * i + 1].record()
        op.backproject(u, out=a)
        ev[3 * i + 2].record()
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    t_fwd = sum(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(args.steps)) * 1e-3 / args.steps
    t_bwd = sum(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(args.steps)) * 1e-3 / args.steps
    terms = float(geom.n_voxels) * geom.n_transducers * L
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = _sm_count(dev)
    peak = {"tflops": n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12,
            "source": f"{src} clock: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz"}
    dom, dom_t = ("k_sph_bwd (H_sph^T)", t_bwd) if t_bwd >= t_fwd else ("k_sph_fwd (H_sph)", t_fwd)
    line = {"metric": "H_sph+H_sph^T complex terms/s (spherical-voxel model, Eqs. dis_sph and sphbwd)",
            "value": 2 * terms / (t_fwd + t_bwd), "unit": "terms/s", "ms_per_step": (t_fwd + t_bwd) * 1e3,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": W.SPH_DESCRIPTION if not args.sph_transducers else
                       W.SPH_DESCRIPTION + f", {geom.n_transducers} transducers", "terms_per_operator": terms},
            "seconds": {"H_sph": t_fwd, "H_sph^T": t_bwd},
            "roofline": {"bound": "alu", "achieved": 8.0 * terms / dom_t * 1e-12, "peak": peak["tflops"],
                         "unit": "TFLOP/s", "frac": 8.0 * terms / dom_t * 1e-12 / peak["tflops"], "traffic": None,
                         "kernel": dom, "flop_per_term": 8.0, "peak_source": peak["source"]},
            "clocks": clocks}
    if not args.no_cpu_baseline:
        from oracle import sph as S
        freqs = f0 + df * np.arange(L)
        an = alpha.cpu().numpy()
        t0 = time.perf_counter()
        S.H_sph(geom, an, freqs[::64], qs=[0])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": float(geom.n_voxels) * len(freqs[::64]) / dt, "unit": "terms/s",
                                "cores": 1, "kind": "oracle",
                                "sample": f"1 transducer x {len(freqs[::64])} frequencies, full grid, numpy FP64, "
                                          f"{dt:.1f} s"}
    op.close()
    print(json.dumps(line), flush=True)


def run_learned(args):
    """PLS-TV time to a 1e-3 relative data residual from zero and from the learned warm start."""
    from paper_1304_2017_gb300 import warmstart
    kw = {}
    for item in filter(None, args.learned_args.split(",")):
        k, v = item.split("=")
        kw[k] = float(v) if "." in v or "e" in v else int(v)
    out = warmstart.run(**kw)
    out["metric"] = "PLS-TV GPU seconds to a 1e-3 relative data residual (zero start vs learned warm start)"
    print(json.dumps(out), flush=True)


def run_conv(args):
    """One 3x3x3 convolution of the warm start's U-Net on the tensor cores (oat_conv3d_bf16,
    tcgen05.mma): 128^3 voxels, 64 -> 64 channels (the bottleneck layer of a 512^3 input), BF16
    in and out, FP32 accumulation; TFLOP/s (2 x 27 x cin x cout FLOP per voxel) against the
    measured dense BF16 peak, CUDA events around K timed calls after W untimed ones."""
    import torch
    from paper_1304_2017_gb300 import unet
    torch.cuda.set_device(0)
    n, cin, cout = args.conv_size, 64, 64
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((n, n, n, cin), device="cuda", generator=g).to(torch.bfloat16)
    w = (0.05 * torch.randn((27, cout, cin), device="cuda", generator=g)).to(torch.bfloat16)
    b = torch.zeros(cout, device="cuda")
    y = torch.empty((n, n, n, cout), dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream

    def call():
        unet._call("oat_conv3d_bf16", n, n, n, cin, cout, unet._p(x), unet._p(w), unet._p(b), 1, unet._p(y),
                   ctypes.c_void_p(s))
    for _ in range(args.warmup):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    unet._call("oat_unet_check")
    sec = e0.elapsed_time(e1) * 1e-3 / args.steps
    # the weight gradient of the same layer (training), on the tensor cores too
    dw = torch.zeros(27 * cout * cin, device="cuda")
    db = torch.zeros(cout, device="cuda")

    def wcall():
        unet._call("oat_conv3d_wgrad", n, n, n, cin, cout, unet._p(x), unet._p(y), unet._p(dw), unet._p(db),
                   ctypes.c_void_p(s))
    for _ in range(args.warmup):
        wcall()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        wcall()
    e1.record()
    torch.cuda.synchronize()
    unet._call("oat_unet_check")
    wsec = e0.elapsed_time(e1) * 1e-3 / args.steps
    flop = 2.0 * 27 * cin * cout * n ** 3
    peaks, src = _peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    line = {"metric": "U-Net 3x3x3 convolution TFLOP/s (tcgen05, BF16 in, FP32 accumulation)",
            "value": flop / sec * 1e-12, "unit": "TFLOP/s", "seconds_per_conv": sec, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"{n}^3 voxels, {cin} -> {cout} channels, channels last"},
            "weight_gradient": {"seconds": wsec, "tflops": flop / wsec * 1e-12},
            "roofline": {"bound": "tensor", "achieved": flop / sec * 1e-12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flop / sec * 1e-12 / peak, "peak_source": f"{src} dense BF16 burst (cuBLAS)"}}
    print(json.dumps(line), flush=True)


def run_capture(n_xdcr=64):
    """The workload restricted to a few transducers, for ncu captures: 64 (rings 10, 30, 50, 64,
    70, 90, 110, 120 x views 0, 20, ..., 140; 2.9e9 interpolations per operator, ~2 GB on the
    device) or 256 (16 rings x 16 views spread over the scan), H and H^T twice."""
    import torch

    from paper_1304_2017_gb300 import oat
    from paper_1304_2017_gb300 import workloads as W
    torch.cuda.set_device(0)
    g = W.config("c2")
    if n_xdcr == 64:
        qs = [r * 180 + v for r in (10, 30, 50, 64, 70, 90, 110, 120) for v in range(0, 160, 20)]
    else:
        side = int(round(n_xdcr ** 0.5))
        qs = [int(r) * 180 + int(v) for r in np.linspace(4, 123, side).round() for v in np.linspace(0, 179, side).round()]
    sub = g.subset(qs)
    plan = oat.Plan(sub)
    alpha = torch.from_numpy(W.phantom("c2", g)).cuda()
    y = torch.from_numpy(W.random_data(sub)).cuda()
    for _ in range(2):
        plan.project(alpha)
        plan.backproject(y)
    torch.cuda.synchronize()
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-pls", action="store_true", help="skip the small PLS-TV figure of the default line")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--learned", action="store_true",
                    help="learned warm start: train the U-Net on PLS-TV targets, compare time to a 1e-3 residual")
    ap.add_argument("--learned-args", default="", help="k=v,... overrides for warmstart.run (e.g. n_train=8)")
    ap.add_argument("--fbp", action="store_true",
                    help="filtered backprojection throughput on the 256^3 / 23,040-transducer workload")
    ap.add_argument("--pls", action="store_true",
                    help="PLS-TV (FISTA-TV) time to a 1e-3 relative data residual on the 160^3 workload")
    ap.add_argument("--pls-iters", type=int, default=400, help="iteration cap of --pls")
    ap.add_argument("--lattice-weights", type=int, default=0,
                    help="1: exact strip-area lattice weights (OAT_LATTICE_EXACT_AREA) in the H / H^T bench")
    ap.add_argument("--eir", default="", choices=["", "gaussian", "bandpass"],
                    help="add a synthetic transducer response (H = H^e D G) to the H / H^T bench")
    ap.add_argument("--sph", action="store_true",
                    help="spherical-voxel model H_sph + H_sph^T on the paper's 210 x 210 x 440 grid")
    ap.add_argument("--sph-transducers", type=int, default=0, help="--sph on this many transducers (0: all)")
    ap.add_argument("--conv", action="store_true",
                    help="one tensor-core 3x3x3 convolution of the U-Net (64 -> 64 channels) on a --conv-size^3 grid")
    ap.add_argument("--conv-size", type=int, default=128)
    ap.add_argument("--capture-transducers", type=int, default=64, help="transducers of --capture (64 or a square)")
    ap.add_argument("--capture", action="store_true",
                    help="small case for ncu captures: the 256^3 workload on 64 transducers, H and H^T twice")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.capture:
        return run_capture(args.capture_transducers)
    if args.conv:
        return run_conv(args)
    if args.learned:
        return run_learned(args)
    if args.pls:
        return run_pls(args)
    if args.fbp:
        return run_fbp(args)
    if args.sph:
        return run_sph(args)

    import torch
    import torch.distributed as dist

    from paper_1304_2017_gb300 import oat
    from paper_1304_2017_gb300 import workloads as W

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    geom = W.config(args.config)
    if args.lattice_weights:
        geom = dataclasses.replace(geom, lattice_weights=args.lattice_weights)
    alpha_np = W.phantom(args.config, geom, seed=1304 + rank)
    y_np = W.random_data(geom, seed=7 + rank)
    plan = oat.Plan(geom, device=local)
    if args.eir:
        plan.set_eir(*W.eir_taps(kind=args.eir))
    st = plan.stats(count_grid_points=True)
    pts = st["points_grid"]
    alpha = torch.from_numpy(alpha_np).to(dev)
    y = torch.from_numpy(y_np).to(dev)
    u = torch.empty(plan.data_shape, dtype=torch.float32, device=dev)
    a = torch.empty(plan.vol_shape, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.project(alpha, out=u)
        plan.backproject(y, out=a)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    plan.set_profiling(True)
    plan.kernel_time(0, reset=True)
    plan.kernel_time(1, reset=True)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    plan.set_profiling(False)
    g_ms, g_n = plan.kernel_time(0, reset=True)
    b_ms, b_n = plan.kernel_time(1, reset=True)
    value, ms_max = replica_throughput(ms, pts, world, dev)

    # end to end through the public API with host buffers: pinned H2D of alpha and y, H and
    # H^T, D2H of u and alpha'
    h_alpha = torch.from_numpy(alpha_np).pin_memory()
    h_y = torch.from_numpy(y_np).pin_memory()
    h_u = torch.empty(plan.data_shape, dtype=torch.float32).pin_memory()
    h_a = torch.empty(plan.vol_shape, dtype=torch.float32).pin_memory()

    def e2e_step():
        alpha.copy_(h_alpha, non_blocking=True)
        y.copy_(h_y, non_blocking=True)
        step()
        h_u.copy_(u, non_blocking=True)
        h_a.copy_(a, non_blocking=True)

    e2e_step()
    barrier()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
    e2e_value, _ = replica_throughput(e2e_ms, pts, world, dev)
    bi = h_alpha.numel() * 4 + h_y.numel() * 4
    bo = h_u.numel() * 4 + h_a.numel() * 4

    # roofline of the dominant kernel, timed by events around its launches on the call's stream
    dom_ms, dom_name = (b_ms / max(b_n, 1), "k_brick_gather_t (H^T)") if b_ms >= g_ms else (g_ms / max(g_n, 1), "k_brick_gather (H)")
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = _sm_count(dev)
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = FLOP_PER_SAMPLE * pts / (dom_ms * 1e-3) / 1e12
    allc = _counters()
    counters = dict(allc.get(dom_name.split()[0], {}))
    counters["source"] = allc.get("source")
    traffic = counters.get("dram_bytes_per_launch")
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": traffic, "kernel": dom_name,
            "kernel_ms": dom_ms, "peak_source": f"{src} clock: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
            "flop_per_sample": FLOP_PER_SAMPLE}
    # on-chip utilisation of the dominant kernel, measured by ncu on the 64-transducer capture case
    # (profiles/counters.json, valid only for the profiled kernel sources): the fraction of issue
    # slots used and of the shared-memory pipe's one wavefront per SM clock, with the shared
    # wavefronts per sample that the second applies to
    onchip = {}
    for key in ("issue_active_pct", "shared_pipe_pct", "shared_wavefronts_per_sample",
                "warp_instructions_per_sample"):
        if counters.get(key) is not None:
            onchip[key] = counters[key]
    l2_peak = l2_read_gbs(dev)
    lts = counters.get("lts_bytes_per_launch")
    onchip["l2"] = {"peak_gbs": l2_peak, "peak_source": "measured here: oat_probe_read over a 48 MB L2-resident buffer",
                    "achieved_gbs": (lts / (dom_ms * 1e-3) / 1e9) if lts else None}
    if lts:
        onchip["l2"]["frac"] = onchip["l2"]["achieved_gbs"] / l2_peak
    onchip["counters_source"] = counters.get("source", "none valid for these kernel sources")

    variant = (", exact strip-area lattice weights" if args.lattice_weights else "") + \
              (f", {args.eir} transducer response (H = H^e D G)" if args.eir else "")
    if args.lattice_weights:
        roof["traffic"] = None          # the committed counters are of the uniform-weight kernels
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_config(geom, world), workload=WORKLOAD + variant),
            "points_per_operator": pts,
            "gpu_launches": args.steps * (LAUNCHES_PER_STEP + (1 if args.eir else 0)),
            "kernel_ms": {"k_brick_gather": g_ms / max(g_n, 1), "k_brick_gather_t": b_ms / max(b_n, 1)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
            "roofline": roof, "onchip": onchip, "clocks": clocks}
    if rank == 0 and not args.no_pls:
        try:
            line["pls_tv"] = pls_small(dev)
        except Exception as exc:  # the PLS-TV figure must not hide the operator line
            line["pls_tv"] = {"value": None, "note": f"failed: {exc}"}
    if rank == 0 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(geom, alpha_np, y_np, n_xdcr=int(os.environ.get("OAT_CPU_XDCR", "16")))
        except Exception as exc:  # the baseline must not hide the GPU line
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
