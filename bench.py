"""Benchmark of the coupled f+h stream+collide step (MLUPS and fraction of the
HBM roofline) and of its adjoint (adjoint/forward time ratio) on synthetic
inputs.

Workload (default): heated sphere in a channel, 384 x 128 x 128 nodes, sphere
diameter 32 at x = 96 (seeded sub-lattice offset), inlet u = 0.02 / T = 0,
sphere wall T = 1, zero-gradient outlet, periodic y/z; D3Q27 cumulant f and
D3Q27 CM-TRT h; nu = 0.032, Pr = 1000; populations stored in FP32 (FP16 and
BF16 storage are timed beside it).  One bench step = one lattice time step
over the whole grid (one kernel launch).  The population arrays (2 x 1.36 GB
read+written per step) are far larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank advances its own replica:
the method has no data-parallel exchange on one grid here ("replicas only").
"""
from __future__ import annotations

import argparse
import hashlib
import itertools
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS of coupled f+h step and % of HBM roofline; adjoint/forward time ratio"
WORKLOAD = dict(nx=384, ny=128, nz=128, D=32.0, cx=96.0, seed=1234, u_in=0.02, T_in=0.0, T_wall=1.0,
                nu=0.032, Pr=1000.0)
BYTES_PER_VALUE = {"f32": 4, "f64": 8, "f16": 2, "bf16": 2}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _between(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


def kernel_source_hash(csrc=None):
    """Hash of the source the timed step kernel is built from: all of
    lbm_device.cuh, and from lbm_kernels.cuh the block size, the step kernel
    with its helpers and launch_step.  Recorded DRAM traffic is reported only
    while this is unchanged."""
    csrc = csrc or os.path.join(ROOT, "paper_2203_01316_gb300", "csrc")
    dev = open(os.path.join(csrc, "lbm_device.cuh")).read()
    ker = open(os.path.join(csrc, "lbm_kernels.cuh")).read()
    parts = [dev,
             _between(ker, "constexpr int kBlock", "\n"),
             _between(ker, "#ifdef LBM_KERNEL_TU", "template <typename S, int QH>\ncudaError_t launch_step("),
             _between(ker, "cudaError_t launch_step(const Buffers& b, const DevParams& p, cudaStream_t s, bool advance_h) {",
                      "\n}\n")]
    h = hashlib.sha256()
    for t in parts:
        h.update(t.encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source is unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel_key)
    if not d or d.get("src_hash") != kernel_source_hash():
        return None
    return d.get("traffic_bytes_per_launch")


def make_workload(scale=1.0):
    from paper_2203_01316_gb300 import inputs as I
    W = WORKLOAD
    nx, ny, nz = (max(8, int(round(W[k] * scale))) for k in ("nx", "ny", "nz"))
    w = I.heated_sphere(nx, ny, nz, D=W["D"] * scale, cx=W["cx"] * scale, seed=W["seed"], u_in=W["u_in"],
                        T_in=W["T_in"])
    return w


def make_solver(w, storage, stream=None):
    from paper_2203_01316_gb300 import Solver
    nx, ny, nz = w["dims"]
    W = WORKLOAD
    s = Solver(nx, ny, nz, nu=W["nu"], Pr=W["Pr"], lat_h=27, hkind="trt", storage=storage, periodic_x=False,
               rho0=1.0, T_ref=W["T_in"], stream=stream)
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.set_bc(0, W["T_wall"])
    s.set_inlet(w["u_in"], w["T_in"])
    return s


def time_steps(s, steps, warmup, stream):
    import torch
    s.step(warmup)
    torch.cuda.synchronize()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if torch.distributed.is_initialized():
        torch.distributed.barrier()
    return e0.elapsed_time(e1) / 1e3


def replica_time(dt, device=None):
    """Timed region of the whole job: the replicas run at the same time, so
    the job ends with the slowest rank (max over ranks; dt itself when not
    distributed)."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return dt
    t = torch.tensor([dt], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, units_per_rank, steps, dt):
    """Whole-job throughput in millions of units per second: every rank
    processed units_per_rank * steps in the job time dt."""
    return world * units_per_rank * steps / dt / 1e6


def oracle_rate(budget_s, max_steps=None):
    """FP64 oracle on a scaled copy of the workload (same shape, fewer
    nodes); returns (MLUPS, cores, sample description, steps run)."""
    from oracle import oracle as O
    probe = make_workload(scale=1 / 16)
    nx, ny, nz = probe["dims"]
    W = WORKLOAD
    def run(w, steps):
        nx, ny, nz = w["dims"]
        p = O.make_params(nx=nx, ny=ny, nz=nz, qh=27, hkind="trt", periodic_x=False, nu=W["nu"],
                          k=W["nu"] / W["Pr"], u_in=w["u_in"], T_in=w["T_in"])
        o = O.Oracle(p)
        o.set_geometry(w["flags"], w["links"], nwalls=1)
        o.set_wall_temperature(0, W["T_wall"])
        o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        t = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t
        o.close()
        return dt
    dt = run(probe, 1)
    rate = nx * ny * nz / dt
    # largest scaled workload whose steps fit the budget
    scale = 1 / 16
    for sc in (1 / 2, 1 / 3, 1 / 4, 1 / 6, 1 / 8, 1 / 12, 1 / 16):
        n = (WORKLOAD["nx"] * sc) * (WORKLOAD["ny"] * sc) * (WORKLOAD["nz"] * sc)
        if n * (max_steps or 2) / rate <= budget_s:
            scale = sc
            break
    w = make_workload(scale)
    nx, ny, nz = w["dims"]
    steps = max_steps or max(1, int(budget_s * rate / (nx * ny * nz)))
    dt = run(w, steps)
    sample = (f"heated-sphere channel scaled by {scale:.4g}: {nx}x{ny}x{nz} nodes, sphere D="
              f"{WORKLOAD['D'] * scale:.3g}, {steps} oracle steps (FP64, OpenMP)")
    return nx * ny * nz * steps / dt / 1e6, O.num_threads(), sample, steps, dt


def oracle_single_thread_rate(budget_s):
    """The oracle on one host thread (the 1/16-scale heated sphere, 24x8x8,
    as many steps as fit the budget): MLUPS and the sample."""
    from oracle import oracle as O
    w = make_workload(scale=1 / 16)
    nx, ny, nz = w["dims"]
    W = WORKLOAD
    threads = O.num_threads()
    O.set_num_threads(1)
    try:
        p = O.make_params(nx=nx, ny=ny, nz=nz, qh=27, hkind="trt", periodic_x=False, nu=W["nu"],
                          k=W["nu"] / W["Pr"], u_in=w["u_in"], T_in=w["T_in"])
        o = O.Oracle(p)
        o.set_geometry(w["flags"], w["links"], nwalls=1)
        o.set_wall_temperature(0, W["T_wall"])
        o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        t = time.perf_counter()
        o.step(1)
        one = time.perf_counter() - t
        steps = max(1, int(budget_s / max(one, 1e-6)))
        t = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t
        o.close()
    finally:
        O.set_num_threads(threads)
    return nx * ny * nz * steps / dt / 1e6, f"{nx}x{ny}x{nz} nodes, {steps} oracle steps (FP64, 1 thread)"


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    # each reference step is one oracle step on a scaled copy of the workload,
    # sized so W + K steps take about a minute of host time
    from oracle import oracle as O  # noqa: F811
    budget = 60.0
    probe = make_workload(scale=1 / 16)
    nx, ny, nz = probe["dims"]
    p = O.make_params(nx=nx, ny=ny, nz=nz, periodic_x=False, nu=WORKLOAD["nu"], k=WORKLOAD["nu"] / WORKLOAD["Pr"],
                      u_in=probe["u_in"], T_in=probe["T_in"])
    o = O.Oracle(p)
    o.set_geometry(probe["flags"], probe["links"], nwalls=1)
    o.init_fields(probe["rho"], probe["u"].reshape(-1), probe["T"])
    t = time.perf_counter(); o.step(1); rate = nx * ny * nz / (time.perf_counter() - t)
    o.close()
    per_step = budget * rate / max(1, args.steps + args.warmup)
    scale = 1 / 16
    for sc in (1 / 2, 1 / 3, 1 / 4, 1 / 6, 1 / 8, 1 / 12, 1 / 16, 1 / 24, 1 / 32):
        if (WORKLOAD["nx"] * sc) * (WORKLOAD["ny"] * sc) * (WORKLOAD["nz"] * sc) <= per_step:
            scale = sc
            break
    w = make_workload(scale)
    nx, ny, nz = w["dims"]
    p = O.make_params(nx=nx, ny=ny, nz=nz, periodic_x=False, nu=WORKLOAD["nu"], k=WORKLOAD["nu"] / WORKLOAD["Pr"],
                      u_in=w["u_in"], T_in=w["T_in"])
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, WORKLOAD["T_wall"])
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    value = nx * ny * nz * args.steps / dt / 1e6
    sample = f"heated-sphere channel scaled by {scale:.4g}: {nx}x{ny}x{nz} nodes per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(),
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(w=None, storage="f32"):
    W = WORKLOAD
    nx, ny, nz = w["dims"] if w is not None else (W["nx"], W["ny"], W["nz"])
    D = w["D"] if w is not None else W["D"]
    traffic = nx * ny * nz * 2 * 54 * BYTES_PER_VALUE[storage] / 1e9
    return {"workload": f"heated sphere channel {nx}x{ny}x{nz}, D={D:g}, "
                        f"D3Q27 cumulant f + D3Q27 CM-TRT h, IBB/IABB, Pr={W['Pr']:g}",
            "grid": [nx, ny, nz], "storage": storage, "lattice": "D3Q27/D3Q27",
            "parallelism": "replicas",
            "l2": f"inputs larger than L2 ({traffic:.2f} GB population traffic per step)"}


def measure_adjoint(w, stream, fwd_ms, steps=200, every=50, accuracy=True):
    """Adjoint/forward time ratio: J = surface heat flux of the sphere summed
    over the last fifth of `steps` steps; backward = restore the checkpoint
    of each segment, recompute its velocities (f only), run the adjoint
    kernel level by level (paper_2203_01316_gb300.autograd)."""
    import torch
    from paper_2203_01316_gb300.autograd import thermal_objective
    s = make_solver(w, "f32", stream=stream.cuda_stream)
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    N = w["flags"].size
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    theta = torch.zeros(N, dtype=torch.float64, device="cuda", requires_grad=True)
    Tw = torch.tensor([WORKLOAD["T_wall"]], dtype=torch.float64, requires_grad=True)
    obj = s.objective("surface", 0, 1.0)
    window = (steps - steps // 5, steps)
    # one untimed pass: device buffers and kernel modules come up here
    Jw = thermal_objective(theta, Tw, s, state0, steps, window, obj, every=every)
    Jw.backward()
    theta.grad = None
    Tw.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = thermal_objective(theta, Tw, s, state0, steps, window, obj, every=every)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    s.close()
    bwd = (t2 - t1) / steps * 1e3
    out = {"steps": steps, "checkpoint_every": every, "objective": "sphere surface heat flux, last 20% of steps",
           "forward_with_checkpoints_ms_per_step": (t1 - t0) / steps * 1e3,
           "backward_ms_per_step": bwd, "forward_ms_per_step": fwd_ms, "ratio": bwd / fwd_ms,
           "dJ_dTwall": float(Tw.grad[0]), "grad_theta_norm": float(theta.grad.norm())}
    if accuracy:
        out["fp32_per_entry"] = adjoint_per_entry_accuracy(w, stream, theta.grad.detach().clone(),
                                                           float(Tw.grad[0]), steps, every)
    return out


def adjoint_per_entry_accuracy(w, stream, g32, dTw32, steps, every):
    """Per-entry error of the FP32 gradient dJ/dtheta against the same
    adjoint run in FP64 storage and arithmetic (which agrees per entry with
    central differences of J to 1e-6): quantiles of |g32 - g64| / |g64| over
    the nodes with g64 != 0, and over those with |g64| >= 1e-3 max|g64|."""
    import torch
    from paper_2203_01316_gb300.autograd import thermal_objective
    t0 = time.perf_counter()
    s = make_solver(w, "f64", stream=stream.cuda_stream)
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    N = w["flags"].size
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    theta = torch.zeros(N, dtype=torch.float64, device="cuda", requires_grad=True)
    Tw = torch.tensor([WORKLOAD["T_wall"]], dtype=torch.float64, requires_grad=True)
    J = thermal_objective(theta, Tw, s, state0, steps, (steps - steps // 5, steps), s.objective("surface", 0, 1.0),
                          every=every)
    J.backward()
    torch.cuda.synchronize()
    s.close()
    g64 = theta.grad.detach()
    a64 = g64.abs()
    nz = a64 > 0
    rel = ((g32 - g64).abs() / a64.clamp_min(1e-300))[nz]
    large = (a64 >= 1e-3 * a64.max())[nz]
    qs = torch.tensor([0.5, 0.9, 0.99], dtype=torch.float64, device=rel.device)

    def summary(r):
        q = torch.quantile(r, qs).tolist() if r.numel() <= (1 << 24) else [float("nan")] * 3
        return {"entries": int(r.numel()), "within_1e-4": float((r <= 1e-4).double().mean()),
                "median": q[0], "p90": q[1], "p99": q[2], "max": float(r.max())}

    dTw64 = float(Tw.grad[0])
    return {"reference": "the same adjoint in FP64 storage", "all_nonzero": summary(rel),
            "above_1e-3_max": summary(rel[large]), "dJ_dTwall_rel_error": abs(dTw32 - dTw64) / abs(dTw64),
            "seconds": round(time.perf_counter() - t0, 1)}


def measure_flow_adjoint(w, stream, fwd_ms, steps=100, every=25):
    """Cost of the coupled f + h adjoint (gradients also with respect to the
    body force and the inlet velocity) on the same objective as
    measure_adjoint: backward time per step against the forward step."""
    import torch
    from paper_2203_01316_gb300.autograd import flow_objective
    s = make_solver(w, "f32", stream=stream.cuda_stream)
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    N = w["flags"].size
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    theta = torch.zeros(N, dtype=torch.float64, device="cuda", requires_grad=True)
    Tw = torch.tensor([WORKLOAD["T_wall"]], dtype=torch.float64, requires_grad=True)
    F = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    uin = torch.tensor(w["u_in"], dtype=torch.float64, requires_grad=True)
    obj = s.objective("surface", 0, 1.0)
    window = (steps - steps // 5, steps)
    Jw = flow_objective(theta, Tw, F, uin, s, state0, 10, (8, 10), obj, every=5)  # warm-up
    Jw.backward()
    for t in (theta, Tw, F, uin):
        t.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = flow_objective(theta, Tw, F, uin, s, state0, steps, window, obj, every=every)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    s.close()
    bwd = (t2 - t1) / steps * 1e3
    return {"steps": steps, "checkpoint_every": every, "objective": "sphere surface heat flux, last 20% of steps",
            "backward_ms_per_step": bwd, "forward_ms_per_step": fwd_ms, "ratio": bwd / fwd_ms,
            "dJ_du_in": uin.grad.tolist(), "dJ_dF": F.grad.tolist(),
            "dJ_dTwall": float(Tw.grad[0])}


def flow_adjoint_study(args):
    import torch
    from paper_2203_01316_gb300 import build
    build.build()
    stream = torch.cuda.Stream()
    w = make_workload(args.scale)
    s = make_solver(w, "f32", stream=stream.cuda_stream)
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    dt = time_steps(s, 200, 20, stream)
    s.close()
    r = measure_flow_adjoint(w, stream, dt / 200 * 1e3, steps=args.adjoint_steps)
    print(json.dumps({"flow_adjoint": r, "workload": _config(w, "f32")["workload"]}), flush=True)


def precision_study(args):
    """Precision form of the heated sphere (Pr = 1000): populations stored
    in FP16 / BF16 (stochastic and nearest rounding) / FP32 with FP32
    arithmetic against the FP64 path, after
    `steps` steps: relative L2 error of u and T over the fluid nodes and the
    relative error of the sphere's Nusselt number averaged over the last 10%
    of the steps.  scale 1: 384x128x128 (D = 32) against the FP64 GPU path;
    --precision-crop: 96x32x32 (D = 8) against the FP64 oracle."""
    import torch
    from paper_2203_01316_gb300 import build
    build.build()
    stream = torch.cuda.Stream()
    scale = 0.25 if args.precision_crop else args.scale
    w = make_workload(scale)
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    D = w["D"]
    fluid = np.asarray(w["flags"]) == 0
    steps = args.steps
    win = max(1, steps // 10)
    k = WORKLOAD["nu"] * scale / WORKLOAD["Pr"]   # nu = U D / Re scales with D
    nu = WORKLOAD["nu"] * scale
    area = math.pi * D * D
    out = {}

    def run(storage, round_nearest=False):
        from paper_2203_01316_gb300 import Solver
        s = Solver(nx, ny, nz, nu=nu, k=k, lat_h=27, hkind="trt", storage=storage, periodic_x=False,
                   rho0=1.0, T_ref=WORKLOAD["T_in"], stream=stream.cuda_stream, round_nearest=round_nearest)
        s.set_geometry(w["flags"], w["links"], n_walls=1)
        s.set_bc(0, WORKLOAD["T_wall"])
        s.set_inlet(w["u_in"], w["T_in"])
        s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        obj = s.objective("surface", 0, D / (k * area * (WORKLOAD["T_wall"] - WORKLOAD["T_in"])) / win)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(steps - win)
        for _ in range(win):
            s.objective_accumulate(obj, J)
            s.step(1)
        rho, u, T = s.macros()
        dt = time.perf_counter() - t0
        Nu = float(J.item())
        s.close()
        return u, T, Nu, dt

    if args.precision_crop:
        from oracle import oracle as O
        O.build()
        p = O.make_params(nx=nx, ny=ny, nz=nz, qh=27, hkind="trt", periodic_x=False, nu=nu, k=k,
                          u_in=w["u_in"], T_in=w["T_in"])
        o = O.Oracle(p)
        o.set_geometry(w["flags"], w["links"], nwalls=1)
        o.set_wall_temperature(0, WORKLOAD["T_wall"])
        o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        # the GPU stores post-collision states; the oracle's level t is its
        # state after t steps, collided once more for the flux of t -> t+1
        o.step(steps - win)
        Nu_ref = 0.0
        for _ in range(win):
            Nu_ref += o.surface_flux(0) * D / (k * area * (WORKLOAD["T_wall"] - WORKLOAD["T_in"])) / win
            o.step(1)
        _, u_ref, T_ref = o.macros()
        ref = "FP64 oracle"
    else:
        u_ref, T_ref, Nu_ref, _ = run("f64")
        ref = "FP64 GPU path"
    for name, storage, rn in (("f32", "f32", False), ("f16", "f16", False), ("f16_round_nearest", "f16", True),
                              ("bf16", "bf16", False), ("bf16_round_nearest", "bf16", True)):
        u, T, Nu, dt = run(storage, rn)
        out[name] = {
            "rel_l2_u": float(np.sqrt(np.sum((u[:, fluid] - u_ref[:, fluid]) ** 2) / np.sum(u_ref[:, fluid] ** 2))),
            "rel_l2_T": float(np.sqrt(np.sum((T[fluid] - T_ref[fluid]) ** 2) / np.sum(T_ref[fluid] ** 2))),
            "Nu": Nu, "Nu_rel_err": abs(Nu - Nu_ref) / abs(Nu_ref)}
    line = {"precision_study": f"heated sphere {nx}x{ny}x{nz}, D={D:g}, Pr={WORKLOAD['Pr']:g}, {steps} steps",
            "reference": ref, "Nu_ref": Nu_ref, "Nu_window_steps": win, "results": out}
    print(json.dumps(line), flush=True)


def porous_study(args):
    """Porous bed: 512x256x256 (33.5M nodes), 200 spheres with D uniform in
    [12, 24], IBB/IABB with T_w = 1, inlet u = 0.01, Pr = 1000, D3Q27
    cumulant f + D3Q7 CM-TRT h, FP32 and FP16 storage.  MLUPS and roofline
    fraction of the step; then `spin` forward steps and a 1000-step adjoint of
    the heat flux through the plane x = nx-2 (summed over the last 100
    levels) with respect to theta, checkpoints every 50 steps."""
    import torch
    from paper_2203_01316_gb300 import Solver, build, inputs as I
    from paper_2203_01316_gb300.autograd import thermal_objective
    build.build()
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    w = I.porous_bed(seed=WORKLOAD["seed"])
    t_geom = time.perf_counter() - t0
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    n_active = int(np.count_nonzero(np.asarray(w["flags"]) != 1))
    nu, Pr = 0.01, 1000.0
    hbm, src = peaks()
    out = {"workload": f"porous bed {nx}x{ny}x{nz}, {len(w['radii'])} spheres D in [12,24], D3Q27 f + "
                       f"D3Q7 CM-TRT h, IBB/IABB, Pr={Pr:g}", "nodes": N, "solid_fraction": 1 - n_active / N,
           "wall_links": int(len(w["links"]["node"])), "geometry_build_s": t_geom}
    for storage in ("f32", "f16"):
        s = Solver(nx, ny, nz, nu=nu, Pr=Pr, lat_h=7, hkind="trt", storage=storage, periodic_x=False,
                   T_ref=w["T_in"], stream=stream.cuda_stream)
        t0 = time.perf_counter()
        s.set_geometry(w["flags"], w["links"], n_walls=1)
        t_set = time.perf_counter() - t0
        s.set_bc(0, 1.0)
        s.set_inlet(w["u_in"], w["T_in"])
        s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        dt = time_steps(s, args.steps, args.warmup, stream)
        alg = n_active * 2 * (27 + 7) * BYTES_PER_VALUE[storage]
        ach = alg / (dt / args.steps) / 1e9
        r = {"MLUPS": N * args.steps / dt / 1e6, "ms_per_step": dt / args.steps * 1e3, "achieved_GBs": ach,
             "frac": ach / hbm, "set_geometry_s": t_set}
        if storage == "f32" and args.adjoint_steps > 0:
            s.step(args.spin)
            torch.cuda.synchronize()
            state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
            theta = torch.zeros(N, dtype=torch.float64, device="cuda", requires_grad=True)
            Tw = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
            obj = s.objective("section", nx - 2, 1.0)
            n = args.adjoint_steps
            every = 50
            torch.cuda.reset_peak_memory_stats()
            tf = time.perf_counter()
            J = thermal_objective(theta, Tw, s, state0, n, (n - 99, n), obj, every=every)
            torch.cuda.synchronize()
            tb = time.perf_counter()
            J.backward()
            torch.cuda.synchronize()
            te = time.perf_counter()
            free, total = torch.cuda.mem_get_info()
            # memory of the checkpointed adjoint: one saved state per segment,
            # the velocity records of one segment, the adjoint state (two h
            # arrays) and the FP64 gradient, against the device's own count
            ss = s.state_size()
            plan = {"checkpoints_GB": -(-n // every) * ss / 1e9, "segment_velocity_records_GB": every * 3 * N * 4 / 1e9,
                    "adjoint_state_GB": (2 * 7 * N * 4 + 8 * N) / 1e9,
                    "solver_state_GB": 2 * 34 * N * BYTES_PER_VALUE[storage] / 1e9}
            plan["planned_total_GB"] = sum(plan.values())
            plan["torch_peak_allocated_GB"] = torch.cuda.max_memory_allocated() / 1e9
            plan["device_used_GB_mem_get_info"] = (total - free) / 1e9
            plan["device_total_GB"] = total / 1e9
            r["adjoint"] = {"steps": n, "checkpoint_every": 50, "spin_up_steps": args.spin,
                            "objective": "heat flux through x = nx-2, last 100 levels",
                            "forward_ms_per_step": (tb - tf) / n * 1e3, "backward_ms_per_step": (te - tb) / n * 1e3,
                            "ratio": (te - tb) / n * 1e3 / r["ms_per_step"], "J": float(J.item()),
                            "grad_theta_norm": float(theta.grad.norm()), "memory": plan,
                            "note": "first (cold) adjoint call: includes allocation of checkpoint buffers"}
        out[storage] = r
        s.close()
    print(json.dumps(out), flush=True)


def sphere_nusselt_study(args):
    """The heated sphere in a channel (192x64x64, D = 16 with a seeded
    sub-node centre offset, plug inlet u = 0.02, T_in = 0, T_w = 1, Re = 20:
    nu = 0.016; --scale s multiplies the grid and D), D3Q27 cumulant f + D3Q27
    CM-TRT h (--kinds) with Eq. IBB / Eq. IABB,
    for Pr = 10, 100, 1000 over `steps` steps (default 20k): the sphere's
    Nusselt number Nu = q D / (k pi D^2 (T_w - T_in)) (the Sec. 4.4
    definition with the sphere's area, reading R10), averaged over the last
    10% of the steps on the device, in FP32 storage and, as a cross-check, in
    FP64 storage."""
    import torch
    from paper_2203_01316_gb300 import Solver, build, inputs as I
    build.build()
    stream = torch.cuda.Stream()
    sc = args.scale  # 2: the same channel at twice the resolution (384x128x128, D = 32)
    D, U, Re = 16.0 * sc, 0.02, 20.0
    nu = U * D / Re
    w = I.heated_sphere(int(round(192 * sc)), int(round(64 * sc)), int(round(64 * sc)), D=D, cx=48.0 * sc,
                        seed=WORKLOAD["seed"], u_in=U, T_in=0.0)
    nx, ny, nz = w["dims"]
    steps = args.steps
    win = max(1, steps // 10)
    out = {"nusselt_study": f"heated sphere {nx}x{ny}x{nz}, D={D:g}, Re={Re:g}, nu={nu:g}, {steps} steps, "
                            f"Nu averaged over the last {win} steps", "results": {}}
    kinds = (args.kinds or "trt").split(",")
    storages = (args.storages or "f32,f64").split(",")
    for Pr, kind in itertools.product([float(v) for v in (args.prs or "10,100,1000").split(",")], kinds):
        k = nu / Pr
        r = {"k": k, "h_kind": kind}
        for storage in storages:
            s = Solver(nx, ny, nz, nu=nu, k=k, lat_h=27, hkind=kind, storage=storage, periodic_x=False,
                       T_ref=w["T_in"], stream=stream.cuda_stream)
            s.set_geometry(w["flags"], w["links"], n_walls=1)
            s.set_bc(0, 1.0)
            s.set_inlet(w["u_in"], w["T_in"])
            s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
            J = torch.zeros(1, dtype=torch.float64, device="cuda")
            obj = s.objective("surface", 0, D / (k * math.pi * D * D * 1.0) / win)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(steps - win)
            half = torch.zeros(1, dtype=torch.float64, device="cuda")
            for i in range(win):
                s.objective_accumulate(obj, J)
                if i == win // 2 - 1:
                    with torch.cuda.stream(stream):  # ordered after the accumulation
                        half.copy_(J)
                s.step(1)
            try:
                mass, energy = s.balances()
            except Exception as e:  # a kind that is unstable on this mesh: say so and go on
                r[storage] = {"diverged": str(e)}
                s.close()
                continue
            dt = time.perf_counter() - t0
            Nu = float(J.item())
            # drift check: the mean over the window's second half against its first half
            first, second = 2.0 * float(half.item()), 2.0 * (Nu - float(half.item()))
            r[storage] = {"Nu": Nu, "Nu_first_half_of_window": first, "Nu_second_half_of_window": second,
                          "wall_s": dt, "MLUPS": nx * ny * nz * steps / dt / 1e6, "mass": mass}
            s.close()
        if "Nu" in r.get("f32", {}) and "Nu" in r.get("f64", {}):
            r["Nu_f32_vs_f64"] = abs(r["f32"]["Nu"] - r["f64"]["Nu"]) / abs(r["f64"]["Nu"])
        out["results"][f"Pr={Pr:g} {kind}"] = r
        print(json.dumps({f"Pr={Pr:g} {kind}": r}), flush=True)
    print(json.dumps(out), flush=True)


def validation_cylinders(args):
    """Sec. 4.3: steady conduction between concentric cylinders (inner
    diameter D/2 at T = 1, outer D at T = 0, k = 0.1, CM-TRT, no flow) on the
    GPU path (FP64 storage), against T(r) = 1 - ln(r/r_in)/ln(r_out/r_in),
    for Eq. IABB, ABB and EQ walls over D = 16 ... 128: normalised L2 error
    and observed order between successive grids."""
    import torch  # noqa: F401
    from paper_2203_01316_gb300 import Solver, build, inputs as I
    build.build()
    Ds = [int(d) for d in args.sizes.split(",")] if args.sizes else [16, 32, 64, 128]
    k = 0.1
    out = {}
    for bc in ("iabb", "abb", "eq"):
        errs = []
        for D in Ds:
            w = I.concentric_cylinders(D)
            n = w["dims"][0]
            s = Solver(n, n, 1, nu=1.0 / 6.0, k=k, lat_h=27, hkind="trt", storage="f64", periodic_x=True,
                       T_ref=0.5, wall_bc=bc)
            s.set_geometry(w["flags"], w["links"], n_walls=2)
            s.set_bc(0, 1.0)
            s.set_bc(1, 0.0)
            s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
            steps = int(12 * (D / 4.0) ** 2 / k) + 200  # about twelve diffusion times across the gap
            s.step(steps)
            _, _, T = s.macros()
            s.close()
            fl = np.asarray(w["flags"]) == 0
            r = w["r"][fl]
            Ta = 1.0 - np.log(r / w["R_inner"]) / np.log(w["R_outer"] / w["R_inner"])
            errs.append(float(np.sqrt(np.sum((Ta - T[fl]) ** 2) / np.sum(Ta ** 2))))
        orders = [math.log(errs[i] / errs[i + 1]) / math.log(Ds[i + 1] / Ds[i]) for i in range(len(Ds) - 1)]
        out[bc] = {"D": Ds, "L2": errs, "observed_order": orders}
    line = {"validation": "concentric cylinders (Sec. 4.3), CM-TRT, k = 0.1, FP64 storage", "results": out}
    print(json.dumps(line), flush=True)
    return line


def lattice_convolution(T0, n, u=(0.0, 0.0)):
    """n steps of T(x) <- sum_a h^eq_a(T(x - e_a), u) on a periodic L x L
    plane: the D3Q27 h step at s^H = 1 (every kind collapses to its
    equilibrium), applied as a product of 1-D transfer functions (Sec. 2.1,
    product-form discrete equilibrium with c_s^2 = 1/3) by FFT in FP64."""
    Ly, Lx = T0.shape
    def sym(L, v):
        th = np.fft.fftfreq(L) * 2.0 * np.pi
        a = 1.0 / 3.0 + v * v
        return (1.0 - a) + 0.5 * (a + v) * np.exp(-1j * th) + 0.5 * (a - v) * np.exp(1j * th)
    G = np.outer(sym(Ly, u[1]), sym(Lx, u[0]))
    return np.real(np.fft.ifft2(np.fft.fft2(T0) * G ** n))


def hill_closed_form(L, s0, k, n, ux):
    """Sec. 4.1 closed form in 2-D (N = 2), centre advected by u_x n and
    wrapped into the periodic box, with the nearest periodic images."""
    yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    s2 = s0 + 2.0 * k * n
    cx = (L / 2.0 + ux * n) % L
    C = np.zeros((L, L))
    for ix in (-1, 0, 1):
        for iy in (-1, 0, 1):
            C += (s0 / s2) * np.exp(-((xx - cx + ix * L) ** 2 + (yy - L / 2.0 + iy * L) ** 2) / (2.0 * s2))
    return C


def validation_hill(args):
    """Sec. 4.1: advection-diffusion of a Gaussian hill on a periodic
    256 x 256 x 1 box (sigma0^2 = 100, t_SI = 100, k_SI = 4, so n = 400/k
    steps), at rest and at u_x = 0.1 (lattice units), for every h kind and
    k from 1/6 down; normalised L2 error of the hill C = T - 1 against the
    closed form, in FP64 (k >= 1e-3: the scheme's own error) and in FP32
    (every k).  At k = 1/6 the FP32 result is also compared with the exact
    lattice convolution the step reduces to there."""
    import torch  # noqa: F401
    from paper_2203_01316_gb300 import Solver, build, inputs as I
    build.build()
    L, s0 = 256, 100.0
    ks = [float(v) for v in args.sizes.split(",")] if args.sizes else [1.0 / 6.0, 1e-2, 1e-3, 1e-4]
    out, lat = {}, {}
    storages = args.storages.split(",") if args.storages else ["f64", "f32"]
    for storage, kind, ux in itertools.product(storages, ("trt", "srt", "1st", "cum1st"), (0.0, 0.1)):
        key = f"{storage}, {kind}, u_x = {ux:g}"
        out[key] = {}
        for k in ks:
            if storage == "f64" and k < 1e-3:
                continue  # 4e6 FP64 steps: about 15 minutes per run on GB300
            n = int(round(400.0 / k))
            w = I.gaussian_hill(L, s0)
            w["u"][0] = ux
            s = Solver(L, L, 1, nu=1.0 / 6.0, k=k, lat_h=27, hkind=kind, storage=storage, periodic_x=True,
                       T_ref=1.0)
            s.set_geometry(w["flags"], None)
            s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
            t0 = time.perf_counter()
            s.step(n)
            _, _, T = s.macros()
            dt = time.perf_counter() - t0
            s.close()
            Cn = T.reshape(L, L) - 1.0
            Ca = hill_closed_form(L, s0, k, n, ux)
            out[key][f"{k:.4g}"] = float(np.sqrt(np.sum((Ca - Cn) ** 2) / np.sum(Ca ** 2)))
            if k == 1.0 / 6.0 and storage == "f32":
                Cl = lattice_convolution(w["T"].reshape(L, L) - 1.0, n, (ux, 0.0))
                lat[key] = float(np.abs(Cl - Cn).max())
            print(f"# {key} k={k:.4g} n={n} {dt:.1f}s L2={out[key][f'{k:.4g}']:.3e}", file=sys.stderr, flush=True)
    line = {"validation": "Gaussian hill (Sec. 4.1), 256x256x1, sigma0^2 = 100, n = 400/k steps",
            "L2": out, "k=1/6: max |C - lattice convolution|": lat}
    print(json.dumps(line), flush=True)
    return line


def confined_nu(S, kind, wall_bc, Pr, storage="f32", max_flow_throughs=4.0, tol=2e-3, xc=None, inlet_bc="zou_he"):
    """Sec. 4.4 confined cylinder on the GPU path: steps until the heat flux
    through the cylinder surface (q_s, Eq. heat_flux_thorough_heater) and the
    heat carried through the outlet section minus the inlet section (q_x,
    Eq. heat_flux_section, sections 50 S and 100 S from the planes) agree to
    tol and the Nusselt number has stopped changing, or until
    max_flow_throughs times L/U steps.  Nu = q D / (k A dT) with A = pi D
    (per unit depth), q the mean of q_s and q_x."""
    from paper_2203_01316_gb300 import Solver, inputs as I
    w = I.confined_cylinder(S, xc=xc)
    nx, ny, nz = w["dims"]
    nu = 0.03
    k = nu / Pr
    s = Solver(nx, ny, nz, nu=nu, k=k, lat_h=27, hkind=kind, storage=storage, periodic_x=False,
               T_ref=w["T_in"], wall_bc=wall_bc, inlet_bc=inlet_bc)
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.set_bc(0, w["T_cyl"])
    s.set_inlet(w["u_in"], w["T_in"])
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    U = w["u_in"][0]
    through = int(nx / U)
    chunk = max(1000, through // 40)
    xin, xout = w["sections"]
    dT = w["T_cyl"] - w["T_in"]
    steps, nu_prev = 0, None
    t0 = time.perf_counter()
    while True:
        s.step(chunk)
        steps += chunk
        qs = s.surface_flux(0)
        qx = s.section_flux(xout) - s.section_flux(xin)
        q = 0.5 * (qs + qx)
        Nu = q / (k * math.pi * dT)
        mism = abs(qs - qx) / max(abs(qs), 1e-30)
        done = (mism < tol and nu_prev is not None and abs(Nu - nu_prev) < 1e-4 * abs(Nu)
                and steps >= through)
        if done or steps >= max_flow_throughs * through or not math.isfinite(Nu):
            break
        nu_prev = Nu
    dt = time.perf_counter() - t0
    s.close()
    return {"Nu": Nu, "q_surface": qs, "q_x": qx, "mismatch": mism, "steps": steps, "converged": bool(done),
            "seconds": round(dt, 1), "MLUPS": round(nx * ny * nz * steps / dt / 1e6)}


def validation_confined(args):
    """Sec. 4.4 Nusselt-number table: four h kernels x first-order (BB + EQ)
    and second-order (Eq. IBB + Eq. IABB) walls x Pr in {10, 100, 1000} on the
    meshes S given by --sizes (default 1: 1000 x 150, D = 30, U = 0.01,
    nu = 0.03, Re = 10), FP32 storage with T_ref = T_in."""
    import torch  # noqa: F401
    from paper_2203_01316_gb300 import build
    build.build()
    Ss = [float(v) if "." in v else int(v) for v in args.sizes.split(",")] if args.sizes else [1]
    kinds = args.kinds.split(",") if args.kinds else ["1st", "srt", "trt", "cum1st"]
    prs = [float(v) for v in args.prs.split(",")] if args.prs else [10.0, 100.0, 1000.0]
    out = []
    for S in Ss:
        for Pr in prs:
            for kind in kinds:
                for order, bc in (("1st", "eq"), ("2nd", "iabb")):
                    if args.orders and order not in args.orders.split(","):
                        continue
                    r = confined_nu(S, kind, bc, Pr, inlet_bc=args.inlet, max_flow_throughs=args.flow_throughs)
                    r.update({"S": S, "Pr": Pr, "kernel": kind, "bc_order": order})
                    out.append(r)
                    print("# " + json.dumps(r), file=sys.stderr, flush=True)
    line = {"validation": f"confined cylinder Nu (Sec. 4.4), Re = 10, FP32, {args.inlet} inlet", "results": out}
    print(json.dumps(line), flush=True)
    return line


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2203_01316_gb300 import build
    build.build()
    # a dedicated stream: the library launches on it and the events bracket it
    stream = torch.cuda.Stream()
    w = make_workload(args.scale)
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    flags = np.asarray(w["flags"])
    n_active = int(np.count_nonzero(flags != 1))
    s = make_solver(w, args.storage, stream=stream.cuda_stream)
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    with ClockSampler(local) as clk:
        dt = time_steps(s, args.steps, args.warmup, stream)
    dt = replica_time(dt, device="cuda")
    mass, energy = s.balances()  # also checks that nothing diverged
    value = replica_value(ws, N, args.steps, dt)
    ms = dt / args.steps * 1e3
    bpv = BYTES_PER_VALUE[args.storage]
    alg_bytes = n_active * 2 * (27 + 27) * bpv
    hbm, src = peaks()
    achieved = alg_bytes / (dt / args.steps) / 1e9
    kname = {"f32": "float", "f64": "double", "f16": "__half", "bf16": "__nv_bfloat16"}[args.storage]
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_source": src, "kernel": f"k_step<{kname},27>",
            "traffic": recorded_traffic(f"k_step_{args.storage}_q27_{nx}x{ny}x{nz}"),
            "algorithmic_bytes_per_launch": alg_bytes}
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic", "config": _config(w, args.storage),
            "fluid_mlups": replica_value(ws, n_active, args.steps, dt),
            "roofline": roof, "gpu_launches": args.steps, "clocks": clk.summary(),
            "balances": {"mass": mass, "energy": energy}}
    if args.no_extras:
        if rank == 0:
            print(json.dumps(line), flush=True)
        s.close()
        return

    # end to end through the public API with host buffers: fields from pinned
    # host memory -> K steps -> macroscopic fields back to pinned host memory
    rho_h = torch.from_numpy(w["rho"]).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(w["u"].reshape(-1))).pin_memory()
    T_h = torch.from_numpy(w["T"]).pin_memory()
    out = [torch.empty(N, dtype=torch.float64).pin_memory(), torch.empty(3 * N, dtype=torch.float64).pin_memory(),
           torch.empty(N, dtype=torch.float64).pin_memory()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.init_fields(rho_h.numpy(), u_h.numpy(), T_h.numpy())
    s.step(args.steps)
    r = s.L.lbm_macros(s._h, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), 0)
    t1 = time.perf_counter()
    if r != 0:
        raise RuntimeError("lbm_macros failed in the end-to-end run")
    e2e = {"value": N * args.steps / (t1 - t0) / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 5 * N * 8 / args.steps, "d2h_bytes_per_step": 5 * N * 8 / args.steps,
           "job": f"lbm_init_fields(host) + lbm_step({args.steps}) + lbm_macros(host)"}
    s.close()
    del s

    variants = {}
    vsteps = max(10, args.steps // 3)
    for storage in ("f16", "bf16"):
        sv = make_solver(w, storage, stream=stream.cuda_stream)
        sv.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        dtv = time_steps(sv, vsteps, max(3, args.warmup // 3), stream)
        bv = n_active * 2 * 54 * BYTES_PER_VALUE[storage]
        variants[storage] = {"value": N * vsteps / dtv / 1e6, "unit": "MLUPS", "steps": vsteps,
                             "achieved_GBs": bv / (dtv / vsteps) / 1e9,
                             "frac": bv / (dtv / vsteps) / 1e9 / hbm}
        sv.close()

    line["e2e"] = e2e
    line["storage_variants"] = variants
    line["adjoint"] = measure_adjoint(w, stream, ms, steps=args.adjoint_steps)
    if args.flow_adjoint_steps > 0:  # the coupled f + h adjoint (gradients for F and u_in too)
        line["flow_adjoint"] = measure_flow_adjoint(w, stream, ms, steps=args.flow_adjoint_steps)
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        v, cores, sample, steps, odt = oracle_rate(budget_s=args.cpu_budget)
        v1, sample1 = oracle_single_thread_rate(budget_s=min(5.0, args.cpu_budget / 3))
        line["cpu_baseline"] = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample,
                                "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1, "sample": sample1}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="scale the workload grid (profiling of a smaller case)")
    ap.add_argument("--storage", choices=["f32", "f64", "f16", "bf16"], default="f32")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--flow-adjoint-steps", type=int, default=100,
                    help="levels of the coupled-adjoint leg of the bench line (0: skip it)")
    ap.add_argument("--flow-adjoint", action="store_true",
                    help="time the coupled f + h adjoint (gradients for F and u_in) on the workload")
    ap.add_argument("--storages", default="", help="validation hill, nusselt study: comma-separated storages")
    ap.add_argument("--kinds", default="", help="validation confined, nusselt study: comma-separated h kinds")
    ap.add_argument("--prs", default="", help="validation confined: comma-separated Prandtl numbers")
    ap.add_argument("--orders", default="", help="validation confined: wall-rule orders, '1st', '2nd' or both")
    ap.add_argument("--inlet", default="zou_he", choices=["zou_he", "equilibrium"],
                    help="validation confined: inlet plane rule")
    ap.add_argument("--validation", choices=["cylinders", "hill", "confined"],
                    help="run one of the paper's validation workloads on the GPU path")
    ap.add_argument("--sizes", default="", help="validation: comma-separated D (cylinders) or k (hill)")
    ap.add_argument("--flow-throughs", type=float, default=4.0,
                    help="validation confined: stop after this many flow-through times L/U at most")
    ap.add_argument("--nusselt-study", action="store_true",
                    help="heated sphere 192x64x64 at Pr 10, 100, 1000 (--prs): mean Nu after --steps steps")
    ap.add_argument("--workload", choices=["sphere", "porous"], default="sphere",
                    help="porous: the 512x256x256 porous bed (see porous_study)")
    ap.add_argument("--spin", type=int, default=2000, help="porous: forward steps before the adjoint")
    ap.add_argument("--precision", action="store_true",
                    help="FP16/BF16/FP32 storage against FP64 (see precision_study)")
    ap.add_argument("--precision-crop", action="store_true",
                    help="with --precision: the 96x32x32 crop against the FP64 oracle")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the end-to-end run and the storage variants")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.flow_adjoint:
        flow_adjoint_study(args)
    elif args.validation == "cylinders":
        validation_cylinders(args)
    elif args.validation == "hill":
        validation_hill(args)
    elif args.validation == "confined":
        validation_confined(args)
    elif args.precision:
        precision_study(args)
    elif args.nusselt_study:
        sphere_nusselt_study(args)
    elif args.workload == "porous":
        porous_study(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
