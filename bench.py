#!/usr/bin/env python
"""Benchmark of the coupled D3Q19 LBGK-LPT step (arXiv:1710.07073) on GB300.

Metric: coupled-step MLUPS (million lattice-site updates per second) with FP32
and with 16-bit (FP16, BF16) shifted population storage, the fraction of the
HBM roofline reached by the fused collide-stream kernel, and the error of the
16-bit runs against the FP64 oracle (terminal rise velocity within 1 %).

A step is one pass of the whole hot path: bubble update with forward coupling,
binning, and the fused collide-stream sweep with backward coupling.  The
default workload is the dispersed swarm: 384x384x768 sites, omega 1.7,
half-way bounce-back on all six walls, 100,000 bubbles with lognormal
diameters (mean 1.5, sd 0.3) released at rest in the bottom 20 % (seed 1234).
The line's ``value`` is the FP32 step; ``fp16`` and ``bf16`` hold the same
measurement with 16-bit storage, and ``precision`` their error against the
oracle's stored 3000-step run of the 64x64x128 crop of the same swarm.  The
population state (17.2 GB FP32, 8.6 GB 16-bit) is far larger than L2, so no
flush is needed between steps.

``--impl reference`` times the FP64 CPU oracle on bounded crops of the same
workload, one per host core.  Under torchrun each rank runs an independent
replica of the column on its own GPU (the method is not sharded), and rank 0
prints one JSON line with the whole-job throughput.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled D3Q19 step MLUPS & % HBM roofline, FP32 vs FP16-store at <=1% u_t error"
FALLBACK_HBM_GBS = 6800.0
STORAGES = {"f32": 0, "f16": 1, "bf16": 2}
STORAGE_SCALE = {"f32": 1.0, "f16": 256.0, "bf16": 1.0}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "collide_stream_traffic.txt")
KERNEL_SOURCES = ("paper_1710_07073_gb300/csrc/lbm_collide.cu",
                  "paper_1710_07073_gb300/csrc/lbm_device.cuh",
                  "paper_1710_07073_gb300/csrc/lbm_internal.cuh")


def workload(name, dims=None):
    """The named workload; ``dims`` resizes it (bubbles re-drawn, the swarm's
    count scaled by volume) for profiling a smaller case."""
    from paper_1710_07073_gb300 import workloads as wl
    if name == "single_large":
        d = tuple(dims) if dims else wl.SINGLE_LARGE
        pos, vel, diam = wl.single_bubble(d)
        return dict(name="single bubble column %dx%dx%d" % d, dims=d, omega=1.6,
                    pos=pos, vel=vel, diam=diam, g=1e-5)
    if name == "batch":
        cols = wl.batch_columns(64, seed=1234)
        return dict(name="batch of 64 single-bubble columns (sizes 32x32x64..128x128x256, omega 1.0-1.9)",
                    columns=cols, dims=None, omega=None, g=1e-5,
                    pos=np.concatenate([c[2] for c in cols]),
                    vel=np.concatenate([c[3] for c in cols]),
                    diam=np.concatenate([c[4] for c in cols]))
    if name == "swarm":
        d = tuple(dims) if dims else wl.SWARM_FULL
        count = wl.swarm_count_for_crop(wl.SWARM_FULL, 100_000, d)
        pos, vel, diam = wl.swarm(d, count, seed=1234)
        return dict(name="dispersed swarm %dx%dx%d, %d bubbles" % (d + (count,)), dims=d,
                    omega=1.7, pos=pos, vel=vel, diam=diam, g=1e-5)
    raise SystemExit("unknown workload %s" % name)


def kernel_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profile_traffic(storage, dims, key=None):
    """DRAM bytes per collide-stream launch from the committed ncu summary, if it
    was taken on the current kernel source for this storage and lattice (or the
    given key)."""
    key = key or "%s_%dx%dx%d" % (storage, *dims)
    try:
        with open(PROFILE_SUMMARY) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) >= 3 and not line.startswith("#") and parts[0] == key:
                    return float(parts[2]) if parts[1] == kernel_hash() else None
    except OSError:
        return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self):
        self.marks.append(time.perf_counter())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        t0, t1 = (self.marks + [0, 0])[:2] if len(self.marks) >= 2 else (0, float("inf"))
        rows = [l for (t, l) in self.lines if t0 <= t <= t1] or [l for (_, l) in self.lines[-5:]]
        window = "timed region" if any(t0 <= t <= t1 for (t, _) in self.lines) else "around timed region"
        mhz, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for row in rows:
            parts = [p.strip() for p in row.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz), "window": window}


def max_over_ranks(value, world, device=None):
    """Largest value over the ranks of the job (the slowest rank's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(world, sites_per_rank, steps, ms_max):
    """Whole-job throughput: all ranks' site updates over the slowest rank's time."""
    return world * sites_per_rank * steps / (ms_max * 1e-3) / 1e6


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _oracle_crop(wl, sample_sites):
    """A wall-bounded crop of about ``sample_sites`` sites centred on the
    workload's bubbles, holding the bubbles that fit inside it."""
    dims = wl["dims"]
    cz = int(min(dims[2], max(16, min(64, sample_sites // 256))))
    cxy = int(max(16, min(dims[0], int((sample_sites / cz) ** 0.5) // 8 * 8)))
    crop = (min(cxy, dims[0]), min(cxy, dims[1]), cz)
    centre = np.median(wl["pos"], axis=0)
    lo = np.array([min(max(int(centre[a] - crop[a] / 2), 0), dims[a] - crop[a]) for a in range(3)],
                  dtype=np.float64)
    rel = wl["pos"] - lo
    r = 0.5 * wl["diam"][:, None]
    sel = ((rel >= r) & (rel <= np.array(crop) - r)).all(axis=1)
    return crop, lo, rel[sel], wl["vel"][sel], wl["diam"][sel]


def _oracle_sim(wl, crop, pos, vel, diam):
    from oracle.step import OracleSim
    from oracle import bubble as obub
    sim = OracleSim(crop, wl["omega"], 0x3F, obub.BubbleParams(wl["omega"], g=wl["g"]))
    sim.set_bubbles(pos, vel, diam)
    return sim


def oracle_mlups(wl, sample_sites, steps, warmup=0):
    """Time the FP64 oracle, single thread, on a crop of the workload centred on
    its bubbles; returns (MLUPS, seconds, description)."""
    crop, lo, pos, vel, diam = _oracle_crop(wl, sample_sites)
    sim = _oracle_sim(wl, crop, pos, vel, diam)
    for _ in range(warmup):
        sim.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.step()
    dt = time.perf_counter() - t0
    sites = crop[0] * crop[1] * crop[2]
    desc = "%dx%dx%d crop of the workload at %s with %d bubble(s), %d step(s)" % (
        crop[0], crop[1], crop[2], lo.astype(int).tolist(), len(diam), steps)
    return sites * steps / dt / 1e6, dt, desc


def _oracle_worker(wl, sample_sites, steps, warmup, barrier, results):
    crop, _, pos, vel, diam = _oracle_crop(wl, sample_sites)
    sim = _oracle_sim(wl, crop, pos, vel, diam)
    for _ in range(warmup):
        sim.step()
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.step()
    results.put(time.perf_counter() - t0)


def oracle_mlups_all_cores(wl, sample_sites, steps, warmup=0, procs=None):
    """The FP64 oracle on every host core: one process per core (spawned, so no
    GPU state is inherited), each stepping its own copy of the crop; the timed
    steps start together.  Returns (aggregate MLUPS, seconds of the slowest
    process, processes, description)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    results = ctx.Queue()
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    small = {k: wl[k] for k in ("dims", "omega", "g", "pos", "vel", "diam")}
    ps = [ctx.Process(target=_oracle_worker, args=(small, sample_sites, steps, warmup, barrier,
                                                   results)) for _ in range(procs)]
    try:
        for p in ps:
            p.start()
        times = [results.get(timeout=600) for _ in range(procs)]
    finally:
        for p in ps:
            p.join(timeout=60)
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    crop, lo, _, _, diam = _oracle_crop(wl, sample_sites)
    sites = crop[0] * crop[1] * crop[2]
    dt = max(times)
    desc = "%d processes, each %dx%dx%d crop of the workload at %s with %d bubble(s), %d step(s)" % (
        procs, crop[0], crop[1], crop[2], lo.astype(int).tolist(), len(diam), steps)
    return procs * sites * steps / dt / 1e6, dt, procs, desc


def run_reference(args, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    # Keep the whole run within about two minutes at ~0.5 MLUPS per core.
    sample = int(max(16384, min(1 << 19, 0.5e8 / max(1, args.steps + args.warmup))))
    t_start = time.perf_counter()
    value, dt, procs, desc = oracle_mlups_all_cores(wl, sample, args.steps, args.warmup,
                                                    procs=args.cpu_procs)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / max(1, args.steps), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "dims": list(wl["dims"]), "omega": wl["omega"],
                   "sample": desc},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": procs,
                         "kind": "oracle", "sample": desc + " (numpy float64)"},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": round(time.perf_counter() - t_start, 2),
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baselines(wl, args):
    """The oracle on all host cores (the reported baseline) and on one core."""
    v1, dt1, desc1 = oracle_mlups(wl, 1 << 19, 6, warmup=1)
    vn, dtn, procs, descn = oracle_mlups_all_cores(wl, 1 << 19, 6, warmup=1,
                                                   procs=args.cpu_procs)
    return {"value": round(vn, 4), "unit": "MLUPS", "cores": procs, "kind": "oracle",
            "sample": descn + " (%.1f s, numpy float64, one process per core)" % dtn,
            "single_core": {"value": round(v1, 4), "unit": "MLUPS", "cores": 1,
                            "sample": desc1 + " (%.1f s, numpy float64)" % dt1}}


def run_batch(args, wl):
    """All columns of the batch in one persistent launch per step (graph replays)."""
    import torch
    from paper_1710_07073_gb300 import lbm

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lbm.lib()
    cols = wl["columns"]
    params = lbm.lbm_default_params()
    params.g = wl["g"]
    storage = args.storage
    b = lbm.Batch([c[0] for c in cols], [c[1] for c in cols], None, STORAGES[storage],
                  STORAGE_SCALE[storage], params=params)
    stream = torch.cuda.Stream()
    lbm.lbm_batch_set_stream(b.h, stream.cuda_stream)
    lbm.lbm_batch_set_bubbles(b.h, [1] * len(cols), wl["pos"].reshape(-1), wl["vel"].reshape(-1),
                              wl["diam"])
    S = lbm.lbm_batch_sites(b.h)
    lbm.lbm_batch_tune(b.h, 8)
    planes, depth, grid = lbm.lbm_batch_launch_shape(b.h)
    lbm.lbm_batch_step(b.h, args.warmup)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3 if sampler.proc else 0.0)
    launches0 = lbm.lbm_batch_launch_count(b.h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.mark()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    lbm.lbm_batch_step(b.h, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    sampler.mark()
    ms = ev0.elapsed_time(ev1)
    launches = lbm.lbm_batch_launch_count(b.h) - launches0
    clocks = sampler.stop()
    # Average duration of the persistent collide-stream launch, timed per launch.
    lbm.lbm_batch_set_kernel_timing(b.h, True)
    lbm.lbm_batch_step(b.h, min(args.steps, 50))
    k_ms, k_n = lbm.lbm_batch_get_kernel_time(b.h)
    lbm.lbm_batch_set_kernel_timing(b.h, False)
    # End to end through the public API with host buffers: bubbles uploaded
    # from pinned memory, the bubbles read back after every graph replay (a
    # pair of steps), every column's fields downloaded at the end.
    pos_h = torch.from_numpy(wl["pos"].reshape(-1).copy()).pin_memory().numpy()
    vel_h = torch.from_numpy(wl["vel"].reshape(-1).copy()).pin_memory().numpy()
    d_h = torch.from_numpy(wl["diam"].copy()).pin_memory().numpy()
    sizes = [int(np.prod(c[0])) for c in cols]
    outs = [(torch.empty(n, dtype=torch.float64).pin_memory().numpy(),
             torch.empty(3 * n, dtype=torch.float64).pin_memory().numpy()) for n in sizes]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_batch_set_bubbles(b.h, [1] * len(cols), pos_h, vel_h, d_h)
    for _ in range(args.steps // 2):
        lbm.lbm_batch_step(b.h, 2)
        lbm.lbm_batch_get_bubbles(b.h)
    for c, (ro, uo) in enumerate(outs):
        lbm.lbm_batch_get_fields(b.h, c, sizes[c], out_rho=ro, out_u=uo)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_steps = 2 * (args.steps // 2)
    nb = int(wl["diam"].size)
    e2e = {"value": round(aggregate_mlups(world, S, e2e_steps, e2e_s * 1e3), 2), "unit": "MLUPS",
           "h2d_bytes_per_step": round(7 * 8 * nb / e2e_steps, 1),
           "d2h_bytes_per_step": round((12 * 8 + 4) * nb / 2 + 4 * 8 * S / e2e_steps, 1)}
    b.close()
    ms = max_over_ranks(ms, world, "cuda")
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    value = aggregate_mlups(world, S, args.steps, ms)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # The oracle on the batch's smallest column, whole, on all host cores.
        small = min(range(len(cols)), key=lambda c: sizes[c])
        dims_c, omega_c, pos_c, vel_c, diam_c = cols[small]
        cpu = cpu_baselines(dict(dims=dims_c, omega=omega_c, g=wl["g"], pos=pos_c, vel=vel_c,
                                 diam=diam_c), args)
    bytes_per_site = 2 * 19 * (4 if storage == "f32" else 2)
    avg_kernel_s = (k_ms / max(1, k_n)) * 1e-3
    achieved = bytes_per_site * S / avg_kernel_s / 1e9
    peak, peak_kind = measured_peak()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl["name"], "columns": len(cols), "sites": S, "storage": storage,
                   "tuned": {"cta_tile": [32, 4, planes], "depth": depth, "grid": grid},
                   "l2": "inputs larger than L2 (%.2f GB populations), no flush" % (
                       19 * S * (4 if storage == "f32" else 2) / 1e9)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": profile_traffic(storage, None, key="%s_batch64" % storage),
                     "kernel": "k_collide_batch<%d,%d>" % (STORAGES[storage], planes),
                     "algorithmic_bytes_per_launch": bytes_per_site * S,
                     "avg_launch_ms": round(avg_kernel_s * 1e3, 5), "launches": k_n,
                     "peak_kind": peak_kind, "timed": "separate per-launch pass after the graph run"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_adjoint(args):
    """Adjoint of 1000 coupled steps of a 128x128x256 column (checkpoint every 50),
    gradients of the terminal-velocity mismatch, checked by central differences."""
    import torch
    from paper_1710_07073_gb300 import lbm, workloads as wlm
    from paper_1710_07073_gb300.adjoint import TerminalVelocityProblem

    torch.cuda.set_device(0)
    lbm.lib()
    dims = (128, 128, 256)
    prob = TerminalVelocityProblem(dims=dims, omega=1.6, positions=np.array([[64.0, 64.0, 32.0]]),
                                   steps=1000, checkpoint_every=50, window=200, target=8e-5,
                                   g=1e-5)
    P = wlm.gaussian_velocity_perturbation(dims, seed=4, amp=1e-4)
    S = int(np.prod(dims))

    def loss_only(sd, d, eps):
        col = prob.column(sd, d, eps * P)
        loss = lbm.lbm_adj_forward(col.ctx, prob.steps, prob.checkpoint_every, prob.window,
                                   prob.target)
        col.close()
        return loss

    col = prob.column(1.0, 2.5, P)
    lbm.lbm_adj_forward(col.ctx, 50, 50, 10, prob.target)   # warm-up
    lbm.lbm_adj_backward(col.ctx, 1.0, want_u0=False)
    col.close()
    col = prob.column(1.0, 2.5, P)
    torch.cuda.synchronize()
    launches0 = lbm.lbm_launch_count(col.ctx)
    t0 = time.perf_counter()
    loss = lbm.lbm_adj_forward(col.ctx, prob.steps, prob.checkpoint_every, prob.window, prob.target)
    t1 = time.perf_counter()
    lbm.lbm_set_kernel_timing(col.ctx, True)
    g_sd, g_d, g_u0 = lbm.lbm_adj_backward(col.ctx, 1.0, want_u0=True)
    t2 = time.perf_counter()
    launches = lbm.lbm_launch_count(col.ctx) - launches0
    k_ms, k_n = lbm.lbm_get_kernel_time(col.ctx)
    col.close()
    # End to end through the autograd.Function, the call a user makes: the
    # initial field goes up from host memory, its gradient comes back.
    from paper_1710_07073_gb300.adjoint import TerminalVelocityLoss
    sd_t = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    d_t = torch.tensor(2.5, dtype=torch.float64, requires_grad=True)
    u0_t = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float64)).requires_grad_()
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    TerminalVelocityLoss.apply(sd_t, d_t, u0_t, prob).backward()
    e2e_s = time.perf_counter() - t3
    nbub = len(prob.positions)
    h2d = 3 * S * 8 + 7 * nbub * 8   # u0, and the bubbles' positions, velocities, diameters
    d2h = 3 * S * 8 + 2 * nbub * 8 + 8   # du0, the per-bubble gradients, the loss
    g_e = float((g_u0 * P.reshape(-1)).sum())
    h, he = 1e-3, 0.05
    fd_sd = (loss_only(1.0 + h, 2.5, 1.0) - loss_only(1.0 - h, 2.5, 1.0)) / (2 * h)
    fd_d = (loss_only(1.0, 2.5 + h, 1.0) - loss_only(1.0, 2.5 - h, 1.0)) / (2 * h)
    fd_e = (loss_only(1.0, 2.5, 1.0 + he) - loss_only(1.0, 2.5, 1.0 - he)) / (2 * he)
    fwd_s, bwd_s = t1 - t0, t2 - t1
    value = S * prob.steps / (fwd_s + bwd_s) / 1e6
    cpu = None
    if not args.no_cpu_baseline:
        # The oracle's gradient is central differences: the loss and two runs
        # per direction (drag scale, diameter, one initial-field direction).
        wl_adj = dict(dims=dims, omega=1.6, g=1e-5, pos=np.array([[64.0, 64.0, 32.0]]),
                      vel=np.zeros((1, 3)), diam=np.array([2.5]))
        vn, dtn, procs, descn = oracle_mlups_all_cores(wl_adj, 1 << 19, 6, warmup=1,
                                                       procs=args.cpu_procs)
        cpu = {"value": round(vn / 7, 4), "unit": "MLUPS", "cores": procs, "kind": "oracle",
               "sample": descn + " (%.1f s, numpy float64, one process per core); forward MLUPS "
                         "%.4f divided by 7 forward runs per gradient (the loss and central "
                         "differences in three directions)" % (dtn, vn)}
    achieved = 3 * 19 * 4 * S / (k_ms / max(1, k_n) * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    line = {
        "metric": "adjoint of the coupled step: forward + reverse MLUPS", "value": round(value, 2),
        "unit": "MLUPS", "n_gpus": 1, "steps": prob.steps, "warmup": 1,
        "ms_per_step": round((fwd_s + bwd_s) * 1e3 / prob.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "adjoint: 128x128x256 column, omega 1.6, d 2.5, 1000 steps, "
                               "checkpoint every 50, loss over the last 200 steps",
                   "forward_s": round(fwd_s, 4), "backward_s": round(bwd_s, 4), "loss": loss},
        "e2e": {"value": round(S * prob.steps / e2e_s / 1e6, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": round(h2d / prob.steps, 1),
                "d2h_bytes_per_step": round(d2h / prob.steps, 1),
                "call": "TerminalVelocityLoss.apply(...).backward() from host tensors, column "
                        "creation included"},
        "cpu_baseline": cpu, "gpu_launches": int(launches),
        "gradients": {"drag_scale": [g_sd, fd_sd, abs(g_sd / fd_sd - 1)],
                      "diameter": [float(g_d[0]), fd_d, abs(g_d[0] / fd_d - 1)],
                      "u0_direction": [g_e, fd_e, abs(g_e / fd_e - 1)],
                      "format": "[adjoint, central FD of the FP32 forward, relative difference]"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "kernel": "k_adj_liquid",
                     "algorithmic_bytes_per_launch": 3 * 19 * 4 * S,
                     "avg_launch_ms": round(k_ms / max(1, k_n), 5), "launches": k_n,
                     "peak_kind": peak_kind},
    }
    print(json.dumps(line), flush=True)
    return 0


GOLDEN_CROP = os.path.join(ROOT, "tests", "golden", "swarm_crop_64x64x128.npz")


def crop_precision(storage, golden=None):
    """The 64x64x128 crop of the swarm (463 bubbles, omega 1.7, seed 1234) run
    for 3000 steps with the given storage, against the FP64 oracle's stored run
    of the same input (tests/golden).  Errors: velocity relative L-inf and
    bubble position relative L-inf after 1000 and 3000 steps (velocity on the
    even sublattice the golden keeps), rho absolute L-inf, and the terminal
    rise velocity (mean u_b,z over all bubbles and steps 2801-3000)."""
    from paper_1710_07073_gb300 import lbm, workloads as wlm
    g = golden if golden is not None else dict(np.load(GOLDEN_CROP))
    dims = wlm.SWARM_CROP
    count = wlm.swarm_count_for_crop(wlm.SWARM_FULL, 100_000, dims)
    pos, vel, diam = wlm.swarm(dims, count, seed=1234)
    p = lbm.lbm_default_params()
    p.g = 1e-5
    col = lbm.Column(dims, 1.7, lbm.LBM_WALL_ALL, STORAGES[storage], STORAGE_SCALE[storage],
                     params=p)
    lbm.lbm_set_bubbles(col.ctx, pos.reshape(-1), vel.reshape(-1), diam)

    def rel(a, b):
        return float(np.abs(a - b).max() / np.abs(b).max())

    lbm.lbm_step(col.ctx, 1000)
    _, u = col.fields()
    e = {"u_rel_linf_1000": rel(u[:, ::2, ::2, ::2], g["u1000"]),
         "pos_rel_1000": rel(lbm.lbm_get_bubbles(col.ctx)["pos"], g["pos1000"])}
    lbm.lbm_step(col.ctx, 1800)
    ubz = []
    for _ in range(200):
        lbm.lbm_step(col.ctx, 1)
        ubz.append(float(lbm.lbm_get_bubbles(col.ctx)["vel"][:, 2].mean()))
    rho, u = col.fields()
    b = lbm.lbm_get_bubbles(col.ctx)
    col.close()
    vt, vt_or = float(np.mean(ubz)), float(np.mean(g["ubz_last200"]))
    e.update({"u_rel_linf_3000": rel(u[:, ::2, ::2, ::2], g["u3000"]),
              "rho_abs_linf_3000": float(np.abs(rho[::2, ::2, ::2] - 1.0 - g["drho3000"]).max()),
              "pos_rel_3000": rel(b["pos"], g["pos3000"]),
              "vt": vt, "vt_oracle": vt_or, "vt_rel": abs(vt / vt_or - 1.0),
              "active_equal": bool(np.array_equal(b["active"], g["active3000"]))})
    return e


def measure(args, wl, storage, stream, world, local, e2e=False):
    """Time ``args.steps`` coupled steps with the given storage; then the sweep
    launch alone (CUDA events around every sweep in a separate pass) and, with
    ``e2e``, the same steps end to end through the C ABI with host buffers."""
    import torch
    from paper_1710_07073_gb300 import lbm

    dims = wl["dims"]
    S = int(np.prod(dims))
    params = lbm.lbm_default_params()
    params.g = wl["g"]
    out = {}
    with torch.cuda.stream(stream):
        col = lbm.Column(dims, wl["omega"], lbm.LBM_WALL_ALL, STORAGES[storage],
                         STORAGE_SCALE[storage], params=params, torch_plumbing=True)
        ctx = col.ctx
        lbm.lbm_set_bubbles(ctx, wl["pos"].reshape(-1), wl["vel"].reshape(-1), wl["diam"])
        lbm.lbm_step(ctx, args.warmup)
        out["kernel"] = lbm.lbm_sweep_kernel(ctx)

        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3 if sampler.proc else 0.0)
        launches0 = lbm.lbm_launch_count(ctx)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler.mark()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lbm.lbm_step(ctx, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        sampler.mark()
        if world > 1:
            torch.distributed.barrier()
        ms = ev0.elapsed_time(ev1)
        out["launches"] = lbm.lbm_launch_count(ctx) - launches0
        time.sleep(0.2 if sampler.proc else 0.0)
        out["clocks"] = sampler.stop()
        # Duration of the collide-stream launch alone: a separate pass with an
        # event pair around every sweep (which keeps plain stream order, so the
        # bubble update does not overlap the timed sweep).
        lbm.lbm_set_kernel_timing(ctx, True)
        lbm.lbm_step(ctx, min(args.steps, 100))
        out["k_ms"], out["k_n"] = lbm.lbm_get_kernel_time(ctx)
        lbm.lbm_set_kernel_timing(ctx, False)
        out["ms"] = max_over_ranks(ms, world, "cuda")
        out["value"] = aggregate_mlups(world, S, args.steps, out["ms"])

        if e2e:
            # End to end through the public API with host buffers: upload the
            # initial fields and bubbles from pinned memory, step, read the
            # bubbles back after every step, download the final fields.
            nb = wl["diam"].size
            rho_h = torch.ones(S, dtype=torch.float64).pin_memory().numpy()
            u_h = torch.zeros(3 * S, dtype=torch.float64).pin_memory().numpy()
            rho_o = torch.empty(S, dtype=torch.float64).pin_memory().numpy()
            u_o = torch.empty(3 * S, dtype=torch.float64).pin_memory().numpy()
            pos_h = torch.from_numpy(wl["pos"].reshape(-1).copy()).pin_memory().numpy()
            vel_h = torch.from_numpy(wl["vel"].reshape(-1).copy()).pin_memory().numpy()
            d_h = torch.from_numpy(wl["diam"].copy()).pin_memory().numpy()
            lbm.lbm_set_fields(ctx, rho_h, u_h)          # warm the allocator's staging blocks
            lbm.lbm_get_fields(ctx, out_rho=rho_o, out_u=u_o)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lbm.lbm_set_fields(ctx, rho_h, u_h)
            lbm.lbm_set_bubbles(ctx, pos_h, vel_h, d_h)
            for _ in range(args.steps):
                lbm.lbm_step(ctx, 1)
                lbm.lbm_get_bubbles(ctx)
            lbm.lbm_get_fields(ctx, out_rho=rho_o, out_u=u_o)
            torch.cuda.synchronize()
            e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
            out["e2e"] = {
                "value": round(aggregate_mlups(world, S, args.steps, e2e_s * 1e3), 2),
                "unit": "MLUPS",
                "h2d_bytes_per_step": round((4 * 8 * S + 7 * 8 * nb) / args.steps, 1),
                "d2h_bytes_per_step": round((4 * 8 * S) / args.steps + (12 * 8 + 4) * nb, 1)}
        col.close()
    bytes_per_site = 2 * 19 * (4 if storage == "f32" else 2)
    avg_kernel_s = (out["k_ms"] / max(1, out["k_n"])) * 1e-3
    achieved = bytes_per_site * S / avg_kernel_s / 1e9
    peak, peak_kind = measured_peak()
    out["roofline"] = {
        "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
        "frac": round(achieved / peak, 4), "traffic": profile_traffic(storage, dims),
        "kernel": out["kernel"], "algorithmic_bytes_per_launch": bytes_per_site * S,
        "avg_launch_ms": round(avg_kernel_s * 1e3, 5), "launches": out["k_n"],
        "peak_kind": peak_kind, "timed": "separate per-launch pass after the timed steps"}
    return out


def run_gpu(args, wl):
    import torch
    from paper_1710_07073_gb300 import lbm

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU; the CPU oracle is only timed with --impl reference")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lbm.lib()   # fails loudly if the CUDA library is missing

    storages = [s for s in args.storages.split(",") if s]
    dims = wl["dims"]
    S = int(np.prod(dims))
    stream = torch.cuda.Stream()
    runs = {}
    for k, st in enumerate(storages):
        runs[st] = measure(args, wl, st, stream, world, local, e2e=(k == 0))
        torch.cuda.empty_cache()
    precision = None
    swarm_workload = wl["name"].startswith("dispersed swarm")
    if swarm_workload and not args.no_precision and os.path.exists(GOLDEN_CROP):
        golden = dict(np.load(GOLDEN_CROP))
        precision = {"crop": "64x64x128 crop of the swarm, 463 bubbles, omega 1.7, seed 1234, "
                             "3000 steps, against the FP64 oracle's stored run",
                     **{st: crop_precision(st, golden) for st in storages}}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    main_st = storages[0]
    r0 = runs[main_st]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(wl, args)
    line = {
        "metric": METRIC, "value": round(r0["value"], 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r0["ms"] / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": main_st,
        "data": "synthetic",
        "config": {"workload": wl["name"], "dims": list(dims), "omega": wl["omega"],
                   "bubbles": int(wl["diam"].size), "storage": main_st,
                   "walls": "bounce-back on all six faces",
                   "l2": "inputs larger than L2 (%.2f GB populations), no flush" % (
                       19 * S * (4 if main_st == "f32" else 2) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": r0["roofline"],
        "cpu_baseline": cpu,
        "e2e": r0.get("e2e"),
        "gpu_launches": int(r0["launches"]),
        "clocks": r0["clocks"],
    }
    for st in storages[1:]:
        r = runs[st]
        line[st] = {"value": round(r["value"], 2), "unit": "MLUPS",
                    "ms_per_step": round(r["ms"] / args.steps, 5),
                    "ratio_vs_%s" % main_st: round(r["value"] / r0["value"], 4),
                    "roofline": r["roofline"], "gpu_launches": int(r["launches"]),
                    "clocks": r["clocks"]}
        if precision is not None:
            line[st]["vt_rel_err"] = precision[st]["vt_rel"]
    if precision is not None:
        line["precision"] = precision
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("gb300", "reference"), default="gb300")
    ap.add_argument("--workload", choices=("swarm", "single_large", "batch", "adjoint"),
                    default="swarm")
    ap.add_argument("--storages", default=None,
                    help="comma-separated storages, the first gives the line's value "
                         "(default f32,f16,bf16 for the swarm, f32 otherwise)")
    ap.add_argument("--storage", choices=tuple(STORAGES), default=None,
                    help="a single storage (same as --storages with one entry)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=None,
                    help="processes for the all-cores oracle timing (default: all cores)")
    ap.add_argument("--dims", default=None,
                    help="override the lattice (nx,ny,nz) for profiling a smaller case")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.storage:
        args.storages = args.storage
    if args.storages is None:
        args.storages = "f32,f16,bf16" if args.workload == "swarm" else "f32"
    for st in args.storages.split(","):
        if st not in STORAGES:
            raise SystemExit("unknown storage %s" % st)
    args.storage = args.storages.split(",")[0]
    if args.workload == "adjoint":
        return run_adjoint(args)
    dims = tuple(int(v) for v in args.dims.split(",")) if args.dims else None
    wl = workload(args.workload, dims)
    if args.impl == "reference":
        if wl.get("columns"):
            raise SystemExit("the reference arm times the single-column workloads")
        return run_reference(args, wl)
    if wl.get("columns"):
        return run_batch(args, wl)
    return run_gpu(args, wl)


if __name__ == "__main__":
    sys.exit(main())
