#!/usr/bin/env python3
"""Benchmark of the pseudo-transient elasto-plastic solve on GB300.

Workload (default): the 3D elasto-plastic box of 127^3 cells under x-z pure
shear with a spherical weak inclusion (radius 0.05, half cohesion) and +-1%
seeded cohesion noise; K = 2, G = 1, c = 1.5e-3 G, phi = 30 deg, strain
increment 1e-4, tolerance 1e-6; FP32 sweeps with FP64 norms, convergence
test and history.  One step is one load increment solved to tolerance
(start state, pseudo-transient sweeps, FP64 commit): the first increment at
which the inclusion yields (increment 5), re-solved from a device checkpoint
each step so that every step does the same work.  The same increment is
then solved once with plain FP64 sweeps ("fp64_plain").

--size 511 runs the 511^3 box of the same setup.  Its first plastic
increment takes about 13,000 iterations with frozen plasticity (about 90 s in
FP32 and 12 minutes in FP64), so it is not the default step.

Metric: effective HBM throughput of the sweeps (algorithmic bytes per cell
per iteration x cells x iterations / device time) and the wall time per
increment.  With --gpus N (torchrun), each rank solves its own replica (the
solve does not shard: no data-path collective) and value is the sum over
ranks divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a smaller grid of the same setup).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HBM GB/s and wall time per increment to tol 1e-6: warm-start FP32 vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=127, help="cells per side of the 3D box")
    ap.add_argument("--increment", type=int, default=5, help="load increment that is timed")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the plain FP64 solve")
    ap.add_argument("--warm", action="store_true", help="also train the warm-start network and time a warm increment")
    ap.add_argument("--warm-increment", type=int, default=7, help="increment timed with and without the warm start")
    ap.add_argument("--warm-train", type=int, default=2, help="held-out setups whose trajectories train the network")
    ap.add_argument("--warm-steps", type=int, default=150, help="training steps")
    ap.add_argument("--warm-base", type=int, default=32, help="base channels of the network")
    ap.add_argument("--batch", type=int, default=0, help="time the batched 2D solve of this many instances")
    ap.add_argument("--batch-increment", type=int, default=3, help="batched increment that is timed")
    ap.add_argument("--batch-freeze", type=int, default=1,
                    help="frozen plasticity after 16 n_x iterations in every instance (Sec. 3.3)")
    ap.add_argument("--batch-tile", type=int, default=-1, help="2D kernel tile (-1: autotune)")
    ap.add_argument("--batch-nchk", type=int, default=1000,
                    help="check interval of the batched FP32 solve (the FP32 stopping test needs long intervals)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-size", type=int, default=24)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--kernel", default="auto", choices=sorted(["auto", "staged", "fused", "tma", "reg"]),
                    help="sweep kernel: auto (library default), staged, fused (cp.async), tma or reg")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def setup_for(size, tol):
    import ep_inputs as E
    return E.config(5, n=(size, size, size), tol=tol)


# ---------------------------------------------------------------- clocks ----
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the samples go to $EP_CLOCKS_DIR (default: the system temporary directory)
        import tempfile
        self.path = os.path.join(os.environ.get("EP_CLOCKS_DIR", tempfile.gettempdir()), "clocks_%d.csv" % index)

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle arm ----
def oracle_increment_rate(size, tol, increment, max_seconds=30.0):
    """Time the FP64 CPU oracle on the same setup at a small size.

    Runs the elastic increments untimed, then times solving `increment`
    (restoring the history first each repetition) until max_seconds is spent.
    Returns (seconds per increment, iterations, cells)."""
    import numpy as np
    import oracle as O
    s = setup_for(size, tol)
    o = O.from_setup(s)
    rates = [s.a, 0.0, -s.a]
    for _ in range(increment - 1):
        o.apply_increment(rates, s.dt)
        o.solve_increment()
    names = ("vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl", "ux", "uy", "uz",
             "exx", "eyy", "ezz", "exy", "exz", "eyz")
    saved = {f: o.get(f) for f in names}
    times, iters = [], 0
    t_start = time.perf_counter()
    while True:
        for f, v in saved.items():
            o.set(f, v)
        t0 = time.perf_counter()
        o.apply_increment(rates, s.dt)
        info = o.solve_increment()
        times.append(time.perf_counter() - t0)
        iters = info["iters"]
        if time.perf_counter() - t_start > max_seconds or len(times) >= 3:
            break
    del np
    return sum(times) / len(times), iters, size ** 3


def alg_bytes_per_cell(ndim, precision):
    """Bytes one fused sweep iteration must move per cell: it reads the
    velocity increment, the stress state and pressure, the base trial and
    base pressure, B c and the rotation weights, and writes the velocity
    increment, the stress state and pressure."""
    nd, ns = ndim, (3 if ndim == 3 else 1)
    words = (nd + (nd + ns) + 1 + (nd + ns) + 1 + 1 + (ns + nd - 1)) + (nd + (nd + ns) + 1)
    return words * (8 if precision == "fp64" else 4)


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    s = setup_for(args.size, args.tol)
    # bounded sample: each step solves the timed increment on a cpu_size^3 grid
    per_inc, iters, cells = None, None, None
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        per_inc, iters, cells = oracle_increment_rate(args.cpu_size, args.tol, args.increment, max_seconds=0.0)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    bpc = alg_bytes_per_cell(3, "fp64")
    gbs = bpc * cells * iters / per_inc / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "3d-ep-xz-inclusion %d^3 (oracle sample of the %d^3 workload), increment %d, tol %g"
                   % (args.cpu_size, s.n[0], args.increment, args.tol),
                   "sample_cells": cells, "iterations": iters},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "increment %d of the %d^3 box solved by the single-threaded FP64 oracle "
                                   "(%d iterations, %.2f s per increment)" % (args.increment, args.cpu_size, iters,
                                                                             per_inc)},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- our arm ----
KERNEL = {"auto": -1, "staged": 0, "fused": 1, "tma": 2, "reg": 3}


def one_step(P, g, s):
    """One pass of the path: back to the checkpoint before the timed
    increment, start it, iterate to tolerance, commit."""
    g.restore()
    g.apply_increment(s.a, s.dt, P.LOAD_XZ)
    return g.solve_increment()


def check_interval(size, precision):
    """Check every 100 iterations, or every 1000 for FP32 boxes above 200^3:
    the FP32 stopping measure needs the longer interval there."""
    return 1000 if precision == "fp32" and size > 200 else 100


def make_grid(P, s, precision, kernel="auto", stream=None):
    g = P.Grid(3, s.n, s.L, precision=P.FP64 if precision == "fp64" else P.FP32_MIXED, stream=stream)
    g.set_kernel(KERNEL[kernel], -1)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    g.set_solver(tol=s.tol, max_iter=2000000, n_chk=check_interval(s.n[0], precision))
    return g


def prepare(P, s, precision, increment, kernel="auto", stream=None):
    """Solve the increments before the timed one, then checkpoint the
    history on the device (every step restarts from it)."""
    g = make_grid(P, s, precision, kernel, stream)
    for inc in range(1, increment):
        g.apply_increment(s.a, s.dt, P.LOAD_XZ)
        g.solve_increment()
    g.snapshot()
    return g


def aggregate(torch, dist, seconds, units, device):
    """The slowest rank's time and the units (bytes) all ranks processed.
    Ranks run replicas (each solves its own copy, no data-path collective);
    this is the only communication besides barriers."""
    if dist is None:
        return seconds, units
    tmax = torch.tensor([seconds], dtype=torch.float64, device=device)
    tot = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(tmax.item()), float(tot.item())


def timed_steps(torch, P, g, s, stream, steps, barrier):
    """Run `steps` steps between CUDA events on the library's stream (with a
    barrier and a device synchronisation on both sides); returns (device
    seconds, solve infos)."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    infos = [one_step(P, g, s) for _ in range(steps)]
    ev1.record(stream)
    barrier()
    return ev0.elapsed_time(ev1) * 1e-3, infos


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu capture of the benchmark command, by kernel and
# box size; the entry must be dropped when the kernel changes.
NCU_TRAFFIC = {("k_fused3d_reg", 127): 271.8e6}


def kernel_names(ktimes, kernel):
    if len(ktimes) == 2:
        return [{"tma": "k_fused3d_tma", "reg": "k_fused3d_reg", "fused": "k_fused3d"}.get(kernel, "k_fused3d_reg")]
    return ["k_strain", "k_trial", "k_return_centres", "k_return_edges", "k_velocity"]


def our_arm(args):
    import torch
    import paper_2305_01701_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    stream = torch.cuda.Stream()
    s = setup_for(args.size, args.tol)
    cells = s.n[0] * s.n[1] * s.n[2]
    g = prepare(P, s, args.precision, args.increment, args.kernel, stream.cuda_stream)
    for _ in range(args.warmup):           # full passes of the timed step
        one_step(P, g, s)
    bpc = g.sweep_bytes_per_cell()
    nchk = check_interval(s.n[0], args.precision)
    clk = Clocks(local)
    clk.start()
    sec, infos = timed_steps(torch, P, g, s, stream, args.steps, barrier)
    clocks = clk.stop()
    iters = sum(i["iters"] for i in infos)
    tmax, total_bytes = aggregate(torch, dist, sec, bpc * cells * iters, "cuda")
    gbs = total_bytes / tmax / 1e9
    ms_per_step = tmax / args.steps * 1e3

    # dominant sweep kernel: CUDA events on the library's stream around a
    # burst of back-to-back launches on the same increment
    ktimes = g.time_sweep(20)
    kernels = kernel_names(ktimes, args.kernel)
    it_ms = ktimes[-1]
    dom = int(max(range(len(kernels)), key=lambda q: ktimes[q]))

    # end to end through the C ABI with host buffers: the step's inputs (load
    # rates, time step) in, the converged fields out to pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        fields = ["vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl"]
        bufs = {f: torch.empty(g.count(f), dtype=torch.float64, pin_memory=True) for f in fields}
        d2h = sum(b.numel() * 8 for b in bufs.values())
        h2d = 8 * 3 + 8
        barrier()
        t0 = time.perf_counter()
        e_iters = 0
        for _ in range(args.e2e_steps):
            e_iters += one_step(P, g, s)["iters"]
            for f in fields:
                g.get_into(f, bufs[f].data_ptr(), bufs[f].numel())
        barrier()
        et = time.perf_counter() - t0
        e2e = {"value": bpc * cells * e_iters * world / et / 1e9, "unit": "GB/s",
               "ms_per_step": et / args.e2e_steps * 1e3, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    fp64 = None
    if not args.no_fp64:
        g.close()
        g64 = prepare(P, s, "fp64", args.increment, "auto", stream.cuda_stream)
        one_step(P, g64, s)
        t64, i64 = timed_steps(torch, P, g64, s, stream, 1, barrier)
        i64 = i64[0]
        fp64 = {"ms_per_increment": t64 * 1e3, "iterations": i64["iters"], "kernel": "staged",
                "GB_per_s": g64.sweep_bytes_per_cell() * cells * i64["iters"] / t64 / 1e9,
                "fp32_speedup": t64 * 1e3 / ms_per_step}
        g64.close()

    warm = None
    if args.warm:
        warm = warm_arm(args, torch, P, stream, barrier, s, cells)
        if fp64 is not None and args.warm_increment == args.increment:
            warm["fp64_plain_ms"] = fp64["ms_per_increment"]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        per_inc, c_iters, c_cells = oracle_increment_rate(args.cpu_size, args.tol, args.increment)
        cpu = {"value": alg_bytes_per_cell(3, "fp64") * c_cells * c_iters / per_inc / 1e9, "unit": "GB/s",
               "cores": 1, "kind": "oracle",
               "sample": "increment %d of the same setup on a %d^3 grid, single-threaded FP64 oracle "
                         "(%d iterations, %.2f s per increment)" % (args.increment, args.cpu_size, c_iters, per_inc)}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    achieved = bpc * cells / (it_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": kernels[0] if len(kernels) == 1 else "staged sweep (5 kernels)",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6800 GB/s",
            "traffic": NCU_TRAFFIC.get((kernels[dom], s.n[0])),
            "traffic_source": "ncu --set full capture of one launch of this command (profiles/)"
                              if (kernels[dom], s.n[0]) in NCU_TRAFFIC else None,
            "kernel_ms": {k: float(ktimes[q]) for q, k in enumerate(kernels)},
            "dominant": kernels[dom], "iteration_ms": float(it_ms), "alg_bytes_per_cell": bpc}
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "3d-ep-xz-inclusion %d^3, increment %d, tol %g, %s sweeps, plain start"
                   % (s.n[0], args.increment, args.tol, args.precision),
                   "sweep_kernel": kernels[0] if len(kernels) == 1 else "staged",
                   "cells": cells, "iterations_per_step": infos[-1]["iters"], "check_every": nchk,
                   "frozen_at": infos[-1].get("frozen_at", -1),
                   "l2": "inputs larger than L2 (%d sweep arrays of %.1f MB)" % (33, cells * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "ms_per_increment": ms_per_step,
        "clocks": clocks,
        # per step: (iters / n_chk + 1) graph chunks (staged: 5 n_chk + 1
        # kernels; fused: one staged check iteration, the check and n_chk - 1
        # fused sweeps), plus about 20 start-of-increment and 7 commit kernels
        "gpu_launches": int(sum((i["iters"] // nchk + 1) * (5 * nchk + 1 if len(kernels) == 5 else nchk + 5) + 27
                                for i in infos)),
        "roofline": roof,
        "e2e": e2e,
        "fp64_plain": fp64,
        "warm_start": warm,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def warm_arm(args, torch, P, stream, barrier, s, cells):
    """The learned warm start on the benchmark box: a 3D U-Net (3 levels,
    BF16 weights, FP32 accumulation) trained on the GPU with the library's
    kernels from trajectories of held-out seeds of the same setup, then the
    increment `--warm-increment` solved from one device checkpoint with the
    plain start and with the network's start (FP32 sweeps, same tolerance)."""
    import time as _t
    import ep_inputs as E
    from paper_2305_01701_gb300 import warmstart as W

    t_train0 = _t.perf_counter()
    net = W.new_net(3, base=args.warm_base, levels=3, seed=7, stream=stream.cuda_stream)
    incs = args.warm_increment + 1
    groups = []
    for q in range(args.warm_train):
        ts = E.config(5, n=s.n, tol=s.tol, seed=s.seed + 101 + q, c0=s.c0 * (1.0 + 0.05 * (q + 1)))
        gt = make_grid(P, ts, "fp32", args.kernel, stream.cuda_stream)
        data = W.Samples(3, gt.warm_dims(), capacity=incs)
        W.collect(gt, ts.a, ts.dt, incs, data, load_plane=P.LOAD_XZ)
        gt.close()
        groups.append(data)
    loss_before = W.evaluate(net, groups)
    losses = W.train(net, groups, steps=args.warm_steps, lr=1e-3, batch=2)
    torch.cuda.synchronize()
    t_train = _t.perf_counter() - t_train0
    loss_after, loss_zero = W.evaluate(net, groups), W.zero_loss(groups)

    g = prepare(P, s, "fp32", args.warm_increment, args.kernel, stream.cuda_stream)
    g.attach_warm_start(net)

    def one(warm):
        g.restore()
        g.apply_increment(s.a, s.dt, P.LOAD_XZ, use_warm_start=warm)
        return g.solve_increment()

    one(False)
    one(True)
    res = {}
    for warm in (False, True):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        info = one(warm)
        ev1.record(stream)
        barrier()
        res[warm] = (ev0.elapsed_time(ev1), info)
    bpc = g.sweep_bytes_per_cell()
    out = {"increment": args.warm_increment,
           "plain_ms": res[False][0], "plain_iterations": res[False][1]["iters"],
           "warm_ms": res[True][0], "warm_iterations": res[True][1]["iters"],
           "warm_GB_per_s": bpc * cells * res[True][1]["iters"] / (res[True][0] * 1e-3) / 1e9,
           "net": "3-level U-Net, base %d, BF16 weights, FP32 accumulation" % args.warm_base,
           "training": {"setups": args.warm_train, "samples": sum(d.n for d in groups), "steps": args.warm_steps,
                        "train_mse_before": loss_before, "train_mse_after": loss_after,
                        "train_mse_zero_net": loss_zero,
                        "last_minibatch_loss": float(sum(losses[-10:]) / 10), "seconds": t_train}}
    g.close()
    net.close()
    return out


def batch_arm(args):
    """Config 4: uneven 2D instances advanced by one persistent, graph-captured
    launch per iteration (FP32 sweeps, FP64 norms and history).  One step is
    one batched increment (`--batch-increment`) re-solved from a device
    checkpoint of every instance."""
    import torch
    import ep_inputs as E
    import paper_2305_01701_gb300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    setups = E.batch_setups(args.batch)
    grids = []
    for s in setups:
        g = P.Grid(2, s.n, precision=P.FP32_MIXED, stream=stream.cuda_stream)
        g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
        g.set_solver(tol=s.tol, max_iter=2000000, n_chk=args.batch_nchk,
                     freeze_iter=16 * s.n[0] if args.batch_freeze else 0)
        grids.append(g)
    B = P.Batch(grids)
    a, dt = setups[0].a, setups[0].dt
    for inc in range(1, args.batch_increment):
        B.apply_increment(a, dt)
        B.solve_increment()
    for g in grids:
        g.snapshot()

    def step():
        for g in grids:
            g.restore()
        B.apply_increment(a, dt)
        return B.solve_increment()[0]

    B.apply_increment(a, dt)
    if args.batch_tile >= 0:
        B.set_tile(args.batch_tile)
        tile = args.batch_tile
    else:
        tile = B.autotune(20)              # restarts the open increments
    B.solve_increment()
    for _ in range(args.warmup):
        step()

    def barrier():
        torch.cuda.synchronize()

    clk = Clocks(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    infos = [step() for _ in range(args.steps)]
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    sec = ev0.elapsed_time(ev1) * 1e-3
    bpc = grids[0].sweep_bytes_per_cell()
    cells = [s.n[0] * s.n[1] for s in setups]
    moved = sum(bpc * c * i["iters"] for inf in infos for c, i in zip(cells, inf))
    gbs = moved / sec / 1e9
    iters = [i["iters"] for i in infos[-1]]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    # the batched kernel with every instance active: a burst of sweeps on the
    # timed increment (CUDA events on the batch's stream)
    for g in grids:
        g.restore()
    B.apply_increment(a, dt)
    sweep_ms = B.time_sweep(20)
    kernel_gbs = bpc * sum(cells) / (sweep_ms * 1e-3) / 1e9

    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O
        import time as _t
        # the smallest instances; of those the one the timed step iterated most
        nmin = min(x.n[0] for x in setups)
        small = max((q for q in range(len(setups)) if setups[q].n[0] == nmin), key=lambda q: iters[q])
        small = setups[small]
        o = O.from_setup(small)
        o.set_solver(tol=small.tol, max_iter=2000000, n_chk=100)
        if args.batch_freeze:
            o.set_freeze(16 * small.n[0], 1e-4)
        for _ in range(args.batch_increment - 1):
            o.apply_increment([a, -a, 0.0], dt)
            o.solve_increment()
        t0 = _t.perf_counter()
        o.apply_increment([a, -a, 0.0], dt)
        oi = o.solve_increment()
        ot = _t.perf_counter() - t0
        ocells = small.n[0] * small.n[1]
        cpu = {"value": alg_bytes_per_cell(2, "fp64") * ocells * max(oi["iters"], 1) / ot / 1e9, "unit": "GB/s",
               "cores": 1, "kind": "oracle",
               "sample": "increment %d of one %dx%d instance (%s), single-threaded FP64 oracle, %d iterations "
                         "in %.2f s" % (args.batch_increment, small.n[0], small.n[1], small.name, oi["iters"], ot)}
    line = {
        "metric": "aggregate sweep GB/s and wall time per batched increment to tol 1e-6",
        "value": gbs, "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "2d-batch %d instances of {127,255,383,511}^2, increment %d, tol 1e-6, fp32 sweeps, "
                               "check every %d iterations%s" % (len(setups), args.batch_increment, args.batch_nchk,
                                                                ", frozen plasticity after 16 n_x iterations"
                                                                if args.batch_freeze else ""),
                   "cells": sum(cells), "tile": tile, "iterations_min_max": [min(iters), max(iters)],
                   "iterations_sum": sum(iters),
                   "l2": "inputs larger than L2 while most instances iterate (%.1f GB per iteration)"
                         % (bpc * sum(cells) / 1e9)},
        "clocks": clocks,
        "roofline": {"bound": "hbm", "kernel": "k_fused2d_strip" if tile >= 3 else "k_fused2d",
                     "achieved": kernel_gbs, "peak": hbm, "unit": "GB/s", "frac": kernel_gbs / hbm,
                     "sweep_ms": sweep_ms, "note": "one batched sweep with all %d instances active" % len(setups),
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6800 GB/s",
                     "traffic": None, "alg_bytes_per_cell": bpc},
        # per step: (max iterations / n_chk + 1) graph chunks of n_chk fused
        # sweeps and one check kernel, plus about 20 start-of-increment and 7
        # commit kernels per instance
        "gpu_launches": int(sum((max(i["iters"] for i in inf) // args.batch_nchk + 1) * (args.batch_nchk + 1)
                                + 27 * len(setups) for inf in infos)),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    B.close()
    for g in grids:
        g.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.batch > 0:
        return batch_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
