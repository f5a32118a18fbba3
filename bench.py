#!/usr/bin/env python3
"""Benchmark of the pseudo-transient elasto-plastic solve on GB300.

Workload (default): the 3D elasto-plastic box of 511^3 cells (133 M cells)
under x-z pure shear with a spherical weak inclusion (radius 0.05, half
cohesion) and +-1 % seeded cohesion noise; K = 2, G = 1, c = 1.5e-3 G,
phi = 30 deg, strain increment 1e-4, tolerance 1e-6, residual check every
1000 iterations, frozen plasticity after 16 n_x iterations (Sec. 3.3); FP32
sweeps with FP64 norms, convergence test and history.

Learned warm start: a 3-level 3D U-Net (base 32, BF16 weights, FP32
accumulation) is trained on the GPU with the library's kernels on the
trajectories of 127^3 boxes of the same setup (other seeds and cohesions),
on coarse cells of 1/64 of the box (2^3 fine cells there, 8^3 here).

Steps: the increment sequence from the first plastic increment (5) on, one
chunk of 1000 sweeps per step; the step that needs a new increment starts it
(warm-start inference and start state), the step whose check converges
commits it.  value = algorithmic sweep bytes of the timed steps / their
device time.  Then the timed increment is solved whole from a device
checkpoint with the warm start (end to end through the C ABI with host
buffers: `e2e`) and with the plain start, and once more with plain FP64
sweeps on an FP64 box ("per_increment": wall time and GB/s of each).

With --gpus N (torchrun), each rank solves its own replica (the solve does
not shard: no data-path collective) and value is the sum over ranks divided
by the slowest rank's time.  --size selects a smaller box of the same setup.

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
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=511, help="cells per side of the 3D box")
    ap.add_argument("--increment", type=int, default=5, help="first increment of the timed sequence")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 increment")
    ap.add_argument("--no-warm", action="store_true", help="plain start instead of the learned warm start")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="precision of the stepped walk (fp64: plain start, for profiling the FP64 sweep)")
    ap.add_argument("--no-increments", action="store_true",
                    help="skip the whole-increment arms (for short profiling runs)")
    ap.add_argument("--coarsen", type=int, default=0,
                    help="fine cells per coarse cell side of the network's grid (0: size / 64)")
    ap.add_argument("--train-size", type=int, default=127, help="box of the training trajectories")
    ap.add_argument("--warm-train", type=int, default=3, help="setups whose trajectories train the network")
    ap.add_argument("--warm-incs", type=int, default=4, help="increments after the first plastic one per setup")
    ap.add_argument("--warm-steps", type=int, default=300, help="training steps")
    ap.add_argument("--warm-base", type=int, default=32, help="base channels of the network")
    ap.add_argument("--batch", type=int, default=0, help="time the batched 2D solve of this many instances")
    ap.add_argument("--batch-increment", type=int, default=3, help="batched increment that is timed")
    ap.add_argument("--batch-freeze", type=int, default=1,
                    help="frozen plasticity after 16 n_x iterations in every instance (Sec. 3.3)")
    ap.add_argument("--batch-tile", type=int, default=-1, help="2D kernel tile (-1: autotune)")
    ap.add_argument("--batch-nchk", type=int, default=1000,
                    help="check interval of the batched FP32 solve (the FP32 stopping test needs long intervals)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--oracle-plan", action="store_true", help="time the CPU oracle per iteration and increment")
    ap.add_argument("--symmetry-study", action="store_true", help="the paper's large vs small increment study")
    ap.add_argument("--warm-study", type=int, default=0, choices=[0, 2, 3],
                    help="the learned warm start on held-out setups: trained vs zero network vs plain start (2D or 3D)")
    ap.add_argument("--sym-strain", type=float, default=1.4e-3, help="total strain of the symmetry study")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-size", type=int, default=48, help="edge of the oracle's sample box (CPU legs)")
    ap.add_argument("--oracle-threads", type=int, default=0,
                    help="threads of the timed oracle: 0 every host core (OpenMP build), 1 the plain build")
    ap.add_argument("--kernel", default="auto", choices=sorted(["auto", "staged", "fused", "tma", "reg"]),
                    help="sweep kernel: auto (library default), staged, fused (cp.async), tma or reg")
    a = ap.parse_args()
    if a.coarsen <= 0:
        a.coarsen = max(1, round(a.size / 64))
    return a


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
def oracle_lib(threads):
    """The oracle build to time and the threads it uses: threads == 1 the
    plain build; otherwise the OpenMP build (same results bit for bit) on
    `threads` threads, 0 meaning every host core (the plain build when the
    compiler has no OpenMP)."""
    import oracle as O
    if threads == 1:
        return None, 1
    path = O.build_omp()
    if path is None:
        return None, 1
    return path, O.threads(threads if threads > 0 else (os.cpu_count() or 1), path)


def oracle_increment_rate(size, tol, increment, max_seconds=30.0, lib_path=None):
    """Time the FP64 CPU oracle on the same setup at a small size.

    Runs the elastic increments untimed, then times solving `increment`
    (restoring the history first each repetition) until max_seconds is spent.
    Returns (seconds per increment, iterations, cells)."""
    import numpy as np
    import oracle as O
    s = setup_for(size, tol)
    o = O.from_setup(s, lib_path=lib_path)
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


def oracle_plan(args):
    """The CPU baseline plan: the FP64 oracle, single-threaded (the plain
    build) and on every host core (the OpenMP build, same results bit for
    bit), timed per iteration at 64^2, 511^2, 63^3 and 127^3 (a perturbed
    start velocity keeps it iterating; a fixed count of iterations) and over
    whole increments at 64^2 (config 1, increments 1-12) and 63^3 (increments
    1-5, the last the first plastic one), with the host's core count and CPU
    model.  Prints one JSON object."""
    import platform
    import numpy as np
    import ep_inputs as E
    import oracle as O

    def cpu_model():
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for line in out.splitlines():
                if line.startswith("Model name"):
                    return line.split(":", 1)[1].strip()
        except Exception:
            pass
        return platform.processor() or "unknown"

    res = {"host": {"nproc": os.cpu_count(), "cpu_model": cpu_model(), "machine": platform.machine()},
           "per_iteration": [], "increments": []}
    builds = [(None, 1)]
    omp = oracle_lib(0)
    if omp[0] is not None:
        builds.append(omp)
    for (path, thr), nd, n, iters in [(b, *c) for b in builds
                                      for c in ((2, 64, 500), (2, 511, 60), (3, 63, 60), (3, 127, 12))]:
        s = E.config(1 if nd == 2 else 3, n=(n,) * nd, tol=1e-30)
        o = O.from_setup(s, lib_path=path, max_iter=iters, n_chk=iters)
        rates = [s.a, -s.a] if nd == 2 else [s.a, 0.0, -s.a]
        o.apply_increment(rates, s.dt)
        rng = np.random.default_rng(0)
        v = np.concatenate([o.get(c).ravel() for c in ("v0x", "v0y", "v0z")[:nd]])
        o.set_start(v * (1.0 + 1e-3 * rng.standard_normal(v.size)))
        t0 = time.perf_counter()
        info = o.solve_increment(commit=False, raise_on_fail=False)
        dt = time.perf_counter() - t0
        cells = n ** nd
        k = max(info["iters"], 1)
        res["per_iteration"].append({"grid": "%d^%d" % (n, nd), "threads": thr, "iterations": k,
                                     "ms_per_iteration": dt / k * 1e3,
                                     "ns_per_cell_iteration": dt / k / cells * 1e9,
                                     "GB_per_s_algorithmic": alg_bytes_per_cell(nd, "fp64") * cells * k / dt / 1e9})
    for (path, thr), nd, n, incs in [(b, *c) for b in builds for c in ((2, 64, 12), (3, 63, 5))]:
        s = E.config(1 if nd == 2 else 3, n=(n,) * nd, tol=1e-8 if nd == 2 else 1e-6)
        o = O.from_setup(s, lib_path=path)
        rates = [s.a, -s.a] if nd == 2 else [s.a, 0.0, -s.a]
        rows = []
        for inc in range(1, incs + 1):
            t0 = time.perf_counter()
            o.apply_increment(rates, s.dt)
            info = o.solve_increment()
            rows.append({"increment": inc, "iterations": info["iters"], "seconds": time.perf_counter() - t0,
                         "n_plastic": info["n_plastic"]})
        res["increments"].append({"grid": "%d^%d" % (n, nd), "threads": thr, "tol": s.tol, "rows": rows,
                                  "seconds_total": sum(r["seconds"] for r in rows)})
    print(json.dumps(res))
    return 0


def warm_study(args):
    """What the learned warm start gains on setups it was not trained on.
    2D: 48^2 boxes with a weak inclusion at varying positions and varying
    friction angle and cohesion, a base-16 network trained on six setups x
    ten increments (800 Adam steps), three held-out setups.  3D: 63^3 boxes of
    the benchmark's setup (other seeds and cohesions), a base-32 network on
    four setups x ten increments (1500 steps), three held-out setups, checks
    every 1000 iterations.  Each held-out increment from the third on is
    solved from the same device checkpoint with the trained network, with the
    zero network (its output is the plain start) and with the plain start;
    the plain solve is kept.  Prints one JSON object."""
    import numpy as np
    import torch
    import ep_inputs as E
    import paper_2305_01701_gb300 as P
    from paper_2305_01701_gb300 import warmstart as W
    nd = args.warm_study
    t0 = time.perf_counter()
    if nd == 2:
        n, incs, steps, base, plane, nchk, kernel = (48, 48), 12, 800, 16, P.LOAD_XY, 100, None

        def setup(q, sd):
            return E.Setup("ws%d" % sd, 2, n, phi_deg=25.0 + 2 * (q % 4), c0=1.3e-3 + 1e-4 * (q % 4),
                           inclusion_radius=0.08, inclusion_centre=(0.03 * ((q % 5) - 2), -0.02 * ((q % 3) - 1), 0.0),
                           seed=sd, tol=1e-6)
        train = [setup(q, 101 + q) for q in range(6)]
        held = [setup(q, 201 + q) for q in range(3)]
    else:
        n, incs, steps, base, plane, nchk, kernel = (63, 63, 63), 12, 1500, 32, P.LOAD_XZ, 1000, P.KERNEL_FUSED_REG
        ref = E.config(5, n=n, tol=1e-6)

        def setup(k):
            return E.config(5, n=n, tol=1e-6, seed=ref.seed + k, c0=ref.c0 * (1.0 + 0.04 * (k % 4)))
        train = [setup(101 + q) for q in range(4)]
        held = [setup(201 + q) for q in range(3)]
    max_iter = 400000

    def grid(s):
        g = P.Grid(nd, s.n, precision=P.FP32_MIXED)
        if kernel is not None:
            g.set_kernel(kernel, 0)
        g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
        g.set_solver(tol=s.tol, max_iter=max_iter, n_chk=nchk)
        return g

    # one pool of samples: a minibatch of consecutive samples spans setups
    data = None
    failed = []
    for s in train:
        g = grid(s)
        if data is None:
            data = W.Samples(nd, g.warm_dims(1), capacity=len(train) * incs)
        try:
            W.collect(g, s.a, s.dt, incs, data, load_plane=plane)
        except P.EPError as e:   # a stalled FP32 solve: keep the samples stored before it
            failed.append("%s: %s" % (s.name, e))
        g.close()
    groups = [data]
    net = W.new_net(nd, base=base, levels=3, seed=7)
    zero = W.new_net(nd, base=base, levels=3, seed=7)
    scale = W.calibrate(net, groups)
    zero.set_output_scale(scale)
    before = W.evaluate(net, groups)
    W.train(net, groups, steps=steps, lr=1e-3, batch=2 if nd == 3 else 8, calibrate_scale=False)
    after = W.evaluate(net, groups)
    t_train = time.perf_counter() - t0
    total = {"trained": 0, "zero": 0, "plain": 0}
    rows = []
    for s in held:
        g = grid(s)
        for inc in range(1, incs + 1):
            if inc < 3:
                g.apply_increment(s.a, s.dt, plane)
                g.solve_increment()
                continue
            g.snapshot()
            out = {}
            for name, nn in (("trained", net), ("zero", zero), ("plain", None)):
                if nn is not None:
                    g.attach_warm_start(nn, 1)
                g.apply_increment(s.a, s.dt, plane, use_warm_start=nn is not None)
                info = g.solve_increment(raise_on_fail=False)
                out[name] = info["iters"] if info["status"] == 0 else max_iter
                total[name] += out[name]
                if name != "plain":
                    g.restore()
            rows.append({"setup": s.name, "increment": inc, **out})
            if out["plain"] == max_iter:   # the plain solve stalled: the rest of this setup is not comparable
                failed.append("%s: plain solve of increment %d did not converge" % (s.name, inc))
                break
        g.close()
    torch.cuda.synchronize()
    res = {"study": "warm start %dD" % nd, "grid": "x".join(map(str, n)), "train_setups": len(train),
           "held_out_setups": len(held), "increments": incs, "adam_steps": steps, "base": base,
           "check_every": nchk, "output_scale": scale, "loss_before": before, "loss_after": after,
           "loss_unit": "mean square of the training targets", "train_seconds": t_train,
           "total_iterations": total, "failures": failed, "samples": data.n, "rows": rows,
           "seconds": time.perf_counter() - t0}
    print(json.dumps(res))
    del np
    return 0


def symmetry_study(args):
    """The paper's symmetry study (Sec. 4.3) on the GPU: the 383 x 191 box
    with a central pressure anomaly (no Jaumann term, elastic limit), loaded
    to the same total strain once in 7 large increments and once in 180
    small ones, FP64 sweeps (warp strips) to tolerance --tol at every
    increment.  Prints, per run, the iterations and the integrated sigma_xx
    on the centre line per increment, and the mirror asymmetry of the final
    accumulated-strain invariant eps_II: |E - E mirrored| / |E| (L2) across
    the vertical and horizontal centre lines and through the centre."""
    import numpy as np
    import torch
    import ep_inputs as E
    import paper_2305_01701_gb300 as P
    torch.cuda.set_device(0)
    total = args.sym_strain
    out = {"box": "383 x 191 (L = 2 x 1), c = 2e-3, mu_s = 1e6, no Jaumann term, p = c/2 within 0.05 of the centre",
           "total_strain": total, "tol": args.tol, "runs": []}
    for incs in (7, 180):
        s = E.anomaly_setup()
        dt = total / incs
        g = P.Grid(2, s.n, s.L, precision=P.FP64)
        g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
        g.set_solver(tol=args.tol, max_iter=10000000, n_chk=100, jaumann=False, freeze_iter=0)
        g.set_kernel(P.KERNEL_FUSED, 3)
        g.set("p", E.pressure_anomaly(s.n, s.L[:2], s.extra["pressure_anomaly"]["value"],
                                     s.extra["pressure_anomaly"]["radius"]))
        rows = []
        t0 = time.perf_counter()
        for inc in range(1, incs + 1):
            g.apply_increment(s.a, dt, P.LOAD_XY)
            info = g.solve_increment()
            rows.append([inc, info["iters"], info["sxx_int_centre"], info["n_plastic"]])
        wall = time.perf_counter() - t0
        e = g.get("eii")
        nrm = float(np.sqrt((e ** 2).sum()))
        asym = {"x_mirror": float(np.sqrt(((e - e[:, ::-1]) ** 2).sum())) / nrm,
                "y_mirror": float(np.sqrt(((e - e[::-1, :]) ** 2).sum())) / nrm,
                "point": float(np.sqrt(((e - e[::-1, ::-1]) ** 2).sum())) / nrm}
        hot = e > 0.5 * e.max()
        out["runs"].append({"increments": incs, "dt": dt, "wall_s": wall, "asymmetry": asym,
                            "band_cells_left_right": [int(hot[:, : s.n[0] // 2].sum()), int(hot[:, s.n[0] // 2:].sum())],
                            "band_cells_bottom_top": [int(hot[: s.n[1] // 2].sum()), int(hot[s.n[1] // 2:].sum())],
                            "eii_max": float(e.max()), "rows": rows})
        g.close()
    print(json.dumps(out))
    return 0


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
    lib_path, thr = oracle_lib(args.oracle_threads)
    # bounded sample: each step solves the timed increment on a cpu_size^3 grid
    per_inc, iters, cells = None, None, None
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        per_inc, iters, cells = oracle_increment_rate(args.cpu_size, args.tol, args.increment, max_seconds=0.0,
                                                      lib_path=lib_path)
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
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": thr, "kind": "oracle",
                         "sample": "increment %d of the %d^3 box solved by the FP64 oracle on %d thread(s) "
                                   "(%d iterations, %.2f s per increment)" % (args.increment, args.cpu_size, thr,
                                                                             iters, per_inc)},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- our arm ----
KERNEL = {"auto": -1, "staged": 0, "fused": 1, "tma": 2, "reg": 3}


def check_interval(size, precision):
    """Check every 100 iterations, or every 1000 for FP32 boxes above 200^3:
    the FP32 stopping measure needs the longer interval there."""
    return 1000 if precision == "fp32" and size > 200 else 100


def make_grid(P, s, precision, kernel="auto", stream=None, nchk=None):
    g = P.Grid(3, s.n, s.L, precision=P.FP64 if precision == "fp64" else P.FP32_MIXED, stream=stream)
    g.set_kernel(KERNEL[kernel], -1)
    g.set_material(s.K, s.G, s.mu_s, s.phi_deg, s.psi_deg, s.cohesion())
    g.set_solver(tol=s.tol, max_iter=2000000, n_chk=nchk or check_interval(s.n[0], precision))
    return g


def prepare(P, s, precision, increment, kernel="auto", stream=None, nchk=None):
    """Solve the increments before the timed one, then checkpoint the
    history on the device (every whole-increment solve restarts from it)."""
    g = make_grid(P, s, precision, kernel, stream, nchk)
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


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu capture of the benchmark command, by kernel and
# box size; the entry must be dropped when the kernel changes.
# DRAM bytes per launch of the dominant kernel from an ncu capture of its
# current build (profiles/k_fused3d_reg_127cube.md)
NCU_TRAFFIC = {("k_fused3d_reg", 127): 271.3e6,
               ("k_fused3d_reg", 511): 271.3e6 * 133432831 / 2048383}
NCU_SOURCE = {("k_fused3d_reg", 127): "ncu --set full capture of one launch at 127^3 (profiles/)",
              ("k_fused3d_reg", 511): "ncu --set full capture of one launch at 127^3 (profiles/), the per-cell "
                                      "traffic scaled to 511^3 by the cell count"}
# FP64 flops per cell of one staged FP64 sweep (dadd + dmul + 2 dfma thread
# instructions of its five kernels, counted by ncu at 127^3; profiles/)
FP64_FLOPS_PER_CELL = 322.5
# algorithmic bytes per cell of a 3D FP32 sweep recast so that its stress is
# no pseudo-time state (reported beside the fraction by the scheme's bytes)
RECAST_BYTES_3D_FP32 = 80.0


def kernel_names(ktimes, kernel):
    if len(ktimes) == 2:
        return [{"tma": "k_fused3d_tma", "reg": "k_fused3d_reg", "fused": "k_fused3d"}.get(kernel, "k_fused3d_reg")]
    return ["k_strain", "k_trial", "k_return_centres", "k_return_edges", "k_velocity"]


class Walk:
    """Steps through the increment sequence one chunk at a time: a step
    applies a new increment when none is open (with the warm start when a
    network is attached) and runs one chunk of n_chk sweeps of the open
    increment's iteration (ep_solve_chunks)."""

    def __init__(self, P, g, s, warm):
        self.P, self.g, self.s, self.warm = P, g, s, warm
        self.open, self.done, self.finished = False, 0, []

    def step(self):
        """Returns the sweeps this step performed."""
        P, g, s = self.P, self.g, self.s
        if not self.open:
            g.apply_increment(s.a, s.dt, P.LOAD_XZ, use_warm_start=self.warm)
            self.open, self.done = True, 0
        info = g.solve_chunks(1)
        if info["status"] == P.PENDING:
            n = info["iters"] - self.done
            self.done = info["iters"]
            return n
        self.open = False
        self.finished.append(info)
        return info["iters"] + 1 - self.done


def train_warm(args, torch, P, stream):
    """The learned warm start for the benchmark box: a 3-level 3D U-Net (BF16
    weights, FP32 accumulation) trained on the GPU with the library's kernels
    on trajectories of smaller boxes of the same setup (other seeds and
    cohesions), on coarse cells of the same physical size as the benchmark
    box's coarse cells."""
    import ep_inputs as E
    from paper_2305_01701_gb300 import warmstart as W
    t0 = time.perf_counter()
    n_tr = args.train_size
    f_tr = max(1, round(args.coarsen * n_tr / args.size))
    net = W.new_net(3, base=args.warm_base, levels=3, seed=7, stream=stream.cuda_stream)
    incs = args.increment + args.warm_incs
    ref = E.config(5, n=(n_tr,) * 3, tol=args.tol)
    dims = None
    groups = []
    iters = []
    for q in range(args.warm_train):
        ts = E.config(5, n=(n_tr,) * 3, tol=args.tol, seed=ref.seed + 101 + q, c0=ref.c0 * (1.0 + 0.04 * q))
        gt = make_grid(P, ts, "fp32", args.kernel, stream.cuda_stream)
        dims = gt.warm_dims(f_tr)
        data = W.Samples(3, dims, capacity=incs)
        iters.append(W.collect(gt, ts.a, ts.dt, incs, data, load_plane=P.LOAD_XZ, coarsen=f_tr))
        gt.close()
        groups.append(data)
    scale = W.calibrate(net, groups)     # losses below in units of the targets' RMS
    zero = W.zero_loss(net, groups)
    before = W.evaluate(net, groups)
    W.train(net, groups, steps=args.warm_steps, lr=1e-3, batch=2, calibrate_scale=False)
    torch.cuda.synchronize()
    after = W.evaluate(net, groups)
    info = {"net": "3-level U-Net, base %d, BF16 weights, FP32 accumulation" % args.warm_base,
            "train_box": "%d^3, coarse cells of %d^3 fine cells (%s per side)" % (n_tr, f_tr, "x".join(map(str, dims[:3]))),
            "setups": args.warm_train, "samples": sum(d.n for d in groups), "steps": args.warm_steps,
            "output_scale": scale, "loss_unit": "mean square of the training targets",
            "train_mse_before": before, "train_mse_after": after, "train_mse_zero_net": zero,
            "train_iterations": iters, "seconds": time.perf_counter() - t0}
    return net, info


def full_increment(torch, P, g, s, stream, barrier, warm, host=None):
    """Solve the checkpointed increment to tolerance from the checkpoint;
    device time by CUDA events on the grid's stream.  With host buffers the
    same solve runs end to end: the FP64 history uploaded from pinned host
    memory first, the converged fields read back to it last, all inside the
    wall-clock region."""
    g.restore()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t0 = time.perf_counter()
    if host is not None:
        for f, b in host["in"].items():
            g.set_from(f, b.data_ptr(), b.numel())
    ev0.record(stream)
    g.apply_increment(s.a, s.dt, P.LOAD_XZ, use_warm_start=warm)
    info = g.solve_increment()
    ev1.record(stream)
    if host is not None:
        for f, b in host["out"].items():
            g.get_into(f, b.data_ptr(), b.numel())
    barrier()
    wall = time.perf_counter() - t0
    return ev0.elapsed_time(ev1), wall, info


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
    nchk = check_interval(s.n[0], "fp32")
    if args.precision == "fp64":
        args.no_warm = True
        nchk = check_interval(s.n[0], "fp64")
    net, training = (None, None) if args.no_warm else train_warm(args, torch, P, stream)

    # the benchmark box: the increments before the timed one, then a checkpoint
    g = prepare(P, s, args.precision, args.increment, args.kernel, stream.cuda_stream, nchk=nchk)
    if net is not None:
        g.attach_warm_start(net, args.coarsen)
    bpc = g.sweep_bytes_per_cell()
    walk = Walk(P, g, s, warm=net is not None)
    for _ in range(args.warmup):
        walk.step()
    clk = Clocks(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    sweeps = [walk.step() for _ in range(args.steps)]
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    sec = ev0.elapsed_time(ev1) * 1e-3
    tmax, total_bytes = aggregate(torch, dist, sec, bpc * cells * sum(sweeps), "cuda")
    gbs = total_bytes / tmax / 1e9
    ms_per_step = tmax / args.steps * 1e3

    # the timed increment solved whole from the checkpoint: warm start end to
    # end through the C ABI with host buffers, and the plain start
    fields_in = ["vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl",
                 "ux", "uy", "uz", "exx", "eyy", "ezz", "exy", "exz", "eyz"]
    fields_out = ["vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz", "p", "epl"]
    g.restore()
    host = {"in": {}, "out": {}}
    for f in ([] if args.no_increments else fields_in):
        b = torch.empty(g.count(f), dtype=torch.float64, pin_memory=True)
        g.get_into(f, b.data_ptr(), b.numel())
        host["in"][f] = b
    for f in ([] if args.no_increments else fields_out):
        host["out"][f] = torch.empty(g.count(f), dtype=torch.float64, pin_memory=True)
    h2d = sum(b.numel() * 8 for b in host["in"].values()) + 8 * 4
    d2h = sum(b.numel() * 8 for b in host["out"].values())
    arms = {}
    for name, warm in (("warm_fp32", net is not None), ("plain_fp32", False)):
        if (name == "warm_fp32" and net is None) or args.no_increments:
            continue
        dev_ms, wall, info = full_increment(torch, P, g, s, stream, barrier, warm,
                                            host if name == "warm_fp32" else None)
        arms[name] = {"ms_per_increment": dev_ms, "iterations": info["iters"], "frozen_at": info["frozen_at"],
                      "GB_per_s": bpc * cells * (info["iters"] + 1) / (dev_ms * 1e-3) / 1e9, "wall_ms": wall * 1e3}
    e2e = None
    if "warm_fp32" in arms:
        w = arms["warm_fp32"]
        e2e = {"value": bpc * cells * (w["iterations"] + 1) * world / (w["wall_ms"] * 1e-3) / 1e9, "unit": "GB/s",
               "ms_per_step": w["wall_ms"], "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "step": "one warm-start increment through the C ABI: FP64 history from pinned host memory, "
                       "start, solve to tolerance, converged fields back to pinned host memory"}

    # dominant sweep kernel: CUDA events on the library's stream around a
    # burst of launches on the open timed increment
    g.restore()
    g.apply_increment(s.a, s.dt, P.LOAD_XZ)
    ktimes = g.time_sweep(10 if s.n[0] > 300 else 20)
    kernels = kernel_names(ktimes, args.kernel)
    it_ms = ktimes[-1]
    dom = int(max(range(len(kernels)), key=lambda q: ktimes[q]))
    g.close()
    if net is not None:
        net.close()

    fp64 = None
    if not args.no_fp64 and not args.no_increments:
        g64 = prepare(P, s, "fp64", args.increment, "auto", stream.cuda_stream, nchk=nchk)
        dev_ms, _, i64 = full_increment(torch, P, g64, s, stream, barrier, False)
        fp64 = {"ms_per_increment": dev_ms, "iterations": i64["iters"], "frozen_at": i64["frozen_at"],
                "kernel": "staged",
                "GB_per_s": g64.sweep_bytes_per_cell() * cells * (i64["iters"] + 1) / (dev_ms * 1e-3) / 1e9}
        # its roof is FP64 arithmetic: flops of the sweeps against the FMA
        # rate measured on this device now
        peak64 = P.measure_fp64_peak()
        tf = FP64_FLOPS_PER_CELL * cells * (i64["iters"] + 1) / (dev_ms * 1e-3) / 1e12
        fp64["roofline"] = {"bound": "fp64-alu", "achieved": tf, "peak": peak64, "unit": "TFLOP/s",
                            "frac": tf / peak64, "flops_per_cell": FP64_FLOPS_PER_CELL,
                            "peak_source": "measured (ep_measure_fp64_peak, FMA chains, 2 flops per FMA)"}
        for name in arms:
            arms[name]["speedup_vs_fp64"] = dev_ms / arms[name]["ms_per_increment"]
        g64.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        lib_path, thr = oracle_lib(args.oracle_threads)
        per_inc, c_iters, c_cells = oracle_increment_rate(args.cpu_size, args.tol, args.increment, lib_path=lib_path)
        cpu = {"value": alg_bytes_per_cell(3, "fp64") * c_cells * c_iters / per_inc / 1e9, "unit": "GB/s",
               "cores": thr, "kind": "oracle",
               "sample": "increment %d of the same setup on a %d^3 grid, FP64 oracle on %d thread(s) "
                         "(%d iterations, %.2f s per increment)" % (args.increment, args.cpu_size, thr, c_iters,
                                                                   per_inc)}

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
            "traffic_source": NCU_SOURCE.get((kernels[dom], s.n[0])),
            "kernel_ms": {k: float(ktimes[q]) for q, k in enumerate(kernels)},
            "dominant": kernels[dom], "iteration_ms": float(it_ms), "alg_bytes_per_cell": bpc,
            "frac_recast_bytes": RECAST_BYTES_3D_FP32 * cells / (it_ms * 1e-3) / 1e9 / hbm}
    warm_desc = "warm start (3D U-Net on coarse cells of %d^3)" % args.coarsen if net is not None else "plain start"
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "3d-ep-xz-inclusion %d^3 (%d cells), increments from %d on, tol %g, %s sweeps, %s"
                   % (s.n[0], cells, args.increment, args.tol, args.precision, warm_desc),
                   "step": "one chunk of %d pseudo-transient sweeps of the increment sequence (a new increment, "
                           "with its warm-start inference and start state, is opened by the step that needs it; "
                           "a converged one is committed by the step that decides it)" % nchk,
                   "sweep_kernel": kernels[0] if len(kernels) == 1 else "staged",
                   "cells": cells, "sweeps_timed": sum(sweeps), "check_every": nchk,
                   "increments_finished": len(walk.finished),
                   "l2": "inputs larger than L2 (33 sweep arrays of %.1f MB)" % (cells * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "clocks": clocks,
        # per step: one graph of n_chk sweep launches plus the staged check (5
        # kernels and the check), and at an increment's start about 20
        # prologue kernels (+ about 40 network kernels with the warm start)
        "gpu_launches": int(args.steps * (nchk + 5) + 60 * (len(walk.finished) + 1)),
        "roofline": roof,
        "e2e": e2e,
        "per_increment": dict(arms, fp64_plain=fp64, increment=args.increment),
        "warm_start": training,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


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
        lib_path, thr = oracle_lib(args.oracle_threads)
        o = O.from_setup(small, lib_path=lib_path)
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
               "cores": thr, "kind": "oracle",
               "sample": "increment %d of one %dx%d instance (%s), FP64 oracle on %d thread(s), %d iterations "
                         "in %.2f s" % (args.batch_increment, small.n[0], small.n[1], small.name, thr, oi["iters"],
                                        ot)}
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
    if args.oracle_plan:
        return oracle_plan(args)
    if args.symmetry_study:
        return symmetry_study(args)
    if args.warm_study:
        return warm_study(args)
    if args.impl == "reference":
        return reference_arm(args)
    if args.batch > 0:
        return batch_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
