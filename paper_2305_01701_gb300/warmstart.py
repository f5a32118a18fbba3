"""Learned warm start: data from the solver's own trajectories, training on
the GPU with the library's network kernels, and use in later solves.

Each sample is one increment n >= 3 of a plain-start solve.  The features,
computed by the library before the increment, describe the previous
increment's velocity change and the state it left (old stress and pressure
over the cohesion, the last return scale, the cohesion, the plastic strain);
the target, computed after the solve, is this increment's velocity change and
the relaxed-return part of its converged stress state (include/ep.h,
ep_warm_features / ep_warm_target).  A network that outputs zero reproduces
the plain start.  PyTorch only supplies the device buffers the library writes
into; every arithmetic step of collection, training and inference runs in the
library.
"""
from __future__ import annotations

import numpy as np

from ._native import LOAD_XY, LOAD_XZ, Net, warm_in, warm_out  # noqa: F401


def new_net(ndim, base=32, levels=3, seed=0, stream=None):
    """A warm-start network for ndim-dimensional grids."""
    return Net(ndim, warm_in(ndim), warm_out(ndim), base=base, levels=levels, seed=seed, stream=stream)


class Samples:
    """Features and targets of one padded size, in device buffers."""

    def __init__(self, ndim, dims, capacity, device="cuda"):
        import torch
        self.ndim, self.dims = ndim, tuple(dims)
        nv = int(np.prod([d for d in dims[:ndim]]))
        self.nv = nv
        self.cin, self.cout = warm_in(ndim), warm_out(ndim)
        self.x = torch.zeros((capacity, self.cin, nv), dtype=torch.float32, device=device)
        self.t = torch.zeros((capacity, self.cout, nv), dtype=torch.float32, device=device)
        torch.cuda.synchronize()   # zeroed before the library writes on its own stream
        self.n = 0

    def ptr_x(self, i):
        return self.x.data_ptr() + i * self.cin * self.nv * 4

    def ptr_t(self, i):
        return self.t.data_ptr() + i * self.cout * self.nv * 4


def collect(grid, a, dt, increments, samples, load_plane=LOAD_XY, coarsen=1, warm=False):
    """Solve `increments` increments on `grid` (plain start, or the attached
    network when warm) and store one sample per increment from the third on.
    Returns the iteration count of each increment."""
    grid.warm_record(True)
    iters = []
    for inc in range(1, increments + 1):
        have = inc >= 3 and samples is not None and samples.n < samples.x.shape[0]
        if have:
            grid.warm_features(samples.ptr_x(samples.n), coarsen)
        grid.apply_increment(a, dt, load_plane, use_warm_start=bool(warm and inc >= 3))
        info = grid.solve_increment()
        iters.append(info["iters"])
        if have:
            grid.warm_target(samples.ptr_t(samples.n), coarsen)
            samples.n += 1
    grid.warm_record(False)
    return iters


def calibrate(net, groups):
    """Set the network's output scale to the root mean square of the stored
    targets (the library's loss of the network with its output scaled to
    zero), so that its head, its loss and its gradients are of order one."""
    net.set_output_scale(0.0)
    ms = evaluate(net, groups)
    net.set_output_scale(float(np.sqrt(ms)) if ms > 0 else 1.0)
    return net.output_scale()


def train(net, groups, steps=400, lr=1e-3, batch=8, seed=0, calibrate_scale=True):
    """Adam on the MSE loss over minibatches of consecutive samples of one
    padded size (drawn at random), after setting the output scale from the
    targets (`calibrate`) unless told otherwise; returns the loss history."""
    rng = np.random.default_rng(seed)
    losses = []
    groups = [g for g in groups if g.n > 0]
    if calibrate_scale:
        calibrate(net, groups)
    for _ in range(steps):
        g = groups[rng.integers(len(groups))]
        nb = min(batch, g.n)
        i0 = int(rng.integers(0, g.n - nb + 1))
        size = list(g.dims[:g.ndim])
        losses.append(net.train_step(g.ptr_x(i0), g.ptr_t(i0), nb, size, lr))
    return losses


def evaluate(net, groups, batch=2):
    """Mean MSE of the network over every stored sample (weighted by sample)."""
    total, count = 0.0, 0
    for g in groups:
        size = list(g.dims[:g.ndim])
        for i0 in range(0, g.n, batch):
            nb = min(batch, g.n - i0)
            total += net.loss(g.ptr_x(i0), g.ptr_t(i0), nb, size) * nb
            count += nb
    return total / max(count, 1)


def zero_loss(net, groups):
    """The same mean loss, in the network's units, for its output scaled to
    zero, i.e. for the plain start (the warm start's fallback)."""
    s = net.output_scale()
    net.set_output_scale(0.0)
    ms = evaluate(net, groups)
    net.set_output_scale(s)
    return ms / (s * s) if s > 0 else ms
