"""FP64 numpy oracle of the warm-start U-Net (forward, loss, gradient).

TEST INFRASTRUCTURE: used only by the tests to check the CUDA network.

The parameter vector follows the library's layout: layers in forward order
(encoder levels, then decoder levels from coarse to fine, then the head);
each layer stores its weights W[c_out][c_in][taps] (taps x fastest, then y,
then z) followed by its c_out biases.  Convolutions zero-pad by one cell;
pooling averages 2^D cells; upsampling repeats each cell 2^D times; the
decoder input concatenates [upsampled coarser output, skip] along channels.

The gradient is taken by central finite differences of the FP64 forward, a
method independent of any back-propagation code.

`forward(..., bf16_inputs=True)` states the precision of the library's
inference forward on the tensor cores: the input of every 3^D convolution
whose output has a multiple of 16 channels (16 to 128) is rounded to BF16
(nearest, ties to even) before the product; everything else stays FP64.
"""
from __future__ import annotations

import numpy as np


def layer_table(ndim, cin, cout, base, levels):
    """(c_in, c_out, k, weight offset, bias offset) in forward order."""
    out, off = [], 0

    def add(ci, co, k):
        nonlocal off
        taps = k ** ndim
        wo = off
        off += ci * co * taps
        bo = off
        off += co
        out.append((ci, co, k, wo, bo))

    cp = cin
    for l in range(levels):
        c = base << l
        add(cp, c, 3)
        add(c, c, 3)
        cp = c
    for l in range(levels - 2, -1, -1):
        c, cup = base << l, base << (l + 1)
        add(cup + c, c, 3)
        add(c, c, 3)
    add(base, cout, 1)
    return out, off


def conv(x, w, b, k):
    """x: (N, Cin, [Z,] Y, X); w: (Cout, Cin, k^D) taps x fastest; zero padding."""
    nd = x.ndim - 2
    r = k // 2
    cout = w.shape[0]
    pad = [(0, 0), (0, 0)] + [(r, r)] * nd
    xp = np.pad(x, pad)
    shape = x.shape[2:]
    y = np.zeros((x.shape[0], cout) + shape)
    y += b.reshape((1, cout) + (1,) * nd)
    taps = w.reshape(cout, w.shape[1], *([k] * nd))  # (co, ci, [kz,] ky, kx)
    for idx in np.ndindex(*([k] * nd)):
        sl = tuple(slice(idx[d], idx[d] + shape[d]) for d in range(nd))
        xs = xp[(slice(None), slice(None)) + sl]
        y += np.einsum("oi,ni...->no...", taps[(slice(None), slice(None)) + idx], xs)
    return y


def pool(x):
    nd = x.ndim - 2
    s = x.shape
    if nd == 2:
        return x.reshape(s[0], s[1], s[2] // 2, 2, s[3] // 2, 2).mean(axis=(3, 5))
    return x.reshape(s[0], s[1], s[2] // 2, 2, s[3] // 2, 2, s[4] // 2, 2).mean(axis=(3, 5, 7))


def up(x):
    y = x
    for ax in range(2, x.ndim):
        y = np.repeat(y, 2, axis=ax)
    return y


def round_bf16(a):
    """Nearest BF16 value (ties to even) of each element, as FP64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, ndim, cin, cout, base, levels, bf16_inputs=False):
    table, n = layer_table(ndim, cin, cout, base, levels)
    assert params.size == n
    li = 0

    def apply(inp, relu):
        nonlocal li
        ci, co, k, wo, bo = table[li]
        li += 1
        w = params[wo:wo + ci * co * k ** ndim].reshape(co, ci, k ** ndim)
        b = params[bo:bo + co]
        if bf16_inputs and k == 3 and co % 16 == 0 and 16 <= co <= 128:
            inp = round_bf16(inp)
        y = conv(inp, w, b, k)
        return np.maximum(y, 0.0) if relu else y

    skips = []
    h = x
    for l in range(levels):
        h = apply(h, True)
        h = apply(h, True)
        skips.append(h)
        if l < levels - 1:
            h = pool(h)
    for l in range(levels - 2, -1, -1):
        h = np.concatenate([up(h), skips[l]], axis=1)
        h = apply(h, True)
        h = apply(h, True)
    return apply(h, False)


def loss(params, x, t, *arch):
    y = forward(params, x, *arch)
    return float(np.mean((y - t) ** 2))


def fd_gradient(params, x, t, *arch, h=1e-6):
    g = np.zeros_like(params)
    for i in range(params.size):
        p1 = params.copy()
        p1[i] += h
        p2 = params.copy()
        p2[i] -= h
        g[i] = (loss(p1, x, t, *arch) - loss(p2, x, t, *arch)) / (2 * h)
    return g
