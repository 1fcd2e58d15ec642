"""Plain FP64 CPU reference of the learned preconditioner's network (oracle;
test infrastructure only: imported by tests/ alone, never by the CUDA path).

The network maps a residual r of a shifted system (z_j I - A) e = r on an
N x N grid (the 2-D convection-diffusion operator of the workloads) to an
approximate correction e.  It is a stack of 3x3 convolutions with zero
padding at the grid boundary (the Dirichlet boundary of the operator):
    a_0 = input image (C channels, zero-padded up to C)
    z_l = conv3x3(a_{l-1}; W_l) + b_l,   a_l = relu(z_l)  (l < L),  out = z_L
with W_l of shape (3, 3, C, C) indexed [dy, dx, c_in, c_out] (tap offset
(dy - 1, dx - 1)) and b_l of shape (C,).  Images are (batch, N, N, C)
channel-last.  The loss is the mean squared error over the first `cout`
output channels, L = sum((out[..., :cout] - target)^2) / target.size.

Every function is the plain definition (explicit loops over the nine taps;
numpy for the channel contractions), so that it can be checked by eye.
The input gradient returned by backward() is d loss / d input, except that
for the layers below the top it already carries relu' of the layer it feeds
(the gradient of the pre-activation).  Pins: tests/test_oracle_net.py."""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in range(3) for dx in range(3)]


def shift(a, dy, dx):
    """s[b, y, x, c] = a[b, y + dy - 1, x + dx - 1, c], zero outside the grid."""
    B, N, M, C = a.shape
    s = np.zeros_like(a)
    oy, ox = dy - 1, dx - 1
    ys, ye = max(0, -oy), min(N, N - oy)
    xs, xe = max(0, -ox), min(M, M - ox)
    s[:, ys:ye, xs:xe, :] = a[:, ys + oy:ye + oy, xs + ox:xe + ox, :]
    return s


def conv3x3(a, W, b):
    """z[b, y, x, o] = b[o] + sum_{dy, dx, i} W[dy, dx, i, o] a[b, y+dy-1, x+dx-1, i]."""
    z = np.zeros(a.shape[:3] + (W.shape[3],))
    for dy, dx in TAPS:
        z += shift(a, dy, dx) @ W[dy, dx]
    return z + b


def bf16(x):
    """Round to bfloat16 (8-bit significand), round-to-nearest-even, as a float.
    The rounding points of the BF16 network: weights, the input and every
    hidden activation, and the stored gradients."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(x, Ws, bs, quant=False):
    """Returns the output and the list of (input, pre-activation) of each layer.
    quant: round weights, input and hidden activations to bfloat16 (biases and
    the last layer's output stay in single precision)."""
    q = bf16 if quant else (lambda v: v)
    a = q(x)
    cache = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = conv3x3(a, q(W), np.float32(b).astype(np.float64) if quant else b)
        cache.append((a, z))
        a = q(np.maximum(z, 0.0)) if l < len(Ws) - 1 else z
    return a, cache


def loss(out, target):
    cout = target.shape[-1]
    d = out[..., :cout] - target
    return float(np.sum(d * d) / target.size)


def backward(out, target, cache, Ws, quant=False):
    """Gradients of loss() with respect to every W_l, b_l and the input.
    quant: the bfloat16 rounding points of the BF16 network (weights, the
    output gradient and every propagated activation gradient)."""
    q = bf16 if quant else (lambda v: v)
    Ws = [q(W) for W in Ws]
    cout = target.shape[-1]
    g = np.zeros_like(out)
    g[..., :cout] = 2.0 * (out[..., :cout] - target) / target.size
    g = q(g)
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        a, z = cache[l]
        dbs[l] = g.sum(axis=(0, 1, 2))
        dW = np.zeros_like(Ws[l])
        for dy, dx in TAPS:
            sa = shift(a, dy, dx)
            dW[dy, dx] = sa.reshape(-1, sa.shape[-1]).T @ g.reshape(-1, g.shape[-1])
        dWs[l] = dW
        # input gradient: the adjoint of conv3x3 (shifts in the opposite direction)
        ga = np.zeros_like(a)
        for dy, dx in TAPS:
            ga += shift(g @ Ws[l][dy, dx].T, 2 - dy, 2 - dx)
        if l > 0:
            ga = q(ga * (cache[l - 1][1] > 0))        # relu' of the layer below
        g = ga
    return dWs, dbs, g
