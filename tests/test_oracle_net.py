"""Pins of the oracle's network reference (oracle/net.py): the tap convention
on an identity and a one-tap shift kernel, and the backward pass against
central finite differences (no GPU)."""
import numpy as np

from oracle import net as ON


def _params(L, C, rng, scale=0.4):
    Ws = [rng.standard_normal((3, 3, C, C)) * scale for _ in range(L)]
    bs = [rng.standard_normal(C) * 0.1 for _ in range(L)]
    return Ws, bs


def test_identity_and_shift_convention():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    W = np.zeros((3, 3, 3, 3))
    W[1, 1] = np.eye(3)                                   # centre tap: out = in
    out, _ = ON.forward(x, [W], [np.zeros(3)])
    assert np.array_equal(out, x)
    W = np.zeros((3, 3, 3, 3))
    W[0, 1] = np.eye(3)                                   # tap (dy, dx) = (0, 1): offset (-1, 0)
    out, _ = ON.forward(x, [W], [np.zeros(3)])
    assert np.array_equal(out[:, 1:], x[:, :-1]) and not out[:, 0].any()
    W = np.zeros((3, 3, 3, 3))
    W[1, 2] = np.eye(3)                                   # offset (0, +1)
    out, _ = ON.forward(x, [W], [np.ones(3)])
    assert np.allclose(out[:, :, :-1], x[:, :, 1:] + 1) and np.allclose(out[:, :, -1], 1)


def test_backward_against_finite_differences():
    rng = np.random.default_rng(1)
    L, C, N = 3, 4, 5
    Ws, bs = _params(L, C, rng)
    x = rng.standard_normal((2, N, N, C))
    t = rng.standard_normal((2, N, N, 2))

    def f(Ws_, bs_, x_):
        out, _ = ON.forward(x_, Ws_, bs_)
        return ON.loss(out, t)

    out, cache = ON.forward(x, Ws, bs)
    dWs, dbs, dx = ON.backward(out, t, cache, Ws)
    h = 1e-6
    for l in range(L):
        for idx in [(0, 0, 0, 1), (1, 1, 2, 3), (2, 1, 3, 0), (1, 2, 1, 1)]:
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (f(Wp, bs, x) - f(Wm, bs, x)) / (2 * h)
            assert abs(fd - dWs[l][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, dWs[l][idx])
        for c in range(C):
            bp = [b.copy() for b in bs]
            bm = [b.copy() for b in bs]
            bp[l][c] += h
            bm[l][c] -= h
            fd = (f(Ws, bp, x) - f(Ws, bm, x)) / (2 * h)
            assert abs(fd - dbs[l][c]) <= 1e-6 * max(1.0, abs(fd))
    # the input gradient of the first layer (no relu below it)
    for idx in [(0, 0, 0, 0), (1, 2, 3, 1), (0, 4, 4, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (f(Ws, bs, xp) - f(Ws, bs, xm)) / (2 * h)
        assert abs(fd - dx[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding():
    # round-to-nearest-even to an 8-bit significand
    # (ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and goes to the even
    # significand 1; 1 + 3*2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6)
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -2.5, 3.0e38])
    r = ON.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6 and r[3] == 1.0 + 2 ** -7 and r[4] == 1.0
    assert r[5] == -2.5 and np.isfinite(r[6])
