"""Pins of the oracle's learned moment filter (a residual 3x3 convolutional
network on the deposited moments with the binomial smoothing as gated
fallback; not from the paper).  Checked against a library convolution
(scipy.signal.correlate2d with periodic wrap), identity networks, finite
differences of the loss, the closed form of bfloat16 rounding and the gate's
definition.  CPU only."""
import numpy as np
import pytest

import oracle as O

scipy_signal = pytest.importorskip("scipy.signal")

RNG = np.random.default_rng(777)
NP = O.FILTER_NPARAM


def grid(nx=10, nz=7, **kw):
    return O.make_grid(nx, 1, nz, 0.25, 1.0, 0.25, 0.01, n_floor=kw.pop("n_floor", 0.05), **kw)


def split(P):
    o = 0
    W1 = P[o:o + 576].reshape(16, 4, 3, 3); o += 576
    b1 = P[o:o + 16]; o += 16
    W2 = P[o:o + 2304].reshape(16, 16, 3, 3); o += 2304
    b2 = P[o:o + 16]; o += 16
    W3 = P[o:o + 576].reshape(4, 16, 3, 3); o += 576
    b3 = P[o:o + 4]
    return W1, b1, W2, b2, W3, b3


def test_bf16_rounding_closed_form():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -7, -2.5, 0.0, 3.0e38])
    got = O.bf16(vals)
    # 1+2^-8 is a tie between 1 and 1+2^-7 and goes to the even 1.0;
    # 1+3*2^-9 rounds up to 1+2^-7
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2 ** -7
    assert got[3] == 1.0 + 2 ** -7 and got[4] == -2.5 and got[5] == 0.0
    assert abs(got[6] - 3.0e38) / 3.0e38 < 2 ** -8


def test_zero_network_is_identity():
    g = grid()
    m = RNG.normal(size=(4, 70))
    m[0] = np.abs(m[0]) + 1.0
    y = O.filter_apply(g, np.zeros(NP), [1.0, 0.5, 0.5, 0.5], 0.0, 1e9, m)
    assert np.array_equal(y, m)


def test_network_conv_matches_scipy_correlate2d_wrap():
    """With non-negative inputs and weights every ReLU is inactive; W2 and W3
    pass channels through at the centre tap, so f_o is the periodic
    cross-correlation of x with W1[o] plus b1[o]."""
    nx, nz = 9, 6
    g = grid(nx, nz)
    P = np.zeros(NP)
    W1, b1, W2, b2, W3, b3 = split(P)
    W1[...] = RNG.uniform(0.0, 1.0, W1.shape)
    b1[...] = RNG.uniform(0.0, 0.5, 16)
    for c in range(16):
        W2[c, c, 1, 1] = 1.0
    for c in range(4):
        W3[c, c, 1, 1] = 1.0
    x = RNG.uniform(0.1, 2.0, (4, nz * nx))
    f, _, _ = O.filter_net(g, P, x, round_bf16=False)
    for o in range(4):
        ref = np.full((nz, nx), b1[o])
        for c in range(4):
            ref += scipy_signal.correlate2d(x[c].reshape(nz, nx), W1[o, c], mode="same",
                                            boundary="wrap")
        assert np.allclose(f[o].reshape(nz, nx), ref, atol=1e-12)


def test_relu_blocks_negative_preactivations():
    g = grid(6, 5)
    P = np.zeros(NP)
    W1, b1, W2, b2, W3, b3 = split(P)
    b1[:] = -1.0  # every layer-1 unit negative -> h1 = 0 -> f = conv(0) + b = b3
    b3[:] = [0.25, -0.5, 0.125, 2.0]
    x = RNG.normal(size=(4, 30))
    f, h1, _ = O.filter_net(g, P, x, round_bf16=False)
    assert np.all(h1 == 0.0)
    assert np.allclose(f, np.array(b3)[:, None])


@pytest.mark.parametrize("round_bf16", [False])
def test_gradient_matches_finite_differences(round_bf16):
    g = grid(5, 4)
    P = RNG.normal(size=NP) * 0.3
    s = np.array([1.0, 0.7, 0.7, 0.7])
    m = RNG.normal(size=(4, 20))
    m[0] = np.abs(m[0]) + 0.5
    t = m + 0.1 * RNG.normal(size=m.shape)
    loss, grad = O.filter_loss_grad(g, P, s, m, t, round_bf16=round_bf16)
    idx = RNG.choice(NP, 60, replace=False)
    idx = np.concatenate([idx, [575, 576, 591, 592, 2896, 2911, 3487, 3491]])
    h = 1e-6
    for q in idx:
        Pp = P.copy(); Pp[q] += h
        Pm = P.copy(); Pm[q] -= h
        lp, _ = O.filter_loss_grad(g, Pp, s, m, t, round_bf16=round_bf16)
        lm, _ = O.filter_loss_grad(g, Pm, s, m, t, round_bf16=round_bf16)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[q]) < 1e-6 * max(1.0, abs(fd)), (q, fd, grad[q])


def test_gate_falls_back_to_binomial():
    g = grid(8, 8, n_floor=0.05)
    m = RNG.uniform(0.5, 1.5, (4, 64))
    m[0, ::5] = 0.01  # below nmin
    P = np.zeros(NP)
    P[-4] = 1e-3  # b3[0]: small residual in the n channel everywhere
    y = O.filter_apply(g, P, [1.0, 1.0, 1.0, 1.0], 0.1, 1.0, m, round_bf16=False)
    sm = O.smooth(g, m, 1).reshape(4, -1)
    low = m[0] < 0.1
    assert np.allclose(y[:, low], sm[:, low])
    assert np.allclose(y[0, ~low], m[0, ~low] + 1e-3)
    # residual gate: a residual larger than rmax * n trips the fallback
    P[-4] = 10.0
    y = O.filter_apply(g, P, [1.0, 1.0, 1.0, 1.0], 0.0, 1.0, m, round_bf16=False)
    assert np.allclose(y, sm)
