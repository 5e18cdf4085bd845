"""Pins of the FP64 network oracle (CPU): convolutions against scipy's
correlation (a library routine), gradients against central finite differences,
parameter count."""
import numpy as np
import pytest
from scipy import signal

from oracle import net_oracle as net


def _rand(*shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("stride,up", [(1, 0), (2, 0), (1, 1)])
def test_conv_matches_scipy_correlate(stride, up):
    x = _rand(2, 3, 8, 8, seed=1)
    w = _rand(4, 3, 3, 3, seed=2)
    b = _rand(4, seed=3)
    y = net.conv(x, w, b, stride, up)
    xu = x.repeat(2, axis=2).repeat(2, axis=3) if up else x
    for bb in range(2):
        for o in range(4):
            full = b[o] + sum(signal.correlate2d(xu[bb, c], w[o, c], mode="same") for c in range(3))
            assert np.allclose(y[bb, o], full[::stride, ::stride], atol=1e-12)


def test_parameter_count():
    _, n = net.layout()
    assert n == 1964690  # 1,963,440 weights + 1,250 biases


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    _, n = net.layout()
    params = np.zeros(n)
    for (wo, bo), (ci, co, *_) in zip(net.layout()[0], net.LAYERS):
        params[wo:wo + co * ci * 9] = rng.standard_normal(co * ci * 9) * np.sqrt(2.0 / (9 * ci))
        params[bo:bo + co] = 0.05 * rng.standard_normal(co)
    I = np.exp(rng.uniform(0, 6, (1, 128, 128)))
    t = rng.standard_normal((1, 2, 64, 64))
    L, g = net.loss_and_grads(params, I, t)
    h = 1e-5
    picks = []
    for l, ((wo, bo), (ci, co, *_)) in enumerate(zip(net.layout()[0], net.LAYERS)):
        picks.append(wo + int(rng.integers(co * ci * 9)))
        if l in (0, 5, 11):
            picks.append(bo + int(rng.integers(co)))
    for i in picks:
        p1 = params.copy()
        p2 = params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (net.loss_and_grads(p1, I, t)[0] - net.loss_and_grads(p2, I, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-4 * abs(fd), (i, fd, g[i])
