"""Pins of the warm-start network oracle: its convolution equals scipy's
n-dimensional correlation, pooling/upsampling backward are the adjoints of
the forward maps, and the hand-written backward pass equals central finite
differences of the forward pass."""
import numpy as np
import pytest

from oracle import wsnet_oracle as N


def test_conv_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 5, 6, 7))
    W = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    out = N.conv(a, W, b)
    for co in range(3):
        want = np.full(a.shape[1:], b[co])
        for ci in range(2):
            k = W[co, ci].reshape(3, 3, 3)  # [dz][dy][dx] with offsets -1, 0, 1
            want += ndimage.correlate(a[ci], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(out[co], want, atol=1e-12)


def test_pool_up_adjoint():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 4, 6, 8))
    g = rng.standard_normal((2, 2, 3, 4))
    assert abs((N.pool(a) * g).sum() - (a * N.pool_backward(g)).sum()) < 1e-12
    h = rng.standard_normal((2, 4, 6, 8))
    assert abs((N.up(g) * h).sum() - (g * N.up_backward(h)).sum()) < 1e-12
    np.testing.assert_allclose(N.pool(N.up(g)), g)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    chans = (2, 3, 4)
    pore = (rng.random((8, 8, 8)) > 0.3).astype(float)
    target = rng.standard_normal((3, 8, 8, 8))
    p = rng.standard_normal(N.n_params(*chans)) * 0.3
    loss, g = N.loss_and_grad(p, pore, target, chans)
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp, _ = N.loss_and_grad(pp, pore, target, chans)
        lm, _ = N.loss_and_grad(pm, pore, target, chans)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_output_is_zero_in_solids():
    rng = np.random.default_rng(3)
    pore = (rng.random((4, 8, 4)) > 0.5).astype(float)
    p = rng.standard_normal(N.n_params(2, 2, 2))
    Y = N.forward(p, pore, (2, 2, 2))
    assert np.all(Y[:, pore == 0] == 0.0)
