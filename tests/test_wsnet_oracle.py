"""Pins of the warm-start network oracle: its convolution equals scipy's
n-dimensional correlation, pooling/upsampling backward are the adjoints of
the forward maps, the parameter packing round-trips, the specified network
(4 levels, 32 base channels) has the stated layer shapes, and the
hand-written backward pass equals central finite differences of the forward
pass at every depth (with entries that have no target)."""
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


def test_pack_unpack_roundtrip_and_layout():
    rng = np.random.default_rng(4)
    p = rng.standard_normal(N.n_params(3, 2))
    np.testing.assert_array_equal(N.pack(N.unpack(p, 3, 2)), p)
    # first layer (cout 2, cin 1): W[co][t][ci] then b[co]
    W, b = N.unpack(p, 3, 2)[0]
    assert W.shape == (2, 1, 27)
    np.testing.assert_array_equal(W[1, 0, :], p[27:54])
    np.testing.assert_array_equal(b, p[54:56])
    # second layer (2 <- 2): tap-major, then input channel
    W1, _ = N.unpack(p, 3, 2)[1]
    np.testing.assert_array_equal(W1[0, 1, 5], p[56 + 5 * 2 + 1])


def test_specified_network_shapes():
    shapes = N.layer_shapes(4, 32)
    assert len(shapes) == 15
    assert shapes[0] == (32, 1) and shapes[-1] == (4, 32)
    assert [co for co, _ in shapes[:8:2]] == [32, 64, 128, 256]
    assert shapes[8] == (128, 256) and shapes[12] == (32, 64)
    assert N.n_params(4, 32) == sum(co * ci * 27 + co for co, ci in shapes)


@pytest.mark.parametrize("levels,base,side", [(3, 2, 8), (4, 2, 8), (2, 3, 4)])
def test_backward_matches_finite_differences(levels, base, side):
    rng = np.random.default_rng(2 + levels)
    pore = (rng.random((side, side, side)) > 0.3).astype(float)
    target = rng.standard_normal((N.NOUT, side, side, side))
    target[3][rng.random(target[3].shape) < 0.3] = np.nan  # entries without a target
    p = rng.standard_normal(N.n_params(levels, base)) * 0.3
    loss, g = N.loss_and_grad(p, pore, target, levels, base)
    # sample parameters from every layer
    idx, k = [], 0
    for co, ci in N.layer_shapes(levels, base):
        n = co * ci * 27 + co
        idx += list(rng.choice(n, 3, replace=False) + k)
        k += n
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp, _ = N.loss_and_grad(pp, pore, target, levels, base)
        lm, _ = N.loss_and_grad(pm, pore, target, levels, base)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_output_is_zero_in_solids():
    rng = np.random.default_rng(3)
    pore = (rng.random((4, 8, 4)) > 0.5).astype(float)
    p = rng.standard_normal(N.n_params(3, 2))
    Y = N.forward(p, pore, 3, 2)
    assert np.all(Y[:, pore == 0] == 0.0)


def test_entries_without_target_add_nothing():
    """A NaN target entry is the same as leaving that entry out of the sum:
    the loss equals the plain masked sum over the other entries."""
    rng = np.random.default_rng(6)
    pore = (rng.random((4, 4, 4)) > 0.3).astype(float)
    p = rng.standard_normal(N.n_params(2, 2)) * 0.3
    t = rng.standard_normal((N.NOUT, 4, 4, 4))
    t[3, 1:3] = np.nan
    loss, _ = N.loss_and_grad(p, pore, t, 2, 2)
    Y = N.forward(p, pore, 2, 2)
    keep = ~np.isnan(t) & (pore[None] > 0)
    want = float(((Y - np.nan_to_num(t)) ** 2)[keep].sum()) / (N.NOUT * pore.sum())
    assert abs(loss - want) <= 1e-12 * want
