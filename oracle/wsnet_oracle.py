"""FP64 numpy oracle of the warm-start network (forward and backward).

TEST INFRASTRUCTURE ONLY (like lbm_oracle): checks the CUDA network kernels.
The paper has no network; this is the library's own learned initial-field
predictor, written out plainly so its gradients can be checked.

Network (c = (c0, c1, c2) channels, volumes with every side divisible by 4):
    X  : pore indicator (1 pore, 0 solid), 1 channel
    L0a = relu(conv(X)),   L0b = relu(conv(L0a))                 full resolution
    L1a = relu(conv(pool(L0b))), L1b = relu(conv(L1a))            1/2
    L2a = relu(conv(pool(L1b))), L2b = relu(conv(L2a))            1/4
    L3a = relu(conv(up(L2b))),   L3b = relu(conv(L3a + L1b))      1/2
    L4a = relu(conv(up(L3b))),   L4b = relu(conv(L4a + L0b))      full
    Y   = conv(L4b) * X                                           3 channels (u / u_D)
    loss = sum over pore voxels and channels of (Y - T)^2 / (3 n_pore)
conv: 3x3x3 cross-correlation with zero padding and a bias; pool: 2x2x2 mean;
up: nearest-neighbour 2x.  Parameters are stored layer by layer as W[co][ci][27]
(taps ordered dz, dy, dx each in -1, 0, 1) followed by b[co].
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def layer_shapes(c0=8, c1=16, c2=32):
    """(cout, cin) of the 11 convolutions in forward order."""
    return [(c0, 1), (c0, c0), (c1, c0), (c1, c1), (c2, c1), (c2, c2),
            (c1, c2), (c1, c1), (c0, c1), (c0, c0), (3, c0)]


def n_params(c0=8, c1=16, c2=32):
    return sum(co * ci * 27 + co for co, ci in layer_shapes(c0, c1, c2))


def unpack(params, c0=8, c1=16, c2=32):
    out, k = [], 0
    for co, ci in layer_shapes(c0, c1, c2):
        W = params[k:k + co * ci * 27].reshape(co, ci, 27)
        k += co * ci * 27
        b = params[k:k + co]
        k += co
        out.append((W, b))
    assert k == params.size
    return out


def shift(a, dz, dy, dx):
    """b[..., z, y, x] = a[..., z + dz, y + dy, x + dx], zero outside."""
    b = np.zeros_like(a)
    nz, ny, nx = a.shape[-3:]
    zs = slice(max(0, -dz), nz - max(0, dz))
    ys = slice(max(0, -dy), ny - max(0, dy))
    xs = slice(max(0, -dx), nx - max(0, dx))
    zs2 = slice(max(0, dz), nz - max(0, -dz))
    ys2 = slice(max(0, dy), ny - max(0, -dy))
    xs2 = slice(max(0, dx), nx - max(0, -dx))
    b[..., zs, ys, xs] = a[..., zs2, ys2, xs2]
    return b


def conv(a, W, b):
    """out[co] = b[co] + sum_ci sum_t W[co, ci, t] a[ci](x + t)."""
    out = np.zeros((W.shape[0],) + a.shape[1:]) + b[:, None, None, None]
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = shift(a, dz, dy, dx)
        out += np.tensordot(W[:, :, t], s, axes=(1, 0))
    return out


def conv_backward(a, W, g):
    """Gradients of sum(g * conv(a, W, b)) w.r.t. a, W, b."""
    ga = np.zeros_like(a)
    gW = np.zeros_like(W)
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = shift(a, dz, dy, dx)
        gW[:, :, t] = np.tensordot(g, s, axes=([1, 2, 3], [1, 2, 3]))
        ga += shift(np.tensordot(W[:, :, t], g, axes=(0, 0)), -dz, -dy, -dx)
    gb = g.sum(axis=(1, 2, 3))
    return ga, gW, gb


def pool(a):
    c, nz, ny, nx = a.shape
    return a.reshape(c, nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(a):
    return np.repeat(np.repeat(np.repeat(a, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(g):
    c, nz, ny, nx = g.shape
    return g.reshape(c, nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(2, 4, 6))


def relu(a):
    return np.maximum(a, 0.0)


def forward(params, pore, chans=(8, 16, 32), keep=False):
    """pore: (nz, ny, nx) 0/1.  Returns Y (3, nz, ny, nx) and, if keep, the
    intermediate activations for backward."""
    Ls = unpack(np.asarray(params, dtype=np.float64), *chans)
    X = np.asarray(pore, dtype=np.float64)[None]
    A = {}
    A["L0a"] = relu(conv(X, *Ls[0]))
    A["L0b"] = relu(conv(A["L0a"], *Ls[1]))
    A["P1"] = pool(A["L0b"])
    A["L1a"] = relu(conv(A["P1"], *Ls[2]))
    A["L1b"] = relu(conv(A["L1a"], *Ls[3]))
    A["P2"] = pool(A["L1b"])
    A["L2a"] = relu(conv(A["P2"], *Ls[4]))
    A["L2b"] = relu(conv(A["L2a"], *Ls[5]))
    A["U1"] = up(A["L2b"])
    A["L3a"] = relu(conv(A["U1"], *Ls[6]))
    A["S1"] = A["L3a"] + A["L1b"]
    A["L3b"] = relu(conv(A["S1"], *Ls[7]))
    A["U0"] = up(A["L3b"])
    A["L4a"] = relu(conv(A["U0"], *Ls[8]))
    A["S0"] = A["L4a"] + A["L0b"]
    A["L4b"] = relu(conv(A["S0"], *Ls[9]))
    A["Z"] = conv(A["L4b"], *Ls[10])
    Y = A["Z"] * X
    A["X"] = X
    return (Y, A) if keep else Y


def loss_and_grad(params, pore, target, chans=(8, 16, 32)):
    """Masked mean squared error and its gradient w.r.t. the packed parameters."""
    params = np.asarray(params, dtype=np.float64)
    Ls = unpack(params, *chans)
    Y, A = forward(params, pore, chans, keep=True)
    X = A["X"]
    npore = X.sum()
    diff = (Y - target) * X
    loss = (diff ** 2).sum() / (3.0 * npore)
    gY = 2.0 * diff / (3.0 * npore)
    grads = [None] * 11

    def back(k, a_in, g_out):
        ga, gW, gb = conv_backward(a_in, Ls[k][0], g_out)
        grads[k] = (gW, gb)
        return ga

    gZ = gY * X
    g = back(10, A["L4b"], gZ)
    g = g * (A["L4b"] > 0)
    g_S0 = back(9, A["S0"], g)
    g = g_S0 * (A["L4a"] > 0)
    g_U0 = back(8, A["U0"], g)
    g_L0b = g_S0.copy()
    g = up_backward(g_U0) * (A["L3b"] > 0)
    g_S1 = back(7, A["S1"], g)
    g = g_S1 * (A["L3a"] > 0)
    g_U1 = back(6, A["U1"], g)
    g_L1b = g_S1.copy()
    g = up_backward(g_U1) * (A["L2b"] > 0)
    g = back(5, A["L2a"], g) * (A["L2a"] > 0)
    g_P2 = back(4, A["P2"], g)
    g_L1b += pool_backward(g_P2)
    g = g_L1b * (A["L1b"] > 0)
    g = back(3, A["L1a"], g) * (A["L1a"] > 0)
    g_P1 = back(2, A["P1"], g)
    g_L0b += pool_backward(g_P1)
    g = g_L0b * (A["L0b"] > 0)
    g = back(1, A["L0a"], g) * (A["L0a"] > 0)
    back(0, X, g)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
