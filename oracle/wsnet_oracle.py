"""FP64 numpy oracle of the warm-start network (forward and backward).

TEST INFRASTRUCTURE ONLY (like lbm_oracle): checks the CUDA network kernels.
The paper has no network; this is the library's own learned initial-field
predictor (a 3-D convolutional U-Net: `levels` resolution levels, `base`
channels at full resolution, doubling per level), written out plainly so its
gradients can be checked.

Network (c_l = base * 2^l channels at level l; every side divisible by
2^(levels - 1)):
    X    : pore indicator (1 pore, 0 solid), 1 channel
    E0a  = relu(conv(X)),        E0b = relu(conv(E0a))            level 0
    El a = relu(conv(pool(E(l-1)b))), El b = relu(conv(El a))     l = 1 .. L-1
    Dl a = relu(conv(up(D(l+1)b)))  (D(L-1)b := E(L-1)b)          l = L-2 .. 0
    Sl   = Dl a + El b,      Dl b = relu(conv(Sl))
    Y    = conv(D0b) * X         4 channels: u / u_D (3) and G = -dp/dz / (nu u_D)
    loss = sum over the entries with a target of (Y - T)^2 / (4 n_pore)
A target entry that is NaN has no target (the G channel is defined only where
a pore voxel's +z neighbour is a pore too); it adds nothing to the loss.
conv: 3x3x3 cross-correlation with zero padding and a bias; pool: 2x2x2 mean;
up: nearest-neighbour 2x.  Parameters are stored layer by layer (in the order
the convolutions run above) as W[co][27][ci] -- the 27 taps ordered dz, dy, dx,
each in -1, 0, 1, then the input channel -- followed by b[co].
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
NOUT = 4  # output channels: u_x, u_y, u_z (over u_D) and the pressure gradient G


def channels(levels=4, base=32):
    return [base * 2 ** l for l in range(levels)]


def layer_shapes(levels=4, base=32):
    """(cout, cin) of the convolutions in forward order."""
    c = channels(levels, base)
    shapes = [(c[0], 1), (c[0], c[0])]
    for l in range(1, levels):
        shapes += [(c[l], c[l - 1]), (c[l], c[l])]
    for l in range(levels - 2, -1, -1):
        shapes += [(c[l], c[l + 1]), (c[l], c[l])]
    shapes.append((NOUT, c[0]))
    return shapes


def n_params(levels=4, base=32):
    return sum(co * ci * 27 + co for co, ci in layer_shapes(levels, base))


def unpack(params, levels=4, base=32):
    """[(W[co][ci][27], b[co])] per layer from the packed W[co][27][ci], b[co] layout."""
    out, k = [], 0
    for co, ci in layer_shapes(levels, base):
        W = params[k:k + co * ci * 27].reshape(co, 27, ci).transpose(0, 2, 1)
        k += co * ci * 27
        b = params[k:k + co]
        k += co
        out.append((W, b))
    assert k == params.size
    return out


def pack(layers):
    """Inverse of unpack."""
    return np.concatenate([np.concatenate([W.transpose(0, 2, 1).ravel(), b]) for W, b in layers])


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


def forward(params, pore, levels=4, base=32, keep=False):
    """pore: (nz, ny, nx) 0/1.  Returns Y (3, nz, ny, nx) and, if keep, the
    intermediate activations for backward."""
    Ls = unpack(np.asarray(params, dtype=np.float64), levels, base)
    X = np.asarray(pore, dtype=np.float64)[None]
    A = {"X": X}
    k = 0
    inp = X
    for l in range(levels):
        if l > 0:
            inp = A["P%d" % l] = pool(A["E%db" % (l - 1)])
        A["E%da" % l] = relu(conv(inp, *Ls[k]))
        A["E%db" % l] = relu(conv(A["E%da" % l], *Ls[k + 1]))
        k += 2
    below = A["E%db" % (levels - 1)]
    for l in range(levels - 2, -1, -1):
        A["U%d" % l] = up(below)
        A["D%da" % l] = relu(conv(A["U%d" % l], *Ls[k]))
        A["S%d" % l] = A["D%da" % l] + A["E%db" % l]
        A["D%db" % l] = relu(conv(A["S%d" % l], *Ls[k + 1]))
        below = A["D%db" % l]
        k += 2
    A["Z"] = conv(below, *Ls[k])
    Y = A["Z"] * X
    return (Y, A) if keep else Y


def loss_and_grad(params, pore, target, levels=4, base=32):
    """Masked mean squared error and its gradient w.r.t. the packed parameters."""
    params = np.asarray(params, dtype=np.float64)
    Ls = unpack(params, levels, base)
    Y, A = forward(params, pore, levels, base, keep=True)
    X = A["X"]
    npore = X.sum()
    target = np.asarray(target, dtype=np.float64)
    has = ~np.isnan(target)
    diff = np.where(has, Y - np.where(has, target, 0.0), 0.0) * X
    loss = (diff ** 2).sum() / (NOUT * npore)
    gY = 2.0 * diff / (NOUT * npore)
    nl = len(Ls)
    grads = [None] * nl

    def back(k, a_in, g_out):
        ga, gW, gb = conv_backward(a_in, Ls[k][0], g_out)
        grads[k] = (gW, gb)
        return ga

    k = nl - 1
    top = "D0b" if levels > 1 else "E0b"
    g = back(k, A[top], gY * X)              # gradient w.r.t. the last feature map
    k -= 1
    g_skip = {}
    for l in range(0, levels - 1):           # decoder, top level first
        g = g * (A["D%db" % l] > 0)
        gS = back(k, A["S%d" % l], g)        # Dl b = relu(conv(Sl))
        g_skip[l] = gS                       # Sl = Dl a + El b
        g = gS * (A["D%da" % l] > 0)
        gU = back(k - 1, A["U%d" % l], g)    # Dl a = relu(conv(Ul))
        g = up_backward(gU)                  # into D(l+1)b, or E(L-1)b at the bottom
        k -= 2
    for l in range(levels - 1, -1, -1):      # encoder, bottom level first
        if l < levels - 1:
            g = g + g_skip[l]
        g = g * (A["E%db" % l] > 0)
        g = back(k, A["E%da" % l], g) * (A["E%da" % l] > 0)
        inp = A["P%d" % l] if l > 0 else X
        g = back(k - 1, inp, g)
        if l > 0:
            g = pool_backward(g)
        k -= 2
    assert k == -1
    return loss, pack([(gW, gb) for gW, gb in grads])
