"""Square-duct Poiseuille series (Section 3.1, Eq. poiseuille_theory).

TEST INFRASTRUCTURE ONLY (see lbm_oracle).

u_z(x, y) = 16 a^2 / (nu pi^3) (-dp/dz) sum_{k odd} (-1)^((k-1)/2)
            [1 - cosh(k pi x / 2w) / cosh(k pi / 2)] cos(k pi y / 2w) / k^3
on -w <= x, y <= w.  The paper leaves "a" undefined; it is read as the
half-width w (the only length in the problem that makes the series satisfy
nu lap(u) = dp/dz).  The series is truncated at k = 200 as in the paper.
"""
from __future__ import annotations

import numpy as np


def duct_velocity(x, y, w, nu, dpdz, kmax=200):
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    s = np.zeros(np.broadcast(x, y).shape)
    for k in range(1, kmax + 1, 2):
        a = k * np.pi / (2.0 * w)
        # cosh(a x) / cosh(k pi / 2) evaluated without overflow
        ratio = np.exp(a * np.abs(x) - k * np.pi / 2.0) * (1.0 + np.exp(-2.0 * a * np.abs(x))) \
            / (1.0 + np.exp(-k * np.pi))
        s = s + (-1.0) ** ((k - 1) // 2) * (1.0 - ratio) * np.cos(a * y) / k ** 3
    return 16.0 * w * w / (nu * np.pi ** 3) * (-dpdz) * s


def duct_flow_rate_per_gradient(w, nu, n=400, kmax=200):
    """Integral of the series over the square for -dp/dz = 1 (midpoint rule, n x n)."""
    h = 2.0 * w / n
    c = -w + h * (np.arange(n) + 0.5)
    X, Y = np.meshgrid(c, c, indexing="ij")
    return duct_velocity(X, Y, w, nu, -1.0, kmax).sum() * h * h
