"""Host helpers of the learned warm start (no GPU): the pore-solid face count
of the Kozeny-Carman estimate against hand counts, the least-squares fit of
its constant, and the seeded He initialisation's layout and spread."""
import math

import numpy as np

from paper_1806_10589_gb300 import warmstart as ws


def test_surface_density_open_box():
    # all pore: only the four lateral box faces count (walls), the z ends do not
    nz, ny, nx = 5, 4, 3
    m = np.zeros((nz, ny, nx), np.uint8)
    assert ws.surface_density(m) == (2 * nz * nx + 2 * nz * ny) / m.size


def test_surface_density_one_interior_solid():
    nz, ny, nx = 5, 5, 5
    m = np.zeros((nz, ny, nx), np.uint8)
    m[2, 2, 2] = 1
    walls = 2 * nz * nx + 2 * nz * ny
    assert ws.surface_density(m) == (walls + 6) / m.size


def test_surface_density_all_solid_and_slab():
    assert ws.surface_density(np.ones((3, 4, 5), np.uint8)) == 0.0
    # a solid x-slab at x = 0 of a 4 x 3 x 6 box: it replaces the x = 0 wall by
    # the slab's face toward x = 1 (same count), the y walls lose the slab's cells
    nz, ny, nx = 4, 3, 6
    m = np.zeros((nz, ny, nx), np.uint8)
    m[:, :, 0] = 1
    faces = nz * ny + nz * ny + 2 * nz * (nx - 1)
    assert ws.surface_density(m) == faces / m.size


def test_kc_features():
    m = np.zeros((5, 5, 5), np.uint8)
    m[2, 2, 2] = 1
    phi, S, x = ws.kc_features(m)
    assert phi == 124 / 125
    assert S == ws.surface_density(m)
    assert math.isclose(x, phi ** 3 / (S * S * (1 - phi) ** 2), rel_tol=1e-15)


def test_fit_kc_recovers_the_constant():
    rng = np.random.default_rng(3)
    masks = [(rng.random((6, 6, 6)) < p).astype(np.uint8) for p in (0.2, 0.3, 0.4, 0.5)]
    x = np.array([ws.kc_features(m)[2] for m in masks])
    assert math.isclose(ws.fit_kc(masks, 0.37 * x), 0.37, rel_tol=1e-12)
    # least squares in log k: multiplicative errors of +-10 % cancel in the geometric mean
    noisy = 0.37 * x * np.array([1.1, 1 / 1.1, 1.1, 1 / 1.1])
    assert math.isclose(ws.fit_kc(masks, noisy), 0.37, rel_tol=1e-12)


class _Net:
    def __init__(self, levels=4, base=32):
        self.levels, self.base = levels, base
        self.n_params = sum(co * ci * 27 + co for co, ci in self.layer_shapes())

    def layer_shapes(self):
        from oracle import wsnet_oracle as N

        return N.layer_shapes(self.levels, self.base)


def test_he_init_layout_and_spread():
    net = _Net()
    p = ws.he_init(net, 7)
    assert p.dtype == np.float32 and p.size == net.n_params
    np.testing.assert_array_equal(p, ws.he_init(net, 7))
    k = 0
    for co, ci in net.layer_shapes():
        w = p[k:k + co * ci * 27]
        b = p[k + co * ci * 27:k + co * ci * 27 + co]
        assert not b.any()
        target = math.sqrt(2.0 / (27 * ci))
        # sample standard deviation of n normal draws: relative error ~ 1/sqrt(2n)
        assert abs(w.std() / target - 1) < 5 / math.sqrt(2 * w.size)
        k += co * ci * 27 + co
    assert k == p.size


def test_pressure_profile_inverts_the_drop_target():
    """For any density field, the predicted-drop profile built from the exact
    targets gives back the plane-mean density of every plane (the outlet
    plane's mean as rho_out); targets exist on the pore voxels of every plane
    but the last."""
    nz, ny, nx = 9, 4, 5
    rng = np.random.default_rng(2)
    m = (rng.random((nz, ny, nx)) < 0.3).astype(np.uint8)
    m[:, 0, 0] = 0  # a pore in every plane
    rho = 1.0 + 1e-3 * rng.random(m.shape)
    Q, tau = 0.02, 0.8
    G = ws.drop_target(rho, m, Q, tau)
    defined = np.zeros(m.shape, bool)
    defined[:-1] = m[:-1] == 0
    np.testing.assert_array_equal(np.isfinite(G), defined)
    pbar = ws.plane_means(rho, m)
    np.testing.assert_allclose(ws.pressure_profile(G, m, Q, tau, rho_out=pbar[-1]), pbar, rtol=0, atol=1e-14)
    # the drop is constant over a plane's pores
    for z in range(nz - 1):
        vals = G[z][m[z] == 0]
        assert np.ptp(vals) == 0.0


def test_kc_profile_is_the_darcy_ramp():
    m = np.zeros((6, 5, 5), np.uint8)
    m[2, 2, 2] = 1
    Q, tau, c = 0.01, 0.7, 0.2
    prof = ws.kc_profile(m, Q, tau, c)
    k_est = c * ws.kc_features(m)[2]
    nu = (tau - 0.5) / 3.0
    dp = nu * Q / 25.0 * 5 / k_est
    np.testing.assert_allclose(prof, 1.0 + 3.0 * dp * (1 - np.arange(6) / 5.0), rtol=1e-14)
    # the permeability the 0.1 % rule reads off this profile is the Kozeny-Carman estimate
    # (rho_in - 1 is ~6e-8 here, so its FP64 rounding is ~2e-9 relative)
    from paper_1806_10589_gb300 import convergence as cv
    assert math.isclose(cv.permeability(Q, m.shape, tau, prof[0], prof[-1]), k_est, rel_tol=1e-7)


def test_fit_net_scale_recovers_a_biased_network():
    """A stand-in network whose pressure drops are twice the true ones implies
    half the permeability; the calibration constant is then exactly 2, and the
    calibrated estimate is the true permeability."""
    from paper_1806_10589_gb300 import convergence as cv

    tau, u_mean = 0.8, 1e-4
    boxes, ks, fields = [], [], []
    rng = np.random.default_rng(5)
    for k in range(3):
        m = (rng.random((8, 6, 6)) < 0.3).astype(np.uint8)
        m[:, 0, 0] = 0
        Q = u_mean * int((m[0] == 0).sum())
        rho = 1.0 + 1e-4 * (7 - np.arange(8))[:, None, None] * (1 + 0.1 * rng.random(m.shape))
        rho[-1] = 1.0
        G = ws.drop_target(rho, m, Q, tau)
        pbar = ws.plane_means(rho, m)
        ks.append(cv.permeability(Q, m.shape, tau, pbar[0], 1.0))
        boxes.append(m)
        fields.append(np.nan_to_num(G))

    class Biased:
        def __init__(self):
            self.k = 0

        def predict(self, mask):
            idx = [i for i, b in enumerate(boxes) if b is mask][0]
            y = np.zeros((4,) + mask.shape, np.float32)
            y[3] = 2.0 * fields[idx]
            return y

    net = Biased()
    c = ws.fit_net_scale(net, boxes, ks, tau, u_mean)
    assert math.isclose(c, 2.0, rel_tol=1e-6)
    for m, k in zip(boxes, ks):
        Q = u_mean * int((m[0] == 0).sum())
        assert math.isclose(ws.net_permeability(net, m, Q, tau, c_net=c), k, rel_tol=1e-6)
