"""Pins of the colour-model oracle (Appendix A): it reduces exactly to the
single-fluid oracle when only one phase is present, conserves the mass of each
phase in a closed box, its gradient stencil is exact on linear fields and equals
a voxel loop, its interfacial terms give the closed-form stress of a unit
normal, its recolouring sends each D3Q7 value as the printed update says, and
the inlet flux stays exact."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import color_oracle as CO
from lbm_inputs import duct_mask, random_mask, uniform_field


def test_single_phase_limit_is_the_single_fluid_oracle():
    """phi = +1 everywhere and solids that look like phase A: no colour
    gradient, so f evolves exactly as in the single-fluid scheme."""
    m = random_mask(7, 6, 9, 0.25, 3)
    c = CO.ColourOracle(m, 0.8, alpha=0.01, beta=0.95, phi_s=1.0, Q=0.004)
    s = O.D3Q19Oracle(m, 0.8, "mrt", Q=0.004)
    for _ in range(12):
        c.step()
        s.step()
    np.testing.assert_array_equal(c.f, s.f)
    phi = c.phase_field()[0]
    np.testing.assert_allclose(phi[m == 0], 1.0, atol=1e-15)


def test_closed_box_conserves_each_phase():
    m = random_mask(8, 7, 8, 0.2, 4)
    m[0] = 1
    m[-1] = 1
    c = CO.ColourOracle(m, 1.0, alpha=0.005, beta=0.9, phi_s=-1.0, inlet=None, outlet=None)
    phi0 = np.tanh(uniform_field(m.shape, 5) * 3)
    c.init_phase(phi0)
    a0 = math.fsum(c.A.ravel().tolist())
    b0 = math.fsum(c.B.ravel().tolist())
    r0 = math.fsum(c.f.ravel().tolist())
    c.step(25)
    assert abs(math.fsum(c.A.ravel().tolist()) - a0) <= 1e-12 * a0
    assert abs(math.fsum(c.B.ravel().tolist()) - b0) <= 1e-12 * b0
    assert abs(math.fsum(c.f.ravel().tolist()) - r0) <= 1e-12 * r0


def test_gradient_exact_on_linear_field_and_matches_loops():
    m = np.zeros((6, 7, 8), np.uint8)
    z, y, x = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    phi = 0.1 * x - 0.2 * y + 0.05 * z
    C = CO.colour_gradient(phi, m, 0.0)
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(C[0][inner], 0.1, atol=1e-14)
    np.testing.assert_allclose(C[1][inner], -0.2, atol=1e-14)
    np.testing.assert_allclose(C[2][inner], 0.05, atol=1e-14)
    mm = random_mask(5, 5, 6, 0.3, 7)
    ph = uniform_field(mm.shape, 8)
    np.testing.assert_allclose(CO.colour_gradient(ph, mm, -0.5), CO.colour_gradient_loops(ph, mm, -0.5), atol=1e-14)


def _unit(rng):
    n = rng.standard_normal(3)
    return n / np.linalg.norm(n)


def _quadratic_with_moments(Pi):
    """The one D3Q19 population g_q = l0 + sum_ab l_ab xi_a xi_b (a quadratic
    polynomial of the velocity, no linear part) with sum_q g_q = 0 and
    sum_q xi_a xi_b g_q = Pi_ab.  Built from the velocity set alone, not from
    the oracle's moment matrix."""
    xi = O.XI.astype(float)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]
    basis = np.stack([np.ones(19)] + [xi[:, a] * xi[:, b] for a, b in pairs], axis=1)  # (19, 7)
    rows = np.stack([np.ones(19)] + [xi[:, a] * xi[:, b] for a, b in pairs], axis=0)   # (7, 19)
    rhs = np.array([0.0] + [Pi[a, b] for a, b in pairs])
    coef = np.linalg.solve(rows @ basis, rhs)
    return basis @ coef


def test_interfacial_terms_give_the_closed_form_stress():
    """Appendix A adds alpha|C| to m1 = e (row 19c^2 - 30), alpha|C|/2 (2nx^2 -
    ny^2 - nz^2) to 3p_xx (row 3cx^2 - c^2), alpha|C|/2 (ny^2 - nz^2) to p_ww
    (row cy^2 - cz^2) and alpha|C|/2 n_a n_b to p_xy, p_yz, p_zx.  Read through
    those row polynomials, the added population carries no mass or momentum,
    its traceless second moment is (|C|/2)(n n - I/3) and its trace is |C|/19
    (sum c^2 g = m1/19).  It lies in the span of the rows e and p, so it is the
    quadratic polynomial of xi with those moments.  All these rows relax at
    s_nu, so the collision adds s_nu alpha times it.  A sign, index or factor
    slip in any of the six terms changes some direction's value."""
    rng = np.random.default_rng(31)
    tau, alpha = 0.8, 0.013
    s_nu = 1.0 / tau
    F = O.W[:, None] * (1.0 + 0.02 * rng.standard_normal((19, 6)))
    for trial in range(6):
        C = np.stack([_unit(rng) * rng.uniform(0.05, 2.0) for _ in range(6)], axis=1)  # (3, 6)
        dm, nvec = CO.interfacial_moments(C)
        diff = CO.collide_colour(F, tau, alpha, dm) - CO.collide_colour(F, tau, 0.0, dm)
        for k in range(6):
            mag = np.linalg.norm(C[:, k])
            n = C[:, k] / mag
            np.testing.assert_allclose(nvec[:, k], n, rtol=0, atol=1e-15)
            Pi = 0.5 * mag * (np.outer(n, n) - np.eye(3) / 3.0) + mag / 57.0 * np.eye(3)
            want = s_nu * alpha * _quadratic_with_moments(Pi)
            scale = s_nu * alpha * mag
            np.testing.assert_allclose(diff[:, k], want, rtol=0, atol=1e-13 * scale)
            # no mass, no momentum (up to the rounding of F ~ 0.3 in the two collisions)
            assert abs(diff[:, k].sum()) <= 1e-15
            np.testing.assert_allclose(O.XI.T.astype(float) @ diff[:, k], 0.0, atol=1e-15)
    # physical direction: the added normal stress is largest along n
    C = np.array([[0.7], [0.0], [0.0]])
    dm, _ = CO.interfacial_moments(C)
    g = CO.collide_colour(F[:, :1], tau, alpha, dm) - CO.collide_colour(F[:, :1], tau, 0.0, dm)
    xi = O.XI.astype(float)
    pxx, pyy, pzz = ((xi[:, a] ** 2) @ g[:, 0] for a in range(3))
    np.testing.assert_allclose(pxx - pyy, s_nu * alpha * 0.35, rtol=1e-13)
    np.testing.assert_allclose(pyy - pzz, 0.0, atol=1e-16)


def test_interfacial_terms_vanish_without_a_gradient():
    dm, n = CO.interfacial_moments(np.zeros((3, 4)))
    assert not dm.any() and not n.any()


def test_recolouring_one_node_through_the_step():
    """A full oracle step on a closed box whose centre node has a known colour
    gradient (linear phase field), phase densities and velocity (every node at
    the equilibrium of one uniform u0): the seven D3Q7 values the centre sends
    arrive at its neighbours (and the rest value stays) as Appendix A's update
    w_q N_A [1 + 9/2 u.xi_q + beta N_B n.xi_q], and likewise for B with
    -beta N_A.  The recolouring pushes A along +n (towards the A-rich side)."""
    m = np.zeros((7, 5, 5), np.uint8)
    m[0] = 1
    m[-1] = 1
    beta = 0.9
    c = CO.ColourOracle(m, 0.9, alpha=0.004, beta=beta, phi_s=-1.0, inlet=None, outlet=None)
    z, y, x = np.meshgrid(np.arange(7), np.arange(5), np.arange(5), indexing="ij")
    g = np.array([0.05, -0.03, 0.02])
    phi = 0.1 + g[0] * (x - 2) + g[1] * (y - 2) + g[2] * (z - 3)
    c.init_phase(phi)
    u0 = np.array([0.004, -0.002, 0.003])
    pore = m == 0
    ones = np.ones(m.shape)
    c.f = O.equilibrium(ones, u0[0] * ones, u0[1] * ones, u0[2] * ones)
    c.f[:, ~pore] = 0.0
    NA, NB = (1.0 + 0.1) / 2.0, (1.0 - 0.1) / 2.0
    n = g / np.linalg.norm(g)
    c.step()
    xi7 = O.XI[:7]
    w7 = [1.0 / 3.0] + [1.0 / 9.0] * 6
    for q in range(7):
        dz, dy, dx = int(xi7[q, 2]), int(xi7[q, 1]), int(xi7[q, 0])
        at = (q, 3 + dz, 2 + dy, 2 + dx)
        xu, xn = float(xi7[q] @ u0), float(xi7[q] @ n)
        np.testing.assert_allclose(c.A[at], w7[q] * NA * (1 + 4.5 * xu + beta * NB * xn), rtol=1e-14)
        np.testing.assert_allclose(c.B[at], w7[q] * NB * (1 + 4.5 * xu - beta * NA * xn), rtol=1e-14)
    # A moves along +n: the value sent along the direction closest to n exceeds the opposite one
    qbest = int(np.argmax([xi7[q] @ n for q in range(1, 7)])) + 1
    opp = [0, 2, 1, 4, 3, 6, 5][qbest]
    sent = lambda arr, q: arr[(q, 3 + int(xi7[q, 2]), 2 + int(xi7[q, 1]), 2 + int(xi7[q, 0]))]
    assert sent(c.A, qbest) - sent(c.A, opp) > 9.0 * w7[qbest] * NA * (xi7[qbest] @ u0)
    assert sent(c.B, qbest) - sent(c.B, opp) < 9.0 * w7[qbest] * NB * (xi7[qbest] @ u0)
    # each phase leaves the centre whole: the seven values sum to N_A and N_B
    np.testing.assert_allclose(sum(sent(c.A, q) for q in range(7)), NA, rtol=1e-14)
    np.testing.assert_allclose(sum(sent(c.B, q) for q in range(7)), NB, rtol=1e-14)


def test_inlet_flux_exact_two_phase():
    m = duct_mask(7, 7, 10)
    c = CO.ColourOracle(m, 0.9, alpha=0.005, beta=0.95, phi_s=-1.0, Q=0.01, phi_in=1.0)
    z = np.arange(10)[:, None, None] * np.ones(m.shape)
    c.init_phase(np.where(z < 4, 1.0, -1.0))
    for _ in range(10):
        c.step()
        _, _, _, uz, _ = c.fields()
        A = int((m[0] == 0).sum())
        assert abs(math.fsum(uz[0][m[0] == 0].tolist()) - 0.01) <= 8 * A * np.finfo(float).eps


def test_box_faces_are_wetting_neutral_and_solids_wet():
    """A uniform phase field has no colour gradient at the box faces whatever
    phi_s is; next to a solid voxel the gradient points away from the solid
    when phi_s < phi (the solid looks like phase B)."""
    m = np.zeros((5, 6, 7), np.uint8)
    phi = np.full(m.shape, 0.3)
    for ps in (-1.0, 0.0, 1.0):
        np.testing.assert_allclose(CO.colour_gradient(phi, m, ps), 0.0, atol=1e-15)
    m[2, 3, 3] = 1
    C = CO.colour_gradient(phi, m, -1.0)
    # the +x neighbour of the solid: C_x > 0 and C_y = C_z = 0 by symmetry
    assert C[0, 2, 3, 4] > 0
    assert abs(C[1, 2, 3, 4]) < 1e-15 and abs(C[2, 2, 3, 4]) < 1e-15
    # stencil weight of one face neighbour: 3 w_1 (phi - phi_s) = (1/6) * 1.3
    np.testing.assert_allclose(C[0, 2, 3, 4], 3.0 / 18.0 * 1.3, rtol=1e-14)


def test_inlet_plane_holds_injected_composition():
    m = duct_mask(6, 6, 8)
    c = CO.ColourOracle(m, 0.9, alpha=0.005, beta=0.95, phi_s=-1.0, Q=0.01, phi_in=0.6)
    c.init_phase(np.tanh(uniform_field(m.shape, 3)))
    c.step(3)
    before_A, before_B = c.A.copy(), c.B.copy()
    c.hold_inlet_composition()
    _, NA, NB = c.phase_field()
    p0 = m[0] == 0
    # phase densities at the reference density rho0 = 1, whatever the inlet pressure
    assert abs(c.rho_in - 1.0) > 1e-4
    np.testing.assert_allclose(NA[0][p0], 0.8, rtol=1e-14)
    np.testing.assert_allclose(NB[0][p0], 0.2, rtol=1e-14)
    # only the value entering through the inlet plane changed
    changed = (c.A != before_A) | (c.B != before_B)
    assert not changed[:5].any() and not changed[6].any() and not changed[5, 1:].any()
