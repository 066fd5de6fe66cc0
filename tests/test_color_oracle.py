"""Pins of the colour-model oracle (Appendix A): it reduces exactly to the
single-fluid oracle when only one phase is present, conserves the mass of each
phase in a closed box, its gradient stencil is exact on linear fields and equals
a voxel loop, recolouring leaves each phase's density unchanged, and the inlet
flux stays exact."""
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


def test_recolouring_conserves_phase_density_per_node():
    """sum_q w_q [1 + 9/2 u.xi + beta N n.xi] = 1, so each node sends out exactly
    its N_A and N_B."""
    rng = np.random.default_rng(9)
    u = 0.01 * rng.standard_normal(3)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    NA, NB, beta = 0.7, 0.3, 0.95
    outA = [CO.W7[q] * NA * (1 + 4.5 * CO.XI7[q] @ u + beta * NB * CO.XI7[q] @ n) for q in range(7)]
    assert abs(sum(outA) - NA) < 1e-15
    # and the first moment carries N_A u plus the recolouring flux
    mom = sum(outA[q] * CO.XI7[q] for q in range(7))
    np.testing.assert_allclose(mom, NA * u + beta * NA * NB * (2.0 / 9.0) * n, atol=1e-15)


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
