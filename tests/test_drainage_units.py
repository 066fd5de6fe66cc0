"""Host arithmetic of the Section 3.2 experiment matching (Ca, M, Q_sim, the
timestep from equal saturation rates, the stable parameter window)."""
import math

import pytest

from paper_1806_10589_gb300 import drainage as D


def test_paper_flux_pairs_share_one_capillary_number():
    """Section 3.2 runs the square tube at Q_sim = 0.02, 0.2, 2.0 and the 256^2
    Bentheimer sub-domain at 0.172, 1.72, 17.2 "such that the capillary numbers
    were the same", with the same gamma_sim = 6e-5 and nu = 1/6.  Equal Ca then
    needs Q_b / Q_t = eps_b A_b / (eps_t A_t): with the open 40 x 40 tube this
    is a sandstone porosity of 0.21, a typical Bentheimer value."""
    mu = D.lattice_viscosity(1.0)
    assert mu == pytest.approx(1.0 / 6.0)
    eps_b = 0.172 / 0.02 * 1600.0 / 65536.0
    assert 0.20 < eps_b < 0.22
    for qt, qb in ((0.02, 0.172), (0.2, 1.72), (2.0, 17.2)):
        ca_t = D.capillary_number(mu, qt, 6e-5, 1.0, 1600.0)
        ca_b = D.capillary_number(mu, qb, 6e-5, eps_b, 65536.0)
        assert ca_b == pytest.approx(ca_t, rel=1e-12)
        assert D.simulated_flux(ca_t, eps_b, 65536.0, 6e-5, mu) == pytest.approx(qb, rel=1e-12)


def test_flux_capillary_number_round_trip():
    for Ca in (1e-6, 1e-5, 3e-4):
        Q = D.simulated_flux(Ca, 0.35, 256 * 256, 0.0102, 1.0 / 6.0)
        assert D.capillary_number(1.0 / 6.0, Q, 0.0102, 0.35, 256 * 256) == pytest.approx(Ca, rel=1e-14)


def test_timestep_equalises_saturation_rates():
    """One lattice step changes s_w by as much as the experiment does in dt."""
    dx = 4.95e-6                      # image resolution of the Section 3.2 sandstone
    L = (256 * dx, 256 * dx, 256 * dx)
    V = L[0] * L[1] * L[2]
    Q = 0.1e-6 / 60.0                 # 0.1 mL/min in m^3/s
    Q_sim, eps = 1.72, 0.21
    dt = D.timestep_seconds(Q_sim, dx, Q)
    per_step_lattice = D.saturation_rate(Q_sim, eps, 256 ** 3)
    per_dt_physical = D.saturation_rate(Q, eps, V) * dt
    assert per_dt_physical == pytest.approx(per_step_lattice, rel=1e-12)
    # by hand: 1.72 * (4.95e-6)^3 / (1.6667e-9) = 1.2516e-7 s
    assert dt == pytest.approx(1.72 * 4.95e-6 ** 3 / (0.1e-6 / 60.0), rel=1e-12)
    assert 1.25e-7 < dt < 1.26e-7


def test_parameter_window():
    assert D.parameter_warnings(6e-5, 1.0, 1.0) == []
    assert any("gamma" in w for w in D.parameter_warnings(0.1, 1.0, 1.0))
    assert any("nu_w" in w for w in D.parameter_warnings(1e-3, 0.6, 1.0))     # nu = 1/30 < 1/15
    assert D.parameter_warnings(1e-3, 0.7, 1.5) == []                          # nu = 1/15 and 1/3 are inside
    assert any("rho_n" in w for w in D.parameter_warnings(1e-3, 1.0, 1.0, 1.0, 0.005))
    assert any("|u|" in w for w in D.parameter_warnings(1e-3, 1.0, 1.0, u_max=0.2))


def test_match_keeps_ca_and_mobility():
    exp = D.Experiment(Q_m3_per_s=0.05e-6 / 60.0, length_m=(1.267e-3, 1.267e-3, 1.267e-3), porosity=0.22,
                       mu_w=1.0e-3, mu_n=1.5e-3, gamma=0.03, dx_m=4.95e-6)
    r = D.match(exp, gamma_sim=6e-5, tau_w=1.0)
    assert r["A_sim"] == 256 * 256
    mu_w_sim = D.lattice_viscosity(1.0)
    mu_n_sim = D.lattice_viscosity(r["tau_n"])
    assert mu_w_sim / mu_n_sim == pytest.approx(exp.mu_w / exp.mu_n, rel=1e-12)
    assert D.capillary_number(mu_w_sim, r["Q_sim"], 6e-5, 0.22, 256 * 256) == pytest.approx(r["Ca"], rel=1e-12)
    assert math.isclose(r["Ca"], 1e-3 * exp.Q_m3_per_s / (0.03 * 0.22 * 1.267e-3 ** 2), rel_tol=1e-12)
    assert r["warnings"] == []
