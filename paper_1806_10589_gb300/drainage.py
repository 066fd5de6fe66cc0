"""Matching a two-fluid displacement experiment to lattice units (Section 3.2,
"Immiscible displacement at constant capillary number").  Host-side arithmetic
only; the simulation itself runs through ColorLattice.

Relations of the paper, in lattice units unless stated:
  * saturation rate of an incompressible displacement (Eq. time_rate_of_Sw):
    d s_w / dt = Q / (eps V);
  * capillary number Ca = mu_w Q / (gamma eps A) and mobility M = mu_w / mu_n;
  * the simulated flux that reproduces Ca: Q_sim = eps A_sim gamma_sim / mu_w_sim * Ca;
  * the timestep follows from equal saturation rates: one lattice step changes s_w by
    Q_sim / (eps V_sim), which the experiment does in (Q_sim / V_sim) / (Q / V) seconds,
    so dt = Q_sim dx^3 / Q (V_sim = V / dx^3);
  * the stable parameter window of the colour model the paper uses:
    1e-5 <= gamma_sim <= 1e-2, 1/15 <= nu <= 1/3, 0.01 <= rho <= 1, |u| below ~0.1.
Lattice viscosity nu = (tau - 1/2)/3 and mu = rho nu (Appendix A).
"""
from __future__ import annotations

from dataclasses import dataclass


def lattice_viscosity(tau: float) -> float:
    return (tau - 0.5) / 3.0


def saturation_rate(Q: float, eps: float, V: float) -> float:
    """d s_w / dt = Q / (eps V) (Eq. time_rate_of_Sw)."""
    return Q / (eps * V)


def capillary_number(mu_w: float, Q: float, gamma: float, eps: float, A: float) -> float:
    """Ca = mu_w Q / (gamma eps A), A the inlet area."""
    return mu_w * Q / (gamma * eps * A)


def mobility(mu_w: float, mu_n: float) -> float:
    return mu_w / mu_n


def simulated_flux(Ca: float, eps: float, A_sim: float, gamma_sim: float, mu_w_sim: float) -> float:
    """Q_sim = eps A_sim (gamma_sim / mu_w_sim) Ca."""
    return eps * A_sim * gamma_sim / mu_w_sim * Ca


def timestep_seconds(Q_sim: float, dx_m: float, Q_m3_per_s: float) -> float:
    """Physical duration of one lattice step from equal saturation rates:
    dt = Q_sim dx^3 / Q (dx in metres, Q in m^3/s)."""
    return Q_sim * dx_m ** 3 / Q_m3_per_s


def parameter_warnings(gamma_sim: float, tau_w: float, tau_n: float, rho_w: float = 1.0, rho_n: float = 1.0,
                       u_max: float | None = None) -> list[str]:
    """Which of the paper's stability limits a parameter set leaves (empty: none)."""
    out = []
    if not 1e-5 <= gamma_sim <= 1e-2:
        out.append(f"gamma_sim {gamma_sim:g} outside [1e-5, 1e-2]")
    for name, tau in (("w", tau_w), ("n", tau_n)):
        nu = lattice_viscosity(tau)
        if not 1.0 / 15.0 - 1e-15 <= nu <= 1.0 / 3.0 + 1e-15:
            out.append(f"nu_{name} {nu:g} outside [1/15, 1/3]")
    for name, rho in (("w", rho_w), ("n", rho_n)):
        if not 0.01 <= rho <= 1.0:
            out.append(f"rho_{name} {rho:g} outside [0.01, 1]")
    if u_max is not None and u_max >= 0.1:
        out.append(f"|u| {u_max:g} reaches 0.1")
    return out


@dataclass
class Experiment:
    """The quantities an experiment provides (SI units)."""
    Q_m3_per_s: float      # volumetric flow rate
    length_m: tuple        # (Lx, Ly, Lz) of the sample
    porosity: float
    mu_w: float            # Pa s
    mu_n: float            # Pa s
    gamma: float           # N/m
    dx_m: float            # image resolution (voxel width)

    @property
    def capillary_number(self) -> float:
        Lx, Ly, _ = self.length_m
        return capillary_number(self.mu_w, self.Q_m3_per_s, self.gamma, self.porosity, Lx * Ly)

    @property
    def mobility(self) -> float:
        return mobility(self.mu_w, self.mu_n)


def match(exp: Experiment, gamma_sim: float, tau_w: float, rho_w: float = 1.0) -> dict:
    """Lattice parameters reproducing the experiment's Ca and M: Q_sim, the
    non-wetting relaxation time, the timestep in seconds and the lattice inlet area."""
    Lx, Ly, Lz = exp.length_m
    A_sim = round(Lx / exp.dx_m) * round(Ly / exp.dx_m)
    mu_w_sim = rho_w * lattice_viscosity(tau_w)
    Q_sim = simulated_flux(exp.capillary_number, exp.porosity, A_sim, gamma_sim, mu_w_sim)
    mu_n_sim = mu_w_sim / exp.mobility
    tau_n = 3.0 * mu_n_sim / rho_w + 0.5
    return {"Ca": exp.capillary_number, "M": exp.mobility, "A_sim": A_sim, "Q_sim": Q_sim, "tau_n": tau_n,
            "dt_s": timestep_seconds(Q_sim, exp.dx_m, exp.Q_m3_per_s),
            "warnings": parameter_warnings(gamma_sim, tau_w, tau_n, rho_w, rho_w)}
