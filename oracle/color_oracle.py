"""Plain FP64 CPU oracle of the two-fluid colour model (Appendix A) with the
paper's flux inlet.

TEST INFRASTRUCTURE ONLY (like lbm_oracle): the correctness reference of the CUDA colour step.

Per step, on the pore nodes of a voxel mask:
  1. phase field phi = (N_A - N_B) / (N_A + N_B), N_A = sum A_q, N_B = sum B_q (D3Q7);
  2. colour gradient C = grad phi, n = C / |C|;
  3. momentum (D3Q19): pull streaming with halfway bounce-back, the inlet density
     of Eq. (potential) with the Appendix B closure, the outlet pressure closure,
     then MRT collision whose equilibrium moments carry the interfacial terms
     m1 += alpha |C|, m9 += alpha |C|/2 (2 nx^2 - ny^2 - nz^2), m11 += alpha |C|/2
     (ny^2 - nz^2), m13 += alpha |C|/2 nx ny, m14 += alpha |C|/2 ny nz,
     m15 += alpha |C|/2 nx nz (Appendix A);
  4. mass transport (Appendix A, D3Q7, w0 = 1/3, w1..6 = 1/9):
     A_q(x + xi_q) = w_q N_A [1 + 9/2 u.xi_q + beta N_B n.xi_q],
     B_q(x + xi_q) = w_q N_B [1 + 9/2 u.xi_q - beta N_A n.xi_q], u = j / rho0.

Readings where the paper is silent (also listed in the design notes):
  * the gradient is the isotropic D3Q19 stencil C = 3 sum_q w_q xi_q phi(x + xi_q);
    a solid voxel contributes phi_s (the wetting parameter: phi_s = +1 means the
    solid looks like phase A), a neighbour outside the box (through any face)
    contributes the node's own phi, so the box faces are wetting-neutral; n = 0
    where |C| = 0;
  * D3Q7 values pushed into a solid (or lateral outside) bounce back to the
    sender in the opposite direction; the inlet plane holds the injected
    composition: at the start of every step the D3Q7 value that entered an inlet
    node through the inlet (direction 5) is set so that the node carries
    N_A = rho0 (1 + phi_in)/2 and N_B = rho0 (1 - phi_in)/2 with rho0 = 1 (the
    phase densities are transported at the reference density of the
    incompressible model; the momentum density carries the pressure) (phi_in =
    +1: the non-wetting phase A is injected); at the outlet the entering value is
    w6 N [1 - 9/2 u_z] with the node's own N_A, N_B, u_z;
  * the collision uses the velocity and colour field of the same step; the
    mass transport uses u = j after the boundary closures.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbm_oracle as L

XI7 = L.XI[:7]
W7 = np.array([1.0 / 3.0] + [1.0 / 9.0] * 6)
OPP7 = np.array([0, 2, 1, 4, 3, 6, 5])


def colour_gradient(phi, mask, phi_s):
    """C = 3 sum_q w_q xi_q phi(x + xi_q) over the D3Q19 set (readings above)."""
    nz, ny, nx = mask.shape
    solid = mask.astype(bool)
    field = np.where(solid, phi_s, phi)
    padded = np.pad(field, 1, constant_values=np.nan)  # nan marks "outside the box"
    C = np.zeros((3,) + mask.shape)
    for q in range(1, L.NQ):
        cx, cy, cz = (int(v) for v in L.XI[q])
        nb = padded[1 + cz:1 + cz + nz, 1 + cy:1 + cy + ny, 1 + cx:1 + cx + nx]
        nb = np.where(np.isnan(nb), phi, nb)
        for a in range(3):
            if L.XI[q, a]:
                C[a] += 3.0 * L.W[q] * L.XI[q, a] * nb
    C[:, solid] = 0.0
    return C


def colour_gradient_loops(phi, mask, phi_s):
    """The same stencil voxel by voxel (brute force, tiny grids only)."""
    nz, ny, nx = mask.shape
    C = np.zeros((3,) + mask.shape)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if mask[z, y, x]:
                    continue
                for q in range(1, L.NQ):
                    sx, sy, sz = x + L.XI[q, 0], y + L.XI[q, 1], z + L.XI[q, 2]
                    if sz < 0 or sz >= nz or sx < 0 or sx >= nx or sy < 0 or sy >= ny:
                        v = phi[z, y, x]
                    elif mask[sz, sy, sx]:
                        v = phi_s
                    else:
                        v = phi[sz, sy, sx]
                    for a in range(3):
                        C[a, z, y, x] += 3.0 * L.W[q] * L.XI[q, a] * v
    return C


def interfacial_moments(C):
    """The alpha-free parts of the Appendix A interfacial terms: returns dm with
    dm[k] multiplying alpha for k in (1, 9, 11, 13, 14, 15)."""
    mag = np.sqrt((C ** 2).sum(axis=0))
    safe = np.where(mag > 0, mag, 1.0)
    n = np.where(mag > 0, C / safe, 0.0)
    nx_, ny_, nz_ = n
    dm = np.zeros((19,) + mag.shape)
    dm[1] = mag
    dm[9] = 0.5 * mag * (2 * nx_ ** 2 - ny_ ** 2 - nz_ ** 2)
    dm[11] = 0.5 * mag * (ny_ ** 2 - nz_ ** 2)
    dm[13] = 0.5 * mag * nx_ * ny_
    dm[14] = 0.5 * mag * ny_ * nz_
    dm[15] = 0.5 * mag * nx_ * nz_
    return dm, n


def collide_colour(F, tau, alpha, dm):
    """Appendix A MRT with m^eq = M f^eq(rho, j) + alpha dm; F, dm are (19, N)."""
    rho, jx, jy, jz = L.moments(F)
    m = L._M @ F
    meq = L._M @ L.equilibrium(rho, jx, jy, jz) + alpha * dm
    S = L.relaxation_rates(1.0 / tau)
    return F + L._MINV @ (S[:, None] * (meq - m))


class ColourOracle:
    """Two-fluid colour LBM on a voxel mask; inlet "flux" (Eq. potential) or None,
    outlet "pressure" or None (None: that z plane must be solid)."""

    def __init__(self, mask, tau, alpha, beta, phi_s=-1.0, Q=0.0, rho_out=1.0, phi_in=1.0,
                 inlet="flux", outlet="pressure"):
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.pore = self.mask == 0
        self.nz, self.ny, self.nx = self.mask.shape
        self.tau, self.alpha, self.beta, self.phi_s = float(tau), float(alpha), float(beta), float(phi_s)
        self.Q, self.rho_out, self.phi_in = float(Q), float(rho_out), float(phi_in)
        self.inlet, self.outlet = inlet, outlet
        self.rho_in = 1.0
        self.init_phase(np.ones(self.mask.shape))

    def init_phase(self, phi, rho=1.0):
        """Rest state with phase field phi (A-rich where phi = +1)."""
        rho = np.broadcast_to(np.asarray(rho, dtype=float), self.mask.shape)
        NA = rho * (1.0 + phi) / 2.0
        NB = rho * (1.0 - phi) / 2.0
        self.A = W7[:, None, None, None] * NA
        self.B = W7[:, None, None, None] * NB
        self.f = L.equilibrium(rho, 0.0 * rho, 0.0 * rho, 0.0 * rho)
        for a in (self.A, self.B, self.f):
            a[:, ~self.pore] = 0.0

    def phase_field(self):
        NA, NB = self.A.sum(axis=0), self.B.sum(axis=0)
        tot = np.where(self.pore, NA + NB, 1.0)
        return np.where(self.pore, (NA - NB) / tot, 0.0), NA, NB

    def step(self, n=1):
        for _ in range(n):
            self._step_once()

    def hold_inlet_composition(self):
        """Set the D3Q7 value that entered each inlet node through the inlet
        (direction 5) so the node carries N_A = rho0 (1 + phi_in)/2 and
        N_B = rho0 (1 - phi_in)/2, rho0 = 1 (reading above)."""
        frac = (1.0 + self.phi_in) / 2.0
        pore0 = self.pore[0]
        for arr, target in ((self.A, L.RHO0 * frac), (self.B, L.RHO0 * (1.0 - frac))):
            others = arr[:, 0].sum(axis=0) - arr[5, 0]
            arr[5, 0] = np.where(pore0, target - others, 0.0)

    def _step_once(self):
        if self.inlet is not None:
            self.hold_inlet_composition()
        phi, NA, NB = self.phase_field()
        C = colour_gradient(phi, self.mask, self.phi_s)
        dm, nvec = interfacial_moments(C)
        # momentum: stream, boundary conditions, collide
        ft = L.stream_pull(self.f, self.mask)
        nz = self.nz
        if self.inlet is not None:
            P = ft[:, 0]
            pore0 = self.pore[0]
            rho, _, _ = L.flux_density(L.inlet_known_sum(P), pore0, self.Q)
            self.rho_in = rho
            L.hh_closure_inlet(P, rho)
            P[:, ~pore0] = 0.0
        if self.outlet is not None:
            P = ft[:, nz - 1]
            L.hh_closure_outlet(P, self.rho_out)
            P[:, ~self.pore[nz - 1]] = 0.0
        F = ft[:, self.pore]
        if np.isnan(F).any():
            raise ValueError("open z face without a boundary condition")
        _, jx, jy, jz = L.moments(F)
        F = collide_colour(F, self.tau, self.alpha, dm[:, self.pore])
        f = np.zeros_like(self.f)
        f[:, self.pore] = F
        self.f = f
        u = np.zeros((3,) + self.mask.shape)
        u[0][self.pore], u[1][self.pore], u[2][self.pore] = jx / L.RHO0, jy / L.RHO0, jz / L.RHO0
        # mass transport: outgoing values at every node, then pull them in
        outA = np.zeros((7,) + self.mask.shape)
        outB = np.zeros((7,) + self.mask.shape)
        for q in range(7):
            xu = sum(XI7[q, a] * u[a] for a in range(3))
            xn = sum(XI7[q, a] * nvec[a] for a in range(3))
            outA[q] = W7[q] * NA * (1.0 + 4.5 * xu + self.beta * NB * xn)
            outB[q] = W7[q] * NB * (1.0 + 4.5 * xu - self.beta * NA * xn)
        self.A = self._transport(outA, NA, NB, u, True)
        self.B = self._transport(outB, NA, NB, u, False)

    def _transport(self, out, NA, NB, u, is_a):
        """new[q](x) = out[q](x - xi_q) for a pore sender, out[opp q](x) when the
        sender is solid or outside laterally, the inlet/outlet value when it is
        outside in z."""
        nz, ny, nx = self.mask.shape
        solid_pad = np.pad(self.mask.astype(bool), 1, constant_values=True)
        new = np.zeros_like(out)
        for q in range(7):
            cx, cy, cz = (int(v) for v in XI7[q])
            sl = (slice(1 - cz, 1 - cz + nz), slice(1 - cy, 1 - cy + ny), slice(1 - cx, 1 - cx + nx))
            src = np.pad(out[q], 1)[sl]
            new[q] = np.where(solid_pad[sl], out[OPP7[q]], src)
            if cz == 1:  # entering through the inlet plane: set at the next step's start
                if self.inlet is not None:
                    new[q, 0] = 0.0
            elif cz == -1:  # entering through the outlet plane
                if self.outlet is not None:
                    N = NA[nz - 1] if is_a else NB[nz - 1]
                    new[q, nz - 1] = W7[q] * N * (1.0 - 4.5 * u[2, nz - 1])
        new[:, ~self.pore] = 0.0
        return new

    def fields(self):
        rho, jx, jy, jz = L.moments(self.f)
        phi, NA, NB = self.phase_field()
        return rho, jx / L.RHO0, jy / L.RHO0, jz / L.RHO0, phi
