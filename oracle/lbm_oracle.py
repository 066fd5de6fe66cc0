"""Plain FP64 CPU oracle of the D3Q19 lattice Boltzmann step with the adaptive
volumetric-flux boundary condition (McClure, Li, Sheppard, Miller, arXiv:1806.10589).

TEST INFRASTRUCTURE ONLY.  This module is the correctness reference for the CUDA
path.  Only the test suite, the smoke check and the benchmark's CPU-baseline /
reference leg may import it; the library itself never does.  It shares no code,
table or helper with the CUDA sources.

Deliberate plainness: dense arrays f[q][z][y][x] over the whole voxel box (not
the pore list the GPU uses), one numpy pass per operation, the collision done in
moment space exactly as Appendix A states it (M, S, M^-1), sums with math.fsum.

Readings where the paper is silent or garbled (each is also listed in the
design notes):
  * velocity order q = 7..18 is fixed by the Appendix B momentum identities;
  * weights 1/3, 1/18, 1/36 and c_s^2 = 1/3 follow from the 1/3 and 1/6
    coefficients of Appendix B;
  * the equilibrium of Appendix B is used with -3/2 u.u (the printed +3/2 would
    break sum_q f_q^eq = rho); rho0 = 1;
  * the equilibrium moments are m^eq = M f^eq(rho, j) (Appendix A prints only an
    abbreviated, rescaled subset);
  * Appendix B's transverse closure rows for f15 and f18 use N_y (the printed
    N_x there is a typo; the simplified rows are taken as authoritative);
  * the outlet closure is Appendix B's relations solved for the xi_z = -1
    members of each pair; tangential velocity at both pressure planes is zero;
  * solid voxels reflect by halfway bounce-back; lateral out-of-box sources are
    solid; the inlet integral runs over pore nodes only and A is their count.
"""
from __future__ import annotations

import math

import numpy as np

# Eq. (d3q19): D3Q19 velocities.  The order inside each +-pair group (7..18)
# is the one for which the Appendix B momentum identities hold as printed.
XI = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
], dtype=np.int64)
NQ = 19
# opposite direction: xi_opp = -xi
OPP = np.array([int(np.where((XI == -XI[q]).all(axis=1))[0][0]) for q in range(NQ)])
# weights: 6 w_q = 1/3 on the axes and 1/6 on the diagonals (Appendix B coefficients)
W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
CS2 = 1.0 / 3.0           # Eq. (pressure): p = c_s^2 rho
RHO0 = 1.0                # reference density of Eq. (m357)

# Eq. (inlet): the known distributions at a z-inlet node
INLET_UNKNOWN = [q for q in range(NQ) if XI[q, 2] == 1]      # 5, 11, 14, 15, 18
TANGENT = [q for q in range(NQ) if XI[q, 2] == 0]            # 0..4, 7..10
INLET_KNOWN_IN = [q for q in range(NQ) if XI[q, 2] == -1]    # 6, 12, 13, 16, 17


def equilibrium(rho, jx, jy, jz):
    """Appendix B equilibrium, incompressible form with j = rho0 u:
    f_q^eq = w_q [rho + rho0 (3 xi.u + 9/2 (xi.u)^2 - 3/2 u.u)]."""
    ux, uy, uz = jx / RHO0, jy / RHO0, jz / RHO0
    uu = ux * ux + uy * uy + uz * uz
    out = np.empty((NQ,) + np.shape(rho))
    for q in range(NQ):
        xu = XI[q, 0] * ux + XI[q, 1] * uy + XI[q, 2] * uz
        out[q] = W[q] * (rho + RHO0 * (3.0 * xu + 4.5 * xu * xu - 1.5 * uu))
    return out


def moment_matrix():
    """Appendix A: the 19 d'Humieres et al. (2002) D3Q19 moments
    (rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pzx,
    mx, my, mz) as polynomials of the velocity components.  Row k gives m_k."""
    M = np.zeros((NQ, NQ))
    for q in range(NQ):
        cx, cy, cz = (float(v) for v in XI[q])
        c2 = cx * cx + cy * cy + cz * cz
        M[0, q] = 1.0
        M[1, q] = 19.0 * c2 - 30.0
        M[2, q] = (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0
        M[3, q] = cx
        M[4, q] = (5.0 * c2 - 9.0) * cx
        M[5, q] = cy
        M[6, q] = (5.0 * c2 - 9.0) * cy
        M[7, q] = cz
        M[8, q] = (5.0 * c2 - 9.0) * cz
        M[9, q] = 3.0 * cx * cx - c2
        M[10, q] = (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2)
        M[11, q] = cy * cy - cz * cz
        M[12, q] = (3.0 * c2 - 5.0) * (cy * cy - cz * cz)
        M[13, q] = cx * cy
        M[14, q] = cy * cz
        M[15, q] = cx * cz
        M[16, q] = (cy * cy - cz * cz) * cx
        M[17, q] = (cz * cz - cx * cx) * cy
        M[18, q] = (cx * cx - cy * cy) * cz
    return M


def relaxation_rates(s_nu, s_q=None):
    """Appendix A: S = diag(0, s_e, s_eps, 0, s_q, 0, s_q, 0, s_q, s_nu, s_pi,
    s_nu, s_pi, s_nu, s_nu, s_nu, s_m, s_m, s_m) with s_e = s_eps = s_pi = s_nu
    and s_q = s_m = 8 (2 - s_nu) / (8 - s_nu) unless s_q is given."""
    if s_q is None:
        s_q = 8.0 * (2.0 - s_nu) / (8.0 - s_nu)
    return np.array([0.0, s_nu, s_nu, 0.0, s_q, 0.0, s_q, 0.0, s_q,
                     s_nu, s_nu, s_nu, s_nu, s_nu, s_nu, s_nu, s_q, s_q, s_q])


_M = moment_matrix()
_MINV = np.linalg.inv(_M)


def moments(F):
    """rho = sum_q f_q (Eq. m0) and j = sum_q f_q xi_q (Eq. m357); F is (19, ...)."""
    rho = F.sum(axis=0)
    j = [np.tensordot(XI[:, a].astype(float), F, axes=(0, 0)) for a in range(3)]
    return rho, j[0], j[1], j[2]


def collide_mrt(F, tau, s_q=None):
    """Appendix A: f' = f + M^-1 S (m^eq - m), m = M f, m^eq = M f^eq(rho, j),
    tau = 1 / s_nu.  F is (19, N)."""
    rho, jx, jy, jz = moments(F)
    m = _M @ F
    meq = _M @ equilibrium(rho, jx, jy, jz)
    S = relaxation_rates(1.0 / tau, s_q)
    return F + _MINV @ (S[:, None] * (meq - m))


def collide_bgk(F, tau):
    """Single-relaxation-time collision f' = f - (f - f^eq) / tau."""
    rho, jx, jy, jz = moments(F)
    return F - (F - equilibrium(rho, jx, jy, jz)) / tau


def stream_pull(f, mask):
    """Eq. (LBE), pull form: ft_q(x) = f_q(x - xi_q).

    A solid source (or one outside the box in x or y) reflects by halfway
    bounce-back: ft_q(x) = f_opp(q)(x).  A source outside the box in z is
    unknown and comes back as NaN; only the xi_z=+1 values at z=0 and the
    xi_z=-1 values at z=nz-1 can be unknown.  Solid cells return 0.
    """
    nz, ny, nx = mask.shape
    solid_pad = np.pad(mask.astype(bool), 1, constant_values=True)
    ft = np.empty_like(f)
    for q in range(NQ):
        cx, cy, cz = (int(v) for v in XI[q])
        sl = (slice(1 - cz, 1 - cz + nz), slice(1 - cy, 1 - cy + ny), slice(1 - cx, 1 - cx + nx))
        src = np.pad(f[q], 1)[sl]
        ft[q] = np.where(solid_pad[sl], f[OPP[q]], src)
        if cz == 1:
            ft[q, 0] = np.nan
        elif cz == -1:
            ft[q, nz - 1] = np.nan
    ft[:, mask.astype(bool)] = 0.0
    return ft


def stream_pull_loops(f, mask):
    """The same pull step written voxel by voxel (brute force, tiny grids only)."""
    nz, ny, nx = mask.shape
    ft = np.zeros_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if mask[z, y, x]:
                    continue
                for q in range(NQ):
                    sx, sy, sz = x - XI[q, 0], y - XI[q, 1], z - XI[q, 2]
                    if sz < 0 or sz >= nz:
                        ft[q, z, y, x] = np.nan
                    elif sx < 0 or sx >= nx or sy < 0 or sy >= ny or mask[sz, sy, sx]:
                        ft[q, z, y, x] = f[OPP[q], z, y, x]
                    else:
                        ft[q, z, y, x] = f[q, sz, sy, sx]
    return ft


def inlet_known_sum(P):
    """The bracket of Eq. (inlet): f0+f1+f2+f3+f4+f7+f8+f9+f10 + 2(f6+f12+f13+f16+f17)
    for a plane P of shape (19, ny, nx)."""
    return (P[0] + P[1] + P[2] + P[3] + P[4] + P[7] + P[8] + P[9] + P[10]
            + 2.0 * (P[6] + P[12] + P[13] + P[16] + P[17]))


def outlet_known_sum(P):
    """Mirror of Eq. (inlet) for a z-outlet node: sum over xi_z=0 plus twice the
    sum over xi_z=+1 (f5, f11, f14, f15, f18)."""
    return (P[0] + P[1] + P[2] + P[3] + P[4] + P[7] + P[8] + P[9] + P[10]
            + 2.0 * (P[5] + P[11] + P[14] + P[15] + P[18]))


def flux_density(K_plane, pore_plane, Q):
    """Eq. (potential): rho = rho0 Q / A + (1/A) sum_{inlet pores} K, A = number of
    inlet pore nodes.  Returns (rho, A, S) with S the sum of K (math.fsum)."""
    vals = K_plane[pore_plane]
    A = int(vals.size)
    S = math.fsum(vals.tolist())
    return (RHO0 * Q + S) / A, A, S


def hh_closure_inlet(P, rho):
    """Appendix B at a z-inlet plane P (19, ny, nx), in place: u_z from Eq. (inlet),
    u_x = u_y = 0, then f5, f11, f14, f15, f18 from the Hecht-Harting relations.
    Returns u_z."""
    ux = uy = 0.0
    uz = rho / RHO0 - inlet_known_sum(P) / RHO0
    nx_ = 0.5 * (P[1] + P[7] + P[9] - (P[2] + P[10] + P[8])) - RHO0 * ux / 3.0
    ny_ = 0.5 * (P[3] + P[7] + P[10] - (P[4] + P[9] + P[8])) - RHO0 * uy / 3.0
    P[5] = P[6] + RHO0 * uz / 3.0
    P[11] = P[12] + RHO0 * (ux + uz) / 6.0 - nx_
    P[14] = P[13] + RHO0 * (-ux + uz) / 6.0 + nx_
    P[15] = P[16] + RHO0 * (uy + uz) / 6.0 - ny_
    P[18] = P[17] + RHO0 * (-uy + uz) / 6.0 + ny_
    return uz


def hh_closure_outlet(P, rho):
    """Appendix B relations solved for the xi_z=-1 unknowns at a z-outlet plane,
    in place: rho0 u_z = sum_{xi_z=0} f + 2 sum_{xi_z=+1} f - rho, u_x = u_y = 0,
    then f6, f12, f13, f16, f17.  Returns u_z."""
    ux = uy = 0.0
    uz = (outlet_known_sum(P) - rho) / RHO0
    nx_ = 0.5 * (P[1] + P[7] + P[9] - (P[2] + P[10] + P[8])) - RHO0 * ux / 3.0
    ny_ = 0.5 * (P[3] + P[7] + P[10] - (P[4] + P[9] + P[8])) - RHO0 * uy / 3.0
    P[6] = P[5] - RHO0 * uz / 3.0
    P[12] = P[11] - RHO0 * (ux + uz) / 6.0 + nx_
    P[13] = P[14] - RHO0 * (-ux + uz) / 6.0 - nx_
    P[16] = P[15] - RHO0 * (uy + uz) / 6.0 + ny_
    P[17] = P[18] - RHO0 * (-uy + uz) / 6.0 - ny_
    return uz


def steady_residual(u_now, u_prev, pore):
    """Section 3.1, Eq. (stopping_criterion): sum_x |u(x,t) - u(x,t-lag)| / sum_x |u(x,t)|
    over pore nodes, |.| the Euclidean norm of the velocity vector; u arrays are
    (3, nz, ny, nx)."""
    du = np.sqrt(((np.asarray(u_now) - np.asarray(u_prev)) ** 2).sum(axis=0))[pore]
    un = np.sqrt((np.asarray(u_now) ** 2).sum(axis=0))[pore]
    return math.fsum(du.tolist()) / math.fsum(un.tolist())


class D3Q19Oracle:
    """Single-fluid D3Q19 LBM on a voxel mask, stepped as Section 2 orders it:
    stream, then (1) the inlet density from Eq. (potential), (2) the pressure
    closure at the inlet with that density and at the outlet with rho_out, then
    collide at every pore node.

    inlet: "flux" (the paper's condition), "pressure" (fixed rho_in) or None
    (no open inlet: the z=0 plane must then be solid); outlet: "pressure" or None.
    model: "mrt" (Appendix A) or "bgk".
    """

    def __init__(self, mask, tau, model="mrt", Q=0.0, rho_in=1.0, rho_out=1.0,
                 inlet="flux", outlet="pressure"):
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.nz, self.ny, self.nx = self.mask.shape
        self.tau = float(tau)
        self.model = model
        self.Q = float(Q)
        self.rho_in = float(rho_in)
        self.rho_out = float(rho_out)
        self.inlet = inlet
        self.outlet = outlet
        self.pore = self.mask == 0
        self.q_in = None
        self.q_out = None
        self.steps = 0
        self.init_equilibrium()

    def init_equilibrium(self, rho=1.0, ux=0.0, uy=0.0, uz=0.0):
        shape = self.mask.shape
        r = np.broadcast_to(np.asarray(rho, dtype=float), shape)
        f = equilibrium(r, np.broadcast_to(ux, shape) * RHO0, np.broadcast_to(uy, shape) * RHO0,
                        np.broadcast_to(uz, shape) * RHO0)
        f[:, ~self.pore] = 0.0
        self.f = np.ascontiguousarray(f)

    def set_distributions(self, f):
        f = np.array(f, dtype=np.float64, copy=True)
        f[:, ~self.pore] = 0.0
        self.f = f

    def step(self, n=1):
        for _ in range(n):
            self._step_once()

    def _step_once(self):
        ft = stream_pull(self.f, self.mask)
        nz = self.nz
        if self.inlet is not None:
            P = ft[:, 0]
            pore0 = self.pore[0]
            if self.inlet == "flux":
                rho, _, _ = flux_density(inlet_known_sum(P), pore0, self.Q)
                self.rho_in = rho
            uz = hh_closure_inlet(P, self.rho_in)
            P[:, ~pore0] = 0.0
            self.q_in = math.fsum(uz[pore0].tolist())
        if self.outlet is not None:
            P = ft[:, nz - 1]
            poreL = self.pore[nz - 1]
            uz = hh_closure_outlet(P, self.rho_out)
            P[:, ~poreL] = 0.0
            self.q_out = math.fsum(uz[poreL].tolist())
        F = ft[:, self.pore]
        if np.isnan(F).any():
            raise ValueError("oracle: unknown distributions left after the boundary step "
                             "(open z face without a boundary condition)")
        if self.model == "mrt":
            F = collide_mrt(F, self.tau)
        elif self.model == "bgk":
            F = collide_bgk(F, self.tau)
        else:
            raise ValueError("unknown model %r" % self.model)
        f = np.zeros_like(self.f)
        f[:, self.pore] = F
        self.f = f
        self.steps += 1

    def fields(self):
        """rho and u = j / rho0 of the stored (post-collision) state; 0 at solids."""
        rho, jx, jy, jz = moments(self.f)
        return rho, jx / RHO0, jy / RHO0, jz / RHO0

    def face_flux(self, z):
        """sum of u_z over the pore nodes of plane z (math.fsum)."""
        _, _, _, uz = self.fields()
        return math.fsum(uz[z][self.pore[z]].tolist())
