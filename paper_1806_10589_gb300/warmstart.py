"""Learned warm start: training data from this library's own steady states, a
Kozeny-Carman pressure-drop estimate calibrated on them, and the warm-started
initial field f = f^eq(rho, u) (host orchestration only; the LBM, the network
forward/backward/Adam and the equilibrium initialisation run in the CUDA
library).

The network predicts, per voxel, u / u_D (u_D = Q / (nx ny)) and the local
pressure gradient G = -(p(z+1) - p(z)) / (nu u_D), p = c_s^2 rho.  Initial
fields of a new geometry with flux Q:
  u = u_D * net_u(mask)                                       (network velocity)
  rho(z) = rho_out + (nu u_D / c_s^2) sum_{z' >= z} Gbar(z')   (network pressure)
with Gbar(z) the mean of the predicted G over the pore voxels of plane z whose
+z neighbour is a pore (the voxels where G is defined); or, without the
network, the analytic ramp
  rho(z) = rho_out + dp_est * (1 - z / (nz - 1)) / c_s^2,
  dp_est = nu u_D (nz - 1) / k_est,  k_est = c_KC phi^3 / (S^2 (1 - phi)^2)
(Darcy with Kozeny-Carman), phi the porosity, S the pore-solid face count per
voxel, c_KC fitted on the training set by least squares in log space.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import convergence as cv

CS2 = 1.0 / 3.0


def he_init(net, seed):
    """Seeded He-normal weights (std sqrt(2 / (27 cin))) and zero biases, in the
    library's parameter layout."""
    rng = np.random.default_rng(seed)
    p = np.zeros(net.n_params, np.float32)
    k = 0
    for co, ci in net.layer_shapes():
        nw = co * ci * 27
        p[k:k + nw] = rng.standard_normal(nw) * math.sqrt(2.0 / (27 * ci))
        k += nw + co
    return p


def surface_density(mask):
    """Pore-solid voxel faces per voxel of a [z][y][x] mask (1 = solid); the
    faces on the lateral box boundary count as walls, z ends do not."""
    m = mask.astype(bool)
    faces = 0
    for ax in (0, 1, 2):
        a = np.moveaxis(m, ax, 0)
        faces += int((a[1:] != a[:-1]).sum())
    faces += int((~m[:, 0, :]).sum() + (~m[:, -1, :]).sum() + (~m[:, :, 0]).sum() + (~m[:, :, -1]).sum())
    return faces / m.size


def kc_features(mask):
    phi = float((mask == 0).mean())
    S = surface_density(mask)
    return phi, S, phi ** 3 / (S * S * (1.0 - phi) ** 2)


def gradient_target(rho, mask, Q, tau):
    """G = -c_s^2 (rho(z+1) - rho(z)) / (nu u_D) on pore voxels whose +z
    neighbour is a pore; NaN (no target) elsewhere and on the last plane."""
    nz, ny, nx = mask.shape
    nu = CS2 * (tau - 0.5)
    uD = Q / (nx * ny)
    G = np.full(mask.shape, np.nan)
    ok = (mask[:-1] == 0) & (mask[1:] == 0)
    G[:-1][ok] = (-CS2 * (rho[1:] - rho[:-1]) / (nu * uD))[ok]
    return G


def steady_targets(batch_cls, masks, tau, u_mean, steps, precision="fp32", stream=None):
    """Run every geometry to (near) steady state in one batched ensemble and
    return (targets as float32 [S][4][z][y][x]: u / u_D and G, permeabilities)."""
    S = len(masks)
    Qs = [u_mean * int((m[0] == 0).sum()) for m in masks]
    targets = np.zeros((S, 4) + masks[0].shape, np.float32)
    ks = np.zeros(S)
    with batch_cls(masks, tau, "mrt", precision, stream=stream) as b:
        for k, q in enumerate(Qs):
            b.set_flux_bc(k, q)
        b.step(steps)
        for k, m in enumerate(masks):
            rho, ux, uy, uz = b.fields(k)
            nz, ny, nx = m.shape
            uD = Qs[k] / (nx * ny)
            targets[k, :3] = (np.stack([ux, uy, uz]) / uD).astype(np.float32)
            targets[k, 3] = gradient_target(rho, m, Qs[k], tau).astype(np.float32)
            _, rho_in = b.get_flux(k, 4)
            ks[k] = cv.permeability(Qs[k], m.shape, tau, rho_in, 1.0)
    return targets, ks


def fit_kc(masks, ks):
    """c_KC of k = c * phi^3 / (S^2 (1 - phi)^2), least squares in log k."""
    x = np.array([kc_features(m)[2] for m in masks])
    return float(np.exp(np.mean(np.log(ks) - np.log(x))))


def pressure_profile(G, mask, Q, tau, rho_out=1.0):
    """rho(z) from a predicted gradient field: the plane means Gbar(z) over the
    voxels where G is defined, summed from the outlet."""
    nz, ny, nx = mask.shape
    nu = CS2 * (tau - 0.5)
    uD = Q / (nx * ny)
    ok = (mask[:-1] == 0) & (mask[1:] == 0)
    cnt = ok.reshape(nz - 1, -1).sum(axis=1)
    gsum = np.where(ok, G[:-1], 0.0).reshape(nz - 1, -1).sum(axis=1)
    gbar = np.where(cnt > 0, gsum / np.maximum(cnt, 1), 0.0)
    drop = np.concatenate([np.cumsum(gbar[::-1])[::-1], [0.0]])  # sum over z' >= z of Gbar(z')
    return rho_out + (nu * uD / CS2) * drop


def kc_profile(mask, Q, tau, c_kc, rho_out=1.0):
    """The linear Kozeny-Carman ramp rho(z)."""
    nz, ny, nx = mask.shape
    uD = Q / (nx * ny)
    k_est = c_kc * kc_features(mask)[2]
    nu = CS2 * (tau - 0.5)
    dp = nu * uD * (nz - 1) / k_est
    return rho_out + (dp / CS2) * (1.0 - np.arange(nz, dtype=np.float64) / (nz - 1))


def initial_fields(net, mask, Q, tau, c_kc, velocity="net", pressure="net"):
    """(rho, ux, uy, uz) float64 arrays for Lattice.set_fields.  velocity:
    "net" (u = u_D * net_u) or "zero"; pressure: "net" (the network's profile),
    "kc" (the Kozeny-Carman ramp) or "uniform" (rho = 1)."""
    nz, ny, nx = mask.shape
    uD = Q / (nx * ny)
    y = net.predict(mask).astype(np.float64) if (velocity == "net" or pressure == "net") else None
    u = y[:3] * uD if velocity == "net" else np.zeros((3,) + mask.shape)
    if pressure == "net":
        prof = pressure_profile(y[3], mask, Q, tau)
    elif pressure == "kc":
        prof = kc_profile(mask, Q, tau, c_kc)
    else:
        prof = np.ones(nz)
    rho = prof[:, None, None] + np.zeros(mask.shape)
    return rho, u[0], u[1], u[2]


def net_permeability(net, mask, Q, tau):
    """Darcy permeability implied by the network's pressure profile (the same
    definition the 0.1 % rule uses)."""
    rho = pressure_profile(net.predict(mask)[3].astype(np.float64), mask, Q, tau)
    return cv.permeability(Q, mask.shape, tau, rho[0], rho[-1])


# start name -> (velocity, pressure) of initial_fields; "cold" sets nothing
STARTS = {"cold": None, "kc_ramp": ("zero", "kc"), "net_velocity": ("net", "uniform"),
          "net_pressure": ("zero", "net"), "net": ("net", "net")}


def run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, start, precision="fp32", stream=None, sync=None,
              max_steps=400000, variant=0):
    """Steps and wall seconds to the 0.1 % rule (k within 1e-3 of k_ref for 10
    checks) from one of STARTS; the time of a warm start includes the network
    inference and the field upload."""
    with lattice_cls(mask, tau, "mrt", precision, stream=stream) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        t_init = 0.0
        if STARTS[start] is not None:
            if sync:
                sync()
            t0 = time.perf_counter()
            rho, ux, uy, uz = initial_fields(net, mask, Q, tau, c_kc, *STARTS[start])
            lat.set_fields(rho, ux, uy, uz)
            if sync:
                sync()
            t_init = time.perf_counter() - t0
        r = cv.run_to_reference(lat, Q, tau, k_ref, max_steps=max_steps, sync=sync)
    return {"steps": r["steps"], "seconds": None if r["seconds"] is None else r["seconds"] + t_init,
            "init_seconds": t_init, "reached": r["reached"], "k": r["k"], "q_out": r["q_out"],
            "steps_run": r["steps_run"]}


def warm_vs_cold(lattice_cls, net, mask, Q, tau, c_kc, k_ref, precision="fp32", stream=None, sync=None,
                 max_steps=400000, variant=0):
    """The cold start and the full learned warm start (network velocity and pressure)."""
    args = (precision, stream, sync, max_steps, variant)
    return {"cold": run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, "cold", *args),
            "warm": run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, "net", *args)}


def ablation(lattice_cls, net, mask, Q, tau, c_kc, k_ref, precision="fp32", stream=None, sync=None,
             max_steps=400000, variant=0):
    """Every start of STARTS to the 0.1 % rule: what the network's velocity and
    pressure each add, and what it adds over the analytic Kozeny-Carman ramp."""
    return {name: run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, name, precision, stream, sync,
                            max_steps, variant) for name in STARTS}
