"""Learned warm start: training data from this library's own steady states, a
Kozeny-Carman pressure-drop estimate calibrated on them, and the warm-started
initial field f = f^eq(rho, u) (host orchestration only; the LBM, the network
forward/backward/Adam and the equilibrium initialisation run in the CUDA
library).

The network predicts, per pore voxel, u / u_D (u_D = Q / (nx ny)) and
G_SCALE * H, H = phi(z) (pbar(z) - pbar(z+1)) / (nu u_D): the drop of the
plane-mean pressure pbar (the mean of p = c_s^2 rho over the pore voxels of a
plane) from the voxel's plane to the next, times the plane's porosity phi(z)
(its pore fraction).  H is a property of the plane that each voxel estimates
from the geometry it sees; the porosity factor removes most of the spread of
the drop itself, which is large across planes with few pores (the mean
interstitial velocity there is u_D / phi).  (A local vertical pressure
difference averaged over vertically connected pores misses the plane-mean drop
by a factor of about two in these packs, so it is not used.)  The sum of the
drops is the whole pressure drop, so these targets reproduce the steady state's
permeability exactly.  G_SCALE makes the squared errors of H weigh about as
much as those of the velocity.  Initial fields of a new geometry with flux Q:
  u = u_D * net_u(mask)                                       (network velocity)
  rho(z) = rho_out + (nu u_D / c_s^2) sum_{z' >= z} Hbar(z') / phi(z')
with Hbar(z) the mean over the pore voxels of plane z of the predicted H
(network pressure), the drops divided by one constant c_net fitted on the
training boxes like c_KC below (least squares in log k of the whole boxes'
permeabilities against the network's); or, without the network, the analytic
ramp
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
G_SCALE = 4.0


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


def plane_means(field, mask):
    """Mean of field over the pore voxels of each z plane (0 for a plane without pores)."""
    pore = mask == 0
    cnt = pore.reshape(mask.shape[0], -1).sum(axis=1)
    tot = np.where(pore, field, 0.0).reshape(mask.shape[0], -1).sum(axis=1)
    return np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)


def plane_porosity(mask):
    return (mask == 0).reshape(mask.shape[0], -1).mean(axis=1)


def drop_target(rho, mask, Q, tau):
    """G_SCALE phi(z) (pbar(z) - pbar(z+1)) / (nu u_D) on the pore voxels of
    plane z, z < nz - 1; NaN (no target) at solids and on the last plane."""
    nz, ny, nx = mask.shape
    nu = CS2 * (tau - 0.5)
    uD = Q / (nx * ny)
    pbar = CS2 * plane_means(rho, mask)
    drop = np.append(G_SCALE * plane_porosity(mask)[:-1] * (pbar[:-1] - pbar[1:]) / (nu * uD), np.nan)
    return np.where(mask == 0, drop[:, None, None], np.nan)


def steady_targets(batch_cls, masks, tau, u_mean, steps, precision="fp32", stream=None, margin=0):
    """Run every geometry to (near) steady state in one batched ensemble and
    return (inputs, targets, permeabilities): with margin > 0 the inputs and
    targets are the interior crops mask[m:-m, m:-m, m:-m] (no lateral walls and
    no inlet or outlet planes inside them), else the whole boxes; targets are
    float32 [S][4][z][y][x] (u / u_D and G_SCALE H, u_D = Q / (nx ny) of the
    whole box); the permeabilities are the whole boxes'."""
    S = len(masks)
    Qs = [u_mean * int((m[0] == 0).sum()) for m in masks]
    sl = (slice(margin, -margin),) * 3 if margin > 0 else (slice(None),) * 3
    inputs = [np.ascontiguousarray(m[sl]) for m in masks]
    targets = np.zeros((S, 4) + inputs[0].shape, np.float32)
    ks = np.zeros(S)
    with batch_cls(masks, tau, "mrt", precision, stream=stream) as b:
        for k, q in enumerate(Qs):
            b.set_flux_bc(k, q)
        b.step(steps)
        for k, m in enumerate(masks):
            rho, ux, uy, uz = b.fields(k)
            nz, ny, nx = m.shape
            uD = Qs[k] / (nx * ny)
            targets[k, :3] = (np.stack([ux[sl], uy[sl], uz[sl]]) / uD).astype(np.float32)
            # drop_target's u_D is Q / (area of the box it is given): hand it the
            # whole box's u_D through an equivalent flux
            cz, cy, cx = inputs[k].shape
            targets[k, 3] = drop_target(rho[sl], inputs[k], uD * cx * cy, tau).astype(np.float32)
            _, rho_in = b.get_flux(k, 4)
            ks[k] = cv.permeability(Qs[k], m.shape, tau, rho_in, 1.0)
    return inputs, targets, ks


def fit_kc(masks, ks):
    """c_KC of k = c * phi^3 / (S^2 (1 - phi)^2), least squares in log k."""
    x = np.array([kc_features(m)[2] for m in masks])
    return float(np.exp(np.mean(np.log(ks) - np.log(x))))


def pressure_profile(G, mask, Q, tau, rho_out=1.0, c_net=1.0):
    """rho(z) from a predicted drop field (G_SCALE H): its plane means over the
    pore voxels, divided by the plane porosity, summed from the outlet, and
    divided by the calibration constant c_net."""
    nz, ny, nx = mask.shape
    nu = CS2 * (tau - 0.5)
    uD = Q / (nx * ny)
    phi = plane_porosity(mask)[:-1]
    hbar = plane_means(np.asarray(G, dtype=np.float64), mask)[:-1] / G_SCALE
    gbar = np.where(phi > 0, hbar / np.maximum(phi, 1e-300), 0.0)
    drop = np.concatenate([np.cumsum(gbar[::-1])[::-1], [0.0]])  # sum over z' >= z of Gbar(z')
    return rho_out + (nu * uD / CS2) * drop / c_net


def kc_profile(mask, Q, tau, c_kc, rho_out=1.0):
    """The linear Kozeny-Carman ramp rho(z)."""
    nz, ny, nx = mask.shape
    uD = Q / (nx * ny)
    k_est = c_kc * kc_features(mask)[2]
    nu = CS2 * (tau - 0.5)
    dp = nu * uD * (nz - 1) / k_est
    return rho_out + (dp / CS2) * (1.0 - np.arange(nz, dtype=np.float64) / (nz - 1))


def initial_fields(net, mask, Q, tau, c_kc, velocity="net", pressure="net", c_net=1.0):
    """(rho, ux, uy, uz) float64 arrays for Lattice.set_fields.  velocity:
    "net" (u = u_D * net_u) or "zero"; pressure: "net" (the network's profile,
    calibrated by c_net), "kc" (the Kozeny-Carman ramp) or "uniform" (rho = 1)."""
    nz, ny, nx = mask.shape
    uD = Q / (nx * ny)
    y = net.predict(mask).astype(np.float64) if (velocity == "net" or pressure == "net") else None
    u = y[:3] * uD if velocity == "net" else np.zeros((3,) + mask.shape)
    if pressure == "net":
        prof = pressure_profile(y[3], mask, Q, tau, c_net=c_net)
    elif pressure == "kc":
        prof = kc_profile(mask, Q, tau, c_kc)
    else:
        prof = np.ones(nz)
    rho = prof[:, None, None] + np.zeros(mask.shape)
    return rho, u[0], u[1], u[2]


def net_permeability(net, mask, Q, tau, c_net=1.0):
    """Darcy permeability implied by the network's pressure profile (the same
    definition the 0.1 % rule uses)."""
    rho = pressure_profile(net.predict(mask)[3].astype(np.float64), mask, Q, tau, c_net=c_net)
    return cv.permeability(Q, mask.shape, tau, rho[0], rho[-1])


def fit_net_scale(net, boxes, ks, tau, u_mean):
    """c_net: least squares in log k of the boxes' permeabilities against the
    network's uncalibrated estimates (the analogue of fit_kc)."""
    r = [np.log(k) - np.log(net_permeability(net, m, u_mean * int((m[0] == 0).sum()), tau))
         for m, k in zip(boxes, ks)]
    return float(np.exp(np.mean(r)))


# start name -> (velocity, pressure) of initial_fields; "cold" sets nothing
STARTS = {"cold": None, "kc_ramp": ("zero", "kc"), "net_velocity": ("net", "uniform"),
          "net_pressure": ("zero", "net"), "net": ("net", "net")}


def run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, start, precision="fp32", stream=None, sync=None,
              max_steps=400000, variant=0, c_net=1.0):
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
            rho, ux, uy, uz = initial_fields(net, mask, Q, tau, c_kc, *STARTS[start], c_net=c_net)
            lat.set_fields(rho, ux, uy, uz)
            if sync:
                sync()
            t_init = time.perf_counter() - t0
        r = cv.run_to_reference(lat, Q, tau, k_ref, max_steps=max_steps, sync=sync)
    return {"steps": r["steps"], "seconds": None if r["seconds"] is None else r["seconds"] + t_init,
            "init_seconds": t_init, "reached": r["reached"], "k": r["k"], "q_out": r["q_out"],
            "steps_run": r["steps_run"]}


def warm_vs_cold(lattice_cls, net, mask, Q, tau, c_kc, k_ref, precision="fp32", stream=None, sync=None,
                 max_steps=400000, variant=0, c_net=1.0):
    """The cold start and the full learned warm start (network velocity and pressure)."""
    args = (precision, stream, sync, max_steps, variant, c_net)
    return {"cold": run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, "cold", *args),
            "warm": run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, "net", *args)}


def ablation(lattice_cls, net, mask, Q, tau, c_kc, k_ref, precision="fp32", stream=None, sync=None,
             max_steps=400000, variant=0, c_net=1.0):
    """Every start of STARTS to the 0.1 % rule: what the network's velocity and
    pressure each add, and what it adds over the analytic Kozeny-Carman ramp."""
    return {name: run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, name, precision, stream, sync,
                            max_steps, variant, c_net) for name in STARTS}
