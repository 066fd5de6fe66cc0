"""Learned warm start: training data from this library's own steady states, a
Kozeny-Carman pressure-drop estimate calibrated on them, and the warm-started
initial field f = f^eq(rho, u) (host orchestration only; the LBM, the network
forward/backward/Adam and the equilibrium initialisation run in the CUDA
library).

Initial field of a new geometry with flux Q:
  u = u_D * net(mask),  u_D = Q / (nx ny)                    (network, u / u_D)
  rho(z) = rho_out + dp_est * (1 - z / (nz - 1)) * 3         (c_s^2 = 1/3)
  dp_est = nu u_D (nz - 1) / k_est                          (Darcy)
  k_est = c_KC * phi^3 / (S^2 (1 - phi)^2)                   (Kozeny-Carman)
with phi the porosity, S the pore-solid face count per voxel, and c_KC fitted
on the training set by least squares in log space.
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


def steady_targets(batch_cls, masks, tau, u_mean, steps, precision="fp32", stream=None):
    """Run every geometry to (near) steady state in one batched ensemble and
    return (targets u / u_D as float32 [S][3][z][y][x], permeabilities)."""
    S = len(masks)
    Qs = [u_mean * int((m[0] == 0).sum()) for m in masks]
    targets = np.zeros((S, 3) + masks[0].shape, np.float32)
    ks = np.zeros(S)
    with batch_cls(masks, tau, "mrt", precision, stream=stream) as b:
        for k, q in enumerate(Qs):
            b.set_flux_bc(k, q)
        b.step(steps)
        for k, m in enumerate(masks):
            _, ux, uy, uz = b.fields(k)
            nz, ny, nx = m.shape
            uD = Qs[k] / (nx * ny)
            targets[k] = (np.stack([ux, uy, uz]) / uD).astype(np.float32)
            _, rho_in = b.get_flux(k, 4)
            ks[k] = cv.permeability(Qs[k], m.shape, tau, rho_in, 1.0)
    return targets, ks


def fit_kc(masks, ks):
    """c_KC of k = c * phi^3 / (S^2 (1 - phi)^2), least squares in log k."""
    x = np.array([kc_features(m)[2] for m in masks])
    return float(np.exp(np.mean(np.log(ks) - np.log(x))))


def initial_fields(net, mask, Q, tau, c_kc, use_net=True, use_ramp=True):
    """(rho, ux, uy, uz) float64 arrays for Lattice.set_fields: u = u_D * net(mask)
    (or 0 without the network), rho the Darcy / Kozeny-Carman ramp (or 1
    without it)."""
    nz, ny, nx = mask.shape
    uD = Q / (nx * ny)
    if use_net:
        y = net.predict(mask).astype(np.float64) * uD
    else:
        y = np.zeros((3,) + mask.shape)
    rho = np.ones(mask.shape)
    if use_ramp:
        k_est = c_kc * kc_features(mask)[2]
        nu = CS2 * (tau - 0.5)
        dp = nu * uD * (nz - 1) / k_est
        z = np.arange(nz, dtype=np.float64)[:, None, None]
        rho = rho + (dp / CS2) * (1.0 - z / (nz - 1))
    return rho, y[0], y[1], y[2]


# start name -> (network velocity, Kozeny-Carman density ramp)
STARTS = {"cold": (False, False), "ramp_only": (False, True), "net_only": (True, False),
          "net_and_ramp": (True, True)}


def run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, start, precision="fp32", stream=None, sync=None,
              max_steps=400000, variant=0):
    """Steps and wall seconds to the 0.1 % rule (k within 1e-3 of k_ref for 10
    checks) from one of STARTS; the time of a warm start includes the network
    inference and the field upload."""
    use_net, use_ramp = STARTS[start]
    with lattice_cls(mask, tau, "mrt", precision, stream=stream) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        t_init = 0.0
        if use_net or use_ramp:
            if sync:
                sync()
            t0 = time.perf_counter()
            rho, ux, uy, uz = initial_fields(net, mask, Q, tau, c_kc, use_net, use_ramp)
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
    """The cold start and the full warm start (network velocity and ramp density)."""
    args = (precision, stream, sync, max_steps, variant)
    return {"cold": run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, "cold", *args),
            "warm": run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, "net_and_ramp", *args)}


def ablation(lattice_cls, net, mask, Q, tau, c_kc, k_ref, precision="fp32", stream=None, sync=None,
             max_steps=400000, variant=0):
    """All four starts (cold, ramp only, network only, both) to the 0.1 % rule:
    what the network adds over the analytic ramp, and the ramp over nothing."""
    return {name: run_start(lattice_cls, net, mask, Q, tau, c_kc, k_ref, name, precision, stream, sync,
                            max_steps, variant) for name in STARTS}
