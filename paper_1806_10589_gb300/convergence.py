"""Time to steady flux: host-side orchestration of a Lattice run (no arithmetic
on the state happens here; every number comes from the library's kernels).

Two stopping rules:
  * Section 3.1 (Eq. stopping_criterion): sum|u(t) - u(t - lag)| / sum|u(t)| <= tol,
    lag = 1000 steps, tol = 1e-6 (lbm_steady_residual);
  * 0.1 % rule: the permeability k(t) is within rtol of a reference k_inf for
    `hold` consecutive checks (optionally also the outlet flux within rtol of Q).
    The outlet-plane sum of u_z is not the discrete mass flux across the outlet:
    warm-started runs reach the reference k (to 1e-8) and a constant total mass
    while that sum can stay ~1 % from Q, so it is reported, not required.

k(t) = nu * u_D * (nz - 1) / dp  (Darcy's law; the paper does not define it),
with nu = (tau - 1/2)/3 (Appendix A), u_D = Q / (nx ny) the superficial velocity
and dp = c_s^2 (rho_in - rho_out) from the inlet density of Eq. (potential).
"""
from __future__ import annotations

import time

CS2 = 1.0 / 3.0


def permeability(Q, shape, tau, rho_in, rho_out):
    nz, ny, nx = shape
    nu = CS2 * (tau - 0.5)
    dp = CS2 * (rho_in - rho_out)
    return nu * (Q / (nx * ny)) * (nz - 1) / dp if dp != 0 else float("inf")


def sample(lat, Q, tau, rho_out=1.0):
    q_out, _ = lat.get_flux(5)
    _, rho_in = lat.get_flux(4)
    return {"k": permeability(Q, lat.shape, tau, rho_in, rho_out), "q_out": q_out, "rho_in": rho_in}


def run_to_residual(lat, Q, tau, lag=1000, tol=1e-6, max_steps=400000, sync=None, min_steps=0):
    """Step until the Section 3.1 residual over `lag` steps is <= tol (and at
    least `min_steps` steps have run).  Returns dict(steps, seconds, residual,
    k, q_out, history)."""
    hist = []
    t0 = time.perf_counter()
    lat.steady_residual()
    steps = 0
    r = float("inf")
    while steps < max_steps:
        lat.step(lag)
        steps += lag
        r = lat.steady_residual()
        s = sample(lat, Q, tau)
        hist.append((steps, r, s["k"], s["q_out"]))
        if r <= tol and steps >= min_steps:
            break
    if sync:
        sync()
    secs = time.perf_counter() - t0
    s = sample(lat, Q, tau)
    return {"steps": steps, "seconds": secs, "residual": r, "k": s["k"], "q_out": s["q_out"],
            "converged": r <= tol, "history": hist}


def run_to_reference(lat, Q, tau, k_ref, rtol=1e-3, hold=10, check_every=100, max_steps=400000,
                     sync=None, require_q_out=False):
    """Step until k(t) stays within rtol of k_ref (and, if require_q_out, the
    outlet flux within rtol of Q) for `hold` consecutive checks.  t_steady is
    the first check of that run of checks.  Returns dict(steps, seconds, k,
    q_out, reached)."""
    t0 = time.perf_counter()
    steps = 0
    streak = 0
    first = None
    first_t = None
    while steps < max_steps:
        lat.step(check_every)
        steps += check_every
        s = sample(lat, Q, tau)
        ok = abs(s["k"] - k_ref) <= rtol * abs(k_ref)
        if require_q_out:
            ok = ok and abs(s["q_out"] - Q) <= rtol * abs(Q)
        if ok:
            if streak == 0:
                first, first_t = steps, time.perf_counter() - t0
            streak += 1
            if streak >= hold:
                break
        else:
            streak = 0
    if sync:
        sync()
    s = sample(lat, Q, tau)
    reached = streak >= hold
    return {"steps": first if reached else None, "seconds": first_t if reached else None,
            "k": s["k"], "q_out": s["q_out"], "reached": reached, "steps_run": steps}
