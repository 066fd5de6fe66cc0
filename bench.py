#!/usr/bin/env python3
"""Throughput of the D3Q19 flux-boundary LBM step on GB300 (MLUPS).

Workload: single-fluid D3Q19 on a seeded synthetic 256^3 sphere pack (radii
U[6,12], voxel porosity 0.35, 6 pure-pore reservoir layers at each z end, pores
not reachable from the inlet filled), tau = 0.7, MRT collision, flux inlet with
mean velocity 1e-4 (Q = 1e-4 * A), fixed-density outlet, FP32 storage.  One
step = one launch of the step kernel over every pore node: pull streaming with
bounce-back, the Appendix B closures with the inlet density of Eq. (potential),
collision, store, and the FP64 reduction that forms the next step's inlet
density.  MLUPS counts pore nodes only.  The default run also reports the
time to steady flux (FP32 vs FP16/BF16 deviation storage, cold starts).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64|fp16dev|bf16dev]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

N > 1 (under torchrun) runs N independent replicas, one per GPU, with no
data-path communication (weak scaling); value = all ranks' pore updates / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from lbm_inputs import sphere_pack  # noqa: E402

METRIC = "MLUPS"
PACK = dict(n=256, rmin=6.0, rmax=12.0, porosity=0.35, seed=2024, reservoir=6)
TAU = 0.7
UBAR = 1e-4
BYTES_PER_VALUE = {"fp64": 8, "fp32": 4, "fp16dev": 2, "bf16dev": 2}
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0  # the ~8 TB/s nominal HBM3e peak (the measured copy bandwidth is the roofline)
PROFILE_TRAFFIC = {0: os.path.join(ROOT, "profiles", "k_step_fp32_sphere256.md"),
                   3: os.path.join(ROOT, "profiles", "k_step_aa_fp32_sphere256.md")}
VARIANT_NAMES = {0: "per-node pull kernel, two buffers", 1: "cp.async-pipelined, 256-node tiles",
                 2: "cp.async-pipelined, 128-node tiles", 3: "AA pattern, one buffer in place"}


# --------------------------------------------------------------- helpers ---
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    mask, info = sphere_pack(PACK["n"], PACK["rmin"], PACK["rmax"], PACK["porosity"], PACK["seed"],
                             reservoir=PACK["reservoir"])
    a_in = int((mask[0] == 0).sum())
    return mask, info, a_in


# the step kernels and their launch configurations; the host API (lbm_api.cu)
# only sequences launches and does not change the traffic of one
STEP_KERNEL_SOURCES = ("lbm_device.cuh", "lbm_internal.h", "lbm_kernels.cu")


def strip_c_comments(src):
    """C/C++ source without its // and /* */ comments (string and character
    literals kept as they are); each comment leaves one space or its newline."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "".join(out)


BATCH_KERNEL_SOURCES = ("lbm_batch.cu", "lbm_device.cuh", "lbm_internal.h")
PROFILE_BATCH = os.path.join(ROOT, "profiles", "k_batch_step_fp16_ensemble64.md")
CONV_KERNEL_SOURCES = ("wsnet.cu", "tc_util.cuh")
PROFILE_CONV = os.path.join(ROOT, "profiles", "k_conv_wgrad_bf16_32x32.md")


def kernel_sources_sha(sources=STEP_KERNEL_SOURCES):
    """Hash of the code (comments stripped, whitespace runs collapsed) of the
    sources that define a kernel and its launch (by default the single-lattice
    step kernel); other modules of the library do not change it, and a comment
    or layout edit does not invalidate a profile."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1806_10589_gb300", "csrc")
    for f in sources:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            code = re.sub(r"\s+", " ", strip_c_comments(fh.read())).strip()
            h.update(f.encode() + b"\0" + code.encode())
    return h.hexdigest()[:16]


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_copy_gbs", "hbm_GBs"):
            if k in d and d[k]:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def measured_bf16_peak():
    """Dense BF16 tensor throughput (TFLOP/s) for a kernel timed alone: the
    burst cuBLAS figure of MEASURED_PEAKS.json, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        if d.get("bf16_tflops"):
            return float(d["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except (OSError, ValueError):
        pass
    return 1900.0, "fallback 1.9 PFLOP/s"


def profiled_traffic(sha, variant=0, path=None):
    """dram bytes per launch of the step kernel (or of the kernel whose summary
    is `path`) from the committed ncu summary, if it was taken on the current
    kernel sources (else None)."""
    try:
        txt = open(path or PROFILE_TRAFFIC[variant]).read()
    except (OSError, KeyError):
        return None
    m_sha = re.search(r"kernel_sources_sha:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not (m_sha and m_b) or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


ORACLE_CHILD = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
m = np.load(sys.argv[2])
steps = int(sys.argv[3]); tau = float(sys.argv[4]); Q = float(sys.argv[5])
o = oracle.D3Q19Oracle(m, tau, "mrt", Q=Q)
o.step(1)  # warm-up (allocations)
t = time.perf_counter()
o.step(steps)
dt = time.perf_counter() - t
print(json.dumps({"seconds": dt, "n_pore": int((m == 0).sum()), "steps": steps}))
"""


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    return env


def oracle_rate(mask, steps, tau=TAU, ubar=UBAR):
    """Run the FP64 CPU oracle on `mask` in a single-threaded child process;
    return (MLUPS, seconds, n_pore)."""
    r = oracle_rate_parallel([mask], steps, tau, ubar)
    return r["mlups"], r["seconds"], r["n_pore"]


def oracle_rate_parallel(masks, steps, tau=TAU, ubar=UBAR):
    """Run one single-threaded FP64 oracle child process per mask, all at the
    same time (one per host core); aggregate MLUPS = all children's pore-node
    updates over the longest child's timed region."""
    with tempfile.TemporaryDirectory() as td:
        procs = []
        for j, m in enumerate(masks):
            p = os.path.join(td, "mask%d.npy" % j)
            np.save(p, m)
            a_in = int((m[0] == 0).sum())
            procs.append(subprocess.Popen([sys.executable, "-c", ORACLE_CHILD, ROOT, p, str(steps), str(tau),
                                           repr(ubar * a_in)], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                          text=True, env=_oracle_env()))
        res = []
        for pr in procs:
            out, err = pr.communicate()
            if pr.returncode != 0:
                raise RuntimeError("oracle child failed: " + err[-2000:])
            res.append(json.loads(out.strip().splitlines()[-1]))
    secs = max(d["seconds"] for d in res)
    n = sum(d["n_pore"] for d in res)
    return {"mlups": n * steps / secs / 1e6, "seconds": secs, "n_pore": n, "children": len(res)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def host_cpu_model():
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def host_mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 16 << 30


def crop_for_budget(mask, seconds_per_step, probe_mlups, z0=0, max_cells=None):
    """A z-slab of the pack starting at plane z0 (full x/y extent, shrunk if
    needed) whose oracle step takes about `seconds_per_step`."""
    nz, ny, nx = mask.shape
    phi = float((mask == 0).mean())
    cells = max(seconds_per_step * probe_mlups * 1e6 / phi, 4 * 4 * 3)
    if max_cells:
        cells = min(cells, max_cells)
    if cells >= nx * ny * 3:
        dz = int(min(nz, max(3, cells // (nx * ny))))
        z0 = max(0, min(z0, nz - dz))
        sub = mask[z0:z0 + dz].copy()
    else:
        side = int(max(4, min(nx, (cells / 3) ** 0.5)))
        z0 = max(0, min(z0, nz - 3))
        sub = mask[z0:z0 + 3, :side, :side].copy()
    for zz in (0, -1):  # the flux inlet and the pressure outlet need pores on their planes
        if not (sub[zz] == 0).any():
            sub[zz] = 0
    return sub


def oracle_samples(mask, seconds_per_step, probe_mlups, cores):
    """One z-slab of the pack per core, spread over the whole depth (slabs may
    overlap; each is an independent problem), sized for `seconds_per_step` of
    single-core oracle time per step and for the host memory left."""
    budget_cells = 0.25 * host_mem_available() / max(1, cores) / 2000.0  # ~2 kB of oracle arrays per cell
    nz = mask.shape[0]
    out = []
    for j in range(cores):
        z0 = int(round(j * max(0, nz - 3) / max(1, cores - 1))) if cores > 1 else 0
        out.append(crop_for_budget(mask, seconds_per_step, probe_mlups, z0=z0, max_cells=budget_cells))
    return out


def aggregate(n_local, K, ms_local, world, device=None):
    """Whole-job MLUPS: every rank's pore-node updates over the slowest rank's
    timed region (max over ranks); returns (MLUPS, max ms)."""
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        ms, total = float(t.item()), float(c.item())
    else:
        ms, total = ms_local, float(n_local)
    return total * K / (ms * 1e-3) / 1e6, ms


def velocity_errors(u, u_ref, pore):
    """Relative L2 error of the velocity over pore nodes, and the largest
    absolute error (also relative to the largest reference speed)."""
    du = np.stack([a[pore] - b[pore] for a, b in zip(u, u_ref)])
    ref = np.stack([b[pore] for b in u_ref])
    n_ref = float(np.sqrt((ref ** 2).sum()))
    mx = float(np.abs(du).max())
    return {"u_l2_rel": float(np.sqrt((du ** 2).sum())) / n_ref, "u_max_abs": mx,
            "u_max_rel": mx / float(np.abs(ref).max())}


def error_block(lat, Q, k_ref, q_ref, u_ref, pore):
    from paper_1806_10589_gb300 import convergence as cv

    s = cv.sample(lat, Q, TAU)
    _, ux, uy, uz = lat.fields()
    out = {"k_rel": (s["k"] - k_ref) / k_ref, "q_out_rel": (s["q_out"] - q_ref) / Q}
    out.update(velocity_errors((ux, uy, uz), u_ref, pore))
    return out


def time_to_steady(mask, a_in, stream, max_steps=150000, variant=3, precs=("fp32", "fp16dev", "bf16dev"),
                   bias_steps=10000):
    """Time to steady flux on the benchmark workload, all on step variant
    `variant`, against an FP64 reference:
      1. FP32 cold run to the Section 3.1 rule (residual over 1000 steps <= 1e-6);
      2. the FP64 GPU path (pinned to the FP64 oracle at 1e-11) from that state's
         distributions, to the same rule and at least 6000 steps: k_inf, Q_out and
         u of FP64;
      3. FP32 / FP16-dev / BF16-dev cold runs until k(t) is within 0.1 % of the
         FP64 k_inf for 10 consecutive checks (every 100 steps); wall times include
         the checks; k, Q_out and u errors against FP64 when the rule is met;
      4. each format started from the FP64 steady state and run `bias_steps`
         steps: its steady-state error against FP64."""
    import torch

    from paper_1806_10589_gb300 import Lattice, convergence as cv

    Q = UBAR * a_in
    pore = mask == 0
    sync = torch.cuda.synchronize
    out = {"criterion": "k within 0.1% of the FP64 k_inf for 10 consecutive checks (every 100 steps)",
           "step_variant": "%d: %s" % (variant, VARIANT_NAMES[variant])}
    with Lattice(mask, TAU, "mrt", "fp32", stream=stream) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        r32 = cv.run_to_residual(lat, Q, TAU, lag=1000, tol=1e-6, max_steps=max_steps, sync=sync)
        f32 = lat.distributions()
    out["fp32_reference_run"] = {"steps": r32["steps"], "seconds": round(r32["seconds"], 3),
                                 "residual": r32["residual"], "converged": r32["converged"], "k": r32["k"]}
    with Lattice(mask, TAU, "mrt", "fp64", stream=stream) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        lat.set_distributions(f32)
        r64 = cv.run_to_residual(lat, Q, TAU, lag=1000, tol=1e-6, max_steps=40000, sync=sync, min_steps=6000)
        f64 = lat.fields()
    del f32
    k_inf, q64 = r64["k"], r64["q_out"]
    u64 = f64[1:]
    out["k_inf"] = k_inf
    out["fp64_reference_run"] = {"start": "the FP32 steady state's distributions", "steps": r64["steps"],
                                 "seconds": round(r64["seconds"], 3), "residual": r64["residual"],
                                 "converged": r64["converged"], "k": k_inf, "q_out_rel_to_Q": (q64 - Q) / Q,
                                 "fp32_reference_k_rel": (r32["k"] - k_inf) / k_inf}
    for prec in precs:
        with Lattice(mask, TAU, "mrt", prec, stream=stream) as lat:
            lat.set_kernel(variant)
            lat.set_flux_bc(Q)
            rr = cv.run_to_reference(lat, Q, TAU, k_inf, max_steps=min(max_steps, 60000), sync=sync)
            at_rule = error_block(lat, Q, k_inf, q64, u64, pore)
        with Lattice(mask, TAU, "mrt", prec, stream=stream) as lat:
            lat.set_kernel(variant)
            lat.set_flux_bc(Q)
            lat.set_fields(*f64)
            lat.step(bias_steps)
            steady = error_block(lat, Q, k_inf, q64, u64, pore)
        out[prec] = {"steps": rr["steps"], "seconds": None if rr["seconds"] is None else round(rr["seconds"], 3),
                     "reached": rr["reached"], "steps_run": rr["steps_run"],
                     "vs_fp64": {"at_rule": at_rule,
                                 "steady": dict(steady, note="from the FP64 steady state, %d steps" % bias_steps)}}
    return out


def ensemble_workload(n_members=64, seed=7):
    """Config-4-shaped ensemble: cubes with edges drawn uniformly from 64..160,
    each its own seeded sphere pack (radii U[6,12], porosity 0.35, no reservoirs),
    flux targets u_mean U[5e-5, 2e-4] times the member's inlet pore count."""
    rng = np.random.default_rng(seed)
    edges = rng.integers(64, 161, size=n_members)
    umean = rng.uniform(5e-5, 2e-4, size=n_members)
    masks = []
    for k, e in enumerate(edges):
        m, _ = sphere_pack(int(e), 6.0, 12.0, 0.35, seed=1000 + k, reservoir=0)
        masks.append(m)
    Qs = [float(u) * int((m[0] == 0).sum()) for u, m in zip(umean, masks)]
    return masks, Qs, edges


def ensemble_steady(masks, Qs, stream, config, prec="fp16dev", max_steps=40000, every=200, hold=10, rtol=1e-3):
    """Cold start of the ensemble in launch configuration `config`, run for
    max_steps, recording every
    member's permeability k(t) (Darcy, from the inlet density) and outlet flux
    every `every` steps.  Each member's k_inf is its value at the end of the run
    (its flatness over the last fifth is reported).  A member is steady from the
    first check after which |k - k_inf| <= rtol k_inf and |Q_out - Q| <= rtol Q
    hold for `hold` consecutive checks; the ensemble is steady when its last
    member is."""
    import torch

    from paper_1806_10589_gb300 import Batch, convergence as cv

    nm = len(masks)
    ks, qs = [], []
    with Batch(masks, TAU, "mrt", prec, stream=stream) as b:
        b.set_config(config)
        for m, q in enumerate(Qs):
            b.set_flux_bc(m, q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max_steps // every):
            b.step(every)
            row_k, row_q = [], []
            for m in range(nm):
                q_out, _ = b.get_flux(m, 5)
                _, rho_in = b.get_flux(m, 4)
                row_k.append(cv.permeability(Qs[m], masks[m].shape, TAU, rho_in, 1.0))
                row_q.append(q_out)
            ks.append(row_k)
            qs.append(row_q)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
    out = steady_summary(np.array(ks), np.array(qs), Qs, every, hold, rtol, max_steps)
    out["seconds_run"] = round(secs, 2)
    return out


def steady_summary(ks, qs, Qs, every, hold, rtol, max_steps):
    """Per-member time to the 0.1 % rule from recorded histories ks, qs
    (checks x members): k_inf = the last k of each member."""
    nm = ks.shape[1]
    Qa = np.asarray(Qs, dtype=float)
    k_inf = ks[-1]
    tail = ks[int(0.8 * len(ks)):]
    flat = float(np.max(np.abs(tail - k_inf) / k_inf))
    ok = (np.abs(ks - k_inf) <= rtol * k_inf) & (np.abs(qs - Qa) <= rtol * Qa)
    first = []
    for m in range(nm):
        run, start = 0, None
        for t in range(len(ok)):
            run = run + 1 if ok[t, m] else 0
            if run == 1:
                start = t
            if run >= hold:
                break
        first.append((start + 1) * every if run >= hold else None)
    reached = [f for f in first if f is not None]
    crit = (f"k within {100 * rtol:g}% of the member's k at the end of a {max_steps}-step run and outlet flux "
            f"within {100 * rtol:g}% of Q_i, for {hold} consecutive checks every {every} steps")
    return {"criterion": crit, "members_reached": len(reached), "members": nm,
            "steps_all_steady": max(reached) if len(reached) == nm else None,
            "steps_median_member": int(np.median(reached)) if reached else None,
            "k_inf_flatness_last_fifth": flat}


def run_ensemble(stream, prec="fp16dev", steps=2000, warmup=64, steady_steps=True):
    """Throughput of the batched ensemble step in the launch configuration the
    library's autotuner picks (per-step launches under a graph or one persistent
    launch; two register caps each), and the step's HBM roofline."""
    import torch

    from paper_1806_10589_gb300 import BATCH_CONFIGS, Batch

    masks, Qs, edges = ensemble_workload()
    with Batch(masks, TAU, "mrt", prec, stream=stream) as b:
        for k, q in enumerate(Qs):
            b.set_flux_bc(k, q)
        b.step(warmup)
        best, trial_ms = b.autotune(128)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        k_ms = b.time_step(100)
        n = b.info()["n_pore"]
        fl = [b.get_flux(k, 4)[0] for k in range(len(masks))]
    steady = ensemble_steady(masks, Qs, stream, best, prec) if steady_steps else None
    s = BYTES_PER_VALUE[prec]
    peak, _ = measured_hbm_peak()
    ach = 2 * 19 * s * n / (k_ms * 1e-3) / 1e9
    return {"workload": "64 sphere packs, edges U{64..160} (%d..%d), porosity 0.35, tau 0.7, "
                        "u_mean U[5e-5,2e-4], %s storage" % (int(edges.min()), int(edges.max()), prec),
            "n_pore": n, "steps": steps, "MLUPS": round(n * steps / (ms * 1e-3) / 1e6, 1),
            "ms_per_step": round(ms / steps, 5),
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4),
                         "traffic": profiled_traffic(kernel_sources_sha(BATCH_KERNEL_SOURCES), path=PROFILE_BATCH)
                         if best in (0, 1) else None,
                         "kernel": {2: "k_batch_persistent", 3: "k_batch_persistent", 4: "k_batch_aa", 5: "k_batch_aa"}.get(best, "k_batch_step"),
                         "kernel_ms": round(k_ms, 5), "bytes_per_unit": 2 * 19 * s},
            "autotune": {"chosen": BATCH_CONFIGS[best],
                         "ms_per_step": {BATCH_CONFIGS[c]: round(t, 5) for c, t in enumerate(trial_ms)}},
            "max_inlet_flux_rel_err": max(abs(f - q) / q for f, q in zip(fl, Qs)),
            "steady": steady}


def laplace_gamma(stream, alpha=0.01, beta=0.95, n=48, R=12.0, steps=3000):
    """Interfacial tension of the colour model for (alpha, beta): Laplace law
    gamma = Delta p R / 2 for a static droplet of phase A in a closed box."""
    from paper_1806_10589_gb300 import ColorLattice

    m = np.zeros((n, n, n), np.uint8)
    m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = 1, 1, 1, 1, 1, 1
    c0 = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - c0) ** 2 + (y - c0) ** 2 + (z - c0) ** 2)
    with ColorLattice(m, 1.0, alpha, beta, -1.0, "fp32", stream=stream) as c:
        c.set_phase(np.where(r < R, 1.0, -1.0))
        c.step(steps)
        rho, _, _, _, _ = c.fields()
    dp = (rho[(r < R - 4) & (m == 0)].mean() - rho[(r > R + 4) & (r < R + 10) & (m == 0)].mean()) / 3.0
    return dp * R / 2.0


def run_two_fluid(stream, steps=500, warmup=20, total_steps=50000):
    """Colour-model step on a 192x192x384 seeded sphere pack (radii U[5,10],
    porosity 0.35), FP32, the sample and the outlet reservoir saturated with the
    wetting phase B, the 6-layer inlet reservoir with the non-wetting phase A,
    A injected at the flux of Ca = mu_w Q / (gamma eps A) = 1e-5
    (Section 3.2), gamma from the Laplace calibration of (alpha, beta).  The step
    is timed over `steps` steps; the run then continues to `total_steps` and
    reports the inlet flux and density there."""
    import torch

    from paper_1806_10589_gb300 import ColorLattice, drainage

    alpha, beta, tau = 0.01, 0.95, 1.0
    gamma = laplace_gamma(stream, alpha, beta)
    mask, info = sphere_pack((192, 192, 384), 5.0, 10.0, 0.35, seed=31, reservoir=6)
    nz, ny, nx = mask.shape
    eps = info["porosity"]
    Q = drainage.simulated_flux(1e-5, eps, nx * ny, gamma, drainage.lattice_viscosity(tau))
    with ColorLattice(mask, tau, alpha, beta, -1.0, "fp32", stream=stream) as c:
        # Section 3.2 set-up: the inlet reservoir holds the non-wetting phase, the
        # sample and the outlet reservoir the wetting phase
        zz = np.arange(nz)[:, None, None] * np.ones(mask.shape)
        c.set_phase(np.where(zz < 6, 1.0, -1.0))
        c.set_flux_bc(Q, 1.0)
        c.step(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        q_in, _ = c.get_flux(4)
        # the rest of the 50,000-step run: the inlet flux stays exact
        c.step(total_steps - warmup - steps)
        q_in_end, rho_in_end = c.get_flux(4)
    n = int((mask == 0).sum())
    unit = 82 * 4  # FP32 values per node and step as built: f 19+19, A/B 14+14, phase 1, pre-pass A/B 14 + phi 1
    unit_min = 66 * 4  # a single pass: f 19+19, A/B 14+14
    peak, _ = measured_hbm_peak()
    ach = unit * n / (ms * 1e-3 / steps) / 1e9
    ach_min = unit_min * n / (ms * 1e-3 / steps) / 1e9
    return {"workload": "two-fluid colour model, 192x192x384 sphere pack (radii 5-10, porosity %.3f, 6+6 "
                        "reservoir layers, inlet reservoir non-wetting), tau 1, alpha %g, beta %g, wetting solid, non-wetting injected "
                        "at Ca 1e-5, FP32" % (eps, alpha, beta),
            "gamma_laplace": gamma, "Q": Q, "n_pore": n, "steps": steps,
            "MLUPS": round(n * steps / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms / steps, 5),
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4), "bytes_per_unit": unit,
                         "kernels": "k_color_pre + k_color_step",
                         "single_pass": {"bytes_per_unit": unit_min, "achieved": round(ach_min, 1),
                                         "frac": round(ach_min / peak, 4),
                                         "note": "against the 66 values a single-pass step must move; the "
                                                 "pre-pass re-reads the 14 D3Q7 values and writes and reads phi"}},
            "inlet_flux_rel_err": abs(q_in - Q) / Q,
            "run_to_step": total_steps,
            "inlet_flux_rel_err_end": abs(q_in_end - Q) / Q, "rho_in_end": rho_in_end}


def cpu_baseline(mask, seconds_per_step, steps):
    """The FP64 oracle as it stands on every host core: one single-threaded
    child per core, each on its own slab of the pack, all at once."""
    cores = host_cores()
    probe_mlups, _, _ = oracle_rate(mask[:16].copy(), 1)
    samples = oracle_samples(mask, seconds_per_step, probe_mlups, cores)
    r = oracle_rate_parallel(samples, steps)
    shp = samples[0].shape
    return {"value": round(r["mlups"], 4), "unit": METRIC, "cores": r["children"], "kind": "oracle",
            "cpu_model": host_cpu_model(), "single_core_probe_mlups": round(probe_mlups, 4),
            "sample": "FP64 numpy oracle, %d single-threaded processes at once (one per host core), %d steps "
                      "each on its own %dx%dx%d z-slab of the same pack (slabs spread over the depth; %d pore "
                      "nodes in all; %.1f s)" % (r["children"], steps, shp[2], shp[1], shp[0], r["n_pore"],
                                                 r["seconds"])}


# ------------------------------------------------------------- our path ---
def timed_launches(W, K, variant, prec, interval=1024, graph=64):
    """Kernel launches of the library inside the timed lbm_step(K) call that
    follows the warm-up lbm_step(W) call on a fresh lattice: the step launches,
    and for the 16-bit formats the reference refresh (re-encode, inlet density)
    every `interval` steps; on the AA pattern (variant 3) the layout swap into
    the in-place layout when the buffer is not already in it, and before a
    refresh the swap back (with an un-stream after a gather-scatter launch).
    Restates the host logic of lbm_step."""
    is16 = prec in ("fp16dev", "bf16dev")
    st = {"since": 0, "resident": False, "phase": 0}

    def call(n):
        c = 0
        if variant == 3:
            done = 0
            while done < n:
                if is16 and st["since"] >= interval:
                    if st["resident"]:
                        c += 1 + st["phase"]
                        st["resident"], st["phase"] = False, 0
                    c += 2
                    st["since"] = 0
                seg = n - done
                if is16:
                    seg = min(seg, interval - st["since"])
                if not st["resident"]:
                    c += 1
                    st["resident"], st["phase"] = True, 0
                c += seg
                st["phase"] = (st["phase"] + seg) & 1
                done += seg
                st["since"] += seg
            return c
        k = 0
        while k < n:
            chunk = graph if n - k >= graph else 1
            if is16 and st["since"] >= interval:
                c += 2
                st["since"] = 0
            c += chunk
            k += chunk
            st["since"] += chunk
        return c

    call(W)
    return call(K)


def run_ours(args, rank, world, local):
    import torch

    from paper_1806_10589_gb300 import Lattice, load_library

    torch.cuda.set_device(local)
    load_library()
    dev_name = torch.cuda.get_device_name(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mask, info, a_in = workload()
    Q = UBAR * a_in
    prec = args.precision
    stream = torch.cuda.current_stream()
    variant = args.variant
    lat = Lattice(mask, TAU, "mrt", prec, stream=stream)
    lat.set_kernel(variant)
    lat.set_flux_bc(Q)
    meta = lat.info()
    n = meta["n_pore"]
    K, W = args.steps, args.warmup

    # warm-up: builds and replays the captured graphs
    lat.step(W)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    value, ms = aggregate(n, K, ms, world, "cuda")
    mon = lat.monitors(raise_unstable=False)
    q_in, rho_in = lat.get_flux(4)

    # dominant kernel: CUDA events around every launch, on the launching stream
    k_prof = max(4, min(K, 400)) // 2 * 2
    ms_step_k, ms_inlet_k = lat.time_kernels(k_prof)
    s = BYTES_PER_VALUE[prec]
    unit_bytes = 2 * 19 * s
    achieved = unit_bytes * n / (ms_step_k * 1e-3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    sha = kernel_sources_sha()
    traffic = profiled_traffic(sha, variant) if prec == "fp32" else None
    per_kernel = None
    if variant == 3:
        # the AA step alternates two launches (each one full step): time the
        # gather-scatter launch alone (a 1-step call) and infer the node-local one
        odd = sum(lat.time_kernels(1)[0] for _ in range(40)) / 40
        even = max(2 * ms_step_k - odd, 1e-6)
        per_kernel = {name: {"ms": round(t, 5), "achieved": round(unit_bytes * n / (t * 1e-3) / 1e9, 1),
                             "frac": round(unit_bytes * n / (t * 1e-3) / 1e9 / peak, 4)}
                      for name, t in (("k_step_aa<odd> (gather-scatter)", odd),
                                      ("k_step_aa<even> (node-local)", even))}
    lat.close()

    # end to end through the public API with host buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with Lattice(mask, TAU, "mrt", prec, stream=stream) as lat2:
        lat2.set_kernel(variant)
        lat2.set_flux_bc(Q)
        lat2.step(K)
        rho, ux, uy, uz = lat2.fields()
    t1 = time.perf_counter()
    nz, ny, nx = mask.shape
    h2d = 4 * (nx + 2) * (ny + 2) * (nz + 2) + 4 * n + 64
    d2h = 4 * 8 * nx * ny * nz
    e2e_mlups = n * K / (t1 - t0) / 1e6

    ens = None
    if rank == 0 and args.ensemble:
        ens = run_ensemble(stream)

    two = None
    if rank == 0 and args.two_fluid:
        two = run_two_fluid(stream)

    steady = None
    if rank == 0 and args.steady:
        steady = time_to_steady(mask, a_in, stream, variant=args.variant)

    warm = None
    if rank == 0 and args.ws_leg:
        warm = run_warmstart_leg(stream, args.ws_samples, 64, args.ws_lbm_steps, args.ws_epochs, 256,
                                 args.variant, args.ws_ref_steps)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mask, seconds_per_step=3.0, steps=3)

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": METRIC, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(ms / K, 6), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32",
                                                          "fp16dev": "f16", "bf16dev": "bf16"}[prec],
        "data": "synthetic",
        "config": {"workload": "D3Q19 MRT flux-BC LBM, 256^3 sphere pack (radii 6-12, porosity %.3f, "
                               "6+6 reservoir layers), tau 0.7, u_mean 1e-4, %s storage" % (info["porosity"], prec),
                   "n_pore": n, "a_in": meta["a_in"], "box": [nx, ny, nz], "precision": prec,
                   "parallelism": "replicas" if world > 1 else "single",
                   "step_variant": "%d: %s" % (variant, VARIANT_NAMES[variant]),
                   "l2": "inputs larger than L2 (%s f buffer%s of %.0f MB)" % (
                       "one" if variant == 3 else "two", "" if variant == 3 else "s", 19 * s * n / 1e6),
                   "device": dev_name},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "frac_vs_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "kernel": "k_step_aa<odd/even> (alternating; each launch is one full step; "
                               "pair mean)" if variant == 3 else "k_step",
                     "kernel_ms": round(ms_step_k, 5), "per_kernel": per_kernel,
                     "bytes_per_unit": unit_bytes, "units_per_launch": n,
                     "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                     if peak_kind == "measured" else "fallback 6.8 TB/s"},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_mlups, 2), "unit": METRIC, "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": d2h / K},
        "gpu_launches": timed_launches(W, K, variant, prec),
        "time_to_steady": steady,
        "warm_start": warm,
        "ensemble": ens,
        "two_fluid": two,
        "clocks": clk,
        "check": {"q_in": q_in, "Q": Q, "rho_in": rho_in, "u_max": mon["u_max"], "status": mon["status"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------ reference (oracle) ---
def run_reference(args, rank, world, local):
    if rank != 0:
        return
    mask, info, a_in = workload()
    K, W = args.steps, args.warmup
    per_step = max(0.02, min(8.0, 60.0 / max(1, K + W)))
    cores = host_cores()
    probe_mlups, _, _ = oracle_rate(mask[:16].copy(), 1)
    samples = oracle_samples(mask, per_step, probe_mlups, cores)
    if W:
        oracle_rate_parallel(samples, W)
    r = oracle_rate_parallel(samples, K)
    shp = samples[0].shape
    desc = ("FP64 numpy oracle, %d single-threaded processes at once (one per host core); each step is one "
            "oracle step of every process on its own %dx%dx%d z-slab of the 256^3 pack (%d pore nodes in all)"
            % (r["children"], shp[2], shp[1], shp[0], r["n_pore"]))
    line = {"impl": "reference", "metric": METRIC, "value": round(r["mlups"], 4), "unit": METRIC,
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": round(1e3 * r["seconds"] / K, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "D3Q19 MRT flux-BC LBM, 256^3 sphere pack (radii 6-12, porosity %.3f, "
                                   "6+6 reservoir layers), tau 0.7, u_mean 1e-4" % info["porosity"],
                       "sample": desc},
            "cpu_baseline": {"kind": "oracle", "cores": r["children"], "cpu_model": host_cpu_model(),
                             "sample": desc, "value": round(r["mlups"], 4), "unit": METRIC},
            "e2e": {"value": round(r["mlups"], 4), "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def net_flops(levels=4, base=32, side=64):
    """Algorithmic FLOPs of one sample's forward pass (2 per multiply-add, real
    channels, interior voxels) and of a training step's forward + backward (data
    gradients of every layer but the first, weight gradients of all)."""
    c = [base << l for l in range(levels)]
    lay = [(c[0], 1, 0), (c[0], c[0], 0)]
    for l in range(1, levels):
        lay += [(c[l], c[l - 1], l), (c[l], c[l], l)]
    for l in range(levels - 2, -1, -1):
        lay += [(c[l], c[l + 1], l), (c[l], c[l], l)]
    lay.append((3, c[0], 0))
    f = [2.0 * 27 * co * ci * (side >> l) ** 3 for co, ci, l in lay]
    return sum(f), 3 * sum(f) - f[0]


def conv_roofline(stream, side=64, batch=8, reps=20):
    """CUDA-event times of the dominant convolution shape of the network (32 ->
    32 channels at full resolution, 8 samples of 64^3: 2.1 M voxels) for the
    forward, data-gradient and weight-gradient kernels, as tensor-core
    throughput on interior voxels against the measured BF16 dense peak."""
    import torch

    from paper_1806_10589_gb300 import conv3d_bf16

    g = torch.Generator(device="cuda").manual_seed(3)
    shp = (batch, side + 2, side + 2, side + 2, 32)
    a = torch.zeros(shp, dtype=torch.bfloat16, device="cuda")
    gr = torch.zeros(shp, dtype=torch.bfloat16, device="cuda")
    a[:, 1:-1, 1:-1, 1:-1] = torch.randn((batch, side, side, side, 32), generator=g, device="cuda").bfloat16()
    gr[:, 1:-1, 1:-1, 1:-1] = torch.randn((batch, side, side, side, 32), generator=g, device="cuda").bfloat16()
    w = (torch.randn((32, 27, 32), generator=g, device="cuda") * 0.03).bfloat16()
    out = torch.empty(shp, dtype=torch.bfloat16, device="cuda")
    gw = torch.zeros((32, 27, 32), dtype=torch.float32, device="cuda")
    args = (batch, side, side, side, 32, 32)
    conv3d_bf16(0, a.data_ptr(), 0, w.data_ptr(), 0, 1, out.data_ptr(), *args, stream=stream)  # warm-up
    ms = {"forward": conv3d_bf16(0, a.data_ptr(), 0, w.data_ptr(), 0, 1, out.data_ptr(), *args, stream=stream,
                                 reps=reps),
          "data_gradient": conv3d_bf16(1, gr.data_ptr(), 0, w.data_ptr(), 0, 0, out.data_ptr(), *args,
                                       stream=stream, reps=reps),
          "weight_gradient": conv3d_bf16(2, a.data_ptr(), gr.data_ptr(), w.data_ptr(), 0, 0, gw.data_ptr(), *args,
                                         stream=stream, reps=reps)}
    flops = 2.0 * 27 * 32 * 32 * batch * side ** 3
    peak, kind = measured_bf16_peak()
    per = {k: {"ms": round(v, 5), "achieved": round(flops / (v * 1e-3) / 1e12, 1),
               "frac": round(flops / (v * 1e-3) / 1e12 / peak, 4)} for k, v in ms.items()}
    return {"bound": "tensor", "unit": "TFLOP/s", "peak": peak, "peak_source": kind,
            "shape": "3x3x3 conv 32 -> 32 channels, %d x %d^3 voxels (BF16, FP32 accumulate)" % (batch, side),
            "flops_per_launch": flops, "per_kernel": per, "achieved": per["forward"]["achieved"],
            "frac": per["forward"]["frac"], "kernel": "k_conv<32,32> (forward)",
            "traffic": profiled_traffic(kernel_sources_sha(CONV_KERNEL_SOURCES), path=PROFILE_CONV)}


def run_warmstart_leg(stream, samples=512, side=64, lbm_steps=8000, epochs=40, test_side=256, variant=3,
                      ref_steps=300000, margin=8):
    """Learned warm start: train the network (4 levels, 32 base channels) on LBM
    steady states of seeded sphere packs (radii U[8,16], porosity U[0.25,0.45])
    computed by this library, 64^3 interior crops of 80^3 packs, then run five starts of a seeded
    test pack (radii 8-16, porosity 0.35) to the 0.1 % rule: cold, the
    Kozeny-Carman density ramp (no network), the network's velocity only, its
    pressure only, and both.  Clocks are sampled over the whole leg."""
    import torch

    from paper_1806_10589_gb300 import Batch, Lattice, WarmStartNet, convergence as cv, warmstart as ws

    sync = torch.cuda.synchronize
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    rng = np.random.default_rng(11)
    t0 = time.perf_counter()
    # packs of side + 2 margin; the network learns from their interior side^3
    # crops, away from the lateral walls (whose channelling raises a small box's
    # permeability) and from the inlet and outlet planes
    boxes = [sphere_pack(side + 2 * margin, 8.0, 16.0, float(rng.uniform(0.25, 0.45)), seed=5000 + k)[0]
             for k in range(samples)]
    t_geo = time.perf_counter() - t0
    t0 = time.perf_counter()
    masks, targets, ks = ws.steady_targets(Batch, boxes, TAU, UBAR, lbm_steps, stream=stream, margin=margin)
    sync()
    t_lbm = time.perf_counter() - t0
    c_kc = ws.fit_kc(boxes, ks)  # the Kozeny-Carman constant of the whole boxes' permeabilities
    net = WarmStartNet(4, 32, stream=stream)
    net.set_params(ws.he_init(net, seed=4))
    ntr = int(0.9 * samples) // 8 * 8
    sync()
    t0 = time.perf_counter()
    hist = net.train(np.stack(masks[:ntr]), targets[:ntr], epochs=epochs, batch=8, lr=1e-3, seed=1)
    t_train = time.perf_counter() - t0
    val_loss = float(np.mean([net.loss_grad(np.stack(masks[j:j + 1]), targets[j:j + 1])[0]
                              for j in range(ntr, samples)]))
    # the network's permeability calibration, fitted on every 4th training box (like c_KC)
    c_net = ws.fit_net_scale(net, boxes[:ntr:4], ks[:ntr:4], TAU, UBAR)
    _, f_step = net_flops(4, 32, side)
    train_flops = f_step * ntr * epochs
    test_mask, _ = sphere_pack(test_side, 8.0, 16.0, 0.35, seed=777)
    Q = UBAR * int((test_mask[0] == 0).sum())
    t0 = time.perf_counter()
    with Lattice(test_mask, TAU, "mrt", "fp32", stream=stream) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        n_test = lat.info()["n_pore"]
        ref = cv.run_to_residual(lat, Q, TAU, lag=1000, tol=1e-6, max_steps=ref_steps, sync=sync)
    t_ref = time.perf_counter() - t0
    abl = ws.ablation(Lattice, net, test_mask, Q, TAU, c_kc, ref["k"], stream=stream, sync=sync,
                      max_steps=ref_steps, variant=variant, c_net=c_net)
    # permeability estimates: the test pack and four more seeded 128^3 packs
    est = []
    for seed, m in [(777, test_mask)] + [(s, sphere_pack(128, 8.0, 16.0, 0.35, seed=s)[0]) for s in (901, 902, 903, 904)]:
        Qm = UBAR * int((m[0] == 0).sum())
        if seed == 777:
            k_true = ref["k"]
        else:
            with Lattice(m, TAU, "mrt", "fp32", stream=stream) as lat:
                lat.set_kernel(variant)
                lat.set_flux_bc(Qm)
                k_true = cv.run_to_residual(lat, Qm, TAU, lag=1000, tol=1e-6, max_steps=ref_steps, sync=sync)["k"]
        k_n = ws.net_permeability(net, m, Qm, TAU, c_net=c_net)
        k_c = c_kc * ws.kc_features(m)[2]
        est.append({"side": m.shape[0], "seed": seed, "k_ref": k_true, "network_rel_err": (k_n - k_true) / k_true,
                    "kozeny_carman_rel_err": (k_c - k_true) / k_true})
    clk = clocks.stop()
    conv = conv_roofline(stream)
    net.close()

    def change(name, base):
        a, b = abl[name], abl[base]
        if not (a["reached"] and b["reached"]):
            return None
        return {"steps": round(a["steps"] / b["steps"] - 1.0, 4), "seconds": round(a["seconds"] / b["seconds"] - 1.0, 4)}

    return {"train": {"network": "U-Net, 4 levels, 32/64/128/256 channels, 15 3x3x3 convolutions, BF16 weights "
                                 "and activations, FP32 accumulate (tcgen05)",
                      "samples": samples, "train_samples": ntr, "side": side,
                      "lbm_box": side + 2 * margin, "lbm_steps": lbm_steps,
                      "epochs": epochs, "batch": 8, "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
                      "val_loss": val_loss, "c_kc": c_kc,
                      "seconds": {"geometry": round(t_geo, 1), "lbm": round(t_lbm, 1), "train": round(t_train, 2)},
                      "train_tflops_algorithmic": round(train_flops / t_train / 1e12, 1)},
            "test": {"side": test_side, "n_pore": n_test, "step_variant": variant, "k_ref": ref["k"],
                     "k_ref_steps": ref["steps"], "k_ref_seconds": round(t_ref, 1), "k_ref_converged": ref["converged"],
                     "criterion": "k within 0.1% of k_ref for 10 consecutive checks (every 100 steps); the time "
                                  "of a warm start includes inference and upload",
                     "starts": abl,
                     "starts_defined": {"cold": "rho 1, u 0", "kc_ramp": "rho: Kozeny-Carman Darcy ramp, u 0 (no "
                                        "network)", "net_velocity": "u: network, rho 1",
                                        "net_pressure": "rho: network pressure profile (calibrated by c_net), u 0",
                                        "net": "u and rho from the network"},
                     "change_vs_cold": {n: change(n, "cold") for n in ("kc_ramp", "net_velocity", "net_pressure",
                                                                       "net")},
                     "net_vs_kc_ramp": change("net", "kc_ramp"),
                     "permeability_estimates": {
                         "packs": est, "c_net": c_net, "c_kc": c_kc,
                         "mean_abs_rel_err": {"network": float(np.mean([abs(e["network_rel_err"]) for e in est])),
                                              "kozeny_carman": float(np.mean([abs(e["kozeny_carman_rel_err"])
                                                                              for e in est]))}}},
            "conv_roofline": conv, "clocks": clk}


def run_warmstart(args):
    """The learned warm-start leg alone (e.g. on a 512^3 test pack)."""
    import torch

    torch.cuda.set_device(0)
    out = {"warmstart": run_warmstart_leg(torch.cuda.current_stream(), args.ws_samples, 64, args.ws_lbm_steps,
                                          args.ws_epochs, args.ws_test, args.variant, args.ws_ref_steps)}
    print(json.dumps(out), flush=True)


def run_profile_case(args):
    """Small, fixed launch sequence for ncu: create the benchmark lattice, W
    single-step warm-up launches, then `steps` steps with per-launch events.
    With --two-fluid-case: the two-fluid pack of the two-fluid leg instead
    (gamma of its Laplace calibration, 0.0102), W + `steps` steps."""
    import torch

    from paper_1806_10589_gb300 import ColorLattice, Lattice, drainage

    torch.cuda.set_device(0)
    if args.conv_case:
        r = conv_roofline(torch.cuda.current_stream(), reps=max(1, args.steps))
        print(json.dumps({"profile_case": "conv", "per_kernel": r["per_kernel"]}))
        return
    if args.ensemble_case:
        from paper_1806_10589_gb300 import Batch

        masks, Qs, _ = ensemble_workload()
        with Batch(masks, TAU, "mrt", "fp16dev", stream=torch.cuda.current_stream()) as b:
            b.set_config(1)  # per-step launches, 48-register cap (the autotuner's usual pick)
            for k, q in enumerate(Qs):
                b.set_flux_bc(k, q)
            for _ in range(args.warmup):
                b.step(1)
            ms = b.time_step(args.steps)
            n = b.info()["n_pore"]
        print(json.dumps({"profile_case": "ensemble fp16dev", "n_pore": n, "step_ms": ms}))
        return
    if args.two_fluid_case:
        mask, info = sphere_pack((192, 192, 384), 5.0, 10.0, 0.35, seed=31, reservoir=6)
        nz, ny, nx = mask.shape
        Q = drainage.simulated_flux(1e-5, info["porosity"], nx * ny, 0.0102, drainage.lattice_viscosity(1.0))
        with ColorLattice(mask, 1.0, 0.01, 0.95, -1.0, "fp32", stream=torch.cuda.current_stream()) as c:
            zz = np.arange(nz)[:, None, None] * np.ones(mask.shape)
            c.set_phase(np.where(zz < 6, 1.0, -1.0))
            c.set_flux_bc(Q, 1.0)
            c.step(args.warmup + args.steps)
            torch.cuda.synchronize()
        print(json.dumps({"profile_case": "two-fluid", "steps": args.warmup + args.steps}))
        return
    mask, info, a_in = workload()
    variant = args.variant
    with Lattice(mask, TAU, "mrt", args.precision, stream=torch.cuda.current_stream()) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(UBAR * a_in)
        for _ in range(args.warmup):
            lat.step(1)
        ms_step, ms_in = lat.time_kernels(args.steps)
        n = lat.info()["n_pore"]
    print(json.dumps({"profile_case": args.precision, "variant": variant, "n_pore": n, "step_ms": ms_step}))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=list(BYTES_PER_VALUE), default="fp32")
    ap.add_argument("--variant", type=int, choices=sorted(VARIANT_NAMES), default=3,
                    help="step kernel (lbm_set_kernel); 3 = AA pattern (one buffer)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--steady", action=argparse.BooleanOptionalAction, default=True,
                    help="also run the time-to-steady-flux comparison (FP32 / FP16 / BF16)")
    ap.add_argument("--ensemble", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the batched 64-member ensemble (FP16 deviation storage)")
    ap.add_argument("--two-fluid", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the two-fluid colour model on a 192x192x384 pack")
    ap.add_argument("--ws-leg", action=argparse.BooleanOptionalAction, default=True,
                    help="also train the warm-start network and run its four-start ablation on a 256^3 pack")
    ap.add_argument("--warmstart", action="store_true",
                    help="run the learned warm-start leg alone instead of the benchmark (see --ws-test)")
    ap.add_argument("--ws-samples", type=int, default=512)
    ap.add_argument("--ws-lbm-steps", type=int, default=8000)
    ap.add_argument("--ws-epochs", type=int, default=40)
    ap.add_argument("--ws-test", type=int, default=256)
    ap.add_argument("--ws-ref-steps", type=int, default=300000)
    ap.add_argument("--two-fluid-case", action="store_true",
                    help="with --profile-case: the two-fluid pack instead of the benchmark lattice")
    ap.add_argument("--conv-case", action="store_true",
                    help="with --profile-case: the network's 32 -> 32 convolution kernels (forward, data and "
                         "weight gradient), --steps launches each")
    ap.add_argument("--ensemble-case", action="store_true",
                    help="with --profile-case: the 64-member FP16-dev ensemble, per-step launches")
    ap.add_argument("--profile-case", action="store_true",
                    help="run the short fixed launch sequence used for ncu captures")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.profile_case:
        run_profile_case(args)
    elif args.warmstart:
        run_warmstart(args)
    elif args.impl == "reference":
        run_reference(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
