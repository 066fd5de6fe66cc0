"""GPU checks of the AA-pattern variant (lbm_set_kernel 3: one distribution
buffer updated in place).

* Parity: FP64 against the oracle (1e-11 relative, as the two-buffer path) for
  even and odd step counts, graph-sized and ragged runs, both collision models.
* Equivalence: FP32 and FP64 states and inlet densities equal those of the
  two-buffer per-node kernel to rounding.  The formulas are the same, but the
  compiler contracts some products into FMAs differently in the two kernels, so
  a step can differ by an ulp of the largest deviation, and such differences
  propagate like rounding errors: max|delta| <= N eps max|d| after N steps.
* Memory: entering the AA pattern releases the second buffer; leaving it
  allocates it again, mid-run, without changing the trajectory.
* 16-bit deviation storage on the AA pattern: oracle bound and a crossing of
  the reference-profile refresh.
* Calls: the buffer stays in the in-place layout between lbm_step calls, so a
  run split into calls equals one call bit for bit; reads in between swap it back.
"""
import numpy as np
import pytest

import oracle as O
from lbm_inputs import random_mask, sphere_pack, uniform_field

pytestmark = pytest.mark.gpu
EPS32 = float(np.finfo(np.float32).eps)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    return torch


def _f0(mask, seed, amp=0.01):
    return O.W[:, None, None, None] * (1.0 + amp * uniform_field((19,) + mask.shape, seed))


def _run(mask, prec, variant, chunks, torch, tau=0.8, model="mrt", Q=0.002, seed=5):
    from paper_1806_10589_gb300 import Lattice

    with Lattice(mask, tau, model, prec, stream=torch.cuda.current_stream()) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        lat.set_distributions(_f0(mask, seed))
        for c in chunks:
            lat.step(c)
        return lat.distributions(), lat.get_flux(4), lat.get_flux(5)


@pytest.mark.parametrize("steps", [1, 2, 15, 16])
@pytest.mark.parametrize("model", ["mrt", "bgk"])
def test_aa_fp64_matches_oracle(torch_cuda, steps, model):
    m = random_mask(9, 8, 12, 0.3, 21)
    got, (q_in, rho_in), _ = _run(m, "fp64", 3, [steps], torch_cuda, model=model)
    ref = O.D3Q19Oracle(m, 0.8, model, Q=0.002)
    ref.set_distributions(_f0(m, 5))
    ref.step(steps)
    assert np.abs(got - ref.f).max() <= 1e-11 * np.abs(ref.f).max()
    assert abs(rho_in - ref.rho_in) <= 1e-12
    assert abs(q_in - 0.002) <= 8 * int((m[0] == 0).sum()) * np.finfo(float).eps


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("chunks", [[130], [1, 64, 3], [65, 65]])
def test_aa_equals_two_buffer_kernel(torch_cuda, prec, chunks):
    """Graph-sized (64) and ragged chunks, odd and even call lengths."""
    m = random_mask(37, 29, 21, 0.3, 8)
    a, fa_in, fa_out = _run(m, prec, 0, chunks, torch_cuda)
    b, fb_in, fb_out = _run(m, prec, 3, chunks, torch_cuda)
    d = np.abs(a - b).max()
    dev = np.abs(a - O.W[:, None, None, None] * (m == 0)).max()
    N = sum(chunks)
    tol = (N * EPS32 * dev) if prec == "fp32" else 1e-14 * np.abs(a).max()
    assert d <= tol, (d, "bit-equal" if d == 0 else "not bit-equal")
    assert abs(fa_in[1] - fb_in[1]) <= (1e-6 if prec == "fp32" else 1e-13)
    assert abs(fa_in[0] - fb_in[0]) <= (1e-6 if prec == "fp32" else 1e-13)
    assert abs(fa_out[0] - fb_out[0]) <= (1e-6 if prec == "fp32" else 1e-13)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("variant, switch", [(3, "GB300_LBM_AA_ADDR64"), (0, "GB300_LBM_STEP_ADDR64")])
def test_32bit_offsets_equal_64bit_addresses(torch_cuda, prec, variant, switch, monkeypatch):
    """The gather-scatter AA launch and the two-buffer step address their
    neighbours as row 0 plus a 32-bit element offset whenever the buffer has
    fewer than 2^32 elements; the 64-bit form (two row pointers) serves larger
    lattices.  Both compute the same step, so the states are bitwise equal (the
    64-bit form is forced by an environment switch; graphs are captured per
    lattice, after it is set)."""
    m = random_mask(37, 29, 21, 0.3, 8)
    chunks = [1, 64, 3]
    a = _run(m, prec, variant, chunks, torch_cuda)
    monkeypatch.setenv(switch, "1")
    b = _run(m, prec, variant, chunks, torch_cuda)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[1] == b[1] and a[2] == b[2]


def test_aa_switching_mid_run_releases_and_restores_memory(torch_cuda):
    from paper_1806_10589_gb300 import Lattice

    torch = torch_cuda
    m, _ = sphere_pack(96, 6.0, 10.0, 0.4, seed=77, cache=False)
    ref, _, _ = _run(m, "fp32", 0, [40], torch)
    with Lattice(m, 0.8, "mrt", "fp32", stream=torch.cuda.current_stream()) as lat:
        lat.set_flux_bc(0.002)
        lat.set_distributions(_f0(m, 5))
        n = lat.info()["n_pore"]
        buf = 19 * ((n + 127) // 128 * 128) * 4
        lat.step(7)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        lat.set_kernel(3)
        free1 = torch.cuda.mem_get_info()[0]
        lat.step(21)
        lat.set_kernel(0)
        free2 = torch.cuda.mem_get_info()[0]
        lat.step(12)
        got = lat.distributions()
    assert free1 - free0 >= buf - (2 << 20), (free0, free1, buf)
    assert free1 - free2 >= buf - (2 << 20), (free1, free2, buf)
    dev = np.abs(ref - O.W[:, None, None, None] * (m == 0)).max()
    assert np.abs(got - ref).max() <= 40 * EPS32 * dev


@pytest.mark.parametrize("prec", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("chunks,whole", [([5, 71], 76), ([1, 64, 2, 1], 68), ([700, 401], 1101)])
def test_aa_calls_continue_in_place(torch_cuda, prec, chunks, whole):
    """Between lbm_step calls the AA buffer stays in its in-place layout and the
    next call continues the alternation of gather-scatter and node-local launches
    (graphs for either starting launch), so splitting a run into calls gives
    bitwise the state, fluxes and inlet density of one call, in every format
    (the 16-bit reference refresh falls on the same step either way)."""
    m = random_mask(13, 11, 10, 0.3, 3)
    a, a_in, a_out = _run(m, prec, 3, chunks, torch_cuda, seed=9)
    b, b_in, b_out = _run(m, prec, 3, [whole], torch_cuda, seed=9)
    assert np.array_equal(a, b), np.abs(a - b).max()
    assert a_in == b_in and a_out == b_out


@pytest.mark.parametrize("steps", [7, 8])
def test_aa_reads_between_calls(torch_cuda, steps):
    """A read between calls swaps the buffer back (with the un-stream after an
    odd step count) and the next call swaps it in again; the layout-changing
    calls in between (monitors, flux, time_kernels) leave the trajectory equal to
    the two-buffer kernel's to FP32 rounding, N eps max|d| after N steps, and the
    FP64 run equal to the oracle."""
    from paper_1806_10589_gb300 import Lattice

    m = random_mask(37, 29, 21, 0.3, 8)
    out = {}
    for prec, v in (("fp32", 0), ("fp32", 3), ("fp64", 3)):
        with Lattice(m, 0.8, "mrt", prec, stream=torch_cuda.cuda.current_stream()) as lat:
            lat.set_kernel(v)
            lat.set_flux_bc(0.002)
            lat.set_distributions(_f0(m, 5))
            lat.step(steps)
            lat.monitors()
            lat.step(steps)
            lat.get_flux(4)
            lat.time_kernels(3)
            lat.step(steps + 1)
            out[(prec, v)] = lat.distributions()
    N = 3 * steps + 4
    a, b = out[("fp32", 0)], out[("fp32", 3)]
    dev = np.abs(a - O.W[:, None, None, None] * (m == 0)).max()
    assert np.abs(a - b).max() <= N * EPS32 * dev
    ref = O.D3Q19Oracle(m, 0.8, "mrt", Q=0.002)
    ref.set_distributions(_f0(m, 5))
    ref.step(N)
    assert np.abs(out[("fp64", 3)] - ref.f).max() <= 1e-11 * np.abs(ref.f).max()


@pytest.mark.parametrize("prec,bits", [("fp16dev", 11), ("bf16dev", 8)])
@pytest.mark.parametrize("chunks", [[10], [3, 4]])
def test_aa_16bit_matches_oracle(torch_cuda, prec, bits, chunks):
    """16-bit deviation storage on the AA pattern (scattered values encoded with
    the destination plane's reference; an odd call re-encodes in the un-stream
    swap): within the stochastic-rounding bound of the two-buffer path,
    8 N 2^-p max|d| after N steps."""
    m = random_mask(13, 11, 10, 0.3, 3)
    N = sum(chunks)
    got, _, _ = _run(m, prec, 3, chunks, torch_cuda, seed=7)
    ref = O.D3Q19Oracle(m, 0.8, "mrt", Q=0.002)
    ref.set_distributions(_f0(m, 7))
    ref.step(N)
    d_ref = ref.f - O.W[:, None, None, None] * (m == 0)
    assert np.isfinite(got).all()
    assert np.abs(got - ref.f).max() <= 8 * N * 2.0 ** -bits * np.abs(d_ref).max()


@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_aa_16bit_crosses_reference_refresh(torch_cuda, prec):
    """1100 steps on the AA pattern cross a refresh of the 16-bit reference
    profile (every 1024 steps, done between segments in the resting layout):
    the flux stays exact to the storage rounding and the state stays close to
    the FP32 run, as for the two-buffer path."""
    from paper_1806_10589_gb300 import Lattice
    from lbm_inputs import duct_mask

    m = duct_mask(10, 9, 40)
    Q = 2e-3 * int((m[0] == 0).sum())
    res = {}
    for p, v in (("fp32", 0), (prec, 3)):
        with Lattice(m, 0.8, "mrt", p, stream=torch_cuda.cuda.current_stream()) as lat:
            lat.set_kernel(v)
            lat.set_flux_bc(Q)
            lat.step(700)
            lat.step(401)
            q_in, rho_in = lat.get_flux(4)
            res[p] = (lat.fields(), q_in, rho_in)
    (rho32, _, _, uz32), _, rin32 = res["fp32"]
    (rho16, _, _, uz16), q16, rin16 = res[prec]
    bits = 11 if prec == "fp16dev" else 8
    dmax = float(np.abs(rho32[m == 0] - 1).max())
    assert abs(q16 - Q) <= 64 * 2.0 ** -bits * dmax * int((m[0] == 0).sum()) / 19
    assert np.abs(uz16 - uz32).max() <= 0.2 * np.abs(uz32).max() * (2.0 ** (11 - bits))
    assert abs(rin16 - rin32) <= 0.05 * abs(rin32 - 1)


def test_aa_fp32_steady_duct_matches_poiseuille_series(torch_cuda):
    """Section 3.1 on the benchmark's step: the 16x16x64 duct (tau = 1, mean inlet
    velocity 1e-3) run on the AA pattern in FP32 until the Section 3.1 residual
    is below 1e-6; the mid-plane profile matches the square-duct series with the
    measured gradient (relative L2 error below 0.5 %, as the oracle at 2000
    steps), and the flux through the mid-plane and the outlet equals Q to 0.1 %."""
    import math

    from paper_1806_10589_gb300 import Lattice, convergence as cv
    from lbm_inputs import duct_mask

    n, nz, tau = 16, 64, 1.0
    m = duct_mask(n, n, nz)
    Q = 1e-3 * (n - 2) ** 2
    with Lattice(m, tau, "mrt", "fp32", stream=torch_cuda.cuda.current_stream()) as lat:
        lat.set_kernel(3)
        lat.set_flux_bc(Q)
        r = cv.run_to_residual(lat, Q, tau, lag=500, tol=1e-6, max_steps=30000)
        rho, ux, uy, uz = lat.fields()
        q_out, _ = lat.get_flux(5)
    assert r["converged"], r["residual"]
    zs = np.arange(nz // 4, 3 * nz // 4)
    rbar = np.array([rho[z][m[z] == 0].mean() for z in zs])
    dpdz = O.CS2 * np.polyfit(zs, rbar, 1)[0]
    c = np.arange(1, n - 1) - (n - 1) / 2.0
    X, Y = np.meshgrid(c, c, indexing="xy")
    th = O.duct_velocity(X, Y, (n - 2) / 2.0, O.CS2 * (tau - 0.5), dpdz)
    sim = uz[nz // 2, 1:n - 1, 1:n - 1]
    err = math.sqrt(((sim - th) ** 2).sum() / (th ** 2).sum())
    assert err < 5e-3, err
    assert abs(sim.sum() - Q) < 1e-3 * Q
    assert abs(q_out - Q) < 1e-3 * Q

