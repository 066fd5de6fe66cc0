"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
identical seeded inputs.

Tolerances (written here, derived in the design notes):
  * FP64 storage and arithmetic: max |f_gpu - f_oracle| <= 1e-11 * max |f|
    (FMA contraction and tree-shaped sums only reorder rounding).
  * FP32 (stores d = f - w, FP32 arithmetic): per step each value picks up a few
    ulps of the largest deviation it is formed from, so after N steps
    max |delta f| <= 20 * N * eps32 * max |d|  (d = f - w).
  * FP16/BF16 deviation storage: every store rounds d/w * 2^10 stochastically to
    11 (FP16) or 8 (BF16) significant bits, an error below one unit in the last
    place (2^(1-p) relative, twice the round-to-nearest bound); the bound is
    8 * N * 2^-p * max |d|.
"""
import math

import numpy as np
import pytest

import oracle as O
from lbm_inputs import duct_mask, random_mask, uniform_field, sphere_pack

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


def _lat(mask, tau, model, prec, torch):
    from paper_1806_10589_gb300 import Lattice

    return Lattice(mask, tau, model, prec, stream=torch.cuda.current_stream())


def _f0(mask, seed, amp=0.01):
    return O.W[:, None, None, None] * (1.0 + amp * uniform_field((19,) + mask.shape, seed))


def _run_pair(mask, tau, model, prec, steps, torch, Q=0.002, seed=3, inlet="flux", rho_in=1.0,
              rho_out=1.0, amp=0.01, chunks=None, variant=None):
    f0 = _f0(mask, seed, amp)
    with _lat(mask, tau, model, prec, torch) as lat:
        if variant is not None:
            lat.set_kernel(variant)
        if inlet == "flux":
            lat.set_flux_bc(Q)
        else:
            lat.set_pressure_bc(4, rho_in)
        lat.set_pressure_bc(5, rho_out)
        lat.set_distributions(f0)
        for c in (chunks or [steps]):
            lat.step(c)
        got = lat.distributions()
        flux = lat.get_flux(4)
        fields = lat.fields()
    ref = O.D3Q19Oracle(mask, tau, model, Q=Q, inlet=inlet, rho_in=rho_in, rho_out=rho_out)
    ref.set_distributions(f0)
    ref.step(steps)
    return got, ref, flux, fields


CASES = [  # (nx, ny, nz, p_solid, seed)
    (4, 4, 6, 0.2, 0),
    (5, 7, 9, 0.3, 1),
    (8, 8, 12, 0.35, 2),
    (13, 11, 10, 0.3, 3),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("model", ["mrt", "bgk"])
def test_fp64_random_masks(torch_cuda, case, model):
    nx, ny, nz, p, seed = case
    m = random_mask(nx, ny, nz, p, seed)
    got, ref, (q_in, rho_in), _ = _run_pair(m, 0.8, model, "fp64", 25, torch_cuda, seed=seed + 50)
    err = np.abs(got - ref.f).max() / np.abs(ref.f).max()
    assert err <= 1e-11, err
    assert abs(rho_in - ref.rho_in) <= 1e-12
    A = int((m[0] == 0).sum())
    assert abs(q_in - 0.002) <= 8 * A * np.finfo(float).eps


def test_fp64_ragged_multi_tile(torch_cuda):
    """~15k pore nodes: many 256-thread tiles, a ragged last tile and several
    inlet-reduction blocks (A > 256)."""
    m = random_mask(37, 29, 21, 0.3, 9)
    got, ref, _, _ = _run_pair(m, 0.65, "mrt", "fp64", 12, torch_cuda, seed=91)
    n = int((m == 0).sum())
    assert n % 256 != 0 and int((m[0] == 0).sum()) > 256
    assert np.abs(got - ref.f).max() / np.abs(ref.f).max() <= 1e-11


def test_fp64_graph_path_matches_single_steps(torch_cuda):
    """lbm_step(n >= 64) replays captured graphs; it must give the same bits as
    the same number of single steps, and match the oracle."""
    m = random_mask(6, 5, 8, 0.25, 4)
    a, ref, _, _ = _run_pair(m, 0.9, "mrt", "fp64", 70, torch_cuda, chunks=[70])
    b, _, _, _ = _run_pair(m, 0.9, "mrt", "fp64", 70, torch_cuda, chunks=[1] * 70)
    c, _, _, _ = _run_pair(m, 0.9, "mrt", "fp64", 70, torch_cuda, chunks=[3, 64, 3])
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    assert np.abs(a - ref.f).max() / np.abs(ref.f).max() <= 1e-11


def test_fp64_pressure_inlet(torch_cuda):
    m = duct_mask(7, 6, 10)
    got, ref, (_, rho_bc), _ = _run_pair(m, 1.0, "mrt", "fp64", 20, torch_cuda, inlet="pressure",
                                         rho_in=1.004, rho_out=0.999)
    assert np.abs(got - ref.f).max() / np.abs(ref.f).max() <= 1e-11
    assert abs(rho_bc - 1.004) < 1e-15


@pytest.fixture(scope="module")
def duct16_pair(torch_cuda):
    """The 16x16x64 duct, tau = 1, mean inlet velocity 1e-3 (Q = 0.196), 2000
    steps from rest, FP64 (graph path)."""
    m = duct_mask(16, 16, 64)
    Q = 1e-3 * 196
    with _lat(m, 1.0, "mrt", "fp64", torch_cuda) as lat:
        lat.set_flux_bc(Q)
        lat.step(2000)
        got = lat.distributions()
        fields = lat.fields()
        mon = lat.monitors()
        flux_in = lat.get_flux(4)
        flux_out = lat.get_flux(5)
    ref = O.D3Q19Oracle(m, 1.0, "mrt", Q=Q)
    ref.step(2000)
    return m, Q, got, fields, mon, flux_in, flux_out, ref


def test_duct16_2000_steps_fp64(duct16_pair):
    m, Q, got, fields, mon, (q_in, rho_in), (q_out, rho_out), ref = duct16_pair
    assert np.abs(got - ref.f).max() / np.abs(ref.f).max() <= 1e-11
    rho, ux, uy, uz = fields
    r_rho, r_ux, r_uy, r_uz = ref.fields()
    assert np.abs(uz - r_uz).max() <= 1e-11 * np.abs(r_uz).max()
    assert np.abs(rho - r_rho).max() <= 1e-11
    assert abs(q_in - Q) <= 1e-12
    assert abs(rho_in - ref.rho_in) <= 1e-12
    assert abs(q_out - ref.face_flux(63)) <= 1e-11 * Q
    assert abs(rho_out - 1.0) == 0.0
    assert abs(mon["mass"] - math.fsum(r_rho[m == 0].tolist())) <= 1e-10
    assert mon["status"] == 0


def test_fields_zero_at_solids(duct16_pair):
    m, _, _, fields, _, _, _, _ = duct16_pair
    for a in fields:
        assert np.all(a[m == 1] == 0.0)


def test_fp64_deterministic(torch_cuda):
    m = random_mask(37, 29, 21, 0.3, 19)
    a, _, _, _ = _run_pair(m, 0.7, "mrt", "fp64", 5, torch_cuda, seed=5)
    b, _, _, _ = _run_pair(m, 0.7, "mrt", "fp64", 5, torch_cuda, seed=5)
    np.testing.assert_array_equal(a, b)


def test_set_fields_is_equilibrium(torch_cuda):
    m = random_mask(9, 7, 8, 0.3, 8)
    rng = np.random.default_rng(1)
    rho = 1 + 0.01 * rng.standard_normal(m.shape)
    u = 0.01 * rng.standard_normal((3,) + m.shape)
    with _lat(m, 1.0, "mrt", "fp64", torch_cuda) as lat:
        lat.set_fields(rho, *u)
        got = lat.distributions()
    want = O.equilibrium(rho, u[0], u[1], u[2])
    want[:, m == 1] = 0
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("model", ["mrt", "bgk"])
def test_fp32_parity(torch_cuda, model):
    m = random_mask(13, 11, 10, 0.3, 3)
    N = 25
    got, ref, (q_in, _), _ = _run_pair(m, 0.8, model, "fp32", N, torch_cuda, seed=7)
    d_ref = ref.f - O.W[:, None, None, None] * (m == 0)
    err = np.abs(got - ref.f).max()
    bound = 20 * N * EPS32 * np.abs(d_ref).max()
    assert err <= bound, (err, bound)
    A = int((m[0] == 0).sum())
    assert abs(q_in - 0.002) <= 19 * A * EPS32 * np.abs(d_ref).max() * 4


@pytest.mark.parametrize("prec,bits", [("fp16dev", 11), ("bf16dev", 8)])
def test_16bit_deviation_storage_error(torch_cuda, prec, bits):
    m = random_mask(13, 11, 10, 0.3, 3)
    N = 10
    got, ref, _, _ = _run_pair(m, 0.8, "mrt", prec, N, torch_cuda, seed=7)
    d_ref = ref.f - O.W[:, None, None, None] * (m == 0)
    err = np.abs(got - ref.f).max()
    bound = 8 * N * 2.0 ** -bits * np.abs(d_ref).max()
    assert np.isfinite(got).all()
    assert err <= bound, (err, bound)


@pytest.fixture(scope="module")
def full_pack():
    """The benchmark workload (256^3 sphere pack, radii U[6,12], porosity 0.35, 6
    reservoir layers, tau 0.7, Q = 1e-4 A) from a seeded perturbed state, and the
    oracle's state after 2 steps (computed once for every format and variant)."""
    m, info = sphere_pack(256, 6, 12, 0.35, seed=2024, reservoir=6)
    Q = 1e-4 * int((m[0] == 0).sum())
    N = 2
    f0 = _f0(m, 77, 0.001)
    ref = O.D3Q19Oracle(m, 0.7, "mrt", Q=Q)
    ref.set_distributions(f0)
    ref.step(N)
    return m, Q, N, f0, ref


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp16dev", "bf16dev"])
def test_full_size_sphere_pack_two_steps(torch_cuda, full_pack, prec, variant):
    """The benchmark's workload at full size, every cell against the oracle after
    2 steps, in every storage format the benchmark reports, on the AA pattern
    the benchmark times (variant 3: layout swap, one gather-scatter and one
    node-local launch, swap back) and on the two-buffer kernel (variant 0), at
    the stated bounds: FP32 20 N eps32 max|d|, FP16 / BF16 8 N 2^-p max|d|."""
    m, Q, N, f0, ref = full_pack
    with _lat(m, 0.7, "mrt", prec, torch_cuda) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        lat.set_distributions(f0)
        lat.step(N)
        got = lat.distributions()
    dmax = float(np.abs(ref.f - O.W[:, None, None, None] * (m == 0)).max())
    err = float(np.abs(got - ref.f).max())
    if prec == "fp32":
        bound = 20 * N * EPS32 * dmax + 4 * EPS32 * 1e-2
    else:
        bound = 8 * N * 2.0 ** -(11 if prec == "fp16dev" else 8) * dmax
    assert np.isfinite(got).all()
    assert err <= bound, (prec, variant, err, bound)


def test_steady_residual_matches_oracle(torch_cuda):
    """lbm_steady_residual against Eq. (stopping_criterion) of the oracle's fields
    over the same lag, FP64."""
    m = duct_mask(8, 7, 16)
    Q = 0.01
    with _lat(m, 0.9, "mrt", "fp64", torch_cuda) as lat:
        lat.set_flux_bc(Q)
        lat.step(40)
        assert lat.steady_residual() == float("inf")
        lat.step(25)
        r_gpu = lat.steady_residual()
    ref = O.D3Q19Oracle(m, 0.9, "mrt", Q=Q)
    ref.step(40)
    _, ux0, uy0, uz0 = ref.fields()
    ref.step(25)
    _, ux1, uy1, uz1 = ref.fields()
    r_ref = O.steady_residual(np.stack([ux1, uy1, uz1]), np.stack([ux0, uy0, uz0]), m == 0)
    assert abs(r_gpu - r_ref) <= 1e-11 * r_ref


def test_convergence_harness_small_duct(torch_cuda):
    """The time-to-steady harness on a small duct: the Section 3.1 rule converges,
    and a second cold run reaches 0.1 % of its permeability and outlet flux."""
    from paper_1806_10589_gb300 import convergence as cv

    m = duct_mask(10, 10, 24)
    Q = 1e-3 * 64
    with _lat(m, 1.0, "mrt", "fp32", torch_cuda) as lat:
        lat.set_flux_bc(Q)
        ref = cv.run_to_residual(lat, Q, 1.0, lag=200, tol=1e-6, max_steps=20000)
    assert ref["converged"] and abs(ref["q_out"] - Q) < 1e-4 * Q
    with _lat(m, 1.0, "mrt", "fp32", torch_cuda) as lat:
        lat.set_flux_bc(Q)
        r = cv.run_to_reference(lat, Q, 1.0, ref["k"], check_every=20, max_steps=20000, require_q_out=True)
    assert r["reached"] and r["steps"] < ref["steps"]


def _run_variant(mask, tau, prec, steps, variant, torch, Q=0.002, seed=3, amp=0.01):
    f0 = _f0(mask, seed, amp)
    with _lat(mask, tau, "mrt", prec, torch) as lat:
        lat.set_kernel(variant)
        lat.set_flux_bc(Q)
        lat.set_distributions(f0)
        lat.step(steps)
        got = lat.distributions()
        q_in, rho_in = lat.get_flux(4)
    return f0, got, q_in, rho_in


@pytest.fixture(scope="module")
def big_random_case():
    """96x96x64 random pore space (~400k nodes: >1500 tiles of 256, so every
    block of the persistent kernels walks several tiles), 70 steps in FP64 with
    the oracle (exercises graphs, the pipelined prologue/steady state/tail)."""
    m = random_mask(96, 96, 64, 0.3, 123)
    f0 = _f0(m, 124)
    ref = O.D3Q19Oracle(m, 0.75, "mrt", Q=0.05)
    ref.set_distributions(f0)
    ref.step(70)
    return m, ref


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_step_variants_fp64_multi_tile(torch_cuda, big_random_case, variant):
    m, ref = big_random_case
    _, got, q_in, rho_in = _run_variant(m, 0.75, "fp64", 70, variant, torch_cuda, Q=0.05, seed=124)
    assert np.abs(got - ref.f).max() / np.abs(ref.f).max() <= 1e-11
    assert abs(rho_in - ref.rho_in) <= 1e-12
    A = int((m[0] == 0).sum())
    assert abs(q_in - 0.05) <= 8 * A * np.finfo(float).eps


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("prec,bound_bits", [("fp32", None), ("fp16dev", 11), ("bf16dev", 8)])
def test_step_variants_reduced_precision(torch_cuda, variant, prec, bound_bits):
    m = random_mask(37, 29, 21, 0.3, 9)
    N = 10
    f0, got, _, _ = _run_variant(m, 0.8, prec, N, variant, torch_cuda, seed=7)
    ref = O.D3Q19Oracle(m, 0.8, "mrt", Q=0.002)
    ref.set_distributions(f0)
    ref.step(N)
    d_ref = ref.f - O.W[:, None, None, None] * (m == 0)
    err = np.abs(got - ref.f).max()
    if bound_bits is None:
        bound = 20 * N * EPS32 * np.abs(d_ref).max()
    else:
        bound = 8 * N * 2.0 ** -bound_bits * np.abs(d_ref).max()
    assert err <= bound, (err, bound)


def test_step_variants_agree_bitwise_on_interior(torch_cuda):
    """Variants differ only in the order of the fused FP64 inlet sum, so after
    one step from the same state every stored value agrees bit for bit."""
    m = random_mask(37, 29, 21, 0.3, 10)
    outs = [_run_variant(m, 0.8, "fp32", 1, v, torch_cuda, seed=11)[1] for v in (0, 1, 2)]
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_16bit_reference_refresh_keeps_state_and_flux(torch_cuda, prec):
    """Crossing a reference-profile refresh (every 1024 steps) of the 16-bit
    formats: the flux through the inlet stays exact to the storage rounding and
    the state stays close to the FP32 run of the same problem."""
    m = duct_mask(10, 9, 40)
    Q = 2e-3 * int((m[0] == 0).sum())
    res = {}
    for p in ("fp32", prec):
        with _lat(m, 0.8, "mrt", p, torch_cuda) as lat:
            lat.set_flux_bc(Q)
            lat.step(1100)
            q_in, rho_in = lat.get_flux(4)
            res[p] = (lat.fields(), q_in, rho_in)
    (rho32, _, _, uz32), _, rin32 = res["fp32"]
    (rho16, _, _, uz16), q16, rin16 = res[prec]
    bits = 11 if prec == "fp16dev" else 8
    dmax = float(np.abs(rho32[m == 0] - 1).max())
    assert abs(q16 - Q) <= 64 * 2.0 ** -bits * dmax * int((m[0] == 0).sum()) / 19
    assert np.abs(uz16 - uz32).max() <= 0.2 * np.abs(uz32).max() * (2.0 ** (11 - bits))
    assert abs(rin16 - rin32) <= 0.05 * abs(rin32 - 1)


@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_16bit_stochastic_rounding_is_reproducible(torch_cuda, prec):
    """The rounding bits come from a counter-based hash of (step seed, node,
    direction): two identical runs give identical states, and changing only the
    step count changes them."""
    m = random_mask(17, 13, 15, 0.3, 4)
    a = _run_variant(m, 0.8, prec, 70, 0, torch_cuda, seed=5)[1]
    b = _run_variant(m, 0.8, prec, 70, 0, torch_cuda, seed=5)[1]
    np.testing.assert_array_equal(a, b)
