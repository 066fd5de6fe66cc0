"""GPU parity of the batched ensemble (lbm_batch_*): every member of one launch
against the FP64 oracle run alone on that member, and against the
single-lattice path."""
import numpy as np
import pytest

import oracle as O
from lbm_inputs import duct_mask, random_mask, uniform_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    return torch


def _members():
    """Uneven members: tiny, ragged, a duct, and one with > 1 inlet tile."""
    return [random_mask(5, 4, 6, 0.25, 1), random_mask(13, 11, 10, 0.3, 2), duct_mask(8, 9, 14),
            random_mask(31, 27, 9, 0.3, 3)]


def _f0(m, seed):
    return O.W[:, None, None, None] * (1.0 + 0.01 * uniform_field((19,) + m.shape, seed))


@pytest.mark.parametrize("steps", [5, 70])
def test_batch_fp64_members_match_oracle(torch_cuda, steps):
    from paper_1806_10589_gb300 import Batch

    masks = _members()
    Qs = [0.001, 0.004, 0.02, 0.03]
    with Batch(masks, 0.8, "mrt", "fp64", stream=torch_cuda.cuda.current_stream()) as b:
        for k, m in enumerate(masks):
            b.set_flux_bc(k, Qs[k])
            b.set_distributions(k, _f0(m, 10 + k))
        b.step(steps)
        got = [b.distributions(k) for k in range(len(masks))]
        flux = [b.get_flux(k, 4) for k in range(len(masks))]
    for k, m in enumerate(masks):
        ref = O.D3Q19Oracle(m, 0.8, "mrt", Q=Qs[k])
        ref.set_distributions(_f0(m, 10 + k))
        ref.step(steps)
        assert np.abs(got[k] - ref.f).max() / np.abs(ref.f).max() <= 1e-11, k
        A = int((m[0] == 0).sum())
        assert abs(flux[k][0] - Qs[k]) <= 8 * A * np.finfo(float).eps, k
        assert abs(flux[k][1] - ref.rho_in) <= 1e-12, k


def test_batch_member_equals_single_lattice_fp32(torch_cuda):
    """Same tiling of the fused reduction, same per-node arithmetic: a member
    of the batch and the same problem on its own agree bit for bit."""
    from paper_1806_10589_gb300 import Batch, Lattice

    masks = _members()
    st = torch_cuda.cuda.current_stream()
    with Batch(masks, 0.7, "mrt", "fp32", stream=st) as b:
        for k, m in enumerate(masks):
            b.set_flux_bc(k, 0.002 * (k + 1))
            b.set_distributions(k, _f0(m, 20 + k))
        b.step(67)
        got = [b.distributions(k) for k in range(len(masks))]
    for k, m in enumerate(masks):
        with Lattice(m, 0.7, "mrt", "fp32", stream=st) as lat:
            lat.set_kernel(0)
            lat.set_flux_bc(0.002 * (k + 1))
            lat.set_distributions(_f0(m, 20 + k))
            lat.step(67)
            np.testing.assert_array_equal(got[k], lat.distributions())


def test_batch_rejects_bad_members(torch_cuda):
    from paper_1806_10589_gb300 import Batch, LBMError

    bad = duct_mask(6, 6, 8)
    bad[0] = 1
    with pytest.raises(LBMError):
        Batch([duct_mask(6, 6, 8), bad], 1.0)


def _run_cfg(masks, prec, config, steps, torch, Qs=(0.001, 0.004, 0.02, 0.03)):
    from paper_1806_10589_gb300 import Batch

    with Batch(masks, 0.8, "mrt", prec, stream=torch.cuda.current_stream()) as b:
        b.set_config(config)
        for k, m in enumerate(masks):
            b.set_flux_bc(k, Qs[k])
            b.set_distributions(k, _f0(m, 10 + k))
        b.step(steps)
        return [b.distributions(k) for k in range(len(masks))], [b.get_flux(k, 4) for k in range(len(masks))]


@pytest.mark.parametrize("config", [1, 2, 3, 4, 5])
def test_batch_configs_fp64_match_oracle(torch_cuda, config):
    """Every launch configuration (per-step launches with the 48-register cap,
    one persistent launch with either cap, the AA pattern with either cap)
    against the oracle, 70 steps: the persistent launch carries all of them,
    with a grid barrier between steps; the AA pattern runs a 64-step graph and
    six single steps."""
    masks = _members()
    Qs = [0.001, 0.004, 0.02, 0.03]
    got, flux = _run_cfg(masks, "fp64", config, 70, torch_cuda)
    for k, m in enumerate(masks):
        ref = O.D3Q19Oracle(m, 0.8, "mrt", Q=Qs[k])
        ref.set_distributions(_f0(m, 10 + k))
        ref.step(70)
        assert np.abs(got[k] - ref.f).max() / np.abs(ref.f).max() <= 1e-11, k
        assert abs(flux[k][1] - ref.rho_in) <= 1e-12, k


@pytest.mark.parametrize("prec", ["fp32", "fp16dev"])
def test_batch_configs_agree(torch_cuda, prec):
    """The configurations compute the same steps.

    Pull forms (configs 1-3 against 0): the same per-node arithmetic, only the
    register cap and the launch form differ, so the compiler may contract a
    product into an FMA differently: each stored value can differ by one
    rounding, eps32 (FP32) of the largest deviation d = f - w, and nothing
    accumulates because every form rounds the same way after that; the bound
    allows 4 eps32 max|d| (FP32) and one FP16 storage unit 2^-9 max|d|
    (2^-10 relative spacing, times 2 for the stochastic rounding).

    AA pattern (configs 4-5): the per-node arithmetic is ordered differently
    (gather-scatter and node-local launches), so each step may round each value
    differently by up to eps32 max|d|.  The collision relaxes every
    non-conserved part by a factor |1 - s| < 1 (rates in (0, 2)), so an earlier
    difference does not grow: after N steps |delta| <= N eps32 max|d|, N = 70
    here.  In 16 bits the AA pattern also encodes a scattered value with its
    destination's plane reference, a different stochastic rounding each step:
    the storage bound of the parity tests, 8 N 2^-11 max|d|."""
    masks = _members()
    ref, _ = _run_cfg(masks, prec, 0, 70, torch_cuda)
    for config in (1, 2, 3, 4, 5):
        got, _ = _run_cfg(masks, prec, config, 70, torch_cuda)
        for k, m in enumerate(masks):
            dev = np.abs(ref[k] - O.W[:, None, None, None] * (m == 0)).max()
            if config >= 4:
                tol = (70 * np.finfo(np.float32).eps if prec == "fp32" else 8 * 70 * 2.0 ** -11) * dev
            else:
                tol = (4 * np.finfo(np.float32).eps if prec == "fp32" else 2.0 ** -9) * dev
            assert np.abs(got[k] - ref[k]).max() <= tol, (config, k)


@pytest.mark.parametrize("prec", ["fp64", "fp16dev"])
@pytest.mark.parametrize("config", [0, 1])
def test_batch_32bit_offsets_equal_64bit_addresses(torch_cuda, prec, config, monkeypatch):
    """The per-step launches address a pulled value as the buffer plus a 32-bit
    element offset when the buffers have fewer than 2^32 elements, else as one
    of two 64-bit addresses; both forms give bitwise the same states (the
    64-bit form is forced by GB300_LBM_BATCH_ADDR64)."""
    masks = _members()
    a = _run_cfg(masks, prec, config, 70, torch_cuda)
    monkeypatch.setenv("GB300_LBM_BATCH_ADDR64", "1")
    b = _run_cfg(masks, prec, config, 70, torch_cuda)
    for fa, fb in zip(a[0], b[0]):
        np.testing.assert_array_equal(fa, fb)
    assert a[1] == b[1]


def test_batch_autotune_keeps_state_and_picks_a_config(torch_cuda):
    from paper_1806_10589_gb300 import Batch

    masks = _members()
    with Batch(masks, 0.8, "mrt", "fp32", stream=torch_cuda.cuda.current_stream()) as b:
        for k, m in enumerate(masks):
            b.set_flux_bc(k, 0.01)
            b.set_distributions(k, _f0(m, 10 + k))
        b.step(5)
        before = [b.distributions(k) for k in range(len(masks))]
        rho_before = [b.get_flux(k, 4)[1] for k in range(len(masks))]
        steps_before = b.info()["steps"]
        best, ms = b.autotune(70)
        assert best in range(6) and len(ms) == 6 and all(t > 0 for t in ms)
        assert ms[best] == min(ms)
        for k in range(len(masks)):
            np.testing.assert_array_equal(b.distributions(k), before[k])
            assert b.get_flux(k, 4)[1] == rho_before[k]
        assert b.info()["steps"] == steps_before
        b.step(30)
        after = [b.distributions(k) for k in range(len(masks))]
    with Batch(masks, 0.8, "mrt", "fp32", stream=torch_cuda.cuda.current_stream()) as c:
        for k, m in enumerate(masks):
            c.set_flux_bc(k, 0.01)
            c.set_distributions(k, _f0(m, 10 + k))
        c.step(35)
        for k, m in enumerate(masks):
            dev = np.abs(after[k] - O.W[:, None, None, None] * (m == 0)).max()
            # the chosen configuration may be the AA pattern: up to one FP32 rounding of
            # max|d| per step, not amplified by the collision (test_batch_configs_agree),
            # over the 35 steps
            assert np.abs(c.distributions(k) - after[k]).max() <= 35 * np.finfo(np.float32).eps * dev, k


def test_batch_barrier_wait_is_bounded(torch_cuda):
    """The persistent launch's grid barrier completes when every block arrives,
    and reports (instead of hanging) when one never does; the ensemble keeps
    working afterwards."""
    from paper_1806_10589_gb300 import Batch

    masks = _members()
    with Batch(masks, 0.8, "mrt", "fp32", stream=torch_cuda.cuda.current_stream()) as b:
        completes, times_out = b.check_barrier(20.0)
        assert completes and times_out
        b.set_config(2)
        b.set_flux_bc(0, 0.001)
        b.step(10)
        assert np.isfinite(b.distributions(0)).all()


@pytest.mark.parametrize("config", [2, 4])
@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_batch_segments_cross_reference_refresh(torch_cuda, prec, config):
    """1100 steps in persistent launches, or AA calls, split at the 16-bit
    reference refresh (every 1024 steps) agree with the per-step launches to the
    storage rounding."""
    masks = _members()[:3]
    ref, fr = _run_cfg(masks, prec, 0, 1100, torch_cuda, Qs=(0.001, 0.004, 0.02))
    got, fg = _run_cfg(masks, prec, config, 1100, torch_cuda, Qs=(0.001, 0.004, 0.02))
    bits = 11 if prec == "fp16dev" else 8
    for k, m in enumerate(masks):
        dev = np.abs(ref[k] - O.W[:, None, None, None] * (m == 0)).max()
        assert np.abs(got[k] - ref[k]).max() <= 2.0 ** (2 - bits) * dev, k
        assert abs(fg[k][1] - fr[k][1]) <= 0.05 * abs(fr[k][1] - 1), k
