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
