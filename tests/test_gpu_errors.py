"""Error paths of the C ABI (every call returns a status and never aborts) and
degenerate geometries: a single pore column and a minimal box, on both step
kernels, against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from lbm_inputs import duct_mask, random_mask, uniform_field

pytestmark = pytest.mark.gpu
EINVAL, EUNSUPPORTED, EUNSTABLE = -1, -4, -5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    return torch


def _status(fn):
    from paper_1806_10589_gb300 import LBMError

    with pytest.raises(LBMError) as ei:
        fn()
    return ei.value.status


def test_create_rejects_bad_arguments(torch_cuda):
    from paper_1806_10589_gb300 import Lattice

    st = torch_cuda.cuda.current_stream()
    m = duct_mask(6, 6, 8)
    closed_inlet = m.copy()
    closed_inlet[0] = 1
    bad_values = m.copy()
    bad_values[3, 3, 3] = 2
    assert _status(lambda: Lattice(closed_inlet, 0.8, "mrt", "fp32", stream=st)) == EINVAL
    assert _status(lambda: Lattice(m, 0.5, "mrt", "fp32", stream=st)) == EINVAL
    assert _status(lambda: Lattice(bad_values, 0.8, "mrt", "fp32", stream=st)) == EINVAL
    assert _status(lambda: Lattice(np.zeros((2, 4, 4), np.uint8), 0.8, "mrt", "fp32", stream=st)) == EINVAL


def test_calls_reject_bad_arguments_and_stay_usable(torch_cuda):
    from paper_1806_10589_gb300 import Lattice

    m = duct_mask(6, 6, 8)
    with Lattice(m, 0.8, "mrt", "fp32", stream=torch_cuda.cuda.current_stream()) as lat:
        assert _status(lambda: lat.set_flux_bc(1e-3, face=5)) == EUNSUPPORTED  # flux only at the inlet
        assert _status(lambda: lat.set_flux_bc(float("nan"))) == EINVAL
        assert _status(lambda: lat.set_pressure_bc(5, -1.0)) == EINVAL
        assert _status(lambda: lat.set_kernel(7)) == EINVAL
        assert _status(lambda: lat.step(-1)) == EINVAL
        lat.set_flux_bc(1e-3)
        lat.step(5)
        q_in, _ = lat.get_flux(4)
        assert abs(q_in - 1e-3) < 1e-9


def test_monitors_report_an_unstable_state(torch_cuda):
    from paper_1806_10589_gb300 import Lattice

    m = duct_mask(6, 6, 8)
    with Lattice(m, 0.8, "mrt", "fp64", stream=torch_cuda.cuda.current_stream()) as lat:
        uz = np.where(m == 0, 0.3, 0.0)  # |u| above the 0.1 stability limit
        lat.set_fields(uz=uz)
        assert _status(lambda: lat.monitors()) == EUNSTABLE
        mon = lat.monitors(raise_unstable=False)
        assert mon["u_max"] > 0.1


def test_other_contexts_reject_bad_arguments(torch_cuda):
    from paper_1806_10589_gb300 import Batch, ColorLattice

    st = torch_cuda.cuda.current_stream()
    m = duct_mask(6, 6, 8)
    assert _status(lambda: ColorLattice(m, 1.0, 0.01, 1.5, -1.0, "fp32", stream=st)) == EINVAL  # beta > 1
    with ColorLattice(m, 1.0, 0.01, 0.95, -1.0, "fp32", stream=st) as c:
        assert _status(lambda: c.set_phase(np.full(m.shape, 2.0))) == EINVAL
    with Batch([m, duct_mask(5, 7, 9)], 0.8, "mrt", "fp32", stream=st) as b:
        assert _status(lambda: b.set_config(9)) == EINVAL
        assert _status(lambda: b.autotune(0)) == EINVAL
        assert _status(lambda: b.check_barrier(0.0)) == EINVAL
        assert _status(lambda: b.set_flux_bc(2, 1e-3)) == EINVAL  # no member 2
        b.step(3)


@pytest.mark.parametrize("variant", [0, 3])
@pytest.mark.parametrize("shape", [(1, 1, 8), (2, 1, 3), (1, 3, 5)])
def test_degenerate_geometries_match_oracle(torch_cuda, variant, shape):
    """A single pore column (every lateral neighbour outside the box), a minimal
    2x1x3 box, and a 1-wide slab: FP64 against the oracle, odd and even step
    counts."""
    from paper_1806_10589_gb300 import Lattice

    nx, ny, nz = shape
    m = np.zeros((nz, ny, nx), np.uint8)
    f0 = O.W[:, None, None, None] * (1.0 + 0.01 * uniform_field((19,) + m.shape, 3))
    Q = 1e-3 * nx * ny
    for steps in (3, 4):
        with Lattice(m, 0.9, "mrt", "fp64", stream=torch_cuda.cuda.current_stream()) as lat:
            lat.set_kernel(variant)
            lat.set_flux_bc(Q)
            lat.set_distributions(f0)
            lat.step(steps)
            got = lat.distributions()
            q_in, _ = lat.get_flux(4)
        ref = O.D3Q19Oracle(m, 0.9, "mrt", Q=Q)
        ref.set_distributions(f0)
        ref.step(steps)
        assert np.abs(got - ref.f).max() <= 1e-11 * np.abs(ref.f).max(), (shape, steps)
        assert abs(q_in - Q) <= 1e-14 * 8, (shape, steps)
