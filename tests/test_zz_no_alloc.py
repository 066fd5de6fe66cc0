"""lbm_inlet_density_noalloc: the inlet density for callers that cannot allocate
device memory when they need it (inside a stream capture, or under a device
memory budget held by another allocator).  Its scratch is a static device array
inside the library, so the call allocates nothing.

The check: on two calls in a row, the value it returns for the current state
equals the density the existing step path then computes and imposes from that
same state (read back through lbm_get_flux after one lbm_step), within the
FP64 parity tolerance of the other GPU tests.  This file is collected last so
that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest

import oracle as O
from lbm_inputs import random_mask, uniform_field

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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_density_matches_step_path_twice(torch_cuda, prec):
    torch = torch_cuda
    from paper_1806_10589_gb300 import Lattice

    m = random_mask(37, 29, 21, 0.3, 9)  # A > 256: several reduction blocks
    f0 = O.W[:, None, None, None] * (1.0 + 0.01 * uniform_field((19,) + m.shape, 33))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with Lattice(m, 0.8, "mrt", prec, stream=torch.cuda.current_stream()) as lat:
        lat.set_flux_bc(0.0031)
        lat.set_distributions(f0)
        for call in range(2):
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            lat.inlet_density_noalloc(out)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            got = float(out.item())
            lat.step(1)
            _, want = lat.get_flux(4)
            assert abs(got - want) <= 1e-11 * abs(want), (call, got, want)
            if call > 0:
                # the first call on a device may make the driver load the
                # library's module (which holds the static scratch); after
                # that, a call changes nothing in device memory
                assert free_after == free_before
            out.zero_()


def test_noalloc_rejects_inlets_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_1806_10589_gb300 import Lattice, LBMError

    m = np.zeros((3, 730, 730), np.uint8)  # 532,900 inlet pore nodes > 524,288
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with Lattice(m, 1.0, "mrt", "fp32", stream=torch.cuda.current_stream()) as lat:
        with pytest.raises(LBMError) as ei:
            lat.inlet_density_noalloc(out)
        assert "at most 524288" in str(ei.value)
