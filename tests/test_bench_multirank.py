"""The N > 1 benchmark path on CPU: two gloo ranks, each a replica with its own
pore count and time; rank 0 must report all ranks' updates over the slowest
rank's time (no GPU, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    n_local = [1000, 3000][rank]
    ms_local = [10.0, 25.0][rank]
    value, ms = bench.aggregate(n_local, 50, ms_local, world, "cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, ms = out[r]
        assert ms == 25.0
        assert abs(value - (4000 * 50) / 25e-3 / 1e6) < 1e-9


def test_single_rank_aggregate_is_local():
    import bench

    v, ms = bench.aggregate(2000, 10, 4.0, 1)
    assert ms == 4.0 and abs(v - 2000 * 10 / 4e-3 / 1e6) < 1e-12


def test_ensemble_steady_summary():
    """Post-processing of the ensemble's steady-state run: a member is steady
    from the first of `hold` consecutive checks within the tolerance."""
    import numpy as np

    import bench

    every, hold = 100, 3
    t = np.arange(1, 21)[:, None]
    # member 0 relaxes like 1 + e^{-t/2}, member 1 never settles its outlet flux
    ks = np.hstack([1.0 + np.exp(-t / 2.0), np.ones_like(t, dtype=float)])
    qs = np.hstack([np.ones_like(t, dtype=float), 1.0 + 0.01 * (-1.0) ** t])
    out = bench.steady_summary(ks, qs, [1.0, 1.0], every, hold, 1e-3, 2000)
    # member 0 is steady from the first check within 1e-3 of its final k (all later ones are too)
    k_inf = ks[-1, 0]
    first_ok = int(np.argmax(np.abs(ks[:, 0] - k_inf) <= 1e-3 * k_inf))
    assert out["members_reached"] == 1 and out["members"] == 2
    assert out["steps_all_steady"] is None
    assert out["steps_median_member"] == (first_ok + 1) * every
    assert "0.1%" in out["criterion"]


def test_timed_launch_count():
    """The benchmark's count of library launches in the timed call.  FP32 on the
    AA pattern: the warm-up call leaves the buffer in the in-place layout, so the
    timed call is its K step launches; the two-buffer kernel is K launches too.
    16-bit AA, warm-up 5 and 1100 timed steps: the refresh falls after 1019
    timed steps, 1024 since the swap-in (an even count: no un-stream), so the
    swap back, re-encode, inlet density and a new swap-in add 4 launches; the
    two-buffer kernel adds the re-encode and the inlet density."""
    import bench

    assert bench.timed_launches(5, 20, 3, "fp32") == 20
    assert bench.timed_launches(3, 10000, 3, "fp32") == 10000
    assert bench.timed_launches(0, 20, 3, "fp32") == 21
    assert bench.timed_launches(5, 200, 0, "fp32") == 200
    assert bench.timed_launches(5, 1100, 3, "fp16dev") == 1100 + 4
    assert bench.timed_launches(5, 1000, 3, "fp16dev") == 1000
    assert bench.timed_launches(5, 2000, 0, "bf16dev") == 2000 + 2
