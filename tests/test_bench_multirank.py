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
