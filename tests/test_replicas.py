"""Multi-GPU form of bench.py: independent replicas, one per rank, combined by the slowest
rank's time and the sum of the units (no collective on the data path).  Checked here with a
world-size-2 gloo group on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) * 10 ms for (r + 1) * 1000 units
    t, u = bench.combine_ranks(dist, 0.010 * (rank + 1), 1000.0 * (rank + 1), "cpu")
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_combine_max_time_and_summed_units():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        t, u = out[r]
        assert t == pytest.approx(0.020) and u == pytest.approx(3000.0)
    # whole-job throughput = summed units / slowest time
    assert out[0][1] / out[0][0] == pytest.approx(150000.0)


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(None, 1.5, 42.0, "cpu") == (1.5, 42.0)
