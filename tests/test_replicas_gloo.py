"""The N > 1 path of bench.py on CPU: two gloo ranks acting as replicas. Units add up over
ranks and the job's time is its slowest rank's; the reference arm prints on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 14.0][rank]
    units = [1000.0, 3000.0][rank]
    res = bench.aggregate_ranks(ms, units, 2 * ms, units / 2, world, torch.device("cpu"))
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_units_and_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
        got = dict(out)
    for rank in (0, 1):
        total, ms_max, e2e_total, e2e_max = got[rank]
        assert total == 4000.0 and ms_max == 14.0
        assert e2e_total == 2000.0 and e2e_max == 28.0


def test_single_rank_passes_values_through():
    import bench
    assert bench.aggregate_ranks(5.0, 7.0, 9.0, 11.0, 1, None) == (7.0, 5.0, 11.0, 9.0)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import argparse

    import bench
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
