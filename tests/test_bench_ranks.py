"""The multi-GPU form of bench.py is independent replicas: every rank solves
its own instance and the whole-job figures combine the ranks.  Checked here on
CPU with two gloo ranks: the combined time is the slowest rank's, the MACs are
summed; the reference arm prints from rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r: device time 1 + r s, e2e 2 + r s, (r + 1) * 1e6 and 2e6 MACs
        got = bench.reduce_over_ranks(1.0 + rank, 2.0 + rank, (rank + 1) * 1e6, 2e6, "cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_replicas_combine_slowest_time_and_summed_work():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t_dev, t_e2e, macs, macs_e2e = out[r]
        assert (t_dev, t_e2e) == (2.0, 3.0)          # max over ranks
        assert (macs, macs_e2e) == (3e6, 4e6)        # sum over ranks


def test_reference_arm_prints_from_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    with redirect_stdout(buf):
        bench.run_reference(bench.parse())
    assert buf.getvalue() == ""
