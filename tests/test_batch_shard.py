"""Sharding of the batched solve across ranks (host logic, CPU): the
longest-processing-time partition, and the gather of per-instance records
over two gloo ranks with a stand-in solver (the real one needs a GPU per
rank)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def sweep(n=64, seed=0):
    """Instances shaped like the batched sweep: N uniform in [100, 600],
    beta from {3/4, 1, 3/2, 2, 3}, P from N (any positive multiple of 32)."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(100, 601, n)
    betas = [(3, 4), (1, 1), (3, 2), (2, 1), (3, 1)]
    bs = rng.integers(0, 5, n)
    return [(int(N), betas[int(b)], 32 * (int(N) // 8 + 8)) for N, b in zip(Ns, bs)]


def test_lpt_partition_assigns_each_instance_once_and_balances():
    from paper_0902_0852_gb300.batch import lpt_partition, work
    inst = sweep()
    for world in (1, 2, 3, 8):
        parts = lpt_partition(inst, world)
        assert sorted(k for p in parts for k in p) == list(range(len(inst)))
        loads = [sum(work(inst[k]) for k in p) for p in parts]
        # the greedy bound: no rank exceeds the lightest by more than one instance
        assert max(loads) - min(loads) <= max(work(x) for x in inst)
        # each rank's instances come in decreasing work (largest first)
        for p in parts:
            assert [work(inst[k]) for k in p] == sorted((work(inst[k]) for k in p), reverse=True)


def _fake_solver(instances, tag=None):
    import torch.distributed as dist
    return [dict(N=N, P=P, rank=dist.get_rank(), tag=tag) for N, _, P in instances]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_0902_0852_gb300.batch import solve_batch_sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        out[rank] = solve_batch_sharded(sweep(20), solver=_fake_solver, tag="x")
    finally:
        dist.destroy_process_group()


def test_sharded_batch_gathers_every_record_in_input_order():
    from paper_0902_0852_gb300.batch import lpt_partition
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    inst = sweep(20)
    parts = lpt_partition(inst, 2)
    assert out[0] == out[1]
    for k, rec in enumerate(out[0]):
        assert (rec["N"], rec["P"], rec["tag"]) == (inst[k][0], inst[k][2], "x")
        assert k in parts[rec["rank"]]
