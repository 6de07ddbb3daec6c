"""Batched solving of many (N, beta) instances with precision escalation.

The instances run through hk_batch_solve (one library call: a worker pool of
contexts on concurrent CUDA streams).  An instance whose rounded pivot fails
(HK_ERR_NOT_PD: the working precision P is too small, as expected for
beta = 3/4 under the batched sweep's precision rule) is regenerated at P + 1024
bits and solved again, up to `max_escalations` times.

Across GPUs the instances shard with no data-path collective: each rank of a
process group (one GPU each) solves its longest-processing-time share and the
small result records are gathered on the host (`solve_batch_sharded`).
"""
from . import hk, inputs


def solve_batch(instances, iters=0, nthreads=16, max_escalations=4, device=0, options=None):
    """instances: list of (N, (p, q), P).  Returns a list of dicts with the final
    P, status, lambda (n, e) and iterations, in input order."""
    ctx = hk.hk_create(device)
    try:
        for opt, val in (options or {}).items():
            hk.hk_set_option(ctx, opt, val)
        cur = [dict(N=N, beta=beta, P=P, status=None, lam=None, iters=0, escalations=0)
               for (N, beta, P) in instances]
        todo = list(range(len(cur)))
        for round_ in range(max_escalations + 1):
            if not todo:
                break
            batch = [(cur[k]["N"], cur[k]["beta"], cur[k]["P"],
                      inputs.moments(cur[k]["N"], cur[k]["beta"], cur[k]["P"])) for k in todo]
            res = hk.hk_batch_solve(ctx, batch, iters=iters, nthreads=nthreads)
            nxt = []
            for k, (st, lam, used) in zip(todo, res):
                cur[k].update(status=st, lam=lam, iters=used)
                if st == hk.HK_ERR_NOT_PD and round_ < max_escalations:
                    cur[k]["P"] += 1024
                    cur[k]["escalations"] += 1
                    nxt.append(k)
            todo = nxt
        return cur
    finally:
        hk.hk_destroy(ctx)


def work(instance):
    """Limb products of an instance's factorisation, N^3 L^2 (L = P / 32): the
    weight of the longest-processing-time order."""
    N, _, P = instance
    return N ** 3 * (P // 32) ** 2


def lpt_partition(instances, world):
    """Indices of `instances` per rank: in decreasing work, each instance goes
    to the rank with the least work so far (ties to the lowest rank)."""
    order = sorted(range(len(instances)), key=lambda k: (-work(instances[k]), k))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += work(instances[k])
    return parts


def solve_batch_sharded(instances, solver=solve_batch, **kwargs):
    """The batched solve over the ranks of the default torch.distributed
    process group (one GPU per rank, `device` = the rank's local GPU in
    kwargs): every rank solves its share with `solver` and every rank returns
    all records in input order, gathered on the host."""
    import torch.distributed as dist
    rank, world = dist.get_rank(), dist.get_world_size()
    mine = lpt_partition(instances, world)[rank]
    res = solver([instances[k] for k in mine], **kwargs) if mine else []
    gathered = [None] * world
    dist.all_gather_object(gathered, list(zip(mine, res)))
    out = [None] * len(instances)
    for part in gathered:
        for k, r in part:
            out[k] = r
    return out
