"""Batched solving of many (N, beta) instances with precision escalation.

The instances run through hk_batch_solve (one library call: a worker pool of
contexts on concurrent CUDA streams).  An instance whose rounded pivot fails
(HK_ERR_NOT_PD: the working precision P is too small, as expected for
beta = 3/4 under the batched sweep's precision rule) is regenerated at P + 1024
bits and solved again, up to `max_escalations` times.
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
