#!/usr/bin/env python3
"""Benchmark: P-bit multiply-accumulates per second of the exact Cholesky
factorisation + inverse iteration of the Hankel moment matrix, and the time
to lambda_min, at the paper-scale workload N = 1000, beta = 1, P = 24576 bits.

One step = load the 2N-1 moments (already resident in device memory),
factor M = R^T R, run inverse iteration until |lambda_t - lambda_{t-1}| <=
2^-136 lambda_t.  The e2e leg repeats the step through the C ABI from pinned
host buffers (host->device moments and device->host lambda inside the timed
region).  `--impl reference` times the CPU oracle on a bounded sample of the
same workload.

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas
(one instance per GPU; the single-instance factorisation does not shard).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "P-bit MAC/s in Cholesky update (+ inverse iteration), time-to-lambda_min"
UNIT = "MAC/s"
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
# DRAM bytes (read + write) per executed limb product of the update kernel, from
# one ncu capture of the current kernel version; None when not measured.
# DRAM bytes (read + write) per executed limb product of the update kernel,
# by Karatsuba depth, from one ncu capture each of the same launch (rows
# 256..271 against t < 256 at N = 512, P = 24576)
UPDATE_TRAFFIC_BYTES_PER_LIMBPROD = {
    3: (8.395456e9 + 0.0322035e9) / (3976 * 256 * 265833),   # k_update_stripe8_N512_P24576_full.md
    4: (39.609636e9 + 0.03896192e9) / (3976 * 256 * 202748),  # k_update_karatsuba4_N512_P24576_full.md
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--N", type=int, default=1000)
    ap.add_argument("--P", type=int, default=24576)
    ap.add_argument("--iters", type=int, default=0, help="0 = until converged (2^-136)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-predicted", action="store_true",
                    help="skip the predicted-precision time-to-lambda comparison (after the timed region)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the after-region comparisons (Secant, INT8 update, batched sweep)")
    ap.add_argument("--paper-cells", default=None, metavar="N:p/q,...|default|all",
                    help="instead of the bench: Table 3 cells at a verified precision, one JSON line")
    return ap.parse_args()


def run_paper_cells(spec):
    """Table 3 cells (N, beta) on the device at a verified precision."""
    from paper_0902_0852_gb300 import build
    from paper_0902_0852_gb300.paper_cells import ALL_CELLS, DEFAULT_CELLS, run_cell
    build.build()
    if spec in ("default", "all"):
        cells = DEFAULT_CELLS if spec == "default" else ALL_CELLS
    else:
        cells = []
        for item in spec.split(","):
            n, b = item.split(":")
            p, q = b.split("/")
            cells.append((int(n), (int(p), int(q))))
    out = []
    for N, beta in cells:
        out.append(run_cell(N, beta))
        print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"paper_cells": out, "matched": sum(r["match"] for r in out), "cells": len(out)}))


def step_macs(N, T):
    """Algorithmic P-bit MACs: factor (N-1)N(N+1)/6, two solves of N(N-1)/2
    per inverse-iteration step, and the two dot products (2N)."""
    return (N - 1) * N * (N + 1) // 6 + T * (N * (N - 1) + 2 * N)


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

ORACLE_STEPS = 16  # panel steps in the timed oracle sample


def oracle_sample_setup(N, P, steps):
    """Inputs of the first `steps` panel steps of the beta = 1 factorisation:
    rows t < steps of R from the exact closed form i! C(i, t) (equal to the
    oracle's own rows at this P; oracle.cholesky_factorial)."""
    import oracle
    return oracle.cholesky_factorial(N, P, rows=steps)


def _oracle_chunk(args):
    """The oracle's exact dot product on one share of the sample: for each
    entry (i, j), i <= j, the contributions sum_{t < min(i, steps)} R_ti R_tj
    of the first panel steps.  Returns (worker pid, MACs, seconds)."""
    import oracle
    rows, cols, steps = args  # rows[t] = {j: R_tj}; cols = list of (i, j)
    t0 = time.perf_counter()
    macs = 0
    for i, j in cols:
        k = min(i, steps)
        if k:
            oracle.exact_dot([(rows[t][i], rows[t][j]) for t in range(k)])
            macs += k
    return os.getpid(), macs, time.perf_counter() - t0


def make_pool(cores):
    """Spawned workers (safe before or after CUDA work)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    pool = ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"))
    # start every worker: each sleeping task holds one, so all must be up
    list(pool.map(time.sleep, [0.3] * (2 * cores)))
    return pool


def oracle_tasks(N, steps, setup, cores):
    """The sample's entries split by column over `cores` workers, each shipped
    only the rows' entries of its columns."""
    Rrows = setup
    tasks = []
    for k in range(cores):
        js = list(range(1 + k, N, cores))
        if not js:
            continue
        need = set(js)
        cols = [(i, j) for j in js for i in range(1, j + 1)]
        need |= {i for i, _ in cols}
        rows = [{c: Rrows[t][c - t] for c in need if c >= t} for t in range(len(Rrows))]
        tasks.append((rows, cols, steps))
    return tasks


def oracle_sample(pool, tasks):
    """The oracle on the first panel steps of the N x N factorisation, split
    over the pool.  Each worker times only the oracle's arithmetic (its share
    of the inputs is shipped before its clock starts); the sample's time is
    the busiest worker's total.  Returns (MACs, seconds)."""
    busy, macs = {}, 0
    for pid, mc, sec in pool.map(_oracle_chunk, tasks):
        busy[pid] = busy.get(pid, 0.0) + sec
        macs += mc
    return macs, max(busy.values())


def oracle_single_thread(tasks, limit=64):
    """The oracle on one core: the first `limit` entries of the first share,
    in this process.  Returns (MACs, seconds)."""
    rows, cols, steps = tasks[0]
    _, macs, sec = _oracle_chunk((rows, cols[-limit:], steps))
    return macs, sec


def sample_macs(N, steps):
    return sum(min(i, steps) * (N - i) for i in range(1, N))


def reduce_over_ranks(t_dev, t_e2e, macs, macs_e2e, device):
    """Whole-job figures of a replicas run (every rank solves its own
    instance): the slowest rank's device and end-to-end times, and the MACs of
    all ranks.  Collective over the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_dev, t_e2e], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    m = torch.tensor([macs, macs_e2e], device=device, dtype=torch.float64)
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(m[0]), float(m[1])


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    def __init__(self, dev):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={SMI_FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(dev)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    N, P = args.N, args.P
    cores = os.cpu_count() or 1
    pool = make_pool(cores)
    tasks = oracle_tasks(N, ORACLE_STEPS, oracle_sample_setup(N, P, ORACLE_STEPS), cores)
    for _ in range(args.warmup):
        oracle_sample(pool, tasks)
    tot_m, tot_t = 0, 0.0
    for _ in range(args.steps):
        m, t = oracle_sample(pool, tasks)
        tot_m += m
        tot_t += t
    pool.shutdown()
    m1, t1 = oracle_single_thread(tasks)
    v = tot_m / tot_t
    sample = (f"the first {ORACLE_STEPS} panel steps of the N={N}, P={P}, beta=1 factorisation: the exact "
              f"contributions sum_(t<min(i,{ORACLE_STEPS})) R_ti R_tj to every entry ({tot_m // args.steps} MACs per "
              f"step; time in the oracle, inputs shipped untimed)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "python-int (exact)",
        "data": "synthetic",
        "config": {"workload": f"Hankel moment matrix N={N}, beta=1 (m_k = k!), P={P} bits; oracle sample", "N": N,
                   "P": P, "beta": "1"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "single_thread": {"value": m1 / t1, "unit": UNIT,
                                           "sample": f"64 entries of the same sample ({m1} MACs, one process)"}},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.paper_cells:
        run_paper_cells(args.paper_cells)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    N, P, beta = args.N, args.P, (1, 1)
    L = P // 32

    # the CPU baseline first (spawn pool, before any CUDA work)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        pool = make_pool(cores)
        tasks = oracle_tasks(N, ORACLE_STEPS, oracle_sample_setup(N, P, ORACLE_STEPS), cores)
        m_, t_ = oracle_sample(pool, tasks)
        pool.shutdown()
        m1, t1 = oracle_single_thread(tasks)
        cpu = {"value": m_ / t_, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the first {ORACLE_STEPS} panel steps of the N={N}, P={P}, beta=1 factorisation: the "
                         f"exact contributions of rows t < {ORACLE_STEPS} to every entry ({m_} MACs, {t_:.1f} s in "
                         f"the oracle, inputs shipped untimed)",
               "single_thread": {"value": m1 / t1, "unit": UNIT,
                                 "sample": f"64 entries of the same sample ({m1} MACs, one process)"}}

    import numpy as np
    import torch
    from paper_0902_0852_gb300 import build, hk, inputs
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    stream = torch.cuda.current_stream()
    moments = inputs.moments(N, beta, P)
    s_h, e_h, l_h = hk.pack(moments, P)
    s_d = torch.from_numpy(s_h).cuda()
    e_d = torch.from_numpy(e_h).cuda()
    l_d = torch.from_numpy(l_h.view(np.int32)).cuda()
    # pinned host copies for the e2e leg
    s_p = torch.from_numpy(s_h).pin_memory()
    e_p = torch.from_numpy(e_h).pin_memory()
    l_p = torch.from_numpy(l_h.view(np.int32)).pin_memory()
    h2d = s_h.nbytes + e_h.nbytes + l_h.nbytes
    d2h = 4 * L + 12

    h = hk.Hankel(local, stream)
    peaks = hk.hk_probe_int_peaks(local)

    def step(device_inputs):
        if device_inputs:
            h.load_device(N, beta, P, s_d, e_d, l_d)
        else:
            hk.hk_load_moments_flat(h.ctx, N, beta, P, s_p, e_p, l_p, on_device=False)
        h.factor()
        lam, used = h.smallest_eig(args.iters)
        return lam, used, h.timings(), h.stats()

    # warm-up; the last warm-up step runs with the lookahead off, so that its
    # per-launch events time the update kernels alone (the roofline below);
    # the timed steps overlap the panel chain with the updates
    serial = None
    for k in range(args.warmup):
        last = k == args.warmup - 1
        if last:
            h.set_option(hk.HK_OPT_LOOKAHEAD, 0)
        r = step(True)
        if last:
            serial = r
            h.set_option(hk.HK_OPT_LOOKAHEAD, 1)
    torch.cuda.synchronize()

    # ---- timed: device-resident inputs ----
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    recs = [step(True) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    t_dev = ev0.elapsed_time(ev1) / 1e3

    # ---- timed: end to end from pinned host buffers ----
    barrier()
    torch.cuda.synchronize()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    recs_e2e = [step(False) for _ in range(args.steps)]
    ee1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_e2e = ee0.elapsed_time(ee1) / 1e3

    lam, used = recs[-1][0], recs[-1][1]
    if lam != recs_e2e[-1][0]:
        raise SystemExit("device-resident and end-to-end runs disagree on lambda")
    macs = sum(step_macs(N, r[1]) for r in recs)
    macs_e2e = sum(step_macs(N, r[1]) for r in recs_e2e)
    if world > 1:
        t_dev, t_e2e, macs, macs_e2e = reduce_over_ranks(t_dev, t_e2e, macs, macs_e2e, "cuda")
    if rank != 0:
        h.close()
        return

    # roofline of the update kernel (factor launches), CUDA events per launch,
    # from the warm-up step without the lookahead (kernels timed alone)
    ref = serial if serial is not None else recs[-1]
    upd_ms = ref[2]["update_ms"]
    fac_ms = sum(r[2]["factor_ms"] for r in recs)
    eig_ms = sum(r[2]["eig_ms"] for r in recs)
    limbprod = (N - 1) * N * (N + 1) // 6 * L * L
    achieved = limbprod / (upd_ms / 1e3) / 1e12
    st = ref[3]
    executed = (N - 1) * N * (N + 1) // 6 * st["limbprod_per_mac"] / (upd_ms / 1e3) / 1e12
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = n_sm * 64 * max_mhz * 1e6 / 2 / 1e12
    # per update launch, averaged like `achieved`: one big update per 16-row
    # block after the first plus one in-block update per row -> N - 1 launches
    per_prod = UPDATE_TRAFFIC_BYTES_PER_LIMBPROD.get(st["karatsuba_levels"])
    traffic = (per_prod * (N - 1) * N * (N + 1) // 6 * st["limbprod_per_mac"] / (N - 1)) if per_prod else None
    n_lam, e_lam = lam
    # decimal rendering of lambda (n * 2^e) with 10 significant digits
    lg = math.log10(abs(n_lam)) + e_lam * math.log10(2)
    ex = math.floor(lg)
    lam_str = f"{10 ** (lg - ex):.9f}e{ex}"

    out = {
        "metric": METRIC, "value": macs / t_dev, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"Hankel moment matrix N={N}, beta=1 (m_k = k!), P={P} bits (L={L}); Cholesky + "
                               f"inverse iteration to 2^-136", "N": N, "beta": "1", "P": P,
                   "iters": "converged" if args.iters == 0 else args.iters,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "no flush: working set (R, its aligned copy and their Karatsuba expansion, about "
                         "22 GB at N=1000) is far larger than L2"},
        "time_to_lambda_s": t_dev / args.steps, "iters_used": used, "lambda_min": lam_str,
        "lambda_min_table3": "1.0892e-52" if (N, P) == (1000, 24576) else None,
        "factor_ms": fac_ms / args.steps, "inverse_iteration_ms": eig_ms / args.steps,
        # per-phase device time (CUDA events around each launch group): update
        # kernels of the factor, its diagonal/row kernels, and the solves; the
        # timed steps overlap the first two (lookahead), the warm-up step
        # without lookahead times them alone
        "phases_ms": {k: sum(r[2][k] for r in recs) / args.steps for k in ("update_ms", "panel_ms", "solve_ms")},
        "phases_ms_serial": {k: ref[2][k] for k in ("update_ms", "panel_ms", "solve_ms", "factor_ms")},
        "factor_macs_per_s": (N - 1) * N * (N + 1) / 6 / (fac_ms / args.steps / 1e3),
        "limb_products_per_s_factor": limbprod / (fac_ms / args.steps / 1e3),
        "e2e": {"value": macs_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # achieved / frac: the algorithmic work (the metric's schoolbook L^2
        # limb products per MAC); executed / executed_frac: the products the
        # Karatsuba expansion actually runs, the kernel's own efficiency
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlimbprod/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_update (exact trailing update), factor launches",
                     "peak_basis": f"{n_sm} SMs x 64 IMAD/clk/SM x {max_mhz:.0f} MHz / 2 IMAD per 32x32->64 "
                                   f"limb product (probe: {peaks['imad_per_clk_sm']:.1f} IMAD/clk/SM)",
                     "achieved_basis": f"schoolbook L^2 = {L * L} limb products per P-bit MAC (the metric's unit); "
                                       f"above 1 because Karatsuba executes fewer products",
                     "executed": executed, "executed_frac": executed / peak,
                     "executed_basis": f"limb products the kernel executes: {st['limbprod_per_mac']} per P-bit MAC "
                                       f"({st['karatsuba_levels']} Karatsuba levels on window W = {st['W']})"},
        "int_probe": peaks,
        "clocks": clocks,
        "gpu_launches": sum(r[3]["launches"] for r in recs),
    }
    out["solve_window_limbs"] = {"max": st.get("solve_wv_max"), "mean": st.get("solve_wv_mean"), "W": st["W"]}
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if world == 1:
        # the GPU on the oracle's sample: the first panel steps' update contributions
        s_ms, s_macs = hk.hk_time_update_slice(h.ctx, ORACLE_STEPS)
        out["gpu_oracle_slice"] = {"panel_steps": ORACLE_STEPS, "macs": s_macs, "ms": s_ms,
                                   "value": s_macs / (s_ms / 1e3), "unit": UNIT,
                                   "what": "the exact update kernel on the same sample as cpu_baseline"}
    if world == 1 and not args.no_extras:
        out["secant"] = secant_comparison(h, N, beta, P, lam, t_dev / args.steps)
    h.close()
    if world == 1 and not args.no_extras:
        out["int8_update"] = int8_comparison(N, beta, P, moments, peaks, clocks)
        out["batched_sweep"] = batched_sweep()
    if not args.no_predicted and world == 1:
        out["time_to_lambda_predicted"] = predicted_comparison(N, beta)
    print(json.dumps(out))


def secant_comparison(h, N, beta, P, lam_ii, t_ii):
    """The paper's own route to lambda_1 on the same instance: the Secant
    recurrence on det(M - xI) (one shifted LDL^T per iterate), then the
    inertia on both sides of the root at P + 160 bits; timed around the
    library calls after the benchmark's timed region."""
    from paper_0902_0852_gb300 import hk
    from paper_0902_0852_gb300.predictor import rel_err_bits
    t0 = time.perf_counter()
    root, dets = hk.hk_secant(h.ctx, P)
    t1 = time.perf_counter()
    out4 = hk.hk_secant_verify(h.ctx, P, root, 130)
    t2 = time.perf_counter()
    agree = rel_err_bits(root, lam_ii)
    return {"t_secant_s": round(t1 - t0, 3), "determinants": dets, "t_verify_s": round(t2 - t1, 3),
            "verified": list(out4) == [0, 1, 1, -1], "inertia": list(out4),
            "t_inverse_iteration_step_s": round(t_ii, 3),
            "agree_bits_with_inverse_iteration": None if agree is None else min(agree, 1e9),
            "speedup_of_inverse_iteration": round((t1 - t0) / t_ii, 3)}


def int8_comparison(N, beta, P, moments, peaks, clocks):
    """The INT8 tensor form of the factor update (mma.sync m16n8k32 u8) on the
    same instance, once, after the timed region: its update time, u8 multiply-
    adds per second over the plain entries (16 W^2 per P-bit MAC), the fraction
    of the measured mma.sync u8 rate, and R equal to the IMAD path's."""
    import torch
    from paper_0902_0852_gb300 import hk
    with hk.Hankel(0) as h:
        h.load(N, beta, P, moments)
        h.factor()
        ref = hk.hk_get_R_flat(h.ctx, N, P)
        ms_imad = h.timings()["update_ms"]
        h.set_update_path(1)
        h.factor()
        tm = h.timings()
        st = h.stats()
        got = hk.hk_get_R_flat(h.ctx, N, P)
    same = all(bool((a == b).all()) for a, b in zip(ref, got))
    W = st["W"]
    u8 = (N - 1) * N * (N + 1) / 6 * 16 * W * W
    rate = u8 / (tm["update_ms"] / 1e3)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = peaks["mma_u8_mac_per_clk_sm"] * n_sm * mhz * 1e6
    return {"update_ms": round(tm["update_ms"], 1), "update_ms_imad": round(ms_imad, 1), "u8_mac_per_s": rate,
            "peak_u8_mac_per_s": peak, "frac_of_mma_u8_peak": rate / peak, "R_bit_identical_to_imad": same,
            "peak_basis": f"probe {peaks['mma_u8_mac_per_clk_sm']:.1f} u8 MAC/clk/SM x {n_sm} SMs x {mhz:.0f} MHz",
            "work_basis": f"16 W^2 u8 MACs per P-bit MAC over plain entries, W = {W}"}


def batched_sweep():
    """The batched sweep: 64 instances (seed 0), N in [100, 600], beta in
    {3/4, 1, 3/2, 2, 3}, P by the sweep's rule, solved to convergence through
    hk_batch_solve (host worker pool of contexts on concurrent streams),
    escalating P by 1024 on a failed pivot; timed around the library calls."""
    from paper_0902_0852_gb300 import batch, inputs
    inst = inputs.batched_instances(64, 0)
    t0 = time.perf_counter()
    res = batch.solve_batch(inst)
    dt = time.perf_counter() - t0
    return {"instances": len(inst), "seconds": round(dt, 3),
            "escalations": sum(r["escalations"] for r in res),
            "iterations": sum(abs(r["iters"]) for r in res),
            "all_ok": all(r["status"] == 0 for r in res),
            "macs": sum((r["N"] - 1) * r["N"] * (r["N"] + 1) // 6 for r in res),
            "scheduler": "host worker pool (16 contexts on non-blocking streams, largest first)"}


def predicted_comparison(N, beta):
    """Time to a verified lambda_min at the precision the trained predictor
    picks (solve at P, verify at P + 1024, escalate on disagreement) against
    the method alone at the conservative precision; both through the library,
    timed around the library calls (which synchronise), after the benchmark's
    timed region.  The two lambdas must agree to 2^-128."""
    from paper_0902_0852_gb300 import predictor as pr
    path = os.path.join(ROOT, "paper_0902_0852_gb300", "data", "predictor.json")
    if not os.path.exists(path):
        return None
    model = pr.load_default()
    c = pr.solve_conservative(N, beta)
    v = pr.solve_verified(N, beta, model)
    agree = pr.rel_err_bits(v["lam"], c["lam"]) if v["lam"] and c["lam"] else None
    return {"P_conservative": c["P"], "t_conservative_s": round(c["seconds"], 4), "iters_conservative": c["iters"],
            "P_predicted": v["P"], "precisions_run": v["tried"], "t_predicted_verified_s": round(v["seconds"], 4),
            "iters_predicted": v["iters"], "verified": v["verified"],
            "agree_bits": None if agree is None else min(agree, 1e9),
            "speedup": round(c["seconds"] / v["seconds"], 3) if v["seconds"] else None,
            "update_path": "IMAD (the INT8 mma.sync path is slower on GB300)"}


if __name__ == "__main__":
    main()
