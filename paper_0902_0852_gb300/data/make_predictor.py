"""Generates the precision predictor's training tuples with the method itself,
trains the network on the device, and evaluates it on held-out instances.
Runs on a machine with the GPU (the solves and the training use the library's
kernels).  Writes, into --out (default: this directory):

  predictor_tuples.json  (N, beta) -> required bits, log2 lambda_min, iterations
  predictor.json         trained parameters, scalings and safety margin
  predictor_eval.json    held-out instances: predicted and verified solve of
                         each; the conservative solve of every --cons-every-th
                         (precisions, seconds, agreement, time gain)

Instances: training N ~ U{32..512}, beta ~ U[0.6, 4] snapped to the rational
grid of predictor.beta_grid() (seed 1, 4096 instances); held-out N ~ U{513..800},
same beta law (seed 2, 256 instances).

The generation can run in pieces: ``--range A:B`` generates the tuples of
training instances A..B-1 only (into predictor_tuples.partA_B.json), and
``--merge DIR`` joins the part files found in DIR (they must cover 0..train-1)
before training and the held-out evaluation.
"""
import glob
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_0902_0852_gb300 import build, predictor as pr  # noqa: E402


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--heldout", type=int, default=256)
    ap.add_argument("--cons-every", type=int, default=1,
                    help="also solve every k-th held-out instance at the conservative precision (time gain)")
    ap.add_argument("--range", default=None, help="A:B -- generate the tuples of training instances A..B-1 only")
    ap.add_argument("--merge", default=None, help="join the part files in this directory, then train and evaluate")
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--out", default=HERE)
    ap.add_argument("--tuples", default=None, help="reuse an existing tuples file")
    ap.add_argument("--workers", type=int, default=12)
    args = ap.parse_args()
    build.build()
    os.makedirs(args.out, exist_ok=True)
    if args.range:
        a, b = (int(v) for v in args.range.split(":"))
        inst = pr.sample_instances(args.train, 1, 32, 512)[a:b]
        t0 = time.time()
        tuples = pr.generate(inst, workers=args.workers, log=log)
        meta = dict(first=a, last=b, seconds=round(time.time() - t0, 1))
        with open(os.path.join(args.out, f"predictor_tuples.part{a}_{b}.json"), "w") as f:
            json.dump(dict(meta=meta, tuples=tuples), f)
        log(f"{len(tuples)} tuples ({a}..{b - 1}) in {meta['seconds']} s")
        return
    if args.merge:
        parts = []
        for path in glob.glob(os.path.join(args.merge, "predictor_tuples.part*_*.json")):
            d = json.load(open(path))
            parts.append((d["meta"]["first"], d["meta"]["last"], d["meta"]["seconds"], d["tuples"]))
        parts.sort()
        assert parts and parts[0][0] == 0 and parts[-1][1] == args.train, "parts must cover 0..train-1"
        assert all(p[1] == q[0] for p, q in zip(parts, parts[1:])), "parts must be contiguous"
        tuples = [t for p in parts for t in p[3]]
        meta = dict(generator="paper_0902_0852_gb300/data/make_predictor.py", count=len(tuples), seed=1,
                    N_range=[32, 512], beta="U[0.6,4] snapped to beta_grid()",
                    seconds=round(sum(p[2] for p in parts), 1), parts=len(parts),
                    agree_bits=pr.AGREE_BITS, delta=pr.DELTA)
        with open(os.path.join(args.out, "predictor_tuples.json"), "w") as f:
            json.dump(dict(meta=meta, tuples=tuples), f, indent=0)
        log(f"{len(tuples)} tuples merged from {len(parts)} parts ({meta['seconds']} s of generation)")
    elif args.tuples:
        tuples = json.load(open(args.tuples))["tuples"]
    else:
        inst = pr.sample_instances(args.train, 1, 32, 512)
        t0 = time.time()
        tuples = pr.generate(inst, workers=args.workers, log=log)
        meta = dict(generator="paper_0902_0852_gb300/data/make_predictor.py", count=len(inst), seed=1,
                    N_range=[32, 512], beta="U[0.6,4] snapped to beta_grid()", seconds=round(time.time() - t0, 1),
                    agree_bits=pr.AGREE_BITS, delta=pr.DELTA)
        with open(os.path.join(args.out, "predictor_tuples.json"), "w") as f:
            json.dump(dict(meta=meta, tuples=tuples), f, indent=0)
        log(f"{len(tuples)} tuples in {meta['seconds']} s")
    model = pr.Predictor()
    hist = model.fit(tuples, steps=args.steps, log=log)
    d = model.to_json()
    d["loss_first_last"] = [float(hist[0]), float(hist[-1])]
    with open(os.path.join(args.out, "predictor.json"), "w") as f:
        json.dump(d, f)
    rows = []
    for k, (N, beta) in enumerate(pr.sample_instances(args.heldout, 2, 513, 800)):
        v = pr.solve_verified(N, beta, model)
        row = dict(N=N, beta=list(beta), P_pred=v["P"], tried=v["tried"], pred_seconds=round(v["seconds"], 4),
                   pred_iters=v["iters"], T_budget=v["T"], verified=v["verified"],
                   log2_lambda=pr.log2_value(v["lam"]) if v["lam"] else None)
        msg = f"held-out N={N} beta={beta}: P {v['P']} ({v['tried']}) {v['seconds']:.2f}s"
        if k % args.cons_every == 0:
            # the plain method at the conservative precision: the reference for
            # the time gain and a second check of the verified value
            c = pr.solve_conservative(N, beta)
            agree = pr.rel_err_bits(v["lam"], c["lam"]) if (v["lam"] and c["lam"]) else None
            row.update(P_cons=c["P"], cons_seconds=round(c["seconds"], 4), cons_iters=c["iters"],
                       cons_converged=c["converged"], agree_bits=None if agree is None else min(agree, 1e9))
            msg += f"; conservative P {c['P']} {c['seconds']:.2f}s, agree {agree}"
        rows.append(row)
        log(msg)
    both = [r for r in rows if "cons_seconds" in r]
    tc = sum(r["cons_seconds"] for r in both)
    tp = sum(r["pred_seconds"] for r in both)
    summary = dict(instances=len(rows), conservative_checked=len(both), conservative_seconds=round(tc, 3),
                   predicted_seconds_same_instances=round(tp, 3),
                   predicted_seconds_all=round(sum(r["pred_seconds"] for r in rows), 3),
                   gain=round(tc / tp, 3) if tp else None, all_verified=all(r["verified"] for r in rows),
                   min_agree_bits=min((r["agree_bits"] for r in both if r["agree_bits"] is not None), default=None),
                   escalated=sum(len(r["tried"]) > 2 for r in rows))
    with open(os.path.join(args.out, "predictor_eval.json"), "w") as f:
        json.dump(dict(summary=summary, rows=rows), f, indent=0)
    log(json.dumps(summary))


if __name__ == "__main__":
    main()
