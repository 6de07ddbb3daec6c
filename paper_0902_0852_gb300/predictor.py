"""Precision predictor: a small network that picks the working precision P
and the iteration budget of the Hankel smallest-eigenvalue solve from (N, beta).

Why.  The paper's precision requirement grows with N (Introduction; the K
column of Table 2), and each P-bit multiply-accumulate of the factorisation
costs about (P/32)^2 limb products, so over-provisioning P is paid
quadratically.  A conservative rule sized on the largest matrix entry is safe
but far above what the floating-point factorisation needs (about 4-7 times the
verified precision on held-out instances); the network learns the gap from
tuples that the method itself generates.

Pieces (all device arithmetic runs in the library: the solves in its
multiprecision kernels, the network in its FP32 kernels):

* ``p_conservative(N, beta)``: the batched sweep's rule
  ceil32(log2((2N-2)!) + 4 sqrt(N) + 256), taken as the maximum with the same
  margins on the largest entry's bits log2(Gamma((2N-1)/beta)/beta).
* ``generate(instances)``: per (N, beta) a reference solve at
  P_ref = P_cons + 1024, then the smallest P (multiple of 32) whose converged
  lambda_min agrees with the reference to 2^-128 relative, found by jumps
  along the measured error (a P-bit solve's relative error falls about one
  bit per bit of P) and a final bisection; targets (required bits,
  log2 lambda_min, iterations).
* ``Predictor``: the 2 -> 64 -> 64 -> 3 network (``hk_mlp_*``) with feature
  and target scaling, trained by full-batch Adam on the device.
* ``solve_verified(N, beta, predictor)``: solve at the predicted P with the
  predicted iteration budget, verify by a rerun at P + 1024, and escalate P by
  1024 while the two disagree (or the iteration did not converge); the
  conservative solve is the fallback.
"""
import json
import math
import os
import time
from fractions import Fraction

import numpy as np

from . import hk, inputs

DELTA = 1024          # verification rerun offset and escalation step (bits)
AGREE_BITS = 128      # required relative agreement 2^-128
P_MIN = 192           # below this the convergence test (2^-136) cannot be met
MAX_ITERS = 400


def _ceil32(x):
    return int(math.ceil(x / 32.0)) * 32


def beta_grid(pmax_den=12):
    """Shape parameters beta = p/q in [0.6, 4] whose moments the input
    generator can produce (p in {1, 2, 3, 4, 5, 7}: Gamma(a/p) constants)."""
    out = set()
    for p in (1, 2, 3, 4, 5, 7):
        for q in range(1, pmax_den + 1):
            if math.gcd(p, q) == 1 and 0.6 <= p / q <= 4.0:
                out.add((p, q))
    return sorted(out, key=lambda b: b[0] / b[1])


def snap_beta(b, grid=None):
    """The grid value nearest to a real beta (ties to the smaller)."""
    grid = grid or beta_grid()
    return min(grid, key=lambda g: (abs(g[0] / g[1] - b), g[0] / g[1]))


def largest_entry_bits(N, beta):
    p, q = inputs.as_ratio(beta)
    x = (2 * N - 1) * q / p
    return (math.lgamma(x) - math.log(p / q)) / math.log(2)


def p_conservative(N, beta):
    base = math.lgamma(2 * N - 1) / math.log(2)
    return _ceil32(max(base, largest_entry_bits(N, beta)) + 4 * math.sqrt(N) + 256)


def sample_instances(count, seed, n_lo, n_hi):
    """N ~ U{n_lo..n_hi}, beta ~ U[0.6, 4] snapped to the rational grid."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_lo, n_hi + 1, count)
    bs = rng.uniform(0.6, 4.0, count)
    grid = beta_grid()
    return [(int(N), snap_beta(float(b), grid)) for N, b in zip(Ns, bs)]


def _frac(v):
    n, e = v
    return Fraction(n) * (Fraction(2) ** e)


def rel_err_bits(v, ref):
    """-log2 |v - ref| / |ref| (inf when equal)."""
    a, b = _frac(v), _frac(ref)
    if a == b:
        return math.inf
    d = abs(a - b) / abs(b)
    return -(math.log2(d.numerator) - math.log2(d.denominator))


def log2_value(v):
    n, e = v
    return math.log2(abs(n)) + e


def _moments_job(args):
    N, beta, P = args
    return inputs.moments(N, beta, P)


class _Pool:
    """Spawned worker processes for the input generator (moments at many P)."""

    def __init__(self, workers):
        self.ex = None
        if workers > 1:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            self.ex = ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))

    def moments(self, jobs):
        if self.ex is None:
            return [_moments_job(j) for j in jobs]
        return list(self.ex.map(_moments_job, jobs, chunksize=1))

    def close(self):
        if self.ex is not None:
            self.ex.shutdown()


def _batch(ctx, pool, jobs, nthreads):
    """Solve (N, beta, P) jobs to convergence: list of (status, lambda, iters,
    converged)."""
    moms = pool.moments(jobs)
    res = hk.hk_batch_solve(ctx, [(N, b, P, m) for (N, b, P), m in zip(jobs, moms)], iters=0,
                            nthreads=nthreads)
    return [(st, lam, abs(it), it > 0) for st, lam, it in res]


def generate(instances, nthreads=16, workers=8, log=None, solve_fn=None):
    """Method-generated training tuples for (N, beta) instances: a list of dicts
    with N, beta, P_cons, P_ref, bits (the required precision), log2_lambda,
    iters, probes, seconds.  ``solve_fn(jobs)`` (jobs: (N, beta, P) triples;
    returns (status, lambda, iterations, converged) per job) replaces the
    library's batched solve, for tests of the search on the host."""
    t0 = time.time()
    ctx = pool = None
    if solve_fn is None:
        ctx = hk.hk_create(0)
        pool = _Pool(workers)
        hk.hk_set_option(ctx, hk.HK_OPT_MAX_ITERS, MAX_ITERS)
        solve_fn = lambda jobs: _batch(ctx, pool, jobs, nthreads)  # noqa: E731
    try:
        recs = []
        for N, beta in instances:
            pc = p_conservative(N, beta)
            recs.append(dict(N=N, beta=list(beta), P_cons=pc, P_ref=pc + DELTA, probes=[]))
        ref = solve_fn([(r["N"], tuple(r["beta"]), r["P_ref"]) for r in recs])
        for r, (st, lam, it, conv) in zip(recs, ref):
            r["ok"] = st == hk.HK_OK and conv
            if r["ok"]:
                r["lam_ref"] = lam
                r["log2_lambda"] = log2_value(lam)
                r["iters"] = it
        # search state: lo = largest failing P, hi = smallest passing P, est =
        # the requirement the error law predicts from the last failing probe
        state = {i: dict(lo=P_MIN - 32, hi=r["P_ref"], est=None, nxt=max(P_MIN + 64, _ceil32(r["P_cons"] / 4)))
                 for i, r in enumerate(recs) if r["ok"]}
        rounds = 0
        while True:
            active = [i for i, s in state.items() if s["hi"] - s["lo"] > 32]
            if not active:
                break
            rounds += 1
            jobs = []
            for i in active:
                s = state[i]
                s["probe"] = min(max(_ceil32(s["nxt"]), s["lo"] + 32), s["hi"] - 32)
                jobs.append((recs[i]["N"], tuple(recs[i]["beta"]), s["probe"]))
            out = solve_fn(jobs)
            for i, (st, lam, it, conv) in zip(active, out):
                s, r = state[i], recs[i]
                P = s["probe"]
                d = rel_err_bits(lam, r["lam_ref"]) if st == hk.HK_OK else None
                r["probes"].append([P, st, None if d is None else (d if math.isfinite(d) else 1e9), it, conv])
                if st == hk.HK_OK and conv and d >= AGREE_BITS:
                    s["hi"] = P
                    # try just below the predicted requirement, else bisect
                    s["nxt"] = _ceil32(s["est"]) - 32 if s["est"] is not None else (s["lo"] + P) // 2
                else:
                    s["lo"] = P
                    if st == hk.HK_OK and d is not None:
                        # the error falls about one bit per bit of P; an
                        # unconverged iteration at enough agreement needs a
                        # little more precision to settle
                        s["est"] = P + AGREE_BITS - d if d < AGREE_BITS else P + 64
                        s["nxt"] = s["est"]
                    elif s["hi"] == r["P_ref"]:
                        s["nxt"] = 2 * P
                    else:
                        s["nxt"] = (P + s["hi"]) // 2
            if log:
                log(f"round {rounds}: {len(active)} probes, {time.time() - t0:.1f}s")
        for i, s in state.items():
            recs[i]["bits"] = s["hi"]
        for r in recs:
            r.pop("lam_ref", None)
        return [dict(r, seconds=round(time.time() - t0, 1)) for r in recs]
    finally:
        if pool is not None:
            pool.close()
        if ctx is not None:
            hk.hk_destroy(ctx)


# ----- network ----------------------------------------------------------------

def features(N, beta):
    """(log2 N - 8, log2 beta)."""
    p, q = beta if isinstance(beta, (tuple, list)) else inputs.as_ratio(beta)
    return [math.log2(N) - 8.0, math.log2(p / q)]


def encode_targets(N, bits, log2_lambda, iters):
    """Network outputs: required bits above the 128-bit accuracy target per
    row, log2 lambda_min per row, log2 of the iteration count.  The method's
    data make the first two nearly independent of N for a fixed beta (the
    requirement grows linearly in N), so the network extrapolates in N
    without bending."""
    return [(bits - AGREE_BITS) / N, log2_lambda / N, math.log2(max(iters, 1))]


def decode_targets(N, y):
    return y[0] * N + AGREE_BITS, y[1] * N, 2.0 ** y[2]


class Predictor:
    """The 2 -> 64 -> 64 -> 3 network on the device, with the scalings above
    and standardisation of features and targets."""

    def __init__(self, params=None, x_mean=None, x_std=None, y_mean=None, y_std=None, margin_bits=32,
                 iter_factor=1.5, device=0, margin_per_row=0.0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        hk.lib()
        if params is None:
            params = self.init_params(0)
        self.params = torch.as_tensor(np.asarray(params, dtype=np.float32), device=self.dev).contiguous()
        self.x_mean = np.zeros(2) if x_mean is None else np.asarray(x_mean, dtype=np.float64)
        self.x_std = np.ones(2) if x_std is None else np.asarray(x_std, dtype=np.float64)
        self.y_mean = np.zeros(3) if y_mean is None else np.asarray(y_mean, dtype=np.float64)
        self.y_std = np.ones(3) if y_std is None else np.asarray(y_std, dtype=np.float64)
        self.margin_bits = margin_bits
        self.margin_per_row = margin_per_row
        self.iter_factor = iter_factor

    @staticmethod
    def init_params(seed):
        """Scaled normal initialisation (variance 1/fan_in), zero biases."""
        rng = np.random.default_rng(seed)
        parts = [rng.normal(0, 1 / math.sqrt(2), 128), np.zeros(64), rng.normal(0, 1 / 8, 4096), np.zeros(64),
                 rng.normal(0, 1 / 8, 192), np.zeros(3)]
        return np.concatenate(parts).astype(np.float32)

    def _x(self, rows):
        X = (np.asarray([features(N, b) for N, b in rows], dtype=np.float64) - self.x_mean) / self.x_std
        return self.torch.as_tensor(X.astype(np.float32), device=self.dev).contiguous()

    def fit(self, tuples, steps=4000, lr=3e-3, seed=0, log=None):
        """Full-batch Adam on the device over the usable tuples; returns the
        loss history (one value per step)."""
        torch = self.torch
        rows = [t for t in tuples if t.get("ok") and "bits" in t]
        F = np.asarray([features(t["N"], tuple(t["beta"])) for t in rows])
        Y = np.asarray([encode_targets(t["N"], t["bits"], t["log2_lambda"], t["iters"]) for t in rows])
        self.x_mean, self.x_std = F.mean(0), F.std(0) + 1e-12
        self.y_mean, self.y_std = Y.mean(0), Y.std(0) + 1e-12
        X = torch.as_tensor(((F - self.x_mean) / self.x_std).astype(np.float32), device=self.dev).contiguous()
        T = torch.as_tensor(((Y - self.y_mean) / self.y_std).astype(np.float32), device=self.dev).contiguous()
        w = torch.ones(3, dtype=torch.float32, device=self.dev)
        self.params = torch.as_tensor(self.init_params(seed), device=self.dev).contiguous()
        m = torch.zeros_like(self.params)
        v = torch.zeros_like(self.params)
        grad = torch.zeros_like(self.params)
        work = torch.empty(hk.hk_mlp_workspace_bytes(len(rows)), dtype=torch.uint8, device=self.dev)
        hist = torch.zeros(steps, dtype=torch.float32, device=self.dev)
        # step schedule: lr, lr/3, lr/10 over the three thirds
        done = 0
        for k, f in enumerate((1.0, 1 / 3, 1 / 10)):
            n = steps // 3 if k < 2 else steps - 2 * (steps // 3)
            hk.hk_mlp_train(self.params, m, v, grad, X, T, w, n, done, lr * f, work, hist[done:])
            done += n
        torch.cuda.synchronize()
        h = hist.cpu().numpy()
        # margin: 32 bits plus, per row, the largest relative under-prediction
        # of the training set (errors grow with N like the requirement itself)
        pred = self.predict_raw([(t["N"], tuple(t["beta"])) for t in rows])
        under = [(t["bits"] - b) / t["N"] for t, (b, _, _) in zip(rows, pred)]
        self.margin_bits = 32
        self.margin_per_row = max(0.0, max(under))
        if log:
            log(f"fit: {len(rows)} tuples, loss {h[0]:.4g} -> {h[-1]:.4g}, margin 32 bits + "
                f"{self.margin_per_row:.3f} bits per row")
        return h

    def predict_raw(self, rows):
        """Decoded network outputs (bits, log2 lambda, iterations) per (N, beta)."""
        torch = self.torch
        X = self._x(rows)
        y = torch.zeros(len(rows), 3, dtype=torch.float32, device=self.dev)
        hk.hk_mlp_forward(self.params, X, y)
        Y = y.cpu().numpy().astype(np.float64) * self.y_std + self.y_mean
        return [decode_targets(N, Y[k]) for k, (N, _) in enumerate(rows)]

    def predict(self, N, beta):
        """(P, iteration budget, log2 lambda_min estimate) for one instance."""
        bits, l2, it = self.predict_raw([(N, beta)])[0]
        P = max(P_MIN, _ceil32(bits + self.margin_bits + self.margin_per_row * N))
        P = min(P, p_conservative(N, beta))
        T = int(min(MAX_ITERS, max(8, math.ceil(it * self.iter_factor) + 4)))
        return P, T, l2

    def to_json(self):
        return dict(params=[float(x) for x in self.params.cpu().numpy()], x_mean=list(self.x_mean),
                    x_std=list(self.x_std), y_mean=list(self.y_mean), y_std=list(self.y_std),
                    margin_bits=self.margin_bits, margin_per_row=self.margin_per_row,
                    iter_factor=self.iter_factor, targets="(bits-128)/N, log2(lambda)/N, log2(iters)")

    @classmethod
    def from_json(cls, d, device=0):
        return cls(d["params"], d["x_mean"], d["x_std"], d["y_mean"], d["y_std"], d["margin_bits"],
                   d["iter_factor"], device, d.get("margin_per_row", 0.0))


# ----- verified solves ----------------------------------------------------------

def _solve_one(h, N, beta, P, T):
    """(lambda or None, iterations, converged, library seconds) of one solve;
    the host-side moment generation is not timed."""
    m = inputs.moments(N, beta, P)
    t0 = time.perf_counter()
    h.load(N, beta, P, m)
    try:
        h.factor()
    except hk.HKError as e:
        if e.code == hk.HK_ERR_NOT_PD:
            return None, 0, False, time.perf_counter() - t0
        raise
    hk.hk_set_option(h.ctx, hk.HK_OPT_MAX_ITERS, T)
    lam, used = h.smallest_eig(0)
    conv = bool(h.stats()["converged"])
    return lam, used, conv, time.perf_counter() - t0


def _solve_loaded(h, N, beta, P, m, T):
    """_solve_one with the moments already generated."""
    t0 = time.perf_counter()
    h.load(N, beta, P, m)
    try:
        h.factor()
    except hk.HKError as e:
        if e.code == hk.HK_ERR_NOT_PD:
            return None, 0, False, time.perf_counter() - t0
        raise
    hk.hk_set_option(h.ctx, hk.HK_OPT_MAX_ITERS, T)
    lam, used = h.smallest_eig(0)
    conv = bool(h.stats()["converged"])
    return lam, used, conv, time.perf_counter() - t0


def _solve_pair(N, beta, Ps, T):
    """Independent solves at the precisions Ps at the same time: one context
    per precision on its own non-blocking stream, driven by its own host
    thread (the library calls release the interpreter lock), so that the
    sequential per-row kernels of one overlap the other's.  Moments are
    generated first, outside the timed span.  Returns the per-solve results
    and the wall time of the pair."""
    import threading
    import torch
    ms = [inputs.moments(N, beta, P) for P in Ps]
    streams = [torch.cuda.Stream() for _ in Ps]
    hs = [hk.Hankel(0, st) for st in streams]
    out = [None] * len(Ps)
    err = []

    def run(k):
        try:
            out[k] = _solve_loaded(hs[k], N, beta, Ps[k], ms[k], T)
        except Exception as e:  # re-raised in the caller's thread
            err.append(e)

    try:
        t0 = time.perf_counter()
        ths = [threading.Thread(target=run, args=(k,)) for k in range(len(Ps))]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        wall = time.perf_counter() - t0
    finally:
        for h in hs:
            h.close()
    if err:
        raise err[0]
    return out, wall


def solve_conservative(N, beta, T=MAX_ITERS):
    """The method without the predictor: one solve at the conservative P."""
    P = p_conservative(N, beta)
    with hk.Hankel(0) as h:
        lam, used, conv, sec = _solve_one(h, N, beta, P, T)
    return dict(lam=lam, P=P, iters=used, converged=conv, seconds=sec)


def solve_verified(N, beta, predictor=None, P=None, T=MAX_ITERS, max_escalations=8):
    """lambda_min of one instance at a verified precision.

    With a predictor, P and the iteration budget T come from it; otherwise P
    defaults to the conservative rule.  The solve at P is accepted when a
    rerun at P + 1024 converges to a value within 2^-128 (relative) of it;
    otherwise P grows by 1024 (and T doubles when the iteration did not
    converge) and the check repeats.  The first solve and its check run at the
    same time on two streams.  Returns a dict with the accepted lambda (the
    P + 1024 value), the precisions tried and the seconds spent in the library
    (wall time; moment generation excluded)."""
    if predictor is not None:
        P, T, _ = predictor.predict(N, beta)
    elif P is None:
        P = p_conservative(N, beta)
    tried = []
    sec = 0.0
    # the solve at P and its check at P + DELTA are independent: run them at
    # the same time (wall time counted once)
    (lo, hi0), wall = _solve_pair(N, beta, [P, P + DELTA], T)
    sec += wall
    tried.append(P)
    with hk.Hankel(0) as h:
        for rnd in range(max_escalations + 1):
            if rnd == 0:
                hi = hi0
            else:
                hi = _solve_one(h, N, beta, P + DELTA, T)
                sec += hi[3]
            tried.append(P + DELTA)
            if lo[0] is not None and hi[0] is not None and lo[2] and hi[2]:
                if rel_err_bits(lo[0], hi[0]) >= AGREE_BITS:
                    return dict(lam=hi[0], P=P, iters=hi[1], tried=tried, seconds=sec, verified=True, T=T)
            elif lo[0] is not None and hi[0] is not None and T < 100000:
                # both factorisations succeeded but an iteration hit its budget:
                # larger budget, same precisions
                T = min(100000, 2 * T)
                lo = _solve_one(h, N, beta, P, T)
                sec += lo[3]
                tried.append(P)
                continue
            P += DELTA
            lo = hi
    return dict(lam=lo[0], P=P, iters=lo[1], tried=tried, seconds=sec, verified=False, T=T)


def load_default(device=0):
    """The predictor trained on the committed method-generated tuples."""
    path = os.path.join(os.path.dirname(__file__), "data", "predictor.json")
    with open(path) as f:
        return Predictor.from_json(json.load(f), device)
