"""Sampled-row check of a factor R against the oracle, usable at sizes the full
oracle cannot reach: row i of R is recomputed by the oracle's own row routine
(oracle.cholesky_row) from R's rows above it, and must equal R's row i bit for
bit.  By induction over the rows this checks exactly what a full comparison
checks for the sampled rows: every rounding step given the finished rows."""
import oracle


def check_rows(moments, R, P, rows, max_cols=None):
    """Return a list of (i, j) where R differs from the oracle's recomputation
    (empty when every sampled entry agrees).  ``R[t][j - t]`` = R_tj."""
    N = len(R)
    bad = []
    for i in rows:
        js = list(range(i, N)) if max_cols is None else list(range(i, min(N, i + max_cols)))
        col_i = [R[t][i - t] for t in range(i)]
        cols = {j: [R[t][j - t] for t in range(i)] for j in js}
        want = oracle.cholesky_row(i, moments, col_i, cols, P)
        bad += [(i, j) for j in js if want[j] != R[i][j - i]]
    return bad


# ---------------------------------------------------------------------------
# full-width rows of a large factor held as flat arrays (the C ABI's packed
# layout), checked in parallel over columns by spawn-started processes
# ---------------------------------------------------------------------------

def _tri(t, j, N):
    return t * N - (t * (t - 1)) // 2 + (j - t)


def _decode(sign, exp, raw, L, k):
    n = int.from_bytes(raw[4 * L * k: 4 * L * (k + 1)], "little")
    if n == 0:
        return (0, 0)
    return (-n if sign[k] else n, int(exp[k]))


def _chunk_task(args):
    """One share of the columns of row i: the oracle's row routine from the
    rows above, compared with the factor's own row i.  Inputs arrive as the
    packed bytes of exactly the entries used."""
    i, js, moments, P, sign, exp, raw = args
    L = P // 32
    # entry order: column i (t < i), then for each j: column j (t < i), R_ij
    k = 0
    col_i = []
    for _ in range(i):
        col_i.append(_decode(sign, exp, raw, L, k))
        k += 1
    cols, have = {}, {}
    for j in js:
        c = []
        for _ in range(i):
            c.append(_decode(sign, exp, raw, L, k))
            k += 1
        cols[j] = c
        have[j] = _decode(sign, exp, raw, L, k)
        k += 1
    want = oracle.cholesky_row(i, moments, col_i, cols, P)
    return [(i, j) for j in js if want[j] != have[j]]


def check_rows_flat(moments, sign, exp, limbs, N, P, rows, workers):
    """Like ``check_rows`` for every column of each sampled row, on a factor
    given as the flat arrays of ``hk_get_R_flat`` (sign int32, exp int64,
    limbs uint32 [entries][L]).  Returns the (i, j) that differ."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import numpy as np
    tasks = []
    for i in rows:
        js = list(range(i, N))
        nch = max(1, min(workers, len(js)))
        for c in range(nch):
            part = js[c::nch]
            idx = [_tri(t, i, N) for t in range(i)]
            for j in part:
                idx += [_tri(t, j, N) for t in range(i)]
                idx.append(_tri(i, j, N))
            ix = np.asarray(idx, dtype=np.int64)
            tasks.append((i, part, moments, P, sign[ix].copy(), exp[ix].copy(),
                          np.ascontiguousarray(limbs[ix]).tobytes()))
    bad = []
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
        for r in pool.map(_chunk_task, tasks):
            bad += r
    return bad
