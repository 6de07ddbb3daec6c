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
