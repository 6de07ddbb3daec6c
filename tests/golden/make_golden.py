"""Writes the stored expected values of the larger parity cases.

Every value here comes from the CPU oracle (oracle/), run on the seeded
moments of the input generator: a SHA-256 digest of R in the C-ABI's packed
layout (sign int32, exp int64, L little-endian limbs per entry, entries in
row-major packed upper-triangle order) and the inverse-iteration history
lambda_1..lambda_T as (mantissa, exponent) pairs.

Usage: python tests/golden/make_golden.py [workers] [case names ...]
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

CASES = [
    # name, N, beta, P, T
    ("config2_beta1", 256, (1, 1), 8192, 10),
    ("config2_beta7_4", 256, (7, 4), 8192, 10),
    # the paper-scale factorial matrix: every step of the factorisation is exact
    # at this P, so the oracle's factor is its closed form (cholesky_factorial)
    ("paper_scale_beta1", 1000, (1, 1), 24576, 3),
    # Table 3 cells whose moments grow fastest (exact factorials 3 (3k+2)! and
    # 2 (2k+1)!), at the precision the cells run at (32 ceil((3.5 N + 512)/32))
    ("cell_N500_beta1_3", 500, (1, 3), 2272, 3),
    ("cell_N500_beta1_2", 500, (1, 2), 2272, 3),
]


def digest_R(R, P):
    L = P // 32
    h = hashlib.sha256()
    for row in R:
        for n, e in row:
            a = -n if n < 0 else n
            h.update((1 if n < 0 else 0).to_bytes(4, "little", signed=True))
            h.update(int(e).to_bytes(8, "little", signed=True))
            h.update(a.to_bytes(4 * L, "little"))
    return h.hexdigest()


def main():
    import oracle
    sys.set_int_max_str_digits(0)  # mantissas of up to 32768 bits as decimal strings
    from paper_0902_0852_gb300 import inputs
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    only = set(sys.argv[2:])
    for name, N, beta, P, T in CASES:
        if only and name not in only:
            continue
        if beta == (1, 1) and N >= 1000:
            R = oracle.cholesky_factorial(N, P)
        else:
            m = inputs.moments(N, beta, P)
            R = oracle.cholesky(m, N, P, workers=workers)
        lam, hist, _ = oracle.inverse_iteration(R, P, T)
        out = {"N": N, "beta": list(beta), "P": P, "T": T, "R_sha256": digest_R(R, P),
               "history": [[str(n), e] for n, e in hist]}
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}.json")
        with open(path, "w") as f:
            json.dump(out, f)
        print(name, "done", flush=True)


if __name__ == "__main__":
    main()
