"""Command line: lambda_min of one Hankel moment matrix on the GPU.

    python -m paper_0902_0852_gb300 --N 500 --beta 7/4             # predicted P
    python -m paper_0902_0852_gb300 --N 500 --beta 7/4 --P 12288   # given P
    python -m paper_0902_0852_gb300 --N 500 --beta 7/4 --conservative

The matrix is M_ij = m_{i+j} with m_k = Gamma((1+k)/beta)/beta; beta = p/q
with p in {1, 2, 3, 4, 5, 7} (the Gamma constants the moment generator holds).
Every answer is verified: the solve at P is accepted when a rerun at P + 1024
agrees to 2^-128 (relative), else P grows by 1024.  Prints one JSON line and
exits 0 when the answer was verified, 1 when it was not.
"""
import argparse
import json
import math
from fractions import Fraction


def _beta(s):
    try:
        fr = Fraction(s)
    except (ValueError, ZeroDivisionError):
        raise argparse.ArgumentTypeError(f"not a ratio: {s!r}")
    if fr <= 0:
        raise argparse.ArgumentTypeError("beta must be positive")
    return fr.numerator, fr.denominator


def decimal(lam, digits=12):
    """A P-bit value (n, e) = n 2^e as a decimal string with `digits`
    significant digits."""
    n, e = lam
    if n == 0:
        return "0"
    lg = math.log10(abs(n)) + e * math.log10(2)
    ex = math.floor(lg)
    return f"{'-' if n < 0 else ''}{10 ** (lg - ex):.{digits - 1}f}e{ex}"


def parse(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_0902_0852_gb300",
                                 description="Smallest eigenvalue of the Hankel moment matrix of order N.")
    ap.add_argument("--N", type=int, required=True, help="matrix order (>= 1)")
    ap.add_argument("--beta", type=_beta, default=(1, 1), help="beta as p/q, e.g. 7/4 (default 1)")
    g = ap.add_mutually_exclusive_group()
    g.add_argument("--P", type=int, help="working precision in bits, a multiple of 32 (default: predicted)")
    g.add_argument("--conservative", action="store_true",
                   help="start at the conservative precision rule instead of the predictor")
    args = ap.parse_args(argv)
    if args.N < 1:
        ap.error("--N must be at least 1")
    if args.P is not None and (args.P < 32 or args.P % 32):
        ap.error("--P must be a positive multiple of 32")
    return args


def main(argv=None):
    args = parse(argv)
    from . import predictor as pr
    model = None if (args.P is not None or args.conservative) else pr.load_default()
    r = pr.solve_verified(args.N, args.beta, model, P=args.P)
    lam = r["lam"]
    out = {
        "N": args.N, "beta": f"{args.beta[0]}/{args.beta[1]}", "P": r["P"],
        "lambda_min": None if lam is None else decimal(lam),
        "lambda_min_exact": None if lam is None else {"mantissa": str(lam[0]), "exp2": lam[1]},
        "iterations": r["iters"], "verified": r["verified"], "precisions_run": r["tried"],
        "seconds": round(r["seconds"], 4),
        "precision_source": "given" if args.P is not None else ("conservative" if args.conservative else "predicted"),
    }
    print(json.dumps(out))
    return 0 if r["verified"] else 1


if __name__ == "__main__":
    raise SystemExit(main())
