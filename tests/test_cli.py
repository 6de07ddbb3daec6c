"""The command line (python -m paper_0902_0852_gb300): help and argument
errors without a GPU, and the decimal rendering of a P-bit value."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, "-m", "paper_0902_0852_gb300", *args], capture_output=True, text=True,
                          cwd=ROOT, timeout=120)


def test_help_and_argument_errors():
    r = _run("--help")
    assert r.returncode == 0 and "--beta" in r.stdout
    for bad in (["--N", "0"], ["--N", "10", "--P", "100"], ["--N", "10", "--beta", "-1/2"],
                ["--N", "10", "--beta", "x"], ["--N", "10", "--P", "256", "--conservative"], []):
        r = _run(*bad)
        assert r.returncode == 2, (bad, r.stderr)


def test_decimal_rendering():
    from paper_0902_0852_gb300.__main__ import decimal
    assert decimal((1 << 31, -31)) == "1.00000000000e0"
    assert decimal((0, 0)) == "0"
    assert decimal((-3 << 30, -30)) == "-3.00000000000e0"
    # lambda_min at N = 1000, beta = 1 (Table 3: 1.0892e-52) as an exact dyadic
    from fractions import Fraction
    x = Fraction(10892, 10 ** 56)
    e = x.numerator.bit_length() - x.denominator.bit_length() - 64
    n = round(x / Fraction(2) ** e)
    assert decimal((n, e)).startswith("1.0892")
