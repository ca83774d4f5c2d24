"""The double-FP32 primitives of csrc/df.cuh, run on the host (no GPU) and
checked with exact rational arithmetic: two_sum, fast_two_sum and two_prod
are error-free (Knuth; Dekker with an FMA), and df_from, df_add, df_mul
and the renormalised dot-product accumulation stay within the bounds the
header states (2^-48 relative, 2^-47 (|a| + |b|), 2^-46 |a b|, and
(n + 4) 2^-46 sum |a_i b_i| for n terms).  The FP64-accurate Legendre
kernels are built from exactly these functions."""
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("dfhost") / "df_host_check"
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_2306_15511_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "df_host_check.cu"), "-o", str(out)])
    res = subprocess.run([str(out)], check=True, capture_output=True, text=True)
    return [ln.split() for ln in res.stdout.splitlines() if ln.strip()]


def _vals(t):
    return [Fr(float.fromhex(x)) for x in t]


def test_error_free_transformations(lines):
    n = 0
    for t in lines:
        if t[0] in ("two_sum", "fast_two_sum"):
            a, b, s, e = _vals(t[1:])
            assert s + e == a + b, t
            n += 1
        elif t[0] == "two_prod":
            a, b, p, e = _vals(t[1:])
            assert p + e == a * b, t
            n += 1
    assert n == 3 * 4000


def test_conversions_and_arithmetic_bounds(lines):
    u = Fr(1, 2 ** 46)
    n = 0
    for t in lines:
        if t[0] == "from":
            x, h, l = _vals(t[1:])
            assert abs(h + l - x) <= abs(x) * u / 4, t
        elif t[0] == "to":
            h, l, d = _vals(t[1:])
            assert abs(d - (h + l)) <= abs(h + l) * Fr(1, 2 ** 53), t
        elif t[0] in ("add", "mul"):
            ah, al, bh, bl, rh, rl = _vals(t[1:])
            a, b, r = ah + al, bh + bl, rh + rl
            if t[0] == "add":
                assert abs(r - (a + b)) <= (abs(a) + abs(b)) * u / 2, t
            else:
                assert abs(r - a * b) <= abs(a * b) * u, t
            n += 1
    assert n == 2 * 4000


def test_dot_product_accumulation(lines):
    u = Fr(1, 2 ** 46)
    dots = [t for t in lines if t[0] == "dot"]
    assert len(dots) == 200
    for t in dots:
        k = int(t[1])
        v = _vals(t[2:])
        terms = [(v[4 * i] + v[4 * i + 1]) * (v[4 * i + 2] + v[4 * i + 3]) for i in range(k)]
        got = v[4 * k] + v[4 * k + 1]
        assert abs(got - sum(terms)) <= (k + 4) * u * sum(abs(x) for x in terms), k
