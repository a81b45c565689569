"""The float-float arithmetic the mixed form's FP64-class kernels execute (csrc/ff.cuh: sums
from TwoSum / FastTwoSum, products with the exact FMA error term, one-correction division,
the compensated Dot2 dot product), compiled for the host from the same header and
checked against exact rational arithmetic on seeded operands of mixed magnitudes and signs,
near cancellations included.  u = 2^-24 is the FP32 unit roundoff; a float-float result is
hi + lo with hi the FP32 rounding of hi + lo (normalised).  Bounds, in units of u^2 = 2^-48:
  a + b:  |r - (a + b)| <= 4 u^2 (|a| + |b|)
  a * b:  |r - ab| <= 5 u^2 |ab|
  a / b:  |r - a/b| <= 10 u^2 |a/b|
  dot of k terms: |r - sum m_i v_i| <= (3 + k) u^2 sum |m_i v_i|
(the measured maxima are about 1.9, 2.8, 4.5 and 3 + k/2).  A dropped cross term, a lost
error term or a sign slip in any of them gives errors of order u, about 2^24 times these."""
import os
import shutil
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_04167_gb300", "csrc")
U2 = F(1, 2 ** 48)


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("ffa") / "ff_arith_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-x", "cu", os.path.join(HERE, "native", "ff_arith_check.cu"),
                    "-o", exe], check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe, "3000"], capture_output=True, text=True, timeout=120, check=True)
    return [ln.split() for ln in r.stdout.splitlines()]


def _ff(h, l):
    return F(float.fromhex(h)) + F(float.fromhex(l))


def _normalised(h, l):
    hi, lo = np.float32(float.fromhex(h)), np.float32(float.fromhex(l))
    return np.float32(hi + lo) == hi


@pytest.mark.parametrize("op,bound", [("add", 4), ("mul", 5), ("div", 10)])
def test_binary_operations(lines, op, bound):
    worst, n = 0.0, 0
    for f in lines:
        if f[0] != op:
            continue
        a, b, r = _ff(f[1], f[2]), _ff(f[3], f[4]), _ff(f[5], f[6])
        assert _normalised(f[5], f[6]), f
        if op == "add":
            exact, scale = a + b, abs(a) + abs(b)
        elif op == "mul":
            exact = a * b
            scale = abs(exact)
        else:
            exact = a / b
            scale = abs(exact)
        ratio = float(abs(r - exact) / (U2 * scale))
        assert ratio <= bound, (op, f, ratio)
        worst, n = max(worst, ratio), n + 1
    assert n == 3000 and worst > 0.1            # the operands do exercise the rounding


def test_compensated_dot(lines):
    n = 0
    for f in lines:
        if f[0] != "dot":
            continue
        k = int(f[1])
        terms = [_ff(f[2 + 4 * j], f[3 + 4 * j]) * _ff(f[4 + 4 * j], f[5 + 4 * j]) for j in range(k)]
        r = _ff(f[-2], f[-1])
        assert _normalised(f[-2], f[-1]), f
        ratio = float(abs(r - sum(terms)) / (U2 * sum(abs(t) for t in terms)))
        assert ratio <= 3 + k, (k, ratio)
        n += 1
    assert n == 750
