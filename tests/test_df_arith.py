"""The double-float operations the true-residual kernel is built from (lqcd_common.cuh: sum by
TwoSum plus the low parts, product by the FMA TwoProduct), compiled for the host and checked with
exact rational arithmetic: the sum errs by at most 2^-45 (|x| + |y|), the product and the fused
multiply-add by 2^-44 of the magnitudes of their terms.  These are the bounds the residual's
accuracy claim (about 1e-13 of ||b|| + ||D|| ||x||) rests on."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def df_program(tmp_path_factory):
    if not os.path.exists(NVCC) and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("df") / "df_arith")
    subprocess.run([NVCC if os.path.exists(NVCC) else "nvcc", "-std=c++17", "-O2",
                    "-I" + os.path.join(ROOT, "paper_2609_37049_b300", "csrc"), "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "host", "df_arith.cu"), "-o", exe], check=True, capture_output=True)
    return exe


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(-1, 1, size=(n, 3))
    expo = rng.integers(-30, 30, size=(n, 3))
    v = mant * np.exp2(expo)
    # cancellation-heavy cases: y close to -x, z close to -x y
    v[: n // 4, 1] = -v[: n // 4, 0] * (1 + rng.uniform(-1e-7, 1e-7, n // 4))
    v[n // 4: n // 2, 2] = -v[n // 4: n // 2, 0] * v[n // 4: n // 2, 1] * (1 + rng.uniform(-1e-6, 1e-6, n // 4))
    return v


def test_double_float_sum_product_fma_error_bounds(df_program):
    v = _cases(400, 2401)
    inp = "\n".join(" ".join(repr(float(x)) for x in r) for r in v) + "\n"
    out = subprocess.run([df_program], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [list(map(float, line.split())) for line in out if line.strip()]
    assert len(rows) == len(v)
    F = lambda h, l: Fraction(h) + Fraction(l)  # noqa: E731  exact value of a (hi, lo) pair
    for r in rows:
        x, y, z = F(r[0], r[1]), F(r[2], r[3]), F(r[4], r[5])
        s, p, f = F(r[6], r[7]), F(r[8], r[9]), F(r[10], r[11])
        assert abs(s - (x + y)) <= Fraction(1, 2 ** 45) * (abs(x) + abs(y))
        assert abs(p - x * y) <= Fraction(1, 2 ** 44) * abs(x * y)
        assert abs(f - (x * y + z)) <= Fraction(1, 2 ** 44) * (abs(x * y) + abs(z))
