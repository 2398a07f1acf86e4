"""CPU pin of the CRT recombination the blind-rotation kernels use (crt_torus in
the CUDA sources): an exact external-product coefficient V is carried modulo the
two 27-bit primes q0, q1 and recombined by Garner's formula, with each residue
anywhere in [0, 2q) (lazy reduction).  That is exact only while |V| stays below
the margin the sign test needs; this checks the worst cases of both gadgets --
l = 3, Bg = 2^7 (6 rows x 1024 terms x 64 x 2^31 < 2^50) and the paper's l = 2,
Bg = 2^10 (4 x 1024 x 512 x 2^31 = 2^52) -- with Python integers: every digit at
its extreme and every key coefficient at +-2^31, plus values around 0, +-q0 and
random ones.  The primes are read from the kernels' header."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def primes():
    text = open(os.path.join(ROOT, "paper_2306_11006_gb300", "csrc", "arx_kernels.h")).read()
    q0 = int(re.search(r"kQ0\s*=\s*(\d+)u", text).group(1))
    q1 = int(re.search(r"kQ1\s*=\s*(\d+)u", text).group(1))
    return q0, q1


def garner_torus(x0, x1, q0, q1):
    """The recombination as the kernels state it, in exact integers: d = x1 + 3 q1
    - x0 (a u32), k = d q0^-1 mod q1, r = q0 k + x0, and r - q0 q1 when k >= q1 / 2;
    all mod 2^32."""
    M32 = 1 << 32
    d = (x1 + 3 * q1 - x0) % M32
    assert 0 < d < M32  # no wrap for x0 < 2 q0, x1 < 2 q1
    k = d * pow(q0, -1, q1) % q1
    r = (q0 * k + x0) % M32
    return (r - q0 * q1) % M32 if k >= q1 // 2 else r


def lazy_residues(v, q):
    """Both representatives of v mod q in [0, 2q)."""
    x = v % q
    return [x, x + q]


@pytest.mark.parametrize("rows,digit_bound", [(6, 64), (4, 512)])  # (2l, Bg/2): l = 3 and l = 2
def test_worst_case_products_recombine_exactly(rows, digit_bound):
    q0, q1 = primes()
    assert q0 % 2048 == 1 and q1 % 2048 == 1 and 32 * max(q0, q1) < 1 << 32
    N = 1024
    worst = rows * N * digit_bound * (1 << 31)
    assert worst < q0 * q1 // 2
    # the extremes: digits all -Bg/2, key coefficients all -2^31 (sum +worst) or +2^31 (sum -worst)
    dig = np.full(N, -digit_bound, dtype=object)
    for key in (-(1 << 31), (1 << 31) - 1, 1 << 31):
        v = rows * int(np.sum(dig * key))
        assert abs(v) <= worst
    rng = np.random.default_rng(rows)
    values = [worst, -worst, 0, 1, -1, q0 - 1, q0, q0 + 1, -q0, -q0 - 1, worst - q0, -worst + q0]
    values += [int(x) for x in rng.integers(-worst, worst, 2000, dtype=np.int64)]
    for v in values:
        for x0 in lazy_residues(v, q0):
            for x1 in lazy_residues(v, q1):
                assert garner_torus(x0, x1, q0, q1) == v % (1 << 32), (v, x0, x1)


def test_sign_test_margin_is_what_the_comment_states():
    q0, q1 = primes()
    for rows, digit_bound, kmax in [(6, 64, 1 << 23), (4, 512, (1 << 25) + (1 << 12))]:
        worst = rows * 1024 * digit_bound * (1 << 31)
        assert worst // q0 < kmax < q1 // 2
