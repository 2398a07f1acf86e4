"""CPU pin of the key-product accumulation the throughput kernel uses (the MAC of
"TGSW BK_i x TLWE temp", Fig. 2).  Per coefficient, a warp adds the products
x_r b_r of its TGSW rows r, with x_r the forward-transform output (below 22q,
the lazy transform's bound) and b_r the NTT-domain key word (fully reduced,
below q, the Montgomery factor 2^32 folded in).  Two forms are in use:

- per product: mont_mul(x, b) = (x b + m q) / 2^32 with m = (x b mod 2^32)(-q^-1)
  mod 2^32, each in [0, 2q), summed in 32 bits (below 12q for six rows);
- exact sum: T = sum_r x_r b_r kept in 64 bits (two 32-bit words added with a
  carry chain in the twelve-warp shapes, whose sums live in tensor memory), then
  one reduction mont_redc(T) = (T + m q) / 2^32, m from the low word of T.

Both must give the same residue T 2^-32 mod q, the 64-bit sum must not wrap,
and the result must stay below the 12q the inverse transform's first stage
assumes, for both gadgets (six rows for l = 3, four for l = 2) and for every
split of the rows over H warps whose partial results an owner warp adds.  The
primes are read from the kernels' header; Python integers do the arithmetic."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M32 = 1 << 32


def primes():
    text = open(os.path.join(ROOT, "paper_2306_11006_gb300", "csrc", "arx_kernels.h")).read()
    q0 = int(re.search(r"kQ0\s*=\s*(\d+)u", text).group(1))
    q1 = int(re.search(r"kQ1\s*=\s*(\d+)u", text).group(1))
    return q0, q1


def qni(q):
    return (-pow(q, -1, M32)) % M32


def mont_mul(x, b, q):
    t = x * b
    m = (t % M32) * qni(q) % M32
    assert (t + m * q) % M32 == 0
    return (t + m * q) >> 32


def mont_redc(t, q):
    m = (t % M32) * qni(q) % M32
    s = t + m * q
    assert s < 1 << 64 and s % M32 == 0
    return s >> 32


def carry_chain_add(lo, hi, x, b):
    """mad.lo.cc.u32 lo, x, b, lo; madc.hi.u32 hi, x, b, hi -- on 32-bit words."""
    p = x * b
    s = lo + p % M32
    return s % M32, (hi + p // M32 + s // M32) % M32


def accumulate(xs, bs):
    lo = hi = 0
    for x, b in zip(xs, bs):
        lo, hi = carry_chain_add(lo, hi, x, b)
    return (hi << 32) | lo


@pytest.mark.parametrize("rows", [6, 4])  # 2l TGSW rows: l = 3 and l = 2
def test_exact_sum_matches_per_product_montgomery(rows):
    rng = np.random.default_rng(rows)
    for q in primes():
        xmax, bmax = 22 * q - 1, q - 1
        cases = [([xmax] * rows, [bmax] * rows), ([0] * rows, [bmax] * rows), ([xmax] * rows, [0] * rows)]
        cases += [([int(v) for v in rng.integers(0, 22 * q, rows)], [int(v) for v in rng.integers(0, q, rows)])
                  for _ in range(2000)]
        for xs, bs in cases:
            t = accumulate(xs, bs)
            assert t == sum(x * b for x, b in zip(xs, bs))  # the carry chain is the exact 64-bit sum
            assert t < 1 << 62
            wide = mont_redc(t, q)
            narrow = sum(mont_mul(x, b, q) for x, b in zip(xs, bs))
            assert all(mont_mul(x, b, q) < 2 * q for x, b in zip(xs, bs))
            assert wide % q == narrow % q == t * pow(M32, -1, q) % q
            assert wide < t / M32 + q and narrow < 2 * q * rows <= 12 * q


@pytest.mark.parametrize("rows,warps", [(6, 1), (6, 2), (6, 3), (4, 1), (4, 2), (4, 4)])
def test_partial_sums_of_split_rows_stay_below_the_inverse_bound(rows, warps):
    """H warps take rows / H rows each, reduce their exact sums, and an owner warp
    adds the H results: the worst case stays below 7.2q, inside the 8q input bound
    the inverse's first stage assumes for these shapes (the throughput shapes with
    H = 1, 2, 3 for l = 3 and H = 1, 2, 4 for l = 2)."""
    for q in primes():
        per = rows // warps
        worst_partial = mont_redc(per * (22 * q - 1) * (q - 1), q)
        bound = per * 22 * q * q / M32 + q
        assert worst_partial < bound
        assert warps * bound < 7.2 * q < 8 * q
        assert 6 * 22 * q * q < 5.2 * q * M32 - q * M32  # six rows reduce below 5.2q (the comment in the kernel)


def test_per_product_montgomery_sums_stay_below_12q():
    """The one-row-per-warp shape (H = 6) reduces every product and adds six of
    them in its owner warp: below 12q, the first stage's other input bound."""
    for q in primes():
        worst = sum(mont_mul(22 * q - 1, b, q) for b in (q - 1, q - 2, 1, 12345, q // 2, q - 3))
        assert worst < 6 * 2 * q == 12 * q
        assert max(mont_mul(x, q - 1, q) for x in (22 * q - 1, 0, 1, q, 2 * q + 7)) < 2 * q


@pytest.mark.parametrize("bound", [2, 8, 12])
def test_first_inverse_stage_reduces_to_2q(bound):
    """The inverse's Gentleman-Sande butterfly as the kernel states it: inputs below
    bound * q; the sum reduced by conditional subtractions of 16q (bound 12 only),
    8q and 4q (bounds 8 and 12) and a last one of 2q lands in [0, 2q); the
    difference x - y + bound q stays in (0, 2^32)."""
    rng = np.random.default_rng(bound)
    for q in primes():
        def csub(v, m):
            return min(v, (v - m) % M32)
        xs = [0, 1, bound * q - 1] + [int(v) for v in rng.integers(0, bound * q, 3000)]
        ys = [bound * q - 1, 0, bound * q - 1] + [int(v) for v in rng.integers(0, bound * q, 3000)]
        for x, y in zip(xs, ys):
            s = (x + y) % M32
            assert s == x + y  # no wrap
            if bound == 12:
                s = csub(s, 16 * q)
            if bound >= 8:
                s = csub(s, 8 * q)
                s = csub(s, 4 * q)
            s = csub(s, 2 * q)
            assert s < 2 * q and s % q == (x + y) % q
            d = x - y + bound * q
            assert 0 < d < M32 and d % q == (x - y) % q
