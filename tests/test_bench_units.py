"""CPU pins of the per-unit work the benchmark's roofline divides by, and of its
wave slicing for the oracle arm.

One CMux (Fig. 2) costs (k+1) l forward and k+1 inverse transforms of N/2 log2 N
butterflies each, and (k+1)^2 l N key products (the MAC), with k = 1, N = 1024:
at one 64-bit modulus that is n [(2l + 2) 5120 + 4 l 1024] modular products per
bootstrap -- 33,546,240 for n = 630, l = 3 -- and the two-prime CRT form
carried here doubles it.  The bench's modmul_per_cmux must equal that count for
both gadgets, written out here from the transform and MAC sizes, and its integer
peak must be 152 SMs x 2.07 GHz x 64 lanes / 3 lane slots per product."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def products_per_cmux(l: int, N: int = 1024, k: int = 1, primes: int = 2) -> int:
    butterflies = N // 2 * int(math.log2(N))
    transforms = (k + 1) * l + (k + 1)
    mac = (k + 1) ** 2 * l * N
    return primes * (transforms * butterflies + mac)


@pytest.mark.parametrize("l", [3, 2])
def test_modmul_per_cmux_is_the_transform_and_mac_count(l):
    assert bench.modmul_per_cmux(l) == products_per_cmux(l)


def test_per_bootstrap_work_at_one_modulus():
    assert 630 * products_per_cmux(3, primes=1) == 33_546_240
    assert bench.MODMUL_PER_CMUX * bench.LWE_N == 2 * 33_546_240


def test_alu_peak():
    assert bench.ALU_PEAK_TMODMUL == pytest.approx(152 * 2.07 * 64 / 3 / 1e3)


@pytest.mark.parametrize("k", [1, 3, 20, 65])
def test_wave_slices_cover_every_wave_once_in_order(k):
    waves = np.repeat(np.arange(65), 7)
    slices = list(bench.wave_slices(waves, k))
    got = np.concatenate([np.asarray(s) for s in slices if len(s)]) if slices else np.array([])
    assert len(slices) == k
    assert np.array_equal(np.sort(got), np.arange(len(waves)))
    # whole waves per slice, slices in wave order
    last = -1
    for s in slices:
        if len(s):
            w = waves[np.asarray(s)]
            assert w.min() > last
            last = w.max()
