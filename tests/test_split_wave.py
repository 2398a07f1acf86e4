"""Host logic of the autotuned wave plan (arx_split_wave, what graph plans use):
the chosen one or two launches, their cost and the capacity that level
balancing fills up to, against a brute-force enumeration of every plan of at
most two launches on random shape tables."""
import math

import numpy as np
import pytest

from paper_2306_11006_gb300 import arx

# measured per-round launch times (ms, 630 CMux) and round sizes of this GPU's
# shapes: the (1,6), (1,4), (2,3), (3,2), (6,1) throughput shapes and the 16-,
# 8-, 4- and 2-CTA cluster kernels
GB300 = [(18.44, 912, 0), (13.80, 608, 0), (9.62, 456, 0), (7.06, 304, 0), (4.82, 152, 0),
         (1.06, 7, 1), (1.32, 8, 1), (1.16, 32, 1), (2.66, 76, 1)]


def _single(table, w):
    return min(math.ceil(w / g) * ms for ms, g, _ in table) if w > 0 else 0.0


def _best(table, w):
    """Cheapest plan of at most two launches: one launch, or k >= 1 whole rounds of a
    non-cluster shape followed by one launch for the rest."""
    best = _single(table, w)
    for ms, g, cl in table:
        if cl:
            continue
        k = 1
        while k * g < w:
            best = min(best, k * ms + _single(table, w - k * g))
            k += 1
    return best


def _check(table, w):
    ms, g, cl = zip(*table)
    bulk, bulk_jobs, tail, cost, cap = arx.split_wave(ms, g, cl, w)
    best = _best(table, w)
    # the cheapest plan, up to the 0.1 % margin a split must win by
    assert best * (1 - 1e-12) <= cost <= best / 0.999 + 1e-12, (w, cost, best)
    # the reported launches cost what is reported and cover the wave
    if tail < 0:
        assert bulk_jobs == w
        assert cost == pytest.approx(math.ceil(w / g[bulk]) * ms[bulk])
    else:
        assert not cl[bulk] and 0 < bulk_jobs < w and bulk_jobs % g[bulk] == 0
        rest = w - bulk_jobs
        assert cost == pytest.approx(bulk_jobs // g[bulk] * ms[bulk] + math.ceil(rest / g[tail]) * ms[tail])
        assert math.ceil(rest / g[tail]) * ms[tail] == pytest.approx(_single(table, rest))
    # capacity: a wave of cap blind rotations runs within the cost, and no wider
    # wave does (checked over the next largest round of widths)
    assert cap >= w
    assert _best(table, cap) <= cost * (1 + 1e-9)
    for w2 in range(cap + 1, cap + max(g) + 1):
        assert _best(table, w2) > cost * (1 + 1e-9), (w, cap, w2)
    return bulk, bulk_jobs, tail, cost, cap


def test_gb300_table_known_cases():
    # 22 full rounds and 8 left over: the 8 on a cluster kernel, not a 23rd round
    bulk, bj, tail, cost, cap = _check(GB300, 22 * 912 + 8)
    assert (bulk, bj) == (0, 22 * 912) and GB300[tail][2] == 1
    # 760: 456 on (2,3) and 304 on (3,2) beat one (1,6) round (16.68 < 18.44 ms)
    bulk, bj, tail, cost, cap = _check(GB300, 760)
    assert cost == pytest.approx(9.62 + 7.06) and {bulk, tail} == {2, 3}
    # exact rounds stay one launch
    assert _check(GB300, 912)[2] == -1 and _check(GB300, 608)[2] == -1
    # narrow waves: the cluster kernels, and a level of 7 has room for nothing more
    assert _check(GB300, 7)[4] == 7


@pytest.mark.parametrize("w", [1, 5, 9, 33, 77, 100, 153, 305, 500, 700, 913, 1000, 1217, 1500, 2000, 3192, 5000])
def test_gb300_table_against_brute_force(w):
    _check(GB300, w)


def test_random_tables_against_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(40):
        k = int(rng.integers(1, 7))
        table = []
        for s in range(k):
            g = int(rng.integers(1, 200))
            ms = float(rng.uniform(0.5, 20.0))
            table.append((ms, g, int(s > 0 and rng.random() < 0.3)))
        for w in rng.integers(1, 1200, 6):
            _check(table, int(w))


def test_bad_arguments_rejected():
    with pytest.raises(arx.ArxError):
        arx.split_wave([1.0], [0], [0], 10)
    with pytest.raises(arx.ArxError):
        arx.split_wave([0.0], [5], [0], 10)
    with pytest.raises(arx.ArxError):
        arx.split_wave([1.0], [5], [0], 0)
    with pytest.raises(arx.ArxError):
        arx.split_wave([], [], [], 10)
