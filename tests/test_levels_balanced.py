"""CPU checks of the balanced levelization (arx_levelize_balanced), the level
assignment graph-mode plans use: the depth of the Sec. 4.2 levelization is kept,
every gate stays between its earliest and its latest level and after its inputs
(so every result is that of the plain levelization), and launches are filled up
to the given capacities.  The earliest / latest levels are recomputed here from
their definitions, independently of the library."""
import numpy as np
import pytest

from paper_2306_11006_gb300 import arx
from paper_2306_11006_gb300 import inputs as I

CAPS = [7, 15, 36, 76]  # co-resident 16-, 8-, 4- and 2-CTA clusters on a GB300


def gate_inputs(nl, g):
    k = I.ARITY[int(nl.type[g])]
    return [int(x[g]) for x in (nl.in0, nl.in1, nl.in2)][:k]


def earliest_latest(nl):
    """Earliest level by the recursive definition; latest by the reverse one."""
    G, NI = nl.num_gates, nl.num_inputs
    memo = {}

    def early(g):
        if g not in memo:
            memo[g] = max([early(w - NI) + 1 for w in gate_inputs(nl, g) if w >= NI], default=0)
        return memo[g]

    import sys
    sys.setrecursionlimit(100000)
    e = np.array([early(g) for g in range(G)])
    depth = int(e.max()) + 1
    readers = [[] for _ in range(G)]
    for g in range(G):
        for w in gate_inputs(nl, g):
            if w >= NI:
                readers[w - NI].append(g)
    late = np.full(G, depth - 1)
    for g in sorted(range(G), key=lambda x: -e[x]):
        for s in readers[g]:
            late[g] = min(late[g], late[s] - 1)
    return e, late, depth


def boots_per_level(nl, wave, depth):
    b = np.zeros(depth, np.int64)
    for g in range(nl.num_gates):
        b[wave[g]] += I.BOOTSTRAPS[int(nl.type[g])]
    return b


NETS = {
    "adder32+mult8": lambda: I.union([I.ripple_carry_adder(32), I.array_multiplier(8)]),
    "cmp16": lambda: I.comparator(16),
    "dag": lambda: I.random_dag(seed=3, total=3000, levels=10, num_inputs=200, wmin=40, wmax=800),
    "matmul_small": lambda: I.matmul4x4(bits=3, acc_bits=6, dim=2),
    "adder4x3": lambda: I.union([I.ripple_carry_adder(4)] * 3),
}


@pytest.mark.parametrize("which", sorted(NETS))
def test_balanced_levels_keep_depth_order_and_slack(which):
    nl = NETS[which]()
    w0, d0 = arx.levelize(nl)
    wave, depth = arx.levelize_balanced(nl, CAPS)
    e, late, d = earliest_latest(nl)
    assert depth == d0 == d
    assert np.array_equal(w0, e)
    assert np.all(wave >= e) and np.all(wave <= late)
    NI = nl.num_inputs
    for g in range(nl.num_gates):
        for w in gate_inputs(nl, g):
            if w >= NI:
                assert wave[w - NI] < wave[g]


def test_config2_launches_fill_the_sixteen_cta_clusters():
    """The 32-bit adder + 8x8 multiplier: the plain levelization has a 128-wide
    first wave and 8 to 15 gates in many others; balanced, every level but one
    fits the 7 co-resident sixteen-CTA clusters."""
    nl = NETS["adder32+mult8"]()
    w0, d0 = arx.levelize(nl)
    b0 = boots_per_level(nl, w0, d0)
    assert b0.max() == 128 and (b0 > 7).sum() > 20
    wave, depth = arx.levelize_balanced(nl, CAPS)
    b = boots_per_level(nl, wave, depth)
    assert b.sum() == b0.sum() == nl.num_bootstraps
    assert (b > 7).sum() <= 1 and b.max() <= 36


def test_no_caps_is_the_plain_levelization_filled_to_nothing():
    nl = NETS["cmp16"]()
    w0, d0 = arx.levelize(nl)
    wave, depth = arx.levelize_balanced(nl, [])
    assert depth == d0
    e, late, _ = earliest_latest(nl)
    assert np.all(wave >= e) and np.all(wave <= late)
    # with no free room a level takes exactly the gates due there: every gate at its latest level
    assert np.array_equal(wave, late)


def test_balanced_levels_errors():
    nl = I.ripple_carry_adder(2)
    with pytest.raises(arx.ArxError) as e:
        arx.levelize_balanced(nl, [7, 7])
    assert e.value.code == -1
    cyc = I.Netlist(nl.num_inputs, nl.type.copy(), nl.in0.copy(), nl.in1.copy(), nl.in2.copy(), nl.outputs.copy())
    cyc.in0[0] = nl.num_inputs + 3
    cyc.in1[3] = nl.num_inputs + 0
    with pytest.raises(arx.ArxError) as e:
        arx.levelize_balanced(cyc, CAPS)
    assert e.value.code == -4
