"""BLIF ingestion and export (host side, no GPU)."""
import numpy as np
import pytest

from paper_2306_11006_gb300 import blif
from paper_2306_11006_gb300 import inputs as I

FULL_ADDER = """
# full adder: sum by two XOR covers, carry by a majority cover
.model fa
.inputs a b c
.outputs s co
.names a b x
01 1
10 1
.names x c s
01 1
10 1
.names a b c \\
  co
11- 1
1-1 1
-11 1
.end
"""

YOSYS_CELLS = """
.model cells
.inputs a b c
.outputs m n o p q r
.subckt $_MUX_ A=c B=b S=a Y=m
.subckt $_ANDNOT_ A=a B=b Y=n
.subckt $_ORNOT_ A=a B=c Y=t
.subckt $_NOT_ A=t Y=o
.subckt $_NMUX_ A=a B=c S=b Y=p
.subckt $_NAND_ A=a B=c Y=u
.subckt $_XNOR_ A=u B=b Y=q
.subckt $_BUF_ A=q Y=r
.end
"""


def _all_inputs(k):
    return [[(m >> (k - 1 - j)) & 1 for j in range(k)] for m in range(1 << k)]


def test_full_adder_covers():
    nl = blif.read_blif(FULL_ADDER)
    assert nl.num_inputs == 3 and len(nl.outputs) == 2
    for a, b, c in _all_inputs(3):
        s, co = nl.plain_eval([a, b, c])
        assert s == (a + b + c) % 2 and co == int(a + b + c >= 2)
    # two XOR gates, the carry from the cover's three cubes (3 AND + 2 OR)
    assert nl.num_gates == 7


def test_yosys_internal_cells():
    nl = blif.read_blif(YOSYS_CELLS)
    for a, b, c in _all_inputs(3):
        m, n, o, p, q, r = nl.plain_eval([a, b, c])
        assert m == (b if a else c)
        assert n == (a & (1 - b))
        assert o == 1 - (a | (1 - c))
        assert p == 1 - (c if b else a)
        assert q == 1 - ((1 - (a & c)) ^ b) and r == q


def test_recognised_gates_and_constants():
    text = """.model g
.inputs a b s
.outputs y0 y1 y2 y3 y4 y5
.names a b y0
00 0
.names s a b y1
11- 1
0-1 1
.names y2
1
.names y3
.names a y4
0 1
.names b s a y5
-0- 0
--0 0
.end
"""
    nl = blif.read_blif(text)
    types = list(nl.type)
    assert I.OR in types and I.MUX in types and I.CONST1 in types and I.CONST0 in types and I.NOT in types
    for a, b, s in _all_inputs(3):
        y0, y1, y2, y3, y4, y5 = nl.plain_eval([a, b, s])
        assert y0 == (a | b) and y1 == (a if s else b) and y2 == 1 and y3 == 0 and y4 == 1 - a
        # OFF-set cover over (b, s, a): zero where s == 0 or a == 0
        assert y5 == int(s == 1 and a == 1)


@pytest.mark.parametrize("make", [lambda: I.ripple_carry_adder(8), lambda: I.array_multiplier(4),
                                  lambda: I.comparator(6)])
def test_round_trip_preserves_function(make):
    nl = make()
    back = blif.read_blif(blif.write_blif(nl))
    assert back.num_inputs == nl.num_inputs and len(back.outputs) == len(nl.outputs)
    rng = np.random.default_rng(5)
    for _ in range(64):
        bits = rng.integers(0, 2, nl.num_inputs)
        assert np.array_equal(back.plain_eval(bits), nl.plain_eval(bits))


def test_deep_chain_is_not_recursive():
    depth = 5000
    lines = [".model chain", ".inputs a b", ".outputs y"]
    prev = "a"
    for k in range(depth):
        lines += [f".names {prev} b w{k}", "01 1", "10 1"]
        prev = f"w{k}"
    lines += [f".names {prev} y", "1 1", ".end"]
    nl = blif.read_blif("\n".join(lines))
    for a, b in _all_inputs(2):
        assert nl.plain_eval([a, b])[0] == (a ^ (b * (depth % 2)))


@pytest.mark.parametrize("text, msg", [
    (".model x\n.inputs a\n.outputs y\n.latch a y re clk 0\n.end\n", "latch"),
    (".model x\n.inputs a\n.outputs y\n.names q y\n1 1\n.end\n", "never defined"),
    (".model x\n.inputs a\n.outputs y\n.names y2 y\n1 1\n.names y y2\n1 1\n.end\n", "cycle"),
    (".model x\n.inputs a\n.outputs y\n.subckt adder A=a Y=y\n.end\n", "unsupported cell"),
    (".model x\n.inputs a\n.outputs y\n.names a y\n1 1\n.model z\n.end\n", "hierarchical"),
    (".model x\n.inputs a b\n.outputs y\n.names a b y\n11 1\n00 0\n.end\n", "only ON-set"),
])
def test_rejects_unsupported_input(text, msg):
    with pytest.raises(ValueError, match=msg):
        blif.read_blif(text)
