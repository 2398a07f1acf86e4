"""BLIF netlists in and out.

The paper's front end synthesises programs into Boolean netlists with Yosys,
weighting a MUX as twice a two-input gate (Sec. 3.2), and the runtime evaluates
gate netlists level by level (Sec. 4).  This module reads the Berkeley Logic
Interchange Format that such a flow writes and returns a `Netlist` the library
evaluates (`arx.eval_netlist`, `arx.Plan`); `write_blif` exports one.

Accepted input (combinational logic only):
- `.model`, `.inputs`, `.outputs`, `.end`, `#` comments, `\\` line continuations;
- `.names` single-output covers (ON-set or OFF-set rows, `-` don't-cares): any
  function of at most three inputs that is one of the library's gates (NOT,
  buffer, the six two-input gates, MUX in any input order, constants) becomes
  that gate, any other cover a sum of products of AND / OR / NOT gates;
- `.subckt` instances of Yosys's internal gate cells `$_BUF_ $_NOT_ $_AND_
  $_NAND_ $_OR_ $_NOR_ $_XOR_ $_XNOR_ $_ANDNOT_ $_ORNOT_ $_MUX_ $_NMUX_` (pins
  A, B, S, Y; `$_MUX_` is Y = S ? B : A), as written by `write_blif` after
  `abc -g ...` or `techmap`.
`.latch`, hierarchical `.subckt` of other models, and cycles raise ValueError.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import inputs as I

_CELLS = {  # Yosys internal cell -> (inputs in order, builder)
    "$_BUF_": ("A",), "$_NOT_": ("A",),
    "$_AND_": ("A", "B"), "$_NAND_": ("A", "B"), "$_OR_": ("A", "B"), "$_NOR_": ("A", "B"),
    "$_XOR_": ("A", "B"), "$_XNOR_": ("A", "B"), "$_ANDNOT_": ("A", "B"), "$_ORNOT_": ("A", "B"),
    "$_MUX_": ("A", "B", "S"), "$_NMUX_": ("A", "B", "S"),
}

_TWO_INPUT = {  # truth table over (a, b) = (0,0), (0,1), (1,0), (1,1) -> gate
    (0, 0, 0, 1): I.AND, (1, 1, 1, 0): I.NAND, (0, 1, 1, 1): I.OR, (1, 0, 0, 0): I.NOR,
    (0, 1, 1, 0): I.XOR, (1, 0, 0, 1): I.XNOR,
}


def _logical_lines(text: str):
    buf = ""
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].rstrip()
        if line.endswith("\\"):
            buf += line[:-1] + " "
            continue
        line = (buf + line).strip()
        buf = ""
        if line:
            yield line


def _cover_table(rows, k: int):
    """Truth table (index = inputs as a binary number, input 0 most significant)."""
    if not rows:
        return [0] * (1 << k)
    on = {r[1] for r in rows}
    if len(on) != 1 or on.pop() not in ("0", "1"):
        raise ValueError("a .names cover must list only ON-set or only OFF-set rows")
    polarity = int(rows[0][1])
    hit = [0] * (1 << k)
    for pat, _ in rows:
        if len(pat) != k or any(ch not in "01-" for ch in pat):
            raise ValueError(f"bad cover row {pat!r}")
        for m in range(1 << k):
            bits = [(m >> (k - 1 - j)) & 1 for j in range(k)]
            if all(ch == "-" or int(ch) == bit for ch, bit in zip(pat, bits)):
                hit[m] = 1
    return [h if polarity else 1 - h for h in hit]


class _Graph:
    """Signals by name; each non-input signal is a node to be emitted as gates."""

    def __init__(self):
        self.inputs, self.outputs = [], []
        self.nodes = {}  # name -> ("table", [in names], table, cover rows) | ("cell", cell, [in names])

    def define(self, name, node):
        if name in self.nodes or name in self.inputs:
            raise ValueError(f"signal {name!r} defined twice")
        self.nodes[name] = node


def _parse(text: str) -> _Graph:
    g = _Graph()
    lines = list(_logical_lines(text))
    i = 0
    models = 0
    while i < len(lines):
        tok = lines[i].split()
        kw = tok[0]
        if kw == ".model":
            models += 1
            if models > 1:
                raise ValueError("hierarchical BLIF (several .model) is not supported")
        elif kw == ".inputs":
            g.inputs += tok[1:]
        elif kw == ".outputs":
            g.outputs += tok[1:]
        elif kw == ".names":
            sigs = tok[1:]
            if not sigs:
                raise ValueError(".names without an output")
            rows = []
            while i + 1 < len(lines) and not lines[i + 1].startswith("."):
                i += 1
                parts = lines[i].split()
                if len(sigs) == 1:
                    rows.append(("", parts[0]))
                else:
                    if len(parts) != 2:
                        raise ValueError(f"bad cover row {lines[i]!r}")
                    rows.append((parts[0], parts[1]))
            g.define(sigs[-1], ("table", sigs[:-1], _cover_table(rows, len(sigs) - 1), rows))
        elif kw in (".subckt", ".gate"):
            cell = tok[1]
            if cell not in _CELLS:
                raise ValueError(f"unsupported cell {cell!r} (only Yosys internal gate cells)")
            pins = dict(p.split("=", 1) for p in tok[2:])
            if "Y" not in pins or any(p not in pins for p in _CELLS[cell]):
                raise ValueError(f"cell {cell} lacks pins")
            g.define(pins["Y"], ("cell", cell, [pins[p] for p in _CELLS[cell]]))
        elif kw == ".end":
            break
        elif kw in (".latch", ".mlatch"):
            raise ValueError("sequential BLIF (.latch) is not supported: netlists are combinational")
        elif kw.startswith("."):
            raise ValueError(f"unsupported BLIF directive {kw}")
        else:
            raise ValueError(f"unexpected line {lines[i]!r}")
        i += 1
    return g


def _find_mux(table):
    """(sel, t, f) input positions when a 3-input table is sel ? t : f."""
    for s, t, f in itertools.permutations(range(3)):
        ok = True
        for m in range(8):
            b = [(m >> (2 - j)) & 1 for j in range(3)]
            if table[m] != (b[t] if b[s] else b[f]):
                ok = False
                break
        if ok:
            return s, t, f
    return None


def read_blif(text: str, name: str = "blif") -> I.Netlist:
    """Parse BLIF text into a Netlist (inputs in .inputs order, outputs in .outputs order)."""
    g = _parse(text)
    if not g.outputs:
        raise ValueError("no .outputs")
    B = I.Builder(len(g.inputs))
    wire = {s: k for k, s in enumerate(g.inputs)}
    state = {}  # name -> 1 visiting, 2 done

    def const(v):
        return B.gate(I.CONST1 if v else I.CONST0)

    def sop(ins, rows):
        # sum of the cover's cubes (AND / OR / NOT gates); an OFF-set cover is negated
        terms = []
        for pat, _ in rows:
            lits = [w if ch == "1" else B.NOT(w) for ch, w in zip(pat, ins) if ch != "-"]
            if not lits:
                return const(int(rows[0][1]))
            acc = lits[0]
            for lit in lits[1:]:
                acc = B.AND(acc, lit)
            terms.append(acc)
        acc = terms[0]
        for t in terms[1:]:
            acc = B.OR(acc, t)
        return acc if rows[0][1] == "1" else B.NOT(acc)

    def build_node(sig, a):
        node = g.nodes[sig]
        if node[0] == "cell":
            cell = node[1]
            if cell == "$_BUF_": return B.gate(I.COPY, a[0])
            if cell == "$_NOT_": return B.NOT(a[0])
            if cell == "$_AND_": return B.AND(a[0], a[1])
            if cell == "$_NAND_": return B.gate(I.NAND, a[0], a[1])
            if cell == "$_OR_": return B.OR(a[0], a[1])
            if cell == "$_NOR_": return B.gate(I.NOR, a[0], a[1])
            if cell == "$_XOR_": return B.XOR(a[0], a[1])
            if cell == "$_XNOR_": return B.XNOR(a[0], a[1])
            if cell == "$_ANDNOT_": return B.AND(a[0], B.NOT(a[1]))
            if cell == "$_ORNOT_": return B.OR(a[0], B.NOT(a[1]))
            if cell == "$_MUX_": return B.MUX(a[2], a[1], a[0])
            return B.NOT(B.MUX(a[2], a[1], a[0]))  # $_NMUX_
        table = node[2]
        k = len(a)
        if all(v == table[0] for v in table):
            return const(table[0])
        if k == 1:
            return B.gate(I.COPY, a[0]) if table == [0, 1] else B.NOT(a[0])
        if k == 2 and tuple(table) in _TWO_INPUT:
            return B.gate(_TWO_INPUT[tuple(table)], a[0], a[1])
        if k == 3 and _find_mux(table) is not None:
            s_, t_, f_ = _find_mux(table)
            return B.MUX(a[s_], a[t_], a[f_])
        return sop(a, node[3])

    def fanin(sig):
        node = g.nodes[sig]
        return node[2] if node[0] == "cell" else node[1]

    def emit(root):
        # depth-first over fan-ins with an explicit stack (netlists can be deep)
        stack = [root]
        while stack:
            sig = stack[-1]
            if sig in wire:
                stack.pop()
                continue
            if sig not in g.nodes:
                raise ValueError(f"signal {sig!r} is used but never defined")
            if state.get(sig) is None:
                state[sig] = 1
                for f in fanin(sig):
                    if f not in wire:
                        if state.get(f) == 1:
                            raise ValueError(f"combinational cycle through {f!r}")
                        stack.append(f)
                continue
            stack.pop()
            ins = fanin(sig)
            if any(f not in wire for f in ins):
                raise ValueError(f"combinational cycle through {sig!r}")
            wire[sig] = build_node(sig, [wire[f] for f in ins])
            state[sig] = 2
        return wire[root]

    outs = [emit(s) for s in g.outputs]
    return B.build(outs, name=name, blif_inputs=list(g.inputs), blif_outputs=list(g.outputs))


_TABLE_OF = {  # gate -> (cover rows over its inputs in order)
    I.AND: ["11 1"], I.NAND: ["0- 1", "-0 1"], I.OR: ["1- 1", "-1 1"], I.NOR: ["00 1"],
    I.XOR: ["01 1", "10 1"], I.XNOR: ["00 1", "11 1"], I.NOT: ["0 1"], I.COPY: ["1 1"],
    I.MUX: ["11- 1", "0-1 1"],  # inputs (sel, t, f)
}


def write_blif(nl: I.Netlist, model: str = "netlist") -> str:
    """BLIF text of a Netlist: inputs i<k>, gates g<k>, outputs o<k> (buffers)."""
    def sig(w):
        w = int(w)
        return f"i{w}" if w < nl.num_inputs else f"g{w - nl.num_inputs}"

    out = [f".model {model}", ".inputs " + " ".join(f"i{k}" for k in range(nl.num_inputs)),
           ".outputs " + " ".join(f"o{k}" for k in range(len(nl.outputs)))]
    for gi in range(nl.num_gates):
        t = int(nl.type[gi])
        ins = [sig(x) for x in (nl.in0[gi], nl.in1[gi], nl.in2[gi])[: I.ARITY[t]]]
        out.append(".names " + " ".join(ins + [f"g{gi}"]))
        if t == I.CONST1:
            out.append("1")
        elif t != I.CONST0:
            out += _TABLE_OF[t]
    for k, w in enumerate(np.asarray(nl.outputs)):
        out += [f".names {sig(w)} o{k}", "1 1"]
    out.append(".end")
    return "\n".join(out) + "\n"
