"""Seeded synthetic inputs: key randomness, message bits and Boolean netlists.

This module holds none of the CGGI arithmetic.  It only draws the random numbers
the scheme consumes (secret-key bits, uniform masks, rounded Gaussian noise in
Torus32 units, message bits) and builds gate netlists shaped like the paper's
workloads (ArctyrEX, arXiv 2306.11006: ripple-carry adders and array multipliers
of Table 1, circuits whose waves are a few hundred to several thousand gates wide
as in Sec. 3.1, many circuits batched together).  The tests, the smoke check and
the benchmark all draw their inputs from here, so the CUDA path and the oracle
always see the same bytes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

N = 1024            # TLWE ring degree
ROWS = 6            # (k+1) l rows per TGSW sample
KS_T = 8            # key-switch digits
LWE_N = 630         # LWE dimension of the standard parameter set
SIGMA_LWE = 2.0 ** -15
SIGMA_TRLWE = 2.0 ** -25

# gate opcodes (numbering shared with the C-ABI)
AND, NAND, OR, NOR, XOR, XNOR, NOT, MUX, COPY, CONST0, CONST1 = range(11)
BINARY_OPS = (AND, NAND, OR, NOR, XOR, XNOR)
ARITY = {AND: 2, NAND: 2, OR: 2, NOR: 2, XOR: 2, XNOR: 2, NOT: 1, MUX: 3, COPY: 1,
         CONST0: 0, CONST1: 0}
BOOTSTRAPS = {t: (2 if t == MUX else (1 if ARITY[t] == 2 else 0)) for t in ARITY}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def torus_noise(rng: np.random.Generator, sigma: float, shape) -> np.ndarray:
    """Rounded Gaussian noise, round(sigma * z * 2^32), as int32 Torus32 values."""
    z = rng.standard_normal(shape)
    return np.rint(z * (sigma * 2.0 ** 32)).astype(np.int64).astype(np.int32)


@dataclass
class KeyRandomness:
    """Every random number key generation consumes, for LWE dimension n."""
    n: int
    s: np.ndarray          # [n] u8 in {0,1}: LWE secret key
    K: np.ndarray          # [N] u8 in {0,1}: TLWE secret key
    bsk_mask: np.ndarray   # [n][6][N] u32 uniform
    bsk_noise: np.ndarray  # [n][6][N] i32
    ksk_mask: np.ndarray   # [N][8][3][n] u32 uniform
    ksk_noise: np.ndarray  # [N][8][3] i32


def key_randomness(seed: int, n: int = LWE_N, noiseless: bool = False,
                   trivial_bsk: bool = False, l: int = 3) -> KeyRandomness:
    """Key randomness from one seed.

    noiseless: all noise terms zero (masks still uniform).
    trivial_bsk: additionally zero the bootstrapping-key masks (a noiseless,
    trivial TGSW encryption), used by closed-form checks of blind rotation.
    l: gadget length (3 rows per key component by default; 2 for the variant).
    """
    rows = 2 * l
    rng = _rng(seed)
    s = rng.integers(0, 2, n, dtype=np.uint8)
    K = rng.integers(0, 2, N, dtype=np.uint8)
    bsk_mask = rng.integers(0, 2 ** 32, (n, rows, N), dtype=np.uint32)
    bsk_noise = torus_noise(rng, SIGMA_TRLWE, (n, rows, N))
    ksk_mask = rng.integers(0, 2 ** 32, (N, KS_T, 3, n), dtype=np.uint32)
    ksk_noise = torus_noise(rng, SIGMA_LWE, (N, KS_T, 3))
    if noiseless or trivial_bsk:
        bsk_noise[:] = 0
        ksk_noise[:] = 0
    if trivial_bsk:
        bsk_mask[:] = 0
    return KeyRandomness(n, s, K, bsk_mask, bsk_noise, ksk_mask, ksk_noise)


def encryption_randomness(seed: int, count: int, n: int = LWE_N, noiseless: bool = False):
    """(mask [count][n] u32, noise [count] i32) for fresh LWE encryptions."""
    rng = _rng(seed)
    mask = rng.integers(0, 2 ** 32, (count, n), dtype=np.uint32)
    noise = torus_noise(rng, SIGMA_LWE, count)
    if noiseless:
        noise[:] = 0
    return mask, noise


def random_bits(seed: int, count: int) -> np.ndarray:
    return _rng(seed).integers(0, 2, count, dtype=np.uint8)


def random_u32(seed: int, shape) -> np.ndarray:
    return _rng(seed).integers(0, 2 ** 32, shape, dtype=np.uint32)


def random_gate_types(seed: int, count: int, ops=BINARY_OPS) -> np.ndarray:
    return np.asarray(ops, np.uint8)[_rng(seed).integers(0, len(ops), count)]


# ----------------------------------------------------------------------------
# netlists
# ----------------------------------------------------------------------------
@dataclass
class Netlist:
    """Gate list over wires: ids 0..num_inputs-1 are inputs, num_inputs+g is gate g."""
    num_inputs: int
    type: np.ndarray
    in0: np.ndarray
    in1: np.ndarray
    in2: np.ndarray
    outputs: np.ndarray
    name: str = "netlist"
    meta: dict = field(default_factory=dict)

    @property
    def num_gates(self) -> int:
        return len(self.type)

    @property
    def num_bootstraps(self) -> int:
        return int(sum(BOOTSTRAPS[int(t)] for t in self.type))

    def plain_eval(self, bits: np.ndarray) -> np.ndarray:
        """Boolean semantics of the netlist on plaintext input bits."""
        w = np.zeros(self.num_inputs + self.num_gates, np.uint8)
        w[: self.num_inputs] = np.asarray(bits, np.uint8)
        done = np.zeros(self.num_inputs + self.num_gates, bool)
        done[: self.num_inputs] = True
        remaining = list(range(self.num_gates))
        while remaining:
            nxt = []
            for g in remaining:
                t = int(self.type[g])
                ins = (int(self.in0[g]), int(self.in1[g]), int(self.in2[g]))[: ARITY[t]]
                if not all(done[i] for i in ins):
                    nxt.append(g)
                    continue
                v = [int(w[i]) for i in ins]
                w[self.num_inputs + g] = _plain_gate(t, v)
                done[self.num_inputs + g] = True
            if len(nxt) == len(remaining):
                raise ValueError("netlist has a cycle")
            remaining = nxt
        return w[self.outputs]


def _plain_gate(t: int, v) -> int:
    if t == AND: return v[0] & v[1]
    if t == NAND: return 1 - (v[0] & v[1])
    if t == OR: return v[0] | v[1]
    if t == NOR: return 1 - (v[0] | v[1])
    if t == XOR: return v[0] ^ v[1]
    if t == XNOR: return 1 - (v[0] ^ v[1])
    if t == NOT: return 1 - v[0]
    if t == COPY: return v[0]
    if t == MUX: return v[1] if v[0] else v[2]
    if t == CONST0: return 0
    if t == CONST1: return 1
    raise ValueError(t)


class Builder:
    """Appends gates in creation order (which is a topological order)."""

    def __init__(self, num_inputs: int):
        self.num_inputs = num_inputs
        self.t, self.a, self.b, self.c = [], [], [], []

    def gate(self, t: int, a: int = 0, b: int = 0, c: int = 0) -> int:
        self.t.append(t); self.a.append(a); self.b.append(b); self.c.append(c)
        return self.num_inputs + len(self.t) - 1

    def AND(self, a, b): return self.gate(AND, a, b)
    def OR(self, a, b): return self.gate(OR, a, b)
    def XOR(self, a, b): return self.gate(XOR, a, b)
    def XNOR(self, a, b): return self.gate(XNOR, a, b)
    def NOT(self, a): return self.gate(NOT, a)
    def MUX(self, s, t, f): return self.gate(MUX, s, t, f)

    def full_adder(self, a, b, c):
        x = self.XOR(a, b)
        s = self.XOR(x, c)
        t1 = self.AND(a, b)
        t2 = self.AND(c, x)
        return s, self.OR(t1, t2)

    def half_adder(self, a, b):
        return self.XOR(a, b), self.AND(a, b)

    def add(self, A, B, width=None):
        """Ripple-carry sum of bit vectors (LSB first; None = constant 0)."""
        n = max(len(A), len(B))
        A = list(A) + [None] * (n - len(A))
        B = list(B) + [None] * (n - len(B))
        out, carry = [], None
        for i in range(n):
            bits = [x for x in (A[i], B[i], carry) if x is not None]
            if len(bits) == 3:
                s, carry = self.full_adder(*bits)
            elif len(bits) == 2:
                s, carry = self.half_adder(*bits)
            elif len(bits) == 1:
                s, carry = bits[0], None
            else:
                s, carry = None, None
            out.append(s)
        out.append(carry)
        if width is not None:
            out = (out + [None] * width)[:width]
        return out

    def build(self, outputs, name="netlist", **meta) -> Netlist:
        outs = [o for o in outputs]
        if any(o is None for o in outs):
            zero = self.gate(CONST0)
            outs = [zero if o is None else o for o in outs]
        u32 = lambda x: np.asarray(x, np.uint32)
        return Netlist(self.num_inputs, np.asarray(self.t, np.uint8), u32(self.a), u32(self.b),
                       u32(self.c), u32(outs), name, dict(meta))


def ripple_carry_adder(bits: int = 32) -> Netlist:
    """a + b + cin with one 5-gate full adder per bit (inputs: a, b LSB first, cin)."""
    B = Builder(2 * bits + 1)
    a = list(range(bits)); b = list(range(bits, 2 * bits)); carry = 2 * bits
    s = []
    for i in range(bits):
        si, carry = B.full_adder(a[i], b[i], carry)
        s.append(si)
    return B.build(s + [carry], name=f"adder{bits}", bits=bits)


def array_multiplier(bits: int = 8) -> Netlist:
    """Unsigned bits x bits -> 2*bits product: AND partial products + ripple rows."""
    B = Builder(2 * bits)
    a = list(range(bits)); b = list(range(bits, 2 * bits))
    acc = [B.AND(a[j], b[0]) for j in range(bits)]
    for i in range(1, bits):
        row = [None] * i + [B.AND(a[j], b[i]) for j in range(bits)]
        acc = B.add(acc, row)
    out = (acc + [None] * (2 * bits))[: 2 * bits]
    return B.build(out, name=f"mult{bits}", bits=bits)


def comparator(bits: int = 16) -> Netlist:
    """(A < B, A == B, A > B) of two unsigned bits-wide operands, LSB-first chain."""
    B = Builder(2 * bits)
    a = list(range(bits)); b = list(range(bits, 2 * bits))
    lt = gt = eq = None
    for i in range(bits):
        e = B.XNOR(a[i], b[i])
        g = B.AND(a[i], B.NOT(b[i]))
        l = B.AND(B.NOT(a[i]), b[i])
        if i == 0:
            lt, gt, eq = l, g, e
        else:
            lt = B.OR(l, B.AND(e, lt))
            gt = B.OR(g, B.AND(e, gt))
            eq = B.AND(e, eq)
    return B.build([lt, eq, gt], name=f"cmp{bits}", bits=bits)


def union(netlists, name="union") -> Netlist:
    """Disjoint union: all inputs first (in order), then all gates (in order)."""
    ni = sum(nl.num_inputs for nl in netlists)
    ng = sum(nl.num_gates for nl in netlists)
    types, ins, outs = [], [[], [], []], []
    ioff, goff = 0, 0
    spans = []
    for nl in netlists:
        def remap(w, nl=nl, ioff=ioff, goff=goff):
            w = np.asarray(w, np.int64)
            return np.where(w < nl.num_inputs, ioff + w, ni + goff + (w - nl.num_inputs))
        types.append(nl.type)
        for k, arr in enumerate((nl.in0, nl.in1, nl.in2)):
            ins[k].append(remap(arr))
        outs.append(remap(nl.outputs))
        spans.append((ioff, nl.num_inputs, sum(len(o) for o in outs[:-1]), len(nl.outputs)))
        ioff += nl.num_inputs
        goff += nl.num_gates
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return Netlist(ni, cat(types, np.uint8), cat(ins[0], np.uint32), cat(ins[1], np.uint32),
                   cat(ins[2], np.uint32), cat(outs, np.uint32), name, {"spans": spans})


def level_widths(seed: int, total: int = 65536, levels: int = 40, wmin: int = 512,
                 wmax: int = 8192) -> np.ndarray:
    """Log-uniform widths in [wmin, wmax], rescaled and clamped to sum to total."""
    rng = _rng(seed)
    w = np.exp(rng.uniform(np.log(wmin), np.log(wmax), levels))
    w = np.clip(np.rint(w * total / w.sum()), wmin, wmax).astype(np.int64)
    diff = total - int(w.sum())
    i = 0
    while diff != 0 and i < 100 * levels:
        k = i % levels
        step = 1 if diff > 0 else -1
        room = (wmax - w[k]) if step > 0 else (w[k] - wmin)
        take = min(abs(diff), int(room))
        w[k] += step * take
        diff -= step * take
        i += 1
    return w


def random_dag(seed: int = 3, total: int = 65536, levels: int = 40, num_inputs: int = 1024,
               wmin: int = 512, wmax: int = 8192, mux_frac: float = 0.05) -> Netlist:
    """Levelized random DAG: in0 from the previous level (exact depth), in1/in2
    uniform over all earlier wires; types uniform over the 6 binary ops with a
    mux_frac share of MUX gates."""
    rng = _rng(seed)
    widths = level_widths(seed, total, levels, wmin, wmax)
    types, a, b, c = [], [], [], []
    prev_lo, prev_hi = 0, num_inputs      # wire range of the previous level
    wires = num_inputs                    # wires defined so far
    for w in widths:
        w = int(w)
        t = np.asarray(BINARY_OPS, np.uint8)[rng.integers(0, 6, w)]
        t[rng.random(w) < mux_frac] = MUX
        types.append(t)
        a.append(rng.integers(prev_lo, prev_hi, w))
        b.append(rng.integers(0, wires, w))
        c.append(rng.integers(0, wires, w))
        prev_lo, prev_hi = wires, wires + w
        wires += w
    last = np.arange(prev_lo, prev_hi)
    return Netlist(num_inputs, np.concatenate(types), np.concatenate(a).astype(np.uint32),
                   np.concatenate(b).astype(np.uint32), np.concatenate(c).astype(np.uint32),
                   last.astype(np.uint32), f"dag{total}x{levels}", {"widths": widths})


def matmul4x4(bits: int = 8, acc_bits: int = 16, dim: int = 4) -> Netlist:
    """C = A B for dim x dim matrices of unsigned bits-wide ints, acc_bits-wide
    (wrapping) accumulators; inputs A row-major then B row-major, LSB first."""
    ni = 2 * dim * dim * bits
    Bd = Builder(ni)
    A = [[list(range((i * dim + k) * bits, (i * dim + k + 1) * bits)) for k in range(dim)]
         for i in range(dim)]
    off = dim * dim * bits
    Bm = [[list(range(off + (k * dim + j) * bits, off + (k * dim + j + 1) * bits))
           for j in range(dim)] for k in range(dim)]

    def mult(x, y):
        acc = [Bd.AND(x[j], y[0]) for j in range(bits)]
        for i in range(1, bits):
            row = [None] * i + [Bd.AND(x[j], y[i]) for j in range(bits)]
            acc = Bd.add(acc, row, width=acc_bits)
        return (acc + [None] * acc_bits)[:acc_bits]

    outs = []
    for i in range(dim):
        for j in range(dim):
            s = mult(A[i][0], Bm[0][j])
            for k in range(1, dim):
                s = Bd.add(s, mult(A[i][k], Bm[k][j]), width=acc_bits)
            outs += s
    return Bd.build(outs, name=f"matmul{dim}x{dim}", bits=bits, acc_bits=acc_bits, dim=dim)


def int_to_bits(x: int, width: int) -> list:
    return [(x >> i) & 1 for i in range(width)]


def bits_to_int(bits) -> int:
    return sum(int(b) << i for i, b in enumerate(bits))
