"""Simon-128/128 as a Boolean netlist: the transciphering workload (App. A).

The paper evaluates Simon and Speck rounds homomorphically as wide-and-shallow
bitwise circuits (App. A).  Written from the cipher's published specification
(Beaulieu et al., "The SIMON and SPECK Families of Lightweight Block Ciphers",
2013): 64-bit words, two key words, 68 rounds, round function
    (x, y) -> (y ^ f(x) ^ k_i, x),   f(x) = (S^1 x & S^8 x) ^ S^2 x,
S^j the left rotation by j, and key schedule (m = 2)
    k_{i+2} = c ^ (z_2)_i ^ k_i ^ S^-3 k_{i+1} ^ S^-4 k_{i+1},   c = 2^64 - 4.
`simon_netlist` turns R rounds over B blocks into gates of the library (64 AND
and 192 XOR gates per round and block; rotations are wiring).  The round keys
are expanded by the key owner (the client) and enter as encrypted inputs, shared
by all blocks.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I

WORD = 64
ROUNDS = 68
MASK = (1 << WORD) - 1
# the constant sequence z_2, first bit on the left, used cyclically
Z2 = "10101111011100000011010010011000101000010001111110010110110011"


def _rol(x: int, r: int) -> int:
    return ((x << r) | (x >> (WORD - r))) & MASK


def _ror(x: int, r: int) -> int:
    return ((x >> r) | (x << (WORD - r))) & MASK


def round_keys(key: tuple[int, int], rounds: int = ROUNDS) -> list[int]:
    """Round keys from key = (k1, k0) (k0 is the first round key)."""
    k = [key[1] & MASK, key[0] & MASK]
    c = MASK ^ 3
    for i in range(rounds - 2):
        t = _ror(k[i + 1], 3)
        t ^= _ror(t, 1)
        k.append(c ^ int(Z2[i % 62]) ^ k[i] ^ t)
    return k[:rounds]


def encrypt(block: tuple[int, int], key: tuple[int, int], rounds: int = ROUNDS) -> tuple[int, int]:
    """Plaintext Simon-128/128 on block = (x, y) (x the high word)."""
    x, y = block
    for k in round_keys(key, rounds):
        x, y = y ^ ((_rol(x, 1) & _rol(x, 8)) ^ _rol(x, 2)) ^ k, x
    return x, y


def word_bits(w: int) -> list[int]:
    return [(w >> j) & 1 for j in range(WORD)]


def bits_word(b) -> int:
    return sum(int(v) << j for j, v in enumerate(b))


def simon_netlist(rounds: int = ROUNDS, blocks: int = 1) -> I.Netlist:
    """Inputs: for each block its x then y word (64 bits each, least significant
    first), then the round keys (rounds x 64 bits).  Outputs: each block's x, y."""
    B = I.Builder(blocks * 2 * WORD + rounds * WORD)
    key0 = blocks * 2 * WORD
    outs = []
    for blk in range(blocks):
        x = [blk * 2 * WORD + j for j in range(WORD)]
        y = [blk * 2 * WORD + WORD + j for j in range(WORD)]
        for r in range(rounds):
            k = [key0 + r * WORD + j for j in range(WORD)]
            nx = []
            for j in range(WORD):
                a = B.AND(x[(j - 1) % WORD], x[(j - 8) % WORD])   # S^1 x & S^8 x
                u = B.XOR(B.XOR(y[j], k[j]), x[(j - 2) % WORD])   # y ^ k ^ S^2 x
                nx.append(B.XOR(a, u))
            x, y = nx, x
        outs += x + y
    return B.build(outs, name=f"simon128x{rounds}x{blocks}", rounds=rounds, blocks=blocks)


def netlist_inputs(blocks_xy, key: tuple[int, int], rounds: int = ROUNDS) -> np.ndarray:
    """Input bits of simon_netlist for the given blocks and key."""
    bits = []
    for x, y in blocks_xy:
        bits += word_bits(x) + word_bits(y)
    for k in round_keys(key, rounds):
        bits += word_bits(k)
    return np.array(bits, np.uint8)


def netlist_outputs(out_bits) -> list[tuple[int, int]]:
    """(x, y) words per block from the netlist's output bits."""
    out_bits = np.asarray(out_bits)
    res = []
    for blk in range(len(out_bits) // (2 * WORD)):
        o = out_bits[blk * 2 * WORD:(blk + 1) * 2 * WORD]
        res.append((bits_word(o[:WORD]), bits_word(o[WORD:])))
    return res
