"""Simon-128/128 transciphering workload (App. A), host side."""
import os

import numpy as np
import pytest

from paper_2306_11006_gb300 import inputs as I
from paper_2306_11006_gb300 import simon as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "simon128_128.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, hi, lo = line.split()
            vals[k] = (int(hi, 16), int(lo, 16))
    return vals


def test_published_test_vector():
    g = _golden()
    assert S.encrypt(g["plaintext"], g["key"]) == g["ciphertext"]


def test_round_keys_start_with_the_key_words():
    k = S.round_keys((0x1111, 0x2222))
    assert len(k) == S.ROUNDS and k[0] == 0x2222 and k[1] == 0x1111


def test_netlist_gate_budget():
    nl = S.simon_netlist(rounds=3, blocks=2)
    assert nl.num_gates == 3 * 2 * 256
    assert set(int(t) for t in nl.type) == {I.AND, I.XOR}
    assert nl.num_inputs == 2 * 128 + 3 * 64 and len(nl.outputs) == 2 * 128


def test_netlist_matches_cipher_on_random_blocks():
    rng = np.random.default_rng(6)
    rounds = 5
    nl = S.simon_netlist(rounds=rounds, blocks=2)
    for _ in range(3):
        key = tuple(int(v) for v in rng.integers(0, 2**63, 2, dtype=np.uint64))
        blocks = [tuple(int(v) for v in rng.integers(0, 2**63, 2, dtype=np.uint64)) for _ in range(2)]
        out = nl.plain_eval(S.netlist_inputs(blocks, key, rounds))
        assert S.netlist_outputs(out) == [S.encrypt(b, key, rounds) for b in blocks]


def test_full_cipher_netlist_reproduces_the_test_vector():
    g = _golden()
    nl = S.simon_netlist()
    out = nl.plain_eval(S.netlist_inputs([g["plaintext"]], g["key"]))
    assert S.netlist_outputs(out) == [g["ciphertext"]]
