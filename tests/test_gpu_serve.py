"""GPU tests of the continuous-batching server (arx_serve_*).

Each request's ciphertexts must be bit-identical (tolerance 0) whether it runs
alone through arx_eval_netlist_ex or mixed with other clients' requests in the
server, whose waves share launches; admission must respect the HBM budget;
requests arriving while others run must join and finish.
"""
import time

import numpy as np
import pytest

from paper_2306_11006_gb300 import arx
from paper_2306_11006_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clients(O, keys630, keys64):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    k630 = arx.load_keys(keys630.bsk, keys630.ksk, 630)
    k64 = arx.load_keys(keys64.bsk, keys64.ksk, 64)
    yield {"a": (keys630, k630), "b": (keys64, k64)}
    arx.unload_keys(k630)
    arx.unload_keys(k64)


def _requests(O, clients):
    reqs = []
    nets = [I.ripple_carry_adder(8), I.array_multiplier(4), I.comparator(6),
            I.random_dag(seed=11, total=1500, levels=6, num_inputs=64, wmin=100, wmax=600)]
    for ci, (name, (keys, ks)) in enumerate(sorted(clients.items())):
        for k, nl in enumerate(nets):
            bits = I.random_bits(1000 + 10 * ci + k, nl.num_inputs)
            ct = keys.encrypt(O, I, bits, 2000 + 10 * ci + k)
            alone = np.zeros((len(nl.outputs), keys.n + 1), np.uint32)
            arx.eval_netlist_ex(nl, ct, alone, keyset=ks)
            reqs.append((nl, bits, ct, keys, ks, alone))
    return reqs


def test_mixed_clients_equal_alone(O, clients):
    reqs = _requests(O, clients)
    with arx.Server(arena_bytes=256 << 20) as srv:
        ids = [srv.submit(nl, ct, keyset=ks, n=keys.n) for nl, bits, ct, keys, ks, alone in reqs]
        outs = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_active"] >= 2
    for (nl, bits, ct, keys, ks, alone), out in zip(reqs, outs):
        assert np.array_equal(out, alone), nl.name
        assert np.array_equal(arx.client_decrypt(keys.n, keys.s, out), nl.plain_eval(bits)), nl.name


def test_admission_respects_hbm_budget(O, clients):
    keys, ks = clients["a"]
    nl = I.ripple_carry_adder(6)
    wire_bytes = (nl.num_inputs + nl.num_gates) * 632 * 4
    budget = arx.resident_bytes() + int(1.5 * wire_bytes)   # room for one request at a time
    cts, bits = [], []
    for k in range(4):
        b = I.random_bits(3000 + k, nl.num_inputs)
        bits.append(b)
        cts.append(keys.encrypt(O, I, b, 3100 + k))
    with arx.Server(hbm_budget=budget, arena_bytes=64 << 20) as srv:
        ids = [srv.submit(nl, ct, keyset=ks) for ct in cts]
        outs = [srv.wait(i) for i in ids]
        st = srv.stats()
        assert st["peak_active"] == 1
        assert st["peak_bytes"] <= budget
        with pytest.raises(arx.ArxError) as e:        # larger than the whole budget
            srv.submit(I.random_dag(seed=1, total=4000, levels=4, num_inputs=64, wmin=500, wmax=2000),
                       np.zeros((64, 631), np.uint32), keyset=ks)
        assert e.value.code == -3
    for b, out in zip(bits, outs):
        assert np.array_equal(arx.client_decrypt(630, keys.s, out), nl.plain_eval(b))


def test_arrivals_while_running_join(O, clients):
    keys, ks = clients["a"]
    big = I.random_dag(seed=12, total=6000, levels=12, num_inputs=128, wmin=200, wmax=900)
    small = I.comparator(8)
    bb = I.random_bits(4000, big.num_inputs)
    sb = I.random_bits(4001, small.num_inputs)
    cb = keys.encrypt(O, I, bb, 4002)
    cs = keys.encrypt(O, I, sb, 4003)
    with arx.Server(arena_bytes=128 << 20) as srv:
        r0 = srv.submit(big, cb, keyset=ks)
        t0 = time.time()
        while srv.stats()["active"] == 0 and time.time() - t0 < 30:
            time.sleep(0.005)
        r1 = srv.submit(small, cs, keyset=ks)          # arrives while the DAG runs
        o1 = srv.wait(r1)
        o0 = srv.wait(r0)
        st = srv.stats()
    assert st["peak_active"] >= 2
    assert np.array_equal(arx.client_decrypt(630, keys.s, o0), big.plain_eval(bb))
    assert np.array_equal(arx.client_decrypt(630, keys.s, o1), small.plain_eval(sb))
    alone = np.zeros_like(o1)
    arx.eval_netlist_ex(small, cs, alone, keyset=ks)
    assert np.array_equal(o1, alone)


def test_bad_requests_rejected_without_disturbing_others(O, clients):
    keys, ks = clients["a"]
    nl = I.ripple_carry_adder(3)
    cyc = I.Netlist(nl.num_inputs, nl.type.copy(), nl.in0.copy(), nl.in1.copy(), nl.in2.copy(), nl.outputs.copy())
    cyc.in0[0] = nl.num_inputs + 3
    cyc.in1[3] = nl.num_inputs + 0
    b = I.random_bits(5000, nl.num_inputs)
    ct = keys.encrypt(O, I, b, 5001)
    with arx.Server(arena_bytes=16 << 20) as srv:
        good = srv.submit(nl, ct, keyset=ks)
        with pytest.raises(arx.ArxError) as e:
            srv.submit(cyc, ct, keyset=ks)
        assert e.value.code == -4
        with pytest.raises(arx.ArxError) as e:
            srv.submit(nl, ct, keyset=77)
        assert e.value.code == -2
        out = srv.wait(good)
    assert np.array_equal(arx.client_decrypt(630, keys.s, out), nl.plain_eval(b))


class _Client:
    def __init__(self, O, seed, n):
        self.n = n
        kr = I.key_randomness(seed, n)
        self.s = kr.s
        self.bsk, self.ksk = O.keygen(kr)
        self.ctx = O.Context(n, self.bsk, self.ksk)

    def encrypt(self, O, I_, bits, seed):
        m, e = I_.encryption_randomness(seed, len(bits), self.n)
        return O.encrypt(self.n, self.s, m, e, np.asarray(bits, np.uint8))


@pytest.fixture(scope="module")
def second630(O, clients):
    """A second client with its own n = 630 keys (same parameter set as client a)."""
    keys = _Client(O, 21, 630)
    ks = arx.load_keys(keys.bsk, keys.ksk, 630)
    yield keys, ks
    arx.unload_keys(ks)


def test_clients_on_different_key_sets_share_launches(O, clients, second630):
    """Two clients with their own key sets of the same parameter set: their
    waves run in the same launches (one blind-rotation and one key-switch launch
    per tick), and each result equals the oracle's and the one computed alone."""
    (ka, sa), (kb, sb) = clients["a"], second630
    nl = I.union([I.ripple_carry_adder(6), I.comparator(4)])
    wave, depth = arx.levelize(nl)
    reqs = []
    for k, (keys, ks) in enumerate(((ka, sa), (kb, sb))):
        bits = I.random_bits(6000 + k, nl.num_inputs)
        reqs.append((keys, ks, bits, keys.encrypt(O, I, bits, 6100 + k)))
    with arx.Server(arena_bytes=64 << 20) as srv:
        ids = [srv.submit(nl, ct, keyset=ks) for keys, ks, bits, ct in reqs]
        outs = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == 2 and st["failed"] == 0
    # merged: at most one tick of offset; apart: two launches per wave per client
    assert st["launches"] <= 2 * depth + 2, st
    assert st["shared_launches"] >= 1 and st["max_keys_per_launch"] == 2, st
    for (keys, ks, bits, ct), out in zip(reqs, outs):
        assert np.array_equal(out, keys.ctx.eval_netlist(nl, ct))
        assert np.array_equal(arx.client_decrypt(630, keys.s, out), nl.plain_eval(bits))


def test_throughput_tiles_never_mix_key_sets(O, clients, second630):
    """Wide waves from two key sets in one launch of the throughput kernel (several
    gates per CTA tile; 301 gates per client, so that each key set's group is
    padded to whole tiles): every sampled ciphertext equals the oracle's."""
    (ka, sa), (kb, sb) = clients["a"], second630
    g = 301
    types = I.random_gate_types(61, g)
    nl = I.Netlist(2 * g, types, np.arange(g, dtype=np.uint32), np.arange(g, 2 * g, dtype=np.uint32),
                   np.zeros(g, np.uint32), np.arange(2 * g, 3 * g, dtype=np.uint32), "gates301")
    reqs = []
    for k, (keys, ks) in enumerate(((ka, sa), (kb, sb))):
        bits = I.random_bits(6200 + k, nl.num_inputs)
        reqs.append((keys, ks, bits, keys.encrypt(O, I, bits, 6300 + k)))
    with arx.Server(arena_bytes=64 << 20) as srv:
        ids = [srv.submit(nl, ct, keyset=ks) for keys, ks, bits, ct in reqs]
        outs = [srv.wait(i) for i in ids]
    rng = np.random.default_rng(5)
    for (keys, ks, bits, ct), out in zip(reqs, outs):
        assert np.array_equal(arx.client_decrypt(630, keys.s, out), nl.plain_eval(bits))
        pick = np.sort(rng.choice(g, 12, replace=False))
        want = keys.ctx.gates(types[pick], ct[pick], ct[g + pick])
        assert np.array_equal(out[pick], want)
