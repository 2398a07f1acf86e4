"""GPU parity: every ciphertext the CUDA path produces is bit-identical to the
CPU oracle's on the same inputs (tolerance 0: the method is exact integer
arithmetic mod 2^32), and every decrypted output is correct.

Sizes the oracle finishes in seconds are compared in full; the full-size
workloads (the 32-bit adder and 8x8 multiplier, the 65,536-gate random DAG, the
eight 4x4 matrix products) are compared on sampled gates, each recomputed by the
oracle from the GPU's own input wires, plus the decrypted results of all outputs.
"""
import numpy as np
import pytest

from paper_2306_11006_gb300 import arx
from paper_2306_11006_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [(96, 1), (48, 1), (24, 1), (12, 1), (6, 1), (3, 1), (3, 2), (2, 1), (2, 3), (1, 1), (1, 2), (1, 4), (1, 6)]


@pytest.fixture(scope="session")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="session")
def _loaded630(torch_cuda, keys630):
    return arx.load_keys(keys630.bsk, keys630.ksk, 630)


@pytest.fixture(scope="session")
def _loaded64(torch_cuda, keys64):
    return arx.load_keys(keys64.bsk, keys64.ksk, 64)


@pytest.fixture(scope="session")
def _loaded512_l2(torch_cuda, keys512_l2):
    return arx.load_keys(keys512_l2.bsk, keys512_l2.ksk, 512, l=2)


@pytest.fixture
def gpu630(_loaded630):
    arx.use_keys(_loaded630)   # the default key set of the calls without an id
    return _loaded630


@pytest.fixture
def gpu64(_loaded64, _loaded630):
    arx.use_keys(_loaded630)
    return _loaded64


def _inputs(O, I_, keys, types, seed):
    m = len(types)
    xs, ys, zs = I_.random_bits(seed, m), I_.random_bits(seed + 1, m), I_.random_bits(seed + 2, m)
    return (xs, ys, zs, keys.encrypt(O, I_, xs, seed + 3), keys.encrypt(O, I_, ys, seed + 4),
            keys.encrypt(O, I_, zs, seed + 5))


def _truth(types, xs, ys, zs):
    return np.array([I._plain_gate(int(t), [int(x), int(y), int(z)]) for t, x, y, z in zip(types, xs, ys, zs)],
                    np.uint8)


def test_config1_64_independent_gates(O, keys630, gpu630):
    types = I.random_gate_types(1, 64)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 10)
    out = np.zeros_like(ca)
    arx.bootstrap_gates(types, ca, cb, out)
    want = keys630.ctx.gates(types, ca, cb)
    assert np.array_equal(out, want)
    assert np.array_equal(arx.client_decrypt(630, keys630.s, out), _truth(types, xs, ys, zs))


def test_all_gate_types_with_mux(O, keys630, gpu630):
    types = np.array(list(range(11)) * 3, np.uint8)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 20)
    out = np.zeros_like(ca)
    arx.bootstrap_gates_ex(types, ca, cb, cc, out, keyset=gpu630)
    want = keys630.ctx.gates(types, ca, cb, cc)
    assert np.array_equal(out, want)
    assert np.array_equal(arx.client_decrypt(630, keys630.s, out), _truth(types, xs, ys, zs))


def test_every_launch_shape_ragged(O, keys630, gpu630):
    """37 gates (a ragged tail for every gates-per-CTA tile) under each shape."""
    types = np.array([I.BINARY_OPS[k % 6] if k % 9 else I.MUX for k in range(37)], np.uint8)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 30)
    want = keys630.ctx.gates(types, ca, cb, cc)
    try:
        for H, GT in SHAPES:
            arx.set_launch_shape(H, GT)
            out = np.zeros_like(ca)
            arx.bootstrap_gates_ex(types, ca, cb, cc, out, keyset=gpu630)
            assert np.array_equal(out, want), (H, GT)
    finally:
        arx.set_launch_shape(0, 0)


def test_persistent_tiles_beyond_one_wave_sampled(O, keys630, gpu630):
    """More tiles than resident CTAs: the persistent loop wraps; sampled gates."""
    count = 2000
    types = I.random_gate_types(40, count)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 41)
    out = np.zeros_like(ca)
    try:
        arx.set_launch_shape(1, 2)
        arx.bootstrap_gates(types, ca, cb, out)
    finally:
        arx.set_launch_shape(0, 0)
    assert np.array_equal(arx.client_decrypt(630, keys630.s, out), _truth(types, xs, ys, zs))
    pick = np.unique(np.concatenate([np.arange(3), np.arange(count - 3, count),
                                     np.random.default_rng(0).choice(count, 26, replace=False)]))
    want = keys630.ctx.gates(types[pick], ca[pick], cb[pick])
    assert np.array_equal(out[pick], want)


def test_device_pointers_and_streams(O, keys630, gpu630, torch_cuda):
    torch = torch_cuda
    types = I.random_gate_types(50, 24)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 51)
    want = keys630.ctx.gates(types, ca, cb)
    da, db = torch.from_numpy(ca.view(np.int32)).cuda(), torch.from_numpy(cb.view(np.int32)).cuda()
    dout = torch.zeros_like(da)
    s = torch.cuda.Stream()
    arx.bootstrap_gates_ex(types, da, db, None, dout, keyset=gpu630, stream=s)
    s.synchronize()
    assert arx.device_status() == 0
    assert np.array_equal(dout.cpu().numpy().view(np.uint32), want)


def _tie_ciphertexts(n, count, seed):
    """Mask and body words on the rounding ties of the mod switch (k 2^21 + 2^20,
    which rounds up), at 2^31, 2^32 - 1 and 0, mixed with random words: not
    encryptions of anything, but every gate is a fixed integer function of its
    input words, so the GPU must reproduce the oracle on them bit for bit."""
    rng = np.random.default_rng(seed)
    ties = (rng.integers(0, 2048, (count, n + 1), dtype=np.uint64) << 21) + (1 << 20)
    special = np.array([1 << 31, (1 << 32) - 1, 0, 1 << 20, (1 << 21) - 1, 1 << 21], np.uint64)
    pick = rng.integers(0, 4, (count, n + 1))
    out = np.where(pick == 0, ties, np.where(pick == 1, special[rng.integers(0, len(special), (count, n + 1))],
                                            rng.integers(0, 1 << 32, (count, n + 1), dtype=np.uint64)))
    out[:, :: 7] = ties[:, :: 7]
    return out.astype(np.uint32)


def test_rounding_ties_bit_exact(O, keys630, gpu630):
    """Linear combinations landing exactly on the mod-switch half points (and the
    words 0, 2^31, 2^32 - 1): with b = 0 the combination of AND / OR / NAND /
    NOR is +-a plus the constant, so ties in a give ties in the combination."""
    n, g = 630, 48
    types = np.array([[I.AND, I.OR, I.NAND, I.NOR, I.XOR, I.XNOR][k % 6] for k in range(g)], np.uint8)
    ca = _tie_ciphertexts(n, g, 71)
    cb = np.zeros_like(ca)
    cb[g // 2:] = _tie_ciphertexts(n, g - g // 2, 72)  # both operands on ties for the second half
    for body in (0, 1 << 20, (1 << 21) + (1 << 20), (1 << 32) - (1 << 29) + (1 << 20)):
        ca[: g // 4, n] = body
    want = keys630.ctx.gates(types, ca, cb)
    out = np.zeros_like(ca)
    arx.bootstrap_gates_ex(types, ca, cb, None, out, keyset=gpu630)
    assert np.array_equal(out, want)


def test_aliased_buffers(O, keys630, gpu630, torch_cuda):
    """ct_out may be ct_a (the inputs reach the device before any output is
    written), and ct_a may be ct_b."""
    torch = torch_cuda
    types = I.random_gate_types(80, 20)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 81)
    want_ab = keys630.ctx.gates(types, ca, cb)
    want_aa = keys630.ctx.gates(types, ca, ca)
    da, db = torch.from_numpy(ca.view(np.int32)).cuda(), torch.from_numpy(cb.view(np.int32)).cuda()
    arx.bootstrap_gates_ex(types, da, db, None, da, keyset=gpu630)  # out == a
    assert np.array_equal(da.cpu().numpy().view(np.uint32), want_ab)
    da2 = torch.from_numpy(ca.view(np.int32)).cuda()
    out = torch.zeros_like(da2)
    arx.bootstrap_gates_ex(types, da2, da2, None, out, keyset=gpu630)  # a == b
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want_aa)
    h = ca.copy()
    arx.bootstrap_gates_ex(types, h, cb, None, h, keyset=gpu630)  # host buffers, out == a
    assert np.array_equal(h, want_ab)


@pytest.mark.parametrize("count", [3, 8, 9, 17, 64, 65])
def test_key_switch_wave_sizes_bit_exact(O, keys630, gpu630, count):
    """The split key switch across wave sizes around its split boundaries (the
    last CTA of each gate reduces the partial sums, counters re-armed for the next
    call): all gate kinds mixed (MUX: two samples, linear gates: no key rows),
    every ciphertext equal to the oracle's, twice in a row."""
    rng = np.random.default_rng(count)
    types = rng.integers(0, 11, count).astype(np.uint8)
    types[: min(count, 3)] = [I.MUX, I.NOT, I.AND][: min(count, 3)]
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 90 + count)
    want = keys630.ctx.gates(types, ca, cb, cc)
    for rep in range(2):
        out = np.zeros_like(ca)
        arx.bootstrap_gates_ex(types, ca, cb, cc, out, keyset=gpu630)
        assert np.array_equal(out, want), rep
    assert np.array_equal(arx.client_decrypt(630, keys630.s, out), _truth(types, xs, ys, zs))


def test_empty_and_single_gate(O, keys630, gpu630):
    arx.bootstrap_gates(np.zeros(0, np.uint8), np.zeros((0, 631), np.uint32), np.zeros((0, 631), np.uint32),
                        np.zeros((0, 631), np.uint32))
    types = np.array([I.NAND], np.uint8)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 60)
    out = np.zeros_like(ca)
    arx.bootstrap_gates(types, ca, cb, out)
    assert np.array_equal(out, keys630.ctx.gates(types, ca, cb))


def test_linear_only_gates(O, keys630, gpu630):
    types = np.array([I.NOT, I.COPY, I.CONST0, I.CONST1] * 5, np.uint8)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 70)
    out = np.zeros_like(ca)
    arx.bootstrap_gates(types, ca, cb, out)
    assert np.array_equal(out, keys630.ctx.gates(types, ca, cb))


def test_second_keyset_smaller_dimension(O, keys64, gpu64, gpu630):
    types = np.array(list(range(11)) * 2, np.uint8)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys64, types, 80)
    out = np.zeros_like(ca)
    arx.bootstrap_gates_ex(types, ca, cb, cc, out, keyset=gpu64)
    assert np.array_equal(out, keys64.ctx.gates(types, ca, cb, cc))


def test_watchdog_expiry_is_reported_and_the_device_stays_usable(O, keys630, gpu630):
    # the token posted: every bounded wait of both wait functions completes
    assert arx.watchdog_selftest(True) == (0, 0)
    # the token withheld: the four waits give up after 2e7 cycles (about 10 ms),
    # the device status word records the expiry and the call reports it
    assert arx.watchdog_selftest(False, 20_000_000) == (-5, 4)
    assert arx.device_status() == 0  # read and cleared by the call
    assert arx.watchdog_selftest(True) == (0, 0)
    # the context is intact: the next bootstraps are still bit-exact
    types = I.random_gate_types(91, 16)
    xs, ys, zs, ca, cb, cc = _inputs(O, I, keys630, types, 92)
    out = np.zeros_like(ca)
    arx.bootstrap_gates(types, ca, cb, out)
    assert np.array_equal(out, keys630.ctx.gates(types, ca, cb))


def test_invalid_arguments_are_rejected(gpu630):
    with pytest.raises(arx.ArxError) as e:
        arx.bootstrap_gates(np.array([11], np.uint8), np.zeros((1, 631), np.uint32),
                            np.zeros((1, 631), np.uint32), np.zeros((1, 631), np.uint32))
    assert e.value.code == -1
    with pytest.raises(arx.ArxError) as e:
        arx.bootstrap_gates_ex(np.array([0], np.uint8), np.zeros((1, 631), np.uint32),
                               np.zeros((1, 631), np.uint32), None, np.zeros((1, 631), np.uint32), keyset=99)
    assert e.value.code == -2
    with pytest.raises(arx.ArxError) as e:
        arx.bootstrap_gates(np.array([I.MUX], np.uint8), np.zeros((1, 631), np.uint32),
                            np.zeros((1, 631), np.uint32), np.zeros((1, 631), np.uint32))
    assert e.value.code == -1


# --------------------------------------------------------------------------
# netlists
# --------------------------------------------------------------------------
def _encrypt_inputs(O, keys, nl, seed):
    bits = I.random_bits(seed, nl.num_inputs)
    return bits, keys.encrypt(O, I, bits, seed + 1)


def test_small_netlists_bit_exact_in_full(O, keys630, gpu630):
    for nl in (I.ripple_carry_adder(4), I.array_multiplier(3), I.comparator(3)):
        bits, ct = _encrypt_inputs(O, keys630, nl, 90)
        out = np.zeros((len(nl.outputs), 631), np.uint32)
        arx.eval_netlist(nl, ct, out)
        assert np.array_equal(out, keys630.ctx.eval_netlist(nl, ct)), nl.name
        assert np.array_equal(arx.client_decrypt(630, keys630.s, out), nl.plain_eval(bits))


def test_blif_netlists_bit_exact_in_full(O, keys630, gpu630):
    from paper_2306_11006_gb300 import blif
    # a Yosys-cell netlist (4-bit adder carry chain with MUX / ANDNOT cells) and a
    # round trip of a generated comparator through BLIF text
    cells = [".model add4", ".inputs " + " ".join(f"a{k} b{k}" for k in range(4)) + " c",
             ".outputs " + " ".join(f"s{k}" for k in range(4)) + " co"]
    carry = "c"
    for k in range(4):
        cells += [f".subckt $_XOR_ A=a{k} B=b{k} Y=p{k}", f".subckt $_XOR_ A=p{k} B={carry} Y=s{k}",
                  f".subckt $_MUX_ A=a{k} B={carry} S=p{k} Y=c{k}"]
        carry = f"c{k}"
    cells += [f".subckt $_ANDNOT_ A={carry} B=b3 Y=t", ".subckt $_ORNOT_ A=t B=b3 Y=co", ".end"]
    for nl in (blif.read_blif("\n".join(cells)), blif.read_blif(blif.write_blif(I.comparator(3)))):
        bits, ct = _encrypt_inputs(O, keys630, nl, 97)
        out = np.zeros((len(nl.outputs), 631), np.uint32)
        arx.eval_netlist(nl, ct, out)
        assert np.array_equal(out, keys630.ctx.eval_netlist(nl, ct)), nl.name
        assert np.array_equal(arx.client_decrypt(630, keys630.s, out), nl.plain_eval(bits))


def test_simon_rounds_transciphering(O, keys630, gpu630):
    from paper_2306_11006_gb300 import simon as S
    rng = np.random.default_rng(11)
    key = tuple(int(v) for v in rng.integers(0, 2**63, 2, dtype=np.uint64))
    blocks = [tuple(int(v) for v in rng.integers(0, 2**63, 2, dtype=np.uint64)) for _ in range(2)]
    # one round: every gate against the oracle
    nl1 = S.simon_netlist(rounds=1, blocks=1)
    ct1 = keys630.encrypt(O, I, S.netlist_inputs(blocks[:1], key, 1), 131)
    out1 = np.zeros((len(nl1.outputs), 631), np.uint32)
    arx.eval_netlist(nl1, ct1, out1)
    assert np.array_equal(out1, keys630.ctx.eval_netlist(nl1, ct1))
    # six rounds on two blocks as one netlist: the decrypted words are the cipher's
    rounds = 6
    nl = S.simon_netlist(rounds=rounds, blocks=2)
    ct = keys630.encrypt(O, I, S.netlist_inputs(blocks, key, rounds), 132)
    out = np.zeros((len(nl.outputs), 631), np.uint32)
    with arx.Plan(nl, mode=arx.MODE_GRAPH) as p:
        p.run(ct, out)
    dec = arx.client_decrypt(630, keys630.s, out)
    assert S.netlist_outputs(dec) == [S.encrypt(b, key, rounds) for b in blocks]


def test_graph_mode_equals_plain_mode(O, keys630, gpu630):
    nl = I.union([I.ripple_carry_adder(5), I.comparator(4)])
    bits, ct = _encrypt_inputs(O, keys630, nl, 95)
    a = np.zeros((len(nl.outputs), 631), np.uint32)
    b = np.zeros_like(a)
    arx.eval_netlist_ex(nl, ct, a, mode=arx.MODE_PLAIN)
    with arx.Plan(nl, mode=arx.MODE_GRAPH) as p:
        p.run(ct, b)
        c = np.zeros_like(a)
        p.run(ct, c)  # replay of the captured graph
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert np.array_equal(arx.client_decrypt(630, keys630.s, a), nl.plain_eval(bits))


def test_split_wave_bulk_and_tail_launches(O, keys630, gpu630):
    """One wave of six full rounds of 152 SMs' tiles plus 8 gates: the autotuned
    plan runs the rounds on the throughput kernel and the 8 left over as a second
    launch on a shape sized for them; every output equals plain mode's, and
    sampled gates from both launches (the tail is the wave's last jobs) equal the
    oracle's."""
    g = 6 * arx.device_sms() + 8
    types = I.random_gate_types(17, g)
    nl = I.Netlist(2 * g, types, np.arange(g, dtype=np.uint32), np.arange(g, 2 * g, dtype=np.uint32),
                   np.zeros(g, np.uint32), np.arange(2 * g, 3 * g, dtype=np.uint32), "gates%d" % g)
    bits, ct = _encrypt_inputs(O, keys630, nl, 97)
    plain = np.zeros((g, 631), np.uint32)
    arx.eval_netlist_ex(nl, ct, plain, mode=arx.MODE_PLAIN)
    out = np.zeros_like(plain)
    with arx.Plan(nl, mode=arx.MODE_GRAPH) as p:
        ls = p.launches()
        assert p.waves == 1 and sum(j for _, _, _, j in ls) == g
        assert len(ls) == 2 and ls[1][3] == 8, ls
        p.run(ct, out)
    assert np.array_equal(out, plain)
    assert np.array_equal(arx.client_decrypt(630, keys630.s, out), nl.plain_eval(bits))
    pick = np.array(sorted(set(list(np.random.default_rng(9).choice(g - 8, 8, replace=False)) +
                               list(range(g - 10, g)))))
    want = keys630.ctx.gates(types[pick], ct[pick], ct[g + pick])
    assert np.array_equal(out[pick], want)


def test_graph_plan_balances_launch_widths(O, keys630, gpu630):
    """Graph plans place gates within their slack: config 2's 128-wide first wave
    and its 8- to 15-gate waves are spread so that at most one launch exceeds the
    co-resident sixteen-CTA clusters; the depth and every ciphertext are those of
    the plain levelization (compared with the oracle on every output)."""
    nl = I.union([I.ripple_carry_adder(32), I.array_multiplier(8)])
    wave, depth = arx.levelize(nl)
    bits, ct = _encrypt_inputs(O, keys630, nl, 77)
    out_plain = np.zeros((len(nl.outputs), 631), np.uint32)
    arx.eval_netlist_ex(nl, ct, out_plain, mode=arx.MODE_PLAIN)
    out = np.zeros_like(out_plain)
    with arx.Plan(nl, mode=arx.MODE_GRAPH) as p:
        sh = p.shapes()
        assert p.waves == depth and sum(j for _, _, j in sh) == p.bootstraps
        assert sum(1 for H, GT, j in sh if j > 7) <= 1, sh
        assert max(j for _, _, j in sh) < 128
        p.run(ct, out)
    assert np.array_equal(out, out_plain)
    assert np.array_equal(out, keys630.ctx.eval_netlist(nl, ct))
    assert np.array_equal(arx.client_decrypt(630, keys630.s, out), nl.plain_eval(bits))


def test_plan_shapes_report_every_wave(gpu630):
    nl = I.union([I.ripple_carry_adder(8), I.array_multiplier(4)])
    wave, depth = arx.levelize(nl)
    with arx.Plan(nl, mode=arx.MODE_PLAIN) as p:
        sh = p.shapes()
        assert len(sh) == p.waves == depth
        assert sum(j for _, _, j in sh) == p.bootstraps
        # narrow waves take the cluster kernels under the heuristic, the sixteen-
        # or eight-CTA one for the narrowest (8 clusters of eight CTAs always fit)
        assert all(H in (96, 48) and GT == 1 for H, GT, j in sh if 0 < j <= 8)
        assert all(H in (12, 24, 48, 96) and GT == 1 for H, GT, j in sh if 0 < j <= arx.device_sms() // 2)
    arx.set_launch_shape(6, 1)
    try:
        with arx.Plan(nl, mode=arx.MODE_PLAIN) as p:
            assert all((H, GT) == (6, 1) for H, GT, j in p.shapes() if j)
    finally:
        arx.set_launch_shape(0, 0)


def _sampled_gate_parity(O, keys, nl, plan, per_level=8, levels=3, seed=0):
    wave, depth = arx.levelize(nl)
    rng = np.random.default_rng(seed)
    lv = sorted(set([0, depth // 2, depth - 1] + list(rng.integers(0, depth, max(0, levels - 3)))))
    gates = []
    for L in lv:
        idx = np.nonzero(wave == L)[0]
        gates += list(rng.choice(idx, min(per_level, len(idx)), replace=False))
    gates = np.array(sorted(gates))
    ins = np.stack([nl.in0[gates], nl.in1[gates], nl.in2[gates]])
    w_in = plan.wires(ins.ravel(), keys.n).reshape(3, len(gates), keys.n + 1)
    w_out = plan.wires(nl.num_inputs + gates, keys.n)
    # inputs a gate does not read are ignored by both sides
    want = keys.ctx.gates(nl.type[gates], w_in[0], w_in[1], w_in[2])
    assert np.array_equal(w_out, want), [int(g) for g in gates[np.any(w_out != want, axis=1)]]
    return len(gates)


@pytest.mark.parametrize("mode", [arx.MODE_PLAIN, arx.MODE_GRAPH])
def test_config2_adder32_and_mult8(O, keys630, gpu630, mode):
    adder, mult = I.ripple_carry_adder(32), I.array_multiplier(8)
    nl = I.union([adder, mult])
    rng = np.random.default_rng(2)
    a, b = (int(x) for x in rng.integers(0, 2 ** 32, 2))
    cin = int(rng.integers(0, 2))
    x, y = (int(v) for v in rng.integers(0, 256, 2))
    bits = I.int_to_bits(a, 32) + I.int_to_bits(b, 32) + [cin] + I.int_to_bits(x, 8) + I.int_to_bits(y, 8)
    ct = keys630.encrypt(O, I, bits, 200)
    out = np.zeros((len(nl.outputs), 631), np.uint32)
    with arx.Plan(nl, mode=mode) as p:
        p.run(ct, out)
        dec = arx.client_decrypt(630, keys630.s, out)
        assert I.bits_to_int(dec[:33]) == a + b + cin
        assert I.bits_to_int(dec[33:]) == x * y
        assert _sampled_gate_parity(O, keys630, nl, p, per_level=6, levels=12) >= 40


def test_config3_random_dag_sampled(O, keys630, gpu630):
    nl = I.random_dag(seed=3)
    bits, ct = _encrypt_inputs(O, keys630, nl, 300)
    out = np.zeros((len(nl.outputs), 631), np.uint32)
    with arx.Plan(nl, mode=arx.MODE_GRAPH) as p:
        assert p.waves == 40 and p.gates == 65536
        p.run(ct, out)
        assert arx.device_status() == 0
        assert np.array_equal(arx.client_decrypt(630, keys630.s, out), nl.plain_eval(bits))
        assert _sampled_gate_parity(O, keys630, nl, p, per_level=6, levels=6, seed=3) >= 30


def test_config4_matmul_instances_sampled(O, keys630, gpu630):
    inst = [I.matmul4x4() for _ in range(8)]
    nl = I.union(inst)
    rng = np.random.default_rng(4)
    A = rng.integers(0, 256, (8, 4, 4))
    B = rng.integers(0, 256, (8, 4, 4))
    bits = []
    for k in range(8):
        for v in list(A[k].ravel()) + list(B[k].ravel()):
            bits += I.int_to_bits(int(v), 8)
    ct = keys630.encrypt(O, I, bits, 400)
    out = np.zeros((len(nl.outputs), 631), np.uint32)
    with arx.Plan(nl, mode=arx.MODE_GRAPH) as p:
        p.run(ct, out)
        dec = arx.client_decrypt(630, keys630.s, out).reshape(8, 16, 16)
        for k in range(8):
            C = (A[k] @ B[k]) % (1 << 16)
            got = np.array([I.bits_to_int(dec[k, e]) for e in range(16)]).reshape(4, 4)
            assert np.array_equal(got, C), k
        assert _sampled_gate_parity(O, keys630, nl, p, per_level=4, levels=6, seed=4) >= 20


def test_netlist_edge_cases(O, keys630, gpu630):
    # no gates: outputs are inputs
    nl0 = I.Netlist(3, np.zeros(0, np.uint8), *(np.zeros(0, np.uint32),) * 3, np.array([2, 0], np.uint32))
    bits, ct = _encrypt_inputs(O, keys630, nl0, 500)
    out = np.zeros((2, 631), np.uint32)
    arx.eval_netlist(nl0, ct, out)
    assert np.array_equal(out, ct[[2, 0]])
    # linear-only chain and constants, MUX-heavy netlist
    B = I.Builder(3)
    w = B.NOT(0)
    w = B.NOT(w)
    c1 = B.gate(I.CONST1)
    m = B.MUX(0, 1, 2)
    m2 = B.MUX(m, c1, B.NOT(1))
    cp = B.gate(I.COPY, m2)
    nl = B.build([w, c1, m, m2, cp])
    for trial in range(2):
        bits, ct = _encrypt_inputs(O, keys630, nl, 510 + trial)
        out = np.zeros((len(nl.outputs), 631), np.uint32)
        arx.eval_netlist(nl, ct, out)
        assert np.array_equal(out, keys630.ctx.eval_netlist(nl, ct))
        assert np.array_equal(arx.client_decrypt(630, keys630.s, out), nl.plain_eval(bits))


def test_plan_keeps_keyset_busy(gpu630, keys64, torch_cuda):
    ks = arx.load_keys(keys64.bsk, keys64.ksk, 64)
    p = arx.Plan(I.comparator(2), keyset=ks, mode=arx.MODE_PLAIN)
    with pytest.raises(arx.ArxError) as e:
        arx.unload_keys(ks)
    assert e.value.code == -7
    p.close()
    arx.unload_keys(ks)
    arx.use_keys(gpu630)


# --------------------------------------------------------------------------
# the paper's own parameter set: n = 512, gadget l = 2 (Bg = 2^10)
# --------------------------------------------------------------------------
def test_gadget_l2_all_gate_types_bit_exact(O, keys512_l2, _loaded512_l2):
    k, ks = keys512_l2, _loaded512_l2
    types = np.array([t for t in range(11) for _ in range(4)], np.uint8)
    xs, ys, zs = (I.random_bits(400 + j, len(types)) for j in range(3))
    ca, cb, cc = (k.encrypt(O, I, v, 410 + j) for j, v in enumerate((xs, ys, zs)))
    out = np.zeros_like(ca)
    arx.bootstrap_gates_ex(types, ca, cb, cc, out, keyset=ks)
    assert np.array_equal(out, k.ctx.gates(types, ca, cb, cc))
    assert np.array_equal(arx.client_decrypt(512, k.s, out), _truth(types, xs, ys, zs))


@pytest.mark.parametrize("mode", [arx.MODE_PLAIN, arx.MODE_GRAPH])
def test_gadget_l2_netlist_and_shapes(O, keys512_l2, _loaded512_l2, mode):
    k, ks = keys512_l2, _loaded512_l2
    nl = I.union([I.ripple_carry_adder(4), I.comparator(3)])
    bits = I.random_bits(420, nl.num_inputs)
    ct = k.encrypt(O, I, bits, 421)
    out = np.zeros((len(nl.outputs), 513), np.uint32)
    with arx.Plan(nl, keyset=ks, mode=mode) as p:
        sh = [(H, GT) for H, GT, j in p.shapes() if j]
        assert set(sh) <= {(80, 1), (40, 1)} and (80, 1) in sh, sh  # the l = 2 cluster kernels
        p.run(ct, out)
    assert np.array_equal(out, k.ctx.eval_netlist(nl, ct))
    assert np.array_equal(arx.client_decrypt(512, k.s, out), nl.plain_eval(bits))


@pytest.mark.parametrize("count", [24, 40])
def test_gadget_l2_wave_wider_than_the_device_sampled(O, keys512_l2, _loaded512_l2, count):
    # 24: more gates than co-resident eight-CTA clusters (the persistent loop
    # takes two tiles per cluster); 40: the throughput kernel br_kernel<H, GT, 2>
    k, ks = keys512_l2, _loaded512_l2
    types = I.random_gate_types(430, count)
    xs, ys = I.random_bits(431, count), I.random_bits(432, count)
    ca, cb = k.encrypt(O, I, xs, 433), k.encrypt(O, I, ys, 434)
    out = np.zeros_like(ca)
    arx.bootstrap_gates_ex(types, ca, cb, ca, out, keyset=ks)
    assert np.array_equal(arx.client_decrypt(512, k.s, out), _truth(types, xs, ys, xs))
    pick = np.array([0, 13, count - 11, count - 1])
    assert np.array_equal(out[pick], k.ctx.gates(types[pick], ca[pick], cb[pick]))


# l = 3 override -> the l = 2 throughput shape it maps to (kGadget2 + H, GT)
GADGET2_SHAPES = [((1, 1), (101, 1)), ((1, 2), (101, 2)), ((1, 4), (101, 4)), ((1, 6), (101, 6)),
                  ((2, 1), (102, 1)), ((2, 3), (102, 3)), ((3, 2), (102, 3)), ((6, 1), (104, 1))]


def test_gadget_l2_every_throughput_shape_ragged(O, keys512_l2, _loaded512_l2):
    """37 gates (a ragged tail for every gates-per-CTA tile) under each l = 2
    throughput shape, every output against the oracle."""
    k, ks = keys512_l2, _loaded512_l2
    types = np.array([I.BINARY_OPS[j % 6] if j % 9 else I.MUX for j in range(37)], np.uint8)
    xs, ys, zs = (I.random_bits(440 + j, len(types)) for j in range(3))
    ca, cb, cc = (k.encrypt(O, I, v, 443 + j) for j, v in enumerate((xs, ys, zs)))
    want = k.ctx.gates(types, ca, cb, cc)
    nl = I.union([I.array_multiplier(6)])
    try:
        for (H, GT), mapped in GADGET2_SHAPES:
            arx.set_launch_shape(H, GT)
            out = np.zeros_like(ca)
            arx.bootstrap_gates_ex(types, ca, cb, cc, out, keyset=ks)
            assert np.array_equal(out, want), (H, GT)
            with arx.Plan(nl, keyset=ks, mode=arx.MODE_PLAIN) as p:
                assert all((h, g) == mapped for h, g, j in p.shapes() if j), (H, GT)
    finally:
        arx.set_launch_shape(0, 0)


def test_gadget_l2_wide_netlist_takes_the_throughput_kernel(O, keys512_l2, _loaded512_l2):
    k, ks = keys512_l2, _loaded512_l2
    nl = I.union([I.array_multiplier(8)])  # a 64-gate first wave, then narrow ones
    bits = I.random_bits(450, nl.num_inputs)
    ct = k.encrypt(O, I, bits, 451)
    out = np.zeros((len(nl.outputs), 513), np.uint32)
    # plain mode keeps the Sec. 4.2 levels (graph plans would spread the wide wave)
    with arx.Plan(nl, keyset=ks, mode=arx.MODE_PLAIN) as p:
        sh = p.shapes()
        assert any(H > 100 for H, GT, j in sh if j > 30) and all(H in (80, 40) for H, GT, j in sh if 0 < j <= 30)
        assert all(H == 40 for H, GT, j in sh if 16 <= j <= 30) and any(H == 80 for H, GT, j in sh if 0 < j <= 7)
        p.run(ct, out)
        assert _sampled_gate_parity(O, k, nl, p, per_level=4, levels=6) >= 6
    assert np.array_equal(arx.client_decrypt(512, k.s, out), nl.plain_eval(bits))


@pytest.mark.parametrize("count", [1, 7, 20])
def test_gadget_l2_sixteen_cta_kernel(O, keys512_l2, _loaded512_l2, count):
    # the sixteen-CTA kernel of the gadget l = 2 (shape (80, 1)): one wave of up
    # to 7 gates by the automatic choice; 20 gates through the (96, 1) override,
    # which maps to it and takes three rounds of its clusters
    k, ks = keys512_l2, _loaded512_l2
    types = np.array([I.BINARY_OPS[j % 6] if j % 5 else I.MUX for j in range(count)], np.uint8)
    xs, ys, zs = (I.random_bits(460 + j, count) for j in range(3))
    ca, cb, cc = (k.encrypt(O, I, v, 463 + j) for j, v in enumerate((xs, ys, zs)))
    out = np.zeros_like(ca)
    try:
        if count > 7:
            arx.set_launch_shape(96, 1)
        arx.bootstrap_gates_ex(types, ca, cb, cc, out, keyset=ks)
        nl = I.union([I.ripple_carry_adder(2)])
        with arx.Plan(nl, keyset=ks, mode=arx.MODE_PLAIN) as p:
            assert all((H, GT) == (80, 1) for H, GT, j in p.shapes() if j)
    finally:
        arx.set_launch_shape(0, 0)
    assert np.array_equal(out, k.ctx.gates(types, ca, cb, cc))
    assert np.array_equal(arx.client_decrypt(512, k.s, out), _truth(types, xs, ys, zs))


def test_gadget_l2_shape_is_not_an_override(gpu630):
    for H, GT in ((40, 1), (80, 1), (101, 6), (104, 1)):
        with pytest.raises(arx.ArxError):
            arx.set_launch_shape(H, GT)
    with pytest.raises(arx.ArxError):
        arx._check(arx.lib().arx_load_keys_gadget(None, None, 512, 2, 7, None))
