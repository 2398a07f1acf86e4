"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own arithmetic: big-integer Python,
closed forms, brute force on small inputs, and special cases whose result is known
exactly.  A plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand, a row-order mix-up) fails at least one of them.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
N = 1024
MASK32 = (1 << 32) - 1


def golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "ntt_constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = int(v)
    return out


def negamul_mod32(a, b):
    """Negacyclic product mod (X^N + 1, 2^32) by the schoolbook definition."""
    a = np.asarray(a, np.uint64)
    b = np.asarray(b, np.uint64)
    m = len(a)
    M = np.multiply.outer(a, b)  # wraps mod 2^64, harmless for a mod 2^32 result
    idx = np.add.outer(np.arange(m), np.arange(m))
    S = np.zeros(2 * m, np.uint64)
    np.add.at(S, idx.ravel(), M.ravel())
    return ((S[:m] - S[m:]) & np.uint64(MASK32)).astype(np.uint32)


def phase_trlwe(mask, body, K):
    return (np.asarray(body, np.uint32) - negamul_mod32(mask, K)).astype(np.uint32)


# --------------------------------------------------------------------------
# Sec. 5.4 constants
# --------------------------------------------------------------------------
def test_golden_constants_match_paper_formula(O):
    c = golden_constants()
    assert c["Q"] == 2 ** 64 - 2 ** 32 + 1
    Q, g = c["Q"], c["g"]
    # g has multiplicative order exactly 2^32: g^(2^32) = 1 and g^(2^31) = -1
    assert pow(g, 2 ** 32, Q) == 1
    assert pow(g, 2 ** 31, Q) == Q - 1
    psi = pow(g, 2 ** 21, Q)
    assert pow(psi, 1024, Q) == Q - 1          # negacyclic 2048-th root
    assert pow(psi, 32, Q) == 8                 # "multiplications become bitshifts"
    assert pow(2, 96, Q) == Q - 1
    assert O.gl_pow(g, 2 ** 31) == Q - 1


def test_goldilocks_mul_matches_bigint(O):
    Q = golden_constants()["Q"]
    rng = np.random.default_rng(11)
    edge = [0, 1, 2, Q - 1, Q - 2, 2 ** 32, 2 ** 32 - 1, 2 ** 63, Q // 2, 2 ** 64 - 2 ** 32]
    vals = edge + [int(x) % Q for x in rng.integers(0, 2 ** 63, 200, dtype=np.int64) * 2 + 1]
    for a in vals:
        for b in vals[:25]:
            assert O.gl_mul(a % Q, b % Q) == (a % Q) * (b % Q) % Q


# --------------------------------------------------------------------------
# negacyclic NTT
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_ntt_is_the_odd_power_evaluation(O, m):
    """A[k] = sum_j a_j psi^((2k+1) j), psi = g^(2^32 / 2m), by big integers."""
    c = golden_constants()
    Q, g = c["Q"], c["g"]
    psi = pow(g, 2 ** 32 // (2 * m), Q)
    rng = np.random.default_rng(m)
    a = [int(x) for x in rng.integers(0, 2 ** 62, m, dtype=np.int64)]
    A = O.ntt(np.array(a, np.uint64))
    for k in range(m):
        want = sum(a[j] * pow(psi, (2 * k + 1) * j, Q) for j in range(m)) % Q
        assert int(A[k]) == want
    back = O.ntt(A, inverse=True)
    assert [int(x) for x in back] == [x % Q for x in a]


def _bigint_negacyclic(a, b):
    m = len(a)
    c = [0] * m
    for i in range(m):
        for j in range(m):
            if i + j < m:
                c[i + j] += a[i] * b[j]
            else:
                c[i + j - m] -= a[i] * b[j]
    return c


@pytest.mark.parametrize("m", [2, 4, 8, 16, 32, 64])
def test_ntt_product_equals_schoolbook_small(O, m):
    rng = np.random.default_rng(100 + m)
    for trial in range(20):
        a = rng.integers(-2 ** 31, 2 ** 31, m, dtype=np.int64)
        b = rng.integers(-64, 64, m, dtype=np.int64)
        want = _bigint_negacyclic([int(x) for x in a], [int(x) for x in b])
        assert [int(x) for x in O.negacyclic_mul(a, b, schoolbook=True)] == want
        assert [int(x) for x in O.negacyclic_mul(a, b)] == want


def test_ntt_product_equals_schoolbook_1024(O):
    rng = np.random.default_rng(7)
    for trial in range(3):
        a = rng.integers(-2 ** 31, 2 ** 31, N, dtype=np.int64)
        b = rng.integers(-64, 64, N, dtype=np.int64)
        assert np.array_equal(O.negacyclic_mul(a, b), O.negacyclic_mul(a, b, schoolbook=True))
    # extreme magnitudes: every term at its bound, the sum still below Q/2
    a = np.full(N, -2 ** 31, np.int64)
    b = np.full(N, -64, np.int64)
    assert np.array_equal(O.negacyclic_mul(a, b), O.negacyclic_mul(a, b, schoolbook=True))


# --------------------------------------------------------------------------
# scalar roundings
# --------------------------------------------------------------------------
EDGES = [0, 1, 2 ** 31, 2 ** 31 - 1, 2 ** 32 - 1, 2 ** 20, 2 ** 20 - 1, 2 ** 21 - 2 ** 20,
         2 ** 10, 2 ** 10 - 1, 2 ** 15, 2 ** 15 - 1, 3 << 29, 5 << 29, 7 << 29]


def _edge_and_random(seed, count=3000):
    rng = np.random.default_rng(seed)
    half_points = [k * 2 ** 11 + 2 ** 10 + d for k in (0, 1, 12345, 2 ** 21 - 1) for d in (-1, 0, 1)]
    half_points += [k * 2 ** 21 + 2 ** 20 + d for k in (0, 1, 777, 2047) for d in (-1, 0, 1)]
    half_points += [k * 2 ** 16 + 2 ** 15 + d for k in (0, 1, 999, 2 ** 16 - 1) for d in (-1, 0, 1)]
    return [x & MASK32 for x in EDGES + half_points] + [int(x) for x in rng.integers(0, 2 ** 32, count)]


def test_modswitch_rounds_half_up_mod_2N(O):
    for x in _edge_and_random(1):
        # floor(x * 2N / 2^32 + 1/2) mod 2N, with exact integer arithmetic
        want = ((2 * x * 2048 + 2 ** 32) // (2 * 2 ** 32)) % 2048
        assert O.modswitch(x) == want


def test_decomposition_recomposes_rounded_value(O):
    for x in _edge_and_random(2):
        d = [int(v) for v in O.decompose(x)]
        assert all(-64 <= v < 64 for v in d)
        rounded = (((2 * x + 2 ** 11) // 2 ** 12) * 2 ** 11) & MASK32   # round to 21 bits
        recomposed = sum(d[p] * 2 ** (32 - 7 * (p + 1)) for p in range(3)) & MASK32
        assert recomposed == rounded


def test_decomposition_unique_brute_force(O):
    """Digits in [-64, 64) with a given recomposition are unique: exhaustive for a
    handful of values over all 128^3 candidate triples (vectorised)."""
    d = np.arange(-64, 64, dtype=np.int64)
    grid = (d[:, None, None] * 2 ** 25 + d[None, :, None] * 2 ** 18 + d[None, None, :] * 2 ** 11) & MASK32
    for x in (0, 2 ** 31, 0xDEADBEEF, 2 ** 32 - 1, 12345678):
        rounded = (((2 * x + 2 ** 11) // 2 ** 12) * 2 ** 11) & MASK32
        hits = np.argwhere(grid == rounded)
        assert len(hits) == 1
        assert [int(v) - 64 for v in hits[0]] == [int(v) for v in O.decompose(x)]


def test_keyswitch_digits_round_to_16_bits(O):
    for x in _edge_and_random(3):
        v = [int(t) for t in O.ks_digits(x)]
        assert all(0 <= t < 4 for t in v)
        rounded16 = ((2 * x + 2 ** 16) // 2 ** 17) % 2 ** 16
        assert sum(v[j] * 4 ** (7 - j) for j in range(8)) == rounded16


# --------------------------------------------------------------------------
# encryption and keys
# --------------------------------------------------------------------------
def test_encrypt_decrypt_phase(O, I):
    n = 630
    kr = I.key_randomness(1, n)
    bits = I.random_bits(2, 300)
    m, e = I.encryption_randomness(3, 300, n)
    ct = O.encrypt(n, kr.s, m, e, bits)
    dec, ph = O.decrypt(n, kr.s, ct)
    assert np.array_equal(dec, bits)
    # phase = b - <a,s> computed by Python integers
    for g in range(0, 300, 37):
        b = int(ct[g, n])
        inner = sum(int(ct[g, j]) * int(kr.s[j]) for j in range(n))
        want = (b - inner) & MASK32
        want = want - 2 ** 32 if want >= 2 ** 31 else want
        assert ph[g] == want
        assert want == int(e[g]) + (2 ** 29 if bits[g] else -2 ** 29)


def test_bsk_rows_encrypt_gadget_times_key_bit(O, I):
    """Phase of BSK row (c, p) is -s_i h_p K (c = 0) or s_i h_p (c = 1), plus noise."""
    n = 4
    kr = I.key_randomness(9, n)
    bsk, ksk = O.keygen(kr)
    for i in range(n):
        for r in range(6):
            c, p = divmod(r, 3)
            h = 2 ** (32 - 7 * (p + 1))
            ph = phase_trlwe(bsk[i, r, 0], bsk[i, r, 1], kr.K).astype(np.int64)
            want = np.zeros(N, np.int64)
            if c == 0:
                want = (-(int(kr.s[i]) * h) * kr.K.astype(np.int64))
            else:
                want[0] = int(kr.s[i]) * h
            want = (want + kr.bsk_noise[i, r].astype(np.int64)) & MASK32
            assert np.array_equal(ph & MASK32, want)
            assert np.array_equal(bsk[i, r, 0, 1:], kr.bsk_mask[i, r, 1:])


def test_ksk_rows_encrypt_scaled_key_bits(O, I):
    n = 16
    kr = I.key_randomness(4, n)
    bsk, ksk = O.keygen(kr)
    rng = np.random.default_rng(0)
    for i in rng.integers(0, N, 20):
        for j in range(1, 9):
            assert not ksk[i, j - 1, 0].any()
            for v in range(1, 4):
                row = ksk[i, j - 1, v]
                ph = (int(row[n]) - sum(int(row[q]) * int(kr.s[q]) for q in range(n))) & MASK32
                want = (v * int(kr.K[i]) * 2 ** (32 - 2 * j) + int(kr.ksk_noise[i, j - 1, v - 1])) & MASK32
                assert ph == want


# --------------------------------------------------------------------------
# bootstrapping pieces
# --------------------------------------------------------------------------
def test_sample_extract_matches_coefficient_zero_phase(O, I):
    rng = np.random.default_rng(5)
    K = rng.integers(0, 2, N).astype(np.uint8)
    acc = rng.integers(0, 2 ** 32, (2, N), dtype=np.uint32)
    lwe = O.sample_extract(acc)
    ph_poly = phase_trlwe(acc[0], acc[1], K)
    ph = (int(lwe[N]) - sum(int(lwe[j]) * int(K[j]) for j in range(N))) & MASK32
    assert ph == int(ph_poly[0])


def test_external_product_noiseless_is_key_bit_times_rounded_input(O, I):
    """With noiseless BSK (uniform masks), phase(BSK_i [x] (t0, t1)) equals
    s_i (round21(t1) - round21(t0) K) exactly, for random t0, t1."""
    n = 6
    kr = I.key_randomness(21, n, noiseless=True)
    bsk, ksk = O.keygen(kr)
    ctx = O.Context(n, bsk, ksk)
    rng = np.random.default_rng(3)
    r21 = lambda t: (((t.astype(np.uint64) + 2 ** 10) >> 11) << 11).astype(np.uint64) & MASK32
    for i in range(n):
        t0 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
        t1 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
        o0, o1 = ctx.external_product(i, t0, t1)
        got = phase_trlwe(o0, o1, kr.K)
        want = (r21(t1) - negamul_mod32(r21(t0).astype(np.uint32), kr.K)) & MASK32
        want = (want * int(kr.s[i])) & MASK32
        assert np.array_equal(got.astype(np.uint64), want.astype(np.uint64)), i


def _rotate_testv(e):
    """X^e * (mu sum_j X^j), coefficients as Python ints mod 2^32."""
    out = [0] * N
    for j in range(N):
        m = (j + e) % (2 * N)
        if m < N:
            out[m] = 2 ** 29
        else:
            out[m - N] = (-2 ** 29) & MASK32
    return out


def test_blind_rotation_trivial_key_closed_form(O, I):
    """Trivial noiseless BSK: ACC ends exactly as (0, X^-(bbar - sum abar_i s_i) testv)."""
    n = 12
    kr = I.key_randomness(8, n, trivial_bsk=True)
    bsk, ksk = O.keygen(kr)
    ctx = O.Context(n, bsk, ksk)
    rng = np.random.default_rng(1)
    for trial in range(4):
        abar = rng.integers(0, 2 * N, n).astype(np.uint32)
        bbar = int(rng.integers(0, 2 * N))
        acc = ctx.blind_rotate(abar, bbar)
        phi = (bbar - sum(int(abar[i]) * int(kr.s[i]) for i in range(n))) % (2 * N)
        assert not acc[0].any()
        assert [int(x) for x in acc[1]] == _rotate_testv((2 * N - phi) % (2 * N))


def test_keyswitch_noiseless_is_rounded_key_change(O, I):
    """Noiseless KSK: phase_s(KS(c)) = b' - sum_i round16(a'_i) K_i exactly."""
    n = 20
    kr = I.key_randomness(30, n, noiseless=True)
    bsk, ksk = O.keygen(kr)
    ctx = O.Context(n, bsk, ksk)
    rng = np.random.default_rng(4)
    for trial in range(3):
        lwe = rng.integers(0, 2 ** 32, N + 1, dtype=np.uint32)
        out = ctx.keyswitch(lwe)
        ph = (int(out[n]) - sum(int(out[q]) * int(kr.s[q]) for q in range(n))) & MASK32
        r16 = [((int(x) + 2 ** 15) >> 16 << 16) & MASK32 for x in lwe[:N]]
        want = (int(lwe[N]) - sum(r16[i] * int(kr.K[i]) for i in range(N))) & MASK32
        assert ph == want


def test_gate_linear_constants(O, I):
    """Fig. 2 top box: phases of the linear pre-combination on exact +-1/8 inputs."""
    n = 8
    kr = I.key_randomness(2, n)
    eighth = 2 ** 29
    table = {0: (-eighth, 1, 1), 1: (eighth, -1, 1), 2: (eighth, 1, 1), 3: (-eighth, -1, 1),
             4: (2 * eighth, 1, 2), 5: (-2 * eighth, -1, 2)}
    for t, (cst, sign, scale) in table.items():
        for x in (0, 1):
            for y in (0, 1):
                m, e = I.encryption_randomness(t * 4 + x * 2 + y, 2, n, noiseless=True)
                ct = O.encrypt(n, kr.s, m, e, np.array([x, y], np.uint8))
                lin = O.gate_linear(n, t, ct[0], ct[1])
                _, ph = O.decrypt(n, kr.s, lin)
                mx = eighth if x else -eighth
                my = eighth if y else -eighth
                want = (cst + sign * scale * (mx + my)) & MASK32
                assert int(ph[0]) & MASK32 == want


# --------------------------------------------------------------------------
# gates end to end
# --------------------------------------------------------------------------
def _truth(I, t, x, y, z=0):
    return I._plain_gate(t, [x, y, z])


@pytest.mark.parametrize("seed", [0, 1])
def test_gate_truth_tables_n630(O, I, keys630, seed):
    types, xs, ys = [], [], []
    for t in range(11):
        if t == 7:
            continue
        for x in (0, 1):
            for y in (0, 1):
                types.append(t); xs.append(x); ys.append(y)
    ca = keys630.encrypt(O, I, xs, 1000 + seed)
    cb = keys630.encrypt(O, I, ys, 2000 + seed)
    out = keys630.ctx.gates(np.array(types, np.uint8), ca, cb)
    dec, ph = O.decrypt(630, keys630.s, out)
    want = [_truth(I, t, x, y) for t, x, y in zip(types, xs, ys)]
    assert list(dec) == want
    # every output phase sits near +-1/8 (fresh bootstrap noise is ~3e-3 of the torus)
    assert np.all(np.abs(np.abs(ph.astype(np.float64)) / 2 ** 32 - 0.125) < 0.03)


def test_mux_truth_table_n630(O, I, keys630):
    combos = [(s, t, f) for s in (0, 1) for t in (0, 1) for f in (0, 1)]
    cs = keys630.encrypt(O, I, [c[0] for c in combos], 31)
    ct = keys630.encrypt(O, I, [c[1] for c in combos], 32)
    cf = keys630.encrypt(O, I, [c[2] for c in combos], 33)
    out = keys630.ctx.gates(np.full(8, 7, np.uint8), cs, ct, cf)
    dec, _ = O.decrypt(630, keys630.s, out)
    assert list(dec) == [t if s else f for s, t, f in combos]


def expected_output_noise(kr):
    """Closed-form mean and variance (torus units) of a fresh gate output's phase
    error, conditional on the realised key noise (fixed for a key), with the
    gadget digits uniform on [-64, 64) (mean -1/2, variance (128^2-1)/12) and the
    key-switch digits uniform on {0,1,2,3}.

    Blind rotation: coefficient 0 of each CMux's external product collects
    sum_r (d_r[0] e_r[0] - sum_{j>0} d_r[j] e_r[N-j]) over the 6 rows' noise e_r.
    Key switch: for each (i, j) the subtracted noise is e_ij(v), v uniform, e(0) = 0.
    Roundings: 16-bit key-switch rounding of N mask terms against a binary key,
    and 21-bit decomposition rounding (about n/2 * (N/2 + 1) * 2^-42 / 12).
    """
    n = kr.n
    var_d = (128.0 ** 2 - 1) / 12
    e = kr.bsk_noise.astype(np.float64) / 2 ** 32                     # [n][6][N]
    signed = np.concatenate([e[..., :1], -e[..., :0:-1]], axis=-1)     # e[0], -e[N-j]
    br_mean = -0.5 * signed.sum()
    br_var = var_d * np.sum(e ** 2)
    ek = kr.ksk_noise.astype(np.float64) / 2 ** 32                    # [N][8][3]
    m_ij = ek.sum(axis=2) / 4
    ks_mean = -m_ij.sum()
    ks_var = np.sum((ek ** 2).sum(axis=2) / 4 - m_ij ** 2)
    rounding = (N / 2) * 2.0 ** -32 / 12 + (n / 2) * (N / 2 + 1) * 2.0 ** -42 / 12
    return br_mean + ks_mean, br_var + ks_var + rounding


@pytest.mark.parametrize("which,m", [("keys64", 1536), ("keys630", 192)])
def test_output_noise_matches_closed_form(O, I, which, m, request):
    from scipy import stats
    keys = request.getfixturevalue(which)
    n = keys.n
    xs = I.random_bits(40, m)
    ys = I.random_bits(41, m)
    types = I.random_gate_types(42, m)
    out = keys.ctx.gates(types, keys.encrypt(O, I, xs, 43), keys.encrypt(O, I, ys, 44))
    dec, ph = O.decrypt(n, keys.s, out)
    want = np.array([_truth(I, int(t), int(x), int(y)) for t, x, y in zip(types, xs, ys)])
    assert np.array_equal(dec, want)
    err = (ph.astype(np.float64) - np.where(want == 1, 2.0 ** 29, -2.0 ** 29)) / 2 ** 32
    mean, var = expected_output_noise(keys.kr)
    assert abs(err.mean() - mean) < 4 * np.sqrt(var / m)
    stat = np.sum((err - mean) ** 2) / var
    lo, hi = stats.chi2.ppf([0.0005, 0.9995], m)
    assert lo < stat < hi, (stat, lo, hi, err.var(), var)
    # and below the worst-case bound (every digit at |64|, every KS digit non-zero)
    bound = n * 6 * N * 64.0 ** 2 * 2.0 ** -50 + N * 8 * 2.0 ** -30 + N * 2.0 ** -32 / 12
    assert err.var() < bound


# --------------------------------------------------------------------------
# netlists (Sec. 4.2)
# --------------------------------------------------------------------------
def _waves_by_definition(I, nl):
    """wave(g) = 0 with no gate inputs, else 1 + max over gate inputs (recursive)."""
    memo = {}

    def wave(g):
        if g in memo:
            return memo[g]
        t = int(nl.type[g])
        ins = (int(nl.in0[g]), int(nl.in1[g]), int(nl.in2[g]))[: I.ARITY[t]]
        preds = [w - nl.num_inputs for w in ins if w >= nl.num_inputs]
        memo[g] = 0 if not preds else 1 + max(wave(p) for p in preds)
        return memo[g]

    import sys
    sys.setrecursionlimit(100000)
    return [wave(g) for g in range(nl.num_gates)]


def test_levelize_matches_definition(O, I):
    for nl in (I.ripple_carry_adder(8), I.array_multiplier(4), I.comparator(6),
               I.random_dag(seed=9, total=600, levels=7, num_inputs=40, wmin=40, wmax=150)):
        rc, wave = O.levelize(nl)
        assert rc == 0
        assert list(wave) == _waves_by_definition(I, nl)


def test_levelize_rejects_cycles_and_bad_wires(O, I):
    nl = I.ripple_carry_adder(2)
    bad = I.Netlist(nl.num_inputs, nl.type.copy(), nl.in0.copy(), nl.in1.copy(), nl.in2.copy(),
                    nl.outputs.copy())
    bad.in0[0] = nl.num_inputs + 3          # gate 0 reads gate 3 which reads gate 0
    bad.in1[3] = nl.num_inputs + 0
    assert O.levelize(bad)[0] == -2
    bad2 = I.Netlist(nl.num_inputs, nl.type.copy(), nl.in0.copy(), nl.in1.copy(), nl.in2.copy(),
                     nl.outputs.copy())
    bad2.in1[1] = nl.num_inputs + nl.num_gates  # out of range
    assert O.levelize(bad2)[0] == -1


def test_netlist_adder_and_multiplier_decrypt_to_integer_results(O, I, keys64):
    rng = np.random.default_rng(77)
    for nl, width, fn in ((I.ripple_carry_adder(4), 4, lambda a, b, c: a + b + c),
                          (I.array_multiplier(3), 3, lambda a, b, c: a * b)):
        a, b = (int(v) for v in rng.integers(0, 2 ** width, 2))
        c = int(rng.integers(0, 2))
        bits = I.int_to_bits(a, width) + I.int_to_bits(b, width)
        if nl.num_inputs > 2 * width:
            bits.append(c)
        assert I.bits_to_int(nl.plain_eval(bits)) == fn(a, b, c)
        ct = keys64.encrypt(O, I, bits, 5)
        out = keys64.ctx.eval_netlist(nl, ct)
        dec, _ = O.decrypt(keys64.n, keys64.s, out)
        assert I.bits_to_int(dec) == fn(a, b, c)
