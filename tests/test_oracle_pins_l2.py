"""Pins of the oracle's l = 2 variant (Bg = 2^10): the paper's own parameter
set (Sec. 6: n = 512; Fig. 2: 4 forward DFTs, i.e. (k+1) l = 4)."""
import numpy as np
import pytest

from test_oracle_pins import MASK32, N, _edge_and_random, _truth, negamul_mod32, phase_trlwe


def _round20(x):
    return (((2 * x + 2 ** 12) // 2 ** 13) * 2 ** 12) & MASK32


def test_decomposition_recomposes_rounded_value_l2(O):
    for x in _edge_and_random(12):
        d = [int(v) for v in O.decompose(x, 2)]
        assert all(-512 <= v < 512 for v in d)
        assert (d[0] * 2 ** 22 + d[1] * 2 ** 12) & MASK32 == _round20(x)


def test_decomposition_unique_brute_force_l2(O):
    """Over all 1024^2 digit pairs exactly one recomposes to the rounded value."""
    d = np.arange(-512, 512, dtype=np.int64)
    grid = (d[:, None] * 2 ** 22 + d[None, :] * 2 ** 12) & MASK32
    for x in (0, 2 ** 31, 0xDEADBEEF, 2 ** 32 - 1, 12345678, 2 ** 11, 2 ** 12 - 1):
        hits = np.argwhere(grid == _round20(x))
        assert len(hits) == 1
        assert [int(v) - 512 for v in hits[0]] == [int(v) for v in O.decompose(x, 2)]


def test_bsk_rows_encrypt_gadget_times_key_bit_l2(O, I):
    n = 3
    kr = I.key_randomness(19, n, l=2)
    bsk, _ = O.keygen(kr)
    assert bsk.shape == (n, 4, 2, N)
    for i in range(n):
        for r in range(4):
            c, p = divmod(r, 2)
            h = 2 ** (32 - 10 * (p + 1))
            ph = phase_trlwe(bsk[i, r, 0], bsk[i, r, 1], kr.K).astype(np.int64)
            want = np.zeros(N, np.int64)
            if c == 0:
                want = -(int(kr.s[i]) * h) * kr.K.astype(np.int64)
            else:
                want[0] = int(kr.s[i]) * h
            assert np.array_equal(ph & MASK32, (want + kr.bsk_noise[i, r].astype(np.int64)) & MASK32)


def test_external_product_noiseless_l2(O, I):
    """phase(BSK_i [x] (t0, t1)) = s_i (round20(t1) - round20(t0) K) exactly."""
    n = 4
    kr = I.key_randomness(23, n, noiseless=True, l=2)
    bsk, ksk = O.keygen(kr)
    ctx = O.Context(n, bsk, ksk)
    assert ctx.l == 2
    rng = np.random.default_rng(4)
    r20 = lambda t: (((t.astype(np.uint64) + 2 ** 11) >> 12) << 12).astype(np.uint64) & MASK32
    for i in range(n):
        t0 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
        t1 = rng.integers(0, 2 ** 32, N, dtype=np.uint32)
        o0, o1 = ctx.external_product(i, t0, t1)
        got = phase_trlwe(o0, o1, kr.K)
        want = (r20(t1) - negamul_mod32(r20(t0).astype(np.uint32), kr.K)) & MASK32
        want = (want * int(kr.s[i])) & MASK32
        assert np.array_equal(got.astype(np.uint64), want.astype(np.uint64)), i


def test_gate_and_mux_truth_tables_n512_l2(O, I, keys512_l2):
    k = keys512_l2
    types, xs, ys = [], [], []
    for t in range(11):
        if t == 7:
            continue
        for x in (0, 1):
            for y in (0, 1):
                types.append(t); xs.append(x); ys.append(y)
    out = k.ctx.gates(np.array(types, np.uint8), k.encrypt(O, I, xs, 301), k.encrypt(O, I, ys, 302))
    dec, ph = O.decrypt(512, k.s, out)
    assert list(dec) == [_truth(I, t, x, y) for t, x, y in zip(types, xs, ys)]
    assert np.all(np.abs(np.abs(ph.astype(np.float64)) / 2 ** 32 - 0.125) < 0.03)
    combos = [(s, t, f) for s in (0, 1) for t in (0, 1) for f in (0, 1)]
    cs, ct, cf = (k.encrypt(O, I, [c[j] for c in combos], 310 + j) for j in range(3))
    dec, _ = O.decrypt(512, k.s, k.ctx.gates(np.full(8, 7, np.uint8), cs, ct, cf))
    assert list(dec) == [t if s else f for s, t, f in combos]


def test_output_noise_matches_closed_form_l2(O, I, keys512_l2):
    """As the l = 3 closed form, with digits uniform on [-512, 512) over 4 rows and
    the 20-bit decomposition rounding."""
    from scipy import stats
    k, m = keys512_l2, 192
    xs, ys, types = I.random_bits(50, m), I.random_bits(51, m), I.random_gate_types(52, m)
    out = k.ctx.gates(types, k.encrypt(O, I, xs, 53), k.encrypt(O, I, ys, 54))
    dec, ph = O.decrypt(512, k.s, out)
    want = np.array([_truth(I, int(t), int(x), int(y)) for t, x, y in zip(types, xs, ys)])
    assert np.array_equal(dec, want)
    err = (ph.astype(np.float64) - np.where(want == 1, 2.0 ** 29, -2.0 ** 29)) / 2 ** 32
    e = k.kr.bsk_noise.astype(np.float64) / 2 ** 32
    signed = np.concatenate([e[..., :1], -e[..., :0:-1]], axis=-1)
    mean = -0.5 * signed.sum()
    var = (1024.0 ** 2 - 1) / 12 * np.sum(e ** 2)
    ek = k.kr.ksk_noise.astype(np.float64) / 2 ** 32
    m_ij = ek.sum(axis=2) / 4
    mean += -m_ij.sum()
    var += np.sum((ek ** 2).sum(axis=2) / 4 - m_ij ** 2)
    var += (N / 2) * 2.0 ** -32 / 12 + (512 / 2) * (N / 2 + 1) * 2.0 ** -40 / 12
    assert abs(err.mean() - mean) < 4 * np.sqrt(var / m)
    stat = np.sum((err - mean) ** 2) / var
    lo, hi = stats.chi2.ppf([0.0005, 0.9995], m)
    assert lo < stat < hi, (stat, lo, hi, err.var(), var)
