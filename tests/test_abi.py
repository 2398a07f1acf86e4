"""CPU checks of the C-ABI library: it loads, exports every symbol include/arx.h
declares, and its host-only entry points (wave levelization, client-side key
generation, encryption, decryption) agree with the oracle and the definitions.
No call here touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2306_11006_gb300 import arx
from paper_2306_11006_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "arx.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(arx_[a-z_0-9]+)\s*\(", text))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 20
    h = ctypes.CDLL(arx.LIB_PATH)
    for n in sorted(names):
        assert hasattr(h, n), n
    assert names == set(arx.SIGNATURES), names ^ set(arx.SIGNATURES)


def test_watchdog_selftest_rejects_bad_limits_without_a_device():
    # checked before the library touches CUDA, so this runs without a GPU
    for limit in (0, 999, 4_000_000_001):
        rc, gave_up = arx.watchdog_selftest(False, limit)
        assert (rc, gave_up) == (-1, -1), limit


def test_header_gate_numbering_matches_oracle(O):
    text = open(HEADER).read()
    body = text[text.index("ARX_AND = 0"): text.index("} arx_gate;")]
    names = [t.strip() for t in body.replace("\n", " ").split(",") if t.strip()]
    names[0] = "ARX_AND"
    assert names == ["ARX_AND", "ARX_NAND", "ARX_OR", "ARX_NOR", "ARX_XOR", "ARX_XNOR", "ARX_NOT",
                     "ARX_MUX", "ARX_COPY", "ARX_CONST0", "ARX_CONST1"]
    assert [O.AND, O.NAND, O.OR, O.NOR, O.XOR, O.XNOR, O.NOT, O.MUX, O.COPY, O.CONST0, O.CONST1] == list(range(11))
    assert [I.AND, I.MUX, I.CONST1] == [0, 7, 10]


@pytest.mark.parametrize("which", ["adder", "mult", "cmp", "dag", "matmul_small"])
def test_levelize_matches_oracle(O, which):
    nl = {"adder": lambda: I.ripple_carry_adder(32), "mult": lambda: I.array_multiplier(8),
          "cmp": lambda: I.comparator(16),
          "dag": lambda: I.random_dag(seed=3, total=4096, levels=12, num_inputs=256, wmin=64, wmax=1024),
          "matmul_small": lambda: I.matmul4x4(bits=3, acc_bits=6, dim=2)}[which]()
    wave, depth = arx.levelize(nl)
    rc, owave = O.levelize(nl)
    assert rc == 0
    assert np.array_equal(wave, owave)
    assert depth == int(owave.max()) + 1


def test_levelize_dag_depth_is_exact():
    nl = I.random_dag(seed=7, total=2000, levels=9, num_inputs=100, wmin=100, wmax=400)
    wave, depth = arx.levelize(nl)
    assert depth == 9
    widths = np.bincount(wave, minlength=9)
    assert np.array_equal(widths, nl.meta["widths"])


def test_levelize_gates_in_any_order(O):
    nl = I.ripple_carry_adder(6)
    perm = np.random.default_rng(0).permutation(nl.num_gates)
    inv = np.argsort(perm)
    remap = lambda w: np.where(w < nl.num_inputs, w, nl.num_inputs + inv[np.maximum(w, nl.num_inputs) - nl.num_inputs])
    shuffled = I.Netlist(nl.num_inputs, nl.type[perm], remap(nl.in0[perm]).astype(np.uint32),
                         remap(nl.in1[perm]).astype(np.uint32), remap(nl.in2[perm]).astype(np.uint32),
                         remap(nl.outputs).astype(np.uint32))
    w0, d0 = arx.levelize(nl)
    w1, d1 = arx.levelize(shuffled)
    assert d0 == d1
    assert np.array_equal(w1, w0[perm])
    assert np.array_equal(w1, O.levelize(shuffled)[1])


def test_levelize_errors():
    nl = I.ripple_carry_adder(2)
    cyc = I.Netlist(nl.num_inputs, nl.type.copy(), nl.in0.copy(), nl.in1.copy(), nl.in2.copy(), nl.outputs.copy())
    cyc.in0[0] = nl.num_inputs + 3
    cyc.in1[3] = nl.num_inputs + 0
    with pytest.raises(arx.ArxError) as e:
        arx.levelize(cyc)
    assert e.value.code == -4
    bad = I.Netlist(nl.num_inputs, nl.type.copy(), nl.in0.copy(), nl.in1.copy(), nl.in2.copy(), nl.outputs.copy())
    bad.in1[1] = nl.num_inputs + nl.num_gates
    with pytest.raises(arx.ArxError) as e:
        arx.levelize(bad)
    assert e.value.code == -1
    badt = I.Netlist(nl.num_inputs, nl.type.copy(), nl.in0.copy(), nl.in1.copy(), nl.in2.copy(), nl.outputs.copy())
    badt.type[0] = 11
    with pytest.raises(arx.ArxError) as e:
        arx.levelize(badt)
    assert e.value.code == -1
    empty = I.Netlist(3, np.zeros(0, np.uint8), *(np.zeros(0, np.uint32),) * 3, np.arange(3, dtype=np.uint32))
    w, d = arx.levelize(empty)
    assert d == 0 and len(w) == 0


@pytest.mark.parametrize("n,seed", [(8, 1), (630, 0)])
def test_client_keygen_matches_oracle(O, n, seed):
    kr = I.key_randomness(seed, n)
    bsk, ksk = arx.client_keygen(kr)
    obsk, oksk = O.keygen(kr)
    assert np.array_equal(bsk, obsk)
    assert np.array_equal(ksk, oksk)


@pytest.mark.parametrize("n", [5, 512])
def test_client_keygen_gadget_l2_matches_oracle(O, n):
    kr = I.key_randomness(8, n, l=2)
    bsk, ksk = arx.client_keygen(kr)
    assert bsk.shape == (n, 4, 2, 1024)
    obsk, oksk = O.keygen(kr)
    assert np.array_equal(bsk, obsk)
    assert np.array_equal(ksk, oksk)


def test_client_keygen_rejects_other_gadgets():
    kr = I.key_randomness(8, 4)
    arrs = [np.ascontiguousarray(a) for a in (kr.s, kr.K, kr.bsk_mask, kr.bsk_noise, kr.ksk_mask, kr.ksk_noise)]
    out = np.zeros((4, 6, 2, 1024), np.uint32), np.zeros((1024, 8, 4, 5), np.uint32)
    rc = arx.lib().arx_client_keygen_gadget(4, 3, 10, *[arx._ptr(a) for a in arrs], arx._ptr(out[0]),
                                            arx._ptr(out[1]))
    assert rc == -1  # ARX_EINVAL


def test_client_encrypt_decrypt_match_oracle(O):
    n = 630
    kr = I.key_randomness(3, n)
    bits = I.random_bits(4, 500)
    m, e = I.encryption_randomness(5, 500, n)
    ct = arx.client_encrypt(n, kr.s, m, e, bits)
    assert np.array_equal(ct, O.encrypt(n, kr.s, m, e, bits))
    assert np.array_equal(arx.client_decrypt(n, kr.s, ct), bits)
    assert np.array_equal(arx.client_decrypt(n, kr.s, ct), O.decrypt(n, kr.s, ct)[0])


def test_keyset_bytes():
    assert arx.keyset_bytes(630) == 630 * 6 * 16384 + (1024 * 8 * 3 * 632 + 640) * 4  # + the zero row
    assert arx.keyset_bytes(0) == 0


class _FakeTensor:
    """Stands in for a torch tensor's metadata (no device memory is touched)."""

    def __init__(self, shape, dtype="torch.int32", is_cuda=True, contiguous=True):
        self.shape, self.dtype, self.is_cuda, self._c = tuple(shape), dtype, is_cuda, contiguous

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return self._c


@pytest.mark.parametrize("case", ["host", "dtype", "noncontig", "rows_N", "rows_n", "count_in", "count_out",
                                  "negative"])
def test_keyswitch_noalloc_argument_checks(case):
    n = 630
    good_in, good_out = _FakeTensor((8, 1025)), _FakeTensor((8, n + 1))
    args = {"host": (_FakeTensor((8, 1025), is_cuda=False), good_out, 8),
            "dtype": (good_in, _FakeTensor((8, n + 1), dtype="torch.int64"), 8),
            "noncontig": (_FakeTensor((8, 1025), contiguous=False), good_out, 8),
            "rows_N": (_FakeTensor((8, 1024)), good_out, 8),
            "rows_n": (good_in, _FakeTensor((8, 513)), 8),
            "count_in": (_FakeTensor((4, 1025)), good_out, 8),
            "count_out": (good_in, _FakeTensor((4, n + 1)), 8),
            "negative": (good_in, good_out, -1)}[case]
    with pytest.raises(arx.ArxError) as e:
        arx._check_noalloc_args(*args, n)
    assert e.value.code == -1
    arx._check_noalloc_args(good_in, good_out, 8, n)  # the valid form passes
