"""ctypes wrapper of the plain C CGGI oracle (oracle/cggi_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only callers.  The product package never imports this
module.  Everything here is argument marshalling; the arithmetic lives in the C
file, which follows the paper (ArctyrEX, arXiv 2306.11006) step by step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cggi_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
# the gadget variants: l -> (library, compile-time definitions)
VARIANTS = {3: (LIB, []), 2: (os.path.join(HERE, "liboracle_l2.so"), ["-DORC_L=2", "-DORC_BG_BITS=10"])}
BG_BITS = {3: 7, 2: 10}

N = 1024
L = 3
ROWS = 6
KS_T = 8
MU = 1 << 29

AND, NAND, OR, NOR, XOR, XNOR, NOT, MUX, COPY, CONST0, CONST1 = range(11)

_lock = threading.Lock()
_libs = {}

_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2): oracle/liboracle.so (l = 3,
    Bg = 2^7) and oracle/liboracle_l2.so (l = 2, Bg = 2^10)."""
    deps = max(os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "cggi_oracle.h")))
    for path, defs in VARIANTS.values():
        if force or not os.path.exists(path) or os.path.getmtime(path) < deps:
            tmp = path + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", *defs, "-shared", "-fPIC", "-o", tmp, SRC, "-lpthread"])
            os.replace(tmp, path)
    return LIB


def lib(l: int = L):
    """The oracle library of gadget length l (3: Bg = 2^7; 2: Bg = 2^10)."""
    with _lock:
        if l not in _libs:
            if l not in VARIANTS:
                raise ValueError(f"no oracle variant with l = {l}")
            build()
            h = ctypes.CDLL(VARIANTS[l][0])
            sig = {
                "orc_gl_mul": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
                "orc_gl_pow": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
                "orc_ntt": (None, [_u64p, ctypes.c_int, ctypes.c_int]),
                "orc_negacyclic_mul_ntt": (None, [_i64p, _i64p, _i64p, ctypes.c_int]),
                "orc_negacyclic_mul_schoolbook": (None, [_i64p, _i64p, _i64p, ctypes.c_int]),
                "orc_modswitch": (ctypes.c_uint32, [ctypes.c_uint32]),
                "orc_decompose": (None, [ctypes.c_uint32, _i32p]),
                "orc_ks_digits": (None, [ctypes.c_uint32, _u32p]),
                "orc_keygen": (None, [ctypes.c_int, _u8p, _u8p, _u32p, _i32p, _u32p, _i32p, _u32p, _u32p]),
                "orc_encrypt": (None, [ctypes.c_int, _u8p, _u32p, _i32p, _u8p, ctypes.c_size_t, _u32p]),
                "orc_decrypt": (None, [ctypes.c_int, _u8p, _u32p, ctypes.c_size_t, _u8p, _i32p]),
                "orc_ctx_create": (ctypes.c_void_p, [ctypes.c_int, _u32p, _u32p]),
                "orc_ctx_destroy": (None, [ctypes.c_void_p]),
                "orc_external_product": (None, [ctypes.c_void_p, ctypes.c_int, _u32p, _u32p, _u32p, _u32p]),
                "orc_blind_rotate": (None, [ctypes.c_void_p, _u32p, ctypes.c_uint32, _u32p]),
                "orc_sample_extract": (None, [_u32p, _u32p]),
                "orc_keyswitch": (None, [ctypes.c_void_p, _u32p, _u32p]),
                "orc_bootstrap_to_N": (None, [ctypes.c_void_p, _u32p, _u32p]),
                "orc_gate_linear": (None, [ctypes.c_int, ctypes.c_int, _u32p, _u32p, _u32p]),
                "orc_gates": (None, [ctypes.c_void_p, _u8p, _u32p, _u32p, _u32p, _u32p, ctypes.c_size_t, ctypes.c_int]),
                "orc_levelize": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, _u8p, _u32p, _u32p, _u32p, _u32p]),
                "orc_eval_netlist": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, _u8p, _u32p, _u32p, _u32p,
                                                    ctypes.c_uint32, _u32p, _u32p, _u32p, ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _libs[l] = h
    return _libs[l]


def _u32(x):
    return np.ascontiguousarray(x, dtype=np.uint32)


def gl_mul(a: int, b: int) -> int:
    return lib().orc_gl_mul(a, b)


def gl_pow(a: int, e: int) -> int:
    return lib().orc_gl_pow(a, e)


def ntt(a, inverse=False):
    x = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().orc_ntt(x, len(x), int(inverse))
    return x


def negacyclic_mul(a, b, schoolbook=False):
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    c = np.zeros_like(a)
    f = lib().orc_negacyclic_mul_schoolbook if schoolbook else lib().orc_negacyclic_mul_ntt
    f(a, b, c, len(a))
    return c


def modswitch(x: int) -> int:
    return lib().orc_modswitch(x)


def decompose(x: int, l: int = L):
    d = np.zeros(l, np.int32)
    lib(l).orc_decompose(x, d)
    return d


def ks_digits(x: int):
    d = np.zeros(KS_T, np.uint32)
    lib().orc_ks_digits(x, d)
    return d


def keygen(kr):
    """kr: inputs.KeyRandomness -> (bsk [n][2l][2][N] u32, ksk [N][8][4][n+1] u32);
    the gadget length l follows the rows of kr.bsk_mask."""
    n = kr.n
    rows = kr.bsk_mask.shape[1]
    bsk = np.zeros((n, rows, 2, N), np.uint32)
    ksk = np.zeros((N, KS_T, 4, n + 1), np.uint32)
    lib(rows // 2).orc_keygen(n, kr.s, kr.K, kr.bsk_mask, kr.bsk_noise, kr.ksk_mask, kr.ksk_noise, bsk, ksk)
    return bsk, ksk


def encrypt(n, s, mask, noise, bits):
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    ct = np.zeros((len(bits), n + 1), np.uint32)
    lib().orc_encrypt(n, s, _u32(mask), np.ascontiguousarray(noise, np.int32), bits, len(bits), ct)
    return ct


def decrypt(n, s, ct):
    ct = _u32(ct).reshape(-1, n + 1)
    bits = np.zeros(len(ct), np.uint8)
    phase = np.zeros(len(ct), np.int32)
    lib().orc_decrypt(n, s, ct, len(ct), bits, phase)
    return bits, phase


def gate_linear(n, gtype, a, b):
    out = np.zeros(n + 1, np.uint32)
    lib().orc_gate_linear(n, gtype, _u32(a), _u32(b), out)
    return out


def sample_extract(acc):
    out = np.zeros(N + 1, np.uint32)
    lib().orc_sample_extract(_u32(acc), out)
    return out


class Context:
    """Bootstrapping context over a (bsk, ksk) pair."""

    def __init__(self, n, bsk, ksk):
        self.n = n
        self._bsk = _u32(bsk)
        self._ksk = _u32(ksk)
        self.l = self._bsk.size // (n * 2 * 2 * N)  # bsk is [n][2l][2][N]
        self.h = lib(self.l).orc_ctx_create(n, self._bsk, self._ksk)

    def __del__(self):
        h = _libs.get(getattr(self, "l", None))
        if getattr(self, "h", None) and h is not None:
            h.orc_ctx_destroy(self.h)
            self.h = None

    def external_product(self, i, t0, t1):
        o0 = np.zeros(N, np.uint32)
        o1 = np.zeros(N, np.uint32)
        lib(self.l).orc_external_product(self.h, i, _u32(t0), _u32(t1), o0, o1)
        return o0, o1

    def blind_rotate(self, abar, bbar):
        acc = np.zeros(2 * N, np.uint32)
        lib(self.l).orc_blind_rotate(self.h, _u32(abar), int(bbar), acc)
        return acc.reshape(2, N)

    def keyswitch(self, lwe_N):
        out = np.zeros(self.n + 1, np.uint32)
        lib(self.l).orc_keyswitch(self.h, _u32(lwe_N), out)
        return out

    def bootstrap_to_N(self, ct):
        out = np.zeros(N + 1, np.uint32)
        lib(self.l).orc_bootstrap_to_N(self.h, _u32(ct), out)
        return out

    def gates(self, types, a, b=None, c=None, nthreads=None):
        types = np.ascontiguousarray(types, dtype=np.uint8)
        a = _u32(a).reshape(-1, self.n + 1)
        b = a if b is None else _u32(b).reshape(-1, self.n + 1)
        c = a if c is None else _u32(c).reshape(-1, self.n + 1)
        out = np.zeros_like(a)
        lib(self.l).orc_gates(self.h, types, a, b, c, out, len(types), nthreads or os.cpu_count() or 1)
        return out

    def eval_netlist(self, nl, ct_in, nthreads=None):
        ct_in = _u32(ct_in).reshape(-1, self.n + 1)
        out = np.zeros((len(nl.outputs), self.n + 1), np.uint32)
        rc = lib(self.l).orc_eval_netlist(
            self.h, nl.num_inputs, nl.num_gates, nl.type, nl.in0, nl.in1, nl.in2,
            len(nl.outputs), nl.outputs, ct_in, out, nthreads or os.cpu_count() or 1,
        )
        if rc:
            raise ValueError(f"oracle netlist evaluation failed: {rc}")
        return out


def levelize(nl):
    wave = np.zeros(max(nl.num_gates, 1), np.uint32)
    rc = lib().orc_levelize(nl.num_inputs, nl.num_gates, nl.type, nl.in0, nl.in1, nl.in2, wave)
    return rc, wave[: nl.num_gates]
