"""Python binding of libarx (include/arx.h): argument marshalling only.

Every step of gate bootstrapping runs in the CUDA kernels behind the C-ABI; this
module turns numpy arrays and torch tensors (host or device) into pointers and
return codes into exceptions.  PyTorch is only used for device memory and
streams.  If libarx.so has not been built, every call raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libarx.so")

N = 1024
LWE_N = 630
MU = 1 << 29
AND, NAND, OR, NOR, XOR, XNOR, NOT, MUX, COPY, CONST0, CONST1 = range(11)
MODE_PLAIN, MODE_GRAPH = 0, 1
STATUS = {0: "ARX_OK", -1: "ARX_EINVAL", -2: "ARX_ENOKEYS", -3: "ARX_ENOMEM", -4: "ARX_ECYCLE",
          -5: "ARX_ETIMEOUT", -6: "ARX_ECUDA", -7: "ARX_EBUSY"}

# every entry point of include/arx.h with its ctypes signature
_vp, _sz, _i, _u32, _u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64


class ServeStats_C(ctypes.Structure):
    _fields_ = [(k, _u64) for k in ("completed", "failed", "gates", "bootstraps", "launches", "ticks", "pending",
                                    "active", "peak_active", "peak_bytes")] + \
               [(k, ctypes.c_double) for k in ("p50_ms", "p99_ms", "busy_s", "elapsed_s")] + \
               [(k, _u64) for k in ("shared_launches", "max_keys_per_launch")]


class Netlist_C(ctypes.Structure):
    _fields_ = [("num_inputs", _u32), ("num_gates", _u32), ("num_outputs", _u32), ("type", _vp),
                ("in0", _vp), ("in1", _vp), ("in2", _vp), ("outputs", _vp)]


_NLP = ctypes.POINTER(Netlist_C)
SIGNATURES = {
    "arx_load_keys": (_i, [_vp, _vp]),
    "arx_load_keys_ex": (_i, [_vp, _vp, _i, _vp]),
    "arx_load_keys_gadget": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "arx_unload_keys": (_i, [_i]),
    "arx_keyset_dims": (_i, [_i, _vp, _vp]),
    "arx_use_keys": (_i, [_i]),
    "arx_keyset_bytes": (_sz, [_i]),
    "arx_resident_bytes": (_sz, []),
    "arx_bootstrap_gates": (_i, [_vp, _vp, _vp, _vp, _sz]),
    "arx_bootstrap_gates_ex": (_i, [_vp, _vp, _vp, _vp, _vp, _sz, _i, _vp]),
    "arx_levelize": (_i, [_NLP, _vp, _vp]),
    "arx_levelize_balanced": (_i, [_NLP, _vp, _u32, _vp, _vp]),
    "arx_eval_netlist": (_i, [_NLP, _vp, _vp]),
    "arx_eval_netlist_ex": (_i, [_NLP, _vp, _vp, _i, _i, _vp]),
    "arx_plan_create": (_i, [_NLP, _i, _i]),
    "arx_plan_run": (_i, [_i, _vp, _vp, _vp]),
    "arx_plan_destroy": (_i, [_i]),
    "arx_plan_info": (_i, [_i, _vp, _vp, _vp]),
    "arx_plan_shapes": (_i, [_i, _vp, _vp, _vp, _u32]),
    "arx_plan_launches": (_i, [_i, _vp, _vp, _vp, _vp, _u32]),
    "arx_split_wave": (_i, [_vp, _vp, _vp, _u32, _u32, _vp, _vp, _vp, _vp, _vp]),
    "arx_plan_wires": (_i, [_i, _vp, _sz, _vp]),
    "arx_set_launch_shape": (_i, [_i, _i]),
    "arx_plan_profile": (_i, [_i, _vp, _vp, _vp, _vp, _vp]),
    "arx_keyswitch_noalloc": (_i, [_vp, _vp, _sz, _i, _vp]),
    "arx_serve_start": (_i, [_sz, _sz, _u32]),
    "arx_serve_submit": (_i, [_i, _NLP, _vp, _vp]),
    "arx_serve_poll": (_i, [_i]),
    "arx_serve_wait": (_i, [_i, ctypes.c_double]),
    "arx_serve_stats": (_i, [ctypes.POINTER(ServeStats_C)]),
    "arx_serve_stop": (_i, []),
    "arx_last_error": (ctypes.c_char_p, []),
    "arx_device_status": (_i, []),
    "arx_watchdog_selftest": (_i, [_i, ctypes.c_longlong, _vp]),
    "arx_device_sms": (_i, []),
    "arx_probe_alu": (_i, [_vp, _i]),
    "arx_client_keygen": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "arx_client_keygen_gadget": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "arx_client_encrypt": (_i, [_i, _vp, _vp, _vp, _vp, _sz, _vp]),
    "arx_client_decrypt": (_i, [_i, _vp, _vp, _sz, _vp]),
}

_lock = threading.Lock()
_lib = None


class ArxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libarx.so (building it first when missing, where nvcc is available)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _build
                _build.build()
            h = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _lib = h
    return _lib


def _check(rc: int) -> int:
    if rc < 0:
        raise ArxError(rc, lib().arx_last_error().decode(errors="replace"))
    return rc


def _ptr(x):
    """Pointer of a numpy array or torch tensor (must be contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(type(x))


def _stream(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def _host_u8(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


# ------------------------------------------------------------------- keys ---
GADGET_BITS = {3: 7, 2: 10}  # gadget length l -> log2 Bg


def load_keys(bsk, ksk, lwe_n: int = LWE_N, stream=None, l: int = 3) -> int:
    """Load a key pair; l = 2 selects the gadget Bg = 2^10 (bsk [n][4][2][N])."""
    if l == 3:
        return _check(lib().arx_load_keys_ex(_ptr(bsk), _ptr(ksk), lwe_n, _stream(stream)))
    return _check(lib().arx_load_keys_gadget(_ptr(bsk), _ptr(ksk), lwe_n, l, GADGET_BITS.get(l, 0),
                                             _stream(stream)))


def keyset_dims(keyset: int = -1) -> tuple:
    """(LWE dimension n, gadget length l) of a loaded key set."""
    n, l = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().arx_keyset_dims(keyset, ctypes.addressof(n), ctypes.addressof(l)))
    return n.value, l.value


def unload_keys(keyset: int) -> None:
    _check(lib().arx_unload_keys(keyset))


def resident_bytes() -> int:
    """Device bytes held by all loaded key sets."""
    return int(lib().arx_resident_bytes())


def use_keys(keyset: int) -> None:
    """Make a loaded key set the default of the calls that take no key set id."""
    _check(lib().arx_use_keys(keyset))


def keyset_bytes(lwe_n: int = LWE_N) -> int:
    return int(lib().arx_keyset_bytes(lwe_n))


# ------------------------------------------------------------------ gates ---
def bootstrap_gates(types, ct_a, ct_b, ct_out) -> None:
    t = _host_u8(types)
    _check(lib().arx_bootstrap_gates(_ptr(t), _ptr(ct_a), _ptr(ct_b), _ptr(ct_out), len(t)))


def bootstrap_gates_ex(types, ct_a, ct_b, ct_c, ct_out, keyset: int = -1, stream=None) -> None:
    t = _host_u8(types)
    _check(lib().arx_bootstrap_gates_ex(_ptr(t), _ptr(ct_a), _ptr(ct_b), _ptr(ct_c), _ptr(ct_out), len(t),
                                        keyset, _stream(stream)))


# --------------------------------------------------------------- netlists ---
class _NetlistRef:
    """Keeps the numpy arrays behind an arx_netlist alive."""

    def __init__(self, nl):
        u32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
        self.type = _host_u8(nl.type)
        self.in0, self.in1, self.in2, self.outputs = u32(nl.in0), u32(nl.in1), u32(nl.in2), u32(nl.outputs)
        self.c = Netlist_C(nl.num_inputs, len(self.type), len(self.outputs), _ptr(self.type), _ptr(self.in0),
                           _ptr(self.in1), _ptr(self.in2), _ptr(self.outputs))

    @property
    def ref(self):
        return ctypes.byref(self.c)


def levelize(nl):
    r = _NetlistRef(nl)
    wave = np.zeros(max(len(r.type), 1), np.uint32)
    depth = ctypes.c_uint32(0)
    _check(lib().arx_levelize(r.ref, _ptr(wave), ctypes.addressof(depth)))
    return wave[: len(r.type)], depth.value


def levelize_balanced(nl, caps):
    """Levels with launch widths evened out within slack (arx_levelize_balanced):
    caps = increasing launch capacities in blind rotations.  Returns (wave, depth)."""
    r = _NetlistRef(nl)
    c = np.ascontiguousarray(np.asarray(caps, dtype=np.uint32))
    wave = np.zeros(max(len(r.type), 1), np.uint32)
    depth = ctypes.c_uint32(0)
    _check(lib().arx_levelize_balanced(r.ref, _ptr(c) if len(c) else None, len(c), _ptr(wave),
                                       ctypes.addressof(depth)))
    return wave[: len(r.type)], depth.value


def split_wave(ms, gates, cluster, jobs):
    """Launch plan of one wave under a table of shapes (arx_split_wave): returns
    (bulk shape, bulk jobs, tail shape or -1, cost in ms, widest wave within it)."""
    m = np.ascontiguousarray(np.asarray(ms, dtype=np.float64))
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.uint32))
    c = np.ascontiguousarray(np.asarray(cluster, dtype=np.uint8))
    if not (len(m) == len(g) == len(c)):
        raise ArxError(-1, "ms, gates and cluster differ in length")
    bulk, bj, cap = ctypes.c_uint32(0), ctypes.c_uint32(0), ctypes.c_uint32(0)
    tail, cost = ctypes.c_int32(0), ctypes.c_double(0)
    _check(lib().arx_split_wave(_ptr(m), _ptr(g), _ptr(c), len(m), int(jobs), ctypes.addressof(bulk),
                                ctypes.addressof(bj), ctypes.addressof(tail), ctypes.addressof(cost),
                                ctypes.addressof(cap)))
    return bulk.value, bj.value, tail.value, cost.value, cap.value


def eval_netlist(nl, ct_in, ct_out) -> None:
    r = _NetlistRef(nl)
    _check(lib().arx_eval_netlist(r.ref, _ptr(ct_in), _ptr(ct_out)))


def eval_netlist_ex(nl, ct_in, ct_out, keyset: int = -1, mode: int = MODE_PLAIN, stream=None) -> None:
    r = _NetlistRef(nl)
    _check(lib().arx_eval_netlist_ex(r.ref, _ptr(ct_in), _ptr(ct_out), keyset, mode, _stream(stream)))


class Plan:
    """A netlist levelized and resident on the device, evaluated many times."""

    def __init__(self, nl, keyset: int = -1, mode: int = MODE_GRAPH):
        r = _NetlistRef(nl)
        self.id = _check(lib().arx_plan_create(r.ref, keyset, mode))
        w, b, g = ctypes.c_uint32(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(lib().arx_plan_info(self.id, ctypes.addressof(w), ctypes.addressof(b), ctypes.addressof(g)))
        self.waves, self.bootstraps, self.gates = w.value, b.value, g.value

    def run(self, ct_in, ct_out, stream=None) -> None:
        _check(lib().arx_plan_run(self.id, _ptr(ct_in), _ptr(ct_out), _stream(stream)))

    def wires(self, ids, n: int = LWE_N):
        ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
        out = np.zeros((len(ids), n + 1), np.uint32)
        _check(lib().arx_plan_wires(self.id, _ptr(ids), len(ids), _ptr(out)))
        return out

    def shapes(self):
        """Launch shape of every wave: list of (H, GT, blind rotations)."""
        cap = max(self.waves, 1)
        H, GT, J = (np.zeros(cap, np.uint32) for _ in range(3))
        w = _check(lib().arx_plan_shapes(self.id, _ptr(H), _ptr(GT), _ptr(J), cap))
        return [(int(H[k]), int(GT[k]), int(J[k])) for k in range(min(w, cap))]

    def launches(self):
        """Every blind-rotation launch: list of (wave, H, GT, blind rotations)."""
        cap = 2 * max(self.waves, 1)
        W, H, GT, J = (np.zeros(cap, np.uint32) for _ in range(4))
        k = _check(lib().arx_plan_launches(self.id, _ptr(W), _ptr(H), _ptr(GT), _ptr(J), cap))
        return [(int(W[i]), int(H[i]), int(GT[i]), int(J[i])) for i in range(min(k, cap))]

    def profile(self, ct_in):
        """One wave-by-wave run timed per launch: (br_ms, ks_ms, br_launches, ks_launches)."""
        bm, km = ctypes.c_float(0), ctypes.c_float(0)
        bl, kl = ctypes.c_uint32(0), ctypes.c_uint32(0)
        _check(lib().arx_plan_profile(self.id, _ptr(ct_in), ctypes.addressof(bm), ctypes.addressof(km),
                                      ctypes.addressof(bl), ctypes.addressof(kl)))
        return bm.value, km.value, bl.value, kl.value

    def close(self) -> None:
        if self.id is not None:
            _check(lib().arx_plan_destroy(self.id))
            self.id = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


KS_NOALLOC_MAX = 1024


def _check_noalloc_args(lwe_N, ct_out, count, n):
    """The shapes the C-ABI cannot see: raises ArxError(ARX_EINVAL) before any
    pointer reaches the library."""
    def bad(msg):
        raise ArxError(-1, msg)

    for name, t in (("lwe_N", lwe_N), ("ct_out", ct_out)):
        if not hasattr(t, "is_cuda") or not t.is_cuda:
            bad(f"{name} must be a CUDA tensor")
        if str(t.dtype) not in ("torch.int32", "torch.uint32"):
            bad(f"{name} must hold 32-bit words, not {t.dtype}")
        if t.dim() != 2 or not t.is_contiguous():
            bad(f"{name} must be a contiguous 2-D tensor")
    if lwe_N.shape[1] != N + 1:
        bad(f"lwe_N rows have {lwe_N.shape[1]} words, not N + 1 = {N + 1}")
    if ct_out.shape[1] != n + 1:
        bad(f"ct_out rows have {ct_out.shape[1]} words, not n + 1 = {n + 1} of the key set")
    if count < 0 or count > lwe_N.shape[0] or count > ct_out.shape[0]:
        bad(f"count {count} exceeds lwe_N ({lwe_N.shape[0]} rows) or ct_out ({ct_out.shape[0]} rows)")


def keyswitch_noalloc(lwe_N, ct_out, count=None, keyset: int = -1, stream=None) -> None:
    """Key switch of LWE_N samples into LWE_n ciphertexts (device tensors) with no
    device allocation inside the call (see include/arx.h).  The tensors' device,
    word size, row widths and count are checked here first."""
    count = len(lwe_N) if count is None else count
    n, _ = keyset_dims(keyset)
    _check_noalloc_args(lwe_N, ct_out, count, n)
    _check(lib().arx_keyswitch_noalloc(_ptr(lwe_N), _ptr(ct_out), count, keyset, _stream(stream)))


class Server:
    """Continuous-batching server (arx_serve_*): submit netlist requests from any
    number of clients (key sets); results arrive in the caller's host buffers."""

    def __init__(self, hbm_budget: int = 0, arena_bytes: int = 1 << 30, max_tick_bootstraps: int = 0):
        _check(lib().arx_serve_start(hbm_budget, arena_bytes, max_tick_bootstraps))
        self._keep = {}

    def submit(self, nl, ct_in, keyset: int = -1, n: int = LWE_N):
        r = _NetlistRef(nl)
        ct_in = np.ascontiguousarray(np.asarray(ct_in, dtype=np.uint32))
        out = np.zeros((len(r.outputs), n + 1), np.uint32)
        rid = _check(lib().arx_serve_submit(keyset, r.ref, _ptr(ct_in), _ptr(out)))
        self._keep[rid] = out
        return rid

    def poll(self, rid: int) -> int:
        return lib().arx_serve_poll(rid)

    def wait(self, rid: int, timeout_s: float = 600.0):
        """Block until request rid completes; returns its output ciphertexts."""
        rc = _check(lib().arx_serve_wait(rid, timeout_s))
        if rc != 1:
            raise TimeoutError(f"request {rid} still pending after {timeout_s} s")
        return self._keep.pop(rid)

    def stats(self) -> dict:
        st = ServeStats_C()
        _check(lib().arx_serve_stats(ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStats_C._fields_}

    def stop(self) -> None:
        _check(lib().arx_serve_stop())

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()


def set_launch_shape(H: int = 0, GT: int = 0) -> None:
    """Force the blind-rotation launch shape; (0, 0) = automatic."""
    _check(lib().arx_set_launch_shape(H, GT))


def device_status() -> int:
    return lib().arx_device_status()


def watchdog_selftest(post_token: bool, limit_cycles: int = 20_000_000) -> tuple:
    """Runs arx_watchdog_selftest; returns (status code, waits given up)."""
    gave_up = ctypes.c_int(-1)
    rc = lib().arx_watchdog_selftest(1 if post_token else 0, int(limit_cycles), ctypes.byref(gave_up))
    return rc, gave_up.value


def device_sms() -> int:
    return lib().arx_device_sms()


PROBE_NAMES = ("imad", "imad_hi", "imad_wide", "alu_x3", "shoup_bfly_q27", "mont_mac_q27", "goldilocks_bfly")


def probe_alu() -> dict:
    """Lane operations per clock per SM of the integer pipes (see arx_probe_alu)."""
    rate = np.zeros(len(PROBE_NAMES), np.float64)
    _check(lib().arx_probe_alu(_ptr(rate), len(rate)))
    return dict(zip(PROBE_NAMES, (float(r) for r in rate)))


# ------------------------------------------------------------ client side ---
def client_keygen(kr):
    """Key pair from an inputs.KeyRandomness: (bsk [n][2l][2][N], ksk [N][8][4][n+1]);
    the gadget length l follows the rows of kr.bsk_mask (6: l = 3, 4: l = 2)."""
    n = kr.n
    rows = kr.bsk_mask.shape[1]
    bsk = np.zeros((n, rows, 2, N), np.uint32)
    ksk = np.zeros((N, 8, 4, n + 1), np.uint32)
    arrs = [np.ascontiguousarray(a) for a in (kr.s, kr.K, kr.bsk_mask, kr.bsk_noise, kr.ksk_mask, kr.ksk_noise)]
    l = rows // 2
    _check(lib().arx_client_keygen_gadget(n, l, GADGET_BITS.get(l, 0), *[_ptr(a) for a in arrs], _ptr(bsk),
                                          _ptr(ksk)))
    return bsk, ksk


def client_encrypt(n: int, s, mask, noise, bits):
    bits = _host_u8(bits)
    s = _host_u8(s)
    mask = np.ascontiguousarray(mask, dtype=np.uint32)
    noise = np.ascontiguousarray(noise, dtype=np.int32)
    ct = np.zeros((len(bits), n + 1), np.uint32)
    _check(lib().arx_client_encrypt(n, _ptr(s), _ptr(mask), _ptr(noise), _ptr(bits), len(bits), _ptr(ct)))
    return ct


def client_decrypt(n: int, s, ct):
    ct = np.ascontiguousarray(np.asarray(ct, dtype=np.uint32)).reshape(-1, n + 1)
    s = _host_u8(s)
    bits = np.zeros(len(ct), np.uint8)
    _check(lib().arx_client_decrypt(n, _ptr(s), _ptr(ct), len(ct), _ptr(bits)))
    return bits
