"""Thin ctypes binding of libmrmod.so (include/mr.h), same names as the C ABI.

Every function marshals arguments only: big integers become little-endian
uint32 limb arrays, torch device tensors become raw device pointers, streams
become cudaStream_t handles.  All arithmetic runs in the library's CUDA
kernels; there is no CPU fallback -- importing this module fails loudly when
the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmrmod.so")

MR_OK = 0
STATUS_NAMES = {
    0: "MR_OK", 1: "MR_ERR_ARG", 2: "MR_ERR_EVEN_MODULUS", 3: "MR_ERR_NOT_COPRIME", 4: "MR_ERR_SIZE",
    5: "MR_ERR_RANGE", 6: "MR_ERR_OOM", 7: "MR_ERR_CUDA", 8: "MR_ERR_TIMEOUT", 9: "MR_ERR_BUSY", 10: "MR_ERR_KEY",
}

EXPORTED = [
    "mr_init", "mr_shutdown", "mr_last_error", "mr_class_for_bits", "mr_rns_setup", "mr_rsa_key_setup",
    "mr_key_info", "mr_key_free", "mr_modexp_batch", "mr_rsa_encrypt", "mr_rsa_decrypt_crt",
    "mr_miller_rabin_batch", "mr_debug_table", "mr_debug_key_table_host", "mr_profile_enable", "mr_profile_read",
    "mr_modexp_batch_noalloc", "mr_class_variants", "mr_lane_variant_info", "mr_set_variant", "mr_debug_mr_setup",
    "mr_rsa_mixed", "mr_plan_create", "mr_plan_launch", "mr_plan_info", "mr_plan_free",
    "mr_imad_peak", "mr_autotune", "mr_debug_big_wait", "mr_prime_test_batch", "mr_debug_trial_table",
    "mr_rsa_keygen_batch", "mr_rsa_message_blocks", "mr_rsa_encrypt_message", "mr_rsa_decrypt_message",
    "mr_get_tuning", "mr_set_tuning", "mr_debug_crt_bin_host", "mr_debug_big_variant",
    "mr_tensor_peak", "mr_debug_tc_mma", "mr_debug_tc_slices", "mr_big_variant_info", "mr_debug_big_phases",
    "mr_set_constant_time", "mr_debug_lane_tc_wait",
]

MR_OP_ENCRYPT = 0
MR_OP_DECRYPT = 1
MR_PLAN_CONCURRENT = 1
MR_PLAN_PERSISTENT = 2
MR_PLAN_GRAPH = 4
MR_PLAN_AUTOTUNE = 8


class KernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint32), ("ms", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("lanes_per_number", ctypes.c_uint32), ("window", ctypes.c_uint32),
                ("configs", ctypes.c_uint32), ("ms", ctypes.c_double), ("ms_default", ctypes.c_double)]


class MRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1305_3699_gb300.build` "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    U32 = ctypes.c_uint32
    PU32 = ctypes.POINTER(ctypes.c_uint32)
    SZ = ctypes.c_size_t
    sig = {
        "mr_init": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(P)]),
        "mr_shutdown": (None, [P]),
        "mr_last_error": (ctypes.c_char_p, [P]),
        "mr_class_for_bits": (ctypes.c_int, [U32, PU32, PU32]),
        "mr_rns_setup": (ctypes.c_int, [P, PU32, U32, ctypes.POINTER(P)]),
        "mr_rsa_key_setup": (ctypes.c_int, [P, PU32, U32, PU32, U32, PU32, PU32, PU32, PU32, PU32, U32,
                                            ctypes.POINTER(P)]),
        "mr_key_info": (ctypes.c_int, [P, PU32, PU32, ctypes.POINTER(ctypes.c_uint64)]),
        "mr_key_free": (ctypes.c_int, [P, P]),
        "mr_modexp_batch": (ctypes.c_int, [P, P, SZ, P, U32, P, U32, P, U32, P, P]),
        "mr_rsa_encrypt": (ctypes.c_int, [P, P, SZ, P, U32, P, U32, P, P]),
        "mr_rsa_decrypt_crt": (ctypes.c_int, [P, P, SZ, P, U32, P, U32, P, P]),
        "mr_miller_rabin_batch": (ctypes.c_int, [P, P, U32, SZ, P, U32, P, P, P]),
        "mr_prime_test_batch": (ctypes.c_int, [P, P, U32, SZ, P, U32, U32, P, P, P]),
        "mr_debug_trial_table": (ctypes.c_int, [PU32, SZ, ctypes.POINTER(SZ)]),
        "mr_rsa_keygen_batch": (ctypes.c_int, [P, U32, SZ, U32, P, P, U32, U32, P, P, P]),
        "mr_rsa_message_blocks": (ctypes.c_int, [P, SZ, ctypes.POINTER(SZ), PU32, PU32]),
        "mr_get_tuning": (ctypes.c_int, [P, U32, PU32, PU32, PU32]),
        "mr_debug_big_variant": (ctypes.c_int, [U32, SZ, U32, U32, PU32, PU32]),
        "mr_debug_crt_bin_host": (ctypes.c_int, [PU32, PU32, PU32, U32, U32, PU32, SZ, ctypes.POINTER(SZ)]),
        "mr_set_tuning": (ctypes.c_int, [P, U32, U32, U32]),
        "mr_rsa_encrypt_message": (ctypes.c_int, [P, P, P, SZ, P, P, P]),
        "mr_rsa_decrypt_message": (ctypes.c_int, [P, P, P, SZ, P, SZ, P, P]),
        "mr_debug_table": (ctypes.c_int, [P, U32, P, ctypes.c_char_p, PU32, SZ, ctypes.POINTER(SZ)]),
        "mr_debug_key_table_host": (ctypes.c_int, [PU32, U32, ctypes.c_char_p, PU32, SZ, ctypes.POINTER(SZ)]),
        "mr_profile_enable": (ctypes.c_int, [P, ctypes.c_int]),
        "mr_modexp_batch_noalloc": (ctypes.c_int, [P, P, SZ, P, U32, P, U32, P, U32, P, P]),
        "mr_class_variants": (ctypes.c_int, [U32, PU32, PU32, U32]),
        "mr_lane_variant_info": (ctypes.c_int, [U32, U32, PU32]),
        "mr_set_variant": (ctypes.c_int, [P, U32, U32]),
        "mr_debug_mr_setup": (ctypes.c_int, [P, P, U32, SZ, P, P]),
        "mr_rsa_mixed": (ctypes.c_int, [P, P, P, SZ, P, U32, P, U32, P, U32, P]),
        "mr_plan_create": (ctypes.c_int, [P, P, P, SZ, P, U32, P, U32, P, U32, ctypes.POINTER(P)]),
        "mr_plan_launch": (ctypes.c_int, [P, P]),
        "mr_plan_info": (ctypes.c_int, [P, PU32, PU32, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
        "mr_plan_free": (None, [P]),
        "mr_profile_read": (ctypes.c_int, [P, ctypes.POINTER(KernelTime), U32]),
        "mr_imad_peak": (ctypes.c_int, [P, U32, P, ctypes.POINTER(ctypes.c_double)]),
        "mr_tensor_peak": (ctypes.c_int, [P, U32, P, ctypes.POINTER(ctypes.c_double)]),
        "mr_debug_tc_mma": (ctypes.c_int, [P, P, P, U32, U32, U32, P, P]),
        "mr_debug_tc_slices": (ctypes.c_int, [U32, PU32, SZ, ctypes.POINTER(SZ)]),
        "mr_big_variant_info": (ctypes.c_int, [U32, U32, PU32, PU32, PU32]),
        "mr_debug_big_phases": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
        "mr_set_constant_time": (ctypes.c_int, [P, ctypes.c_int]),
        "mr_autotune": (ctypes.c_int, [P, U32, U32, U32, ctypes.POINTER(TuneResult)]),
        "mr_debug_big_wait": (ctypes.c_int, [P, U32, ctypes.c_int32]),
        "mr_debug_lane_tc_wait": (ctypes.c_int, [P, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _limbs(x: int, n: Optional[int] = None) -> np.ndarray:
    if x < 0:
        raise ValueError("negative integer")
    nl = max(1, (x.bit_length() + 31) // 32) if n is None else n
    return np.frombuffer(x.to_bytes(4 * nl, "little"), dtype="<u4").astype(np.uint32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _dev(t) -> int:
    """Device pointer of a torch tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _rows(t) -> tuple:
    if t.dim() != 2 or t.element_size() != 4:
        raise ValueError("expected a 2-D tensor of 32-bit limbs (rows x limbs)")
    return t.shape[0], t.shape[1]


def mr_class_for_bits(bits: int):
    L, k = ctypes.c_uint32(), ctypes.c_uint32()
    rc = lib.mr_class_for_bits(bits, ctypes.byref(L), ctypes.byref(k))
    if rc:
        raise MRError(rc, f"no size class for {bits} bits")
    return L.value, k.value


def mr_lane_variant_info(class_bits: int, variant: int) -> dict:
    """One lane mapping of a lane-group size class (see mr.h)."""
    out = (ctypes.c_uint32 * 4)()
    rc = lib.mr_lane_variant_info(class_bits, variant, out)
    if rc != 0:
        raise MRError(rc, "mr_lane_variant_info")
    return {"lanes_per_number": out[0], "threads": out[1], "numbers_per_block": out[2], "tensor": bool(out[3])}


def mr_class_variants(class_bits: int) -> List[int]:
    """Lanes per number of each compiled lane mapping of a size class."""
    cnt = ctypes.c_uint32()
    buf = (ctypes.c_uint32 * 8)()
    rc = lib.mr_class_variants(class_bits, ctypes.byref(cnt), buf, 8)
    if rc:
        raise MRError(rc, f"no size class {class_bits}")
    return [buf[i] for i in range(min(cnt.value, 8))]


def mr_debug_key_table_host(N: int, name: str) -> List[int]:
    nl = _limbs(N)
    cnt = ctypes.c_size_t()
    rc = lib.mr_debug_key_table_host(_ptr(nl), len(nl), name.encode(), None, 0, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, f"table {name}")
    out = np.zeros(cnt.value, dtype=np.uint32)
    rc = lib.mr_debug_key_table_host(_ptr(nl), len(nl), name.encode(), _ptr(out), cnt.value, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, f"table {name}")
    return [int(v) for v in out]


def mr_debug_trial_table() -> np.ndarray:
    """The trial-division tables as built on the host: 131 rows of 10,016 words (see mr.h)."""
    cnt = ctypes.c_size_t()
    rc = lib.mr_debug_trial_table(None, 0, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, "trial table")
    out = np.zeros(cnt.value, dtype=np.uint32)
    rc = lib.mr_debug_trial_table(_ptr(out), cnt.value, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, "trial table")
    return out.reshape(131, -1)


def mr_debug_big_variant(class_bits: int, n_items: int, sms: int = 152, ctas_per_sm: int = 1):
    """(variant, slots) the large-class launch picks for n_items numbers (see mr.h)."""
    v, sl = ctypes.c_uint32(), ctypes.c_uint32()
    rc = lib.mr_debug_big_variant(class_bits, n_items, sms, ctas_per_sm, ctypes.byref(v), ctypes.byref(sl))
    if rc:
        raise MRError(rc, "big variant")
    return v.value, sl.value


def mr_debug_crt_bin_host(p: int, q: int, qinv: int, W: int) -> List[int]:
    """The binary Garner block of CRT halves p, q in a class of W limbs (see mr.h)."""
    nl = max(1, (max(p.bit_length(), q.bit_length()) + 31) // 32)
    a, b, c = _limbs(p, nl), _limbs(q, nl), _limbs(qinv % p, nl)
    cnt = ctypes.c_size_t()
    rc = lib.mr_debug_crt_bin_host(_ptr(a), _ptr(b), _ptr(c), nl, W, None, 0, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, "crt block")
    out = np.zeros(cnt.value, dtype=np.uint32)
    rc = lib.mr_debug_crt_bin_host(_ptr(a), _ptr(b), _ptr(c), nl, W, _ptr(out), cnt.value, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, "crt block")
    return [int(v) for v in out]


def mr_debug_class_table(class_bits: int, name: str) -> List[int]:
    cnt = ctypes.c_size_t()
    rc = lib.mr_debug_table(None, class_bits, None, name.encode(), None, 0, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, f"table {name}")
    out = np.zeros(cnt.value, dtype=np.uint32)
    rc = lib.mr_debug_table(None, class_bits, None, name.encode(), _ptr(out), cnt.value, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, f"table {name}")
    return [int(v) for v in out]


class Key:
    """A modulus (or RSA key) set up on the device; owned by its Context."""

    def __init__(self, ctx: "Context", handle: int, N: int, e: Optional[int] = None, private: bool = False):
        self.ctx, self.handle, self.N, self.e, self.private = ctx, handle, N, e, private
        self.half_bits = 0  # bit length of the larger RSA prime when the private CRT parts are set

    @property
    def limbs(self) -> int:
        return max(1, (self.N.bit_length() + 31) // 32)

    def info(self):
        k, kh, nb = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        self.ctx._check(lib.mr_key_info(self.handle, ctypes.byref(k), ctypes.byref(kh), ctypes.byref(nb)))
        return {"k": k.value, "k_half": kh.value, "device_bytes": nb.value}

    def free(self):
        if self.handle:
            self.ctx._check(lib.mr_key_free(self.ctx.handle, self.handle))
            self.handle = None


class KeyList:
    """A reusable host array of key handles for batched calls."""

    def __init__(self, keys: Sequence[Key]):
        self.keys = list(keys)
        self.arr = (ctypes.c_void_p * len(self.keys))(*[k.handle for k in self.keys])

    def __len__(self):
        return len(self.keys)


class Plan:
    """A prepared mixed batch (mr_plan_create); launch() enqueues one execution."""

    def __init__(self, ctx: "Context", handle: int, refs):
        self.ctx, self.handle, self._refs = ctx, handle, refs

    def launch(self, stream=None):
        self.ctx._check(lib.mr_plan_launch(self.handle, _stream(stream)))

    def info(self):
        k, g, b, p = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_double()
        self.ctx._check(lib.mr_plan_info(self.handle, ctypes.byref(k), ctypes.byref(g), ctypes.byref(b), ctypes.byref(p)))
        return {"kernels": k.value, "groups": g.value, "device_bytes": b.value, "products": p.value}

    def free(self):
        if self.handle:
            lib.mr_plan_free(self.handle)
            self.handle = None


def _ops(ops):
    a = np.ascontiguousarray(np.asarray(ops, dtype=np.uint8))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _keylist(keys) -> KeyList:
    return keys if isinstance(keys, KeyList) else KeyList(keys)


class Context:
    """mr_init / mr_shutdown around one CUDA device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        rc = lib.mr_init(device, ctypes.byref(h))
        if rc:
            raise MRError(rc, f"mr_init(device={device}) failed")
        self.handle = h.value
        self.device = device

    def _check(self, rc: int):
        if rc:
            raise MRError(rc, lib.mr_last_error(self.handle).decode(errors="replace"))

    def last_error(self) -> str:
        return lib.mr_last_error(self.handle).decode(errors="replace")

    def close(self):
        if self.handle:
            lib.mr_shutdown(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- setup
    def mr_rns_setup(self, N: int) -> Key:
        nl = _limbs(N)
        h = ctypes.c_void_p()
        self._check(lib.mr_rns_setup(self.handle, _ptr(nl), len(nl), ctypes.byref(h)))
        return Key(self, h.value, N)

    def mr_rsa_key_setup(self, N: int, e: int, p: Optional[int] = None, q: Optional[int] = None,
                         dp: Optional[int] = None, dq: Optional[int] = None, qinv: Optional[int] = None) -> Key:
        nl, el = _limbs(N), _limbs(e)
        h = ctypes.c_void_p()
        if p is None:
            self._check(lib.mr_rsa_key_setup(self.handle, _ptr(nl), len(nl), _ptr(el), len(el), None, None, None,
                                             None, None, 0, ctypes.byref(h)))
            return Key(self, h.value, N, e, False)
        hl = max(_limbs(v).size for v in (p, q, dp, dq, qinv))
        parts = [_limbs(v, hl) for v in (p, q, dp, dq, qinv)]
        self._check(lib.mr_rsa_key_setup(self.handle, _ptr(nl), len(nl), _ptr(el), len(el),
                                         *[_ptr(a) for a in parts], hl, ctypes.byref(h)))
        key = Key(self, h.value, N, e, True)
        key.half_bits = max(p.bit_length(), q.bit_length())
        return key

    # ---- batched calls (torch tensors: rows x limbs, 32-bit, contiguous, on this device)
    def mr_modexp_batch(self, keys, x, e, out, status=None, stream=None):
        kl = _keylist(keys)
        n, xs = _rows(x)
        _, es = _rows(e)
        _, os_ = _rows(out)
        self._check(lib.mr_modexp_batch(self.handle, kl.arr, len(kl), _dev(x), xs, _dev(e), es, _dev(out), os_,
                                        _dev(status), _stream(stream)))

    def mr_modexp_batch_noalloc(self, key: Key, x, e, out, status=None, stream=None):
        """Allocation-free exponentiation for one modulus (see mr_modexp_batch_noalloc in mr.h)."""
        n, xs = _rows(x)
        _, es = _rows(e)
        _, os_ = _rows(out)
        self._check(lib.mr_modexp_batch_noalloc(self.handle, key.handle, n, _dev(x), xs, _dev(e), es, _dev(out), os_,
                                                _dev(status), _stream(stream)))

    def mr_rsa_encrypt(self, keys, m, c, status=None, stream=None):
        kl = _keylist(keys)
        _, ms = _rows(m)
        _, cs = _rows(c)
        self._check(lib.mr_rsa_encrypt(self.handle, kl.arr, len(kl), _dev(m), ms, _dev(c), cs, _dev(status),
                                       _stream(stream)))

    def mr_rsa_decrypt_crt(self, keys, c, m, status=None, stream=None):
        kl = _keylist(keys)
        _, cs = _rows(c)
        _, ms = _rows(m)
        self._check(lib.mr_rsa_decrypt_crt(self.handle, kl.arr, len(kl), _dev(c), cs, _dev(m), ms, _dev(status),
                                           _stream(stream)))

    def mr_rsa_mixed(self, keys, ops, inp, out, status=None, flags: int = 0, stream=None):
        """Mixed RSA encryptions / CRT decryptions of any sizes in one call (ops: MR_OP_* per row)."""
        kl = _keylist(keys)
        oa, op = _ops(ops)
        _, is_ = _rows(inp)
        _, os_ = _rows(out)
        self._check(lib.mr_rsa_mixed(self.handle, kl.arr, op, len(kl), _dev(inp), is_, _dev(out), os_, _dev(status),
                                     flags, _stream(stream)))

    def mr_plan_create(self, keys, ops, inp, out, status=None, flags: int = 0) -> Plan:
        kl = _keylist(keys)
        oa, op = _ops(ops)
        _, is_ = _rows(inp)
        _, os_ = _rows(out)
        h = ctypes.c_void_p()
        self._check(lib.mr_plan_create(self.handle, kl.arr, op, len(kl), _dev(inp), is_, _dev(out), os_, _dev(status),
                                       flags, ctypes.byref(h)))
        return Plan(self, h.value, (kl, inp, out, status))

    def mr_miller_rabin_batch(self, cand, witness, rounds: int, is_prime, round_mask=None, stream=None):
        n, nl = _rows(cand)
        self._check(lib.mr_miller_rabin_batch(self.handle, _dev(cand), nl, n, _dev(witness), rounds, _dev(is_prime),
                                              _dev(round_mask), _stream(stream)))

    def mr_prime_test_batch(self, cand, witness, rounds: int, verdict, n_primes: int = 10000, survivors=None,
                            stream=None):
        """verdict[i] = 0 (fails trial division), 1 (a Miller-Rabin round fails), 2 (probable prime)."""
        n, nl = _rows(cand)
        self._check(lib.mr_prime_test_batch(self.handle, _dev(cand), nl, n, _dev(witness), rounds, n_primes,
                                            _dev(verdict), _dev(survivors), _stream(stream)))

    def mr_rsa_keygen_batch(self, cand, witness, rounds: int, n_keys: int, pool: int, out, e: int = 65537,
                            status=None, stream=None):
        """Keys from candidate pools: out rows of 9 * half_limbs limbs (N, d, p, q, dp, dq, qinv)."""
        n, nl = _rows(cand)
        if n != n_keys * 2 * pool:
            raise ValueError("cand must hold n_keys * 2 * pool rows")
        self._check(lib.mr_rsa_keygen_batch(self.handle, nl, n_keys, pool, _dev(cand), _dev(witness), rounds, e,
                                            _dev(out), _dev(status), _stream(stream)))

    def mr_rsa_message_blocks(self, key: Key, length: int):
        """(n_blocks, bytes per block, limbs per ciphertext row) of a `length`-byte message."""
        nb, B, W = ctypes.c_size_t(), ctypes.c_uint32(), ctypes.c_uint32()
        self._check(lib.mr_rsa_message_blocks(key.handle, length, ctypes.byref(nb), ctypes.byref(B), ctypes.byref(W)))
        return nb.value, B.value, W.value

    def mr_rsa_encrypt_message(self, key: Key, msg, c, status=None, stream=None):
        """msg: contiguous uint8 CUDA tensor; c: n_blocks rows of W limbs."""
        self._check(lib.mr_rsa_encrypt_message(self.handle, key.handle, _dev(msg), msg.numel(), _dev(c), _dev(status),
                                               _stream(stream)))

    def mr_rsa_decrypt_message(self, key: Key, c, msg, status=None, stream=None):
        n, _ = _rows(c)
        self._check(lib.mr_rsa_decrypt_message(self.handle, key.handle, _dev(c), n, _dev(msg), msg.numel(),
                                               _dev(status), _stream(stream)))

    def mr_get_tuning(self, class_bits: int) -> dict:
        v, w, t = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        self._check(lib.mr_get_tuning(self.handle, class_bits, ctypes.byref(v), ctypes.byref(w), ctypes.byref(t)))
        return {"variant": v.value, "window_cap": w.value, "tuned": bool(t.value)}

    def mr_set_tuning(self, class_bits: int, variant: int, window_cap: int = 0):
        self._check(lib.mr_set_tuning(self.handle, class_bits, variant, window_cap))

    def save_tuning(self, path: str, classes: Sequence[int] = (512, 1024, 1536, 2048, 3072, 4096, 8192, 16384)):
        """Write the tuned classes' (variant, window cap) to a JSON file (an autotune cache)."""
        import json
        state = {}
        for L in classes:
            t = self.mr_get_tuning(L)
            if t["tuned"]:
                state[str(L)] = {"variant": t["variant"], "window_cap": t["window_cap"]}
        with open(path, "w") as f:
            json.dump({"mr_tuning": 1, "classes": state}, f, indent=1, sort_keys=True)
        return state

    def load_tuning(self, path: str) -> dict:
        """Install the tuning saved by save_tuning."""
        import json
        with open(path) as f:
            d = json.load(f)
        for L, t in d.get("classes", {}).items():
            self.mr_set_tuning(int(L), int(t["variant"]), int(t["window_cap"]))
        return d.get("classes", {})

    def mr_debug_mr_setup(self, cand, out, stream=None):
        n, nl = _rows(cand)
        self._check(lib.mr_debug_mr_setup(self.handle, _dev(cand), nl, n, _dev(out), _stream(stream)))

    def mr_set_variant(self, class_bits: int, variant: int):
        self._check(lib.mr_set_variant(self.handle, class_bits, variant))

    def mr_profile_enable(self, on: bool = True):
        self._check(lib.mr_profile_enable(self.handle, 1 if on else 0))

    def mr_profile_read(self):
        """[(launches, ms) for the exponentiation kernels, (launches, ms) for the CRT kernels]"""
        arr = (KernelTime * 2)()
        self._check(lib.mr_profile_read(self.handle, arr, 2))
        return [(arr[i].launches, arr[i].ms) for i in range(2)]

    def mr_autotune(self, class_bits: int, n_items: int, exp_bits: int) -> dict:
        """Time the lane mappings and window widths of a size class; keep the fastest (see mr.h)."""
        r = TuneResult()
        self._check(lib.mr_autotune(self.handle, class_bits, n_items, exp_bits, ctypes.byref(r)))
        return {"variant": r.variant, "lanes_per_number": r.lanes_per_number, "window": r.window,
                "configs": r.configs, "ms": r.ms, "ms_default": r.ms_default}

    def mr_set_constant_time(self, on: bool = True):
        """Constant-time exponentiation schedule for later calls and plans (see mr.h)."""
        self._check(lib.mr_set_constant_time(self.handle, 1 if on else 0))

    def mr_debug_big_phases(self, on: bool = True) -> List[int]:
        """Phase cycle counters of the large classes' tensor-core form (see mr.h): returns the 8 sums
        and the block count accumulated so far, then restarts them (on) or releases them (off)."""
        buf = (ctypes.c_uint64 * 9)()
        self._check(lib.mr_debug_big_phases(self.handle, 1 if on else 0, buf))
        return [int(v) for v in buf]

    def mr_debug_lane_tc_wait(self, skip: bool):
        """Test hook: the lane-group tensor-core kernels issue no product (see mr.h)."""
        self._check(lib.mr_debug_lane_tc_wait(self.handle, 1 if skip else 0))

    def mr_debug_big_wait(self, spin_limit: int = 0, absent_slice: int = -1):
        """Test hook of the large classes' bounded waits (see mr.h)."""
        self._check(lib.mr_debug_big_wait(self.handle, spin_limit, absent_slice))

    def mr_imad_peak(self, kind: int = 0, stream=None) -> float:
        """Measured multiply-adds per second: kind 0 mad.wide.u32, 1 mad.lo.u32, 2 carry pair, 3 mad.hi.u32."""
        v = ctypes.c_double()
        self._check(lib.mr_imad_peak(self.handle, kind, _stream(stream), ctypes.byref(v)))
        return v.value

    def mr_tensor_peak(self, kind: int = 0, stream=None) -> float:
        """Measured tensor operations per second: kind 0 tcgen05 kind::f16, 1 mma.sync s8, 2 mma.sync f16."""
        v = ctypes.c_double()
        self._check(lib.mr_tensor_peak(self.handle, kind, _stream(stream), ctypes.byref(v)))
        return v.value

    def mr_debug_tc_mma(self, a: np.ndarray, b: np.ndarray, swap_strides: int = 0, stream=None) -> np.ndarray:
        """D = A B^T (fp16 in, fp32 out) through one tcgen05 CTA (layout test hook, see mr.h)."""
        a = np.ascontiguousarray(a, dtype=np.float16)
        b = np.ascontiguousarray(b, dtype=np.float16)
        n, kdim = b.shape
        d = np.zeros((a.shape[0], n), dtype=np.float32)
        self._check(lib.mr_debug_tc_mma(self.handle, a.ctypes.data, b.ctypes.data, n, kdim, swap_strides,
                                        d.ctypes.data, _stream(stream)))
        return d

    def mr_debug_table(self, name: str, key: Optional[Key] = None, class_bits: int = 0) -> List[int]:
        cnt = ctypes.c_size_t()
        kh = key.handle if key else None
        self._check(lib.mr_debug_table(self.handle, class_bits, kh, name.encode(), None, 0, ctypes.byref(cnt)))
        out = np.zeros(cnt.value, dtype=np.uint32)
        self._check(lib.mr_debug_table(self.handle, class_bits, kh, name.encode(), _ptr(out), cnt.value,
                                       ctypes.byref(cnt)))
        return [int(v) for v in out]


def mr_big_variant_info(class_bits: int, variant: int) -> dict:
    """Channels per block, blocks per group and tensor-core flag of a large-class variant (see mr.h)."""
    sc, sl, tc = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    rc = lib.mr_big_variant_info(class_bits, variant, ctypes.byref(sc), ctypes.byref(sl), ctypes.byref(tc))
    if rc:
        raise MRError(rc, f"no variant {variant} of large class {class_bits}")
    return {"slice_channels": sc.value, "slices": sl.value, "tensor": bool(tc.value)}


def mr_debug_tc_slices(class_bits: int) -> np.ndarray:
    """The tensor-core operand table of a size class as fp16 values (see mr.h), host-built."""
    cnt = ctypes.c_size_t()
    rc = lib.mr_debug_tc_slices(class_bits, None, 0, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, f"no tensor-core table for class {class_bits}")
    out = np.zeros(cnt.value, dtype=np.uint32)
    rc = lib.mr_debug_tc_slices(class_bits, _ptr(out), cnt.value, ctypes.byref(cnt))
    if rc:
        raise MRError(rc, "tensor-core table")
    return out.view(np.float16)


def to_tensor(values: Iterable[int], n_limbs: int, device="cuda"):
    """Pack Python ints into a (rows x n_limbs) int32 tensor of little-endian limbs."""
    import torch
    vals = list(values)
    arr = np.zeros((len(vals), n_limbs), dtype=np.uint32)
    for i, v in enumerate(vals):
        arr[i] = _limbs(v, n_limbs)
    return torch.from_numpy(arr.view(np.int32)).to(device)


def from_tensor(t) -> List[int]:
    """Unpack a (rows x limbs) 32-bit tensor into Python ints."""
    a = t.detach().cpu().contiguous().numpy().view(np.uint32)
    return [int.from_bytes(row.astype("<u4").tobytes(), "little") for row in a]
