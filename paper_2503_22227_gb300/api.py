"""Thin Python binding of the C ABI in ``include/catfhe.h``.

Argument marshalling only: every step of every operation runs in the CUDA
kernels of ``libcatfhe.so``.  PyTorch supplies device memory (ciphertexts
and workspaces are ``torch.int64`` CUDA tensors holding the uint64
residues bit for bit) and the current CUDA stream.  There is no CPU
fallback: if the library is missing, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads as W

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcatfhe.so")

CKKS, BFV, BGV = 0, 1, 2
OP_MUL_RELIN, OP_MUL_RELIN_RESCALE, OP_ROTATE, OP_RESCALE, OP_DECRYPT, OP_EXPORT, OP_NTT = range(1, 8)
OP_ADD, OP_SUB, OP_MUL_INT, OP_ADD_CONST, OP_DROP = range(8, 13)
OP_ROTATE_HOISTED = 13
OP_MUL_PLAIN = 14
OP_ENCODE, OP_DECODE = 15, 16
FORM_COEFF, FORM_NATIVE = 0, 1
FORM_ASYNC = 0x100      # OR-ed into a form: import / export without synchronising

# every symbol include/catfhe.h declares
EXPORTS = [
    "catfhe_strerror", "catfhe_ctx_create", "catfhe_ctx_destroy", "catfhe_ctx_info",
    "catfhe_ctx_moduli", "catfhe_galois_elt", "catfhe_keygen", "catfhe_gen_galois_key",
    "catfhe_keys_destroy", "catfhe_keys_export", "catfhe_encrypt", "catfhe_ct_uniform",
    "catfhe_ct_import", "catfhe_ct_export", "catfhe_add", "catfhe_mul_relin",
    "catfhe_mul_relin_rescale", "catfhe_rotate", "catfhe_rescale", "catfhe_decrypt",
    "catfhe_ntt", "catfhe_workspace_bytes", "catfhe_measure_int_peak", "catfhe_kernel_launches",
    "catfhe_rescale_noalloc", "catfhe_batch_workspace_bytes", "catfhe_run_batch",
    "catfhe_batch_capture", "catfhe_graph_launch", "catfhe_graph_nodes", "catfhe_graph_destroy",
    "catfhe_tune_ntt", "catfhe_ntt_schedule", "catfhe_set_ntt_schedule",
    "catfhe_sub", "catfhe_mul_int", "catfhe_add_const", "catfhe_drop_level",
    "catfhe_rotate_hoisted", "catfhe_plain_import", "catfhe_mul_plain",
    "catfhe_encode_ckks", "catfhe_decode_ckks", "catfhe_device_status", "catfhe_wait_selftest",
    "catfhe_packed_words", "catfhe_ct_import_packed", "catfhe_ct_export_packed",
    "catfhe_pack_host", "catfhe_unpack_host", "catfhe_sync", "catfhe_measure_imad_rates",
]


class Params(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("log_n", ctypes.c_int32),
                ("log_n_max", ctypes.c_int32), ("L", ctypes.c_int32), ("K", ctypes.c_int32),
                ("dnum", ctypes.c_int32), ("q_bits", ctypes.c_int32 * 64),
                ("p_bits", ctypes.c_int32 * 16), ("t", ctypes.c_uint64),
                ("aux_count", ctypes.c_int32), ("aux_bits", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("L", ctypes.c_int32), ("K", ctypes.c_int32),
                ("nb", ctypes.c_int32), ("alpha", ctypes.c_int32), ("beta", ctypes.c_int32)]


class Op(ctypes.Structure):
    """One entry of an uneven batch (catfhe_op)."""
    _fields_ = [("op", ctypes.c_int32), ("level", ctypes.c_uint32), ("count", ctypes.c_uint32),
                ("level_out", ctypes.c_uint32), ("ctx", ctypes.c_void_p), ("keys", ctypes.c_void_p),
                ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("arg", ctypes.c_uint64)]


class CatfheError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_lib.catfhe_strerror(code).decode()} ({code})")


_lib = None
_lock = threading.Lock()
vp, u64, i64, u32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
u8p = ctypes.POINTER(ctypes.c_uint8)


def load(path: str = LIB_PATH):
    """Loads libcatfhe.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libcatfhe.so not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        sig = {
            "catfhe_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "catfhe_ctx_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(vp)]),
            "catfhe_ctx_destroy": (None, [vp]),
            "catfhe_ctx_info": (ctypes.c_int, [vp, ctypes.POINTER(Info)]),
            "catfhe_ctx_moduli": (ctypes.c_int, [vp, vp, vp, vp]),
            "catfhe_galois_elt": (u64, [vp, i64]),
            "catfhe_keygen": (ctypes.c_int, [vp, u8p, ctypes.POINTER(vp)]),
            "catfhe_gen_galois_key": (ctypes.c_int, [vp, vp, u64]),
            "catfhe_keys_destroy": (None, [vp]),
            "catfhe_keys_export": (ctypes.c_int, [vp, vp, u64, vp, vp, vp]),
            "catfhe_encrypt": (ctypes.c_int, [vp, vp, vp, u8p, vp, vp]),
            "catfhe_ct_uniform": (ctypes.c_int, [vp, u8p, u32, u32, vp, vp]),
            "catfhe_ct_import": (ctypes.c_int, [vp, vp, u32, u32, ctypes.c_int, vp, vp]),
            "catfhe_ct_export": (ctypes.c_int, [vp, vp, u32, u32, ctypes.c_int, vp, vp, sz, vp]),
            "catfhe_packed_words": (sz, [vp, u32, u32]),
            "catfhe_ct_import_packed": (ctypes.c_int, [vp, vp, u32, u32, vp, vp, sz, ctypes.c_int, vp]),
            "catfhe_ct_export_packed": (ctypes.c_int, [vp, vp, u32, u32, vp, vp, sz, ctypes.c_int, vp]),
            "catfhe_pack_host": (ctypes.c_int, [vp, u32, u32, u32, vp, vp]),
            "catfhe_unpack_host": (ctypes.c_int, [vp, u32, u32, u32, vp, vp]),
            "catfhe_add": (ctypes.c_int, [vp, vp, vp, vp, u32, u32, vp]),
            "catfhe_mul_relin": (ctypes.c_int, [vp, vp, vp, vp, vp, u32, u32, vp, sz, vp]),
            "catfhe_mul_relin_rescale": (ctypes.c_int, [vp, vp, vp, vp, vp, u32, u32, vp, sz, vp]),
            "catfhe_rotate": (ctypes.c_int, [vp, vp, vp, u64, vp, u32, u32, vp, sz, vp]),
            "catfhe_rotate_hoisted": (ctypes.c_int, [vp, vp, vp, vp, u32, vp, u32, u32, vp, sz, vp]),
            "catfhe_plain_import": (ctypes.c_int, [vp, vp, u32, vp, vp]),
            "catfhe_mul_plain": (ctypes.c_int, [vp, vp, vp, vp, u32, u32, vp]),
            "catfhe_encode_ckks": (ctypes.c_int, [vp, vp, ctypes.c_double, u32, vp, vp, sz, vp]),
            "catfhe_device_status": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, vp]),
            "catfhe_wait_selftest": (ctypes.c_int, [vp, u64, vp]),
            "catfhe_decode_ckks": (ctypes.c_int, [vp, vp, vp, u32, ctypes.c_double, vp, vp, sz, vp]),
            "catfhe_rescale": (ctypes.c_int, [vp, vp, vp, u32, u32, vp, sz, vp]),
            "catfhe_decrypt": (ctypes.c_int, [vp, vp, vp, u32, u64, vp, vp, sz, vp]),
            "catfhe_ntt": (ctypes.c_int, [vp, vp, u32, u32, ctypes.c_int, vp]),
            "catfhe_workspace_bytes": (sz, [vp, ctypes.c_int, u32, u32]),
            "catfhe_measure_int_peak": (ctypes.c_int, [vp, vp, vp, vp]),
            "catfhe_measure_imad_rates": (ctypes.c_int, [vp, vp, vp, vp]),
            "catfhe_kernel_launches": (u64, []),
            "catfhe_rescale_noalloc": (ctypes.c_int, [vp, vp, vp, u32, u32, vp]),
            "catfhe_sync": (ctypes.c_int, [vp, vp]),
            "catfhe_batch_workspace_bytes": (sz, [vp, u32, u32]),
            "catfhe_run_batch": (ctypes.c_int, [vp, u32, u32, vp, sz, vp]),
            "catfhe_batch_capture": (ctypes.c_int, [vp, u32, u32, vp, sz, ctypes.POINTER(vp)]),
            "catfhe_graph_launch": (ctypes.c_int, [vp, vp]),
            "catfhe_graph_nodes": (sz, [vp]),
            "catfhe_graph_destroy": (None, [vp]),
            "catfhe_tune_ntt": (ctypes.c_int, [vp, u32, vp, ctypes.POINTER(ctypes.c_int32), vp]),
            "catfhe_ntt_schedule": (ctypes.c_int, [vp, u32, ctypes.POINTER(ctypes.c_int32),
                                                   ctypes.POINTER(ctypes.c_int32), vp]),
            "catfhe_set_ntt_schedule": (ctypes.c_int, [vp, ctypes.c_int32]),
            "catfhe_sub": (ctypes.c_int, [vp, vp, vp, vp, u32, u32, vp]),
            "catfhe_mul_int": (ctypes.c_int, [vp, vp, i64, vp, u32, u32, vp]),
            "catfhe_add_const": (ctypes.c_int, [vp, vp, i64, vp, u32, u32, vp]),
            "catfhe_drop_level": (ctypes.c_int, [vp, vp, u32, u32, vp, u32, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise CatfheError(rc, what)


def _seed(seed: bytes):
    assert len(seed) == 32
    return (ctypes.c_uint8 * 32).from_buffer_copy(seed)


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def params_from_preset(p: W.Preset) -> Params:
    prm = Params()
    prm.scheme, prm.log_n = p.scheme, p.log_n
    prm.log_n_max = p.log_n_max or p.log_n
    prm.L, prm.K, prm.dnum = p.L, p.K, p.dnum
    for i, b in enumerate(p.q_bits):
        prm.q_bits[i] = b
    for i, b in enumerate(p.p_bits):
        prm.p_bits[i] = b
    prm.t = p.t
    prm.aux_count = 0
    prm.aux_bits = p.b_bits
    return prm


class Context:
    """A parameter set on the current CUDA device (primes, NTT tables)."""

    def __init__(self, preset: W.Preset | Params):
        L = load()
        prm = params_from_preset(preset) if isinstance(preset, W.Preset) else preset
        self.preset = preset if isinstance(preset, W.Preset) else None
        h = vp()
        _check(L.catfhe_ctx_create(ctypes.byref(prm), ctypes.byref(h)), "catfhe_ctx_create")
        self._h = h
        info = Info()
        _check(L.catfhe_ctx_info(h, ctypes.byref(info)), "catfhe_ctx_info")
        self.n, self.L, self.K, self.nb = info.n, info.L, info.K, info.nb
        self.alpha, self.beta = info.alpha, info.beta
        self.scheme, self.t = prm.scheme, prm.t
        q = (ctypes.c_uint64 * self.L)()
        p = (ctypes.c_uint64 * self.K)()
        b = (ctypes.c_uint64 * max(1, self.nb))()
        _check(L.catfhe_ctx_moduli(h, q, p, b), "catfhe_ctx_moduli")
        self.q, self.p, self.b = list(q), list(p), list(b)[: self.nb]
        self._ws = {}

    def close(self):
        if getattr(self, "_h", None):
            load().catfhe_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- buffers
    def empty_ct(self, count: int, level: int):
        torch = _torch()
        return torch.empty((count, 2, level, self.n), dtype=torch.int64, device="cuda")

    def workspace(self, op: int, level: int, count: int):
        torch = _torch()
        need = load().catfhe_workspace_bytes(self._h, op, level, count)
        key = (op, level, count)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
            self._ws[key] = ws
        return ws

    def galois_elt(self, steps: int) -> int:
        return int(load().catfhe_galois_elt(self._h, steps))

    # ---------------------------------------------------------------- keys
    def keygen(self, seed: bytes) -> "Keys":
        return Keys(self, seed)

    # ---------------------------------------------------------------- ciphertext I/O
    def encrypt(self, keys: "Keys", msg: np.ndarray, seed: bytes):
        m = np.ascontiguousarray(np.asarray(msg, dtype=np.int64))
        assert m.shape == (self.n,)
        out = self.empty_ct(1, self.L)
        _check(load().catfhe_encrypt(self._h, keys._h, m.ctypes.data_as(vp), _seed(seed), _ptr(out),
                                     _stream()), "catfhe_encrypt")
        return out

    def ct_uniform(self, seed: bytes, index: int, level: int):
        out = self.empty_ct(1, level)
        _check(load().catfhe_ct_uniform(self._h, _seed(seed), index, level, _ptr(out), _stream()),
               "catfhe_ct_uniform")
        return out

    def import_ct(self, host, form: int = FORM_COEFF, out=None):
        """host: uint64 numpy array, or a (pinned) CPU int64 tensor, shaped
        [count][2][level][N] -> device tensor in the at-rest form."""
        torch = _torch()
        if isinstance(host, torch.Tensor):
            assert host.device.type == "cpu" and host.is_contiguous() and host.dtype == torch.int64
            count, _, level, _ = host.shape
            hp = ctypes.c_void_p(host.data_ptr())
            keep = host
        else:
            h = np.ascontiguousarray(host, dtype=np.uint64)
            if h.ndim == 3:
                h = h[None]
            count, _, level, _ = h.shape
            hp = h.ctypes.data_as(vp)
            keep = h
        out = self.empty_ct(count, level) if out is None else out
        _check(load().catfhe_ct_import(self._h, hp, level, count, form, _ptr(out), _stream()),
               "catfhe_ct_import")
        del keep
        return out

    def export_into(self, ct, host, form: int = FORM_NATIVE, ws=None):
        """Device ciphertexts -> a (pinned) CPU int64 tensor of the same shape
        (ws: a workspace from workspace(OP_EXPORT, level, count), or None)."""
        count, _, level, _ = ct.shape
        if ws is None:
            ws = self.workspace(OP_EXPORT, level, count)
        _check(load().catfhe_ct_export(self._h, _ptr(ct), level, count, form,
                                       ctypes.c_void_p(host.data_ptr()), _ptr(ws), ws.numel(),
                                       _stream()), "catfhe_ct_export")
        return host

    # ------------------------------------------------ bit-packed transfers
    def bits(self, level: int) -> np.ndarray:
        """Bit length of q_0 .. q_{level-1}: the packed form's field widths."""
        return np.array([int(q).bit_length() for q in self.q[:level]], dtype=np.uint8)

    def packed_words(self, level: int, count: int) -> int:
        return int(load().catfhe_packed_words(self._h, level, count))

    def pack(self, limbs, out=None):
        """Host [count][2][level][N] residues (numpy uint64 or CPU int64
        tensor) -> the packed words (a flat array of the same kind)."""
        count, _, level, n = limbs.shape
        words = self.packed_words(level, count)
        if out is None:
            out = (np.empty(words, dtype=np.uint64) if isinstance(limbs, np.ndarray)
                   else _torch().empty(words, dtype=_torch().int64))
        bits = self.bits(level)
        _check(load().catfhe_pack_host(bits.ctypes.data_as(vp), level, 2 * count,
                                       n.bit_length() - 1, _hptr(limbs), _hptr(out)),
               "catfhe_pack_host")
        return out

    def unpack(self, packed, count: int, level: int) -> np.ndarray:
        out = np.empty((count, 2, level, self.n), dtype=np.uint64)
        bits = self.bits(level)
        _check(load().catfhe_unpack_host(bits.ctypes.data_as(vp), level, 2 * count,
                                         self.n.bit_length() - 1, _hptr(packed), _hptr(out)),
               "catfhe_unpack_host")
        return out

    def import_packed(self, packed, level: int, count: int, out=None, ws=None, flags: int = 0):
        """Packed host words -> device ciphertexts (at-rest form); ws: a
        device buffer of at least packed_words * 8 bytes (None: the
        context's scratch)."""
        out = self.empty_ct(count, level) if out is None else out
        nb = 0 if ws is None else ws.numel() * ws.element_size()
        _check(load().catfhe_ct_import_packed(self._h, _hptr(packed), level, count, _ptr(out),
                                              None if ws is None else _ptr(ws), nb, flags,
                                              _stream()), "catfhe_ct_import_packed")
        return out

    def export_packed(self, ct, packed=None, ws=None, flags: int = 0):
        count, _, level, _ = ct.shape
        if packed is None:
            packed = np.empty(self.packed_words(level, count), dtype=np.uint64)
        nb = 0 if ws is None else ws.numel() * ws.element_size()
        _check(load().catfhe_ct_export_packed(self._h, _ptr(ct), level, count, _hptr(packed),
                                              None if ws is None else _ptr(ws), nb, flags,
                                              _stream()), "catfhe_ct_export_packed")
        return packed

    def export_ct(self, ct, form: int = FORM_COEFF) -> np.ndarray:
        count, _, level, n = ct.shape
        host = np.empty((count, 2, level, n), dtype=np.uint64)
        ws = self.workspace(OP_EXPORT, level, count)
        _check(load().catfhe_ct_export(self._h, _ptr(ct), level, count, form, host.ctypes.data_as(vp),
                                       _ptr(ws), ws.numel(), _stream()), "catfhe_ct_export")
        return host

    def decrypt(self, keys: "Keys", ct, factor: int = 1) -> np.ndarray:
        level = ct.shape[-2]
        out = np.empty(self.n, dtype=np.int64)
        ws = self.workspace(OP_DECRYPT, level, 1)
        _check(load().catfhe_decrypt(self._h, keys._h, _ptr(ct), level, factor, out.ctypes.data_as(vp),
                                     _ptr(ws), ws.numel(), _stream()), "catfhe_decrypt")
        return out

    # ---------------------------------------------------------------- operations
    def add(self, a, b, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level) if out is None else out
        _check(load().catfhe_add(self._h, _ptr(a), _ptr(b), _ptr(out), level, count, _stream()),
               "catfhe_add")
        return out

    def sub(self, a, b, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level) if out is None else out
        _check(load().catfhe_sub(self._h, _ptr(a), _ptr(b), _ptr(out), level, count, _stream()),
               "catfhe_sub")
        return out

    def mul_int(self, a, k: int, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level) if out is None else out
        _check(load().catfhe_mul_int(self._h, _ptr(a), k, _ptr(out), level, count, _stream()),
               "catfhe_mul_int")
        return out

    def add_const(self, a, k: int, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level) if out is None else out
        _check(load().catfhe_add_const(self._h, _ptr(a), k, _ptr(out), level, count, _stream()),
               "catfhe_add_const")
        return out

    def drop_level(self, a, new_level: int, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, new_level) if out is None else out
        _check(load().catfhe_drop_level(self._h, _ptr(a), level, new_level, _ptr(out), count,
                                        _stream()), "catfhe_drop_level")
        return out

    def mul_relin(self, keys: "Keys", a, b, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level) if out is None else out
        ws = self.workspace(OP_MUL_RELIN, level, count)
        _check(load().catfhe_mul_relin(self._h, keys._h, _ptr(a), _ptr(b), _ptr(out), level, count,
                                       _ptr(ws), ws.numel(), _stream()), "catfhe_mul_relin")
        return out

    def mul_relin_rescale(self, keys: "Keys", a, b, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level - 1) if out is None else out
        ws = self.workspace(OP_MUL_RELIN_RESCALE, level, count)
        _check(load().catfhe_mul_relin_rescale(self._h, keys._h, _ptr(a), _ptr(b), _ptr(out), level,
                                               count, _ptr(ws), ws.numel(), _stream()),
               "catfhe_mul_relin_rescale")
        return out

    def rotate(self, keys: "Keys", a, galois_elt: int, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level) if out is None else out
        ws = self.workspace(OP_ROTATE, level, count)
        _check(load().catfhe_rotate(self._h, keys._h, _ptr(a), galois_elt, _ptr(out), level, count,
                                    _ptr(ws), ws.numel(), _stream()), "catfhe_rotate")
        return out

    def plain_import(self, coeffs, level: int | None = None):
        """Signed plaintext coefficients (int64[N]) -> device plaintext
        [level][N] in NTT form, for mul_plain."""
        level = self.L if level is None else level
        m = np.ascontiguousarray(np.asarray(coeffs, dtype=np.int64))
        assert m.shape == (self.n,)
        torch = _torch()
        pt = torch.empty((level, self.n), dtype=torch.int64, device="cuda")
        _check(load().catfhe_plain_import(self._h, m.ctypes.data_as(vp), level, _ptr(pt), _stream()),
               "catfhe_plain_import")
        return pt

    def encode_ckks(self, slots, scale: float, level: int | None = None):
        """N/2 complex slots -> device plaintext [level][N] (NTT form), encoded
        on the device."""
        level = self.L if level is None else level
        z = np.ascontiguousarray(np.asarray(slots, dtype=np.complex128))
        assert z.shape == (self.n // 2,)
        torch = _torch()
        pt = torch.empty((level, self.n), dtype=torch.int64, device="cuda")
        ws = self.workspace(OP_ENCODE, level, 1)
        _check(load().catfhe_encode_ckks(self._h, z.ctypes.data_as(vp), float(scale), level,
                                         _ptr(pt), _ptr(ws), ws.numel(), _stream()),
               "catfhe_encode_ckks")
        return pt

    def decode_ckks(self, keys: "Keys", ct, scale: float) -> np.ndarray:
        """Decrypts one ciphertext and decodes its slots on the device."""
        level = ct.shape[-2]
        z = np.empty(self.n // 2, dtype=np.complex128)
        ws = self.workspace(OP_DECODE, level, 1)
        _check(load().catfhe_decode_ckks(self._h, keys._h, _ptr(ct), level, float(scale),
                                         z.ctypes.data_as(vp), _ptr(ws), ws.numel(), _stream()),
               "catfhe_decode_ckks")
        return z

    def device_status(self, clear: bool = True) -> int:
        """Status word of the kernels' bounded waits (0: none timed out)."""
        v = ctypes.c_int32(0)
        _check(load().catfhe_device_status(self._h, ctypes.byref(v), 1 if clear else 0, _stream()),
               "catfhe_device_status")
        return v.value

    def sync(self) -> None:
        """Waits for the current stream; raises CatfheError (ETIMEOUT) if a
        bounded wait of this context's kernels has given up."""
        _check(load().catfhe_sync(self._h, _stream()), "catfhe_sync")

    def wait_selftest(self, limit_ns: int = 20_000_000) -> None:
        _check(load().catfhe_wait_selftest(self._h, int(limit_ns), _stream()), "catfhe_wait_selftest")

    def mul_plain(self, a, pt, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level) if out is None else out
        _check(load().catfhe_mul_plain(self._h, _ptr(a), _ptr(pt), _ptr(out), level, count,
                                       _stream()), "catfhe_mul_plain")
        return out

    def rotate_hoisted(self, keys: "Keys", a, galois_elts, out=None):
        """Rotations of the same ciphertexts by every Galois element, one
        shared ModUp: returns (or fills) [n_rot][count][2][level][N]."""
        count, _, level, n = a.shape
        gs = np.ascontiguousarray(np.asarray(galois_elts, dtype=np.uint64))
        torch = _torch()
        if out is None:
            out = torch.empty((len(gs), count, 2, level, n), dtype=torch.int64, device="cuda")
        ws = self.workspace(OP_ROTATE_HOISTED, level, count)
        _check(load().catfhe_rotate_hoisted(self._h, keys._h, _ptr(a), gs.ctypes.data_as(vp),
                                            len(gs), _ptr(out), level, count, _ptr(ws), ws.numel(),
                                            _stream()), "catfhe_rotate_hoisted")
        return out

    def rescale(self, a, out=None):
        count, _, level, _ = a.shape
        out = self.empty_ct(count, level - 1) if out is None else out
        ws = self.workspace(OP_RESCALE, level, count)
        _check(load().catfhe_rescale(self._h, _ptr(a), _ptr(out), level, count, _ptr(ws), ws.numel(),
                                     _stream()), "catfhe_rescale")
        return out

    def rescale_noalloc(self, a, out):
        """catfhe_rescale_noalloc: the rescale with the library's static
        scratch, for callers that cannot allocate device memory."""
        count, _, level, _ = a.shape
        _check(load().catfhe_rescale_noalloc(self._h, _ptr(a), _ptr(out), level, count, _stream()),
               "catfhe_rescale_noalloc")
        return out

    def tune_ntt(self, limbs: int):
        """Times every NTT schedule of this ring degree on `limbs` limbs; keeps
        the fastest for launches of that size class."""
        chosen = ctypes.c_int32()
        us = (ctypes.c_float * 8)()
        _check(load().catfhe_tune_ntt(self._h, limbs, _stream(), ctypes.byref(chosen), us),
               "catfhe_tune_ntt")
        idx, count, shape = self.ntt_schedule(limbs)
        return chosen.value, [round(us[i], 2) for i in range(count)]

    def ntt_schedule(self, limbs: int = 1 << 20):
        """(index, count, shape) of the schedule used for launches of `limbs`
        limbs (default: the largest size class)."""
        idx, count = ctypes.c_int32(), ctypes.c_int32()
        shape = (ctypes.c_int32 * 4)()
        _check(load().catfhe_ntt_schedule(self._h, limbs, ctypes.byref(idx), ctypes.byref(count),
                                          shape), "catfhe_ntt_schedule")
        return idx.value, count.value, list(shape)

    def set_ntt_schedule(self, index: int):
        _check(load().catfhe_set_ntt_schedule(self._h, index), "catfhe_set_ntt_schedule")

    def ntt(self, limbs, inverse: bool = False):
        """limbs: int64 tensor [count][level][N], transformed in place."""
        count, level, _ = limbs.shape
        _check(load().catfhe_ntt(self._h, _ptr(limbs), level, count, int(inverse), _stream()),
               "catfhe_ntt")
        return limbs


def _hptr(x):
    """Host address of a contiguous numpy array or CPU tensor."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"] and x.dtype.itemsize == 8
        return x.ctypes.data_as(vp)
    assert x.device.type == "cpu" and x.is_contiguous() and x.element_size() == 8
    return ctypes.c_void_p(x.data_ptr())


def measure_int_peak() -> tuple[float, float, float]:
    """(Shoup modmul/s, forward butterfly/s for primes of 57 bits or more,
    forward butterfly/s for smaller primes) ceilings of the current device."""
    mm, bf, bw = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().catfhe_measure_int_peak(ctypes.byref(mm), ctypes.byref(bf), ctypes.byref(bw),
                                          _stream()),
           "catfhe_measure_int_peak")
    return mm.value, bf.value, bw.value


def measure_imad_rates() -> tuple[float, float, float]:
    """(mad.lo.u32, mad.hi.u32, mad.wide.u32) thread instructions per second."""
    lo, hi, wide = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().catfhe_measure_imad_rates(ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(wide),
                                            _stream()), "catfhe_measure_imad_rates")
    return lo.value, hi.value, wide.value


def kernel_launches() -> int:
    return int(load().catfhe_kernel_launches())


def make_op(kind: int, ctx: "Context", a, out, keys: "Keys" = None, b=None, galois_elt: int = 0,
            const: int = 0) -> Op:
    """An entry of an uneven batch: `a`, `b`, `out` are device tensors
    [count][2][level][N] of ctx's ring degree (for MUL_PLAIN `b` is a
    plaintext from plain_import).  galois_elt for rotations, const (int64)
    for MUL_INT / ADD_CONST; DROP takes the level of `out`."""
    count, _, level, _ = a.shape
    return make_op_ptr(kind, ctx, count, level, out.shape[2], a.data_ptr(),
                       b.data_ptr() if b is not None else None, out.data_ptr(), keys=keys,
                       galois_elt=galois_elt, const=const)


def make_op_ptr(kind: int, ctx: "Context", count: int, level: int, level_out: int, a: int,
                b, out: int, keys: "Keys" = None, galois_elt: int = 0, const: int = 0) -> Op:
    """make_op from device addresses: `a` (and `b`, or None) hold
    [count][2][level][N] words, `out` [count][2][level_out][N]."""
    o = Op()
    o.op = kind
    o.count, o.level, o.level_out = count, level, level_out
    o.ctx = ctx._h.value
    o.keys = keys._h.value if keys is not None else None
    o.a = a
    o.b = b
    o.out = out
    o.arg = galois_elt if kind == OP_ROTATE else (const & 0xFFFFFFFFFFFFFFFF)
    return o


def _op_array(ops):
    arr = (Op * len(ops))(*ops)
    return arr


def batch_workspace_bytes(ops, lanes: int) -> int:
    return int(load().catfhe_batch_workspace_bytes(_op_array(ops), len(ops), lanes))


def run_batch(ops, lanes: int, ws=None):
    """Runs independent operations of any ring degree and level concurrently."""
    torch = _torch()
    arr = _op_array(ops)
    need = load().catfhe_batch_workspace_bytes(arr, len(ops), lanes)
    if need == 0:
        raise CatfheError(-1, "catfhe_batch_workspace_bytes")
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    _check(load().catfhe_run_batch(arr, len(ops), lanes, _ptr(ws), ws.numel(), _stream()),
           "catfhe_run_batch")
    return ws


class Batch:
    """An uneven batch marshalled once: the entry array serves both the
    workspace query and the submission."""

    def __init__(self, ops):
        self.n = len(ops)
        self.arr = _op_array(ops)

    def workspace_bytes(self, lanes: int) -> int:
        need = int(load().catfhe_batch_workspace_bytes(self.arr, self.n, lanes))
        if need == 0:
            raise CatfheError(-1, "catfhe_batch_workspace_bytes")
        return need

    def run(self, lanes: int, ws) -> None:
        _check(load().catfhe_run_batch(self.arr, self.n, lanes, _ptr(ws), ws.numel(), _stream()),
               "catfhe_run_batch")


class Graph:
    """A captured uneven batch, replayed with launch()."""

    def __init__(self, ops, lanes: int):
        torch = _torch()
        self._arr = _op_array(ops)
        need = load().catfhe_batch_workspace_bytes(self._arr, len(ops), lanes)
        if need == 0:
            raise CatfheError(-1, "catfhe_batch_workspace_bytes")
        self.ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        h = vp()
        _check(load().catfhe_batch_capture(self._arr, len(ops), lanes, _ptr(self.ws), self.ws.numel(),
                                           ctypes.byref(h)), "catfhe_batch_capture")
        self._h = h
        self.nodes = int(load().catfhe_graph_nodes(h))

    def launch(self):
        _check(load().catfhe_graph_launch(self._h, _stream()), "catfhe_graph_launch")

    def close(self):
        if getattr(self, "_h", None):
            load().catfhe_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Keys:
    def __init__(self, ctx: Context, seed: bytes):
        self.ctx = ctx
        h = vp()
        _check(load().catfhe_keygen(ctx._h, _seed(seed), ctypes.byref(h)), "catfhe_keygen")
        self._h = h

    def gen_galois(self, g: int) -> None:
        _check(load().catfhe_gen_galois_key(self.ctx._h, self._h, g), "catfhe_gen_galois_key")

    def export(self, key_id: int = 0, s=True, pk=True, ksk=True):
        c = self.ctx
        S = np.empty(c.n, dtype=np.int64) if s else None
        PK = np.empty((2, c.L, c.n), dtype=np.uint64) if pk else None
        KS = np.empty((c.beta, 2, c.L + c.K, c.n), dtype=np.uint64) if ksk else None
        _check(load().catfhe_keys_export(c._h, self._h, key_id,
                                         S.ctypes.data_as(vp) if s else None,
                                         PK.ctypes.data_as(vp) if pk else None,
                                         KS.ctypes.data_as(vp) if ksk else None), "catfhe_keys_export")
        return S, PK, KS

    def close(self):
        if getattr(self, "_h", None):
            load().catfhe_keys_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
