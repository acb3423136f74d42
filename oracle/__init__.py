"""CPU oracle for the RNS hot path of CKKS / BFV / BGV (arXiv 2503.22227).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import this package.  The product library never links or calls it, and it
shares no code with the CUDA path.

The C sources (``oc_*.c``) hold the plain definitions; this module builds
them with gcc into ``oracle/_build/liboracle.so`` and wraps them with
ctypes.  ``encode_ckks`` / ``decode_ckks`` are the oracle's own canonical
embedding, evaluated directly at the roots (O(N^2)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_DIR, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
SOURCES = ["oc_num.c", "oc_bigint.c", "oc_ntt.c", "oc_chacha.c", "oc_fhe.c"]

CKKS, BFV, BGV = 0, 1, 2
TAG_SK, TAG_PK_A, TAG_PK_E, TAG_KSK_A, TAG_KSK_E = 1, 2, 3, 4, 5
TAG_ENC_V, TAG_ENC_E0, TAG_ENC_E1, TAG_CT_UNIFORM = 6, 7, 8, 9

_lock = threading.Lock()
_lib = None

u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
u8p = ctypes.POINTER(ctypes.c_uint8)
intp = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_DIR, s) for s in SOURCES]
    hdr = os.path.join(_DIR, "oracle.h")
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs + [hdr]):
            return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            sig = {
                "oc_mulmod": (ctypes.c_uint64, [ctypes.c_uint64] * 3),
                "oc_powmod": (ctypes.c_uint64, [ctypes.c_uint64] * 3),
                "oc_invmod": (ctypes.c_uint64, [ctypes.c_uint64] * 2),
                "oc_is_prime": (ctypes.c_int, [ctypes.c_uint64]),
                "oc_gen_primes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                 u64p, ctypes.c_int, u64p]),
                "oc_min_psi": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_int]),
                "oc_ntt_fwd": (None, [u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]),
                "oc_ntt_inv": (None, [u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]),
                "oc_negacyclic_mul": (None, [u64p, u64p, u64p, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_uint64]),
                "oc_chacha20_block": (None, [u8p, ctypes.c_uint32, u8p, u8p]),
                "oc_stream_word": (ctypes.c_uint64, [u8p, ctypes.c_uint32, ctypes.c_uint32,
                                                     ctypes.c_uint32, ctypes.c_uint64]),
                "oc_cdt_table": (None, [u64p]),
                "oc_sample_uniform": (None, [u8p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             u64p, ctypes.c_int, ctypes.c_int, u64p]),
                "oc_sample_ternary": (None, [u8p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_int, i64p]),
                "oc_sample_gaussian": (None, [u8p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_int, i64p]),
                "oc_ctx_new": (ctypes.c_void_p, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 intp, ctypes.c_int, intp, ctypes.c_int, ctypes.c_uint64,
                                                 ctypes.c_int, ctypes.c_int]),
                "oc_ctx_free": (None, [ctypes.c_void_p]),
                "oc_ctx_moduli": (None, [ctypes.c_void_p, u64p, u64p, u64p, intp]),
                "oc_lift_centred": (None, [u64p, u64p, ctypes.c_int, u64p, ctypes.c_int, u64p,
                                           ctypes.c_uint64]),
                "oc_div_round": (None, [u64p, u64p, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_uint64]),
                "oc_div_t_exact": (None, [u64p, u64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                          u64p, ctypes.c_uint64]),
                "oc_automorphism": (None, [u64p, u64p, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_uint64]),
                "oc_keygen": (ctypes.c_void_p, [ctypes.c_void_p, u8p]),
                "oc_gen_galois": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
                "oc_keys_free": (None, [ctypes.c_void_p]),
                "oc_keys_export": (None, [ctypes.c_void_p, ctypes.c_void_p, i64p, u64p]),
                "oc_ksk_export": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, u64p]),
                "oc_encrypt": (None, [ctypes.c_void_p, ctypes.c_void_p, i64p, u8p, u64p]),
                "oc_ct_uniform": (None, [ctypes.c_void_p, u8p, ctypes.c_uint32, ctypes.c_int, u64p]),
                "oc_decrypt": (None, [ctypes.c_void_p, ctypes.c_void_p, u64p, ctypes.c_int,
                                      ctypes.c_uint64, i64p]),
                "oc_add": (None, [ctypes.c_void_p, u64p, u64p, u64p, ctypes.c_int]),
                "oc_sub": (None, [ctypes.c_void_p, u64p, u64p, u64p, ctypes.c_int]),
                "oc_mul_int": (None, [ctypes.c_void_p, u64p, ctypes.c_int64, u64p, ctypes.c_int]),
                "oc_add_const": (None, [ctypes.c_void_p, u64p, ctypes.c_int64, u64p, ctypes.c_int]),
                "oc_drop": (None, [ctypes.c_void_p, u64p, ctypes.c_int, ctypes.c_int, u64p]),
                "oc_mul_plain": (None, [ctypes.c_void_p, u64p, i64p, u64p, ctypes.c_int]),
                "oc_keyswitch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, u64p, ctypes.c_int,
                                                ctypes.c_uint64, u64p]),
                "oc_rescale": (None, [ctypes.c_void_p, u64p, u64p, ctypes.c_int]),
                "oc_tensor": (None, [ctypes.c_void_p, u64p, u64p, u64p, ctypes.c_int]),
                "oc_mul_relin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, u64p, u64p, u64p,
                                                ctypes.c_int]),
                "oc_rotate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, u64p, u64p,
                                             ctypes.c_int, ctypes.c_uint64]),
                "oc_galois_elt": (ctypes.c_uint64, [ctypes.c_int, ctypes.c_int64]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _u64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(u64p)


def _i64(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(i64p)


def _bytes(b: bytes):
    assert len(b) in (12, 32, 64)
    return (ctypes.c_uint8 * len(b)).from_buffer_copy(b)


# ---------------------------------------------------------------- primitives

def is_prime(n: int) -> bool:
    return bool(lib().oc_is_prime(n))


def gen_primes(bits: int, count: int, two_n: int, exclude=()) -> list[int]:
    ex = np.array(list(exclude) or [0], dtype=np.uint64)
    out = np.zeros(count, dtype=np.uint64)
    k = lib().oc_gen_primes(bits, count, two_n, _u64(ex), len(exclude), _u64(out))
    return [int(x) for x in out[:k]]


def min_psi(q: int, log_n: int) -> int:
    return int(lib().oc_min_psi(q, log_n))


def ntt(a, log_n: int, q: int, psi: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).copy()
    lib().oc_ntt_fwd(_u64(x), log_n, q, psi)
    return x


def intt(a, log_n: int, q: int, psi: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).copy()
    lib().oc_ntt_inv(_u64(x), log_n, q, psi)
    return x


def negacyclic_mul(a, b, log_n: int, q: int, psi: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    y = np.ascontiguousarray(np.asarray(b, dtype=np.uint64))
    out = np.empty_like(x)
    lib().oc_negacyclic_mul(_u64(out), _u64(x), _u64(y), log_n, q, psi)
    return out


def chacha20_block(key: bytes, counter: int, nonce: bytes) -> bytes:
    out = (ctypes.c_uint8 * 64)()
    lib().oc_chacha20_block(_bytes(key), counter, _bytes(nonce), out)
    return bytes(out)


def stream_word(key: bytes, tag: int, i0: int, i1: int, w: int) -> int:
    return int(lib().oc_stream_word(_bytes(key), tag, i0, i1, w))


def cdt_table() -> list[int]:
    out = np.zeros(19, dtype=np.uint64)
    lib().oc_cdt_table(_u64(out))
    return [int(x) for x in out]


def sample_uniform(key, tag, i0, i1, mods, log_n) -> np.ndarray:
    m = np.array(mods, dtype=np.uint64)
    out = np.zeros((len(mods), 1 << log_n), dtype=np.uint64)
    lib().oc_sample_uniform(_bytes(key), tag, i0, i1, _u64(m), len(mods), log_n, _u64(out))
    return out


def sample_ternary(key, tag, i0, i1, log_n) -> np.ndarray:
    out = np.zeros(1 << log_n, dtype=np.int64)
    lib().oc_sample_ternary(_bytes(key), tag, i0, i1, log_n, _i64(out))
    return out


def sample_gaussian(key, tag, i0, i1, log_n) -> np.ndarray:
    out = np.zeros(1 << log_n, dtype=np.int64)
    lib().oc_sample_gaussian(_bytes(key), tag, i0, i1, log_n, _i64(out))
    return out


def lift_centred(src: np.ndarray, src_mods, dst_mods) -> np.ndarray:
    src = np.ascontiguousarray(src, dtype=np.uint64)
    n = src.shape[-1]
    sm = np.array(src_mods, dtype=np.uint64)
    dm = np.array(dst_mods, dtype=np.uint64)
    out = np.zeros((len(dst_mods), n), dtype=np.uint64)
    lib().oc_lift_centred(_u64(src), _u64(sm), len(src_mods), _u64(dm), len(dst_mods), _u64(out), n)
    return out


def div_round(src: np.ndarray, q_mods, d_mods) -> np.ndarray:
    src = np.ascontiguousarray(src, dtype=np.uint64)
    n = src.shape[-1]
    m = np.array(list(q_mods) + list(d_mods), dtype=np.uint64)
    out = np.zeros((len(q_mods), n), dtype=np.uint64)
    lib().oc_div_round(_u64(src), _u64(m), len(q_mods), len(d_mods), _u64(out), n)
    return out


def div_t_exact(src: np.ndarray, q_mods, d_mods, t: int) -> np.ndarray:
    src = np.ascontiguousarray(src, dtype=np.uint64)
    n = src.shape[-1]
    m = np.array(list(q_mods) + list(d_mods), dtype=np.uint64)
    out = np.zeros((len(q_mods), n), dtype=np.uint64)
    lib().oc_div_t_exact(_u64(src), _u64(m), len(q_mods), len(d_mods), t, _u64(out), n)
    return out


def automorphism(a, g: int, q: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    out = np.zeros_like(x)
    lib().oc_automorphism(_u64(out), _u64(x), x.shape[-1], g, q)
    return out


def galois_elt(log_n: int, r: int) -> int:
    return int(lib().oc_galois_elt(log_n, r))


# ---------------------------------------------------------------- schemes

class Context:
    """An oracle parameter set: the prime chain and the per-prime NTT roots."""

    def __init__(self, scheme: int, log_n: int, q_bits, p_bits, dnum: int, t: int = 0,
                 log_n_max: int | None = None, nb: int = 0, b_bits: int = 60):
        L = lib()
        qb = (ctypes.c_int * len(q_bits))(*q_bits)
        pb = (ctypes.c_int * max(1, len(p_bits)))(*p_bits)
        self.scheme, self.log_n, self.n = scheme, log_n, 1 << log_n
        self.t = t
        self._h = L.oc_ctx_new(scheme, log_n, log_n_max if log_n_max else log_n, len(q_bits), qb,
                               len(p_bits), pb, dnum, t, nb, b_bits)
        if not self._h:
            raise RuntimeError("oracle: prime generation failed")
        counts = (ctypes.c_int * 5)()
        L.oc_ctx_moduli(self._h, None, None, None, counts)
        self.L, self.K, self.nb, self.alpha, self.beta = list(counts)
        q = np.zeros(self.L, dtype=np.uint64)
        p = np.zeros(max(1, self.K), dtype=np.uint64)
        b = np.zeros(max(1, self.nb), dtype=np.uint64)
        L.oc_ctx_moduli(self._h, _u64(q), _u64(p), _u64(b), counts)
        self.q = [int(x) for x in q]
        self.p = [int(x) for x in p[: self.K]]
        self.b = [int(x) for x in b[: self.nb]]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oc_ctx_free(self._h)
            self._h = None

    # -- keys
    def keygen(self, seed: bytes) -> "Keys":
        return Keys(self, seed)

    # -- ciphertexts are numpy uint64 arrays [2][level][N] in coefficient form
    def encrypt(self, keys: "Keys", msg, seed: bytes) -> np.ndarray:
        m = np.ascontiguousarray(np.asarray(msg, dtype=np.int64))
        assert m.shape == (self.n,)
        out = np.zeros((2, self.L, self.n), dtype=np.uint64)
        lib().oc_encrypt(self._h, keys._h, _i64(m), _bytes(seed), _u64(out))
        return out

    def ct_uniform(self, seed: bytes, index: int, level: int) -> np.ndarray:
        out = np.zeros((2, level, self.n), dtype=np.uint64)
        lib().oc_ct_uniform(self._h, _bytes(seed), index, level, _u64(out))
        return out

    def decrypt(self, keys: "Keys", ct: np.ndarray, factor: int = 1) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        out = np.zeros(self.n, dtype=np.int64)
        lib().oc_decrypt(self._h, keys._h, _u64(ct), ct.shape[1], factor, _i64(out))
        return out

    def add(self, a, b):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros_like(a)
        lib().oc_add(self._h, _u64(a), _u64(b), _u64(out), a.shape[1])
        return out

    def sub(self, a, b):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros_like(a)
        lib().oc_sub(self._h, _u64(a), _u64(b), _u64(out), a.shape[1])
        return out

    def mul_int(self, a, k: int):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.zeros_like(a)
        lib().oc_mul_int(self._h, _u64(a), int(k), _u64(out), a.shape[1])
        return out

    def add_const(self, a, k: int):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.zeros_like(a)
        lib().oc_add_const(self._h, _u64(a), int(k), _u64(out), a.shape[1])
        return out

    def drop(self, a, new_level: int):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.zeros((2, new_level, self.n), dtype=np.uint64)
        lib().oc_drop(self._h, _u64(a), a.shape[1], new_level, _u64(out))
        return out

    def mul_plain(self, a, pt):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        pt = np.ascontiguousarray(pt, dtype=np.int64)
        out = np.zeros_like(a)
        lib().oc_mul_plain(self._h, _u64(a), _i64(pt), _u64(out), a.shape[1])
        return out

    def tensor(self, a, b):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros((3, a.shape[1], self.n), dtype=np.uint64)
        lib().oc_tensor(self._h, _u64(a), _u64(b), _u64(out), a.shape[1])
        return out

    def keyswitch(self, keys: "Keys", c, key_id: int) -> np.ndarray:
        c = np.ascontiguousarray(c, dtype=np.uint64)
        level = c.shape[0]
        out = np.zeros((2, level, self.n), dtype=np.uint64)
        if lib().oc_keyswitch(self._h, keys._h, _u64(c), level, key_id, _u64(out)) != 0:
            raise KeyError(key_id)
        return out

    def mul_relin(self, keys: "Keys", a, b) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros_like(a)
        if lib().oc_mul_relin(self._h, keys._h, _u64(a), _u64(b), _u64(out), a.shape[1]) != 0:
            raise KeyError(0)
        return out

    def rescale(self, a) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        level = a.shape[1]
        out = np.zeros((2, level - 1, self.n), dtype=np.uint64)
        lib().oc_rescale(self._h, _u64(a), _u64(out), level)
        return out

    def rotate(self, keys: "Keys", a, g: int) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.zeros_like(a)
        if lib().oc_rotate(self._h, keys._h, _u64(a), _u64(out), a.shape[1], g) != 0:
            raise KeyError(g)
        return out

    def galois_elt(self, r: int) -> int:
        return galois_elt(self.log_n, r)

    def bgv_factor_after_rescale(self, factor: int, level: int) -> int:
        """Plaintext factor after switching from `level` to `level-1`."""
        q = self.q[level - 1]
        return factor * pow(q, -1, self.t) % self.t


class Keys:
    def __init__(self, ctx: Context, seed: bytes):
        self.ctx = ctx
        self._h = lib().oc_keygen(ctx._h, _bytes(seed))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oc_keys_free(self._h)
            self._h = None

    def gen_galois(self, g: int) -> None:
        if lib().oc_gen_galois(self.ctx._h, self._h, g) != 0:
            raise ValueError(g)

    def secret(self) -> np.ndarray:
        s = np.zeros(self.ctx.n, dtype=np.int64)
        lib().oc_keys_export(self.ctx._h, self._h, _i64(s), None)
        return s

    def public(self) -> np.ndarray:
        pk = np.zeros((2, self.ctx.L, self.ctx.n), dtype=np.uint64)
        lib().oc_keys_export(self.ctx._h, self._h, None, _u64(pk))
        return pk

    def ksk(self, key_id: int) -> np.ndarray:
        c = self.ctx
        out = np.zeros((c.beta, 2, c.L + c.K, c.n), dtype=np.uint64)
        if lib().oc_ksk_export(c._h, self._h, key_id, _u64(out)) != 0:
            raise KeyError(key_id)
        return out


# ---------------------------------------------------------------- CKKS encoding

def _slot_roots(n: int) -> np.ndarray:
    """zeta^(5^k mod 2N) for the N/2 slots, zeta = exp(i pi / N)."""
    two_n = 2 * n
    e = np.ones(n // 2, dtype=np.int64)
    for k in range(1, n // 2):
        e[k] = e[k - 1] * 5 % two_n
    return np.exp(1j * np.pi * e / n)


def encode_ckks(z, n: int, scale: float) -> np.ndarray:
    """Integer coefficients m with m(zeta_k) ~ scale z_k (canonical embedding),
    m_j = (2/N) Re(sum_k scale z_k zeta_k^(-j)), rounded half away from zero."""
    z = np.asarray(z, dtype=np.complex128)
    assert z.shape == (n // 2,)
    roots = _slot_roots(n)
    coeffs = np.zeros(n)
    j = np.arange(n)
    for k0 in range(0, n // 2, 512):
        r = roots[k0:k0 + 512]
        w = scale * z[k0:k0 + 512]
        coeffs += (2.0 / n) * np.real((w[:, None] * r[:, None] ** (-j[None, :])).sum(axis=0))
    return (np.sign(coeffs) * np.floor(np.abs(coeffs) + 0.5)).astype(np.int64)


def decode_ckks(m, n: int, scale: float) -> np.ndarray:
    """z_k = m(zeta_k) / scale."""
    m = np.asarray(m, dtype=np.float64)
    roots = _slot_roots(n)
    j = np.arange(n)
    out = np.zeros(n // 2, dtype=np.complex128)
    for k0 in range(0, n // 2, 512):
        r = roots[k0:k0 + 512]
        out[k0:k0 + 512] = (m[None, :] * r[:, None] ** j[None, :]).sum(axis=1)
    return out / scale
