"""CKKS canonical-embedding encoder and decoder (host side, numpy FFT).

Slot k of a plaintext polynomial m is its value at zeta^(5^k mod 2N),
zeta = exp(i pi / N), k = 0 .. N/2-1 (the paper's Table 1 "encode" /
"decode" operators; the GPU path works on the encoded integers).  With
omega = zeta^2, m(zeta^(2j+1)) = sum_i (m_i zeta^i) omega^(j i), so all N
evaluations are one length-N DFT of the twisted coefficients; encoding
places the scaled slots and their conjugates at the matching j and inverts
that DFT.  Coefficients are rounded half away from zero.
"""
from __future__ import annotations

import numpy as np


def _slot_index(n: int) -> tuple[np.ndarray, np.ndarray]:
    """DFT index j of slot k (root zeta^(5^k)) and of its conjugate."""
    two_n = 2 * n
    e = np.empty(n // 2, dtype=np.int64)
    v = 1
    for k in range(n // 2):
        e[k] = v
        v = v * 5 % two_n
    j = (e - 1) // 2
    jc = (two_n - e - 1) // 2
    return j, jc


_cache: dict[int, tuple] = {}


def _tables(n: int):
    t = _cache.get(n)
    if t is None:
        j, jc = _slot_index(n)
        twist = np.exp(1j * np.pi * np.arange(n) / n)   # zeta^i
        t = (j, jc, twist)
        _cache[n] = t
    return t


def encode(z, n: int, scale: float) -> np.ndarray:
    """Slots z (N/2 complex) -> int64 coefficients of m with m(zeta_k) ~ scale z_k."""
    z = np.asarray(z, dtype=np.complex128)
    assert z.shape == (n // 2,)
    j, jc, twist = _tables(n)
    E = np.zeros(n, dtype=np.complex128)
    E[j] = scale * z
    E[jc] = np.conj(scale * z)
    # E_j = sum_i (m_i zeta^i) omega^(j i)  =>  m_i zeta^i = IDFT(E)_i (numpy's
    # forward FFT uses omega^-1, so the evaluation is n * ifft)
    m = np.real(np.fft.fft(E) / n * np.conj(twist))
    return (np.sign(m) * np.floor(np.abs(m) + 0.5)).astype(np.int64)


def decode(m, n: int, scale: float) -> np.ndarray:
    """int coefficients -> slots m(zeta_k) / scale."""
    m = np.asarray(m, dtype=np.float64)
    j, _, twist = _tables(n)
    E = np.fft.ifft(m * twist) * n
    return E[j] / scale


def encode_constant(c: float, scale: float) -> int:
    """The constant vector c encodes to the constant polynomial round(c scale)."""
    v = c * scale
    return int(np.sign(v) * np.floor(abs(v) + 0.5))
