"""Named parameter sets and seeded synthetic inputs.

This module holds no arithmetic of the method: only the parameter presets
(ring degree, prime bit sizes, digit count, plaintext modulus, batch shape)
and seeded generators of inputs (seeds, messages, uniform residues).  Both
the CUDA path and the CPU oracle take their inputs from here.

The presets follow the paper's parameter style (Sec. 5.1: N = 2^15, L = 16,
log Q = 881 for its operator tables) at the sizes this library is measured
on:

  ckks_n12      CKKS, N = 2^12, 3 x 40-bit q, 1 x 40-bit p, dnum = 3
  ckks_n16      CKKS, N = 2^16, 24 x 50-bit q, 4 x 60-bit p, dnum = 3,
                batch of 8 ciphertext pairs (the headline workload)
  ckks_n16_k8   the same chain with 8 x 60-bit special primes, so that
                key-switching noise stays below the scale (decryption checks)
  bfv_n14       BFV, N = 2^14, t = 65537, 8 x 55-bit q, 1 x 60-bit p,
                dnum = 8, auxiliary basis of 60-bit primes, batch 16
  bgv_n14       BGV with the same chain, batch 16

Prime chains for N up to 2^16 use q = 1 mod 2^17 so that one chain serves
every ring degree of the uneven mix.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

CKKS, BFV, BGV = 0, 1, 2


@dataclass(frozen=True)
class Preset:
    name: str
    scheme: int
    log_n: int
    q_bits: tuple
    p_bits: tuple
    dnum: int
    t: int = 0
    log_n_max: int = 0
    batch: int = 1
    log_scale: float = 0.0
    b_bits: int = 60
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def L(self) -> int:
        return len(self.q_bits)

    @property
    def K(self) -> int:
        return len(self.p_bits)


PRESETS = {
    "ckks_n12": Preset("ckks_n12", CKKS, 12, (40,) * 3, (40,), 3, log_n_max=12, batch=1,
                       log_scale=40.0),
    "ckks_n16": Preset("ckks_n16", CKKS, 16, (50,) * 24, (60,) * 4, 3, log_n_max=16, batch=8,
                       log_scale=50.0),
    "ckks_n16_k8": Preset("ckks_n16_k8", CKKS, 16, (50,) * 24, (60,) * 8, 3, log_n_max=16,
                          batch=8, log_scale=50.0),
    "bfv_n14": Preset("bfv_n14", BFV, 14, (55,) * 8, (60,), 8, t=65537, log_n_max=14, batch=16),
    "bgv_n14": Preset("bgv_n14", BGV, 14, (55,) * 8, (60,), 8, t=65537, log_n_max=14, batch=16),
}


def seed_for(name: str) -> bytes:
    """32-byte seed derived from a name (SHA-256), so inputs are reproducible."""
    return hashlib.sha256(name.encode()).digest()


def rng_for(name: str) -> np.random.Generator:
    return np.random.default_rng(int.from_bytes(seed_for(name)[:8], "little"))


def int_messages(rng: np.random.Generator, n: int, t: int) -> np.ndarray:
    """Messages uniform mod t (BFV / BGV), one per coefficient."""
    return rng.integers(0, t, size=n, dtype=np.int64)


def complex_slots(rng: np.random.Generator, n: int) -> np.ndarray:
    """N/2 complex slots with real and imaginary parts uniform in [-1, 1]."""
    return rng.uniform(-1, 1, n // 2) + 1j * rng.uniform(-1, 1, n // 2)


def uniform_residues(rng: np.random.Generator, mods, shape_prefix, n: int) -> np.ndarray:
    """Residues uniform in [0, m_i) for every limb i: shape prefix + (len(mods), n)."""
    mods = [int(m) for m in mods]
    out = np.empty(tuple(shape_prefix) + (len(mods), n), dtype=np.uint64)
    for i, m in enumerate(mods):
        out[..., i, :] = rng.integers(0, m, size=tuple(shape_prefix) + (n,), dtype=np.uint64)
    return out
