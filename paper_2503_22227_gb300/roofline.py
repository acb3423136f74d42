"""Algorithmic work of the hot-path operations, for roofline accounting.

Counts are the algorithmic ones (what the operation has to do), not what a
kernel happens to execute:

* a limb-NTT of size N is (N/2) log2 N butterflies, one modular product each;
* an exact base conversion of one coefficient from k source primes to T
  target primes costs k + k*T products (one per source, one per source and
  target);
* the tensor costs 4 products per coefficient and limb, the key-switching
  inner product 2 per digit, extended limb and coefficient, the ModDown
  combine 1 per output limb and coefficient of each of the two polynomials.

Bytes are the minimum HBM traffic: every input ciphertext read once, every
output written once, and the evaluation key read once per batch (shared by
the batch).
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass
class Work:
    limb_ntts: int          # number of length-N transforms
    coeff_products: int     # products counted per coefficient (times N)
    n: int

    @property
    def butterflies(self) -> int:
        return self.limb_ntts * (self.n // 2) * int(math.log2(self.n))

    @property
    def modmuls(self) -> int:
        return self.butterflies + self.coeff_products * self.n


def digits(level: int, alpha: int) -> list[int]:
    """Sizes of the key-switching digits at `level`."""
    out, i = [], 0
    while i < level:
        out.append(min(alpha, level - i))
        i += alpha
    return out


def ckks_mul_relin_rescale(n: int, level: int, K: int, alpha: int) -> Work:
    """CKKS HMult + relinearise + rescale, ModDown fused with the rescale."""
    M = level + K
    ds = digits(level, alpha)
    ntt = level                                   # INTT of d2
    ntt += sum(M - a for a in ds)                 # NTT of the lifted digits
    ntt += 2 * (K + 1) + 2 * (level - 1)          # ModDown+rescale: INTT, NTT
    prod = 4 * level                              # tensor
    prod += sum(a + a * (M - a) for a in ds)      # ModUp conversions
    prod += 2 * len(ds) * M                       # inner product with the key
    prod += 2 * ((K + 1) + (K + 1) * (level - 1)) # ModDown conversion
    prod += 2 * (level - 1)                       # final (y - lift) * D^-1
    return Work(ntt, prod, n)


def ckks_rotate(n: int, level: int, K: int, alpha: int) -> Work:
    M = level + K
    ds = digits(level, alpha)
    ntt = level + sum(M - a for a in ds) + 2 * K + 2 * level
    prod = sum(a + a * (M - a) for a in ds) + 2 * len(ds) * M
    prod += 2 * (K + K * level) + 2 * level
    return Work(ntt, prod, n)


def bytes_mul_relin_rescale(n: int, level: int, L: int, K: int, alpha: int, batch: int) -> float:
    """Minimum HBM bytes per operation in a batch of `batch`."""
    beta_l = len(digits(L, alpha))
    inputs = 2 * 2 * level * n * 8
    output = 2 * (level - 1) * n * 8
    key = beta_l * 2 * (L + K) * n * 8
    return inputs + output + key / batch


def ntt_bytes(n: int, limbs: int) -> int:
    """A transform reads and writes each limb once at minimum."""
    return 2 * 8 * n * limbs
