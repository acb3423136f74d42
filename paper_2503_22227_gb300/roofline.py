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
    limb_ntts: float        # number of length-N transforms (a share, for hoisted work)
    coeff_products: float   # products counted per coefficient (times N)
    n: int

    @property
    def butterflies(self) -> float:
        return self.limb_ntts * (self.n // 2) * int(math.log2(self.n))

    @property
    def modmuls(self) -> float:
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


def ckks_mul_relin(n: int, level: int, K: int, alpha: int) -> Work:
    """CKKS HMult + relinearise without the rescale: the tensor, then the same
    key switching as a rotation (ModDown divides by P alone)."""
    w = ckks_rotate(n, level, K, alpha)
    return Work(w.limb_ntts, w.coeff_products + 4 * level, n)


def ckks_rotate(n: int, level: int, K: int, alpha: int) -> Work:
    M = level + K
    ds = digits(level, alpha)
    ntt = level + sum(M - a for a in ds) + 2 * K + 2 * level
    prod = sum(a + a * (M - a) for a in ds) + 2 * len(ds) * M
    prod += 2 * (K + K * level) + 2 * level
    return Work(ntt, prod, n)


def ckks_rotate_hoisted(n: int, level: int, K: int, alpha: int, rotations: int) -> Work:
    """One of `rotations` hoisted rotations of a ciphertext: the INTT, ModUp
    and NTT of c1 are shared by all of them; each rotation permutes (in NTT
    form, no products), runs the inner product and ModDown."""
    M = level + K
    ds = digits(level, alpha)
    shared_ntt = level + sum(M - a for a in ds)
    shared_prod = sum(a + a * (M - a) for a in ds)
    ntt = 2 * K + 2 * level
    prod = 2 * len(ds) * M + 2 * (K + K * level) + 2 * level
    # each rotation's share of the hoisted part (a fraction of a transform)
    return Work(ntt + shared_ntt / rotations, prod + shared_prod / rotations, n)


def bgv_mul_relin(n: int, level: int, K: int, alpha: int) -> Work:
    """BGV HMult + relinearise (no modulus switch): tensor in NTT form, then
    key switching of d2 with the t-preserving ModDown."""
    r = ckks_rotate(n, level, K, alpha)
    return Work(r.limb_ntts, r.coeff_products + 4 * level, n)


def bfv_mul_relin(n: int, level: int, K: int, alpha: int, nb: int) -> Work:
    """BFV HMult + relinearise: lift the four input polynomials from Q to
    the auxiliary basis B (nb primes), NTT over Q u B, tensor, INTT, exact
    round(t x / Q) back to Q (a conversion Q -> B, then B -> Q), then key
    switching of d2 in coefficient form (ModUp transforms every digit
    position, ModDown's combine works in coefficient form)."""
    kb = level + nb
    M = level + K
    ds = digits(level, alpha)
    ntt = 4 * kb + 3 * kb                         # NTT of the lifted inputs, INTT of the tensor
    ntt += len(ds) * M                            # NTT of every digit position
    ntt += 2 * M                                  # INTT of the inner product
    prod = 4 * (level + level * nb)               # lift Q -> B of the 4 polynomials
    prod += 4 * kb                                # tensor over Q u B
    prod += 3 * 2 * (level + level * nb)          # scale-and-round: Q -> B, then B -> Q
    prod += sum(a + a * (M - a) for a in ds)      # ModUp conversions
    prod += 2 * len(ds) * M                       # inner product
    prod += 2 * (K + K * level) + 2 * level       # ModDown conversion and combine
    return Work(ntt, prod, n)


def bytes_keyswitch(n: int, level: int, L: int, inputs: int, out_level: int, K: int,
                    alpha: int, batch: int, inputs_shared: int = 1) -> float:
    """Minimum HBM bytes per operation of a key-switching operation in a
    batch of `batch`: `inputs` ciphertexts at `level` read once (shared by
    `inputs_shared` operations, as hoisted rotations share their input), the
    output at `out_level` written once, the key read once per batch."""
    beta_l = len(digits(L, alpha))
    key = beta_l * 2 * (L + K) * n * 8
    return (inputs * 2 * level * n * 8 / inputs_shared + 2 * out_level * n * 8
            + key / batch)


# Issue bound of the integer pipes: 152 SMs x 4 warp schedulers x one warp
# instruction per cycle.  The instruction counts per operation are ncu's
# counts (smsp__inst_executed) for the register-resident loops of
# catfhe_measure_int_peak on GB300: the fully reduced Shoup product, the
# forward butterfly with a conditional subtraction and the wide one.
SMS = 152
INSTR_PER_MODMUL = 19.1
INSTR_PER_BUTTERFLY = 23.2
INSTR_PER_BUTTERFLY_WIDE = 17.2


# The integer multiply pipe (ncu: fmaheavy) is the one the arithmetic fills:
# a 32-bit low product occupies it 2 cycles per warp instruction, a high or
# widening product 4 (catfhe_measure_imad_rates, and ncu's pipe counters on
# those loops).  ncu puts the wide-butterfly loop of catfhe_measure_int_peak
# at this fraction of the pipe's cycles, so its rate divided by this is the
# rate of that butterfly with the pipe busy on every cycle.
LOOP_MUL_PIPE_BUSY = 0.954


def issue_bounds(sm_mhz: float) -> dict:
    """Operations per second if the loops issued an instruction on every
    scheduler cycle at `sm_mhz`."""
    thread_instr = SMS * 4 * 32 * sm_mhz * 1e6
    return {"sm_mhz": sm_mhz, "thread_instr_per_s": thread_instr,
            "modmul_per_s": thread_instr / INSTR_PER_MODMUL,
            "butterfly_per_s": thread_instr / INSTR_PER_BUTTERFLY,
            "butterfly_wide_per_s": thread_instr / INSTR_PER_BUTTERFLY_WIDE}


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
