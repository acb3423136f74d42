"""The bit-packed transfer form's host codec (catfhe_pack_host /
catfhe_unpack_host, no GPU needed): residue k of a limb with field width b
occupies bits [k b, (k+1) b) of the limb's little-endian bit stream.  The
words are checked against that definition written with Python integers."""
import ctypes

import numpy as np
import pytest

from paper_2503_22227_gb300 import api

vp = ctypes.c_void_p


def _pack(bits, limbs, log_n):
    polys, level, n = limbs.shape
    words = polys * sum(n * int(b) // 64 for b in bits)
    out = np.empty(words, dtype=np.uint64)
    b = np.asarray(bits, dtype=np.uint8)
    rc = api.load().catfhe_pack_host(b.ctypes.data_as(vp), level, polys, log_n,
                                     np.ascontiguousarray(limbs).ctypes.data_as(vp),
                                     out.ctypes.data_as(vp))
    return rc, out


def _unpack(bits, packed, polys, log_n):
    level, n = len(bits), 1 << log_n
    out = np.empty((polys, level, n), dtype=np.uint64)
    b = np.asarray(bits, dtype=np.uint8)
    rc = api.load().catfhe_unpack_host(b.ctypes.data_as(vp), level, polys, log_n,
                                       packed.ctypes.data_as(vp), out.ctypes.data_as(vp))
    return rc, out


def _reference_words(bits, limbs):
    """The definition: per limb, the integer sum_k v_k 2^(k b), cut into
    64-bit words, limbs one after another."""
    words = []
    for poly in limbs:
        for b, limb in zip(bits, poly):
            stream = 0
            for k, v in enumerate(limb):
                stream |= (int(v) & ((1 << b) - 1)) << (k * b)
            for w in range(len(limb) * b // 64):
                words.append((stream >> (64 * w)) & (2 ** 64 - 1))
    return np.array(words, dtype=np.uint64)


@pytest.mark.parametrize("log_n", [6, 7])
def test_layout_matches_the_definition(log_n):
    rng = np.random.default_rng(5 + log_n)
    bits = [50, 61, 20, 33, 64, 1]
    n = 1 << log_n
    limbs = np.stack([np.stack([rng.integers(0, 2 ** 63, n, dtype=np.uint64) * 2 +
                                rng.integers(0, 2, n, dtype=np.uint64) for _ in bits])
                      for _ in range(2)])
    rc, packed = _pack(bits, limbs, log_n)
    assert rc == 0
    assert np.array_equal(packed, _reference_words(bits, limbs))
    rc, back = _unpack(bits, packed, 2, log_n)
    assert rc == 0
    masks = np.array([(1 << b) - 1 if b < 64 else 2 ** 64 - 1 for b in bits], dtype=np.uint64)
    assert np.array_equal(back, limbs & masks[None, :, None])


def test_round_trip_of_residues_at_size():
    """Residues below 2^b survive unchanged; the stream is b/64 of the words."""
    rng = np.random.default_rng(11)
    log_n, bits = 12, [50] * 24
    n = 1 << log_n
    limbs = rng.integers(0, 2 ** 50, (4, 24, n), dtype=np.uint64)
    rc, packed = _pack(bits, limbs, log_n)
    assert rc == 0 and packed.size == 4 * 24 * n * 50 // 64
    rc, back = _unpack(bits, packed, 4, log_n)
    assert rc == 0 and np.array_equal(back, limbs)


def test_bad_arguments_are_rejected():
    limbs = np.zeros((1, 1, 64), dtype=np.uint64)
    for bits, log_n in (([0], 6), ([65], 6), ([50], 5), ([50], 21)):
        b = np.asarray(bits, dtype=np.uint8)
        out = np.empty(64, dtype=np.uint64)
        rc = api.load().catfhe_pack_host(b.ctypes.data_as(vp), 1, 1, log_n,
                                         limbs.ctypes.data_as(vp), out.ctypes.data_as(vp))
        assert rc == -1, (bits, log_n)
    b = np.asarray([50], dtype=np.uint8)
    assert api.load().catfhe_pack_host(b.ctypes.data_as(vp), 1, 1, 6, None, None) == -1
    assert api.load().catfhe_pack_host(b.ctypes.data_as(vp), 1, 0, 6, None, None) == 0
