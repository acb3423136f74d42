"""The FFT-based CKKS encoder against the oracle's direct O(N^2) canonical
embedding (CPU)."""
import numpy as np

import oracle
from paper_2503_22227_gb300 import encoding, workloads as W


def test_encoder_matches_oracle_embedding():
    n, scale = 1 << 11, 2.0 ** 40
    rng = W.rng_for("encoder")
    z = W.complex_slots(rng, n)
    fast = encoding.encode(z, n, scale)
    slow = oracle.encode_ckks(z, n, scale)
    assert np.max(np.abs(fast - slow)) <= 1      # both round m, float order differs
    assert np.mean(fast == slow) > 0.98        # a rounding tie-break differs rarely
    assert np.max(np.abs(encoding.decode(fast, n, scale) - oracle.decode_ckks(fast, n, scale))) < 1e-9
    assert np.max(np.abs(encoding.decode(fast, n, scale) - z)) < 1e-9


def test_encoder_constant_and_rotation():
    n, scale = 1 << 10, 2.0 ** 30
    m = encoding.encode(np.full(n // 2, -0.625, dtype=complex), n, scale)
    assert m[0] == encoding.encode_constant(-0.625, scale) and not m[1:].any()
    rng = np.random.default_rng(3)
    z = W.complex_slots(rng, n)
    m = encoding.encode(z, n, scale)
    rot = np.zeros(n, dtype=np.int64)
    for i in range(n):          # X -> X^5 rotates slots left by one
        k = 5 * i % (2 * n)
        if k < n:
            rot[k] = m[i]
        else:
            rot[k - n] = -m[i]
    assert np.max(np.abs(encoding.decode(rot, n, scale) - np.roll(z, -1))) < 1e-7
