"""The algorithmic counts behind the benchmark's roofline (CPU only)."""
from paper_2503_22227_gb300 import roofline as R


def test_config2_counts():
    w = R.ckks_mul_relin_rescale(1 << 16, 24, 4, 8)
    assert w.limb_ntts == 140
    assert w.coeff_products == 1054
    assert abs(w.modmuls - 1.42e8) / 1.42e8 < 0.01
    r = R.ckks_rotate(1 << 16, 24, 4, 8)
    assert r.limb_ntts == 140
    assert abs(r.modmuls - 1.34e8) / 1.34e8 < 0.01


def test_small_config_counts():
    w = R.ckks_mul_relin_rescale(1 << 12, 3, 1, 1)
    assert w.limb_ntts == 3 + 3 * 3 + 4 + 4 == 20
    assert R.digits(5, 2) == [2, 2, 1]


def test_bytes():
    b = R.bytes_mul_relin_rescale(1 << 16, 24, 24, 4, 8, 8)
    mib = b / 2 ** 20
    assert 80 < mib < 83   # 48 in + 23 out + 84/8 key
    assert R.ntt_bytes(1 << 16, 1) == 2 ** 20
