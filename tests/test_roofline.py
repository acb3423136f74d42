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


def test_secondary_counts():
    """The integer-scheme and hoisted-rotation counts at N = 2^14, L = 8,
    K = 1, dnum = 8 (alpha = 1) and N = 2^16, L = 24, K = 4, alpha = 8."""
    n = 1 << 14
    bgv = R.bgv_mul_relin(n, 8, 1, 1)
    # INTT of d2, 8 digits x 8 lifted limbs, INTT of 2 P limbs, NTT of 2 x 8
    assert bgv.limb_ntts == 8 + 64 + 2 + 16
    assert bgv.coeff_products == 32 + 72 + 144 + 18 + 16
    bfv = R.bfv_mul_relin(n, 8, 1, 1, 8)
    assert bfv.limb_ntts == 64 + 48 + 72 + 18
    assert bfv.coeff_products == 4 * 72 + 64 + 3 * 144 + 72 + 144 + 18 + 16
    # one hoisted rotation alone is a plain rotation
    one = R.ckks_rotate_hoisted(1 << 16, 24, 4, 8, 1)
    rot = R.ckks_rotate(1 << 16, 24, 4, 8)
    assert one.limb_ntts == rot.limb_ntts and one.coeff_products == rot.coeff_products
    # 16 rotations share the INTT + ModUp + NTT (84 transforms, 504 N products)
    h = R.ckks_rotate_hoisted(1 << 16, 24, 4, 8, 16)
    assert abs(h.limb_ntts - (56 + 84 / 16)) < 1e-9
    assert abs(h.coeff_products - (416 + 504 / 16)) < 1e-9


def test_mul_relin_without_rescale_counts():
    """HMult + relinearise alone at N = 2^16, L = 24, K = 4, alpha = 8: INTT of
    d2 (24), 3 digits x 20 lifted limbs (60), INTT of the 4 P limbs of both
    polynomials (8), NTT of their lift to the 24 q limbs (48); products: the
    tensor (96), ModUp 3 x (8 + 8 x 20) = 504, the key inner product
    2 x 3 x 28 = 168, ModDown 2 x (4 + 4 x 24) = 200 and the final 2 x 24."""
    w = R.ckks_mul_relin(1 << 16, 24, 4, 8)
    assert w.limb_ntts == 24 + 60 + 8 + 48
    assert w.coeff_products == 96 + 504 + 168 + 200 + 48


def test_keyswitch_bytes_and_issue_bounds():
    n = 1 << 16
    # a rotation reads one ciphertext, writes one, and shares the key over 8
    b = R.bytes_keyswitch(n, 24, 24, 1, 24, 4, 8, 8)
    assert b == 2 * 24 * n * 8 + 2 * 24 * n * 8 + 3 * 2 * 28 * n * 8 / 8
    assert R.bytes_keyswitch(n, 24, 24, 2, 23, 4, 8, 8) == R.bytes_mul_relin_rescale(n, 24, 24, 4, 8, 8)
    ib = R.issue_bounds(2000.0)
    assert abs(ib["thread_instr_per_s"] - 152 * 4 * 32 * 2e9) < 1
    assert ib["butterfly_wide_per_s"] > ib["modmul_per_s"] > ib["butterfly_per_s"]
