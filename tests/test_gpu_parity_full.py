"""Bit-exact parity with the CPU oracle at the full sizes of the remaining
configurations, in the launch configurations the benchmark and the serving
loop use:

- the noise-valid N = 2^16 chain (24 x 50-bit q, K = 8 x 60-bit p, dnum = 3)
  that the private-query serving loop runs on: a batched HMult+relin+rescale
  (its ModDown+rescale divides by 9 primes at once) and HRotate(1);
- the standalone CKKS rescale at N = 2^16, level 24 (Table 1 "rescale");
- the BGV modulus switch at N = 2^14, 8 x 55-bit q, t = 65537, batch 16.

The oracle's full-size operations take seconds each; they run on threads
(the oracle's C calls release the interpreter lock and share no mutable
state), one per sampled output.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2503_22227_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402


def _octx(p: W.Preset):
    return oracle.Context(p.scheme, p.log_n, p.q_bits, p.p_bits, p.dnum, t=p.t,
                          log_n_max=p.log_n_max or p.log_n, b_bits=p.b_bits)


def _run_all(jobs):
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        return list(ex.map(lambda f: f(), jobs))


@pytest.mark.slow
def test_ckks_n16_k8_chain_matches_oracle():
    """K = 8: a batch of 8 uniform pairs at level 24 through one fused
    HMult+relin+rescale launch (two halves of 4 on two streams, as in the
    serving loop's batched ticks) and HRotate(1) on the batch; the first and
    last ciphertexts limb for limb against the oracle's HMult+relin, then
    rescale, and its rotation."""
    p = W.PRESETS["ckks_n16_k8"]
    g_ctx, o_ctx = api.Context(p), _octx(p)
    seed_k = W.seed_for("k8-parity-keys")
    gk = g_ctx.keygen(seed_k)
    g = g_ctx.galois_elt(1)
    gk.gen_galois(g)
    seed = W.seed_for("k8-parity-inputs")
    a = torch.cat([g_ctx.ct_uniform(seed, 2 * i, p.L) for i in range(8)])
    b = torch.cat([g_ctx.ct_uniform(seed, 2 * i + 1, p.L) for i in range(8)])
    got = g_ctx.export_ct(g_ctx.mul_relin_rescale(gk, a, b))
    rot = g_ctx.export_ct(g_ctx.rotate(gk, a, g))
    assert got.shape == (8, 2, p.L - 1, p.n)
    ok = o_ctx.keygen(seed_k)
    ok.gen_galois(g)
    ins = {i: (o_ctx.ct_uniform(seed, 2 * i, p.L), o_ctx.ct_uniform(seed, 2 * i + 1, p.L))
           for i in (0, 7)}
    jobs = []
    for i in (0, 7):
        oa, ob = ins[i]
        jobs.append(lambda oa=oa, ob=ob: o_ctx.rescale(o_ctx.mul_relin(ok, oa, ob)))
        jobs.append(lambda oa=oa: o_ctx.rotate(ok, oa, g))
    want = _run_all(jobs)
    for j, i in enumerate((0, 7)):
        assert np.array_equal(got[i], want[2 * j]), ("mul_relin_rescale", i)
        assert np.array_equal(rot[i], want[2 * j + 1]), ("rotate", i)


@pytest.mark.slow
def test_ckks_n16_rescale_matches_oracle():
    """Standalone rescale of the benchmark's 8 input ciphertexts (N = 2^16,
    level 24 -> 23): first, middle and last against the oracle's
    round(c / q_23)."""
    p = W.PRESETS["ckks_n16"]
    g_ctx, o_ctx = api.Context(p), _octx(p)
    seed = W.seed_for("bench-inputs")
    a = torch.cat([g_ctx.ct_uniform(seed, 2 * i, p.L) for i in range(8)])
    got = g_ctx.export_ct(g_ctx.rescale(a))
    picks = (0, 3, 7)
    want = _run_all([lambda i=i: o_ctx.rescale(o_ctx.ct_uniform(seed, 2 * i, p.L))
                     for i in picks])
    for i, w in zip(picks, want):
        assert np.array_equal(got[i], w), i
    # and again from level 23 (a different last prime and target count)
    a2 = a[:, :, :p.L - 1].contiguous()
    got2 = g_ctx.export_ct(g_ctx.rescale(a2))
    o_in = o_ctx.ct_uniform(seed, 0, p.L)[:, :p.L - 1]
    assert np.array_equal(got2[0], o_ctx.rescale(o_in))


def test_bgv_n14_modswitch_matches_oracle():
    """BGV modulus switch (c - t [c t^-1]_q) / q on the benchmark's batch of
    16 (N = 2^14, level 8 -> 7): first and last against the oracle; then the
    decryption invariant on a real encryption: the plaintext becomes
    m q_7^-1 mod t, which the factor passed to decrypt undoes."""
    p = W.PRESETS["bgv_n14"]
    g_ctx, o_ctx = api.Context(p), _octx(p)
    seed = W.seed_for("bench-inputs-bgv_n14")
    x = torch.cat([g_ctx.ct_uniform(seed, 2 * i, p.L) for i in range(p.batch)])
    got = g_ctx.export_ct(g_ctx.rescale(x))
    for i in (0, p.batch - 1):
        assert np.array_equal(got[i], o_ctx.rescale(o_ctx.ct_uniform(seed, 2 * i, p.L))), i
    keys_seed = W.seed_for("bgv-modswitch-keys")
    gk, ok = g_ctx.keygen(keys_seed), o_ctx.keygen(keys_seed)
    m = W.int_messages(W.rng_for("bgv-modswitch-msg"), p.n, p.t)
    es = W.seed_for("bgv-modswitch-enc")
    ct = g_ctx.encrypt(gk, m, es)
    sw = g_ctx.rescale(ct)
    o_sw = o_ctx.rescale(o_ctx.encrypt(ok, m, es))
    assert np.array_equal(g_ctx.export_ct(sw)[0], o_sw)
    factor = o_ctx.bgv_factor_after_rescale(1, p.L)
    assert np.array_equal(o_ctx.decrypt(ok, o_sw, factor), m)
