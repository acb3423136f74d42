"""NTT schedules, the schedule tuner, and uneven batches (many operations of
different ring degrees and levels in one submission, run over concurrent
lanes and replayed from a captured CUDA graph): every result must equal the
single-operation results (which the parity tests tie to the oracle)."""
import numpy as np
import pytest

import oracle
from paper_2503_22227_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402


@pytest.mark.parametrize("log_n", [12, 13, 14, 15, 16])
def test_every_ntt_schedule_matches_oracle(log_n):
    p = W.Preset("sched", W.CKKS, log_n, (50, 58, 61), (60,), 1, log_n_max=16)
    ctx = api.Context(p)
    _, count, _ = ctx.ntt_schedule()
    assert count >= 1
    rng = np.random.default_rng(100 + log_n)
    host = W.uniform_residues(rng, ctx.q, (1,), ctx.n)
    want = [oracle.ntt(host[0, i], log_n, q, oracle.min_psi(q, log_n)) for i, q in enumerate(ctx.q)]
    for k in range(count):
        ctx.set_ntt_schedule(k)
        dev = torch.from_numpy(host.view(np.int64).copy()).cuda()
        ctx.ntt(dev)
        got = dev.cpu().numpy().view(np.uint64)
        for i in range(ctx.L):
            assert np.array_equal(got[0, i], want[i]), (k, i)
        ctx.ntt(dev, inverse=True)
        assert np.array_equal(dev.cpu().numpy().view(np.uint64), host), k
    # one choice per launch size class: tuning the small class leaves the
    # large one as it was
    ctx.set_ntt_schedule(count - 1)
    chosen, times = ctx.tune_ntt(3 * 8)
    assert 0 <= chosen < count and len(times) == count and all(t > 0 for t in times)
    assert ctx.ntt_schedule(24)[0] == chosen
    assert ctx.ntt_schedule(3 * 200)[0] == count - 1
    big, _ = ctx.tune_ntt(3 * 100)
    assert ctx.ntt_schedule(300)[0] == big and ctx.ntt_schedule(24)[0] == chosen


def test_every_ntt_schedule_gives_the_same_key_switching():
    """At N = 2^16 every schedule (row passes of one or several tiles per
    CTA) must give the same HMult+relin+rescale and HRotate limbs as the
    default one, which the parity tests tie to the oracle: this runs the
    unreduced and the combine row passes of each schedule."""
    p = W.PRESETS["ckks_n16"]
    ctx = api.Context(p)
    keys = ctx.keygen(W.seed_for("sched-ks-keys"))
    g = ctx.galois_elt(3)
    keys.gen_galois(g)
    seed = W.seed_for("sched-ks-inputs")
    level = 6
    a = torch.cat([ctx.ct_uniform(seed, 2 * i, level) for i in range(4)])
    b = torch.cat([ctx.ct_uniform(seed, 2 * i + 1, level) for i in range(4)])
    _, count, _ = ctx.ntt_schedule()
    ctx.set_ntt_schedule(0)
    want_m = ctx.mul_relin_rescale(keys, a, b).clone()
    want_r = ctx.rotate(keys, a, g).clone()
    for k in range(1, count):
        ctx.set_ntt_schedule(k)
        assert torch.equal(ctx.mul_relin_rescale(keys, a, b), want_m), k
        assert torch.equal(ctx.rotate(keys, a, g), want_r), k
    ctx.set_ntt_schedule(0)


def _ctx(preset, rots):
    ctx = api.Context(preset)
    keys = ctx.keygen(W.seed_for("batch-keys-" + preset.name))
    gs = [ctx.galois_elt(r) for r in rots]
    for g in gs:
        keys.gen_galois(g)
    return ctx, keys, gs


def test_uneven_batch_and_graph_equal_single_ops():
    c12, k12, g12 = _ctx(W.PRESETS["ckks_n12"], (1, 3))
    c13, k13, g13 = _ctx(W.Preset("ckks_n13", W.CKKS, 13, (45,) * 6, (50, 50), 3, log_n_max=13),
                         (1, 5))
    rng = np.random.default_rng(7)
    jobs = []  # (kind, ctx, keys, level, count, galois)
    for i in range(14):
        ctx, keys, gs = (c12, k12, g12) if i % 2 == 0 else (c13, k13, g13)
        level = int(rng.integers(2, ctx.L + 1))
        kind = [api.OP_MUL_RELIN, api.OP_MUL_RELIN_RESCALE, api.OP_ROTATE, api.OP_RESCALE][i % 4]
        count = int(rng.integers(1, 3))
        jobs.append((kind, ctx, keys, level, count, gs[i % 2]))
    ops, outs, wants = [], [], []
    for j, (kind, ctx, keys, level, count, g) in enumerate(jobs):
        a = torch.cat([ctx.ct_uniform(W.seed_for("batch-in"), 2 * (8 * j + c), level)
                       for c in range(count)])
        b = torch.cat([ctx.ct_uniform(W.seed_for("batch-in"), 2 * (8 * j + c) + 1, level)
                       for c in range(count)])
        if kind == api.OP_MUL_RELIN:
            want = ctx.mul_relin(keys, a, b)
        elif kind == api.OP_MUL_RELIN_RESCALE:
            want = ctx.mul_relin_rescale(keys, a, b)
        elif kind == api.OP_ROTATE:
            want = ctx.rotate(keys, a, g)
        else:
            want = ctx.rescale(a)
        out = torch.zeros_like(want)
        ops.append(api.make_op(kind, ctx, a, out, keys=keys, b=b, galois_elt=g))
        outs.append(out)
        wants.append(want.clone())
        # keep inputs alive for the graph replays
        outs[-1]._keep = (a, b)
    api.run_batch(ops, lanes=4)
    torch.cuda.synchronize()
    for j, (o, w) in enumerate(zip(outs, wants)):
        assert torch.equal(o, w), j
    graph = api.Graph(ops, lanes=4)
    assert graph.nodes > len(ops)
    for o in outs:
        o.zero_()
    for _ in range(2):
        graph.launch()
    torch.cuda.synchronize()
    for j, (o, w) in enumerate(zip(outs, wants)):
        assert torch.equal(o, w), j


def test_batch_rejects_bad_entries():
    ctx, keys, gs = _ctx(W.PRESETS["ckks_n12"], (1,))
    a = ctx.ct_uniform(W.seed_for("bad"), 0, 1)
    out = torch.zeros_like(a)
    with pytest.raises(api.CatfheError) as e:
        api.run_batch([api.make_op(api.OP_RESCALE, ctx, a, out)], lanes=1)
    assert e.value.code in (-1, -2)   # rescale at level 1
    a3 = ctx.ct_uniform(W.seed_for("bad"), 1, 3)
    out3 = torch.zeros_like(a3)
    with pytest.raises(api.CatfheError) as e:
        api.run_batch([api.make_op(api.OP_ROTATE, ctx, a3, out3, keys=keys,
                                   galois_elt=ctx.galois_elt(9))], lanes=1)
    assert e.value.code in (-1, -3)   # missing Galois key


def test_compatible_entries_are_merged_and_exact():
    """Single-ciphertext HMult+relin(+rescale) and HRotate entries of the same
    context, keys, level (and Galois element) are gathered into one batched
    operation by the batch planner; every output must equal the single call,
    eager and from a captured graph, whatever the lane count."""
    ctx, keys, gs = _ctx(W.PRESETS["ckks_n12"], (1, 3))
    ctx2, keys2, gs2 = _ctx(W.Preset("ckks_n13", W.CKKS, 13, (45,) * 6, (50, 50), 3, log_n_max=13),
                            (1,))
    seed = W.seed_for("merge-in")
    jobs = []
    for j in range(11):
        jobs.append((api.OP_MUL_RELIN_RESCALE, ctx, keys, 3, gs[0]))
    for j in range(5):
        jobs.append((api.OP_MUL_RELIN, ctx, keys, 2, gs[0]))
    for j in range(7):
        jobs.append((api.OP_ROTATE, ctx, keys, 3, gs[j % 2]))
    for j in range(6):
        jobs.append((api.OP_MUL_RELIN_RESCALE, ctx2, keys2, 4, gs2[0]))
    ops, outs, wants, keep = [], [], [], []
    for j, (kind, c, k, level, g) in enumerate(jobs):
        a = c.ct_uniform(seed, 2 * j, level)
        b = c.ct_uniform(seed, 2 * j + 1, level)
        if kind == api.OP_MUL_RELIN:
            want = c.mul_relin(k, a, b)
        elif kind == api.OP_MUL_RELIN_RESCALE:
            want = c.mul_relin_rescale(k, a, b)
        else:
            want = c.rotate(k, a, g)
        out = torch.full_like(want, -1)
        ops.append(api.make_op(kind, c, a, out, keys=k, b=b, galois_elt=g))
        outs.append(out)
        wants.append(want.clone())
        keep.append((a, b))
    for lanes in (1, 2, 5):
        for o in outs:
            o.fill_(-1)
        api.run_batch(ops, lanes=lanes)
        torch.cuda.synchronize()
        for j, (o, w) in enumerate(zip(outs, wants)):
            assert torch.equal(o, w), (lanes, j)
    graph = api.Graph(ops, lanes=3)
    for o in outs:
        o.fill_(-1)
    graph.launch()
    torch.cuda.synchronize()
    for j, (o, w) in enumerate(zip(outs, wants)):
        assert torch.equal(o, w), ("graph", j)


@pytest.mark.slow
def test_uneven_mix_full_sizes_sampled():
    """The uneven mix at its real sizes (N from 2^13 to 2^16 on one prime
    chain, levels 2..24, HMult+relin / HRotate / rescale, tuned NTT schedules,
    one captured graph over 8 lanes), 48 operations: every output equals the
    single call, two N = 2^13 key-switching outputs and every rescale entry
    (all four ring degrees) equal the oracle."""
    base = W.PRESETS["ckks_n16"]
    rng = W.rng_for("mix-test")
    ctxs = {}
    for log_n in (13, 14, 15, 16):
        pr = W.Preset(f"mix_n{log_n}", W.CKKS, log_n, base.q_bits, base.p_bits, base.dnum,
                      log_n_max=16)
        c = api.Context(pr)
        k = c.keygen(W.seed_for(f"mix-keys-{log_n}"))
        gs = [c.galois_elt(r) for r in (1, 7)]
        for g in gs:
            k.gen_galois(g)
        c.tune_ntt(2 * c.L * 2)
        ctxs[log_n] = (pr, c, k, gs)
    kinds = [api.OP_MUL_RELIN, api.OP_ROTATE, api.OP_RESCALE]
    seed = W.seed_for("mix-test-inputs")
    ops, outs, wants, meta = [], [], [], []
    for i in range(48):
        log_n = int(rng.choice([13, 14, 15, 16]))
        level = int(rng.integers(2, 25))
        kind = kinds[i % 3]
        pr, c, k, gs = ctxs[log_n]
        g = gs[i % 2]
        a = c.ct_uniform(seed, 2 * i, level)
        b = c.ct_uniform(seed, 2 * i + 1, level)
        if kind == api.OP_MUL_RELIN:
            want = c.mul_relin(k, a, b)
        elif kind == api.OP_ROTATE:
            want = c.rotate(k, a, g)
        else:
            want = c.rescale(a)
        out = torch.full_like(want, -1)
        ops.append(api.make_op(kind, c, a, out, keys=k, b=b, galois_elt=g))
        outs.append(out)
        wants.append(want.clone())
        meta.append((log_n, level, kind, i, g, a, b))
    graph = api.Graph(ops, lanes=8)
    graph.launch()
    torch.cuda.synchronize()
    for j, (o, w) in enumerate(zip(outs, wants)):
        assert torch.equal(o, w), j
    checked = 0
    for (log_n, level, kind, i, g, a, b), o in zip(meta, outs):
        if log_n != 13 or kind == api.OP_RESCALE or checked >= 2:
            continue
        pr, c, k, gs = ctxs[13]
        oc = oracle.Context(pr.scheme, pr.log_n, pr.q_bits, pr.p_bits, pr.dnum, log_n_max=16)
        ok = oc.keygen(W.seed_for("mix-keys-13"))
        oa, ob = oc.ct_uniform(seed, 2 * i, level), oc.ct_uniform(seed, 2 * i + 1, level)
        if kind == api.OP_MUL_RELIN:
            want = oc.mul_relin(ok, oa, ob)
        else:
            ok.gen_galois(g)
            want = oc.rotate(ok, oa, g)
        assert np.array_equal(c.export_ct(o)[0], want), (kind, level)
        checked += 1
    assert checked == 2
    # every rescale entry against the oracle's round(c / q_{l-1})
    octxs, seen = {}, set()
    for (log_n, level, kind, i, g, a, b), o in zip(meta, outs):
        if kind != api.OP_RESCALE:
            continue
        pr, c, k, gs = ctxs[log_n]
        if log_n not in octxs:
            octxs[log_n] = oracle.Context(pr.scheme, pr.log_n, pr.q_bits, pr.p_bits, pr.dnum,
                                          log_n_max=16)
        oc = octxs[log_n]
        want = oc.rescale(oc.ct_uniform(seed, 2 * i, level))
        assert np.array_equal(c.export_ct(o)[0], want), (log_n, level)
        seen.add(log_n)
    assert seen == {13, 14, 15, 16}
