"""Host-side logic of the serving workload, without a device: the circuit
builder (Chebyshev baby-step/giant-step evaluation against numpy's own
Chebyshev series, levels, scales, stage schedule, buffer release), the
committed sign polynomial, Poisson arrivals, and the continuous-batching
scheduler with HBM admission driven by a simulated device."""
import types

import numpy as np
import pytest

from paper_2503_22227_gb300 import circuit as C
from paper_2503_22227_gb300 import serving as S
from paper_2503_22227_gb300.data import make_sign_poly

PRIMES = [(1 << 50) - 27 - 2 * i * 131072 for i in range(24)]   # ~2^50, for scale tracking only


def _ctx(L=24, log_n=16):
    return types.SimpleNamespace(q=PRIMES[:L], n=1 << log_n, L=L, galois_elt=lambda r: 2 * r + 1)


def test_sign_coefficients_are_the_committed_interpolant():
    c = S.sign_coefficients()
    assert np.array_equal(c, make_sign_poly.coefficients())
    assert np.all(c[0::2] == 0.0)
    x = np.linspace(-1, 1, 2001)
    approx = np.polynomial.chebyshev.chebval(x, c)
    # analytic in the Bernstein ellipse up to the poles of tanh at +-i pi / 16:
    # error ~ rho^-64, rho = a + sqrt(a^2 + 1), a = pi / 16, i.e. ~4e-6
    assert np.max(np.abs(approx - np.tanh(8 * x))) < 1e-5


@pytest.mark.parametrize("deg", [1, 2, 5, 7, 8, 13, 31, 63])
def test_chebyshev_circuit_equals_series(deg):
    rng = np.random.default_rng(deg)
    coeffs = rng.uniform(-1, 1, deg + 1) / (1 + np.arange(deg + 1))
    z = rng.uniform(-1, 1, 512)
    want = np.polynomial.chebyshev.chebval(z, coeffs)
    # every modulus equal to the scale: all scales stay exactly 2^50, and the
    # only error is the integer constants round(c q) / q (~2^-50 each)
    c = C.Circuit([1 << 50] * 24, 2.0 ** 50, 16)
    x = c.input("x", 24)
    c.output("p", c.chebyshev(x, coeffs))
    got = c.evaluate_float({"x": z})["p"].real
    assert np.max(np.abs(got - want)) < 1e-12
    depth = 24 - c.level(c.outputs["p"])
    assert depth <= int(np.ceil(np.log2(deg + 1))) + 1
    # moduli spread by ~6e-9 relative: sums of terms whose scales differ by
    # that much, the error stays of that order
    c2 = C.Circuit(PRIMES, 2.0 ** 50, 16)
    x2 = c2.input("x", 24)
    c2.output("p", c2.chebyshev(x2, coeffs))
    got2 = c2.evaluate_float({"x": z})["p"].real
    assert np.max(np.abs(got2 - want)) < 1e-6


def test_pdq_circuit_levels_scales_and_answer():
    ctx = _ctx()
    coeffs = S.sign_coefficients()
    c = C.pdq_circuit(ctx, 2.0 ** 50, coeffs, sum_slots=1024)
    out = c.nodes[c.outputs["sum"]]
    assert out.level >= 2
    assert abs(out.scale / 2.0 ** 50 - 1) < 1e-4
    counts = c.counts()
    assert counts["rotate"] == 10 and counts["input"] == 4
    for nd in c.nodes:
        if nd.kind in ("mul", "rescale"):
            assert c.nodes[nd.args[0]].level >= 2
        if nd.kind in ("add", "sub", "mul"):
            assert c.level(nd.args[0]) == c.level(nd.args[1])
            if nd.kind != "mul":
                assert abs(c.nodes[nd.args[0]].scale / c.nodes[nd.args[1]].scale - 1) < 1e-3
    rng = np.random.default_rng(5)
    half = ctx.n // 2
    x = np.zeros(half)
    y = np.zeros(half)
    x[:1000], y[:1000] = rng.random(1000), rng.random(1000)
    lo, hi = 0.3, 0.7
    vals = {"x": x, "y": y, "lo": np.full(half, lo), "hi": np.full(half, hi)}
    got = c.evaluate_float(vals)
    p = lambda t: np.polynomial.chebyshev.chebval(t, coeffs)
    want = np.sum((1 + p(x - lo)) * (1 + p(hi - x)) / 4 * y)
    assert abs(got["sum"][0].real - want) < 1e-4 * abs(want)     # scale spread of the moduli
    ctx_eq = types.SimpleNamespace(q=[1 << 50] * 24, n=ctx.n, L=24, galois_elt=ctx.galois_elt)
    exact = C.pdq_circuit(ctx_eq, 2.0 ** 50, coeffs).evaluate_float(vals)
    assert abs(exact["sum"][0].real - want) < 1e-9
    # the soft predicate approaches the hard one
    hard = np.sum(y[(x >= lo) & (x <= hi)])
    assert abs(want - hard) < 0.1 * hard


def test_schedule_releases_every_intermediate_once():
    ctx = _ctx()
    c = C.pdq_circuit(ctx, 2.0 ** 50, S.sign_coefficients())
    sch = C.schedule(c)
    seen = set()
    produced_at = {}
    for k, st in enumerate(sch.stages):
        for i, kind, args, level, arg in st:
            for a in args:
                assert a in c.inputs.values() or (a in produced_at and produced_at[a] < k)
                assert a not in seen, "argument released before its last use"
            produced_at[i] = k
        seen.update(sch.release[k])
    keep = set(c.outputs.values()) | set(c.inputs.values())
    assert seen == set(produced_at) - keep
    assert C.schedule(c) is sch


def test_poisson_arrivals_and_percentiles():
    t = S.poisson_arrivals(50.0, 20000, np.random.default_rng(1))
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 0.02) < 0.001
    assert abs(np.std(gaps) - 0.02) < 0.001               # exponential: std = mean
    st = S.latency_stats(np.arange(1, 101) / 1000.0)
    assert st["p50_ms"] == pytest.approx(50.5) and st["p99_ms"] == pytest.approx(99.01)


class FakeEngine:
    """A simulated device: each batch takes `cost(entries)` seconds after the
    previous one ends; the clock only moves when the loop waits or idles."""

    def __init__(self, stages=5, need=100, cost=lambda n: 0.001 * (1 + n)):
        self.now = 0.0
        self.stages, self.need_b, self.cost = stages, need, cost
        self.device_end = 0.0
        self.batches = []
        self.active_ids = set()
        self.max_active_seen = 0
        self.results = {}
        self.retired = []

    def clock(self):
        return self.now

    def idle(self, s):
        self.now += s

    def need(self, req):
        return self.need_b

    def start(self, req):
        req.state = {"pos": 0, "acc": req.id}
        self.active_ids.add(req.id)
        self.max_active_seen = max(self.max_active_seen, len(self.active_ids))

    def stage(self, reqs):
        entries = []
        for r in reqs:
            entries.append((r.id, r.state["pos"]))
            r.state["acc"] = (r.state["acc"] * 31 + r.state["pos"]) % 1000003
            r.state["pos"] += 1
        return entries

    def submit(self, entries):
        self.batches.append(entries)
        self.device_end = max(self.device_end, self.now) + self.cost(len(entries))
        self.now += 1e-5                                    # host time to enqueue

    def is_done(self, req):
        return req.state["pos"] >= self.stages

    def finish(self, req):
        self.results[req.id] = req.state["acc"]
        self.active_ids.discard(req.id)
        req.state = None

    def mark(self):
        return self.device_end

    def retire(self, req):
        self.retired.append(req.id)

    def ready(self, token):
        return self.now >= token

    def wait(self, token):
        self.now = max(self.now, token)


def _reqs(times):
    return [S.Request(id=i, arrival=float(t)) for i, t in enumerate(times)]


def test_serve_completes_all_and_batches_continuously():
    eng = FakeEngine(stages=6)
    times = S.poisson_arrivals(400.0, 200, np.random.default_rng(3))
    reqs = _reqs(times)
    st = S.serve(reqs, eng, budget_bytes=10 ** 9, max_active=16, clock=eng.clock, idle=eng.idle)
    assert st.served == 200
    assert all(r.finished >= r.admitted >= r.arrival for r in reqs)
    assert all(r.latency >= 6 * 0.001 for r in reqs)
    assert st.admitted_while_busy > 0 and st.max_active > 1
    assert eng.max_active_seen <= 16
    # some batch mixes requests at different stage positions (continuous batching)
    assert any(len({pos for _, pos in b}) > 1 for b in eng.batches)
    # every request ran each of its stages exactly once, in order
    seen = {}
    for b in eng.batches:
        for rid, pos in b:
            assert seen.get(rid, -1) == pos - 1
            seen[rid] = pos
    assert all(seen[r.id] == 5 for r in reqs)
    assert sorted(eng.retired) == list(range(200))
    # the result does not depend on the mix
    alone = _reqs(times)
    for r in alone:
        e1 = FakeEngine(stages=6)
        r.arrival = 0.0
        S.serve([r], e1, budget_bytes=10 ** 9, clock=e1.clock, idle=e1.idle)
        assert e1.results[r.id] == eng.results[r.id]


def test_oldest_first_batches_are_bounded_and_exact():
    """max_batch = 3: no tick carries more than 3 requests, each tick takes
    the oldest active ones, and every result equals the unbounded run's."""
    arr = np.linspace(0, 0.004, 12)
    eng = FakeEngine(stages=5)
    st = S.serve(_reqs(arr), eng, budget_bytes=10 ** 9, max_active=16, clock=eng.clock,
                 idle=eng.idle, max_batch=3)
    assert st.served == 12 and len(eng.results) == 12
    assert all(len(b) <= 3 for b in eng.batches)
    for b in eng.batches:
        ids = [i for i, _ in b]
        assert ids == sorted(ids)
    ref = FakeEngine(stages=5)
    S.serve(_reqs(arr), ref, budget_bytes=10 ** 9, max_active=16, clock=ref.clock, idle=ref.idle)
    assert eng.results == ref.results


def test_admission_respects_budget_and_slots():
    eng = FakeEngine(stages=4, need=300)
    reqs = _reqs(np.zeros(20))
    st = S.serve(reqs, eng, budget_bytes=1000, max_active=8, clock=eng.clock, idle=eng.idle)
    assert st.served == 20
    assert eng.max_active_seen == 3 and st.max_active == 3       # 3 x 300 <= 1000 < 4 x 300
    assert st.peak_reserved == 900
    order = sorted(reqs, key=lambda r: r.admitted)
    assert [r.id for r in order] == list(range(20))                # first come, first admitted
    eng2 = FakeEngine(stages=4, need=10)
    st2 = S.serve(_reqs(np.zeros(20)), eng2, budget_bytes=1000, max_active=5, clock=eng2.clock,
                  idle=eng2.idle)
    assert eng2.max_active_seen == 5 and st2.max_active == 5


def test_request_above_budget_is_refused():
    eng = FakeEngine(need=2000)
    with pytest.raises(ValueError):
        S.serve(_reqs([0.0]), eng, budget_bytes=1000, clock=eng.clock, idle=eng.idle)


def test_idle_gaps_do_not_count_as_latency():
    eng = FakeEngine(stages=3, cost=lambda n: 0.001)
    reqs = _reqs([0.0, 10.0])
    st = S.serve(reqs, eng, budget_bytes=10 ** 9, clock=eng.clock, idle=eng.idle)
    assert reqs[1].admitted >= 10.0
    assert all(r.latency < 0.05 for r in reqs)
    assert st.latency["max_ms"] < 50


# ----------------------------------------------------------------------------
# The GPU engine's memory, with a fake allocator of real sizes that recycles
# an address as soon as its buffer is dropped (as a caching allocator may).

class _Alloc:
    def __init__(self):
        self.free, self.next, self.live = {}, 1 << 20, {}

    def take(self, size):
        spare = self.free.get(size)
        if spare:
            addr = spare.pop()
        else:
            addr = self.next
            self.next += (size + 4095) // 4096 * 4096
        self.live[addr] = size
        return addr

    def give(self, addr):
        size = self.live.pop(addr)
        self.free.setdefault(size, []).append(addr)

    def holds(self, lo, hi):
        import bisect
        bases = sorted(self.live)
        k = bisect.bisect_right(bases, lo) - 1
        return k >= 0 and hi <= bases[k] + self.live[bases[k]]


class _Buf:
    def __init__(self, alloc, shape=None, nbytes=None):
        import weakref
        self.shape = shape
        self.nbytes = nbytes if nbytes is not None else 8 * int(np.prod(shape))
        self._p = alloc.take(self.nbytes)
        weakref.finalize(self, alloc.give, self._p)

    def data_ptr(self):
        return self._p

    def numel(self):
        return self.nbytes

    # the views a runner takes of its arena for its results
    def narrow(self, dim, start, length):
        return self

    def view(self, *shape):
        if shape and all(isinstance(d, int) for d in shape):
            return types.SimpleNamespace(shape=shape, data_ptr=self.data_ptr)
        return self


def _fake_table(alloc, batches):
    import bisect
    import ctypes
    from paper_2503_22227_gb300 import api as real_api

    ctx = _ctx()
    ctx._h = ctypes.c_void_p(1)
    ctx.empty_ct = lambda count, level: _Buf(alloc, (count, 2, level, ctx.n))
    ctx.import_ct = lambda host, form: _Buf(alloc, (1, 2, ctx.L, ctx.n))
    ctx.export_into = lambda ct, host, form: host
    keys = types.SimpleNamespace(_h=ctypes.c_void_p(2))

    def span(ptr, count, level):
        return ptr, ptr + count * 2 * level * ctx.n * 8

    def run_batch(entries, lanes, ws):
        outs = sorted(span(e.out, e.count, e.level_out) for e in entries)
        ins = [span(e.a, e.count, e.level) for e in entries]
        ins += [span(e.b, e.count, e.level) for e in entries if e.b]
        for (a0, a1), (b0, b1) in zip(outs, outs[1:]):
            assert a1 <= b0, "two outputs of one batch share memory"
        starts = [o[0] for o in outs]
        for lo, hi in ins:
            k = bisect.bisect_left(starts, hi) - 1
            assert k < 0 or outs[k][1] <= lo, "an output overwrites an input of the same batch"
        for lo, hi in ins + outs:
            assert alloc.holds(lo, hi), "a batch touches memory that is not allocated"
        batches.append(len(entries))

    class _Batch:
        def __init__(self, entries):
            self.entries = entries

        def workspace_bytes(self, lanes):
            return 1

        def run(self, lanes, ws):
            run_batch(self.entries, lanes, ws)

    fake_api = types.SimpleNamespace(
        FORM_NATIVE=real_api.FORM_NATIVE, FORM_ASYNC=real_api.FORM_ASYNC, Batch=_Batch)

    class _Event:
        def record(self):
            pass

        def query(self):
            return True

        def synchronize(self):
            pass

    class _Host:
        def clone(self):
            return self

    def empty(*a, **k):
        if k.get("pin_memory"):
            return _Host()
        return _Buf(alloc, nbytes=int(a[0]))

    fake_torch = types.SimpleNamespace(uint8=None, int64=None, empty=empty,
                                       cuda=types.SimpleNamespace(Event=_Event))
    t = S.Table.__new__(S.Table)
    t.api, t.torch, t.ctx, t.keys = fake_api, fake_torch, ctx, keys
    t.circuit = C.pdq_circuit(ctx, 2.0 ** 50, S.sign_coefficients())
    t.columns = [_Buf(alloc, (1, 2, ctx.L, ctx.n)) for _ in range(S.COLS)]
    t.uploads = [(None, None)] * 4
    t.arena_bytes = C.memory_plan(t.circuit).size
    t.ct_bytes = 2 * ctx.L * ctx.n * 8
    t.need = t.arena_bytes + 2 * t.ct_bytes
    return t


def test_memory_plan_keeps_every_stage_disjoint():
    """In every stage the buffers live then (written in it, read in it or
    later) occupy disjoint bytes of the arena, within its size, which is at
    least the circuit's peak of live bytes and not far above it."""
    c = C.pdq_circuit(_ctx(), 2.0 ** 50, S.sign_coefficients())
    plan = C.memory_plan(c)
    assert set(plan.offsets) == {i for st in c.stages() for i in st}
    for st in c.stages():
        s = c.nodes[st[0]].stage
        spans = sorted((plan.offsets[i], plan.offsets[i] + plan.sizes[i])
                       for i in plan.offsets if plan.live[i][0] <= s <= plan.live[i][1])
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0, s
        assert spans[-1][1] <= plan.size
        # every argument read in this stage is live in it
        for i in st:
            for a in c.nodes[i].args:
                if a in plan.live:
                    assert plan.live[a][0] < s <= plan.live[a][1]
    assert c.peak_bytes() <= plan.size <= 1.1 * c.peak_bytes()


def test_gpu_engine_batches_touch_only_their_own_live_memory():
    alloc, batches = _Alloc(), []
    table = _fake_table(alloc, batches)
    eng = S.GpuEngine(table, lanes=4)
    reqs = [S.Request(id=i, arrival=0.002 * i, col_a=i % 4, col_b=(i + 1) % 4, bounds=i % 4)
            for i in range(12)]
    clock = iter(np.arange(0, 1e3, 1e-4))
    st = S.serve(reqs, eng, budget_bytes=5 * table.need, max_active=5,
                 clock=lambda: next(clock), idle=lambda s: None)
    assert st.served == 12 and max(batches) > 45
    assert all(r.result is not None for r in reqs)
    del reqs, eng
    # every request's arena and uploads went back: only the table columns stay
    assert len(alloc.live) == S.COLS
