"""Private-query serving: continuous batching of encrypted range-predicate
sums over a resident encrypted table (the paper's PDQ setting, Sec. 4: the
client uploads ciphertexts, the server keeps its data and keys in GPU
memory for the lifetime of the queries and returns encrypted results).

Each request carries two encrypted bounds lo, hi and names two table
columns a, b; the answer is the encrypted sum over the rows of
mask(a) * b, mask = (1 + p(u)) (1 + p(v)) / 4, u = kappa (a - lo),
v = kappa (hi - a), p a degree-63 odd Chebyshev interpolant of tanh(8x)
standing in for the sign (the paper's comparison method is only cited),
followed by log2(1024) rotate-and-add steps.

Serving loop (`serve`): requests arrive over time; at every tick the loop
retires finished GPU work, admits arrived requests in order while both the
slot limit and the device-memory budget allow (each request reserves its
circuit's peak of live ciphertexts plus its uploaded inputs), then submits
the next circuit stage of EVERY active request as one uneven batch.  A
request admitted while others are half-way through joins the very next
batch (continuous batching); its operations run on the device beside
theirs.  Up to `depth` ticks are in flight, so the host builds tick k+1
while the device runs tick k.  A request's latency runs from its arrival
to the completion of the copy of its result into host memory.

The scheduling logic takes an `engine` (the GPU engine `GpuEngine`, or a
host-only stand-in in the tests), so admission and batching are testable
without a device.
"""
from __future__ import annotations

import os
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import workloads as W

ROWS, COLS, SUM_SLOTS = 1000, 4, 1024


def sign_coefficients() -> np.ndarray:
    """Chebyshev coefficients c_0 .. c_63 of the committed sign approximation."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "sign_cheb63.txt")
    vals = [float(x) for x in open(path) if x.strip() and not x.startswith("#")]
    assert len(vals) == 64
    return np.array(vals)


def poisson_arrivals(rate: float, count: int, rng: np.random.Generator) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of `rate` per second."""
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def latency_stats(lat_s) -> dict:
    lat = np.asarray(lat_s, dtype=np.float64) * 1e3
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "max_ms": None}
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}


# --------------------------------------------------------------------------- requests
@dataclass
class Request:
    id: int
    arrival: float                   # seconds after the start of serving
    col_a: int = 0
    col_b: int = 1
    bounds: int = 0                  # index of the client's uploaded bound pair
    admitted: float = -1.0
    finished: float = -1.0
    need: int = 0                    # reserved device bytes
    state: object = None             # engine state while active
    result: object = None            # host copy of the encrypted answer

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    served: int
    wall_s: float
    throughput: float                # requests / (last completion - first arrival)
    latency: dict
    max_active: int
    mean_active: float
    ticks: int
    peak_reserved: int
    admitted_while_busy: int         # requests that joined a batch already running


class Admission:
    """Device-memory budget and slot limit for active requests."""

    def __init__(self, budget_bytes: int, max_active: int):
        self.budget, self.max_active = int(budget_bytes), int(max_active)
        self.reserved, self.active, self.peak = 0, 0, 0

    def fits(self, need: int) -> bool:
        return self.active < self.max_active and self.reserved + need <= self.budget

    def take(self, need: int) -> None:
        assert self.fits(need)
        self.reserved += need
        self.active += 1
        self.peak = max(self.peak, self.reserved)

    def give(self, need: int) -> None:
        self.reserved -= need
        self.active -= 1
        assert self.reserved >= 0 and self.active >= 0


def serve(requests: list, engine, budget_bytes: int, max_active: int = 64, depth: int = 2,
          clock=time.perf_counter, idle=None, max_batch: int | None = None) -> ServeStats:
    """Runs `requests` (sorted by arrival) to completion; see the module text.

    max_batch: at most this many active requests advance per tick, the
    oldest first (None: every active request advances every tick).

    engine protocol:
      need(req) -> bytes          device memory the request reserves
      start(req)                  upload its inputs, set req.state
      stage(reqs) -> list         build the next stage's entries of each
      submit(entries)             enqueue them as one batch (non-blocking) and move
                                  each request past that stage
      is_done(req) -> bool        no stage left
      finish(req)                 enqueue the copy of the result to the host, drop buffers
      mark() -> token             a marker after everything enqueued so far
      ready(token) -> bool, wait(token)
      retire(req)                 its result has reached the host
    """
    reqs = sorted(requests, key=lambda r: r.arrival)
    for r in reqs:
        if engine.need(r) > budget_bytes:
            raise ValueError(f"request {r.id} needs {engine.need(r)} bytes, above the "
                             f"budget of {budget_bytes}")
    adm = Admission(budget_bytes, max_active)
    pending = deque(reqs)
    active: list = []
    inflight: deque = deque()        # (token, requests that finish with it)
    t0 = clock()
    ticks, act_sum, max_act, joined = 0, 0, 0, 0

    def retire(token, done):
        now = clock() - t0
        for r in done:
            r.finished = now
            engine.retire(r)
            adm.give(r.need)

    while pending or active or inflight:
        while inflight and engine.ready(inflight[0][0]):
            retire(*inflight.popleft())
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            r = pending[0]
            r.need = engine.need(r)
            if not adm.fits(r.need):
                break
            pending.popleft()
            adm.take(r.need)
            r.admitted = now
            if active:
                joined += 1
            engine.start(r)
            active.append(r)
        if not active:
            if inflight:
                token, done = inflight.popleft()
                engine.wait(token)
                retire(token, done)
            elif pending:
                wait_s = pending[0].arrival - (clock() - t0)
                if wait_s > 0:
                    (idle or time.sleep)(min(wait_s, 0.01))
            continue
        if len(inflight) >= depth:
            token, done = inflight.popleft()
            engine.wait(token)
            retire(token, done)
            continue
        batch = active if max_batch is None else active[:max_batch]
        engine.submit(engine.stage(batch))
        ticks += 1
        act_sum += len(active)
        max_act = max(max_act, len(active))
        done = [r for r in batch if engine.is_done(r)]
        if done:
            active = [r for r in active if not engine.is_done(r)]
        for r in done:
            engine.finish(r)
        inflight.append((engine.mark(), done))
    wall = clock() - t0
    lat = [r.latency for r in reqs]
    span = max((r.finished for r in reqs), default=0.0) - min((r.arrival for r in reqs), default=0.0)
    return ServeStats(served=len(reqs), wall_s=wall,
                      throughput=len(reqs) / span if span > 0 else 0.0,
                      latency=latency_stats(lat), max_active=max_act,
                      mean_active=act_sum / max(1, ticks), ticks=ticks,
                      peak_reserved=adm.peak, admitted_while_busy=joined)


# --------------------------------------------------------------------------- GPU side
class Table:
    """The server's resident state: context, keys (relinearisation and the
    rotations 1, 2, 4, ..., 512), the encrypted columns, the query circuit,
    and the clients' uploaded bound pairs (pinned host ciphertexts)."""

    def __init__(self, preset: W.Preset = W.PRESETS["ckks_n16_k8"], bound_pairs: int = 8,
                 kappa: float = 1.0, seed: str = "pdq"):
        from . import api, circuit, encoding
        import torch
        self.api, self.torch, self.encoding = api, torch, encoding
        self.ctx = ctx = api.Context(preset)
        self.delta = 2.0 ** preset.log_scale
        self.keys = ctx.keygen(W.seed_for(seed + "-keys"))
        self.galois = {}
        r = 1
        while r < SUM_SLOTS:
            g = ctx.galois_elt(r)
            self.keys.gen_galois(g)
            self.galois[r] = g
            r *= 2
        rng = W.rng_for(seed + "-table")
        self.values = rng.random((COLS, ROWS))                   # uniform in [0, 1)
        self.slots = np.zeros((COLS, ctx.n // 2))
        self.slots[:, :ROWS] = self.values
        self.columns = [ctx.encrypt(self.keys, encoding.encode(self.slots[c], ctx.n, self.delta),
                                    W.seed_for(f"{seed}-col{c}")) for c in range(COLS)]
        self.ones_slots = np.zeros(ctx.n // 2)
        self.ones_slots[:ROWS] = 1.0
        self.ones = ctx.encrypt(self.keys, encoding.encode(self.ones_slots, ctx.n, self.delta),
                                W.seed_for(f"{seed}-ones"))
        self.seed = seed
        self.circuit = circuit.pdq_circuit(ctx, self.delta, sign_coefficients(), kappa=kappa,
                                           sum_slots=SUM_SLOTS, galois=self.galois)
        brng = W.rng_for(seed + "-bounds")
        self.bounds = []
        self.uploads = []
        for i in range(bound_pairs):
            lo, hi = np.sort(brng.random(2))
            self.bounds.append((float(lo), float(hi)))
            pair = []
            for j, v in enumerate((lo, hi)):
                m = np.zeros(ctx.n, dtype=np.int64)
                m[0] = encoding.encode_constant(float(v), self.delta)
                ct = ctx.encrypt(self.keys, m, W.seed_for(f"{seed}-bound{i}-{j}"))
                host = torch.empty(tuple(ct.shape), dtype=torch.int64, pin_memory=True)
                ctx.export_into(ct, host, api.FORM_NATIVE)
                pair.append(host)
            self.uploads.append(pair)
        torch.cuda.synchronize()
        self.ct_bytes = 2 * ctx.L * ctx.n * 8
        # one arena per request for the circuit's intermediates, plus the two
        # uploaded bounds
        self.arena_bytes = circuit.memory_plan(self.circuit).size
        self.need = self.arena_bytes + 2 * self.ct_bytes

    def avg_circuit(self):
        if getattr(self, "_avg_circuit", None) is None:
            from . import circuit
            self._avg_circuit = circuit.pdq_circuit(self.ctx, self.delta, sign_coefficients(),
                                                    sum_slots=SUM_SLOTS, galois=self.galois,
                                                    with_count=True)
        return self._avg_circuit

    def float_answer(self, col_a: int, col_b: int, bounds: int) -> float:
        """The float64 evaluation of the same circuit (same integer constants
        and scales) on the plaintext slots; slot 0 holds the sum."""
        lo, hi = self.bounds[bounds]
        lo_v = self.encoding.encode_constant(lo, self.delta) / self.delta
        hi_v = self.encoding.encode_constant(hi, self.delta) / self.delta
        half = self.ctx.n // 2
        out = self.circuit.evaluate_float({"x": self.slots[col_a], "y": self.slots[col_b],
                                           "lo": np.full(half, lo_v), "hi": np.full(half, hi_v)})
        return float(out["sum"][0].real)

    def float_avg_parts(self, col_a: int, col_b: int, bounds: int) -> tuple:
        """(sum, count) of the search-and-average circuit evaluated in float64
        with the same integer constants and scales."""
        lo, hi = self.bounds[bounds]
        lo_v = self.encoding.encode_constant(lo, self.delta) / self.delta
        hi_v = self.encoding.encode_constant(hi, self.delta) / self.delta
        half = self.ctx.n // 2
        out = self.avg_circuit().evaluate_float(
            {"x": self.slots[col_a], "y": self.slots[col_b], "ones": self.ones_slots,
             "lo": np.full(half, lo_v), "hi": np.full(half, hi_v)})
        return float(out["sum"][0].real), float(out["count"][0].real)

    def decrypt_answer(self, result_host) -> float:
        """Client side: decrypt and decode slot 0 of a host result."""
        ct = self.ctx.import_ct(result_host, self.api.FORM_NATIVE)
        m = self.ctx.decrypt(self.keys, ct)
        scale = self.circuit.nodes[self.circuit.outputs["sum"]].scale
        return float(self.encoding.decode(m, self.ctx.n, scale)[0].real)


class GpuEngine:
    """Runs requests' circuit stages as uneven batches over `lanes` streams.
    Uploads and result copies are asynchronous (page-locked host buffers,
    stream-ordered), so no tick waits for the host; result buffers come from
    a pool and return to it when the request retires.  Each request's
    intermediates live in one device arena laid out by the circuit's memory
    plan, and its batch entries are built once when it starts (a tick
    concatenates them), so the host does no allocation and no marshalling
    per operation."""

    def __init__(self, table: Table, lanes: int = 8, keep_results: bool = True,
                 profile: bool = False):
        from . import circuit
        self.t = table
        self.api, self.torch = table.api, table.torch
        self.circuit_mod = circuit
        self.lanes = lanes
        self.keep = keep_results
        self.ws = None
        self.staged: list = []
        self.free_hosts: list = []
        self.profile = profile
        self.reset_profile()

    def reset_profile(self) -> None:
        self.host_stage_s = self.host_submit_s = 0.0
        self.n_ops = self.n_ticks = 0
        self.tick_events: list = []

    def device_busy_s(self) -> float:
        """Sum over profiled ticks of the device time from the start to the
        end of each batch (synchronises)."""
        self.torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in self.tick_events) * 1e-3

    def need(self, req) -> int:
        return self.t.need

    def start(self, req) -> None:
        ctx, api = self.t.ctx, self.api
        lo_h, hi_h = self.t.uploads[req.bounds]
        lo = ctx.import_ct(lo_h, api.FORM_NATIVE | api.FORM_ASYNC)
        hi = ctx.import_ct(hi_h, api.FORM_NATIVE | api.FORM_ASYNC)
        arena = self.torch.empty(self.t.arena_bytes, dtype=self.torch.uint8, device="cuda")
        req.state = self.circuit_mod.Runner(self.t.circuit, ctx, self.t.keys,
                                            {"x": self.t.columns[req.col_a],
                                             "y": self.t.columns[req.col_b], "lo": lo, "hi": hi},
                                            arena=arena)

    def stage(self, reqs) -> list:
        t0 = time.perf_counter()
        entries = []
        for r in reqs:
            entries.extend(r.state.stage_ops())
        self.staged = list(reqs)
        self.host_stage_s += time.perf_counter() - t0
        return entries

    def submit(self, entries):
        api, torch = self.api, self.torch
        t0 = time.perf_counter()
        batch = api.Batch(entries)
        need = batch.workspace_bytes(self.lanes)
        if self.ws is None or self.ws.numel() < need:
            self.ws = None
            self.ws = torch.empty(max(need, 1 << 20), dtype=torch.uint8, device="cuda")
        if self.profile:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
        batch.run(self.lanes, self.ws)
        if self.profile:
            e1.record()
            self.tick_events.append((e0, e1))
        self.n_ops += len(entries)
        self.n_ticks += 1
        # Buffers whose last reader is in this batch go back to the allocator
        # only now: released before the submission, their memory could be
        # handed to another request's output within the same batch.
        for r in self.staged:
            r.state.advance()
        self.staged = []
        self.host_submit_s += time.perf_counter() - t0

    def is_done(self, req) -> bool:
        return req.state.done

    def finish(self, req) -> None:
        ct = req.state.result("sum")
        host = self.free_hosts.pop() if self.free_hosts else \
            self.torch.empty(tuple(ct.shape), dtype=self.torch.int64, pin_memory=True)
        self.t.ctx.export_into(ct, host, self.api.FORM_NATIVE | self.api.FORM_ASYNC)
        req.result = host
        req.state.release()
        req.state = None

    def retire(self, req) -> None:
        host = req.result
        req.result = host.clone() if self.keep else None
        self.free_hosts.append(host)

    def mark(self):
        ev = self.torch.cuda.Event()
        ev.record()
        return ev

    def ready(self, token) -> bool:
        return token.query()

    def wait(self, token) -> None:
        token.synchronize()


def make_requests(table: Table, count: int, rate: float, seed: str) -> list:
    rng = W.rng_for(seed)
    t = poisson_arrivals(rate, count, rng) if rate > 0 else np.zeros(count)
    out = []
    for i in range(count):
        a, b = rng.choice(COLS, size=2, replace=False)
        out.append(Request(id=i, arrival=float(t[i]), col_a=int(a), col_b=int(b),
                           bounds=int(rng.integers(len(table.uploads)))))
    return out


# --------------------------------------------------------------------------- search-and-average
def _scalar(ctx, ct, r: float):
    """Server-side multiplication by the real r at unchanged scale: the
    integer k = round(r q_top) then a rescale by q_top; returns the
    ciphertext and the multiplier k / q_top it actually applied."""
    level = ct.shape[-2]
    q = ctx.q[level - 1]
    k = int(round(r * q))
    return ctx.rescale(ctx.mul_int(ct, k)), k / q


def multiply_inverse(table: Table, ct, scale: float, rng) -> tuple:
    """The two-party multiply-inverse (the paper's Algorithm 2), slot 0:
    the server masks Enc(x) by a random real r and sends Enc(r x); the
    client decrypts, inverts and sends back Enc(1 / (r x)) (a fresh
    encryption of the constant); the server multiplies by r again, leaving
    Enc(1 / x).  Returns (Enc(1/x), the masked value the client saw)."""
    ctx, keys, enc = table.ctx, table.keys, table.encoding
    r = float(rng.uniform(0.5, 2.0))
    c1, r_eff = _scalar(ctx, ct, r)                                # server
    x1 = float(ctx.decode_ckks(keys, c1, scale)[0].real)           # client
    m = np.zeros(ctx.n, dtype=np.int64)
    m[0] = enc.encode_constant(1.0 / x1, table.delta)
    c2 = ctx.encrypt(keys, m, W.seed_for(f"{table.seed}-inv-{rng.integers(1 << 62)}"))
    c3, _ = _scalar(ctx, c2, r_eff)                                # server
    return c3, x1


def search_and_average(table: Table, col_a: int, col_b: int, bounds: int, rng=None) -> dict:
    """Avg(column b) where lo <= column a <= hi (soft predicate): the circuit
    computes Enc(sum of mask * b) and Enc(sum of mask) together, the
    multiply-inverse turns the count into Enc(1 / count), one HMult gives
    the average; returns the decrypted average and the intermediate values."""
    from . import api, circuit
    ctx, keys = table.ctx, table.keys
    rng = rng or W.rng_for(f"{table.seed}-avg")
    c = table.avg_circuit()
    lo_h, hi_h = table.uploads[bounds]
    inputs = {"x": table.columns[col_a], "y": table.columns[col_b], "ones": table.ones,
              "lo": ctx.import_ct(lo_h, api.FORM_NATIVE), "hi": ctx.import_ct(hi_h, api.FORM_NATIVE)}
    run = circuit.Runner(c, ctx, keys, inputs)
    ws = None
    while not run.done:
        ops = run.stage_ops()
        batch = api.Batch(ops)
        need = batch.workspace_bytes(8)
        if ws is None or ws.numel() < need:
            ws = table.torch.empty(need, dtype=table.torch.uint8, device="cuda")
        batch.run(8, ws)
        run.advance()
    s_ct, n_ct = run.result("sum"), run.result("count")
    s_scale = c.nodes[c.outputs["sum"]].scale
    n_scale = c.nodes[c.outputs["count"]].scale
    inv, masked = multiply_inverse(table, n_ct, n_scale, rng)
    # bring 1/count down to the sum's level, then one HMult + rescale
    lv = s_ct.shape[-2]
    if inv.shape[-2] > lv:
        inv = ctx.drop_level(inv, lv)
    elif inv.shape[-2] < lv:
        s_ct = ctx.drop_level(s_ct, inv.shape[-2])
        lv = inv.shape[-2]
    avg_ct = ctx.mul_relin_rescale(keys, s_ct, inv)
    avg_scale = s_scale * table.delta / ctx.q[lv - 1]
    avg = float(ctx.decode_ckks(keys, avg_ct, avg_scale)[0].real)
    return {"avg": avg, "masked_count_seen_by_client": masked,
            "sum": float(ctx.decode_ckks(keys, s_ct, s_scale)[0].real),
            "count": float(ctx.decode_ckks(keys, n_ct, n_scale)[0].real)}
