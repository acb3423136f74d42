#!/usr/bin/env python
"""Throughput of batched CKKS homomorphic multiplication with
relinearisation (and rescale) at N = 2^16, L = 24, K = 4, dnum = 3 on GB300.

One step = one batched HMult+relin+rescale of 8 ciphertext pairs at level 24
(the whole hot path: tensor, INTT, exact ModUp, NTT, key inner product,
exact ModDown fused with the rescale), inputs resident in HBM.  Prints one
JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl catfhe|reference]

N > 1 runs under torchrun as independent replicas (one process per GPU, no
data-path collective: the batch is independent ciphertexts), value = all
ranks' operations / the slowest rank's time.  ``--impl reference`` times the
CPU oracle on this host's cores on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HMult+relin/s at N=2^16 L=24, batched vs single; NTT % of roofline; p99 ms"
UNIT = "HMult+relin/s"
PRESET = "ckks_n16"
BATCH = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="catfhe", choices=["catfhe", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the rotation and N=2^14 BFV/BGV side measurements")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the private-query serving sweep")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed helpers

def dist_init(n_gpus):
    from paper_2503_22227_gb300 import replicas
    return replicas.init_from_env()


def barrier(world):
    from paper_2503_22227_gb300 import replicas
    replicas.barrier(world)


def max_over_ranks(x, world):
    from paper_2503_22227_gb300 import replicas
    return replicas.max_over_ranks(x, world, "cuda")


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle leg

def oracle_op_seconds(n_ops: int = 1, warm: int = 0):
    """Times the CPU oracle on `n_ops` HMult+relin+rescale of the workload
    (one ciphertext pair each), single-threaded, after `warm` untimed ones;
    keygen untimed."""
    import oracle
    from paper_2503_22227_gb300 import workloads as W
    p = W.PRESETS[PRESET]
    ctx = oracle.Context(p.scheme, p.log_n, p.q_bits, p.p_bits, p.dnum, log_n_max=p.log_n_max)
    keys = ctx.keygen(W.seed_for("bench-keys"))
    seed = W.seed_for("bench-inputs")
    times = []
    for i in range(warm + n_ops):
        a = ctx.ct_uniform(seed, 2 * i, p.L)
        b = ctx.ct_uniform(seed, 2 * i + 1, p.L)
        t0 = time.perf_counter()
        ctx.rescale(ctx.mul_relin(keys, a, b))
        if i >= warm:
            times.append(time.perf_counter() - t0)
    return times


def _ref_worker(args):
    idx, n_ops, warm = args
    return oracle_op_seconds(n_ops, warm)


def oracle_pool(k: int, warm: int = 0):
    """k oracle operations spread over min(k, cores) spawned processes (a
    spawned pool: safe after CUDA has been initialised in this process),
    each process first running ceil(warm / processes) untimed ones.
    Returns (ops/s from the slowest worker's op time, processes, wall s,
    s per op, warm-up ops run)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    procs = max(1, min(k, cores))
    per = [k // procs + (1 if i < k % procs else 0) for i in range(procs)]
    w = -(-warm // procs) if warm > 0 else 0
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(procs) as pool:
        results = pool.map(_ref_worker, [(i, per[i], w) for i in range(procs)])
    wall = time.perf_counter() - t0
    busy = max(sum(r) for r in results)
    return k / busy, procs, wall, busy / max(per), w * procs


def run_reference(args):
    """The CPU oracle on this host's cores: each step is one HMult+relin+
    rescale of one pair; steps are spread over worker processes (spawned)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    # one operation per step, at most two per core, so the run stays bounded
    k = max(1, min(args.steps, 2 * cores))
    value, procs, wall, per_op, warmed = oracle_pool(k, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": k, "warmup": warmed, "ms_per_step": 1e3 * per_op,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "ckks_n16: CKKS N=2^16 L=24 K=4 dnum=3, HMult+relin+rescale "
                               "of uniform ciphertext pairs", "N": 1 << 16, "L": 24, "K": 4,
                   "dnum": 3},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{k} HMult+relin+rescale ops (one pair each; steps capped at "
                                   f"2 per core) over {procs} processes, after {warmed} untimed "
                                   f"warm-up ops (one or more per process); keygen untimed; "
                                   f"wall {wall:.1f}s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg

def _time(fn, reps):
    import torch
    s = torch.cuda.current_stream()
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / reps


def uneven_mix(api, W, R, mm_peak, n_ops=256, lanes=8, reps=5):
    """256 CKKS operations with N drawn from {2^13 .. 2^16}, levels uniform in
    2..24, kinds uniform over HMult+relin / HRotate(r in 1..16) / rescale, on
    one prime chain (q = 1 mod 2^17), tuned NTT schedules, captured once into
    a CUDA graph over concurrent lanes and replayed."""
    import numpy as np
    import torch
    rng = W.rng_for("uneven-mix")
    base = W.PRESETS["ckks_n16"]
    ctxs = {}
    tuned = {}
    for log_n in (13, 14, 15, 16):
        pr = W.Preset(f"mix_n{log_n}", W.CKKS, log_n, base.q_bits, base.p_bits, base.dnum,
                      log_n_max=16)
        c = api.Context(pr)
        k = c.keygen(W.seed_for(f"mix-keys-{log_n}"))
        gs = [c.galois_elt(r) for r in range(1, 17)]
        for g in gs:
            k.gen_galois(g)
        # one schedule per launch size class: one ciphertext (2L limbs),
        # four, sixteen
        tuned[log_n] = {cls: c.tune_ntt(2 * c.L * m)
                        for cls, m in (("<=64", 1), ("<=256", 4), (">256", 16))}
        ctxs[log_n] = (c, k, gs)
    ops, keep, work = [], [], 0.0
    kinds = [api.OP_MUL_RELIN, api.OP_ROTATE, api.OP_RESCALE]
    seed = W.seed_for("mix-inputs")
    for i in range(n_ops):
        log_n = int(rng.choice([13, 14, 15, 16]))
        level = int(rng.integers(2, 25))
        kind = kinds[int(rng.integers(0, 3))]
        c, k, gs = ctxs[log_n]
        a = c.ct_uniform(seed, 2 * i, level)
        b = c.ct_uniform(seed, 2 * i + 1, level) if kind == api.OP_MUL_RELIN else None
        out = c.empty_ct(1, level - 1 if kind == api.OP_RESCALE else level)
        g = gs[int(rng.integers(0, 16))]
        ops.append(api.make_op(kind, c, a, out, keys=k, b=b, galois_elt=g))
        keep.append((a, b, out))
        if kind == api.OP_MUL_RELIN:
            w = R.ckks_mul_relin_rescale(c.n, level, c.K, c.alpha).modmuls
        elif kind == api.OP_ROTATE:
            w = R.ckks_rotate(c.n, level, c.K, c.alpha).modmuls
        else:
            w = (2 + 2 * (level - 1)) * c.n // 2 * log_n + 4 * level * c.n
        work += w
    res = {}
    for nl in (lanes, 1):
        graph = api.Graph(ops, lanes=nl)
        t = _time(graph.launch, reps)
        res[nl] = (t, graph.nodes)
        graph.close()
    t, nodes = res[lanes]
    return {"value": n_ops / t, "unit": "ops/s", "n_ops": n_ops, "lanes": lanes,
            "graph_nodes": nodes, "ms_per_graph": t * 1e3,
            "one_lane_ops_per_s": n_ops / res[1][0],
            "modmul_frac_of_peak": work / t / mm_peak,
            "ntt_schedules": {f"2^{k}": {cls: {"chosen": cv[0], "us_per_schedule": cv[1]}
                                         for cls, cv in v.items()}
                              for k, v in tuned.items()},
            "note": "HMult+relin / HRotate / rescale mix over N=2^13..2^16, levels 2..24; "
                    "frac = sum of per-op modular products / (time x modmul peak)"}


def secondary(ctx, keys, a, api, W):
    """HRotate by r = 1..16 on the batch of 8 (one Galois key each), and
    HMult+relin on 16 pairs of the N=2^14 BFV and BGV chains."""
    import torch
    out = {}
    gs = [ctx.galois_elt(r) for r in range(1, 17)]
    for g in gs:
        keys.gen_galois(g)
    rot = ctx.empty_ct(*a.shape[:1], a.shape[2])

    def rotate_all():
        for g in gs:
            ctx.rotate(keys, a, g, rot)
    t = _time(rotate_all, 5)
    out["hrotate_r1_16"] = {"value": a.shape[0] * len(gs) / t, "unit": "HRotate/s",
                            "note": "8 ciphertexts at level 24, r = 1..16 (16 Galois keys)"}
    hoisted = torch.empty((len(gs),) + tuple(a.shape), dtype=a.dtype, device=a.device)
    th = _time(lambda: ctx.rotate_hoisted(keys, a, gs, hoisted), 5)
    out["hrotate_r1_16_hoisted"] = {
        "value": a.shape[0] * len(gs) / th, "unit": "HRotate/s",
        "note": "the same 128 rotations with one shared ModUp per ciphertext "
                "(catfhe_rotate_hoisted; outputs equal catfhe_rotate bit for bit)"}
    for name in ("bfv_n14", "bgv_n14"):
        p = W.PRESETS[name]
        c2 = api.Context(p)
        k2 = c2.keygen(W.seed_for("bench-keys-" + name))
        seed = W.seed_for("bench-inputs-" + name)
        x = torch.cat([c2.ct_uniform(seed, 2 * i, p.L) for i in range(p.batch)])
        y = torch.cat([c2.ct_uniform(seed, 2 * i + 1, p.L) for i in range(p.batch)])
        o = c2.empty_ct(p.batch, p.L)
        t = _time(lambda: c2.mul_relin(k2, x, y, o), 10)
        out[name] = {"value": p.batch / t, "unit": "HMult+relin/s",
                     "note": f"N=2^14, 8 x 55-bit q, t=65537, batch {p.batch}"}
        del c2, k2
    return out

def serving_sweep(W, fracs=(0.1, 0.5, 0.8, 1.5), lanes=8, max_active=64):
    """The private-query workload (1000 x 4 encrypted table, N=2^16, L=24,
    K=8): the saturation rate from a burst of 64 requests, then Poisson
    arrivals at fractions of it; p50/p99 latency (arrival to result in host
    memory) and throughput per rate."""
    import torch

    from paper_2503_22227_gb300 import serving as S
    table = S.Table(W.PRESETS["ckks_n16_k8"], bound_pairs=8)
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(max_active * table.need, 0.8 * free))
    eng = S.GpuEngine(table, lanes=lanes, keep_results=False)
    # warm-up: a full burst, so the allocator holds the memory of 64 requests
    S.serve(S.make_requests(table, max_active, 0.0, "serve-warm"), eng, budget, max_active)
    torch.cuda.synchronize()
    # one request alone, and a burst of 64, with host and device time split
    prof = {}
    for name, count in (("alone", 1), ("burst64", max_active)):
        eng.profile = True
        eng.reset_profile()
        st = S.serve(S.make_requests(table, count, 0.0, "serve-prof"), eng, budget, max_active)
        dev = eng.device_busy_s()
        prof[name] = {"wall_ms": st.wall_s * 1e3, "device_busy_ms": dev * 1e3,
                      "host_stage_ms": eng.host_stage_s * 1e3,
                      "host_submit_ms": eng.host_submit_s * 1e3, "ticks": eng.n_ticks,
                      "ops": eng.n_ops}
        eng.profile = False
    burst = S.serve(S.make_requests(table, max_active, 0.0, "serve-burst"), eng, budget, max_active)
    mu = burst.throughput
    points = []
    for f in fracs:
        rate = f * mu
        count = int(min(192, max(32, rate * 3.0)))
        st = S.serve(S.make_requests(table, count, rate, f"serve-{f}"), eng, budget, max_active)
        points.append({"offered_per_s": rate, "requests": count, "throughput_per_s": st.throughput,
                       **st.latency, "mean_active": st.mean_active, "max_active": st.max_active,
                       "joined_running_batch": st.admitted_while_busy, "ticks": st.ticks})
    # search-and-average: circuit (sum and count) + two-party inverse + HMult,
    # one query at a time, wall time including the client's decrypt/encrypt
    import numpy as np
    avg_ms = []
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.search_and_average(table, k % S.COLS, (k + 1) % S.COLS, k % len(table.bounds),
                             rng=np.random.default_rng(k))
        torch.cuda.synchronize()
        avg_ms.append((time.perf_counter() - t0) * 1e3)
    counts = table.circuit.counts()
    head = points[1] if len(points) > 1 else points[0]
    out = {"unit": "queries/s", "saturation_per_s": mu,
           "burst64": {"throughput_per_s": mu, **burst.latency, "ticks": burst.ticks},
           "profile": prof,
           "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
           "at_offered_per_s": head["offered_per_s"], "sweep": points,
           "request": {"rows": S.ROWS, "columns": S.COLS, "stages": len(table.circuit.stages()),
                       "ops": {k: v for k, v in counts.items() if k != "input"},
                       "reserved_bytes": table.need},
           "search_and_average_ms": {"first": avg_ms[0], "median_of_rest": float(np.median(avg_ms[1:])),
                                     "note": "Avg(b) where lo <= a <= hi: sum and count circuit, the "
                                             "two-party multiply-inverse (client decrypts the masked "
                                             "count, inverts, re-encrypts), one HMult; one query alone"},
           "budget_bytes": budget, "max_active": max_active, "lanes": lanes,
           "note": "latency from Poisson arrival to the encrypted answer in pinned host memory; "
                   "p50/p99 at the second sweep point (0.5 x saturation)"}
    del eng, table
    torch.cuda.empty_cache()
    return out


NTT_TRAFFIC = os.path.join(ROOT, "profiles", "ntt_fwd_ckks_n16_384limbs.md")
NTT_SOURCE = os.path.join(ROOT, "paper_2503_22227_gb300", "csrc", "ntt.cu")


def ntt_traffic():
    """DRAM bytes per forward transform of the 384 limbs (both passes), from
    the committed ncu summary, if it was taken on the current NTT source."""
    import hashlib
    try:
        text = open(NTT_TRAFFIC).read()
        src = hashlib.sha256(open(NTT_SOURCE, "rb").read()).hexdigest()
    except OSError:
        return None
    fields = {}
    for line in text.splitlines():
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("ntt.cu sha256") != src:
        return None
    try:
        return int(fields["traffic bytes per transform"])
    except (KeyError, ValueError):
        return None


def run_catfhe(args):
    import numpy as np
    import torch

    from paper_2503_22227_gb300 import api, roofline as R, workloads as W

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    p = W.PRESETS[PRESET]
    ctx = api.Context(p)
    keys = ctx.keygen(W.seed_for("bench-keys"))
    seed = W.seed_for("bench-inputs")
    L = p.L
    a = torch.cat([ctx.ct_uniform(seed, 2 * i, L) for i in range(BATCH)])
    b = torch.cat([ctx.ct_uniform(seed, 2 * i + 1, L) for i in range(BATCH)])
    out = ctx.empty_ct(BATCH, L - 1)
    stream = torch.cuda.current_stream()

    def step():
        ctx.mul_relin_rescale(keys, a, b, out)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None

    # ---- timed region: exactly K steps, CUDA events on the launching stream
    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    launches0 = api.kernel_launches()
    torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed steps
    ev[0].record(stream)
    for i in range(K):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = api.kernel_launches() - launches0
    barrier(world)
    clk = clocks.stop() if clocks else None
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    total_s = max_over_ranks(ev[0].elapsed_time(ev[K]) * 1e-3, world)
    from paper_2503_22227_gb300 import replicas
    value = replicas.throughput(BATCH * K, world, total_s)

    # ---- single-ciphertext launches for the same work
    def single_step():
        for i in range(BATCH):
            ctx.mul_relin_rescale(keys, a[i:i + 1], b[i:i + 1], out[i:i + 1])

    for _ in range(2):
        single_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ks = max(3, K // 3)
    e0.record(stream)
    for _ in range(ks):
        single_step()
    e1.record(stream)
    torch.cuda.synchronize()
    single_value = BATCH * ks / (e0.elapsed_time(e1) * 1e-3)

    # ---- NTT roofline: the batched forward NTT of the step's input volume
    mm_peak, bf_narrow_peak, bf_peak = api.measure_int_peak()
    limbs = torch.cat([a.reshape(2 * BATCH, L, p.n)]).clone()
    for _ in range(3):
        ctx.ntt(limbs)
    torch.cuda.synchronize()
    reps = 20
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("ntt_roofline")
    f0.record(stream)
    for _ in range(reps):
        ctx.ntt(limbs)
    f1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ntt_s = f0.elapsed_time(f1) * 1e-3 / reps
    n_limbs = 2 * BATCH * L
    bfly = n_limbs * (p.n // 2) * 16
    ntt_rate = bfly / ntt_s
    ntt_gbs = R.ntt_bytes(p.n, n_limbs) / ntt_s / 1e9

    # ---- step roofline: max(bytes / HBM, modmuls / modmul peak) per operation
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    work = R.ckks_mul_relin_rescale(p.n, L, p.K, ctx.alpha)
    bytes_op = R.bytes_mul_relin_rescale(p.n, L, L, p.K, ctx.alpha, BATCH)
    t_roof = max(bytes_op / hbm, work.modmuls / mm_peak)
    t_meas = total_s / (BATCH * K) * world

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # Every step: upload both input batches from pinned host memory,
        # HMult+relin+rescale, copy the result batch back to pinned host
        # memory, all through the C ABI.  Steps are pipelined over two buffer
        # sets and three streams (uploads, compute, downloads), so step k+1's
        # upload and step k-1's download overlap step k's compute; every
        # step's copies stay inside the timed region.
        ha = torch.empty(a.shape, dtype=torch.int64, pin_memory=True)
        hb = torch.empty(b.shape, dtype=torch.int64, pin_memory=True)
        ha.copy_(a.cpu())
        hb.copy_(b.cpu())
        ref = out.cpu()
        # the client's ciphertexts in the bit-packed transfer form (50-bit
        # fields), packed once on the host before the timed region
        pa, pb = ctx.pack(ha).pin_memory(), ctx.pack(hb).pin_memory()
        lo = out.shape[2]
        wo = ctx.packed_words(lo, BATCH)
        hpo = [torch.empty(wo, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        da = [torch.empty_like(a) for _ in range(2)]
        db = [torch.empty_like(b) for _ in range(2)]
        do = [torch.empty_like(out) for _ in range(2)]
        sa = [torch.empty(pa.numel(), dtype=torch.int64, device="cuda") for _ in range(2)]
        sb = [torch.empty(pb.numel(), dtype=torch.int64, device="cuda") for _ in range(2)]
        so = [torch.empty(wo, dtype=torch.int64, device="cuda") for _ in range(2)]
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_cmp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        asyn = api.FORM_ASYNC

        def upload(k):
            ctx.import_packed(pa, L, BATCH, out=da[k], ws=sa[k], flags=asyn)
            ctx.import_packed(pb, L, BATCH, out=db[k], ws=sb[k], flags=asyn)

        def download(k):
            ctx.export_packed(do[k], hpo[k], ws=so[k], flags=asyn)

        def e2e_run(steps):
            for e in ev_cmp + ev_out:
                e.record()
            for i in range(steps):
                k = i % 2
                with torch.cuda.stream(s_in):
                    s_in.wait_event(ev_cmp[k])
                    upload(k)
                    ev_in[k].record(s_in)
                with torch.cuda.stream(s_cmp):
                    s_cmp.wait_event(ev_in[k])
                    s_cmp.wait_event(ev_out[k])
                    ctx.mul_relin_rescale(keys, da[k], db[k], do[k])
                    ev_cmp[k].record(s_cmp)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_cmp[k])
                    download(k)
                    ev_out[k].record(s_out)
            torch.cuda.synchronize()

        # the host link's own rates, through the same calls: uploads alone,
        # downloads alone, both at once (two streams)
        def link_s(up, down, reps=5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                if up:
                    with torch.cuda.stream(s_in):
                        upload(0)
                if down:
                    with torch.cuda.stream(s_out):
                        download(1)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps

        h2d_b, d2h_b = (pa.numel() + pb.numel()) * 8, wo * 8
        link_s(True, True, 2)
        t_up, t_down, t_both = link_s(True, False), link_s(False, True), link_s(True, True)
        link = {"h2d_gbs": h2d_b / t_up / 1e9, "d2h_gbs": d2h_b / t_down / 1e9,
                "both_gbs": (h2d_b + d2h_b) / t_both / 1e9,
                "bound_per_s": BATCH / t_both,
                "note": "one step's packed uploads and download alone and at once, through "
                        "the same calls (unpack / pack kernels included); bound_per_s = "
                        "operations per second if a step took only its transfers"}
        e2e_run(3)
        ke = max(3, K // 3)
        barrier(world)
        t0 = time.perf_counter()
        e2e_run(ke)
        te = max_over_ranks(time.perf_counter() - t0, world)
        last = ctx.unpack(hpo[(ke - 1) % 2].numpy().view(np.uint64), BATCH, lo)
        if not np.array_equal(last, ref.numpy().view(np.uint64)):
            raise RuntimeError("end-to-end result differs from the device-resident result")
        e2e = {"value": world * BATCH * ke / te, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d_b), "d2h_bytes_per_step": int(d2h_b),
               "note": "pinned host in/out in the bit-packed transfer form (50-bit fields; the "
                       "client packs its inputs once before timing) through "
                       "catfhe_ct_import_packed / catfhe_ct_export_packed (asynchronous), "
                       "pipelined over 2 buffer sets and 3 streams; the last result is "
                       "unpacked and checked against the device-resident result",
               "link": link}

    side = None
    if not args.no_secondary:
        side = secondary(ctx, keys, a, api, W)
        side["uneven_mix"] = uneven_mix(api, W, R, mm_peak)
    serving = None
    if not args.no_serving:
        serving = serving_sweep(W)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands on every host core (one op per process),
        # and on one thread
        pv, procs, wall, _, _ = oracle_pool(os.cpu_count() or 1)
        ts = oracle_op_seconds(1)
        cpu = {"value": pv, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} HMult+relin+rescale ops of the workload (N=2^16, L=24; one "
                         f"uniform pair each), one per spawned process on {procs} cores; "
                         f"keygen untimed; wall {wall:.1f}s",
               "single_thread": {"value": 1.0 / ts[0], "cores": 1,
                                 "sample": "1 op of the same workload on one thread"}}
    step_ms_sorted = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": 1e3 * total_s / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "ckks_n16: CKKS N=2^16 L=24 (50-bit q) K=4 (60-bit p) dnum=3, "
                               "batch of 8 uniform ciphertext pairs, fused HMult+relin+rescale",
                   "N": p.n, "L": L, "K": p.K, "dnum": p.dnum, "batch": BATCH,
                   "l2": "inputs 384 MiB + key 84 MiB per step, larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": "batched forward NTT (k_ntt_fwd_cols + k_ntt_fwd_rows)",
                     "achieved": ntt_rate / 1e9, "peak": bf_peak / 1e9, "unit": "Gbutterfly/s",
                     "frac": ntt_rate / bf_peak, "traffic": ntt_traffic(),
                     "peak_source": "measured: register-resident loop of the forward "
                                    "butterfly the transform runs on these 50-bit primes "
                                    "(catfhe_measure_int_peak, wide form), whole GPU",
                     "peak_narrow_form": bf_narrow_peak / 1e9,
                     "hbm_view": {"achieved_gbs": ntt_gbs, "peak_gbs": hbm / 1e9,
                                  "frac": ntt_gbs * 1e9 / hbm},
                     "limbs_per_launch": n_limbs, "us_per_launch": ntt_s * 1e6},
        "step_roofline": {"modmuls_per_op": work.modmuls, "bytes_per_op": bytes_op,
                          "modmul_peak_per_s": mm_peak, "hbm_bytes_per_s": hbm,
                          "roofline_us_per_op": t_roof * 1e6, "measured_us_per_op": t_meas * 1e6,
                          "frac": t_roof / t_meas},
        "single": {"value": single_value, "unit": UNIT,
                   "note": "same 8 pairs as 8 single-ciphertext launches"},
        "latency_ms": {"p50": step_ms_sorted[len(step_ms) // 2],
                       "p99": step_ms_sorted[min(len(step_ms) - 1, int(0.99 * len(step_ms)))],
                       "unit": "ms per batched step of 8"},
        "gpu_launches": int(launches),
        "p99_ms": serving["p99_ms"] if serving else None,
        "serving": serving,
        "secondary": side,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_catfhe(args)


if __name__ == "__main__":
    main()
