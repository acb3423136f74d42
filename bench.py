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
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default NTT schedules (for profiler runs, whose replays "
                         "would skew the tuner's timings)")
    ap.add_argument("--detail", default=os.path.join(ROOT, "bench_out", "bench_detail.json"),
                    help="where the full measurement record (sweeps, schedule tables) goes")
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


# ---------------------------------------------------------------- workload description

def workload_config(world: int = 1) -> dict:
    """The `config` object of both arms' lines (the same workload)."""
    return {"workload": "ckks_n16: CKKS N=2^16 L=24 (50-bit q) K=4 (60-bit p) dnum=3, batch "
                        "of 8 uniform pairs, HMult+relin+rescale",
            "N": 1 << 16, "L": 24, "K": 4, "dnum": 3, "batch": BATCH,
            "l2": "inputs 384 MiB + key 84 MiB per step > L2, no flush",
            "parallelism": f"replicas x{world}"}


# ---------------------------------------------------------------- CPU oracle leg

def _oracle_setup():
    import oracle
    from paper_2503_22227_gb300 import workloads as W
    p = W.PRESETS[PRESET]
    ctx = oracle.Context(p.scheme, p.log_n, p.q_bits, p.p_bits, p.dnum, log_n_max=p.log_n_max)
    keys = ctx.keygen(W.seed_for("bench-keys"))
    return ctx, keys, W.seed_for("bench-inputs"), p


def _oracle_op(ctx, keys, seed, p, pair):
    """One HMult+relin+rescale of uniform pair `pair` of the workload; seconds."""
    a = ctx.ct_uniform(seed, 2 * pair, p.L)
    b = ctx.ct_uniform(seed, 2 * pair + 1, p.L)
    t0 = time.perf_counter()
    ctx.rescale(ctx.mul_relin(keys, a, b))
    return time.perf_counter() - t0


def oracle_single_op_seconds() -> float:
    """The oracle on one thread, one operation alone (keygen untimed)."""
    ctx, keys, seed, p = _oracle_setup()
    return _oracle_op(ctx, keys, seed, p, 0)


def _ref_proc(first, n_ops, warm, barrier, q):
    """One worker: keygen and `warm` untimed ops, then a barrier shared by all
    workers, then `n_ops` timed ops on pairs first, first+1, ...; reports
    (wall-clock start, end, per-op seconds)."""
    ctx, keys, seed, p = _oracle_setup()
    for i in range(warm):
        _oracle_op(ctx, keys, seed, p, 100000 + first + i)
    barrier.wait()
    t_start = time.time()
    times = [_oracle_op(ctx, keys, seed, p, first + i) for i in range(n_ops)]
    q.put((first, t_start, time.time(), times))


def oracle_pool(k: int, warm: int = 0):
    """k timed oracle operations over min(k, cores) spawned processes (safe
    after CUDA has been initialised in this process), after `warm` untimed
    ones spread over the same processes.  All processes start their timed
    operations together (a barrier); the timed region runs from that start
    to the last process's end.  Returns (ops/s over the region, processes,
    region seconds, seconds per op on one core)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    procs = max(1, min(k, cores))
    per = [k // procs + (1 if i < k % procs else 0) for i in range(procs)]
    wper = [warm // procs + (1 if i < warm % procs else 0) for i in range(procs)]
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(procs), ctx.Queue()
    firsts = [sum(per[:i]) for i in range(procs)]
    ps = [ctx.Process(target=_ref_proc, args=(firsts[i], per[i], wper[i], barrier, q))
          for i in range(procs)]
    for pr in ps:
        pr.start()
    res = [q.get() for _ in ps]
    for pr in ps:
        pr.join()
    t0 = min(r[1] for r in res)
    t1 = max(r[2] for r in res)
    per_op = statistics.median([t for r in res for t in r[3]])
    return k / (t1 - t0), procs, t1 - t0, per_op


def run_reference(args):
    """The CPU oracle on this host's cores: each step is one HMult+relin+
    rescale of one ciphertext pair of the workload (a bounded sample of the
    batched step); steps run in parallel over worker processes.  Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    # at most four operations per core (about a minute), so the run stays bounded
    k = max(1, min(args.steps, 4 * cores))
    w = max(0, args.warmup)
    value, procs, region, per_op = oracle_pool(k, w)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": k, "warmup": w, "ms_per_step": 1e3 * region / k,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": workload_config(args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{k} HMult+relin+rescale ops of the workload, one ciphertext "
                                   f"pair each (a step = one op), over {procs} processes started "
                                   f"together after {w} untimed warm-up ops; keygen untimed; "
                                   f"timed region {region:.1f}s; {per_op:.1f}s per op on one core"},
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
            w = R.ckks_mul_relin(c.n, level, c.K, c.alpha).modmuls
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
            "frac": work / t / mm_peak,
            "ntt_schedules": {f"2^{k}": {cls: {"chosen": cv[0], "us_per_schedule": cv[1]}
                                         for cls, cv in v.items()}
                              for k, v in tuned.items()},
            "note": "HMult+relin / HRotate / rescale mix over N=2^13..2^16, levels 2..24; "
                    "frac = sum of per-op modular products / (time x modmul peak)"}


def secondary(ctx, keys, a, api, W, R, mm_peak, hbm):
    """HRotate by r = 1..16 on the batch of 8 (one Galois key each), the same
    rotations hoisted, and HMult+relin on 16 pairs of the N=2^14 BFV and BGV
    chains; each with its roofline fraction (the slower of algorithmic bytes
    over HBM and algorithmic modular products over the measured modmul peak,
    divided by the measured time per operation)."""
    import torch
    out, det = {}, {}
    gs = [ctx.galois_elt(r) for r in range(1, 17)]
    for g in gs:
        keys.gen_galois(g)
    rot = ctx.empty_ct(*a.shape[:1], a.shape[2])
    n, L, K, alpha, batch = ctx.n, a.shape[2], ctx.K, ctx.alpha, a.shape[0]

    def frac(work, nbytes, t_op):
        return max(nbytes / hbm, work.modmuls / mm_peak) / t_op

    def rotate_all():
        for g in gs:
            ctx.rotate(keys, a, g, rot)
    t = _time(rotate_all, 5) / (batch * len(gs))
    rb = R.bytes_keyswitch(n, L, L, 1, L, K, alpha, batch)
    out["hrotate_r1_16"] = {"value": 1 / t, "unit": "HRotate/s",
                            "frac": frac(R.ckks_rotate(n, L, K, alpha), rb, t)}
    hoisted = torch.empty((len(gs),) + tuple(a.shape), dtype=a.dtype, device=a.device)
    th = _time(lambda: ctx.rotate_hoisted(keys, a, gs, hoisted), 5) / (batch * len(gs))
    hb = R.bytes_keyswitch(n, L, L, 1, L, K, alpha, batch, inputs_shared=len(gs))
    out["hrotate_r1_16_hoisted"] = {
        "value": 1 / th, "unit": "HRotate/s",
        "frac": frac(R.ckks_rotate_hoisted(n, L, K, alpha, len(gs)), hb, th)}
    det["rotations"] = "8 ciphertexts at level 24, r = 1..16 (16 Galois keys); hoisted: one " \
                       "shared ModUp per ciphertext (catfhe_rotate_hoisted)"
    # device CKKS encode (host slots -> NTT-form plaintext at level 24) and
    # decode (decrypt + decode -> host slots), one call at a time, wall time
    # with the host copies of the N/2 slots
    from paper_2503_22227_gb300 import encoding
    z = W.complex_slots(W.rng_for("bench-encode"), n)
    scale = 2.0 ** 50
    ctx.encode_ckks(z, scale)
    ct = ctx.encrypt(keys, encoding.encode(z, n, scale), W.seed_for("bench-encode"))
    ctx.decode_ckks(keys, ct, scale)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        ctx.encode_ckks(z, scale)
    torch.cuda.synchronize()
    t_enc = (time.perf_counter() - t0) / 10
    t0 = time.perf_counter()
    for _ in range(10):
        ctx.decode_ckks(keys, ct, scale)
    t_dec = (time.perf_counter() - t0) / 10
    det["ckks_encode_decode_ms"] = {"encode": t_enc * 1e3, "decode": t_dec * 1e3,
                                    "note": "N=2^16, level 24, one call at a time, wall time "
                                            "with the N/2 host slots' copies"}
    for name in ("bfv_n14", "bgv_n14"):
        p = W.PRESETS[name]
        c2 = api.Context(p)
        k2 = c2.keygen(W.seed_for("bench-keys-" + name))
        seed = W.seed_for("bench-inputs-" + name)
        x = torch.cat([c2.ct_uniform(seed, 2 * i, p.L) for i in range(p.batch)])
        y = torch.cat([c2.ct_uniform(seed, 2 * i + 1, p.L) for i in range(p.batch)])
        o = c2.empty_ct(p.batch, p.L)
        torch.cuda.nvtx.range_push(name)  # a profiler's filter for this configuration
        t = _time(lambda: c2.mul_relin(k2, x, y, o), 10) / p.batch
        torch.cuda.nvtx.range_pop()
        if p.scheme == W.BFV:
            w = R.bfv_mul_relin(c2.n, p.L, c2.K, c2.alpha, c2.nb)
        else:
            w = R.bgv_mul_relin(c2.n, p.L, c2.K, c2.alpha)
        nbytes = R.bytes_keyswitch(c2.n, p.L, p.L, 2, p.L, c2.K, c2.alpha, p.batch)
        out[name] = {"value": 1 / t, "unit": "HMult+relin/s", "frac": frac(w, nbytes, t)}
        det[name] = {"modmuls_per_op": w.modmuls, "bytes_per_op": nbytes,
                     "note": f"N=2^14, 8 x 55-bit q, t=65537, batch {p.batch}"}
        del c2, k2
    return out, det


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
    # the same offered load as the headline point, with ticks bounded to the
    # 16 oldest active requests (oldest first) instead of all of them
    half = fracs[1] if len(fracs) > 1 else fracs[0]
    rate = half * mu
    count = int(min(192, max(32, rate * 3.0)))
    st = S.serve(S.make_requests(table, count, rate, f"serve-{half}"), eng, budget, max_active,
                 max_batch=16)
    oldest16 = {"offered_per_s": rate, "requests": count, "throughput_per_s": st.throughput,
                **st.latency, "ticks": st.ticks}
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
           "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "oldest16": oldest16,
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
NTT_SOURCES = [os.path.join(ROOT, "paper_2503_22227_gb300", "csrc", f)
               for f in ("ntt.cu", "ntt_kernels.cuh", "ntt_part.cuh", "ntt_n16.cu",
                         "butterfly.cuh", "modarith.cuh")]


def ntt_source_sha() -> str:
    """SHA-256 over the sources of the N = 2^16 transform's kernels."""
    import hashlib
    h = hashlib.sha256()
    for f in NTT_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def ntt_traffic():
    """DRAM bytes per forward transform of the 384 limbs (both passes), from
    the committed ncu summary, if it was taken on the current NTT sources."""
    try:
        text = open(NTT_TRAFFIC).read()
        src = ntt_source_sha()
    except OSError:
        return None
    fields = {}
    for line in text.splitlines():
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("ntt sources sha256") != src:
        return None
    try:
        return int(fields["traffic bytes per transform"])
    except (KeyError, ValueError):
        return None


def e2e_leg(ctx, keys, a, b, out, K, world, api, np, torch):
    """End to end through the public API with host buffers.  Every step:
    upload both input batches from page-locked host memory in coefficient
    form (catfhe_ct_import: copy, then NTT on the device), HMult+relin+
    rescale, and read the result batch back to page-locked host memory in
    coefficient form (catfhe_ct_export: INTT on the device, then copy); all
    asynchronous on three streams (uploads, compute, downloads) over two
    buffer sets, so step k+1's upload and step k-1's download overlap step
    k's compute.  Every step's copies and transforms are in the timed
    region.  The link bound runs the same pipeline with the compute left out
    (uploads and downloads only, same calls, same overlap), so it is the
    rate the transfers alone allow."""
    L = a.shape[2]
    lo = out.shape[2]
    BATCHn = a.shape[0]
    ha = [torch.empty(a.shape, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    hb = [torch.empty(b.shape, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    coeff_a = ctx.export_ct(a)
    coeff_b = ctx.export_ct(b)
    for k in range(2):
        ha[k].numpy().view(np.uint64)[...] = coeff_a
        hb[k].numpy().view(np.uint64)[...] = coeff_b
    ctx.mul_relin_rescale(keys, a, b, out)
    ref = ctx.export_ct(out)
    ho = [torch.empty(out.shape, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    da = [torch.empty_like(a) for _ in range(2)]
    db = [torch.empty_like(b) for _ in range(2)]
    do = [torch.empty_like(out) for _ in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    form_in = api.FORM_COEFF | api.FORM_ASYNC
    form_out = api.FORM_COEFF | api.FORM_ASYNC
    # every export runs on s_out in order, so one workspace serves both sets
    with torch.cuda.stream(s_out):
        ws_out = ctx.workspace(api.OP_EXPORT, lo, BATCHn)

    def run(steps, compute=True):
        for e in ev_cmp + ev_out:
            e.record()
        for i in range(steps):
            k = i % 2
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_cmp[k])
                ctx.import_ct(ha[k], form_in, out=da[k])
                ctx.import_ct(hb[k], form_in, out=db[k])
                ev_in[k].record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in[k])
                s_cmp.wait_event(ev_out[k])
                if compute:
                    ctx.mul_relin_rescale(keys, da[k], db[k], do[k])
                ev_cmp[k].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_cmp[k])
                ctx.export_into(do[k], ho[k], form_out, ws=ws_out)
                ev_out[k].record(s_out)
        torch.cuda.synchronize()

    run(3)
    run(3, compute=False)
    # the same number of steps as the device-resident measurement, so that the
    # pipeline's fill (first upload) and drain (last compute and download) are
    # spread over as many steps
    ke = max(3, K)
    from paper_2503_22227_gb300 import replicas
    barrier(world)
    t0 = time.perf_counter()
    run(ke)
    te = max_over_ranks(time.perf_counter() - t0, world)
    got = [ho[k].numpy().view(np.uint64) for k in range((ke - 1) % 2, (ke - 1) % 2 + 1)]
    if not np.array_equal(got[0], ref):
        raise RuntimeError("end-to-end result differs from the device-resident result")
    t_link = []
    for _ in range(3):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        run(ke, compute=False)
        t_link.append((time.perf_counter() - t1) / ke)
    tl = min(t_link)
    h2d = 2 * a.numel() * 8
    d2h = out.numel() * 8
    return {"value": world * BATCHn * ke / te, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": te / ke * 1e3,
            "note": "pinned coefficient-form u64 limbs through catfhe_ct_import/export "
                    "around the step, every step",
            "link": {"bound_per_s": BATCHn / tl, "ms_per_step": tl * 1e3,
                     "gbs": (h2d + d2h) / tl / 1e9}}


def _rounded(x):
    """The line's floats to 4 significant digits (the full values go to the
    detail file), so that the one line stays short."""
    if isinstance(x, float):
        return float(f"{x:.4g}")
    if isinstance(x, dict):
        return {k: _rounded(v) for k, v in x.items()}
    if isinstance(x, list):
        return [_rounded(v) for v in x]
    return x


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
    # the NTT schedule of each launch size class this workload uses, picked by
    # the library's tuner (the step's transforms run on 40 to 240 limbs per
    # half batch; the roofline's on 384)
    tuned = {} if args.no_tune else {"<=64": ctx.tune_ntt(2 * L), "<=256": ctx.tune_ntt(4 * L),
                                     ">256": ctx.tune_ntt(2 * BATCH * L)}

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
    issue = R.issue_bounds(float((clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)))
    work = R.ckks_mul_relin_rescale(p.n, L, p.K, ctx.alpha)
    bytes_op = R.bytes_mul_relin_rescale(p.n, L, L, p.K, ctx.alpha, BATCH)
    t_roof = max(bytes_op / hbm, work.modmuls / mm_peak)
    t_meas = total_s / (BATCH * K) * world
    t_roof_issue = max(bytes_op / hbm, work.modmuls / issue["modmul_per_s"])

    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg(ctx, keys, a, b, out, K, world, api, np, torch)

    detail = {}
    side = None
    if not args.no_secondary:
        side, sdet = secondary(ctx, keys, a, api, W, R, mm_peak, hbm)
        detail["secondary"] = sdet
        mix = uneven_mix(api, W, R, mm_peak)
        detail["uneven_mix"] = mix
        side["uneven_mix"] = {k: mix[k] for k in ("value", "unit", "n_ops", "frac")}
        side["uneven_mix"]["schedules_timed_2^16"] = [len(v["us_per_schedule"])
                                                       for v in mix["ntt_schedules"]["2^16"].values()]
    serving = None
    if not args.no_serving:
        serving = serving_sweep(W)
        detail["serving"] = serving
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands on every host core (one op per process),
        # and one op alone on one thread
        pv, procs, region, _ = oracle_pool(os.cpu_count() or 1)
        ts = oracle_single_op_seconds()
        cpu = {"value": pv, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} ops of the workload, one per process, {region:.1f}s; "
                         f"1 op on 1 thread {ts:.1f}s"}
    step_ms_sorted = sorted(step_ms)
    side_short = None
    if side:
        side_short = {k: [round(v["value"]), round(v.get("frac", 0), 3)] for k, v in side.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": 1e3 * total_s / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": workload_config(world),
        "single": {"value": single_value, "batched_over_single": value / world / single_value},
        "p50_ms": serving["p50_ms"] if serving else None,
        "p99_ms": serving["p99_ms"] if serving else None,
        "roofline": {"bound": "alu", "kernel": "fwd NTT, 384 limbs",
                     "achieved": ntt_rate / 1e9, "peak": bf_peak / 1e9, "unit": "Gbutterfly/s",
                     "frac": ntt_rate / bf_peak, "traffic": ntt_traffic(),
                     "frac_of_mul_pipe_bound": ntt_rate * R.LOOP_MUL_PIPE_BUSY / bf_peak,
                     "frac_of_issue_bound": ntt_rate / issue["butterfly_wide_per_s"],
                     "us": ntt_s * 1e6},
        "step_roofline": {"frac": t_roof / t_meas, "frac_of_issue_bound": t_roof_issue / t_meas,
                          "us_per_op": t_meas * 1e6, "roof_us_per_op": t_roof * 1e6},
        "gpu_launches": int(launches),
        "e2e": ({"value": e2e["value"], "unit": UNIT,
                 "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                 "d2h_bytes_per_step": e2e["d2h_bytes_per_step"],
                 "link_bound_per_s": e2e["link"]["bound_per_s"]} if e2e else None),
        "cpu_baseline": cpu, "clocks": clk,
        "secondary": side_short,
        "saturation_qps": serving["saturation_per_s"] if serving else None,
    }
    line = _rounded(line)
    detail["e2e"] = e2e
    detail["secondary_line"] = side
    detail["step_latency_ms"] = {"p50": step_ms_sorted[len(step_ms) // 2],
                                 "p99": step_ms_sorted[min(len(step_ms) - 1,
                                                           int(0.99 * len(step_ms)))]}
    detail["line"] = line
    detail["ntt_schedules_headline"] = {k: {"chosen": v[0], "us_per_schedule": v[1]}
                                        for k, v in tuned.items()}
    lo, hi, wide = api.measure_imad_rates()
    detail["step_roofline"] = {"modmuls_per_op": work.modmuls, "bytes_per_op": bytes_op,
                               "hbm_bytes_per_s": hbm, "issue_bounds": issue,
                               "butterfly_narrow_peak": bf_narrow_peak,
                               "imad_rates_per_s": {"mad.lo.u32": lo, "mad.hi.u32": hi,
                                                    "mad.wide.u32": wide}}
    try:
        os.makedirs(os.path.dirname(args.detail), exist_ok=True)
        with open(args.detail, "w") as f:
            json.dump(detail, f, indent=1)
    except OSError:
        pass
    print(json.dumps(line, separators=(",", ":")), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_catfhe(args)


if __name__ == "__main__":
    main()
