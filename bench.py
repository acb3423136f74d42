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
    return ap.parse_args()


# ---------------------------------------------------------------- distributed helpers

def dist_init(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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

def oracle_op_seconds(n_ops: int = 1):
    """Times the CPU oracle on `n_ops` HMult+relin+rescale of the workload
    (one ciphertext pair each), single-threaded, keygen untimed."""
    import oracle
    from paper_2503_22227_gb300 import workloads as W
    p = W.PRESETS[PRESET]
    ctx = oracle.Context(p.scheme, p.log_n, p.q_bits, p.p_bits, p.dnum, log_n_max=p.log_n_max)
    keys = ctx.keygen(W.seed_for("bench-keys"))
    seed = W.seed_for("bench-inputs")
    times = []
    for i in range(n_ops):
        a = ctx.ct_uniform(seed, 2 * i, p.L)
        b = ctx.ct_uniform(seed, 2 * i + 1, p.L)
        t0 = time.perf_counter()
        ctx.rescale(ctx.mul_relin(keys, a, b))
        times.append(time.perf_counter() - t0)
    return times


def _ref_worker(args):
    idx, n_ops = args
    return oracle_op_seconds(n_ops)


def run_reference(args):
    """The CPU oracle on this host's cores: each step is one HMult+relin+
    rescale of one pair; steps are spread over worker processes (spawned)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    # one operation per step, at most two per core, so the run stays bounded
    k = max(1, min(args.steps, 2 * cores))
    procs = max(1, min(k, cores))
    per = [k // procs + (1 if i < k % procs else 0) for i in range(procs)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        results = pool.map(_ref_worker, [(i, per[i]) for i in range(procs)])
    wall = time.perf_counter() - t0
    busy = max(sum(r) for r in results)      # slowest worker's op time
    value = k / busy
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": k, "warmup": 0, "ms_per_step": 1e3 * busy / max(per),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "ckks_n16: CKKS N=2^16 L=24 K=4 dnum=3, HMult+relin+rescale "
                               "of uniform ciphertext pairs", "N": 1 << 16, "L": 24, "K": 4,
                   "dnum": 3},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{k} HMult+relin+rescale ops (one pair each; steps capped at "
                                   f"2 per core) over {procs} processes; keygen untimed; "
                                   f"wall {wall:.1f}s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg

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
    ev[0].record(stream)
    for i in range(K):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    launches = api.kernel_launches() - launches0
    barrier(world)
    clk = clocks.stop() if clocks else None
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    total_s = max_over_ranks(ev[0].elapsed_time(ev[K]) * 1e-3, world)
    value = world * BATCH * K / total_s

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
    mm_peak, bf_peak = api.measure_int_peak()
    limbs = torch.cat([a.reshape(2 * BATCH, L, p.n)]).clone()
    for _ in range(3):
        ctx.ntt(limbs)
    torch.cuda.synchronize()
    reps = 20
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(reps):
        ctx.ntt(limbs)
    f1.record(stream)
    torch.cuda.synchronize()
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
        ha = torch.empty(a.shape, dtype=torch.int64, pin_memory=True)
        hb = torch.empty(b.shape, dtype=torch.int64, pin_memory=True)
        ho = torch.empty(out.shape, dtype=torch.int64, pin_memory=True)
        ha.copy_(a.cpu())
        hb.copy_(b.cpu())
        da, db = torch.empty_like(a), torch.empty_like(b)

        def e2e_step():
            ctx.import_ct(ha, api.FORM_NATIVE, out=da)
            ctx.import_ct(hb, api.FORM_NATIVE, out=db)
            ctx.mul_relin_rescale(keys, da, db, out)
            ctx.export_into(out, ho, api.FORM_NATIVE)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        ke = max(3, K // 3)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * BATCH * ke / te, "unit": UNIT,
               "h2d_bytes_per_step": int(ha.numel() * 8 + hb.numel() * 8),
               "d2h_bytes_per_step": int(ho.numel() * 8)}

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ts = oracle_op_seconds(1)
        cpu = {"value": 1.0 / ts[0], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "1 HMult+relin+rescale of one uniform pair of the workload "
                         "(N=2^16, L=24), single thread, keygen untimed"}
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
                     "frac": ntt_rate / bf_peak, "traffic": None,
                     "peak_source": "measured: register-resident Shoup butterfly loop "
                                    "(catfhe_measure_int_peak), whole GPU",
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
