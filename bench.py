"""Benchmark of the multi-vector MaxSim hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gem|reference] [--workload text|small]

One step = one exhaustive search over the text-corpus workload (500,000 sets,
lognormal lengths mean 70 clipped 20..180, d = 128, 4,096-centre mixture;
1,000 queries of 32 vectors): BF16 tensor-core MaxSim of every (query, set)
pair -> top-1000 per query -> exact FP32 Kahan rerank of those 1,000 ->
top-100.  The metric is doc-sets scored per second (query-set x doc-set pairs of
the exhaustive pass).  Inputs are synthetic (seeded) and resident in HBM before
the timed region; the 9 GB bf16 store exceeds L2, so no flush is needed.

Under torchrun each rank scores its own 1,000 queries against its own replica
of the store (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    "text": dict(n_sets=500_000, n_queries=1000, rerank=1000, k=100),
    "small": dict(n_sets=20_000, n_queries=100, rerank=1000, k=100),
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        rank = int(os.environ["RANK"])
        local = int(os.environ.get("LOCAL_RANK", rank))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return dist, rank, ws, local
    return None, 0, 1, 0


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


def cpu_baseline(docs_host: torch.Tensor, offsets: np.ndarray, q_host: torch.Tensor, q_offsets: np.ndarray,
                 n_docs: int, budget_s: float, k: int):
    """The FP64 oracle (exact CH of every pair + exact top-k), timed on host cores
    over the first n_docs sets for as many queries as fit in budget_s."""
    import oracle
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    off = offsets[: n_docs + 1]
    X = docs_host[: int(off[-1])].numpy()
    t0 = time.perf_counter()
    done = 0
    while done < len(q_offsets) - 1:
        qo = q_offsets[done: done + 2] - q_offsets[done]
        Q = q_host[int(q_offsets[done]): int(q_offsets[done + 1])].numpy()
        S = oracle.score_all(Q, qo, X, off)
        oracle.topk(S[0], k)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done * n_docs / dt, "unit": "doc-sets/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} queries x first {n_docs} sets (FP64 numpy, exact CH + top-{k})",
            "seconds": dt}


def run_reference(args, dist, rank, world):
    """The oracle as the reference arm: host cores, bounded sample per step."""
    if rank != 0:
        return
    cfg = WORKLOADS[args.workload]
    w = synth.text_corpus(n_sets=20_000, n_queries=max(args.steps + args.warmup, 1), device="cpu")
    per_step = []
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(w.docs.vecs, w.docs.offsets, w.queries.vecs[32 * s: 32 * (s + 1)],
                         np.array([0, 32]), 20_000, 0.0, cfg["k"])
        if s >= args.warmup:
            per_step.append(r)
    value = statistics.mean(r["value"] for r in per_step)
    ms = 1000.0 * statistics.mean(r["seconds"] for r in per_step)
    line = {"impl": "reference", "metric": "doc-sets scored/s (exact MaxSim)", "value": value,
            "unit": "doc-sets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "text-corpus 500k sets (sample: 1 query x first 20k sets per step)",
                       "queries_per_step": 1, "m_q": 32},
            "cpu_baseline": {"value": value, "unit": "doc-sets/s", "cores": per_step[0]["cores"],
                             "kind": "oracle", "sample": "1 query x first 20,000 sets per step"},
            "e2e": {"value": value, "unit": "doc-sets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gem(args, dist, rank, world, local):
    import paper_2603_20336_b300 as gem
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = WORKLOADS[args.workload]
    seed = 1236
    w = synth.text_corpus(seed=seed, n_sets=cfg["n_sets"], n_queries=cfg["n_queries"], device=dev)
    # each rank scores its own queries (weak scaling)
    if rank:
        w.queries = synth.vector_sets(np.full(cfg["n_queries"], 32, np.int64), synth.centres(4096, seed),
                                      seed + 7919 + 104729 * rank, dev)
    store = gem.Store(w.docs.vecs, w.docs.offsets, keep=("f32", "bf16"))
    B = cfg["n_queries"]
    R, K = cfg["rerank"], cfg["k"]
    q = w.queries.vecs
    qo = torch.from_numpy(w.queries.offsets).to(dev)
    rows = int(w.queries.offsets[-1])
    ws = gem.Workspace(store, max_queries=B, max_q_rows=rows, max_q_len=32, max_cands=B * R, max_k=R)
    n_pairs = B * store.n_sets
    V = store.n_vecs

    scores = torch.empty((B, store.n_sets), dtype=torch.float32, device=dev)
    pool_ids = torch.empty((B, R), dtype=torch.int64, device=dev)
    pool_off = torch.arange(B + 1, dtype=torch.int64, device=dev) * R
    pool_sc = torch.empty(B * R, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(st)
        gem.score_all(store, ws, q, qo, "bf16", out=scores)
        if ev:
            ev[1].record(st)
        pid, _ = gem.topk(ws, scores, R)
        pool_ids.copy_(pid)
        gem.score_ids(store, ws, q, qo, pool_off, pool_ids.view(-1), "f32", out=pool_sc)
        out = gem.topk(ws, pool_sc.view(B, R), K, ids=pool_ids.view(-1).view(B, R).contiguous())
        if ev:
            ev[2].record(st)
        return out

    # correctness of the explicit stage sequence against the single-call pipeline
    ids_a, sc_a = step()
    ids_b, sc_b = gem.search(store, ws, q, qo, "bf16", rerank_depth=R, k=K)
    assert torch.equal(ids_a, ids_b) and torch.equal(sc_a, sc_b), "stage sequence != gem_search"
    assert ws.status() == 0

    for _ in range(args.warmup):
        step()
    _barrier(dist)
    launches0 = gem.lib.gem_kernel_launches()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(st)
    for s in range(args.steps):
        step(evs[s])
    t_end.record(st)
    _barrier(dist)
    clk = clocks.stop()
    launches = (gem.lib.gem_kernel_launches() - launches0) // max(1, args.steps)
    ms = t_start.elapsed_time(t_end) / args.steps
    ms = _max_over_ranks(dist, ms)
    k1_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    assert ws.status() == 0

    # end to end through the host-buffer entry point: H2D queries, search, D2H results
    qh = w.queries.vecs.cpu().pin_memory()
    qoh = torch.from_numpy(w.queries.offsets)
    oi = torch.empty((B, K), dtype=torch.int64, pin_memory=True)
    osc = torch.empty((B, K), dtype=torch.float32, pin_memory=True)
    gem.search_host(store, ws, qh, qoh, "bf16", R, K, oi, osc)
    _barrier(dist)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gem.search_host(store, ws, qh, qoh, "bf16", R, K, oi, osc)
    e2e_ms = _max_over_ranks(dist, 1000 * (time.perf_counter() - t0) / args.steps)
    assert torch.equal(oi, ids_a.cpu())

    peaks, peak_kind = _peaks()
    flops = 2.0 * rows * V * 128
    achieved = flops / (k1_ms * 1e-3) / 1e12
    peak = peaks["bf16_tflops"]
    line = {
        "metric": "doc-sets scored/s (exact MaxSim, BF16 tensor cores + FP32 rerank)",
        "value": world * n_pairs / (ms * 1e-3), "unit": "doc-sets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"text-corpus {store.n_sets} sets / {V} vectors, {B} queries x 32, "
                               f"top-{R} -> FP32 rerank -> top-{K}",
                   "n_sets": store.n_sets, "n_vecs": V, "queries": B, "m_q": 32, "rerank": R, "k": K,
                   "l2": "inputs larger than L2 (bf16 store %.2f GB)" % (V * 256 / 1e9)},
        "stages_ms": {"maxsim_bf16": k1_ms,
                      "topk_rerank_topk": statistics.mean(e[1].elapsed_time(e[2]) for e in evs)},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "tc_score_all_kernel<2,false> (+ query packing)",
                     "peak_kind": f"{peak_kind} bf16 burst"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": world * n_pairs / (e2e_ms * 1e-3), "unit": "doc-sets/s",
                "h2d_bytes_per_step": int(qh.numel() * 4 + qoh.numel() * 8),
                "d2h_bytes_per_step": int(oi.numel() * 8 + osc.numel() * 4)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        n_cpu = 20_000
        line["cpu_baseline"] = cpu_baseline(w.docs.vecs[: int(w.docs.offsets[n_cpu])].cpu(), w.docs.offsets,
                                            w.queries.vecs.cpu(), w.queries.offsets, n_cpu,
                                            args.cpu_budget, K)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gem", choices=["gem", "reference"])
    ap.add_argument("--workload", default="text", choices=list(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        # the oracle runs on host cores only: rank 0 times it, other ranks exit
        run_reference(args, None, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    dist, rank, world, local = _dist()
    run_gem(args, dist, rank, world, local)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
