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

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# BF16 tensor-core kernel over its algorithmic bytes (unpadded bf16 store + FP32
# score matrix), per schedule (m_tiles, variant, chunk_rows), from one ncu
# capture of one launch on the medium text case (1,000 queries x 50,000 sets,
# 1.090 GB algorithmic); the reported traffic is this ratio times the run's own
# algorithmic bytes (the store is read once per launch and the scores written
# once, so traffic grows in proportion).  An entry is removed when the kernel
# changes, until it is captured again; a schedule without an entry reports null.
TC_TRAFFIC_RATIO = {
    (2, "plain", 65536): 1.19538e9 / 1.08980e9,     # 1.0009 GB read + 0.1945 GB written
    (2, "two_sets", 16384): 1.14127e9 / 1.08980e9,  # 0.9468 GB read + 0.1945 GB written
    (2, "plain", 16384): 1.14045e9 / 1.08980e9,     # 0.9464 GB read + 0.1940 GB written
    (2, "plain", 32768): 1.16730e9 / 1.08980e9,     # 0.9729 GB read + 0.1944 GB written
    (2, "two_sets", 32768): 1.16270e9 / 1.08980e9,  # 0.9683 GB read + 0.1944 GB written
    (2, "two_sets", 65536): 1.19810e9 / 1.08980e9,  # 1.0028 GB read + 0.1953 GB written
}

# the headline metric: (query set, stored set) pairs scored per second by the
# exhaustive search step (both arms report it under this name)
METRIC = "doc-sets scored/s (exact MaxSim, BF16 tensor cores + FP32 rerank)"

WORKLOADS = {
    "text": dict(n_sets=500_000, n_queries=1000, rerank=1000, k=100),
    "small": dict(n_sets=20_000, n_queries=100, rerank=1000, k=100),
    # the text-corpus recipe at 50,000 sets (3.5M vectors, about 3 GB of store
    # copies): the size of the small-case kernel profiles
    "medium": dict(n_sets=50_000, n_queries=1000, rerank=1000, k=100),
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
    """One process per GPU (torchrun); NCCL for the barrier and the max over ranks.
    GEM_BENCH_BACKEND=gloo keeps those host-side (ranks sharing a GPU can then run
    the whole path: their kernels never wait on one another)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        rank = int(os.environ["RANK"])
        local = int(os.environ.get("LOCAL_RANK", rank)) % max(1, torch.cuda.device_count())
        torch.cuda.set_device(local)
        backend = os.environ.get("GEM_BENCH_BACKEND", "nccl")
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
        return dist, rank, ws, local
    return None, 0, 1, 0


def _max_over_ranks(dist, x: float) -> float:
    """The slowest rank's time: the job's time."""
    if dist is None:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_query_seed(seed: int, rank: int) -> int:
    """Seed of the query sets a rank scores (rank 0 keeps the workload's own)."""
    return seed + 7919 + 104729 * rank


def _barrier(dist):
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


def _cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


_ONE_THREAD_CODE = """
import json, sys, time
sys.path.insert(0, {root!r})
import oracle, synth
w = synth.text_corpus(n_sets={n}, n_queries={nq}, device="cpu")
X, Q = w.docs.vecs.numpy(), w.queries.vecs.numpy()
t0 = time.perf_counter()
S = oracle.score_all(Q, w.queries.offsets, X, w.docs.offsets)
for b in range({nq}):
    oracle.topk(S[b], {k})
print(json.dumps({{"seconds": time.perf_counter() - t0}}))
"""


def cpu_baseline_one_thread(k: int, n_sets: int = 5_000, n_queries: int = 4) -> dict:
    """The oracle on one host thread: a child process with every BLAS / OpenMP
    pool limited to one thread scores the first n_queries queries of the
    text-corpus workload against its first n_sets sets (the device-independent
    generator gives the same data on the host; generating it takes most of the
    child's wall time, so the sample is small)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        code = _ONE_THREAD_CODE.format(root=ROOT, n=n_sets, nq=n_queries, k=k)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": n_queries * n_sets / d["seconds"], "unit": "doc-sets/s", "cores": 1,
                "sample": f"{n_queries} queries x the first {n_sets} sets (FP64 numpy, exact CH + top-{k})",
                "seconds": d["seconds"]}
    except Exception as e:  # a failing extra must not hide the headline line
        return {"unavailable": repr(e)[:200]}


def cpu_baseline(docs_host: torch.Tensor, offsets: np.ndarray, q_host: torch.Tensor, q_offsets: np.ndarray,
                 n_queries: int, k: int, n_docs=None, one_thread: bool = False):
    """The FP64 oracle (exact CH of every pair + exact top-k), timed on host cores
    for the first n_queries queries against the first n_docs sets (all by default).
    Returns the timing and the oracle's top-k (ids, scores) of those queries: the
    ground truth for recall.  one_thread: also time one query on a single thread."""
    import oracle
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    n_docs = len(offsets) - 1 if n_docs is None else n_docs
    off = offsets[: n_docs + 1]
    X = docs_host[: int(off[-1])].numpy()
    n_queries = min(n_queries, len(q_offsets) - 1)
    qo = q_offsets[: n_queries + 1]
    Q = q_host[: int(qo[-1])].numpy()
    t0 = time.perf_counter()
    S = oracle.score_all(Q, qo, X, off)
    truth = [oracle.topk(S[b], k) for b in range(n_queries)]
    dt = time.perf_counter() - t0
    res = {"value": n_queries * n_docs / dt, "unit": "doc-sets/s", "cores": cores, "kind": "oracle",
           "sample": f"{n_queries} queries x {n_docs} sets (FP64 numpy, exact CH + top-{k})",
           "seconds": dt, "cpu_model": _cpu_model(), "logical_cpus": os.cpu_count()}
    if one_thread:
        res["one_thread"] = cpu_baseline_one_thread(k)
    return res, truth


TRUTH_FILE = os.path.join(ROOT, "tests", "golden", "text500k_truth.npz")


def load_truth(w):
    """The stored exact FP64 top-100 of all text-corpus queries, if it was
    computed on exactly this data (fingerprint), else None."""
    if not os.path.exists(TRUTH_FILE):
        return None, "no stored ground truth"
    d = np.load(TRUTH_FILE)
    fp = synth.fingerprint(w.docs, w.queries)
    if str(d["fingerprint"]) != fp or d["ids"].shape[0] != w.queries.n_sets:
        return None, "stored ground truth was computed on other data (fingerprint differs)"
    return (d["ids"].astype(np.int64), d["scores"]), "stored"


def recall_vs_truth(found: np.ndarray, truth) -> dict:
    """Mean |found_top100 ∩ exact_top100| / 100 over all queries; boundary_ties
    counts queries whose exact 100th and 101st scores tie within 1e-6 (there the
    exact top-100 itself is ambiguous)."""
    ids, sc = truth
    r = [len(set(found[b, :100].tolist()) & set(ids[b].tolist())) / 100.0 for b in range(ids.shape[0])]
    ties = int(np.sum(np.abs(sc[:, 99] - sc[:, 100]) <= 1e-6 * np.maximum(1.0, np.abs(sc[:, 99]))))
    return {"recall": float(np.mean(r)), "min": float(np.min(r)), "queries": int(ids.shape[0]),
            "boundary_ties": ties}


def _recall(found: np.ndarray, truth):
    """Mean |found ∩ exact| / k over the queries the oracle finished, plus the
    swaps that are ties of the exact scores within 1e-6."""
    rs = []
    for b, (ids, sc) in enumerate(truth):
        rs.append(len(set(found[b].tolist()) & set(ids.tolist())) / len(ids))
    return float(np.mean(rs)) if rs else None


def _time(fn, reps=3, st=None):
    st = st or torch.cuda.current_stream()
    fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_stages(gem, store, ws, w, q, qo, R, K, recall, stages, dev, step_ms, only=None, qch_k1="",
                 schedule=None, bp=None):
    """Every hot-path row measured on its own (after the headline timing)."""
    B = qo.numel() - 1
    rows = q.shape[0]
    flops = 2.0 * rows * store.n_vecs * 128
    out = torch.empty((B, store.n_sets), dtype=torch.float32, device=dev)

    def guard(name, fn):
        if only and name not in only:
            return
        try:
            stages[name] = fn()
        except Exception as e:  # a failing extra must not hide the headline line
            stages[name] = {"error": repr(e)[:300]}

    def fp8():
        # both E4M3 storage forms: per-vector scales (a multiply per stored
        # column in the epilogue) and one power-of-two scale per set (a multiply
        # per set score)
        res = {}
        for dt, name in (("fp8", "per_vector_scale"), ("fp8_set", "per_set_scale")):
            ch = gem.autotune_score_all(store, ws, q, qo, dt, scores=out)
            ms = _time(lambda: gem.score_all(store, ws, q, qo, dt, out=out))
            ms_s = _time(lambda: gem.search(store, ws, q, qo, dt, rerank_depth=R, k=K))
            ids, _ = gem.search(store, ws, q, qo, dt, rerank_depth=R, k=K)
            res[name] = {"ms": ms, "pairs_per_s": B * store.n_sets / (ms * 1e-3), "tflops_equiv": flops / ms / 1e9,
                         "schedule": ch, "search_step_ms": ms_s, "step_speedup_vs_bf16": step_ms / ms_s,
                         "recall_at_100_after_rerank": recall(ids.cpu().numpy())}
        return res

    def fp32():
        ms = _time(lambda: gem.score_all(store, ws, q, qo, "f32", out=out), reps=1)
        ids, _ = gem.search(store, ws, q, qo, "f32", rerank_depth=R, k=K)
        return {"ms": ms, "pairs_per_s": B * store.n_sets / (ms * 1e-3), "tflops": flops / ms / 1e9,
                "frac_of_builder_fp32_peak": (flops / ms / 1e9) / bp["fp32_tflops"] if bp else None,
                "recall_at_100": recall(ids.cpu().numpy()),
                "bf16_rerank_step_speedup_vs_fp32_exhaustive": ms / step_ms}

    def qch():
        # Sec. 5.1 codebook size by default; --qch-k1 sweeps it (Sec. 5.4 varies
        # |C_quant|).  Each size is measured in both estimate forms.
        V = store.n_vecs
        k1_formula = 1 << int(np.floor(np.log2(16.0 * np.sqrt(V))))
        sizes = [int(x) for x in qch_k1.split(",")] if qch_k1 else [k1_formula]
        nq = B if recall.full else min(B, 64)
        runs = []
        for k1 in sizes:
            t0 = time.perf_counter()
            C = gem.train_codebook(store, k1=k1, iters=10, sample=min(V, 2_000_000), seed=5)
            gem.set_codebook(store, C)
            t_build = time.perf_counter() - t0
            ws2 = gem.Workspace(store, max_queries=B, max_q_rows=rows, max_q_len=32, max_cands=B * R, max_k=R)
            est = torch.empty((nq, store.n_sets), dtype=torch.float32, device=dev)
            qn, qon = q[: 32 * nq], qo[: nq + 1]
            for form in ("symmetric", "asymmetric"):
                gem.set_qch_form(ws2, form)
                ms = _time(lambda: gem.estimate_codes(store, ws2, qn, qon, out=est), reps=1)
                # the whole codes-first search in one call: qCH of every set ->
                # top-R -> exact FP32 rerank -> top-K (Algorithm 5's order)
                ms_s = _time(lambda: gem.search(store, ws2, qn, qon, "codes", rerank_depth=R, k=K), reps=1)
                ids, _ = gem.search(store, ws2, qn, qon, "codes", rerank_depth=R, k=K)
                est_top, _ = gem.search(store, ws2, qn, qon, "codes", rerank_depth=0, k=K)
                assert ws2.status() == 0
                gather_gbs = nq * V * 128 / (ms * 1e-3) / 1e9   # one 128-byte table row per stored vector
                runs.append({"k1": k1, "form": form, "codebook_and_codes_s": t_build, "ms": ms,
                             "pairs_per_s": nq * store.n_sets / (ms * 1e-3), "search_ms": ms_s,
                             "table_gather_gbs": gather_gbs,
                             "frac_of_builder_l2_gather_peak": gather_gbs / bp["l2_gather_gbs"] if bp else None,
                             "recall_at_100_after_rerank": recall(ids.cpu().numpy()),
                             "recall_at_100_of_the_estimate": recall(est_top.cpu().numpy())})
            ws2.close()
        head = runs[0]
        return {"k1": head["k1"], "codebook_and_codes_s": head["codebook_and_codes_s"], "queries": nq,
                "ms": head["ms"], "pairs_per_s": head["pairs_per_s"],
                "recall_at_100_after_rerank": head["recall_at_100_after_rerank"], "runs": runs}

    def cluster():
        # Sec. 4.5.1: C_index = k-means of C_quant (second stage, k2 = 2,048),
        # then C_query of every query set with t = 4
        if getattr(store, "k1", 0) <= 0:
            return {"error": "no codebook (the qch stage trains it)"}
        Cq = store.export("codebook")
        k2, t = 2048, 4
        t0 = time.perf_counter()
        Ci = gem.kmeans(Cq, k2, iters=10, seed=5)
        torch.cuda.synchronize()
        km_s = time.perf_counter() - t0
        ms = _time(lambda: gem.cluster_filter(q, qo, Ci, t=t, max_q_len=32))
        _, lst, cnt = gem.cluster_filter(q, qo, Ci, t=t, max_q_len=32)
        # multi-entry points (Sec. 4.5.2): C_index codes and member lists of the
        # store, then one random member set per cluster of every C_query
        t0 = time.perf_counter()
        gem.set_index_centroids(store, Ci)
        torch.cuda.synchronize()
        idx_s = time.perf_counter() - t0
        ms_e = _time(lambda: gem.entry_points(store, lst, cnt, seed=7))
        seeds = gem.entry_points(store, lst, cnt, seed=7)
        return {"k1": int(Cq.shape[0]), "k2": k2, "t": t, "kmeans_s": km_s, "ms": ms,
                "query_vectors_x_centroids_per_s": rows * k2 / (ms * 1e-3),
                "tflops": 2.0 * rows * k2 * 128 / ms / 1e9, "mean_c_query": float(cnt.float().mean()),
                "index_codes_and_members_s": idx_s, "entry_points_ms": ms_e,
                "entry_points": int((seeds >= 0).sum())}

    def graph_search():
        # Algorithm 5 end to end on a 50,000-set text-shaped store: a 16-NN graph
        # by the BF16 scorer (symmetrised), C_quant (Sec. 5.1 size) and C_index
        # (k2 = 256), cluster filter (t = 4), entry points, beam search (ef = 64),
        # exact FP32 rerank of R, top-10 against the exhaustive FP32 top-10
        n = 50_000
        wg = synth.text_corpus(seed=1240, n_sets=n, n_queries=B, device=dev)
        sg = gem.Store(wg.docs.vecs, wg.docs.offsets, keep=("f32", "bf16"))
        qg = wg.queries.vecs
        qog = torch.from_numpy(wg.queries.offsets).to(dev)
        lens = wg.docs.lengths()
        t0 = time.perf_counter()
        rows_max = max(int(wg.docs.offsets[min(n, a + 5000)] - wg.docs.offsets[a]) for a in range(0, n, 5000))
        wsg = gem.Workspace(sg, max_queries=5000, max_q_rows=rows_max, max_q_len=int(lens.max()), max_k=17)
        nbr = []
        for a in range(0, n, 5000):
            b1 = min(n, a + 5000)
            qd = wg.docs.vecs[int(wg.docs.offsets[a]):int(wg.docs.offsets[b1])]
            qod = torch.from_numpy(wg.docs.offsets[a:b1 + 1] - wg.docs.offsets[a]).to(dev)
            sc = gem.score_all(sg, wsg, qd, qod, "bf16")
            ids, _ = gem.topk(wsg, sc, 17)
            nbr.append(ids.cpu().numpy())
        wsg.close()
        nbr = np.concatenate(nbr)
        src = np.repeat(np.arange(n), nbr.shape[1])
        dst = nbr.ravel()
        keep = dst != src
        a_, b_ = np.concatenate([src[keep], dst[keep]]), np.concatenate([dst[keep], src[keep]])
        key = np.unique(a_.astype(np.int64) * n + b_)
        go = np.zeros(n + 1, dtype=np.int64)
        np.add.at(go, key // n + 1, 1)
        go = np.cumsum(go)
        gn = (key % n).astype(np.int32)
        graph_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        V = sg.n_vecs
        k1 = 1 << int(np.floor(np.log2(16.0 * np.sqrt(V))))
        Cg = gem.train_codebook(sg, k1=k1, iters=10, sample=min(V, 1_000_000), seed=5)
        gem.set_codebook(sg, Cg)
        Ci = gem.kmeans(Cg, 256, iters=10, seed=6)
        gem.set_index_centroids(sg, Ci)
        torch.cuda.synchronize()
        index_s = time.perf_counter() - t0
        # qEMD (Sec. 4.2.2), the paper's edge weight, over the first 100,000 edges
        # whose two sets have at most 128 vectors
        lens_np = np.asarray(lens)
        ok = (lens_np[key // n] <= 128) & (lens_np[key % n] <= 128)
        ea = torch.from_numpy(np.ascontiguousarray((key // n)[ok][:100_000])).to(dev)
        eb = torch.from_numpy(np.ascontiguousarray((key % n)[ok][:100_000])).to(dev)
        wqe = gem.Workspace(sg, max_queries=1, max_q_rows=32, max_q_len=32)
        qe = torch.empty(ea.numel(), dtype=torch.float32, device=dev)
        gem.qemd(sg, wqe, ea[:2000], eb[:2000], out=qe[:2000])
        qemd_ms = _time(lambda: gem.qemd(sg, wqe, ea, eb, out=qe), reps=1)
        assert wqe.status() == 0 and bool(torch.isfinite(qe).all())
        wqe.close()
        wsq = gem.Workspace(sg, max_queries=B, max_q_rows=qg.shape[0], max_q_len=32, max_cands=B * 64, max_k=64)
        go_d, gn_d = torch.from_numpy(go).to(dev), torch.from_numpy(gn).to(dev)
        res = {}

        def search():
            mask, lst, cnt = gem.cluster_filter(qg, qog, Ci, t=4, max_q_len=32)
            ent = gem.entry_points(sg, lst, cnt, seed=11)
            ids, _, rounds = gem.beam_search(sg, wsq, qg, qog, go_d, gn_d, mask, ent, ef=64)
            pool = ids.clamp(min=0).view(-1)
            po = torch.arange(B + 1, dtype=torch.int64, device=dev) * 64
            rs = gem.score_ids(sg, wsq, qg, qog, po, pool, "f32")
            rs = torch.where(ids.view(-1) >= 0, rs, torch.full_like(rs, -float("inf")))
            top, _ = gem.topk(wsq, rs.view(B, 64), 10, ids=ids.contiguous())
            res["rounds"] = rounds
            return top

        search()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        top = search()
        torch.cuda.synchronize()
        ms = 1000 * (time.perf_counter() - t0)
        exact = gem.score_all(sg, wsq, qg, qog, "f32")
        ex10 = torch.topk(exact, 10, dim=1).indices.cpu().numpy()
        rec = float(np.mean([len(set(a.tolist()) & set(e.tolist())) / 10 for a, e in zip(top.cpu().numpy(), ex10)]))
        out = {"n_sets": n, "queries": B, "graph_degree_mean": float(len(gn) / n), "graph_build_s": graph_s,
               "k1": k1, "k2": 256, "index_build_s": index_s, "ef": 64, "t": 4, "rounds": res["rounds"],
               "search_ms": ms, "queries_per_s": B / (ms * 1e-3), "recall_at_10_vs_exact_fp32": rec,
               "qemd_edges": int(ea.numel()), "qemd_ms": qemd_ms, "qemd_pairs_per_s": ea.numel() / (qemd_ms * 1e-3),
               "qemd_mean": float(qe.mean())}
        wsq.close()
        sg.close()
        return out

    def beam():
        nq, rounds = 4096, 20
        qs = synth.vector_sets(synth.lengths_uniform(nq, 8, 64, 1238 + 7919), synth.centres(4096, 1236),
                               1238 + 7919, dev)
        co, ci0 = synth.candidate_lists(nq, store.n_sets, 64, 512, 0.3, 10_000, 1238)
        qv, qoff = qs.vecs, torch.from_numpy(qs.offsets).to(dev)
        co_d = torch.from_numpy(co).to(dev)
        lists = [torch.from_numpy(synth.shift_lists(ci0, r, store.n_sets)).to(dev) for r in range(rounds)]
        ch = gem.autotune_batch(store, qv, qoff, co_d, lists[0], mode="f32", max_q_len=64)
        bt = gem.Batch(store, "f32", max_queries=nq, max_q_rows=qv.shape[0], max_q_len=64, max_cands=len(ci0),
                       seg=ch["seg"], ctas_per_sm=ch["ctas_per_sm"])
        bt.run(qv, qoff, co_d, lists[0])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(rounds):
            bt.run(qv, qoff, co_d, lists[r])
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / rounds
        # flop of one round: 2 m_q m_p 128 per (query, candidate) pair (every round
        # has the same lengths: its ids are a bijection of round 0's)
        dl = np.diff(w.docs.offsets)
        fl = 2.0 * 128 * float(np.sum(np.repeat(np.diff(qs.offsets), np.diff(co)) * dl[ci0]))
        # bit-match of the last round with the per-query path on 8 queries
        got = bt.scores[: len(ci0)].clone()
        ws3 = gem.Workspace(store, max_queries=1, max_q_rows=64, max_q_len=64)
        ok = True
        for b in range(0, nq, nq // 8):
            lo, hi = int(co[b]), int(co[b + 1])
            one = gem.score_ids(store, ws3, qv[qs.offsets[b]:qs.offsets[b + 1]],
                                torch.tensor([0, qs.offsets[b + 1] - qs.offsets[b]], device=dev),
                                torch.tensor([0, hi - lo], device=dev), lists[-1][lo:hi], "f32")
            ok &= bool(torch.equal(one, got[lo:hi]))
        assert bt.status() == 0
        bt.close()
        res = {"queries": nq, "pairs_per_round": int(len(ci0)), "rounds": rounds, "ms_per_round": ms,
               "pairs_per_s": len(ci0) / (ms * 1e-3), "schedule": ch, "bit_match_per_query_path": ok,
               "tflops": fl / (ms * 1e-3) / 1e12,
               "frac_of_builder_fp32_peak": fl / (ms * 1e-3) / 1e12 / bp["fp32_tflops"] if bp else None}
        # the codes form of the same rounds (the qCH estimate per pair), when the
        # store has a codebook (the qch stage trains one)
        try:
            btc = gem.Batch(store, "codes", max_queries=nq, max_q_rows=qv.shape[0], max_q_len=64,
                            max_cands=len(ci0))
        except gem.GemError as e:
            res["codes"] = {"skipped": str(e)[:120]}
            return res
        btc.run(qv, qoff, co_d, lists[0])
        e0.record()
        for r in range(rounds):
            btc.run(qv, qoff, co_d, lists[r])
        e1.record()
        e1.synchronize()
        msc = e0.elapsed_time(e1) / rounds
        gotc = btc.scores[: len(ci0)].clone()
        wsc = gem.Workspace(store, max_queries=nq, max_q_rows=qv.shape[0], max_q_len=64)
        refc = gem.score_ids(store, wsc, qv, qoff, co_d, lists[-1], "codes")
        assert btc.status() == 0 and wsc.status() == 0
        res["codes"] = {"ms_per_round": msc, "pairs_per_s": len(ci0) / (msc * 1e-3),
                        "bit_match_id_list_path": bool(torch.equal(gotc, refc))}
        wsc.close()
        btc.close()
        return res

    def backward():
        wb = synth.contrastive_batch(device=dev)
        nb, per_q = 256, 64
        po = torch.arange(nb + 1, dtype=torch.int64, device=dev) * per_q
        pid = torch.arange(nb * per_q, dtype=torch.int64, device=dev)
        qo5 = torch.from_numpy(wb.queries.offsets).to(dev)
        do5 = torch.from_numpy(wb.docs.offsets).to(dev)
        s, am = gem.maxsim_fwd(wb.queries.vecs, qo5, wb.docs.vecs, do5, po, pid, "bf16", max_q_len=32)
        g = torch.randn_like(s)
        ms_f = _time(lambda: gem.maxsim_fwd(wb.queries.vecs, qo5, wb.docs.vecs, do5, po, pid, "bf16", max_q_len=32))
        ms_b = _time(lambda: gem.maxsim_bwd(wb.queries.vecs, qo5, wb.docs.vecs, do5, po, pid, am, g))
        # algorithmic work: the forward reads every set row once as FP32 and
        # does 2 * m_q * m_p * 128 flop per pair; the backward writes every row of
        # grad_docs and of grad_q once and reads one set row per (pair, query row)
        n_dv = int(wb.docs.n_vecs)
        q_rows = int(wb.queries.offsets[-1])
        fwd_gb = n_dv * 512 / 1e9
        fwd_tf = 2.0 * 32 * n_dv * 128 / (ms_f * 1e-3) / 1e12
        bwd_gb = (n_dv * 512 + q_rows * 512 + nb * per_q * 32 * 512) / 1e9
        pk, kind = _peaks()
        return {"pairs": nb * per_q, "fwd_ms": ms_f, "bwd_ms": ms_b, "doc_vectors": n_dv,
                "fwd": {"algorithmic_gb": fwd_gb, "hbm_gbs": fwd_gb / (ms_f * 1e-3),
                        "frac_of_hbm_peak": fwd_gb / (ms_f * 1e-3) / pk["hbm_gbs"], "tflops": fwd_tf,
                        "frac_of_bf16_peak": fwd_tf / pk["bf16_tflops"], "bound": "hbm",
                        "includes": "query rounding launch + forward kernel"},
                "bwd": {"algorithmic_gb": bwd_gb, "hbm_gbs": bwd_gb / (ms_b * 1e-3),
                        "frac_of_hbm_peak": bwd_gb / (ms_b * 1e-3) / pk["hbm_gbs"], "bound": "hbm",
                        "includes": "dQ kernel + set counts + owner rows + atomic pass"},
                "peak_kind": kind}

    def pages():
        # the multi-modal page configuration: 50,000 sets x 1,024 vectors, 500
        # queries of 16..32 vectors; per dtype: exhaustive time, the pipeline
        # (top-2,000, FP32 rerank, top-100) and its recall against the exact
        # FP32 exhaustive top-100 computed on the GPU
        wp = synth.multimodal_pages(device=dev)
        sp = gem.Store(wp.docs.vecs, wp.docs.offsets, keep=("f32", "bf16", "fp8", "fp8_set"))
        del wp.docs.vecs
        qp = wp.queries.vecs
        qop = torch.from_numpy(wp.queries.offsets).to(dev)
        Bp = qop.numel() - 1
        wsp = gem.Workspace(sp, max_queries=Bp, max_q_rows=qp.shape[0], max_q_len=32, max_cands=Bp * 2000,
                            max_k=2000)
        outp = torch.empty((Bp, sp.n_sets), dtype=torch.float32, device=dev)
        gem.score_all(sp, wsp, qp, qop, "f32", out=outp)
        exact = torch.topk(outp, 100, dim=1).indices.cpu().numpy()
        fl = 2.0 * float(wp.queries.lengths().sum()) * sp.n_vecs * 128
        res = {"n_sets": sp.n_sets, "n_vecs": sp.n_vecs, "queries": Bp}
        for dt in ("bf16", "fp8", "fp8_set"):
            ch = gem.autotune_score_all(sp, wsp, qp, qop, dt, scores=outp)
            ms = _time(lambda: gem.score_all(sp, wsp, qp, qop, dt, out=outp))
            ms_s = _time(lambda: gem.search(sp, wsp, qp, qop, dt, rerank_depth=2000, k=100))
            ids, _ = gem.search(sp, wsp, qp, qop, dt, rerank_depth=2000, k=100)
            res[dt] = {"exhaustive_ms": ms, "tflops_equiv": fl / ms / 1e9, "schedule": ch,
                       "search_ms": ms_s, "doc_sets_per_s": Bp * sp.n_sets / (ms_s * 1e-3),
                       "recall_at_100_vs_exact_fp32": float(np.mean(
                           [len(set(r.tolist()) & set(e.tolist())) / 100 for r, e in zip(ids.cpu().numpy(), exact)]))}
        res["fp32_exhaustive_ms"] = _time(lambda: gem.score_all(sp, wsp, qp, qop, "f32", out=outp), reps=1)
        wsp.close()
        sp.close()
        return res

    def fp32_l2():
        # Sim = -(L2 distance) against the inner product on the FP32 scorer, first
        # 100 queries against every set
        nq = min(B, 100)
        o = torch.empty((nq, store.n_sets), dtype=torch.float32, device=dev)
        qs, qos = q[: 32 * nq], qo[: nq + 1]
        ms_ip = _time(lambda: gem.score_all(store, ws, qs, qos, "f32", out=o), reps=1)
        gem.set_similarity(ws, "l2")
        try:
            ms_l2 = _time(lambda: gem.score_all(store, ws, qs, qos, "f32", out=o), reps=1)
        finally:
            gem.set_similarity(ws, "ip")
        assert ws.status() == 0
        return {"queries": nq, "ip_ms": ms_ip, "l2_ms": ms_l2, "l2_pairs_per_s": nq * store.n_sets / (ms_l2 * 1e-3)}

    def nm_scaling():
        # Sec. 5.4 (effect of N and m): the corpus sampled to 1/8, 1/4 and 1/2 of its
        # sets (the sets are i.i.d., so a prefix is a random sample), or every set cut
        # to the same fraction of its vectors (i.i.d. within a set: a prefix again),
        # one factor at a time; the headline search step (BF16 scoring of every set,
        # top-R, FP32 rerank, top-K) on each, same queries and schedule
        off = w.docs.offsets
        lens = np.diff(off)
        runs = []
        for kind in ("N", "m"):
            for f in (8, 4, 2):
                if kind == "N":
                    sub_off = off[: len(lens) // f + 1].copy()
                    sub = w.docs.vecs[: int(sub_off[-1])]
                else:
                    nl = np.maximum(1, -(-lens // f))
                    sub_off = np.concatenate([[0], np.cumsum(nl)]).astype(np.int64)
                    idx = np.repeat(off[:-1], nl) + (np.arange(int(sub_off[-1])) - np.repeat(sub_off[:-1], nl))
                    sub = w.docs.vecs[torch.from_numpy(idx).to(dev)]
                sp = gem.Store(sub, sub_off, keep=("f32", "bf16"))
                del sub
                wsp = gem.Workspace(sp, max_queries=B, max_q_rows=rows, max_q_len=32, max_cands=B * R, max_k=R)
                if schedule:
                    gem.set_schedule(wsp, schedule["m_tiles"], schedule["chunk_rows"], variant=schedule["variant"])
                ms = _time(lambda: gem.search(sp, wsp, q, qo, "bf16", rerank_depth=R, k=K), reps=2)
                assert wsp.status() == 0
                runs.append({"vary": kind, "fraction": 1.0 / f, "n_sets": sp.n_sets, "n_vecs": sp.n_vecs,
                             "mean_m": sp.n_vecs / sp.n_sets, "search_ms": ms,
                             "doc_sets_per_s": B * sp.n_sets / (ms * 1e-3),
                             "vectors_per_s": B * sp.n_vecs / (ms * 1e-3)})
                wsp.close()
                sp.close()
        runs.append({"vary": "none", "fraction": 1.0, "n_sets": store.n_sets, "n_vecs": store.n_vecs,
                     "mean_m": store.n_vecs / store.n_sets, "search_ms": step_ms,
                     "doc_sets_per_s": B * store.n_sets / (step_ms * 1e-3),
                     "vectors_per_s": B * store.n_vecs / (step_ms * 1e-3)})
        return {"queries": B, "runs": runs}

    def exact_2k():
        # config 1, the parity-sized case (launch-bound, reported, not a bench
        # line): 2,000 sets of 16..64 vectors, 10 queries of 32, top-10 (its
        # parity against the oracle is in the tests; here the BF16 top-10 is
        # compared with the FP32 path's)
        w1 = synth.exact_fp32(device=dev)
        s1 = gem.Store(w1.docs.vecs, w1.docs.offsets, keep=("f32", "bf16"))
        ws1 = gem.Workspace(s1, max_queries=10, max_q_rows=320, max_q_len=32)
        q1, qo1 = w1.queries.vecs, torch.from_numpy(w1.queries.offsets).to(dev)
        res = {"n_sets": s1.n_sets, "queries": 10}
        top = {}
        for dt in ("f32", "bf16"):
            def run():
                return gem.topk(ws1, gem.score_all(s1, ws1, q1, qo1, dt), 10)
            ms1 = _time(run, reps=20)
            top[dt] = run()[0].cpu().numpy()
            res[dt] = {"ms": ms1, "pairs_per_s": 10 * s1.n_sets / (ms1 * 1e-3)}
        res["bf16_top10_overlap_with_f32"] = float(np.mean(
            [len(set(top["bf16"][b].tolist()) & set(top["f32"][b].tolist())) / 10.0 for b in range(10)]))
        ws1.close()
        s1.close()
        return res

    guard("exact_fp32_2k", exact_2k)
    guard("fp8_exhaustive", fp8)
    guard("fp32_exhaustive", fp32)
    guard("pages_50k", pages)
    guard("qch_estimate", qch)
    guard("cluster_filter", cluster)
    guard("graph_search", graph_search)
    guard("beam_batch", beam)
    guard("backward", backward)
    guard("nm_scaling", nm_scaling)
    guard("fp32_l2", fp32_l2)


def run_reference(args, dist, rank, world):
    """The oracle as the reference arm: host cores, bounded sample per step."""
    if rank != 0:
        return
    cfg = WORKLOADS[args.workload]
    w = synth.text_corpus(n_sets=20_000, n_queries=max(args.steps + args.warmup, 1), device="cpu")
    per_step = []
    for s in range(args.warmup + args.steps):
        r, _ = cpu_baseline(w.docs.vecs, w.docs.offsets, w.queries.vecs[32 * s: 32 * (s + 1)],
                            np.array([0, 32]), 1, cfg["k"])
        if s >= args.warmup:
            per_step.append(r)
    value = statistics.mean(r["value"] for r in per_step)
    ms = 1000.0 * statistics.mean(r["seconds"] for r in per_step)
    # the GEM arm's workload (same sizes and recipe), of which each step scores a sample
    V = int(synth.lengths_lognormal(cfg["n_sets"], 70.0, 0.5, 20, 180, 1236).sum())
    B, R, K = cfg["n_queries"], cfg["rerank"], cfg["k"]
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "doc-sets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"text-corpus {cfg['n_sets']} sets / {V} vectors, {B} queries x 32, "
                                   f"top-{R} -> FP32 rerank -> top-{K}",
                       "n_sets": cfg["n_sets"], "n_vecs": V, "queries": B, "m_q": 32, "rerank": R, "k": K,
                       "sample_per_step": "1 query x the first 20,000 sets of the same recipe, drawn on the host; "
                                          "exact CH (FP64) + top-100"},
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
                                      rank_query_seed(seed, rank), dev)
    store = gem.Store(w.docs.vecs, w.docs.offsets, keep=("f32", "bf16", "fp8", "fp8_set"))
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
    pool_sc = torch.empty(B * R, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    if args.schedule:
        mt, var, cr = args.schedule.split(",")
        gem.set_schedule(ws, int(mt), int(cr), variant=var)
        schedule = {"m_tiles": int(mt), "variant": var, "chunk_rows": int(cr), "fixed": True}
    else:
        schedule = gem.autotune_score_all(store, ws, q, qo, "bf16", scores=scores)

    def step(ev=None):
        if ev:
            ev[0].record(st)
        gem.score_all(store, ws, q, qo, "bf16", out=scores)
        if ev:
            ev[1].record(st)
        pid, _ = gem.topk(ws, scores, R)
        pool_ids.copy_(pid)
        if ev:
            ev[3].record(st)
        gem.rerank_pool(store, ws, q, qo, pool_ids, out=pool_sc.view(B, R))
        if ev:
            ev[4].record(st)
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
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
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
    launches = gem.lib.gem_kernel_launches() - launches0   # the library's launches in the timed region
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
    # each step is a fraction of a second: the burst peak is the denominator; the
    # fraction of the sustained (seconds-long, power-capped) peak is reported beside it
    peak = peaks["bf16_tflops"]
    key = (schedule["m_tiles"], schedule["variant"], schedule["chunk_rows"])
    line = {
        "metric": METRIC,
        "value": world * n_pairs / (ms * 1e-3), "unit": "doc-sets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"text-corpus {store.n_sets} sets / {V} vectors, {B} queries x 32, "
                               f"top-{R} -> FP32 rerank -> top-{K}",
                   "n_sets": store.n_sets, "n_vecs": V, "queries": B, "m_q": 32, "rerank": R, "k": K,
                   "l2": "inputs larger than L2 (bf16 store %.2f GB)" % (V * 256 / 1e9)},
        "stages": {"maxsim_bf16_ms": k1_ms,
                   "topk_rerank_topk_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in evs),
                   "topk_1000_of_500k_ms": statistics.mean(e[1].elapsed_time(e[3]) for e in evs),
                   "fp32_rerank_ms": statistics.mean(e[3].elapsed_time(e[4]) for e in evs),
                   "topk_100_of_1000_ms": statistics.mean(e[4].elapsed_time(e[2]) for e in evs)},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": (TC_TRAFFIC_RATIO[key] * (V * 256 + n_pairs * 4) if key in TC_TRAFFIC_RATIO
                                 else None),
                     "traffic_basis": "ncu DRAM bytes of one launch on the medium case (1,000 x 50,000 sets), "
                                      "as a ratio to algorithmic bytes, times this run's algorithmic bytes",
                     "frac_of_sustained_peak": achieved / peaks["bf16_tflops_sustained"],
                     "algorithmic_bytes": V * 256 + n_pairs * 4,
                     "kernel": "tc_score_all_kernel<%d,bf16,%s> (+ query packing)" % (schedule["m_tiles"], schedule["variant"]),
                     "peak_kind": f"{peak_kind} bf16 dense burst"},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": int(launches) // max(1, args.steps),
        "clocks": clk,
        "e2e": {"value": world * n_pairs / (e2e_ms * 1e-3), "unit": "doc-sets/s",
                "h2d_bytes_per_step": int(qh.numel() * 4 + qoh.numel() * 8),
                "d2h_bytes_per_step": int(oi.numel() * 8 + osc.numel() * 4)},
    }
    line["config"]["schedule"] = schedule
    bp = None
    if rank == 0:
        # builder-measured denominators of the FP32 and L2-gather kernels
        bp = gem.measure_peaks()
        line["builder_peaks"] = dict(bp, how="gem_measure_peaks on this GPU in this run: packed FP32 FMA chains "
                                              "over a full grid; 128-byte row gathers from a 64 MB L2-resident "
                                              "buffer (best of three launches)")
        lens_d = torch.from_numpy(np.diff(w.docs.offsets)).to(dev)
        pool_vecs = float(lens_d[pool_ids.view(-1)].sum())
        rr_ms = line["stages"]["fp32_rerank_ms"]
        tk_ms = line["stages"]["topk_1000_of_500k_ms"]
        rr = 2.0 * 32 * 128 * pool_vecs / (rr_ms * 1e-3) / 1e12
        tk = n_pairs * 4 / (tk_ms * 1e-3) / 1e9
        line["rooflines_other"] = {
            "fp32_rerank": {"kernel": "f32_ids_stream_kernel", "bound": "alu", "achieved": rr,
                            "peak": bp["fp32_tflops"], "unit": "TFLOP/s", "frac": rr / bp["fp32_tflops"],
                            "peak_kind": "builder-measured FP32 FMA", "gathered_gb": pool_vecs * 512 / 1e9,
                            # how much a doc-major grouping of the pool could save: the
                            # FP32 bytes of the distinct sets against those gathered
                            "distinct_sets": int(torch.unique(pool_ids).numel()),
                            "distinct_gb": float(lens_d[torch.unique(pool_ids)].sum()) * 512 / 1e9},
            "topk_1000_of_500k": {"kernel": "topk_sample/filter/select", "bound": "hbm", "achieved": tk,
                                  "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": tk / peaks["hbm_gbs"],
                                  "peak_kind": f"{peak_kind} HBM copy", "algorithmic_gb": n_pairs * 4 / 1e9}}
    truth = []
    full_truth, truth_note = (load_truth(w) if rank == 0 and args.workload == "text"
                              else (None, "not the text-corpus workload"))
    if rank == 0 and not args.no_cpu_baseline:
        docs_host = w.docs.vecs.cpu()
        line["cpu_baseline"], truth = cpu_baseline(docs_host, w.docs.offsets, w.queries.vecs.cpu(),
                                                   w.queries.offsets, args.cpu_queries, K, one_thread=True)
        del docs_host

    def recall(found):
        """recall@100 against the exact FP64 top-100: the stored ground truth of
        all queries when it matches this data, else the oracle's sample above."""
        if full_truth is not None:
            ids, sc = full_truth
            r = recall_vs_truth(found, (ids[: found.shape[0]], sc[: found.shape[0]]))
            r["reference"] = "stored exact FP64 top-100 of every query (tests/golden/text500k_truth.npz)"
            return r
        n = min(len(truth), found.shape[0])
        return {"recall": _recall(found, truth[:n]) if n else None, "queries": n,
                "reference": f"oracle top-100 of the first {n} queries ({truth_note})"}
    recall.full = full_truth is not None
    if rank == 0 and (full_truth is not None or truth):
        line["recall_at_100"] = {"bf16_rerank": recall(ids_a.cpu().numpy())}
    if rank == 0 and not args.no_extras:
        stages = line["stages"]
        extra_stages(gem, store, ws, w, q, qo, R, K, recall, stages, dev, ms,
                     only=set(args.stages.split(",")) if args.stages else None, qch_k1=args.qch_k1,
                     schedule=schedule, bp=bp)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gem", choices=["gem", "reference"])
    ap.add_argument("--workload", default="text", choices=list(WORKLOADS))
    ap.add_argument("--cpu-queries", type=int, default=4, help="queries the FP64 oracle scores (ground truth)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the per-row stage measurements")
    ap.add_argument("--stages", default="", help="comma-separated extra stages to run (default: all)")
    ap.add_argument("--qch-k1", default="", help="comma-separated codebook sizes for the qch stage "
                    "(default: the Sec. 5.1 formula)")
    ap.add_argument("--schedule", default="", help="fixed tensor-core schedule 'm_tiles,variant,chunk_rows' "
                    "instead of the autotuner (for profiling)")
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
