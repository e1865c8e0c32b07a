#!/usr/bin/env python
"""Benchmark: PiPNN index build (Alg. 4) on GB300, points per second.

One step = one full build (sketches, partition, leaf all-pairs + pick, HashPrune, final prune) of
the spacev-like-i8 workload: 100,000,000 points x 128 int8 (10,000-cluster mixture, the largest
workload that fits one GPU), squared L2, C_max 2048, l_max 64, R 64, multi-level fanout [10, 3],
k = 2, m = 12 hash bits, alpha 1.2, the leaf step in memory-bounded waves and HashPrune once per
group of waves.  The
input is resident in HBM when a step starts (and far larger than L2); L2 is also flushed (256 MB
write) before every step, outside the timed events.  Each rank builds its own independently
seeded instance (independent indexes: no collective on the data path), so the job's throughput is
the number of points all ranks built divided by the slowest rank's time.

Beside the headline line (rank 0, one GPU) the JSON carries: recall@10 of the 100M graph on a
sample of the workload's queries; the 1M-point bigann-like-u8 build with its recall gate against
the oracle's graph (the oracle cannot build 100M points inside a run); and the 1M-point
deep-like-ip float build at every leaf precision with each precision's error against FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--engine tc|simt]
                  [--impl reference]

--impl reference times the CPU oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "spacev-like-i8"
CONTEXT = "bigann-like-u8"
METRIC = "build points/sec at recall@10>=oracle-0.3pp; GEMM tensor-pipe % and prune HBM GB/s"
CPU_SAMPLE = 200_000
CONTEXT_CPU_SAMPLE = 50_000
REF_SAMPLE = 20_000
HEADLINE_QUERIES = 200
DTYPE_NAME = {synth.F32: "f32", synth.U8: "u8", synth.I8: "i8"}


def workload_params(w):
    return dict(c_max=w["c_max"], l_max=w["l_max"], R=w["R"], fanout=tuple(w["fanout"]))


def config_dict(name, w, engine, n):
    return {"workload": name, "n": n, "d": w["d"], "dtype": DTYPE_NAME[w["dtype"]],
            "metric": "IP" if w["metric"] == synth.IP else "L2", "c_max": w["c_max"], "c_min": w["c_max"] // 16,
            "l_max": w["l_max"], "R": w["R"], "fanout": list(w["fanout"]), "leaf_k": 2, "hash_bits": 12,
            "alpha": 1.2, "p_samp": 0.005, "max_leaders": 1000, "leaf_engine": engine,
            "l2": "flushed before every step (256 MB write); inputs larger than L2", "input": "resident in HBM",
            "data": "synthetic, seeded per rank"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def profiled_traffic(kernel_file, profile_file):
    """DRAM bytes per build of a kernel recorded by an ncu capture (scaled to the bench's build),
    if that capture is of the current source."""
    src = os.path.join(ROOT, "paper_2602_21247_gb300", "csrc", kernel_file)
    prof = os.path.join(ROOT, "profiles", profile_file)
    if not (os.path.exists(src) and os.path.exists(prof)):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    text = open(prof).read()
    m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_build:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_data_seed(w, rank):
    """Every rank builds its own seeded instance of the workload (replicas only: no exchange)."""
    return w["data_seed"] + 7919 * rank


def max_over_ranks(x, world, device):
    """The largest of every rank's x: the whole job takes as long as its slowest rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank, world, seconds):
    """Points built per second by the whole job (world ranks, n_per_rank points each)."""
    return world * n_per_rank / seconds


def cpu_baseline(X, H, w, name, n_sample):
    import oracle  # the CPU oracle: timed here as a reported baseline only

    n = min(n_sample, X.shape[0])
    bp = oracle.params(**workload_params(w))
    t = time.perf_counter()
    oracle.build(np.ascontiguousarray(X[:n]), bp, H, synth.BUILD_SEED, metric=w["metric"])
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "points/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"first {n:,} points of the {name} workload, full Alg. 4 build ({dt:.1f} s)"}


RECALL_L = (16, 32, 64, 128)


KNN_L = (16, 32, 64)


def multi_index_block(pk, steps):
    """The multi-index workload: 512 independent float indexes (sizes log-uniform in 2,000 ..
    200,000, 128-d, L2; C_max 1024, l_max 64, R 48, fanout [2]) built by one batched pipeline
    (pipnn_build_batched), timed with CUDA events, against a loop of one pipnn_build per index
    over the same points; every batched graph is checked equal to its single build."""
    import torch

    sizes = synth.multi_index_sizes()
    d = 128
    pts = [synth.mixture_device(int(s), d, synth.F32, max(10, int(s) // 200), 0.3, 10000 + i)
           for i, s in enumerate(sizes)]
    H = torch.from_numpy(synth.hyperplanes(12, d)).cuda()
    bp = pk.params(dtype=pk.PIPNN_F32, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, prec=pk.PIPNN_PREC_BF16X3,
                   c_max=1024, l_max=64, R=48, fanout=(2,))
    seeds = [synth.BUILD_SEED] * len(sizes)
    total = int(sizes.sum())

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    pk.pipnn_build_batched(pts, bp, seeds)
    ms_b = []
    for _ in range(steps):
        graphs, ms = timed(lambda: pk.pipnn_build_batched(pts, bp, seeds))
        ms_b.append(ms)
    pk.pipnn_build(pts[0], bp, seeds[0])
    serial, ms_s = timed(lambda: [pk.pipnn_build(p, bp, sd) for p, sd in zip(pts, seeds)])
    same = all(torch.equal(ga, sa) and torch.equal(gd, sd_) for (ga, gd), (sa, sd_) in zip(graphs, serial))
    mb = statistics.mean(ms_b)
    return {"indexes": len(sizes), "points": total, "d": d, "dtype": "f32", "metric": "L2", "c_max": 1024,
            "l_max": 64, "R": 48, "fanout": [2], "leaf_engine": "tc", "prec": "bf16x3",
            "batched": {"ms": mb, "points_per_s": total / (mb / 1e3), "steps": steps},
            "serial_loop": {"ms": ms_s, "points_per_s": total / (ms_s / 1e3)},
            "speedup": ms_s / mb, "batched_graphs_equal_single_builds": bool(same),
            "data": "synthetic: index i drawn with seed 10000 + i, max(10, n_i / 200) centres, sigma 0.3"}


def knn_graph_block(pk, Xd, X, adj, deg, steps, n_sample=2000):
    """The k-NN graph application of Sec. 5 on the built graph: every point runs Alg. 1 on the GPU
    with itself as the query and keeps its 10 nearest others (pipnn_knn_graph), timed with CUDA
    events for several beam widths; recall@10 against the exact 10-NN (without self) of a sample of
    points; the GPU start (pipnn_medoid) checked against the oracle's."""
    import oracle
    import torch

    start = pk.pipnn_medoid(Xd)
    start_o = oracle.medoid(X)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(X.shape[0], n_sample, replace=False))
    t = time.perf_counter()
    gt = oracle.knn_bytes(X, X[sample], 11)
    t_gt = time.perf_counter() - t
    gt10 = [[int(j) for j in r if j != p][:10] for r, p in zip(gt, sample)]
    rows = []
    for L in KNN_L:
        pk.pipnn_knn_graph(Xd, adj, deg, L, k=10, start=start)
        ms = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            knn, nd = pk.pipnn_knn_graph(Xd, adj, deg, L, k=10, start=start)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        kh = knn.view(torch.int32).cpu().numpy().view(np.uint32)[sample]
        rec = float(np.mean([len(set(a.tolist()) & set(b)) / 10 for a, b in zip(kh, gt10)]))
        m = statistics.mean(ms)
        rows.append({"L": L, "ms": m, "points_per_s": X.shape[0] / (m / 1e3), "recall_at_10": rec,
                     "evaluations_per_point": nd / X.shape[0]})
    return {"k": 10, "start": "medoid (exact, GPU)", "start_equals_oracle": bool(start == start_o),
            "sample": f"recall over {n_sample} random points against exact 10-NN without self ({t_gt:.1f} s)",
            "runs": rows}


def recall_gate(X, H, w, adj_gpu, deg_gpu, n_queries, Xd=None, pk=None):
    """The metric's gate, measured outside the timed region: the oracle builds the same graph
    (Alg. 4 on the same points, parameters and seed); both graphs are searched with the oracle's
    beam search (Alg. 1) from the medoid at every beam width L for the workload's queries, and
    recall@10 (Def. 2) is taken against exact ground truth.  The oracle build is also timed as the
    CPU baseline (the full workload, not a sample)."""
    import oracle

    bp = oracle.params(**workload_params(w))
    t = time.perf_counter()
    adj_o, deg_o, _ = oracle.build(X, bp, H, synth.BUILD_SEED)
    dt = time.perf_counter() - t
    cpu = {"value": X.shape[0] / dt, "unit": "points/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
           "sample": f"the full {X.shape[0]:,}-point {CONTEXT} workload, full Alg. 4 build ({dt:.1f} s)"}
    identical = bool(np.array_equal(deg_o, deg_gpu) and np.array_equal(adj_o, adj_gpu))
    rows_differ = int(((adj_o != adj_gpu).any(axis=1) | (deg_o != deg_gpu)).sum())
    Q = synth.queries(CONTEXT, n_queries)
    t = time.perf_counter()
    gt = oracle.knn_bytes(X, Q, 10)
    t_gt = time.perf_counter() - t
    start = oracle.medoid(X)
    rec_g, rec_o, same_search = [], [], []
    for L in RECALL_L:
        ids_g, _ = oracle.beam_search(X, adj_gpu, deg_gpu, Q, L, start=start)
        ids_o, _ = oracle.beam_search(X, adj_o, deg_o, Q, L, start=start)
        rec_g.append(oracle.recall(ids_g, gt))
        rec_o.append(oracle.recall(ids_o, gt))
        if pk is not None:
            # the GPU's Alg. 1 on the GPU graph returns the oracle's results query for query
            import torch

            adj_t = torch.from_numpy(adj_gpu.view(np.int32)).cuda().view(torch.uint32)
            deg_t = torch.from_numpy(deg_gpu.view(np.int32)).cuda().view(torch.uint32)
            ids_d, _ = pk.pipnn_beam_search(Xd, adj_t, deg_t, torch.from_numpy(Q).cuda(), L, k=10, start=start)
            same_search.append(bool(np.array_equal(ids_d.view(torch.int32).cpu().numpy().view(np.uint32), ids_g)))
    gate = all(g >= o - 0.003 for g, o in zip(rec_g, rec_o))
    rec = {"k": 10, "L": list(RECALL_L), "gpu": rec_g, "oracle": rec_o, "gate_pp": 0.3, "pass": gate,
           "graph_identical_to_oracle": identical, "rows_differing": rows_differ, "queries": int(Q.shape[0]),
           "start": "medoid", "ground_truth": f"exact 10-NN by (L2, id) ({t_gt:.1f} s)"}
    if same_search:
        rec["gpu_beam_search_identical_to_oracle"] = same_search
    return rec, cpu


PREC_MODES = (("fp32", "simt", 0), ("bf16x3", "tc", 4), ("bf16", "tc", 1), ("fp8", "tc", 2))


def precision_modes(steps, warmup, n_queries=1000, error_leaves=48):
    """The deep-like-ip workload (1M x 96 float32, unit norm, inner product) built with every leaf
    precision: the defining FP32 evaluation on the CUDA cores, and the tensor-core Gram at split
    BF16 (three BF16 products), BF16 and FP8 e4m3, each with its exact FP32 re-rank.  Reports
    points/s per mode, whether each graph equals the FP32 one, the rows whose error band did not
    fit and were evaluated in full, the recall@10 of the (shared) graph, and the error of each
    mode's leaf dissimilarities against FP64 on a sample of the partition's leaves."""
    import torch

    import oracle
    import paper_2602_21247_gb300 as pk

    name = "deep-like-ip"
    w = synth.WORKLOADS[name]
    X, Q = synth.workload(name, n_queries=n_queries)
    n, d = X.shape
    H = synth.hyperplanes(12, d)
    Xd = torch.from_numpy(X).cuda()
    Hd = torch.from_numpy(H).cuda()
    kw = workload_params(w)
    R = w["R"]
    adj = torch.empty((n, R), dtype=torch.int32, device="cuda")
    deg = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    out = {"workload": name, "n": n, "d": d, "metric": "IP", "c_max": w["c_max"], "l_max": w["l_max"], "R": R,
           "fanout": list(w["fanout"]), "modes": {}}
    ref = None
    for mode, eng, prec in PREC_MODES:
        bp = pk.params(dtype=pk.PIPNN_F32, hyperplanes=Hd, prec=prec,
                       leaf_engine=pk.PIPNN_LEAF_TC if eng == "tc" else pk.PIPNN_LEAF_SIMT, **kw)
        for _ in range(warmup):
            pk.pipnn_build_into(Xd, bp, synth.BUILD_SEED, adj, deg, metric=w["metric"])
        torch.cuda.synchronize()
        times, stats = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pk.pipnn_build_into(Xd, bp, synth.BUILD_SEED, adj, deg, metric=w["metric"])
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(pk.pipnn_get_stats())
        a_np = adj.cpu().numpy().view(np.uint32)
        d_np = deg.cpu().numpy().view(np.uint32)
        if ref is None:
            ref = (a_np.copy(), d_np.copy())
            same = True
        else:
            same = bool(np.array_equal(a_np, ref[0]) and np.array_equal(d_np, ref[1]))
        ms = statistics.mean(times)
        st = stats[-1]
        out["modes"][mode] = {"engine": eng, "ms_per_step": ms, "points_per_s": n / (ms / 1e3),
                              "ms_leaf": statistics.mean(x["ms_leaf"] for x in stats),
                              "ms_leaf_kernel": statistics.mean(x["ms_leaf_kernel"] for x in stats),
                              "rows_evaluated_in_full": int(st["leaf_full_rows"]),
                              "leaf_rows": int(st["leaf_members"]), "graph_equals_fp32": same}
    # recall of the graph (every mode's graph is the FP32 one when graph_equals_fp32 holds)
    gt = oracle.knn(X, Q, 10, metric=w["metric"])
    start = oracle.medoid(X, metric=w["metric"])
    out["recall_at_10"] = {str(L): oracle.recall(oracle.beam_search(X, ref[0], ref[1], Q, L, start=start,
                                                                    metric=w["metric"])[0], gt) for L in RECALL_L}
    out["recall_queries"] = int(Q.shape[0])
    # leaf dissimilarity error against FP64 on a sample of the partition's leaves
    bp = pk.params(dtype=pk.PIPNN_F32, hyperplanes=Hd, **kw)
    off, mem, _ = pk.pipnn_partition(Xd, bp, synth.BUILD_SEED, metric=w["metric"])
    off_h = off.view(torch.int64).cpu().numpy()
    mem_h = mem.view(torch.int32).cpu().numpy().view(np.uint32)
    pick = np.linspace(0, len(off_h) - 2, error_leaves).astype(np.int64)
    sub_off = [0]
    sub_mem = []
    for b in pick:
        sub_mem.append(mem_h[off_h[b]:off_h[b + 1]])
        sub_off.append(sub_off[-1] + len(sub_mem[-1]))
    sub_mem = np.concatenate(sub_mem).astype(np.uint32)
    sub_off = np.array(sub_off, np.uint64)
    D64, D32 = [], []
    for b in range(len(pick)):
        Xl = X[sub_mem[sub_off[b]:sub_off[b + 1]]]
        G = Xl.astype(np.float64) @ Xl.astype(np.float64).T
        D64.append(1.0 - G)
        s_ = Xl.shape[0]
        ii, jj = np.meshgrid(np.arange(s_), np.arange(s_), indexing="ij")
        ids = sub_mem[sub_off[b]:sub_off[b + 1]]
        D32.append(oracle.dissimilarity(X, ids[ii.ravel()], ids[jj.ravel()], metric=w["metric"]).reshape(s_, s_))

    def err_stats(approx):
        ab, rel = [], []
        for b in range(len(pick)):
            m_ = ~np.eye(D64[b].shape[0], dtype=bool)
            e = np.abs(approx[b] - D64[b])[m_]
            ab.append(e)
            rel.append(e / np.maximum(np.abs(D64[b][m_]), 1e-12))
        ab, rel = np.concatenate(ab), np.concatenate(rel)
        return {"max_abs": float(ab.max()), "mean_abs": float(ab.mean()), "max_rel": float(rel.max()),
                "mean_rel": float(rel.mean())}

    errs = {"fp32": err_stats(D32)}
    for mode, eng, prec in PREC_MODES[1:]:
        g = pk.pipnn_leaf_gram(Xd, torch.from_numpy(sub_off).cuda(), torch.from_numpy(sub_mem).cuda(), prec,
                               metric=w["metric"]).cpu().numpy()
        blocks, at = [], 0
        for b in range(len(pick)):
            s_ = int(sub_off[b + 1] - sub_off[b])
            blocks.append(g[at:at + s_ * s_].reshape(s_, s_).astype(np.float64))
            at += s_ * s_
        errs[mode] = err_stats(blocks)
    out["distance_error_vs_fp64"] = errs
    out["error_sample"] = f"{len(pick)} leaves of the partition, {int(sum(x.size for x in D64)):,} ordered pairs"
    return out


def timed_builds(pk, Xd, bp, adj, deg, steps, warmup, metric, barrier, sampler=None):
    """W untimed builds, then K builds each bracketed by CUDA events on the current stream (L2
    flushed before each, outside the events).  Returns the per-step ms and the library's stats."""
    import torch

    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")  # 256 MB > 129 MB L2
    for _ in range(warmup):
        pk.pipnn_build_into(Xd, bp, synth.BUILD_SEED, adj, deg, metric=metric)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stats = []
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        pk.pipnn_build_into(Xd, bp, synth.BUILD_SEED, adj, deg, metric=metric)
        evs[i][1].record(stream)
        stats.append(pk.pipnn_get_stats())
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    del flush
    return [a.elapsed_time(b) for a, b in evs], stats, clocks


def leaf_roofline(stats, d, engine, kernel_file, profile_file):
    """The leaf all-pairs kernel against the burst BF16 peak: unique-pair flops of every build
    (sum over leaves of |b| (|b| - 1) d) over the kernel time of that build (summed over its
    launches, one per wave)."""
    flops = sum(s["leaf_pairs"] * d for s in stats)
    ms = sum(s["ms_leaf_kernel"] for s in stats)
    launches = sum(s["leaf_kernel_launches"] for s in stats)
    peaks, peak_kind = measured_peaks()
    # the kernel runs for milliseconds to a second inside a build: the burst peak applies
    peak = peaks["bf16_tflops"]
    achieved = flops / (ms / 1e3) / 1e12
    per_build = profiled_traffic(kernel_file, profile_file) if engine == "tc" else None
    # DRAM bytes of the kernel per launch (a build launches it once per wave)
    traffic = per_build / (launches / len(stats)) if per_build else None
    return {"kernel": "leaf all-pairs Gram + k-NN pick (" + engine + ")", "bound": "tensor", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": f"{peak_kind} bf16 burst",
            "traffic": traffic, "algorithmic_flops_per_build": flops / len(stats),
            "ms_per_build": ms / len(stats), "launches_per_build": launches / len(stats)}


def prune_roofline(stats, w, n):
    """The final prune's kernel (A6) against the measured HBM copy bandwidth: per build, every
    reservoir slot read (8 B) with its candidate's vector gathered in the stored element type, the
    node's own vector, count, adjacency row and degree -- over the kernel's launch time."""
    elem = 4 if w["dtype"] == synth.F32 else 1
    d, R = w["d"], w["R"]
    bytes_ = [s["reservoir_slots"] * (8 + d * elem) + n * (d * elem + 4 + R * 4 + 4) for s in stats]
    ms = sum(s["ms_prune_kernel"] for s in stats)
    peaks, kind = measured_peaks()
    achieved = sum(bytes_) / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    return {"kernel": "final RobustPrune (prune_tc_kernel)" if w["dtype"] != synth.F32 else "final RobustPrune",
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{kind} HBM copy", "traffic": None,
            "algorithmic_bytes_per_build": sum(bytes_) / len(stats), "ms_per_build": ms / len(stats),
            "reservoir_slots_per_build": sum(s["reservoir_slots"] for s in stats) / len(stats)}


def phases(stats):
    return {k: statistics.mean(s[k] for s in stats)
            for k in ("ms_sketch", "ms_partition", "ms_leaf", "ms_hashprune", "ms_prune")}


def context_block(pk, steps, warmup, engine, n_queries, cpu_sample, recall=True, knn=True):
    """The 1M-point bigann-like-u8 build (the configuration the oracle can build inside a run):
    points/s, and the recall gate against the oracle's graph of the same points."""
    import torch

    w = dict(synth.WORKLOADS[CONTEXT])
    X = synth.mixture(w["n"], w["d"], w["dtype"], w["centers"], w["sigma"], w["data_seed"])
    H = synth.hyperplanes(12, w["d"])
    Xd = torch.from_numpy(X).cuda()
    eng = pk.PIPNN_LEAF_TC if engine == "tc" else pk.PIPNN_LEAF_SIMT
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=torch.from_numpy(H).cuda(), leaf_engine=eng, **workload_params(w))
    n, R = w["n"], w["R"]
    adj = torch.empty((n, R), dtype=torch.int32, device="cuda")
    deg = torch.empty(n, dtype=torch.int32, device="cuda")
    times, stats, _ = timed_builds(pk, Xd, bp, adj, deg, steps, warmup, w["metric"], lambda: None)
    ms = statistics.mean(times)
    out = {"config": config_dict(CONTEXT, w, engine, n), "value": n / (ms / 1e3), "unit": "points/s",
           "ms_per_step": ms, "steps": steps, "phases_ms": phases(stats),
           "roofline": leaf_roofline(stats, w["d"], engine, "leaf_tc.cu", "leaf_gram_tc_bigann-like-u8.md"),
           "roofline_prune": prune_roofline(stats, w, n)}
    if recall:
        adj_g = adj.cpu().numpy().view(np.uint32)
        deg_g = deg.cpu().numpy().view(np.uint32)
        out["recall"], out["cpu_baseline"] = recall_gate(X, H, w, adj_g, deg_g, n_queries, Xd, pk)
    else:
        out["cpu_baseline"] = cpu_baseline(X, H, w, CONTEXT, cpu_sample)
    if knn:
        import torch

        out["knn_graph"] = knn_graph_block(pk, Xd, X, adj.view(torch.uint32), deg.view(torch.uint32), steps)
    del Xd, adj, deg
    return out


def headline_recall(Xh, adj_h, deg_h, w, n_queries):
    """Recall@10 (Def. 2) of the GPU graph of the headline workload under the oracle's beam search
    (Alg. 1) from the medoid, on a sample of the workload's queries, against exact ground truth."""
    import oracle

    Q = synth.queries_device(n_queries, w["d"], w["dtype"], w["centers"], w["sigma"], w["data_seed"],
                             w["query_seed"])
    t = time.perf_counter()
    gt = oracle.knn_bytes(Xh, Q, 10, chunk=n_queries, db_chunk=1 << 20)
    t_gt = time.perf_counter() - t
    start = oracle.medoid(Xh)
    rec = [oracle.recall(oracle.beam_search(Xh, adj_h, deg_h, Q, L, start=start)[0], gt) for L in RECALL_L]
    return {"k": 10, "L": list(RECALL_L), "gpu": rec, "oracle": None, "queries": int(Q.shape[0]), "start": "medoid",
            "ground_truth": f"exact 10-NN by (L2, id) over all points ({t_gt:.1f} s)",
            "oracle_graph": "not built at this size (hours on the host); the oracle-gated recall is in "
                            "the bigann_like_u8 block, and the wave-split build equals the oracle's graph "
                            "in the parity tests"}


def run_reference(args, w):
    """Reference arm: the CPU oracle as it stands, on bounded samples of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    n = REF_SAMPLE
    X = synth.mixture(n, w["d"], w["dtype"], w["centers"], w["sigma"], w["data_seed"])
    H = synth.hyperplanes(12, w["d"])
    bp = oracle.params(**workload_params(w))
    for _ in range(args.warmup):
        oracle.build(X, bp, H, synth.BUILD_SEED, metric=w["metric"])
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.build(X, bp, H, synth.BUILD_SEED, metric=w["metric"])
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = n / (ms / 1e3)
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[w["dtype"]], "data": "synthetic",
            "config": {**config_dict(args.workload, w, "cpu-oracle", w["n"]),
                       "sample": f"{n:,} points of the workload's mixture per step"},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n:,} points of the {args.workload} workload's mixture per step"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def make_points(name, w, n, rank):
    """The workload's points on the device: drawn on the GPU for the 100M workload (its host draw
    would take minutes), else drawn on the host and copied."""
    import torch

    seed = rank_data_seed(w, rank)
    if n > 20_000_000:
        return synth.mixture_device(n, w["d"], w["dtype"], w["centers"], w["sigma"], seed,
                                    normalize=w["metric"] == synth.IP)
    X = synth.mixture(n, w["d"], w["dtype"], w["centers"], w["sigma"], seed, normalize=w["metric"] == synth.IP)
    return torch.from_numpy(X).cuda()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--engine", default="tc", choices=["tc", "simt"])
    ap.add_argument("--prec", default=None, choices=["fp32", "bf16", "fp8", "bf16x3"],
                    help="leaf precision for float workloads (default bf16x3 on the tc engine)")
    ap.add_argument("--n", type=int, default=None, help="override the workload size (tests)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-recall", action="store_true", help="skip the recall measurements")
    ap.add_argument("--no-context", action="store_true", help="skip the 1M bigann-like-u8 block")
    ap.add_argument("--no-knn", action="store_true", help="skip the k-NN graph application in that block")
    ap.add_argument("--no-multi-index", action="store_true", help="skip the 512-index batched block")
    ap.add_argument("--no-precision-modes", action="store_true",
                    help="skip the float workload built at every leaf precision")
    ap.add_argument("--queries", type=int, default=None, help="queries of the recall measurement")
    ap.add_argument("--profile", action="store_true", help="timed steps only (for profiler launch lists)")
    ap.add_argument("--wave-members", type=int, default=0,
                    help="with --profile: leaf members per wave (0: sized from free memory)")
    ap.add_argument("--merge-waves", type=int, default=0,
                    help="with --profile: leaf waves per HashPrune merge (0: sized from free memory)")
    ap.add_argument("--profile-knn", action="store_true",
                    help="with --profile: also one k-NN graph construction on the built graph (byte data)")
    args = ap.parse_args()
    w = dict(synth.WORKLOADS[args.workload])
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import torch.distributed as dist

    import paper_2602_21247_gb300 as pk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    n = args.n or w["n"]
    Xd = make_points(args.workload, w, n, rank)
    H = synth.hyperplanes(12, w["d"])
    Hd = torch.from_numpy(H).cuda()
    engine = pk.PIPNN_LEAF_TC if args.engine == "tc" else pk.PIPNN_LEAF_SIMT
    prec_names = {"fp32": pk.PIPNN_PREC_FP32, "bf16": pk.PIPNN_PREC_BF16, "fp8": pk.PIPNN_PREC_FP8,
                  "bf16x3": pk.PIPNN_PREC_BF16X3}
    prec = prec_names[args.prec] if args.prec else (
        pk.PIPNN_PREC_BF16X3 if (w["dtype"] == synth.F32 and args.engine == "tc") else pk.PIPNN_PREC_FP32)
    dt_code = {synth.F32: pk.PIPNN_F32, synth.U8: pk.PIPNN_U8, synth.I8: pk.PIPNN_I8}[w["dtype"]]
    split = dict(wave_members=args.wave_members, merge_waves=args.merge_waves) if args.profile else {}
    bp = pk.params(dtype=dt_code, hyperplanes=Hd, leaf_engine=engine, prec=prec, **split, **workload_params(w))
    R = w["R"]
    adj = torch.empty((n, R), dtype=torch.int32, device="cuda")
    deg = torch.empty(n, dtype=torch.int32, device="cuda")

    sampler = ClockSampler(torch.cuda.current_device())
    step_ms, stats, clocks = timed_builds(pk, Xd, bp, adj, deg, args.steps, args.warmup, w["metric"], barrier,
                                          sampler)
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, "cuda")
    value = job_throughput(n, world, ms / 1e3)
    roofline = leaf_roofline(stats, w["d"], args.engine, "leaf_tc.cu" if w["dtype"] != synth.F32 else "leaf_tcf.cu",
                             f"leaf_gram_tc_{args.workload}.md")
    if args.profile:
        if rank == 0:
            st = stats[-1]
            out = {"profile_run": True, "ms_per_step": ms, "phases_ms": phases(stats),
                   "leaf_pairs": st["leaf_pairs"], "leaf_members": st["leaf_members"],
                   "leaves": st["leaves"], "candidates": st["candidates"], "waves": st["waves"],
                   "hashprune_merges": st["hashprune_merges"]}
            if args.profile_knn and w["dtype"] != synth.F32:
                # one k-NN graph construction (Sec. 5) on the built graph, L = 32, k = 10, after one
                # untimed call
                start = pk.pipnn_medoid(Xd)
                pk.pipnn_knn_graph(Xd, adj.view(torch.uint32), deg.view(torch.uint32), 32, k=10, start=start)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                _, nd = pk.pipnn_knn_graph(Xd, adj.view(torch.uint32), deg.view(torch.uint32), 32, k=10, start=start)
                e1.record()
                torch.cuda.synchronize()
                out["knn_graph_ms"] = e0.elapsed_time(e1)
                out["knn_evaluations_per_point"] = nd / n
            print(json.dumps(out), flush=True)
        return 0

    # end to end through the public call: pinned host input, host output, copies inside the region
    Xh = torch.empty(tuple(Xd.shape), dtype=Xd.dtype, pin_memory=True)
    Xh.copy_(Xd)
    adj_h = torch.empty((n, R), dtype=torch.int32, pin_memory=True)
    deg_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
    del adj, deg, Xd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    bp_h = pk.params(dtype=dt_code, hyperplanes=torch.from_numpy(H), leaf_engine=engine, prec=prec,
                     **workload_params(w))
    pk.pipnn_build_into(Xh, bp_h, synth.BUILD_SEED, adj_h, deg_h, metric=w["metric"])
    e2e_steps = max(3, min(args.steps, 5)) if n <= 20_000_000 else 3
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pk.pipnn_build_into(Xh, bp_h, synth.BUILD_SEED, adj_h, deg_h, metric=w["metric"])
        int(deg_h[0])  # the result is read on the host
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, "cuda")
    e2e = {"value": job_throughput(n, world, e2e_s), "unit": "points/s",
           "h2d_bytes_per_step": int(Xh.numel() * Xh.element_size() + H.nbytes),
           "d2h_bytes_per_step": int(n * R * 4 + n * 4)}

    if rank == 0:
        st = stats[-1]
        line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE_NAME[w["dtype"]], "data": "synthetic",
                "config": config_dict(args.workload, w, args.engine, n), "roofline": roofline,
                "roofline_prune": prune_roofline(stats, w, n), "e2e": e2e,
                "gpu_launches": int(sum(s["kernel_launches"] for s in stats)), "clocks": clocks,
                "phases_ms": phases(stats), "leaves": st["leaves"], "candidates": st["candidates"],
                "waves_per_build": st["waves"], "hashprune_merges_per_build": st["hashprune_merges"],
                "peak_device_bytes": st["peak_device_bytes"]}
        if w["dtype"] == synth.F32:
            line["config"]["prec"] = args.prec or ("bf16x3" if args.engine == "tc" else "fp32")
        Xnp = Xh.numpy()
        adj_np = adj_h.numpy().view(np.uint32)
        deg_np = deg_h.numpy().view(np.uint32)
        if world == 1 and not args.no_recall:
            if args.workload == CONTEXT and n == w["n"]:
                line["recall"], cpu = recall_gate(Xnp, H, w, adj_np, deg_np, args.queries or w["queries"])
                if not args.no_cpu_baseline:
                    line["cpu_baseline"] = cpu
            elif w["dtype"] != synth.F32:
                line["recall"] = headline_recall(Xnp, adj_np, deg_np, w, args.queries or HEADLINE_QUERIES)
        if world == 1 and not args.no_cpu_baseline and "cpu_baseline" not in line:
            line["cpu_baseline"] = cpu_baseline(Xnp, H, w, args.workload, CPU_SAMPLE)
        del Xh, adj_h, deg_h, Xnp, adj_np, deg_np
        pk.pipnn_trim_pool()
        torch.cuda.empty_cache()
        if world == 1 and not args.no_context and args.workload != CONTEXT:
            line["bigann_like_u8"] = context_block(pk, min(args.steps, 10), min(args.warmup, 3), args.engine,
                                                   args.queries or synth.WORKLOADS[CONTEXT]["queries"],
                                                   CONTEXT_CPU_SAMPLE, recall=not args.no_recall,
                                                   knn=not args.no_knn)
            pk.pipnn_trim_pool()
            torch.cuda.empty_cache()
        if world == 1 and not args.no_multi_index:
            line["multi_index"] = multi_index_block(pk, min(args.steps, 3))
            pk.pipnn_trim_pool()
            torch.cuda.empty_cache()
        if world == 1 and not args.no_precision_modes:
            line["precision_modes"] = precision_modes(min(args.steps, 5), min(args.warmup, 2))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
