"""Pins of the CPU oracle against facts fixed outside it: published known-answer vectors,
hand-worked sequences of Alg. 2 and Alg. 3, exact integer arithmetic, error bounds, brute force
on tiny inputs, the history-independence theorem (Sec. 3) and the invariants of Alg. 5."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -24  # binary32 unit roundoff


# --------------------------------------------------------------------------------------------
# Philox4x32-10: the published known-answer vectors
# --------------------------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(w[0:4], w[4:6])
        assert out.tolist() == w[6:10]


# --------------------------------------------------------------------------------------------
# Dissimilarity (Sec. 2): exact for bytes, within the binary32 error bound for floats
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [synth.U8, synth.I8])
def test_dissimilarity_bytes_exact(dtype):
    X = synth.uniform_points(300, 128, dtype, seed=11)
    a = np.arange(300) % 300
    b = (np.arange(300) * 7 + 3) % 300
    got = oracle.dissimilarity(X, a, b)
    ref = ((X[a].astype(np.int64) - X[b].astype(np.int64)) ** 2).sum(1)
    assert np.array_equal(got, ref.astype(np.float64))


@pytest.mark.parametrize("metric", [synth.L2, synth.IP])
def test_dissimilarity_float_within_bound(metric):
    X = synth.mixture(400, 96, synth.F32, 10, 0.3, seed=12, normalize=(metric == synth.IP))
    a = np.arange(400)
    b = (a * 13 + 5) % 400
    got = oracle.dissimilarity(X, a, b, metric=metric)
    x = X[a].astype(np.float64)
    y = X[b].astype(np.float64)
    d = X.shape[1]
    if metric == synth.L2:
        ref = ((x - y) ** 2).sum(1)
        bound = (d + 3) * U * ref
    else:
        dot = (x * y).sum(1)
        ref = 1.0 - dot
        bound = (d + 1) * U * np.abs(x * y).sum(1) + U * np.abs(ref) + 1e-12
    assert np.all(np.abs(got - ref) <= bound)
    # the double-precision reference path agrees with numpy to rounding
    f64 = oracle.dissimilarity(X, a, b, metric=metric, f64=True)
    assert np.allclose(f64, ref, rtol=1e-12, atol=1e-12)


def test_dissimilarity_integer_valued_floats_exact():
    # small integers in binary32: every product and partial sum is exact, so d_def is the exact sum
    X = synth.uniform_points(200, 128, synth.I8, seed=13).astype(np.float32)
    a = np.arange(200)
    b = (a * 3 + 1) % 200
    got = oracle.dissimilarity(X, a, b)
    ref = ((X[a].astype(np.int64) - X[b].astype(np.int64)) ** 2).sum(1)
    assert np.array_equal(got, ref.astype(np.float64))


# --------------------------------------------------------------------------------------------
# Sketches and the residualised hash (Sec. 3, Eq. 1)
# --------------------------------------------------------------------------------------------
def test_sketch_and_hash_bits():
    X = synth.mixture(500, 128, synth.F32, 10, 0.3, seed=14)
    H = synth.hyperplanes(12, 128, seed=3)
    S, nrm = oracle.sketch(X, H)
    ref = X.astype(np.float64) @ H.astype(np.float64).T
    scale = np.abs(X.astype(np.float64)) @ np.abs(H.astype(np.float64)).T
    assert np.all(np.abs(S - ref) <= 130 * U * scale + 1e-30)
    assert np.allclose(nrm, (X.astype(np.float64) ** 2).sum(1), rtol=1e-12)
    # bit i of h_p(c) is the sign of H_i . (c - p); where the exact margin exceeds the sketches'
    # error the oracle's bits must agree with it
    rng = np.random.default_rng(0)
    p = rng.integers(0, 500, 2000)
    c = rng.integers(0, 500, 2000)
    margin = (X[c].astype(np.float64) - X[p].astype(np.float64)) @ H.astype(np.float64).T
    err = 2 * 130 * U * (scale[c] + scale[p])
    bits = (S[c] >= S[p])
    sure = np.abs(margin) > err
    assert sure.mean() > 0.99
    assert np.array_equal(bits[sure], (margin >= 0)[sure])


def test_sketch_bytes_exact():
    X = synth.uniform_points(100, 128, synth.U8, seed=15)
    H = np.round(synth.hyperplanes(8, 128, seed=4) * 4).astype(np.float32)  # small integers
    S, nrm = oracle.sketch(X, H)
    ref = X.astype(np.int64) @ H.astype(np.int64).T
    assert np.array_equal(S.astype(np.int64), ref)
    assert np.array_equal(nrm, (X.astype(np.int64) ** 2).sum(1).astype(np.float64))


def test_slot_packing_orders_by_bf16_distance_then_id():
    # 1.0 is 0x3F80 in bf16; 1.00390625 is halfway to 0x3F81 and rounds to even (0x3F80);
    # 1.01171875 is halfway between 0x3F81 and 0x3F82 and rounds to even (0x3F82).
    s = oracle.slot(1.0, 5, 3)
    assert s >> 48 == (0x3F80 | 0x8000)
    assert (s >> 16) & 0xFFFFFFFF == 5 and s & 0xFFFF == 3
    assert oracle.slot(1.00390625, 0, 0) >> 48 == (0x3F80 | 0x8000)
    assert oracle.slot(1.01171875, 0, 0) >> 48 == (0x3F82 | 0x8000)
    assert oracle.slot(-2.0, 0, 0) >> 48 == (~0xC000) & 0xFFFF
    vals = np.sort(np.random.default_rng(1).normal(0, 100, 500).astype(np.float32))
    keys = [oracle.slot(float(v), 7, 0) for v in vals]
    assert keys == sorted(keys)
    assert oracle.slot(2.0, 3, 9) < oracle.slot(2.0, 4, 0)


# --------------------------------------------------------------------------------------------
# HashPrune (Alg. 3): hand-worked sequences, permutation invariance, closed form
# --------------------------------------------------------------------------------------------
def _load_hashprune_cases():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "hashprune_worked.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "case":
            cur = dict(name=t[1], l_max=int(t[2]), m=int(t[3]), ins=[], expect=None)
            cases.append(cur)
        elif t[0] == "ins":
            cur["ins"].append((int(t[1]), float(t[2]), int(t[3])))
        elif t[0] == "expect":
            cur["expect"] = [int(x) for x in t[1:]]
    return cases


def _case_stream(case):
    ids = [c[0] for c in case["ins"]]
    n = max(ids) + 1
    m = case["m"]
    S = np.zeros((n, m), dtype=np.float32)
    for ident, _, h in case["ins"]:
        if ident != 0:
            S[ident] = [1.0 if (h >> i) & 1 else -1.0 for i in range(m)]
    dst = np.zeros(len(ids), np.uint32)
    src = np.array(ids, np.uint32)
    dist = np.array([c[1] for c in case["ins"]], np.float32)
    return dst, src, dist, S, n


@pytest.mark.parametrize("case", _load_hashprune_cases(), ids=lambda c: c["name"])
def test_hashprune_worked_sequences(case):
    dst, src, dist, S, n = _case_stream(case)
    for fn in (oracle.hashprune_stream, oracle.hashprune_closed):
        res, cnt = fn(dst, src, dist, S, n, case["l_max"])
        got = [int(s >> np.uint64(16)) & 0xFFFFFFFF for s in res[0, :cnt[0]]]
        assert got == case["expect"], fn.__name__
    # history independence (Sec. 3 theorem): every insertion order gives the same reservoir
    for perm in itertools.permutations(range(len(src))):
        p = np.array(perm)
        res, cnt = oracle.hashprune_stream(dst[p], src[p], dist[p], S, n, case["l_max"])
        got = [int(s >> np.uint64(16)) & 0xFFFFFFFF for s in res[0, :cnt[0]]]
        assert got == case["expect"]


def _random_stream(rng, n, count, m, spread=4.0):
    dst = rng.integers(0, n, count).astype(np.uint32)
    src = rng.integers(0, n, count).astype(np.uint32)
    # a candidate's distance is a function of the (dst, src) pair, as in the build
    key = (dst.astype(np.uint64) * np.uint64(1000003) + src.astype(np.uint64)) % np.uint64(977)
    dist = (key.astype(np.float32) / np.float32(977.0) * np.float32(spread)).astype(np.float32)
    S = rng.standard_normal((n, m)).astype(np.float32)
    return dst, src, dist, S


@pytest.mark.parametrize("m,l_max", [(3, 4), (6, 16), (12, 64)])
def test_hashprune_stream_equals_closed_form_and_merges(m, l_max):
    rng = np.random.default_rng(m * 100 + l_max)
    n = 60
    dst, src, dist, S = _random_stream(rng, n, 6000, m)
    r1, c1 = oracle.hashprune_stream(dst, src, dist, S, n, l_max)
    r2, c2 = oracle.hashprune_closed(dst, src, dist, S, n, l_max)
    assert np.array_equal(c1, c2) and np.array_equal(r1, r2)
    # reservoir bound: min(l_max, number of distinct buckets among non-self candidates)
    for v in range(n):
        sel = (dst == v) & (src != v)
        hs = {int(sum(1 << i for i in range(m) if S[s, i] >= S[v, i])) for s in src[sel]}
        assert c1[v] == min(l_max, len(hs))
    # associativity: streaming a second batch into the first batch's reservoirs equals the
    # closed form of the union, for random splits
    for split in (1, 1500, 3000, 5999):
        ra, ca = oracle.hashprune_stream(dst[:split], src[:split], dist[:split], S, n, l_max)
        rb, cb = oracle.hashprune_stream(dst[split:], src[split:], dist[split:], S, n, l_max,
                                         res=ra, cnt=ca)
        assert np.array_equal(cb, c2) and np.array_equal(rb, r2)


# --------------------------------------------------------------------------------------------
# RobustPrune (Alg. 2): hand-worked example, standard == lazy, alpha -> infinity
# --------------------------------------------------------------------------------------------
def test_robustprune_worked_example():
    pts, cases = {}, []
    for line in open(os.path.join(GOLDEN, "robustprune_worked.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "point":
            pts[int(t[1])] = (float(t[2]), float(t[3]))
        else:
            cases.append((float(t[1]), int(t[2]), [int(x) for x in t[3:]]))
    X = np.array([pts[i] for i in range(len(pts))], np.float32)
    n = len(pts)
    l_max = 8
    res = np.full((n, l_max), np.uint64(~np.uint64(0)), np.uint64)
    cnt = np.zeros(n, np.uint32)
    for t, c in enumerate(range(1, n)):
        res[0, t] = oracle.slot(0.0, c, 0)
    cnt[0] = n - 1
    for alpha, R, want in cases:
        for lazy in (False, True):
            adj, deg = oracle.final_prune(X, res, cnt, R, alpha, lazy=lazy)
            assert adj[0, :deg[0]].tolist() == want
            assert np.all(adj[0, deg[0]:] == 0xFFFFFFFF)


def _random_reservoirs(X, n, l_max, rng):
    res = np.full((n, l_max), np.uint64(~np.uint64(0)), np.uint64)
    cnt = np.zeros(n, np.uint32)
    for v in range(n):
        c = rng.integers(0, l_max + 1)
        ids = rng.choice(np.delete(np.arange(n), v), size=c, replace=False)
        for t, i in enumerate(ids):
            res[v, t] = oracle.slot(0.0, int(i), 0)
        cnt[v] = c
    return res, cnt


@pytest.mark.parametrize("dtype", [synth.F32, synth.U8])
def test_robustprune_standard_equals_lazy(dtype):
    rng = np.random.default_rng(5)
    n, l_max = 300, 48
    X = (synth.mixture(n, 32, synth.F32, 5, 0.5, seed=16) if dtype == synth.F32
         else synth.uniform_points(n, 32, synth.U8, seed=16))
    res, cnt = _random_reservoirs(X, n, l_max, rng)
    for alpha, R in ((1.0, 16), (1.2, 32), (1.5, 48)):
        a1, d1 = oracle.final_prune(X, res, cnt, R, alpha, lazy=False)
        a2, d2 = oracle.final_prune(X, res, cnt, R, alpha, lazy=True)
        assert np.array_equal(a1, a2) and np.array_equal(d1, d2)
        assert np.all(d1 <= R)
        for v in range(n):
            got = set(a1[v, :d1[v]].tolist())
            assert v not in got
            assert got <= {int(s >> np.uint64(16)) & 0xFFFFFFFF for s in res[v, :cnt[v]]}


def test_robustprune_large_alpha_keeps_R_nearest():
    rng = np.random.default_rng(6)
    n, l_max, R = 200, 32, 10
    X = synth.uniform_points(n, 16, synth.U8, seed=17)
    res, cnt = _random_reservoirs(X, n, l_max, rng)
    adj, deg = oracle.final_prune(X, res, cnt, R, 1e18)
    for v in range(n):
        ids = np.array([int(s >> np.uint64(16)) & 0xFFFFFFFF for s in res[v, :cnt[v]]], np.int64)
        dd = ((X[ids].astype(np.int64) - X[v].astype(np.int64)) ** 2).sum(1)
        # duplicates at distance 0 from an admitted neighbour are the only thing alpha cannot keep
        order = np.lexsort((ids, dd))
        if np.unique(X[ids], axis=0).shape[0] == len(ids):
            assert adj[v, :deg[v]].tolist() == ids[order][:R].tolist()


# --------------------------------------------------------------------------------------------
# Pick (Sec. 4.2): brute-force k-NN inside leaves
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 4])
def test_leaf_pick_brute_force(k):
    X = synth.uniform_points(400, 24, synth.U8, lo=0, hi=6, seed=18)  # many exact ties
    rng = np.random.default_rng(k)
    leaves = [rng.choice(400, size=s, replace=False) for s in (1, 2, 3, 50, 137)]
    leaves.append(np.concatenate([leaves[3][:10], leaves[3][:10]]))  # repeated ids count once
    off = np.cumsum([0] + [len(l) for l in leaves]).astype(np.uint32)
    mem = np.concatenate(leaves).astype(np.uint32)
    dst, src, dist = oracle.leaf_pick(X, off, mem, k=k)
    got = sorted(zip(dst.tolist(), src.tolist(), dist.tolist()))
    want = []
    for l in leaves:
        u = np.unique(l)
        D = ((X[u][:, None, :].astype(np.int64) - X[u][None, :, :].astype(np.int64)) ** 2).sum(2)
        for a in range(len(u)):
            cand = [(D[a, b], u[b]) for b in range(len(u)) if b != a]
            for dv, j in sorted(cand)[:k]:
                want.append((int(u[a]), int(j), float(dv)))
                want.append((int(j), int(u[a]), float(dv)))
    assert got == sorted(want)


# --------------------------------------------------------------------------------------------
# Partition (Alg. 5): single leaf, invariants, brute-force level 0, determinism, guard
# --------------------------------------------------------------------------------------------
def _leaf_sets(off, mem):
    return sorted(tuple(sorted(mem[off[b]:off[b + 1]].tolist())) for b in range(len(off) - 1))


def test_partition_single_leaf_and_exact_knn_graph():
    X = synth.uniform_points(700, 32, synth.U8, seed=19)
    bp = oracle.params(c_max=1024, l_max=32, R=32, fanout=(10, 3))
    off, mem, _ = oracle.partition(X, bp, seed=1)
    assert len(off) == 2 and sorted(mem.tolist()) == list(range(700))
    # one leaf: the candidates are the exact bi-directed 2-NN graph
    dst, src, dist = oracle.leaf_pick(X, off, mem, k=2)
    D = ((X[:, None, :].astype(np.int64) - X[None, :, :].astype(np.int64)) ** 2).sum(2)
    np.fill_diagonal(D, np.iinfo(np.int64).max)
    nn = np.lexsort((np.broadcast_to(np.arange(700), D.shape), D), axis=1)[:, :2]
    want = set()
    for i in range(700):
        for j in nn[i]:
            want.add((i, int(j)))
            want.add((int(j), i))
    assert {(int(a), int(b)) for a, b in zip(dst, src)} == want


def _level0_reference(X, bp, seed):
    """Level 0 of Alg. 5 computed independently: leaders are the l smallest (Philox priority, id)
    under subproblem 0, every point joins its f nearest leaders (ties to the earlier-drawn one)."""
    n = X.shape[0]
    l = int(max(2, min(math.ceil(Fraction(float(np.float32(bp.p_samp))) * n), bp.max_leaders)))
    prio = np.array([oracle.philox4x32_10([i, 0, 0, 0x1EAD], [seed & 0xFFFFFFFF, seed >> 32])[0]
                     for i in range(n)], np.uint64)
    leaders = np.lexsort((np.arange(n), prio))[:l]
    f = min(bp.fanout[0], l)
    D = ((X[:, None, :].astype(np.int64) - X[leaders][None, :, :].astype(np.int64)) ** 2).sum(2)
    order = np.argsort(D, axis=1, kind="stable")[:, :f]
    buckets = [sorted(np.nonzero((order == r).any(1))[0].tolist()) for r in range(l)]
    return leaders, buckets


def test_partition_level0_matches_brute_force():
    X = synth.mixture(3000, 16, synth.U8, 20, 10.0, seed=20)
    bp = oracle.params(c_max=2900, c_min=0, p_samp=0.01, fanout=(3,), l_max=32, R=32)
    off, mem, levels = oracle.partition(X, bp, seed=77)
    leaders, buckets = _level0_reference(X, bp, 77)
    assert len(leaders) == 30
    want = sorted(tuple(b) for b in buckets if len(b) > 0)
    assert all(len(b) <= 2900 for b in want)
    assert _leaf_sets(off, mem) == want
    # every point sits in exactly min(fanout, l) leaves
    assert np.array_equal(np.bincount(mem, minlength=3000), np.full(3000, 3))


@pytest.mark.parametrize("dtype,metric", [(synth.F32, synth.L2), (synth.U8, synth.L2),
                                          (synth.F32, synth.IP)])
def test_partition_invariants_and_determinism(dtype, metric):
    X = synth.mixture(12000, 32, dtype, 30, 0.3 if dtype == synth.F32 else 10.0, seed=21,
                      normalize=(metric == synth.IP))
    bp = oracle.params(c_max=512, fanout=(4, 2), p_samp=0.01, l_max=32, R=32)
    off, mem, levels = oracle.partition(X, bp, seed=5, metric=metric)
    sizes = np.diff(off.astype(np.int64))
    assert sizes.max() <= 512 and sizes.min() >= 1
    assert levels >= 2
    assert np.all(np.bincount(mem, minlength=12000) >= 1)
    for b in range(len(off) - 1):
        seg = mem[off[b]:off[b + 1]]
        assert len(np.unique(seg)) == len(seg)
    off2, mem2, _ = oracle.partition(X, bp, seed=5, metric=metric)
    assert np.array_equal(off, off2) and np.array_equal(mem, mem2)
    off3, mem3, _ = oracle.partition(X, bp, seed=6, metric=metric)
    assert _leaf_sets(off, mem) != _leaf_sets(off3, mem3)


def test_partition_merge_packs_small_buckets():
    X = synth.mixture(5000, 16, synth.U8, 200, 10.0, seed=22)
    bp = oracle.params(c_max=400, c_min=100, p_samp=0.02, fanout=(1,), l_max=32, R=32)
    off, mem, _ = oracle.partition(X, bp, seed=3)
    sizes = np.diff(off.astype(np.int64))
    assert sizes.max() <= 400
    # fanout 1 and no recursion beyond carving: every point lands in exactly one leaf
    assert np.array_equal(np.sort(mem), np.arange(5000))
    # small buckets were merged: fewer leaves than leaders, and few leaves below C_min
    assert len(sizes) < 100
    assert (sizes < 100).sum() <= 1 + len(sizes) // 4


def test_partition_duplicates_guard():
    X = np.zeros((5000, 8), np.uint8)
    X[::7] = 3
    bp = oracle.params(c_max=256, fanout=(3, 2), l_max=16, R=16)
    off, mem, _ = oracle.partition(X, bp, seed=9)
    sizes = np.diff(off.astype(np.int64))
    assert sizes.max() <= 256
    assert np.all(np.bincount(mem, minlength=5000) >= 1)


# --------------------------------------------------------------------------------------------
# End to end (Alg. 4): graph structure and quality
# --------------------------------------------------------------------------------------------
def test_build_graph_quality_and_structure():
    X, Q = synth.mixture(8000, 32, synth.F32, 40, 0.3, seed=23, n_queries=200)
    H = synth.hyperplanes(12, 32, seed=5)
    bp = oracle.params(c_max=512, l_max=64, R=32, fanout=(10, 3))
    adj, deg, st = oracle.build(X, bp, H, seed=42)
    assert st["candidates"] <= 4 * st["leaf_members"]
    assert deg.max() <= 32 and deg.min() >= 1
    for v in range(0, 8000, 97):
        nb = adj[v, :deg[v]]
        assert v not in nb.tolist() and len(set(nb.tolist())) == len(nb)
        assert np.all(adj[v, deg[v]:] == 0xFFFFFFFF)
    gt = oracle.knn(X, Q, 10)
    ids, _ = oracle.beam_search(X, adj, deg, Q, 64)
    assert oracle.recall(ids, gt) >= 0.95
    # without the final prune a node keeps its reservoir's nearest R entries
    bp.final_prune = 0
    adj2, deg2, _ = oracle.build(X, bp, H, seed=42)
    assert deg2.max() <= 32
    ids2, _ = oracle.beam_search(X, adj2, deg2, Q, 64)
    assert oracle.recall(ids2, gt) >= 0.9


def test_replicated_build_pins():
    # Sec. 4.1 replication.  One replica composes the stages exactly as Alg. 4 (orc_build); more
    # replicas feed one HashPrune, whose closed form over the union must equal streaming the
    # replicas' candidates one replica after another (history independence, Sec. 3), and every
    # replica must be a different RBC run (its own seed).
    X, Q = synth.mixture(5000, 24, synth.U8, 25, 10.0, seed=26, n_queries=150)
    H = synth.hyperplanes(12, 24, seed=6)
    bp = oracle.params(c_max=256, l_max=48, R=24, fanout=(3,))
    adj1, deg1 = oracle.build_replicated(X, bp, H, 42, 1)
    adj, deg, _ = oracle.build(X, bp, H, seed=42)
    assert np.array_equal(adj1, adj) and np.array_equal(deg1, deg)
    assert oracle.replica_seed(42, 0) == 42 and oracle.replica_seed(2**64 - 1, 1) == 0x9E3779B97F4A7C14
    S, _ = oracle.sketch(X, H)
    res, cnt = None, None
    leafsets = []
    for r in range(3):
        off, mem, _ = oracle.partition(X, bp, oracle.replica_seed(42, r))
        leafsets.append(sorted(tuple(sorted(mem[off[b]:off[b + 1]].tolist())) for b in range(len(off) - 1)))
        dst, src, dist = oracle.leaf_pick(X, off, mem, k=bp.leaf_k)
        res, cnt = oracle.hashprune_stream(dst, src, dist, S, X.shape[0], bp.l_max, res, cnt)
    assert leafsets[0] != leafsets[1] and leafsets[1] != leafsets[2]
    adj3, deg3 = oracle.build_replicated(X, bp, H, 42, 3)
    adj_s, deg_s = oracle.final_prune(X, res, cnt, bp.R, bp.alpha)
    assert np.array_equal(adj3, adj_s) and np.array_equal(deg3, deg_s)
    # the extra replicates add candidates (Sec. 5: an extra replicate buys quality): with fanout 3
    # alone one replica reaches recall@10 ~0.6 at L = 32 here, three ~0.94
    gt = oracle.knn(X, Q, 10)
    r1 = oracle.recall(oracle.beam_search(X, adj1, deg1, Q, 32)[0], gt)
    r3 = oracle.recall(oracle.beam_search(X, adj3, deg3, Q, 32)[0], gt)
    assert r3 > r1 + 0.1
    # without the final prune: the nearest R reservoir entries, as orc_build keeps them
    bp.final_prune = 0
    a0, d0 = oracle.build_replicated(X, bp, H, 42, 1)
    a1, d1, _ = oracle.build(X, bp, H, seed=42)
    assert np.array_equal(a0, a1) and np.array_equal(d0, d1)


def test_knn_and_beam_search_exact_on_complete_graph():
    X, Q = synth.mixture(300, 8, synth.F32, 5, 0.5, seed=24, n_queries=20)
    gt = oracle.knn(X, Q, 10)
    D = ((Q[:, None, :].astype(np.float64) - X[None, :, :].astype(np.float64)) ** 2).sum(2)
    assert np.array_equal(gt, np.argsort(D, axis=1, kind="stable")[:, :10])
    # on the complete graph Alg. 1 with L >= 10 finds the exact neighbours after one expansion
    R = 299
    adj = np.array([[j for j in range(300) if j != i] for i in range(300)], np.uint32)
    deg = np.full(300, R, np.uint32)
    ids, _ = oracle.beam_search(X, adj, deg, Q, 16)
    assert oracle.recall(ids, gt) == 1.0


@pytest.mark.parametrize("dtype", [np.float32, np.uint8, np.int8])
def test_beam_search_walks_a_path_graph(dtype):
    """Alg. 1 worked by hand on ten points on a line (x_i = i, edges i <-> i +- 1), query at 7,
    start 0.  L = 1 walks greedily 0 -> 7 and evaluates points 0 .. 8 (9 evaluations); L = 3 also
    expands 8 and evaluates 9 (10 evaluations) and returns 7, then the tie 6 / 8 by id."""
    X = np.zeros((10, 4), dtype=dtype)
    X[:, 0] = np.arange(10)
    adj = np.full((10, 2), 0xFFFFFFFF, np.uint32)
    deg = np.zeros(10, np.uint32)
    for i in range(10):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < 10]
        adj[i, :len(nb)] = nb
        deg[i] = len(nb)
    Q = X[7:8].copy()
    for defined in (False, True):
        ids, nd = oracle.beam_search(X, adj, deg, Q, 1, k=1, start=0, defined=defined)
        assert ids.tolist() == [[7]] and nd == 9
        ids, nd = oracle.beam_search(X, adj, deg, Q, 3, k=3, start=0, defined=defined)
        assert ids.tolist() == [[7, 6, 8]] and nd == 10


@pytest.mark.parametrize("dtype", [np.float32, np.uint8, np.int8])
def test_defined_beam_search_and_knn_graph_on_complete_graph(dtype):
    """On the complete graph one expansion evaluates every point, so Alg. 1 returns the exact k
    nearest by (dissimilarity, id), and the k-NN graph is the brute-force one without self.
    Integer-valued data keeps the binary32 evaluation exact, so the brute force is in integers;
    duplicated points plant exact ties."""
    rng = np.random.default_rng(33)
    n, d = 240, 6
    lo, hi = (0, 12) if dtype == np.uint8 else (-6, 7)
    X = rng.integers(lo, hi, size=(n, d)).astype(dtype)
    X[100:110] = X[99]
    adj = np.array([[j for j in range(n) if j != i] for i in range(n)], np.uint32)
    deg = np.full(n, n - 1, np.uint32)
    Xi = X.astype(np.int64)
    D = ((Xi[:, None, :] - Xi[None, :, :]) ** 2).sum(2)
    order = np.lexsort((np.broadcast_to(np.arange(n), (n, n)), D), axis=1)
    Q = X[[5, 99, 104, 200]]
    ids, _ = oracle.beam_search(X, adj, deg, Q, 20, k=12, start=17, defined=True)
    for r, qi in enumerate([5, 99, 104, 200]):
        assert ids[r].tolist() == order[qi, :12].tolist()
    knn, _ = oracle.knn_graph(X, adj, deg, 20, k=10, start=17)
    for p in range(n):
        want = [int(j) for j in order[p] if j != p][:10]
        assert knn[p].tolist() == want


def test_invalid_parameters_rejected():
    X = synth.uniform_points(100, 8, synth.U8, seed=25)
    for kw in (dict(c_max=1), dict(hash_bits=17), dict(R=65, l_max=64), dict(leaf_k=0)):
        bp = oracle.params(**{**dict(c_max=64, l_max=64, R=64), **kw})
        with pytest.raises(RuntimeError):
            oracle.partition(X, bp, seed=1) if "hash_bits" not in kw else \
                oracle.build(X, bp, np.zeros((17, 8), np.float32), seed=1)
    Xf = synth.uniform_points(100, 8, synth.F32, seed=25)
    Xf[3, 2] = np.nan
    with pytest.raises(RuntimeError):
        oracle.partition(Xf, oracle.params(c_max=64), seed=1)


# --------------------------------------------------------------------------------------------
# Leader count (Sec. 4.1: ceil(P_samp |P|)) and the beam-search start (medoid)
# --------------------------------------------------------------------------------------------
def test_leader_count_ceiling_is_exact():
    """ceil of the exact real product of the binary32 P_samp and |P|, checked with rationals,
    including products that are integers and products just above one (where a rounded
    double product can land on the integer below)."""
    rng = np.random.default_rng(5)
    ps = [0.005, 0.01, 0.5, 1.0, 2.0 ** -20, float(np.float32(1 / 3)), 1e-30]
    ps += [float(np.float32(v)) for v in rng.uniform(1e-4, 1.0, 40)]
    ns = [1, 2, 3, 199, 200, 201, 1 << 20, (1 << 32) - 2, 123456789, 4000000001]
    ns += [int(v) for v in rng.integers(1, 1 << 32, 40)]
    for p in ps:
        pf = Fraction(float(np.float32(p)))
        for n in ns:
            assert oracle.ceil_of_product(p, n) == math.ceil(pf * n), (p, n)
    # p = M 2^-24 with M odd and n = M^-1 (mod 2^24) + 200 2^24: the exact product is an integer
    # plus 2^-24, which a binary64 product of this size rounds away
    M = (1 << 23) + 12345
    n = pow(M, -1, 1 << 24) + 200 * (1 << 24)
    p = M / 2.0 ** 24
    k = (M * n) >> 24
    assert float(np.float64(p) * np.float64(n)) == k  # the rounded product sits on the integer
    assert oracle.ceil_of_product(p, n) == k + 1


@pytest.mark.parametrize("dtype", [synth.F32, synth.U8, synth.I8])
def test_medoid_is_point_nearest_to_mean(dtype):
    X = synth.mixture(2000, 24, dtype, 10, 0.3 if dtype == synth.F32 else 10.0, seed=31)
    Xd = X.astype(np.float64)
    dist = ((Xd - Xd.mean(0)) ** 2).sum(1)
    want = int(np.argmin(dist))  # first index among equals, like the oracle's strict comparison
    assert oracle.medoid(X) == want
    # a planted exact centre: the mean of a symmetric set is one of its points
    Y = np.array([[0, 0], [2, 0], [-2, 0], [0, 2], [0, -2], [1, 1], [-1, -1]], np.float32)
    assert oracle.medoid(Y) == 0


@pytest.mark.parametrize("dtype", [synth.U8, synth.I8])
def test_byte_medoid_is_exact(dtype):
    """Byte data: the start is the point nearest to the exact rational mean, checked with Python
    integers, including a near tie (mirrored points around a mean just off the lattice) and an
    exact tie (broken towards the smaller index)."""
    X = synth.mixture(700, 16, dtype, 5, 10.0, seed=32)
    n = X.shape[0]
    Xi = [[int(v) for v in r] for r in X]
    S = [sum(r[t] for r in Xi) for t in range(16)]
    val = [sum((n * r[t] - S[t]) ** 2 for t in range(16)) for r in Xi]
    assert oracle.medoid(X) == min(range(n), key=lambda i: (val[i], i))
    # exact tie: two mirrored points around an integer mean, the rest symmetric too
    npdt = np.uint8 if dtype == synth.U8 else np.int8
    lo, hi = (0, 200) if dtype == synth.U8 else (-100, 100)
    mid = (lo + hi) // 2
    Y = np.array([[mid + 3, mid], [mid - 3, mid], [mid, mid + 3], [mid, mid - 3],
                  [lo, lo], [hi, hi], [lo, hi], [hi, lo]], dtype=npdt)
    assert oracle.medoid(Y) == 0
    # near tie: the mean is just off the lattice point between the mirrored candidates
    Z = np.zeros((1000, 2), dtype=npdt)
    Z[:, :] = mid
    Z[0] = (mid + 1, mid)
    Z[1] = (mid - 1, mid)
    Z[2] = (mid + 1, mid)   # mean x = mid + 1/1000: point 0/2 (x = mid + 1) nearer than point 1
    Z[3:] = (mid + 5, mid + 5)
    Zi = [[int(v) for v in r] for r in Z]
    S = [sum(r[t] for r in Zi) for t in range(2)]
    val = [sum((1000 * r[t] - S[t]) ** 2 for t in range(2)) for r in Zi]
    assert oracle.medoid(Z) == min(range(1000), key=lambda i: (val[i], i))


@pytest.mark.parametrize("dtype", [synth.U8, synth.I8])
def test_knn_bytes_equals_plain_knn_and_brute_force(dtype):
    """The matrix-product ground truth equals the plain scan (Def. 1, ties by id), including rows
    with planted ties at the k-th distance."""
    X, Q = synth.mixture(3000, 128, dtype, 20, 10.0, seed=44, n_queries=60, query_seed=45)
    X = X.copy()
    X[100:130] = X[99]  # 31 identical points: ties across the k-th position for queries near them
    Q = np.concatenate([Q, X[99:100], X[5:6]])
    want = oracle.knn(X, Q, 10)
    got = oracle.knn_bytes(X, Q, 10, chunk=16)
    assert np.array_equal(got, want)
    # the points in blocks: every block's own top 10, merged by (distance, id)
    assert np.array_equal(oracle.knn_bytes(X, Q, 10, chunk=16, db_chunk=77), want)
    D = ((Q[:, None, :].astype(np.int64) - X[None, :, :].astype(np.int64)) ** 2).sum(2)
    brute = np.lexsort((np.broadcast_to(np.arange(X.shape[0]), D.shape), D), axis=1)[:, :10]
    assert np.array_equal(got, brute)


# --------------------------------------------------------------------------------------------
# App. A.3 pick variants: directed, inverted and bi-directed k-NN
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 5])
def test_pick_directions(k):
    X = synth.uniform_points(400, 16, synth.U8, lo=0, hi=6, seed=23)  # many ties
    rng = np.random.default_rng(k)
    sizes = [1, 2, 3, 40, 157, 199]
    mem = np.concatenate([rng.choice(400, s, replace=False) for s in sizes]).astype(np.uint32)
    off = np.cumsum([0] + sizes).astype(np.uint32)
    fwd = oracle.leaf_pick(X, off, mem, k=k, direction=oracle.DIRECTED)
    inv = oracle.leaf_pick(X, off, mem, k=k, direction=oracle.INVERTED)
    bi = oracle.leaf_pick(X, off, mem, k=k)
    # directed: exactly each member's k nearest other members by (distance, id), brute force
    want = []
    for b in range(len(sizes)):
        m = mem[off[b]:off[b + 1]].astype(np.int64)
        D = ((X[m][:, None, :].astype(np.int64) - X[m][None, :, :].astype(np.int64)) ** 2).sum(2)
        for i in range(len(m)):
            order = sorted((int(D[i, j]), int(m[j])) for j in range(len(m)) if j != i)
            for dv, j in order[:k]:
                want.append((int(m[i]), j, dv))
    got = [(int(a), int(b_), int(c)) for a, b_, c in zip(*fwd)]
    assert sorted(got) == sorted(want)  # as lists: a point in two leaves yields its edges twice
    # inverted is directed with every edge reversed; bi-directed is the union of both, as lists
    assert sorted(zip(inv[1].tolist(), inv[0].tolist(), inv[2].tolist())) == \
        sorted(zip(fwd[0].tolist(), fwd[1].tolist(), fwd[2].tolist()))
    both = sorted(zip(*[np.concatenate([f, i_]).tolist() for f, i_ in zip(fwd, inv)]))
    assert both == sorted(zip(*[a.tolist() for a in bi]))


def test_build_with_pick_directions_runs_and_differs():
    X = synth.mixture(3000, 32, synth.U8, 20, 10.0, seed=24)
    H = synth.hyperplanes(12, 32, seed=3)
    graphs = [oracle.build(X, oracle.params(c_max=256, fanout=(3,), l_max=32, R=24, pick_direction=m), H, 5)
              for m in (oracle.BIDIRECTED, oracle.DIRECTED, oracle.INVERTED)]
    st = [g[2]["candidates"] for g in graphs]
    assert st[0] == st[1] + st[2] and st[1] == st[2]
    assert not np.array_equal(graphs[1][0], graphs[2][0])
