"""CPU oracle of the PiPNN index-build path (numpy front end of pipnn_oracle.c).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA path and the CUDA path never calls it.

Every function returns numpy arrays and follows the paper's definitions:
  sketch ............ Sec. 3 "Implementation" (Sketch(v) = [v . H_i]) and squared norms
  partition ......... Alg. 5 randomized ball carving with multi-level fanout and Merge
  leaf_pick ......... Sec. 4.2 / App. A.3 bi-directed k-NN candidates inside every leaf
  hashprune_stream .. Alg. 3 streamed in candidate order
  hashprune_closed .. the closed form of the history-independence lemma (App. A.6)
  final_prune ....... Alg. 2 RobustPrune (standard or lazy) to degree R
  build ............. Alg. 4 end to end
  build_replicated .. Alg. 4 with Sec. 4.1 replication (independent RBC copies, one HashPrune)
  knn / knn_bytes / beam_search / recall .. Def. 1, Alg. 1 and Def. 2 for evaluating graphs
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

F32, U8, I8 = 0, 1, 2
L2, IP = 0, 1

_lib = None


class Params(C.Structure):
    """Hyper-parameters BP of Alg. 4 (fields as named in Sec. 3, Sec. 4.1, App. A.3 and Alg. 2)."""
    _fields_ = [("c_max", C.c_uint32), ("c_min", C.c_uint32), ("max_leaders", C.c_uint32),
                ("p_samp", C.c_float), ("fanout", C.c_uint32 * 4), ("fanout_levels", C.c_uint32),
                ("leaf_k", C.c_uint32), ("hash_bits", C.c_uint32), ("l_max", C.c_uint32),
                ("R", C.c_uint32), ("alpha", C.c_float), ("final_prune", C.c_int32),
                ("pick_direction", C.c_int32)]


class _Leaves(C.Structure):
    _fields_ = [("off", C.POINTER(C.c_uint32)), ("mem", C.POINTER(C.c_uint32)),
                ("nleaves", C.c_uint64), ("nmem", C.c_uint64), ("levels", C.c_uint64)]


class _Edges(C.Structure):
    _fields_ = [("dst", C.POINTER(C.c_uint32)), ("src", C.POINTER(C.c_uint32)),
                ("dist", C.POINTER(C.c_float)), ("count", C.c_uint64)]


class _Stats(C.Structure):
    _fields_ = [("leaves", C.c_uint64), ("leaf_members", C.c_uint64), ("levels", C.c_uint64),
                ("candidates", C.c_uint64)]


BIDIRECTED, DIRECTED, INVERTED = 0, 1, 2


def params(c_max=1024, c_min=None, max_leaders=1000, p_samp=0.005, fanout=(2,), leaf_k=2,
           hash_bits=12, l_max=64, R=64, alpha=1.2, final_prune=True, pick_direction=BIDIRECTED) -> Params:
    p = Params()
    p.c_max = c_max
    p.c_min = c_max // 16 if c_min is None else c_min
    p.max_leaders = max_leaders
    p.p_samp = p_samp
    for i in range(4):
        p.fanout[i] = fanout[i] if i < len(fanout) else 1
    p.fanout_levels = len(fanout)
    p.leaf_k = leaf_k
    p.hash_bits = hash_bits
    p.l_max = l_max
    p.R = R
    p.alpha = alpha
    p.final_prune = 1 if final_prune else 0
    p.pick_direction = pick_direction
    return p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_philox4x32_10.restype = None
        L.orc_dissimilarity_pairs.argtypes = [vp, u32, i32, i32, vp, vp, u64, vp]
        L.orc_dissimilarity_pairs.restype = None
        L.orc_dissimilarity_f64_pairs.argtypes = [vp, u32, i32, i32, vp, vp, u64, vp]
        L.orc_dissimilarity_f64_pairs.restype = None
        L.orc_sketch.argtypes = [vp, u64, u32, i32, vp, u32, vp, vp]
        L.orc_slot.argtypes = [C.c_float, u32, u32]
        L.orc_slot.restype = u64
        L.orc_partition.argtypes = [vp, u64, u32, i32, i32, C.POINTER(Params), u64, C.POINTER(_Leaves)]
        L.orc_leaves_free.argtypes = [C.POINTER(_Leaves)]
        L.orc_leaves_free.restype = None
        L.orc_leaf_pick.argtypes = [vp, u64, u32, i32, i32, vp, vp, u64, u32, i32, C.POINTER(_Edges)]
        L.orc_edges_free.argtypes = [C.POINTER(_Edges)]
        L.orc_edges_free.restype = None
        for f in (L.orc_hashprune_stream, L.orc_hashprune_closed):
            f.argtypes = [vp, vp, vp, u64, vp, u32, u64, u32, vp, vp]
        L.orc_final_prune.argtypes = [vp, u64, u32, i32, i32, vp, vp, u32, u32, C.c_float, i32, vp, vp]
        L.orc_build.argtypes = [vp, u64, u32, i32, i32, C.POINTER(Params), vp, u64, vp, vp,
                                C.POINTER(_Stats)]
        L.orc_knn.argtypes = [vp, u64, vp, u64, u32, i32, i32, u32, vp]
        L.orc_ceil_of_product.argtypes = [C.c_float, u64]
        L.orc_ceil_of_product.restype = u64
        L.orc_medoid.argtypes = [vp, u64, u32, i32, i32]
        L.orc_medoid.restype = u32
        L.orc_beam_search.argtypes = [vp, u64, u32, i32, i32, vp, vp, u32, vp, u64, u32, u32, u32,
                                      vp, vp]
        L.orc_beam_search_as.argtypes = [vp, u64, u32, i32, i32, vp, vp, u32, vp, u64, u32, u32, u32,
                                         i32, vp, vp]
        _lib = L
    return _lib


def _dtype_code(x: np.ndarray) -> int:
    if x.dtype == np.float32:
        return F32
    if x.dtype == np.uint8:
        return U8
    if x.dtype == np.int8:
        return I8
    raise TypeError(f"unsupported point dtype {x.dtype}")


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def dissimilarity(X, a, b, metric=L2, f64=False):
    """Dissimilarity of the pairs (a[i], b[i]): binary32/exact-integer decision values, or the
    double-precision reference when f64 is set."""
    X = np.ascontiguousarray(X)
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    out = np.zeros(a.shape[0], dtype=np.float64)
    fn = lib().orc_dissimilarity_f64_pairs if f64 else lib().orc_dissimilarity_pairs
    fn(_p(X), X.shape[1], _dtype_code(X), metric, _p(a), _p(b), a.shape[0], _p(out))
    return out


def sketch(X, H):
    X = np.ascontiguousarray(X)
    H = np.ascontiguousarray(H, dtype=np.float32)
    n, d = X.shape
    m = H.shape[0]
    S = np.zeros((n, m), dtype=np.float32)
    nrm = np.zeros(n, dtype=np.float64)
    _check(lib().orc_sketch(_p(X), n, d, _dtype_code(X), _p(H), m, _p(S), _p(nrm)), "sketch")
    return S, nrm


def partition(X, bp: Params, seed, metric=L2):
    """Leaves of Alg. 5 as (offsets, members); leaf b holds members[offsets[b]:offsets[b+1]]."""
    X = np.ascontiguousarray(X)
    n, d = X.shape
    out = _Leaves()
    _check(lib().orc_partition(_p(X), n, d, _dtype_code(X), metric, C.byref(bp), seed,
                               C.byref(out)), "partition")
    try:
        off = np.ctypeslib.as_array(out.off, shape=(out.nleaves + 1,)).copy() if out.nleaves else \
            np.zeros(1, dtype=np.uint32)
        mem = np.ctypeslib.as_array(out.mem, shape=(out.nmem,)).copy() if out.nmem else \
            np.zeros(0, dtype=np.uint32)
        levels = out.levels
    finally:
        lib().orc_leaves_free(C.byref(out))
    return off, mem, levels


def leaf_pick(X, off, mem, k=2, metric=L2, direction=BIDIRECTED):
    """k-NN candidates (dst, src, dist) of every leaf: bi-directed (Sec. 4.2), or App. A.3's
    directed (dst = the member, src = its neighbour) or inverted (the reverse) variant."""
    X = np.ascontiguousarray(X)
    n, d = X.shape
    off = np.ascontiguousarray(off, dtype=np.uint32)
    mem = np.ascontiguousarray(mem, dtype=np.uint32)
    out = _Edges()
    _check(lib().orc_leaf_pick(_p(X), n, d, _dtype_code(X), metric, _p(off), _p(mem),
                               len(off) - 1, k, direction, C.byref(out)), "leaf_pick")
    try:
        cnt = out.count
        if cnt:
            dst = np.ctypeslib.as_array(out.dst, shape=(cnt,)).copy()
            src = np.ctypeslib.as_array(out.src, shape=(cnt,)).copy()
            dist = np.ctypeslib.as_array(out.dist, shape=(cnt,)).copy()
        else:
            dst = np.zeros(0, np.uint32)
            src = np.zeros(0, np.uint32)
            dist = np.zeros(0, np.float32)
    finally:
        lib().orc_edges_free(C.byref(out))
    return dst, src, dist


def _hashprune(fn, dst, src, dist, S, n, l_max, res=None, cnt=None):
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dist = np.ascontiguousarray(dist, dtype=np.float32)
    S = np.ascontiguousarray(S, dtype=np.float32)
    m = S.shape[1]
    res = np.full((n, l_max), np.uint64(~np.uint64(0)), dtype=np.uint64) if res is None else \
        np.ascontiguousarray(res, dtype=np.uint64).copy()
    cnt = np.zeros(n, dtype=np.uint32) if cnt is None else np.ascontiguousarray(cnt, np.uint32).copy()
    _check(fn(_p(dst), _p(src), _p(dist), dst.shape[0], _p(S), m, n, l_max, _p(res), _p(cnt)),
           "hashprune")
    return res, cnt


def hashprune_stream(dst, src, dist, S, n, l_max, res=None, cnt=None):
    """Alg. 3 over the stream in its given order; returns (slots n x l_max sorted, counts)."""
    return _hashprune(lib().orc_hashprune_stream, dst, src, dist, S, n, l_max, res, cnt)


def hashprune_closed(dst, src, dist, S, n, l_max, res=None, cnt=None):
    """Closed form of Alg. 3's result (history-independence lemma)."""
    return _hashprune(lib().orc_hashprune_closed, dst, src, dist, S, n, l_max, res, cnt)


def slot(dist, ident, h):
    """Reservoir slot [ordered bf16 distance:16][id:32][hash:16] as the oracle packs it."""
    return int(lib().orc_slot(float(dist), int(ident), int(h)))


def final_prune(X, res, cnt, R, alpha, metric=L2, lazy=False):
    X = np.ascontiguousarray(X)
    n, d = X.shape
    res = np.ascontiguousarray(res, dtype=np.uint64)
    cnt = np.ascontiguousarray(cnt, dtype=np.uint32)
    l_max = res.shape[1]
    adj = np.zeros((n, R), dtype=np.uint32)
    deg = np.zeros(n, dtype=np.uint32)
    _check(lib().orc_final_prune(_p(X), n, d, _dtype_code(X), metric, _p(res), _p(cnt), l_max, R,
                                 alpha, 1 if lazy else 0, _p(adj), _p(deg)), "final_prune")
    return adj, deg


def build(X, bp: Params, H, seed, metric=L2):
    """Alg. 4: returns (adjacency n x R padded with 0xFFFFFFFF, degrees, stats dict)."""
    X = np.ascontiguousarray(X)
    n, d = X.shape
    H = np.ascontiguousarray(H, dtype=np.float32)
    if H.shape != (bp.hash_bits, d):
        raise ValueError("hyperplanes must be hash_bits x d")
    adj = np.zeros((n, bp.R), dtype=np.uint32)
    deg = np.zeros(n, dtype=np.uint32)
    st = _Stats()
    _check(lib().orc_build(_p(X), n, d, _dtype_code(X), metric, C.byref(bp), _p(H), seed, _p(adj),
                           _p(deg), C.byref(st)), "build")
    return adj, deg, dict(leaves=st.leaves, leaf_members=st.leaf_members, levels=st.levels,
                          candidates=st.candidates)


REPLICA_SEED_STEP = 0x9E3779B97F4A7C15


def replica_seed(seed, r):
    """Seed of replica r: seed + r * 0x9E3779B97F4A7C15 (mod 2^64); replica 0 keeps the build seed."""
    return (int(seed) + int(r) * REPLICA_SEED_STEP) % (1 << 64)


def build_replicated(X, bp: Params, H, seed, replicas, metric=L2):
    """Alg. 4 with Sec. 4.1 replication: `replicas` independent runs of Alg. 5 (replica r with
    replica_seed(seed, r)), every replica's bi-directed candidates into one HashPrune (Alg. 3 in
    its closed form over the union, which the history-independence lemma makes equal to streaming
    the replicas one after another), then Alg. 2 as in build().  Returns (adjacency, degrees)."""
    X = np.ascontiguousarray(X)
    n = X.shape[0]
    S, _ = sketch(X, H)
    parts = []
    for r in range(replicas):
        off, mem, _ = partition(X, bp, replica_seed(seed, r), metric)
        parts.append(leaf_pick(X, off, mem, k=bp.leaf_k, metric=metric, direction=bp.pick_direction))
    dst, src, dist = (np.concatenate([p[i] for p in parts]) for i in range(3))
    res, cnt = hashprune_closed(dst, src, dist, S, n, bp.l_max)
    if bp.final_prune:
        return final_prune(X, res, cnt, bp.R, bp.alpha, metric)
    # without the final prune: the first R reservoir entries in (distance, id) order
    R = bp.R
    c = np.minimum(cnt, R).astype(np.uint32)
    ids = ((res[:, :R] >> np.uint64(16)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ids[np.arange(R)[None, :] >= c[:, None]] = 0xFFFFFFFF
    return ids, c


def knn(X, Q, k=10, metric=L2):
    X = np.ascontiguousarray(X)
    Q = np.ascontiguousarray(Q, dtype=X.dtype)
    ids = np.zeros((Q.shape[0], k), dtype=np.uint32)
    _check(lib().orc_knn(_p(X), X.shape[0], _p(Q), Q.shape[0], X.shape[1], _dtype_code(X), metric,
                         k, _p(ids)), "knn")
    return ids


def knn_bytes(X, Q, k=10, chunk=256, db_chunk=1 << 22):
    """Exact k nearest points of every query by (squared L2, id) for byte data (Def. 1), the same
    result as knn() but through float32 matrix products: u8 / i8 coordinates are integers of
    magnitude <= 255, so every product and every partial sum of a d <= 128 dot product is an
    integer below 2^24 and exact in binary32 whatever the summation order; the distances
    ||q||^2 + ||x||^2 - 2<q, x> are then formed exactly in int64.  The points are taken in blocks
    of db_chunk; every block contributes its own exact k smallest by (distance, id), ties at the
    k-th distance resolved by id, and the blocks' lists are merged by (distance, id)."""
    import torch

    X = np.ascontiguousarray(X)
    Q = np.ascontiguousarray(Q, dtype=X.dtype)
    if X.dtype not in (np.uint8, np.int8) or X.shape[1] > 128:
        raise ValueError("knn_bytes takes byte data with d <= 128")
    n, nq = X.shape[0], Q.shape[0]
    kk = min(k, n)
    best_d = np.full((nq, 0), 0, np.int64)
    best_i = np.full((nq, 0), 0, np.int64)
    for b0 in range(0, n, db_chunk):
        Xb = X[b0:b0 + db_chunk]
        Xf = torch.from_numpy(Xb.astype(np.float32))
        nx = torch.from_numpy((Xb.astype(np.int64) ** 2).sum(1))
        cd = np.zeros((nq, min(kk, Xb.shape[0])), np.int64)
        ci = np.zeros_like(cd)
        for s in range(0, nq, chunk):
            q = Q[s:s + chunk]
            dot = (torch.from_numpy(q.astype(np.float32)) @ Xf.T).to(torch.int64)
            nq_ = torch.from_numpy((q.astype(np.int64) ** 2).sum(1))
            D = nq_[:, None] + nx[None, :] - 2 * dot
            m = min(kk, Xb.shape[0])
            val, idx = torch.topk(D, m, dim=1, largest=False, sorted=True)
            val, idx = val.numpy(), idx.numpy()
            Dn = None
            for r in range(q.shape[0]):
                th = val[r, m - 1]
                # every candidate up to the m-th distance, ordered by (distance, id)
                if m < Xb.shape[0] or len(set(val[r].tolist())) < m:
                    if Dn is None:
                        Dn = D.numpy()
                    c = np.nonzero(Dn[r] <= th)[0]
                    if len(c) > m or len(set(val[r].tolist())) < m:
                        o = np.lexsort((c, Dn[r, c]))[:m]
                        cd[s + r], ci[s + r] = Dn[r, c[o]], c[o]
                        continue
                cd[s + r], ci[s + r] = val[r], idx[r]
                o = np.lexsort((ci[s + r], cd[s + r]))
                cd[s + r], ci[s + r] = cd[s + r, o], ci[s + r, o]
        ci += b0
        alld = np.concatenate([best_d, cd], 1)
        alli = np.concatenate([best_i, ci], 1)
        o = np.lexsort((alli, alld), axis=1)[:, :kk]
        best_d = np.take_along_axis(alld, o, 1)
        best_i = np.take_along_axis(alli, o, 1)
    return best_i.astype(np.uint32)


def ceil_of_product(p, n):
    """ceil(p * n) of the exact real product of the binary32 value p and the integer n (the leader
    count of Alg. 5 before its clamps)."""
    return int(lib().orc_ceil_of_product(float(p), int(n)))


def medoid(X, metric=L2):
    X = np.ascontiguousarray(X)
    return int(lib().orc_medoid(_p(X), X.shape[0], X.shape[1], _dtype_code(X), metric))


def knn_graph(X, adj, deg, L, k=10, start=None, metric=L2, defined=True):
    """k-NN graph construction with the built index (Sec. 5): every point p queries the graph with
    itself (Alg. 1, beam L, the k + 1 closest kept) and p's k nearest are the first k of those
    other than p.  Returns (knn n x k, number of distance evaluations)."""
    X = np.ascontiguousarray(X)
    if k + 1 > L:
        raise ValueError("need k + 1 <= L")
    ids, nd = beam_search(X, adj, deg, X, L, k=k + 1, start=start, metric=metric, defined=defined)
    out = np.full((X.shape[0], k), 0xFFFFFFFF, dtype=np.uint32)
    for p in range(X.shape[0]):
        row = [int(v) for v in ids[p] if int(v) != p][:k]
        out[p, :len(row)] = row
    return out, nd


def beam_search(X, adj, deg, Q, L, k=10, start=None, metric=L2, defined=False):
    """Alg. 1 for every query; returns (ids nq x k, number of distance evaluations).  Query
    dissimilarities in double precision, or with defined=True as the build's defining binary32 /
    exact-integer value."""
    X = np.ascontiguousarray(X)
    Q = np.ascontiguousarray(Q, dtype=X.dtype)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    deg = np.ascontiguousarray(deg, dtype=np.uint32)
    start = medoid(X, metric) if start is None else start
    ids = np.zeros((Q.shape[0], k), dtype=np.uint32)
    nd = np.zeros(1, dtype=np.uint64)
    _check(lib().orc_beam_search_as(_p(X), X.shape[0], X.shape[1], _dtype_code(X), metric, _p(adj),
                                    _p(deg), adj.shape[1], _p(Q), Q.shape[0], start, L, k,
                                    1 if defined else 0, _p(ids), _p(nd)), "beam_search")
    return ids, int(nd[0])


def recall(found, truth):
    """Mean k@k recall (Def. 2) of found ids against exact ids, row by row."""
    k = truth.shape[1]
    hits = 0
    for f, t in zip(found, truth):
        hits += len(set(f[:k].tolist()) & set(t.tolist()))
    return hits / (k * len(truth))
