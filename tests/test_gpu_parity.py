"""Parity of the CUDA path (through the C ABI) with the CPU oracle, stage by stage and end to end.

Bar: bit-exact.  Every decision on the path (leader choice, pick, HashPrune, prune) is made on
values both sides evaluate identically -- exact integers for byte data, the binary32
fused-multiply-add chain in index order for float data -- so sketches, leaves, candidate edges,
reservoirs and graphs must be identical, not merely close.  Squared norms of float data are the
one value compared with a tolerance (the oracle keeps them in double): |err| <= (d+1) u ||x||^2.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

U = 2.0 ** -24
CODE = {np.float32: pk.PIPNN_F32, np.uint8: pk.PIPNN_U8, np.int8: pk.PIPNN_I8}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    if t.dtype == torch.uint64:
        return t.view(torch.int64).cpu().numpy().view(np.uint64)
    return t.cpu().numpy()


def leaf_sets(off, mem):
    off = np.asarray(off, np.int64)
    return sorted(tuple(sorted(np.asarray(mem)[off[b]:off[b + 1]].tolist())) for b in range(len(off) - 1))


def edge_rows(dst, src, dist):
    a = np.stack([np.asarray(dst, np.int64), np.asarray(src, np.int64),
                  np.asarray(dist, np.float32).view(np.int32).astype(np.int64)], 1)
    return a[np.lexsort(a.T[::-1])]


CASES = {
    "u8-l2": (lambda: synth.mixture(9000, 64, synth.U8, 40, 10.0, seed=31), synth.L2),
    "i8-l2": (lambda: synth.mixture(7000, 48, synth.I8, 30, 10.0, seed=32), synth.L2),
    "f32-l2": (lambda: synth.mixture(8000, 40, synth.F32, 40, 0.3, seed=33), synth.L2),
    "f32-ip": (lambda: synth.mixture(7000, 36, synth.F32, 30, 0.3, seed=34, normalize=True), synth.IP),
}
KW = dict(c_max=300, p_samp=0.01, fanout=(4, 2), l_max=48, R=32)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    X, metric = CASES[request.param][0](), CASES[request.param][1]
    H = synth.hyperplanes(12, X.shape[1], seed=8)
    return request.param, X, metric, H


# ---------------------------------------------------------------- A0
@pytest.mark.parametrize("d,dtype,m", [(37, synth.U8, 12), (30, synth.I8, 16), (45, synth.F32, 5),
                                       (128, synth.U8, 16), (8, synth.I8, 1), (4, synth.F32, 12)])
def test_sketch_parity_widths(d, dtype, m):
    # four coordinates per step (d % 4 == 0) and one at a time (otherwise): both bit-exact
    X = synth.mixture(3000, d, dtype, 10, 10.0 if dtype != synth.F32 else 0.3, seed=37 + d)
    H = synth.hyperplanes(m, d, seed=9)
    S, nrm = pk.pipnn_sketch(dev(X), dev(H))
    S_o, nrm_o = oracle.sketch(X, H)
    assert np.array_equal(host(S).view(np.uint32), S_o.view(np.uint32))
    if X.dtype == np.float32:
        assert np.all(np.abs(host(nrm).astype(np.float64) - nrm_o) <= (d + 1) * U * nrm_o)
    else:
        assert np.array_equal(host(nrm).astype(np.float64), nrm_o)


def test_sketch_parity(case):
    name, X, metric, H = case
    S, nrm = pk.pipnn_sketch(dev(X), dev(H))
    S_o, nrm_o = oracle.sketch(X, H)
    assert np.array_equal(host(S).view(np.uint32), S_o.view(np.uint32))
    if X.dtype == np.float32:
        bound = (X.shape[1] + 1) * U * nrm_o
        assert np.all(np.abs(host(nrm).astype(np.float64) - nrm_o) <= bound)
    else:
        assert np.array_equal(host(nrm).astype(np.float64), nrm_o)


# ---------------------------------------------------------------- A1
def test_partition_parity(case):
    name, X, metric, H = case
    bp_o = oracle.params(**KW)
    off_o, mem_o, lev_o = oracle.partition(X, bp_o, seed=11, metric=metric)
    bp = pk.params(dtype=CODE[X.dtype.type], hyperplanes=H, **KW)
    off, mem, lev = pk.pipnn_partition(dev(X), bp, seed=11, metric=metric)
    assert lev == lev_o and lev >= 2
    assert leaf_sets(host(off), host(mem)) == leaf_sets(off_o, mem_o)


# ---------------------------------------------------------------- A2-A4
@pytest.mark.parametrize("k", [1, 2, 3])
def test_leaf_pick_parity(case, k):
    name, X, metric, H = case
    off_o, mem_o, _ = oracle.partition(X, oracle.params(**KW), seed=12, metric=metric)
    want = edge_rows(*oracle.leaf_pick(X, off_o, mem_o, k=k, metric=metric))
    dst, src, dist = pk.pipnn_leaf_pick(dev(X), dev(off_o.astype(np.uint64)), dev(mem_o), k=k, metric=metric)
    got = edge_rows(host(dst), host(src), host(dist))
    assert got.shape == want.shape and np.array_equal(got, want)


def test_leaf_pick_ragged_and_tiny_leaves():
    X = synth.uniform_points(3000, 20, synth.U8, lo=0, hi=4, seed=35)  # heavy ties
    rng = np.random.default_rng(3)
    sizes = [1, 2, 3, 5, 127, 128, 129, 255, 256, 257, 1000]
    leaves = [rng.choice(3000, size=s, replace=False) for s in sizes]
    off = np.cumsum([0] + sizes).astype(np.uint64)
    mem = np.concatenate(leaves).astype(np.uint32)
    for k in (2, 5, 16):
        want = edge_rows(*oracle.leaf_pick(X, off, mem, k=k))
        got = edge_rows(*[host(t) for t in pk.pipnn_leaf_pick(dev(X), dev(off), dev(mem), k=k)])
        assert np.array_equal(got, want)


# ---------------------------------------------------------------- A5
def test_hashprune_parity_and_associativity(case):
    name, X, metric, H = case
    off_o, mem_o, _ = oracle.partition(X, oracle.params(**KW), seed=13, metric=metric)
    dst, src, dist = oracle.leaf_pick(X, off_o, mem_o, k=2, metric=metric)
    S, _ = oracle.sketch(X, H)
    n = X.shape[0]
    for l_max in (8, 48, 256):
        res_o, cnt_o = oracle.hashprune_stream(dst, src, dist, S, n, l_max)
        res, cnt = pk.pipnn_hashprune(dev(dst), dev(src), dev(dist), dev(S), n, l_max)
        assert np.array_equal(host(cnt), cnt_o)
        assert np.array_equal(host(res), res_o)
    # two and three batches merge to the same reservoirs (history independence)
    l_max = 48
    res_o, cnt_o = oracle.hashprune_closed(dst, src, dist, S, n, l_max)
    perm = np.random.default_rng(0).permutation(len(dst))
    d2, s2, w2 = dst[perm], src[perm], dist[perm]
    res, cnt = None, None
    for a, b in ((0, len(d2) // 3), (len(d2) // 3, len(d2) // 2), (len(d2) // 2, len(d2))):
        res, cnt = pk.pipnn_hashprune(dev(d2[a:b]), dev(s2[a:b]), dev(w2[a:b]), dev(S), n, l_max, res, cnt)
    assert np.array_equal(host(cnt), cnt_o) and np.array_equal(host(res), res_o)


def test_hashprune_grouped_pick_stream_odd_sketch_width():
    # the leaf pick's k = 2 stream, (v, c1), (c1, v), (v, c2), (c2, v) per member, with a sketch
    # width that is not a multiple of four, a count that is not a multiple of four, and a prefix
    # shifted by one so the groups straddle members
    rng = np.random.default_rng(5)
    X = synth.mixture(4000, 24, synth.U8, 20, 10.0, seed=36)
    off_o, mem_o, _ = oracle.partition(X, oracle.params(**KW), seed=15)
    dst, src, dist = oracle.leaf_pick(X, off_o, mem_o, k=2)
    n, m = X.shape[0], 10
    S = rng.standard_normal((n, m)).astype(np.float32)
    for a, b in ((0, len(dst) - 3), (1, len(dst))):
        res_o, cnt_o = oracle.hashprune_closed(dst[a:b], src[a:b], dist[a:b], S, n, 32)
        res, cnt = pk.pipnn_hashprune(dev(dst[a:b]), dev(src[a:b]), dev(dist[a:b]), dev(S), n, 32)
        assert np.array_equal(host(cnt), cnt_o) and np.array_equal(host(res), res_o)


def test_hashprune_grouped_stream_with_self_edges_and_bad_ids():
    # the k = 2 pick stream with some groups broken by a self edge (skipped by both sides); then an
    # id past the last node in each position of a group and in the ragged tail, which is an error
    # (and the next call still works)
    rng = np.random.default_rng(6)
    X = synth.mixture(3000, 16, synth.U8, 15, 10.0, seed=37)
    off_o, mem_o, _ = oracle.partition(X, oracle.params(**KW), seed=16)
    dst, src, dist = oracle.leaf_pick(X, off_o, mem_o, k=2)
    n = X.shape[0]
    S = rng.standard_normal((n, 12)).astype(np.float32)
    src = src.copy()
    at = rng.choice(len(dst), size=len(dst) // 50, replace=False)
    src[at] = dst[at]
    res_o, cnt_o = oracle.hashprune_closed(dst, src, dist, S, n, 24)
    res, cnt = pk.pipnn_hashprune(dev(dst), dev(src), dev(dist), dev(S), n, 24)
    assert np.array_equal(host(cnt), cnt_o) and np.array_equal(host(res), res_o)
    tail = len(dst) - 1 - 4 * ((len(dst) - 1) // 4)
    for pos in (28, 29, 30, 31, len(dst) - 1 - tail, len(dst) - 1):
        for which in (0, 1):
            bd, bs = dst.copy(), src.copy()
            (bd if which == 0 else bs)[pos] = n
            with pytest.raises(pk.PipnnError) as e:
                pk.pipnn_hashprune(dev(bd), dev(bs), dev(dist), dev(S), n, 24)
            assert e.value.code == -1
    res, cnt = pk.pipnn_hashprune(dev(dst), dev(src), dev(dist), dev(S), n, 24)
    assert np.array_equal(host(cnt), cnt_o) and np.array_equal(host(res), res_o)


def _small_batches(n, batches, rng, most=40):
    """Batches of 0..most slots per node (in shuffled order): fresh random pairs, the same pair as an
    earlier slot with its distance (an exact duplicate) or with another distance (the same bucket,
    another slot); distances on a coarse grid, so that many tie in their 16-bit form."""
    hist_s = [np.zeros(0, np.uint32) for _ in range(n)]
    hist_w = [np.zeros(0, np.float32) for _ in range(n)]
    out = []
    for _ in range(batches):
        D, Sx, W = [], [], []
        for v in range(n):
            c = int(rng.integers(0, most + 1))
            if c == 0:
                continue
            s_ = rng.integers(0, n - 1, size=c).astype(np.uint32)
            s_ += (s_ >= v).astype(np.uint32)
            w_ = (rng.integers(0, 200, size=c) * 0.25).astype(np.float32)
            if len(hist_s[v]):
                pick = rng.integers(0, len(hist_s[v]), size=c)
                r = rng.random(c)
                dup, rebucket = r < 0.35, (r >= 0.35) & (r < 0.45)
                s_[dup | rebucket] = hist_s[v][pick[dup | rebucket]]
                w_[dup] = hist_w[v][pick[dup]]
            D.append(np.full(c, v, np.uint32))
            Sx.append(s_)
            W.append(w_)
            hist_s[v] = np.concatenate([hist_s[v], s_])
            hist_w[v] = np.concatenate([hist_w[v], w_])
        d, s_, w_ = (np.concatenate(z) for z in (D, Sx, W))
        perm = rng.permutation(len(d))
        out.append((d[perm], s_[perm], w_[perm]))
    return out


@pytest.mark.parametrize("m", [4, 12, 13])
@pytest.mark.parametrize("l_max", [16, 96, 200])
@pytest.mark.parametrize("most", [40, 140])
def test_hashprune_small_batches_into_filled_reservoirs(m, l_max, most):
    # many batches merged into the same reservoirs: per node up to 128 new slots (in chunks of 32)
    # into up to 128 kept ones (with at most 12 hash bits) take the bucket-lookup path, the rest
    # the sorting paths; after every batch the reservoirs equal the oracle's over the whole stream
    rng = np.random.default_rng(100 + m + l_max + most)
    n = 2000
    S = rng.standard_normal((n, m)).astype(np.float32)
    Sd = dev(S)
    res = cnt = None
    seen = []
    for d, s_, w_ in _small_batches(n, 8 if most < 100 else 4, rng, most):
        seen.append((d, s_, w_))
        res, cnt = pk.pipnn_hashprune(dev(d), dev(s_), dev(w_), Sd, n, l_max, res, cnt)
        res_o, cnt_o = oracle.hashprune_closed(*(np.concatenate(z) for z in zip(*seen)), S, n, l_max)
        assert np.array_equal(host(cnt), cnt_o) and np.array_equal(host(res), res_o)
    if l_max > 128 and m >= 12:
        assert (cnt_o > 128).any()   # some reservoirs outgrow the bucket-lookup path


@pytest.mark.parametrize("engine,dtype", [("tc", synth.U8), ("simt", synth.F32)])
def test_build_replicas_parity(engine, dtype):
    # Sec. 4.1 replication: three independent RBC runs feed one set of reservoirs
    X = synth.mixture(5000, 24, dtype, 25, 10.0 if dtype != synth.F32 else 0.3, seed=26)
    H = synth.hyperplanes(12, 24, seed=6)
    kw = dict(c_max=256, l_max=48, R=24, fanout=(3,))
    adj_o, deg_o = oracle.build_replicated(X, oracle.params(**kw), H, 42, 3)
    code = {np.uint8: pk.PIPNN_U8, np.float32: pk.PIPNN_F32}[X.dtype.type]
    eng = pk.PIPNN_LEAF_TC if engine == "tc" else pk.PIPNN_LEAF_SIMT
    bp = pk.params(dtype=code, hyperplanes=H, leaf_engine=eng, replicas=3, **kw)
    adj, deg = pk.pipnn_build(dev(X), bp, 42)
    assert np.array_equal(host(deg), deg_o) and np.array_equal(host(adj), adj_o)
    st = pk.pipnn_get_stats()
    assert st["leaf_kernel_launches"] == 3


def test_hashprune_hub_node_many_candidates():
    # one node receives far more candidates than a warp buffer holds
    rng = np.random.default_rng(4)
    n, m = 5000, 10
    S = rng.standard_normal((n, m)).astype(np.float32)
    src = rng.integers(1, n, 30000).astype(np.uint32)
    dst = np.zeros_like(src)
    dist = rng.uniform(0, 100, 30000).astype(np.float32)
    for l_max in (16, 200):
        res_o, cnt_o = oracle.hashprune_closed(dst, src, dist, S, n, l_max)
        res, cnt = pk.pipnn_hashprune(dev(dst), dev(src), dev(dist), dev(S), n, l_max)
        assert np.array_equal(host(cnt), cnt_o) and np.array_equal(host(res), res_o)


# ---------------------------------------------------------------- A6
def test_final_prune_parity(case):
    name, X, metric, H = case
    off_o, mem_o, _ = oracle.partition(X, oracle.params(**KW), seed=14, metric=metric)
    dst, src, dist = oracle.leaf_pick(X, off_o, mem_o, k=3, metric=metric)
    S, _ = oracle.sketch(X, H)
    n = X.shape[0]
    res, cnt = oracle.hashprune_closed(dst, src, dist, S, n, 64)
    for R, alpha in ((32, 1.2), (64, 1.0), (7, 2.0)):
        adj_o, deg_o = oracle.final_prune(X, res, cnt, R, alpha, metric=metric)
        adj, deg = pk.pipnn_final_prune(dev(X), dev(res), dev(cnt), R, alpha, metric=metric)
        assert np.array_equal(host(deg), deg_o)
        assert np.array_equal(host(adj), adj_o)


# ---------------------------------------------------------------- Alg. 4 end to end
def _build_both(X, metric, H, seed=42, **kw):
    bp_o = oracle.params(**kw)
    adj_o, deg_o, st = oracle.build(X, bp_o, H, seed, metric=metric)
    bp = pk.params(dtype=CODE[X.dtype.type], hyperplanes=H, **kw)
    adj, deg = pk.pipnn_build(dev(X), bp, seed, metric=metric)
    return host(adj), host(deg), adj_o, deg_o, st


def test_build_parity(case):
    name, X, metric, H = case
    adj, deg, adj_o, deg_o, st = _build_both(X, metric, H, **KW)
    assert st["levels"] >= 2
    assert np.array_equal(deg, deg_o) and np.array_equal(adj, adj_o)


def test_build_small_workload_both_fanout_readings():
    X = synth.workload("small-f32-l2", n_queries=1)[0]
    H = synth.hyperplanes(12, 128)
    for fanout in ((2,), (10, 3)):
        kw = dict(c_max=1024, l_max=64, R=64, fanout=fanout)
        adj, deg, adj_o, deg_o, _ = _build_both(X, synth.L2, H, **kw)
        assert np.array_equal(deg, deg_o) and np.array_equal(adj, adj_o)


def test_build_host_input_and_host_graph():
    X = synth.mixture(5000, 32, synth.U8, 20, 10.0, seed=36)
    H = synth.hyperplanes(12, 32, seed=2)
    kw = dict(c_max=256, l_max=32, R=24, fanout=(3, 2), p_samp=0.01)
    adj_o, deg_o, _ = oracle.build(X, oracle.params(**kw), H, seed=5)
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, **kw)
    adj, deg = pk.pipnn_build(X, bp, 5, graph_on_host=True)
    assert isinstance(adj, np.ndarray)
    assert np.array_equal(deg, deg_o) and np.array_equal(adj, adj_o)


def test_build_without_final_prune():
    X = synth.mixture(4000, 32, synth.F32, 20, 0.3, seed=37)
    H = synth.hyperplanes(8, 32, seed=2)
    kw = dict(c_max=256, l_max=32, R=20, fanout=(3, 2), p_samp=0.01, hash_bits=8, final_prune=False)
    adj, deg, adj_o, deg_o, _ = _build_both(X, synth.L2, H, **kw)
    assert np.array_equal(deg, deg_o) and np.array_equal(adj, adj_o)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 300])
def test_build_single_leaf_sizes(n):
    X = synth.uniform_points(n, 16, synth.U8, seed=38)
    H = synth.hyperplanes(12, 16, seed=2)
    kw = dict(c_max=300, l_max=16, R=8, fanout=(2,))
    adj, deg, adj_o, deg_o, _ = _build_both(X, synth.L2, H, **kw)
    assert np.array_equal(deg, deg_o) and np.array_equal(adj, adj_o)


def test_build_batched_independent_indexes():
    # several independent indexes of one dimension in one call, each with its own seed: every graph
    # equals the oracle's build of that index alone (sizes span a multi-level partition, a single
    # leaf and a three-point index; host and device inputs mixed)
    H = synth.hyperplanes(12, 16, seed=2)
    kw = dict(c_max=300, l_max=16, R=8, fanout=(3, 2), p_samp=0.01)
    Xs = [synth.mixture(n, 16, synth.U8, 10, 10.0, seed=40 + n) for n in (4000, 250, 3)]
    seeds = [11, 12, 13]
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, **kw)
    got = pk.pipnn_build_batched([dev(Xs[0]), Xs[1], dev(Xs[2])], bp, seeds)
    assert len(got) == 3
    for X, s, (adj, deg) in zip(Xs, seeds, got):
        adj_o, deg_o, _ = oracle.build(X, oracle.params(**kw), H, seed=s)
        assert np.array_equal(host(deg), deg_o) and np.array_equal(host(adj), adj_o)
    # one invalid index (no points): an error, and no graph is returned
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_build_batched([dev(Xs[0]), dev(Xs[0][:0])], bp, [1, 2])
    assert e.value.code == -1


def test_build_duplicate_points_guard():
    X = np.zeros((4000, 8), np.uint8)
    X[::5] = 7
    X[1::11] = 3
    H = synth.hyperplanes(12, 8, seed=2)
    kw = dict(c_max=128, l_max=16, R=16, fanout=(3, 2))
    adj, deg, adj_o, deg_o, _ = _build_both(X, synth.L2, H, **kw)
    assert np.array_equal(deg, deg_o) and np.array_equal(adj, adj_o)


def test_invalid_arguments_return_errors():
    X = dev(synth.uniform_points(100, 8, synth.U8, seed=39))
    H = synth.hyperplanes(12, 8, seed=2)
    for kw in (dict(c_max=1), dict(R=65, l_max=64), dict(hash_bits=17), dict(leaf_k=0), dict(l_max=300, R=10),
               dict(fanout=(33,)), dict(alpha=0.5)):
        bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, **{**dict(c_max=64), **kw})
        with pytest.raises(pk.PipnnError) as e:
            pk.pipnn_build(X, bp, 1)
        assert e.value.code == -1
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, c_max=64)
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_build(X, bp, 1, metric=pk.PIPNN_IP)
    assert e.value.code == -5
    Xf = synth.uniform_points(100, 8, synth.F32, seed=39)
    Xf[7, 3] = np.nan
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_build(dev(Xf), pk.params(dtype=pk.PIPNN_F32, hyperplanes=H, c_max=64), 1)
    assert e.value.code == -1
    # the context stays usable after every rejected call
    adj, deg = pk.pipnn_build(X, pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, c_max=64, l_max=16, R=8), 1)
    assert int(deg.view(torch.int32).max()) <= 8
