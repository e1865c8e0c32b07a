"""Alg. 2 RobustPrune on the tensor cores (byte data): identical graphs to the oracle.

The engine reads every distance it needs from one exact Gram matrix per node and turns the
binary32 removal test fl(alpha^2 * D(y, z)) < D(x, z) into an integer threshold on D(z, y); the
candidate order comes from the reservoir's BF16 keys (checked, with a full count as fallback).
The cases cover HashPrune reservoirs (sorted), shuffled reservoirs (fallback order), heavy ties,
duplicate points, empty and one-entry reservoirs, counts above l_max, alpha = 1 and very large
alpha, l_max up to 127 and d from 8 to 128."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def reservoirs(X, l_max, seed, k=3, c_max=300):
    off, mem, _ = oracle.partition(X, oracle.params(c_max=c_max, p_samp=0.01, fanout=(4, 2)), seed=seed)
    dst, src, dist = oracle.leaf_pick(X, off, mem, k=k)
    S, _ = oracle.sketch(X, synth.hyperplanes(12, X.shape[1], seed=8))
    return oracle.hashprune_closed(dst, src, dist, S, X.shape[0], l_max)


def check(X, res, cnt, R, alpha):
    adj_o, deg_o = oracle.final_prune(X, res, cnt, R, alpha)
    for engine in (pk.PIPNN_LEAF_TC, pk.PIPNN_LEAF_SIMT):
        adj, deg = pk.pipnn_final_prune(dev(X), dev(res), dev(cnt), R, alpha, engine=engine)
        assert np.array_equal(host(deg), deg_o), f"engine {engine}"
        assert np.array_equal(host(adj), adj_o), f"engine {engine}"


@pytest.mark.parametrize("d,dtype", [(8, synth.U8), (64, synth.I8), (100, synth.U8), (128, synth.U8),
                                     (128, synth.I8)])
def test_tc_prune_row_widths(d, dtype):
    X = synth.mixture(6000, d, dtype, 30, 10.0, seed=71 + d)
    res, cnt = reservoirs(X, 96, seed=3)
    for R, alpha in ((64, 1.2), (32, 1.0), (7, 2.0)):
        check(X, res, cnt, R, alpha)


@pytest.mark.parametrize("l_max", [1, 16, 33, 64, 127, 128])
def test_tc_prune_reservoir_sizes(l_max):
    X = synth.mixture(5000, 128, synth.U8, 25, 10.0, seed=72)
    res, cnt = reservoirs(X, l_max, seed=4, k=4)
    for R in sorted({1, max(1, l_max // 3), l_max}):
        check(X, res, cnt, R, 1.2)


def test_tc_prune_shuffled_reservoirs_use_the_full_order():
    X = synth.mixture(4000, 64, synth.U8, 20, 10.0, seed=73)
    res, cnt = reservoirs(X, 80, seed=5)
    rng = np.random.default_rng(2)
    for v in range(X.shape[0]):
        c = int(cnt[v])
        res[v, :c] = res[v, rng.permutation(c)]
    check(X, res, cnt, 40, 1.2)


@pytest.mark.parametrize("kind", ["ties", "duplicates", "all-255"])
def test_tc_prune_ties_and_duplicates(kind):
    n = 4000
    if kind == "ties":
        X = synth.uniform_points(n, 128, synth.U8, lo=0, hi=3, seed=74)
    elif kind == "duplicates":
        base = synth.mixture(300, 96, synth.U8, 10, 10.0, seed=75)
        X = base[np.random.default_rng(3).integers(0, 300, n)]
    else:
        X = np.full((n, 128), 255, np.uint8)
        X[::3, :64] = 0
        X[1::7] = synth.uniform_points(len(X[1::7]), 128, synth.U8, seed=76)
    res, cnt = reservoirs(X, 64, seed=6, c_max=256)
    for alpha in (1.0, 1.2):
        check(X, res, cnt, 32, alpha)


def test_tc_prune_small_counts_clipping_and_huge_alpha():
    X = synth.mixture(3000, 32, synth.I8, 15, 10.0, seed=77)
    res, cnt = reservoirs(X, 48, seed=7)
    cnt = cnt.copy()
    cnt[::5] = 0
    cnt[1::7] = np.minimum(cnt[1::7], 1)
    full = cnt == 48
    cnt[full] = 1000  # above l_max (only where the reservoir is full): clipped to l_max
    check(X, res, cnt, 24, 1.2)
    check(X, res, cnt, 48, 1e18)


@pytest.mark.parametrize("n", [4001, 4002])
def test_tc_prune_every_tile_kind(n):
    """Reservoirs filled from 400 random candidates per node and cut to sizes spread over
    0 .. l_max, so that nodes go four to a tile (up to 31 candidates), two to a tile (32 .. 63) and
    alone (64 and more), in every interleaving, with a lone node left over in the last two-node
    tile when their number is odd."""
    X = synth.mixture(n, 128, synth.U8, 8, 10.0, seed=78)
    rng = np.random.default_rng(n)
    dst = np.repeat(np.arange(n, dtype=np.uint32), 400)
    src = rng.integers(0, n, size=dst.size).astype(np.uint32)
    Xi = X.astype(np.int64)
    dist = ((Xi[dst] - Xi[src]) ** 2).sum(1).astype(np.float32)
    S, _ = oracle.sketch(X, synth.hyperplanes(12, X.shape[1], seed=8))
    res, cnt = oracle.hashprune_closed(dst, src, dist, S, n, 96)
    cnt = np.minimum(cnt, rng.integers(0, 97, size=n)).astype(cnt.dtype)
    assert ((cnt >= 32) & (cnt <= 63)).sum() > 500 and (cnt >= 64).sum() > 500 and (cnt <= 31).sum() > 500
    for R, alpha in ((64, 1.2), (20, 1.0), (96, 1.5)):
        check(X, res, cnt, R, alpha)
