"""The tcgen05 tensor-core leaf engine (byte data) against the oracle: identical candidate edges.

BF16 holds every u8 / i8 value and the byte-wide pieces of the halved squared norms exactly and,
for d <= 128, every partial sum of the accumulated <x_i, x_j> - n_i / 2 - n_j / 2 (= -D_ij / 2) is a
multiple of 1/2 below 2^23 in magnitude, so the tensor-core result is exact and the picks must
equal the oracle's integer picks bit for bit -- including extreme values (all 255, int8 -128),
leaves whose size is not a multiple of the 128-row / 128-column tiles, and many leaves per CTA
(the engine carries loads across consecutive tiles and units)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

CODE = {np.float32: pk.PIPNN_F32, np.uint8: pk.PIPNN_U8, np.int8: pk.PIPNN_I8}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def edge_rows(dst, src, dist):
    a = np.stack([np.asarray(dst, np.int64), np.asarray(src, np.int64),
                  np.asarray(dist, np.float32).view(np.int32).astype(np.int64)], 1)
    return a[np.lexsort(a.T[::-1])]


def random_leaves(n, sizes, seed):
    rng = np.random.default_rng(seed)
    leaves = [rng.choice(n, size=s, replace=False) for s in sizes]
    off = np.cumsum([0] + list(sizes)).astype(np.uint64)
    return off, np.concatenate(leaves).astype(np.uint32)


def check(X, off, mem, k):
    want = edge_rows(*oracle.leaf_pick(X, off, mem, k=k))
    got = edge_rows(*[host(t) for t in pk.pipnn_leaf_pick(dev(X), dev(off), dev(mem), k=k,
                                                           engine=pk.PIPNN_LEAF_TC)])
    assert got.shape == want.shape
    assert np.array_equal(got, want)


SIZES = [1, 2, 3, 15, 16, 17, 127, 128, 129, 255, 256, 257, 383, 511, 600, 1024, 1500, 2048]


@pytest.mark.parametrize("k", [1, 2, 3, 5, 16])
def test_tc_pick_ragged_leaves_u8(k):
    X = synth.mixture(12000, 128, synth.U8, 50, 10.0, seed=51)
    off, mem = random_leaves(12000, SIZES, seed=k)
    check(X, off, mem, k)


@pytest.mark.parametrize("k", [2, 4])
def test_tc_pick_many_leaves_per_cta(k):
    # ~1,700 row tiles over ~600 leaves of 1 .. 700 members: every persistent CTA walks a dozen
    # units of mixed sizes (one-tile leaves, leaves of <= 32 members, ragged last tiles)
    rng = np.random.default_rng(57)
    sizes = np.concatenate([rng.integers(1, 33, 150), rng.integers(33, 700, 450)])
    rng.shuffle(sizes)
    n = 30000
    X = synth.mixture(n, 128, synth.U8, 80, 10.0, seed=58)
    off, mem = random_leaves(n, sizes.tolist(), seed=k + 10)
    check(X, off, mem, k)


@pytest.mark.parametrize("kind", ["u8-full-range", "u8-all-255", "u8-ties", "i8-full-range"])
def test_tc_pick_extreme_values_exact(kind):
    n = 5000
    if kind == "u8-full-range":
        X = synth.uniform_points(n, 128, synth.U8, seed=52)
    elif kind == "u8-all-255":
        X = np.full((n, 128), 255, np.uint8)
        X[::3, :64] = 0
        X[1::7] = synth.uniform_points(len(X[1::7]), 128, synth.U8, seed=53)
    elif kind == "u8-ties":
        X = synth.uniform_points(n, 128, synth.U8, lo=0, hi=3, seed=54)
    else:
        X = synth.uniform_points(n, 128, synth.I8, lo=-128, hi=128, seed=55)
    off, mem = random_leaves(n, [2048, 1000, 700, 129, 5], seed=9)
    check(X, off, mem, 2)


@pytest.mark.parametrize("k", [2, 3])
def test_tc_pick_ties_across_tiles_of_a_large_leaf(k):
    # values in 0..2: most distances tie, so the id order inside every 128-member tile and the
    # (D, id) merge across 36 tiles both decide picks; the leaf is larger than any the partition makes
    n = 6000
    X = synth.uniform_points(n, 128, synth.U8, lo=0, hi=3, seed=60)
    off, mem = random_leaves(n, [4500, 257, 31], seed=11)
    check(X, off, mem, k)


@pytest.mark.parametrize("d,dtype", [(8, synth.U8), (64, synth.I8), (100, synth.I8), (100, synth.U8),
                                     (127, synth.U8), (128, synth.I8)])
def test_tc_pick_dimensions(d, dtype):
    X = synth.mixture(6000, d, dtype, 30, 10.0, seed=56 + d)
    off, mem = random_leaves(6000, [2048, 777, 300, 64, 1], seed=d)
    check(X, off, mem, 2)


def test_tc_engine_rejects_d_beyond_exactness_bound():
    X = dev(synth.uniform_points(300, 129, synth.U8, seed=59))
    off = dev(np.array([0, 300], np.uint64))
    mem = dev(np.arange(300, dtype=np.uint32))
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_leaf_pick(X, off, mem, k=2, engine=pk.PIPNN_LEAF_TC)
    assert e.value.code == -5


@pytest.mark.parametrize("dtype", [synth.U8, synth.I8])
def test_tc_build_parity(dtype):
    X = synth.mixture(20000, 128, dtype, 80, 10.0, seed=57)
    H = synth.hyperplanes(12, 128, seed=4)
    kw = dict(c_max=1024, l_max=64, R=48, fanout=(6, 2), p_samp=0.005)
    adj_o, deg_o, _ = oracle.build(X, oracle.params(**kw), H, 42)
    bp = pk.params(dtype=CODE[X.dtype.type], hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, **kw)
    adj, deg = pk.pipnn_build(dev(X), bp, 42)
    assert np.array_equal(host(deg), deg_o) and np.array_equal(host(adj), adj_o)


def test_tc_engine_rejects_float_data():
    X = dev(synth.uniform_points(100, 8, synth.F32, seed=58))
    off = dev(np.array([0, 100], np.uint64))
    mem = dev(np.arange(100, dtype=np.uint32))
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_leaf_pick(X, off, mem, k=2, engine=pk.PIPNN_LEAF_TC)
    assert e.value.code == -5
