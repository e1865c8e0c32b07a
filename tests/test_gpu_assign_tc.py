"""Alg. 5 leader assignment on the tensor cores (byte data): the partition built with the
PIPNN_LEAF_TC engine must equal the oracle's leaf for leaf.

The engine ranks leaders by <x, l> - n_l / 2 accumulated in FP32 from BF16 operands; for u8 / i8
and d <= 128 that is exact, so the picks -- including the draw-order tie break between
equidistant leaders -- must be the oracle's integer picks.  Cases span every fanout bucket of the
engine (1..16, and 17 on the CUDA-core path), leader counts that are not multiples of the 16 / 32 /
128-column tiles (2 up to the 1024 cap), one- and two-K-block rows (d = 8 .. 128) and inputs built
to tie."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

CODE = {np.uint8: pk.PIPNN_U8, np.int8: pk.PIPNN_I8}


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


def check(X, seed, **kw):
    off_o, mem_o, lev_o = oracle.partition(X, oracle.params(**kw), seed=seed)
    want = leaf_sets(off_o, mem_o)
    H = synth.hyperplanes(12, X.shape[1], seed=8)
    for engine in (pk.PIPNN_LEAF_TC, pk.PIPNN_LEAF_SIMT):
        bp = pk.params(dtype=CODE[X.dtype.type], leaf_engine=engine, hyperplanes=H, **kw)
        off, mem, lev = pk.pipnn_partition(dev(X), bp, seed=seed)
        assert lev == lev_o
        assert leaf_sets(host(off), host(mem)) == want, f"engine {engine}"
    return lev_o


@pytest.mark.parametrize("fanout", [(1,), (2,), (3, 2), (4,), (5, 3), (8,), (10, 3), (16,), (17, 2)])
def test_tc_assign_every_fanout_bucket(fanout):
    X = synth.mixture(12000, 128, synth.U8, 60, 10.0, seed=61)
    check(X, 21, c_max=400, p_samp=0.02, max_leaders=300, fanout=fanout)


@pytest.mark.parametrize("d,dtype", [(8, synth.U8), (64, synth.I8), (65, synth.U8), (100, synth.I8),
                                     (127, synth.U8), (128, synth.I8)])
def test_tc_assign_row_widths(d, dtype):
    X = synth.mixture(9000, d, dtype, 40, 10.0, seed=62 + d)
    check(X, 22, c_max=300, p_samp=0.01, fanout=(4, 2))


def test_tc_assign_1024_leaders_and_ragged_counts():
    # level 0: 1024 leaders (eight 128-column tiles); deeper levels: small, odd leader counts
    X = synth.mixture(40000, 128, synth.U8, 200, 10.0, seed=63)
    lev = check(X, 23, c_max=2048, p_samp=0.03, max_leaders=1024, fanout=(10, 3))
    assert lev >= 2
    X = synth.mixture(20000, 96, synth.U8, 80, 10.0, seed=64)
    check(X, 24, c_max=700, p_samp=0.0013, max_leaders=1000, fanout=(6, 2))


@pytest.mark.parametrize("kind", ["u8-ties", "u8-duplicates", "u8-all-255", "i8-full-range"])
def test_tc_assign_ties_and_extremes(kind):
    n = 8000
    if kind == "u8-ties":
        X = synth.uniform_points(n, 128, synth.U8, lo=0, hi=3, seed=65)
    elif kind == "u8-duplicates":
        base = synth.mixture(400, 64, synth.U8, 10, 10.0, seed=66)
        X = base[np.random.default_rng(1).integers(0, 400, n)]
    elif kind == "u8-all-255":
        X = np.full((n, 128), 255, np.uint8)
        X[::3, :64] = 0
        X[1::7] = synth.uniform_points(len(X[1::7]), 128, synth.U8, seed=67)
    else:
        X = synth.uniform_points(n, 128, synth.I8, lo=-128, hi=128, seed=68)
    check(X, 25, c_max=256, p_samp=0.02, fanout=(5, 2))


def test_tc_assign_deep_recursion_and_guard():
    # a tight C_max and fanout 1 drive the recursion to the depth cap on clustered data
    X = synth.mixture(6000, 32, synth.U8, 3, 2.0, seed=69)
    check(X, 26, c_max=40, p_samp=0.01, fanout=(1,))
