"""Alg. 1 (BeamSearch) on the GPU and the k-NN graph construction of Sec. 5 against the oracle.

The GPU search evaluates the defining dissimilarity (binary32 fused multiply-add chain for float
data, exact integers for byte data), so for every query its k results must equal the oracle's
sequential Alg. 1 on the same values (oracle.beam_search(..., defined=True)) id for id, on graphs
the oracle built, for every dtype / metric, for row widths that take the 16-byte path and ones that
do not, for beam widths 1 .. 512, and on graphs whose evaluated-id sets overflow the GPU's per-query
table (where ids get evaluated twice and the result must not change)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

NPDT = {synth.F32: np.float32, synth.U8: np.uint8, synth.I8: np.int8}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def graph(X, metric, R=32, seed=42):
    H = synth.hyperplanes(12, X.shape[1], seed=5)
    kw = dict(c_max=512, l_max=48, R=R, fanout=(4, 2), p_samp=0.01)
    adj, deg, _ = oracle.build(X, oracle.params(**kw), H, seed, metric=metric)
    return adj, deg


def data(dtype, n, d, metric=oracle.L2, nq=200, seed=61):
    sigma = 0.3 if dtype == synth.F32 else 10.0
    X, Q = synth.mixture(n, d, dtype, 30, sigma, seed=seed, n_queries=nq, query_seed=seed + 1,
                         normalize=metric == oracle.IP)
    return X, Q


CASES = [(synth.U8, 128, oracle.L2), (synth.I8, 128, oracle.L2), (synth.U8, 20, oracle.L2),
         (synth.I8, 37, oracle.L2), (synth.F32, 96, oracle.L2), (synth.F32, 33, oracle.L2),
         (synth.F32, 96, oracle.IP), (synth.F32, 35, oracle.IP)]


@pytest.mark.parametrize("dtype,d,metric", CASES)
@pytest.mark.parametrize("L", [1, 10, 32, 100])
def test_beam_search_equals_oracle(dtype, d, metric, L):
    X, Q = data(dtype, 4000, d, metric)
    adj, deg = graph(X, metric)
    start = oracle.medoid(X, metric)
    k = min(10, L)
    want, nd_o = oracle.beam_search(X, adj, deg, Q, L, k=k, start=start, metric=metric, defined=True)
    got, nd_g = pk.pipnn_beam_search(dev(X), dev(adj), dev(deg), dev(Q), L, k=k, start=start, metric=metric)
    assert np.array_equal(host(got), want)
    # every id the oracle evaluates the GPU evaluates too, some possibly twice
    assert nd_g >= nd_o


@pytest.mark.parametrize("dtype,d,metric", CASES[:2] + CASES[4:5] + CASES[6:7])
def test_knn_graph_equals_oracle(dtype, d, metric):
    X, _ = data(dtype, 3000, d, metric, nq=1)
    adj, deg = graph(X, metric)
    start = oracle.medoid(X, metric)
    want, _ = oracle.knn_graph(X, adj, deg, 40, k=10, start=start, metric=metric)
    got, _ = pk.pipnn_knn_graph(dev(X), dev(adj), dev(deg), 40, k=10, start=start, metric=metric)
    assert np.array_equal(host(got), want)
    # nobody is its own neighbour
    assert not np.any(host(got) == np.arange(3000, dtype=np.uint32)[:, None])


@pytest.mark.parametrize("dtype", [synth.U8, synth.I8])
def test_medoid_equals_oracle(dtype):
    X = synth.mixture(50000, 128, dtype, 40, 10.0, seed=62)
    assert pk.pipnn_medoid(dev(X)) == oracle.medoid(X)
    # planted exact tie: mirrored points around an integer mean, and a far pair
    npdt = NPDT[dtype]
    mid = 100 if dtype == synth.U8 else 0
    Y = np.full((9, 16), mid, dtype=npdt)
    Y[0, 0] += 3
    Y[1, 0] -= 3
    Y[2, 1] += 3
    Y[3, 1] -= 3
    Y[4, 2] += 90
    Y[5, 2] -= 90
    Y[6, 3] += 90
    Y[7, 3] -= 90
    Y[8] = mid
    Y[8, 4] += 1
    Y[8, 5] -= 1
    assert pk.pipnn_medoid(dev(Y)) == oracle.medoid(Y)
    # the k-NN graph's own start (start omitted) is this medoid
    adj, deg = graph(X[:3000], oracle.L2)
    want, _ = oracle.knn_graph(X[:3000], adj, deg, 24, k=8)
    got, _ = pk.pipnn_knn_graph(dev(X[:3000]), dev(adj), dev(deg), 24, k=8)
    assert np.array_equal(host(got), want)


def test_medoid_rejects_float_data():
    X = dev(synth.uniform_points(100, 8, synth.F32, seed=63))
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_medoid(X)
    assert e.value.code == -5


@pytest.mark.parametrize("dtype", [synth.U8, synth.F32])
def test_dense_graph_overflows_the_evaluated_id_table(dtype):
    """Rows of 1024 random neighbours: every expansion brings hundreds of new ids, so the per-query
    table is emptied many times and ids are evaluated again; the results must not change."""
    n, d = 6000, 64
    X, Q = data(dtype, n, d, nq=64)
    rng = np.random.default_rng(64)
    R = 1024
    adj = np.stack([rng.choice(n, size=R, replace=False) for _ in range(n)]).astype(np.uint32)
    deg = rng.integers(R // 2, R + 1, size=n).astype(np.uint32)
    for L in (16, 64):
        want, nd_o = oracle.beam_search(X, adj, deg, Q, L, k=10, start=7, defined=True)
        got, nd_g = pk.pipnn_beam_search(dev(X), dev(adj), dev(deg), dev(Q), L, k=10, start=7)
        assert np.array_equal(host(got), want)
        assert nd_g > nd_o   # re-evaluations happened


def test_wide_beam_and_duplicate_neighbours():
    """L = 512 (the maximum; more than the reachable set on a sparse graph, so the beam ends
    partly empty and the tail of ids is 0xFFFFFFFF), and rows that repeat an id."""
    X, Q = data(synth.U8, 700, 128, nq=20)
    adj, deg = graph(X, oracle.L2, R=8)
    adj = adj.copy()
    adj[:, 1] = np.where(deg > 1, adj[:, 0], adj[:, 1])   # the first neighbour twice
    want, _ = oracle.beam_search(X, adj, deg, Q, 512, k=512, start=3, defined=True)
    got, _ = pk.pipnn_beam_search(dev(X), dev(adj), dev(deg), dev(Q), 512, k=512, start=3)
    assert np.array_equal(host(got), want)


def test_isolated_start_and_empty_batch():
    X, Q = data(synth.F32, 500, 16, nq=5)
    adj = np.full((500, 4), 0xFFFFFFFF, np.uint32)
    deg = np.zeros(500, np.uint32)
    got, nd = pk.pipnn_beam_search(dev(X), dev(adj), dev(deg), dev(Q), 8, k=3, start=11)
    assert host(got).tolist() == [[11, 0xFFFFFFFF, 0xFFFFFFFF]] * 5 and nd == 5
    got, nd = pk.pipnn_beam_search(dev(X), dev(adj), dev(deg), dev(Q[:0]), 8, k=3, start=11)
    assert got.shape == (0, 3) and nd == 0


def test_invalid_arguments():
    X, Q = data(synth.U8, 500, 16, nq=5)
    adj, deg = graph(X, oracle.L2, R=8)
    Xd, Qd, ad, dd = dev(X), dev(Q), dev(adj), dev(deg)
    for kw in (dict(L=4, k=5), dict(L=513, k=5), dict(L=8, k=3, start=500)):
        with pytest.raises(pk.PipnnError) as e:
            pk.pipnn_beam_search(Xd, ad, dd, Qd, **kw)
        assert e.value.code == -1
    with pytest.raises(pk.PipnnError):
        pk.pipnn_knn_graph(Xd, ad, dd, 10, k=10)   # k + 1 > L
    bad = adj.copy()
    bad[:, 0] = 100000   # an id outside the points
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_beam_search(Xd, dev(bad), dd, Qd, 8, k=3, start=0)
    assert e.value.code == -1
    # host arrays are refused
    with pytest.raises(pk.PipnnError):
        pk.pipnn_beam_search(Xd, torch.from_numpy(adj), dd, Qd, 8, k=3, start=0)
    # the context is still usable
    got, _ = pk.pipnn_beam_search(Xd, ad, dd, Qd, 8, k=3, start=0)
    want, _ = oracle.beam_search(X, adj, deg, Q, 8, k=3, start=0, defined=True)
    assert np.array_equal(host(got), want)
