"""Parity at the benchmark's own configuration (Alg. 4 end to end).

The benchmark builds the bigann-like-u8 workload (1,000,000 x 128 uint8, squared L2, C_max 2048,
C_min 128, fanout [10, 3], k = 2, m = 12, l_max 96, R 64, alpha 1.2) with the tensor-core engines.
Here the first 200,000 points of that workload are built with exactly those parameters on the GPU
and by the oracle, and the graphs are compared element by element: a build of this size runs
every level of the multi-level fanout (levels 0, 1 and the recursion below), leaves up to C_max,
the F = 10 and F = 3 assignment buckets and reservoirs that fill to l_max.  The recall of both
graphs under the oracle's beam search (Alg. 1, Def. 2) is then equal by construction; it is
checked anyway on a few hundred queries, because the metric is stated as recall."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

W = synth.WORKLOADS["bigann-like-u8"]
KW = dict(c_max=W["c_max"], l_max=W["l_max"], R=W["R"], fanout=tuple(W["fanout"]))


def host_u32(t):
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("engine", ["tc", "simt"])
def test_bench_parameters_graph_equals_oracle(engine):
    n = 200_000 if engine == "tc" else 60_000
    X, Q = synth.workload("bigann-like-u8", n=n, n_queries=300)
    H = synth.hyperplanes(12, W["d"])
    want_adj, want_deg, st = oracle.build(X, oracle.params(**KW), H, synth.BUILD_SEED)
    assert st["levels"] >= 3  # the fanout-10 level, the fanout-3 level and the recursion below
    eng = pk.PIPNN_LEAF_TC if engine == "tc" else pk.PIPNN_LEAF_SIMT
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=torch.from_numpy(H).cuda(), leaf_engine=eng, **KW)
    adj, deg = pk.pipnn_build(torch.from_numpy(X).cuda(), bp, seed=synth.BUILD_SEED)
    torch.cuda.synchronize()
    adj, deg = host_u32(adj), host_u32(deg)
    stats = pk.pipnn_get_stats()
    assert stats["leaves"] == st["leaves"] and stats["candidates"] == st["candidates"]
    assert np.array_equal(deg, want_deg)
    assert np.array_equal(adj, want_adj)
    gt = oracle.knn_bytes(X, Q, 10)
    start = oracle.medoid(X)
    for L in (16, 64):
        r_gpu = oracle.recall(oracle.beam_search(X, adj, deg, Q, L, start=start)[0], gt)
        r_orc = oracle.recall(oracle.beam_search(X, want_adj, want_deg, Q, L, start=start)[0], gt)
        assert r_gpu >= r_orc - 0.003
