"""Many independent indexes in one pipeline (pipnn_build_batched): the indexes are partitioned
together -- each with its own seed and index-relative ids in Alg. 5's randomness -- and share the
leaf, HashPrune and prune launches; every index's graph must equal the oracle's build of that
index alone, bit for bit, on every engine and for indexes that are a single leaf."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402


def host(t):
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("engine", ["u8-tc", "u8-simt", "f32-bf16x3", "f32-simt-ip"])
def test_batch_of_many_indexes_equals_separate_oracle_builds(engine):
    rng = np.random.default_rng(61)
    sizes = np.rint(np.exp(rng.uniform(np.log(20), np.log(9000), size=24))).astype(int).tolist() + [1, 2, 512, 513]
    dt = synth.U8 if engine.startswith("u8") else synth.F32
    metric = oracle.IP if engine.endswith("ip") else oracle.L2
    d = 32
    Xs = [synth.mixture(s, d, dt, max(2, s // 200), 10.0 if dt == synth.U8 else 0.3, seed=1000 + i,
                        normalize=metric == oracle.IP) for i, s in enumerate(sizes)]
    seeds = [int(x) for x in rng.integers(1, 1 << 62, size=len(sizes))]
    H = synth.hyperplanes(12, d, seed=5)
    kw = dict(c_max=512, l_max=32, R=24, fanout=(4, 2), p_samp=0.01)
    eng = pk.PIPNN_LEAF_TC if "tc" in engine or "bf16" in engine else pk.PIPNN_LEAF_SIMT
    prec = pk.PIPNN_PREC_BF16X3 if "bf16x3" in engine else pk.PIPNN_PREC_FP32
    bp = pk.params(dtype=pk.PIPNN_U8 if dt == synth.U8 else pk.PIPNN_F32, hyperplanes=H, leaf_engine=eng,
                   prec=prec, **kw)
    got = pk.pipnn_build_batched([torch.from_numpy(X).cuda() for X in Xs], bp, seeds, metric=metric)
    st = pk.pipnn_get_stats()
    cand = 0
    for X, s, (adj, deg) in zip(Xs, seeds, got):
        adj_o, deg_o, st_o = oracle.build(X, oracle.params(**kw), H, seed=s, metric=metric)
        cand += st_o["candidates"]
        assert np.array_equal(host(deg), deg_o) and np.array_equal(host(adj), adj_o)
    assert st["candidates"] == cand


def test_batch_with_replicas_and_waves():
    sizes = [3000, 40, 2500, 700]
    Xs = [synth.mixture(s, 16, synth.I8, 8, 10.0, seed=77 + i) for i, s in enumerate(sizes)]
    seeds = [3, 1 << 40, 5, 7]
    H = synth.hyperplanes(12, 16, seed=2)
    kw = dict(c_max=256, l_max=24, R=16, fanout=(3,), p_samp=0.01)
    bp = pk.params(dtype=pk.PIPNN_I8, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, replicas=2, wave_members=700,
                   **kw)
    got = pk.pipnn_build_batched([torch.from_numpy(X).cuda() for X in Xs], bp, seeds)
    assert pk.pipnn_get_stats()["waves"] > 4
    for X, s, (adj, deg) in zip(Xs, seeds, got):
        adj_o, deg_o = oracle.build_replicated(X, oracle.params(**kw), H, s, replicas=2)
        assert np.array_equal(host(deg), deg_o) and np.array_equal(host(adj), adj_o)
