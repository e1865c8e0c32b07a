"""A2..A5 in waves of leaves: the build merges each wave's candidates into the reservoirs before the
next wave's are formed, which bounds the memory of a large build.  HashPrune's history
independence (Sec. 3) makes the graph independent of the split, so a build in forced small waves
must equal the oracle's graph bit for bit on every engine, including waves of a single leaf and
the split float engine."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402


def host_u32(t):
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


KW = dict(c_max=1024, l_max=64, R=48, fanout=(6, 2), p_samp=0.005)


@pytest.mark.parametrize("engine", ["tc", "simt"])
@pytest.mark.parametrize("wave", [1, 3000, 25000, 0])
def test_wave_split_build_equals_oracle_bytes(engine, wave):
    X = synth.mixture(20000, 128, synth.I8, 80, 10.0, seed=91)
    H = synth.hyperplanes(12, 128, seed=4)
    adj_o, deg_o, st_o = oracle.build(X, oracle.params(**KW), H, 42)
    eng = pk.PIPNN_LEAF_TC if engine == "tc" else pk.PIPNN_LEAF_SIMT
    bp = pk.params(dtype=pk.PIPNN_I8, hyperplanes=H, leaf_engine=eng, wave_members=wave, **KW)
    adj, deg = pk.pipnn_build(torch.from_numpy(X).cuda(), bp, 42)
    st = pk.pipnn_get_stats()
    if wave == 1:
        assert st["waves"] == st["leaves"]
    elif wave == 3000:
        assert st["waves"] > 10
    elif wave == 0:
        assert st["waves"] == 1
    # caller-sized waves, merges sized by memory: this build's candidates fit in one merge
    assert st["hashprune_merges"] == 1
    assert st["candidates"] == st_o["candidates"]
    assert np.array_equal(host_u32(deg), deg_o) and np.array_equal(host_u32(adj), adj_o)


@pytest.mark.parametrize("prec", [pk.PIPNN_PREC_BF16X3, pk.PIPNN_PREC_FP8])
def test_wave_split_build_equals_oracle_float(prec):
    X = synth.mixture(15000, 96, synth.F32, 60, 0.3, seed=92, normalize=True)
    H = synth.hyperplanes(12, 96, seed=4)
    adj_o, deg_o, _ = oracle.build(X, oracle.params(**KW), H, 42, metric=oracle.IP)
    bp = pk.params(dtype=pk.PIPNN_F32, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, prec=prec, wave_members=4000,
                   **KW)
    adj, deg = pk.pipnn_build(torch.from_numpy(X).cuda(), bp, 42, metric=oracle.IP)
    assert pk.pipnn_get_stats()["waves"] > 5
    assert np.array_equal(host_u32(deg), deg_o) and np.array_equal(host_u32(adj), adj_o)


def test_replicas_in_waves():
    X = synth.mixture(12000, 64, synth.U8, 50, 10.0, seed=93)
    H = synth.hyperplanes(12, 64, seed=4)
    want_adj, want_deg = oracle.build_replicated(X, oracle.params(**KW), H, 7, replicas=3)
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, replicas=3, wave_members=2500,
                   **KW)
    adj, deg = pk.pipnn_build(torch.from_numpy(X).cuda(), bp, 7)
    assert pk.pipnn_get_stats()["waves"] > 3
    assert np.array_equal(host_u32(deg), want_deg) and np.array_equal(host_u32(adj), want_adj)


@pytest.mark.parametrize("merge_waves", [1, 2, 7])
def test_merge_groups_equal_oracle(merge_waves):
    """HashPrune once per group of consecutive leaf waves (the candidate edges of a group kept until
    its last wave is done): every grouping gives the oracle's graph."""
    X = synth.mixture(20000, 128, synth.U8, 80, 10.0, seed=94)
    H = synth.hyperplanes(12, 128, seed=4)
    adj_o, deg_o, _ = oracle.build(X, oracle.params(**KW), H, 42)
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, wave_members=3000,
                   merge_waves=merge_waves, **KW)
    adj, deg = pk.pipnn_build(torch.from_numpy(X).cuda(), bp, 42)
    st = pk.pipnn_get_stats()
    assert st["waves"] > 10
    assert st["hashprune_merges"] == -(-st["waves"] // merge_waves)
    assert np.array_equal(host_u32(deg), deg_o) and np.array_equal(host_u32(adj), adj_o)
