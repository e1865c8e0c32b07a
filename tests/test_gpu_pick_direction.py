"""App. A.3 leaf-pick variants on every engine: the directed k-NN (member -> neighbour) and the
inverted k-NN (neighbour -> member) keep one edge of each picked pair; candidate streams and built
graphs must equal the oracle's bit for bit."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

DIRS = {"directed": (pk.PIPNN_PICK_DIRECTED, oracle.DIRECTED), "inverted": (pk.PIPNN_PICK_INVERTED, oracle.INVERTED)}
ENGINES = {"u8-tc": (synth.U8, pk.PIPNN_LEAF_TC, pk.PIPNN_PREC_FP32),
           "u8-simt": (synth.U8, pk.PIPNN_LEAF_SIMT, pk.PIPNN_PREC_FP32),
           "f32-simt": (synth.F32, pk.PIPNN_LEAF_SIMT, pk.PIPNN_PREC_FP32),
           "f32-bf16x3": (synth.F32, pk.PIPNN_LEAF_TC, pk.PIPNN_PREC_BF16X3)}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def rows(dst, src, dist):
    a = np.stack([np.asarray(dst, np.int64), np.asarray(src, np.int64),
                  np.asarray(dist, np.float32).view(np.int32).astype(np.int64)], 1)
    return a[np.lexsort(a.T[::-1])]


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("direction", sorted(DIRS))
@pytest.mark.parametrize("k", [1, 3])
def test_leaf_pick_direction(engine, direction, k):
    dt, eng, prec = ENGINES[engine]
    X = synth.mixture(8000, 64, dt, 40, 0.3 if dt == synth.F32 else 10.0, seed=95)
    rng = np.random.default_rng(k)
    sizes = [1, 2, 17, 128, 129, 700, 2048]
    mem = np.concatenate([rng.choice(8000, s, replace=False) for s in sizes]).astype(np.uint32)
    off = np.cumsum([0] + sizes).astype(np.uint64)
    gd, od = DIRS[direction]
    want = rows(*oracle.leaf_pick(X, off, mem, k=k, direction=od))
    got = rows(*[host(t) for t in pk.pipnn_leaf_pick(dev(X), dev(off), dev(mem), k=k, engine=eng, prec=prec,
                                                     direction=gd)])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("engine", ["u8-tc", "f32-bf16x3"])
@pytest.mark.parametrize("direction", sorted(DIRS))
def test_build_direction(engine, direction):
    dt, eng, prec = ENGINES[engine]
    X = synth.mixture(12000, 64, dt, 50, 0.3 if dt == synth.F32 else 10.0, seed=96)
    H = synth.hyperplanes(12, 64, seed=4)
    gd, od = DIRS[direction]
    kw = dict(c_max=512, l_max=48, R=32, fanout=(4, 2), p_samp=0.01)
    want_adj, want_deg, st = oracle.build(X, oracle.params(pick_direction=od, **kw), H, 9)
    code = pk.PIPNN_U8 if dt == synth.U8 else pk.PIPNN_F32
    bp = pk.params(dtype=code, hyperplanes=H, leaf_engine=eng, prec=prec, pick_direction=gd, **kw)
    adj, deg = pk.pipnn_build(dev(X), bp, 9)
    assert pk.pipnn_get_stats()["candidates"] == st["candidates"]
    assert np.array_equal(host(deg), want_deg) and np.array_equal(host(adj), want_adj)
