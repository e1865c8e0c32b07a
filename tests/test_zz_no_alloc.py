"""pipnn_hashprune_noalloc: HashPrune for callers that cannot allocate device memory (for example a
serving process whose own allocator reserved the GPU up front).  It must return exactly what
pipnn_hashprune returns, on consecutive calls that share its fixed library scratch, and refuse
inputs that do not fit that scratch before doing any GPU work.

This file is collected last so that a run stopping at the first failure has already run every
other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

STATIC_BYTES = 64 << 20


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def empty_reservoirs(n, l_max):
    res = torch.full((n, l_max), -1, dtype=torch.int64, device="cuda").view(torch.uint64)
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda").view(torch.uint32)
    return res, cnt


def as_np(t):
    return t.view(torch.int64 if t.dtype == torch.uint64 else torch.int32).cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    X = synth.mixture(6000, 32, synth.U8, 30, 10.0, seed=41)
    H = synth.hyperplanes(12, 32, seed=6)
    off, mem, _ = oracle.partition(X, oracle.params(c_max=256, p_samp=0.01, fanout=(4, 2)), seed=3)
    dst, src, dist = oracle.leaf_pick(X, off, mem, k=2)
    S, _ = oracle.sketch(X, H)
    n, l_max = X.shape[0], 48
    half = len(dst) // 2
    batches = [(dst[:half], src[:half], dist[:half]), (dst[half:], src[half:], dist[half:])]
    Sd = dev(S)

    ref_res, ref_cnt = empty_reservoirs(n, l_max)
    got_res, got_cnt = empty_reservoirs(n, l_max)
    for d_, s_, w_ in batches:  # two calls in a row, each merging into the previous result
        pk.pipnn_hashprune(dev(d_), dev(s_), dev(w_), Sd, n, l_max, ref_res, ref_cnt)
        pk.pipnn_hashprune_noalloc(dev(d_), dev(s_), dev(w_), Sd, n, l_max, got_res, got_cnt)
        torch.cuda.synchronize()
        assert np.array_equal(as_np(got_cnt), as_np(ref_cnt))
        assert np.array_equal(as_np(got_res), as_np(ref_res))

    # and both equal the oracle's closed form of Alg. 3 over the whole stream
    want_res, want_cnt = oracle.hashprune_closed(dst, src, dist, S, n, l_max)
    assert np.array_equal(as_np(got_cnt).astype(np.uint32), want_cnt)
    assert np.array_equal(as_np(got_res).view(np.uint64), want_res)

    # a fresh pair of reservoirs after the scratch holds the previous call's contents
    ref2, rc2 = empty_reservoirs(n, l_max)
    got2, gc2 = empty_reservoirs(n, l_max)
    pk.pipnn_hashprune(dev(dst), dev(src), dev(dist), Sd, n, l_max, ref2, rc2)
    pk.pipnn_hashprune_noalloc(dev(dst), dev(src), dev(dist), Sd, n, l_max, got2, gc2)
    torch.cuda.synchronize()
    assert np.array_equal(as_np(gc2), as_np(rc2)) and np.array_equal(as_np(got2), as_np(ref2))


def test_noalloc_rejects_inputs_beyond_its_scratch():
    n, l_max = 1000, 16
    S = dev(np.zeros((n, 12), np.float32))
    res, cnt = empty_reservoirs(n, l_max)
    count = STATIC_BYTES // 8  # the slots alone exceed the scratch
    dst = torch.zeros(count, dtype=torch.int32, device="cuda").view(torch.uint32)
    src = torch.ones(count, dtype=torch.int32, device="cuda").view(torch.uint32)
    dist = torch.zeros(count, dtype=torch.float32, device="cuda")
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_hashprune_noalloc(dst, src, dist, S, n, l_max, res, cnt)
    assert e.value.code == pk.PIPNN_OK - 1
    assert "static scratch" in str(e.value)
    assert int(cnt.view(torch.int32).max()) == 0  # nothing was written
