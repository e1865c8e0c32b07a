"""Failure paths without a GPU fault: a bounded device wait that runs out, and device
allocations that fail part-way through a build.

* The tensor-core engines bound every mbarrier wait by %globaltimer.  pipnn_debug_wait_probe runs
  that same wait on an mbarrier nothing completes: it must give up after the stated limit and
  return PIPNN_ETIMEOUT, and the context must stay usable for the next build.
* pipnn_debug_set_alloc_limit caps the library's device allocations (host-side injection, the
  same error a failing cudaMallocAsync gives).  Builds under caps that run out at different points
  of Alg. 4 must fail with PIPNN_ENOMEM, return no graph, leave caller buffers untouched, and the
  next uncapped build must equal the oracle's graph."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

KW = dict(c_max=512, l_max=48, R=32, fanout=(4, 2), p_samp=0.01)


def small_case():
    X = synth.mixture(6000, 64, synth.U8, 40, 10.0, seed=97)
    H = synth.hyperplanes(12, 64, seed=3)
    return X, H


def host_u32(t):
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


def check_build_equals_oracle(X, H):
    want_adj, want_deg, _ = oracle.build(X, oracle.params(**KW), H, 42)
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, **KW)
    adj, deg = pk.pipnn_build(torch.from_numpy(X).cuda(), bp, seed=42)
    assert np.array_equal(host_u32(deg), want_deg) and np.array_equal(host_u32(adj), want_adj)


@pytest.mark.parametrize("limit_ms", [1, 50])
def test_bounded_wait_gives_up_and_context_survives(limit_ms):
    t0 = time.perf_counter()
    with pytest.raises(pk.PipnnError) as e:
        pk.pipnn_debug_wait_probe(limit_ms * 1_000_000)
    dt = time.perf_counter() - t0
    assert e.value.code == -4  # PIPNN_ETIMEOUT
    assert dt >= limit_ms / 1e3 and dt < 1.5 + limit_ms / 1e3
    X, H = small_case()
    check_build_equals_oracle(X, H)


@pytest.mark.parametrize("cap_mb", [0.001, 0.1, 1, 2, 4])
def test_allocation_failure_returns_nothing_and_next_build_succeeds(cap_mb):
    X, H = small_case()
    Xd = torch.from_numpy(X).cuda()
    bp = pk.params(dtype=pk.PIPNN_U8, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, **KW)
    adj = torch.full((X.shape[0], KW["R"]), 7, dtype=torch.int32, device="cuda")
    deg = torch.full((X.shape[0],), 7, dtype=torch.int32, device="cuda")
    pk.pipnn_debug_set_alloc_limit(int(cap_mb * (1 << 20)))
    try:
        with pytest.raises(pk.PipnnError) as e:
            pk.pipnn_build_into(Xd, bp, 42, adj, deg)
        assert e.value.code == -2  # PIPNN_ENOMEM
        with pytest.raises(pk.PipnnError):
            pk.pipnn_build(Xd, bp, seed=42)
    finally:
        pk.pipnn_debug_set_alloc_limit(0)
    # the caller's buffers are untouched: nothing partial is written
    assert int((adj != 7).sum()) == 0 and int((deg != 7).sum()) == 0
    check_build_equals_oracle(X, H)
