"""The reduced-precision tensor-core leaf engine for float data (BF16 and FP8 e4m3 operands, FP32
accumulation, exact re-rank) against the oracle: identical candidate edges.

The engine forms every leaf's Gram matrix at reduced precision, keeps per row the candidates within
a proven error band of the row's k-th, and evaluates those with the defining binary32 fused
multiply-add chain; so its edges (dst, src, binary32 distance) must equal the oracle's pick of the
k nearest by (binary32 distance, id) bit for bit, for L2 and inner product, for ragged leaves of
1 .. 2048 members, for k = 1 .. 16, and for rows built to defeat the band (exact duplicates, points
one unit in the last place apart, many equidistant points), where the engine must fall back to a
full evaluation rather than pick wrongly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2602_21247_gb300 as pk  # noqa: E402

PRECS = {"bf16": pk.PIPNN_PREC_BF16, "fp8": pk.PIPNN_PREC_FP8, "bf16x3": pk.PIPNN_PREC_BF16X3}
SIZES = [1, 2, 3, 15, 16, 17, 127, 128, 129, 255, 256, 257, 383, 511, 600, 1024, 1500, 2048]


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


def check(X, off, mem, k, prec, metric=oracle.L2):
    want = edge_rows(*oracle.leaf_pick(X, off, mem, k=k, metric=metric))
    got = edge_rows(*[host(t) for t in pk.pipnn_leaf_pick(dev(X), dev(off), dev(mem), k=k, metric=metric,
                                                           engine=pk.PIPNN_LEAF_TC, prec=PRECS[prec])])
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 16])
def test_ragged_leaves_l2(prec, k):
    X = synth.mixture(12000, 128, synth.F32, 50, 0.3, seed=71)
    off, mem = random_leaves(12000, SIZES, seed=k)
    check(X, off, mem, k, prec)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_ragged_leaves_inner_product_unit_vectors(prec, k):
    X = synth.mixture(12000, 96, synth.F32, 50, 0.3, seed=72, normalize=True)
    off, mem = random_leaves(12000, SIZES, seed=20 + k)
    check(X, off, mem, k, prec, metric=oracle.IP)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
def test_inner_product_unnormalised_and_negative_dissimilarities(prec):
    # |x| up to ~30: 1 - <x, y> is far below zero for many pairs, which the per-leaf key offset
    # must keep ordered
    X = synth.mixture(6000, 64, synth.F32, 20, 0.5, seed=73) * np.float32(3.0)
    off, mem = random_leaves(6000, [2048, 700, 129, 33, 2], seed=5)
    check(X, off, mem, 2, prec, metric=oracle.IP)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("d", [8, 33, 64, 96, 100, 128])
def test_dimensions(prec, d):
    X = synth.mixture(6000, d, synth.F32, 30, 0.3, seed=74 + d)
    off, mem = random_leaves(6000, [2048, 777, 300, 64, 1], seed=d)
    check(X, off, mem, 2, prec)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("kind", ["duplicates", "ulp-apart", "equidistant", "offset-far-from-origin"])
def test_adversarial_near_ties(prec, kind):
    rng = np.random.default_rng(75)
    n, d = 5000, 64
    X = synth.mixture(n, d, synth.F32, 10, 0.3, seed=76)
    if kind == "duplicates":
        X[1000:1400] = X[999]
    elif kind == "ulp-apart":
        base = X[2000].copy()
        for i in range(1, 300):
            X[2000 + i] = base
            X[2000 + i, i % d] = np.nextafter(base[i % d], np.float32(np.inf))
    elif kind == "equidistant":
        # points on a sphere around a centre: every distance to the centre is (nearly) equal
        c = X[3000].copy()
        v = rng.standard_normal((400, d)).astype(np.float32)
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        X[3001:3401] = c + np.float32(0.25) * v
    else:
        X = X + np.float32(1000.0)  # norms far above the distances (the centring's purpose)
    off, mem = random_leaves(n, [2048, 1500, 600, 129], seed=77)
    if kind != "offset-far-from-origin":
        # the planted groups inside the first leaf
        lo = {"duplicates": 999, "ulp-apart": 2000, "equidistant": 3000}[kind]
        grp = np.arange(lo, lo + 401, dtype=np.uint32)
        rest = np.setdiff1d(np.arange(n, dtype=np.uint32), grp)[:2048 - 401]
        mem[:2048] = np.concatenate([grp, rest])
    check(X, off, mem, 2, prec)
    check(X, off, mem, 5, prec)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
def test_partition_leaves_of_a_clustered_ip_set(prec):
    # the leaves Alg. 5 makes (merged buckets of several clusters among them)
    X = synth.mixture(30000, 96, synth.F32, 200, 0.3, seed=78, normalize=True)
    off, mem, _ = oracle.partition(X, oracle.params(c_max=2048, fanout=(10, 3)), seed=3, metric=oracle.IP)
    check(X, off.astype(np.uint64), mem, 2, prec, metric=oracle.IP)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("metric", [oracle.L2, oracle.IP])
def test_build_parity(prec, metric):
    X = synth.mixture(20000, 96, synth.F32, 80, 0.3, seed=79, normalize=metric == oracle.IP)
    H = synth.hyperplanes(12, 96, seed=4)
    kw = dict(c_max=1024, l_max=64, R=48, fanout=(6, 2), p_samp=0.005)
    adj_o, deg_o, _ = oracle.build(X, oracle.params(**kw), H, 42, metric=metric)
    bp = pk.params(dtype=pk.PIPNN_F32, hyperplanes=H, leaf_engine=pk.PIPNN_LEAF_TC, prec=PRECS[prec], **kw)
    adj, deg = pk.pipnn_build(dev(X), bp, 42, metric=metric)
    assert np.array_equal(host(deg), deg_o) and np.array_equal(host(adj), adj_o)
    st = pk.pipnn_get_stats()
    assert st["leaf_full_rows"] < st["leaf_members"]


def test_float_tc_needs_reduced_precision():
    X = dev(synth.uniform_points(100, 8, synth.F32, seed=58))
    off = dev(np.array([0, 100], np.uint64))
    mem = dev(np.arange(100, dtype=np.uint32))
    for prec in (pk.PIPNN_PREC_FP32, pk.PIPNN_PREC_INT8):
        with pytest.raises(pk.PipnnError) as e:
            pk.pipnn_leaf_pick(X, off, mem, k=2, engine=pk.PIPNN_LEAF_TC, prec=prec)
        assert e.value.code == -5


def _model_bound(Xl, metric, prec, d):
    """The error bound E_ij (D units) the engine's band assumes, restated from its stated
    ingredients (without the 25 % safety factor): operand rounding of the centred Gram, the
    binary32 centring / norm terms, a tensor-core FP32 accumulation error of at most u_acc of the
    accumulated magnitudes per MMA instruction, and the defining binary32 evaluation's own error."""
    uc = 2.0 ** -24
    uq, a0, uacc, kstep = (2.0 ** -4, 2.0 ** -10, 2.0 ** -11, 32) if prec == "fp8" else (2.0 ** -8, 0.0, 2.0 ** -22, 16)
    steps = (3 if prec == "bf16x3" else 1) * -(-d // kstep) + 1
    X64 = Xl.astype(np.float64)
    mu = X64.mean(0)
    r = np.linalg.norm(X64 - mu, axis=1)
    ext = np.abs(X64 - mu).max()
    s = 448.0 * (1 - 2.0 ** -8) / ext if prec == "fp8" else 1.0
    ri, rj = r[:, None], r[None, :]
    gram = (3 * 2.0 ** -16 + 2.0 ** -22 if prec == "bf16x3" else 2 * uq + uq * uq) * (1 + 4 * uc)
    lin = a0 * (1 + uq) * np.sqrt(d) * (ri + rj) / s + d * a0 * a0 / s ** 2
    if metric == oracle.L2:
        return (2 * gram * ri * rj + 2 * lin + ((d + 6) * uc + steps * uacc) * (ri ** 2 + rj ** 2)
                + 2 * steps * uacc * (1 + uq) ** 2 * ri * rj + (d + 12) * uc * (ri + rj) ** 2)
    m = np.linalg.norm(mu)
    P = max(0.0, (np.linalg.norm(X64, axis=1) ** 2).max() - 1.0)
    W = 0.5 * (1 + m * m + P) + (r.max() + m) * m
    return (gram * ri * rj + lin + 2 * (d + 6) * uc * W + steps * uacc * ((1 + uq) ** 2 * ri * rj + 2 * W)
            + (d + 6) * uc * (ri + m) * (rj + m) + 2 * uc)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x3"])
@pytest.mark.parametrize("metric", [oracle.L2, oracle.IP])
def test_leaf_gram_error_within_the_band_model(prec, metric):
    """Every approximate dissimilarity the engine forms lies within the error model its band is
    built on, measured against FP64 over all pairs of several leaves (about 4.7 million pairs)."""
    d = 96
    X = synth.mixture(20000, d, synth.F32, 40, 0.3, seed=81, normalize=metric == oracle.IP)
    sizes = [2048, 1024, 700, 129, 64, 3]
    off, mem = random_leaves(20000, sizes, seed=8)
    gram = host(pk.pipnn_leaf_gram(dev(X), dev(off), dev(mem), PRECS[prec], metric=metric))
    g0 = 0
    worst = 0.0
    for b, sz in enumerate(sizes):
        Xl = X[mem[off[b]:off[b + 1]]].astype(np.float64)
        G = Xl @ Xl.T
        if metric == oracle.L2:
            n2 = (Xl * Xl).sum(1)
            D64 = n2[:, None] + n2[None, :] - 2 * G
        else:
            D64 = 1.0 - G
        Dt = gram[g0:g0 + sz * sz].reshape(sz, sz).astype(np.float64)
        g0 += sz * sz
        bound = _model_bound(X[mem[off[b]:off[b + 1]]], metric, prec, d)
        ratio = np.abs(Dt - D64) / bound
        np.fill_diagonal(ratio, 0.0)
        worst = max(worst, float(ratio.max()))
    print(f"{prec} metric {metric}: largest |D~ - D_fp64| / model bound = {worst:.3f}")
    assert worst <= 1.0
