"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and bench.py.

This module holds no arithmetic of the method itself: it only draws points, queries and the
random hyperplanes that HashPrune's residualised hash (Sec. 3, Eq. 1) consumes.  The paper
measures on BigANN-benchmarks datasets (BigANN, MS-SPACEV, DEEP, Wikipedia-Cohere, Text2Image);
those are not available here, so every workload below is a seeded stand-in with the same
dimensionality, element type and metric, and clustered structure (a mixture of Gaussians).

Workloads (n / d / type / metric):
  small-f32-l2   20,000 / 128 / f32 / L2   100 centres ~N(0,I), sigma 0.3
  bigann-like-u8 1,000,000 / 128 / u8 / L2  1,000 centres with coords ~Gamma(2, 20),
                 x = round(clip(c + N(0, 10^2), 0, 255))
  deep-like-ip   1,000,000 / 96 / f32 / IP  500 centres ~N(0,I), sigma 0.3, then unit-normalised
  multi-index    512 indexes, log-uniform sizes 2e3..2e5, 128-d f32 L2
  spacev-like-i8 100,000,000 / 128 / i8 / L2  10,000 centres ~N(0, 40^2),
                 x = clip(rint(c + N(0, 10^2)), -127, 127)
"""
from __future__ import annotations

import numpy as np

F32, U8, I8 = 0, 1, 2
L2, IP = 0, 1

# Parameter sets of the five workloads.  fanout is the multi-level fanout schedule of Sec. 4.1.
WORKLOADS = {
    "small-f32-l2": dict(n=20_000, d=128, dtype=F32, metric=L2, centers=100, sigma=0.3,
                         c_max=1024, l_max=64, R=64, fanout=(2,), queries=1_000, data_seed=1001,
                         query_seed=2001),
    "bigann-like-u8": dict(n=1_000_000, d=128, dtype=U8, metric=L2, centers=1_000, sigma=10.0,
                           c_max=2048, l_max=96, R=64, fanout=(10, 3), queries=10_000,
                           data_seed=1002, query_seed=2002),
    "deep-like-ip": dict(n=1_000_000, d=96, dtype=F32, metric=IP, centers=500, sigma=0.3,
                         c_max=2048, l_max=96, R=64, fanout=(10, 3), queries=10_000,
                         data_seed=1003, query_seed=2003),
    "spacev-like-i8": dict(n=100_000_000, d=128, dtype=I8, metric=L2, centers=10_000, sigma=10.0,
                           c_max=2048, l_max=64, R=64, fanout=(10, 3), queries=10_000,
                           data_seed=1005, query_seed=2005),
}

BUILD_SEED = 42
HYPERPLANE_SEED = 7


def _mixture_f32(n, d, centers, sigma, rng_c, rng_x, normalize):
    c = rng_c.standard_normal((centers, d))
    lab = rng_x.integers(0, centers, size=n)
    x = c[lab] + sigma * rng_x.standard_normal((n, d))
    if normalize:
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    return np.ascontiguousarray(x, dtype=np.float32)


def _mixture_u8(n, d, centers, sigma, rng_c, rng_x):
    c = rng_c.gamma(2.0, 20.0, size=(centers, d))
    out = np.empty((n, d), dtype=np.uint8)
    step = 1 << 18
    for s in range(0, n, step):
        e = min(n, s + step)
        lab = rng_x.integers(0, centers, size=e - s)
        v = c[lab] + sigma * rng_x.standard_normal((e - s, d))
        out[s:e] = np.rint(np.clip(v, 0.0, 255.0)).astype(np.uint8)
    return out


def _mixture_i8(n, d, centers, sigma, rng_c, rng_x):
    c = 40.0 * rng_c.standard_normal((centers, d))
    out = np.empty((n, d), dtype=np.int8)
    step = 1 << 18
    for s in range(0, n, step):
        e = min(n, s + step)
        lab = rng_x.integers(0, centers, size=e - s)
        v = c[lab] + sigma * rng_x.standard_normal((e - s, d))
        out[s:e] = np.clip(np.rint(v), -127.0, 127.0).astype(np.int8)
    return out


def mixture(n, d, dtype, centers, sigma, seed, normalize=False, n_queries=0, query_seed=None):
    """Points (and optionally queries from the same mixture) as a C-contiguous array.

    dtype F32 draws centres ~N(0, I) and points c + sigma*N(0, I) (optionally unit-normalised);
    U8 draws centres ~Gamma(2, 20) per coordinate and rounds/clips to [0, 255];
    I8 draws centres ~N(0, 40^2) and rounds/clips to [-127, 127].
    """
    rng_c = np.random.default_rng([seed, 0])
    rng_x = np.random.default_rng([seed, 1])
    rng_q = np.random.default_rng([query_seed if query_seed is not None else seed, 2])

    def draw(count, rng):
        # the centres are re-drawn from an identical generator so points and queries share them
        rc = np.random.default_rng([seed, 0])
        if dtype == F32:
            return _mixture_f32(count, d, centers, sigma, rc, rng, normalize)
        if dtype == U8:
            return _mixture_u8(count, d, centers, sigma, rc, rng)
        if dtype == I8:
            return _mixture_i8(count, d, centers, sigma, rc, rng)
        raise ValueError("dtype")

    del rng_c
    pts = draw(n, rng_x)
    if n_queries:
        return pts, draw(n_queries, rng_q)
    return pts


def queries(name, n_queries=None):
    """Only the queries of a named workload (the same draws workload() returns beside the points)."""
    w = WORKLOADS[name]
    nq = w["queries"] if n_queries is None else n_queries
    rng_q = np.random.default_rng([w["query_seed"], 2])
    rc = np.random.default_rng([w["data_seed"], 0])
    if w["dtype"] == F32:
        return _mixture_f32(nq, w["d"], w["centers"], w["sigma"], rc, rng_q, w["metric"] == IP)
    if w["dtype"] == U8:
        return _mixture_u8(nq, w["d"], w["centers"], w["sigma"], rc, rng_q)
    return _mixture_i8(nq, w["d"], w["centers"], w["sigma"], rc, rng_q)


def workload(name, n=None, n_queries=None):
    """Points and queries of a named workload (n may be overridden for reduced test sizes)."""
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    nq = w["queries"] if n_queries is None else n_queries
    return mixture(n, w["d"], w["dtype"], w["centers"], w["sigma"], w["data_seed"],
                   normalize=(w["metric"] == IP), n_queries=nq, query_seed=w["query_seed"])


def _centres(centers, d, dtype, seed):
    """The mixture's centres, drawn exactly as mixture() draws them (float64, host)."""
    rng_c = np.random.default_rng([seed, 0])
    if dtype == F32:
        return rng_c.standard_normal((centers, d))
    if dtype == U8:
        return rng_c.gamma(2.0, 20.0, size=(centers, d))
    return 40.0 * rng_c.standard_normal((centers, d))


def mixture_device(n, d, dtype, centers, sigma, seed, device="cuda", chunk=1 << 23, normalize=False):
    """The same mixture recipes drawn with torch's generator on `device` (for workloads too large to
    draw on the host in reasonable time, e.g. 100M x 128 int8).  Seeded and reproducible on one
    kind of device; its values differ from mixture()'s numpy draws."""
    import torch

    def gen(tag):
        g = torch.Generator(device=device)
        g.manual_seed((int(seed) * 1000003 + tag) % (1 << 63))
        return g

    gx = gen(1)
    c = torch.from_numpy(_centres(centers, d, dtype, seed)).to(device)
    tdt = {F32: torch.float32, U8: torch.uint8, I8: torch.int8}[dtype]
    out = torch.empty((n, d), dtype=tdt, device=device)
    for s0 in range(0, n, chunk):
        e = min(n, s0 + chunk)
        lab = torch.randint(0, centers, (e - s0,), generator=gx, device=device)
        v = c[lab] + sigma * torch.randn(e - s0, d, generator=gx, device=device, dtype=torch.float64)
        if dtype == F32:
            if normalize:
                v = v / torch.linalg.norm(v, dim=1, keepdim=True)
            out[s0:e] = v.to(torch.float32)
        elif dtype == U8:
            out[s0:e] = torch.round(torch.clamp(v, 0.0, 255.0)).to(torch.uint8)
        else:
            out[s0:e] = torch.clamp(torch.round(v), -127.0, 127.0).to(torch.int8)
    return out


def queries_device(n_queries, d, dtype, centers, sigma, seed, query_seed, device="cuda"):
    """Queries from the same mixture as mixture_device(..., seed) (same centres), as a host array."""
    import torch

    if dtype not in (I8, F32):
        raise ValueError("queries_device draws int8 and float32 mixtures")
    c = torch.from_numpy(_centres(centers, d, dtype, seed)).to(device)
    gq = torch.Generator(device=device)
    gq.manual_seed((int(query_seed) * 1000003 + 2) % (1 << 63))
    lab = torch.randint(0, centers, (n_queries,), generator=gq, device=device)
    v = c[lab] + sigma * torch.randn(n_queries, d, generator=gq, device=device, dtype=torch.float64)
    if dtype == I8:
        return torch.clamp(torch.round(v), -127.0, 127.0).to(torch.int8).cpu().numpy()
    return v.to(torch.float32).cpu().numpy()


def multi_index_sizes(count=512, lo=2_000, hi=200_000, seed=1004):
    """Sizes of the batched multi-index workload: log-uniform in [lo, hi]."""
    rng = np.random.default_rng([seed, 3])
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


def hyperplanes(m, d, seed=HYPERPLANE_SEED):
    """The m random hyperplanes through the origin of Sec. 3 (rows ~N(0, I_d)), float32 m x d."""
    rng = np.random.default_rng([seed, 4])
    return np.ascontiguousarray(rng.standard_normal((m, d)), dtype=np.float32)


def uniform_points(n, d, dtype, seed, lo=None, hi=None):
    """Unstructured points for edge-case tests (uniform on a box)."""
    rng = np.random.default_rng([seed, 5])
    if dtype == F32:
        return rng.uniform(-1.0 if lo is None else lo, 1.0 if hi is None else hi,
                           size=(n, d)).astype(np.float32)
    if dtype == U8:
        return rng.integers(0 if lo is None else lo, 256 if hi is None else hi,
                            size=(n, d)).astype(np.uint8)
    return rng.integers(-127 if lo is None else lo, 128 if hi is None else hi,
                        size=(n, d)).astype(np.int8)
