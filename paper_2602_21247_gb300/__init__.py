"""GB300 (sm_103a) PiPNN index build: thin ctypes binding of libpipnn.so (include/pipnn.h).

The binding only marshals arguments: torch tensors in device memory are passed as raw pointers,
library-owned outputs are copied into torch tensors.  Every step of the path runs in the CUDA
library; if it has not been built, importing works but every call raises.

Entry points (same names as the C ABI):
  pipnn_sketch       A0  sketches and squared norms (Sec. 3 "Implementation")
  pipnn_partition    A1  Alg. 5 randomized ball carving with multi-level fanout and Merge
  pipnn_leaf_pick    A2-A4 in-leaf all pairs + bi-directed k-NN candidates (Sec. 4.2)
  pipnn_hashprune    A5  Alg. 3 HashPrune batch merge into reservoirs
  pipnn_final_prune  A6  Alg. 2 RobustPrune to degree R (Sec. 4.3)
  pipnn_build        Alg. 4 end to end (host or device input)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpipnn.so")

PIPNN_F32, PIPNN_U8, PIPNN_I8 = 0, 1, 2
PIPNN_L2, PIPNN_IP = 0, 1
PIPNN_LEAF_SIMT, PIPNN_LEAF_TC = 0, 1
PIPNN_PREC_FP32, PIPNN_PREC_BF16, PIPNN_PREC_FP8, PIPNN_PREC_INT8, PIPNN_PREC_BF16X3 = 0, 1, 2, 3, 4
PIPNN_PICK_BIDIRECTED, PIPNN_PICK_DIRECTED, PIPNN_PICK_INVERTED = 0, 1, 2
PIPNN_OK = 0

# symbols declared in include/pipnn.h
EXPORTS = ("pipnn_set_stream", "pipnn_last_error", "pipnn_sketch", "pipnn_partition", "pipnn_leaves_free",
           "pipnn_leaf_pick", "pipnn_edges_free", "pipnn_hashprune", "pipnn_final_prune", "pipnn_build",
           "pipnn_free", "pipnn_build_into", "pipnn_get_stats", "pipnn_hashprune_noalloc", "pipnn_build_batched",
           "pipnn_leaf_gram", "pipnn_trim_pool", "pipnn_debug_set_alloc_limit", "pipnn_debug_wait_probe",
           "pipnn_medoid", "pipnn_beam_search", "pipnn_knn_graph")


class PipnnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pipnn error {code}: {msg}")
        self.code = code


class pipnn_params(C.Structure):
    _fields_ = [("c_max", C.c_uint32), ("c_min", C.c_uint32), ("max_leaders", C.c_uint32),
                ("p_samp", C.c_float), ("fanout", C.c_uint32 * 4), ("fanout_levels", C.c_uint32),
                ("leaf_k", C.c_uint32), ("hash_bits", C.c_uint32), ("l_max", C.c_uint32),
                ("R", C.c_uint32), ("alpha", C.c_float), ("final_prune", C.c_int32),
                ("dtype", C.c_int32), ("leaf_engine", C.c_int32), ("hyperplanes", C.c_void_p),
                ("replicas", C.c_uint32), ("prec", C.c_int32), ("wave_members", C.c_uint64),
                ("pick_direction", C.c_int32), ("merge_waves", C.c_uint32)]


class pipnn_graph(C.Structure):
    _fields_ = [("ids", C.c_void_p), ("deg", C.c_void_p), ("n", C.c_uint64), ("R", C.c_uint32),
                ("on_device", C.c_int32)]


class pipnn_leaves(C.Structure):
    _fields_ = [("offsets", C.c_void_p), ("members", C.c_void_p), ("num_leaves", C.c_uint64),
                ("num_members", C.c_uint64), ("levels", C.c_uint32)]


class pipnn_edges(C.Structure):
    _fields_ = [("dst", C.c_void_p), ("src", C.c_void_p), ("dist", C.c_void_p), ("count", C.c_uint64)]


class pipnn_stats(C.Structure):
    _fields_ = [("ms_total", C.c_float), ("ms_sketch", C.c_float), ("ms_partition", C.c_float),
                ("ms_leaf", C.c_float), ("ms_hashprune", C.c_float), ("ms_prune", C.c_float),
                ("ms_leaf_kernel", C.c_float), ("leaf_kernel_launches", C.c_uint32), ("levels", C.c_uint32),
                ("leaves", C.c_uint64), ("leaf_members", C.c_uint64), ("candidates", C.c_uint64),
                ("leaf_pairs", C.c_double), ("leaf_pairs_executed", C.c_double),
                ("kernel_launches", C.c_uint64), ("leaf_full_rows", C.c_uint64), ("waves", C.c_uint32),
                ("hashprune_merges", C.c_uint32), ("peak_device_bytes", C.c_uint64), ("ms_prune_kernel", C.c_float),
                ("pad2_", C.c_uint32), ("reservoir_slots", C.c_uint64)]


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        vp, u64, u32, i32, f32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32, C.c_float
        L.pipnn_set_stream.argtypes = [vp]
        L.pipnn_last_error.restype = C.c_char_p
        L.pipnn_sketch.argtypes = [vp, u64, u32, i32, vp, u32, vp, vp]
        L.pipnn_partition.argtypes = [vp, u64, u32, i32, C.POINTER(pipnn_params), u64, C.POINTER(pipnn_leaves)]
        L.pipnn_leaves_free.argtypes = [C.POINTER(pipnn_leaves)]
        L.pipnn_leaves_free.restype = None
        L.pipnn_leaf_pick.argtypes = [vp, u64, u32, i32, i32, vp, vp, u64, u32, i32, i32, i32, C.POINTER(pipnn_edges)]
        L.pipnn_leaf_gram.argtypes = [vp, u64, u32, i32, vp, vp, u64, i32, vp]
        L.pipnn_edges_free.argtypes = [C.POINTER(pipnn_edges)]
        L.pipnn_edges_free.restype = None
        L.pipnn_hashprune.argtypes = [vp, vp, vp, u64, vp, u32, u64, u32, vp, vp]
        L.pipnn_hashprune_noalloc.argtypes = [vp, vp, vp, u64, vp, u32, u64, u32, vp, vp]
        L.pipnn_final_prune.argtypes = [vp, u64, u32, i32, i32, vp, vp, u32, u32, f32, i32, vp, vp]
        L.pipnn_build.argtypes = [vp, u64, u32, i32, C.POINTER(pipnn_params), u64, i32, C.POINTER(pipnn_graph)]
        L.pipnn_free.argtypes = [C.POINTER(pipnn_graph)]
        L.pipnn_free.restype = None
        L.pipnn_build_into.argtypes = [vp, u64, u32, i32, C.POINTER(pipnn_params), u64, vp, vp]
        L.pipnn_build_batched.argtypes = [C.POINTER(C.c_void_p), C.POINTER(C.c_uint64), u32, u32, i32,
                                          C.POINTER(pipnn_params), C.POINTER(C.c_uint64), C.POINTER(pipnn_graph)]
        L.pipnn_get_stats.argtypes = [C.POINTER(pipnn_stats)]
        L.pipnn_debug_set_alloc_limit.argtypes = [u64]
        L.pipnn_debug_wait_probe.argtypes = [u64]
        L.pipnn_medoid.argtypes = [vp, u64, u32, i32, C.POINTER(C.c_uint32)]
        L.pipnn_beam_search.argtypes = [vp, u64, u32, i32, i32, vp, vp, u32, vp, u64, u32, u32, u32, vp,
                                        C.POINTER(C.c_uint64)]
        L.pipnn_knn_graph.argtypes = [vp, u64, u32, i32, i32, vp, vp, u32, u32, u32, u32, vp,
                                      C.POINTER(C.c_uint64)]
        _lib = L
    return _lib


def _check(rc):
    if rc != PIPNN_OK:
        raise PipnnError(rc, lib().pipnn_last_error().decode(errors="replace"))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def dtype_code(t) -> int:
    dt = t.dtype
    if dt in (torch.float32, np.float32):
        return PIPNN_F32
    if dt in (torch.uint8, np.uint8):
        return PIPNN_U8
    if dt in (torch.int8, np.int8):
        return PIPNN_I8
    raise TypeError(f"unsupported point dtype {dt}")


class _DevView:
    """Library-owned device memory seen through __cuda_array_interface__ (copied immediately)."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


def _take(ptr, count, typestr, view=None):
    if count == 0:
        t = torch.empty(0, dtype={"<i4": torch.int32, "<i8": torch.int64, "<f4": torch.float32}[typestr],
                        device="cuda")
    else:
        t = torch.as_tensor(_DevView(ptr, count, typestr), device="cuda").clone()
    return t.view(view) if view is not None else t


def params(dtype=PIPNN_F32, c_max=1024, c_min=None, max_leaders=1000, p_samp=0.005, fanout=(2,), leaf_k=2,
           hash_bits=12, l_max=64, R=64, alpha=1.2, final_prune=True, leaf_engine=PIPNN_LEAF_SIMT,
           hyperplanes=None, replicas=1, prec=PIPNN_PREC_FP32, wave_members=0,
           pick_direction=PIPNN_PICK_BIDIRECTED, merge_waves=0) -> pipnn_params:
    """BP of Alg. 4.  `hyperplanes` (hash_bits x d float32, numpy or torch) must stay alive for the call."""
    p = pipnn_params()
    p.c_max = c_max
    p.c_min = c_max // 16 if c_min is None else c_min
    p.max_leaders = max_leaders
    p.p_samp = p_samp
    for i in range(4):
        p.fanout[i] = fanout[i] if i < len(fanout) else 1
    p.fanout_levels = len(fanout)
    p.leaf_k = leaf_k
    p.hash_bits = hash_bits
    p.l_max = l_max
    p.R = R
    p.alpha = alpha
    p.final_prune = 1 if final_prune else 0
    p.dtype = dtype
    p.leaf_engine = leaf_engine
    p.hyperplanes = _ptr(hyperplanes)
    p.replicas = replicas
    p.prec = prec
    p.wave_members = wave_members
    p.pick_direction = pick_direction
    p.merge_waves = merge_waves
    p._keep = hyperplanes
    return p


def pipnn_set_stream(stream=None):
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    _check(lib().pipnn_set_stream(C.c_void_p(s)))


def pipnn_last_error() -> str:
    return lib().pipnn_last_error().decode(errors="replace")


def pipnn_sketch(points: torch.Tensor, hyperplanes: torch.Tensor):
    """A0: returns (sketch n x m float32, squared norms n: float32 for float data, int32 for bytes)."""
    n, d = points.shape
    m = hyperplanes.shape[0]
    S = torch.empty((n, m), dtype=torch.float32, device=points.device)
    nrm = torch.empty(n, dtype=torch.float32 if points.dtype == torch.float32 else torch.int32,
                      device=points.device)
    pipnn_set_stream()
    _check(lib().pipnn_sketch(_ptr(points), n, d, dtype_code(points), _ptr(hyperplanes), m, _ptr(S), _ptr(nrm)))
    return S, nrm


def pipnn_partition(points: torch.Tensor, bp: pipnn_params, seed: int, metric=PIPNN_L2):
    """A1: returns (offsets uint64 [L+1], members uint32, levels)."""
    n, d = points.shape
    out = pipnn_leaves()
    pipnn_set_stream()
    _check(lib().pipnn_partition(_ptr(points), n, d, metric, C.byref(bp), seed, C.byref(out)))
    try:
        off = _take(out.offsets, out.num_leaves + 1, "<i8", torch.uint64)
        mem = _take(out.members, out.num_members, "<i4", torch.uint32)
        levels = out.levels
    finally:
        lib().pipnn_leaves_free(C.byref(out))
    return off, mem, levels


def pipnn_leaf_pick(points: torch.Tensor, offsets: torch.Tensor, members: torch.Tensor, k=2, metric=PIPNN_L2,
                    engine=PIPNN_LEAF_SIMT, prec=PIPNN_PREC_FP32, direction=PIPNN_PICK_BIDIRECTED):
    """A2-A4: returns (dst uint32, src uint32, dist float32) candidate edges."""
    n, d = points.shape
    out = pipnn_edges()
    pipnn_set_stream()
    _check(lib().pipnn_leaf_pick(_ptr(points), n, d, dtype_code(points), metric, _ptr(offsets), _ptr(members),
                                 offsets.numel() - 1, k, engine, prec, direction, C.byref(out)))
    try:
        dst = _take(out.dst, out.count, "<i4", torch.uint32)
        src = _take(out.src, out.count, "<i4", torch.uint32)
        dist = _take(out.dist, out.count, "<f4")
    finally:
        lib().pipnn_edges_free(C.byref(out))
    return dst, src, dist


def pipnn_leaf_gram(points: torch.Tensor, offsets: torch.Tensor, members: torch.Tensor, prec, metric=PIPNN_L2):
    """The reduced-precision engine's leaf dissimilarities before the re-rank: a flat float32
    tensor holding every leaf's |b| x |b| block in leaf order."""
    n, d = points.shape
    o = offsets.view(torch.int64) if offsets.dtype == torch.uint64 else offsets.to(torch.int64)
    sizes = o[1:] - o[:-1]
    total = int((sizes * sizes).sum())
    gram = torch.empty(max(total, 1), dtype=torch.float32, device=points.device)
    pipnn_set_stream()
    _check(lib().pipnn_leaf_gram(_ptr(points), n, d, metric, _ptr(offsets), _ptr(members), offsets.numel() - 1, prec,
                                 _ptr(gram)))
    return gram[:total]


def pipnn_hashprune(dst, src, dist, sketch, n, l_max, reservoir=None, count=None):
    """A5: merges the candidates into (reservoir n x l_max uint64, count n uint32), in place if given."""
    m = sketch.shape[1]
    dev = sketch.device
    if reservoir is None:
        reservoir = torch.full((n, l_max), -1, dtype=torch.int64, device=dev).view(torch.uint64)
    if count is None:
        count = torch.zeros(n, dtype=torch.int32, device=dev).view(torch.uint32)
    pipnn_set_stream()
    _check(lib().pipnn_hashprune(_ptr(dst), _ptr(src), _ptr(dist), dst.numel(), _ptr(sketch), m, n, l_max,
                                 _ptr(reservoir), _ptr(count)))
    return reservoir, count


def pipnn_hashprune_noalloc(dst, src, dist, sketch, n, l_max, reservoir, count):
    """A5 without device allocation (fixed 64 MiB library scratch); reservoir/count are updated
    in place and must be provided by the caller."""
    m = sketch.shape[1]
    pipnn_set_stream()
    _check(lib().pipnn_hashprune_noalloc(_ptr(dst), _ptr(src), _ptr(dist), dst.numel(), _ptr(sketch), m, n, l_max,
                                         _ptr(reservoir), _ptr(count)))
    return reservoir, count


def pipnn_final_prune(points, reservoir, count, R, alpha, metric=PIPNN_L2, engine=PIPNN_LEAF_SIMT):
    """A6: returns (adjacency n x R uint32 padded with 0xFFFFFFFF, degree n uint32)."""
    n, d = points.shape
    l_max = reservoir.shape[1]
    adj = torch.empty((n, R), dtype=torch.int32, device=points.device).view(torch.uint32)
    deg = torch.empty(n, dtype=torch.int32, device=points.device).view(torch.uint32)
    pipnn_set_stream()
    _check(lib().pipnn_final_prune(_ptr(points), n, d, dtype_code(points), metric, _ptr(reservoir), _ptr(count),
                                   l_max, R, alpha, engine, _ptr(adj), _ptr(deg)))
    return adj, deg


def pipnn_build(points, bp: pipnn_params, seed: int, metric=PIPNN_L2, graph_on_host=False):
    """Alg. 4 end to end.  points: torch tensor (cuda or cpu) or numpy array.  Returns
    (adjacency n x R uint32, degree n uint32) as torch tensors on the device, or numpy arrays on
    the host when graph_on_host is set."""
    n, d = points.shape
    bp.dtype = dtype_code(points)
    g = pipnn_graph()
    pipnn_set_stream()
    _check(lib().pipnn_build(_ptr(points), n, d, metric, C.byref(bp), seed, 1 if graph_on_host else 0, C.byref(g)))
    try:
        R = g.R
        if g.on_device:
            adj = _take(g.ids, n * R, "<i4", torch.uint32).view(n, R)
            deg = _take(g.deg, n, "<i4", torch.uint32)
        else:
            adj = np.ctypeslib.as_array((C.c_uint32 * (n * R)).from_address(g.ids)).reshape(n, R).copy()
            deg = np.ctypeslib.as_array((C.c_uint32 * n).from_address(g.deg)).copy()
    finally:
        lib().pipnn_free(C.byref(g))
    return adj, deg


def pipnn_build_into(points, bp: pipnn_params, seed: int, adj, deg, metric=PIPNN_L2):
    """Alg. 4 end to end into caller-owned adj (n x R) / deg (n) uint32 buffers, host or device
    (torch tensors or numpy arrays)."""
    n, d = points.shape
    bp.dtype = dtype_code(points)
    pipnn_set_stream()
    _check(lib().pipnn_build_into(_ptr(points), n, d, metric, C.byref(bp), seed, _ptr(adj), _ptr(deg)))
    return adj, deg


def pipnn_build_batched(points_list, bp: pipnn_params, seeds, metric=PIPNN_L2):
    """Alg. 4 for several independent indexes of one dimension and dtype (torch tensors or numpy
    arrays, host or device), seeds[i] for index i.  Returns a list of (adjacency n_i x R uint32,
    degree n_i uint32) device tensors."""
    count = len(points_list)
    if count != len(seeds):
        raise ValueError("one seed per index")
    d = points_list[0].shape[1] if count else 0
    if any(p.shape[1] != d or dtype_code(p) != dtype_code(points_list[0]) for p in points_list):
        raise ValueError("every index needs the same dimension and dtype")
    if count:
        bp.dtype = dtype_code(points_list[0])
    ptrs = (C.c_void_p * max(1, count))(*[_ptr(p) for p in points_list])
    ns = (C.c_uint64 * max(1, count))(*[p.shape[0] for p in points_list])
    sd = (C.c_uint64 * max(1, count))(*[int(s) for s in seeds])
    outs = (pipnn_graph * max(1, count))()
    pipnn_set_stream()
    _check(lib().pipnn_build_batched(ptrs, ns, count, d, metric, C.byref(bp), sd, outs))
    graphs = []
    try:
        for i, p in enumerate(points_list):
            n, R = p.shape[0], outs[i].R
            graphs.append((_take(outs[i].ids, n * R, "<i4", torch.uint32).view(n, R),
                           _take(outs[i].deg, n, "<i4", torch.uint32)))
    finally:
        for i in range(count):
            lib().pipnn_free(C.byref(outs[i]))
    return graphs


def pipnn_debug_set_alloc_limit(nbytes):
    """Caps the device bytes the library may allocate (0 lifts the cap): failure injection."""
    _check(lib().pipnn_debug_set_alloc_limit(int(nbytes)))


def pipnn_debug_wait_probe(limit_ns):
    """The engines' bounded wait on an mbarrier nothing completes; raises PipnnError(-4) after
    limit_ns."""
    _check(lib().pipnn_debug_wait_probe(int(limit_ns)))


def pipnn_medoid(points) -> int:
    """The search start for byte data: the point nearest to the exact mean (device points)."""
    n, d = points.shape
    out = C.c_uint32(0)
    pipnn_set_stream()
    _check(lib().pipnn_medoid(_ptr(points), n, d, dtype_code(points), C.byref(out)))
    return int(out.value)


def pipnn_beam_search(points, adj, deg, queries, L, k=10, start=None, metric=PIPNN_L2):
    """Alg. 1 for every row of queries (device tensors).  start None: pipnn_medoid's start (byte
    data).  Returns (ids nq x k uint32 on the device, number of dissimilarity evaluations)."""
    n, d = points.shape
    nq = queries.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=points.device).view(torch.uint32)
    nd = C.c_uint64(0)
    if start is None:
        start = pipnn_medoid(points)
    pipnn_set_stream()
    _check(lib().pipnn_beam_search(_ptr(points), n, d, dtype_code(points), metric, _ptr(adj), _ptr(deg),
                                   adj.shape[1], _ptr(queries), nq, int(start), L, k, _ptr(ids), C.byref(nd)))
    return ids, int(nd.value)


def pipnn_knn_graph(points, adj, deg, L, k=10, start=None, metric=PIPNN_L2):
    """k-NN graph construction with the built graph (Sec. 5): every point queries with itself.
    start None: pipnn_medoid's start (byte data).  Returns (knn n x k uint32 on the device,
    number of dissimilarity evaluations)."""
    n, d = points.shape
    knn = torch.empty((n, k), dtype=torch.int32, device=points.device).view(torch.uint32)
    nd = C.c_uint64(0)
    pipnn_set_stream()
    _check(lib().pipnn_knn_graph(_ptr(points), n, d, dtype_code(points), metric, _ptr(adj), _ptr(deg),
                                 adj.shape[1], 0xFFFFFFFF if start is None else int(start), L, k, _ptr(knn),
                                 C.byref(nd)))
    return knn, int(nd.value)


def pipnn_trim_pool():
    """Releases the device memory the library's pool keeps between builds."""
    _check(lib().pipnn_trim_pool())


def pipnn_get_stats() -> dict:
    st = pipnn_stats()
    _check(lib().pipnn_get_stats(C.byref(st)))
    return {name: getattr(st, name) for name, _ in pipnn_stats._fields_}
