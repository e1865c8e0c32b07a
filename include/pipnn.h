/*
 * pipnn.h -- C ABI of the GB300 (sm_103a) PiPNN index-build library.
 *
 * PiPNN (Pick-in-Partitions Nearest Neighbors, arXiv 2602.21247) builds a graph index for
 * approximate nearest-neighbour search without beam search (Alg. 4):
 *   A0  sketches:   Sketch(v) = [v . H_i] for the m random hyperplanes of Sec. 3
 *   A1  partition:  randomized ball carving with multi-level fanout and Merge (Alg. 5)
 *   A2-A4 pick:     all-pairs dissimilarities inside every leaf and the bi-directed k-NN
 *                   candidate edges (Sec. 4.2, App. A.3)
 *   A5  HashPrune:  candidates streamed into per-node reservoirs of at most l_max slots (Alg. 3)
 *   A6  prune:      RobustPrune of every reservoir down to degree R (Alg. 2, Sec. 4.3)
 *
 * Conventions for every entry point:
 *  - Status: 0 on success, a negative PIPNN_E* code otherwise; pipnn_last_error() returns a
 *    message for the calling thread's last failure.  A failed call writes no partial output
 *    object (graph, leaves, edges) and frees everything it allocated.
 *  - Pointers are device pointers unless the entry point says "host or device"; those accept
 *    either and detect which with cudaPointerGetAttributes.  Inputs are read only and remain
 *    owned by the caller.
 *  - Work is issued on the stream set by pipnn_set_stream (default: the legacy default stream)
 *    on the current CUDA device.  Entry points return after their results are complete (they
 *    synchronise that stream).
 *  - Points are n rows of d elements, row-major and contiguous, of type PIPNN_F32 (float),
 *    PIPNN_U8 (uint8) or PIPNN_I8 (int8).  n < 2^32 - 1 (point ids are 32-bit).
 *  - Dissimilarity (Sec. 2): PIPNN_L2 is the squared Euclidean distance, PIPNN_IP is
 *    1 - <x, y> (for unit-norm data half the squared distance; float data only).  For float
 *    data every decision (leader choice, pick, prune) uses the binary32 value accumulated with
 *    one fused multiply-add per coordinate in index order; for byte data the exact integer.
 *  - Library-owned outputs live in device memory allocated from the stream-ordered pool and are
 *    released by the matching *_free call.
 */
#ifndef PIPNN_H
#define PIPNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIPNN_OK 0
#define PIPNN_EINVAL (-1)      /* invalid argument or parameter (message says which)         */
#define PIPNN_ENOMEM (-2)      /* device or host allocation failed                            */
#define PIPNN_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed                 */
#define PIPNN_ETIMEOUT (-4)    /* a bounded device-side wait gave up                          */
#define PIPNN_EUNSUPPORTED (-5)/* valid but unsupported combination (e.g. IP on byte data)    */

enum { PIPNN_F32 = 0, PIPNN_U8 = 1, PIPNN_I8 = 2 };
enum { PIPNN_L2 = 0, PIPNN_IP = 1 };

/* Engine of the distance contractions: the leaf all-pairs step (A2) and the leader assignment
 * of Alg. 5 (A1).  Both engines give identical results.
 *  PIPNN_LEAF_SIMT: CUDA-core arithmetic in the defining order (binary32 FMA chain / exact
 *                   integer dot products).
 *  PIPNN_LEAF_TC:   tcgen05 tensor-core tiles with BF16 operands and FP32 accumulation in TMEM
 *                   that produce n_j - 2<x_i, x_j> directly (the norm enters as extra K
 *                   columns).  For byte data with d <= 128 every product and partial sum is an
 *                   integer below 2^24, so the result is exact.  Float data runs the leaf
 *                   step at the reduced precision chosen by pipnn_params.prec (BF16 or FP8,
 *                   below) with an exact re-rank; the leaf step returns PIPNN_EUNSUPPORTED for
 *                   d > 128 and for float data at PIPNN_PREC_FP32; the assignment (byte data,
 *                   d <= 128, fanout of the level <= 16) and the final prune (byte data,
 *                   d <= 128, l_max <= 127) run on the tensor cores where they apply and on the
 *                   CUDA cores otherwise. */
enum { PIPNN_LEAF_SIMT = 0, PIPNN_LEAF_TC = 1 };

/* App. A.3 leaf-pick variants (pipnn_params.pick_direction, pipnn_leaf_pick's direction). */
enum { PIPNN_PICK_BIDIRECTED = 0, PIPNN_PICK_DIRECTED = 1, PIPNN_PICK_INVERTED = 2 };

/* Operand precision of the leaf Gram GEMM on the tensor cores (Sec. 4.2 forms the leaf's
 * all-pairs distances with a GEMM; the conclusion names quantised GEMMs as the next step).
 * Every precision gives the same picks -- those of the defining binary32 / exact-integer
 * dissimilarity -- so the graph does not depend on it:
 *  PIPNN_PREC_FP32: the defining precision.  Float data runs the leaf step on the CUDA cores
 *                   (the tensor-core engine rejects it); byte data runs exactly on either engine.
 *  PIPNN_PREC_BF16: float data on PIPNN_LEAF_TC: leaf-centred BF16 operands, FP32 accumulation
 *                   in TMEM, then the candidates within a proven error band of every row's k-th
 *                   are re-ranked with the defining binary32 evaluation (rows whose band does
 *                   not fit the tracked candidates are evaluated in full).
 *  PIPNN_PREC_FP8:  as BF16 with e4m3 operands and one scale per leaf (448 over the leaf's
 *                   largest centred coordinate).
 *  PIPNN_PREC_INT8: byte data only; the exact integer Gram (the tensor-core engine holds u8 / i8
 *                   values exactly in BF16 with FP32 accumulation, exact for d <= 128).
 *  PIPNN_PREC_BF16X3: float data on PIPNN_LEAF_TC: every centred coordinate split into a BF16
 *                   high part and a BF16 remainder, and the Gram formed from three BF16 products
 *                   (hi.hi + lo.hi + hi.lo) with FP32 accumulation: relative operand error about
 *                   2^-16 instead of 2^-8, so the error band stays narrower than the gaps between
 *                   a row's nearest neighbours even in leaves whose spread is far larger than
 *                   those distances, where single BF16 or FP8 leave most rows to the full
 *                   evaluation.
 * For byte data every precision is exact and they are interchangeable. */
enum { PIPNN_PREC_FP32 = 0, PIPNN_PREC_BF16 = 1, PIPNN_PREC_FP8 = 2, PIPNN_PREC_INT8 = 3, PIPNN_PREC_BF16X3 = 4 };

/* Hyper-parameters BP of Alg. 4. */
typedef struct pipnn_params {
    uint32_t c_max;         /* Alg. 5: maximum leaf size C_max (>= 2)                           */
    uint32_t c_min;         /* Alg. 5 Merge: buckets smaller than C_min are merged (<= C_max)   */
    uint32_t max_leaders;   /* Sec. 4.1: cap on leaders per subproblem (2..1024)                */
    float p_samp;           /* Sec. 4.1: leaders = max(2, min(ceil(p_samp*|P|), cap)), (0, 1]   */
    uint32_t fanout[4];     /* Sec. 4.1 multi-level fanout: fanout at depth 0..3 (1..32)       */
    uint32_t fanout_levels; /* number of valid fanout entries; deeper levels use fanout 1       */
    uint32_t leaf_k;        /* App. A.3: k of the bi-directed k-NN pick (1..16)                 */
    uint32_t hash_bits;     /* Sec. 3: m, number of hyperplanes / hash bits (1..16)             */
    uint32_t l_max;         /* Alg. 3: reservoir capacity (1..256)                              */
    uint32_t R;             /* Alg. 2: final degree bound (1..l_max)                            */
    float alpha;            /* Alg. 2: pruning factor (>= 1), applied as alpha^2 on D           */
    int32_t final_prune;    /* Alg. 4 BP.final_prune: 1 = RobustPrune every node, 0 = keep the
                               first R reservoir entries in (distance, id) order               */
    int32_t dtype;          /* PIPNN_F32 / PIPNN_U8 / PIPNN_I8                                  */
    int32_t leaf_engine;    /* PIPNN_LEAF_SIMT / PIPNN_LEAF_TC                                  */
    const float *hyperplanes; /* Sec. 3: the m x d random hyperplanes H (row i = H_i), float32,
                                 host or device; required                                      */
    uint32_t replicas;      /* Sec. 4.1 replication (Sec. 5 "extra replicate"): independent RBC
                               copies whose candidates feed the same HashPrune reservoirs
                               (1..16; 0 means 1).  Replica r partitions with the seed
                               seed + r * 0x9E3779B97F4A7C15 (mod 2^64), so replica 0 is the
                               single-replica build.                                          */
    int32_t prec;           /* PIPNN_PREC_*: operand precision of the tensor-core leaf Gram      */
    uint64_t wave_members;  /* A2..A4 run in waves of consecutive leaves holding at most this many
                               members (a larger leaf forms a wave of its own), which bounds the
                               staging memory; A5 merges the candidates of a group of waves
                               (merge_waves) into the reservoirs before the next group's are
                               formed, which bounds the candidate memory.  By the history
                               independence of Alg. 3 (Sec. 3) the graph does not depend on the
                               split.  0: sized from the free device memory (one wave whenever
                               everything fits).                                              */
    int32_t pick_direction; /* App. A.3 leaf-pick variant: PIPNN_PICK_BIDIRECTED (Sec. 4.2's
                               choice: both edges of every picked pair), PIPNN_PICK_DIRECTED
                               (only member -> neighbour: the neighbour enters the member's
                               reservoir) or PIPNN_PICK_INVERTED (only neighbour -> member)  */
    uint32_t merge_waves;   /* leaf waves whose candidates HashPrune merges into the reservoirs
                               together (their candidate edges are kept until then): k = after
                               every k waves, 0 = automatic (as many consecutive waves as the
                               memory left beside the leaf step holds; with wave_members also
                               0, the leaf waves are then sized a quarter of that).  Like the
                               wave split, the grouping does not change the graph.            */
} pipnn_params;

/* Output graph: ids[v*R + j] for j < deg[v] are v's out-neighbours in prune order; the rest of
 * the row is 0xFFFFFFFF. */
typedef struct pipnn_graph {
    uint32_t *ids;
    uint32_t *deg;
    uint64_t n;
    uint32_t R;
    int32_t on_device;      /* 1: ids/deg are device memory; 0: pinned host memory              */
} pipnn_graph;

/* Leaves of the partition: leaf b holds members[offsets[b] .. offsets[b+1]). */
typedef struct pipnn_leaves {
    uint64_t *offsets;      /* num_leaves + 1 entries, device                                    */
    uint32_t *members;      /* point ids, device                                                 */
    uint64_t num_leaves;
    uint64_t num_members;
    uint32_t levels;        /* recursion levels of Alg. 5 that carved at least one subproblem   */
} pipnn_leaves;

/* Candidate edges: dst[e] receives src[e] at dissimilarity dist[e]. */
typedef struct pipnn_edges {
    uint32_t *dst;
    uint32_t *src;
    float *dist;            /* binary32 value of the dissimilarity (byte data: exact integer
                               converted to binary32, round to nearest)                       */
    uint64_t count;
} pipnn_edges;

/* Timings (CUDA events on the library stream) and counters of the last pipnn_build. */
typedef struct pipnn_stats {
    float ms_total, ms_sketch, ms_partition, ms_leaf, ms_hashprune, ms_prune;
    float ms_leaf_kernel;        /* summed duration of the leaf all-pairs kernel launches       */
    uint32_t leaf_kernel_launches;
    uint32_t levels;
    uint64_t leaves, leaf_members, candidates;
    double leaf_pairs;           /* sum over leaves of |b| (|b| - 1), the unordered-pair work x2 */
    double leaf_pairs_executed;  /* sum over leaves of |b|^2: the full square the leaf kernels
                                    evaluate (both orders and the diagonal; the tensor-core
                                    kernel also evaluates the padding of ragged tiles)          */
    uint64_t kernel_launches;    /* kernels this library launched during the build              */
    uint64_t leaf_full_rows;     /* reduced-precision leaf engine: rows whose error band did not
                                    fit the tracked candidates and were evaluated in full        */
    uint32_t waves;              /* leaf waves of the build (summed over replicas)              */
    uint32_t hashprune_merges;   /* HashPrune merges of the build (summed over replicas): one per
                                    group of merge_waves leaf waves                            */
    uint64_t peak_device_bytes;  /* device memory in use (total minus free, so including memory
                                    the allocators hold in reserve) at the fullest point the
                                    build sampled: after the partition and inside every wave  */
    float ms_prune_kernel;       /* duration of the final prune's kernel launch (A6, without
                                    the staging of its operand rows)                           */
    uint32_t pad2_;
    uint64_t reservoir_slots;    /* sum over nodes of the final reservoir sizes: the candidates
                                    the final prune reads                                       */
} pipnn_stats;

/* Sets the CUDA stream (a cudaStream_t, or NULL for the default stream) used by later calls. */
int pipnn_set_stream(void *stream);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *pipnn_last_error(void);

/* A0 -- sketches and squared norms (Sec. 3 "Implementation").
 * points: n x d device; hyperplanes: m x d float32 device; sketch: n x m float32 device output,
 * sketch[p*m + i] = sum_t x_t * H_i[t] as a binary32 FMA chain in index order; sqnorm: n
 * entries device output (may be NULL): float32 FMA chain for float data, exact int32 for byte
 * data (reinterpret the buffer).  Non-finite float input returns PIPNN_EINVAL. */
int pipnn_sketch(const void *points, uint64_t n, uint32_t d, int32_t dtype, const float *hyperplanes,
                 uint32_t m, float *sketch, void *sqnorm);

/* A1 -- Alg. 5 randomized ball carving with multi-level fanout and Merge, seeded by `seed`
 * (determinism lemma, App. A.5: the result is a function of the inputs and the seed).
 * points: device.  On success *out holds library-owned device arrays; free with
 * pipnn_leaves_free.  Leaves are listed in no particular order; members inside a leaf are in
 * no particular order and distinct.  The leader assignment runs on bp->leaf_engine. */
int pipnn_partition(const void *points, uint64_t n, uint32_t d, int32_t metric, const pipnn_params *bp,
                    uint64_t seed, pipnn_leaves *out);
void pipnn_leaves_free(pipnn_leaves *leaves);

/* A2-A4 -- for every leaf (offsets/members as produced by pipnn_partition, device, distinct
 * members), the k nearest other members of every member by (dissimilarity, id), emitted in both
 * directions (Sec. 4.2, App. A.3): 2 * |b| * min(k, |b|-1) edges per leaf, in no particular
 * order; direction PIPNN_PICK_DIRECTED / _INVERTED keeps one edge of each pair (half as many).  engine: PIPNN_LEAF_SIMT or PIPNN_LEAF_TC; prec: PIPNN_PREC_* (float data on the
 * tensor cores needs BF16, FP8 or BF16X3; the edges are the same for every engine and precision).  Free
 * the result with pipnn_edges_free. */
int pipnn_leaf_pick(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric,
                    const uint64_t *offsets, const uint32_t *members, uint64_t num_leaves,
                    uint32_t k, int32_t engine, int32_t prec, int32_t direction, pipnn_edges *out);
void pipnn_edges_free(pipnn_edges *edges);

/* The leaf dissimilarities as the reduced-precision tensor-core engine forms them (Sec. 4.2's
 * leaf GEMM at BF16 or FP8 operands, before the exact re-rank), for error reports against FP64:
 * for leaf b, gram[g_b + i |b| + j] = D~(members[off_b + i], members[off_b + j]) with
 * g_b = sum over earlier leaves of |c|^2 (the diagonal included).  points: float32, n x d,
 * device; offsets/members as for pipnn_leaf_pick; prec: PIPNN_PREC_BF16, _FP8 or _BF16X3;
 * gram: caller-owned device buffer of sum |b|^2 floats.  The picks never use these values
 * directly: every pick is re-ranked with the defining binary32 evaluation. */
int pipnn_leaf_gram(const void *points, uint64_t n, uint32_t d, int32_t metric, const uint64_t *offsets,
                    const uint32_t *members, uint64_t num_leaves, int32_t prec, float *gram);

/* A5 -- Alg. 3 HashPrune of a candidate stream into the reservoirs of n nodes.
 * dst/src/dist: `count` candidates, device.  sketch: n x m float32 device (from pipnn_sketch).
 * reservoir: n x l_max uint64 device, in/out; count_inout: n uint32 device, in/out (0 = empty).
 * Slot layout: [ordered bf16(dist):16][src:32][h_dst(src):16]; unsigned order of slots is
 * (distance, id).  h_p(c) bit i = [Sketch(c)_i >= Sketch(p)_i] (Eq. 1).  On return node v's
 * slots are reservoir[v*l_max .. + count[v]) in ascending order, the rest 0xFF..FF.  By the
 * history-independence theorem (Sec. 3) the result is the l_max smallest per-hash-bucket
 * minima of the old reservoir together with the new candidates, whatever their order; calling
 * twice on two halves of a stream equals one call on the whole.  Self candidates are dropped. */
int pipnn_hashprune(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count,
                    const float *sketch, uint32_t m, uint64_t n, uint32_t l_max, uint64_t *reservoir,
                    uint32_t *count_inout);

/* pipnn_hashprune without any device allocation (the paper has no counterpart; this is a
 * deployment variant of A5).  Some callers cannot call cudaMalloc or let a library do it: a
 * serving process whose own allocator has reserved the GPU's memory up front, or a host thread
 * that must not block on the driver's allocator.  This entry point takes the same arguments
 * and returns the same reservoirs as pipnn_hashprune, bit for bit, but keeps its scratch in a
 * fixed 64 MiB device array inside the library, which every GPU that loads the library holds
 * until the process exits.  The call needs
 *   256 + 8(n+1) + 4n + 8*(ceil(n/4096) + ceil(n/4096^2) + ... + 1) + 8*count  bytes
 * (each term rounded up to 256); larger inputs return PIPNN_EINVAL with the sizes in the
 * message, before any GPU work.  The first call on each device looks up the array's device
 * address (with that device current) and remembers it; make that first call before any stream
 * capture.  The remembered address does not survive cudaDeviceReset: after a reset of a device,
 * do not call this entry point on it again in the same process.  All calls share the array and
 * clear what they need on entry, so calls that overlap
 * on the GPU (different streams or threads on one device) race and must be serialised by the
 * caller.  No cudaMalloc, cudaFree or allocating library routine is called. */
int pipnn_hashprune_noalloc(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count,
                            const float *sketch, uint32_t m, uint64_t n, uint32_t l_max, uint64_t *reservoir,
                            uint32_t *count_inout);

/* A6 -- Alg. 2 RobustPrune of every node's reservoir to at most R neighbours (Sec. 4.3).
 * Candidates are ordered by (dissimilarity to the node, id); candidate z is removed by the
 * admitted y when alpha^2 * D(y,z) < D(x,z), evaluated in binary32 with
 * alpha^2 = (float)((double)alpha * alpha).  points, reservoir (n x l_max), count, adj (n x R)
 * and deg (n) are device pointers.  engine: PIPNN_LEAF_SIMT, or PIPNN_LEAF_TC, which forms every
 * node's candidate Gram matrix on the tensor cores where it applies (byte data, d <= 128,
 * l_max <= 127; elsewhere the CUDA cores).  Both give the same graph. */
int pipnn_final_prune(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric,
                      const uint64_t *reservoir, const uint32_t *count, uint32_t l_max, uint32_t R,
                      float alpha, int32_t engine, uint32_t *adj, uint32_t *deg);

/* Alg. 4 end to end: A0 .. A6 on the GPU.  points: host or device (host input is copied to the
 * device inside the call).  graph_on_host = 1 returns the graph in pinned host memory, 0 in
 * device memory.  Free with pipnn_free. */
int pipnn_build(const void *points, uint64_t n, uint32_t d, int32_t metric, const pipnn_params *bp,
                uint64_t seed, int32_t graph_on_host, pipnn_graph *out);
void pipnn_free(pipnn_graph *graph);

/* Alg. 4 for `count` independent indexes of one dimension d (independent point sets, each with
 * its own seed: points[i] holds n[i] rows, host or device), in one pipeline: the indexes are laid
 * out one after another and partitioned together -- every index with its own seed and with its
 * point ids taken relative to it wherever the randomness of Alg. 5 sees them, so each index gets
 * the leaves a separate build would -- and their leaves, HashPrune and prune share the launches of
 * a single build.  outs[i] receives index i's graph (index-local ids) in device memory; free each
 * with pipnn_free.  On an error no graph is returned (every outs[i] is zeroed).  pipnn_get_stats
 * describes the whole batch. */
int pipnn_build_batched(const void *const *points, const uint64_t *n, uint32_t count, uint32_t d, int32_t metric,
                        const pipnn_params *bp, const uint64_t *seeds, pipnn_graph *outs);

/* Alg. 4 end to end into caller-owned outputs: adj (n x R uint32) and deg (n uint32), host or
 * device pointers, written completely on success (rows padded with 0xFFFFFFFF).  points: host or
 * device.  Allocates only its device workspace. */
int pipnn_build_into(const void *points, uint64_t n, uint32_t d, int32_t metric, const pipnn_params *bp,
                     uint64_t seed, uint32_t *adj, uint32_t *deg);

/* Search start for byte data (u8 / i8): the point nearest to the mean of all points, found
 * exactly as the argmin of the integer sum_t (n x_t - S_t)^2 with S the exact coordinate sums
 * (ties to the smaller index).  The paper does not name a start node for Alg. 1; this is the
 * medoid reading.  points: device, n x d row-major.  Float data: PIPNN_EUNSUPPORTED (the caller
 * passes its own start).  Synchronises the stream. */
int pipnn_medoid(const void *points, uint64_t n, uint32_t d, int32_t dtype, uint32_t *medoid);

/* Alg. 1 (BeamSearch) for nq queries at once: from `start`, repeatedly expand the nearest
 * unvisited node of the beam, evaluate its not yet evaluated out-neighbours, keep the L nearest
 * by (dissimilarity, id); stop when every beam node is visited; return the k nearest.  The
 * dissimilarity is the defining one of Sec. 2 (binary32 fused multiply-add chain in index order
 * for float data, 1 - <x, q> for PIPNN_IP; exact integer squared L2 for byte data), so the result
 * equals a sequential Alg. 1 on the same values.
 *   points: device, n x d (dtype); adj: device, n x R uint32 rows, the first deg[v] entries of row
 *   v are v's out-neighbours (other entries ignored; ids >= n are an error); deg: device, n
 *   uint32; queries: device, nq x d of the same dtype; ids: device, nq x k uint32, written
 *   completely (0xFFFFFFFF where the beam holds fewer than k nodes).  1 <= k <= L <= 512,
 *   1 <= R <= 1024, start < n.  ndist (host, may be NULL) receives the number of dissimilarity
 *   evaluations (each node evaluated at least once per query it reaches; a node may be evaluated
 *   twice when a query's evaluated-id set outgrows its table).  Synchronises the stream. */
int pipnn_beam_search(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric,
                      const uint32_t *adj, const uint32_t *deg, uint32_t R, const void *queries, uint64_t nq,
                      uint32_t start, uint32_t L, uint32_t k, uint32_t *ids, uint64_t *ndist);

/* k-NN graph construction with a built index (Sec. 5): every point p runs Alg. 1 with itself as
 * the query (beam L) and its row of knn (device, n x k uint32) receives the first k beam nodes
 * other than p (0xFFFFFFFF where fewer exist).  start = 0xFFFFFFFF takes pipnn_medoid's start
 * (byte data only).  1 <= k < L <= 512.  Other arguments as pipnn_beam_search. */
int pipnn_knn_graph(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric,
                    const uint32_t *adj, const uint32_t *deg, uint32_t R, uint32_t start, uint32_t L,
                    uint32_t k, uint32_t *knn, uint64_t *ndist);

/* Returns to the driver the device memory the library's stream-ordered pool keeps for reuse
 * between builds (the pool otherwise holds its high-water mark, so that repeated builds of one
 * size allocate nothing new).  Call it between builds of very different sizes, or before handing
 * the memory to another allocator.  Synchronises the device. */
int pipnn_trim_pool(void);

/* Failure injection for tests (no counterpart in the paper).  pipnn_debug_set_alloc_limit caps
 * the device bytes the library may allocate from now on (0 lifts the cap); an allocation beyond
 * it fails exactly as a failed cudaMallocAsync does (PIPNN_ENOMEM, nothing partial returned).
 * pipnn_debug_wait_probe runs the engines' bounded device-side wait on an mbarrier that nothing
 * completes: after limit_ns it must return PIPNN_ETIMEOUT, with the context still usable. */
int pipnn_debug_set_alloc_limit(uint64_t bytes);
int pipnn_debug_wait_probe(uint64_t limit_ns);

/* Statistics of the last successful pipnn_build / pipnn_build_into on the calling thread. */
int pipnn_get_stats(pipnn_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* PIPNN_H */
