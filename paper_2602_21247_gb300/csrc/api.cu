// api.cu -- the extern "C" entry points declared in include/pipnn.h: argument validation,
// host/device input handling, the Alg. 4 pipeline (A0 .. A6) and per-phase timing.
#include "internal.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace pipnn {
void set_stream(cudaStream_t s);
void set_device_error_word(unsigned *p);
int sketch_points(const void *X, uint64_t n, uint32_t d, int dtype, const float *H, uint32_t m, float *S,
                  void *sqnorm);
int partition_points(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
                     const pipnn_params *bp, uint64_t seed, pipnn_leaves *out);
int partition_points_batch(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
                           const pipnn_params *bp, const uint64_t *idx_off, const uint64_t *seeds, uint64_t count,
                           pipnn_leaves *out);
int leaf_pick(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
              const uint64_t *off, const uint32_t *mem, uint64_t L, uint32_t k, int engine, int prec,
              int direction, pipnn_edges *out, float *ms_kernel, uint32_t *launches, uint64_t *full_rows);
int hashprune_merge(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count, const float *S,
                    uint32_t m, uint64_t n, uint32_t l_max, uint64_t *res, uint32_t *cnt, int padded);
int hashprune_merge_segments(const EdgeSegment *seg, uint32_t nseg, const float *S, uint32_t m, uint64_t n,
                             uint32_t l_max, uint64_t *res, uint32_t *cnt, int padded);
int final_prune(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
                const uint64_t *res, const uint32_t *cnt, uint32_t l_max, uint32_t R, float alpha, int engine,
                uint32_t *adj, uint32_t *deg, float *ms_kernel);
int reservoir_total(const uint32_t *cnt, uint64_t n, uint32_t l_max, uint64_t *total);
int reservoir_graph(uint64_t n, const uint64_t *res, const uint32_t *cnt, uint32_t l_max, uint32_t R, uint32_t *adj,
                    uint32_t *deg);
int leaf_gram_tcf(const float *X, uint32_t d, int metric, int prec, const uint64_t *off, const uint32_t *mem,
                  uint64_t L, float *gram, Workspace &ws);
int medoid_bytes(const void *X, uint64_t n, uint32_t d, int dtype, uint32_t *medoid_host, Workspace &ws);
int beam_search_batch(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const uint32_t *adj,
                      const uint32_t *deg, uint32_t R, const void *Q, uint64_t nq, uint32_t start, uint32_t L,
                      uint32_t k, int exclude_self, uint32_t *ids, uint64_t *ndist_host, Workspace &ws);

namespace {
thread_local pipnn_stats g_stats;

// Per-call device error word, installed for the duration of an entry point.
struct CallScope {
    Workspace ws;
    unsigned *err = nullptr;
    int init() {
        clear_error();
        PIPNN_TRY(ws.zeros(&err, 1));
        set_device_error_word(err);
        return PIPNN_OK;
    }
    ~CallScope() { set_device_error_word(nullptr); }
};

size_t elem_size(int dtype) { return dtype == PIPNN_F32 ? 4 : 1; }

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_points(const void *X, uint64_t n, uint32_t d, int dtype, int metric) {
    if (!X) return set_error(PIPNN_EINVAL, "points is NULL");
    if (n == 0) return set_error(PIPNN_EINVAL, "n must be positive");
    if (n >= 0xFFFFFFFFull) return set_error(PIPNN_EINVAL, "n must be below 2^32 - 1");
    if (d == 0) return set_error(PIPNN_EINVAL, "d must be positive");
    if (dtype < PIPNN_F32 || dtype > PIPNN_I8) return set_error(PIPNN_EINVAL, "unknown dtype %d", dtype);
    if (metric != PIPNN_L2 && metric != PIPNN_IP) return set_error(PIPNN_EINVAL, "unknown metric %d", metric);
    if (metric == PIPNN_IP && dtype != PIPNN_F32)
        return set_error(PIPNN_EUNSUPPORTED, "inner product is supported for float data only");
    // the CUDA-core all-pairs kernel keeps a 128-row tile resident in shared memory
    const size_t dw = dtype == PIPNN_F32 ? d : (d + 3) / 4;
    if ((128 + 32) * dw * 4 > 227 * 1024)
        return set_error(PIPNN_EUNSUPPORTED, "d = %u exceeds the resident-tile limit", d);
    return PIPNN_OK;
}

int check_params(const pipnn_params *bp) {
    if (!bp) return set_error(PIPNN_EINVAL, "params is NULL");
    if (bp->c_max < 2) return set_error(PIPNN_EINVAL, "c_max must be at least 2");
    if (bp->c_min > bp->c_max) return set_error(PIPNN_EINVAL, "c_min must not exceed c_max");
    if (bp->max_leaders < 2 || bp->max_leaders > 1024) return set_error(PIPNN_EINVAL, "max_leaders outside 2..1024");
    if (!(bp->p_samp > 0.0f) || !(bp->p_samp <= 1.0f)) return set_error(PIPNN_EINVAL, "p_samp outside (0, 1]");
    if (bp->fanout_levels > 4) return set_error(PIPNN_EINVAL, "fanout_levels above 4");
    for (uint32_t i = 0; i < bp->fanout_levels; i++)
        if (bp->fanout[i] < 1 || bp->fanout[i] > 32) return set_error(PIPNN_EINVAL, "fanout[%u] outside 1..32", i);
    if (bp->leaf_k < 1 || bp->leaf_k > 16) return set_error(PIPNN_EINVAL, "leaf_k outside 1..16");
    if (bp->hash_bits < 1 || bp->hash_bits > 16) return set_error(PIPNN_EINVAL, "hash_bits outside 1..16");
    if (bp->l_max < 1 || bp->l_max > 256) return set_error(PIPNN_EINVAL, "l_max outside 1..256");
    if (bp->R < 1 || bp->R > bp->l_max) return set_error(PIPNN_EINVAL, "R outside 1..l_max");
    if (!(bp->alpha >= 1.0f) || !std::isfinite(bp->alpha)) return set_error(PIPNN_EINVAL, "alpha must be finite and >= 1");
    if (bp->leaf_engine != PIPNN_LEAF_SIMT && bp->leaf_engine != PIPNN_LEAF_TC)
        return set_error(PIPNN_EINVAL, "unknown leaf_engine %d", bp->leaf_engine);
    if (!bp->hyperplanes) return set_error(PIPNN_EINVAL, "hyperplanes is NULL");
    if (bp->replicas > 16) return set_error(PIPNN_EINVAL, "replicas above 16");
    if (bp->pick_direction < PIPNN_PICK_BIDIRECTED || bp->pick_direction > PIPNN_PICK_INVERTED)
        return set_error(PIPNN_EINVAL, "unknown pick_direction %d", bp->pick_direction);
    if (bp->prec < PIPNN_PREC_FP32 || bp->prec > PIPNN_PREC_BF16X3) return set_error(PIPNN_EINVAL, "unknown prec %d", bp->prec);
    if (bp->dtype == PIPNN_F32 && bp->prec == PIPNN_PREC_INT8)
        return set_error(PIPNN_EUNSUPPORTED, "PIPNN_PREC_INT8 takes byte data");
    return PIPNN_OK;
}

struct Timer {
    cudaEvent_t ev[8] = {};
    int init() {
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return set_error(PIPNN_ECUDA, "event creation failed");
        return PIPNN_OK;
    }
    void mark(int i) { cudaEventRecord(ev[i], stream()); }
    float ms(int a, int b) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) cudaGetLastError();
        return t;
    }
    ~Timer() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
};

// sum over leaves of |b| (|b| - 1), in 64-bit integers
__global__ void leaf_pairs_kernel(const uint64_t *off, uint64_t L, unsigned long long *acc) {
    unsigned long long local = 0;
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < L; b += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long s = off[b + 1] - off[b];
        local += s * (s ? s - 1 : 0);
    }
    atomicAdd(acc, local);
}

__global__ void rebase_offsets(const uint64_t *off, uint64_t count, uint64_t *out) {
    const uint64_t base = off[0];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = off[i] - base;
}

int leaf_offsets_to_host(const uint64_t *off, uint64_t L, std::vector<uint64_t> *h) {
    h->assign(L + 1, 0);
    PIPNN_CUDA(cudaMemcpyAsync(h->data(), off, (L + 1) * 8, cudaMemcpyDeviceToHost, stream()));
    PIPNN_CUDA(cudaStreamSynchronize(stream()));
    return PIPNN_OK;
}

// Device memory in use now (total minus free, so including what the allocators hold in reserve),
// kept as the build's peak.
void note_peak(pipnn_stats *st) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const uint64_t used = (uint64_t)(tot - fr);
    if (used > st->peak_device_bytes) st->peak_device_bytes = used;
}

// Leaf waves per HashPrune merge when both are sized automatically: fewer merges mean fewer passes
// over every node's reservoir, at the price of keeping the earlier waves' candidate edges while the
// later ones run their leaf step.
constexpr uint64_t kLeafWavesPerMerge = 4;

// Members of one leaf wave (*wave) and of one HashPrune merge group (*group, consecutive waves whose
// candidate edges are kept and merged together), from the free device memory less the per-node
// HashPrune arrays and a reserve.  A member costs, in the leaf step, the engine's staged operand
// row and per-member buffers plus the 2k candidate edges it writes (12 B each); while its group is
// open, its edges; in the merge, its edges and their 8-byte grouped slots.  A group of G members
// whose last wave has W members needs 12·2k·(G − W) + leaf·W in the leaf step and 20·2k·G in the
// merge.  Waves stay below the tensor maps' 2^31 rows.
void wave_plan(uint64_t n, uint32_t d, int dtype, const pipnn_params *bp, uint64_t *wave, uint64_t *group) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = 0;
    }
    // memory the stream-ordered pool holds but no allocation uses is available too
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            fr += (size_t)(reserved - used);
    }
    cudaGetLastError();
    const uint64_t kp = ((uint64_t)d + 63) / 64 * 64;
    const uint64_t k2 = 2ull * bp->leaf_k;
    uint64_t stage = 32;  // CUDA-core engines read the rows in place
    if (bp->leaf_engine == PIPNN_LEAF_TC) {
        if (dtype != PIPNN_F32) stage = kp * 2 + 12;
        else if (bp->prec == PIPNN_PREC_BF16X3) stage = kp * 4 + 96;
        else if (bp->prec == PIPNN_PREC_FP8) stage = 128 * ((kp + 127) / 128) + 96;
        else stage = kp * 2 + 96;
    }
    const uint64_t keep = k2 * 12, leaf_step = stage + keep + 32, hp_step = k2 * (12 + 8) + 16;
    const uint64_t reserve = (2ull << 30) + 24 * n;
    const uint64_t F = fr > reserve ? fr - reserve : 0;
    const uint64_t lo = 1ull << 20, cap = 0x7FF00000ull;
    uint64_t W = bp->wave_members, G = 0;
    if (!W) {
        // one wave per merge: the larger step bounds it; several: the leaf step of the group's
        // last wave beside the kept edges of the others
        const uint64_t one = leaf_step > hp_step ? leaf_step : hp_step;
        W = F / one;
        if (bp->merge_waves != 1) {
            const uint64_t s = bp->merge_waves ? bp->merge_waves : kLeafWavesPerMerge;
            G = F / (keep + (leaf_step + s - 1) / s);
            if (G > F / hp_step) G = F / hp_step;
            W = G / s;
        }
        if (W < lo) W = lo;
        if (W > cap) W = cap;
    } else if (bp->merge_waves == 0) {
        // caller-sized waves: as many per merge as fit beside one wave's leaf step
        const uint64_t left = F > leaf_step * W ? F - leaf_step * W : 0;
        G = W + left / keep;
        if (G > F / hp_step) G = F / hp_step;
    }
    if (G < W) G = W;
    *wave = W;
    *group = G;
}

// Keeps freed stream-ordered allocations in the device's default pool (the build allocates and
// frees the same large buffers every call).
void keep_pool_memory() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}

// Several independent indexes built by one pipeline (pipnn_build_batched).
struct BatchDesc {
    const void *const *points;  // per index, host or device
    const uint64_t *n;          // per index
    const uint64_t *seeds;      // per index
    uint32_t count;
    pipnn_graph *outs;          // per index, device graphs
};

// Rows lo .. lo + rows of the batch's graph as index-local ids (padding stays 0xFFFFFFFF).
__global__ void local_rows(const uint32_t *adj, const uint32_t *deg, uint64_t lo, uint64_t rows, uint32_t R,
                           uint32_t *out_adj, uint32_t *out_deg) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < rows * R; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = adj[lo * R + i];
        out_adj[i] = v == 0xFFFFFFFFu ? v : v - (uint32_t)lo;
        if (i % R == 0) out_deg[i / R] = deg[lo + i / R];
    }
}

// graph_on_host: 0 device graph, 1 pinned host graph, 2 caller buffers (user_adj/user_deg),
// 3 a batch (batch->outs, device graphs per index)
int build_impl(const void *points, uint64_t n, uint32_t d, int metric, const pipnn_params *bp, uint64_t seed,
               int graph_on_host, pipnn_graph *out, uint32_t *user_adj = nullptr, uint32_t *user_deg = nullptr,
               const BatchDesc *batch = nullptr) {
    memset(out, 0, sizeof(*out));
    // the indexes of the build: one, or a batch laid out one after another
    std::vector<uint64_t> idx_off{0}, idx_seed;
    if (batch) {
        for (uint32_t i = 0; i < batch->count; i++) {
            idx_off.push_back(idx_off.back() + batch->n[i]);
            idx_seed.push_back(batch->seeds[i]);
        }
        n = idx_off.back();
        points = batch->count ? batch->points[0] : nullptr;
    } else {
        idx_off.push_back(n);
        idx_seed.push_back(seed);
    }
    keep_pool_memory();
    PIPNN_TRY(check_params(bp));
    const int dtype = bp->dtype;
    PIPNN_TRY(check_points(points, n, d, dtype, metric));
    if (bp->leaf_engine == PIPNN_LEAF_TC && dtype == PIPNN_F32 && bp->prec != PIPNN_PREC_BF16 &&
        bp->prec != PIPNN_PREC_FP8 && bp->prec != PIPNN_PREC_BF16X3)
        return set_error(PIPNN_EUNSUPPORTED, "float data on the tensor-core leaf engine needs prec BF16, FP8 or BF16X3");
    CallScope cs;
    PIPNN_TRY(cs.init());
    Workspace &ws = cs.ws;
    Timer tm;
    PIPNN_TRY(tm.init());
    pipnn_stats st;
    memset(&st, 0, sizeof(st));
    const uint64_t launches0 = launch_count();
    tm.mark(0);

    // inputs on the device (a batch: every index's points copied one after another)
    const void *X = points;
    if (batch) {
        char *dx = nullptr;
        PIPNN_TRY(ws.alloc(&dx, n * d * elem_size(dtype)));
        for (uint32_t i = 0; i < batch->count; i++)
            if (batch->n[i])
                PIPNN_CUDA(cudaMemcpyAsync(dx + idx_off[i] * d * elem_size(dtype), batch->points[i],
                                           batch->n[i] * d * elem_size(dtype), cudaMemcpyDefault, stream()));
        X = dx;
    } else if (!is_device_ptr(points)) {
        void *dx = nullptr;
        PIPNN_TRY(ws.alloc((char **)&dx, n * d * elem_size(dtype)));
        PIPNN_CUDA(cudaMemcpyAsync(dx, points, n * d * elem_size(dtype), cudaMemcpyHostToDevice, stream()));
        X = dx;
    }
    const uint32_t m = bp->hash_bits;
    const float *H = bp->hyperplanes;
    if (!is_device_ptr(H)) {
        float *dh = nullptr;
        PIPNN_TRY(ws.alloc(&dh, (size_t)m * d));
        PIPNN_CUDA(cudaMemcpyAsync(dh, H, (size_t)m * d * 4, cudaMemcpyHostToDevice, stream()));
        H = dh;
    }

    // A0
    float *S;
    int32_t *sqn;
    PIPNN_TRY(ws.alloc(&S, n * m));
    PIPNN_TRY(ws.alloc(&sqn, n));
    PIPNN_TRY(sketch_points(X, n, d, dtype, H, m, S, sqn));
    tm.mark(1);
    const int32_t *sqn_bytes = dtype == PIPNN_F32 ? nullptr : sqn;

    // A1 .. A5 once per replica (Sec. 4.1 replication): an independent RBC with its own seed whose
    // candidates join the same reservoirs; HashPrune's result does not depend on the order in
    // which candidates arrive (Alg. 3, history independence), so the replicas simply run in turn
    const uint32_t replicas = bp->replicas ? bp->replicas : 1;
    std::vector<Timer> rt(replicas);
    for (auto &t : rt) PIPNN_TRY(t.init());
    unsigned long long *acc;
    PIPNN_TRY(ws.zeros(&acc, 1));
    uint64_t *res = nullptr;
    uint32_t *cnt = nullptr;
    for (uint32_t r = 0; r < replicas; r++) {
        std::vector<uint64_t> seed_r(idx_seed.size());
        for (size_t i = 0; i < idx_seed.size(); i++) seed_r[i] = idx_seed[i] + (uint64_t)r * 0x9E3779B97F4A7C15ull;
        rt[r].mark(0);
        // A1 (every index of a batch with its own seed, in one pass)
        pipnn_leaves leaves;
        PIPNN_TRY(partition_points_batch(X, n, d, dtype, metric, sqn_bytes, bp, idx_off.data(), seed_r.data(),
                                         idx_seed.size(), &leaves));
        rt[r].mark(1);
        st.levels = leaves.levels > st.levels ? leaves.levels : st.levels;
        st.leaves += leaves.num_leaves;
        st.leaf_members += leaves.num_members;
        if (leaves.num_leaves) {
            leaf_pairs_kernel<<<grid_for(leaves.num_leaves, 256, 1024), 256, 0, stream()>>>(leaves.offsets,
                                                                                           leaves.num_leaves, acc);
        }

        // A5's reservoirs (once, for every replica and wave)
        int rc = PIPNN_OK;
        if (r == 0) {
            rc = ws.alloc(&res, n * bp->l_max);
            if (rc == PIPNN_OK) rc = ws.zeros(&cnt, n);
            if (rc == PIPNN_OK) {
                cudaError_t e = cudaMemsetAsync(res, 0xFF, n * bp->l_max * 8, stream());
                if (e != cudaSuccess) rc = set_error(PIPNN_ECUDA, "memset: %s", cudaGetErrorString(e));
            }
        }
        // A2 .. A4 in waves of consecutive leaves, A5 once per group of consecutive waves: a group's
        // candidate edges are kept until its last wave's leaf step is done and are then merged
        // into the reservoirs before the next group's are formed (Alg. 3's history independence
        // makes the result independent of both splits)
        std::vector<uint64_t> hoff;
        uint64_t W = 0, G = 0;
        if (rc == PIPNN_OK) rc = leaf_offsets_to_host(leaves.offsets, leaves.num_leaves, &hoff);
        if (rc == PIPNN_OK) {
            note_peak(&st);
            wave_plan(n, d, dtype, bp, &W, &G);
        }
        std::vector<uint64_t> wave_lo;  // first leaf of every wave, then num_leaves (none after an error)
        for (uint64_t b0 = 0; rc == PIPNN_OK && b0 < leaves.num_leaves;) {
            wave_lo.push_back(b0);
            uint64_t b1 = b0 + 1;
            while (b1 < leaves.num_leaves && hoff[b1 + 1] - hoff[b0] <= W) b1++;
            b0 = b1;
        }
        if (rc == PIPNN_OK) wave_lo.push_back(leaves.num_leaves);
        std::vector<pipnn_edges> group;  // the open group's candidate edges, one entry per wave
        uint64_t group_members = 0;
        auto free_group = [&]() {
            for (auto &e : group) {
                dev_free_raw(e.dst);
                dev_free_raw(e.src);
                dev_free_raw(e.dist);
            }
            group.clear();
            group_members = 0;
        };
        auto merge_group = [&]() -> int {
            Timer mt;
            PIPNN_TRY(mt.init());
            note_peak(&st);
            std::vector<EdgeSegment> seg;
            for (auto &e : group) seg.push_back(EdgeSegment{e.dst, e.src, e.dist, e.count});
            mt.mark(0);
            int r2 = hashprune_merge_segments(seg.data(), (uint32_t)seg.size(), S, m, n, bp->l_max, res, cnt, 1);
            mt.mark(1);
            free_group();
            if (r2 == PIPNN_OK) {
                cudaStreamSynchronize(stream());
                st.ms_hashprune += mt.ms(0, 1);
                st.hashprune_merges++;
            }
            return r2;
        };
        for (size_t wi = 0; rc == PIPNN_OK && wi + 1 < wave_lo.size(); wi++) {
            const uint64_t b0 = wave_lo[wi], b1 = wave_lo[wi + 1], Lw = b1 - b0;
            const uint64_t members = hoff[b1] - hoff[b0];
            // close the open group first if this wave does not fit in it
            if (!group.empty() && (bp->merge_waves ? group.size() >= bp->merge_waves : group_members + members > G))
                rc = merge_group();
            Timer wt;
            if (rc == PIPNN_OK) rc = wt.init();
            uint64_t *off_w = nullptr;
            Workspace wave_ws;
            if (rc == PIPNN_OK) rc = wave_ws.alloc(&off_w, Lw + 1);
            if (rc == PIPNN_OK) {
                wt.mark(0);
                rebase_offsets<<<grid_for(Lw + 1, 256), 256, 0, stream()>>>(leaves.offsets + b0, Lw + 1, off_w);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) rc = set_error(PIPNN_ECUDA, "rebase: %s", cudaGetErrorString(e));
                count_launch();
            }
            if (rc == PIPNN_OK) {
                pipnn_edges edges{};
                float leaf_ms = 0.0f;
                uint32_t leaf_launches = 0;
                uint64_t full_rows = 0;
                rc = leaf_pick(X, n, d, dtype, metric, sqn_bytes, off_w, leaves.members + hoff[b0], Lw, bp->leaf_k,
                               bp->leaf_engine, bp->prec, bp->pick_direction, &edges, &leaf_ms, &leaf_launches,
                               &full_rows);
                if (rc == PIPNN_OK || edges.dst || edges.src || edges.dist) group.push_back(edges);
                group_members += members;
                if (rc == PIPNN_OK) {
                    st.leaf_full_rows += full_rows;
                    st.ms_leaf_kernel += leaf_ms;
                    st.leaf_kernel_launches += leaf_launches;
                    st.candidates += edges.count;
                    wt.mark(1);
                    note_peak(&st);
                    cudaStreamSynchronize(stream());
                    st.ms_leaf += wt.ms(0, 1);
                    st.waves++;
                }
            }
        }
        if (rc == PIPNN_OK && !group.empty()) rc = merge_group();
        free_group();
        dev_free_raw(leaves.offsets);
        dev_free_raw(leaves.members);
        if (rc != PIPNN_OK) return rc;
        rt[r].mark(2);
    }
    unsigned long long leaf_pairs = 0;
    PIPNN_CUDA(cudaMemcpyAsync(&leaf_pairs, acc, 8, cudaMemcpyDeviceToHost, stream()));
    tm.mark(4);
    int rc = PIPNN_OK;

    // A6
    uint32_t *adj = nullptr, *deg = nullptr;
    PIPNN_TRY(dev_alloc_raw((void **)&adj, n * bp->R * 4));
    rc = dev_alloc_raw((void **)&deg, n * 4);
    if (rc == PIPNN_OK) {
        if (bp->final_prune)
            rc = final_prune(X, n, d, dtype, metric, sqn_bytes, res, cnt, bp->l_max, bp->R, bp->alpha, bp->leaf_engine,
                             adj, deg, &st.ms_prune_kernel);
        else
            rc = reservoir_graph(n, res, cnt, bp->l_max, bp->R, adj, deg);
    }
    if (rc == PIPNN_OK) rc = check_device_error("final prune");
    tm.mark(5);
    if (rc == PIPNN_OK) rc = reservoir_total(cnt, n, bp->l_max, &st.reservoir_slots);
    if (rc == PIPNN_OK && graph_on_host == 3) {
        // per index, its rows with index-local ids
        uint32_t i = 0;
        for (; rc == PIPNN_OK && i < batch->count; i++) {
            const uint64_t lo = idx_off[i], rows = batch->n[i];
            pipnn_graph &g = batch->outs[i];
            rc = dev_alloc_raw((void **)&g.ids, rows * bp->R * 4);
            if (rc == PIPNN_OK) rc = dev_alloc_raw((void **)&g.deg, rows * 4);
            if (rc == PIPNN_OK && rows) {
                local_rows<<<grid_for(rows * bp->R, 256), 256, 0, stream()>>>(adj, deg, lo, rows, bp->R, g.ids, g.deg);
                count_launch();
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) rc = set_error(PIPNN_ECUDA, "graph split: %s", cudaGetErrorString(e));
            }
            g.n = rows;
            g.R = bp->R;
            g.on_device = 1;
        }
        if (rc == PIPNN_OK) rc = check_device_error("graph split");
        dev_free_raw(adj);
        dev_free_raw(deg);
        adj = deg = nullptr;
        if (rc != PIPNN_OK) {
            for (uint32_t j = 0; j < batch->count; j++) {
                dev_free_raw(batch->outs[j].ids);
                dev_free_raw(batch->outs[j].deg);
                memset(&batch->outs[j], 0, sizeof(pipnn_graph));
            }
            return rc;
        }
    } else if (rc == PIPNN_OK && graph_on_host == 2) {
        cudaError_t e = cudaMemcpyAsync(user_adj, adj, n * bp->R * 4, cudaMemcpyDefault, stream());
        if (e == cudaSuccess) e = cudaMemcpyAsync(user_deg, deg, n * 4, cudaMemcpyDefault, stream());
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream());
        dev_free_raw(adj);
        dev_free_raw(deg);
        adj = deg = nullptr;
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(PIPNN_ECUDA, "graph copy: %s", cudaGetErrorString(e));
        }
    } else if (rc == PIPNN_OK && graph_on_host) {
        uint32_t *hadj = nullptr, *hdeg = nullptr;
        cudaError_t e = cudaMallocHost(&hadj, n * bp->R * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&hdeg, n * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hadj, adj, n * bp->R * 4, cudaMemcpyDeviceToHost, stream());
        if (e == cudaSuccess) e = cudaMemcpyAsync(hdeg, deg, n * 4, cudaMemcpyDeviceToHost, stream());
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream());
        dev_free_raw(adj);
        dev_free_raw(deg);
        adj = deg = nullptr;
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (hadj) cudaFreeHost(hadj);
            if (hdeg) cudaFreeHost(hdeg);
            return set_error(PIPNN_ECUDA, "graph copy to host: %s", cudaGetErrorString(e));
        }
        out->ids = hadj;
        out->deg = hdeg;
        out->on_device = 0;
    } else if (rc == PIPNN_OK) {
        out->ids = adj;
        out->deg = deg;
        out->on_device = 1;
    }
    if (rc != PIPNN_OK) {
        dev_free_raw(adj);
        dev_free_raw(deg);
        return rc;
    }
    out->n = n;
    out->R = bp->R;
    tm.mark(6);
    cudaStreamSynchronize(stream());
    st.ms_sketch = tm.ms(0, 1);
    for (auto &t : rt) st.ms_partition += t.ms(0, 1);
    st.ms_prune = tm.ms(4, 5);
    st.leaf_pairs = (double)leaf_pairs;
    st.leaf_pairs_executed = st.leaf_pairs + (double)st.leaf_members;
    st.ms_total = tm.ms(0, 6);
    st.kernel_launches = launch_count() - launches0;
    g_stats = st;
    return PIPNN_OK;
}
}  // namespace
}  // namespace pipnn

using namespace pipnn;

extern "C" {

int pipnn_set_stream(void *s) {
    set_stream(static_cast<cudaStream_t>(s));
    return PIPNN_OK;
}

const char *pipnn_last_error(void) { return error_message(); }

int pipnn_sketch(const void *points, uint64_t n, uint32_t d, int32_t dtype, const float *hyperplanes, uint32_t m,
                 float *sketch, void *sqnorm) {
    CallScope cs;
    PIPNN_TRY(cs.init());
    PIPNN_TRY(check_points(points, n, d, dtype, PIPNN_L2));
    if (!hyperplanes || !sketch) return set_error(PIPNN_EINVAL, "hyperplanes and sketch are required");
    if (m < 1 || m > 16) return set_error(PIPNN_EINVAL, "m outside 1..16");
    PIPNN_TRY(sketch_points(points, n, d, dtype, hyperplanes, m, sketch, sqnorm));
    return check_device_error("sketch");
}

int pipnn_partition(const void *points, uint64_t n, uint32_t d, int32_t metric, const pipnn_params *bp, uint64_t seed,
                    pipnn_leaves *out) {
    if (!out) return set_error(PIPNN_EINVAL, "out is NULL");
    memset(out, 0, sizeof(*out));
    CallScope cs;
    PIPNN_TRY(cs.init());
    PIPNN_TRY(check_params(bp));
    PIPNN_TRY(check_points(points, n, d, bp->dtype, metric));
    return partition_points(points, n, d, bp->dtype, metric, nullptr, bp, seed, out);
}

void pipnn_leaves_free(pipnn_leaves *l) {
    if (!l) return;
    dev_free_raw(l->offsets);
    dev_free_raw(l->members);
    cudaStreamSynchronize(stream());
    memset(l, 0, sizeof(*l));
}

int pipnn_leaf_pick(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric, const uint64_t *offsets,
                    const uint32_t *members, uint64_t num_leaves, uint32_t k, int32_t engine, int32_t prec,
                    int32_t direction, pipnn_edges *out) {
    if (!out) return set_error(PIPNN_EINVAL, "out is NULL");
    memset(out, 0, sizeof(*out));
    CallScope cs;
    PIPNN_TRY(cs.init());
    PIPNN_TRY(check_points(points, n, d, dtype, metric));
    if (!offsets || (!members && num_leaves)) return set_error(PIPNN_EINVAL, "offsets/members are NULL");
    if (k < 1 || k > 16) return set_error(PIPNN_EINVAL, "k outside 1..16");
    if (engine != PIPNN_LEAF_SIMT && engine != PIPNN_LEAF_TC) return set_error(PIPNN_EINVAL, "unknown engine");
    if (prec < PIPNN_PREC_FP32 || prec > PIPNN_PREC_BF16X3) return set_error(PIPNN_EINVAL, "unknown prec %d", prec);
    return leaf_pick(points, n, d, dtype, metric, nullptr, offsets, members, num_leaves, k, engine, prec, direction,
                     out, nullptr, nullptr, nullptr);
}

int pipnn_leaf_gram(const void *points, uint64_t n, uint32_t d, int32_t metric, const uint64_t *offsets,
                    const uint32_t *members, uint64_t num_leaves, int32_t prec, float *gram) {
    CallScope cs;
    PIPNN_TRY(cs.init());
    PIPNN_TRY(check_points(points, n, d, PIPNN_F32, metric));
    if (!offsets || !gram || (!members && num_leaves)) return set_error(PIPNN_EINVAL, "offsets/members/gram are NULL");
    PIPNN_TRY(leaf_gram_tcf(static_cast<const float *>(points), d, metric, prec, offsets, members, num_leaves, gram,
                            cs.ws));
    return check_device_error("leaf gram");
}

void pipnn_edges_free(pipnn_edges *e) {
    if (!e) return;
    dev_free_raw(e->dst);
    dev_free_raw(e->src);
    dev_free_raw(e->dist);
    cudaStreamSynchronize(stream());
    memset(e, 0, sizeof(*e));
}

int pipnn_hashprune(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count, const float *sketch,
                    uint32_t m, uint64_t n, uint32_t l_max, uint64_t *reservoir, uint32_t *count_inout) {
    CallScope cs;
    PIPNN_TRY(cs.init());
    if (count && (!dst || !src || !dist)) return set_error(PIPNN_EINVAL, "candidate arrays are NULL");
    if (!sketch || !reservoir || !count_inout) return set_error(PIPNN_EINVAL, "sketch/reservoir/count are NULL");
    if (n == 0 || n >= 0xFFFFFFFFull) return set_error(PIPNN_EINVAL, "n outside 1..2^32-2");
    return hashprune_merge(dst, src, dist, count, sketch, m, n, l_max, reservoir, count_inout, 0);
}

int pipnn_final_prune(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric,
                      const uint64_t *reservoir, const uint32_t *count, uint32_t l_max, uint32_t R, float alpha,
                      int32_t engine, uint32_t *adj, uint32_t *deg) {
    CallScope cs;
    PIPNN_TRY(cs.init());
    PIPNN_TRY(check_points(points, n, d, dtype, metric));
    if (!reservoir || !count || !adj || !deg) return set_error(PIPNN_EINVAL, "NULL array");
    if (l_max < 1 || l_max > 256 || R < 1 || R > l_max) return set_error(PIPNN_EINVAL, "need 1 <= R <= l_max <= 256");
    if (!(alpha >= 1.0f) || !std::isfinite(alpha)) return set_error(PIPNN_EINVAL, "alpha must be finite and >= 1");
    if (engine != PIPNN_LEAF_SIMT && engine != PIPNN_LEAF_TC) return set_error(PIPNN_EINVAL, "unknown engine %d", engine);
    PIPNN_TRY(final_prune(points, n, d, dtype, metric, nullptr, reservoir, count, l_max, R, alpha, engine, adj, deg,
                          nullptr));
    return check_device_error("final prune");
}

int pipnn_build(const void *points, uint64_t n, uint32_t d, int32_t metric, const pipnn_params *bp, uint64_t seed,
                int32_t graph_on_host, pipnn_graph *out) {
    if (!out) return set_error(PIPNN_EINVAL, "out is NULL");
    return build_impl(points, n, d, metric, bp, seed, graph_on_host ? 1 : 0, out);
}

int pipnn_build_into(const void *points, uint64_t n, uint32_t d, int32_t metric, const pipnn_params *bp,
                     uint64_t seed, uint32_t *adj, uint32_t *deg) {
    if (!adj || !deg) return set_error(PIPNN_EINVAL, "adj/deg are NULL");
    pipnn_graph g;
    return build_impl(points, n, d, metric, bp, seed, 2, &g, adj, deg);
}

void pipnn_free(pipnn_graph *g) {
    if (!g) return;
    if (g->on_device) {
        dev_free_raw(g->ids);
        dev_free_raw(g->deg);
        cudaStreamSynchronize(stream());
    } else {
        if (g->ids) cudaFreeHost(g->ids);
        if (g->deg) cudaFreeHost(g->deg);
    }
    memset(g, 0, sizeof(*g));
}

int pipnn_build_batched(const void *const *points, const uint64_t *n, uint32_t count, uint32_t d, int32_t metric,
                        const pipnn_params *bp, const uint64_t *seeds, pipnn_graph *outs) {
    if (count && (!points || !n || !seeds || !outs)) return set_error(PIPNN_EINVAL, "points/n/seeds/outs are NULL");
    for (uint32_t i = 0; i < count; i++) memset(&outs[i], 0, sizeof(pipnn_graph));
    if (count == 0) return PIPNN_OK;
    uint64_t total = 0;
    for (uint32_t i = 0; i < count; i++) {
        if (n[i] == 0) return set_error(PIPNN_EINVAL, "index %u has no points", i);
        if (!points[i]) return set_error(PIPNN_EINVAL, "points[%u] is NULL", i);
        total += n[i];
    }
    if (total >= 0xFFFFFFFFull) return set_error(PIPNN_EINVAL, "the batch holds 2^32 - 1 points or more");
    BatchDesc b{points, n, seeds, count, outs};
    pipnn_graph whole;
    return build_impl(points[0], total, d, metric, bp, 0, 3, &whole, nullptr, nullptr, &b);
}

int pipnn_medoid(const void *points, uint64_t n, uint32_t d, int32_t dtype, uint32_t *medoid) {
    CallScope cs;
    PIPNN_TRY(cs.init());
    PIPNN_TRY(check_points(points, n, d, dtype, PIPNN_L2));
    if (!medoid) return set_error(PIPNN_EINVAL, "medoid is NULL");
    if (!is_device_ptr(points)) return set_error(PIPNN_EINVAL, "points must be a device pointer");
    PIPNN_TRY(medoid_bytes(points, n, d, dtype, medoid, cs.ws));
    return check_device_error("medoid");
}

static int search_common(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric,
                         const uint32_t *adj, const uint32_t *deg, uint32_t R, const void *queries, uint64_t nq,
                         uint32_t *start, uint32_t L, uint32_t k, int exclude_self, uint32_t *ids, uint64_t *ndist,
                         const char *what) {
    if (ndist) *ndist = 0;
    CallScope cs;
    PIPNN_TRY(cs.init());
    PIPNN_TRY(check_points(points, n, d, dtype, metric));
    if (!adj || !deg || !ids || !queries) return set_error(PIPNN_EINVAL, "%s: NULL array", what);
    if (!is_device_ptr(points) || !is_device_ptr(adj) || !is_device_ptr(deg) || !is_device_ptr(queries) ||
        !is_device_ptr(ids))
        return set_error(PIPNN_EINVAL, "%s: points, adj, deg, queries and the output must be device pointers", what);
    if (R < 1 || R > 1024) return set_error(PIPNN_EINVAL, "%s: R outside 1..1024", what);
    if (L < 1 || L > 512) return set_error(PIPNN_EINVAL, "%s: L outside 1..512", what);
    if (k < 1 || k + (exclude_self ? 1u : 0u) > L)
        return set_error(PIPNN_EINVAL, exclude_self ? "%s: need 1 <= k < L" : "%s: need 1 <= k <= L", what);
    if (*start == 0xFFFFFFFFu) PIPNN_TRY(medoid_bytes(points, n, d, dtype, start, cs.ws));
    if (*start >= n) return set_error(PIPNN_EINVAL, "%s: start %u is not a point", what, *start);
    PIPNN_TRY(beam_search_batch(points, n, d, dtype, metric, adj, deg, R, queries, nq, *start, L, k, exclude_self,
                                ids, ndist, cs.ws));
    return check_device_error(what);
}

int pipnn_beam_search(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric, const uint32_t *adj,
                      const uint32_t *deg, uint32_t R, const void *queries, uint64_t nq, uint32_t start, uint32_t L,
                      uint32_t k, uint32_t *ids, uint64_t *ndist) {
    if (nq == 0) {
        if (ndist) *ndist = 0;
        return PIPNN_OK;
    }
    if (start == 0xFFFFFFFFu) return set_error(PIPNN_EINVAL, "beam search: start %u is not a point", start);
    return search_common(points, n, d, dtype, metric, adj, deg, R, queries, nq, &start, L, k, 0, ids, ndist,
                         "beam search");
}

int pipnn_knn_graph(const void *points, uint64_t n, uint32_t d, int32_t dtype, int32_t metric, const uint32_t *adj,
                    const uint32_t *deg, uint32_t R, uint32_t start, uint32_t L, uint32_t k, uint32_t *knn,
                    uint64_t *ndist) {
    return search_common(points, n, d, dtype, metric, adj, deg, R, points, n, &start, L, k, 1, knn, ndist,
                         "k-NN graph");
}

int pipnn_trim_pool(void) {
    clear_error();
    int dev = 0;
    PIPNN_CUDA(cudaGetDevice(&dev));
    PIPNN_CUDA(cudaDeviceSynchronize());
    cudaMemPool_t pool;
    PIPNN_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    PIPNN_CUDA(cudaMemPoolTrimTo(pool, 0));
    return PIPNN_OK;
}

int pipnn_get_stats(pipnn_stats *out) {
    if (!out) return set_error(PIPNN_EINVAL, "out is NULL");
    *out = g_stats;
    return PIPNN_OK;
}

}  // extern "C"
