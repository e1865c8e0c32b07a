// leaf.cu -- A2..A4: all-pairs dissimilarities inside every leaf and the bi-directed k-NN pick
// (Sec. 4.2, App. A.3).  Every member keeps its k nearest other members by (dissimilarity, id)
// and emits the edge in both directions; a leaf of u members yields 2 u min(k, u-1) candidates,
// written at a precomputed offset so the stream is compact.
#include "allpairs.cuh"

namespace pipnn {

int sketch_points(const void *X, uint64_t n, uint32_t d, int dtype, const float *H, uint32_t m, float *S,
                  void *sqnorm);
int leaf_pick_tc(const void *X, uint64_t n, uint32_t d, int dtype, const int32_t *sqnorm, const uint64_t *off,
                 const uint32_t *mem, uint64_t L, const uint32_t *leaf_size, const uint64_t *cand_off, uint32_t k,
                 uint32_t *out_dst, uint32_t *out_src, float *out_dist, Workspace &ws, cudaEvent_t ev0,
                 cudaEvent_t ev1, uint32_t *launches);
int leaf_pick_tcf(const float *X, uint64_t n, uint32_t d, int metric, int prec, const uint64_t *off,
                  const uint32_t *mem, uint64_t L, const uint32_t *leaf_size, const uint64_t *cand_off, uint32_t k,
                  uint32_t *out_dst, uint32_t *out_src, float *out_dist, Workspace &ws, cudaEvent_t ev0,
                  cudaEvent_t ev1, uint32_t *launches, uint64_t *fallback_rows);

namespace {
// caller-supplied leaves: offsets non-decreasing, member ids below n
__global__ void check_leaves(const uint64_t *off, uint64_t L, const uint32_t *mem, uint64_t n, unsigned *err) {
    const uint64_t M = off[L];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < M || i < L;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < M && mem[i] >= n) atomicOr(err, DERR_RANGE);
        if (i < L && off[i + 1] < off[i]) atomicOr(err, DERR_RANGE);
    }
}

__global__ void leaf_sizes(const uint64_t *off, uint64_t L, uint32_t k, uint32_t *size, uint64_t *cand) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < L; b += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = off[b + 1] - off[b];
        size[b] = (uint32_t)s;
        uint64_t kk = s > 0 ? (s - 1 < k ? s - 1 : k) : 0;
        cand[b] = 2 * s * kk;
    }
}
}  // namespace

// App. A.3 variants: every engine writes the two edges of a picked pair at (2e, 2e + 1) --
// member -> neighbour first -- so a directed or inverted pick keeps one parity.
__global__ void keep_direction(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t half,
                               uint32_t parity, uint32_t *od, uint32_t *os, float *ow) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < half; e += (uint64_t)gridDim.x * blockDim.x) {
        od[e] = dst[2 * e + parity];
        os[e] = src[2 * e + parity];
        ow[e] = dist[2 * e + parity];
    }
}

int leaf_pick(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
              const uint64_t *off, const uint32_t *mem, uint64_t L, uint32_t k, int engine, int prec,
              int direction, pipnn_edges *out, float *ms_kernel, uint32_t *launches, uint64_t *full_rows) {
    if (direction < PIPNN_PICK_BIDIRECTED || direction > PIPNN_PICK_INVERTED)
        return set_error(PIPNN_EINVAL, "unknown pick direction %d", direction);
    if (full_rows) *full_rows = 0;
    if (engine == PIPNN_LEAF_TC && dtype == PIPNN_F32 && prec != PIPNN_PREC_BF16 && prec != PIPNN_PREC_FP8 &&
        prec != PIPNN_PREC_BF16X3)
        return set_error(PIPNN_EUNSUPPORTED, "float data on the tensor-core leaf engine needs prec BF16, FP8 or BF16X3");
    memset(out, 0, sizeof(*out));
    Workspace ws;
    const int32_t *sqn = sqnorm_bytes;
    if (dtype != PIPNN_F32 && !sqn) {
        int32_t *tmp = nullptr;
        PIPNN_TRY(ws.alloc(&tmp, n));
        PIPNN_TRY(sketch_points(X, n, d, dtype, nullptr, 0, nullptr, tmp));
        sqn = tmp;
    }
    uint32_t *size;
    uint64_t *cand_off, *tot, E = 0;
    PIPNN_TRY(ws.alloc(&size, L));
    PIPNN_TRY(ws.alloc(&cand_off, L));
    PIPNN_TRY(ws.alloc(&tot, 1));
    if (L) {
        check_leaves<<<grid_for(L * 64, 256), 256, 0, stream()>>>(off, L, mem, n, device_error_word());
        PIPNN_LAUNCH_CHECK();
        PIPNN_TRY(check_device_error("leaf pick input"));
        leaf_sizes<<<grid_for(L, 256), 256, 0, stream()>>>(off, L, k, size, cand_off);
        PIPNN_LAUNCH_CHECK();
    }
    PIPNN_TRY(exclusive_scan_u64(cand_off, cand_off, L, tot, ws));
    PIPNN_TRY(read_u64(tot, &E));

    uint32_t *dst = nullptr, *src = nullptr;
    float *dist = nullptr;
    int rc = dev_alloc_raw((void **)&dst, E * 4);
    if (rc == PIPNN_OK) rc = dev_alloc_raw((void **)&src, E * 4);
    if (rc == PIPNN_OK) rc = dev_alloc_raw((void **)&dist, E * 4);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (rc == PIPNN_OK && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess))
        rc = set_error(PIPNN_ECUDA, "event creation failed");
    uint32_t nl = 0;
    if (rc == PIPNN_OK) {
        if (engine == PIPNN_LEAF_TC && dtype == PIPNN_F32) {
            rc = leaf_pick_tcf(static_cast<const float *>(X), n, d, metric, prec, off, mem, L, size, cand_off, k, dst,
                               src, dist, ws, ev0, ev1, &nl, full_rows);
        } else if (engine == PIPNN_LEAF_TC) {
            rc = leaf_pick_tc(X, n, d, dtype, sqn, off, mem, L, size, cand_off, k, dst, src, dist, ws, ev0, ev1, &nl);
        } else {
            uint32_t *tile_grp = nullptr, *tile_row0 = nullptr;
            uint64_t ntiles = 0;
            rc = make_tiles(size, L, AP_ROWS, &tile_grp, &tile_row0, &ntiles, ws);
            if (rc == PIPNN_OK) {
                AllPairsArgs a{};
                a.X = X;
                a.d = d;
                a.sqnorm = sqn;
                a.tile_grp = tile_grp;
                a.tile_row0 = tile_row0;
                a.leaf_off = off;
                a.members = mem;
                a.cand_off = cand_off;
                a.k = k;
                a.out_dst = dst;
                a.out_src = src;
                a.out_dist = dist;
                cudaEventRecord(ev0, stream());
                rc = launch_allpairs<MODE_PICK>(dtype, metric, k, a, ntiles);
                cudaEventRecord(ev1, stream());
                nl = ntiles ? 1 : 0;
            }
        }
    }
    if (rc == PIPNN_OK) rc = check_device_error("leaf pick");
    if (rc == PIPNN_OK && ms_kernel) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) *ms_kernel = ms;
        else cudaGetLastError();
    }
    if (launches) *launches = nl;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (rc != PIPNN_OK) {
        dev_free_raw(dst);
        dev_free_raw(src);
        dev_free_raw(dist);
        return rc;
    }
    if (direction != PIPNN_PICK_BIDIRECTED) {
        uint32_t *d2 = nullptr, *s2 = nullptr;
        float *w2 = nullptr;
        const uint64_t half = E / 2;
        rc = dev_alloc_raw((void **)&d2, half * 4);
        if (rc == PIPNN_OK) rc = dev_alloc_raw((void **)&s2, half * 4);
        if (rc == PIPNN_OK) rc = dev_alloc_raw((void **)&w2, half * 4);
        if (rc == PIPNN_OK && half) {
            keep_direction<<<grid_for(half, 256), 256, 0, stream()>>>(dst, src, dist, half,
                                                                      direction == PIPNN_PICK_DIRECTED ? 0u : 1u, d2,
                                                                      s2, w2);
            count_launch();
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = set_error(PIPNN_ECUDA, "keep_direction: %s", cudaGetErrorString(e));
        }
        dev_free_raw(dst);
        dev_free_raw(src);
        dev_free_raw(dist);
        if (rc != PIPNN_OK) {
            dev_free_raw(d2);
            dev_free_raw(s2);
            dev_free_raw(w2);
            return rc;
        }
        dst = d2;
        src = s2;
        dist = w2;
        E = half;
    }
    out->dst = dst;
    out->src = src;
    out->dist = dist;
    out->count = E;
    return PIPNN_OK;
}

}  // namespace pipnn
