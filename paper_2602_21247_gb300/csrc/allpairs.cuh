// allpairs.cuh -- CUDA-core "rows x columns, keep the k smallest per row" kernel.
//
// Two steps of the path share it:
//  * Alg. 5 leader assignment: rows are the instances of one subproblem, columns its leaders;
//    every row keeps its f nearest leaders (payload = leader rank).
//  * Sec. 4.2 pick: rows and columns are the members of one leaf; every row keeps its k
//    nearest other members (payload = member id) and emits both edge directions.
// Dissimilarities are evaluated in the defining order: a binary32 fused-multiply-add chain over
// coordinates 0..d-1 for float data, an exact integer dot product (n_i + n_j - 2<x_i,x_j>) for
// byte data.  A row's key is (order-preserving dissimilarity : 32, payload : 32), so ties go to
// the smaller payload.
#pragma once

#include "internal.cuh"

namespace pipnn {

enum { MODE_ASSIGN = 0, MODE_PICK = 1 };

constexpr int AP_ROWS = 128;   // rows per block (one per thread)
constexpr int AP_COLS = 32;    // columns per shared-memory tile
constexpr int AP_PREFETCH = 8; // 16-byte column chunks each thread keeps in flight (rows <= 512 B)

struct AllPairsArgs {
    const void *X;
    uint32_t d;
    const int32_t *sqnorm;       // byte data: exact squared norms
    const uint32_t *tile_grp;    // tile -> group
    const uint32_t *tile_row0;   // tile -> first row inside the group
    // MODE_ASSIGN: group = subproblem
    const uint64_t *seg_start;   // first instance of the subproblem
    const uint32_t *seg_size;
    const uint32_t *inst;        // instance -> point id
    const uint64_t *lead_off;    // first leader of the subproblem
    const uint32_t *lead_cnt;
    const uint32_t *lead;        // leader point ids in rank order
    uint32_t fanout;             // F: stride of `assign`; a subproblem uses min(F, leaders)
    uint16_t *assign;            // instance -> F leader ranks
    uint32_t *bucket_cnt;        // (subproblem, rank) -> bucket size
    // MODE_PICK: group = leaf
    const uint64_t *leaf_off;    // CSR offsets of leaf members
    const uint32_t *members;
    const uint64_t *cand_off;    // first candidate slot of the leaf
    uint32_t k;
    uint32_t *out_dst, *out_src;
    float *out_dist;
};

template <int KMAX>
__device__ __forceinline__ void topk_insert(uint64_t (&kv)[KMAX], uint64_t key) {
    if (key >= kv[KMAX - 1]) return;
    // skip an exact duplicate of a kept key
#pragma unroll
    for (int p = 0; p < KMAX; p++)
        if (kv[p] == key) return;
    kv[KMAX - 1] = key;
#pragma unroll
    for (int p = KMAX - 1; p > 0; p--) {
        uint64_t a = kv[p - 1], b = kv[p];
        bool sw = b < a;
        kv[p - 1] = sw ? b : a;
        kv[p] = sw ? a : b;
    }
}

template <int DT>
__device__ __forceinline__ float coord_f(const void *X, uint64_t row, uint32_t d, uint32_t t) {
    return static_cast<const float *>(X)[row * d + t];
}

// Packs byte coordinates 4 per word (zero padded past d).
template <int DT>
__device__ __forceinline__ uint32_t coord_word(const void *X, uint64_t row, uint32_t d, uint32_t w) {
    const uint8_t *p = static_cast<const uint8_t *>(X) + row * d;
    uint32_t v = 0;
    uint32_t t0 = w * 4;
    if (t0 + 4 <= d && (((uintptr_t)(p + t0)) & 3u) == 0) return *reinterpret_cast<const uint32_t *>(p + t0);
#pragma unroll
    for (int b = 0; b < 4; b++)
        if (t0 + b < d) v |= (uint32_t)p[t0 + b] << (8 * b);
    return v;
}

template <int DT>
__device__ __forceinline__ int dot4(uint32_t a, uint32_t b, int acc) {
    if (DT == PIPNN_U8) return (int)__dp4a(a, b, (unsigned)acc);
    return __dp4a((int)a, (int)b, acc);
}

// Shared memory words needed per block.
inline size_t allpairs_smem_bytes(int dtype, uint32_t d) {
    size_t dw = dtype == PIPNN_F32 ? d : (d + 3) / 4;
    return (size_t)(AP_ROWS + AP_COLS) * dw * 4 + 2 * AP_COLS * 4;
}

template <int DT, int MET, int KMAX, int MODE>
__global__ void __launch_bounds__(AP_ROWS) allpairs_topk(AllPairsArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t d = a.d;
    const uint32_t dw = DT == PIPNN_F32 ? d : (d + 3) / 4;
    uint32_t *Rs = smem;                       // [dw][AP_ROWS]
    uint32_t *Cs = smem + (size_t)dw * AP_ROWS;  // [dw][AP_COLS]
    uint32_t *Cid = Cs + (size_t)dw * AP_COLS;   // column ids of the tile
    int *Cn = reinterpret_cast<int *>(Cid + AP_COLS);  // their exact squared norms (byte data)

    const uint32_t g = a.tile_grp[blockIdx.x];
    const uint32_t row0 = a.tile_row0[blockIdx.x];
    const int tid = threadIdx.x;

    uint32_t nrows, ncols;
    const uint32_t *row_ids, *col_ids;
    if (MODE == MODE_ASSIGN) {
        nrows = a.seg_size[g];
        row_ids = a.inst + a.seg_start[g];
        ncols = a.lead_cnt[g];
        col_ids = a.lead + a.lead_off[g];
    } else {
        uint64_t s = a.leaf_off[g], e = a.leaf_off[g + 1];
        nrows = (uint32_t)(e - s);
        ncols = nrows;
        row_ids = a.members + s;
        col_ids = row_ids;
    }
    const uint32_t r = row0 + tid;
    const bool row_ok = r < nrows;
    const uint32_t my_id = row_ok ? row_ids[r] : 0u;

    // resident row tile, transposed
    for (uint32_t w = 0; w < dw; w++) {
        uint32_t v = 0;
        if (row_ok) {
            if (DT == PIPNN_F32) v = __float_as_uint(coord_f<DT>(a.X, my_id, d, w));
            else v = coord_word<DT>(a.X, my_id, d, w);
        }
        Rs[(size_t)w * AP_ROWS + tid] = v;
    }
    int my_norm = 0;
    if (DT != PIPNN_F32 && row_ok) my_norm = a.sqnorm[my_id];

    uint64_t kv[KMAX];
#pragma unroll
    for (int p = 0; p < KMAX; p++) kv[p] = ~0ull;

    // Column tiles: rows that are whole 16-byte chunks are fetched as uint4, and the next tile's
    // chunks are in flight while the current tile is consumed.
    const uint32_t row_bytes = DT == PIPNN_F32 ? d * 4 : d;
    const uint32_t nch = row_bytes / 16;                       // chunks per column row
    const bool vec = row_bytes % 16 == 0 && nch * AP_COLS <= AP_PREFETCH * AP_ROWS;
    uint4 pre[AP_PREFETCH];
    uint32_t pre_id = 0xFFFFFFFFu;
    int pre_n = 0;
    auto fetch_info = [&](uint32_t c0) {
        if (tid < AP_COLS) {
            pre_id = c0 + tid < ncols ? col_ids[c0 + tid] : 0xFFFFFFFFu;
            pre_n = (DT != PIPNN_F32 && pre_id != 0xFFFFFFFFu) ? a.sqnorm[pre_id] : 0;
        }
    };
    auto fetch = [&](uint32_t c0) {
#pragma unroll
        for (int u = 0; u < AP_PREFETCH; u++) {
            const uint32_t idx = u * AP_ROWS + tid;
            pre[u] = make_uint4(0, 0, 0, 0);
            if (idx < nch * AP_COLS) {
                const uint32_t c = idx / nch, ch = idx - c * nch;
                if (c0 + c < ncols) {
                    const uint32_t cid = col_ids[c0 + c];
                    pre[u] = __ldg(reinterpret_cast<const uint4 *>(static_cast<const char *>(a.X) +
                                                                   (uint64_t)cid * row_bytes) + ch);
                }
            }
        }
    };
    if (vec && ncols) fetch(0);
    if (ncols) fetch_info(0);
    for (uint32_t c0 = 0; c0 < ncols; c0 += AP_COLS) {
        __syncthreads();  // previous column tile fully consumed (and row tile written)
        if (tid < AP_COLS) {
            Cid[tid] = pre_id;
            Cn[tid] = pre_n;
        }
        if (c0 + AP_COLS < ncols && !vec) fetch_info(c0 + AP_COLS);
        if (vec) {
#pragma unroll
            for (int u = 0; u < AP_PREFETCH; u++) {
                const uint32_t idx = u * AP_ROWS + tid;
                if (idx < nch * AP_COLS) {
                    const uint32_t c = idx / nch, w0 = (idx - c * nch) * 4;
                    Cs[(size_t)(w0 + 0) * AP_COLS + c] = pre[u].x;
                    Cs[(size_t)(w0 + 1) * AP_COLS + c] = pre[u].y;
                    Cs[(size_t)(w0 + 2) * AP_COLS + c] = pre[u].z;
                    Cs[(size_t)(w0 + 3) * AP_COLS + c] = pre[u].w;
                }
            }
            __syncthreads();
            if (c0 + AP_COLS < ncols) {
                fetch(c0 + AP_COLS);
                fetch_info(c0 + AP_COLS);
            }
        } else {
            // thread (tid % 32) owns column c0 + tid%32, strides over words by 4
            const uint32_t c = tid % AP_COLS;
            const uint32_t cc = c0 + c;
            const bool ok = cc < ncols;
            const uint32_t cid = ok ? col_ids[cc] : 0u;
            for (uint32_t w = tid / AP_COLS; w < dw; w += AP_ROWS / AP_COLS) {
                uint32_t v = 0;
                if (ok) {
                    if (DT == PIPNN_F32) v = __float_as_uint(coord_f<DT>(a.X, cid, d, w));
                    else v = coord_word<DT>(a.X, cid, d, w);
                }
                Cs[(size_t)w * AP_COLS + c] = v;
            }
            __syncthreads();
        }
        if (!row_ok) continue;

        if (DT == PIPNN_F32) {
            float acc[AP_COLS];
#pragma unroll
            for (int c = 0; c < AP_COLS; c++) acc[c] = 0.0f;
            for (uint32_t t = 0; t < d; t++) {
                const float x = __uint_as_float(Rs[(size_t)t * AP_ROWS + tid]);
                const float4 *crow = reinterpret_cast<const float4 *>(Cs + (size_t)t * AP_COLS);
#pragma unroll
                for (int q = 0; q < AP_COLS / 4; q++) {
                    float4 y = crow[q];
                    if (MET == PIPNN_L2) {
                        float d0 = __fsub_rn(x, y.x), d1 = __fsub_rn(x, y.y);
                        float d2 = __fsub_rn(x, y.z), d3 = __fsub_rn(x, y.w);
                        acc[4 * q + 0] = __fmaf_rn(d0, d0, acc[4 * q + 0]);
                        acc[4 * q + 1] = __fmaf_rn(d1, d1, acc[4 * q + 1]);
                        acc[4 * q + 2] = __fmaf_rn(d2, d2, acc[4 * q + 2]);
                        acc[4 * q + 3] = __fmaf_rn(d3, d3, acc[4 * q + 3]);
                    } else {
                        acc[4 * q + 0] = __fmaf_rn(x, y.x, acc[4 * q + 0]);
                        acc[4 * q + 1] = __fmaf_rn(x, y.y, acc[4 * q + 1]);
                        acc[4 * q + 2] = __fmaf_rn(x, y.z, acc[4 * q + 2]);
                        acc[4 * q + 3] = __fmaf_rn(x, y.w, acc[4 * q + 3]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < AP_COLS; c++) {
                const uint32_t cc = c0 + c;
                if (cc < ncols) {
                    float D = MET == PIPNN_L2 ? acc[c] : __fsub_rn(1.0f, acc[c]);
                    uint32_t pay = MODE == MODE_ASSIGN ? cc : Cid[c];
                    if (MODE == MODE_PICK && pay == my_id) continue;
                    topk_insert<KMAX>(kv, ((uint64_t)f32_order(D) << 32) | pay);
                }
            }
        } else {
            int acc[AP_COLS];
#pragma unroll
            for (int c = 0; c < AP_COLS; c++) acc[c] = 0;
            for (uint32_t w = 0; w < dw; w++) {
                const uint32_t x = Rs[(size_t)w * AP_ROWS + tid];
                const uint4 *crow = reinterpret_cast<const uint4 *>(Cs + (size_t)w * AP_COLS);
#pragma unroll
                for (int q = 0; q < AP_COLS / 4; q++) {
                    uint4 y = crow[q];
                    acc[4 * q + 0] = dot4<DT>(x, y.x, acc[4 * q + 0]);
                    acc[4 * q + 1] = dot4<DT>(x, y.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = dot4<DT>(x, y.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = dot4<DT>(x, y.w, acc[4 * q + 3]);
                }
            }
#pragma unroll
            for (int c = 0; c < AP_COLS; c++) {
                const uint32_t cc = c0 + c;
                if (cc < ncols) {
                    const uint32_t cid = Cid[c];
                    if (MODE == MODE_PICK && cid == my_id) continue;
                    int D = my_norm + Cn[c] - 2 * acc[c];
                    uint32_t pay = MODE == MODE_ASSIGN ? cc : cid;
                    topk_insert<KMAX>(kv, ((uint64_t)(uint32_t)D << 32) | pay);
                }
            }
        }
    }
    if (!row_ok) return;

    if (MODE == MODE_ASSIGN) {
        const uint32_t f = a.fanout < ncols ? a.fanout : ncols;
        const uint64_t inst_idx = a.seg_start[g] + r;
#pragma unroll
        for (int p = 0; p < KMAX; p++) {
            if ((uint32_t)p < f) {
                uint32_t rank = (uint32_t)kv[p];
                a.assign[inst_idx * a.fanout + p] = (uint16_t)rank;
                atomicAdd(&a.bucket_cnt[a.lead_off[g] + rank], 1u);
            }
        }
    } else {
        const uint32_t kk = nrows - 1 < a.k ? nrows - 1 : a.k;
        uint64_t w = a.cand_off[g] + (uint64_t)r * 2 * kk;
#pragma unroll
        for (int p = 0; p < KMAX; p++) {
            if ((uint32_t)p < kk) {
                // a leaf with repeated ids has fewer distinct neighbours: emit a self edge,
                // which HashPrune drops
                uint32_t src = kv[p] == ~0ull ? my_id : (uint32_t)kv[p];
                uint32_t o = (uint32_t)(kv[p] >> 32);
                float D = DT == PIPNN_F32 ? f32_unorder(o) : __uint2float_rn(o);
                a.out_dst[w] = my_id;
                a.out_src[w] = src;
                a.out_dist[w] = D;
                a.out_dst[w + 1] = src;
                a.out_src[w + 1] = my_id;
                a.out_dist[w + 1] = D;
                w += 2;
            }
        }
    }
}

// Smallest instantiated KMAX that holds k keys (0 if none).
inline int kmax_for(uint32_t k) {
    if (k <= 2) return 2;
    if (k <= 4) return 4;
    if (k <= 8) return 8;
    if (k <= 16) return 16;
    if (k <= 32) return 32;
    return 0;
}

// Launches allpairs_topk<DT, MET, KMAX, MODE> with the right shared memory size.
template <int DT, int MET, int KMAX, int MODE>
int launch_allpairs_inst(const AllPairsArgs &args, uint64_t num_tiles) {
    size_t smem = allpairs_smem_bytes(DT, args.d);
    auto kern = allpairs_topk<DT, MET, KMAX, MODE>;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (uint64_t t0 = 0; t0 < num_tiles; t0 += 0x7FFFFFFFull) {
        uint64_t cnt = num_tiles - t0 < 0x7FFFFFFFull ? num_tiles - t0 : 0x7FFFFFFFull;
        AllPairsArgs a = args;
        a.tile_grp += t0;
        a.tile_row0 += t0;
        kern<<<(unsigned)cnt, AP_ROWS, smem, stream()>>>(a);
        PIPNN_LAUNCH_CHECK();
    }
    return PIPNN_OK;
}

template <int MODE>
int launch_allpairs(int dtype, int metric, uint32_t k, const AllPairsArgs &args, uint64_t num_tiles) {
    if (num_tiles == 0) return PIPNN_OK;
    int km = kmax_for(k);
#define PIPNN_AP_K(DT, MET)                                                                   \
    switch (km) {                                                                             \
    case 2: return launch_allpairs_inst<DT, MET, 2, MODE>(args, num_tiles);                    \
    case 4: return launch_allpairs_inst<DT, MET, 4, MODE>(args, num_tiles);                    \
    case 8: return launch_allpairs_inst<DT, MET, 8, MODE>(args, num_tiles);                    \
    case 16: return launch_allpairs_inst<DT, MET, 16, MODE>(args, num_tiles);                  \
    case 32: return launch_allpairs_inst<DT, MET, 32, MODE>(args, num_tiles);                  \
    default: return set_error(PIPNN_EINVAL, "k or fanout %u exceeds 32", k);                   \
    }
    if (dtype == PIPNN_F32 && metric == PIPNN_L2) { PIPNN_AP_K(PIPNN_F32, PIPNN_L2) }
    if (dtype == PIPNN_F32 && metric == PIPNN_IP) { PIPNN_AP_K(PIPNN_F32, PIPNN_IP) }
    if (dtype == PIPNN_U8) { PIPNN_AP_K(PIPNN_U8, PIPNN_L2) }
    if (dtype == PIPNN_I8) { PIPNN_AP_K(PIPNN_I8, PIPNN_L2) }
#undef PIPNN_AP_K
    return set_error(PIPNN_EUNSUPPORTED, "dtype %d with metric %d", dtype, metric);
}

}  // namespace pipnn
