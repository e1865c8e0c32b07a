// search.cu -- Alg. 1 (BeamSearch) for a batch of queries over a built graph, the k-NN graph
// construction of Sec. 5 that queries every point with itself, and the search start for byte
// data (the point nearest to the exact mean).
//
// One warp runs one query at a time; warps take queries from a global counter.  Per warp, shared
// memory holds the beam (L packed keys (dissimilarity, id) kept sorted, with a visited flag per
// slot, double-buffered for the merge), the unseen neighbours of the node being expanded, the
// query, and a small hash set of evaluated ids.
//
// Exactness.  The beam after every expansion is the L smallest keys of everything evaluated so
// far, and the next node expanded is the first unvisited slot, as in Alg. 1.  The hash set only
// saves work: it holds exact ids (no false positives), so skipping an id it holds is safe, and
// when it fills it is emptied, after which an id may be evaluated twice.  A second evaluation
// changes nothing: the id is either in the beam now (its key equals the beam's copy and the merge
// drops it), or it left the beam or never entered it, in which case L smaller keys exist and keep
// existing, so the beam rejects it again.  The dissimilarity is the defining one of Sec. 2 (the
// binary32 fused multiply-add chain in index order for float data, the exact integer for byte
// data), so the result equals a sequential Alg. 1 on the same dissimilarity key for key.
#include "internal.cuh"

namespace pipnn {
namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kProbes = 8;
// evaluated-id slots per beam slot (the per-query table holds 1024 .. 8192 ids)
#ifndef PIPNN_SEARCH_SLOTS_PER_BEAM
#define PIPNN_SEARCH_SLOTS_PER_BEAM 32
#endif

struct SearchArgs {
    const void *X;
    uint64_t n;
    uint32_t d;
    const uint32_t *adj;
    const uint32_t *deg;
    uint32_t R;
    const void *Q;
    uint64_t nq;
    uint32_t start, L, k;
    int exclude_self;
    int vec;                 // 16-byte row loads are legal (aligned base, row bytes a multiple of 16)
    uint32_t hbits;          // the hash set holds 1 << hbits ids
    uint32_t warp_bytes;     // shared memory per warp
    uint32_t *ids;           // nq x k
    unsigned long long *ndist;
    unsigned long long *next;
    unsigned *err;
};

// Per-warp shared-memory layout (identical on host and device).
struct WarpLayout {
    uint32_t keys, newk, cid, hash, flags, query, bytes;
};
__host__ __device__ inline WarpLayout warp_layout(uint32_t L, uint32_t R, uint32_t hbits, uint32_t row_bytes) {
    WarpLayout w;
    uint32_t o = 0;
    w.keys = o;
    o += 2 * L * 8;
    w.newk = o;
    o += 32 * 8;
    w.cid = o;
    o += ((R + 31) / 32) * 32 * 4;
    w.hash = o;
    o += (1u << hbits) * 4;
    w.flags = o;
    o += (2 * L + 15) / 16 * 16;
    w.query = o;
    o += (row_bytes + 15) / 16 * 16;
    w.bytes = (o + 15) / 16 * 16;
    return w;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// number of entries of the sorted a[0, n) below key
__device__ __forceinline__ uint32_t lower_bound(const uint64_t *a, uint32_t n, uint64_t key) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ascending bitonic sort of one key per lane across the warp
__device__ __forceinline__ uint64_t warp_sort(uint64_t key, uint32_t lane) {
#pragma unroll
    for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            const uint64_t other = __shfl_xor_sync(kFull, key, j);
            const bool up = (lane & k) == 0;
            const bool lower = (lane & j) == 0;
            key = (lower == up) ? (key < other ? key : other) : (key < other ? other : key);
        }
    }
    return key;
}

// Inserts id u into the warp's hash set; returns false iff u was already there.  Lanes insert
// concurrently, so an empty slot is claimed with a compare-and-swap.  After kProbes occupied
// slots the id is reported as new without being stored (it may then be evaluated again).
__device__ __forceinline__ bool hash_insert(uint32_t *tab, uint32_t hbits, uint32_t u) {
    const uint32_t mask = (1u << hbits) - 1;
    const uint32_t h = (u * 0x9E3779B1u) >> (32 - hbits);
#pragma unroll 1
    for (int p = 0; p < kProbes; p++) {
        uint32_t *slot = &tab[(h + (uint32_t)p) & mask];
        uint32_t v = *reinterpret_cast<volatile uint32_t *>(slot);
        if (v == u) return false;
        if (v == kEmpty) {
            v = atomicCAS(slot, kEmpty, u);
            if (v == kEmpty) return true;
            if (v == u) return false;
        }
    }
    return true;
}

// ---- dissimilarities (Sec. 2, defining evaluation) ---------------------------------------------
template <int MET>
__device__ __forceinline__ float dis_f32(const float *x, const float *q, uint32_t d, bool vec) {
    float acc = 0.0f;
    if (vec) {
        for (uint32_t t = 0; t < d; t += 4) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(x + t));
            const float4 b = *reinterpret_cast<const float4 *>(q + t);
            if (MET == PIPNN_L2) {
                float df = __fsub_rn(a.x, b.x);
                acc = __fmaf_rn(df, df, acc);
                df = __fsub_rn(a.y, b.y);
                acc = __fmaf_rn(df, df, acc);
                df = __fsub_rn(a.z, b.z);
                acc = __fmaf_rn(df, df, acc);
                df = __fsub_rn(a.w, b.w);
                acc = __fmaf_rn(df, df, acc);
            } else {
                acc = __fmaf_rn(a.x, b.x, acc);
                acc = __fmaf_rn(a.y, b.y, acc);
                acc = __fmaf_rn(a.z, b.z, acc);
                acc = __fmaf_rn(a.w, b.w, acc);
            }
        }
    } else {
        for (uint32_t t = 0; t < d; t++) {
            const float a = __ldg(x + t), b = q[t];
            if (MET == PIPNN_L2) {
                const float df = __fsub_rn(a, b);
                acc = __fmaf_rn(df, df, acc);
            } else {
                acc = __fmaf_rn(a, b, acc);
            }
        }
    }
    return MET == PIPNN_L2 ? acc : __fsub_rn(1.0f, acc);
}

template <typename T>
__device__ __forceinline__ uint32_t dis_bytes_scalar(const T *x, const T *q, uint32_t d) {
    int32_t acc = 0;
    for (uint32_t t = 0; t < d; t++) {
        const int32_t df = (int32_t)__ldg(x + t) - (int32_t)q[t];
        acc += df * df;
    }
    return (uint32_t)acc;
}

// One 8-lane group's share of a byte row (16-byte chunks g, g + 8, ...): sum of squared byte
// differences.  flip = 0x80808080 maps int8 to uint8 by adding 128 to both sides, which keeps
// every difference.  The query chunk in shared memory is stored flipped already.
__device__ __forceinline__ uint32_t dis_bytes_chunks(const uint8_t *x, const uint8_t *q, uint32_t nch, uint32_t g,
                                                     uint32_t flip) {
    uint32_t acc = 0;
    for (uint32_t c = g; c < nch; c += 8) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(x) + c);
        const uint4 b = reinterpret_cast<const uint4 *>(q)[c];
        uint32_t v = __vabsdiffu4(a.x ^ flip, b.x);
        acc = __dp4a(v, v, acc);
        v = __vabsdiffu4(a.y ^ flip, b.y);
        acc = __dp4a(v, v, acc);
        v = __vabsdiffu4(a.z ^ flip, b.z);
        acc = __dp4a(v, v, acc);
        v = __vabsdiffu4(a.w ^ flip, b.w);
        acc = __dp4a(v, v, acc);
    }
    return acc;
}

// Keys (dissimilarity, id) of the m <= 32 candidates cid[0, m): one per lane (lane < m), else ~0.
// GROUPED: byte rows of whole 16-byte chunks, eight lanes per candidate, four candidates a pass.
template <int DT, int MET, bool GROUPED>
__device__ __forceinline__ uint64_t eval_keys(const SearchArgs &a, const uint32_t *cid, uint32_t m,
                                              const uint8_t *q, uint64_t *scratch, uint32_t lane) {
    if (GROUPED) {
        const uint32_t nch = a.d / 16, g = lane & 7, slot = lane >> 3;
        const uint32_t flip = DT == PIPNN_I8 ? 0x80808080u : 0u;
        const uint8_t *X = static_cast<const uint8_t *>(a.X);
        const uint4 qg = g < nch ? reinterpret_cast<const uint4 *>(q)[g] : make_uint4(0, 0, 0, 0);
        // sixteen candidates at a time: the first chunk of all four passes is loaded before any is
        // reduced, so the row gathers overlap
        for (uint32_t p0 = 0; p0 < m; p0 += 16) {
            uint4 v[4];
            uint32_t u[4];
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const uint32_t c = p0 + 4 * s + slot;
                u[s] = c < m ? cid[c] : 0u;
                v[s] = (c < m && g < nch) ? __ldg(reinterpret_cast<const uint4 *>(X + (size_t)u[s] * a.d) + g)
                                          : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const uint32_t c = p0 + 4 * s + slot;
                uint32_t acc = 0;
                if (c < m && g < nch) {
                    uint32_t w = __vabsdiffu4(v[s].x ^ flip, qg.x);
                    acc = __dp4a(w, w, acc);
                    w = __vabsdiffu4(v[s].y ^ flip, qg.y);
                    acc = __dp4a(w, w, acc);
                    w = __vabsdiffu4(v[s].z ^ flip, qg.z);
                    acc = __dp4a(w, w, acc);
                    w = __vabsdiffu4(v[s].w ^ flip, qg.w);
                    acc = __dp4a(w, w, acc);
                    if (nch > 8) acc += dis_bytes_chunks(X + (size_t)u[s] * a.d, q, nch, g + 8, flip);
                }
                acc += __shfl_xor_sync(kFull, acc, 1);
                acc += __shfl_xor_sync(kFull, acc, 2);
                acc += __shfl_xor_sync(kFull, acc, 4);
                if (c < m && g == 0) scratch[c] = ((uint64_t)acc << 32) | u[s];
            }
        }
        __syncwarp();
        const uint64_t key = lane < m ? scratch[lane] : ~0ull;
        __syncwarp();
        return key;
    } else {
        if (lane >= m) return ~0ull;
        const uint32_t u = cid[lane];
        if (DT == PIPNN_F32) {
            const float v = dis_f32<MET>(static_cast<const float *>(a.X) + (size_t)u * a.d,
                                         reinterpret_cast<const float *>(q), a.d, a.vec != 0);
            if (!(v == v) || isinf(v)) atomicOr(a.err, DERR_NONFINITE);
            return ((uint64_t)f32_order(v) << 32) | u;
        } else if (DT == PIPNN_U8) {
            const uint32_t v = dis_bytes_scalar(static_cast<const uint8_t *>(a.X) + (size_t)u * a.d, q, a.d);
            return ((uint64_t)v << 32) | u;
        } else {
            const uint32_t v = dis_bytes_scalar(static_cast<const int8_t *>(a.X) + (size_t)u * a.d,
                                                reinterpret_cast<const int8_t *>(q), a.d);
            return ((uint64_t)v << 32) | u;
        }
    }
}

// Merges one key per lane into the sorted beam src[0, nb) (flags fsrc) and writes the L smallest
// of the union to dst / fdst.  Keys equal to a beam key, repeated within the batch, or no smaller
// than the last key of a full beam are dropped.  Returns the new beam size, with bit 31 set when
// dst was written (otherwise src stays current).
constexpr uint32_t kMoved = 0x80000000u;
__device__ __forceinline__ uint32_t merge_batch(const uint64_t *src, const uint8_t *fsrc, uint64_t *dst, uint8_t *fdst,
                                                uint32_t nb, uint32_t L, uint64_t key, uint64_t *newk, uint32_t lane) {
    if (key != ~0ull) {
        if (nb == L && key >= src[L - 1]) {
            key = ~0ull;
        } else {
            const uint32_t r = lower_bound(src, nb, key);
            if (r < nb && src[r] == key) key = ~0ull;
        }
    }
    key = warp_sort(key, lane);
    const uint64_t prev = __shfl_up_sync(kFull, key, 1);
    if (lane > 0 && key == prev) key = ~0ull;
    const unsigned vm = __ballot_sync(kFull, key != ~0ull);
    if (vm == 0) return nb;
    const uint32_t cnt = __popc(vm);
    const uint32_t j = __popc(vm & lanemask_lt());
    if (key != ~0ull) newk[j] = key;
    __syncwarp();
    if (key != ~0ull) {
        const uint32_t pos = lower_bound(src, nb, key) + j;
        if (pos < L) {
            dst[pos] = key;
            fdst[pos] = 0;
        }
    }
    for (uint32_t t = lane; t < nb; t += 32) {
        const uint64_t v = src[t];
        const uint32_t pos = t + lower_bound(newk, cnt, v);
        if (pos < L) {
            dst[pos] = v;
            fdst[pos] = fsrc[t];
        }
    }
    __syncwarp();
    return min(L, nb + cnt) | kMoved;
}

// MINB: blocks of 8 warps per SM the register budget is sized for (4: 64 registers, for the small
// per-warp footprints of narrow beams; 3: 80 registers)
template <int DT, int MET, bool GROUPED, int MINB>
__global__ void __launch_bounds__(256, MINB) beam_search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t esz = DT == PIPNN_F32 ? 4 : 1;
    const uint32_t row_bytes = (uint32_t)(a.d * esz);
    const WarpLayout W = warp_layout(a.L, a.R, a.hbits, row_bytes);
    uint8_t *base = smem + (size_t)warp * a.warp_bytes;
    uint64_t *const keys0 = reinterpret_cast<uint64_t *>(base + W.keys);
    uint8_t *const flags0 = base + W.flags;
    // beam buffer b (0 or 1)
    auto keys = [&](uint32_t b) { return keys0 + b * a.L; };
    auto flags = [&](uint32_t b) { return flags0 + b * a.L; };
    uint64_t *newk = reinterpret_cast<uint64_t *>(base + W.newk);
    uint32_t *cid = reinterpret_cast<uint32_t *>(base + W.cid);
    uint32_t *tab = reinterpret_cast<uint32_t *>(base + W.hash);
    uint8_t *q = base + W.query;
    const uint32_t H = 1u << a.hbits;
    uint64_t evals = 0;

    for (;;) {
        unsigned long long qi = 0;
        if (lane == 0) qi = atomicAdd(a.next, 1ull);
        qi = __shfl_sync(kFull, qi, 0);
        if (qi >= a.nq) break;

        // the query row, into shared memory (int8 rows of the grouped path stored flipped)
        const uint8_t *qs = static_cast<const uint8_t *>(a.Q) + qi * row_bytes;
        if (a.vec) {
            for (uint32_t t = lane; t < row_bytes / 16; t += 32) {
                uint4 v = __ldg(reinterpret_cast<const uint4 *>(qs) + t);
                if (GROUPED && DT == PIPNN_I8) {
                    v.x ^= 0x80808080u;
                    v.y ^= 0x80808080u;
                    v.z ^= 0x80808080u;
                    v.w ^= 0x80808080u;
                }
                reinterpret_cast<uint4 *>(q)[t] = v;
            }
        } else {
            for (uint32_t t = lane; t < row_bytes; t += 32) q[t] = qs[t];
        }
        for (uint32_t t = lane; t < H; t += 32) tab[t] = kEmpty;
        __syncwarp();

        // the beam starts as the start node alone
        uint32_t cur = 0, nb = 0, inserted = 0;
        if (lane == 0) {
            cid[0] = a.start;
            hash_insert(tab, a.hbits, a.start);
        }
        __syncwarp();
        {
            const uint64_t key = eval_keys<DT, MET, GROUPED>(a, cid, 1, q, newk, lane);
            evals += lane == 0 ? 1 : 0;
            const uint32_t r = merge_batch(keys(cur), flags(cur), keys(cur ^ 1), flags(cur ^ 1), nb, a.L, key, newk, lane);
            nb = r & ~kMoved;
            if (r & kMoved) cur ^= 1;
        }
        inserted = 1;

        // every expansion visits a distinct node, so n + 1 rounds bound the loop
        for (uint64_t round = 0; round <= a.n; round++) {
            int p = -1;
            for (uint32_t c0 = 0; c0 < nb; c0 += 32) {
                const uint32_t t = c0 + lane;
                const unsigned um = __ballot_sync(kFull, t < nb && flags(cur)[t] == 0);
                if (um) {
                    p = (int)(c0 + __ffs(um) - 1);
                    break;
                }
            }
            if (p < 0) break;
            const uint32_t node = (uint32_t)keys(cur)[p];
            __syncwarp();
            if (lane == 0) flags(cur)[p] = 1;
            if (inserted > H / 2) {
                // the set is emptied and refilled with the beam's ids, the ones most likely met again
                for (uint32_t t = lane; t < H; t += 32) tab[t] = kEmpty;
                __syncwarp();
                for (uint32_t t = lane; t < nb; t += 32) hash_insert(tab, a.hbits, (uint32_t)keys(cur)[t]);
                inserted = nb;
            }
            __syncwarp();
            const uint32_t dg = min(__ldg(a.deg + node), a.R);
            uint32_t cnt = 0;
            for (uint32_t j0 = 0; j0 < dg; j0 += 32) {
                const uint32_t j = j0 + lane;
                const uint32_t u = j < dg ? __ldg(a.adj + (uint64_t)node * a.R + j) : kEmpty;
                bool fresh = false;
                if (u != kEmpty) {
                    if (u >= a.n) atomicOr(a.err, DERR_RANGE);
                    else fresh = hash_insert(tab, a.hbits, u);
                }
                const unsigned fm = __ballot_sync(kFull, fresh);
                if (fresh) cid[cnt + __popc(fm & lanemask_lt())] = u;
                cnt += __popc(fm);
            }
            inserted += cnt;
            __syncwarp();
            for (uint32_t c0 = 0; c0 < cnt; c0 += 32) {
                const uint32_t m = min(32u, cnt - c0);
                const uint64_t key = eval_keys<DT, MET, GROUPED>(a, cid + c0, m, q, newk, lane);
                evals += lane < m ? 1 : 0;
                const uint32_t r =
                    merge_batch(keys(cur), flags(cur), keys(cur ^ 1), flags(cur ^ 1), nb, a.L, key, newk, lane);
                nb = r & ~kMoved;
                if (r & kMoved) cur ^= 1;
            }
        }

        // the first k beam entries (other than the query itself for the k-NN graph)
        uint32_t written = 0;
        uint32_t *out = a.ids + qi * a.k;
        for (uint32_t c0 = 0; c0 < nb && written < a.k; c0 += 32) {
            const uint32_t t = c0 + lane;
            const uint32_t id = t < nb ? (uint32_t)keys(cur)[t] : kEmpty;
            const bool keep = t < nb && !(a.exclude_self && id == (uint32_t)qi);
            const unsigned km = __ballot_sync(kFull, keep);
            if (keep) {
                const uint32_t r = written + __popc(km & lanemask_lt());
                if (r < a.k) out[r] = id;
            }
            written += __popc(km);
        }
        for (uint32_t t = written + lane; t < a.k; t += 32) out[t] = kEmpty;
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(kFull, evals, o);
    if (lane == 0 && evals) atomicAdd(a.ndist, (unsigned long long)evals);
}

// Launches one persistent grid: the block size (1 .. 8 warps) that keeps the most warps resident
// per SM under the per-warp shared-memory footprint; the 64-register build where 32 warps fit.
template <int DT, int MET, bool GROUPED>
int launch_search(const SearchArgs &a) {
    auto kern = 32ull * a.warp_bytes <= 200ull * 1024 ? beam_search_kernel<DT, MET, GROUPED, 4>
                                                      : beam_search_kernel<DT, MET, GROUPED, 3>;
    int sms = 0, dev = 0, smem_max = 0;
    PIPNN_CUDA(cudaGetDevice(&dev));
    PIPNN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PIPNN_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    uint32_t warps = 0;
    int per_sm = 0, best = 0;
    for (uint32_t w = 8; w >= 1; w--) {
        const size_t sm = (size_t)w * a.warp_bytes;
        if (sm > (size_t)smem_max) continue;
        PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int b = 0;
        PIPNN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, (int)(w * 32), sm));
        if (b * (int)w > best) {
            best = b * (int)w;
            warps = w;
            per_sm = b;
        }
    }
    if (best < 1)
        return set_error(PIPNN_EUNSUPPORTED, "beam search: %u bytes of shared memory per warp do not fit",
                         a.warp_bytes);
    const size_t smem = (size_t)warps * a.warp_bytes;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    uint64_t blocks = (uint64_t)per_sm * sms;
    const uint64_t need = (a.nq + warps - 1) / warps;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, warps * 32, smem, stream()>>>(a);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

// ---- the search start for byte data --------------------------------------------------------------
__global__ void column_sums_kernel(const uint8_t *X, uint64_t n, uint32_t d, int is_signed, uint64_t rows_per_block,
                                   unsigned long long *S) {
    const uint64_t r0 = (uint64_t)blockIdx.x * rows_per_block;
    const uint64_t r1 = min(n, r0 + rows_per_block);
    for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) {
        long long acc = 0;
        for (uint64_t i = r0; i < r1; i++) {
            const uint8_t v = X[i * d + t];
            acc += is_signed ? (long long)(int8_t)v : (long long)v;
        }
        atomicAdd(S + t, (unsigned long long)acc);   // two's complement: exact modulo 2^64
    }
}

struct Best128 {
    unsigned long long hi, lo;
    uint32_t id, pad;
};

__device__ __forceinline__ bool less128(unsigned long long ah, unsigned long long al, uint32_t ai,
                                        unsigned long long bh, unsigned long long bl, uint32_t bi) {
    if (ah != bh) return ah < bh;
    if (al != bl) return al < bl;
    return ai < bi;
}

// per point sum_t (n x_t - S_t)^2 as a 128-bit integer (hi, lo); each block writes its argmin
__global__ void medoid_kernel(const uint8_t *X, uint64_t n, uint32_t d, int is_signed, const long long *S,
                              Best128 *block_best) {
    extern __shared__ long long s_sum[];
    __shared__ Best128 wbest[32];
    for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) s_sum[t] = S[t];
    __syncthreads();
    unsigned long long bh = ~0ull, bl = ~0ull;
    uint32_t bi = kEmpty;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long hi = 0, lo = 0;
        const uint8_t *x = X + i * d;
        for (uint32_t t = 0; t < d; t++) {
            const long long v = is_signed ? (long long)(int8_t)x[t] : (long long)x[t];
            const long long e = (long long)n * v - s_sum[t];
            const unsigned long long m = e < 0 ? (unsigned long long)(-e) : (unsigned long long)e;
            const unsigned long long pl = m * m, ph = __umul64hi(m, m);
            lo += pl;
            hi += ph + (lo < pl ? 1ull : 0ull);
        }
        if (less128(hi, lo, (uint32_t)i, bh, bl, bi)) {
            bh = hi;
            bl = lo;
            bi = (uint32_t)i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long oh = __shfl_xor_sync(kFull, bh, o), ol = __shfl_xor_sync(kFull, bl, o);
        const uint32_t oi = __shfl_xor_sync(kFull, bi, o);
        if (less128(oh, ol, oi, bh, bl, bi)) {
            bh = oh;
            bl = ol;
            bi = oi;
        }
    }
    if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = Best128{bh, bl, bi, 0};
    __syncthreads();
    if (threadIdx.x == 0) {
        Best128 b = wbest[0];
        for (uint32_t w = 1; w < blockDim.x / 32; w++)
            if (less128(wbest[w].hi, wbest[w].lo, wbest[w].id, b.hi, b.lo, b.id)) b = wbest[w];
        block_best[blockIdx.x] = b;
    }
}

__global__ void medoid_final_kernel(const Best128 *bb, uint32_t nblocks, uint32_t *out) {
    if (threadIdx.x != 0) return;
    Best128 b = bb[0];
    for (uint32_t i = 1; i < nblocks; i++)
        if (less128(bb[i].hi, bb[i].lo, bb[i].id, b.hi, b.lo, b.id)) b = bb[i];
    *out = b.id;
}

}  // namespace

int medoid_bytes(const void *X, uint64_t n, uint32_t d, int dtype, uint32_t *medoid_host, Workspace &ws) {
    if (dtype != PIPNN_U8 && dtype != PIPNN_I8)
        return set_error(PIPNN_EUNSUPPORTED, "the exact medoid is defined for byte data; pass a start node");
    unsigned long long *S = nullptr;
    PIPNN_TRY(ws.zeros(&S, d));
    const uint64_t rpb = 4096;
    const uint64_t blocks = (n + rpb - 1) / rpb;
    column_sums_kernel<<<(unsigned)blocks, 128, 0, stream()>>>(static_cast<const uint8_t *>(X), n, d,
                                                                dtype == PIPNN_I8, rpb, S);
    PIPNN_LAUNCH_CHECK();
    const unsigned mb = grid_for(n, 256, 152u * 8u);
    Best128 *bb = nullptr;
    uint32_t *out = nullptr;
    PIPNN_TRY(ws.alloc(&bb, mb));
    PIPNN_TRY(ws.alloc(&out, 1));
    medoid_kernel<<<mb, 256, (size_t)d * sizeof(long long), stream()>>>(
        static_cast<const uint8_t *>(X), n, d, dtype == PIPNN_I8, reinterpret_cast<const long long *>(S), bb);
    PIPNN_LAUNCH_CHECK();
    medoid_final_kernel<<<1, 32, 0, stream()>>>(bb, mb, out);
    PIPNN_LAUNCH_CHECK();
    PIPNN_CUDA(cudaMemcpyAsync(medoid_host, out, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream()));
    PIPNN_CUDA(cudaStreamSynchronize(stream()));
    return PIPNN_OK;
}

// hash-set size (1024 .. 8192 slots); it is emptied when half full
static uint32_t search_hash_bits(uint32_t L) {
    uint32_t b = 10;
    while (b < 13 && (1u << b) < (uint32_t)PIPNN_SEARCH_SLOTS_PER_BEAM * L) b++;
    return b;
}

int beam_search_batch(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const uint32_t *adj,
                      const uint32_t *deg, uint32_t R, const void *Q, uint64_t nq, uint32_t start, uint32_t L,
                      uint32_t k, int exclude_self, uint32_t *ids, uint64_t *ndist_host, Workspace &ws) {
    if (nq == 0) {
        if (ndist_host) *ndist_host = 0;
        return PIPNN_OK;
    }
    SearchArgs a{};
    a.X = X;
    a.n = n;
    a.d = d;
    a.adj = adj;
    a.deg = deg;
    a.R = R;
    a.Q = Q;
    a.nq = nq;
    a.start = start;
    a.L = L;
    a.k = k;
    a.exclude_self = exclude_self;
    a.ids = ids;
    a.err = device_error_word();
    const size_t esz = dtype == PIPNN_F32 ? 4 : 1;
    const size_t row_bytes = (size_t)d * esz;
    const bool aligned = (reinterpret_cast<uintptr_t>(X) % 16 == 0) && (reinterpret_cast<uintptr_t>(Q) % 16 == 0);
    a.vec = aligned && row_bytes % 16 == 0;
    a.hbits = search_hash_bits(L);
    const WarpLayout W = warp_layout(L, R, a.hbits, (uint32_t)row_bytes);
    a.warp_bytes = W.bytes;
    unsigned long long *cnt = nullptr;
    PIPNN_TRY(ws.zeros(&cnt, 2));
    a.ndist = cnt;
    a.next = cnt + 1;
    const bool grouped = dtype != PIPNN_F32 && a.vec;
    int rc;
    if (dtype == PIPNN_F32)
        rc = metric == PIPNN_L2 ? launch_search<PIPNN_F32, PIPNN_L2, false>(a)
                                : launch_search<PIPNN_F32, PIPNN_IP, false>(a);
    else if (dtype == PIPNN_U8)
        rc = grouped ? launch_search<PIPNN_U8, PIPNN_L2, true>(a) : launch_search<PIPNN_U8, PIPNN_L2, false>(a);
    else
        rc = grouped ? launch_search<PIPNN_I8, PIPNN_L2, true>(a) : launch_search<PIPNN_I8, PIPNN_L2, false>(a);
    PIPNN_TRY(rc);
    if (ndist_host) {
        PIPNN_CUDA(cudaMemcpyAsync(ndist_host, cnt, sizeof(uint64_t), cudaMemcpyDeviceToHost, stream()));
    }
    return PIPNN_OK;
}

}  // namespace pipnn
