// partition.cu -- A1: Alg. 5 randomized ball carving with multi-level fanout and Merge.
//
// The recursion is processed level by level.  A level holds S subproblems ("segments"), each a
// contiguous run of instances (point ids) with a 64-bit identity.  Per level:
//   1. leader sample  -- the l = max(2, min(ceil(P_samp*|P|), cap)) members with the smallest
//                        (Philox priority, id); candidates under a per-subproblem threshold are
//                        collected, then sorted in shared memory (retried if too few)
//   2. assignment     -- every instance joins its min(fanout(depth), l) nearest leaders,
//                        equidistant leaders in draw order: on the tensor cores for byte data
//                        with the PIPNN_LEAF_TC engine (assign_tc.cu), else on the CUDA cores
//                        (allpairs_topk, MODE_ASSIGN)
//   3. Merge plan     -- buckets below C_min are packed next-fit in leader-rank order into
//                        groups of at most C_max (one thread per subproblem walks its ranks)
//   4. scatter        -- instances move to their leaf / next-level bucket; a point that reaches
//                        one merged group twice is stored once
//   5. guard          -- a bucket as large as its subproblem (no progress) or at the depth cap
//                        is cut into ceil(|b|/C_max) runs of its members in id order
// Leaves are compacted into one CSR array at the end.
#include "allpairs.cuh"
#include "tc_common.cuh"

#include <memory>

namespace pipnn {

int sketch_points(const void *X, uint64_t n, uint32_t d, int dtype, const float *H, uint32_t m, float *S,
                  void *sqnorm);

namespace {
constexpr uint32_t CAND_CAP = 2048;
constexpr uint32_t DEPTH_CAP = 12;
constexpr uint32_t OB_NONE = 0xFFFFFFFFu;
enum : uint8_t { OB_LEAF = 0, OB_MERGED = 1, OB_RECURSE = 2, OB_GUARD = 3 };

// ceil(p * np) of the exact real product of the binary32 p = M * 2^E and the integer np, in
// integer arithmetic (M < 2^24 and np < 2^32, so M * np fits 64 bits).
__device__ __forceinline__ uint64_t ceil_mul_f32(float p, uint64_t np) {
    const uint32_t bits = __float_as_uint(p);
    const uint32_t ex = (bits >> 23) & 0xFFu;
    const uint64_t M = ex ? ((bits & 0x7FFFFFu) | 0x800000u) : (bits & 0x7FFFFFu);
    const int E = ex ? (int)ex - 150 : -149;
    const uint64_t prod = M * np;
    if (E >= 0) return prod << E;  // p <= 1 keeps E negative; kept for completeness
    const int sh = -E;
    if (sh >= 64) return prod ? 1 : 0;
    const uint64_t q = prod >> sh;
    return q + ((prod & ((1ull << sh) - 1)) ? 1 : 0);
}

__device__ __forceinline__ uint32_t leader_count(uint64_t np, float p_samp, uint32_t cap) {
    uint64_t l = ceil_mul_f32(p_samp, np);
    if (l > cap) l = cap;
    if (l < 2) l = 2;
    if (l > np) l = np;
    return (uint32_t)l;
}

__device__ __forceinline__ uint32_t isqrt_u32(uint32_t v) {
    uint32_t s = 0;
    while ((s + 1) * (s + 1) <= v) s++;
    return s;
}

// Candidate threshold of the leader sample: a member is collected when its 32-bit priority is
// below thr = min(2^32, expect * 2^32 / n), so about `expect` of the n members are collected.
// Any threshold gives the same leaders (the l smallest priorities of those collected, retried
// when fewer than l or more than the buffer arrive); this only sizes the work.
__device__ __forceinline__ unsigned long long sample_threshold(uint64_t expect, uint32_t n) {
    return expect >= n ? (1ull << 32) : (unsigned long long)((expect << 32) / n);
}

__global__ void seg_setup(uint64_t S, const uint32_t *seg_size, float p_samp, uint32_t cap_leaders,
                          uint32_t *lead_cnt, uint64_t *lead_cnt64, uint64_t *cand_cap, uint64_t *expect,
                          unsigned long long *thr, uint8_t *active, uint32_t *ccnt) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S; s += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t n = seg_size[s];
        uint32_t l = leader_count(n, p_samp, cap_leaders);
        lead_cnt[s] = l;
        lead_cnt64[s] = l;
        cand_cap[s] = n < CAND_CAP ? n : CAND_CAP;
        const uint64_t e = (uint64_t)l + 5u * isqrt_u32(l) + 10u;
        expect[s] = e;
        thr[s] = sample_threshold(e, n);
        active[s] = 1;
        ccnt[s] = 0;
    }
}

// The sample's randomness is that of the subproblem's own index: its seed and its points' ids
// relative to the index (seg_base), so a batch of indexes draws what separate builds would.
__global__ void collect_candidates(uint64_t N, const uint32_t *inst, const uint32_t *inst_seg,
                                   const uint64_t *seg_id, const unsigned long long *thr, const uint8_t *active,
                                   const uint64_t *cand_off, const uint64_t *cand_cap, uint32_t *ccnt,
                                   uint64_t *cbuf, const uint64_t *seg_seed, const uint32_t *seg_base) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t s = inst_seg[i];
        if (!active[s]) continue;
        uint32_t pt = inst[i];
        uint32_t prio = leader_priority(seg_seed[s], seg_id[s], pt - seg_base[s]);
        if ((unsigned long long)prio < thr[s]) {
            uint32_t pos = atomicAdd(&ccnt[s], 1u);
            if (pos < cand_cap[s]) cbuf[cand_off[s] + pos] = ((uint64_t)prio << 32) | pt;
        }
    }
}

// Too few candidates: expect twice as many; too many: three fifths as many.
__global__ void check_candidates(uint64_t S, const uint32_t *seg_size, const uint32_t *lead_cnt,
                                 const uint64_t *cand_cap, uint32_t *ccnt, uint64_t *expect,
                                 unsigned long long *thr, uint8_t *active, unsigned *nbad) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S; s += (uint64_t)gridDim.x * blockDim.x) {
        if (!active[s]) continue;
        uint32_t c = ccnt[s];
        bool under = c < lead_cnt[s], over = c > cand_cap[s];
        if (!under && !over) {
            active[s] = 0;
            continue;
        }
        atomicAdd(nbad, 1u);
        uint64_t e = expect[s];
        e = under ? 2 * e : (3 * e) / 5;
        if (e < 1) e = 1;
        if (e > (1ull << 32)) e = 1ull << 32;
        expect[s] = e;
        thr[s] = sample_threshold(e, seg_size[s]);
        ccnt[s] = 0;
    }
}

// One block per subproblem: bitonic sort of the collected (priority, id) keys, first l are the
// leaders in rank order.
__global__ void __launch_bounds__(1024) sort_leaders(const uint64_t *cbuf, const uint64_t *cand_off,
                                                     const uint32_t *ccnt, const uint32_t *lead_cnt,
                                                     const uint64_t *lead_off, uint32_t *lead) {
    __shared__ uint64_t sh[CAND_CAP];
    const uint32_t s = blockIdx.x;
    const uint32_t c = ccnt[s];
    uint32_t P = 1;
    while (P < c) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < c ? cbuf[cand_off[s] + i] : ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                uint32_t ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = sh[i], b = sh[ixj];
                    bool asc = (i & k) == 0;
                    if ((a > b) == asc) {
                        sh[i] = b;
                        sh[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    const uint32_t l = lead_cnt[s];
    for (uint32_t r = threadIdx.x; r < l; r += blockDim.x) lead[lead_off[s] + r] = (uint32_t)sh[r];
}

// Merge(B, C_min, C_max) and the leaf / recurse / guard decision, one thread per subproblem.
// pass 0 counts output buckets; pass 1 writes them at ob_base[s].
__global__ void merge_plan(uint64_t S, int pass, const uint32_t *seg_size, const uint64_t *seg_id,
                           const uint64_t *lead_off, const uint32_t *lead_cnt, const uint32_t *lead,
                           const uint32_t *bucket_cnt, uint32_t c_min, uint32_t c_max, uint32_t depth,
                           const uint64_t *seg_seed, const uint32_t *seg_base, uint64_t *ob_count,
                           const uint64_t *ob_base, uint32_t *rank_ob, uint32_t *ob_raw, uint8_t *ob_kind,
                           uint64_t *ob_child, uint32_t *ob_parent) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S; s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t lo = lead_off[s];
        const uint32_t l = lead_cnt[s], n_s = seg_size[s];
        const uint64_t base = pass ? ob_base[s] : 0;
        uint64_t nb = 0, gidx = 0;
        uint32_t gsz = 0;
        bool gopen = false;
        for (uint32_t r = 0; r < l; r++) {
            const uint32_t c = bucket_cnt[lo + r];
            if (c == 0) {
                if (pass) rank_ob[lo + r] = OB_NONE;
                continue;
            }
            if (c >= c_min) {
                uint8_t kind = c <= c_max ? OB_LEAF
                                          : ((c == n_s || depth + 1 >= DEPTH_CAP) ? OB_GUARD : OB_RECURSE);
                uint64_t ob = base + nb++;
                if (pass) {
                    rank_ob[lo + r] = (uint32_t)ob;
                    ob_raw[ob] = c;
                    ob_kind[ob] = kind;
                    ob_child[ob] = kind == OB_RECURSE
                                       ? child_identity(seg_seed[s], seg_id[s], lead[lo + r] - seg_base[s])
                                       : 0ull;
                    ob_parent[ob] = (uint32_t)s;
                }
                continue;
            }
            if (!gopen || gsz + c > c_max) {
                gopen = true;
                gidx = base + nb++;
                gsz = 0;
                if (pass) {
                    ob_kind[gidx] = OB_MERGED;
                    ob_child[gidx] = 0ull;
                }
            }
            gsz += c;
            if (pass) {
                rank_ob[lo + r] = (uint32_t)gidx;
                ob_raw[gidx] = gsz;
            }
        }
        if (!pass) ob_count[s] = nb;
    }
}

__global__ void classify_buckets(uint64_t OB, const uint8_t *ob_kind, const uint32_t *ob_raw, uint64_t *leafsz,
                                 uint64_t *nextsz, uint64_t *is_leaf, uint64_t *is_rec, uint64_t *is_guard) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < OB; b += (uint64_t)gridDim.x * blockDim.x) {
        uint8_t k = ob_kind[b];
        uint32_t c = ob_raw[b];
        leafsz[b] = k != OB_RECURSE ? c : 0;
        nextsz[b] = k == OB_RECURSE ? c : 0;
        is_leaf[b] = (k == OB_LEAF || k == OB_MERGED) ? 1 : 0;
        is_rec[b] = k == OB_RECURSE ? 1 : 0;
        is_guard[b] = k == OB_GUARD ? 1 : 0;
    }
}

// Instances per block and hash-table entries (at most half full) of the block-aggregated scatter.
template <int FMAX>
struct ScatterCfg {
    static constexpr uint32_t IB = FMAX <= 16 ? 256 : 128;
    static constexpr uint32_t HT = FMAX <= 2 ? 1024 : FMAX <= 4 ? 2048 : FMAX <= 8 ? 4096 : 8192;
    static constexpr uint32_t SMEM = HT * 12;  // key, count, base
    static_assert(HT >= 2 * IB * FMAX, "load factor");
};

// Every instance joins the output buckets of its (distinct) picks.  A block first ranks its picks
// per bucket in a shared-memory hash table, then reserves each bucket's run with one global
// atomic and writes; the order inside a bucket is arbitrary (as with one atomic per pick).
template <int FMAX>
__global__ void __launch_bounds__(256) scatter_instances(
    uint64_t N, uint32_t F, const uint32_t *inst, const uint32_t *inst_seg, const uint64_t *lead_off,
    const uint32_t *lead_cnt, const uint16_t *assign, const uint32_t *rank_ob, const uint8_t *ob_kind,
    const uint32_t *ob_raw, const uint64_t *leaf_pos, const uint64_t *next_pos, const uint64_t *rec_idx,
    uint32_t *ob_fill, uint32_t *leafmem, uint32_t *next_inst, uint32_t *next_seg, unsigned *err) {
    using C = ScatterCfg<FMAX>;
    extern __shared__ uint32_t sc_smem[];
    uint32_t *key = sc_smem, *cnt = sc_smem + C::HT, *base = sc_smem + 2 * C::HT;
    for (uint32_t e = threadIdx.x; e < C::HT; e += blockDim.x) {
        key[e] = OB_NONE;
        cnt[e] = 0;
    }
    __syncthreads();
    for (uint64_t i0 = (uint64_t)blockIdx.x * C::IB; i0 < N; i0 += (uint64_t)gridDim.x * C::IB) {
        const uint64_t i = i0 + threadIdx.x;
        const bool live = threadIdx.x < C::IB && i < N;
        uint32_t f = 0, pt = 0, s = 0;
        if (live) {
            s = inst_seg[i];
            f = F < lead_cnt[s] ? F : lead_cnt[s];
            pt = inst[i];
        }
        // the instance's buckets (duplicates and OB_NONE dropped), their table slots and ranks
        uint32_t ob[FMAX], sl[FMAX], lr[FMAX];
#pragma unroll
        for (int j = 0; j < FMAX; j++) {
            ob[j] = OB_NONE;
            if ((uint32_t)j >= f) continue;
            const uint32_t o = rank_ob[lead_off[s] + assign[i * F + j]];
            bool dup = false;
#pragma unroll
            for (int q = 0; q < j; q++) dup = dup || ob[q] == o;
            if (dup || o == OB_NONE) continue;
            ob[j] = o;
            uint32_t h = (o * 0x9E3779B1u) & (C::HT - 1);
            for (;;) {
                const uint32_t old = atomicCAS(&key[h], OB_NONE, o);
                if (old == OB_NONE || old == o) break;
                h = (h + 1) & (C::HT - 1);
            }
            sl[j] = h;
            lr[j] = atomicAdd(&cnt[h], 1u);
        }
        __syncthreads();
        // one reservation per bucket touched by the block
        for (uint32_t e = threadIdx.x; e < C::HT; e += blockDim.x)
            if (key[e] != OB_NONE) base[e] = atomicAdd(&ob_fill[key[e]], cnt[e]);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < FMAX; j++) {
            if (ob[j] == OB_NONE) continue;
            const uint32_t o = ob[j];
            const uint32_t pos = base[sl[j]] + lr[j];
            if (pos >= ob_raw[o]) {
                atomicOr(err, DERR_CAPACITY);
                continue;
            }
            if (ob_kind[o] == OB_RECURSE) {
                const uint64_t q = next_pos[o] + pos;
                next_inst[q] = pt;
                next_seg[q] = (uint32_t)rec_idx[o];
            } else {
                leafmem[leaf_pos[o] + pos] = pt;
            }
        }
        __syncthreads();
        // empty the slots this thread filled (several threads may clear one slot: same values)
#pragma unroll
        for (int j = 0; j < FMAX; j++) {
            if (ob[j] == OB_NONE) continue;
            key[sl[j]] = OB_NONE;
            cnt[sl[j]] = 0;
        }
        __syncthreads();
    }
}

template <int FMAX>
int launch_scatter(uint64_t N, uint32_t F, const uint32_t *inst, const uint32_t *inst_seg, const uint64_t *lead_off,
                   const uint32_t *lead_cnt, const uint16_t *assign, const uint32_t *rank_ob, const uint8_t *ob_kind,
                   const uint32_t *ob_raw, const uint64_t *leaf_pos, const uint64_t *next_pos,
                   const uint64_t *rec_idx, uint32_t *ob_fill, uint32_t *leafmem, uint32_t *next_inst,
                   uint32_t *next_seg, unsigned *err) {
    using C = ScatterCfg<FMAX>;
    auto kern = scatter_instances<FMAX>;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    kern<<<grid_for(N, C::IB, 152u * 8u), 256, C::SMEM, stream()>>>(N, F, inst, inst_seg, lead_off, lead_cnt, assign,
                                                                  rank_ob, ob_kind, ob_raw, leaf_pos, next_pos,
                                                                  rec_idx, ob_fill, leafmem, next_inst, next_seg, err);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

__global__ void emit_descriptors(uint64_t OB, const uint8_t *ob_kind, const uint32_t *ob_fill, const uint64_t *ob_child,
                                 const uint64_t *leaf_pos, const uint64_t *next_pos, const uint64_t *leaf_idx,
                                 const uint64_t *rec_idx, const uint64_t *guard_idx, uint64_t *leaf_start,
                                 uint32_t *leaf_size, uint64_t *nseg_start, uint32_t *nseg_size, uint64_t *nseg_id,
                                 uint64_t *guard_pos, uint64_t *guard_size, const uint32_t *ob_parent,
                                 const uint64_t *seg_seed, const uint32_t *seg_base, uint64_t *nseg_seed,
                                 uint32_t *nseg_base) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < OB; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint8_t k = ob_kind[b];
        if (k == OB_LEAF || k == OB_MERGED) {
            leaf_start[leaf_idx[b]] = leaf_pos[b];
            leaf_size[leaf_idx[b]] = ob_fill[b];
        } else if (k == OB_RECURSE) {
            nseg_start[rec_idx[b]] = next_pos[b];
            nseg_size[rec_idx[b]] = ob_fill[b];
            nseg_id[rec_idx[b]] = ob_child[b];
            nseg_seed[rec_idx[b]] = seg_seed[ob_parent[b]];
            nseg_base[rec_idx[b]] = seg_base[ob_parent[b]];
        } else {
            guard_pos[guard_idx[b]] = leaf_pos[b];
            guard_size[guard_idx[b]] = ob_fill[b];
        }
    }
}

// ---- guard: rank members by id through a flag array over all points ----
__global__ void guard_mark(const uint32_t *mem, uint64_t size, uint64_t *flags) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < size; q += (uint64_t)gridDim.x * blockDim.x)
        flags[mem[q]] = 1;
}
__global__ void guard_place(const uint32_t *mem, uint64_t size, const uint64_t *rank, uint32_t *tmp) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < size; q += (uint64_t)gridDim.x * blockDim.x)
        tmp[rank[mem[q]]] = mem[q];
}
__global__ void guard_runs(uint64_t pos, uint64_t size, uint32_t c_max, uint64_t *leaf_start, uint32_t *leaf_size) {
    const uint64_t k = (size + c_max - 1) / c_max;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < k; j += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = j * size / k, e = (j + 1) * size / k;
        leaf_start[j] = pos + s;
        leaf_size[j] = (uint32_t)(e - s);
    }
}

__global__ void iota_u32(uint32_t *a, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        a[i] = (uint32_t)i;
}

__global__ void widen_u32(const uint32_t *a, uint64_t n, uint64_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = a[i];
}

// one block per leaf: copy its members into the final CSR position
__global__ void compact_leaves(uint64_t L, const uint64_t *leaf_start, const uint32_t *leaf_size,
                               const uint32_t *leafmem, const uint64_t *dst_off, uint32_t *dst) {
    for (uint64_t b = blockIdx.x; b < L; b += gridDim.x) {
        const uint64_t s = leaf_start[b], o = dst_off[b];
        const uint32_t c = leaf_size[b];
        for (uint32_t q = threadIdx.x; q < c; q += blockDim.x) dst[o + q] = leafmem[s + q];
    }
}

struct LevelLeaves {
    uint32_t *mem;          // level leaf storage
    uint64_t *start;        // leaf -> first member inside `mem`
    uint32_t *size;
    uint64_t count;
};

struct Level {
    uint64_t S = 0, N = 0;
    uint64_t *seg_start = nullptr;
    uint32_t *seg_size = nullptr;
    uint64_t *seg_id = nullptr;
    uint64_t *seg_seed = nullptr;  // the seed of the subproblem's index
    uint32_t *seg_base = nullptr;  // the first point id of the subproblem's index
    uint32_t *inst = nullptr;
    uint32_t *inst_seg = nullptr;
    std::unique_ptr<Workspace> ws{new Workspace()};
};

uint32_t fanout_at(const pipnn_params *bp, uint32_t depth) {
    if (depth < bp->fanout_levels && depth < 4) return bp->fanout[depth] ? bp->fanout[depth] : 1;
    return 1;
}
}  // namespace

// Points of the `count` indexes of a batch: index i holds point ids idx_off[i] .. idx_off[i+1).
__global__ void batch_level0(uint64_t count, const uint64_t *big_off, const uint64_t *big_start,
                             const uint64_t *big_seed, uint32_t *seg_size, uint64_t *seg_start, uint64_t *seg_seed,
                             uint32_t *seg_base) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < count; s += (uint64_t)gridDim.x * blockDim.x) {
        seg_size[s] = (uint32_t)(big_off[2 * s + 1] - big_off[2 * s]);
        seg_start[s] = big_start[s];
        seg_seed[s] = big_seed[s];
        seg_base[s] = (uint32_t)big_off[2 * s];
    }
}

// instance j of the level-0 segments: the points of the large indexes in order, and their segment
__global__ void batch_instances(uint64_t count, const uint64_t *big_off, const uint64_t *big_start, uint32_t *inst,
                                uint32_t *inst_seg) {
    for (uint64_t s = blockIdx.x; s < count; s += gridDim.x) {
        const uint64_t lo = big_off[2 * s], hi = big_off[2 * s + 1], at = big_start[s];
        for (uint64_t q = threadIdx.x; q < hi - lo; q += blockDim.x) {
            inst[at + q] = (uint32_t)(lo + q);
            inst_seg[at + q] = (uint32_t)s;
        }
    }
}

// Alg. 5 over a batch of `count` independent indexes at once: index i holds the points
// idx_off[i] .. idx_off[i+1) (host array) and is partitioned with seeds[i] (host array), with its
// point ids taken relative to idx_off[i] wherever the randomness sees them, so every index gets the
// leaves a separate partition of it would get (its members as global ids).
int partition_points_batch(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
                           const pipnn_params *bp, const uint64_t *idx_off, const uint64_t *seeds, uint64_t count,
                           pipnn_leaves *out) {
    memset(out, 0, sizeof(*out));
    Workspace leaf_ws;
    std::vector<LevelLeaves> levels;
    unsigned *err = device_error_word();
    if (count == 0 || idx_off[count] != n) return set_error(PIPNN_EINVAL, "index offsets do not cover the points");

    // byte data needs exact squared norms for the dot-product form
    const int32_t *sqn = sqnorm_bytes;
    if (dtype != PIPNN_F32 && !sqn) {
        int32_t *tmp = nullptr;
        PIPNN_TRY(leaf_ws.alloc(&tmp, n));
        PIPNN_TRY(sketch_points(X, n, d, dtype, nullptr, 0, nullptr, tmp));
        sqn = tmp;
    }

    // tensor-core assignment: one padded BF16 copy of the points, made at the first level that uses it
    Workspace tc_ws;
    AssignTcPlan tc_plan;

    // level 0: an index of at most C_max points is one leaf; the others are the first subproblems
    std::vector<uint64_t> small_start, big_off, big_start, big_seed;
    std::vector<uint32_t> small_size;
    uint64_t big_total = 0;
    for (uint64_t i = 0; i < count; i++) {
        const uint64_t lo = idx_off[i], hi = idx_off[i + 1];
        if (hi < lo) return set_error(PIPNN_EINVAL, "index offsets decrease");
        if (hi == lo) continue;
        if (hi - lo <= bp->c_max) {
            small_start.push_back(lo);
            small_size.push_back((uint32_t)(hi - lo));
        } else {
            big_off.push_back(lo);
            big_off.push_back(hi);
            big_start.push_back(big_total);
            big_seed.push_back(seeds[i]);
            big_total += hi - lo;
        }
    }
    if (!small_start.empty()) {
        // the leaf storage of these leaves is the point ids themselves: mem = 0 .. n-1
        LevelLeaves lv{};
        const uint64_t ns = small_start.size();
        PIPNN_TRY(leaf_ws.alloc(&lv.mem, n));
        PIPNN_TRY(leaf_ws.alloc(&lv.start, ns));
        PIPNN_TRY(leaf_ws.alloc(&lv.size, ns));
        iota_u32<<<grid_for(n, 256), 256, 0, stream()>>>(lv.mem, n);
        PIPNN_LAUNCH_CHECK();
        PIPNN_CUDA(cudaMemcpyAsync(lv.start, small_start.data(), ns * 8, cudaMemcpyHostToDevice, stream()));
        PIPNN_CUDA(cudaMemcpyAsync(lv.size, small_size.data(), ns * 4, cudaMemcpyHostToDevice, stream()));
        PIPNN_CUDA(cudaStreamSynchronize(stream()));
        lv.count = ns;
        levels.push_back(lv);
    }
    std::unique_ptr<Level> cur(new Level());
    uint32_t nlevels = 0;
    const uint64_t nbig = big_start.size();
    cur->S = nbig;
    cur->N = big_total;
    if (nbig) {
        Workspace &w = *cur->ws;
        uint64_t *dbig_off, *dbig_start, *dbig_seed;
        PIPNN_TRY(w.alloc(&cur->seg_start, nbig));
        PIPNN_TRY(w.alloc(&cur->seg_size, nbig));
        PIPNN_TRY(w.zeros(&cur->seg_id, nbig));
        PIPNN_TRY(w.alloc(&cur->seg_seed, nbig));
        PIPNN_TRY(w.alloc(&cur->seg_base, nbig));
        PIPNN_TRY(w.alloc(&cur->inst, big_total));
        PIPNN_TRY(w.alloc(&cur->inst_seg, big_total));
        PIPNN_TRY(w.alloc(&dbig_off, 2 * nbig));
        PIPNN_TRY(w.alloc(&dbig_start, nbig));
        PIPNN_TRY(w.alloc(&dbig_seed, nbig));
        PIPNN_CUDA(cudaMemcpyAsync(dbig_off, big_off.data(), 2 * nbig * 8, cudaMemcpyHostToDevice, stream()));
        PIPNN_CUDA(cudaMemcpyAsync(dbig_start, big_start.data(), nbig * 8, cudaMemcpyHostToDevice, stream()));
        PIPNN_CUDA(cudaMemcpyAsync(dbig_seed, big_seed.data(), nbig * 8, cudaMemcpyHostToDevice, stream()));
        batch_level0<<<grid_for(nbig, 256), 256, 0, stream()>>>(nbig, dbig_off, dbig_start, dbig_seed, cur->seg_size,
                                                                 cur->seg_start, cur->seg_seed, cur->seg_base);
        PIPNN_LAUNCH_CHECK();
        batch_instances<<<grid_for(nbig, 1, 152u * 16u), 256, 0, stream()>>>(nbig, dbig_off, dbig_start, cur->inst,
                                                                              cur->inst_seg);
        PIPNN_LAUNCH_CHECK();
        PIPNN_CUDA(cudaStreamSynchronize(stream()));
    }

    for (uint32_t depth = 0; cur->S > 0; depth++) {
        nlevels++;
        const uint64_t S = cur->S, N = cur->N;
        const uint32_t F = fanout_at(bp, depth);
        Workspace tw;  // temporaries of this level
        uint32_t *lead_cnt, *ccnt, *lead, *bucket_cnt;
        uint64_t *lead_cnt64, *lead_off, *cand_cap, *cand_off, *cbuf, *tot;
        uint64_t *expect;
        unsigned long long *thr;
        uint8_t *active;
        unsigned *nbad;
        PIPNN_TRY(tw.alloc(&lead_cnt, S));
        PIPNN_TRY(tw.alloc(&lead_cnt64, S));
        PIPNN_TRY(tw.alloc(&lead_off, S));
        PIPNN_TRY(tw.alloc(&cand_cap, S));
        PIPNN_TRY(tw.alloc(&cand_off, S));
        PIPNN_TRY(tw.alloc(&expect, S));
        PIPNN_TRY(tw.alloc(&thr, S));
        PIPNN_TRY(tw.alloc(&active, S));
        PIPNN_TRY(tw.alloc(&ccnt, S));
        PIPNN_TRY(tw.alloc(&tot, 8));  // scan totals, read back several at a time
        PIPNN_TRY(tw.zeros(&nbad, 1));
        const unsigned gs = grid_for(S, 256);
        seg_setup<<<gs, 256, 0, stream()>>>(S, cur->seg_size, bp->p_samp, bp->max_leaders, lead_cnt, lead_cnt64,
                                            cand_cap, expect, thr, active, ccnt);
        PIPNN_LAUNCH_CHECK();
        uint64_t h2[2];
        PIPNN_TRY(exclusive_scan_u64(lead_cnt64, lead_off, S, tot, tw));
        PIPNN_TRY(exclusive_scan_u64(cand_cap, cand_off, S, tot + 1, tw));
        PIPNN_CUDA(cudaMemcpyAsync(h2, tot, sizeof(h2), cudaMemcpyDeviceToHost, stream()));
        PIPNN_CUDA(cudaStreamSynchronize(stream()));
        const uint64_t total_leaders = h2[0], total_cand = h2[1];
        PIPNN_TRY(tw.alloc(&cbuf, total_cand));
        PIPNN_TRY(tw.alloc(&lead, total_leaders));
        PIPNN_TRY(tw.zeros(&bucket_cnt, total_leaders));

        // 1. leader sample (bounded retries of under/over-full candidate sets)
        int tries = 0;
        for (;; tries++) {
            collect_candidates<<<grid_for(N, 256), 256, 0, stream()>>>(N, cur->inst, cur->inst_seg, cur->seg_id, thr,
                                                                       active, cand_off, cand_cap, ccnt, cbuf,
                                                                       cur->seg_seed, cur->seg_base);
            PIPNN_LAUNCH_CHECK();
            PIPNN_CUDA(cudaMemsetAsync(nbad, 0, sizeof(unsigned), stream()));
            check_candidates<<<gs, 256, 0, stream()>>>(S, cur->seg_size, lead_cnt, cand_cap, ccnt, expect, thr, active,
                                                       nbad);
            PIPNN_LAUNCH_CHECK();
            unsigned hb = 0;
            PIPNN_CUDA(cudaMemcpyAsync(&hb, nbad, sizeof(unsigned), cudaMemcpyDeviceToHost, stream()));
            PIPNN_CUDA(cudaStreamSynchronize(stream()));
            if (hb == 0) break;
            if (tries >= 16) return set_error(PIPNN_ECUDA, "leader sample did not converge");
        }
        sort_leaders<<<(unsigned)S, 1024, 0, stream()>>>(cbuf, cand_off, ccnt, lead_cnt, lead_off, lead);
        PIPNN_LAUNCH_CHECK();

        // 2. assignment to the f nearest leaders
        uint16_t *assign;
        PIPNN_TRY(tw.alloc(&assign, N * F));
        uint32_t *tile_grp, *tile_row0;
        uint64_t ntiles = 0;
        PIPNN_TRY(make_tiles(cur->seg_size, S, AP_ROWS, &tile_grp, &tile_row0, &ntiles, tw));
        AllPairsArgs a{};
        a.X = X;
        a.d = d;
        a.sqnorm = sqn;
        a.tile_grp = tile_grp;
        a.tile_row0 = tile_row0;
        a.seg_start = cur->seg_start;
        a.seg_size = cur->seg_size;
        a.inst = cur->inst;
        a.lead_off = lead_off;
        a.lead_cnt = lead_cnt;
        a.lead = lead;
        a.fanout = F;
        a.assign = assign;
        a.bucket_cnt = bucket_cnt;
        if (bp->leaf_engine == PIPNN_LEAF_TC && assign_tc_eligible(dtype, d, n, F)) {
            if (!tc_plan.rows) PIPNN_TRY(assign_tc_plan(X, n, d, dtype, tc_ws, &tc_plan));
            PIPNN_TRY(assign_tc(tc_plan, X, d, dtype, sqn, tile_grp, tile_row0, ntiles, cur->seg_start,
                                cur->seg_size, cur->inst, lead_off, lead_cnt, lead, total_leaders, N, F, assign,
                                bucket_cnt, tw));
        } else {
            PIPNN_TRY(launch_allpairs<MODE_ASSIGN>(dtype, metric, F, a, ntiles));
        }

        // 3. Merge plan
        uint64_t *ob_count, *ob_base, OB = 0;
        PIPNN_TRY(tw.alloc(&ob_count, S));
        PIPNN_TRY(tw.alloc(&ob_base, S));
        merge_plan<<<gs, 256, 0, stream()>>>(S, 0, cur->seg_size, cur->seg_id, lead_off, lead_cnt, lead, bucket_cnt,
                                             bp->c_min, bp->c_max, depth, cur->seg_seed, cur->seg_base, ob_count,
                                             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
        PIPNN_LAUNCH_CHECK();
        PIPNN_TRY(exclusive_scan_u64(ob_count, ob_base, S, tot, tw));
        PIPNN_TRY(read_u64(tot, &OB));
        uint32_t *rank_ob, *ob_raw, *ob_fill;
        uint8_t *ob_kind;
        uint64_t *ob_child;
        PIPNN_TRY(tw.alloc(&rank_ob, total_leaders));
        PIPNN_TRY(tw.alloc(&ob_raw, OB));
        PIPNN_TRY(tw.zeros(&ob_fill, OB));
        PIPNN_TRY(tw.alloc(&ob_kind, OB));
        PIPNN_TRY(tw.alloc(&ob_child, OB));
        uint32_t *ob_parent;
        PIPNN_TRY(tw.alloc(&ob_parent, OB));
        merge_plan<<<gs, 256, 0, stream()>>>(S, 1, cur->seg_size, cur->seg_id, lead_off, lead_cnt, lead, bucket_cnt,
                                             bp->c_min, bp->c_max, depth, cur->seg_seed, cur->seg_base, nullptr,
                                             ob_base, rank_ob, ob_raw, ob_kind, ob_child, ob_parent);
        PIPNN_LAUNCH_CHECK();

        uint64_t *leafsz, *nextsz, *is_leaf, *is_rec, *is_guard;
        PIPNN_TRY(tw.alloc(&leafsz, OB));
        PIPNN_TRY(tw.alloc(&nextsz, OB));
        PIPNN_TRY(tw.alloc(&is_leaf, OB));
        PIPNN_TRY(tw.alloc(&is_rec, OB));
        PIPNN_TRY(tw.alloc(&is_guard, OB));
        classify_buckets<<<grid_for(OB, 256), 256, 0, stream()>>>(OB, ob_kind, ob_raw, leafsz, nextsz, is_leaf,
                                                                  is_rec, is_guard);
        PIPNN_LAUNCH_CHECK();
        uint64_t h5[5];
        PIPNN_TRY(exclusive_scan_u64(leafsz, leafsz, OB, tot, tw));
        PIPNN_TRY(exclusive_scan_u64(nextsz, nextsz, OB, tot + 1, tw));
        PIPNN_TRY(exclusive_scan_u64(is_leaf, is_leaf, OB, tot + 2, tw));
        PIPNN_TRY(exclusive_scan_u64(is_rec, is_rec, OB, tot + 3, tw));
        PIPNN_TRY(exclusive_scan_u64(is_guard, is_guard, OB, tot + 4, tw));
        PIPNN_CUDA(cudaMemcpyAsync(h5, tot, sizeof(h5), cudaMemcpyDeviceToHost, stream()));
        PIPNN_CUDA(cudaStreamSynchronize(stream()));
        const uint64_t leaf_members_raw = h5[0], N_next = h5[1], n_leafobs = h5[2], n_rec = h5[3], n_guard = h5[4];

        // 4. scatter
        std::unique_ptr<Level> next(new Level());
        next->S = n_rec;
        next->N = N_next;
        Workspace &nw = *next->ws;
        PIPNN_TRY(nw.alloc(&next->seg_start, n_rec));
        PIPNN_TRY(nw.alloc(&next->seg_size, n_rec));
        PIPNN_TRY(nw.alloc(&next->seg_id, n_rec));
        PIPNN_TRY(nw.alloc(&next->seg_seed, n_rec));
        PIPNN_TRY(nw.alloc(&next->seg_base, n_rec));
        PIPNN_TRY(nw.alloc(&next->inst, N_next));
        PIPNN_TRY(nw.alloc(&next->inst_seg, N_next));
        LevelLeaves lv{};
        PIPNN_TRY(leaf_ws.alloc(&lv.mem, leaf_members_raw));
        uint64_t *guard_pos, *guard_size;
        PIPNN_TRY(tw.alloc(&guard_pos, n_guard));
        PIPNN_TRY(tw.alloc(&guard_size, n_guard));
        // guards add at least two runs each; the exact count is known after the scatter
        {
#define PIPNN_SCATTER(FM)                                                                                         \
    PIPNN_TRY(launch_scatter<FM>(N, F, cur->inst, cur->inst_seg, lead_off, lead_cnt, assign, rank_ob, ob_kind,     \
                                 ob_raw, leafsz, nextsz, is_rec, ob_fill, lv.mem, next->inst, next->inst_seg, err))
            if (F <= 2) PIPNN_SCATTER(2);
            else if (F <= 4) PIPNN_SCATTER(4);
            else if (F <= 8) PIPNN_SCATTER(8);
            else if (F <= 16) PIPNN_SCATTER(16);
            else PIPNN_SCATTER(32);
#undef PIPNN_SCATTER
        }
        uint64_t *lstart_tmp;
        uint32_t *lsize_tmp;
        PIPNN_TRY(tw.alloc(&lstart_tmp, n_leafobs));
        PIPNN_TRY(tw.alloc(&lsize_tmp, n_leafobs));
        emit_descriptors<<<grid_for(OB, 256), 256, 0, stream()>>>(OB, ob_kind, ob_fill, ob_child, leafsz, nextsz,
                                                                  is_leaf, is_rec, is_guard, lstart_tmp, lsize_tmp,
                                                                  next->seg_start, next->seg_size, next->seg_id,
                                                                  guard_pos, guard_size, ob_parent, cur->seg_seed,
                                                                  cur->seg_base, next->seg_seed, next->seg_base);
        PIPNN_LAUNCH_CHECK();

        // 5. guard buckets: runs of members in id order
        std::vector<uint64_t> gpos(n_guard), gsize(n_guard);
        uint64_t guard_runs_total = 0;
        if (n_guard) {
            PIPNN_CUDA(cudaMemcpyAsync(gpos.data(), guard_pos, n_guard * 8, cudaMemcpyDeviceToHost, stream()));
            PIPNN_CUDA(cudaMemcpyAsync(gsize.data(), guard_size, n_guard * 8, cudaMemcpyDeviceToHost, stream()));
            PIPNN_CUDA(cudaStreamSynchronize(stream()));
            for (uint64_t g = 0; g < n_guard; g++) guard_runs_total += (gsize[g] + bp->c_max - 1) / bp->c_max;
        }
        lv.count = n_leafobs + guard_runs_total;
        PIPNN_TRY(leaf_ws.alloc(&lv.start, lv.count));
        PIPNN_TRY(leaf_ws.alloc(&lv.size, lv.count));
        if (n_leafobs) {
            PIPNN_CUDA(cudaMemcpyAsync(lv.start, lstart_tmp, n_leafobs * 8, cudaMemcpyDeviceToDevice, stream()));
            PIPNN_CUDA(cudaMemcpyAsync(lv.size, lsize_tmp, n_leafobs * 4, cudaMemcpyDeviceToDevice, stream()));
        }
        if (n_guard) {
            uint64_t *flags, *tot2;
            uint32_t *tmp;
            PIPNN_TRY(tw.alloc(&flags, n));
            PIPNN_TRY(tw.alloc(&tot2, 1));
            uint64_t maxg = 0;
            for (uint64_t g = 0; g < n_guard; g++) maxg = gsize[g] > maxg ? gsize[g] : maxg;
            PIPNN_TRY(tw.alloc(&tmp, maxg));
            uint64_t at = n_leafobs;
            for (uint64_t g = 0; g < n_guard; g++) {
                uint32_t *m = lv.mem + gpos[g];
                PIPNN_CUDA(cudaMemsetAsync(flags, 0, n * 8, stream()));
                guard_mark<<<grid_for(gsize[g], 256), 256, 0, stream()>>>(m, gsize[g], flags);
                PIPNN_LAUNCH_CHECK();
                PIPNN_TRY(exclusive_scan_u64(flags, flags, n, tot2, tw));
                guard_place<<<grid_for(gsize[g], 256), 256, 0, stream()>>>(m, gsize[g], flags, tmp);
                PIPNN_LAUNCH_CHECK();
                PIPNN_CUDA(cudaMemcpyAsync(m, tmp, gsize[g] * 4, cudaMemcpyDeviceToDevice, stream()));
                uint64_t k = (gsize[g] + bp->c_max - 1) / bp->c_max;
                guard_runs<<<grid_for(k, 256), 256, 0, stream()>>>(gpos[g], gsize[g], bp->c_max, lv.start + at,
                                                                    lv.size + at);
                PIPNN_LAUNCH_CHECK();
                at += k;
            }
        }
        PIPNN_TRY(check_device_error("partition"));
        levels.push_back(lv);
        cur = std::move(next);
    }

    // compaction into CSR
    uint64_t L = 0;
    for (auto &lv : levels) L += lv.count;
    uint64_t *offsets = nullptr;
    uint32_t *members = nullptr;
    {
        Workspace tw;
        uint64_t *sizes, *tot;
        PIPNN_TRY(tw.alloc(&sizes, L + 1));
        PIPNN_TRY(tw.alloc(&tot, 1));
        uint64_t at = 0;
        for (auto &lv : levels) {
            widen_u32<<<grid_for(lv.count, 256), 256, 0, stream()>>>(lv.size, lv.count, sizes + at);
            PIPNN_LAUNCH_CHECK();
            at += lv.count;
        }
        PIPNN_TRY(dev_alloc_raw((void **)&offsets, (L + 1) * sizeof(uint64_t)));
        uint64_t M = 0;
        int rc = exclusive_scan_u64(sizes, offsets, L, tot, tw);
        if (rc == PIPNN_OK) rc = read_u64(tot, &M);
        if (rc == PIPNN_OK) {
            cudaMemcpyAsync(offsets + L, tot, 8, cudaMemcpyDeviceToDevice, stream());
            rc = dev_alloc_raw((void **)&members, M * sizeof(uint32_t));
        }
        if (rc != PIPNN_OK) {
            dev_free_raw(offsets);
            return rc;
        }
        at = 0;
        for (auto &lv : levels) {
            if (lv.count)
                compact_leaves<<<grid_for(lv.count, 1, 152u * 32u), 256, 0, stream()>>>(lv.count, lv.start, lv.size,
                                                                                         lv.mem, offsets + at, members);
            at += lv.count;
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream());
        if (e != cudaSuccess) {
            dev_free_raw(offsets);
            dev_free_raw(members);
            return set_error(PIPNN_ECUDA, "leaf compaction: %s", cudaGetErrorString(e));
        }
        out->offsets = offsets;
        out->members = members;
        out->num_leaves = L;
        out->num_members = M;
        out->levels = nlevels;
    }
    return PIPNN_OK;
}

int partition_points(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
                     const pipnn_params *bp, uint64_t seed, pipnn_leaves *out) {
    const uint64_t off[2] = {0, n};
    return partition_points_batch(X, n, d, dtype, metric, sqnorm_bytes, bp, off, &seed, 1, out);
}

}  // namespace pipnn
