// hashprune.cu -- A5: Alg. 3 HashPrune as a batch merge.
//
// Alg. 3 is history independent (Sec. 3 theorem): a node's reservoir ends up holding the l_max
// smallest per-hash-bucket minima of all its candidates, in whatever order they arrive.  The
// same fact makes the reservoir of a prefix plus the rest of the stream merge to the reservoir
// of the whole stream, so the GPU inserts a whole batch at once:
//   1. count candidates per destination, prefix-sum, scatter each candidate's slot
//      [ordered bf16 dist:16][src:32][h_dst(src):16] next to its destination's others;
//   2. one warp per node first drops exact duplicate slots (the same pair reached through several
//      leaves: about four of every five candidates of a build) with a shared-memory hash set,
//      sorts the distinct ones in registers with shuffles, and walks them in ascending order,
//      keeping a slot iff its hash bucket has not been seen yet (__match_any_sync within a chunk
//      of 32, a bitmap of 2^m bits across chunks), until l_max are kept.  Nodes with more than
//      128 distinct slots sort everything (in registers up to 256, else in shared memory, chunk
//      by chunk for batches larger than the buffer).  A node with at most 32 new slots and at
//      most 128 kept ones (hash bits <= 12) skips the sort: see the small-batch path below.
#include "internal.cuh"

#include <type_traits>

namespace pipnn {

namespace {
constexpr int HP_WARPS = 8;
constexpr int HP_BUF = 512;   // slots per warp buffer
constexpr uint32_t HP_HT = 256;       // per-warp hash set of distinct slots
constexpr uint32_t HP_DISTINCT = 128; // distinct slots the fast path sorts in registers

// Four consecutive candidates per thread, grouped like hp_scatter below: a group (v, c1), (c1, v),
// (v, c2), (c2, v) takes three atomics (v's two at once) instead of four.
__global__ void hp_count(const uint32_t *dst, const uint32_t *src, uint64_t count, uint64_t n, unsigned *per_node,
                         unsigned *err) {
    const uint64_t ngroups = (count + 3) / 4;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < ngroups; g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = 4 * g;
        uint32_t v[4], c[4];
        bool ok[4];
        bool bad = false;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const bool in = e + q < count;
            v[q] = in ? dst[e + q] : 0u;
            c[q] = in ? src[e + q] : 0u;
            bad |= in && (v[q] >= n || c[q] >= n);
            ok[q] = in && v[q] < n && c[q] < n && v[q] != c[q];
        }
        if (bad) atomicOr(err, DERR_RANGE);
        if (ok[0] && ok[1] && ok[2] && ok[3] && v[2] == v[0] && v[1] == c[0] && c[1] == v[0] && v[3] == c[2] &&
            c[3] == v[2]) {
            atomicAdd(&per_node[v[0]], 2u);
            atomicAdd(&per_node[v[1]], 1u);
            atomicAdd(&per_node[v[3]], 1u);
            continue;
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (ok[q]) atomicAdd(&per_node[v[q]], 1u);
    }
}

// start[v] = per_node[v] (to be prefix-summed); per_node[v] = 0 (it becomes the fill counter).
__global__ void hp_widen(unsigned *per_node, uint64_t n, uint64_t *start) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        start[v] = per_node[v];
        per_node[v] = 0;
    }
}

// Residualised hash h_v(c) (Eq. 1): bit i = [Sketch(c)_i >= Sketch(v)_i]; with both sketch rows
// loaded once, also h_c(v), whose bit i is [Sketch(v)_i >= Sketch(c)_i].
__device__ __forceinline__ void hash_pair(const float *S, uint32_t m, uint32_t v, uint32_t c, uint32_t &h_vc,
                                          uint32_t &h_cv) {
    h_vc = 0;
    h_cv = 0;
    const float *sv = S + (uint64_t)v * m, *sc = S + (uint64_t)c * m;
    if ((m & 3u) == 0) {
        // rows of a multiple of four floats start 16-byte aligned: vector loads
        const float4 *v4 = reinterpret_cast<const float4 *>(sv), *c4 = reinterpret_cast<const float4 *>(sc);
        for (uint32_t i = 0; i < m / 4; i++) {
            const float4 a = __ldg(c4 + i), b = __ldg(v4 + i);
            h_vc |= ((a.x >= b.x ? 1u : 0u) | (a.y >= b.y ? 2u : 0u) | (a.z >= b.z ? 4u : 0u) |
                     (a.w >= b.w ? 8u : 0u)) << (4 * i);
            h_cv |= ((b.x >= a.x ? 1u : 0u) | (b.y >= a.y ? 2u : 0u) | (b.z >= a.z ? 4u : 0u) |
                     (b.w >= a.w ? 8u : 0u)) << (4 * i);
        }
    } else {
        for (uint32_t i = 0; i < m; i++) {
            const float a = __ldg(sc + i), b = __ldg(sv + i);
            h_vc |= (a >= b ? 1u : 0u) << i;
            h_cv |= (b >= a ? 1u : 0u) << i;
        }
    }
}

// Residualised hashes of node v against c1 and c2 and back, with v's sketch row loaded once.
__device__ __forceinline__ void hash_fan(const float *S, uint32_t m, uint32_t v, uint32_t c1, uint32_t c2,
                                         uint32_t &h_v1, uint32_t &h_1v, uint32_t &h_v2, uint32_t &h_2v) {
    h_v1 = h_1v = h_v2 = h_2v = 0;
    const float *sv = S + (uint64_t)v * m, *s1 = S + (uint64_t)c1 * m, *s2 = S + (uint64_t)c2 * m;
    if ((m & 3u) == 0) {
        const float4 *v4 = reinterpret_cast<const float4 *>(sv), *a4 = reinterpret_cast<const float4 *>(s1),
                     *b4 = reinterpret_cast<const float4 *>(s2);
        for (uint32_t i = 0; i < m / 4; i++) {
            const float4 x = __ldg(v4 + i), a = __ldg(a4 + i), b = __ldg(b4 + i);
            h_v1 |= ((a.x >= x.x ? 1u : 0u) | (a.y >= x.y ? 2u : 0u) | (a.z >= x.z ? 4u : 0u) |
                     (a.w >= x.w ? 8u : 0u)) << (4 * i);
            h_1v |= ((x.x >= a.x ? 1u : 0u) | (x.y >= a.y ? 2u : 0u) | (x.z >= a.z ? 4u : 0u) |
                     (x.w >= a.w ? 8u : 0u)) << (4 * i);
            h_v2 |= ((b.x >= x.x ? 1u : 0u) | (b.y >= x.y ? 2u : 0u) | (b.z >= x.z ? 4u : 0u) |
                     (b.w >= x.w ? 8u : 0u)) << (4 * i);
            h_2v |= ((x.x >= b.x ? 1u : 0u) | (x.y >= b.y ? 2u : 0u) | (x.z >= b.z ? 4u : 0u) |
                     (x.w >= b.w ? 8u : 0u)) << (4 * i);
        }
    } else {
        for (uint32_t i = 0; i < m; i++) {
            const float x = __ldg(sv + i), a = __ldg(s1 + i), b = __ldg(s2 + i);
            h_v1 |= (a >= x ? 1u : 0u) << i;
            h_1v |= (x >= a ? 1u : 0u) << i;
            h_v2 |= (b >= x ? 1u : 0u) << i;
            h_2v |= (x >= b ? 1u : 0u) << i;
        }
    }
}

// Four consecutive candidates per thread.  The leaf pick emits every pair in both directions next
// to each other, (v, c) then (c, v), and a node's picks one after another: for k = 2 a group of
// four is (v, c1), (c1, v), (v, c2), (c2, v), which needs three sketch rows and three cursor
// updates instead of six and four.  Any other group is taken as two pairs (mirrored pairs load
// their two rows once) or one candidate at a time.
// cursor[v] starts at v's first slot (the exclusive prefix sum) and is advanced atomically, so
// afterwards it holds the first slot of v + 1 and v's run is [cursor[v - 1], cursor[v]).
__global__ void hp_scatter(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count, uint64_t n,
                           const float *S, uint32_t m, unsigned long long *cursor, uint64_t *slots) {
    const uint64_t ngroups = (count + 3) / 4;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < ngroups; g += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = 4 * g;
        uint32_t v[4], c[4];
        float w[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const bool in = e + q < count;
            v[q] = in ? dst[e + q] : 0u;
            c[q] = in ? src[e + q] : 0u;
            w[q] = in ? dist[e + q] : 0.0f;
            ok[q] = in && v[q] < n && c[q] < n && v[q] != c[q];
        }
        const bool mirror01 = ok[0] && ok[1] && v[1] == c[0] && c[1] == v[0];
        const bool mirror23 = ok[2] && ok[3] && v[3] == c[2] && c[3] == v[2];
        if (mirror01 && mirror23 && v[2] == v[0]) {
            uint32_t h01, h10, h02, h20;
            hash_fan(S, m, v[0], c[0], c[2], h01, h10, h02, h20);
            const unsigned long long p = atomicAdd(&cursor[v[0]], 2ull);
            slots[p] = reservoir_slot(w[0], c[0], h01);
            slots[p + 1] = reservoir_slot(w[2], c[2], h02);
            slots[atomicAdd(&cursor[v[1]], 1ull)] = reservoir_slot(w[1], c[1], h10);
            slots[atomicAdd(&cursor[v[3]], 1ull)] = reservoir_slot(w[3], c[3], h20);
            continue;
        }
#pragma unroll
        for (int pr = 0; pr < 2; pr++) {
            const int q0 = 2 * pr, q1 = q0 + 1;
            uint32_t h0 = 0, h1 = 0;
            if (ok[q0]) {
                uint32_t back;
                hash_pair(S, m, v[q0], c[q0], h0, back);
                if (ok[q1]) {
                    if (v[q1] == c[q0] && c[q1] == v[q0]) h1 = back;
                    else hash_pair(S, m, v[q1], c[q1], h1, back);
                }
            } else if (ok[q1]) {
                uint32_t back;
                hash_pair(S, m, v[q1], c[q1], h1, back);
            }
            if (ok[q0]) slots[atomicAdd(&cursor[v[q0]], 1ull)] = reservoir_slot(w[q0], c[q0], h0);
            if (ok[q1]) slots[atomicAdd(&cursor[v[q1]], 1ull)] = reservoir_slot(w[q1], c[q1], h1);
        }
    }
}

// Ascending bitonic sort of 32 * E keys held E per lane (element E * lane + q in K[q]):
// exchanges within a lane for distances below E, shuffles across lanes for the rest.
template <int E>
__device__ __forceinline__ void warp_sort_regs(uint64_t (&K)[E], int lane) {
#pragma unroll
    for (uint32_t k = 2; k <= 32u * E; k <<= 1) {
#pragma unroll
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            if (j >= (uint32_t)E) {
#pragma unroll
                for (int q = 0; q < E; q++) {
                    const uint32_t i = E * lane + q;
                    const uint64_t o = __shfl_xor_sync(0xffffffffu, K[q], j / E);
                    const bool take_min = ((i & j) == 0) == ((i & k) == 0);
                    K[q] = take_min ? (o < K[q] ? o : K[q]) : (o > K[q] ? o : K[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < E; q++) {
                    if ((q & j) == 0) {
                        const uint32_t i = E * lane + q;
                        const uint64_t lo = K[q], hi = K[q | j];
                        const bool up = (i & k) == 0;
                        const bool sw = (lo > hi) == up;
                        K[q] = sw ? hi : lo;
                        K[q | j] = sw ? lo : hi;
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ void warp_bitonic_sort(uint64_t *buf, uint32_t P, int lane) {
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < P; i += 32) {
                uint32_t ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = buf[i], b = buf[ixj];
                    bool asc = (i & k) == 0;
                    if ((a > b) == asc) {
                        buf[i] = b;
                        buf[ixj] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// padded: rows past cnt[v] already hold 0xFF..FF (a node without new slots is then left alone)
__global__ void __launch_bounds__(HP_WARPS * 32, 4) hp_merge(uint64_t n, uint32_t m, uint32_t l_max,
                                                         const uint64_t *start, const uint64_t *slots,
                                                         uint64_t *res, uint32_t *cnt, int padded) {
    extern __shared__ __align__(16) unsigned char hp_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bm_words = m >= 5 ? (1u << (m - 5)) : 1u;
    uint64_t *buf = reinterpret_cast<uint64_t *>(hp_smem) + (size_t)warp * HP_BUF;
    uint32_t *seen = reinterpret_cast<uint32_t *>(hp_smem + (size_t)HP_WARPS * HP_BUF * 8) + (size_t)warp * bm_words;
    unsigned long long *ht = reinterpret_cast<unsigned long long *>(
                                 hp_smem + (size_t)HP_WARPS * HP_BUF * 8 + (((size_t)HP_WARPS * bm_words * 4 + 7) & ~(size_t)7)) +
                             (size_t)warp * HP_HT;
    for (uint32_t w = lane; w < bm_words; w += 32) seen[w] = 0;
    for (uint32_t w = lane; w < HP_HT; w += 32) ht[w] = ~0ull;
    __syncwarp();

    // start[] is the scatter's advanced cursor: v's run is [start[v - 1], start[v]); a node's
    // count and run bounds are requested one node ahead
    const uint64_t stride = (uint64_t)gridDim.x * HP_WARPS;
    uint64_t v = (uint64_t)blockIdx.x * HP_WARPS + warp;
    uint32_t n_cur = 0;
    uint64_t n_a = 0, n_b = 0;
    if (v < n) {
        n_cur = cnt[v];
        n_a = v ? start[v - 1] : 0ull;
        n_b = start[v];
    }
    for (; v < n; v += stride) {
        const uint32_t cnt_in = n_cur;
        uint32_t cur = n_cur;
        if (cur > l_max) cur = l_max;
        uint64_t a = n_a;
        const uint64_t b = n_b;
        if (v + stride < n) {
            n_cur = cnt[v + stride];
            n_a = start[v + stride - 1];
            n_b = start[v + stride];
        }
        if (a == b) {
            // no new candidates: the reservoir is unchanged (normalise the padding unless the
            // caller keeps it)
            if (!padded)
                for (uint32_t t = cur + lane; t < l_max; t += 32) res[v * l_max + t] = ~0ull;
            continue;
        }
        // walk buf[0 .. nb) ascending, keep the first slot of every unseen hash bucket (compacted
        // to the front of buf); returns how many were kept, at most l_max
        auto walk = [&](uint32_t nb) {
            uint32_t out = 0;
            for (uint32_t base = 0; base < nb && out < l_max; base += 32) {
                const uint32_t i = base + lane;
                const bool valid = i < nb;
                const uint64_t key = valid ? buf[i] : ~0ull;
                const uint32_t h = (uint32_t)(key & 0xFFFFu);
                const unsigned vmask = __ballot_sync(0xffffffffu, valid);
                const unsigned same = __match_any_sync(0xffffffffu, valid ? h : 0xFFFFFFFFu);
                const bool leader = valid && (__ffs(same & vmask) - 1) == lane;
                const bool unseen = valid && !((seen[h >> 5] >> (h & 31)) & 1u);
                const bool keep = leader && unseen;
                __syncwarp();
                if (valid) atomicOr(&seen[h >> 5], 1u << (h & 31));
                const unsigned km = __ballot_sync(0xffffffffu, keep);
                const uint32_t pos = out + __popc(km & ((1u << lane) - 1u));
                if (keep && pos < l_max) buf[pos] = key;
                out += __popc(km);
                __syncwarp();
            }
            for (uint32_t w = lane; w < bm_words; w += 32) seen[w] = 0;
            __syncwarp();
            return out < l_max ? out : l_max;
        };
        // small-batch path (hash bits <= 12, at most 128 new slots, at most 128 kept at any point):
        // the kept slots have distinct buckets, so each new slot needs only the kept slot of its
        // own bucket.  The new slots go 32 at a time: the smallest of every bucket in the chunk
        // (exact duplicates: the lowest lane) is looked up in a bucket -> position byte table; it
        // is dropped if the kept slot is not larger, else it replaces it (or enters a bucket not
        // kept yet).  Every survivor's place in the merged order is its rank among the surviving
        // kept slots plus its rank among the entering ones; places from l_max on fall off.  The
        // merged order stays in shared memory and registers between chunks and is written once; a
        // batch that changes nothing writes nothing.  (An empty reservoir with more than 32 new
        // slots goes to the hash-set path below, which was faster there.)
        if (m <= 12 && b - a <= (cur > 0 ? 128u : 32u) && cur <= 128 && (l_max <= 128 || cur + (b - a) <= 128)) {
            const uint32_t nn_all = (uint32_t)(b - a);
            uint64_t o[4];  // kept slot t = 32 q + lane in o[q]
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t t = 32 * q + lane;
                o[q] = t < cur ? res[v * l_max + t] : ~0ull;
            }
            uint64_t x = (uint32_t)lane < nn_all ? slots[a + lane] : ~0ull;
            // the table (2^m bytes, position + 1, 0 = bucket not kept) in buf, the kept slots in ht
            unsigned char *tbl = reinterpret_cast<unsigned char *>(buf);
            uint64_t *oldsm = reinterpret_cast<uint64_t *>(ht);
            const uint32_t hmask = (1u << m) - 1u;
            for (uint32_t i = lane; i < ((1u << m) + 15) / 16; i += 32)
                reinterpret_cast<uint4 *>(buf)[i] = make_uint4(0u, 0u, 0u, 0u);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t t = 32 * q + lane;
                if (t < cur) {
                    tbl[(uint32_t)o[q] & hmask] = (unsigned char)(t + 1);
                    oldsm[t] = o[q];
                }
            }
            uint32_t kc = cur;
            bool changed = false;
            for (uint32_t c0 = 0; c0 < nn_all; c0 += 32) {
                const bool valid = c0 + lane < nn_all;
                const uint32_t h = (uint32_t)x & hmask;
                const unsigned same = __match_any_sync(0xffffffffu, valid ? h : 0xFFFFFFFFu);
                bool keep = valid;
                if (valid) {
                    for (unsigned r = same; r; r &= r - 1) {
                        const int j = __ffs(r) - 1;
                        const uint64_t y = __shfl_sync(same, x, j);
                        if (y < x || (y == x && j < lane)) keep = false;
                    }
                }
                __syncwarp();
                const uint32_t p = keep ? tbl[h] : 0u;
                const uint64_t ov = p ? oldsm[p - 1] : 0ull;
                const bool ins = keep && (p == 0 || ov > x);
                const bool repl = ins && p != 0;
                const unsigned insm = __ballot_sync(0xffffffffu, ins);
                // the next chunk is requested before this one is ranked
                const uint64_t xn = c0 + 32 + lane < nn_all ? slots[a + c0 + 32 + lane] : ~0ull;
                if (insm) {
                    unsigned dead[4];
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        dead[q] = __reduce_or_sync(0xffffffffu, (repl && ((p - 1) >> 5) == (uint32_t)q)
                                                                    ? 1u << ((p - 1) & 31)
                                                                    : 0u);
                    // kept slots below index s (0 .. 128) that were replaced
                    const uint32_t dc0 = __popc(dead[0]), dc1 = dc0 + __popc(dead[1]), dc2 = dc1 + __popc(dead[2]),
                                   dc3 = dc2 + __popc(dead[3]);
                    auto dead_below = [&](uint32_t s) {
                        const uint32_t q = s >> 5;
                        const uint32_t base = q == 0 ? 0u : q == 1 ? dc0 : q == 2 ? dc1 : q == 3 ? dc2 : dc3;
                        const unsigned w = q == 0 ? dead[0] : q == 1 ? dead[1] : q == 2 ? dead[2] : q == 3 ? dead[3] : 0u;
                        return base + __popc(w & ((1u << (s & 31)) - 1u));
                    };
                    const bool wide = kc > 64;  // kept slots in o[2], o[3] too
                    uint32_t pos_x = 0;
                    if (ins) {
                        uint32_t lo = 0, hi = kc;
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (oldsm[mid] < x) lo = mid + 1;
                            else hi = mid;
                        }
                        pos_x = lo - dead_below(lo);
                    }
                    uint32_t pos_o[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) pos_o[q] = 32u * q + lane - dead_below(32u * q + lane);
                    for (unsigned r = insm; r; r &= r - 1) {
                        const uint64_t y = __shfl_sync(0xffffffffu, x, __ffs(r) - 1);
                        pos_x += y < x ? 1u : 0u;
                        pos_o[0] += y < o[0] ? 1u : 0u;
                        pos_o[1] += y < o[1] ? 1u : 0u;
                        if (wide) {
                            pos_o[2] += y < o[2] ? 1u : 0u;
                            pos_o[3] += y < o[3] ? 1u : 0u;
                        }
                    }
                    const uint32_t total = kc - dc3 + __popc(insm);
                    const uint32_t nk = total < l_max ? total : l_max;  // >= kc: a replaced slot's successor enters
                    __syncwarp();
                    // the merged order into shared memory, then back into registers and the table
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (32u * q + lane < kc) tbl[(uint32_t)o[q] & hmask] = 0;
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const uint32_t t = 32 * q + lane;
                        if (t < kc && !((dead[q] >> lane) & 1u) && pos_o[q] < l_max) oldsm[pos_o[q]] = o[q];
                    }
                    if (ins && pos_x < l_max) oldsm[pos_x] = x;
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const uint32_t t = 32 * q + lane;
                        o[q] = t < nk ? oldsm[t] : ~0ull;
                        if (t < nk) tbl[(uint32_t)o[q] & hmask] = (unsigned char)(t + 1);
                    }
                    kc = nk;
                    changed = true;
                    __syncwarp();
                }
                x = xn;
            }
            if (changed) {
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (32u * q + lane < kc) res[v * l_max + 32 * q + lane] = o[q];
            }
            if (lane == 0 && kc != cnt_in) cnt[v] = kc;
            if (!padded)
                for (uint32_t t = kc + lane; t < l_max; t += 32) res[v * l_max + t] = ~0ull;
            __syncwarp();
            // ht is all ones again for the next node's hash set
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (32u * q + lane < kc) oldsm[32 * q + lane] = ~0ull;
            __syncwarp();
            continue;
        }
        // incremental path: a reservoir that already holds slots (from an earlier batch or wave) is
        // sorted with distinct hash buckets, so a short run of new slots is sorted on its own and
        // merged into it by rank (a stable merge: old before new on equal keys), then walked; the
        // walk keeps the first slot of each bucket, which also drops exact duplicates
        if (cur > 0 && b - a <= 32 && cur + (b - a) <= (uint64_t)HP_BUF / 2) {
            const uint32_t nn = (uint32_t)(b - a);
            uint64_t nk[1] = {(uint32_t)lane < nn ? slots[a + lane] : ~0ull};
            warp_sort_regs<1>(nk, lane);
            // the old reservoir and the sorted new slots, in the upper half of the buffer, for the
            // two rank searches (cur + nn <= HP_BUF / 2)
            uint64_t *old = buf + HP_BUF / 2;
            uint64_t *fresh = old + cur;
            for (uint32_t t = lane; t < cur; t += 32) old[t] = res[v * l_max + t];
            if ((uint32_t)lane < nn) fresh[lane] = nk[0];
            __syncwarp();
            // each old slot's position: its index plus the new slots strictly below it (binary search)
            for (uint32_t t = lane; t < cur; t += 32) {
                const uint64_t x = old[t];
                uint32_t lo = 0, hi = nn;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (fresh[mid] < x) lo = mid + 1;
                    else hi = mid;
                }
                buf[t + lo] = x;
            }
            // each new slot's position: its rank plus the old slots at or below it (binary search)
            if ((uint32_t)lane < nn) {
                uint32_t lo = 0, hi = cur;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (old[mid] <= nk[0]) lo = mid + 1;
                    else hi = mid;
                }
                buf[lane + lo] = nk[0];
            }
            __syncwarp();
            cur = walk(cur + nn);
            for (uint32_t t = lane; t < l_max; t += 32) res[v * l_max + t] = t < cur ? buf[t] : ~0ull;
            if (lane == 0) cnt[v] = cur;
            __syncwarp();
            continue;
        }
        // fast path: the distinct slots (old reservoir and new run) through the hash set, sorted
        // in registers when at most HP_DISTINCT; exact duplicates are interchangeable, so dropping
        // them leaves the walk's result unchanged.  (A valid slot is never all ones: its id is < n.)
        const uint64_t total = (uint64_t)cur + (b - a);
        uint32_t u = 0;
        bool fast = true;
        for (uint64_t base0 = 0; base0 < total && fast; base0 += 128) {
            // up to 128 slots requested at once, then inserted 32 at a time
            uint64_t kq[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint64_t t = base0 + 32 * q + lane;
                kq[q] = t < total ? (t < cur ? res[v * l_max + t] : slots[a + (t - cur)]) : ~0ull;
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
            const uint64_t base = base0 + 32 * q;
            if (base >= total) break;
            const uint64_t t = base + lane;
            const bool valid = t < total;
            const uint64_t key = kq[q];
            bool fresh = false;
            if (valid) {
                uint32_t h = (uint32_t)(((key ^ (key >> 31)) * 0x9E3779B97F4A7C15ull) >> 56);
                for (uint32_t it = 0; it < HP_HT; it++) {
                    const unsigned long long old = atomicCAS(&ht[h], ~0ull, (unsigned long long)key);
                    if (old == ~0ull) {
                        fresh = true;
                        break;
                    }
                    if (old == key) break;
                    h = (h + 1) & (HP_HT - 1);
                }
            }
            const unsigned fm = __ballot_sync(0xffffffffu, fresh);
            const uint32_t pos = u + __popc(fm & ((1u << lane) - 1u));
            if (fresh && pos < HP_DISTINCT) buf[pos] = key;
            u += __popc(fm);
            if (u > HP_DISTINCT) {  // uniform: the table then holds at most HP_DISTINCT + 32 < HP_HT
                fast = false;
                break;
            }
            }
        }
        for (uint32_t w = lane; w < HP_HT; w += 32) ht[w] = ~0ull;
        __syncwarp();
        auto sort_distinct = [&](auto tag) {
            constexpr int E = decltype(tag)::value;
            uint64_t K[E];
#pragma unroll
            for (int q = 0; q < E; q++) {
                const uint32_t t = E * lane + q;
                K[q] = t < u ? buf[t] : ~0ull;
            }
            __syncwarp();
            warp_sort_regs<E>(K, lane);
#pragma unroll
            for (int q = 0; q < E; q++) buf[E * lane + q] = K[q];
            __syncwarp();
            cur = walk(u);
        };
        // old + new slots, E per lane, sorted in registers
        auto sort_regs = [&](auto tag) {
            constexpr int E = decltype(tag)::value;
            const uint32_t nb = cur + (uint32_t)(b - a);
            uint64_t K[E];
#pragma unroll
            for (int q = 0; q < E; q++) {
                const uint32_t t = E * lane + q;
                K[q] = t < cur ? res[v * l_max + t] : (t < nb ? slots[a + (t - cur)] : ~0ull);
            }
            warp_sort_regs<E>(K, lane);
#pragma unroll
            for (int q = 0; q < E; q++) buf[E * lane + q] = K[q];
            __syncwarp();
            cur = walk(nb);
        };
        // (eight per lane would cover 256 but doubles the kernel's registers, which costs more
        // occupancy than the larger nodes gain)
        if (fast) {
            if (u <= 32) sort_distinct(std::integral_constant<int, 1>());
            else if (u <= 64) sort_distinct(std::integral_constant<int, 2>());
            else sort_distinct(std::integral_constant<int, 4>());
        } else if (total <= 128) {
            sort_regs(std::integral_constant<int, 4>());
        } else if (total <= 256) {
            // two runs of 128 sorted in registers (the second written descending), then the 8
            // merge stages of a 256-element bitonic network in shared memory
            const uint32_t nb = (uint32_t)total;
#pragma unroll
            for (int run = 0; run < 2; run++) {
                uint64_t K[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t t = 128 * run + 4 * lane + q;
                    K[q] = t < cur ? res[v * l_max + t] : (t < nb ? slots[a + (t - cur)] : ~0ull);
                }
                warp_sort_regs<4>(K, lane);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t i = 4 * lane + q;
                    buf[run == 0 ? i : 255 - i] = K[q];
                }
            }
            __syncwarp();
            for (uint32_t jm = 128; jm > 0; jm >>= 1) {
                for (uint32_t i = lane; i < 256; i += 32) {
                    const uint32_t ixj = i ^ jm;
                    if (ixj > i) {
                        const uint64_t x = buf[i], y = buf[ixj];
                        if (x > y) {
                            buf[i] = y;
                            buf[ixj] = x;
                        }
                    }
                }
                __syncwarp();
            }
            cur = walk(nb);
        } else {
            for (uint32_t t = lane; t < cur; t += 32) buf[t] = res[v * l_max + t];
            while (a < b) {
                uint32_t take = (uint32_t)((b - a) < (uint64_t)(HP_BUF - cur) ? (b - a) : (uint64_t)(HP_BUF - cur));
                for (uint32_t t = lane; t < take; t += 32) buf[cur + t] = slots[a + t];
                a += take;
                const uint32_t nb = cur + take;
                uint32_t P = 32;
                while (P < nb) P <<= 1;
                for (uint32_t t = nb + lane; t < P; t += 32) buf[t] = ~0ull;
                __syncwarp();
                warp_bitonic_sort(buf, P, lane);
                cur = walk(nb);
            }
        }
        for (uint32_t t = lane; t < l_max; t += 32) res[v * l_max + t] = t < cur ? buf[t] : ~0ull;
        if (lane == 0) cnt[v] = cur;
        __syncwarp();
    }
}
}  // namespace

size_t hashprune_smem_bytes(uint32_t m) {
    uint32_t bm_words = m >= 5 ? (1u << (m - 5)) : 1u;
    return (size_t)HP_WARPS * HP_BUF * 8 + (((size_t)HP_WARPS * bm_words * 4 + 7) & ~(size_t)7) +
           (size_t)HP_WARPS * HP_HT * 8;
}

// Several runs of candidate edges merged as one stream: counted and grouped run by run, then merged
// per node once.
int hashprune_merge_segments(const EdgeSegment *seg, uint32_t nseg, const float *S, uint32_t m, uint64_t n,
                             uint32_t l_max, uint64_t *res, uint32_t *cnt, int padded) {
    if (m < 1 || m > 16) return set_error(PIPNN_EINVAL, "hash_bits %u outside 1..16", m);
    if (l_max < 1 || l_max > 256) return set_error(PIPNN_EINVAL, "l_max %u outside 1..256", l_max);
    Workspace ws;
    unsigned *err = device_error_word();
    uint64_t *start, *tot;
    unsigned *fill;
    uint64_t *slots;
    uint64_t E = 0, count = 0;
    PIPNN_TRY(ws.zeros(&start, n + 1));
    PIPNN_TRY(ws.zeros(&fill, n));
    PIPNN_TRY(ws.alloc(&tot, 1));
    for (uint32_t i = 0; i < nseg; i++) {
        if (!seg[i].count) continue;
        hp_count<<<grid_for((seg[i].count + 3) / 4, 256), 256, 0, stream()>>>(seg[i].dst, seg[i].src, seg[i].count, n,
                                                                               fill, err);
        PIPNN_LAUNCH_CHECK();
        count += seg[i].count;
    }
    if (count) {
        hp_widen<<<grid_for(n, 256), 256, 0, stream()>>>(fill, n, start);
        PIPNN_LAUNCH_CHECK();
    }
    PIPNN_TRY(exclusive_scan_u64(start, start, n, tot, ws));
    PIPNN_CUDA(cudaMemcpyAsync(start + n, tot, 8, cudaMemcpyDeviceToDevice, stream()));
    PIPNN_TRY(read_u64(tot, &E));
    PIPNN_TRY(ws.alloc(&slots, E));
    for (uint32_t i = 0; i < nseg; i++) {
        if (!seg[i].count) continue;
        hp_scatter<<<grid_for((seg[i].count + 3) / 4, 256), 256, 0, stream()>>>(
            seg[i].dst, seg[i].src, seg[i].dist, seg[i].count, n, S, m, reinterpret_cast<unsigned long long *>(start),
            slots);
        PIPNN_LAUNCH_CHECK();
    }
    size_t smem = hashprune_smem_bytes(m);
    PIPNN_CUDA(cudaFuncSetAttribute(hp_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    hp_merge<<<grid_for(n, HP_WARPS, 152u * 8u), HP_WARPS * 32, smem, stream()>>>(n, m, l_max, start, slots, res, cnt,
                                                                                   padded);
    PIPNN_LAUNCH_CHECK();
    return check_device_error("hashprune");
}

int hashprune_merge(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count, const float *S,
                    uint32_t m, uint64_t n, uint32_t l_max, uint64_t *res, uint32_t *cnt, int padded) {
    const EdgeSegment seg{dst, src, dist, count};
    return hashprune_merge_segments(&seg, 1, S, m, n, l_max, res, cnt, padded);
}

}  // namespace pipnn

// ---------------------------------------------------------------------------------------------
// pipnn_hashprune_noalloc: HashPrune for callers that cannot allocate device memory.
//
// Its scratch (per-node run offsets and fill counters, the scan's per-tile totals, the grouped
// slots and the error word) lives in one file-scope device array of HP_STATIC_BYTES that every
// GPU loading this library keeps until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device, with that device current, asks
// the runtime for the address once (cudaGetSymbolAddress) and later calls reuse it; the remembered
// address does not survive cudaDeviceReset (the library's module is reloaded afterwards, possibly
// elsewhere), so a process that resets a device must not call this entry point again.  Every call
// shares the array and reuses whatever the previous call left there, so the parts that must
// start at zero are cleared on each call; two calls whose work overlaps on the GPU (different
// streams or host threads on the same device) race on it.
// ---------------------------------------------------------------------------------------------
#include <mutex>

namespace pipnn {
void set_device_error_word(unsigned *p);

namespace {
constexpr size_t HP_STATIC_BYTES = 64ull << 20;
constexpr int HP_STATIC_MAX_DEVICES = 64;
static __device__ __align__(256) unsigned char g_hp_static_scratch[HP_STATIC_BYTES];
std::mutex g_hp_static_mu;
void *g_hp_static_addr[HP_STATIC_MAX_DEVICES];

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct StaticLayout {
    size_t err, total, start, fill, scan, slots, bytes;
};

StaticLayout static_layout(uint64_t n, uint64_t count) {
    StaticLayout L;
    L.err = 0;
    L.total = 8;
    L.start = 256;
    L.fill = L.start + round256((n + 1) * 8);
    L.scan = L.fill + round256(n * 4);
    L.slots = L.scan + round256(scan_scratch_elems(n) * 8);
    L.bytes = L.slots + count * 8;
    return L;
}

int static_scratch_address(unsigned char **base) {
    int dev = 0;
    PIPNN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= HP_STATIC_MAX_DEVICES) return set_error(PIPNN_EUNSUPPORTED, "device %d", dev);
    std::lock_guard<std::mutex> lock(g_hp_static_mu);
    if (!g_hp_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_hp_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(PIPNN_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                             cudaGetErrorString(e));
        }
        g_hp_static_addr[dev] = p;
    }
    *base = static_cast<unsigned char *>(g_hp_static_addr[dev]);
    return PIPNN_OK;
}

int hashprune_noalloc_impl(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count,
                           const float *S, uint32_t m, uint64_t n, uint32_t l_max, uint64_t *res, uint32_t *cnt) {
    if (count && (!dst || !src || !dist)) return set_error(PIPNN_EINVAL, "candidate arrays are NULL");
    if (!S || !res || !cnt) return set_error(PIPNN_EINVAL, "sketch/reservoir/count are NULL");
    if (n == 0 || n >= 0xFFFFFFFFull) return set_error(PIPNN_EINVAL, "n outside 1..2^32-2");
    if (m < 1 || m > 16) return set_error(PIPNN_EINVAL, "hash_bits %u outside 1..16", m);
    if (l_max < 1 || l_max > 256) return set_error(PIPNN_EINVAL, "l_max %u outside 1..256", l_max);
    // bound n and count first, so the layout arithmetic below cannot wrap around
    const bool too_big = count > HP_STATIC_BYTES / 8 || n > HP_STATIC_BYTES / 12;
    const StaticLayout L = too_big ? StaticLayout{0, 0, 0, 0, 0, 0, ~(size_t)0} : static_layout(n, count);
    if (too_big || L.bytes > HP_STATIC_BYTES)
        return set_error(PIPNN_EINVAL,
                         "n = %llu nodes and %llu candidates need more than the %zu bytes the static scratch "
                         "holds (use pipnn_hashprune or split the stream)",
                         (unsigned long long)n, (unsigned long long)count, HP_STATIC_BYTES);
    unsigned char *base = nullptr;
    PIPNN_TRY(static_scratch_address(&base));
    unsigned *err = reinterpret_cast<unsigned *>(base + L.err);
    uint64_t *total = reinterpret_cast<uint64_t *>(base + L.total);
    uint64_t *start = reinterpret_cast<uint64_t *>(base + L.start);
    unsigned *fill = reinterpret_cast<unsigned *>(base + L.fill);
    uint64_t *scan = reinterpret_cast<uint64_t *>(base + L.scan);
    uint64_t *slots = reinterpret_cast<uint64_t *>(base + L.slots);

    PIPNN_CUDA(cudaMemsetAsync(base, 0, 256, stream()));
    PIPNN_CUDA(cudaMemsetAsync(start, 0, (n + 1) * 8, stream()));
    PIPNN_CUDA(cudaMemsetAsync(fill, 0, n * 4, stream()));
    set_device_error_word(err);
    struct Restore {
        ~Restore() { set_device_error_word(nullptr); }
    } restore;

    if (count) {
        hp_count<<<grid_for((count + 3) / 4, 256), 256, 0, stream()>>>(dst, src, count, n, fill, err);
        PIPNN_LAUNCH_CHECK();
        hp_widen<<<grid_for(n, 256), 256, 0, stream()>>>(fill, n, start);
        PIPNN_LAUNCH_CHECK();
    }
    PIPNN_TRY(exclusive_scan_u64_scratch(start, start, n, total, scan));
    PIPNN_CUDA(cudaMemcpyAsync(start + n, total, 8, cudaMemcpyDeviceToDevice, stream()));
    if (count) {
        hp_scatter<<<grid_for((count + 3) / 4, 256), 256, 0, stream()>>>(dst, src, dist, count, n, S, m,
                                                                          reinterpret_cast<unsigned long long *>(start),
                                                                          slots);
        PIPNN_LAUNCH_CHECK();
    }
    const size_t smem = hashprune_smem_bytes(m);
    PIPNN_CUDA(cudaFuncSetAttribute(hp_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    hp_merge<<<grid_for(n, HP_WARPS, 152u * 8u), HP_WARPS * 32, smem, stream()>>>(n, m, l_max, start, slots, res, cnt,
                                                                                   0);
    PIPNN_LAUNCH_CHECK();
    return check_device_error("hashprune (static scratch)");
}
}  // namespace
}  // namespace pipnn

extern "C" int pipnn_hashprune_noalloc(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count,
                                       const float *sketch, uint32_t m, uint64_t n, uint32_t l_max,
                                       uint64_t *reservoir, uint32_t *count_inout) {
    pipnn::clear_error();
    return pipnn::hashprune_noalloc_impl(dst, src, dist, count, sketch, m, n, l_max, reservoir, count_inout);
}
