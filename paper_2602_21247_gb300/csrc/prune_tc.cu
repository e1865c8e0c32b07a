// prune_tc.cu -- A6: Alg. 2 RobustPrune on the tensor cores (byte data, d <= 128, l_max <= 127).
//
// For a node x with candidates z_0..z_{c-1} (its reservoir in slot order, invalid ids dropped)
// one MMA forms the Gram matrix of the c + 1 rows [z_0, .., z_{c-1}, x] with the norm fold of the
// leaf engine:  acc[r][s] = <x_r, x_s> - n_s / 2,  so  D(r, s) = n_r - 2 acc[r][s]  exactly.
// Alg. 2 then needs only comparisons of entries of this matrix:
//  * order: candidates by (D(x, z), id).  D(x, z_r) is column c of row r.  The reservoir is sorted
//    by the BF16 rounding of the same distance (then id), and rounding is monotone, so the rank of
//    z_r is the first slot of its run of equal BF16 keys plus its place inside the run.  Both
//    premises are checked per node; if either fails the rank is a full count.
//  * removal: admitted y removes z iff fl(alpha^2 * D(y, z)) < D(x, z).  fl(alpha^2 * t) is
//    monotone in t, so there is an integer T_z with  fl(alpha^2 * t) < D(x, z)  <=>  t < T_z,
//    and D(y, z) = D(z, y); hence y removes z iff acc[z][y] > (n_z - T_z) / 2.  Row z of the
//    accumulator gives, one compare per entry, the set of candidates that would remove z (its
//    "column mask").
//  * walk: in rank order a candidate is admitted unless its column mask meets the admitted set
//    (the removal loop of Alg. 2 and its lazy form coincide), up to R admissions.
//
// Persistent CTA (one per SM, 21 warps):
//   warp 0       node info: reservoir slots and norms (loaded a node ahead), compaction of the
//                valid ids, BF16 keys, norm pieces
//   warp 20      TMA gather4 of the node's rows (ids from the node info)
//   warp 1       owns TMEM (4 x 128 columns); one thread issues the Gram MMAs
//   warps 2-13   epilogue: three groups of four warps (one per TMEM lane quarter, a thread per
//                row) take turns on nodes: D(x, .), thresholds, ranks, column masks -> walk slot
//   warps 14-19  walkers: one node at a time each, write adj / deg
// Waits are bounded as in the other engines (DERR_TIMEOUT; TMEM is still released).
#include "tc_common.cuh"

namespace pipnn {

namespace {

using namespace tc;

constexpr int PT_GROUPS = 3;                                     // epilogue groups of 4 warps
constexpr int PT_EPI_WARPS = 4 * PT_GROUPS;
constexpr int PT_WALKERS = 6;
constexpr int PT_WALK_WARP0 = 2 + PT_EPI_WARPS;
constexpr int PT_GATHER_WARP = PT_WALK_WARP0 + PT_WALKERS;
constexpr int PT_THREADS = (PT_GATHER_WARP + 1) * 32;
constexpr uint32_t PT_MAXC = 127;                                 // candidates per node (+ the node)

struct PtArgs {
    const uint64_t *res;   // n x l_max reservoir slots
    const uint32_t *cnt;   // entries per reservoir
    const int32_t *sqn;    // exact squared norms
    uint64_t n;
    uint32_t l_max, R;
    float alpha2, inv_alpha2;
    uint32_t *adj, *deg;
    unsigned *err;
};

template <int KB>
struct PtCfg {
    static constexpr int A = 4;            // gathered row tiles in flight
    static constexpr int T = 4;            // accumulator buffers = node-info slots
    static constexpr int W = PT_WALKERS;   // walk slots (walker w owns slot w)
    // node info, producer -> epilogue: ids[128] u32, norms[128] i32, BF16 keys[128] u16, c, v
    static constexpr int I_IDS = 0, I_NRM = 512, I_BKEY = 1024, I_MISC = 1280, I_BYTES = 1296;
    // walk slot, epilogue -> walker: column masks[128] x 4 u32, ids[128], order[128] u8, c, v
    static constexpr int W_MASK = 0, W_IDS = 2048, W_ORDER = 2560, W_MISC = 2688, W_BYTES = 2704;
    static constexpr int OFF_A0 = 0;
    static constexpr int OFF_AN = OFF_A0 + A * KB * REGION;
    static constexpr int OFF_BN = OFF_AN + REGION;          // a 32-byte norm slice per A buffer
    static constexpr int OFF_INFO = OFF_BN + REGION;
    static constexpr int OFF_WS = OFF_INFO + T * I_BYTES;
    static constexpr int OFF_DX = OFF_WS + W * W_BYTES;     // per group 2 x 128 u32: D(x, z_r) by row
    static constexpr int OFF_BAR = OFF_DX + PT_GROUPS * 2 * 128 * 4;
    static constexpr int BAR_FULL_A = 0, BAR_EMPTY_A = A, BAR_CFULL = 2 * A, BAR_TFULL = 2 * A + T,
                         BAR_TEMPTY = 2 * A + 2 * T, BAR_WFULL = 2 * A + 3 * T, BAR_WEMPTY = 2 * A + 3 * T + W,
                         NBAR = 2 * A + 3 * T + 2 * W;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;     // tmem base, abort flag
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr int SMEM = BYTES + 1024;
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(T * 128 <= (int)TMEM_COLS, "TMEM budget");
    static_assert(A <= 4, "norm slices per 128-byte row");
    static_assert(I_BYTES % 16 == 0 && W_BYTES % 16 == 0, "slot alignment");
};

// Register g[j] for a run-time j (five-level select tree).
__device__ __forceinline__ uint32_t pick32(const uint32_t (&g)[32], uint32_t j) {
    uint32_t a[16], b[8], c[4], e[2];
#pragma unroll
    for (int i = 0; i < 16; i++) a[i] = (j & 16u) ? g[i + 16] : g[i];
#pragma unroll
    for (int i = 0; i < 8; i++) b[i] = (j & 8u) ? a[i + 8] : a[i];
#pragma unroll
    for (int i = 0; i < 4; i++) c[i] = (j & 4u) ? b[i + 4] : b[i];
#pragma unroll
    for (int i = 0; i < 2; i++) e[i] = (j & 2u) ? c[i + 2] : c[i];
    return (j & 1u) ? e[1] : e[0];
}

// Smallest integer t >= 0 with !(fl(alpha2 * t) < dx): a candidate at distance dx from the node is
// removed by y exactly when D(y, z) < T.  (alpha2 = +inf gives T = 0: nothing is removed, as
// inf * t < dx never holds and 0 * inf is NaN.)
// The estimate dx * (1 / alpha2) is within a few units of T (relative error ~2^-22 on values
// below 2^24), and the two bounded walks make it exact.
__device__ __forceinline__ uint32_t removal_threshold(uint32_t dx, float alpha2, float inv_alpha2) {
    if (dx == 0) return 0;
    const float f = (float)dx;  // dx < 2^24: exact
    uint32_t t = (uint32_t)fminf(__fmul_rn(f, inv_alpha2), 16777216.0f);
    for (int i = 0; i < 8 && t > 0 && !(__fmul_rn(alpha2, (float)(t - 1)) < f); i++) t--;
    for (int i = 0; i < 8 && __fmul_rn(alpha2, (float)t) < f; i++) t++;
    return t;
}

// Order-preserving image of bf16_rn(f), as stored in the top 16 bits of a reservoir slot.
__device__ __forceinline__ uint32_t bf16_key(float f) {
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(f));
    return (b & 0x8000u) ? (~b & 0xFFFFu) : (b | 0x8000u);
}

template <int KB>
__global__ void __launch_bounds__(PT_THREADS, 1)
    prune_tc_kernel(const __grid_constant__ CUtensorMap xmap, const PtArgs a) {
    using C = PtCfg<KB>;
    extern __shared__ unsigned char pt_smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(pt_smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + C::OFF_MISC);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + C::OFF_MISC + 4);
    auto bar = [&](int i) { return sbase + C::OFF_BAR + 8 * i; };
    auto info = [&](uint32_t tb) { return smem + C::OFF_INFO + tb * C::I_BYTES; };
    auto wslot = [&](uint32_t ws) { return smem + C::OFF_WS + ws * C::W_BYTES; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t n = a.n;

    if (threadIdx.x == 0) {
        for (int i = 0; i < C::A; i++) {
            mbar_init(bar(C::BAR_FULL_A + i), 64);  // info warp + gather warp
            mbar_init(bar(C::BAR_EMPTY_A + i), 1);
        }
        for (int i = 0; i < C::T; i++) {
            mbar_init(bar(C::BAR_CFULL + i), 32);
            mbar_init(bar(C::BAR_TFULL + i), 1);
            mbar_init(bar(C::BAR_TEMPTY + i), 128);
        }
        for (int i = 0; i < C::W; i++) {
            mbar_init(bar(C::BAR_WFULL + i), 128);
            mbar_init(bar(C::BAR_WEMPTY + i), 32);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == MMA_WARP) tmem_alloc(sbase + C::OFF_MISC, TMEM_COLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == PRODUCER_WARP) {
        // ------------------------------------------------------------ producer (one warp)
        for (uint32_t r = lane; r < 128u; r += 32) {
            const uint32_t one = 0x3F80u;  // bf16 1.0
            const uint32_t base = sbase + C::OFF_AN + r * 128;
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(base + ((0u ^ (r & 7)) << 4)),
                         "r"(one | (one << 16)), "r"(one | (one << 16)), "r"(0u), "r"(0u)
                         : "memory");
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(base + ((1u ^ (r & 7)) << 4)), "r"(0u),
                         "r"(0u), "r"(0u), "r"(0u)
                         : "memory");
            // every buffer's 32-byte norm slice starts zero; a node rewrites only its first 8 bytes
            for (uint32_t q = 0; q < 2u * C::A; q++)
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(sbase + C::OFF_BN + r * 128 +
                                                                              ((q ^ (r & 7)) << 4)),
                             "r"(0u), "r"(0u), "r"(0u), "r"(0u)
                             : "memory");
        }
        fence_proxy_async();
        // Software pipeline: the reservoir slots of node j + 1 and the norms of its valid
        // candidates are loaded while node j is issued (two dependent global round trips that a
        // node would otherwise wait for in turn).
        struct Pre {
            uint64_t key[4];
            int32_t nr[4];
            int32_t nv;
            uint32_t c;
        };
        auto load_keys = [&](uint64_t v, Pre &p) {
            p.c = 0;
            p.nv = 0;
            if (v >= n) return;
            p.nv = a.sqn[v];
            const uint32_t c = a.cnt[v];
            p.c = c < a.l_max ? c : a.l_max;
            // every slot of the row is read, so these loads do not wait for the count
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t s = 32 * k + lane;
                p.key[k] = s < a.l_max ? a.res[v * a.l_max + s] : 0ull;
            }
        };
        auto load_norms = [&](Pre &p) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t s = 32 * k + lane;
                const uint32_t id = (uint32_t)(p.key[k] >> 16);
                p.nr[k] = (s < p.c && (uint64_t)id < n) ? a.sqn[id] : 0;
            }
        };
        Pre cur, nxt;
        load_keys(blockIdx.x, cur);
        load_norms(cur);
        load_keys(blockIdx.x + (uint64_t)gridDim.x, nxt);
        for (uint32_t j = 0;; j++) {
            const uint64_t v = blockIdx.x + (uint64_t)j * gridDim.x;
            if (v >= n) break;
            const uint32_t ua = j % C::A, tb = j % C::T;
            Pre nn;
            load_keys(v + 2 * (uint64_t)gridDim.x, nn);
            load_norms(nxt);
            const uint32_t c = cur.c;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_TEMPTY + tb), ((j / C::T) & 1) ^ 1, abort, a.err)))
                break;
            unsigned char *in = info(tb);
            uint32_t *ids = reinterpret_cast<uint32_t *>(in + C::I_IDS);
            int32_t *nrm = reinterpret_cast<int32_t *>(in + C::I_NRM);
            uint16_t *bkey = reinterpret_cast<uint16_t *>(in + C::I_BKEY);
            uint32_t cc = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t s = 32 * k + lane;
                const uint32_t id = (uint32_t)(cur.key[k] >> 16);
                const bool in_range = s < c && (uint64_t)id < n;
                if (s < c && !in_range) atomicOr(a.err, DERR_RANGE);
                const unsigned m = __ballot_sync(0xffffffffu, in_range);
                if (in_range) {
                    const uint32_t pos = cc + __popc(m & ((1u << lane) - 1u));
                    ids[pos] = id;
                    nrm[pos] = cur.nr[k];
                    bkey[pos] = (uint16_t)(cur.key[k] >> 48);
                }
                cc += __popc(m);
            }
            if (lane == 0) {
                ids[cc] = (uint32_t)v;
                nrm[cc] = cur.nv;
                reinterpret_cast<uint32_t *>(in + C::I_MISC)[0] = cc;
                reinterpret_cast<uint32_t *>(in + C::I_MISC)[1] = (uint32_t)v;
            }
            __syncwarp();
            mbar_arrive(bar(C::BAR_CFULL + tb));
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_EMPTY_A + ua), ((j / C::A) & 1) ^ 1, abort, a.err)))
                break;
            // -(n_r / 2) pieces of every row in this buffer's norm slice; zero past the rows
            const uint32_t rows = cc + 1;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t r = 4 * lane + e;
                const uint2 pc = neg_half_norm_pieces(r < rows ? (uint32_t)nrm[r] : 0u);
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(sbase + C::OFF_BN + r * 128 +
                                                                     (((2 * ua) ^ (r & 7)) << 4)),
                             "r"(pc.x), "r"(pc.y)
                             : "memory");
            }
            fence_proxy_async();
            mbar_arrive(bar(C::BAR_FULL_A + ua));
            cur = nxt;
            nxt = nn;
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t issued_j = 0;
            bool any = false, stop = false;
            for (uint32_t j = 0;; j++) {
                const uint64_t v = blockIdx.x + (uint64_t)j * gridDim.x;
                if (v >= n) break;
                const uint32_t ua = j % C::A, tb = j % C::T;
                if (!mbar_wait(bar(C::BAR_CFULL + tb), (j / C::T) & 1, abort, a.err) ||
                    !mbar_wait(bar(C::BAR_FULL_A + ua), (j / C::A) & 1, abort, a.err) ||
                    !mbar_wait(bar(C::BAR_TEMPTY + tb), ((j / C::T) & 1) ^ 1, abort, a.err)) {
                    stop = true;
                    break;
                }
                fence_after();
                const uint32_t rows = reinterpret_cast<const uint32_t *>(info(tb) + C::I_MISC)[0] + 1;
                const uint32_t idesc = idesc_bf16(128, (rows + 15) & ~15u);
                const uint32_t aB = sbase + C::OFF_A0 + ua * KB * REGION;
                const uint32_t d = tmem + tb * 128;
#pragma unroll
                for (int kk = 0; kk < KB * 4; kk++) {
                    const uint64_t desc = smem_desc_sw128(aB + (kk >> 2) * REGION + (kk & 3) * 32);
                    mma_bf16(d, desc, desc, idesc, kk > 0 ? 1u : 0u);
                }
                mma_bf16(d, smem_desc_sw128(sbase + C::OFF_AN), smem_desc_sw128(sbase + C::OFF_BN + ua * 32), idesc,
                         1u);
                mma_commit(bar(C::BAR_EMPTY_A + ua));
                mma_commit(bar(C::BAR_TFULL + tb));
                any = true;
                issued_j = j;
            }
            if (stop && any)
                mbar_wait(bar(C::BAR_TFULL + issued_j % C::T), (issued_j / C::T) & 1, abort, a.err);
        }
        __syncwarp();
    } else if (warp < PT_WALK_WARP0) {
        // ------------------------------------------------------------ epilogue (groups of 4 warps)
        const uint32_t grp = (warp - EPI_WARP0) >> 2;  // group: nodes j = grp, grp + PT_GROUPS, ...
        const int quarter = warp & 3;                   // TMEM lane quarter this warp may access
        const uint32_t r = quarter * 32 + lane;         // row = candidate slot
        const uint32_t bar_id = 1 + grp;
        bool stop = false;
        for (uint32_t k = 0;; k++) {
            const uint32_t j = grp + k * PT_GROUPS;
            const uint64_t vv = blockIdx.x + (uint64_t)j * gridDim.x;
            if (vv >= n) break;
            const uint32_t tb = j % C::T, ws = j % C::W;
            const bool ok = !stop && __all_sync(0xffffffffu,
                                                 mbar_wait(bar(C::BAR_TFULL + tb), (j / C::T) & 1, abort, a.err) &&
                                                     mbar_wait(bar(C::BAR_CFULL + tb), (j / C::T) & 1, abort, a.err) &&
                                                     mbar_wait(bar(C::BAR_WEMPTY + ws), ((j / C::W) & 1) ^ 1, abort,
                                                               a.err));
            const unsigned char *in = info(tb);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(in + C::I_IDS);
            const int32_t *nrm = reinterpret_cast<const int32_t *>(in + C::I_NRM);
            const uint16_t *bkey = reinterpret_cast<const uint16_t *>(in + C::I_BKEY);
            uint32_t *dx = reinterpret_cast<uint32_t *>(smem + C::OFF_DX) + (grp * 2 + (k & 1)) * 128;
            unsigned char *wsl = wslot(ws);
            uint32_t c = 0, DX = 0;
            float theta = 0.0f;
            bool bad = false;
            if (ok) {
                fence_after();
                c = reinterpret_cast<const uint32_t *>(in + C::I_MISC)[0];
                // E1: D(x, z_r) from column c of row r; the removal threshold of z_r
                uint32_t g[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + tb * 128 + (c & ~31u), g);
                if (r < c) {
                    const float acc = __uint_as_float(pick32(g, c & 31u));
                    const int32_t nr = nrm[r];
                    const float dxf = __fmaf_rn(-2.0f, acc, (float)nr);  // exact integer
                    DX = (uint32_t)dxf;
                    const uint32_t T = removal_threshold(DX, a.alpha2, a.inv_alpha2);
                    theta = ((float)nr - (float)T) * 0.5f;             // exact (multiple of 1/2)
                    dx[r] = DX;
                    bad = bf16_key(dxf) != bkey[r] || (r > 0 && bkey[r - 1] > bkey[r]);
                }
            }
            const bool full_count = named_barrier_or(bar_id, 128, ok && bad);
            if (ok) {
                // E2: rank of z_r in (D(x, z), id, slot) order
                if (r < c) {
                    const uint32_t id = ids[r];
                    uint32_t lo = 0;
                    if (!full_count) {
                        lo = r;
                        while (lo > 0 && bkey[lo - 1] == bkey[r]) lo--;
                    }
                    uint32_t rank = lo;
                    for (uint32_t s = lo; s < c && (full_count || bkey[s] == bkey[r]); s++) {
                        const uint32_t ds = dx[s], is = ids[s];
                        rank += (ds < DX || (ds == DX && (is < id || (is == id && s < r)))) ? 1u : 0u;
                    }
                    wsl[C::W_ORDER + rank] = (unsigned char)r;
                    reinterpret_cast<uint32_t *>(wsl + C::W_IDS)[r] = id;
                }
                if (r == 0) {
                    reinterpret_cast<uint32_t *>(wsl + C::W_MISC)[0] = c;
                    reinterpret_cast<uint32_t *>(wsl + C::W_MISC)[1] =
                        reinterpret_cast<const uint32_t *>(in + C::I_MISC)[1];
                }
                // E3: column mask of z_r -- the candidates y with acc[r][y] > theta_r
                uint32_t mw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    if (q * 32 < c) {
                        uint32_t g[32];
                        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + tb * 128 + q * 32, g);
                        uint32_t m = 0;
#pragma unroll
                        for (int jj = 0; jj < 32; jj++) m |= __uint_as_float(g[jj]) > theta ? (1u << jj) : 0u;
                        const uint32_t live = c - q * 32;
                        if (live < 32) m &= (1u << live) - 1u;
                        if (r / 32 == q) m &= ~(1u << (r & 31));
                        mw[q] = m;
                    }
                }
                if (r < c) reinterpret_cast<uint4 *>(wsl + C::W_MASK)[r] = make_uint4(mw[0], mw[1], mw[2], mw[3]);
                fence_before();
                mbar_arrive(bar(C::BAR_TEMPTY + tb));
                mbar_arrive(bar(C::BAR_WFULL + ws));
            }
            stop = named_barrier_or(bar_id, 128, !ok || *abort);
            if (stop) break;
        }
    } else if (warp < PT_GATHER_WARP) {
        // ------------------------------------------------------------ walkers
        const uint32_t w = warp - PT_WALK_WARP0;
        for (uint32_t k = 0;; k++) {
            const uint32_t j = w + k * C::W;
            const uint64_t vv = blockIdx.x + (uint64_t)j * gridDim.x;
            if (vv >= n) break;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_WFULL + w), k & 1, abort, a.err))) break;
            const unsigned char *wsl = wslot(w);
            const uint32_t c = reinterpret_cast<const uint32_t *>(wsl + C::W_MISC)[0];
            const uint64_t v = reinterpret_cast<const uint32_t *>(wsl + C::W_MISC)[1];
            const uint4 *mask = reinterpret_cast<const uint4 *>(wsl + C::W_MASK);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(wsl + C::W_IDS);
            const unsigned char *order = wsl + C::W_ORDER;
            const uint32_t R = a.R;
            uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0;  // admitted slots
            uint32_t e = 0;
            uint32_t out[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
            for (uint32_t b = 0; b * 32 < c && e < R; b++) {
                const uint32_t i = b * 32 + lane;
                const uint32_t tl = i < c ? order[i] : 0u;
                const uint4 cm = i < c ? mask[tl] : make_uint4(0, 0, 0, 0);
                const uint32_t nb = c - b * 32 < 32 ? c - b * 32 : 32;
#pragma unroll 4
                for (uint32_t jj = 0; jj < nb; jj++) {
                    const uint32_t t = __shfl_sync(0xffffffffu, tl, jj);
                    const uint32_t cx = __shfl_sync(0xffffffffu, cm.x, jj), cy = __shfl_sync(0xffffffffu, cm.y, jj);
                    const uint32_t cz = __shfl_sync(0xffffffffu, cm.z, jj), cw = __shfl_sync(0xffffffffu, cm.w, jj);
                    if (((cx & A0) | (cy & A1) | (cz & A2) | (cw & A3)) == 0u) {
                        const uint32_t bit = 1u << (t & 31);
                        const uint32_t wd = t >> 5;
                        A0 |= wd == 0 ? bit : 0u;
                        A1 |= wd == 1 ? bit : 0u;
                        A2 |= wd == 2 ? bit : 0u;
                        A3 |= wd == 3 ? bit : 0u;
                        const uint32_t id = ids[t];
                        const bool mine = (e & 31) == (uint32_t)lane;
                        const uint32_t o = e >> 5;
                        out[0] = (mine && o == 0) ? id : out[0];
                        out[1] = (mine && o == 1) ? id : out[1];
                        out[2] = (mine && o == 2) ? id : out[2];
                        out[3] = (mine && o == 3) ? id : out[3];
                        if (++e == R) break;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t p = lane + 32 * q;
                if (p < R) a.adj[v * R + p] = p < e ? out[q] : 0xFFFFFFFFu;
            }
            if (lane == 0) a.deg[v] = e;
            __syncwarp();
            mbar_arrive(bar(C::BAR_WEMPTY + w));
        }
    } else {
        // ------------------------------------------------------------ row gathers (one warp)
        for (uint32_t j = 0;; j++) {
            const uint64_t v = blockIdx.x + (uint64_t)j * gridDim.x;
            if (v >= n) break;
            const uint32_t ua = j % C::A, tb = j % C::T;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_CFULL + tb), (j / C::T) & 1, abort, a.err) &&
                                             mbar_wait(bar(C::BAR_EMPTY_A + ua), ((j / C::A) & 1) ^ 1, abort,
                                                       a.err)))
                break;
            const unsigned char *in = info(tb);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(in + C::I_IDS);
            const uint32_t rows = reinterpret_cast<const uint32_t *>(in + C::I_MISC)[0] + 1;
            const uint32_t ng = (rows + 3) / 4;  // gathers of four rows
            const uint32_t fb = bar(C::BAR_FULL_A + ua);
            if (lane == 0) mbar_arrive_tx(fb, ng * 512u * KB);
            __syncwarp();
            if ((uint32_t)lane < ng) {
                int32_t y[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const uint32_t r = 4 * lane + e;
                    y[e] = (int32_t)(r < rows ? ids[r] : ids[rows - 1]);
                }
                const uint32_t dst = sbase + C::OFF_A0 + ua * KB * REGION + lane * 4 * 128;
#pragma unroll
                for (int kb = 0; kb < KB; kb++) tma_gather4(dst + kb * REGION, &xmap, kb * 64, y[0], y[1], y[2], y[3], fb);
            }
            if (lane != 0) mbar_arrive(fb);
        }
    }

    fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

template <int KB>
int launch_pt(const CUtensorMap &xmap, const PtArgs &args) {
    using C = PtCfg<KB>;
    auto kern = prune_tc_kernel<KB>;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int dev = 0, sms = 0;
    PIPNN_CUDA(cudaGetDevice(&dev));
    PIPNN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)(args.n < (uint64_t)sms ? args.n : (uint64_t)sms);
    kern<<<grid, PT_THREADS, C::SMEM, stream()>>>(xmap, args);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

}  // namespace

bool prune_tc_eligible(int dtype, uint32_t d, uint64_t n, uint32_t l_max) {
    return (dtype == PIPNN_U8 || dtype == PIPNN_I8) && d >= 1 && d <= 128 && n >= 1 && n < 0x7FFFFF00ull &&
           l_max >= 1 && l_max <= PT_MAXC;
}

int final_prune_tc(const void *X, uint64_t n, uint32_t d, int dtype, const int32_t *sqn, const uint64_t *res,
                   const uint32_t *cnt, uint32_t l_max, uint32_t R, float alpha2, uint32_t *adj, uint32_t *deg,
                   Workspace &ws) {
    if (!prune_tc_eligible(dtype, d, n, l_max))
        return set_error(PIPNN_EUNSUPPORTED, "the tensor-core prune takes byte data, d <= 128, l_max <= %u", PT_MAXC);
    if (R < 1 || R > l_max) return set_error(PIPNN_EINVAL, "R outside 1..l_max");
    const uint32_t kp = d <= 64 ? 64 : 128;
    __nv_bfloat16 *rows = nullptr;
    PIPNN_TRY(ws.alloc(&rows, n * kp));
    PIPNN_TRY(stage_rows_bf16(X, d, kp, dtype, nullptr, n, rows));
    CUtensorMap map;
    PIPNN_TRY(encode_rows_map(&map, rows, n, kp, true));
    PtArgs a{};
    a.res = res;
    a.cnt = cnt;
    a.sqn = sqn;
    a.n = n;
    a.l_max = l_max;
    a.R = R;
    a.alpha2 = alpha2;
    a.inv_alpha2 = 1.0f / alpha2;
    a.adj = adj;
    a.deg = deg;
    a.err = device_error_word();
    if (kp == 64) return launch_pt<1>(map, a);
    return launch_pt<2>(map, a);
}

}  // namespace pipnn
