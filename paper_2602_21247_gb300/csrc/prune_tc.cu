// prune_tc.cu -- A6: Alg. 2 RobustPrune on the tensor cores (byte data, d <= 128, l_max <= 127).
//
// For a node x with candidates z_0..z_{c-1} (its reservoir in slot order, invalid ids dropped)
// one MMA forms the Gram matrix G of the c + 1 rows [z_0, .., z_{c-1}, x] (BF16 operands, FP32
// accumulation; exact for bytes).  Its diagonal holds the squared norms n_r = G[r][r], so
// D(r, s) = n_r + n_s - 2 G[r][s] needs no other input.
// Alg. 2 then needs only comparisons of entries of this matrix:
//  * order: candidates by (D(x, z), id).  D(x, z_r) is column c of row r.  The reservoir is sorted
//    by the BF16 rounding of the same distance (then id), and rounding is monotone, so the rank of
//    z_r is the first slot of its run of equal BF16 keys plus its place inside the run.  Both
//    premises are checked per node; if either fails the rank is a full count.
//  * removal: admitted y removes z iff fl(alpha^2 * D(y, z)) < D(x, z).  fl(alpha^2 * t) is
//    monotone in t, so there is an integer T_z with  fl(alpha^2 * t) < D(x, z)  <=>  t < T_z,
//    and D(y, z) = D(z, y); hence y removes z iff G[z][y] - n_y / 2 > (n_z - T_z) / 2.  Row z of
//    the accumulator gives, with one subtraction and one compare per entry, the set of
//    candidates that would remove z (its "column mask").
//  * walk: in rank order a candidate is admitted unless its column mask meets the admitted set
//    (the removal loop of Alg. 2 and its lazy form coincide), up to R admissions.
//
// Persistent CTA (one per SM, 20 warps):
//   warps 0-11   epilogue: three groups of four warps (one per TMEM lane quarter, a thread per
//                row) take turns on nodes: norms, D(x, .), thresholds, ranks, column masks
//   warp 12      owns TMEM (4 x 128 columns); one thread issues the Gram MMAs
//   warp 15      node info: reservoir slots (loaded two nodes ahead), compaction of the valid
//                ids, BF16 keys
//   warps 17-18  TMA gather4 of the rows of alternate nodes (ids from the node info)
//   warps 13, 14, 16, 19  walkers: write adj / deg
// Waits are bounded as in the other engines (DERR_TIMEOUT; TMEM is still released).
#include "tc_common.cuh"

namespace pipnn {

namespace {

using namespace tc;

// Warp roles.  A warp reaches TMEM lanes 32 (w % 4) .. +31 and runs on scheduler w % 4, so the
// epilogue groups are warps 4g .. 4g + 3, and the other roles are placed so that each scheduler
// carries a similar load (the rows of lane quarter 0, the nearest candidates, are always
// occupied; quarter 3 is the lightest).
constexpr int PT_GROUPS = 3;                 // epilogue groups of 4 warps: warps 0 .. 11
constexpr int PT_EPI_WARPS = 4 * PT_GROUPS;
constexpr int PT_MMA_WARP = 12;              // scheduler 0
constexpr int PT_INFO_WARP = 15;             // scheduler 3
constexpr int PT_WALKERS = 4;                // warps 13, 14, 16, 19
constexpr int PT_GATHERERS = 2;              // warps 17, 18
constexpr int PT_THREADS = 20 * 32;
__host__ __device__ constexpr int walker_of(int warp) {
    return warp == 13 ? 0 : warp == 14 ? 1 : warp == 16 ? 2 : warp == 19 ? 3 : -1;
}
__host__ __device__ constexpr int gatherer_of(int warp) { return warp == 17 ? 0 : warp == 18 ? 1 : -1; }
constexpr uint32_t PT_MAXC = 127;                                 // candidates per node (+ the node)
constexpr int W_MASK_OFF = 0, W_IDS_OFF = 2048, W_ORDER_OFF = 2560, W_MISC_OFF = 2688, W_SLOT_BYTES = 2704;

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
    static constexpr int T = 4;            // accumulator buffers
    static constexpr int I = 8;            // node-info slots (info and gathers run ahead)
    static constexpr int W = 2 * PT_WALKERS;  // walk slots (walker w alternates between w and w + PT_WALKERS)
    // node info, producer -> epilogue: ids[128] u32, BF16 keys[128] u16, c, v, n_x
    static constexpr int I_IDS = 0, I_BKEY = 512, I_MISC = 768, I_BYTES = 784;
    // walk slot, epilogue -> walker: column masks[128] x 4 u32, ids[128], order[128] u8, c, v
    static constexpr int W_MASK = W_MASK_OFF, W_IDS = W_IDS_OFF, W_ORDER = W_ORDER_OFF, W_MISC = W_MISC_OFF,
                         W_BYTES = W_SLOT_BYTES;
    static constexpr int OFF_A0 = 0;
    static constexpr int OFF_INFO = OFF_A0 + A * KB * REGION;
    static constexpr int OFF_WS = OFF_INFO + I * I_BYTES;
    // per group, two node buffers of: D(x, z_r) u32[128], n_r / 2 float[128]
    static constexpr int OFF_DX = OFF_WS + W * W_BYTES;
    static constexpr int OFF_BAR = OFF_DX + PT_GROUPS * 2 * 1024;
    static constexpr int BAR_FULL_A = 0, BAR_EMPTY_A = A, BAR_CFULL = 2 * A, BAR_IEMPTY = 2 * A + I,
                         BAR_TFULL = 2 * A + 2 * I, BAR_TEMPTY = 2 * A + 2 * I + T,
                         BAR_WFULL = 2 * A + 2 * I + 2 * T, BAR_WEMPTY = 2 * A + 2 * I + 2 * T + W,
                         NBAR = 2 * A + 2 * I + 2 * T + 2 * W;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;     // tmem base, abort flag
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr int SMEM = BYTES + 1024;
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(T * 128 <= (int)TMEM_COLS, "TMEM budget");
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
            mbar_init(bar(C::BAR_FULL_A + i), 32);  // the gather warp
            mbar_init(bar(C::BAR_EMPTY_A + i), 1);
        }
        for (int i = 0; i < C::I; i++) {
            mbar_init(bar(C::BAR_CFULL + i), 32);
            mbar_init(bar(C::BAR_IEMPTY + i), 128);
        }
        for (int i = 0; i < C::T; i++) {
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
    if (warp == PT_MMA_WARP) tmem_alloc(sbase + C::OFF_MISC, TMEM_COLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == PT_INFO_WARP) {
        // ------------------------------------------------------------ node info (one warp)
        // Software pipeline: the reservoir row, count and node norm of node j + 2 are requested
        // while node j is compacted, so their latency is hidden behind two nodes of work.
        struct Pre {
            uint64_t key[4];
            int32_t nv;
            uint32_t c;
        };
        auto load = [&](uint64_t v, Pre &p) {
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
        Pre p0, p1;
        load(blockIdx.x, p0);
        load(blockIdx.x + (uint64_t)gridDim.x, p1);
        for (uint32_t j = 0;; j++) {
            const uint64_t v = blockIdx.x + (uint64_t)j * gridDim.x;
            if (v >= n) break;
            const uint32_t ib = j % C::I;
            Pre p2;
            load(v + 2 * (uint64_t)gridDim.x, p2);
            const uint32_t c = p0.c;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_IEMPTY + ib), ((j / C::I) & 1) ^ 1, abort, a.err)))
                break;
            unsigned char *in = info(ib);
            uint32_t *ids = reinterpret_cast<uint32_t *>(in + C::I_IDS);
            uint16_t *bkey = reinterpret_cast<uint16_t *>(in + C::I_BKEY);
            uint32_t cc = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t s = 32 * k + lane;
                const uint32_t id = (uint32_t)(p0.key[k] >> 16);
                const bool in_range = s < c && (uint64_t)id < n;
                if (s < c && !in_range) atomicOr(a.err, DERR_RANGE);
                const unsigned m = __ballot_sync(0xffffffffu, in_range);
                if (in_range) {
                    const uint32_t pos = cc + __popc(m & ((1u << lane) - 1u));
                    ids[pos] = id;
                    bkey[pos] = (uint16_t)(p0.key[k] >> 48);
                }
                cc += __popc(m);
            }
            if (lane == 0) {
                ids[cc] = (uint32_t)v;
                uint32_t *misc = reinterpret_cast<uint32_t *>(in + C::I_MISC);
                misc[0] = cc;
                misc[1] = (uint32_t)v;
                misc[2] = (uint32_t)p0.nv;
            }
            __syncwarp();
            mbar_arrive(bar(C::BAR_CFULL + ib));
            p0 = p1;
            p1 = p2;
        }
    } else if (warp == PT_MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t issued_j = 0;
            bool any = false, stop = false;
            for (uint32_t j = 0;; j++) {
                const uint64_t v = blockIdx.x + (uint64_t)j * gridDim.x;
                if (v >= n) break;
                const uint32_t ua = j % C::A, tb = j % C::T, ib = j % C::I;
                if (!mbar_wait(bar(C::BAR_CFULL + ib), (j / C::I) & 1, abort, a.err) ||
                    !mbar_wait(bar(C::BAR_FULL_A + ua), (j / C::A) & 1, abort, a.err) ||
                    !mbar_wait(bar(C::BAR_TEMPTY + tb), ((j / C::T) & 1) ^ 1, abort, a.err)) {
                    stop = true;
                    break;
                }
                fence_after();
                const uint32_t rows = reinterpret_cast<const uint32_t *>(info(ib) + C::I_MISC)[0] + 1;
                const uint32_t idesc = idesc_bf16(128, (rows + 15) & ~15u);
                const uint32_t aB = sbase + C::OFF_A0 + ua * KB * REGION;
                const uint32_t d = tmem + tb * 128;
#pragma unroll
                for (int kk = 0; kk < KB * 4; kk++) {
                    const uint64_t desc = smem_desc_sw128(aB + (kk >> 2) * REGION + (kk & 3) * 32);
                    mma_bf16(d, desc, desc, idesc, kk > 0 ? 1u : 0u);
                }
                mma_commit(bar(C::BAR_EMPTY_A + ua));
                mma_commit(bar(C::BAR_TFULL + tb));
                any = true;
                issued_j = j;
            }
            if (stop && any)
                mbar_wait(bar(C::BAR_TFULL + issued_j % C::T), (issued_j / C::T) & 1, abort, a.err);
        }
        __syncwarp();
    } else if (warp < PT_EPI_WARPS) {
        // ------------------------------------------------------------ epilogue (groups of 4 warps)
        const uint32_t grp = warp >> 2;                 // group: nodes j = grp, grp + PT_GROUPS, ...
        const int quarter = warp & 3;                   // TMEM lane quarter this warp may access
        const uint32_t r = quarter * 32 + lane;         // row = candidate slot
        const uint32_t bar_id = 1 + grp;
        bool stop = false;
        for (uint32_t k = 0;; k++) {
            const uint32_t j = grp + k * PT_GROUPS;
            const uint64_t vv = blockIdx.x + (uint64_t)j * gridDim.x;
            if (vv >= n) break;
            const uint32_t tb = j % C::T, ws = j % C::W, ib = j % C::I;
            const bool ok = !stop && __all_sync(0xffffffffu,
                                                 mbar_wait(bar(C::BAR_TFULL + tb), (j / C::T) & 1, abort, a.err) &&
                                                     mbar_wait(bar(C::BAR_CFULL + ib), (j / C::I) & 1, abort, a.err) &&
                                                     mbar_wait(bar(C::BAR_WEMPTY + ws), ((j / C::W) & 1) ^ 1, abort,
                                                               a.err));
            const unsigned char *in = info(ib);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(in + C::I_IDS);
            const uint16_t *bkey = reinterpret_cast<const uint16_t *>(in + C::I_BKEY);
            uint32_t *dx = reinterpret_cast<uint32_t *>(smem + C::OFF_DX + (grp * 2 + (k & 1)) * 1024);
            float *hn = reinterpret_cast<float *>(dx + 128);
            unsigned char *wsl = wslot(ws);
            uint32_t c = 0, DX = 0;
            float theta = 0.0f;
            bool bad = false;
            if (ok) {
                fence_after();
                c = reinterpret_cast<const uint32_t *>(in + C::I_MISC)[0];
                const float nx = (float)reinterpret_cast<const int32_t *>(in + C::I_MISC)[2];
                // E1: n_r from the diagonal (column r lies in chunk `quarter`), D(x, z_r) from
                // column c, the removal threshold of z_r
                const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + tb * 128;
                uint32_t g[32];
                tmem_ld32(trow + quarter * 32, g);
                const float nr = __uint_as_float(pick32(g, lane));  // exact integer < 2^23
                hn[r] = 0.5f * nr;
                tmem_ld32(trow + (c & ~31u), g);
                if (r < c) {
                    const float gx = __uint_as_float(pick32(g, c & 31u));
                    const float dxf = __fmaf_rn(-2.0f, gx, nr + nx);    // exact integer < 2^24
                    DX = (uint32_t)dxf;
                    const uint32_t T = removal_threshold(DX, a.alpha2, a.inv_alpha2);
                    theta = (nr - (float)T) * 0.5f;                    // exact (multiple of 1/2)
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
                mbar_arrive(bar(C::BAR_IEMPTY + ib));  // node info no longer read
                // E3: column mask of z_r -- the candidates y with G[r][y] - n_y / 2 > theta_r
                // (both sides multiples of 1/2 below 2^23: exact)
                uint32_t mw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    if (q * 32 < c) {
                        uint32_t g[32];
                        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + tb * 128 + q * 32, g);
                        const float4 *h4 = reinterpret_cast<const float4 *>(hn + q * 32);
                        uint32_t m = 0;
#pragma unroll
                        for (int j4 = 0; j4 < 8; j4++) {
                            const float4 h = h4[j4];
                            m |= __fsub_rn(__uint_as_float(g[4 * j4 + 0]), h.x) > theta ? (1u << (4 * j4 + 0)) : 0u;
                            m |= __fsub_rn(__uint_as_float(g[4 * j4 + 1]), h.y) > theta ? (1u << (4 * j4 + 1)) : 0u;
                            m |= __fsub_rn(__uint_as_float(g[4 * j4 + 2]), h.z) > theta ? (1u << (4 * j4 + 2)) : 0u;
                            m |= __fsub_rn(__uint_as_float(g[4 * j4 + 3]), h.w) > theta ? (1u << (4 * j4 + 3)) : 0u;
                        }
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
    } else if (walker_of(warp) >= 0) {
        // ------------------------------------------------------------ walkers
        // Walker w takes nodes j = w, w + PT_WALKERS, ... and alternates between its two walk slots
        // (w and w + PT_WALKERS).  Per block of 32 ranks the lanes drop, with one vote, every
        // candidate removed by an earlier admission; then each admission (the first remaining
        // lane) removes, with one vote, the later lanes whose column mask holds it.
        const uint32_t w = walker_of(warp);
        const uint32_t R = a.R;
        for (uint32_t k = 0;; k++) {
            const uint32_t j = w + k * PT_WALKERS;
            if (blockIdx.x + (uint64_t)j * gridDim.x >= n) break;
            const uint32_t sl = j % C::W;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_WFULL + sl), (j / C::W) & 1, abort, a.err))) break;
            const unsigned char *wsl = wslot(sl);
            const uint32_t c = reinterpret_cast<const uint32_t *>(wsl + C::W_MISC)[0];
            const uint64_t v = reinterpret_cast<const uint32_t *>(wsl + C::W_MISC)[1];
            const uint4 *mask = reinterpret_cast<const uint4 *>(wsl + C::W_MASK);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(wsl + C::W_IDS);
            const unsigned char *order = wsl + C::W_ORDER;
            uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0;  // admitted slots
            uint32_t e = 0;
            uint32_t out[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
            for (uint32_t b = 0; b * 32 < c && e < R; b++) {
                const uint32_t i = b * 32 + lane;
                const bool valid = i < c;
                const uint32_t tl = valid ? order[i] : 0u;
                const uint4 cm = valid ? mask[tl] : make_uint4(0, 0, 0, 0);
                unsigned U = __ballot_sync(0xffffffffu,
                                           valid && ((cm.x & A0) | (cm.y & A1) | (cm.z & A2) | (cm.w & A3)) == 0u);
                while (U != 0u && e < R) {
                    const uint32_t u = __ffs(U) - 1;
                    const uint32_t t = __shfl_sync(0xffffffffu, tl, u);
                    const uint32_t wd = t >> 5, bit = 1u << (t & 31);
                    A0 |= wd == 0 ? bit : 0u;
                    A1 |= wd == 1 ? bit : 0u;
                    A2 |= wd == 2 ? bit : 0u;
                    A3 |= wd == 3 ? bit : 0u;
                    const uint32_t id = ids[t];
                    const uint32_t o = e >> 5;
                    const bool mine = (e & 31) == (uint32_t)lane;
                    out[0] = (mine && o == 0) ? id : out[0];
                    out[1] = (mine && o == 1) ? id : out[1];
                    out[2] = (mine && o == 2) ? id : out[2];
                    out[3] = (mine && o == 3) ? id : out[3];
                    e++;
                    const uint32_t mw = wd == 0 ? cm.x : wd == 1 ? cm.y : wd == 2 ? cm.z : cm.w;
                    U &= ~__ballot_sync(0xffffffffu, (mw >> (t & 31)) & 1u) & ~(1u << u);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t p = lane + 32 * q;
                if (p < R) a.adj[v * R + p] = p < e ? out[q] : 0xFFFFFFFFu;
            }
            if (lane == 0) a.deg[v] = e;
            __syncwarp();
            mbar_arrive(bar(C::BAR_WEMPTY + sl));
        }
    } else if (gatherer_of(warp) >= 0) {
        // ------------------------------------------------------------ row gathers (two warps)
        for (uint32_t j = gatherer_of(warp);; j += PT_GATHERERS) {
            const uint64_t v = blockIdx.x + (uint64_t)j * gridDim.x;
            if (v >= n) break;
            const uint32_t ua = j % C::A, ib = j % C::I;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_CFULL + ib), (j / C::I) & 1, abort, a.err) &&
                                             mbar_wait(bar(C::BAR_EMPTY_A + ua), ((j / C::A) & 1) ^ 1, abort,
                                                       a.err)))
                break;
            const unsigned char *in = info(ib);
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
    if (warp == PT_MMA_WARP) {
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
