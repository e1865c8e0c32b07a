// leaf_tc.cu -- A2..A4 on the 5th-generation tensor cores (tcgen05 + TMEM), byte data.
//
// For every leaf b and every 128-row tile of it, the kernel forms, for all |b| members j,
//     -D_ij / 2 = <x_i, x_j> - n_i / 2 - n_j / 2      (D = squared L2, n = squared norm)
// directly in the tensor-core accumulator, and keeps per row the k nearest other members by
// (D, id) (Sec. 4.2: the all-pairs distance matrix of a leaf; App. A.3: bi-directed k-NN pick).
// The distance matrix never leaves TMEM / registers.
//
// The MMA operands come from one leaf-ordered BF16 copy of the members' rows, extended by one
// K = 16 norm step: A_i = [x_i | 1,1,1,1, -a1,-a2,-a3,-ha] and B_j = [x_j | -b1,-b2,-b3,-hb, 1,1,1,1]
// where n / 2 = p1 + p2 + p3 + h is split into byte-wide pieces and h = (n mod 2) / 2 (the B row's
// pieces b, the A row's a).  Exactness: u8 / i8 values and the pieces are exact in BF16, every
// product is an integer or a half, and for d <= 128 every partial sum is a multiple of 1/2 below
// 2^23 in magnitude, so FP32 accumulation in any order is exact and the picks equal those of the
// defining integer arithmetic.
//
// Persistent CTA (one per SM, 10 warps) over units (leaf, 128-row tile):
//   warp 0     producer: TMA tiled loads (128 rows x 64 columns, 128-byte swizzle) of the A and B
//              tiles from the leaf-ordered copy; both also get their norm pieces (a 32-byte slice
//              per buffer / stage) and B tiles a column-id list
//   warp 1     owns TMEM; one thread issues tcgen05.mma M=128, N<=128, K=16 steps into one of four
//              accumulator buffers and commits to the stage / accumulator barriers
//   warps 2-9  epilogue: tcgen05.ld 32 columns at a time, two smallest per row (k <= 2; the next
//              chunk's load always in flight) or exact (D, id) insertion (k > 2); two warps share
//              each TMEM lane quarter
// Every mbarrier wait is bounded by %globaltimer (2 s); on expiry the CTA records DERR_TIMEOUT,
// every role stops at the same points, and the TMEM is still released.
#include "tc_common.cuh"

namespace pipnn {

namespace {

using namespace tc;

// ------------------------------------------------------------------ kernel
struct TcUnit {
    uint64_t off;   // first member of the leaf
    uint64_t out;   // first output slot of the tile's first row
    uint32_t s;     // leaf size
    uint32_t row0;  // first row of the tile
};

struct TcArgs {
    const TcUnit *units;
    const uint32_t *members;     // leaf members, ascending ids inside every 128-member tile
    const uint2 *member_pieces;  // -(n / 2) of every leaf member as four BF16 pieces
    uint32_t k;
    uint32_t *out_dst, *out_src;
    float *out_dist;
    unsigned *err;
};

template <int KB, int KMAX>
struct TcCfg {
    static constexpr int NMAX = 128;                                     // columns per B tile
    static constexpr int S = 3;                                          // B stages
    static constexpr int T = 4;                                          // accumulator buffers
    static constexpr int REGION = tc::REGION;
    static constexpr int OFF_A0 = 0;                                     // A data, 2 buffers
    static constexpr int OFF_AN = OFF_A0 + 2 * KB * REGION;              // A norm blocks (a 32-byte slice per buffer)
    static constexpr int OFF_B0 = OFF_AN + REGION;                       // B data, S stages
    static constexpr int OFF_BN = OFF_B0 + S * KB * REGION;              // B norm blocks (32-byte slice per stage)
    static constexpr int OFF_CI = OFF_BN + REGION;                       // T x NMAX column ids
    static constexpr int MVBUF = KMAX == 2 ? 2 : 1;                      // k <= 2: one per unit parity
    static constexpr int OFF_MV = OFF_CI + T * NMAX * 4;                 // MVBUF x 128 rows x KMAX (D, id)
    static constexpr int OFF_BAR = OFF_MV + MVBUF * ROWS * KMAX * 8;
    static constexpr int BAR_FULL_A = 0, BAR_EMPTY_A = 2, BAR_FULL = 4, BAR_EMPTY = BAR_FULL + S,
                         BAR_TFULL = BAR_EMPTY + S, BAR_TEMPTY = BAR_TFULL + T, BAR_CFULL = BAR_TEMPTY + T,
                         NBAR = BAR_CFULL + T;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;                  // tmem base, abort flag
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr int SMEM = BYTES + 1024;                            // + alignment slack
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(T * NMAX <= (int)TMEM_COLS, "TMEM budget");
    static_assert(S <= 4, "norm slices per 128-byte row");
};

template <int KMAX>
__device__ __forceinline__ void topk_insert(float (&kv)[KMAX], uint32_t (&ki)[KMAX], float v, uint32_t id) {
    if (v > kv[KMAX - 1] || (v == kv[KMAX - 1] && id >= ki[KMAX - 1])) return;
    kv[KMAX - 1] = v;
    ki[KMAX - 1] = id;
#pragma unroll
    for (int p = KMAX - 1; p > 0; p--) {
        const bool sw = kv[p] < kv[p - 1] || (kv[p] == kv[p - 1] && ki[p] < ki[p - 1]);
        const float tv = kv[p - 1];
        const uint32_t ti = ki[p - 1];
        kv[p - 1] = sw ? kv[p] : tv;
        ki[p - 1] = sw ? ki[p] : ti;
        kv[p] = sw ? tv : kv[p];
        ki[p] = sw ? ti : ki[p];
    }
}

// Persistent: CTA b processes units b, b + grid, ...; every role walks the same unit sequence.
// B job j (one 128-column tile) uses B stage j % S (phase (j / S) % 2) and accumulator buffer /
// column-id slot j % T (phase (j / T) % 2); unit i uses A buffer i % 2 (phase (i / 2) % 2).
template <int KB, int KMAX>
__global__ void __launch_bounds__(THREADS, 1)
    leaf_gram_tc(const __grid_constant__ CUtensorMap map, const TcArgs a, uint32_t nunits) {
    using C = TcCfg<KB, KMAX>;
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    uint32_t *colid = reinterpret_cast<uint32_t *>(smem + C::OFF_CI);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + C::OFF_MISC);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + C::OFF_MISC + 4);
    auto bar = [&](int i) { return sbase + C::OFF_BAR + 8 * i; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) {
            mbar_init(bar(C::BAR_FULL_A + i), 32);
            mbar_init(bar(C::BAR_EMPTY_A + i), 1);
        }
        for (int i = 0; i < C::S; i++) {
            mbar_init(bar(C::BAR_FULL + i), 32);
            mbar_init(bar(C::BAR_EMPTY + i), 1);
        }
        for (int i = 0; i < C::T; i++) {
            mbar_init(bar(C::BAR_TFULL + i), 1);
            mbar_init(bar(C::BAR_TEMPTY + i), EPI_WARPS * 32);
            mbar_init(bar(C::BAR_CFULL + i), 32);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == MMA_WARP) {
        tmem_alloc(sbase + C::OFF_MISC, TMEM_COLS);
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == PRODUCER_WARP) {
        // ------------------------------------------------------------ producer (one warp)
        // norm slices (K = 16 BF16 = 32 bytes = logical chunks 2 x, 2 x + 1 of a 128-byte row):
        // A buffer x: [1,1,1,1, a-pieces, 0 x 8], B stage x: [b-pieces, 1,1,1,1, 0 x 8]; the A and B
        // jobs rewrite only the pieces
        for (uint32_t r = lane; r < (uint32_t)ROWS; r += 32) {
            const uint32_t one2 = 0x3F803F80u;  // two bf16 1.0
            for (uint32_t q = 0; q < 4; q++) {
                const bool lo = (q & 1) == 0;
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(sbase + C::OFF_AN + r * 128 +
                                                                              ((q ^ (r & 7)) << 4)),
                             "r"(lo ? one2 : 0u), "r"(lo ? one2 : 0u), "r"(0u), "r"(0u)
                             : "memory");
            }
            for (uint32_t q = 0; q < 2u * C::S; q++) {
                const bool lo = (q & 1) == 0;
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(sbase + C::OFF_BN + r * 128 +
                                                                              ((q ^ (r & 7)) << 4)),
                             "r"(0u), "r"(0u), "r"(lo ? one2 : 0u), "r"(lo ? one2 : 0u)
                             : "memory");
            }
        }
        fence_proxy_async();
        // job stream: per unit one A job, then one B job per 128-column tile.  The member ids
        // and norms of the next B job are loaded while the current one is issued.
        struct Job {
            uint32_t kind;  // 0 A, 1 B, 2 end
            uint32_t i, u, t, s, first;
            uint64_t off;
        };
        auto unit_job = [&](uint32_t i, uint32_t u) {
            Job q;
            if (u >= nunits) {
                q.kind = 2;
                return q;
            }
            const TcUnit un = a.units[u];
            q.kind = 0;
            q.i = i;
            q.u = u;
            q.t = 0;
            q.s = un.s;
            q.first = un.row0;
            q.off = un.off;
            return q;
        };
        auto next_job = [&](const Job &c) {
            Job q = c;
            if (c.kind == 0) {
                q.kind = 1;
                q.t = 0;
                q.first = 0;
                return q;
            }
            const uint32_t nct = (c.s + C::NMAX - 1) / C::NMAX;
            if (c.t + 1 < nct) {
                q.t = c.t + 1;
                q.first = q.t * C::NMAX;
                return q;
            }
            return unit_job(c.i + 1, c.u + gridDim.x);
        };
        // an A job's rows need their norm pieces, a B job's columns pieces and ids
        auto load_ids = [&](const Job &q, uint32_t (&id)[4], uint2 (&nr)[4]) {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t r = q.first + 4 * lane + e;
                const bool in = q.kind <= 1 && r < q.s;
                id[e] = (in && q.kind == 1) ? a.members[q.off + r] : 0u;
                nr[e] = in ? a.member_pieces[q.off + r] : make_uint2(0u, 0u);
            }
        };
        Job cur = unit_job(0, blockIdx.x);
        uint32_t id[4];
        uint2 nr[4];
        load_ids(cur, id, nr);
        uint32_t j = 0;
        while (cur.kind != 2) {
            const Job nxt = next_job(cur);
            uint32_t nid[4];
            uint2 nnr[4];
            bool ok;
            if (cur.kind == 0) {
                const uint32_t ua = cur.i & 1;
                ok = mbar_wait(bar(C::BAR_EMPTY_A + ua), ((cur.i >> 1) & 1) ^ 1, abort, a.err);
                // the next job's ids and norm pieces: requested here, consumed next iteration
                load_ids(nxt, nid, nnr);
                if (ok) {
                    // -(n_i / 2) of the tile's rows (zero past the leaf): bytes 8..15 of logical
                    // chunk 2 ua
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const uint32_t r = 4 * lane + e;
                        asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(sbase + C::OFF_AN + r * 128 +
                                                                             (((2 * ua) ^ (r & 7)) << 4) + 8),
                                     "r"(nr[e].x), "r"(nr[e].y)
                                     : "memory");
                    }
                    fence_proxy_async();
                    const uint32_t fb = bar(C::BAR_FULL_A + ua);
                    if (lane == 0) {
                        mbar_arrive_tx(fb, KB * C::REGION);
                        const uint32_t dst = sbase + C::OFF_A0 + ua * KB * C::REGION;
#pragma unroll
                        for (int kb = 0; kb < KB; kb++)
                            tma_load_tile(dst + kb * C::REGION, &map, kb * 64, (int32_t)(cur.off + cur.first), fb);
                    } else {
                        mbar_arrive(fb);
                    }
                }
            } else {
                const uint32_t st = j % C::S, tb = j % C::T;
                ok = mbar_wait(bar(C::BAR_EMPTY + st), ((j / C::S) & 1) ^ 1, abort, a.err) &&
                     mbar_wait(bar(C::BAR_TEMPTY + tb), ((j / C::T) & 1) ^ 1, abort, a.err);
                if (ok) {
                    uint32_t *ci = colid + tb * C::NMAX;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const uint32_t r = 4 * lane + e;
                        ci[r] = cur.first + r < cur.s ? id[e] : 0xFFFFFFFFu;
                        // -(n_j / 2) as four BF16-exact pieces (zero past the leaf) in the first 8
                        // bytes of this stage's 32-byte slice (logical chunk 2 st)
                        asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(sbase + C::OFF_BN + r * 128 +
                                                                             (((2 * st) ^ (r & 7)) << 4)),
                                     "r"(nr[e].x), "r"(nr[e].y)
                                     : "memory");
                    }
                    fence_proxy_async();
                    mbar_arrive(bar(C::BAR_CFULL + tb));
                }
                // requested after the proxy fence, which would otherwise wait for them
                load_ids(nxt, nid, nnr);
                if (ok) {
                    const uint32_t fb = bar(C::BAR_FULL + st);
                    if (lane == 0) {
                        mbar_arrive_tx(fb, KB * C::REGION);
                        const uint32_t dst = sbase + C::OFF_B0 + st * KB * C::REGION;
#pragma unroll
                        for (int kb = 0; kb < KB; kb++)
                            tma_load_tile(dst + kb * C::REGION, &map, kb * 64, (int32_t)(cur.off + cur.first), fb);
                    } else {
                        mbar_arrive(fb);
                    }
                }
                j++;
            }
            if (!__all_sync(0xffffffffu, ok)) break;
            cur = nxt;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                id[e] = nid[e];
                nr[e] = nnr[e];
            }
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t j = 0, issued_j = 0;
            bool any = false, stop = false;
            for (uint32_t i = 0, u = blockIdx.x; u < nunits && !stop; i++, u += gridDim.x) {
                const uint32_t s = a.units[u].s;
                const uint32_t ua = i & 1;
                if (!mbar_wait(bar(C::BAR_FULL_A + ua), (i >> 1) & 1, abort, a.err)) break;
                const uint32_t aB = sbase + C::OFF_A0 + ua * KB * C::REGION;
                const uint32_t nct = (s + C::NMAX - 1) / C::NMAX;
                for (uint32_t t = 0; t < nct; t++, j++) {
                    const uint32_t st = j % C::S, tb = j % C::T;
                    if (!mbar_wait(bar(C::BAR_FULL + st), (j / C::S) & 1, abort, a.err) ||
                        !mbar_wait(bar(C::BAR_TEMPTY + tb), ((j / C::T) & 1) ^ 1, abort, a.err)) {
                        stop = true;
                        break;
                    }
                    fence_after();
                    const uint32_t c0 = t * C::NMAX;
                    const uint32_t ncols = s - c0 < (uint32_t)C::NMAX ? s - c0 : C::NMAX;
                    const uint32_t idesc = idesc_bf16(128, (ncols + 15) & ~15u);
                    const uint32_t bB = sbase + C::OFF_B0 + st * KB * C::REGION;
                    const uint32_t d = tmem + tb * C::NMAX;
#pragma unroll
                    for (int kk = 0; kk < KB * 4; kk++) {
                        const uint64_t ad = smem_desc_sw128(aB + (kk >> 2) * C::REGION + (kk & 3) * 32);
                        const uint64_t bd = smem_desc_sw128(bB + (kk >> 2) * C::REGION + (kk & 3) * 32);
                        mma_bf16(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    // - n_i / 2 - n_j / 2: the norm slices of this A buffer and this B stage
                    mma_bf16(d, smem_desc_sw128(sbase + C::OFF_AN + ua * 32),
                             smem_desc_sw128(sbase + C::OFF_BN + st * 32), idesc, 1u);
                    mma_commit(bar(C::BAR_EMPTY + st));
                    mma_commit(bar(C::BAR_TFULL + tb));
                    any = true;
                    issued_j = j;
                }
                if (!stop) mma_commit(bar(C::BAR_EMPTY_A + ua));
            }
            // after an early stop, let the issued MMAs drain before TMEM is released
            if (stop && any)
                mbar_wait(bar(C::BAR_TFULL + issued_j % C::T), (issued_j / C::T) & 1, abort, a.err);
        }
        __syncwarp();
    } else if constexpr (KMAX == 2) {
        // ------------------------------------------------------------ epilogue, k <= 2
        // D_ij = -2 acc is an integer below 2^23 (d <= 128 bytes), so fma(-2, acc, 2^23) = D + 2^23
        // exactly and its bit pattern is 0x4B000000 + D: times 128 plus the column in the tile it is
        // a 32-bit key ordered by (D, column), i.e. by (D, id) -- every 128-member tile of a leaf is
        // in ascending id order.  Two smallest per chain: k2 = min(k2, max(k1, key)), k1 = min(k1, key).  Warp
        // (quarter, half) takes chunks half and half + 2 of every tile; one chunk's TMEM load is
        // always in flight while the other is ranked, across tiles and units.
        const int ew = warp - EPI_WARP0;
        const int half = ew >> 2;
        const int quarter = warp & 3;
        const uint32_t r = quarter * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
        uint64_t *mv = reinterpret_cast<uint64_t *>(smem + C::OFF_MV);
        // warp-uniform: tcgen05.ld is a warp-collective instruction
        auto open_tile = [&](uint32_t jj) {
            const uint32_t tb = jj % C::T, ph = (jj / C::T) & 1;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_TFULL + tb), ph, abort, a.err) &&
                                                        mbar_wait(bar(C::BAR_CFULL + tb), ph, abort, a.err));
            fence_after();
            return ok;
        };
        // two smallest keys of chunk q (columns base .. base + 31 of the leaf) folded into T1 <= T2
        auto rank_chunk = [&](uint32_t (&g)[32], uint32_t q, uint32_t base, uint32_t s, uint32_t self_col,
                              uint32_t &T1, uint32_t &T2) {
            uint32_t key[32];
#pragma unroll
            for (int jj = 0; jj < 32; jj++)
                key[jj] = __float_as_uint(__fmaf_rn(-2.0f, __uint_as_float(g[jj]), 8388608.0f)) * 128u +
                          (q * 32 + jj);
            // the row's own column and columns past the leaf never qualify (both tests are uniform
            // over the warp: a warp's rows are 32 consecutive columns)
            if (self_col - base < 32u || base + 32 > s) {
#pragma unroll
                for (int jj = 0; jj < 32; jj++)
                    if (base + jj == self_col || base + jj >= s) key[jj] = ~0u;
            }
            uint32_t k1[4], k2[4];
#pragma unroll
            for (int ch = 0; ch < 4; ch++) {
                k1[ch] = key[ch];
                k2[ch] = ~0u;
            }
#pragma unroll
            for (int jj = 4; jj < 32; jj++) {
                const int ch = jj & 3;
                k2[ch] = min(k2[ch], max(k1[ch], key[jj]));
                k1[ch] = min(k1[ch], key[jj]);
            }
#pragma unroll
            for (int ch = 0; ch < 4; ch++) {
                const uint32_t m2 = min(max(T1, k1[ch]), min(T2, k2[ch]));
                T1 = min(T1, k1[ch]);
                T2 = m2;
            }
        };
        uint32_t u = blockIdx.x, i = 0, j = 0, t = 0;
        TcUnit un = a.units[u];
        TcUnit unx = a.units[u + gridDim.x < nunits ? u + gridDim.x : u];
        uint32_t my_id = un.row0 + r < un.s ? a.members[un.off + un.row0 + r] : 0xFFFFFFFFu;
        uint64_t RK1 = ~0ull, RK2 = ~0ull;  // running two smallest (D << 32 | id) of this half
        uint32_t gA[32], gB[32];
#pragma unroll
        for (int jj = 0; jj < 32; jj++) gA[jj] = gB[jj] = 0u;
        bool failed = !open_tile(0);
        bool cur_ok = !failed;  // tile j is open (its accumulator and column ids are ready)
        if (!failed && half * 32 < (un.s < (uint32_t)C::NMAX ? un.s : (uint32_t)C::NMAX))
            tmem_ld32_async(tq + half * 32, gA);
        for (;;) {
            const uint32_t tb = j % C::T;
            const uint32_t c0 = t * C::NMAX;
            const uint32_t ncols = un.s - c0 < (uint32_t)C::NMAX ? un.s - c0 : C::NMAX;
            const uint32_t nct = (un.s + C::NMAX - 1) / C::NMAX;
            const uint32_t self_col = un.row0 + r;
            const bool v0 = cur_ok && half * 32 < ncols;
            const bool v1 = cur_ok && (half + 2) * 32 < ncols;
            tmem_wait_ld_regs(gA);
            if (v1) tmem_ld32_async(tq + tb * C::NMAX + (half + 2) * 32, gB);
            uint32_t T1 = ~0u, T2 = ~0u;
            if (v0) rank_chunk(gA, half, c0 + half * 32, un.s, self_col, T1, T2);
            tmem_wait_ld_regs(gB);
            // open the next tile -- the rest of this unit, else the next unit's first -- and start
            // its first chunk's load before ranking this tile's second chunk
            const bool last = t + 1 == nct;
            bool nxt_ok = false;
            if (!failed && (!last || u + gridDim.x < nunits)) {
                nxt_ok = open_tile(j + 1);
                failed = !nxt_ok;
                const uint32_t nrem = last ? unx.s : un.s - c0 - C::NMAX;
                if (nxt_ok && half * 32 < nrem) tmem_ld32_async(tq + ((j + 1) % C::T) * C::NMAX + half * 32, gA);
            }
            if (v1) rank_chunk(gB, half + 2, c0 + (half + 2) * 32, un.s, self_col, T1, T2);
            if (cur_ok) {
                // the tile's pair as (D << 32 | id), merged into the running pair
                const uint32_t *ci = colid + tb * C::NMAX;
                const uint64_t K1 =
                    T1 == ~0u ? ~0ull : ((uint64_t)((T1 & 0x7FFFFFFFu) >> 7) << 32) | ci[T1 & 127u];
                const uint64_t K2 =
                    T2 == ~0u ? ~0ull : ((uint64_t)((T2 & 0x7FFFFFFFu) >> 7) << 32) | ci[T2 & 127u];
                const uint64_t m2 = min(max(RK1, K1), min(RK2, K2));
                RK1 = min(RK1, K1);
                RK2 = m2;
                // the accumulator buffer and the column ids of tile j are free again
                fence_before();
                mbar_arrive(bar(C::BAR_TEMPTY + tb));
            }
            cur_ok = nxt_ok;
            j++;
            if (!last) {
                t++;
                continue;
            }
            // unit done: merge the two halves of each row (one buffer per unit parity, so the next
            // unit's writes cannot meet this unit's reads) and emit
            uint64_t *m = mv + ((i & 1) * ROWS + r) * 2;
            if (half == 1) {
                m[0] = RK1;
                m[1] = RK2;
            }
            failed = named_barrier_or(1, EPI_WARPS * 32, failed || *abort);
            if (half == 0 && un.row0 + r < un.s && !failed) {
                const uint64_t P1 = m[0], P2 = m[1];
                const uint64_t R2 = min(max(RK1, P1), min(RK2, P2));
                const uint64_t R1 = min(RK1, P1);
                const uint32_t kk = un.s - 1 < a.k ? un.s - 1 : a.k;
                uint64_t w = un.out + (uint64_t)r * 2 * kk;
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    if ((uint32_t)p < kk) {
                        const uint64_t R = p == 0 ? R1 : R2;
                        const bool none = R == ~0ull;
                        const uint32_t src = none ? my_id : (uint32_t)R;
                        const float D = none ? __int_as_float(0x7f800000) : (float)(uint32_t)(R >> 32);
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
            u += gridDim.x;
            i++;
            if (failed || u >= nunits) break;
            un = unx;
            unx = a.units[u + gridDim.x < nunits ? u + gridDim.x : u];
            my_id = un.row0 + r < un.s ? a.members[un.off + un.row0 + r] : 0xFFFFFFFFu;
            t = 0;
            RK1 = ~0ull;
            RK2 = ~0ull;
        }
        // a load started for a tile that a failure left unused completes before TMEM is released
        tmem_wait_ld();
    } else {
        // ------------------------------------------------------------ epilogue, k > 2
        const int ew = warp - EPI_WARP0;          // 0..7
        const int half = ew >> 2;                    // which column chunks
        const int quarter = warp & 3;                // TMEM lane quarter this warp may access
        const uint32_t r = quarter * 32 + lane;      // row inside the tile
        float2 *mv = reinterpret_cast<float2 *>(smem + C::OFF_MV);
        uint32_t j = 0;
        bool failed = false;
        for (uint32_t i = 0, u = blockIdx.x; u < nunits; i++, u += gridDim.x) {
            const TcUnit un = a.units[u];
            const uint64_t off = un.off;
            const uint32_t s = un.s, row0 = un.row0;
            const bool row_ok = row0 + r < s;
            const uint32_t my_id = row_ok ? a.members[off + row0 + r] : 0xFFFFFFFFu;
            float kv[KMAX];
            uint32_t ki[KMAX];
#pragma unroll
            for (int p = 0; p < KMAX; p++) {
                kv[p] = __int_as_float(0x7f800000);
                ki[p] = 0xFFFFFFFFu;
            }
            const uint32_t nct = (s + C::NMAX - 1) / C::NMAX;
            for (uint32_t t = 0; t < nct; t++, j++) {
                const uint32_t tb = j % C::T, ph = (j / C::T) & 1;
                if (failed) continue;
                // warp-uniform waits: tcgen05.ld below is a warp-collective instruction
                const bool ok = __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_TFULL + tb), ph, abort, a.err) &&
                                                            mbar_wait(bar(C::BAR_CFULL + tb), ph, abort, a.err));
                if (!ok) {
                    failed = true;
                    continue;
                }
                fence_after();
                const uint32_t c0 = t * C::NMAX;
                const uint32_t ncols = s - c0 < (uint32_t)C::NMAX ? s - c0 : C::NMAX;
                const uint32_t *info = colid + tb * C::NMAX;
                for (uint32_t q = half; q * 32 < ncols; q += 2) {
                    uint32_t gv[32];
                    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + tb * C::NMAX + q * 32, gv);
                    if (!row_ok) continue;
                    // the accumulator holds -D/2; rank by D/2 (same order, exact)
                    float v[32];
#pragma unroll
                    for (int jj = 0; jj < 32; jj++) v[jj] = -__uint_as_float(gv[jj]);
                    float m0 = fminf(fminf(v[0], v[1]), fminf(v[2], v[3]));
                    float m1 = fminf(fminf(v[4], v[5]), fminf(v[6], v[7]));
                    float m2 = fminf(fminf(v[8], v[9]), fminf(v[10], v[11]));
                    float m3 = fminf(fminf(v[12], v[13]), fminf(v[14], v[15]));
                    m0 = fminf(m0, fminf(fminf(v[16], v[17]), fminf(v[18], v[19])));
                    m1 = fminf(m1, fminf(fminf(v[20], v[21]), fminf(v[22], v[23])));
                    m2 = fminf(m2, fminf(fminf(v[24], v[25]), fminf(v[26], v[27])));
                    m3 = fminf(m3, fminf(fminf(v[28], v[29]), fminf(v[30], v[31])));
                    const float mn = fminf(fminf(m0, m1), fminf(m2, m3));
                    if (mn <= kv[KMAX - 1]) {
#pragma unroll
                        for (int jj = 0; jj < 32; jj++) {
                            if (v[jj] <= kv[KMAX - 1]) {
                                const uint32_t id = info[q * 32 + jj];
                                if (id != my_id && id != 0xFFFFFFFFu) topk_insert<KMAX>(kv, ki, v[jj], id);
                            }
                        }
                    }
                }
                fence_before();
                mbar_arrive(bar(C::BAR_TEMPTY + tb));
            }
            // merge the two halves of each row, then emit
            if (half == 1) {
#pragma unroll
                for (int p = 0; p < KMAX; p++) mv[r * KMAX + p] = make_float2(kv[p], __uint_as_float(ki[p]));
            }
            failed = named_barrier_or(1, EPI_WARPS * 32, failed || *abort);
            if (half == 0 && row_ok && !failed) {
#pragma unroll
                for (int p = 0; p < KMAX; p++) {
                    const float2 e = mv[r * KMAX + p];
                    const uint32_t id = __float_as_uint(e.y);
                    if (id != 0xFFFFFFFFu) topk_insert<KMAX>(kv, ki, e.x, id);
                }
                const uint32_t kk = s - 1 < a.k ? s - 1 : a.k;
                uint64_t w = un.out + (uint64_t)r * 2 * kk;
#pragma unroll
                for (int p = 0; p < KMAX; p++) {
                    if ((uint32_t)p < kk) {
                        const uint32_t src = ki[p] == 0xFFFFFFFFu ? my_id : ki[p];
                        const float D = __fmul_rn(2.0f, kv[p]);
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
            // mv is rewritten by the next unit only after every reader is done
            failed = named_barrier_or(1, EPI_WARPS * 32, failed || *abort);
            if (failed) break;
        }
    }

    fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

__global__ void build_units(const uint32_t *tile_grp, const uint32_t *tile_row0, uint64_t nunits,
                            const uint64_t *leaf_off, const uint64_t *cand_off, uint32_t k, TcUnit *units) {
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < nunits; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = tile_grp[u];
        TcUnit x;
        x.off = leaf_off[g];
        x.s = (uint32_t)(leaf_off[g + 1] - x.off);
        x.row0 = tile_row0[u];
        // row r of a leaf of s members writes 2 min(s - 1, k) slots from cand_off + r 2 min(s - 1, k)
        const uint32_t kk = x.s - 1 < k ? x.s - 1 : k;
        x.out = cand_off[g] + (uint64_t)x.row0 * 2 * kk;
        units[u] = x;
    }
}

// Ascending bitonic sort of 32 * E keys held E per lane (element E * lane + q in K[q]): exchanges
// within a lane for distances below E, shuffles across lanes for the rest.
template <int E>
__device__ __forceinline__ void warp_sort_u32(uint32_t (&K)[E], int lane) {
#pragma unroll
    for (uint32_t k = 2; k <= 32u * E; k <<= 1) {
#pragma unroll
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            if (j >= (uint32_t)E) {
#pragma unroll
                for (int q = 0; q < E; q++) {
                    const uint32_t i = E * lane + q;
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, K[q], j / E);
                    const bool take_min = ((i & j) == 0) == ((i & k) == 0);
                    K[q] = take_min ? min(o, K[q]) : max(o, K[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < E; q++) {
                    if ((q & j) == 0) {
                        const uint32_t i = E * lane + q;
                        const uint32_t lo = K[q], hi = K[q | j];
                        const bool up = (i & k) == 0;
                        K[q] = up ? min(lo, hi) : max(lo, hi);
                        K[q | j] = up ? max(lo, hi) : min(lo, hi);
                    }
                }
            }
        }
    }
}

// Sorts the members of every 128-member tile of every leaf ascending, one warp per tile in
// registers.  Column order inside a B tile is then id order, which is all the packed (D, column)
// keys of the k <= 2 epilogue need to break ties by id; across tiles (and halves) the epilogue
// compares (D, id) itself, and the general-k epilogue compares (D, id) throughout.
__global__ void __launch_bounds__(256) sort_tile_members(const uint32_t *tile_grp, const uint32_t *tile_row0,
                                                         uint64_t ntiles, const uint64_t *off, uint32_t *mem) {
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nw) {
        const uint32_t g = tile_grp[t], row0 = tile_row0[t];
        const uint64_t o = off[g] + row0;
        const uint64_t rest = off[g + 1] - o;
        const uint32_t nn = rest < (uint64_t)ROWS ? (uint32_t)rest : (uint32_t)ROWS;
        if (nn < 2) continue;
        uint32_t K[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = 4 * lane + q;
            K[q] = i < nn ? mem[o + i] : 0xFFFFFFFFu;
        }
        warp_sort_u32<4>(K, lane);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = 4 * lane + q;
            if (i < nn) mem[o + i] = K[q];
        }
    }
}

__global__ void member_pieces(const uint32_t *members, uint64_t M, const int32_t *sqnorm, uint2 *pieces) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < M; i += (uint64_t)gridDim.x * blockDim.x)
        pieces[i] = neg_half_norm_pieces((uint32_t)sqnorm[members[i]]);
}

template <int KB, int KMAX>
int launch_tc(const CUtensorMap &map, const TcArgs &args, uint64_t ntiles) {
    using C = TcCfg<KB, KMAX>;
    auto kern = leaf_gram_tc<KB, KMAX>;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int dev = 0, sms = 0;
    PIPNN_CUDA(cudaGetDevice(&dev));
    PIPNN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (uint64_t t0 = 0; t0 < ntiles; t0 += 0xFFFFFFFFull) {
        const uint64_t cnt = ntiles - t0 < 0xFFFFFFFFull ? ntiles - t0 : 0xFFFFFFFFull;
        TcArgs a = args;
        a.units += t0;
        const unsigned grid = (unsigned)(cnt < (uint64_t)sms ? cnt : (uint64_t)sms);
        kern<<<grid, THREADS, C::SMEM, stream()>>>(map, a, (uint32_t)cnt);
        PIPNN_LAUNCH_CHECK();
    }
    return PIPNN_OK;
}

template <int KB>
int launch_tc_k(const CUtensorMap &map, const TcArgs &args, uint64_t ntiles, uint32_t k) {
    if (k <= 2) return launch_tc<KB, 2>(map, args, ntiles);
    if (k <= 4) return launch_tc<KB, 4>(map, args, ntiles);
    if (k <= 8) return launch_tc<KB, 8>(map, args, ntiles);
    return launch_tc<KB, 16>(map, args, ntiles);
}

}  // namespace

int leaf_pick_tc(const void *X, uint64_t n, uint32_t d, int dtype, const int32_t *sqnorm, const uint64_t *off,
                 const uint32_t *mem, uint64_t L, const uint32_t *leaf_size, const uint64_t *cand_off, uint32_t k,
                 uint32_t *out_dst, uint32_t *out_src, float *out_dist, Workspace &ws, cudaEvent_t ev0,
                 cudaEvent_t ev1, uint32_t *launches) {
    if (dtype == PIPNN_F32) return set_error(PIPNN_EUNSUPPORTED, "the tensor-core leaf engine takes byte data only");
    if (d > 128) return set_error(PIPNN_EUNSUPPORTED, "the tensor-core leaf engine is exact for d <= 128");
    if (k > 16) return set_error(PIPNN_EINVAL, "k above 16");
    const uint32_t kb = (d + 63) / 64;
    const uint32_t kp = kb * 64;
    uint64_t M = 0;
    PIPNN_TRY(read_u64(off + L, &M));
    if (M >= 0x7FFFFF00ull) return set_error(PIPNN_EUNSUPPORTED, "the tensor-core leaf engine takes < 2^31 leaf members");
    uint32_t *tile_grp = nullptr, *tile_row0 = nullptr;
    uint64_t ntiles = 0;
    PIPNN_TRY(make_tiles(leaf_size, L, ROWS, &tile_grp, &tile_row0, &ntiles, ws));
    // a copy of the members with every 128-member tile of a leaf in ascending id order
    uint32_t *tile_members = nullptr;
    PIPNN_TRY(ws.alloc(&tile_members, M));
    uint2 *mpieces = nullptr;
    PIPNN_TRY(ws.alloc(&mpieces, M));
    if (M) {
        PIPNN_CUDA(cudaMemcpyAsync(tile_members, mem, M * 4, cudaMemcpyDeviceToDevice, stream()));
        sort_tile_members<<<grid_for(ntiles, 8, 152u * 32u), 256, 0, stream()>>>(tile_grp, tile_row0, ntiles, off,
                                                                                 tile_members);
        PIPNN_LAUNCH_CHECK();
        mem = tile_members;
        member_pieces<<<grid_for(M, 256), 256, 0, stream()>>>(mem, M, sqnorm, mpieces);
        PIPNN_LAUNCH_CHECK();
    }
    __nv_bfloat16 *staged = nullptr;
    PIPNN_TRY(ws.alloc(&staged, (M ? M : 1) * kp));
    if (M) {
        PIPNN_TRY(stage_rows_bf16(X, d, kp, dtype, mem, M, staged));
    }
    TcUnit *units = nullptr;
    PIPNN_TRY(ws.alloc(&units, ntiles));
    if (ntiles) {
        build_units<<<grid_for(ntiles, 256), 256, 0, stream()>>>(tile_grp, tile_row0, ntiles, off, cand_off, k,
                                                                 units);
        PIPNN_LAUNCH_CHECK();
    }
    CUtensorMap map;
    PIPNN_TRY(encode_rows_map(&map, staged, M ? M : 1, kp, false));
    TcArgs a{};
    a.units = units;
    a.members = mem;
    a.member_pieces = mpieces;
    a.k = k;
    a.out_dst = out_dst;
    a.out_src = out_src;
    a.out_dist = out_dist;
    a.err = device_error_word();
    *launches = 0;
    if (ntiles == 0) return PIPNN_OK;
    cudaEventRecord(ev0, stream());
    int rc;
    if (kb == 1) rc = launch_tc_k<1>(map, a, ntiles, k);
    else rc = launch_tc_k<2>(map, a, ntiles, k);
    cudaEventRecord(ev1, stream());
    *launches = 1;
    return rc;
}

}  // namespace pipnn
