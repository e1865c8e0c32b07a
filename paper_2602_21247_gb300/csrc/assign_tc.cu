// assign_tc.cu -- Alg. 5 leader assignment on the 5th-generation tensor cores (byte data, d <= 128).
//
// Every instance x of a subproblem joins its F nearest leaders l_0..l_{L-1} (L <= 1024), nearest by
// (D(x, l), rank) with D the squared L2 distance (equidistant leaders in draw order).  For a
// fixed instance D(x, l_c) = n_x - 2 w_c with
//     w_c = <x, l_c> - n_{l_c} / 2,
// so the F largest (w, -c) give the assignment.  w is formed in the accumulator by the same
// norm fold as the leaf engine: A_x = [x, 1,1,1,1] and B_c = [l_c, -pieces of n_{l_c} / 2], all
// exact in BF16, FP32 sums exact for d <= 128.
//
// Operands: A rows (instances, in subproblem order) are fetched with TMA tile::gather4 straight
// from a padded BF16 copy of all points made once per partition; B rows (the level's leaders, in
// rank order) come from a small per-level BF16 copy with tiled TMA loads.
//
// Persistent CTA (one per SM, 12 warps) over units (subproblem, 128-instance tile):
//   warp 0     producer: B tiles + the leaders' norm pieces
//   warps 10-11 A gathers, one warp per A buffer (each lane fetches four instance rows)
//   warp 1     owns TMEM (4 x 128 accumulator columns); one thread issues the MMAs
//   warps 2-9  epilogue: per row the F best (w, c) of its half of the columns, kept sorted in
//              registers; columns that beat the current F-th are collected as a bit mask and
//              inserted one by one, so a warp's work per 32 columns is set by its busiest row, not
//              by the union of all rows' candidates.  The two halves are merged in shared memory.
//              Bucket sizes are counted in a shared-memory histogram and flushed to global memory
//              once per run of units of the same subproblem.
// Waits are bounded like the leaf engine's (DERR_TIMEOUT, TMEM still released).
#include "tc_common.cuh"

#include <type_traits>

namespace pipnn {

namespace {

using namespace tc;

// warps: 0 producer (B tiles), 1 MMA, 2 .. 9 epilogue, 10 .. 11 A-row gathers (one per A buffer:
// a warp issues TMA gathers at a bounded rate, so two issuing warps double the rows in flight)
constexpr int AS_GATHER_WARP0 = EPI_WARP0 + EPI_WARPS;
constexpr int AS_THREADS = (AS_GATHER_WARP0 + 2) * 32;
constexpr uint32_t AS_HIST = 1024;            // leaders per subproblem (max_leaders is at most 1024)
constexpr uint32_t AS_SENT = 0xFFFFFFFEu;     // padding entry in front of the F live ones
constexpr uint32_t AS_NONE = 0xFFFFFFFFu;     // live entry not filled yet

struct AsUnit {
    uint64_t inst0;  // first instance of the subproblem
    uint64_t lead0;  // its rank-0 leader inside the level's leader rows
    uint32_t nrows;  // subproblem size
    uint32_t row0;   // first row of the tile
    uint32_t ncols;  // leader count
    uint32_t seg;    // subproblem index
};

struct AsArgs {
    const AsUnit *units;
    const uint32_t *inst;       // instance -> point id
    const int32_t *inst_norm;   // instance -> exact squared norm of its point
    const int32_t *lead_norm;   // exact squared norm of every leader row
    uint32_t fanout;            // F <= KMAX; stride of assign
    uint16_t *assign;           // instance -> F leader ranks
    uint32_t *bucket_cnt;       // (lead0 + rank) -> bucket size
    unsigned *err;
};

template <int KB, int KMAX>
struct AsCfg {
    static constexpr int NMAX = 128;                              // columns per B tile
    static constexpr int S = 3;                                   // B stages
    static constexpr int T = 4;                                   // accumulator buffers
    static constexpr int OFF_A0 = 0;                              // A data, 2 buffers
    static constexpr int OFF_AN = OFF_A0 + 2 * KB * REGION;       // A norm block (constant)
    static constexpr int OFF_B0 = OFF_AN + REGION;                // B data, S stages
    static constexpr int OFF_BN = OFF_B0 + S * KB * REGION;       // B norm pieces, a 32-byte slice per stage
    static constexpr int OFF_MV = OFF_BN + REGION;                // 128 rows x KMAX (w, c): half merge
    static constexpr int OFF_HIST = OFF_MV + ROWS * KMAX * 8;     // bucket histogram of the subproblem
    static constexpr int OFF_BAR = OFF_HIST + AS_HIST * 4;
    static constexpr int BAR_FULL_A = 0, BAR_EMPTY_A = 2, BAR_FULL = 4, BAR_EMPTY = BAR_FULL + S,
                         BAR_TFULL = BAR_EMPTY + S, BAR_TEMPTY = BAR_TFULL + T, NBAR = BAR_TEMPTY + T;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;           // tmem base, abort flag
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr int SMEM = BYTES + 1024;                     // + alignment slack
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(T * NMAX <= (int)TMEM_COLS, "TMEM budget");
    static_assert(S <= 4, "norm slices per 128-byte row");
};

// Register g[j] for a run-time j, by a five-level select tree (no local-memory indexing).
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

// Sorted ascending list of K keys: insert x, the largest drops out.  Branch free, every slot
// computed from the old list (depth two).
template <int K, typename T>
__device__ __forceinline__ void key_insert(T (&L)[K], T x) {
#pragma unroll
    for (int p = K - 1; p > 0; p--) L[p] = min(L[p], max(L[p - 1], x));
    L[0] = min(L[0], x);
}

// Sorted list, best first.  Inserts (w, c) given gt[p] = "(w, c) goes before entry p"; the last
// entry drops out.  All predicates are taken on the old list, so the slots update independently.
template <int KMAX>
__device__ __forceinline__ void list_insert(float (&kv)[KMAX], uint32_t (&ki)[KMAX], const bool (&gt)[KMAX],
                                            float w, uint32_t c) {
#pragma unroll
    for (int p = KMAX - 1; p > 0; p--) {
        kv[p] = gt[p - 1] ? kv[p - 1] : (gt[p] ? w : kv[p]);
        ki[p] = gt[p - 1] ? ki[p - 1] : (gt[p] ? c : ki[p]);
    }
    kv[0] = gt[0] ? w : kv[0];
    ki[0] = gt[0] ? c : ki[0];
}

// Columns arrive in increasing order: an equal w never overtakes (the earlier column wins).
template <int KMAX>
__device__ __forceinline__ void insert_in_order(float (&kv)[KMAX], uint32_t (&ki)[KMAX], float w, uint32_t c) {
    bool gt[KMAX];
#pragma unroll
    for (int p = 0; p < KMAX; p++) gt[p] = w > kv[p];
    list_insert<KMAX>(kv, ki, gt, w, c);
}

// Any order: larger w first, then smaller column.
template <int KMAX>
__device__ __forceinline__ void insert_lex(float (&kv)[KMAX], uint32_t (&ki)[KMAX], float w, uint32_t c) {
    bool gt[KMAX];
#pragma unroll
    for (int p = 0; p < KMAX; p++) gt[p] = w > kv[p] || (w == kv[p] && c < ki[p]);
    if (!gt[KMAX - 1]) return;
    list_insert<KMAX>(kv, ki, gt, w, c);
}

// Persistent: CTA b processes units b, b + grid, ...; every role walks the same unit sequence.
// B job j uses B stage j % S (phase (j / S) % 2) and accumulator buffer j % T (phase (j / T) % 2);
// unit i uses A buffer i % 2 (phase (i / 2) % 2).
template <int KB, int KMAX>
__global__ void __launch_bounds__(AS_THREADS, 1)
    assign_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap lmap,
                     const AsArgs a, uint32_t nunits) {
    using C = AsCfg<KB, KMAX>;
    extern __shared__ unsigned char as_smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(as_smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + C::OFF_HIST);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + C::OFF_MISC);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + C::OFF_MISC + 4);
    auto bar = [&](int i) { return sbase + C::OFF_BAR + 8 * i; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (uint32_t i = threadIdx.x; i < AS_HIST; i += AS_THREADS) hist[i] = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) {
            mbar_init(bar(C::BAR_FULL_A + i), 1);
            mbar_init(bar(C::BAR_EMPTY_A + i), 1);
        }
        for (int i = 0; i < C::S; i++) {
            mbar_init(bar(C::BAR_FULL + i), 32);
            mbar_init(bar(C::BAR_EMPTY + i), 1);
        }
        for (int i = 0; i < C::T; i++) {
            mbar_init(bar(C::BAR_TFULL + i), 1);
            mbar_init(bar(C::BAR_TEMPTY + i), EPI_WARPS * 32);
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
        // A's norm block: [1, 1, 1, 1, 0, ...] in logical chunk 0 of every row, zeros in chunk 1
        for (uint32_t r = lane; r < (uint32_t)ROWS; r += 32) {
            const uint32_t one = 0x3F80u;  // bf16 1.0
            const uint32_t base = sbase + C::OFF_AN + r * 128;
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(base + ((0u ^ (r & 7)) << 4)),
                         "r"(one | (one << 16)), "r"(one | (one << 16)), "r"(0u), "r"(0u)
                         : "memory");
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(base + ((1u ^ (r & 7)) << 4)), "r"(0u),
                         "r"(0u), "r"(0u), "r"(0u)
                         : "memory");
        }
        fence_proxy_async();
        // Per unit i of this CTA (u = blockIdx.x + i gridDim.x): one B job per 128 leaders (the A
        // rows are the gather warps').  The leader norms of the next B job (of this unit or the
        // next) are requested during the current one, unit descriptors a unit ahead.
        const uint32_t G = gridDim.x;
        auto desc = [&](uint32_t i) {
            const uint64_t u = blockIdx.x + (uint64_t)i * G;
            AsUnit x{};  // nrows = 0: past the last unit
            if (u < nunits) x = a.units[u];
            return x;
        };
        auto lead_norms = [&](const AsUnit &un, uint32_t t, uint32_t (&v)[4]) {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t c = t * C::NMAX + 4 * lane + e;
                v[e] = (un.nrows && c < un.ncols) ? (uint32_t)a.lead_norm[un.lead0 + c] : 0u;
            }
        };
        AsUnit d0 = desc(0), d1 = desc(1);
        uint32_t nrm[4];
        lead_norms(d0, 0, nrm);
        uint32_t j = 0;
        bool ok = true;
        for (uint32_t i = 0; ok && blockIdx.x + (uint64_t)i * G < nunits; i++) {
            const AsUnit d2 = desc(i + 2);
            const uint32_t nct = (d0.ncols + C::NMAX - 1) / C::NMAX;
            for (uint32_t t = 0; t < nct; t++, j++) {
                uint32_t nn[4];
                if (t + 1 < nct) lead_norms(d0, t + 1, nn);
                else lead_norms(d1, 0, nn);
                const uint32_t st = j % C::S;
                ok = __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_EMPTY + st), ((j / C::S) & 1) ^ 1, abort, a.err));
                if (!ok) break;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const uint32_t r = 4 * lane + e;
                    const uint2 pc = neg_half_norm_pieces(nrm[e]);
                    const uint32_t nb = sbase + C::OFF_BN + r * 128;
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(nb + (((2 * st) ^ (r & 7)) << 4)),
                                 "r"(pc.x), "r"(pc.y), "r"(0u), "r"(0u)
                                 : "memory");
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(nb + (((2 * st + 1) ^ (r & 7)) << 4)),
                                 "r"(0u), "r"(0u), "r"(0u), "r"(0u)
                                 : "memory");
                }
                fence_proxy_async();
                const uint32_t fb = bar(C::BAR_FULL + st);
                if (lane == 0) {
                    mbar_arrive_tx(fb, KB * REGION);
                    const uint32_t dst = sbase + C::OFF_B0 + st * KB * REGION;
                    const int32_t y = (int32_t)(d0.lead0 + (uint64_t)t * C::NMAX);
#pragma unroll
                    for (int kb = 0; kb < KB; kb++) tma_load_tile(dst + kb * REGION, &lmap, kb * 64, y, fb);
                } else {
                    mbar_arrive(fb);
                }
#pragma unroll
                for (int e = 0; e < 4; e++) nrm[e] = nn[e];
            }
            d0 = d1;
            d1 = d2;
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t j = 0, issued_j = 0;
            bool any = false, stop = false;
            // the next unit's leader count is requested one unit ahead
            uint32_t nc_next = blockIdx.x < nunits ? a.units[blockIdx.x].ncols : 0u;
            for (uint32_t i = 0, u = blockIdx.x; u < nunits && !stop; i++, u += gridDim.x) {
                const uint32_t ncols = nc_next;
                nc_next = u + gridDim.x < nunits ? a.units[u + gridDim.x].ncols : 0u;
                const uint32_t ua = i & 1;
                if (!mbar_wait(bar(C::BAR_FULL_A + ua), (i >> 1) & 1, abort, a.err)) break;
                const uint32_t aB = sbase + C::OFF_A0 + ua * KB * REGION;
                const uint32_t nct = (ncols + C::NMAX - 1) / C::NMAX;
                for (uint32_t t = 0; t < nct; t++, j++) {
                    const uint32_t st = j % C::S, tb = j % C::T;
                    if (!mbar_wait(bar(C::BAR_FULL + st), (j / C::S) & 1, abort, a.err) ||
                        !mbar_wait(bar(C::BAR_TEMPTY + tb), ((j / C::T) & 1) ^ 1, abort, a.err)) {
                        stop = true;
                        break;
                    }
                    fence_after();
                    const uint32_t c0 = t * C::NMAX;
                    const uint32_t nc = ncols - c0 < (uint32_t)C::NMAX ? ncols - c0 : C::NMAX;
                    const uint32_t idesc = idesc_bf16(128, (nc + 15) & ~15u);
                    const uint32_t bB = sbase + C::OFF_B0 + st * KB * REGION;
                    const uint32_t d = tmem + tb * C::NMAX;
#pragma unroll
                    for (int kk = 0; kk < KB * 4; kk++) {
                        const uint64_t ad = smem_desc_sw128(aB + (kk >> 2) * REGION + (kk & 3) * 32);
                        const uint64_t bd = smem_desc_sw128(bB + (kk >> 2) * REGION + (kk & 3) * 32);
                        mma_bf16(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    // - n_l / 2: ones x norm pieces (this stage's 32-byte slice)
                    mma_bf16(d, smem_desc_sw128(sbase + C::OFF_AN), smem_desc_sw128(sbase + C::OFF_BN + st * 32),
                             idesc, 1u);
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
    } else if (warp < AS_GATHER_WARP0) {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - EPI_WARP0;             // 0..7
        const int half = ew >> 2;                    // which column chunks
        const int quarter = warp & 3;                // TMEM lane quarter this warp may access
        const uint32_t r = quarter * 32 + lane;      // row inside the tile
        const uint32_t et = ew * 32 + lane;          // 0..255
        const uint32_t F = a.fanout;
        float2 *mv = reinterpret_cast<float2 *>(smem + C::OFF_MV);
        uint32_t j = 0;
        bool failed = false;
        // unit descriptors are requested two units ahead and the row's instance norm one unit
        // ahead, so no unit starts with a wait on a chain of loads
        auto desc = [&](uint64_t u) {
            AsUnit x{};
            if (u < nunits) x = a.units[u];
            return x;
        };
        auto row_norm = [&](const AsUnit &x) {
            return (KMAX <= 4 && x.row0 + r < x.nrows) ? a.inst_norm[x.inst0 + x.row0 + r] : 0;
        };
        AsUnit un = desc(blockIdx.x), un1 = desc(blockIdx.x + (uint64_t)gridDim.x);
        int32_t nrm = row_norm(un);
        for (uint32_t i = 0, u = blockIdx.x; u < nunits; i++, u += gridDim.x) {
            const AsUnit un2 = desc(u + 2 * (uint64_t)gridDim.x);
            const int32_t nrm1 = row_norm(un1);
            const bool row_ok = un.row0 + r < un.nrows;
            // F <= 4: the KMAX smallest (D << 32 | rank), D = n_x - 2 w the squared distance
            uint64_t RK[KMAX];
            float nb23 = 0.0f;
            if constexpr (KMAX <= 4) {
#pragma unroll
                for (int p = 0; p < KMAX; p++) RK[p] = ~0ull;
                nb23 = (float)(row_ok ? nrm : 0) + 8388608.0f;  // n_x + 2^23
            }
            // KMAX - F padding entries (+inf) in front, then the F live ones
            float kv[KMAX];
            uint32_t ki[KMAX];
#pragma unroll
            for (int p = 0; p < KMAX; p++) {
                const bool pad = (uint32_t)p + F < (uint32_t)KMAX;
                kv[p] = __int_as_float(pad ? 0x7f800000 : 0xff800000);
                ki[p] = pad ? AS_SENT : AS_NONE;
            }
            const uint32_t nct = (un.ncols + C::NMAX - 1) / C::NMAX;
            for (uint32_t t = 0; t < nct; t++, j++) {
                const uint32_t tb = j % C::T, ph = (j / C::T) & 1;
                if (failed) continue;
                // warp-uniform wait: tcgen05.ld below is a warp-collective instruction
                if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_TFULL + tb), ph, abort, a.err))) {
                    failed = true;
                    continue;
                }
                fence_after();
                const uint32_t c0 = t * C::NMAX;
                const uint32_t nc = un.ncols - c0 < (uint32_t)C::NMAX ? un.ncols - c0 : C::NMAX;
                if constexpr (KMAX <= 4) {
                    // D = n_x - 2 w is an integer below 2^23 (d <= 128 bytes): fma(-2, w, n_x + 2^23)
                    // is exact with bit pattern 0x4B000000 + D, so bits * 128 + column is a 32-bit
                    // key ordered by (D, rank); the tile's KMAX smallest via a min/max network
                    uint32_t L0[KMAX], L1[KMAX];
#pragma unroll
                    for (int p = 0; p < KMAX; p++) L0[p] = L1[p] = ~0u;
                    uint32_t g[2][32];
                    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + tb * C::NMAX;
                    const bool two = (half + 2) * 32 < nc;
                    // the second chunk loads while the first is ranked
                    if (half * 32 < nc) tmem_ld32_async(tbase + half * 32, g[0]);
                    tmem_wait_ld();
                    if (two) tmem_ld32_async(tbase + (half + 2) * 32, g[1]);
                    auto rank = [&](uint32_t (&gc)[32], uint32_t q, auto full_tag) {
                        constexpr bool FULL = decltype(full_tag)::value;
                        const uint32_t live = nc - q * 32;
#pragma unroll
                        for (int jj = 0; jj < 32; jj += 2) {
                            uint32_t k0 = __float_as_uint(__fmaf_rn(-2.0f, __uint_as_float(gc[jj]), nb23)) * 128u +
                                          (q * 32 + jj);
                            uint32_t k1 = __float_as_uint(__fmaf_rn(-2.0f, __uint_as_float(gc[jj + 1]), nb23)) *
                                              128u + (q * 32 + jj + 1);
                            if (!FULL) {
                                k0 = (uint32_t)jj < live ? k0 : ~0u;
                                k1 = (uint32_t)jj + 1 < live ? k1 : ~0u;
                            }
                            key_insert<KMAX>(L0, k0);
                            key_insert<KMAX>(L1, k1);
                        }
                    };
                    // columns past the tile's leaders are masked only in a ragged last chunk
                    if (half * 32 < nc) {
                        if (nc - half * 32 >= 32) rank(g[0], half, std::true_type());
                        else rank(g[0], half, std::false_type());
                    }
                    if (two) {
                        tmem_wait_ld_regs(g[1]);
                        if (nc - (half + 2) * 32 >= 32) rank(g[1], half + 2, std::true_type());
                        else rank(g[1], half + 2, std::false_type());
                    }
#pragma unroll
                    for (int p = 0; p < KMAX; p++) key_insert<KMAX>(L0, L1[p]);
                    // the tile's keys as (D << 32 | rank), merged into the running list
#pragma unroll
                    for (int p = 0; p < KMAX; p++) {
                        const uint64_t K = L0[p] == ~0u ? ~0ull
                                                        : ((uint64_t)((L0[p] & 0x7FFFFFFFu) >> 7) << 32) |
                                                              (c0 + (L0[p] & 127u));
                        key_insert<KMAX>(RK, K);
                    }
                } else {
                for (uint32_t q = half; q * 32 < nc; q += 2) {
                    uint32_t g[32];
                    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + tb * C::NMAX + q * 32, g);
                    uint32_t m = 0;
                    if (row_ok) {
                        const float thr = kv[KMAX - 1];
#pragma unroll
                        for (int jj = 0; jj < 32; jj++) m |= __uint_as_float(g[jj]) > thr ? (1u << jj) : 0u;
                        const uint32_t live = nc - q * 32;  // columns of this chunk inside the tile
                        if (live < 32) m &= (1u << live) - 1u;
                    }
                    const uint32_t base = c0 + q * 32;
                    while (__any_sync(0xffffffffu, m != 0)) {
                        if (m) {
                            const uint32_t jj = __ffs(m) - 1;
                            m &= m - 1;
                            const float w = __uint_as_float(pick32(g, jj));
                            if (w > kv[KMAX - 1]) insert_in_order<KMAX>(kv, ki, w, base + jj);
                        }
                    }
                }
                }
                fence_before();
                mbar_arrive(bar(C::BAR_TEMPTY + tb));
            }
            // merge the two halves of each row, then emit
            if constexpr (KMAX <= 4) {
                uint64_t *mk = reinterpret_cast<uint64_t *>(mv);
                if (half == 1) {
#pragma unroll
                    for (int p = 0; p < KMAX; p++) mk[r * KMAX + p] = RK[p];
                }
                failed = named_barrier_or(1, EPI_WARPS * 32, failed || *abort);
                if (half == 0 && row_ok && !failed) {
#pragma unroll
                    for (int p = 0; p < KMAX; p++) key_insert<KMAX>(RK, mk[r * KMAX + p]);
                    const uint32_t f = F < un.ncols ? F : un.ncols;
                    const uint64_t out = (un.inst0 + un.row0 + r) * (uint64_t)F;
#pragma unroll
                    for (int p = 0; p < KMAX; p++) {
                        const uint32_t rank = (uint32_t)RK[p];
                        if ((uint32_t)p < f && RK[p] != ~0ull && rank < AS_HIST) {
                            a.assign[out + p] = (uint16_t)rank;
                            atomicAdd(&hist[rank], 1u);
                        }
                    }
                }
            } else {
            if (half == 1) {
#pragma unroll
                for (int p = 0; p < KMAX; p++) mv[r * KMAX + p] = make_float2(kv[p], __uint_as_float(ki[p]));
            }
            failed = named_barrier_or(1, EPI_WARPS * 32, failed || *abort);
            if (half == 0 && row_ok && !failed) {
#pragma unroll
                for (int p = 0; p < KMAX; p++) {
                    const float2 e = mv[r * KMAX + p];
                    const uint32_t c = __float_as_uint(e.y);
                    if (c < AS_SENT) insert_lex<KMAX>(kv, ki, e.x, c);
                }
                const uint32_t f = F < un.ncols ? F : un.ncols;
                const uint64_t out = (un.inst0 + un.row0 + r) * (uint64_t)F;
#pragma unroll
                for (int p = 0; p < KMAX; p++) {
                    const int slot = p - (KMAX - (int)F);
                    if (slot >= 0 && (uint32_t)slot < f && ki[p] < AS_HIST) {
                        a.assign[out + slot] = (uint16_t)ki[p];
                        atomicAdd(&hist[ki[p]], 1u);
                    }
                }
            }
            }
            // mv is rewritten, and the histogram counted into, only after every thread is done
            failed = named_barrier_or(1, EPI_WARPS * 32, failed || *abort);
            if (failed) break;
            const uint32_t nu = u + gridDim.x;
            if (nu >= nunits || un1.seg != un.seg) {
                for (uint32_t c = et; c < un.ncols && c < AS_HIST; c += EPI_WARPS * 32) {
                    const uint32_t h = hist[c];
                    if (h) {
                        atomicAdd(&a.bucket_cnt[un.lead0 + c], h);
                        hist[c] = 0;
                    }
                }
            }
            un = un1;
            un1 = un2;
            nrm = nrm1;
        }
    } else {
        // ------------------------------------------------------------ A-row gathers (two warps)
        // Gather warp g fills A buffer g with the instance rows of units g, g + 2, ...: lane L
        // fetches tile rows 4L .. 4L + 3 of every K block.  Its unit descriptors are requested
        // two own units ahead and the instance ids one own unit ahead.
        const uint32_t g = (uint32_t)(warp - AS_GATHER_WARP0);
        const uint32_t G = gridDim.x;
        auto desc = [&](uint32_t i) {
            const uint64_t u = blockIdx.x + (uint64_t)i * G;
            AsUnit x{};  // nrows = 0: past the last unit
            if (u < nunits) x = a.units[u];
            return x;
        };
        auto inst_ids = [&](const AsUnit &un, uint32_t (&v)[4]) {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                // rows past the subproblem repeat its last instance; their results are unused
                uint32_t r = un.row0 + 4 * lane + e;
                r = r < un.nrows ? r : un.nrows - 1;
                v[e] = un.nrows ? a.inst[un.inst0 + r] : 0u;
            }
        };
        AsUnit e1 = desc(g + 2), e2 = desc(g + 4);
        uint32_t rows0[4], rows1[4];
        inst_ids(desc(g), rows0);
        inst_ids(e1, rows1);
        for (uint32_t i = g; blockIdx.x + (uint64_t)i * G < nunits; i += 2) {
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_EMPTY_A + g), ((i >> 1) & 1) ^ 1, abort, a.err))) break;
            const uint32_t fb = bar(C::BAR_FULL_A + g);
            if (lane == 0) mbar_arrive_tx(fb, KB * REGION);
            __syncwarp();
            const uint32_t dst = sbase + C::OFF_A0 + g * KB * REGION + lane * 4 * 128;
#pragma unroll
            for (int kb = 0; kb < KB; kb++)
                tma_gather4(dst + kb * REGION, &xmap, kb * 64, (int32_t)rows0[0], (int32_t)rows0[1],
                            (int32_t)rows0[2], (int32_t)rows0[3], fb);
            uint32_t rows2[4];
            inst_ids(e2, rows2);
            const AsUnit e3 = desc(i + 6);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                rows0[e] = rows1[e];
                rows1[e] = rows2[e];
            }
            e2 = e3;
        }
    }

    fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

__global__ void build_as_units(const uint32_t *tile_grp, const uint32_t *tile_row0, uint64_t nunits,
                               const uint64_t *seg_start, const uint32_t *seg_size, const uint64_t *lead_off,
                               const uint32_t *lead_cnt, AsUnit *units) {
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < nunits; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = tile_grp[u];
        AsUnit x;
        x.inst0 = seg_start[g];
        x.lead0 = lead_off[g];
        x.nrows = seg_size[g];
        x.row0 = tile_row0[u];
        x.ncols = lead_cnt[g];
        x.seg = g;
        units[u] = x;
    }
}

__global__ void gather_norms(const uint32_t *ids, uint64_t M, const int32_t *sqnorm, int32_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < M; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = sqnorm[ids[i]];
}

template <int KB, int KMAX>
int launch_as(const CUtensorMap &xmap, const CUtensorMap &lmap, const AsArgs &args, uint64_t nunits) {
    using C = AsCfg<KB, KMAX>;
    auto kern = assign_tc_kernel<KB, KMAX>;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int dev = 0, sms = 0;
    PIPNN_CUDA(cudaGetDevice(&dev));
    PIPNN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (uint64_t t0 = 0; t0 < nunits; t0 += 0xFFFFFFFFull) {
        const uint64_t cnt = nunits - t0 < 0xFFFFFFFFull ? nunits - t0 : 0xFFFFFFFFull;
        AsArgs a = args;
        a.units += t0;
        const unsigned grid = (unsigned)(cnt < (uint64_t)sms ? cnt : (uint64_t)sms);
        kern<<<grid, AS_THREADS, C::SMEM, stream()>>>(xmap, lmap, a, (uint32_t)cnt);
        PIPNN_LAUNCH_CHECK();
    }
    return PIPNN_OK;
}

template <int KB>
int launch_as_k(const CUtensorMap &xmap, const CUtensorMap &lmap, const AsArgs &args, uint64_t nunits, uint32_t F) {
    // the smallest list that holds F: each column costs 2 KMAX - 1 min / max operations
    if (F == 1) return launch_as<KB, 1>(xmap, lmap, args, nunits);
    if (F == 2) return launch_as<KB, 2>(xmap, lmap, args, nunits);
    if (F == 3) return launch_as<KB, 3>(xmap, lmap, args, nunits);
    if (F <= 4) return launch_as<KB, 4>(xmap, lmap, args, nunits);
    if (F <= 8) return launch_as<KB, 8>(xmap, lmap, args, nunits);
    return launch_as<KB, 16>(xmap, lmap, args, nunits);
}

}  // namespace

bool assign_tc_eligible(int dtype, uint32_t d, uint64_t n, uint32_t F) {
    return (dtype == PIPNN_U8 || dtype == PIPNN_I8) && d >= 1 && d <= 128 && n < 0x7FFFFF00ull && F >= 1 &&
           F <= ASSIGN_TC_MAX_F;
}

int assign_tc_plan(const void *X, uint64_t n, uint32_t d, int dtype, Workspace &ws, AssignTcPlan *plan) {
    plan->kp = d <= 64 ? 64 : 128;
    PIPNN_TRY(ws.alloc(&plan->rows, (n ? n : 1) * plan->kp));
    PIPNN_TRY(stage_rows_bf16(X, d, plan->kp, dtype, nullptr, n, plan->rows));
    PIPNN_TRY(encode_rows_map(&plan->map, plan->rows, n ? n : 1, plan->kp, true));
    return PIPNN_OK;
}

int assign_tc(const AssignTcPlan &plan, const void *X, uint32_t d, int dtype, const int32_t *sqnorm,
              const uint32_t *tile_grp, const uint32_t *tile_row0, uint64_t ntiles, const uint64_t *seg_start,
              const uint32_t *seg_size, const uint32_t *inst, const uint64_t *lead_off, const uint32_t *lead_cnt,
              const uint32_t *lead, uint64_t total_leaders, uint64_t ninst, uint32_t F, uint16_t *assign,
              uint32_t *bucket_cnt, Workspace &ws) {
    if (F < 1 || F > ASSIGN_TC_MAX_F) return set_error(PIPNN_EINVAL, "fanout %u outside 1..%u", F, ASSIGN_TC_MAX_F);
    if (ntiles == 0) return PIPNN_OK;
    if (total_leaders >= 0x7FFFFF00ull) return set_error(PIPNN_EUNSUPPORTED, "too many leaders in one level");
    __nv_bfloat16 *lrows = nullptr;
    int32_t *lnorm = nullptr, *inorm = nullptr;
    AsUnit *units = nullptr;
    PIPNN_TRY(ws.alloc(&lrows, total_leaders * plan.kp));
    PIPNN_TRY(ws.alloc(&lnorm, total_leaders));
    PIPNN_TRY(ws.alloc(&units, ntiles));
    PIPNN_TRY(stage_rows_bf16(X, d, plan.kp, dtype, lead, total_leaders, lrows));
    gather_norms<<<grid_for(total_leaders, 256), 256, 0, stream()>>>(lead, total_leaders, sqnorm, lnorm);
    PIPNN_LAUNCH_CHECK();
    if (F <= 4) {
        PIPNN_TRY(ws.alloc(&inorm, ninst ? ninst : 1));
        if (ninst) {
            gather_norms<<<grid_for(ninst, 256), 256, 0, stream()>>>(inst, ninst, sqnorm, inorm);
            PIPNN_LAUNCH_CHECK();
        }
    }
    build_as_units<<<grid_for(ntiles, 256), 256, 0, stream()>>>(tile_grp, tile_row0, ntiles, seg_start, seg_size,
                                                                lead_off, lead_cnt, units);
    PIPNN_LAUNCH_CHECK();
    CUtensorMap lmap;
    PIPNN_TRY(encode_rows_map(&lmap, lrows, total_leaders, plan.kp, false));
    AsArgs a{};
    a.units = units;
    a.inst = inst;
    a.inst_norm = inorm;
    a.lead_norm = lnorm;
    a.fanout = F;
    a.assign = assign;
    a.bucket_cnt = bucket_cnt;
    a.err = device_error_word();
    if (plan.kp == 64) return launch_as_k<1>(plan.map, lmap, a, ntiles, F);
    return launch_as_k<2>(plan.map, lmap, a, ntiles, F);
}

}  // namespace pipnn
