// leaf_tcf.cu -- A2..A4 for float data on the tensor cores at reduced precision, with an exact
// FP32 re-rank of the candidates near every row's k-th.
//
// Sec. 4.2 builds the leaf's all-pairs dissimilarity matrix with a GEMM, and the conclusion names
// quantised GEMMs as the way to make that step cheaper.  Here the Gram matrix of every leaf is
// formed by tcgen05.mma from BF16 (kind::f16) or FP8 e4m3 (kind::f8f6f4, one scale per leaf)
// operands with FP32 accumulation in TMEM, and the picks still equal those of the defining
// binary32 evaluation (one fused multiply-add per coordinate in index order) bit for bit:
//
//  1. Staging (leaf_stage_f32, one block per leaf).  The leaf centroid mu is subtracted first
//     (x' = fl(x - mu)); squared L2 is shift invariant, and for the inner product
//     1 - <x_i, x_j> + P = w_i + w_j - <x'_i, x'_j> with w = (1 + |mu|^2 + P) / 2 - <x, mu>, where
//     the per-leaf offset P >= max(0, max |x|^2 - 1) keeps every key non-negative.  Centring
//     shrinks the operands to the leaf's own spread, which the rounding error scales with.  The
//     operands are
//     rounded to BF16 (or s x' to e4m3, s = 448 (1 - 2^-8) / max |x'_t| over the leaf); the
//     per-row term v = n'/2 (L2) or w (IP), times s^2, enters the MMA as one extra K = 16 step of
//     four exact BF16 pieces, so the accumulator holds -sigma D~ with sigma = s^2 / 2 (L2) or s^2
//     (IP, shifted by P).
//  2. Approximate pick (leaf_gram_tcf).  Per row the KP smallest keys (the binary32 value -acc
//     with its low CB bits replaced by the leaf column, so keys are unique and ordered by value)
//     are tracked with a branch-free insertion network.
//  3. Band.  With E an upper bound on |D~_ij - D_ij| over the row (below), every member of the
//     exact top k (by the binary32 D and id) has D~ <= tau + 2E, where tau is the k-th smallest
//     D~ of the row: the k approximately nearest have D <= D~ + E <= tau + E, so the k-th exact
//     distance is at most tau + E, and a member of the exact top k has D~ <= D + E <= tau + 2E.
//     If the KP-th tracked key lies beyond tau + 2E, every untracked column lies beyond it too
//     and the tracked keys up to tau + 2E hold the exact top k; the row's candidates are those.
//     Otherwise the row is listed for a full evaluation.
//  4. Re-rank (rerank_rows, rerank_full).  The candidates' dissimilarities are evaluated in the
//     defining binary32 order and the k smallest by (D, id) are emitted in both directions.
//
// The error bound E (D units) adds: operand rounding of the Gram (unit roundoff u_q = 2^-8 for
// BF16, 2^-4 plus an absolute 2^-10 below the e4m3 normal range, in scaled units, for FP8), the
// binary32 rounding of the centring, the norms / w and their pieces, the tensor-core FP32
// accumulation (taken as relative error at most u_acc = 2^-16 (kind::f16) or 2^-11
// (kind::f8f6f4) of the accumulated magnitudes per MMA instruction -- an assumption about the
// hardware accumulator, checked against FP64 by the tests), the error of the defining binary32
// evaluation itself, and a 25 % safety factor.  Truncating a key's low CB bits moves it by less
// than 2^(CB-23) of its value, which the threshold adds as well.
#include <cuda_fp8.h>

#include "allpairs.cuh"
#include "tc_common.cuh"

namespace pipnn {

namespace {

using namespace tc;

enum : int { PREC_BF16 = PIPNN_PREC_BF16, PREC_FP8 = PIPNN_PREC_FP8, PREC_SPLIT = PIPNN_PREC_BF16X3 };

struct LeafInfoF {
    float R;      // max over the leaf of |x'_j| (rounded up)
    float m;      // |mu| (rounded up)
    float P;      // inner product: the key offset (>= max(0, max |x_j|^2 - 1)); L2: 0
    float scale;  // operand scale s (FP8), 1 for BF16
};

struct TcUnitF {
    uint64_t off;   // first member of the leaf
    uint64_t out;   // first output slot of the tile's first row
    uint32_t s;     // leaf size
    uint32_t row0;  // first row of the tile
    uint32_t leaf;
    uint32_t pad;
};

// Coefficients of the row bound E(r, R) in D units; per leaf the FP8 terms scale with 1/s.
struct BandCoef {
    float rR, sq, lin, zero;  // L2: rR * r R + sq * (r^2 + R^2) + lin * (r + R) / s + zero / s^2
    float W, mm, one;         // IP: + W * W(leaf) + mm * (r + m)(R + m) + one
    float safety;
};

struct TcfArgs {
    const TcUnitF *units;
    const uint2 *pieces;       // -(v) of every leaf member as four BF16 pieces
    const float *rnorm;        // |x'_j| of every leaf member (rounded up)
    const LeafInfoF *info;
    BandCoef bc;
    int metric;
    uint32_t colbits;          // CB: low key bits that hold the leaf column
    uint32_t k;
    uint16_t *cand;            // KP leaf columns per member row
    uint8_t *ccnt;             // candidates per member row; 0xFF: full evaluation
    uint32_t *ovf;             // (unit << 7 | row) of rows that need a full evaluation
    unsigned *novf;
    unsigned *leaf_ovf;        // rows of every leaf that need a full evaluation
    unsigned *err;
    float *gram;               // dump mode: the approximate dissimilarities, leaf by leaf
    const uint64_t *gram_off;  // dump mode: first entry of every leaf's |b| x |b| block
};

// KB: 128-byte K blocks of one operand (for the split form: of each of its hi and lo halves).
template <int PREC, int KB, int KP>
struct TcfCfg {
    static constexpr bool SPLIT = PREC == PREC_SPLIT;
    static constexpr int NMAX = 128;
    static constexpr int KBA = SPLIT ? 2 * KB : KB;    // K blocks of an A tile (hi then lo)
    static constexpr int KBB = KB;                     // K blocks of one B job (hi or lo half)
    static constexpr int JPT = SPLIT ? 2 : 1;          // B jobs per 128-column tile
    static constexpr int S = SPLIT ? (KB == 2 ? 2 : 4) : (PREC == PREC_FP8 ? 4 : 3);  // B stages
    static constexpr int T = 4;                        // accumulator buffers
    static constexpr int REGION = tc::REGION;
    // norm slices (32 bytes per row each, four per 128-byte row): A buffer x uses slice x of the
    // AN region; B stage x slice BSLICE0 + x of the BN region, which is the AN region itself when
    // the operand tiles leave no room for a second one
    static constexpr bool MERGED = SPLIT && KB == 2;
    static constexpr int BSLICE0 = MERGED ? 2 : 0;
    static constexpr int OFF_A0 = 0;
    static constexpr int OFF_AN = OFF_A0 + 2 * KBA * REGION;
    static constexpr int OFF_B0 = OFF_AN + REGION;
    static constexpr int OFF_BN = MERGED ? OFF_AN : OFF_B0 + S * KBB * REGION;
    static constexpr int OFF_MV = (MERGED ? OFF_B0 + S * KBB * REGION : OFF_BN + REGION);  // 2 x 128 x KP keys
    static constexpr int OFF_BAR = OFF_MV + 2 * ROWS * KP * 4;
    static constexpr int BAR_FULL_A = 0, BAR_EMPTY_A = 2, BAR_FULL = 4, BAR_EMPTY = BAR_FULL + S,
                         BAR_TFULL = BAR_EMPTY + S, BAR_TEMPTY = BAR_TFULL + T, BAR_DRAIN = BAR_TEMPTY + T,
                         NBAR = BAR_DRAIN + 1;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr int SMEM = BYTES + 1024;
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(T * NMAX <= (int)TMEM_COLS, "TMEM budget");
    static_assert(BSLICE0 + S <= 4, "norm slices per 128-byte row");
};

// Keeps K[0] < K[1] < ... < K[KP-1], the KP smallest keys seen (keys are unique).
template <int KP>
__device__ __forceinline__ void keep_smallest(uint32_t (&K)[KP], uint32_t key) {
#pragma unroll
    for (int p = KP - 1; p > 0; p--) K[p] = min(K[p], max(K[p - 1], key));
    K[0] = min(K[0], key);
}

// Half-width E of the band in key units for a row with |x'_i| = r in a leaf with `li`.
__device__ __forceinline__ float band_key(const BandCoef &c, int metric, float r, const LeafInfoF &li) {
    const float R = li.R, inv_s = 1.0f / li.scale;
    float e = c.rR * r * R + c.lin * (r + R) * inv_s + c.zero * inv_s * inv_s;
    float sigma;
    if (metric == PIPNN_L2) {
        e += c.sq * (r * r + R * R);
        sigma = 0.5f * li.scale * li.scale;
    } else {
        const float m = li.m;
        const float W = 0.5f * (1.0f + m * m + li.P) + (R + m) * m;
        e += c.W * W + c.mm * (r + m) * (R + m) + c.one;
        sigma = li.scale * li.scale;
    }
    return c.safety * e * sigma;
}

// DUMP: instead of ranking, every row writes its approximate dissimilarities (the accumulator
// converted back to D units, before any re-rank) to a.gram.
template <int PREC, int KB, int KP, bool DUMP>
__global__ void __launch_bounds__(THREADS, 1)
    leaf_gram_tcf(const __grid_constant__ CUtensorMap map, const TcfArgs a, uint32_t nunits, uint32_t ksteps) {
    using C = TcfCfg<PREC, KB, KP>;
    extern __shared__ unsigned char tcf_smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tcf_smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
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
        }
        mbar_init(bar(C::BAR_DRAIN), 1);
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
        // norm slices: A buffer x = [1,1,1,1, a-pieces, 0 x 8], B stage x = [b-pieces, 1,1,1,1, 0 x 8]
        for (uint32_t r = lane; r < (uint32_t)ROWS; r += 32) {
            const uint32_t one2 = 0x3F803F80u;
            for (uint32_t q = 0; q < 8; q++) {
                const bool first = (q & 1) == 0;
                const bool b_type = C::MERGED && (q >> 1) >= 2;
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(sbase + C::OFF_AN + r * 128 +
                                                                              ((q ^ (r & 7)) << 4)),
                             "r"(first && !b_type ? one2 : 0u), "r"(first && !b_type ? one2 : 0u),
                             "r"(first && b_type ? one2 : 0u), "r"(first && b_type ? one2 : 0u)
                             : "memory");
            }
            if (!C::MERGED) {
                for (uint32_t q = 0; q < 8; q++) {
                    const bool first = (q & 1) == 0;
                    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(sbase + C::OFF_BN + r * 128 +
                                                                                  ((q ^ (r & 7)) << 4)),
                                 "r"(0u), "r"(0u), "r"(first ? one2 : 0u), "r"(first ? one2 : 0u)
                                 : "memory");
                }
            }
        }
        fence_proxy_async();
        // job stream: per unit one A job, then per 128-column tile one B job (two for the split
        // form: its hi half, which carries the column norms, then its lo half)
        struct Job {
            uint32_t kind;  // 0 A, 1 B, 2 end
            uint32_t i, u, t, s, first, h;
            uint64_t off;
        };
        auto unit_job = [&](uint32_t i, uint32_t u) {
            Job q;
            if (u >= nunits) {
                q.kind = 2;
                return q;
            }
            const TcUnitF un = a.units[u];
            q.kind = 0;
            q.i = i;
            q.u = u;
            q.t = 0;
            q.h = 0;
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
                q.h = 0;
                q.first = 0;
                return q;
            }
            if (C::SPLIT && c.h == 0) {
                q.h = 1;
                return q;
            }
            const uint32_t nct = (c.s + C::NMAX - 1) / C::NMAX;
            if (c.t + 1 < nct) {
                q.t = c.t + 1;
                q.h = 0;
                q.first = q.t * C::NMAX;
                return q;
            }
            return unit_job(c.i + 1, c.u + gridDim.x);
        };
        auto load_pieces = [&](const Job &q, uint2 (&nr)[4]) {
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const uint32_t r = q.first + 4 * lane + e;
                nr[e] = (q.kind <= 1 && q.h == 0 && r < q.s) ? a.pieces[q.off + r] : make_uint2(0u, 0u);
            }
        };
        // TMA x coordinate of K block kb: 64 BF16 elements or 128 e4m3 bytes
        constexpr int XSTEP = PREC == PREC_FP8 ? 128 : 64;
        Job cur = unit_job(0, blockIdx.x);
        uint2 nr[4];
        load_pieces(cur, nr);
        uint32_t j = 0;
        while (cur.kind != 2) {
            const Job nxt = next_job(cur);
            uint2 nnr[4];
            bool ok;
            if (cur.kind == 0) {
                const uint32_t ua = cur.i & 1;
                ok = mbar_wait(bar(C::BAR_EMPTY_A + ua), ((cur.i >> 1) & 1) ^ 1, abort, a.err);
                load_pieces(nxt, nnr);
                if (ok) {
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
                        mbar_arrive_tx(fb, C::KBA * C::REGION);
                        const uint32_t dst = sbase + C::OFF_A0 + ua * C::KBA * C::REGION;
#pragma unroll
                        for (int kb = 0; kb < C::KBA; kb++)
                            tma_load_tile(dst + kb * C::REGION, &map, kb * XSTEP, (int32_t)(cur.off + cur.first), fb);
                    } else {
                        mbar_arrive(fb);
                    }
                }
            } else {
                const uint32_t st = j % C::S;
                ok = mbar_wait(bar(C::BAR_EMPTY + st), ((j / C::S) & 1) ^ 1, abort, a.err);
                if (ok && cur.h == 0) {
                    const uint32_t sl = C::BSLICE0 + st;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const uint32_t r = 4 * lane + e;
                        asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(sbase + C::OFF_BN + r * 128 +
                                                                             (((2 * sl) ^ (r & 7)) << 4)),
                                     "r"(nr[e].x), "r"(nr[e].y)
                                     : "memory");
                    }
                    fence_proxy_async();
                }
                load_pieces(nxt, nnr);
                if (ok) {
                    const uint32_t fb = bar(C::BAR_FULL + st);
                    if (lane == 0) {
                        mbar_arrive_tx(fb, C::KBB * C::REGION);
                        const uint32_t dst = sbase + C::OFF_B0 + st * C::KBB * C::REGION;
#pragma unroll
                        for (int kb = 0; kb < C::KBB; kb++)
                            tma_load_tile(dst + kb * C::REGION, &map, (cur.h * KB + kb) * XSTEP,
                                          (int32_t)(cur.off + cur.first), fb);
                    } else {
                        mbar_arrive(fb);
                    }
                }
                j++;
            }
            if (!__all_sync(0xffffffffu, ok)) break;
            cur = nxt;
#pragma unroll
            for (int e = 0; e < 4; e++) nr[e] = nnr[e];
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        // B job jb (one stage load) uses stage jb % S; tile j uses accumulator buffer j % T.  The
        // split form issues hi.hi and lo.hi and the norm step on the tile's hi job, hi.lo on its
        // lo job.
        if (lane == 0) {
            uint32_t j = 0, jb = 0, issued_j = 0;
            bool any = false, stop = false;
            auto products = [&](uint32_t d, uint32_t aB, uint32_t bB, uint32_t nn, bool first) {
                for (uint32_t kk = 0; kk < ksteps; kk++) {
                    const uint64_t ad = smem_desc_sw128(aB + (kk >> 2) * C::REGION + (kk & 3) * 32);
                    const uint64_t bd = smem_desc_sw128(bB + (kk >> 2) * C::REGION + (kk & 3) * 32);
                    const uint32_t acc = (first && kk == 0) ? 0u : 1u;
                    if (PREC == PREC_FP8) mma_e4m3(d, ad, bd, idesc_e4m3(128, nn), acc);
                    else mma_bf16(d, ad, bd, idesc_bf16(128, nn), acc);
                }
            };
            for (uint32_t i = 0, u = blockIdx.x; u < nunits && !stop; i++, u += gridDim.x) {
                const uint32_t s = a.units[u].s;
                const uint32_t ua = i & 1;
                if (!mbar_wait(bar(C::BAR_FULL_A + ua), (i >> 1) & 1, abort, a.err)) break;
                const uint32_t aB = sbase + C::OFF_A0 + ua * C::KBA * C::REGION;
                const uint32_t nct = (s + C::NMAX - 1) / C::NMAX;
                for (uint32_t t = 0; t < nct; t++, j++) {
                    const uint32_t st = jb % C::S, tb = j % C::T;
                    if (!mbar_wait(bar(C::BAR_FULL + st), (jb / C::S) & 1, abort, a.err) ||
                        !mbar_wait(bar(C::BAR_TEMPTY + tb), ((j / C::T) & 1) ^ 1, abort, a.err)) {
                        stop = true;
                        break;
                    }
                    fence_after();
                    const uint32_t c0 = t * C::NMAX;
                    const uint32_t ncols = s - c0 < (uint32_t)C::NMAX ? s - c0 : C::NMAX;
                    const uint32_t nn = (ncols + 15) & ~15u;
                    const uint32_t bB = sbase + C::OFF_B0 + st * C::KBB * C::REGION;
                    const uint32_t d = tmem + tb * C::NMAX;
                    products(d, aB, bB, nn, true);                                   // hi . hi
                    if (C::SPLIT) products(d, aB + KB * C::REGION, bB, nn, false);    // lo . hi
                    // - v_i - v_j from the BF16 norm slices of this A buffer and this B stage
                    mma_bf16(d, smem_desc_sw128(sbase + C::OFF_AN + ua * 32),
                             smem_desc_sw128(sbase + C::OFF_BN + (C::BSLICE0 + st) * 32), idesc_bf16(128, nn), 1u);
                    mma_commit(bar(C::BAR_EMPTY + st));
                    jb++;
                    if (C::SPLIT) {
                        const uint32_t st2 = jb % C::S;
                        if (!mbar_wait(bar(C::BAR_FULL + st2), (jb / C::S) & 1, abort, a.err)) {
                            stop = true;
                            any = true;
                            issued_j = j;
                            break;
                        }
                        fence_after();
                        products(d, aB, sbase + C::OFF_B0 + st2 * C::KBB * C::REGION, nn, false);  // hi . lo
                        mma_commit(bar(C::BAR_EMPTY + st2));
                        jb++;
                    }
                    mma_commit(bar(C::BAR_TFULL + tb));
                    any = true;
                    issued_j = j;
                }
                if (!stop) mma_commit(bar(C::BAR_EMPTY_A + ua));
            }
            if (stop && any) {
                // let the MMAs already issued complete before TMEM is released: a commit to a
                // barrier of its own, waited for with a time bound only (the abort flag is set)
                (void)issued_j;
                mma_commit(bar(C::BAR_DRAIN));
                const unsigned long long t0 = globaltimer();
                while (!mbar_try_wait(bar(C::BAR_DRAIN), 0) && globaltimer() - t0 < WAIT_NS) {
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue (8 warps)
        // Warp (quarter, half) reads TMEM lanes 32 quarter .. + 31 (its rows) and ranks chunks half
        // and half + 2 of every 128-column tile; one chunk's load is in flight while the other is
        // ranked, across tiles and units.
        const int ew = warp - EPI_WARP0;
        const int half = ew >> 2;
        const int quarter = warp & 3;
        const uint32_t r = quarter * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
        const uint32_t cmask = (1u << a.colbits) - 1u;
        uint32_t *mv = reinterpret_cast<uint32_t *>(smem + C::OFF_MV);
        auto open_tile = [&](uint32_t jj) {
            const uint32_t tb = jj % C::T, ph = (jj / C::T) & 1;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_TFULL + tb), ph, abort, a.err));
            fence_after();
            return ok;
        };
        uint32_t u = blockIdx.x, i = 0, j = 0, t = 0;
        TcUnitF un = a.units[u];
        TcUnitF unx = a.units[u + gridDim.x < nunits ? u + gridDim.x : u];
        auto rank_chunk = [&](uint32_t (&g)[32], uint32_t base, uint32_t s, uint32_t self_col, uint32_t (&K)[KP]) {
            if constexpr (DUMP) {
                // self_col is this row's leaf column; rows past the leaf write nothing
                if (self_col >= s) return;
                const LeafInfoF li = a.info[un.leaf];
                const float sigma = (a.metric == PIPNN_L2 ? 0.5f : 1.0f) * li.scale * li.scale;
                float *row = a.gram + a.gram_off[un.leaf] + (uint64_t)self_col * s;
#pragma unroll
                for (int jj = 0; jj < 32; jj++) {
                    if (base + jj < s) {
                        const float D = __fdiv_rn(-__uint_as_float(g[jj]), sigma);
                        row[base + jj] = a.metric == PIPNN_L2 ? D : __fsub_rn(D, li.P);
                    }
                }
                return;
            }
            uint32_t key[32];
#pragma unroll
            for (int jj = 0; jj < 32; jj++)
                key[jj] = (__float_as_uint(fmaxf(-__uint_as_float(g[jj]), 0.0f)) & ~cmask) | (base + jj);
            if (self_col - base < 32u || base + 32 > s) {
#pragma unroll
                for (int jj = 0; jj < 32; jj++)
                    if (base + jj == self_col || base + jj >= s) key[jj] = ~0u;
            }
#pragma unroll
            for (int jj = 0; jj < 32; jj++) keep_smallest<KP>(K, key[jj]);
        };
        uint32_t K[KP];
#pragma unroll
        for (int p = 0; p < KP; p++) K[p] = ~0u;
        uint32_t gA[32], gB[32];
#pragma unroll
        for (int jj = 0; jj < 32; jj++) gA[jj] = gB[jj] = 0u;
        bool failed = !open_tile(0);
        bool cur_ok = !failed;
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
            if (v0) rank_chunk(gA, c0 + half * 32, un.s, self_col, K);
            tmem_wait_ld_regs(gB);
            const bool last = t + 1 == nct;
            bool nxt_ok = false;
            if (!failed && (!last || u + gridDim.x < nunits)) {
                nxt_ok = open_tile(j + 1);
                failed = !nxt_ok;
                const uint32_t nrem = last ? unx.s : un.s - c0 - C::NMAX;
                if (nxt_ok && half * 32 < nrem) tmem_ld32_async(tq + ((j + 1) % C::T) * C::NMAX + half * 32, gA);
            }
            if (v1) rank_chunk(gB, c0 + (half + 2) * 32, un.s, self_col, K);
            if (cur_ok) {
                fence_before();
                mbar_arrive(bar(C::BAR_TEMPTY + tb));
            }
            cur_ok = nxt_ok;
            j++;
            if (!last) {
                t++;
                continue;
            }
            // unit done: merge the halves of each row, find the band, write the candidates
            uint32_t *m = mv + ((i & 1) * ROWS + r) * KP;
            if (half == 1) {
#pragma unroll
                for (int p = 0; p < KP; p++) m[p] = K[p];
            }
            failed = named_barrier_or(1, EPI_WARPS * 32, failed || *abort);
            if (!DUMP && half == 0 && un.row0 + r < un.s && !failed) {
#pragma unroll
                for (int p = 0; p < KP; p++) keep_smallest<KP>(K, m[p]);
                const uint64_t row = un.off + un.row0 + r;
                const uint32_t kk = un.s - 1 < a.k ? un.s - 1 : a.k;
                uint32_t cnt = 0;
                bool full = false;
                if (kk > 0) {
                    const LeafInfoF li = a.info[un.leaf];
                    const float E = band_key(a.bc, a.metric, a.rnorm[row], li);
                    uint32_t kth = 0;  // K[kk - 1], selected without a dynamic register index
#pragma unroll
                    for (int p = 0; p < KP; p++)
                        if ((uint32_t)p + 1 == kk) kth = K[p];
                    const float tau = __uint_as_float(kth & ~cmask);
                    const float grow = 1.0f + __uint_as_float((uint32_t)(127 + a.colbits - 22) << 23);
                    const float thr = (tau * grow + 2.0f * E) * 1.0000005f;
                    const uint32_t tb_ = __float_as_uint(thr);
                    const bool complete = un.s - 1 <= (uint32_t)KP || (K[KP - 1] & ~cmask) > tb_;
                    if (complete) {
#pragma unroll
                        for (int p = 0; p < KP; p++) {
                            if (K[p] != ~0u && (K[p] & ~cmask) <= tb_) {
                                a.cand[row * KP + cnt] = (uint16_t)(K[p] & cmask);
                                cnt++;
                            }
                        }
                    } else {
                        full = true;
                    }
                }
                a.ccnt[row] = full ? (uint8_t)0xFF : (uint8_t)cnt;
                if (full) {
                    const unsigned slot = atomicAdd(a.novf, 1u);
                    a.ovf[slot] = (u << 7) | r;
                    atomicAdd(a.leaf_ovf + un.leaf, 1u);
                }
            }
            u += gridDim.x;
            i++;
            if (failed || u >= nunits) break;
            un = unx;
            unx = a.units[u + gridDim.x < nunits ? u + gridDim.x : u];
            t = 0;
#pragma unroll
            for (int p = 0; p < KP; p++) K[p] = ~0u;
        }
        tmem_wait_ld();
    }

    fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ------------------------------------------------------------------ staging (one block per leaf)
constexpr int STAGE_THREADS = 256;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float round_up_rel(float v) { return v * 1.000001f + 1e-30f; }

// Four BF16 pieces whose sum is -v exactly (a binary32 value has 24 significant bits; every
// residual below is exact in binary32).
__device__ __forceinline__ uint2 neg_pieces_f32(float v) {
    float rest = -v;
    uint32_t b[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const __nv_bfloat16 h = __float2bfloat16_rn(rest);
        b[q] = __bfloat16_as_ushort(h);
        rest = __fsub_rn(rest, __bfloat162float(h));
    }
    return make_uint2(b[0] | (b[1] << 16), b[2] | (b[3] << 16));
}

template <int MET, int PREC>
__global__ void __launch_bounds__(STAGE_THREADS) leaf_stage_f32(const float *X, uint32_t d, const uint64_t *off,
                                                                const uint32_t *mem, uint64_t L, uint32_t row_bytes,
                                                                LeafInfoF *info, uint2 *pieces, float *rnorm,
                                                                unsigned char *staged) {
    __shared__ float mu[128];
    __shared__ float part[2][128], lo_s[2][128], hi_s[2][128];
    __shared__ float red[3][STAGE_THREADS / 32];
    __shared__ LeafInfoF li_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NW = STAGE_THREADS / 32;
    for (uint64_t b = blockIdx.x; b < L; b += gridDim.x) {
        const uint64_t o = off[b];
        const uint32_t s = (uint32_t)(off[b + 1] - o);
        // A: centroid and per-coordinate extent (two groups of 128 threads, members split by parity)
        {
            const uint32_t g = tid >> 7, t = tid & 127;
            float sum = 0.0f, lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
            if (t < d) {
#pragma unroll 4
                for (uint32_t jm = g; jm < s; jm += 2) {
                    const float v = X[(uint64_t)mem[o + jm] * d + t];
                    sum += v;
                    lo = fminf(lo, v);
                    hi = fmaxf(hi, v);
                }
            }
            part[g][t] = sum;
            lo_s[g][t] = lo;
            hi_s[g][t] = hi;
        }
        __syncthreads();
        float ext = 0.0f, mu2 = 0.0f;
        if (tid < 128) {
            const uint32_t t = tid;
            float m = 0.0f;
            if (t < d && s > 0) {
                m = __fdiv_rn(part[0][t] + part[1][t], (float)s);
                const float lo = fminf(lo_s[0][t], lo_s[1][t]), hi = fmaxf(hi_s[0][t], hi_s[1][t]);
                ext = fmaxf(__fsub_rn(hi, m), __fsub_rn(m, lo));
                mu2 = m * m;
            }
            mu[t] = m;
        }
        ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, 16));
        ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, 8));
        ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, 4));
        ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, 2));
        ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, 1));
        mu2 = warp_sum(mu2);
        if (lane == 0) {
            red[0][warp] = ext;
            red[1][warp] = mu2;
        }
        __syncthreads();
        // B: |x'| and (inner product) |x|^2 of every member, one warp per member
        float rmax = 0.0f, pmax = 0.0f;
        for (uint32_t jm = warp; jm < s; jm += NW) {
            const float *x = X + (uint64_t)mem[o + jm] * d;
            float sq = 0.0f, raw = 0.0f;
            for (uint32_t t = lane; t < d; t += 32) {
                const float v = x[t], c = __fsub_rn(v, mu[t]);
                sq = __fmaf_rn(c, c, sq);
                raw = __fmaf_rn(v, v, raw);
            }
            sq = warp_sum(sq);
            raw = warp_sum(raw);
            rmax = fmaxf(rmax, sqrtf(sq));
            pmax = fmaxf(pmax, raw);
        }
        if (lane == 0) red[2][warp] = rmax;
        __syncthreads();
        if (tid == 0) {
            float e = 0.0f, m2 = 0.0f, R = 0.0f;
            for (int w = 0; w < NW; w++) {
                e = fmaxf(e, red[0][w]);
                m2 += red[1][w];
                R = fmaxf(R, red[2][w]);
            }
            LeafInfoF li;
            li.R = round_up_rel(R);
            li.m = round_up_rel(sqrtf(m2));
            li.P = 0.0f;
            li.scale = (PREC == PREC_FP8 && e > 0.0f) ? __fdiv_rn(448.0f * (1.0f - 1.0f / 256.0f), e) : 1.0f;
            li_s = li;
        }
        __syncthreads();
        if (MET == PIPNN_IP) {
            // P = max |x|^2 over the leaf
            if (lane == 0) red[2][warp] = pmax;
            __syncthreads();
            if (tid == 0) {
                // offset P >= max(0, max |x|^2 - 1) (the binary32 norms are raised past their
                // rounding error), so D + P = 1 - <x_i, x_j> + P >= 1 - max |x|^2 + P >= 0
                float P = 0.0f;
                for (int w = 0; w < NW; w++) P = fmaxf(P, red[2][w]);
                li_s.P = fmaxf(__fsub_rn(P * 1.0000153f, 1.0f), 0.0f) + 1e-6f;
            }
            __syncthreads();
        }
        const LeafInfoF li = li_s;
        if (tid == 0) info[b] = li;
        const float sc = li.scale, sc2 = __fmul_rn(li.scale, li.scale);
        const float wbase = MET == PIPNN_IP ? 0.5f * (1.0f + li.m * li.m + li.P) : 0.0f;
        // C: the operand row, the -v pieces and |x'| of every member
        for (uint32_t jm = warp; jm < s; jm += NW) {
            const uint64_t row = o + jm;
            const float *x = X + (uint64_t)mem[row] * d;
            float sq = 0.0f, dot = 0.0f;
            for (uint32_t t = lane; t < d; t += 32) {
                const float v = x[t], c = __fsub_rn(v, mu[t]);
                sq = __fmaf_rn(c, c, sq);
                dot = __fmaf_rn(v, mu[t], dot);
            }
            sq = warp_sum(sq);
            dot = warp_sum(dot);
            // operand row: lane writes coordinates 4 lane .. 4 lane + 3 (zero past d)
            float c4[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t t = 4 * lane + q;
                c4[q] = t < d ? __fsub_rn(x[t], mu[t]) : 0.0f;
            }
            if (PREC == PREC_SPLIT) {
                // [hi (dp) | lo (dp)] with dp = row_bytes / 4 BF16 values per half
                const uint32_t dp = row_bytes / 4;
                uint32_t hw[2], lw[2];
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(c4[2 * q]), h1 = __float2bfloat16_rn(c4[2 * q + 1]);
                    const __nv_bfloat16 l0 = __float2bfloat16_rn(__fsub_rn(c4[2 * q], __bfloat162float(h0)));
                    const __nv_bfloat16 l1 = __float2bfloat16_rn(__fsub_rn(c4[2 * q + 1], __bfloat162float(h1)));
                    hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                    lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                }
                if (4 * lane < dp) {
                    uint2 *rowp = reinterpret_cast<uint2 *>(staged + row * row_bytes);
                    rowp[lane] = make_uint2(hw[0], hw[1]);
                    rowp[dp / 4 + lane] = make_uint2(lw[0], lw[1]);
                }
            } else if (PREC == PREC_FP8) {
                uint32_t w = 0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const __nv_fp8_storage_t e8 = __nv_cvt_float_to_fp8(__fmul_rn(sc, c4[q]), __NV_SATFINITE, __NV_E4M3);
                    w |= (uint32_t)e8 << (8 * q);
                }
                if (4 * lane < row_bytes) reinterpret_cast<uint32_t *>(staged + row * row_bytes)[lane] = w;
            } else {
                const uint32_t w0 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(c4[0])) |
                                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(c4[1])) << 16);
                const uint32_t w1 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(c4[2])) |
                                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(c4[3])) << 16);
                if (8 * lane < row_bytes)
                    reinterpret_cast<uint2 *>(staged + row * row_bytes)[lane] = make_uint2(w0, w1);
            }
            if (lane == 0) {
                const float v = MET == PIPNN_L2 ? __fmul_rn(sc2, 0.5f * sq) : __fmul_rn(sc2, __fsub_rn(wbase, dot));
                pieces[row] = neg_pieces_f32(v);
                rnorm[row] = round_up_rel(sqrtf(sq));
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ re-rank
// Dissimilarity in the defining binary32 order: one fused multiply-add per coordinate, index
// order (L2: of the differences; IP: 1 - the products' chain).
template <int MET, int NC>
__device__ __forceinline__ void defined_dis(const float *xi, const float *const (&xj)[NC], uint32_t d, uint32_t nc,
                                            float (&acc)[NC]) {
#pragma unroll
    for (int p = 0; p < NC; p++) acc[p] = 0.0f;
    for (uint32_t t = 0; t < d; t++) {
        const float a = __ldg(xi + t);
#pragma unroll
        for (int p = 0; p < NC; p++) {
            if ((uint32_t)p < nc) {
                const float b = __ldg(xj[p] + t);
                if (MET == PIPNN_L2) {
                    const float df = __fsub_rn(a, b);
                    acc[p] = __fmaf_rn(df, df, acc[p]);
                } else {
                    acc[p] = __fmaf_rn(a, b, acc[p]);
                }
            }
        }
    }
    if (MET == PIPNN_IP) {
#pragma unroll
        for (int p = 0; p < NC; p++) acc[p] = __fsub_rn(1.0f, acc[p]);
    }
}

// The same chain reading four coordinates per load (d a multiple of four: every row starts on a
// 16-byte boundary); the fused multiply-adds still run one coordinate at a time in index order.
template <int MET, int NC>
__device__ __forceinline__ void defined_dis4(const float *xi, const float *const (&xj)[NC], uint32_t d, uint32_t nc,
                                             float (&acc)[NC]) {
#pragma unroll
    for (int p = 0; p < NC; p++) acc[p] = 0.0f;
    for (uint32_t t = 0; t < d; t += 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(xi + t));
#pragma unroll
        for (int p = 0; p < NC; p++) {
            if ((uint32_t)p < nc) {
                const float4 b = __ldg(reinterpret_cast<const float4 *>(xj[p] + t));
                if (MET == PIPNN_L2) {
                    float df = __fsub_rn(a.x, b.x);
                    acc[p] = __fmaf_rn(df, df, acc[p]);
                    df = __fsub_rn(a.y, b.y);
                    acc[p] = __fmaf_rn(df, df, acc[p]);
                    df = __fsub_rn(a.z, b.z);
                    acc[p] = __fmaf_rn(df, df, acc[p]);
                    df = __fsub_rn(a.w, b.w);
                    acc[p] = __fmaf_rn(df, df, acc[p]);
                } else {
                    acc[p] = __fmaf_rn(a.x, b.x, acc[p]);
                    acc[p] = __fmaf_rn(a.y, b.y, acc[p]);
                    acc[p] = __fmaf_rn(a.z, b.z, acc[p]);
                    acc[p] = __fmaf_rn(a.w, b.w, acc[p]);
                }
            }
        }
    }
    if (MET == PIPNN_IP) {
#pragma unroll
        for (int p = 0; p < NC; p++) acc[p] = __fsub_rn(1.0f, acc[p]);
    }
}

__device__ __forceinline__ uint64_t dis_key(float D, uint32_t id) { return ((uint64_t)f32_order(D) << 32) | id; }

__device__ __forceinline__ void emit_pair(uint32_t *dst, uint32_t *src, float *dist, uint64_t w, uint32_t me,
                                          uint64_t key) {
    const uint32_t other = (uint32_t)key;
    const float D = f32_unorder((uint32_t)(key >> 32));
    dst[w] = me;
    src[w] = other;
    dist[w] = D;
    dst[w + 1] = other;
    src[w + 1] = me;
    dist[w + 1] = D;
}

// One block per unit, one thread per row: the row's listed candidates, evaluated exactly.
// vec4: d is a multiple of four and X starts on a 16-byte boundary (four coordinates per load).
template <int MET, int KP>
__global__ void __launch_bounds__(128) rerank_rows(const float *X, uint32_t d, bool vec4, const TcUnitF *units,
                                                   uint64_t nunits, const uint32_t *members, const uint16_t *cand,
                                                   const uint8_t *ccnt, uint32_t k, uint32_t *out_dst,
                                                   uint32_t *out_src, float *out_dist) {
    for (uint64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const TcUnitF un = units[u];
        const uint32_t row = un.row0 + threadIdx.x;
        if (row >= un.s) continue;
        const uint64_t g = un.off + row;
        const uint32_t c = ccnt[g];
        if (c == 0xFF) continue;  // evaluated in full by rerank_full
        const uint32_t kk = un.s - 1 < k ? un.s - 1 : k;
        if (kk == 0) continue;
        const uint32_t me = members[g];
        const float *xi = X + (uint64_t)me * d;
        const float *xj[KP];
        uint32_t id[KP];
#pragma unroll
        for (int p = 0; p < KP; p++) {
            id[p] = (uint32_t)p < c ? members[un.off + cand[g * KP + p]] : me;
            xj[p] = X + (uint64_t)id[p] * d;
        }
        float D[KP];
        if (vec4) defined_dis4<MET, KP>(xi, xj, d, c, D);
        else defined_dis<MET, KP>(xi, xj, d, c, D);
        uint64_t key[KP];
#pragma unroll
        for (int p = 0; p < KP; p++) key[p] = (uint32_t)p < c ? dis_key(D[p], id[p]) : ~0ull;
        // selection of the kk smallest (c <= KP is small)
        uint64_t w = un.out + (uint64_t)threadIdx.x * 2 * kk;
        for (uint32_t q = 0; q < kk; q++) {
            uint64_t best = ~0ull;
#pragma unroll
            for (int p = 0; p < KP; p++) best = min(best, key[p]);
#pragma unroll
            for (int p = 0; p < KP; p++)
                if (key[p] == best) key[p] = ~0ull;
            emit_pair(out_dst, out_src, out_dist, w, me, best);
            w += 2;
        }
    }
}

// One warp per listed row: every other member of the leaf, evaluated exactly; each lane keeps
// its 16 smallest (D, id), then the warp takes the kk smallest of all lanes.
template <int MET>
__global__ void __launch_bounds__(256) rerank_full(const float *X, uint32_t d, bool vec4, const TcUnitF *units,
                                                   const uint32_t *ovf, uint32_t novf, const uint32_t *members,
                                                   const uint32_t *simt_size, uint32_t k, uint32_t *out_dst,
                                                   uint32_t *out_src, float *out_dist) {
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t w_ = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; w_ < novf; w_ += nw) {
        const uint32_t e = ovf[w_];
        const TcUnitF un = units[e >> 7];
        if (simt_size[un.leaf]) continue;  // the whole leaf is evaluated on the CUDA cores
        const uint32_t r = e & 127u, row = un.row0 + r;
        const uint32_t kk = un.s - 1 < k ? un.s - 1 : k;
        const uint32_t me = members[un.off + row];
        const float *xi = X + (uint64_t)me * d;
        uint64_t best[16];
#pragma unroll
        for (int p = 0; p < 16; p++) best[p] = ~0ull;
        for (uint32_t jm = lane; jm < un.s; jm += 32) {
            if (jm == row) continue;
            const uint32_t id = members[un.off + jm];
            const float *xj[1] = {X + (uint64_t)id * d};
            float D[1];
            if (vec4) defined_dis4<MET, 1>(xi, xj, d, 1, D);
            else defined_dis<MET, 1>(xi, xj, d, 1, D);
            const uint64_t key = dis_key(D[0], id);
            if (key < best[15]) {
                best[15] = key;
#pragma unroll
                for (int p = 15; p > 0; p--) {
                    const uint64_t lo = min(best[p - 1], best[p]), hi = max(best[p - 1], best[p]);
                    best[p - 1] = lo;
                    best[p] = hi;
                }
            }
        }
        // warp-wide: kk rounds of "smallest head over the lanes"
        uint32_t head = 0;
        uint64_t w = un.out + (uint64_t)r * 2 * kk;
        for (uint32_t q = 0; q < kk; q++) {
            uint64_t h = ~0ull;
#pragma unroll
            for (int p = 0; p < 16; p++)
                if ((uint32_t)p == head) h = best[p];
            uint64_t m = h;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, (uint64_t)__shfl_xor_sync(0xffffffffu, m, o));
            if (h == m && m != ~0ull) head++;
            if (lane == 0) emit_pair(out_dst, out_src, out_dist, w, me, m);
            w += 2;
        }
    }
}

__global__ void build_units_f(const uint32_t *tile_grp, const uint32_t *tile_row0, uint64_t nunits,
                              const uint64_t *leaf_off, const uint64_t *cand_off, uint32_t k, TcUnitF *units) {
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < nunits; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = tile_grp[u];
        TcUnitF x;
        x.off = leaf_off[g];
        x.s = (uint32_t)(leaf_off[g + 1] - x.off);
        x.row0 = tile_row0[u];
        x.leaf = g;
        x.pad = 0;
        const uint32_t kk = x.s - 1 < k ? x.s - 1 : k;
        x.out = cand_off[g] + (uint64_t)x.row0 * 2 * kk;
        units[u] = x;
    }
}

// Leaves where more than one row in eight needs a full evaluation are evaluated whole by the
// CUDA-core all-pairs kernel (tiled, far cheaper per row than one warp per row).
__global__ void simt_leaves(const uint32_t *size, const unsigned *leaf_ovf, uint64_t L, uint32_t *simt_size) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < L; b += (uint64_t)gridDim.x * blockDim.x)
        simt_size[b] = (uint64_t)leaf_ovf[b] * 8 > size[b] ? size[b] : 0u;
}

__global__ void max_leaf_size(const uint32_t *size, uint64_t L, unsigned *out) {
    unsigned m = 0;
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < L; b += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, size[b]);
    atomicMax(out, m);
}

template <int PREC, int KB, int KP, bool DUMP = false>
int launch_tcf(const CUtensorMap &map, const TcfArgs &args, uint64_t ntiles, uint32_t ksteps) {
    using C = TcfCfg<PREC, KB, KP>;
    auto kern = leaf_gram_tcf<PREC, KB, KP, DUMP>;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int dev = 0, sms = 0;
    PIPNN_CUDA(cudaGetDevice(&dev));
    PIPNN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)(ntiles < (uint64_t)sms ? ntiles : (uint64_t)sms);
    kern<<<grid, THREADS, C::SMEM, stream()>>>(map, args, (uint32_t)ntiles, ksteps);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

template <int MET>
int launch_stage(int prec, const float *X, uint32_t d, const uint64_t *off, const uint32_t *mem, uint64_t L,
                 uint32_t row_bytes, LeafInfoF *info, uint2 *pieces, float *rnorm, unsigned char *staged) {
    const unsigned g = grid_for(L, 1, 152u * 8u);
    if (prec == PREC_FP8)
        leaf_stage_f32<MET, PREC_FP8><<<g, STAGE_THREADS, 0, stream()>>>(X, d, off, mem, L, row_bytes, info, pieces,
                                                                        rnorm, staged);
    else if (prec == PREC_SPLIT)
        leaf_stage_f32<MET, PREC_SPLIT><<<g, STAGE_THREADS, 0, stream()>>>(X, d, off, mem, L, row_bytes, info, pieces,
                                                                          rnorm, staged);
    else
        leaf_stage_f32<MET, PREC_BF16><<<g, STAGE_THREADS, 0, stream()>>>(X, d, off, mem, L, row_bytes, info, pieces,
                                                                         rnorm, staged);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

// The bound's coefficients (D units) for precision prec at dimension d.
BandCoef band_coefficients(int prec, uint32_t d, int metric) {
    const double uc = std::ldexp(1.0, -24);
    const double uq = prec == PREC_FP8 ? std::ldexp(1.0, -4) : std::ldexp(1.0, -8);
    const double a0 = prec == PREC_FP8 ? std::ldexp(1.0, -10) : 0.0;
    const double uacc = prec == PREC_FP8 ? std::ldexp(1.0, -11) : std::ldexp(1.0, -22);
    const uint32_t kstep = prec == PREC_FP8 ? 32 : 16;
    const uint32_t products = prec == PREC_SPLIT ? 3 : 1;
    const double steps = (double)(products * ((d + kstep - 1) / kstep) + 1);
    const double sd = std::sqrt((double)d);
    // |G~ - G| / sum |x_t y_t|: one rounding per operand, or for the split form x = hi + lo + e with
    // |e| <= 2^-16 |x| and |lo| <= 2^-8 (1 + 2^-8) |x| (the dropped lo.lo term included)
    const double gram = (prec == PREC_SPLIT ? 3.0 * std::ldexp(1.0, -16) + std::ldexp(1.0, -22)
                                            : 2.0 * uq + uq * uq) * (1.0 + 4.0 * uc);
    BandCoef c{};
    if (metric == PIPNN_L2) {
        // 2|dG| + |dn_i| + |dn_j| + accumulation + defining-order error + centring perturbation
        c.rR = (float)(2.0 * gram + 2.0 * steps * uacc * (1.0 + uq) * (1.0 + uq) * 1.02 + 2.0 * (d + 4) * uc + 8.0 * uc);
        c.sq = (float)((d + 6) * uc + steps * uacc + (d + 4) * uc + 4.0 * uc);
        c.lin = (float)(2.0 * a0 * (1.0 + uq) * sd);
        c.zero = (float)(2.0 * d * a0 * a0);
    } else {
        c.rR = (float)(gram + steps * uacc * (1.0 + uq) * (1.0 + uq) * 1.02);
        c.lin = (float)(a0 * (1.0 + uq) * sd);
        c.zero = (float)(d * a0 * a0);
        c.W = (float)(2.0 * (d + 6) * uc + 2.0 * steps * uacc);
        c.mm = (float)((d + 6) * uc);
        c.one = (float)(2.0 * uc);
    }
    c.safety = 1.25f;
    return c;
}

__global__ void gram_sizes(const uint32_t *size, uint64_t L, uint64_t *sq) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < L; b += (uint64_t)gridDim.x * blockDim.x)
        sq[b] = (uint64_t)size[b] * size[b];
}

__global__ void sizes_of(const uint64_t *off, uint64_t L, uint32_t *size) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < L; b += (uint64_t)gridDim.x * blockDim.x)
        size[b] = (uint32_t)(off[b + 1] - off[b]);
}

}  // namespace

// The approximate dissimilarities of the reduced-precision engine, before any re-rank: for leaf b
// the |b| x |b| block gram[sum_{c<b} |c|^2 ..] (row = member i, column = member j, both in the
// leaf's member order).  For the FP64 error reports and the error-bound tests.
int leaf_gram_tcf(const float *X, uint32_t d, int metric, int prec, const uint64_t *off, const uint32_t *mem,
                  uint64_t L, float *gram, Workspace &ws) {
    if (prec != PREC_BF16 && prec != PREC_FP8 && prec != PREC_SPLIT)
        return set_error(PIPNN_EUNSUPPORTED, "the reduced-precision leaf engine takes BF16, FP8 or BF16X3");
    if (d > 128) return set_error(PIPNN_EUNSUPPORTED, "the reduced-precision leaf engine takes d <= 128");
    uint64_t M = 0;
    PIPNN_TRY(read_u64(off + L, &M));
    if (M == 0 || L == 0) return PIPNN_OK;
    if (M >= 0x7FFFFF00ull) return set_error(PIPNN_EUNSUPPORTED, "the tensor-core leaf engine takes < 2^31 leaf members");
    uint32_t *size;
    uint64_t *goff, *tot;
    PIPNN_TRY(ws.alloc(&size, L));
    PIPNN_TRY(ws.alloc(&goff, L));
    PIPNN_TRY(ws.alloc(&tot, 1));
    sizes_of<<<grid_for(L, 256), 256, 0, stream()>>>(off, L, size);
    PIPNN_LAUNCH_CHECK();
    gram_sizes<<<grid_for(L, 256), 256, 0, stream()>>>(size, L, goff);
    PIPNN_LAUNCH_CHECK();
    PIPNN_TRY(exclusive_scan_u64(goff, goff, L, tot, ws));
    const uint32_t KB = prec == PREC_FP8 ? 1 : (d + 63) / 64;
    // 64 BF16 or 128 e4m3 values per K block; the split form stores a hi and a lo half
    const uint32_t row_bytes = 128 * KB * (prec == PREC_SPLIT ? 2 : 1);
    const uint32_t ksteps = prec == PREC_FP8 ? (d + 31) / 32 : (d + 15) / 16;
    LeafInfoF *info;
    uint2 *pieces;
    float *rnorm;
    unsigned char *staged;
    PIPNN_TRY(ws.alloc(&info, L));
    PIPNN_TRY(ws.alloc(&pieces, M));
    PIPNN_TRY(ws.alloc(&rnorm, M));
    PIPNN_TRY(ws.alloc(&staged, M * row_bytes));
    if (metric == PIPNN_L2) PIPNN_TRY(launch_stage<PIPNN_L2>(prec, X, d, off, mem, L, row_bytes, info, pieces, rnorm, staged));
    else PIPNN_TRY(launch_stage<PIPNN_IP>(prec, X, d, off, mem, L, row_bytes, info, pieces, rnorm, staged));
    uint32_t *tile_grp = nullptr, *tile_row0 = nullptr;
    uint64_t ntiles = 0;
    PIPNN_TRY(make_tiles(size, L, ROWS, &tile_grp, &tile_row0, &ntiles, ws));
    TcUnitF *units;
    PIPNN_TRY(ws.alloc(&units, ntiles));
    build_units_f<<<grid_for(ntiles, 256), 256, 0, stream()>>>(tile_grp, tile_row0, ntiles, off, goff, 0, units);
    PIPNN_LAUNCH_CHECK();
    CUtensorMap map;
    if (prec == PREC_FP8) PIPNN_TRY(encode_bytes_map(&map, staged, M, row_bytes));
    else PIPNN_TRY(encode_rows_map(&map, reinterpret_cast<const __nv_bfloat16 *>(staged), M, row_bytes / 2, false));
    TcfArgs a{};
    a.units = units;
    a.pieces = pieces;
    a.rnorm = rnorm;
    a.info = info;
    a.metric = metric;
    a.colbits = 16;
    a.err = device_error_word();
    a.gram = gram;
    a.gram_off = goff;
    if (prec == PREC_FP8) return launch_tcf<PREC_FP8, 1, 4, true>(map, a, ntiles, ksteps);
    if (prec == PREC_SPLIT)
        return KB == 1 ? launch_tcf<PREC_SPLIT, 1, 4, true>(map, a, ntiles, ksteps)
                       : launch_tcf<PREC_SPLIT, 2, 4, true>(map, a, ntiles, ksteps);
    if (KB == 1) return launch_tcf<PREC_BF16, 1, 4, true>(map, a, ntiles, ksteps);
    return launch_tcf<PREC_BF16, 2, 4, true>(map, a, ntiles, ksteps);
}

// A2..A4 for float data on the reduced-precision tensor-core engine (see the file comment).
// X: n x d float32 device; off/mem: leaves; leaf_size/cand_off: per-leaf size and first output
// slot; writes 2 |b| min(k, |b| - 1) edges per leaf.  *fallback_rows receives the number of rows
// whose band overflowed the tracked keys (evaluated in full).
int leaf_pick_tcf(const float *X, uint64_t n, uint32_t d, int metric, int prec, const uint64_t *off,
                  const uint32_t *mem, uint64_t L, const uint32_t *leaf_size, const uint64_t *cand_off, uint32_t k,
                  uint32_t *out_dst, uint32_t *out_src, float *out_dist, Workspace &ws, cudaEvent_t ev0,
                  cudaEvent_t ev1, uint32_t *launches, uint64_t *fallback_rows) {
    (void)n;
    if (prec != PREC_BF16 && prec != PREC_FP8 && prec != PREC_SPLIT)
        return set_error(PIPNN_EUNSUPPORTED, "the reduced-precision leaf engine takes BF16, FP8 or BF16X3");
    if (d > 128) return set_error(PIPNN_EUNSUPPORTED, "the reduced-precision leaf engine takes d <= 128");
    if (k > 16) return set_error(PIPNN_EINVAL, "k above 16");
    *launches = 0;
    if (fallback_rows) *fallback_rows = 0;
    uint64_t M = 0;
    PIPNN_TRY(read_u64(off + L, &M));
    if (M == 0 || L == 0) return PIPNN_OK;
    if (M >= 0x7FFFFF00ull) return set_error(PIPNN_EUNSUPPORTED, "the tensor-core leaf engine takes < 2^31 leaf members");
    unsigned *dmax;
    PIPNN_TRY(ws.zeros(&dmax, 1));
    max_leaf_size<<<grid_for(L, 256), 256, 0, stream()>>>(leaf_size, L, dmax);
    PIPNN_LAUNCH_CHECK();
    unsigned smax = 0;
    PIPNN_CUDA(cudaMemcpyAsync(&smax, dmax, 4, cudaMemcpyDeviceToHost, stream()));
    PIPNN_CUDA(cudaStreamSynchronize(stream()));
    if (smax > 65536) return set_error(PIPNN_EUNSUPPORTED, "the reduced-precision leaf engine takes leaves of <= 65536");
    uint32_t colbits = 1;
    while ((1u << colbits) < smax) colbits++;
    if (colbits < 7) colbits = 7;

    const uint32_t KB = prec == PREC_FP8 ? 1 : (d + 63) / 64;
    // 64 BF16 or 128 e4m3 values per K block; the split form stores a hi and a lo half
    const uint32_t row_bytes = 128 * KB * (prec == PREC_SPLIT ? 2 : 1);
    const uint32_t ksteps = prec == PREC_FP8 ? (d + 31) / 32 : (d + 15) / 16;
    LeafInfoF *info;
    uint2 *pieces;
    float *rnorm;
    unsigned char *staged;
    PIPNN_TRY(ws.alloc(&info, L));
    PIPNN_TRY(ws.alloc(&pieces, M));
    PIPNN_TRY(ws.alloc(&rnorm, M));
    PIPNN_TRY(ws.alloc(&staged, M * row_bytes));  // every byte of every row is written by the staging
    if (metric == PIPNN_L2) PIPNN_TRY(launch_stage<PIPNN_L2>(prec, X, d, off, mem, L, row_bytes, info, pieces, rnorm, staged));
    else PIPNN_TRY(launch_stage<PIPNN_IP>(prec, X, d, off, mem, L, row_bytes, info, pieces, rnorm, staged));

    uint32_t *tile_grp = nullptr, *tile_row0 = nullptr;
    uint64_t ntiles = 0;
    PIPNN_TRY(make_tiles(leaf_size, L, ROWS, &tile_grp, &tile_row0, &ntiles, ws));
    if (ntiles >= (1ull << 25)) return set_error(PIPNN_EUNSUPPORTED, "too many leaf tiles for one launch");
    TcUnitF *units;
    PIPNN_TRY(ws.alloc(&units, ntiles));
    build_units_f<<<grid_for(ntiles, 256), 256, 0, stream()>>>(tile_grp, tile_row0, ntiles, off, cand_off, k, units);
    PIPNN_LAUNCH_CHECK();

    const int KP = prec == PREC_BF16 ? (k <= 2 ? 4 : (k <= 4 ? 8 : 16)) : (k <= 2 ? 8 : 16);
    uint16_t *cand;
    uint8_t *ccnt;
    uint32_t *ovf;
    unsigned *novf;
    PIPNN_TRY(ws.alloc(&cand, M * KP));
    PIPNN_TRY(ws.alloc(&ccnt, M));
    unsigned *leaf_ovf;
    uint32_t *simt_size;
    PIPNN_TRY(ws.alloc(&ovf, M));
    PIPNN_TRY(ws.zeros(&novf, 1));
    PIPNN_TRY(ws.zeros(&leaf_ovf, L));
    PIPNN_TRY(ws.alloc(&simt_size, L));

    CUtensorMap map;
    if (prec == PREC_FP8) PIPNN_TRY(encode_bytes_map(&map, staged, M, row_bytes));
    else PIPNN_TRY(encode_rows_map(&map, reinterpret_cast<const __nv_bfloat16 *>(staged), M, row_bytes / 2, false));
    TcfArgs a{};
    a.units = units;
    a.pieces = pieces;
    a.rnorm = rnorm;
    a.info = info;
    a.bc = band_coefficients(prec, d, metric);
    a.metric = metric;
    a.colbits = colbits;
    a.k = k;
    a.cand = cand;
    a.ccnt = ccnt;
    a.ovf = ovf;
    a.novf = novf;
    a.leaf_ovf = leaf_ovf;
    a.err = device_error_word();

    cudaEventRecord(ev0, stream());
    int rc;
    if (prec == PREC_FP8) {
        rc = KP == 8 ? launch_tcf<PREC_FP8, 1, 8>(map, a, ntiles, ksteps) : launch_tcf<PREC_FP8, 1, 16>(map, a, ntiles, ksteps);
    } else if (prec == PREC_SPLIT) {
        if (KB == 1)
            rc = KP == 8 ? launch_tcf<PREC_SPLIT, 1, 8>(map, a, ntiles, ksteps)
                         : launch_tcf<PREC_SPLIT, 1, 16>(map, a, ntiles, ksteps);
        else
            rc = KP == 8 ? launch_tcf<PREC_SPLIT, 2, 8>(map, a, ntiles, ksteps)
                         : launch_tcf<PREC_SPLIT, 2, 16>(map, a, ntiles, ksteps);
    } else if (KB == 1) {
        rc = KP == 4 ? launch_tcf<PREC_BF16, 1, 4>(map, a, ntiles, ksteps)
                     : KP == 8 ? launch_tcf<PREC_BF16, 1, 8>(map, a, ntiles, ksteps)
                               : launch_tcf<PREC_BF16, 1, 16>(map, a, ntiles, ksteps);
    } else {
        rc = KP == 4 ? launch_tcf<PREC_BF16, 2, 4>(map, a, ntiles, ksteps)
                     : KP == 8 ? launch_tcf<PREC_BF16, 2, 8>(map, a, ntiles, ksteps)
                               : launch_tcf<PREC_BF16, 2, 16>(map, a, ntiles, ksteps);
    }
    cudaEventRecord(ev1, stream());
    PIPNN_TRY(rc);
    *launches = 1;

    // exact re-rank of the listed candidates, then the rows listed for a full evaluation
    const unsigned gr = grid_for(ntiles, 1, 152u * 16u);
    const bool vec4 = (d & 3u) == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
    if (metric == PIPNN_L2) {
        if (KP == 4) rerank_rows<PIPNN_L2, 4><<<gr, 128, 0, stream()>>>(X, d, vec4, units, ntiles, mem, cand, ccnt, k, out_dst, out_src, out_dist);
        else if (KP == 8) rerank_rows<PIPNN_L2, 8><<<gr, 128, 0, stream()>>>(X, d, vec4, units, ntiles, mem, cand, ccnt, k, out_dst, out_src, out_dist);
        else rerank_rows<PIPNN_L2, 16><<<gr, 128, 0, stream()>>>(X, d, vec4, units, ntiles, mem, cand, ccnt, k, out_dst, out_src, out_dist);
    } else {
        if (KP == 4) rerank_rows<PIPNN_IP, 4><<<gr, 128, 0, stream()>>>(X, d, vec4, units, ntiles, mem, cand, ccnt, k, out_dst, out_src, out_dist);
        else if (KP == 8) rerank_rows<PIPNN_IP, 8><<<gr, 128, 0, stream()>>>(X, d, vec4, units, ntiles, mem, cand, ccnt, k, out_dst, out_src, out_dist);
        else rerank_rows<PIPNN_IP, 16><<<gr, 128, 0, stream()>>>(X, d, vec4, units, ntiles, mem, cand, ccnt, k, out_dst, out_src, out_dist);
    }
    PIPNN_LAUNCH_CHECK();
    unsigned hovf = 0;
    PIPNN_CUDA(cudaMemcpyAsync(&hovf, novf, 4, cudaMemcpyDeviceToHost, stream()));
    PIPNN_CUDA(cudaStreamSynchronize(stream()));
    if (hovf) {
        simt_leaves<<<grid_for(L, 256), 256, 0, stream()>>>(leaf_size, leaf_ovf, L, simt_size);
        PIPNN_LAUNCH_CHECK();
        const unsigned gf = grid_for((uint64_t)hovf * 32, 256);
        if (metric == PIPNN_L2)
            rerank_full<PIPNN_L2><<<gf, 256, 0, stream()>>>(X, d, vec4, units, ovf, hovf, mem, simt_size, k, out_dst, out_src,
                                                            out_dist);
        else
            rerank_full<PIPNN_IP><<<gf, 256, 0, stream()>>>(X, d, vec4, units, ovf, hovf, mem, simt_size, k, out_dst, out_src,
                                                            out_dist);
        PIPNN_LAUNCH_CHECK();
        uint32_t *sg = nullptr, *sr = nullptr;
        uint64_t nst = 0;
        PIPNN_TRY(make_tiles(simt_size, L, AP_ROWS, &sg, &sr, &nst, ws));
        if (nst) {
            AllPairsArgs ap{};
            ap.X = X;
            ap.d = d;
            ap.tile_grp = sg;
            ap.tile_row0 = sr;
            ap.leaf_off = off;
            ap.members = mem;
            ap.cand_off = cand_off;
            ap.k = k;
            ap.out_dst = out_dst;
            ap.out_src = out_src;
            ap.out_dist = out_dist;
            PIPNN_TRY(launch_allpairs<MODE_PICK>(PIPNN_F32, metric, k, ap, nst));
        }
    }
    if (fallback_rows) *fallback_rows = hovf;
    return PIPNN_OK;
}

}  // namespace pipnn
