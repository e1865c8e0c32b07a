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
// Tiles.  Most reservoirs of a build are small (after duplicate candidates collapse, a node keeps
// ~20), so nodes with at most 31 valid candidates are packed four to a 128-row tile: node q owns
// rows 32q .. 32q + c_q (its candidates, then itself), i.e. exactly TMEM lane quarter q, and the
// columns it needs are the same 32.  The 128 x 128 Gram of a packed tile costs the tensor cores
// little; only its four diagonal 32 x 32 blocks are read.  Nodes with 32 .. 63 candidates (most of
// them in builds of 100M points, whose reservoirs fill further) go two to a tile: node h owns rows
// and columns 64h .. 64h + c_h, TMEM lane quarters 2h and 2h + 1, and the group's two warps on
// those quarters handle it.  A larger node gets a tile of its own.
//
// Persistent CTA (one per SM, 16 warps):
//   warps 0-11   epilogue: three groups of four warps (one per TMEM lane quarter) take turns on
//                tiles.  In a packed tile each warp handles its quarter's node alone (norms,
//                D(x, .), thresholds, ranks, masks, walk, output) with warp-level sync only; a
//                large node is handled by the group together (named barrier) and walked by one
//                of its warps.
//   warp 12      owns TMEM (4 x 128 columns); one thread issues the Gram MMAs
//   warp 13      node info: reservoir rows copied eight nodes ahead (cp.async ring), compaction
//                of the valid ids, packing; writes the tile sequence, ended by one end marker per
//                consumer
//   warps 14-15  TMA gather4 of the rows of alternate tiles
// A warp reaches TMEM lanes 32 (w % 4) .. +31 and runs on scheduler w % 4; the single-warp roles
// sit one on each scheduler.  Waits are bounded as in the other engines (DERR_TIMEOUT; TMEM is
// still released).
#include "tc_common.cuh"

namespace pipnn {

namespace {

using namespace tc;

constexpr int PT_GROUPS = 3;                 // epilogue groups of 4 warps: warps 0 .. 11
constexpr int PT_EPI_WARPS = 4 * PT_GROUPS;
constexpr int PT_MMA_WARP = 12;
constexpr int PT_INFO_WARP = 13;
constexpr int PT_GATHER_WARP0 = 14;          // and 15
constexpr int PT_GATHERERS = 2;
constexpr int PT_THREADS = 16 * 32;
constexpr uint32_t PT_MAXC = 127;            // candidates per node (+ the node)
constexpr uint32_t PT_SMALL = 31;            // packed nodes: at most this many valid candidates
constexpr uint32_t PT_MEDIUM = 63;           // two to a tile: at most this many
constexpr uint32_t PT_ENDS = PT_GROUPS > PT_GATHERERS ? PT_GROUPS : PT_GATHERERS;  // end markers

enum : uint32_t { TK_PACK = 1, TK_LARGE = 2, TK_END = 3, TK_MED = 4 };

struct PtArgs {
    const uint64_t *res;   // n x l_max reservoir slots
    const uint32_t *cnt;   // entries per reservoir
    const int32_t *sqn;    // exact squared norms
    uint64_t n;
    uint32_t l_max, R;
    float alpha2, inv_alpha2;
    uint32_t *adj, *deg;
    unsigned *err;
    uint32_t medium;  // largest candidate count that goes two to a tile (PT_SMALL: none do)
};

// Tile info, info warp -> gathers, MMA, epilogue: row ids (a packed node's rows start at 32q; the
// row after its candidates is the node itself), BF16 keys of the candidate rows, and
// misc = {kind, nodes, (c_q, v_q, n_x q) for q < 4}.
constexpr int I_IDS = 0, I_BKEY = 512, I_MISC = 768, I_BYTES = 832;
constexpr int M_KIND = 0, M_NODES = 1, M_NODE = 2;  // node q: misc[2 + 3q + {0, 1, 2}] = c, v, n_x

template <int KB>
struct PtCfg {
    static constexpr int A = 4;            // gathered row tiles in flight
    static constexpr int T = 4;            // accumulator buffers
    static constexpr int I = 8;            // tile-info slots (info and gathers run ahead)
    static constexpr int OFF_A0 = 0;
    static constexpr int OFF_INFO = OFF_A0 + A * KB * REGION;
    static constexpr int OFF_STAGE = OFF_INFO + I * I_BYTES;          // the info warp's packed tile
    static constexpr int OFF_STAGE2 = OFF_STAGE + I_BYTES;            // and its two-node tile
    // per group (large nodes): column masks 128 x 4 u32, ids 128, order 128 u8, D(x, .) 128,
    // n / 2 128 floats
    static constexpr int G_MASK = 0, G_IDS = 2048, G_ORDER = 2560, G_DX = 2688, G_HN = 3200, G_BYTES = 3712;
    static constexpr int OFF_GROUP = OFF_STAGE2 + I_BYTES;
    // per epilogue warp (packed nodes): D(x, .) 32, n / 2 32 floats, order 32 u8
    static constexpr int W_DX = 0, W_HN = 128, W_ORDER = 256, W_BYTES = 288;
    static constexpr int OFF_WARP = OFF_GROUP + PT_GROUPS * G_BYTES;
    // the info warp's prefetch ring: per node its reservoir row (up to 128 slots), count and norm
    static constexpr int P = 16;                                      // nodes in flight (<= 32)
    static constexpr int P_KEYS = 0, P_CNT = 1024, P_NRM = 1028, P_BYTES = 1040;
    static constexpr int OFF_PRE = OFF_WARP + PT_EPI_WARPS * W_BYTES;
    static constexpr int OFF_BAR = OFF_PRE + P * P_BYTES;
    static constexpr int BAR_FULL_A = 0, BAR_EMPTY_A = A, BAR_CFULL = 2 * A, BAR_IEMPTY = 2 * A + I,
                         BAR_TFULL = 2 * A + 2 * I, BAR_TEMPTY = 2 * A + 2 * I + T, NBAR = 2 * A + 2 * I + 2 * T;
    static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;               // tmem base, abort flag
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr int SMEM = BYTES + 1024;
    static_assert(SMEM <= 232448, "shared memory budget");
    static_assert(T * 128 <= (int)TMEM_COLS, "TMEM budget");
    static_assert(I_BYTES % 16 == 0 && G_BYTES % 16 == 0 && W_BYTES % 16 == 0 && P_BYTES % 16 == 0, "alignment");
    static_assert(I >= (int)PT_ENDS, "end markers fit the ring");
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

// Rank of candidate r among c in (D(x, .), id, slot) order: the start of its run of equal BF16
// keys plus its place inside the run, or (full) a count over all c.
__device__ __forceinline__ uint32_t candidate_rank(uint32_t r, uint32_t c, uint32_t DX, uint32_t id,
                                                   const uint32_t *dx, const uint32_t *ids, const uint16_t *bkey,
                                                   bool full) {
    uint32_t lo = 0;
    if (!full) {
        lo = r;
        while (lo > 0 && bkey[lo - 1] == bkey[r]) lo--;
    }
    uint32_t rank = lo;
    for (uint32_t s = lo; s < c && (full || bkey[s] == bkey[r]); s++) {
        const uint32_t ds = dx[s], is = ids[s];
        rank += (ds < DX || (ds == DX && (is < id || (is == id && s < r)))) ? 1u : 0u;
    }
    return rank;
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
    auto info = [&](uint32_t ib) { return smem + C::OFF_INFO + ib * I_BYTES; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t n = a.n;
    const uint32_t R = a.R;

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
        // ------------------------------------------------------------ tile info (one warp)
        // Prefetch: the reservoir row, count and norm of node j + P are copied (cp.async, no
        // registers in flight) into ring slot (j + P) % P while node j is compacted.
        // node j of this CTA: blockIdx.x + j * gridDim.x (n past the last)
        auto node_at = [&](uint32_t j) {
            const uint64_t v = blockIdx.x + (uint64_t)j * gridDim.x;
            return v < n ? v : n;
        };
        auto fetch = [&](uint32_t j) {
            const uint64_t v = node_at(j);
            if (v < n) {
                const uint32_t slot = sbase + C::OFF_PRE + (j % C::P) * C::P_BYTES;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t s_ = 32 * k + lane;
                    if (s_ < a.l_max) cp_async8(slot + C::P_KEYS + 8 * s_, a.res + v * a.l_max + s_);
                }
                if (lane == 0) {
                    cp_async4(slot + C::P_CNT, a.cnt + v);
                    cp_async4(slot + C::P_NRM, a.sqn + v);
                }
            }
            cp_async_commit();  // one group per node, empty past the end
        };
        unsigned char *stage = smem + C::OFF_STAGE, *stage2 = smem + C::OFF_STAGE2;
        uint32_t tile = 0, packed = 0, paired = 0;  // tiles written; nodes in the two staged tiles
        bool stop = false;
        // the next tile slot; false if the kernel aborted
        auto acquire = [&]() {
            return __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_IEMPTY + tile % C::I), ((tile / C::I) & 1) ^ 1,
                                                     abort, a.err));
        };
        auto publish = [&]() {
            __syncwarp();
            mbar_arrive(bar(C::BAR_CFULL + tile % C::I));
            tile++;
        };
        auto flush_staged = [&](unsigned char *st, uint32_t kind, uint32_t &count) {
            if (lane == 0) {
                reinterpret_cast<uint32_t *>(st + I_MISC)[M_KIND] = kind;
                reinterpret_cast<uint32_t *>(st + I_MISC)[M_NODES] = count;
            }
            __syncwarp();
            if (!acquire()) return false;
            const uint4 *srcv = reinterpret_cast<const uint4 *>(st);
            uint4 *dstv = reinterpret_cast<uint4 *>(info(tile % C::I));
            for (int q = lane; q < I_BYTES / 16; q += 32) dstv[q] = srcv[q];
            publish();
            count = 0;
            return true;
        };
        auto flush_packed = [&]() { return flush_staged(stage, TK_PACK, packed); };
        auto flush_paired = [&]() { return flush_staged(stage2, TK_MED, paired); };
        for (uint32_t j = 0; j < (uint32_t)C::P; j++) fetch(j);
        for (uint32_t j = 0; !stop; j++) {
            const uint64_t v = node_at(j);
            if (v >= n) break;
            cp_async_wait<C::P - 1>();  // node j's group (every later one may still be in flight)
            __syncwarp();
            const unsigned char *pre = smem + C::OFF_PRE + (j % C::P) * C::P_BYTES;
            const uint32_t c0 = *reinterpret_cast<const uint32_t *>(pre + C::P_CNT);
            const uint32_t pc = c0 < a.l_max ? c0 : a.l_max;
            const int32_t pnv = *reinterpret_cast<const int32_t *>(pre + C::P_NRM);
            uint64_t key[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t s = 32 * k + lane;
                key[k] = s < pc ? reinterpret_cast<const uint64_t *>(pre + C::P_KEYS)[s] : 0ull;
            }
            __syncwarp();
            fetch(j + C::P);  // the slot is free again
            // valid candidates (id < n), in slot order
            uint32_t cc = 0;
            bool in_range[4] = {false, false, false, false};
            uint32_t pos[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (32u * k >= pc) break;  // uniform: most reservoirs need one round
                const uint32_t s = 32 * k + lane;
                const uint32_t id = (uint32_t)(key[k] >> 16);
                in_range[k] = s < pc && (uint64_t)id < n;
                if (s < pc && !in_range[k]) atomicOr(a.err, DERR_RANGE);
                const unsigned m = __ballot_sync(0xffffffffu, in_range[k]);
                pos[k] = cc + __popc(m & ((1u << lane) - 1u));
                cc += __popc(m);
            }
            unsigned char *dst;
            uint32_t row0;
            if (cc <= PT_SMALL) {
                dst = stage;
                row0 = 32 * packed;
            } else if (cc <= a.medium) {
                dst = stage2;
                row0 = 64 * paired;
            } else {
                // a large node: its own tile, written straight into the ring
                if (!acquire()) {
                    stop = true;
                    break;
                }
                dst = info(tile % C::I);
                row0 = 0;
            }
            uint32_t *ids = reinterpret_cast<uint32_t *>(dst + I_IDS);
            uint16_t *bkey = reinterpret_cast<uint16_t *>(dst + I_BKEY);
            uint32_t *misc = reinterpret_cast<uint32_t *>(dst + I_MISC);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (in_range[k]) {
                    ids[row0 + pos[k]] = (uint32_t)(key[k] >> 16);
                    bkey[row0 + pos[k]] = (uint16_t)(key[k] >> 48);
                }
            }
            if (lane == 0) {
                ids[row0 + cc] = (uint32_t)v;
                const uint32_t q = cc <= PT_SMALL ? packed : cc <= a.medium ? paired : 0;
                misc[M_NODE + 3 * q + 0] = cc;
                misc[M_NODE + 3 * q + 1] = (uint32_t)v;
                misc[M_NODE + 3 * q + 2] = (uint32_t)pnv;
                if (cc > a.medium) {
                    misc[M_KIND] = TK_LARGE;
                    misc[M_NODES] = 1;
                }
            }
            if (cc <= PT_SMALL) {
                __syncwarp();
                if (++packed == 4 && !flush_packed()) stop = true;
            } else if (cc <= a.medium) {
                __syncwarp();
                if (++paired == 2 && !flush_paired()) stop = true;
            } else {
                publish();
            }
        }
        cp_async_wait<0>();  // no copy outlives the warp's loop
        if (!stop && packed > 0 && !flush_packed()) stop = true;
        if (!stop && paired > 0 && !flush_paired()) stop = true;
        // one end marker for every consumer that walks the tiles in a stride
        for (uint32_t e = 0; e < PT_ENDS && !stop; e++) {
            if (!acquire()) break;
            if (lane == 0) reinterpret_cast<uint32_t *>(info(tile % C::I) + I_MISC)[M_KIND] = TK_END;
            publish();
        }
    } else if (warp == PT_MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t issued = 0;
            bool any = false, stop = false;
            for (uint32_t k = 0;; k++) {
                const uint32_t ua = k % C::A, tb = k % C::T, ib = k % C::I;
                if (!mbar_wait(bar(C::BAR_CFULL + ib), (k / C::I) & 1, abort, a.err)) {
                    stop = true;
                    break;
                }
                const uint32_t *misc = reinterpret_cast<const uint32_t *>(info(ib) + I_MISC);
                const uint32_t kind = misc[M_KIND];
                if (kind == TK_END) break;
                if (!mbar_wait(bar(C::BAR_FULL_A + ua), (k / C::A) & 1, abort, a.err) ||
                    !mbar_wait(bar(C::BAR_TEMPTY + tb), ((k / C::T) & 1) ^ 1, abort, a.err)) {
                    stop = true;
                    break;
                }
                fence_after();
                const uint32_t ncol = kind != TK_LARGE ? 128u : ((misc[M_NODE] + 1 + 15) & ~15u);
                const uint32_t idesc = idesc_bf16(128, ncol);
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
                issued = k;
            }
            if (stop && any) mbar_wait(bar(C::BAR_TFULL + issued % C::T), (issued / C::T) & 1, abort, a.err);
        }
        __syncwarp();
    } else if (warp < PT_EPI_WARPS) {
        // ------------------------------------------------------------ epilogue (groups of 4 warps)
        const uint32_t grp = warp >> 2;                 // group: tiles k = grp, grp + PT_GROUPS, ...
        const int quarter = warp & 3;                   // TMEM lane quarter this warp may access
        const uint32_t r = quarter * 32 + lane;         // row of the tile
        const uint32_t bar_id = 1 + grp;
        unsigned char *gs = smem + C::OFF_GROUP + grp * C::G_BYTES;
        unsigned char *wsm = smem + C::OFF_WARP + warp * C::W_BYTES;
        for (uint32_t k = grp;; k += PT_GROUPS) {
            const uint32_t tb = k % C::T, ib = k % C::I;
            // the tile kind first (an end marker is never followed by an accumulator), then one
            // decision for the whole group, so that its warps always meet the same named barriers
            bool ok = __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_CFULL + ib), (k / C::I) & 1, abort, a.err));
            const unsigned char *in = info(ib);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(in + I_IDS);
            const uint16_t *bkey = reinterpret_cast<const uint16_t *>(in + I_BKEY);
            const uint32_t *misc = reinterpret_cast<const uint32_t *>(in + I_MISC);
            const uint32_t kind = ok ? misc[M_KIND] : 0u;
            if (ok && kind != TK_END)
                ok = __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_TFULL + tb), (k / C::T) & 1, abort, a.err));
            if (named_barrier_or(bar_id, 128, !ok) || kind == TK_END) break;
            fence_after();
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + tb * 128;

            if (kind == TK_PACK) {
                // ---- this warp's node, alone: rows and columns 32q .. 32q + c
                const uint32_t nodes = misc[M_NODES];
                if ((uint32_t)quarter < nodes) {
                    const uint32_t c = misc[M_NODE + 3 * quarter + 0];
                    const uint64_t v = misc[M_NODE + 3 * quarter + 1];
                    const float nx = (float)(int32_t)misc[M_NODE + 3 * quarter + 2];
                    const uint32_t *nid = ids + 32 * quarter;
                    const uint16_t *nkey = bkey + 32 * quarter;
                    uint32_t *wdx = reinterpret_cast<uint32_t *>(wsm + C::W_DX);
                    float *whn = reinterpret_cast<float *>(wsm + C::W_HN);
                    unsigned char *word = wsm + C::W_ORDER;
                    uint32_t g[32];
                    tmem_ld32(trow + quarter * 32, g);
                    const bool valid = (uint32_t)lane < c;
                    const float nr = __uint_as_float(pick32(g, lane));  // diagonal: exact integer
                    const float gx = __uint_as_float(pick32(g, c));
                    const float dxf = __fmaf_rn(-2.0f, gx, nr + nx);   // exact integer < 2^24
                    const uint32_t DX = valid ? (uint32_t)dxf : 0u;
                    const uint32_t T = removal_threshold(DX, a.alpha2, a.inv_alpha2);
                    const float theta = (nr - (float)T) * 0.5f;         // exact
                    wdx[lane] = DX;
                    whn[lane] = 0.5f * nr;
                    const bool bad =
                        valid && (bf16_key(dxf) != nkey[lane] || (lane > 0 && nkey[lane - 1] > nkey[lane]));
                    const bool full = __any_sync(0xffffffffu, bad);
                    __syncwarp();  // every lane's D(x, .) and n / 2 are visible
                    if (valid) word[candidate_rank(lane, c, DX, nid[lane], wdx, nid, nkey, full)] = (unsigned char)lane;
                    // column mask: candidates y < c (not itself) with G[r][y] - n_y / 2 > theta
                    uint32_t m = 0;
                    const float4 *h4 = reinterpret_cast<const float4 *>(whn);
#pragma unroll
                    for (int j4 = 0; j4 < 8; j4++) {
                        const float4 h = h4[j4];
                        m |= __fsub_rn(__uint_as_float(g[4 * j4 + 0]), h.x) > theta ? (1u << (4 * j4 + 0)) : 0u;
                        m |= __fsub_rn(__uint_as_float(g[4 * j4 + 1]), h.y) > theta ? (1u << (4 * j4 + 1)) : 0u;
                        m |= __fsub_rn(__uint_as_float(g[4 * j4 + 2]), h.z) > theta ? (1u << (4 * j4 + 2)) : 0u;
                        m |= __fsub_rn(__uint_as_float(g[4 * j4 + 3]), h.w) > theta ? (1u << (4 * j4 + 3)) : 0u;
                    }
                    m &= ((1u << c) - 1u) & ~(1u << lane);  // c <= 31
                    __syncwarp();
                    // walk: lane i holds the candidate of rank i and its mask
                    const uint32_t tl = valid ? word[lane] : 0u;
                    const uint32_t cm = __shfl_sync(0xffffffffu, m, tl);
                    unsigned U = __ballot_sync(0xffffffffu, valid);
                    uint32_t e = 0, out = 0xFFFFFFFFu;
                    while (U != 0u && e < R) {
                        const uint32_t u = __ffs(U) - 1;
                        const uint32_t t = __shfl_sync(0xffffffffu, tl, u);
                        if ((uint32_t)lane == e) out = nid[t];
                        e++;
                        U &= ~__ballot_sync(0xffffffffu, (cm >> t) & 1u) & ~(1u << u);
                    }
                    for (uint32_t p = lane; p < R; p += 32) a.adj[v * R + p] = p < e ? out : 0xFFFFFFFFu;
                    if (lane == 0) a.deg[v] = e;
                    __syncwarp();
                }
                fence_before();
                mbar_arrive(bar(C::BAR_TEMPTY + tb));
                mbar_arrive(bar(C::BAR_IEMPTY + ib));
                continue;
            }

            if (kind == TK_MED) {
                // ---- two nodes: node h by the warps on lane quarters 2h and 2h + 1, rows and
                // columns 64h .. 64h + c_h; the pair meets at its own named barrier
                uint32_t *gmask = reinterpret_cast<uint32_t *>(gs + C::G_MASK);
                uint32_t *gids = reinterpret_cast<uint32_t *>(gs + C::G_IDS);
                unsigned char *gorder = gs + C::G_ORDER;
                uint32_t *dx = reinterpret_cast<uint32_t *>(gs + C::G_DX);
                float *hn = reinterpret_cast<float *>(gs + C::G_HN);
                const uint32_t h = (uint32_t)quarter >> 1;
                const uint32_t base = 64 * h, lr = r - base;
                const uint32_t pair_id = 1 + PT_GROUPS + 2 * grp + h;
                const bool mine = h < misc[M_NODES];
                uint32_t c = 0;
                uint64_t v = 0;
                if (mine) {
                    c = misc[M_NODE + 3 * h + 0];
                    v = misc[M_NODE + 3 * h + 1];
                    const float nx = (float)(int32_t)misc[M_NODE + 3 * h + 2];
                    uint32_t DX = 0;
                    float theta = 0.0f;
                    bool bad = false;
                    {
                        uint32_t g[32];
                        tmem_ld32(trow + quarter * 32, g);
                        const float nr = __uint_as_float(pick32(g, lane));  // diagonal: exact integer
                        hn[r] = 0.5f * nr;
                        const uint32_t xc = base + c;  // the node's column
                        tmem_ld32(trow + (xc & ~31u), g);
                        if (lr < c) {
                            const float gx = __uint_as_float(pick32(g, xc & 31u));
                            const float dxf = __fmaf_rn(-2.0f, gx, nr + nx);
                            DX = (uint32_t)dxf;
                            const uint32_t T = removal_threshold(DX, a.alpha2, a.inv_alpha2);
                            theta = (nr - (float)T) * 0.5f;
                            dx[r] = DX;
                            bad = bf16_key(dxf) != bkey[r] || (lr > 0 && bkey[r - 1] > bkey[r]);
                        }
                    }
                    const bool full = named_barrier_or(pair_id, 64, bad);
                    uint32_t rk = 0;
                    if (lr < c) {
                        rk = candidate_rank(lr, c, DX, ids[r], dx + base, ids + base, bkey + base, full);
                        gorder[base + rk] = (unsigned char)lr;
                        gids[r] = ids[r];
                    }
                    uint32_t mw[2] = {0u, 0u};
#pragma unroll
                    for (uint32_t qq = 0; qq < 2; qq++) {
                        if (qq * 32 < c) {
                            uint32_t g[32];
                            tmem_ld32(trow + (2 * h + qq) * 32, g);
                            const float4 *h4 = reinterpret_cast<const float4 *>(hn + base + qq * 32);
                            uint32_t m = 0;
#pragma unroll
                            for (int j4 = 0; j4 < 8; j4++) {
                                const float4 hv = h4[j4];
                                m |= __fsub_rn(__uint_as_float(g[4 * j4 + 0]), hv.x) > theta ? (1u << (4 * j4 + 0)) : 0u;
                                m |= __fsub_rn(__uint_as_float(g[4 * j4 + 1]), hv.y) > theta ? (1u << (4 * j4 + 1)) : 0u;
                                m |= __fsub_rn(__uint_as_float(g[4 * j4 + 2]), hv.z) > theta ? (1u << (4 * j4 + 2)) : 0u;
                                m |= __fsub_rn(__uint_as_float(g[4 * j4 + 3]), hv.w) > theta ? (1u << (4 * j4 + 3)) : 0u;
                            }
                            const uint32_t live = c - qq * 32;
                            if (live < 32) m &= (1u << live) - 1u;
                            if (lr / 32 == qq) m &= ~(1u << (lr & 31));
                            mw[qq] = m;
                        }
                    }
                    // masks stored by rank, so the walk reads them in order without a dependent lookup
                    if (lr < c) reinterpret_cast<uint2 *>(gmask)[base + rk] = make_uint2(mw[0], mw[1]);
                }
                fence_before();
                mbar_arrive(bar(C::BAR_TEMPTY + tb));
                mbar_arrive(bar(C::BAR_IEMPTY + ib));
                if (mine) {
                    named_barrier_or(pair_id, 64, false);  // masks, order and ids of the pair complete
                    if ((uint32_t)quarter == 2 * h) {
                        // the walk, in one lane: rank i is admitted unless its mask (the candidates
                        // that remove it) meets the admitted set, up to R admissions; then the
                        // warp writes the admitted ids in rank order
                        const uint2 *mask = reinterpret_cast<const uint2 *>(gmask) + base;
                        uint64_t adm = 0;
                        if (lane == 0) {
                            uint64_t A = 0;
                            uint32_t e = 0;
                            for (uint32_t i = 0; i < c && e < R; i++) {
                                const uint2 mm = mask[i];
                                const uint32_t t = gorder[base + i];
                                if (((((uint64_t)mm.y << 32) | mm.x) & A) == 0ull) {
                                    A |= 1ull << t;
                                    adm |= 1ull << i;
                                    e++;
                                }
                            }
                        }
                        adm = __shfl_sync(0xffffffffu, adm, 0);
                        const uint32_t e = (uint32_t)__popcll(adm);
                        for (uint32_t i = lane; i < c; i += 32) {
                            if ((adm >> i) & 1ull) {
                                const uint32_t pos = (uint32_t)__popcll(adm & ((1ull << i) - 1ull));
                                a.adj[v * R + pos] = gids[base + gorder[base + i]];
                            }
                        }
                        for (uint32_t p = e + lane; p < R; p += 32) a.adj[v * R + p] = 0xFFFFFFFFu;
                        if (lane == 0) a.deg[v] = e;
                    }
                }
                // the group's arrays are rewritten by its next tile only after this barrier
                if (named_barrier_or(bar_id, 128, *abort != 0)) break;
                continue;
            }

            // ---- a large node, by the group: rows 0 .. c
            uint32_t *gmask = reinterpret_cast<uint32_t *>(gs + C::G_MASK);
            uint32_t *gids = reinterpret_cast<uint32_t *>(gs + C::G_IDS);
            unsigned char *gorder = gs + C::G_ORDER;
            uint32_t *dx = reinterpret_cast<uint32_t *>(gs + C::G_DX);
            float *hn = reinterpret_cast<float *>(gs + C::G_HN);
            const uint32_t c = misc[M_NODE + 0];
            const uint64_t v = misc[M_NODE + 1];
            const float nx = (float)(int32_t)misc[M_NODE + 2];
            uint32_t DX = 0;
            float theta = 0.0f;
            bool bad = false;
            {
                uint32_t g[32];
                tmem_ld32(trow + quarter * 32, g);
                const float nr = __uint_as_float(pick32(g, lane));  // diagonal: exact integer
                hn[r] = 0.5f * nr;
                tmem_ld32(trow + (c & ~31u), g);
                if (r < c) {
                    const float gx = __uint_as_float(pick32(g, c & 31u));
                    const float dxf = __fmaf_rn(-2.0f, gx, nr + nx);
                    DX = (uint32_t)dxf;
                    const uint32_t T = removal_threshold(DX, a.alpha2, a.inv_alpha2);
                    theta = (nr - (float)T) * 0.5f;
                    dx[r] = DX;
                    bad = bf16_key(dxf) != bkey[r] || (r > 0 && bkey[r - 1] > bkey[r]);
                }
            }
            const bool full = named_barrier_or(bar_id, 128, bad);
            if (r < c) {
                gorder[candidate_rank(r, c, DX, ids[r], dx, ids, bkey, full)] = (unsigned char)r;
                gids[r] = ids[r];
            }
            uint32_t mw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                if (q * 32 < c) {
                    uint32_t g[32];
                    tmem_ld32(trow + q * 32, g);
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
            if (r < c) reinterpret_cast<uint4 *>(gmask)[r] = make_uint4(mw[0], mw[1], mw[2], mw[3]);
            fence_before();
            mbar_arrive(bar(C::BAR_TEMPTY + tb));
            mbar_arrive(bar(C::BAR_IEMPTY + ib));
            named_barrier_or(bar_id, 128, false);  // masks, order and ids complete
            if (quarter == 0) {
                // the walk: per block of 32 ranks one vote drops every candidate removed by an
                // earlier admission, then each admission removes, with one vote, the later lanes
                // it prunes
                const uint4 *mask = reinterpret_cast<const uint4 *>(gmask);
                uint32_t A0 = 0, A1 = 0, A2 = 0, A3 = 0, e = 0;
                uint32_t out[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
                for (uint32_t b = 0; b * 32 < c && e < R; b++) {
                    const uint32_t i = b * 32 + lane;
                    const bool valid = i < c;
                    const uint32_t tl = valid ? gorder[i] : 0u;
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
                        const uint32_t id = gids[t];
                        const uint32_t o = e >> 5;
                        const bool mine = (e & 31) == (uint32_t)lane;
                        out[0] = (mine && o == 0) ? id : out[0];
                        out[1] = (mine && o == 1) ? id : out[1];
                        out[2] = (mine && o == 2) ? id : out[2];
                        out[3] = (mine && o == 3) ? id : out[3];
                        e++;
                        const uint32_t mwd = wd == 0 ? cm.x : wd == 1 ? cm.y : wd == 2 ? cm.z : cm.w;
                        U &= ~__ballot_sync(0xffffffffu, (mwd >> (t & 31)) & 1u) & ~(1u << u);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t p = lane + 32 * q;
                    if (p < R) a.adj[v * R + p] = p < e ? out[q] : 0xFFFFFFFFu;
                }
                if (lane == 0) a.deg[v] = e;
            }
            // the group's walk data is rewritten by its next large tile only after this barrier
            if (named_barrier_or(bar_id, 128, *abort != 0)) break;
        }
    } else {
        // ------------------------------------------------------------ row gathers (two warps)
        // Warp g gathers the rows of tiles g, g + 2, ...: lane L rows 4L .. 4L + 3 if any of them
        // is in use.  A tile's row ids are read one own tile ahead (while the current tile waits
        // for its A buffer); no tile past an end marker is read (none may exist).
        struct Rows {
            uint32_t y[4];
            bool use;
            uint32_t kind;
        };
        auto prepare = [&](uint32_t k, Rows &t) {
            const uint32_t ib = k % C::I;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_CFULL + ib), (k / C::I) & 1, abort, a.err)))
                return false;
            const unsigned char *in = info(ib);
            const uint32_t *ids = reinterpret_cast<const uint32_t *>(in + I_IDS);
            const uint32_t *misc = reinterpret_cast<const uint32_t *>(in + I_MISC);
            t.kind = misc[M_KIND];
            t.use = false;
            if (t.kind == TK_END) return true;
            if (t.kind == TK_PACK) {
                const uint32_t q = (uint32_t)lane >> 3;
                const uint32_t nodes = misc[M_NODES];
                const uint32_t c = q < nodes ? misc[M_NODE + 3 * q] : 0u;
                const uint32_t node_row = 32 * q + c;  // the node itself
                t.use = q < nodes && 4 * ((uint32_t)lane & 7) <= c;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const uint32_t row = 4 * lane + e;
                    t.y[e] = t.use ? ids[(row & 31) <= c ? row : node_row] : 0u;
                }
            } else if (t.kind == TK_MED) {
                const uint32_t h = (uint32_t)lane >> 4;
                const uint32_t nodes = misc[M_NODES];
                const uint32_t c = h < nodes ? misc[M_NODE + 3 * h] : 0u;
                const uint32_t node_row = 64 * h + c;  // the node itself
                t.use = h < nodes && 4 * ((uint32_t)lane & 15) <= c;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const uint32_t row = 4 * lane + e;
                    t.y[e] = t.use ? ids[(row & 63) <= c ? row : node_row] : 0u;
                }
            } else {
                const uint32_t rows = misc[M_NODE] + 1;
                t.use = 4u * lane < rows;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const uint32_t row = 4 * lane + e;
                    t.y[e] = t.use ? ids[row < rows ? row : rows - 1] : 0u;
                }
            }
            return true;
        };
        uint32_t k = warp - PT_GATHER_WARP0;
        Rows cur, nxt;
        bool live = prepare(k, cur) && (cur.kind == TK_END || prepare(k + PT_GATHERERS, nxt));
        while (live && cur.kind != TK_END) {
            const uint32_t ua = k % C::A;
            if (!__all_sync(0xffffffffu, mbar_wait(bar(C::BAR_EMPTY_A + ua), ((k / C::A) & 1) ^ 1, abort, a.err)))
                break;
            const unsigned um = __ballot_sync(0xffffffffu, cur.use);
            const uint32_t fb = bar(C::BAR_FULL_A + ua);
            if (lane == 0) mbar_arrive_tx(fb, __popc(um) * 512u * KB);
            __syncwarp();
            if (cur.use) {
                const uint32_t dst = sbase + C::OFF_A0 + ua * KB * REGION + lane * 4 * 128;
#pragma unroll
                for (int kb = 0; kb < KB; kb++)
                    tma_gather4(dst + kb * REGION, &xmap, kb * 64, (int32_t)cur.y[0], (int32_t)cur.y[1],
                                (int32_t)cur.y[2], (int32_t)cur.y[3], fb);
            }
            if (lane != 0) mbar_arrive(fb);
            cur = nxt;
            k += PT_GATHERERS;
            if (cur.kind != TK_END) live = prepare(k + PT_GATHERERS, nxt);
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

int reservoir_total(const uint32_t *cnt, uint64_t n, uint32_t l_max, uint64_t *total);

int final_prune_tc(const void *X, uint64_t n, uint32_t d, int dtype, const int32_t *sqn, const uint64_t *res,
                   const uint32_t *cnt, uint32_t l_max, uint32_t R, float alpha2, uint32_t *adj, uint32_t *deg,
                   float *ms_kernel, Workspace &ws) {
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
    // Two-node tiles pay off where reservoirs are full (average above 32 slots, as in builds of
    // 100M points: 1.68 -> 1.11 s) and cost a little where most are small (1M points, average 21:
    // 5.4 -> 6.1 ms), so they are used by that average.
    uint64_t slots = 0;
    PIPNN_TRY(reservoir_total(cnt, n, l_max, &slots));
    a.medium = slots > 32 * n ? PT_MEDIUM : PT_SMALL;
    LaunchTimer lt(ms_kernel);
    PIPNN_TRY(kp == 64 ? launch_pt<1>(map, a) : launch_pt<2>(map, a));
    lt.stop();
    return PIPNN_OK;
}

}  // namespace pipnn
