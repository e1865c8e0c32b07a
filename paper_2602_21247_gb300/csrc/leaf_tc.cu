// leaf_tc.cu -- A2..A4 on the 5th-generation tensor cores (tcgen05 + TMEM), byte data.
//
// For every leaf b and every 128-row tile of it, one CTA computes the Gram block
// G = X_rows X_colsᵀ against all |b| members, 256 columns at a time, and keeps, per row, the
// k nearest other members by (D, id) with D = n_i + n_j - 2 G_ij (Sec. 4.2: the all-pairs
// distance matrix of a leaf; App. A.3: bi-directed k-NN pick).  The distance matrix never
// leaves TMEM / registers.
//
// Exactness: u8 / i8 coordinates are exact in BF16; every product is an integer of magnitude
// <= 65,536 and for d <= 256 every partial sum of d products, n_j - 2G and D stay below 2^24,
// so FP32 accumulation in the tensor core is exact in any order and the picks equal those of
// the defining integer arithmetic.
//
// CTA layout (13 warps):
//   warps 0-3  producers: gather the tile's rows from the BF16 copy of the points (16-byte
//              loads), store them in the 128-byte-swizzled K-major layout the MMA descriptors
//              describe, fence the async proxy, arrive on the stage's "full" barrier
//   warp 4     allocates 512 TMEM columns; one thread issues tcgen05.mma (M=128, N<=256, K=16
//              steps) into accumulator buffer t%2 and commits to "empty[stage]" / "tmem_full"
//   warps 5-12 epilogue: tcgen05.ld 32 columns at a time, v = n_j - 2G (exact), per 32-column
//              chunk a min filter against the row's current k-th best, exact (v, id) insertion;
//              two warps share each TMEM lane quarter and split the columns, then merge
// Every mbarrier wait is bounded by %globaltimer (2 s); on expiry the CTA records
// DERR_TIMEOUT, stops all roles, and still frees its TMEM.
#include "internal.cuh"

namespace pipnn {

namespace {

constexpr int TC_PRODUCER_WARPS = 4;
constexpr int TC_MMA_WARP = 4;
constexpr int TC_EPI_WARP0 = 5;
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = (TC_PRODUCER_WARPS + 1 + TC_EPI_WARPS) * 32;  // 416
constexpr int TC_ROWS = 128;
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false if the CTA aborted or the wait ran past TC_WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, unsigned *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t i = 1;; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (*abort) return false;
            if (globaltimer() - t0 > TC_WAIT_NS) {
                *abort = 1;
                atomicOr(err, DERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier that also ORs a predicate over the participating threads, so a stop decision
// is identical for all of them (no thread can leave a loop its peers are still in).
__device__ __forceinline__ bool named_barrier_or(uint32_t id, uint32_t count, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major.
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t M, uint32_t N) {
    return (1u << 4)              // D: FP32
           | (1u << 7)            // A: BF16
           | (1u << 10)           // B: BF16
           | ((N >> 3) << 17)     // N / 8
           | ((M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ kernel
struct TcArgs {
    const __nv_bfloat16 *Xb;     // n x Kp BF16 copy of the points (zero padded)
    const int32_t *sqnorm;       // exact squared norms
    const uint32_t *tile_grp, *tile_row0;
    const uint64_t *leaf_off;
    const uint32_t *members;
    const uint64_t *cand_off;
    uint32_t k;
    uint32_t *out_dst, *out_src;
    float *out_dist;
    unsigned *err;
};

template <int KB, int KMAX>
struct TcCfg {
    static constexpr int KP = 64 * KB;                       // padded K (elements)
    static constexpr int NMAX = KB <= 2 ? 256 : 128;         // columns per B tile
    static constexpr int A_REGION = TC_ROWS * 128;           // bytes per 64-wide K block of A
    static constexpr int B_REGION = NMAX * 128;              // bytes per 64-wide K block of B
    static constexpr int A_BYTES = A_REGION * KB;
    static constexpr int B_BYTES = B_REGION * KB;
    static constexpr int OFF_A = 0;
    static constexpr int OFF_B0 = OFF_A + A_BYTES;
    static constexpr int OFF_B1 = OFF_B0 + B_BYTES;
    static constexpr int OFF_NB = OFF_B1 + B_BYTES;          // 2 x NMAX floats
    static constexpr int OFF_GB = OFF_NB + 2 * NMAX * 4;     // 2 x NMAX ids
    static constexpr int OFF_MV = OFF_GB + 2 * NMAX * 4;     // 128 rows x KMAX (v, id) merge buffer
    static constexpr int OFF_BAR = OFF_MV + TC_ROWS * KMAX * 8;
    static constexpr int BAR_FULL_A = 0, BAR_FULL = 1, BAR_EMPTY = 3, BAR_TFULL = 5, BAR_TEMPTY = 7;
    static constexpr int OFF_MISC = OFF_BAR + 9 * 8;         // tmem base, abort flag
    static constexpr int BYTES = OFF_MISC + 16;
    static constexpr int SMEM = BYTES + 1024;                // + alignment slack
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

template <int KB, int KMAX>
__global__ void __launch_bounds__(TC_THREADS, 1) leaf_gram_tc(const TcArgs a) {
    using C = TcCfg<KB, KMAX>;
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    float *nbuf = reinterpret_cast<float *>(smem + C::OFF_NB);
    uint32_t *gbuf = reinterpret_cast<uint32_t *>(smem + C::OFF_GB);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(smem + C::OFF_MISC);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + C::OFF_MISC + 4);
    auto bar = [&](int i) { return sbase + C::OFF_BAR + 8 * i; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t g = a.tile_grp[blockIdx.x];
    const uint32_t row0 = a.tile_row0[blockIdx.x];
    const uint64_t off = a.leaf_off[g];
    const uint32_t s = (uint32_t)(a.leaf_off[g + 1] - off);
    const uint32_t nct = (s + C::NMAX - 1) / C::NMAX;  // column tiles
    const uint32_t *mem = a.members + off;

    if (threadIdx.x == 0) {
        mbar_init(bar(C::BAR_FULL_A), TC_PRODUCER_WARPS * 32);
        for (int i = 0; i < 2; i++) {
            mbar_init(bar(C::BAR_FULL + i), TC_PRODUCER_WARPS * 32);
            mbar_init(bar(C::BAR_EMPTY + i), 1);
            mbar_init(bar(C::BAR_TFULL + i), 1);
            mbar_init(bar(C::BAR_TEMPTY + i), TC_EPI_WARPS * 32);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == TC_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         sbase + C::OFF_MISC),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < TC_PRODUCER_WARPS) {
        // ---------------- producers
        const int pt = threadIdx.x;  // 0..127
        constexpr int CHUNKS = KB * 8;  // 16-byte chunks per row
        auto load_rows = [&](uint32_t dst_base, int region, uint32_t first, uint32_t nrows_alloc) {
            // rows r < nrows_alloc of the tile starting at member `first`; rows past the leaf
            // repeat its first member (their columns / rows are masked later).  All of a
            // thread's 16-byte copies are in flight at once (cp.async, L2 only); the thread
            // waits for its own copies, then makes them visible to the tensor core's proxy.
            for (uint32_t idx = pt; idx < nrows_alloc * CHUNKS; idx += TC_PRODUCER_WARPS * 32) {
                const uint32_t r = idx / CHUNKS, c = idx % CHUNKS;
                const uint32_t m = first + r < s ? mem[first + r] : mem[0];
                const __nv_bfloat16 *src = a.Xb + (uint64_t)m * C::KP + c * 8;
                const uint32_t kb = c >> 3, ch = c & 7;
                const uint32_t addr = dst_base + kb * region + r * 128 + ((ch ^ (r & 7)) << 4);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(addr), "l"(src) : "memory");
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            fence_proxy_async();
        };
        load_rows(sbase + C::OFF_A, C::A_REGION, row0, TC_ROWS);
        mbar_arrive(bar(C::BAR_FULL_A));
        for (uint32_t t = 0; t < nct; t++) {
            const uint32_t st = t & 1;
            if (!mbar_wait(bar(C::BAR_EMPTY + st), ((t >> 1) & 1) ^ 1, abort, a.err)) break;
            const uint32_t c0 = t * C::NMAX;
            const uint32_t ncols = s - c0 < (uint32_t)C::NMAX ? s - c0 : C::NMAX;
            const uint32_t nalloc = (ncols + 15) & ~15u;
            load_rows(sbase + (st ? C::OFF_B1 : C::OFF_B0), C::B_REGION, c0, nalloc);
            mbar_arrive(bar(C::BAR_FULL + st));
        }
    } else if (warp == TC_MMA_WARP) {
        // ---------------- MMA issuer
        if (lane == 0) {
            bool ok = mbar_wait(bar(C::BAR_FULL_A), 0, abort, a.err);
            uint32_t issued = 0;
            for (uint32_t t = 0; ok && t < nct; t++) {
                const uint32_t st = t & 1;
                if (!mbar_wait(bar(C::BAR_FULL + st), (t >> 1) & 1, abort, a.err)) break;
                if (!mbar_wait(bar(C::BAR_TEMPTY + st), ((t >> 1) & 1) ^ 1, abort, a.err)) break;
                tc_fence_after();
                const uint32_t c0 = t * C::NMAX;
                const uint32_t ncols = s - c0 < (uint32_t)C::NMAX ? s - c0 : C::NMAX;
                const uint32_t N = (ncols + 15) & ~15u;
                const uint32_t idesc = idesc_bf16(128, N);
                const uint32_t aB = sbase + C::OFF_A, bB = sbase + (st ? C::OFF_B1 : C::OFF_B0);
#pragma unroll
                for (int kk = 0; kk < KB * 4; kk++) {
                    const uint64_t ad = smem_desc_sw128(aB + (kk >> 2) * C::A_REGION + (kk & 3) * 32);
                    const uint64_t bd = smem_desc_sw128(bB + (kk >> 2) * C::B_REGION + (kk & 3) * 32);
                    mma_bf16(tmem + st * C::NMAX, ad, bd, idesc, kk > 0 ? 1u : 0u);
                }
                mma_commit(bar(C::BAR_EMPTY + st));
                mma_commit(bar(C::BAR_TFULL + st));
                issued = t + 1;
            }
            // on an early stop, let the last issued MMAs finish before TMEM is released
            if (issued && issued < nct) mbar_wait(bar(C::BAR_TFULL + ((issued - 1) & 1)), ((issued - 1) >> 1) & 1, abort, a.err);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue
        const int ew = warp - TC_EPI_WARP0;          // 0..7
        const int half = ew >> 2;                    // which column chunks
        const int quarter = warp & 3;                // TMEM lane quarter this warp may access
        const uint32_t r = quarter * 32 + lane;      // row inside the tile
        const uint32_t et = (uint32_t)(threadIdx.x - TC_EPI_WARP0 * 32);  // 0..255
        const bool row_ok = row0 + r < s;
        const uint32_t my_id = row_ok ? mem[row0 + r] : 0xFFFFFFFFu;
        float kv[KMAX];
        uint32_t ki[KMAX];
#pragma unroll
        for (int p = 0; p < KMAX; p++) {
            kv[p] = __int_as_float(0x7f800000);
            ki[p] = 0xFFFFFFFFu;
        }
        bool failed = false;
        for (uint32_t t = 0; t < nct; t++) {
            const uint32_t st = t & 1;
            const uint32_t c0 = t * C::NMAX;
            if (et < (uint32_t)C::NMAX) {
                const uint32_t col = c0 + et;
                uint32_t gid = 0xFFFFFFFFu;
                float nb = __int_as_float(0x7f800000);
                if (col < s) {
                    gid = mem[col];
                    nb = (float)a.sqnorm[gid];
                }
                nbuf[st * C::NMAX + et] = nb;
                gbuf[st * C::NMAX + et] = gid;
            }
            if (named_barrier_or(1, TC_EPI_WARPS * 32, failed || *abort)) {
                failed = true;
                break;
            }
            // warp-uniform wait: tcgen05.ld below is a warp-collective instruction
            const bool ok = __all_sync(0xffffffffu, mbar_wait(bar(C::BAR_TFULL + st), (t >> 1) & 1, abort, a.err));
            if (!ok) {
                failed = true;
                continue;
            }
            tc_fence_after();
            const uint32_t ncols = s - c0 < (uint32_t)C::NMAX ? s - c0 : C::NMAX;
            const float *nbt = nbuf + st * C::NMAX;
            const uint32_t *gbt = gbuf + st * C::NMAX;
            for (uint32_t q = half; q * 32 < ncols; q += 2) {
                uint32_t gv[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + st * C::NMAX + q * 32, gv);
                if (!row_ok) continue;
                float v[32];
                const float4 *n4 = reinterpret_cast<const float4 *>(nbt + q * 32);
#pragma unroll
                for (int j4 = 0; j4 < 8; j4++) {
                    const float4 nn = n4[j4];
                    v[4 * j4 + 0] = __fmaf_rn(-2.0f, __uint_as_float(gv[4 * j4 + 0]), nn.x);
                    v[4 * j4 + 1] = __fmaf_rn(-2.0f, __uint_as_float(gv[4 * j4 + 1]), nn.y);
                    v[4 * j4 + 2] = __fmaf_rn(-2.0f, __uint_as_float(gv[4 * j4 + 2]), nn.z);
                    v[4 * j4 + 3] = __fmaf_rn(-2.0f, __uint_as_float(gv[4 * j4 + 3]), nn.w);
                }
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
                    for (int j = 0; j < 32; j++) {
                        if (v[j] <= kv[KMAX - 1]) {
                            const uint32_t id = gbt[q * 32 + j];
                            if (id != my_id && id != 0xFFFFFFFFu) topk_insert<KMAX>(kv, ki, v[j], id);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(bar(C::BAR_TEMPTY + st));
        }
        // merge the two halves of each row
        float2 *mv = reinterpret_cast<float2 *>(smem + C::OFF_MV);
        if (half == 1) {
#pragma unroll
            for (int p = 0; p < KMAX; p++) mv[r * KMAX + p] = make_float2(kv[p], __uint_as_float(ki[p]));
        }
        failed = named_barrier_or(1, TC_EPI_WARPS * 32, failed || *abort);
        if (half == 0 && row_ok && !failed) {
#pragma unroll
            for (int p = 0; p < KMAX; p++) {
                const float2 e = mv[r * KMAX + p];
                const uint32_t id = __float_as_uint(e.y);
                if (id != 0xFFFFFFFFu) topk_insert<KMAX>(kv, ki, e.x, id);
            }
            const uint32_t kk = s - 1 < a.k ? s - 1 : a.k;
            const float ni = (float)a.sqnorm[my_id];
            uint64_t w = a.cand_off[g] + (uint64_t)(row0 + r) * 2 * kk;
#pragma unroll
            for (int p = 0; p < KMAX; p++) {
                if ((uint32_t)p < kk) {
                    const uint32_t src = ki[p] == 0xFFFFFFFFu ? my_id : ki[p];
                    const float D = __fadd_rn(ni, kv[p]);
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

    tc_fence_before();
    __syncthreads();
    if (warp == TC_MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

__global__ void to_bf16_padded(const void *X, uint64_t n, uint32_t d, uint32_t kp, int dtype, __nv_bfloat16 *out) {
    const uint64_t total = n * kp;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = i / kp;
        const uint32_t t = (uint32_t)(i % kp);
        float v = 0.0f;
        if (t < d) {
            v = dtype == PIPNN_U8 ? (float)static_cast<const uint8_t *>(X)[p * d + t]
                                  : (float)static_cast<const int8_t *>(X)[p * d + t];
        }
        out[i] = __float2bfloat16_rn(v);
    }
}

template <int KB, int KMAX>
int launch_tc(const TcArgs &args, uint64_t ntiles) {
    using C = TcCfg<KB, KMAX>;
    auto kern = leaf_gram_tc<KB, KMAX>;
    PIPNN_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    for (uint64_t t0 = 0; t0 < ntiles; t0 += 0x7FFFFFFFull) {
        const uint64_t cnt = ntiles - t0 < 0x7FFFFFFFull ? ntiles - t0 : 0x7FFFFFFFull;
        TcArgs a = args;
        a.tile_grp += t0;
        a.tile_row0 += t0;
        kern<<<(unsigned)cnt, TC_THREADS, C::SMEM, stream()>>>(a);
        PIPNN_LAUNCH_CHECK();
    }
    return PIPNN_OK;
}

template <int KB>
int launch_tc_k(const TcArgs &args, uint64_t ntiles, uint32_t k) {
    if (k <= 2) return launch_tc<KB, 2>(args, ntiles);
    if (k <= 4) return launch_tc<KB, 4>(args, ntiles);
    if (k <= 8) return launch_tc<KB, 8>(args, ntiles);
    return launch_tc<KB, 16>(args, ntiles);
}
}  // namespace

int leaf_pick_tc(const void *X, uint64_t n, uint32_t d, int dtype, const int32_t *sqnorm, const uint64_t *off,
                 const uint32_t *mem, uint64_t L, const uint32_t *leaf_size, const uint64_t *cand_off, uint32_t k,
                 uint32_t *out_dst, uint32_t *out_src, float *out_dist, Workspace &ws, cudaEvent_t ev0,
                 cudaEvent_t ev1, uint32_t *launches) {
    if (dtype == PIPNN_F32) return set_error(PIPNN_EUNSUPPORTED, "the tensor-core leaf engine takes byte data only");
    if (d > 256) return set_error(PIPNN_EUNSUPPORTED, "the tensor-core leaf engine is exact for d <= 256");
    if (k > 16) return set_error(PIPNN_EINVAL, "k above 16");
    const uint32_t kb = (d + 63) / 64;
    const uint32_t kp = kb * 64;
    __nv_bfloat16 *Xb = nullptr;
    PIPNN_TRY(ws.alloc(&Xb, n * kp));
    to_bf16_padded<<<grid_for(n * kp, 256), 256, 0, stream()>>>(X, n, d, kp, dtype, Xb);
    PIPNN_LAUNCH_CHECK();
    uint32_t *tile_grp = nullptr, *tile_row0 = nullptr;
    uint64_t ntiles = 0;
    PIPNN_TRY(make_tiles(leaf_size, L, TC_ROWS, &tile_grp, &tile_row0, &ntiles, ws));
    TcArgs a{};
    a.Xb = Xb;
    a.sqnorm = sqnorm;
    a.tile_grp = tile_grp;
    a.tile_row0 = tile_row0;
    a.leaf_off = off;
    a.members = mem;
    a.cand_off = cand_off;
    a.k = k;
    a.out_dst = out_dst;
    a.out_src = out_src;
    a.out_dist = out_dist;
    a.err = device_error_word();
    *launches = 0;
    if (ntiles == 0) return PIPNN_OK;
    cudaEventRecord(ev0, stream());
    int rc;
    switch (kb) {
    case 1: rc = launch_tc_k<1>(a, ntiles, k); break;
    case 2: rc = launch_tc_k<2>(a, ntiles, k); break;
    case 3: rc = launch_tc_k<3>(a, ntiles, k); break;
    default: rc = launch_tc_k<4>(a, ntiles, k); break;
    }
    cudaEventRecord(ev1, stream());
    *launches = 1;
    return rc;
}

}  // namespace pipnn
