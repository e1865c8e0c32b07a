// tc_common.cuh -- pieces shared by the tcgen05 engines (leaf pick and leader assignment):
// inline-PTX wrappers for mbarriers, TMA, tcgen05.mma / ld and TMEM, the persistent-CTA role
// layout, and host helpers that build the BF16 operand copies and their tensor maps.
//
// Operand layout (both engines): K-major BF16 rows, 64 columns (128 bytes) per K block, 128 rows
// per 16 KB region, 128-byte swizzle (16-byte chunk c of row r stored at chunk c ^ (r & 7)).  For
// byte data every value is exact in BF16 and FP32 accumulation of integer products is exact while
// partial sums stay below 2^24, which holds for d <= 128.
#pragma once

#include "internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace pipnn {
namespace tc {

constexpr int PRODUCER_WARP = 0;
constexpr int MMA_WARP = 1;
constexpr int EPI_WARP0 = 2;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = (2 + EPI_WARPS) * 32;  // 320
constexpr int ROWS = 128;
constexpr int REGION = 128 * 128;              // bytes of one 128-row x 64-column K block
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long WAIT_NS = 2000000000ull;

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

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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

// Bounded wait: false if the CTA aborted or the wait ran past limit_ns (then the CTA is marked
// aborted and DERR_TIMEOUT is recorded).
__device__ __forceinline__ bool mbar_wait_limit(uint32_t bar, uint32_t parity, volatile int *abort, unsigned *err,
                                                unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (uint32_t i = 1;; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (*abort) return false;
            if (globaltimer() - t0 > limit_ns) {
                *abort = 1;
                atomicOr(err, DERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, unsigned *err) {
    return mbar_wait_limit(bar, parity, abort, err, WAIT_NS);
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

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
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

// Instruction descriptor, kind::f8f6f4: E4M3 x E4M3 -> FP32, both operands K-major (32 K per MMA).
__device__ __forceinline__ uint32_t idesc_e4m3(uint32_t M, uint32_t N) {
    return (1u << 4)              // D: FP32
           | (0u << 7)            // A: E4M3
           | (0u << 10)           // B: E4M3
           | ((N >> 3) << 17)     // N / 8
           | ((M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (lane = row).
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

// The same load without the wait: several may be in flight before one tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
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
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The wait, with r passed through it: no use of r can be scheduled before the load completed.
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Asynchronous global -> shared copies (no registers hold the data in flight): committed in
// groups, waited for with "at most N groups still pending".  Completion is visible to the copying
// thread only; a __syncwarp after the wait publishes a warp's copies to all its lanes.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// TMA tiled load of a 128-row x 64-column BF16 box at (x, y) into 16 KB of shared memory,
// 128-byte swizzled -- the layout the MMA descriptors read.  Rows past the tensor read as zero.
__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y,
                                              uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// TMA gather of four rows y0..y3, columns x..x+63, into four consecutive 128-byte rows of shared
// memory.  The 128-byte swizzle is keyed to the destination address, so four rows written at
// row offset 4g of a 1024-byte-aligned region land exactly where a tiled load would put rows
// 4g..4g+3.  The map's box is one row high.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y0, int32_t y1,
                                            int32_t y2, int32_t y3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(bar)
        : "memory");
}

// The four pieces of -(n / 2) for a non-negative integer n < 2^25, each exact in BF16: minus the
// three bytes of floor(n / 2) and -(n mod 2) / 2, packed as two words (pieces 0,1 and 2,3).
__device__ __forceinline__ uint2 neg_half_norm_pieces(uint32_t n) {
    const uint32_t h = n >> 1;
    const uint32_t b1 = __bfloat16_as_ushort(__float2bfloat16_rn(-(float)(h & 0xFF0000u)));
    const uint32_t b2 = __bfloat16_as_ushort(__float2bfloat16_rn(-(float)(h & 0x00FF00u)));
    const uint32_t b3 = __bfloat16_as_ushort(__float2bfloat16_rn(-(float)(h & 0x0000FFu)));
    const uint32_t b4 = __bfloat16_as_ushort(__float2bfloat16_rn((n & 1u) ? -0.5f : 0.0f));
    return make_uint2(b1 | (b2 << 16), b3 | (b4 << 16));
}

}  // namespace tc

// Row-major BF16 copy of rows of X, zero padded to kp columns (a multiple of 64): row i holds
// point ids[i], or point i when ids is null.  Exact for byte data.
int stage_rows_bf16(const void *X, uint32_t d, uint32_t kp, int dtype, const uint32_t *ids, uint64_t M,
                    __nv_bfloat16 *out);

// Tensor map over an n x kp BF16 row-major matrix with 128-byte swizzle: boxes of 128 rows x 64
// columns (tiled loads) or, with gather = true, of 1 row x 64 columns (tile::gather4).
int encode_rows_map(CUtensorMap *map, const __nv_bfloat16 *base, uint64_t n, uint32_t kp, bool gather);

// Tensor map over an n x kpb byte matrix (8-bit operands, kpb a multiple of 128) with 128-byte
// swizzle: boxes of 128 rows x 128 bytes.
int encode_bytes_map(CUtensorMap *map, const void *base, uint64_t n, uint32_t kpb);

// ---------------------------------------------------------------- Alg. 5 assignment engine
constexpr uint32_t ASSIGN_TC_MAX_F = 16;

// Padded BF16 copy of all points and its gather map, made once per partition.  Once the rows are
// restaged in a locality order (assign_tc_plan_reorder), point v's row is row pos[v].
struct AssignTcPlan {
    __nv_bfloat16 *rows = nullptr;
    CUtensorMap map;
    uint32_t kp = 0;
};

// True if a level with fanout F can run on the tensor-core assignment engine: byte data,
// d <= 128, fewer than 2^31 points, F <= ASSIGN_TC_MAX_F.
bool assign_tc_eligible(int dtype, uint32_t d, uint64_t n, uint32_t F);

int assign_tc_plan(const void *X, uint64_t n, uint32_t d, int dtype, Workspace &ws, AssignTcPlan *plan);

// One level's assignment: for every instance of every subproblem, the min(F, L) nearest of the
// subproblem's L leaders by (squared distance, rank), written to assign[instance * F + slot], and
// every pick counted into bucket_cnt[lead_off + rank] (which the caller zeroed).  Tiles are the
// 128-instance tiles of make_tiles(seg_size).
int assign_tc(const AssignTcPlan &plan, const void *X, uint32_t d, int dtype, const int32_t *sqnorm,
              const uint32_t *tile_grp, const uint32_t *tile_row0, uint64_t ntiles, const uint64_t *seg_start,
              const uint32_t *seg_size, const uint32_t *inst, const uint64_t *lead_off, const uint32_t *lead_cnt,
              const uint32_t *lead, uint64_t total_leaders, uint64_t ninst, uint32_t F, uint16_t *assign,
              uint32_t *bucket_cnt, Workspace &ws);

}  // namespace pipnn
