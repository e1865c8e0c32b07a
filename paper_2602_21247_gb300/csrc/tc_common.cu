// tc_common.cu -- host helpers of the tcgen05 engines: BF16 operand copies and TMA tensor maps.
#include "tc_common.cuh"

namespace pipnn {

namespace {

// Eight bytes -> eight BF16 values (exact for u8 / i8), as four packed words.
template <int DT>
__device__ __forceinline__ void bytes_to_bf16x8(uint32_t lo, uint32_t hi, uint32_t (&w)[4]) {
    const uint32_t b[2] = {lo, hi};
#pragma unroll
    for (int h = 0; h < 4; h++) {
        const uint32_t word = b[h >> 1], sh = (h & 1) * 16;
        const uint32_t x0 = (word >> sh) & 0xFFu, x1 = (word >> (sh + 8)) & 0xFFu;
        const float f0 = DT == PIPNN_U8 ? (float)x0 : (float)(int8_t)x0;
        const float f1 = DT == PIPNN_U8 ? (float)x1 : (float)(int8_t)x1;
        w[h] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f0)) |
               ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f1)) << 16);
    }
}

// One thread per 16-byte output chunk (8 BF16 values) of the padded copy.  Rows whose width is a
// multiple of 8 bytes are read 8 bytes at a time; others byte by byte.
template <int DT, bool WIDE>
__global__ void stage_rows_kernel(const void *X, uint32_t d, uint32_t kp, const uint32_t *ids, uint64_t M,
                                  __nv_bfloat16 *out) {
    const uint32_t per_row = kp / 8;
    const uint64_t total = M * per_row;
    const uint8_t *Xb = static_cast<const uint8_t *>(X);
    // chunks per row: a power of two (d <= 128: 8 or 16) splits the index with a shift and a mask
    const bool pow2 = (per_row & (per_row - 1)) == 0;
    const uint32_t shift = __ffs(per_row) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t row = pow2 ? i >> shift : i / per_row;
        const uint32_t c = (uint32_t)(i - row * per_row);
        const uint64_t src = (uint64_t)(ids ? ids[row] : row) * d;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (WIDE) {
            if (c * 8 < d) {
                const uint2 v = *reinterpret_cast<const uint2 *>(Xb + src + c * 8);
                bytes_to_bf16x8<DT>(v.x, v.y, w);
            }
        } else {
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const uint32_t col = c * 8 + t;
                const uint32_t x = col < d ? Xb[src + col] : 0u;
                if (t < 4) lo |= x << (8 * t);
                else hi |= x << (8 * (t - 4));
            }
            bytes_to_bf16x8<DT>(lo, hi, w);
        }
        reinterpret_cast<uint4 *>(out)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace

int stage_rows_bf16(const void *X, uint32_t d, uint32_t kp, int dtype, const uint32_t *ids, uint64_t M,
                    __nv_bfloat16 *out) {
    if (dtype != PIPNN_U8 && dtype != PIPNN_I8) return set_error(PIPNN_EUNSUPPORTED, "BF16 staging takes byte data");
    if (kp % 64 != 0 || kp < d) return set_error(PIPNN_EINVAL, "padded width %u", kp);
    if (M == 0) return PIPNN_OK;
    const unsigned g = grid_for(M * (kp / 8), 256);
    const bool wide = d % 8 == 0 && (reinterpret_cast<uintptr_t>(X) & 7) == 0;
    if (dtype == PIPNN_U8) {
        if (wide) stage_rows_kernel<PIPNN_U8, true><<<g, 256, 0, stream()>>>(X, d, kp, ids, M, out);
        else stage_rows_kernel<PIPNN_U8, false><<<g, 256, 0, stream()>>>(X, d, kp, ids, M, out);
    } else {
        if (wide) stage_rows_kernel<PIPNN_I8, true><<<g, 256, 0, stream()>>>(X, d, kp, ids, M, out);
        else stage_rows_kernel<PIPNN_I8, false><<<g, 256, 0, stream()>>>(X, d, kp, ids, M, out);
    }
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            !fn) {
            cudaGetLastError();
            return nullptr;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return encode;
}
}  // namespace

int encode_bytes_map(CUtensorMap *map, const void *base, uint64_t n, uint32_t kpb) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return set_error(PIPNN_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    if (n >= 0x7FFFFFFFull) return set_error(PIPNN_EUNSUPPORTED, "a tensor map addresses fewer than 2^31 rows");
    if (kpb % 128 != 0) return set_error(PIPNN_EINVAL, "byte rows of %u bytes (a multiple of 128 is needed)", kpb);
    const cuuint64_t gdim[2] = {kpb, n};
    const cuuint64_t gstride[1] = {(cuuint64_t)kpb};
    const cuuint32_t box[2] = {128, 128};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult rc = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), gdim, gstride, box,
                               estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) return set_error(PIPNN_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)rc);
    return PIPNN_OK;
}

int encode_rows_map(CUtensorMap *map, const __nv_bfloat16 *base, uint64_t n, uint32_t kp, bool gather) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return set_error(PIPNN_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    if (n >= 0x7FFFFFFFull) return set_error(PIPNN_EUNSUPPORTED, "a tensor map addresses fewer than 2^31 rows");
    const cuuint64_t gdim[2] = {kp, n};
    const cuuint64_t gstride[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {64, gather ? 1u : 128u};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult rc = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), gdim,
                               gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) return set_error(PIPNN_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)rc);
    return PIPNN_OK;
}

namespace {
// One warp waits, through the engines' bounded wait, on an mbarrier that nothing ever arrives on.
__global__ void wait_probe_kernel(unsigned long long limit_ns, unsigned *err) {
    __shared__ __align__(8) unsigned long long bar_storage;
    __shared__ int abort_flag;
    const uint32_t bar = tc::smem_u32(&bar_storage);
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool ok = tc::mbar_wait_limit(bar, 0, &abort_flag, err, limit_ns);
    (void)__all_sync(0xffffffffu, ok);
}
}  // namespace

}  // namespace pipnn

// Exercises the bounded device-side wait that every tensor-core engine uses: a wait on an
// mbarrier that is never completed must give up after limit_ns and report PIPNN_ETIMEOUT, and the
// context must stay usable.  Failure detection without a fault: no GPU state is harmed.
extern "C" int pipnn_debug_wait_probe(uint64_t limit_ns) {
    using namespace pipnn;
    clear_error();
    unsigned *err = nullptr;
    if (!alloc_budget_take(4)) return set_error(PIPNN_ENOMEM, "allocation budget spent");
    PIPNN_CUDA(cudaMallocAsync(&err, sizeof(unsigned), stream()));
    cudaMemsetAsync(err, 0, sizeof(unsigned), stream());
    wait_probe_kernel<<<1, 32, 0, stream()>>>(limit_ns, err);
    cudaError_t e = cudaGetLastError();
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream());
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream());
    cudaFreeAsync(err, stream());
    if (e != cudaSuccess) return set_error(PIPNN_ECUDA, "wait probe: %s", cudaGetErrorString(e));
    if (h & DERR_TIMEOUT) return set_error(PIPNN_ETIMEOUT, "wait probe: the bounded wait gave up after %llu ns",
                                           (unsigned long long)limit_ns);
    return PIPNN_OK;
}
