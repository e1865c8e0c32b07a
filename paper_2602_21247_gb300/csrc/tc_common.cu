// tc_common.cu -- host helpers of the tcgen05 engines: BF16 operand copies and TMA tensor maps.
#include "tc_common.cuh"

namespace pipnn {

namespace {

// One thread per 16-byte output chunk (8 BF16 values) of the padded copy.
__global__ void stage_rows_kernel(const void *X, uint32_t d, uint32_t kp, int dtype, const uint32_t *ids,
                                  uint64_t M, __nv_bfloat16 *out) {
    const uint32_t per_row = kp / 8;
    const uint64_t total = M * per_row;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t row = i / per_row;
        const uint32_t c = (uint32_t)(i % per_row);
        const uint64_t src = (uint64_t)(ids ? ids[row] : row) * d;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            float lo = 0.0f, hi = 0.0f;
            const uint32_t t = c * 8 + 2 * h;
            if (t < d) lo = dtype == PIPNN_U8 ? (float)static_cast<const uint8_t *>(X)[src + t]
                                              : (float)static_cast<const int8_t *>(X)[src + t];
            if (t + 1 < d) hi = dtype == PIPNN_U8 ? (float)static_cast<const uint8_t *>(X)[src + t + 1]
                                                  : (float)static_cast<const int8_t *>(X)[src + t + 1];
            w[h] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
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
    stage_rows_kernel<<<grid_for(M * (kp / 8), 256), 256, 0, stream()>>>(X, d, kp, dtype, ids, M, out);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

int encode_rows_map(CUtensorMap *map, const __nv_bfloat16 *base, uint64_t n, uint32_t kp, bool gather) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            !fn) {
            cudaGetLastError();
            return set_error(PIPNN_ECUDA, "cuTensorMapEncodeTiled is unavailable");
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
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

}  // namespace pipnn
