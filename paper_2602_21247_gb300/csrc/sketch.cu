// sketch.cu -- A0: sketches Sketch(v) = [v . H_i] (Sec. 3 "Implementation") and squared norms.
//
// One thread per point.  Every sketch coordinate is a binary32 fused-multiply-add chain over the
// point's coordinates in index order, so it equals the CPU evaluation of the same definition bit
// for bit.  Squared norms: binary32 FMA chain for float data, exact int32 for byte data.  The
// pass also rejects non-finite float coordinates (NaN would make every comparison false).
#include "internal.cuh"

namespace pipnn {

namespace {
constexpr int MMAX = 16;

template <int DT>
__device__ __forceinline__ float coordf(const void *X, uint64_t i) {
    if (DT == PIPNN_F32) return static_cast<const float *>(X)[i];
    if (DT == PIPNN_U8) return (float)static_cast<const uint8_t *>(X)[i];
    return (float)static_cast<const int8_t *>(X)[i];
}

template <int DT>
__global__ void __launch_bounds__(128) sketch_kernel(const void *X, uint64_t n, uint32_t d, const float *H,
                                                     uint32_t m, float *S, void *sqnorm, unsigned *err) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        float acc[MMAX];
#pragma unroll
        for (int i = 0; i < MMAX; i++) acc[i] = 0.0f;
        float nf = 0.0f;
        int ni = 0;
        bool finite = true;
        const uint64_t base = p * d;
        for (uint32_t t = 0; t < d; t++) {
            const float x = coordf<DT>(X, base + t);
            if (DT == PIPNN_F32) {
                finite = finite && isfinite(x);
                nf = __fmaf_rn(x, x, nf);
            } else {
                const int xi = (int)x;
                ni += xi * xi;
            }
#pragma unroll
            for (int i = 0; i < MMAX; i++)
                if ((uint32_t)i < m) acc[i] = __fmaf_rn(x, __ldg(H + (size_t)i * d + t), acc[i]);
        }
#pragma unroll
        for (int i = 0; i < MMAX; i++)
            if ((uint32_t)i < m) S[p * m + i] = acc[i];
        if (sqnorm) {
            if (DT == PIPNN_F32) static_cast<float *>(sqnorm)[p] = nf;
            else static_cast<int32_t *>(sqnorm)[p] = ni;
        }
        if (!finite) atomicOr(err, DERR_NONFINITE);
    }
}

template <int DT>
__global__ void to_bf16_kernel(const void *X, uint64_t count, __nv_bfloat16 *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(coordf<DT>(X, i));
}
}  // namespace

int sketch_points(const void *X, uint64_t n, uint32_t d, int dtype, const float *H, uint32_t m, float *S,
                  void *sqnorm) {
    // m == 0 with S == nullptr computes squared norms only
    if (m > MMAX || (m < 1 && S)) return set_error(PIPNN_EINVAL, "hash_bits %u outside 1..16", m);
    unsigned *err = device_error_word();
    unsigned grid = grid_for(n, 128);
    if (dtype == PIPNN_F32) sketch_kernel<PIPNN_F32><<<grid, 128, 0, stream()>>>(X, n, d, H, m, S, sqnorm, err);
    else if (dtype == PIPNN_U8) sketch_kernel<PIPNN_U8><<<grid, 128, 0, stream()>>>(X, n, d, H, m, S, sqnorm, err);
    else sketch_kernel<PIPNN_I8><<<grid, 128, 0, stream()>>>(X, n, d, H, m, S, sqnorm, err);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

int points_to_bf16(const void *X, uint64_t count, int dtype, __nv_bfloat16 *out) {
    unsigned grid = grid_for(count, 256);
    if (dtype == PIPNN_F32) to_bf16_kernel<PIPNN_F32><<<grid, 256, 0, stream()>>>(X, count, out);
    else if (dtype == PIPNN_U8) to_bf16_kernel<PIPNN_U8><<<grid, 256, 0, stream()>>>(X, count, out);
    else to_bf16_kernel<PIPNN_I8><<<grid, 256, 0, stream()>>>(X, count, out);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

}  // namespace pipnn
