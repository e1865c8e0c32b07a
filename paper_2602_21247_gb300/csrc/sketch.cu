// sketch.cu -- A0: sketches Sketch(v) = [v . H_i] (Sec. 3 "Implementation") and squared norms.
//
// One thread per point (four coordinates per step when d % 4 == 0).  Every sketch coordinate is a
// binary32 fused-multiply-add chain over the point's coordinates in index order, so it equals the
// CPU evaluation of the same definition bit for bit.  Squared norms: binary32 FMA chain for float data, exact int32 for byte data.  The
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

// The same chains, four coordinates at a time: the hyperplanes staged in shared memory (one
// 16-byte read gives four coefficients of one hyperplane), the point's coordinates read four at a
// time (d % 4 == 0, rows aligned).  Every accumulator still adds its terms in index order.
template <int DT>
__global__ void __launch_bounds__(128) sketch_kernel_vec(const void *X, uint64_t n, uint32_t d, const float *H,
                                                         uint32_t m, float *S, void *sqnorm, unsigned *err) {
    extern __shared__ float4 sk_h[];  // m rows of d / 4 float4
    const uint32_t d4 = d / 4;
    for (uint32_t e = threadIdx.x; e < m * d4; e += blockDim.x) sk_h[e] = reinterpret_cast<const float4 *>(H)[e];
    __syncthreads();
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        float acc[MMAX];
#pragma unroll
        for (int i = 0; i < MMAX; i++) acc[i] = 0.0f;
        float nf = 0.0f;
        int ni = 0;
        bool finite = true;
        for (uint32_t t4 = 0; t4 < d4; t4++) {
            float x[4];
            if (DT == PIPNN_F32) {
                const float4 v = reinterpret_cast<const float4 *>(X)[p * d4 + t4];
                x[0] = v.x;
                x[1] = v.y;
                x[2] = v.z;
                x[3] = v.w;
            } else {
                const uint32_t w = reinterpret_cast<const uint32_t *>(X)[p * d4 + t4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t b = (w >> (8 * q)) & 0xFFu;
                    x[q] = DT == PIPNN_U8 ? (float)b : (float)(int)(int8_t)(uint8_t)b;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                if (DT == PIPNN_F32) {
                    finite = finite && isfinite(x[q]);
                    nf = __fmaf_rn(x[q], x[q], nf);
                } else {
                    const int xi = (int)x[q];
                    ni += xi * xi;
                }
            }
#pragma unroll
            for (int i = 0; i < MMAX; i++) {
                if ((uint32_t)i < m) {
                    const float4 h = sk_h[i * d4 + t4];
                    acc[i] = __fmaf_rn(x[0], h.x, acc[i]);
                    acc[i] = __fmaf_rn(x[1], h.y, acc[i]);
                    acc[i] = __fmaf_rn(x[2], h.z, acc[i]);
                    acc[i] = __fmaf_rn(x[3], h.w, acc[i]);
                }
            }
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

}  // namespace

int sketch_points(const void *X, uint64_t n, uint32_t d, int dtype, const float *H, uint32_t m, float *S,
                  void *sqnorm) {
    // m == 0 with S == nullptr computes squared norms only
    if (m > MMAX || (m < 1 && S)) return set_error(PIPNN_EINVAL, "hash_bits %u outside 1..16", m);
    unsigned *err = device_error_word();
    unsigned grid = grid_for(n, 128);
    const size_t hbytes = (size_t)m * d * 4;
    const size_t xalign = dtype == PIPNN_F32 ? 16 : 4;
    if (m >= 1 && S && d % 4 == 0 && hbytes <= 48 * 1024 && reinterpret_cast<uintptr_t>(X) % xalign == 0 &&
        reinterpret_cast<uintptr_t>(H) % 16 == 0) {
        if (dtype == PIPNN_F32)
            sketch_kernel_vec<PIPNN_F32><<<grid, 128, hbytes, stream()>>>(X, n, d, H, m, S, sqnorm, err);
        else if (dtype == PIPNN_U8)
            sketch_kernel_vec<PIPNN_U8><<<grid, 128, hbytes, stream()>>>(X, n, d, H, m, S, sqnorm, err);
        else
            sketch_kernel_vec<PIPNN_I8><<<grid, 128, hbytes, stream()>>>(X, n, d, H, m, S, sqnorm, err);
        PIPNN_LAUNCH_CHECK();
        return PIPNN_OK;
    }
    if (dtype == PIPNN_F32) sketch_kernel<PIPNN_F32><<<grid, 128, 0, stream()>>>(X, n, d, H, m, S, sqnorm, err);
    else if (dtype == PIPNN_U8) sketch_kernel<PIPNN_U8><<<grid, 128, 0, stream()>>>(X, n, d, H, m, S, sqnorm, err);
    else sketch_kernel<PIPNN_I8><<<grid, 128, 0, stream()>>>(X, n, d, H, m, S, sqnorm, err);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

}  // namespace pipnn
