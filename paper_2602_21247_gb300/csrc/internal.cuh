// internal.cuh -- shared host/device plumbing of the PiPNN CUDA library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "pipnn.h"

namespace pipnn {

// One run of candidate edges for HashPrune: dst[e] receives src[e] at dissimilarity dist[e].
struct EdgeSegment {
    const uint32_t *dst;
    const uint32_t *src;
    const float *dist;
    uint64_t count;
};

// ---------------------------------------------------------------------------------------------
// Errors.  Every host routine returns a PIPNN_* status; the message goes to a thread-local
// buffer read by pipnn_last_error().
// ---------------------------------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
const char *error_message();
void clear_error();

#define PIPNN_CUDA(call)                                                                      \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (e_ == cudaErrorMemoryAllocation)                                              \
                return ::pipnn::set_error(PIPNN_ENOMEM, "%s: %s (%s:%d)", #call,              \
                                          cudaGetErrorString(e_), __FILE__, __LINE__);        \
            return ::pipnn::set_error(PIPNN_ECUDA, "%s: %s (%s:%d)", #call,                   \
                                      cudaGetErrorString(e_), __FILE__, __LINE__);            \
        }                                                                                     \
    } while (0)

#define PIPNN_TRY(expr)                                                                       \
    do {                                                                                      \
        int rc_ = (expr);                                                                     \
        if (rc_ != PIPNN_OK) return rc_;                                                      \
    } while (0)

// counts this thread's kernel launches (every launch site is followed by this check)
void count_launch();
uint64_t launch_count();
#define PIPNN_LAUNCH_CHECK()                                                                  \
    do {                                                                                      \
        ::pipnn::count_launch();                                                              \
        PIPNN_CUDA(cudaGetLastError());                                                       \
    } while (0)

cudaStream_t stream();

// Device-side error word: kernels OR bits into it; checked at synchronisation points.
enum : unsigned {
    DERR_NONFINITE = 1u,   // a float input coordinate is NaN or infinite
    DERR_RANGE = 2u,       // an id or index outside its valid range
    DERR_CAPACITY = 4u,    // a bounded buffer overflowed (the host retries or fails)
    DERR_TIMEOUT = 8u,     // a bounded wait gave up
};
unsigned *device_error_word();
int check_device_error(const char *where);   // synchronises the stream

// ---------------------------------------------------------------------------------------------
// Failure injection on the host (pipnn_debug_set_alloc_limit): every device allocation of the
// library is charged against an optional byte budget and fails with PIPNN_ENOMEM once the budget
// is spent, exactly as a failing cudaMallocAsync would.
// ---------------------------------------------------------------------------------------------
bool alloc_budget_take(size_t bytes);

// ---------------------------------------------------------------------------------------------
// Stream-ordered device allocations released when the owning Workspace goes out of scope.
// ---------------------------------------------------------------------------------------------
class Workspace {
  public:
    Workspace() = default;
    Workspace(const Workspace &) = delete;
    Workspace &operator=(const Workspace &) = delete;
    ~Workspace() { release(); }
    template <typename T>
    int alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        if (!alloc_budget_take(count * sizeof(T)))
            return set_error(PIPNN_ENOMEM, "device allocation of %zu bytes refused: allocation budget spent",
                             count * sizeof(T));
        cudaError_t e = cudaMallocAsync(&q, count * sizeof(T), stream());
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(PIPNN_ENOMEM, "device allocation of %zu bytes failed: %s",
                             count * sizeof(T), cudaGetErrorString(e));
        }
        ptrs_.push_back(q);
        *p = static_cast<T *>(q);
        return PIPNN_OK;
    }
    template <typename T>
    int zeros(T **p, size_t count) {
        PIPNN_TRY(alloc(p, count));
        PIPNN_CUDA(cudaMemsetAsync(*p, 0, (count ? count : 1) * sizeof(T), stream()));
        return PIPNN_OK;
    }
    // hands ownership of p to the caller
    void detach(void *p) {
        for (auto &q : ptrs_)
            if (q == p) q = nullptr;
    }
    void release() {
        for (void *q : ptrs_)
            if (q) cudaFreeAsync(q, stream());
        ptrs_.clear();
    }

  private:
    std::vector<void *> ptrs_;
};

int dev_alloc_raw(void **p, size_t bytes);   // outside any workspace (library-owned outputs)
void dev_free_raw(void *p);

// CUDA-event time of the launches issued on the library stream between construction and stop()
// (nothing is recorded when out is null or the events cannot be made).
struct LaunchTimer {
    float *out;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    explicit LaunchTimer(float *o) : out(o) {
        if (!out) return;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            cudaGetLastError();
            out = nullptr;
            return;
        }
        cudaEventRecord(e0, stream());
    }
    void stop() {
        if (!out) return;
        cudaEventRecord(e1, stream());
        if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(out, e0, e1);
        else cudaGetLastError();
    }
    ~LaunchTimer() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// ---------------------------------------------------------------------------------------------
// Small device utilities
// ---------------------------------------------------------------------------------------------
// exclusive prefix sum of n uint64 values (in may equal out); total written to *total_dev
int exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *total_dev,
                       Workspace &ws);
// the same with caller-provided scratch for the per-tile totals (no allocation);
// scratch holds scan_scratch_elems(n) values
size_t scan_scratch_elems(uint64_t n);
int exclusive_scan_u64_scratch(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *total_dev,
                               uint64_t *scratch);
// copy one device value to the host (synchronises the stream)
int read_u64(const uint64_t *dev, uint64_t *host);

// Tiles: for groups of sizes size[g], tile t covers rows [row0, row0 + tile) of group grp[t].
// Produces tile_grp/tile_row0 arrays of total ceil(size/tile) entries; total on host.
int make_tiles(const uint32_t *size, uint64_t groups, uint32_t tile, uint32_t **tile_grp,
               uint32_t **tile_row0, uint64_t *num_tiles, Workspace &ws);

inline unsigned grid_for(uint64_t work, unsigned block, unsigned cap = 152u * 64u) {
    uint64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ---------------------------------------------------------------------------------------------
// Device arithmetic shared by the kernels
// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, Weyl key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c0), lo0 = m0 * c0;
        uint32_t hi1 = __umulhi(m1, c2), lo1 = m1 * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Leader-sample priority of point pt in subproblem `sub` (Alg. 5 SampleLeaders).
__device__ __forceinline__ uint32_t leader_priority(uint64_t seed, uint64_t sub, uint32_t pt) {
    uint32_t c0 = pt, c1 = (uint32_t)sub, c2 = (uint32_t)(sub >> 32), c3 = 0x1EADu;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    return c0;
}

// Identity of the subproblem carved around `leader` inside `parent`.
__device__ __forceinline__ uint64_t child_identity(uint64_t seed, uint64_t parent, uint32_t leader) {
    uint32_t c0 = leader, c1 = (uint32_t)parent, c2 = (uint32_t)(parent >> 32), c3 = 0xC41Du;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    return ((uint64_t)c1 << 32) | c0;
}

// Order-preserving 32-bit image of a binary32 value (no NaN; -0 never arises here).
__device__ __forceinline__ uint32_t f32_order(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float f32_unorder(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// Reservoir slot of Alg. 3: [ordered bf16(dist):16][id:32][hash:16].
__device__ __forceinline__ uint64_t reservoir_slot(float dist, uint32_t id, uint32_t h) {
    __nv_bfloat16 b = __float2bfloat16_rn(dist);
    uint16_t bits = __bfloat16_as_ushort(b);
    uint16_t ord = (bits & 0x8000u) ? (uint16_t)~bits : (uint16_t)(bits | 0x8000u);
    return ((uint64_t)ord << 48) | ((uint64_t)id << 16) | (uint64_t)(h & 0xFFFFu);
}

}  // namespace pipnn
