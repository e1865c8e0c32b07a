// util.cu -- error state, stream, device error word, prefix sums and tile tables.
#include "internal.cuh"

#include <atomic>

#include <cstring>

namespace pipnn {

static thread_local char g_msg[1024];
static thread_local cudaStream_t g_stream = nullptr;
static thread_local unsigned *g_err_word = nullptr;
static thread_local uint64_t g_launches = 0;

void count_launch() { g_launches++; }
uint64_t launch_count() { return g_launches; }

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}
const char *error_message() { return g_msg; }
void clear_error() { g_msg[0] = 0; }

cudaStream_t stream() { return g_stream; }
void set_stream(cudaStream_t s) { g_stream = s; }
unsigned *device_error_word() { return g_err_word; }
void set_device_error_word(unsigned *p) { g_err_word = p; }

int check_device_error(const char *where) {
    PIPNN_CUDA(cudaStreamSynchronize(stream()));
    unsigned *w = device_error_word();
    if (!w) return PIPNN_OK;
    unsigned h = 0;
    PIPNN_CUDA(cudaMemcpy(&h, w, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (h & DERR_NONFINITE) return set_error(PIPNN_EINVAL, "%s: non-finite input coordinate", where);
    if (h & DERR_RANGE) return set_error(PIPNN_EINVAL, "%s: id or index out of range", where);
    if (h & DERR_TIMEOUT) return set_error(PIPNN_ETIMEOUT, "%s: bounded device wait gave up", where);
    if (h & DERR_CAPACITY) return set_error(PIPNN_ECUDA, "%s: internal buffer capacity exceeded", where);
    return PIPNN_OK;
}

namespace {
std::atomic<uint64_t> g_alloc_left{~0ull};  // bytes the budget still allows; ~0 = unlimited
}  // namespace

bool alloc_budget_take(size_t bytes) {
    uint64_t left = g_alloc_left.load();
    for (;;) {
        if (left == ~0ull) return true;
        if (left < bytes) return false;
        if (g_alloc_left.compare_exchange_weak(left, left - bytes)) return true;
    }
}

int dev_alloc_raw(void **p, size_t bytes) {
    *p = nullptr;
    if (!alloc_budget_take(bytes))
        return set_error(PIPNN_ENOMEM, "device allocation of %zu bytes refused: allocation budget spent", bytes);
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 1, stream());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(PIPNN_ENOMEM, "device allocation of %zu bytes failed: %s", bytes,
                         cudaGetErrorString(e));
    }
    return PIPNN_OK;
}
void dev_free_raw(void *p) {
    if (p) cudaFreeAsync(p, stream());
}

int read_u64(const uint64_t *dev, uint64_t *host) {
    PIPNN_CUDA(cudaMemcpyAsync(host, dev, sizeof(uint64_t), cudaMemcpyDeviceToHost, stream()));
    PIPNN_CUDA(cudaStreamSynchronize(stream()));
    return PIPNN_OK;
}

// ---------------------------------------------------------------------------------------------
// Exclusive prefix sum: each block scans 4096 values (1024 threads x 4), block totals are scanned
// recursively and added back.
// ---------------------------------------------------------------------------------------------
namespace {
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *warp_tot, uint64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    return warp_tot[warp] + inc - v;
}

__global__ void scan_tiles(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *tile_sums) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t total;
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t v[SCAN_ITEMS];
    uint64_t local = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        v[i] = base + i < n ? in[base + i] : 0;
        local += v[i];
    }
    uint64_t ex = block_exclusive_scan(local, warp_tot, &total);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void scan_add(uint64_t *out, uint64_t n, const uint64_t *tile_offsets) {
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    const uint64_t add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++)
        if (base + i < n) out[base + i] += add;
}

__global__ void copy_one(const uint64_t *src, uint64_t *dst) { *dst = *src; }

__global__ void tile_counts(const uint32_t *size, uint64_t groups, uint32_t tile, uint64_t *cnt) {
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < groups;
         g += (uint64_t)gridDim.x * blockDim.x)
        cnt[g] = (size[g] + tile - 1) / tile;
}

__global__ void tile_fill(const uint64_t *off, uint64_t groups, uint64_t total, uint32_t tile,
                          uint32_t *tile_grp, uint32_t *tile_row0) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        // largest g with off[g] <= q
        uint64_t lo = 0, hi = groups;
        while (hi - lo > 1) {
            uint64_t mid = (lo + hi) / 2;
            if (off[mid] <= q) lo = mid;
            else hi = mid;
        }
        tile_grp[q] = (uint32_t)lo;
        tile_row0[q] = (uint32_t)((q - off[lo]) * tile);
    }
}
}  // namespace

int exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *total_dev, Workspace &ws) {
    if (n == 0) {
        PIPNN_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), stream()));
        return PIPNN_OK;
    }
    uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint64_t *sums = nullptr;
    PIPNN_TRY(ws.alloc(&sums, tiles));
    scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, stream()>>>(in, out, n, sums);
    PIPNN_LAUNCH_CHECK();
    if (tiles == 1) {
        copy_one<<<1, 1, 0, stream()>>>(sums, total_dev);
        PIPNN_LAUNCH_CHECK();
        return PIPNN_OK;
    }
    PIPNN_TRY(exclusive_scan_u64(sums, sums, tiles, total_dev, ws));
    scan_add<<<(unsigned)tiles, SCAN_THREADS, 0, stream()>>>(out, n, sums);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

size_t scan_scratch_elems(uint64_t n) {
    size_t total = 1;
    for (uint64_t t = n;;) {
        uint64_t tiles = (t + SCAN_TILE - 1) / SCAN_TILE;
        total += tiles;
        if (tiles <= 1) break;
        t = tiles;
    }
    return total;
}

int exclusive_scan_u64_scratch(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *total_dev,
                               uint64_t *scratch) {
    if (n == 0) {
        PIPNN_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), stream()));
        return PIPNN_OK;
    }
    const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint64_t *sums = scratch;
    scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, stream()>>>(in, out, n, sums);
    PIPNN_LAUNCH_CHECK();
    if (tiles == 1) {
        copy_one<<<1, 1, 0, stream()>>>(sums, total_dev);
        PIPNN_LAUNCH_CHECK();
        return PIPNN_OK;
    }
    PIPNN_TRY(exclusive_scan_u64_scratch(sums, sums, tiles, total_dev, scratch + tiles));
    scan_add<<<(unsigned)tiles, SCAN_THREADS, 0, stream()>>>(out, n, sums);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

int make_tiles(const uint32_t *size, uint64_t groups, uint32_t tile, uint32_t **tile_grp,
               uint32_t **tile_row0, uint64_t *num_tiles, Workspace &ws) {
    *num_tiles = 0;
    if (groups == 0) return PIPNN_OK;
    uint64_t *cnt = nullptr, *tot = nullptr;
    PIPNN_TRY(ws.alloc(&cnt, groups));
    PIPNN_TRY(ws.alloc(&tot, 1));
    tile_counts<<<grid_for(groups, 256), 256, 0, stream()>>>(size, groups, tile, cnt);
    PIPNN_LAUNCH_CHECK();
    PIPNN_TRY(exclusive_scan_u64(cnt, cnt, groups, tot, ws));
    PIPNN_TRY(read_u64(tot, num_tiles));
    PIPNN_TRY(ws.alloc(tile_grp, *num_tiles));
    PIPNN_TRY(ws.alloc(tile_row0, *num_tiles));
    if (*num_tiles) {
        tile_fill<<<grid_for(*num_tiles, 256), 256, 0, stream()>>>(cnt, groups, *num_tiles, tile,
                                                                    *tile_grp, *tile_row0);
        PIPNN_LAUNCH_CHECK();
    }
    return PIPNN_OK;
}

}  // namespace pipnn

extern "C" int pipnn_debug_set_alloc_limit(uint64_t bytes) {
    pipnn::g_alloc_left.store(bytes ? bytes : ~0ull);
    return PIPNN_OK;
}
