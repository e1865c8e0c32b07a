// prune.cu -- A6: Alg. 2 RobustPrune of every node's reservoir down to degree R (Sec. 4.3).
//
// One warp per node.  The reservoir's ids are ordered by (dissimilarity to the node, id) with a
// shared-memory bitonic sort; then the warp repeatedly admits the nearest live candidate y and
// removes, in parallel over lanes, every live z with alpha^2 * D(y,z) < D(x,z) (binary32).
// Dissimilarities use the defining order (binary32 FMA chain / exact integer), so the result
// equals the CPU evaluation of Alg. 2 bit for bit.
#include "allpairs.cuh"

namespace pipnn {

int sketch_points(const void *X, uint64_t n, uint32_t d, int dtype, const float *H, uint32_t m, float *S,
                  void *sqnorm);
bool prune_tc_eligible(int dtype, uint32_t d, uint64_t n, uint32_t l_max);
int final_prune_tc(const void *X, uint64_t n, uint32_t d, int dtype, const int32_t *sqn, const uint64_t *res,
                   const uint32_t *cnt, uint32_t l_max, uint32_t R, float alpha2, uint32_t *adj, uint32_t *deg,
                   float *ms_kernel, Workspace &ws);

namespace {
constexpr int PR_WARPS = 8;
constexpr int PR_MAX = 256;  // l_max bound

template <int DT, int MET>
struct Dis {
    // decision value as (order key, binary32 value)
    __device__ __forceinline__ static void eval(const void *X, uint32_t d, const int32_t *sqn, uint32_t a, uint32_t b,
                                                uint32_t &key, float &val) {
        if (DT == PIPNN_F32) {
            const float *x = static_cast<const float *>(X) + (uint64_t)a * d;
            const float *y = static_cast<const float *>(X) + (uint64_t)b * d;
            float acc = 0.0f;
            if (MET == PIPNN_L2) {
                for (uint32_t t = 0; t < d; t++) {
                    float df = __fsub_rn(__ldg(x + t), __ldg(y + t));
                    acc = __fmaf_rn(df, df, acc);
                }
            } else {
                for (uint32_t t = 0; t < d; t++) acc = __fmaf_rn(__ldg(x + t), __ldg(y + t), acc);
                acc = __fsub_rn(1.0f, acc);
            }
            key = f32_order(acc);
            val = acc;
        } else {
            const uint32_t dw = (d + 3) / 4;
            int dot = 0;
            for (uint32_t w = 0; w < dw; w++) dot = dot4<DT>(coord_word<DT>(X, a, d, w), coord_word<DT>(X, b, d, w), dot);
            const int D = sqn[a] + sqn[b] - 2 * dot;
            key = (uint32_t)D;
            val = __int2float_rn(D);
        }
    }
};

template <int DT, int MET>
__global__ void __launch_bounds__(PR_WARPS * 32) robust_prune(const void *X, uint64_t n, uint32_t d,
                                                             const int32_t *sqn, const uint64_t *res,
                                                             const uint32_t *cnt, uint32_t l_max, uint32_t R,
                                                             float alpha2, uint32_t *adj, uint32_t *deg,
                                                             unsigned *err) {
    __shared__ uint64_t keys[PR_WARPS][PR_MAX];
    __shared__ float dx[PR_WARPS][PR_MAX];
    __shared__ uint32_t alive[PR_WARPS][PR_MAX / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *K = keys[warp];
    float *DX = dx[warp];
    uint32_t *A = alive[warp];

    for (uint64_t v = (uint64_t)blockIdx.x * PR_WARPS + warp; v < n; v += (uint64_t)gridDim.x * PR_WARPS) {
        uint32_t c = cnt[v];
        if (c > l_max) c = l_max;
        uint32_t P = 32;
        while (P < c) P <<= 1;
        // (dissimilarity to v, id) keys
        for (uint32_t t = lane; t < P; t += 32) {
            uint64_t kk = ~0ull;
            if (t < c) {
                uint32_t id = (uint32_t)(res[v * l_max + t] >> 16);
                if (id < n) {
                    uint32_t ok;
                    float val;
                    Dis<DT, MET>::eval(X, d, sqn, (uint32_t)v, id, ok, val);
                    kk = ((uint64_t)ok << 32) | id;
                } else {
                    atomicOr(err, DERR_RANGE);
                }
            }
            K[t] = kk;
        }
        __syncwarp();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = lane; i < P; i += 32) {
                    uint32_t ixj = i ^ j;
                    if (ixj > i) {
                        uint64_t a = K[i], b = K[ixj];
                        bool asc = (i & k) == 0;
                        if ((a > b) == asc) {
                            K[i] = b;
                            K[ixj] = a;
                        }
                    }
                }
                __syncwarp();
            }
        }
        {
            uint32_t bad = 0;
            for (uint32_t t = lane; t < c; t += 32) bad += K[t] == ~0ull ? 1u : 0u;
            for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
            c -= bad;
        }
        for (uint32_t t = lane; t < c; t += 32) {
            uint32_t ord = (uint32_t)(K[t] >> 32);
            DX[t] = DT == PIPNN_F32 ? f32_unorder(ord) : __int2float_rn((int)ord);
        }
        for (uint32_t w = lane; w < PR_MAX / 32; w += 32) {
            uint32_t lo = w * 32;
            A[w] = lo >= c ? 0u : (c - lo >= 32 ? 0xFFFFFFFFu : ((1u << (c - lo)) - 1u));
        }
        __syncwarp();

        uint32_t e = 0, head = 0;
        while (e < R) {
            // next live candidate at or after head
            uint32_t h = 0xFFFFFFFFu;
            for (uint32_t w = head / 32; w < (c + 31) / 32; w++) {
                uint32_t bits = A[w] & (w == head / 32 ? (0xFFFFFFFFu << (head & 31)) : 0xFFFFFFFFu);
                if (bits) {
                    h = w * 32 + (__ffs(bits) - 1);
                    break;
                }
            }
            __syncwarp();
            if (h == 0xFFFFFFFFu) break;
            const uint32_t y = (uint32_t)K[h];
            if (lane == 0) {
                adj[v * R + e] = y;
                A[h / 32] &= ~(1u << (h & 31));
            }
            e++;
            head = h + 1;
            __syncwarp();
            for (uint32_t z = head + lane; z < c; z += 32) {
                if (!((A[z / 32] >> (z & 31)) & 1u)) continue;
                uint32_t ok;
                float dyz;
                Dis<DT, MET>::eval(X, d, sqn, y, (uint32_t)K[z], ok, dyz);
                if (__fmul_rn(alpha2, dyz) < DX[z]) atomicAnd(&A[z / 32], ~(1u << (z & 31)));
            }
            __syncwarp();
        }
        for (uint32_t t = e + lane; t < R; t += 32) adj[v * R + t] = 0xFFFFFFFFu;
        if (lane == 0) deg[v] = e;
        __syncwarp();
    }
}

// Shared-memory variant: the node's candidate rows (and its own) are staged once per node --
// with 16-byte cp.async copies all in flight when a row is a whole number of 16-byte chunks,
// else with word loads -- into rows whose 16-byte chunks are XOR-swizzled by row index (lanes
// reading different rows then hit different banks); keys (D(x,c), id) are sorted with the slot as
// payload and every D(y,z) of the prune loop reads shared memory only.  Same arithmetic and
// order as robust_prune.
struct PruneSmem {
    uint32_t dw, lmax, P, stride, smask;
    bool async16;
    size_t rows, keys, perm, dx, nz, alive, per_warp;
};

__host__ __device__ inline PruneSmem prune_smem_layout(int dtype, uint32_t d, uint32_t l_max) {
    PruneSmem L;
    L.dw = dtype == PIPNN_F32 ? d : (d + 3) / 4;
    L.lmax = l_max;
    L.P = 32;
    while (L.P < l_max) L.P <<= 1;
    const uint32_t row_bytes = dtype == PIPNN_F32 ? d * 4 : d;
    L.async16 = row_bytes % 16 == 0;
    L.stride = (L.dw + 3) & ~3u;                 // words per staged row (whole 16-byte chunks)
    const uint32_t nch = L.stride / 4;
    // the XOR must keep every chunk inside its row: full groups of 8 chunks, or a power of two
    L.smask = nch % 8 == 0 ? 7u : ((nch & (nch - 1)) == 0 ? nch - 1 : 0u);
    size_t o = 0;
    L.rows = o;
    o += (size_t)(l_max + 1) * L.stride * 4;
    o = (o + 7) & ~(size_t)7;
    L.keys = o;
    o += (size_t)L.P * 8;
    L.perm = o;
    o += (size_t)L.P * 2;
    o = (o + 3) & ~(size_t)3;
    L.dx = o;
    o += (size_t)l_max * 4;
    L.nz = o;
    o += (size_t)(l_max + 1) * 4;
    L.alive = o;
    o += (size_t)((l_max + 31) / 32) * 4;
    L.per_warp = (o + 15) & ~(size_t)15;
    return L;
}

// word w of a staged row sits at w ^ (xor_a << 2) (chunk index XOR-swizzled by row)
template <int DT, int MET>
__device__ __forceinline__ void dis_smem(const uint32_t *ra, uint32_t xa, const uint32_t *rb, uint32_t xb,
                                         uint32_t dw, int na, int nb, uint32_t &key, float &val) {
    xa <<= 2;
    xb <<= 2;
    if (DT == PIPNN_F32) {
        float acc = 0.0f;
        if (MET == PIPNN_L2) {
            for (uint32_t t = 0; t < dw; t++) {
                const float df = __fsub_rn(__uint_as_float(ra[t ^ xa]), __uint_as_float(rb[t ^ xb]));
                acc = __fmaf_rn(df, df, acc);
            }
        } else {
            for (uint32_t t = 0; t < dw; t++)
                acc = __fmaf_rn(__uint_as_float(ra[t ^ xa]), __uint_as_float(rb[t ^ xb]), acc);
            acc = __fsub_rn(1.0f, acc);
        }
        key = f32_order(acc);
        val = acc;
    } else {
        int dot = 0;
        for (uint32_t w = 0; w < dw; w++) dot = dot4<DT>(ra[w ^ xa], rb[w ^ xb], dot);
        const int D = na + nb - 2 * dot;
        key = (uint32_t)D;
        val = __int2float_rn(D);
    }
}

// Byte data with staged rows of at most 8 chunks (d <= 128): one operand's row in registers,
// the other read with 16-byte shared loads, four independent integer partial sums (exact in any
// order).
template <int DT>
__device__ __forceinline__ void row_to_regs(const uint32_t *row, uint32_t x, uint32_t nch, uint4 (&r)[8]) {
#pragma unroll
    for (int c = 0; c < 8; c++)
        r[c] = (uint32_t)c < nch ? *reinterpret_cast<const uint4 *>(row + (((uint32_t)c ^ x) << 2)) : make_uint4(0, 0, 0, 0);
}

template <int DT>
__device__ __forceinline__ int dot_regs(const uint4 (&y)[8], const uint32_t *zrow, uint32_t zx, uint32_t nch) {
    int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        if ((uint32_t)c < nch) {
            const uint4 z = *reinterpret_cast<const uint4 *>(zrow + (((uint32_t)c ^ zx) << 2));
            a0 = dot4<DT>(y[c].x, z.x, a0);
            a1 = dot4<DT>(y[c].y, z.y, a1);
            a2 = dot4<DT>(y[c].z, z.z, a2);
            a3 = dot4<DT>(y[c].w, z.w, a3);
        }
    }
    return (a0 + a1) + (a2 + a3);
}

template <int DT, int MET>
__global__ void robust_prune_smem(const void *X, uint64_t n, uint32_t d, const int32_t *sqn, const uint64_t *res,
                                  const uint32_t *cnt, uint32_t l_max, uint32_t R, float alpha2, uint32_t *adj,
                                  uint32_t *deg, unsigned *err) {
    extern __shared__ __align__(16) unsigned char pr_smem[];
    const PruneSmem L = prune_smem_layout(DT, d, l_max);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    unsigned char *base = pr_smem + (size_t)warp * L.per_warp;
    uint32_t *rows = reinterpret_cast<uint32_t *>(base + L.rows);   // (l_max + 1) x (dw + 1); row l_max = node
    uint64_t *K = reinterpret_cast<uint64_t *>(base + L.keys);
    uint16_t *perm = reinterpret_cast<uint16_t *>(base + L.perm);
    float *DX = reinterpret_cast<float *>(base + L.dx);
    int *NZ = reinterpret_cast<int *>(base + L.nz);
    uint32_t *A = reinterpret_cast<uint32_t *>(base + L.alive);
    const uint32_t stride = L.stride, sm = L.smask;

    for (uint64_t v = (uint64_t)blockIdx.x * nwarps + warp; v < n; v += (uint64_t)gridDim.x * nwarps) {
        uint32_t c = cnt[v];
        if (c > l_max) c = l_max;
        // stage the node and its candidates; invalid ids are dropped (and reported)
        uint32_t nvalid = 0;
        for (uint32_t t0 = 0; t0 < c; t0 += 32) {
            const uint32_t t = t0 + lane;
            uint32_t id = 0xFFFFFFFFu;
            if (t < c) {
                id = (uint32_t)(res[v * l_max + t] >> 16);
                if (id >= n) {
                    atomicOr(err, DERR_RANGE);
                    id = 0xFFFFFFFFu;
                }
            }
            const unsigned okm = __ballot_sync(0xffffffffu, id != 0xFFFFFFFFu);
            const uint32_t slot = nvalid + __popc(okm & ((1u << lane) - 1u));
            if (id != 0xFFFFFFFFu) {
                K[slot] = id;  // ids first; keys are formed below
                NZ[slot] = DT == PIPNN_F32 ? 0 : sqn[id];
            }
            nvalid += __popc(okm);
        }
        c = nvalid;
        __syncwarp();
        // candidate rows into rows 0..c-1, the node's own row into row l_max
        if (L.async16) {
            const uint32_t nch = stride / 4, row_bytes = DT == PIPNN_F32 ? d * 4 : d;
            const uint32_t total = (c + 1) * nch;
            for (uint32_t idx = lane; idx < total; idx += 32) {
                const uint32_t t = idx / nch, ch = idx - t * nch;
                const uint32_t id = t < c ? (uint32_t)K[t] : (uint32_t)v;
                const uint32_t row = t < c ? t : l_max;
                const char *src = static_cast<const char *>(X) + (uint64_t)id * row_bytes + ch * 16;
                const uint32_t dst = static_cast<uint32_t>(
                    __cvta_generic_to_shared(rows + (size_t)row * stride + ((ch ^ (row & sm)) << 2)));
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
        } else {
            // four independent loads per lane are in flight before their stores; the padding
            // words of a row (stride > dw) are written as zeros, as whole chunks are read back
            const uint32_t total = (c + 1) * stride;
            for (uint32_t b0 = 0; b0 < total; b0 += 128) {
                uint32_t vals[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t idx = b0 + u * 32 + lane;
                    vals[u] = 0;
                    if (idx < total) {
                        const uint32_t t = idx / stride, w = idx - t * stride;
                        const uint32_t id = t < c ? (uint32_t)K[t] : (uint32_t)v;
                        if (w < L.dw) {
                            if (DT == PIPNN_F32)
                                vals[u] = __float_as_uint(__ldg(static_cast<const float *>(X) + (uint64_t)id * d + w));
                            else
                                vals[u] = coord_word<DT>(X, id, d, w);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t idx = b0 + u * 32 + lane;
                    if (idx < total) {
                        const uint32_t t = idx / stride, w = idx - t * stride;
                        const uint32_t row = t < c ? t : l_max;
                        rows[(size_t)row * stride + (w ^ ((row & sm) << 2))] = vals[u];
                    }
                }
            }
        }
        if (lane == 0) NZ[l_max] = DT == PIPNN_F32 ? 0 : sqn[v];
        __syncwarp();
        const uint32_t *xr = rows + (size_t)l_max * stride;
        uint32_t P = 32;
        while (P < c) P <<= 1;
        const bool regs = DT != PIPNN_F32 && stride <= 32;
        uint4 xw[8];
        if (regs) row_to_regs<DT>(xr, l_max & sm, stride / 4, xw);
        for (uint32_t t = lane; t < P; t += 32) {
            uint64_t kk = ~0ull;
            if (t < c) {
                uint32_t ok;
                float val;
                if (regs) {
                    const int D = NZ[l_max] + NZ[t] - 2 * dot_regs<DT>(xw, rows + (size_t)t * stride, t & sm, stride / 4);
                    ok = (uint32_t)D;
                } else {
                    dis_smem<DT, MET>(xr, l_max & sm, rows + (size_t)t * stride, t & sm, L.dw, NZ[l_max], NZ[t], ok,
                                      val);
                }
                kk = ((uint64_t)ok << 32) | (uint32_t)K[t];
            }
            K[t] = kk;
            perm[t] = (uint16_t)t;
        }
        __syncwarp();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = lane; i < P; i += 32) {
                    const uint32_t ixj = i ^ j;
                    if (ixj > i) {
                        const uint64_t a = K[i], b = K[ixj];
                        const bool asc = (i & k) == 0;
                        if ((a > b) == asc) {
                            K[i] = b;
                            K[ixj] = a;
                            const uint16_t pa = perm[i];
                            perm[i] = perm[ixj];
                            perm[ixj] = pa;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (uint32_t t = lane; t < c; t += 32) {
            const uint32_t ord = (uint32_t)(K[t] >> 32);
            DX[t] = DT == PIPNN_F32 ? f32_unorder(ord) : __int2float_rn((int)ord);
        }
        for (uint32_t w = lane; w < (l_max + 31) / 32; w += 32) {
            const uint32_t lo = w * 32;
            A[w] = lo >= c ? 0u : (c - lo >= 32 ? 0xFFFFFFFFu : ((1u << (c - lo)) - 1u));
        }
        __syncwarp();

        uint32_t e = 0, head = 0;
        while (e < R) {
            uint32_t h = 0xFFFFFFFFu;
            for (uint32_t w = head / 32; w < (c + 31) / 32; w++) {
                const uint32_t bits = A[w] & (w == head / 32 ? (0xFFFFFFFFu << (head & 31)) : 0xFFFFFFFFu);
                if (bits) {
                    h = w * 32 + (__ffs(bits) - 1);
                    break;
                }
            }
            __syncwarp();
            if (h == 0xFFFFFFFFu) break;
            const uint32_t y = (uint32_t)K[h];
            const uint32_t ys = perm[h];
            if (lane == 0) {
                adj[v * R + e] = y;
                A[h / 32] &= ~(1u << (h & 31));
            }
            e++;
            head = h + 1;
            __syncwarp();
            const uint32_t *yr = rows + (size_t)ys * stride;
            const int ny = NZ[ys];
            uint4 yw[8];
            if (regs) row_to_regs<DT>(yr, ys & sm, stride / 4, yw);
            for (uint32_t z = head + lane; z < c; z += 32) {
                if (!((A[z / 32] >> (z & 31)) & 1u)) continue;
                const uint32_t zs = perm[z];
                uint32_t ok;
                float dyz;
                if (regs) {
                    dyz = __int2float_rn(ny + NZ[zs] - 2 * dot_regs<DT>(yw, rows + (size_t)zs * stride, zs & sm, stride / 4));
                } else {
                    dis_smem<DT, MET>(yr, ys & sm, rows + (size_t)zs * stride, zs & sm, L.dw, ny, NZ[zs], ok, dyz);
                }
                if (__fmul_rn(alpha2, dyz) < DX[z]) atomicAnd(&A[z / 32], ~(1u << (z & 31)));
            }
            __syncwarp();
        }
        for (uint32_t t = e + lane; t < R; t += 32) adj[v * R + t] = 0xFFFFFFFFu;
        if (lane == 0) deg[v] = e;
        __syncwarp();
    }
}

// Without the final prune: the first R reservoir entries in (distance, id) order.
__global__ void reservoir_to_graph(uint64_t n, const uint64_t *res, const uint32_t *cnt, uint32_t l_max, uint32_t R,
                                   uint32_t *adj, uint32_t *deg) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n * R; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = i / R;
        uint32_t t = (uint32_t)(i % R);
        uint32_t c = cnt[v] < R ? cnt[v] : R;
        adj[i] = t < c ? (uint32_t)(res[v * l_max + t] >> 16) : 0xFFFFFFFFu;
        if (t == 0) deg[v] = c;
    }
}
}  // namespace

int final_prune(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const int32_t *sqnorm_bytes,
                const uint64_t *res, const uint32_t *cnt, uint32_t l_max, uint32_t R, float alpha, int engine,
                uint32_t *adj, uint32_t *deg, float *ms_kernel) {
    if (l_max > PR_MAX) return set_error(PIPNN_EINVAL, "l_max %u exceeds %d", l_max, PR_MAX);
    Workspace ws;
    const int32_t *sqn = sqnorm_bytes;
    if (dtype != PIPNN_F32 && !sqn) {
        int32_t *tmp = nullptr;
        PIPNN_TRY(ws.alloc(&tmp, n));
        PIPNN_TRY(sketch_points(X, n, d, dtype, nullptr, 0, nullptr, tmp));
        sqn = tmp;
    }
    const float alpha2 = (float)((double)alpha * (double)alpha);
    if (n == 0) return PIPNN_OK;
    if (engine == PIPNN_LEAF_TC && prune_tc_eligible(dtype, d, n, l_max))
        return final_prune_tc(X, n, d, dtype, sqn, res, cnt, l_max, R, alpha2, adj, deg, ms_kernel, ws);
    const PruneSmem L = prune_smem_layout(dtype, d, l_max);
    const size_t budget = 200 * 1024;
    if (L.per_warp <= budget) {
        uint32_t wpb = (uint32_t)(budget / L.per_warp);
        if (wpb > 8) wpb = 8;
        const size_t smem = wpb * L.per_warp;
        const unsigned grid = grid_for(n, wpb, 152u * 64u);
        unsigned *err = device_error_word();
        LaunchTimer lt(ms_kernel);
#define PIPNN_PRS(DT, MET)                                                                                   \
    do {                                                                                                     \
        PIPNN_CUDA(cudaFuncSetAttribute(robust_prune_smem<DT, MET>,                                           \
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));            \
        robust_prune_smem<DT, MET><<<grid, wpb * 32, smem, stream()>>>(X, n, d, sqn, res, cnt, l_max, R, alpha2, \
                                                                      adj, deg, err);                        \
    } while (0)
        if (dtype == PIPNN_F32 && metric == PIPNN_L2) PIPNN_PRS(PIPNN_F32, PIPNN_L2);
        else if (dtype == PIPNN_F32) PIPNN_PRS(PIPNN_F32, PIPNN_IP);
        else if (dtype == PIPNN_U8) PIPNN_PRS(PIPNN_U8, PIPNN_L2);
        else PIPNN_PRS(PIPNN_I8, PIPNN_L2);
#undef PIPNN_PRS
        PIPNN_LAUNCH_CHECK();
        lt.stop();
        return PIPNN_OK;
    }
    const unsigned grid = grid_for(n, PR_WARPS, 152u * 16u);
    LaunchTimer lt(ms_kernel);
#define PIPNN_PR(DT, MET) \
    robust_prune<DT, MET><<<grid, PR_WARPS * 32, 0, stream()>>>(X, n, d, sqn, res, cnt, l_max, R, alpha2, adj, deg, \
                                                                device_error_word())
    if (dtype == PIPNN_F32 && metric == PIPNN_L2) PIPNN_PR(PIPNN_F32, PIPNN_L2);
    else if (dtype == PIPNN_F32) PIPNN_PR(PIPNN_F32, PIPNN_IP);
    else if (dtype == PIPNN_U8) PIPNN_PR(PIPNN_U8, PIPNN_L2);
    else PIPNN_PR(PIPNN_I8, PIPNN_L2);
#undef PIPNN_PR
    PIPNN_LAUNCH_CHECK();
    lt.stop();
    return PIPNN_OK;
}

namespace {
__global__ void sum_counts(const uint32_t *cnt, uint64_t n, uint32_t l_max, unsigned long long *out) {
    unsigned long long s = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        s += cnt[i] < l_max ? cnt[i] : l_max;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}
}  // namespace

int reservoir_total(const uint32_t *cnt, uint64_t n, uint32_t l_max, uint64_t *total) {
    Workspace ws;
    unsigned long long *d = nullptr;
    PIPNN_TRY(ws.zeros(&d, 1));
    if (n) {
        sum_counts<<<grid_for(n, 256, 152u * 8u), 256, 0, stream()>>>(cnt, n, l_max, d);
        PIPNN_LAUNCH_CHECK();
    }
    return read_u64(reinterpret_cast<uint64_t *>(d), total);
}

int reservoir_graph(uint64_t n, const uint64_t *res, const uint32_t *cnt, uint32_t l_max, uint32_t R, uint32_t *adj,
                    uint32_t *deg) {
    reservoir_to_graph<<<grid_for(n * R, 256), 256, 0, stream()>>>(n, res, cnt, l_max, R, adj, deg);
    PIPNN_LAUNCH_CHECK();
    return PIPNN_OK;
}

}  // namespace pipnn
