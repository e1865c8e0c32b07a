/*
 * pipnn_oracle.c -- plain, slow, CPU-only oracle of the PiPNN index-build path.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header, table or helper with the CUDA path;
 * every function restates the paper's definition in plain loops, in the paper's order:
 *
 *   Philox4x32-10 ........ counter-based generator of Salmon et al. (SC'11), used for the
 *                          random leader sample of Alg. 5 and for subproblem identities
 *   dissimilarity ........ Sec. 2 "dissimilarity measure"; squared L2, or 1 - <x,y> for inner
 *                          product.  Float data: one fused multiply-add per coordinate in index
 *                          order, binary32 round-to-nearest.  Byte data: exact integer sum.
 *   sketch ............... Sec. 3 "Implementation": Sketch(v) = [v . H_i]
 *   residualised hash .... Sec. 3, Eq. 1: bit i = [H_i . (c - p) >= 0], taken as
 *                          Sketch(c)_i >= Sketch(p)_i
 *   partition ............ Alg. 5 (randomized ball carving with multi-level fanout, Merge)
 *   pick ................. Sec. 4.2 / App. A.3: bi-directed k-NN inside every leaf
 *   HashPrune ............ Alg. 3 (streaming, reservoir sorted by hash, cached farthest) and
 *                          its closed form from the history-independence lemma (App. A.6)
 *   final prune .......... Alg. 2 RobustPrune, standard and lazy (App. A.3 "Optimizing
 *                          RobustPrune") variants
 *   evaluation ........... Alg. 1 BeamSearch, exact k-NN (Def. 1), k@k' recall (Def. 2)
 *
 * Readings where the paper is silent or ambiguous are listed in the design notes; the ones that
 * change arithmetic are restated at the function that takes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_F32 0
#define ORC_U8 1
#define ORC_I8 2
#define ORC_L2 0
#define ORC_IP 1

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* Depth at which Alg. 5 stops recursing and cuts an oversized bucket into runs (guard; the
 * paper's recursion has no explicit bound). */
#define ORC_DEPTH_CAP 12

typedef struct {
    uint32_t c_max, c_min, max_leaders;
    float p_samp;
    uint32_t fanout[4];
    uint32_t fanout_levels;
    uint32_t leaf_k, hash_bits, l_max, R;
    float alpha;
    int32_t final_prune;
    int32_t pick_direction; /* App. A.3: 0 bi-directed k-NN, 1 directed k-NN, 2 inverted k-NN */
} orc_params;

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",   */
/* SC'11): ten rounds of two 32x32->64 multiplications on a 4-word counter, with the 2-word key */
/* advanced by the Weyl constants between rounds.                                              */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random priority of point `pt` inside subproblem `sub` (leader sample of Alg. 5): word 0 of
 * Philox(counter = (pt, sub_lo, sub_hi, 0x1EAD), key = seed). */
static uint32_t leader_priority(uint64_t seed, uint64_t sub, uint32_t pt)
{
    uint32_t c[4] = {pt, (uint32_t)sub, (uint32_t)(sub >> 32), 0x1EADu};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(c, k, o);
    return o[0];
}

/* Identity of the child subproblem carved around leader `leader` of subproblem `parent`:
 * words 0,1 of Philox(counter = (leader, parent_lo, parent_hi, 0xC41D), key = seed).  The root
 * subproblem has identity 0.  Identities make the partition a function of the seed alone
 * (determinism lemma, App. A.5). */
static uint64_t child_identity(uint64_t seed, uint64_t parent, uint32_t leader)
{
    uint32_t c[4] = {leader, (uint32_t)parent, (uint32_t)(parent >> 32), 0xC41Du};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(c, k, o);
    return ((uint64_t)o[1] << 32) | o[0];
}

/* ------------------------------------------------------------------------------------------ */
/* Dissimilarity (Sec. 2).  Returned as a double that holds the exact decision value: the      */
/* binary32 result for float data, the exact integer for byte data.                            */
/* ------------------------------------------------------------------------------------------ */
static size_t elem_size(int dtype) { return dtype == ORC_F32 ? 4 : 1; }

static double dis_vec(const void *a, const void *b, uint32_t d, int dtype, int metric)
{
    if (dtype == ORC_F32) {
        const float *x = (const float *)a, *y = (const float *)b;
        float acc = 0.0f;
        if (metric == ORC_L2) {
            for (uint32_t t = 0; t < d; t++) {
                float df = x[t] - y[t];
                acc = fmaf(df, df, acc);
            }
            return (double)acc;
        }
        for (uint32_t t = 0; t < d; t++) acc = fmaf(x[t], y[t], acc);
        return (double)(1.0f - acc);
    }
    int64_t s = 0;
    if (dtype == ORC_U8) {
        const uint8_t *x = (const uint8_t *)a, *y = (const uint8_t *)b;
        for (uint32_t t = 0; t < d; t++) {
            int64_t df = (int64_t)x[t] - (int64_t)y[t];
            s += df * df;
        }
    } else {
        const int8_t *x = (const int8_t *)a, *y = (const int8_t *)b;
        for (uint32_t t = 0; t < d; t++) {
            int64_t df = (int64_t)x[t] - (int64_t)y[t];
            s += df * df;
        }
    }
    return (double)s;
}

static const void *row(const void *X, uint64_t i, uint32_t d, int dtype)
{
    return (const char *)X + (size_t)i * d * elem_size(dtype);
}

double orc_dissimilarity(const void *X, uint32_t d, int dtype, int metric, uint64_t a, uint64_t b)
{
    return dis_vec(row(X, a, d, dtype), row(X, b, d, dtype), d, dtype, metric);
}

/* Exact reference value in double precision (error reports only). */
static double dis_vec_f64(const void *a, const void *b, uint32_t d, int dtype, int metric)
{
    double acc = 0.0;
    for (uint32_t t = 0; t < d; t++) {
        double x, y;
        if (dtype == ORC_F32) { x = ((const float *)a)[t]; y = ((const float *)b)[t]; }
        else if (dtype == ORC_U8) { x = ((const uint8_t *)a)[t]; y = ((const uint8_t *)b)[t]; }
        else { x = ((const int8_t *)a)[t]; y = ((const int8_t *)b)[t]; }
        if (metric == ORC_L2) acc += (x - y) * (x - y);
        else acc += x * y;
    }
    return metric == ORC_L2 ? acc : 1.0 - acc;
}

void orc_dissimilarity_f64_pairs(const void *X, uint32_t d, int dtype, int metric,
                                 const uint32_t *a, const uint32_t *b, uint64_t count, double *out)
{
    for (uint64_t i = 0; i < count; i++)
        out[i] = dis_vec_f64(row(X, a[i], d, dtype), row(X, b[i], d, dtype), d, dtype, metric);
}

void orc_dissimilarity_pairs(const void *X, uint32_t d, int dtype, int metric,
                             const uint32_t *a, const uint32_t *b, uint64_t count, double *out)
{
    for (uint64_t i = 0; i < count; i++) out[i] = orc_dissimilarity(X, d, dtype, metric, a[i], b[i]);
}

/* ------------------------------------------------------------------------------------------ */
/* Sketches (Sec. 3 "Implementation"): S[p][i] = sum_t x_t * H[i][t], one fused multiply-add   */
/* per coordinate in index order (binary32).  Squared norms are returned in double.           */
/* ------------------------------------------------------------------------------------------ */
static float coord(const void *x, uint32_t t, int dtype)
{
    if (dtype == ORC_F32) return ((const float *)x)[t];
    if (dtype == ORC_U8) return (float)((const uint8_t *)x)[t];
    return (float)((const int8_t *)x)[t];
}

int orc_sketch(const void *X, uint64_t n, uint32_t d, int dtype, const float *H, uint32_t m,
               float *S, double *sqnorm)
{
    if (!X || !H || !S || m == 0 || m > 16 || d == 0) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)n; p++) {
        const void *x = row(X, (uint64_t)p, d, dtype);
        for (uint32_t i = 0; i < m; i++) {
            float acc = 0.0f;
            for (uint32_t t = 0; t < d; t++) acc = fmaf(coord(x, t, dtype), H[(size_t)i * d + t], acc);
            S[(size_t)p * m + i] = acc;
        }
        if (sqnorm) {
            double s = 0.0;
            for (uint32_t t = 0; t < d; t++) {
                double v = coord(x, t, dtype);
                s += v * v;
            }
            sqnorm[p] = s;
        }
    }
    return ORC_OK;
}

/* Residualised hash h_p(c) (Eq. 1): bit i is set iff H_i . (c - p) >= 0, evaluated on the
 * sketches as Sketch(c)_i >= Sketch(p)_i.  Bit i sits at 2^i. */
static uint32_t residual_hash(const float *S, uint32_t m, uint32_t p, uint32_t c)
{
    uint32_t h = 0;
    for (uint32_t i = 0; i < m; i++)
        if (S[(size_t)c * m + i] >= S[(size_t)p * m + i]) h |= 1u << i;
    return h;
}

/* bf16 of a binary32 value, round to nearest, ties to even (the reservoir keeps a 2-byte float
 * distance, Sec. 3 "Implementation"). */
static uint16_t to_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return (uint16_t)((u >> 16) | 0x40u);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

/* Order-preserving map of a bf16 bit pattern onto unsigned 16-bit integers. */
static uint16_t bf16_order(uint16_t b) { return (b & 0x8000u) ? (uint16_t)~b : (uint16_t)(b | 0x8000u); }

/* Reservoir slot: [ordered bf16 distance : 16][candidate id : 32][hash : 16].  Unsigned order
 * of slots is the order (distance, id) that decides every comparison of Alg. 3. */
static uint64_t slot_of(float dist, uint32_t id, uint32_t h)
{
    return ((uint64_t)bf16_order(to_bf16(dist)) << 48) | ((uint64_t)id << 16) | (uint64_t)(h & 0xFFFFu);
}

uint64_t orc_slot(float dist, uint32_t id, uint32_t h) { return slot_of(dist, id, h); }

/* ------------------------------------------------------------------------------------------ */
/* Alg. 5 -- Randomized Ball Carving with multi-level fanout and Merge.                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint32_t *off, *mem;
    uint64_t nleaves, cap_leaves, nmem, cap_mem;
    int err;
} orc_leafset;

typedef struct {
    const void *X;
    uint32_t d;
    int dtype, metric;
    const orc_params *bp;
    uint64_t seed;
    uint64_t levels_seen;
} part_ctx;

static void leafset_emit(orc_leafset *L, const uint32_t *ids, uint64_t cnt)
{
    if (L->err) return;
    if (L->nleaves + 2 > L->cap_leaves) {
        uint64_t nc = L->cap_leaves ? 2 * L->cap_leaves : 1024;
        uint32_t *p = (uint32_t *)realloc(L->off, nc * sizeof(uint32_t));
        if (!p) { L->err = 1; return; }
        L->off = p; L->cap_leaves = nc;
    }
    if (L->nmem + cnt > L->cap_mem) {
        uint64_t nc = L->cap_mem ? 2 * L->cap_mem : 65536;
        while (nc < L->nmem + cnt) nc *= 2;
        uint32_t *p = (uint32_t *)realloc(L->mem, nc * sizeof(uint32_t));
        if (!p) { L->err = 1; return; }
        L->mem = p; L->cap_mem = nc;
    }
    if (L->nleaves == 0) L->off[0] = 0;
    memcpy(L->mem + L->nmem, ids, cnt * sizeof(uint32_t));
    L->nmem += cnt;
    L->nleaves++;
    L->off[L->nleaves] = (uint32_t)L->nmem;
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : x > y;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* Number of leaders of a subproblem of size np: l = max(2, min(ceil(P_samp * np), cap)), and
 * never more than np.  The ceiling is of the exact real product P_samp * np, where P_samp is the
 * binary32 parameter: writing P_samp = M * 2^E (M the integer significand), it is the integer
 * ceil(M * np / 2^-E), evaluated with a quotient and a remainder. */
static uint64_t ceil_of_product(float p, uint64_t np)
{
    uint32_t bits;
    memcpy(&bits, &p, 4);
    uint32_t biased = (bits >> 23) & 0xFFu;
    uint64_t M = biased ? ((bits & 0x7FFFFFu) | 0x800000u) : (bits & 0x7FFFFFu);
    int E = biased ? (int)biased - 150 : -149;
    uint64_t prod = M * np;
    if (E >= 0) return prod << E;
    int sh = -E;
    if (sh >= 64) return prod != 0;
    uint64_t q = prod >> sh, rem = prod - (q << sh);
    return q + (rem != 0);
}

uint64_t orc_ceil_of_product(float p, uint64_t np) { return ceil_of_product(p, np); }

static uint64_t leader_count(const orc_params *bp, uint64_t np)
{
    uint64_t l = ceil_of_product(bp->p_samp, np);
    if (l > bp->max_leaders) l = bp->max_leaders;
    if (l < 2) l = 2;
    if (l > np) l = np;
    return l;
}

static uint32_t fanout_at(const orc_params *bp, uint32_t depth)
{
    if (depth < bp->fanout_levels && depth < 4) return bp->fanout[depth] ? bp->fanout[depth] : 1;
    return 1;
}

/* Guard for a bucket that cannot be carved further (it is as large as its parent, or the depth
 * cap is reached): sort its members by id and cut them into ceil(|b| / C_max) consecutive runs
 * of near-equal size. */
static void cut_into_runs(orc_leafset *L, uint32_t *b, uint64_t nb, uint32_t c_max)
{
    qsort(b, nb, sizeof(uint32_t), cmp_u32);
    uint64_t k = (nb + c_max - 1) / c_max;
    for (uint64_t j = 0; j < k; j++) {
        uint64_t s = j * nb / k, e = (j + 1) * nb / k;
        leafset_emit(L, b + s, e - s);
    }
}

static void partition_rec(part_ctx *C, uint32_t *P, uint64_t np, uint32_t depth, uint64_t sub,
                          orc_leafset *L);

/* One leaf or subproblem produced by carving.  kind 0: leaf, 1: recurse with identity `child`. */
static void settle_bucket(part_ctx *C, uint32_t *b, uint64_t nb, uint64_t np_parent, uint32_t depth,
                          uint64_t child, orc_leafset *L)
{
    const orc_params *bp = C->bp;
    if (nb <= bp->c_max) {
        leafset_emit(L, b, nb);
        return;
    }
    if (nb == np_parent || depth + 1 >= ORC_DEPTH_CAP) {
        cut_into_runs(L, b, nb, bp->c_max);
        return;
    }
    partition_rec(C, b, nb, depth + 1, child, L);
}

static void partition_rec(part_ctx *C, uint32_t *P, uint64_t np, uint32_t depth, uint64_t sub,
                          orc_leafset *L)
{
    const orc_params *bp = C->bp;
    if (L->err) return;
    if (depth + 1 > C->levels_seen) C->levels_seen = depth + 1;
    /* line "if |P| <= C_max return {P}" */
    if (np <= bp->c_max) {
        leafset_emit(L, P, np);
        return;
    }
    /* SampleLeaders(P, P_samp * |P|): the l members with the smallest (priority, id). */
    uint64_t l = leader_count(bp, np);
    uint64_t *prio = (uint64_t *)malloc(np * sizeof(uint64_t));
    if (!prio) { L->err = 1; return; }
    for (uint64_t i = 0; i < np; i++)
        prio[i] = ((uint64_t)leader_priority(C->seed, sub, P[i]) << 32) | P[i];
    qsort(prio, np, sizeof(uint64_t), cmp_u64);
    uint32_t *lead = (uint32_t *)malloc(l * sizeof(uint32_t));
    if (!lead) { free(prio); L->err = 1; return; }
    for (uint64_t r = 0; r < l; r++) lead[r] = (uint32_t)prio[r];
    free(prio);

    /* local_fanout <- min(fanout(depth), l)  (the paper prints |P|; the number of leaders is the
     * only bound that makes sense, reading C1 of the design notes) */
    uint32_t f = fanout_at(bp, depth);
    if (f > l) f = (uint32_t)l;

    /* every point joins the buckets of its f nearest leaders; equidistant leaders are taken in
     * the order they were drawn (leader rank) */
    uint32_t *assign = (uint32_t *)malloc(np * f * sizeof(uint32_t));
    uint64_t *cnt = (uint64_t *)calloc(l, sizeof(uint64_t));
    if (!assign || !cnt) { free(lead); free(assign); free(cnt); L->err = 1; return; }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < (int64_t)np; i++) {
        double bd[64];
        uint32_t br[64];
        uint32_t have = 0;
        const void *x = row(C->X, P[i], C->d, C->dtype);
        for (uint64_t r = 0; r < l; r++) {
            double dv = dis_vec(x, row(C->X, lead[r], C->d, C->dtype), C->d, C->dtype, C->metric);
            /* ranks arrive in increasing order, so an equal distance never displaces */
            if (have == f && dv >= bd[f - 1]) continue;
            uint32_t pos = have < f ? have++ : f - 1;
            while (pos > 0 && dv < bd[pos - 1]) {
                bd[pos] = bd[pos - 1]; br[pos] = br[pos - 1];
                pos--;
            }
            bd[pos] = dv; br[pos] = (uint32_t)r;
        }
        for (uint32_t j = 0; j < f; j++) assign[(uint64_t)i * f + j] = br[j];
    }
    for (uint64_t i = 0; i < np * f; i++) cnt[assign[i]]++;
    uint64_t *start = (uint64_t *)malloc((l + 1) * sizeof(uint64_t));
    uint32_t *members = (uint32_t *)malloc(np * f * sizeof(uint32_t));
    if (!start || !members) { free(lead); free(assign); free(cnt); free(start); free(members); L->err = 1; return; }
    start[0] = 0;
    for (uint64_t r = 0; r < l; r++) start[r + 1] = start[r] + cnt[r];
    memset(cnt, 0, l * sizeof(uint64_t));
    for (uint64_t i = 0; i < np; i++)
        for (uint32_t j = 0; j < f; j++) {
            uint32_t r = assign[i * f + j];
            members[start[r] + cnt[r]++] = P[i];
        }
    free(assign);

    /* Merge(B, C_min, C_max): buckets below C_min, visited in leader-rank order (a uniformly
     * random order), are packed next-fit into groups that never exceed C_max.  A merged group
     * is a leaf (a point that reached two merged buckets appears once). */
    uint32_t *group = (uint32_t *)malloc((size_t)bp->c_max * sizeof(uint32_t));
    if (!group) { free(lead); free(cnt); free(start); free(members); L->err = 1; return; }
    uint64_t gsz = 0;
    for (uint64_t r = 0; r < l; r++) {
        uint64_t nb = start[r + 1] - start[r];
        if (nb == 0) continue;
        uint32_t *b = members + start[r];
        if (nb >= bp->c_min) {
            settle_bucket(C, b, nb, np, depth, child_identity(C->seed, sub, lead[r]), L);
            continue;
        }
        if (gsz + nb > bp->c_max) {
            qsort(group, gsz, sizeof(uint32_t), cmp_u32);
            uint64_t u = 0;
            for (uint64_t t = 0; t < gsz; t++)
                if (t == 0 || group[t] != group[t - 1]) group[u++] = group[t];
            leafset_emit(L, group, u);
            gsz = 0;
        }
        memcpy(group + gsz, b, nb * sizeof(uint32_t));
        gsz += nb;
    }
    if (gsz) {
        qsort(group, gsz, sizeof(uint32_t), cmp_u32);
        uint64_t u = 0;
        for (uint64_t t = 0; t < gsz; t++)
            if (t == 0 || group[t] != group[t - 1]) group[u++] = group[t];
        leafset_emit(L, group, u);
    }
    free(group);
    free(lead);
    free(cnt);
    free(start);
    free(members);
}

typedef struct {
    uint32_t *off, *mem;
    uint64_t nleaves, nmem;
    uint64_t levels;
} orc_leaves;

static int params_ok(const orc_params *bp)
{
    if (!bp) return 0;
    if (bp->c_max < 2 || bp->c_min > bp->c_max || bp->max_leaders < 2 || bp->max_leaders > 1024) return 0;
    if (!(bp->p_samp > 0.0f) || !(bp->p_samp <= 1.0f)) return 0;
    if (bp->fanout_levels > 4) return 0;
    for (uint32_t i = 0; i < bp->fanout_levels; i++)
        if (bp->fanout[i] < 1 || bp->fanout[i] > 32) return 0;
    if (bp->leaf_k < 1 || bp->leaf_k > 16) return 0;
    if (bp->hash_bits < 1 || bp->hash_bits > 16) return 0;
    if (bp->l_max < 1 || bp->l_max > 1024 || bp->R < 1 || bp->R > bp->l_max) return 0;
    if (!(bp->alpha >= 1.0f)) return 0;
    if (bp->pick_direction < 0 || bp->pick_direction > 2) return 0;
    return 1;
}

static int input_ok(const void *X, uint64_t n, uint32_t d, int dtype, int metric)
{
    if (!X || n == 0 || d == 0 || n >= 0xFFFFFFFFull) return 0;
    if (dtype < 0 || dtype > 2 || metric < 0 || metric > 1) return 0;
    if (dtype != ORC_F32 && metric == ORC_IP) return 0;
    if (dtype == ORC_F32) {
        const float *x = (const float *)X;
        for (uint64_t i = 0; i < n * (uint64_t)d; i++)
            if (!isfinite(x[i])) return 0;
    }
    return 1;
}

int orc_partition(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const orc_params *bp,
                  uint64_t seed, orc_leaves *out)
{
    if (!out || !params_ok(bp) || !input_ok(X, n, d, dtype, metric)) return ORC_EINVAL;
    memset(out, 0, sizeof(*out));
    uint32_t *all = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!all) return ORC_ENOMEM;
    for (uint64_t i = 0; i < n; i++) all[i] = (uint32_t)i;
    part_ctx C = {X, d, dtype, metric, bp, seed, 0};
    orc_leafset L;
    memset(&L, 0, sizeof(L));
    partition_rec(&C, all, n, 0, 0, &L);
    free(all);
    if (L.err) { free(L.off); free(L.mem); return ORC_ENOMEM; }
    out->off = L.off;
    out->mem = L.mem;
    out->nleaves = L.nleaves;
    out->nmem = L.nmem;
    out->levels = C.levels_seen;
    return ORC_OK;
}

void orc_leaves_free(orc_leaves *l)
{
    if (!l) return;
    free(l->off);
    free(l->mem);
    memset(l, 0, sizeof(*l));
}

/* ------------------------------------------------------------------------------------------ */
/* Pick (Sec. 4.2, App. A.3): for every member i of a leaf, its k nearest other members by     */
/* (dissimilarity, id); every picked pair (i, j) yields the candidates j -> reservoir(i) and   */
/* i -> reservoir(j) ("bi-directed k-NN").  App. A.3's variants keep one of the two: the       */
/* directed k-NN the edge from i to its neighbour j (j -> reservoir(i)), the inverted k-NN the */
/* edge to i from j (i -> reservoir(j)).  A leaf with repeated ids counts each id once.        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint32_t *dst, *src;
    float *dist;
    uint64_t count;
} orc_edges;

int orc_leaf_pick(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const uint32_t *off,
                  const uint32_t *mem, uint64_t nleaves, uint32_t k, int direction, orc_edges *out)
{
    if (!out || !X || !off || !mem || k < 1 || k > 16 || direction < 0 || direction > 2) return ORC_EINVAL;
    const uint64_t per_pick = direction == 0 ? 2 : 1;
    memset(out, 0, sizeof(*out));
    uint64_t *cnt = (uint64_t *)calloc(nleaves + 1, sizeof(uint64_t));
    uint32_t **uniq = (uint32_t **)calloc(nleaves ? nleaves : 1, sizeof(uint32_t *));
    uint64_t *usz = (uint64_t *)calloc(nleaves ? nleaves : 1, sizeof(uint64_t));
    if (!cnt || !uniq || !usz) { free(cnt); free(uniq); free(usz); return ORC_ENOMEM; }
    int err = 0;
    for (uint64_t b = 0; b < nleaves; b++) {
        uint64_t s = off[b], e = off[b + 1];
        uniq[b] = (uint32_t *)malloc((e - s + 1) * sizeof(uint32_t));
        if (!uniq[b]) { err = 1; break; }
        memcpy(uniq[b], mem + s, (e - s) * sizeof(uint32_t));
        qsort(uniq[b], e - s, sizeof(uint32_t), cmp_u32);
        uint64_t u = 0;
        for (uint64_t t = 0; t < e - s; t++) {
            if (uniq[b][t] >= n) { err = 1; break; }
            if (t == 0 || uniq[b][t] != uniq[b][t - 1]) uniq[b][u++] = uniq[b][t];
        }
        usz[b] = u;
        uint64_t kk = u > 0 ? (u - 1 < k ? u - 1 : k) : 0;
        cnt[b + 1] = cnt[b] + per_pick * u * kk;
    }
    if (!err) {
        uint64_t total = cnt[nleaves];
        out->dst = (uint32_t *)malloc((total + 1) * sizeof(uint32_t));
        out->src = (uint32_t *)malloc((total + 1) * sizeof(uint32_t));
        out->dist = (float *)malloc((total + 1) * sizeof(float));
        if (!out->dst || !out->src || !out->dist) err = 1;
        out->count = total;
    }
    if (!err) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t b = 0; b < (int64_t)nleaves; b++) {
            const uint32_t *m = uniq[b];
            uint64_t u = usz[b];
            uint64_t kk = u > 0 ? (u - 1 < k ? u - 1 : k) : 0;
            uint64_t w = cnt[b];
            for (uint64_t i = 0; i < u; i++) {
                double bd[16];
                uint32_t bid[16];
                uint32_t have = 0;
                for (uint64_t j = 0; j < u; j++) {
                    if (j == i) continue;
                    double dv = orc_dissimilarity(X, d, dtype, metric, m[i], m[j]);
                    uint32_t id = m[j];
                    if (have == kk && (dv > bd[kk - 1] || (dv == bd[kk - 1] && id > bid[kk - 1]))) continue;
                    uint32_t pos = have < kk ? have++ : (uint32_t)kk - 1;
                    while (pos > 0 && (dv < bd[pos - 1] || (dv == bd[pos - 1] && id < bid[pos - 1]))) {
                        bd[pos] = bd[pos - 1]; bid[pos] = bid[pos - 1];
                        pos--;
                    }
                    bd[pos] = dv; bid[pos] = id;
                }
                for (uint32_t t = 0; t < have; t++) {
                    if (direction != 2) {  /* the edge from i to its neighbour */
                        out->dst[w] = m[i]; out->src[w] = bid[t]; out->dist[w] = (float)bd[t]; w++;
                    }
                    if (direction != 1) {  /* the edge to i from its neighbour */
                        out->dst[w] = bid[t]; out->src[w] = m[i]; out->dist[w] = (float)bd[t]; w++;
                    }
                }
            }
        }
    }
    for (uint64_t b = 0; b < nleaves; b++) free(uniq[b]);
    free(uniq);
    free(usz);
    free(cnt);
    if (err) {
        free(out->dst); free(out->src); free(out->dist);
        memset(out, 0, sizeof(*out));
        return ORC_EINVAL;
    }
    return ORC_OK;
}

void orc_edges_free(orc_edges *e)
{
    if (!e) return;
    free(e->dst); free(e->src); free(e->dist);
    memset(e, 0, sizeof(*e));
}

/* ------------------------------------------------------------------------------------------ */
/* Alg. 3 -- HashPrune, streaming form.  One reservoir per node: an array of at most l_max     */
/* (hash, slot) entries kept sorted by hash and searched by bisection, plus the cached index of */
/* the farthest entry (Sec. 3 "Implementation").  "Closer" compares reservoir slots, i.e. the  */
/* bf16 distance with ties to the smaller id.                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint32_t size;
    int32_t far;      /* cached index of the farthest entry, -1 if stale */
    uint16_t *hash;
    uint64_t *slot;
} reservoir;

static int32_t res_find(const reservoir *M, uint32_t h, uint32_t *ins)
{
    uint32_t lo = 0, hi = M->size;
    while (lo < hi) {
        uint32_t mid = (lo + hi) / 2;
        if (M->hash[mid] < h) lo = mid + 1;
        else hi = mid;
    }
    *ins = lo;
    return (lo < M->size && M->hash[lo] == h) ? (int32_t)lo : -1;
}

static void res_insert_at(reservoir *M, uint32_t pos, uint32_t h, uint64_t s)
{
    memmove(M->hash + pos + 1, M->hash + pos, (M->size - pos) * sizeof(uint16_t));
    memmove(M->slot + pos + 1, M->slot + pos, (M->size - pos) * sizeof(uint64_t));
    M->hash[pos] = (uint16_t)h;
    M->slot[pos] = s;
    M->size++;
}

static void res_remove_at(reservoir *M, uint32_t pos)
{
    memmove(M->hash + pos, M->hash + pos + 1, (M->size - pos - 1) * sizeof(uint16_t));
    memmove(M->slot + pos, M->slot + pos + 1, (M->size - pos - 1) * sizeof(uint64_t));
    M->size--;
}

static void hashprune_insert(reservoir *M, uint32_t l_max, uint32_t h, uint64_t s)
{
    uint32_t ins;
    int32_t at = res_find(M, h, &ins);
    if (at >= 0) {                       /* M.HasKey(h_p(c)) */
        if (s < M->slot[at]) {           /* ||p,c|| < ||p, M.Get(h_p(c))|| */
            M->slot[at] = s;
            M->far = -1;
        }
        return;
    }
    if (M->size < l_max) {               /* |M| < l_max */
        res_insert_at(M, ins, h, s);
        M->far = -1;
        return;
    }
    if (M->far < 0) {                    /* z = argmax_y ||p,y||, by linear scan, then cached */
        uint32_t z = 0;
        for (uint32_t t = 1; t < M->size; t++)
            if (M->slot[t] > M->slot[z]) z = t;
        M->far = (int32_t)z;
    }
    if (s < M->slot[M->far]) {           /* ||p,c|| < ||p,z||: evict z, insert c */
        uint32_t z = (uint32_t)M->far;
        res_remove_at(M, z);
        res_find(M, h, &ins);
        res_insert_at(M, ins, h, s);
        M->far = -1;
    }
}

/* Group a candidate stream by destination, keeping stream order inside each group. */
static int group_by_dst(const uint32_t *dst, uint64_t count, uint64_t n, uint64_t **start_out,
                        uint64_t **order_out)
{
    uint64_t *start = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
    uint64_t *order = (uint64_t *)malloc((count + 1) * sizeof(uint64_t));
    if (!start || !order) { free(start); free(order); return ORC_ENOMEM; }
    for (uint64_t e = 0; e < count; e++) {
        if (dst[e] >= n) { free(start); free(order); return ORC_EINVAL; }
        start[dst[e] + 1]++;
    }
    for (uint64_t v = 0; v < n; v++) start[v + 1] += start[v];
    uint64_t *fill = (uint64_t *)malloc((n + 1) * sizeof(uint64_t));
    if (!fill) { free(start); free(order); return ORC_ENOMEM; }
    memcpy(fill, start, (n + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < count; e++) order[fill[dst[e]]++] = e;
    free(fill);
    *start_out = start;
    *order_out = order;
    return ORC_OK;
}

/* Streams the candidates (dst[e] receives src[e] at dissimilarity dist[e]) through Alg. 3 in
 * stream order, starting from the reservoirs given in res/cnt (cnt[v] = 0 for an empty one).
 * On return res[v*l_max ...] holds node v's slots sorted ascending and cnt[v] their number.
 * A candidate equal to its destination is dropped. */
int orc_hashprune_stream(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count,
                         const float *S, uint32_t m, uint64_t n, uint32_t l_max, uint64_t *res,
                         uint32_t *cnt)
{
    if ((count && (!dst || !src || !dist)) || !S || !res || !cnt || m < 1 || m > 16 || l_max < 1)
        return ORC_EINVAL;
    uint64_t *start, *order;
    int rc = group_by_dst(dst, count, n, &start, &order);
    if (rc) return rc;
    for (uint64_t e = 0; e < count; e++)
        if (src[e] >= n) { free(start); free(order); return ORC_EINVAL; }
    int err = 0;
#pragma omp parallel
    {
        reservoir M;
        M.hash = (uint16_t *)malloc((l_max + 1) * sizeof(uint16_t));
        M.slot = (uint64_t *)malloc((l_max + 1) * sizeof(uint64_t));
        if (!M.hash || !M.slot) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 512)
            for (int64_t v = 0; v < (int64_t)n; v++) {
                /* load the existing reservoir (re-sorted by hash) */
                M.size = 0;
                M.far = -1;
                uint32_t c0 = cnt[v] > l_max ? l_max : cnt[v];
                for (uint32_t t = 0; t < c0; t++) {
                    uint64_t s = res[(uint64_t)v * l_max + t];
                    uint32_t ins;
                    res_find(&M, (uint32_t)(s & 0xFFFFu), &ins);
                    res_insert_at(&M, ins, (uint32_t)(s & 0xFFFFu), s);
                }
                for (uint64_t q = start[v]; q < start[v + 1]; q++) {
                    uint64_t e = order[q];
                    if (src[e] == (uint32_t)v) continue;
                    uint32_t h = residual_hash(S, m, (uint32_t)v, src[e]);
                    hashprune_insert(&M, l_max, h, slot_of(dist[e], src[e], h));
                }
                qsort(M.slot, M.size, sizeof(uint64_t), cmp_u64);
                for (uint32_t t = 0; t < M.size; t++) res[(uint64_t)v * l_max + t] = M.slot[t];
                for (uint32_t t = M.size; t < l_max; t++) res[(uint64_t)v * l_max + t] = ~0ull;
                cnt[v] = M.size;
            }
        }
        free(M.hash);
        free(M.slot);
    }
    free(start);
    free(order);
    return err ? ORC_ENOMEM : ORC_OK;
}

/* Closed form of HashPrune (history-independence lemma, App. A.6): node v's reservoir is the
 * l_max smallest among the per-hash-bucket minima of all its candidates (the existing reservoir
 * entries count as candidates). */
int orc_hashprune_closed(const uint32_t *dst, const uint32_t *src, const float *dist, uint64_t count,
                         const float *S, uint32_t m, uint64_t n, uint32_t l_max, uint64_t *res,
                         uint32_t *cnt)
{
    if ((count && (!dst || !src || !dist)) || !S || !res || !cnt || m < 1 || m > 16 || l_max < 1)
        return ORC_EINVAL;
    uint64_t *start, *order;
    int rc = group_by_dst(dst, count, n, &start, &order);
    if (rc) return rc;
    for (uint64_t e = 0; e < count; e++)
        if (src[e] >= n) { free(start); free(order); return ORC_EINVAL; }
    int err = 0;
#pragma omp parallel
    {
        uint64_t *best = (uint64_t *)malloc(sizeof(uint64_t) << 16);
        uint64_t *mins = (uint64_t *)malloc(sizeof(uint64_t) << 16);
        if (!best || !mins) {
#pragma omp atomic write
            err = 1;
        } else {
            for (uint32_t h = 0; h < (1u << 16); h++) best[h] = ~0ull;
#pragma omp for schedule(dynamic, 512)
            for (int64_t v = 0; v < (int64_t)n; v++) {
                uint32_t c0 = cnt[v] > l_max ? l_max : cnt[v];
                for (uint32_t t = 0; t < c0; t++) {
                    uint64_t s = res[(uint64_t)v * l_max + t];
                    uint32_t h = (uint32_t)(s & 0xFFFFu);
                    if (s < best[h]) best[h] = s;
                }
                for (uint64_t q = start[v]; q < start[v + 1]; q++) {
                    uint64_t e = order[q];
                    if (src[e] == (uint32_t)v) continue;
                    uint32_t h = residual_hash(S, m, (uint32_t)v, src[e]);
                    uint64_t s = slot_of(dist[e], src[e], h);
                    if (s < best[h]) best[h] = s;
                }
                uint32_t nm = 0;
                for (uint32_t h = 0; h < (1u << m); h++)
                    if (best[h] != ~0ull) { mins[nm++] = best[h]; best[h] = ~0ull; }
                qsort(mins, nm, sizeof(uint64_t), cmp_u64);
                uint32_t keep = nm < l_max ? nm : l_max;
                for (uint32_t t = 0; t < keep; t++) res[(uint64_t)v * l_max + t] = mins[t];
                for (uint32_t t = keep; t < l_max; t++) res[(uint64_t)v * l_max + t] = ~0ull;
                cnt[v] = keep;
            }
        }
        free(best);
        free(mins);
    }
    free(start);
    free(order);
    return err ? ORC_ENOMEM : ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Alg. 2 -- RobustPrune of every node's reservoir down to degree R (final prune, Sec. 4.3).   */
/* Candidates are ordered by (dissimilarity to x, id); "argmin" reads as the nearest remaining */
/* candidate.  z is removed when alpha * ||y,z|| < ||x,z||; on squared distances this is       */
/* alpha^2 * D(y,z) < D(x,z), evaluated in binary32 with alpha^2 = (float)(alpha * alpha).     */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    double d;
    uint32_t id;
} cand;

static int cmp_cand(const void *a, const void *b)
{
    const cand *x = (const cand *)a, *y = (const cand *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return x->id < y->id ? -1 : x->id > y->id;
}

static int prunes(const void *X, uint32_t d, int dtype, int metric, float alpha2, uint32_t y, const cand *z)
{
    float dyz = (float)orc_dissimilarity(X, d, dtype, metric, y, z->id);
    float dxz = (float)z->d;
    float lhs = alpha2 * dyz;
    return lhs < dxz;
}

int orc_final_prune(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const uint64_t *res,
                    const uint32_t *cnt, uint32_t l_max, uint32_t R, float alpha, int lazy, uint32_t *adj,
                    uint32_t *deg)
{
    if (!X || !res || !cnt || !adj || !deg || R < 1 || l_max < 1) return ORC_EINVAL;
    float alpha2 = (float)((double)alpha * (double)alpha);
    int err = 0;
#pragma omp parallel
    {
        cand *N = (cand *)malloc((l_max + 1) * sizeof(cand));
        uint8_t *alive = (uint8_t *)malloc(l_max + 1);
        if (!N || !alive) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (int64_t v = 0; v < (int64_t)n; v++) {
                uint32_t c = cnt[v] > l_max ? l_max : cnt[v];
                for (uint32_t t = 0; t < c; t++) {
                    uint32_t id = (uint32_t)(res[(uint64_t)v * l_max + t] >> 16);
                    N[t].id = id;
                    N[t].d = orc_dissimilarity(X, d, dtype, metric, (uint64_t)v, id);
                }
                qsort(N, c, sizeof(cand), cmp_cand);
                uint32_t e = 0;
                if (!lazy) {
                    memset(alive, 1, c);
                    for (uint32_t head = 0; head < c && e < R; head++) {
                        if (!alive[head]) continue;
                        uint32_t y = N[head].id;              /* y <- argmin over N */
                        adj[(uint64_t)v * R + e++] = y;       /* E.Add((x, y)); N.Remove(y) */
                        alive[head] = 0;
                        for (uint32_t z = head + 1; z < c; z++)
                            if (alive[z] && prunes(X, d, dtype, metric, alpha2, y, &N[z])) alive[z] = 0;
                    }
                } else {
                    /* lazy: admit a candidate unless an already admitted neighbour prunes it */
                    for (uint32_t t = 0; t < c && e < R; t++) {
                        int pruned = 0;
                        for (uint32_t q = 0; q < e && !pruned; q++)
                            pruned = prunes(X, d, dtype, metric, alpha2, adj[(uint64_t)v * R + q], &N[t]);
                        if (!pruned) adj[(uint64_t)v * R + e++] = N[t].id;
                    }
                }
                deg[v] = e;
                for (uint32_t t = e; t < R; t++) adj[(uint64_t)v * R + t] = 0xFFFFFFFFu;
            }
        }
        free(N);
        free(alive);
    }
    return err ? ORC_ENOMEM : ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Alg. 4 -- PiPNN: partition, pick in every leaf, stream the candidates through HashPrune,    */
/* then (BP.final_prune) RobustPrune every node.  Without the final prune a node's neighbours  */
/* are its first R reservoir entries in (distance, id) order.                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t leaves, leaf_members, levels, candidates;
} orc_stats;

int orc_build(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const orc_params *bp,
              const float *H, uint64_t seed, uint32_t *adj, uint32_t *deg, orc_stats *st)
{
    if (!params_ok(bp) || !input_ok(X, n, d, dtype, metric) || !H || !adj || !deg) return ORC_EINVAL;
    float *S = (float *)malloc(n * bp->hash_bits * sizeof(float));
    if (!S) return ORC_ENOMEM;
    int rc = orc_sketch(X, n, d, dtype, H, bp->hash_bits, S, NULL);
    orc_leaves L;
    if (!rc) rc = orc_partition(X, n, d, dtype, metric, bp, seed, &L);
    if (rc) { free(S); return rc; }
    orc_edges E;
    rc = orc_leaf_pick(X, n, d, dtype, metric, L.off, L.mem, L.nleaves, bp->leaf_k, bp->pick_direction, &E);
    if (st) {
        st->leaves = L.nleaves;
        st->leaf_members = L.nmem;
        st->levels = L.levels;
        st->candidates = E.count;
    }
    orc_leaves_free(&L);
    if (rc) { free(S); return rc; }
    uint64_t *res = (uint64_t *)malloc(n * bp->l_max * sizeof(uint64_t));
    uint32_t *cnt = (uint32_t *)calloc(n, sizeof(uint32_t));
    if (!res || !cnt) { free(S); free(res); free(cnt); orc_edges_free(&E); return ORC_ENOMEM; }
    rc = orc_hashprune_stream(E.dst, E.src, E.dist, E.count, S, bp->hash_bits, n, bp->l_max, res, cnt);
    orc_edges_free(&E);
    free(S);
    if (!rc) {
        if (bp->final_prune) {
            rc = orc_final_prune(X, n, d, dtype, metric, res, cnt, bp->l_max, bp->R, bp->alpha, 0, adj, deg);
        } else {
            for (uint64_t v = 0; v < n; v++) {
                uint32_t c = cnt[v] < bp->R ? cnt[v] : bp->R;
                for (uint32_t t = 0; t < bp->R; t++)
                    adj[v * bp->R + t] = t < c ? (uint32_t)(res[v * bp->l_max + t] >> 16) : 0xFFFFFFFFu;
                deg[v] = c;
            }
        }
    }
    free(res);
    free(cnt);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Evaluation: exact k-NN (Def. 1, ties to the smaller id), Alg. 1 BeamSearch, medoid start.  */
/* Query-side dissimilarities are taken in double precision, or (defined = 1) as the defining    */
/* binary32 / exact-integer value the build uses.                                              */
/* ------------------------------------------------------------------------------------------ */
static double qdis_as(const void *X, uint64_t i, const void *q, uint32_t d, int dtype, int metric, int defined)
{
    return defined ? dis_vec(row(X, i, d, dtype), q, d, dtype, metric)
                   : dis_vec_f64(row(X, i, d, dtype), q, d, dtype, metric);
}

static double qdis(const void *X, uint64_t i, const void *q, uint32_t d, int dtype, int metric)
{
    return qdis_as(X, i, q, d, dtype, metric, 0);
}

int orc_knn(const void *X, uint64_t n, const void *Q, uint64_t nq, uint32_t d, int dtype, int metric,
            uint32_t k, uint32_t *ids)
{
    if (!X || !Q || !ids || k < 1 || k > n || k > 1024) return ORC_EINVAL;
    int err = 0;
#pragma omp parallel
    {
        cand *best = (cand *)malloc((k + 1) * sizeof(cand));
        if (!best) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t qi = 0; qi < (int64_t)nq; qi++) {
                const void *q = row(Q, (uint64_t)qi, d, dtype);
                uint32_t have = 0;
                for (uint64_t i = 0; i < n; i++) {
                    double dv = qdis(X, i, q, d, dtype, metric);
                    if (have == k && (dv > best[k - 1].d || (dv == best[k - 1].d && i > best[k - 1].id))) continue;
                    uint32_t pos = have < k ? have++ : k - 1;
                    while (pos > 0 && (dv < best[pos - 1].d || (dv == best[pos - 1].d && i < best[pos - 1].id))) {
                        best[pos] = best[pos - 1];
                        pos--;
                    }
                    best[pos].d = dv;
                    best[pos].id = (uint32_t)i;
                }
                for (uint32_t t = 0; t < k; t++) ids[(uint64_t)qi * k + t] = best[t].id;
            }
        }
        free(best);
    }
    return err ? ORC_ENOMEM : ORC_OK;
}

/* Byte data: the point nearest to the exact mean, found without rounding.  With S the exact
 * coordinate sums, |x - S/n|^2 = |n x - S|^2 / n^2, so the argmin of the integer
 * sum_t (n x_t - S_t)^2 (below 2^92 for any admissible n and d) is the point nearest to the mean;
 * ties go to the smaller index. */
static uint32_t medoid_bytes_exact(const void *X, uint64_t n, uint32_t d, int dtype)
{
    int64_t *S = (int64_t *)calloc(d, sizeof(int64_t));
    if (!S) return 0;
    for (uint64_t i = 0; i < n; i++)
        for (uint32_t t = 0; t < d; t++) S[t] += (int64_t)coord(row(X, i, d, dtype), t, dtype);
    uint32_t best = 0;
    unsigned __int128 bv = 0;
    int have = 0;
#pragma omp parallel
    {
        uint32_t lb = 0;
        unsigned __int128 lv = 0;
        int lh = 0;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; i++) {
            unsigned __int128 v = 0;
            for (uint32_t t = 0; t < d; t++) {
                int64_t e = (int64_t)n * (int64_t)coord(row(X, (uint64_t)i, d, dtype), t, dtype) - S[t];
                uint64_t a = e < 0 ? (uint64_t)(-e) : (uint64_t)e;
                v += (unsigned __int128)a * a;
            }
            if (!lh || v < lv) { lv = v; lb = (uint32_t)i; lh = 1; }
        }
#pragma omp critical
        {
            if (lh && (!have || lv < bv || (lv == bv && lb < best))) { bv = lv; best = lb; have = 1; }
        }
    }
    free(S);
    return best;
}

/* The beam-search start: the point nearest to the mean of all points (ties to the smaller
 * index).  Byte data: exact (above).  Float data: in double precision, the mean summed in fixed
 * chunks of 65,536 points whose partial sums are added in chunk order, so the result does not
 * depend on the thread count. */
uint32_t orc_medoid(const void *X, uint64_t n, uint32_t d, int dtype, int metric)
{
    (void)metric;
    if (dtype != ORC_F32) return medoid_bytes_exact(X, n, d, dtype);
    const uint64_t CH = 65536;
    const uint64_t nch = (n + CH - 1) / CH;
    double *part = (double *)calloc(nch * d, sizeof(double));
    double *mean = (double *)calloc(d, sizeof(double));
    if (!part || !mean) {
        free(part);
        free(mean);
        return 0;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < (int64_t)nch; c++) {
        uint64_t lo = (uint64_t)c * CH, hi = lo + CH < n ? lo + CH : n;
        for (uint64_t i = lo; i < hi; i++)
            for (uint32_t t = 0; t < d; t++) part[(uint64_t)c * d + t] += coord(row(X, i, d, dtype), t, dtype);
    }
    for (uint64_t c = 0; c < nch; c++)
        for (uint32_t t = 0; t < d; t++) mean[t] += part[c * d + t];
    for (uint32_t t = 0; t < d; t++) mean[t] /= (double)n;
    uint32_t best = 0;
    double bd = INFINITY;
#pragma omp parallel
    {
        uint32_t lb = 0;
        double ld = INFINITY;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; i++) {
            double s = 0.0;
            for (uint32_t t = 0; t < d; t++) {
                double df = coord(row(X, (uint64_t)i, d, dtype), t, dtype) - mean[t];
                s += df * df;
            }
            if (s < ld || (s == ld && (uint32_t)i < lb)) { ld = s; lb = (uint32_t)i; }
        }
#pragma omp critical
        {
            if (ld < bd || (ld == bd && lb < best)) { bd = ld; best = lb; }
        }
    }
    free(part);
    free(mean);
    return best;
}

/* Alg. 1: beam B (kept sorted by (distance, id)) and visited set V; visit the nearest unvisited
 * beam member, add its neighbours, trim the beam to the L closest.  Returns the k closest of the
 * final beam and the number of distance evaluations. */
int orc_beam_search_as(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const uint32_t *adj,
                       const uint32_t *deg, uint32_t R, const void *Q, uint64_t nq, uint32_t start,
                       uint32_t L, uint32_t k, int defined, uint32_t *ids, uint64_t *ndist);

int orc_beam_search(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const uint32_t *adj,
                    const uint32_t *deg, uint32_t R, const void *Q, uint64_t nq, uint32_t start,
                    uint32_t L, uint32_t k, uint32_t *ids, uint64_t *ndist)
{
    return orc_beam_search_as(X, n, d, dtype, metric, adj, deg, R, Q, nq, start, L, k, 0, ids, ndist);
}

int orc_beam_search_as(const void *X, uint64_t n, uint32_t d, int dtype, int metric, const uint32_t *adj,
                       const uint32_t *deg, uint32_t R, const void *Q, uint64_t nq, uint32_t start,
                       uint32_t L, uint32_t k, int defined, uint32_t *ids, uint64_t *ndist)
{
    if (!X || !adj || !deg || !Q || !ids || L < 1 || k < 1 || k > L || start >= n) return ORC_EINVAL;
    uint64_t total = 0;
    int err = 0;
#pragma omp parallel reduction(+ : total)
    {
        cand *B = (cand *)malloc((L + R + 1) * sizeof(cand));
        uint8_t *vis = (uint8_t *)calloc(n, 1);  /* 1 = in beam or seen, 2 = visited */
        uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (n < 1000000 ? n : 1000000));
        uint64_t cap_t = n < 1000000 ? n : 1000000;
        if (!B || !vis || !touched) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t qi = 0; qi < (int64_t)nq; qi++) {
                const void *q = row(Q, (uint64_t)qi, d, dtype);
                uint64_t nt = 0;
                uint32_t nb = 1;
                B[0].id = start;
                B[0].d = qdis_as(X, start, q, d, dtype, metric, defined);
                total++;
                vis[start] = 1;
                touched[nt++] = start;
                for (;;) {
                    int32_t p = -1;
                    for (uint32_t t = 0; t < nb; t++)
                        if (vis[B[t].id] != 2) { p = (int32_t)t; break; }
                    if (p < 0) break;
                    uint32_t pid = B[p].id;
                    vis[pid] = 2;
                    for (uint32_t j = 0; j < deg[pid] && j < R; j++) {
                        uint32_t u = adj[(uint64_t)pid * R + j];
                        if (u >= n || vis[u]) continue;
                        vis[u] = 1;
                        if (nt < cap_t) touched[nt++] = u;
                        double dv = qdis_as(X, u, q, d, dtype, metric, defined);
                        total++;
                        if (nb == L && (dv > B[L - 1].d || (dv == B[L - 1].d && u > B[L - 1].id))) continue;
                        uint32_t pos = nb < L ? nb++ : L - 1;
                        while (pos > 0 && (dv < B[pos - 1].d || (dv == B[pos - 1].d && u < B[pos - 1].id))) {
                            B[pos] = B[pos - 1];
                            pos--;
                        }
                        B[pos].d = dv;
                        B[pos].id = u;
                    }
                }
                for (uint32_t t = 0; t < k; t++) ids[(uint64_t)qi * k + t] = t < nb ? B[t].id : 0xFFFFFFFFu;
                if (nt < cap_t) {
                    for (uint64_t t = 0; t < nt; t++) vis[touched[t]] = 0;
                } else {
                    memset(vis, 0, n);
                }
            }
        }
        free(B);
        free(vis);
        free(touched);
    }
    if (ndist) *ndist = total;
    return err ? ORC_ENOMEM : ORC_OK;
}
