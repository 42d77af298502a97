/*
 * EVP oracle: a plain, slow, obviously correct CPU statement of what the
 * GPU hot path computes.  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the CPU-baseline leg of the benchmark call it; the product
 * path never does.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Paper: R. Connor, A. Dearle, B. Claydon, "Ultra-Quantisation: Efficient
 * Embedding Search via 1.58-bit Encodings" (arXiv 2506.00528).
 *
 * Representation used here: a ternary vector is an int8 array of d values
 * in {-1, 0, +1} (the set T of the notation table, Table 1).  Distances
 * are integer sums over those arrays; no bitplane or popcount is used, so
 * this file is independent of the GPU's bit-level route.  Packing to the
 * paper's two-bitplane form (v+, v-) is a separate pair of functions.
 *
 * Plain C99, single thread, no intrinsics: the same results on x86-64 and
 * aarch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* Choice of x (Sec. 5.1.1): the x in [1, d] that maximises the vertex  */
/* count C(d, x) * 2^x (Sec. 2.3).  Successive counts have the exact   */
/* ratio f(x+1)/f(x) = 2(d-x)/(x+1); f rises while that ratio exceeds  */
/* 1 and falls after, so walking x upward while f(x+1) > f(x) gives the */
/* smallest maximiser (at d = 500 the counts for 333 and 334 are equal  */
/* and 333 is returned, as in Table 2).                                 */
/* ------------------------------------------------------------------ */
int evpo_default_x(int d)
{
    int x = 1;
    if (d < 1) return 0;
    while (x < d && 2 * (int64_t)(d - x) > (int64_t)(x + 1)) /* f(x+1) > f(x) */
        x++;
    return x;
}

/* ------------------------------------------------------------------ */
/* Encoding (Sec. 2.4): the nearest {x,d} vertex to u is found by       */
/* (1) taking the x elements of largest absolute value, (2) giving +1   */
/* to the positive and -1 to the negative ones among them, (3) giving 0 */
/* to the rest.                                                         */
/* Readings where the paper is silent:                                  */
/*  - |u_i| is compared through its IEEE-754 bit pattern with the sign  */
/*    bit cleared (an exact total order for finite values); equal       */
/*    magnitudes are taken lowest index first.                          */
/*  - a selected element with u_i < 0 gets -1, every other selected     */
/*    element (including +0.0 and -0.0) gets +1, so a code always has   */
/*    exactly x non-zero elements (Sec. 2.3).                           */
/*  - any NaN or infinity in a row sets *nonfinite (the code of that    */
/*    row is still written but carries no meaning).                     */
/* ------------------------------------------------------------------ */
typedef struct { uint32_t mag; int32_t idx; } evpo_mag_t;

static uint32_t evpo_abs_bits(float f)
{
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    return b & 0x7fffffffu;
}

static int evpo_cmp_mag_desc(const void* pa, const void* pb)
{
    const evpo_mag_t* a = (const evpo_mag_t*)pa;
    const evpo_mag_t* b = (const evpo_mag_t*)pb;
    if (a->mag != b->mag) return a->mag > b->mag ? -1 : 1;   /* larger first */
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0); /* lower index first */
}

int evpo_encode(const float* U, int64_t n, int d, int x, int8_t* V)
{
    int nonfinite = 0;
    evpo_mag_t* order;
    int64_t r;
    int j;
    if (n <= 0) return 0;
    order = (evpo_mag_t*)malloc(sizeof(evpo_mag_t) * (size_t)d);
    if (!order) return -1;
    for (r = 0; r < n; ++r) {
        const float* u = U + r * (int64_t)d;
        int8_t* v = V + r * (int64_t)d;
        for (j = 0; j < d; ++j) {
            if (!isfinite(u[j])) nonfinite = 1;
            order[j].mag = evpo_abs_bits(u[j]);
            order[j].idx = j;
        }
        qsort(order, (size_t)d, sizeof(evpo_mag_t), evpo_cmp_mag_desc);
        for (j = 0; j < d; ++j) v[j] = 0;
        for (j = 0; j < x; ++j) {
            int i = order[j].idx;
            v[i] = (u[i] < 0.0f) ? (int8_t)-1 : (int8_t)1;
        }
    }
    free(order);
    return nonfinite;
}

/* ------------------------------------------------------------------ */
/* Bitplanes (Sec. 5.1.2 and Table 3): v+ has a bit set where v_i = 1, */
/* v- where v_i = -1.  Layout chosen for this library: W = ceil(d/64)   */
/* 64-bit words per plane, v+ in words [0, W) and v- in words [W, 2W);  */
/* dimension j is bit (j mod 64) of word floor(j/64); unused bits are 0.*/
/* ------------------------------------------------------------------ */
int evpo_words(int d) { return (d + 63) / 64; }

void evpo_pack(const int8_t* V, int64_t n, int d, uint64_t* T)
{
    int W = evpo_words(d);
    int64_t r;
    int j;
    for (r = 0; r < n; ++r) {
        const int8_t* v = V + r * (int64_t)d;
        uint64_t* t = T + r * (int64_t)(2 * W);
        for (j = 0; j < 2 * W; ++j) t[j] = 0;
        for (j = 0; j < d; ++j) {
            uint64_t bit = (uint64_t)1 << (j % 64);
            if (v[j] == 1) t[j / 64] |= bit;
            else if (v[j] == -1) t[W + j / 64] |= bit;
        }
    }
}

/* Returns the number of rows that are not a valid packed ternary code
 * (a dimension set in both planes, or a set bit beyond d). */
int64_t evpo_unpack(const uint64_t* T, int64_t n, int d, int8_t* V)
{
    int W = evpo_words(d);
    int64_t r, bad = 0;
    int j;
    for (r = 0; r < n; ++r) {
        const uint64_t* t = T + r * (int64_t)(2 * W);
        int8_t* v = V + r * (int64_t)d;
        int row_bad = 0;
        for (j = 0; j < d; ++j) {
            int p = (int)((t[j / 64] >> (j % 64)) & 1u);
            int m = (int)((t[W + j / 64] >> (j % 64)) & 1u);
            if (p && m) row_bad = 1;
            v[j] = (int8_t)(p - m);
        }
        for (j = d; j < 64 * W; ++j) {
            if ((t[j / 64] >> (j % 64)) & 1u) row_bad = 1;
            if ((t[W + j / 64] >> (j % 64)) & 1u) row_bad = 1;
        }
        bad += row_bad;
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* Scalar product of two ternary vectors: what b2sp computes from the  */
/* four bitplane counts (Sec. 5.1.2), written as the plain sum.         */
/* ------------------------------------------------------------------ */
int64_t evpo_dot(const int8_t* v, const int8_t* w, int d)
{
    int64_t s = 0;
    int j;
    for (j = 0; j < d; ++j) s += (int64_t)v[j] * (int64_t)w[j];
    return s;
}

/* Proxy distance Delta (notation table; Sec. 2.6): read as the squared  */
/* Euclidean distance between the two ternary vectors.  For two codes   */
/* with x non-zeros each this equals 2x - 2*b2sp.                        */
int64_t evpo_delta(const int8_t* v, const int8_t* w, int d)
{
    int64_t s = 0;
    int j;
    for (j = 0; j < d; ++j) {
        int64_t e = (int64_t)v[j] - (int64_t)w[j];
        s += e * e;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Exhaustive kNN in the proxy space (Sec. 5.3, and the 100-query       */
/* exhaustive scans of Table 5): for each query, every database code is */
/* compared, and the k smallest (Delta, index) pairs are returned in    */
/* ascending order.  Equal Delta is broken by the lower database index. */
/* ------------------------------------------------------------------ */
typedef struct { int64_t delta; int64_t idx; } evpo_cand_t;

static int evpo_cmp_cand(const void* pa, const void* pb)
{
    const evpo_cand_t* a = (const evpo_cand_t*)pa;
    const evpo_cand_t* b = (const evpo_cand_t*)pb;
    if (a->delta != b->delta) return a->delta < b->delta ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

int evpo_knn(const int8_t* Vq, int64_t nq, const int8_t* Vs, int64_t ns, int d,
             int k, int64_t* ids, int32_t* dist)
{
    evpo_cand_t* all;
    int64_t q, s;
    int j;
    if (nq <= 0) return 0;
    if (k < 1 || (int64_t)k > ns) return -1;
    all = (evpo_cand_t*)malloc(sizeof(evpo_cand_t) * (size_t)ns);
    if (!all) return -1;
    for (q = 0; q < nq; ++q) {
        const int8_t* v = Vq + q * (int64_t)d;
        for (s = 0; s < ns; ++s) {
            all[s].delta = evpo_delta(v, Vs + s * (int64_t)d, d);
            all[s].idx = s;
        }
        qsort(all, (size_t)ns, sizeof(evpo_cand_t), evpo_cmp_cand);
        for (j = 0; j < k; ++j) {
            ids[q * k + j] = all[j].idx;
            dist[q * k + j] = (int32_t)all[j].delta;
        }
    }
    free(all);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Re-ordering of a shortlist in the original space (Sec. 5.3: n > k    */
/* proxy results are re-ordered with respect to the original vectors    */
/* and the best k kept).  Score = scalar product <q, s> in double       */
/* precision; for l2-normalised rows this orders exactly as cosine      */
/* similarity and as Euclidean distance (Sec. 1.1).  Larger score first,*/
/* equal scores by lower index.  Shortlist entries of -1 are empty and  */
/* skipped; when fewer than k entries remain, the tail of the output is */
/* id -1 with score -infinity.  absdot receives sum_i |q_i s_i| for each */
/* output (the scale of the rounding error of any float evaluation).    */
/* Returns -1 if a shortlist id lies outside [-1, ns).                  */
/* ------------------------------------------------------------------ */
typedef struct { double score; int64_t idx; double absdot; } evpo_scored_t;

static int evpo_cmp_scored(const void* pa, const void* pb)
{
    const evpo_scored_t* a = (const evpo_scored_t*)pa;
    const evpo_scored_t* b = (const evpo_scored_t*)pb;
    if (a->score != b->score) return a->score > b->score ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

int evpo_rerank(const float* Q, int64_t nq, const float* S, int64_t ns, int d,
                const int64_t* shortlist, int n, int k,
                int64_t* ids, double* scores, double* absdot)
{
    evpo_scored_t* c;
    int64_t q;
    int j, i, m;
    if (nq <= 0) return 0;
    c = (evpo_scored_t*)malloc(sizeof(evpo_scored_t) * (size_t)(n > 0 ? n : 1));
    if (!c) return -1;
    for (q = 0; q < nq; ++q) {
        const float* qv = Q + q * (int64_t)d;
        m = 0;
        for (j = 0; j < n; ++j) {
            int64_t id = shortlist[q * n + j];
            const float* sv;
            double s = 0.0, a = 0.0;
            if (id == -1) continue;
            if (id < 0 || id >= ns) { free(c); return -1; }
            sv = S + id * (int64_t)d;
            for (i = 0; i < d; ++i) {
                double p = (double)qv[i] * (double)sv[i];
                s += p;
                a += fabs(p);
            }
            c[m].score = s;
            c[m].idx = id;
            c[m].absdot = a;
            m++;
        }
        qsort(c, (size_t)m, sizeof(evpo_scored_t), evpo_cmp_scored);
        for (j = 0; j < k; ++j) {
            if (j < m) {
                ids[q * k + j] = c[j].idx;
                scores[q * k + j] = c[j].score;
                absdot[q * k + j] = c[j].absdot;
            } else {
                ids[q * k + j] = -1;
                scores[q * k + j] = -INFINITY;
                absdot[q * k + j] = 0.0;
            }
        }
    }
    free(c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Single-operand translation (Sec. 6): only the database is mapped to  */
/* EVP vertices; the query keeps (almost) its original values.  Here     */
/* the query is held as int8 so that every score stays an exact integer. */
/* The paper does not fix this precision; the reading used is symmetric  */
/* per-query scaling: m = max_i |q_i|, scale = 127 / m (float32), and    */
/* q8_i = q_i * scale rounded to the nearest integer, ties to even, all  */
/* in float32 (m = 0 gives the zero vector).  Returns 1 if some q_i is   */
/* NaN or infinite (that row is then left zero), 0 otherwise.            */
/* ------------------------------------------------------------------ */
int evpo_quantize_i8(const float* Q, int64_t nq, int d, int8_t* Q8)
{
    int64_t r;
    int j, bad = 0;
    for (r = 0; r < nq; ++r) {
        const float* q = Q + r * (int64_t)d;
        int8_t* o = Q8 + r * (int64_t)d;
        float m = 0.0f, scale;
        int finite = 1;
        for (j = 0; j < d; ++j) {
            float a = fabsf(q[j]);
            if (!(a <= 3.4028234663852886e38f)) finite = 0;   /* NaN or infinity */
            else if (a > m) m = a;
        }
        if (!finite) {
            for (j = 0; j < d; ++j) o[j] = 0;
            bad = 1;
            continue;
        }
        if (m == 0.0f) {
            for (j = 0; j < d; ++j) o[j] = 0;
            continue;
        }
        scale = 127.0f / m;
        for (j = 0; j < d; ++j) {
            float p = q[j] * scale;
            o[j] = (int8_t)rintf(p);
        }
    }
    return bad;
}

/* Masked addition (Sec. 5.1.2): the scalar product of a query with a    */
/* ternary vector v needs no multiplication -- the query elements where  */
/* v is +1 are added and those where v is -1 subtracted.  Exhaustive     */
/* search with that score (Sec. 5.3 with the single-operand translation */
/* of Sec. 6): per query the k rows with the largest score, equal scores */
/* by lower row index.                                                  */
int64_t evpo_masked_sum(const int8_t* q8, const int8_t* v, int d)
{
    int64_t s = 0;
    int j;
    for (j = 0; j < d; ++j) {
        if (v[j] == 1) s += q8[j];
        else if (v[j] == -1) s -= q8[j];
    }
    return s;
}

int evpo_knn_i8q(const int8_t* Q8, int64_t nq, const int8_t* Vs, int64_t ns, int d,
                 int k, int64_t* ids, int32_t* score)
{
    evpo_cand_t* all;
    int64_t q, s;
    int j;
    if (nq <= 0) return 0;
    if (k < 1 || (int64_t)k > ns) return -1;
    all = (evpo_cand_t*)malloc(sizeof(evpo_cand_t) * (size_t)ns);
    if (!all) return -1;
    for (q = 0; q < nq; ++q) {
        const int8_t* q8 = Q8 + q * (int64_t)d;
        for (s = 0; s < ns; ++s) {
            /* ascending (-score, index) = descending score, lower index first */
            all[s].delta = -evpo_masked_sum(q8, Vs + s * (int64_t)d, d);
            all[s].idx = s;
        }
        qsort(all, (size_t)ns, sizeof(evpo_cand_t), evpo_cmp_cand);
        for (j = 0; j < k; ++j) {
            ids[q * k + j] = all[j].idx;
            score[q * k + j] = (int32_t)(-all[j].delta);
        }
    }
    free(all);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sparse representation for small x (Sec. 6, "different EVPs": fewer    */
/* non-zeros).  A code is the list of its x non-zero dimensions in       */
/* ascending order, each a 16-bit entry: bits 0-14 the dimension, bit 15 */
/* set for -1.  Requires d <= 32768.  Returns the number of rows whose   */
/* count of non-zeros is not x (those rows are left zero-filled).        */
/* ------------------------------------------------------------------ */
int64_t evpo_sparse_pack(const int8_t* V, int64_t n, int d, int x, uint16_t* E)
{
    int64_t r, bad = 0;
    int j, c;
    for (r = 0; r < n; ++r) {
        const int8_t* v = V + r * (int64_t)d;
        uint16_t* e = E + r * (int64_t)x;
        for (c = 0, j = 0; j < d; ++j)
            if (v[j] != 0) c++;
        if (c != x) {
            for (j = 0; j < x; ++j) e[j] = 0;
            bad++;
            continue;
        }
        for (c = 0, j = 0; j < d; ++j) {
            if (v[j] == 1) e[c++] = (uint16_t)j;
            else if (v[j] == -1) e[c++] = (uint16_t)(0x8000u | (unsigned)j);
        }
    }
    return bad;
}

/* Inverse of evpo_sparse_pack; returns the number of malformed rows (a  */
/* dimension >= d, or entries not strictly ascending).                   */
int64_t evpo_sparse_unpack(const uint16_t* E, int64_t n, int d, int x, int8_t* V)
{
    int64_t r, bad = 0;
    int j;
    for (r = 0; r < n; ++r) {
        const uint16_t* e = E + r * (int64_t)x;
        int8_t* v = V + r * (int64_t)d;
        int prev = -1, row_bad = 0;
        for (j = 0; j < d; ++j) v[j] = 0;
        for (j = 0; j < x; ++j) {
            int dim = (int)(e[j] & 0x7FFFu);
            if (dim >= d || dim <= prev) { row_bad = 1; break; }
            v[dim] = (e[j] & 0x8000u) ? (int8_t)-1 : (int8_t)1;
            prev = dim;
        }
        if (row_bad) bad++;
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* The float baseline of the paper's speed comparison ("Euclidean" in    */
/* Tables 4 and 5): exhaustive kNN by squared Euclidean distance over    */
/* the original float32 vectors, summed in float32 in index order, the  */
/* k smallest (distance, index) pairs ascending.  A CPU baseline, not    */
/* part of the method.                                                  */
/* ------------------------------------------------------------------ */
typedef struct { float dist; int64_t idx; } evpo_fcand_t;

static int evpo_cmp_fcand(const void* pa, const void* pb)
{
    const evpo_fcand_t* a = (const evpo_fcand_t*)pa;
    const evpo_fcand_t* b = (const evpo_fcand_t*)pb;
    if (a->dist != b->dist) return a->dist < b->dist ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

int evpo_l2_knn(const float* Q, int64_t nq, const float* S, int64_t ns, int d, int k,
                int64_t* ids, float* dist)
{
    evpo_fcand_t* all;
    int64_t q, s;
    int j;
    if (nq <= 0) return 0;
    if (k < 1 || (int64_t)k > ns) return -1;
    all = (evpo_fcand_t*)malloc(sizeof(evpo_fcand_t) * (size_t)ns);
    if (!all) return -1;
    for (q = 0; q < nq; ++q) {
        const float* qv = Q + q * (int64_t)d;
        for (s = 0; s < ns; ++s) {
            const float* sv = S + s * (int64_t)d;
            float acc = 0.0f;
            for (j = 0; j < d; ++j) {
                float e = qv[j] - sv[j];
                acc += e * e;
            }
            all[s].dist = acc;
            all[s].idx = s;
        }
        qsort(all, (size_t)ns, sizeof(evpo_fcand_t), evpo_cmp_fcand);
        for (j = 0; j < k; ++j) {
            ids[q * k + j] = all[j].idx;
            dist[q * k + j] = all[j].dist;
        }
    }
    free(all);
    return 0;
}
