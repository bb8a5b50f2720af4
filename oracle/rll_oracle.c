/*
 * Reinforcement Lightcuts Learning -- plain CPU reference ("oracle").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct
 * restatement of the method of Pantaleoni, "Importance Sampling of Many
 * Lights with Reinforcement Lightcuts Learning" (arXiv 1911.10217) that the
 * CUDA library is checked against. Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code, header or
 * constant table with the CUDA library.
 *
 * Precision. Continuous quantities (contributions, pdfs, Q, C) are computed in
 * double. Wherever a floating-point value decides an integer -- the cell a
 * point is hashed to, the Morton code of a light, which child a descent step
 * takes, whether a shadow segment is blocked, which leaf is split and which
 * parent collapsed -- that value is computed in IEEE binary32 with one
 * correctly rounded operation per step, the precision the device kernels
 * decide in. Build with -ffp-contract=off so that no multiply-add is fused.
 * Comparisons of a 24-bit uniform against a product (u * total) are made in
 * double, where the product is exact.
 *
 * Stored tables. Q and C are stored in the table precision (binary32,
 * binary16 or bfloat16): the oracle rounds them once when a pass ends.
 *
 * Parity pins: see tests/test_oracle_*.py (brute-force direct lighting,
 * Lambert's closed form, closed form of Eq. 1, pdf normalisation, the split
 * example of Fig. "TreeCuts", the power-sampler special case, cuRAND Philox).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EMPTY 0xFFFFFFFFFFFFFFFFull
#define ORC_MAX_PROBES 64
#define ORC_PREC_F32 0
#define ORC_PREC_F16 1
#define ORC_PREC_BF16 2
#define ORC_MODE_DESCENT 0
#define ORC_MODE_UNIFORM 1
#define ORC_MODE_DESCENT2 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random        */
/* numbers: as easy as 1, 2, 3"): 10 rounds of the 4x32 Philox S-box with the */
/* two published multipliers, the key bumped by the two Weyl constants       */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in [0, 1): the top 24 bits of a 32-bit word, times 2^-24. Exact in
 * binary32 and binary64. */
static float orc_u24(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

/* The draws of one light sample, indexed linearly: draw i is word (i mod 4) of
 * Philox(counter = (sample id, frame, i / 4, 0), key = (seed lo, seed hi)).
 *   0 cut search   1,2 triangle point   3 in-cluster (uniform mode)
 *   4..7 jitter x, y, z, normal u       8 jitter normal v
 *   9 + k descent level k                                                   */
#define ORC_DRAW_CUT 0
#define ORC_DRAW_TRI_A 1
#define ORC_DRAW_TRI_B 2
#define ORC_DRAW_UNIFORM 3
#define ORC_DRAW_JIT 4
#define ORC_DRAW_DESCENT 9

typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t cached_block;
    uint32_t words[4];
} orc_stream;

static void orc_stream_init(orc_stream* s, uint64_t seed, uint32_t sample_id, uint32_t frame)
{
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->ctr[0] = sample_id;
    s->ctr[1] = frame;
    s->ctr[2] = 0;
    s->ctr[3] = 0;
    s->cached_block = 0xFFFFFFFFu;
}

static float orc_draw(orc_stream* s, uint32_t i)
{
    uint32_t block = i >> 2;
    if (block != s->cached_block) {
        s->ctr[2] = block;
        orc_philox4x32_10(s->ctr, s->key, s->words);
        s->cached_block = block;
    }
    return orc_u24(s->words[i & 3]);
}

/* ------------------------------------------------------------------------ */
/* binary16 / bfloat16 rounding (round to nearest even), written from the   */
/* IEEE 754 format definitions.                                             */
/* ------------------------------------------------------------------------ */
static double orc_round_format(double v, int mant_bits, int emin, double maxval)
{
    if (!(v == v)) return v;
    double a = fabs(v);
    if (a == 0.0) return v;
    if (a >= maxval) {
        /* saturate: values past the largest finite are stored as the largest */
        return v < 0 ? -maxval : maxval;
    }
    int e;
    frexp(a, &e);               /* a = f 2^e, f in [0.5, 1) => exponent e-1 */
    int ex = e - 1;
    if (ex < emin) ex = emin;   /* subnormal range: fixed step */
    double step = ldexp(1.0, ex - mant_bits);
    double q = nearbyint(a / step) * step;  /* default rounding: to nearest even */
    if (q > maxval) q = maxval;
    return v < 0 ? -q : q;
}

double orc_round_storage(double v, int precision)
{
    if (precision == ORC_PREC_F16) return orc_round_format(v, 10, -14, 65504.0);
    if (precision == ORC_PREC_BF16) return orc_round_format(v, 7, -126, 3.3895313892515355e38);
    return (double)(float)v;
}

/* The next representable value above a non-negative v in the format. */
static double orc_next_up(double v, int precision)
{
    int mant = precision == ORC_PREC_F16 ? 10 : (precision == ORC_PREC_BF16 ? 7 : 23);
    int emin = precision == ORC_PREC_F16 ? -14 : -126;
    if (v <= 0.0) return ldexp(1.0, emin - mant);
    int e;
    frexp(v, &e);
    int ex = e - 1;
    if (ex < emin) ex = emin;
    return v + ldexp(1.0, ex - mant);
}

static double orc_next_down(double v, int precision)
{
    int mant = precision == ORC_PREC_F16 ? 10 : (precision == ORC_PREC_BF16 ? 7 : 23);
    int emin = precision == ORC_PREC_F16 ? -14 : -126;
    int e;
    frexp(v, &e);
    int ex = e - 1;
    /* at an exact power of two the step below is half the step above */
    if (v == ldexp(1.0, ex) && ex > emin) ex -= 1;
    if (ex < emin) ex = emin;
    return v - ldexp(1.0, ex - mant);
}

/* ------------------------------------------------------------------------ */
/* Eq. 2 (Section 3): C(0) = Q(0), C(s) = C(s-1) + Q(s), computed after the  */
/* pass. Reading (the paper is silent on zero probabilities): every leaf     */
/* gets a floor eps * sum(Q) / m added before the prefix sum, so no cluster  */
/* with a possible contribution has probability zero; a cell whose largest Q */
/* is below the smallest normal binary32 value (2^-126; in particular a cell */
/* whose Q are all zero) samples its clusters uniformly. With a 16-bit table */
/* the cdf is stored normalised (C(m-1) = 1) and forced strictly increasing. */
/* ------------------------------------------------------------------------ */
void orc_cdf(int m, const double* q, double eps, int precision, double* c_out)
{
    double sum = 0.0, qmax = 0.0;
    for (int s = 0; s < m; ++s) {
        sum += q[s];
        if (q[s] > qmax) qmax = q[s];
    }
    double acc = 0.0;
    int uniform = !(qmax >= 0x1p-126) || !isfinite(sum);
    for (int s = 0; s < m; ++s) {
        double qt = uniform ? 1.0 : q[s] + eps * sum / (double)m;
        acc += qt;
        c_out[s] = acc;
    }
    if (precision == ORC_PREC_F32) {
        for (int s = 0; s < m; ++s) c_out[s] = (double)(float)c_out[s];
        return;
    }
    double total = c_out[m - 1];
    for (int s = 0; s < m - 1; ++s) c_out[s] = orc_round_storage(c_out[s] / total, precision);
    c_out[m - 1] = 1.0;
    double prev = 0.0;
    for (int s = 0; s < m - 1; ++s) {
        if (c_out[s] <= prev) c_out[s] = orc_next_up(prev, precision);
        prev = c_out[s];
    }
    for (int s = m - 2; s >= 0; --s)
        if (c_out[s] >= c_out[s + 1]) c_out[s] = orc_next_down(c_out[s + 1], precision);
}

/* ------------------------------------------------------------------------ */
/* Light tree (Section 3.1: a linear BVH built from the light positions     */
/* alone). Lights are sorted by the 30-bit Morton code of their              */
/* centroid (ties: input index); the tree is the binary radix tree over the   */
/* 64-bit keys (code << 32 | index). Node numbering: internal nodes 0..n-2,   */
/* leaf of sorted light l is n-1+l, the root is node 0; an internal node's   */
/* id is the end of its range that it shares with its parent's split, i.e.   */
/* a left child covering [b, g] is node g and a right child covering         */
/* [g+1, e] is node g+1 (the layout of Karras, HPG 2012).                     */
/*                                                                          */
/* Node record (binary32, decides descent): AABB of all vertices, power      */
/* phi = sum lum(Le) * area (bottom-up, phi(left) + phi(right)), orientation */
/* cone: axis = normalised bottom-up sum of the unnormalised winding normals, */
/* cos_theta = min over the node's lights of axis . n_l (clamped to [-1, 1]). */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    uint32_t* perm;      /* [n] sorted light -> input index            */
    uint32_t* code;      /* [n] Morton code of sorted light            */
    int32_t* left;       /* [n-1]                                       */
    int32_t* right;      /* [n-1]                                       */
    int32_t* parent;     /* [2n-1], -1 at the root                      */
    uint32_t* begin;     /* [2n-1] first sorted light                   */
    uint32_t* end;       /* [2n-1] one past the last sorted light       */
    float* rec;          /* [2n-1][11] bmin xyz, bmax xyz, phi, axis xyz, cos_theta */
    double* phi64;       /* [2n-1] power in double                      */
} orc_tree;

#define REC(t, i) ((t)->rec + (size_t)(i) * 11)

static int orc_cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static uint32_t orc_spread10(uint32_t v)
{
    uint32_t r = 0;
    for (int i = 0; i < 10; ++i) r |= ((v >> i) & 1u) << (3 * i);
    return r;
}

static int orc_clz64(uint64_t v)
{
    int n = 0;
    for (int i = 63; i >= 0; --i) {
        if ((v >> i) & 1u) break;
        ++n;
    }
    return n;
}

static float orc_lum32(const float* le)
{
    return (0.2126f * le[0] + 0.7152f * le[1]) + 0.0722f * le[2];
}

static double orc_lum64(double r, double g, double b) { return 0.2126 * r + 0.7152 * g + 0.0722 * b; }

/* binary32 winding cross product and its length (decision data) */
static void orc_cross32(const float* v, float cr[3], float* len)
{
    float e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    float e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
    cr[0] = e1y * e2z - e1z * e2y;
    cr[1] = e1z * e2x - e1x * e2z;
    cr[2] = e1x * e2y - e1y * e2x;
    *len = sqrtf((cr[0] * cr[0] + cr[1] * cr[1]) + cr[2] * cr[2]);
}

typedef struct {
    const orc_tree* t;
    const uint64_t* keys;
    int64_t n;
} orc_build_ctx;

static void orc_build_rec(orc_build_ctx* b, int64_t lo, int64_t hi, int32_t id, int32_t parent)
{
    const orc_tree* t = b->t;
    int64_t n = b->n;
    t->parent[id] = parent;
    t->begin[id] = (uint32_t)lo;
    t->end[id] = (uint32_t)(hi + 1);
    if (lo == hi) return;
    int prefix = orc_clz64(b->keys[lo] ^ b->keys[hi]);
    int64_t g = lo;
    for (int64_t j = lo; j < hi; ++j)
        if (orc_clz64(b->keys[lo] ^ b->keys[j]) > prefix) g = j;
    int32_t lid = (g == lo) ? (int32_t)(n - 1 + g) : (int32_t)g;
    int32_t rid = (g + 1 == hi) ? (int32_t)(n - 1 + g + 1) : (int32_t)(g + 1);
    t->left[id] = lid;
    t->right[id] = rid;
    orc_build_rec(b, lo, g, lid, id);
    orc_build_rec(b, g + 1, hi, rid, id);
}

/* bottom-up binary32 bounds; returns the unnormalised axis sum in s[3] */
static void orc_bounds_rec(const orc_tree* t, int32_t id, const float* tri, const float* emis, float s[3])
{
    int64_t n = t->n;
    float* r = REC(t, id);
    if (id >= n - 1) {
        int64_t l = id - (n - 1);
        const float* v = tri + (size_t)t->perm[l] * 9;
        float cr[3], len;
        orc_cross32(v, cr, &len);
        for (int k = 0; k < 3; ++k) {
            float a = fminf(fminf(v[k], v[3 + k]), v[6 + k]);
            float c = fmaxf(fmaxf(v[k], v[3 + k]), v[6 + k]);
            r[k] = a;
            r[3 + k] = c;
            s[k] = cr[k];
        }
        float area = 0.5f * len;
        r[6] = orc_lum32(emis + (size_t)t->perm[l] * 3) * area;
        return;
    }
    float sl[3], sr[3];
    orc_bounds_rec(t, t->left[id], tri, emis, sl);
    orc_bounds_rec(t, t->right[id], tri, emis, sr);
    const float* a = REC(t, t->left[id]);
    const float* c = REC(t, t->right[id]);
    for (int k = 0; k < 3; ++k) {
        r[k] = fminf(a[k], c[k]);
        r[3 + k] = fmaxf(a[3 + k], c[3 + k]);
        s[k] = sl[k] + sr[k];
    }
    r[6] = a[6] + c[6];
}

/* ------------------------------------------------------------------------ */
/* Surface-area-orientation split positions (Section 3.1 leaves a hierarchy   */
/* that considers light orientations and a surface area heuristic as future  */
/* work). Reading: the lights keep their Morton order, so every node is still */
/* a contiguous range; only the split position of each node changes. For a   */
/* range of m lights the candidates are every position when m <= 17, else    */
/* the 15 positions b + floor(m j / 16) (j = 1..15) and the Morton split; the */
/* chosen one minimises cost(L) + cost(R) (ties: the smallest position),     */
/* with cost(S) = phi(S) * SA(box(S)) * (2 - |sum_S c_i| / sum_S |c_i|),     */
/* c_i the winding cross product of light i (twice its area times its unit  */
/* normal), SA the box's surface area. phi, |c| and c are summed exactly in  */
/* 64-bit fixed point (scale 2^(30 - e), e the exponent of the largest       */
/* value), so that any summation order gives the same sums; the cost is     */
/* then evaluated in binary32 from the sums converted to float. Internal    */
/* node ids are (split position - split position of the root) mod (n - 1),  */
/* so the root is 0; leaves keep n - 1 + l.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_tree* t;
    const uint64_t* keys;
    int64_t n;
    const int64_t* pphi;   /* [n+1] prefix sums, fixed point */
    const int64_t* parea;  /* [n+1] */
    const int64_t* pc;     /* [3][n+1] */
    const float* lbox;     /* [n][6] light boxes */
    int64_t groot;
    int median;            /* split every range at its middle instead */
} orc_saoh_ctx;

static int orc_exponent(double v)
{
    int e = 0;
    frexp(v, &e);
    return e;
}

static float orc_box_area(const float b[6])
{
    float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return 2.0f * ((dx * dy + dy * dz) + dz * dx);
}

static float orc_saoh_cost(const orc_saoh_ctx* x, int64_t lo, int64_t hi, const float box[6])
{
    float phi = (float)(x->pphi[hi] - x->pphi[lo]);
    float area = (float)(x->parea[hi] - x->parea[lo]);
    float cx = (float)(x->pc[hi] - x->pc[lo]);
    float cy = (float)(x->pc[(x->n + 1) + hi] - x->pc[(x->n + 1) + lo]);
    float cz = (float)(x->pc[2 * (x->n + 1) + hi] - x->pc[2 * (x->n + 1) + lo]);
    float om = 1.0f;
    if (area > 0.0f) om = 2.0f - sqrtf((cx * cx + cy * cy) + cz * cz) / area;
    return (phi * orc_box_area(box)) * om;
}

/* Morton split of [lo, hi] (inclusive): last g with a longer common prefix with lo than hi has */
static int64_t orc_morton_split(const uint64_t* keys, int64_t lo, int64_t hi)
{
    int prefix = orc_clz64(keys[lo] ^ keys[hi]);
    int64_t g = lo;
    for (int64_t j = lo; j < hi; ++j)
        if (orc_clz64(keys[lo] ^ keys[j]) > prefix) g = j;
    return g;
}

/* split position k (first index of the right child) of the range [b, e) */
int64_t orc_saoh_split(const orc_saoh_ctx* x, int64_t b, int64_t e)
{
    int64_t m = e - b;
    int64_t cand[17];
    int nc = 0;
    if (m <= 17) {
        for (int64_t k = b + 1; k < e; ++k) cand[nc++] = k;
    } else {
        int64_t km = orc_morton_split(x->keys, b, e - 1) + 1;
        int dup = 0;
        for (int j = 1; j <= 15; ++j) {
            cand[nc++] = b + (m * j) / 16;
            dup |= cand[nc - 1] == km;
        }
        if (!dup) cand[nc++] = km;
    }
    float best = INFINITY;
    int64_t bk = b + 1;
    for (int c = 0; c < nc; ++c) {
        int64_t k = cand[c];
        float lb[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        float rb[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int64_t l = b; l < e; ++l) {
            float* bb = l < k ? lb : rb;
            for (int q = 0; q < 3; ++q) {
                bb[q] = fminf(bb[q], x->lbox[l * 6 + q]);
                bb[3 + q] = fmaxf(bb[3 + q], x->lbox[l * 6 + 3 + q]);
            }
        }
        float cst = orc_saoh_cost(x, b, k, lb) + orc_saoh_cost(x, k, e, rb);
        if (cst < best || (cst == best && k < bk)) {
            best = cst;
            bk = k;
        }
    }
    return bk;
}

static int32_t orc_saoh_id(const orc_saoh_ctx* x, int64_t g)
{
    int64_t nm1 = x->n - 1;
    return (int32_t)(((g - x->groot) % nm1 + nm1) % nm1);
}

/* node [b, e) with split k; returns its id, fills the arrays below it */
static int32_t orc_saoh_rec(orc_saoh_ctx* x, int64_t b, int64_t e, int32_t parent)
{
    orc_tree* t = x->t;
    if (e - b == 1) {
        int32_t id = (int32_t)(x->n - 1 + b);
        t->parent[id] = parent;
        t->begin[id] = (uint32_t)b;
        t->end[id] = (uint32_t)e;
        return id;
    }
    int64_t k = x->median ? b + (e - b) / 2 : orc_saoh_split(x, b, e);
    if (parent < 0) x->groot = k - 1;
    int32_t id = orc_saoh_id(x, k - 1);
    t->parent[id] = parent;
    t->begin[id] = (uint32_t)b;
    t->end[id] = (uint32_t)e;
    t->left[id] = orc_saoh_rec(x, b, k, id);
    t->right[id] = orc_saoh_rec(x, k, e, id);
    return id;
}

static int orc_build_tree_with(int64_t n, const float* tri, const float* emis, orc_tree* t, int builder)
{
    if (n <= 0) return -1;
    t->n = n;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float* cen = (float*)malloc(sizeof(float) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const float* v = tri + (size_t)i * 9;
        for (int k = 0; k < 3; ++k) {
            float c = ((v[k] + v[3 + k]) + v[6 + k]) / 3.0f;
            cen[i * 3 + k] = c;
            lo[k] = fminf(lo[k], c);
            hi[k] = fmaxf(hi[k], c);
        }
    }
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            float ext = hi[k] - lo[k];
            float u = ext > 0.0f ? (cen[i * 3 + k] - lo[k]) / ext : 0.0f;
            float f = floorf(u * 1024.0f);
            int iq = (int)f;
            if (iq < 0) iq = 0;
            if (iq > 1023) iq = 1023;
            q[k] = (uint32_t)iq;
        }
        uint32_t code = (orc_spread10(q[0]) << 2) | (orc_spread10(q[1]) << 1) | orc_spread10(q[2]);
        keys[i] = ((uint64_t)code << 32) | (uint64_t)i;
    }
    qsort(keys, (size_t)n, sizeof(uint64_t), orc_cmp_u64);
    for (int64_t l = 0; l < n; ++l) {
        t->perm[l] = (uint32_t)(keys[l] & 0xFFFFFFFFu);
        t->code[l] = (uint32_t)(keys[l] >> 32);
    }
    if (builder == 0 || n < 2) {
        orc_build_ctx b = {t, keys, n};
        orc_build_rec(&b, 0, n - 1, 0, -1);
    } else {
        /* fixed-point prefix sums of power, |c| and c over the sorted lights */
        int64_t* pphi = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
        int64_t* parea = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
        int64_t* pc = (int64_t*)calloc((size_t)(3 * (n + 1)), sizeof(int64_t));
        float* lbox = (float*)malloc(sizeof(float) * 6 * (size_t)n);
        float* phi = (float*)malloc(sizeof(float) * (size_t)n);
        float* cr = (float*)malloc(sizeof(float) * 4 * (size_t)n);
        double mphi = 0.0, mc = 0.0;
        for (int64_t l = 0; l < n; ++l) {
            const float* v = tri + (size_t)t->perm[l] * 9;
            float c[3], len;
            orc_cross32(v, c, &len);
            for (int k = 0; k < 3; ++k) {
                lbox[l * 6 + k] = fminf(fminf(v[k], v[3 + k]), v[6 + k]);
                lbox[l * 6 + 3 + k] = fmaxf(fmaxf(v[k], v[3 + k]), v[6 + k]);
                cr[l * 4 + k] = c[k];
                if (fabs((double)c[k]) > mc) mc = fabs((double)c[k]);
            }
            cr[l * 4 + 3] = len;
            if ((double)len > mc) mc = len;
            phi[l] = orc_lum32(emis + (size_t)t->perm[l] * 3) * (0.5f * len);
            if ((double)phi[l] > mphi) mphi = phi[l];
        }
        int sp = 30 - orc_exponent(mphi), sc = 30 - orc_exponent(mc);
        for (int64_t l = 0; l < n; ++l) {
            pphi[l + 1] = pphi[l] + llrint(ldexp((double)phi[l], sp));
            parea[l + 1] = parea[l] + llrint(ldexp((double)cr[l * 4 + 3], sc));
            for (int k = 0; k < 3; ++k)
                pc[k * (n + 1) + l + 1] = pc[k * (n + 1) + l] + llrint(ldexp((double)cr[l * 4 + k], sc));
        }
        orc_saoh_ctx x = {t, keys, n, pphi, parea, pc, lbox, 0, builder == 2};
        orc_saoh_rec(&x, 0, n, -1);
        free(pphi);
        free(parea);
        free(pc);
        free(lbox);
        free(phi);
        free(cr);
    }

    float s[3];
    orc_bounds_rec(t, 0, tri, emis, s);
    /* axes and cones need the axis sum of every node: recompute per node */
    int64_t nn = 2 * n - 1;
    float* sums = (float*)calloc((size_t)nn * 3, sizeof(float));
    /* leaves first, then internal nodes in an order where children precede
       parents: a post-order walk with an explicit stack */
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)nn * 2);
    int64_t sp = 0;
    stack[sp++] = 0;
    uint8_t* done = (uint8_t*)calloc((size_t)nn, 1);
    while (sp > 0) {
        int32_t id = stack[sp - 1];
        if (id >= n - 1) {
            float cr[3], len;
            orc_cross32(tri + (size_t)t->perm[id - (n - 1)] * 9, cr, &len);
            sums[id * 3 + 0] = cr[0];
            sums[id * 3 + 1] = cr[1];
            sums[id * 3 + 2] = cr[2];
            done[id] = 1;
            --sp;
            continue;
        }
        int32_t a = t->left[id], c = t->right[id];
        if (!done[a]) { stack[sp++] = a; continue; }
        if (!done[c]) { stack[sp++] = c; continue; }
        for (int k = 0; k < 3; ++k) sums[id * 3 + k] = sums[a * 3 + k] + sums[c * 3 + k];
        done[id] = 1;
        --sp;
    }
    free(stack);
    free(done);
    /* unit normals of the sorted lights (binary32) */
    float* nl = (float*)malloc(sizeof(float) * 3 * (size_t)n);
    for (int64_t l = 0; l < n; ++l) {
        float cr[3], len;
        orc_cross32(tri + (size_t)t->perm[l] * 9, cr, &len);
        for (int k = 0; k < 3; ++k) nl[l * 3 + k] = cr[k] / len;
    }
    for (int64_t id = 0; id < nn; ++id) {
        float* r = REC(t, id);
        float sx = sums[id * 3], sy = sums[id * 3 + 1], sz = sums[id * 3 + 2];
        float len = sqrtf((sx * sx + sy * sy) + sz * sz);
        if (len > 0.0f) {
            r[7] = sx / len;
            r[8] = sy / len;
            r[9] = sz / len;
            float cmin = 1.0f;
            for (uint32_t l = t->begin[id]; l < t->end[id]; ++l) {
                float d = (r[7] * nl[l * 3] + r[8] * nl[l * 3 + 1]) + r[9] * nl[l * 3 + 2];
                cmin = fminf(cmin, d);
            }
            r[10] = fmaxf(-1.0f, cmin);
        } else {
            r[7] = 0.0f;
            r[8] = 0.0f;
            r[9] = 1.0f;
            r[10] = -1.0f;
        }
        /* power in double: sum over the node's lights */
        double p = 0.0;
        for (uint32_t l = t->begin[id]; l < t->end[id]; ++l) {
            const float* v = tri + (size_t)t->perm[l] * 9;
            double e1[3], e2[3];
            for (int k = 0; k < 3; ++k) {
                e1[k] = (double)v[3 + k] - v[k];
                e2[k] = (double)v[6 + k] - v[k];
            }
            double cx = e1[1] * e2[2] - e1[2] * e2[1];
            double cy = e1[2] * e2[0] - e1[0] * e2[2];
            double cz = e1[0] * e2[1] - e1[1] * e2[0];
            double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
            const float* le = emis + (size_t)t->perm[l] * 3;
            p += orc_lum64(le[0], le[1], le[2]) * area;
        }
        t->phi64[id] = p;
    }
    free(nl);
    free(sums);
    free(cen);
    free(keys);
    return 0;
}

int orc_build_tree(int64_t n, const float* tri, const float* emis, orc_tree* t)
{
    return orc_build_tree_with(n, tri, emis, t, 0);
}

/* builder 0: the radix tree of the Morton codes (Section 3.1); 1: the
 * surface-area-orientation split positions above; 2: the same light order
 * with every range [b, e) split at b + floor((e - b) / 2) (a balanced tree) */
int orc_build_tree_ex(int64_t n, const float* tri, const float* emis, orc_tree* t, int builder)
{
    return orc_build_tree_with(n, tri, emis, t, builder);
}

/* ------------------------------------------------------------------------ */
/* Initial cut (Section 3: any heuristic may pick it; the paper suggests a   */
/* breadth-first descent until M nodes are collected): a FIFO queue seeded with the */
/* root; pop the front node, push its two children (a single light is pushed */
/* back unchanged) until the queue holds min(M, n) nodes. Stored sorted by    */
/* range begin, i.e. as the monotone list of cluster ends of Section 3.       */
/* ------------------------------------------------------------------------ */
static const orc_tree* orc_sort_tree;
static int orc_cmp_begin(const void* a, const void* b)
{
    uint32_t x = orc_sort_tree->begin[*(const int32_t*)a], y = orc_sort_tree->begin[*(const int32_t*)b];
    return x < y ? -1 : (x > y ? 1 : 0);
}

int orc_initial_cut(const orc_tree* t, int M, int32_t* cut)
{
    int64_t n = t->n;
    int m = (int64_t)M < n ? M : (int)n;
    int cap = 2 * m + 4;
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap * 4);
    int head = 0, tail = 0, size = 0;
    int qcap = cap * 4;
    q[tail] = 0; tail = (tail + 1) % qcap; size = 1;
    while (size < m) {
        int32_t id = q[head];
        head = (head + 1) % qcap;
        --size;
        if (id >= n - 1) {
            q[tail] = id; tail = (tail + 1) % qcap; ++size;
        } else {
            q[tail] = t->left[id]; tail = (tail + 1) % qcap; ++size;
            q[tail] = t->right[id]; tail = (tail + 1) % qcap; ++size;
        }
    }
    for (int i = 0; i < m; ++i) cut[i] = q[(head + i) % qcap];
    orc_sort_tree = t;
    qsort(cut, (size_t)m, sizeof(int32_t), orc_cmp_begin);
    free(q);
    return m;
}

/* ------------------------------------------------------------------------ */
/* 5-d hash grid (Section 3: jittered quantised position (3) and normal (2)). */
/* Reading: fixed cell size h from the grid origin; normals by the octahedral */
/* map (y up) quantised to nb bins per axis; jitter of +-1/2 cell or bin per  */
/* lookup; 16-bit position fields biased by 2^15, 8-bit normal fields.       */
/* All quantisation arithmetic is binary32.                                  */
/* ------------------------------------------------------------------------ */
/* Multi-resolution reading of the footprint-sized cells (Section 3: cells  */
/* sized from the ray footprint of each path vertex, coarser on later        */
/* bounces): `levels` tables of Hl slots each (H = levels * Hl); level l has  */
/* cell size h * 2^l and its own slot range [l * Hl, (l + 1) * Hl). A point   */
/* with footprint f uses the smallest level whose cell is at least f wide:   */
/* l = ceil(log2(f / h)) clamped to [0, levels - 1], from the binary32       */
/* quotient; points without a footprint use level 0.                        */
typedef struct {
    uint32_t H, M, m;
    float origin[3];
    float h;
    uint32_t nb, jitter, mode, reward_mode, precision;
    double alpha, T, eps;
    uint64_t* keys;   /* [H] */
    int32_t* cut;     /* [H*M] node ids */
    double* Q;        /* [H*M] stored (table precision) values */
    double* C;        /* [H*M] stored (table precision) values */
    const int32_t* def_cut;  /* [m] */
    const double* def_Q;     /* [m] */
    const double* def_C;     /* [m] */
    uint32_t levels;  /* resolution levels (1: a single grid of cell size h) */
    uint32_t Hl;      /* slots per level (H / levels) */
} orc_grid;

/* level of a point with footprint f (see orc_grid) */
uint32_t orc_footprint_level(float f, float h, uint32_t levels)
{
    float r = f / h;
    if (!(r > 1.0f)) return 0;
    uint32_t b;
    memcpy(&b, &r, sizeof b);
    uint32_t e = ((b >> 23) & 0xFFu) - 127u;       /* r > 1: biased exponent >= 127 */
    uint32_t l = e + ((b & 0x7FFFFFu) != 0u);      /* ceil(log2 r) */
    uint32_t top = levels > 0 ? levels - 1 : 0;
    return l < top ? l : top;
}

static int32_t orc_qpos(float p, float o, float h, int jit, float u)
{
    float t = (p - o) / h;
    if (jit) t = t + (u - 0.5f);
    float f = floorf(t);
    if (f < -32767.0f) f = -32767.0f;
    if (f > 32766.0f) f = 32766.0f;
    return (int32_t)f + 32768;
}

static uint32_t orc_qnrm(float a, uint32_t nb, int jit, float u)
{
    float q = ((a + 1.0f) * 0.5f) * (float)nb;
    if (jit) q = q + (u - 0.5f);
    float f = floorf(q);
    if (f < 0.0f) f = 0.0f;
    if (f > (float)(nb - 1)) f = (float)(nb - 1);
    return (uint32_t)f;
}

/* key of the cell of cell size h_cell (h * 2^level) */
static uint64_t orc_cell_key_h(const orc_grid* g, float h_cell, const float p[3], const float nrm[3],
                               const float jit[5])
{
    int j = g->jitter != 0;
    uint32_t fx = (uint32_t)orc_qpos(p[0], g->origin[0], h_cell, j, j ? jit[0] : 0.0f);
    uint32_t fy = (uint32_t)orc_qpos(p[1], g->origin[1], h_cell, j, j ? jit[1] : 0.0f);
    uint32_t fz = (uint32_t)orc_qpos(p[2], g->origin[2], h_cell, j, j ? jit[2] : 0.0f);
    float ax = fabsf(nrm[0]), ay = fabsf(nrm[1]), az = fabsf(nrm[2]);
    float s = (ax + ay) + az;
    float a = 0.0f, b = 0.0f;
    if (s > 0.0f) {
        a = nrm[0] / s;
        b = nrm[2] / s;
        if (nrm[1] < 0.0f) {
            float sa = a >= 0.0f ? 1.0f : -1.0f, sb = b >= 0.0f ? 1.0f : -1.0f;
            float na = (1.0f - fabsf(b)) * sa;
            float nbv = (1.0f - fabsf(a)) * sb;
            a = na;
            b = nbv;
        }
    }
    uint32_t iu = orc_qnrm(a, g->nb, j, j ? jit[3] : 0.0f);
    uint32_t iv = orc_qnrm(b, g->nb, j, j ? jit[4] : 0.0f);
    return (uint64_t)fx | ((uint64_t)fy << 16) | ((uint64_t)fz << 32) | ((uint64_t)iu << 48) |
           ((uint64_t)iv << 56);
}

uint64_t orc_cell_key(const orc_grid* g, const float p[3], const float nrm[3], const float jit[5])
{
    return orc_cell_key_h(g, g->h, p, nrm, jit);
}

/* key at a level: cell size h * 2^level (exact in binary32) */
uint64_t orc_cell_key_level(const orc_grid* g, uint32_t level, const float p[3], const float nrm[3],
                            const float jit[5])
{
    return orc_cell_key_h(g, ldexpf(g->h, (int)level), p, nrm, jit);
}

/* MurmurHash3 64-bit finaliser (Appleby), slot = hash mod H */
uint64_t orc_fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

/* Lookup with lazy creation (Section 3: the initial cut is copied into a cell
 * the first time it is used): linear probing from fmix64(key) mod H for at most
 * 64 slots. Returns the slot, or -1 when the probe limit is reached. */
static int64_t orc_lookup_insert_level(orc_grid* g, uint32_t level, uint64_t key)
{
    uint64_t h = orc_fmix64(key);
    uint32_t hl = g->Hl ? g->Hl : g->H;
    for (uint32_t i = 0; i < ORC_MAX_PROBES; ++i) {
        uint64_t slot = (uint64_t)level * hl + ((h + i) & (uint64_t)(hl - 1));
        if (g->keys[slot] == key) return (int64_t)slot;
        if (g->keys[slot] == ORC_EMPTY) {
            g->keys[slot] = key;
            for (uint32_t s = 0; s < g->m; ++s) {
                g->cut[slot * g->M + s] = g->def_cut[s];
                g->Q[slot * g->M + s] = g->def_Q[s];
                g->C[slot * g->M + s] = g->def_C[s];
            }
            return (int64_t)slot;
        }
    }
    return -1;
}

int64_t orc_lookup_insert(orc_grid* g, uint64_t key) { return orc_lookup_insert_level(g, 0, key); }

/* ------------------------------------------------------------------------ */
/* Node importance for the stochastic descent below a cut node (binary32).   */
/* Reading (the paper picks the light inside a cluster at random; a descent by */
/* unoccluded bounds follows the bound-based samplers it cites, Section 2):   */
/*   I = phi * Brecv * Bemit / d^2,  d = AABB centre - x, r = half diagonal,  */
/*   sin(beta) = r / |d|; Brecv bounds max(0, n . w) and Bemit bounds         */
/*   max(0, -n_l . w) over directions w within beta of d/|d| and normals n_l */
/*   within the node's cone (axis, half angle theta); a point inside the      */
/*   bounding sphere gets I = phi / r^2. Angle sums by the addition formulas; */
/*   every cosine and sine is carried multiplied by |d| so that only         */
/*   sqrt(d^2 - r^2) and two more square roots are needed; the bound is kept */
/*   as num / den = (phi A B) / d^6 and two bounds are compared by cross      */
/*   multiplication, without a division.                                    */
/*   Node constants are binary32 values of the node record, computed with    */
/*   the same operations on both sides, and kept compact: r = the square     */
/*   root of the squared half diagonal rounded up by one ulp, r^2 = r r      */
/*   (not below the box's own r^2); the cone as 1 - cos theta rounded up to  */
/*   binary16 (a cone at least as wide) and sin theta of that cone rounded   */
/*   up to binary16 (orc_node_consts32).                                     */
/* ------------------------------------------------------------------------ */

/* x rounded to binary16 toward -inf (up = 0) or +inf (up = 1); |x| < 65504.  */
/* The binary16 values of the binade of |x| are multiples of its ulp          */
/* 2^(E - 10) (2^-24 below 2^-14), so the rounding is a floor or ceiling of   */
/* x / ulp, exact in double.                                                  */
static double orc_half_round64(double x, int up)
{
    if (x == 0.0) return x;
    int e = 0;
    frexp(fabs(x), &e);
    int E = e - 1;                 /* 2^E <= |x| < 2^(E+1) */
    if (E < -14) E = -14;
    double q = ldexp(1.0, E - 10);
    double k = x / q;
    return (up ? ceil(k) : floor(k)) * q;
}

float orc_half_round(float x, int up) { return (float)orc_half_round64((double)x, up); }

/* The compact constants of a node's descent bound (reading of the stored
 * bound, see above), from its record r = bmin xyz, bmax xyz, phi, cone axis
 * xyz, cone cos: k[0..2] the box centre (binary32), k[3] the radius r
 * (binary32 square root of the squared half diagonal, one ulp up), k[4] =
 * r r; the cone as k[5] = cos theta' = 1 - v, where v is 1 - cos theta
 * rounded up to binary16 (a cone at least as wide; binary16 keeps 11
 * significant bits of v, so narrow cones stay narrow), and k[6] = sin theta'
 * rounded up to binary16, from the exact 1 - cos^2 theta' = v (2 - v). */
void orc_node_consts32(const float* r, float k[7])
{
    k[0] = (r[0] + r[3]) * 0.5f;
    k[1] = (r[1] + r[4]) * 0.5f;
    k[2] = (r[2] + r[5]) * 0.5f;
    float ex = r[3] - r[0], ey = r[4] - r[1], ez = r[5] - r[2];
    float rb2 = 0.25f * ((ex * ex + ey * ey) + ez * ez);
    k[3] = nextafterf(sqrtf(rb2), INFINITY);
    k[4] = k[3] * k[3];
    double v = orc_half_round64(1.0 - (double)r[10], 1);  /* 1 - cos exact in double */
    k[5] = (float)(1.0 - v);                             /* exact in binary32 */
    k[6] = (float)orc_half_round64(sqrt(v * (2.0 - v)), 1);
}

void orc_importance32(const float* r, const float x[3], const float n[3], float* num, float* den)
{
    float k[7];
    orc_node_consts32(r, k);
    float cx = k[0], cy = k[1], cz = k[2];
    float rr = k[3], r2 = k[4], ct = k[5], st = k[6];
    float phi = r[6];
    float dx = cx - x[0], dy = cy - x[1], dz = cz - x[2];
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (d2 <= r2) {
        *num = phi;
        *den = fmaxf(r2, 1e-30f);
        return;
    }
    float cb = sqrtf(d2 - r2);                              /* |d| cos(beta)        */
    float nd = fmaf(n[2], dz, fmaf(n[1], dy, n[0] * dx));   /* |d| cos(gamma)       */
    float A;                                                /* |d|^2 Brecv          */
    if (nd >= cb) A = d2;
    else A = fmaxf(0.0f, fmaf(nd, cb, sqrtf(fmaxf(0.0f, fmaf(-nd, nd, d2))) * rr));
    float ad = -fmaf(r[9], dz, fmaf(r[8], dy, r[7] * dx));  /* |d| cos(psi)         */
    float sphi = fmaf(st, cb, ct * rr);                     /* |d| sin(theta+beta)  */
    float cphi = fmaf(ct, cb, -(st * rr));                  /* |d| cos(theta+beta)  */
    float B;                                                /* |d|^2 Bemit          */
    if (sphi <= 0.0f || cphi <= ad) B = d2;
    else B = fmaxf(0.0f, fmaf(ad, cphi, sqrtf(fmaxf(0.0f, fmaf(-ad, ad, d2))) * sphi));
    *num = (phi * A) * B;
    *den = (d2 * d2) * d2;
}

/* The same bound written out plainly in double precision, as a check of the
 * binary32 form above (which carries the cosines multiplied by |d| and
 * compares bounds without dividing). Inputs are the node's constants:
 * centre c, radius r, cone cos theta and sin theta, cone axis a (unit),
 * power phi; x the shading point, n its unit normal.
 *   w = d / |d| with d = c - x is the direction to the centre; the sphere of
 *   radius r subtends the half angle beta, sin beta = r / |d|.
 *   Receiver: gamma = angle(n, w). Over directions within beta of w,
 *   max(0, n . omega) is 1 if gamma <= beta, else max(0, cos(gamma - beta)).
 *   Emitter: psi = angle(a, -w), the angle between the cone axis and the
 *   direction from the node back to x. Over normals within theta of a and
 *   directions within beta of w, max(0, -n_l . omega) is 1 if
 *   psi <= theta + beta (or theta + beta >= pi), else
 *   max(0, cos(psi - (theta + beta))).
 *   I = phi * Brecv * Bemit / |d|^2; inside the sphere (|d| <= r) I = phi / r^2.
 * The cosines of the angle differences and sums come from the addition
 * formulas with the sines sqrt(1 - cos^2). */
double orc_bound64(const double c[3], double r, double cos_t, double sin_t, const double a[3], double phi,
                   const double x[3], const double n[3])
{
    double d[3] = {c[0] - x[0], c[1] - x[1], c[2] - x[2]};
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (d2 <= r * r) return phi / (r * r);
    double dist = sqrt(d2);
    double w[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
    double sin_b = r / dist;
    double cos_b = sqrt(1.0 - sin_b * sin_b);

    double cos_g = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
    double sin_g = sqrt(fmax(0.0, 1.0 - cos_g * cos_g));
    double recv;
    if (cos_g >= cos_b) recv = 1.0;                          /* gamma <= beta */
    else recv = fmax(0.0, cos_g * cos_b + sin_g * sin_b);   /* cos(gamma - beta) */

    double cos_p = -(a[0] * w[0] + a[1] * w[1] + a[2] * w[2]);
    double sin_p = sqrt(fmax(0.0, 1.0 - cos_p * cos_p));
    double cos_tb = cos_t * cos_b - sin_t * sin_b;          /* cos(theta + beta) */
    double sin_tb = sin_t * cos_b + cos_t * sin_b;          /* sin(theta + beta) */
    double emit;
    if (sin_tb <= 0.0 || cos_p >= cos_tb) emit = 1.0;         /* psi <= theta + beta */
    else emit = fmax(0.0, cos_p * cos_tb + sin_p * sin_tb); /* cos(psi - theta - beta) */

    return phi * recv * emit / d2;
}

/* Branch weights of the two children a, c of a descent step: the bounds
 * I = num / den compared without a division, w_a = num_a den_c and
 * w_c = num_c den_a (binary32); if both are zero, the children's powers. */
static void orc_branch_weights(const float* ra, const float* rc, const float x[3], const float n[3],
                               float* wa, float* wc)
{
    float na, da, nc, dc;
    orc_importance32(ra, x, n, &na, &da);
    orc_importance32(rc, x, n, &nc, &dc);
    *wa = na * dc;
    *wc = nc * da;
    if (!((*wa + *wc) > 0.0f)) {
        *wa = ra[6];
        *wc = rc[6];
    }
}

/* ------------------------------------------------------------------------ */
/* Shadow test (binary32): segment from o = x + 1e-4 n to the light point y, */
/* parameter t in (0, 0.9999), slab test against every box (open intervals). */
/* Each slab plane is t = fma(b, 1/d, -(o * (1/d))): one fused multiply-add, */
/* correctly rounded (C99 fmaf). A direction component with |d| < 2^-100     */
/* (the segment does not move along that axis; 1/d would be infinite and the */
/* planes undefined) is taken as 2^-100 with the sign of d: o * 2^100 is     */
/* exact, so the planes lie at t = (b - o) 2^100 rounded, and the segment is */
/* inside that slab exactly when b_min < o < b_max, as the double test below */
/* decides for a parallel segment (one lying on a face plane goes by the     */
/* sign given to d).                                                         */
/* ------------------------------------------------------------------------ */
static int orc_occluded32(const float o[3], const float y[3], int nbox, const float* boxes)
{
    float d[3], inv[3], oi[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = y[k] - o[k];
        if (!(fabsf(d[k]) >= 0x1p-100f)) d[k] = copysignf(0x1p-100f, d[k]);
        inv[k] = 1.0f / d[k];
        oi[k] = o[k] * inv[k];
    }
    for (int b = 0; b < nbox; ++b) {
        const float* bx = boxes + (size_t)b * 6;
        float tn = 0.0f, tf = 0.9999f;
        for (int k = 0; k < 3; ++k) {
            float t0 = fmaf(bx[k], inv[k], -oi[k]);
            float t1 = fmaf(bx[3 + k], inv[k], -oi[k]);
            tn = fmaxf(tn, fminf(t0, t1));
            tf = fminf(tf, fmaxf(t0, t1));
        }
        if (tn < tf) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One light sample (Section 3, "Main contribution"): binary search in C for  */
/* the cluster s, a light l in s, the contribution c_l with its shadow test.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t light;       /* sorted light index */
    int64_t slot;        /* -1: no cell (probe limit) */
    int32_t s;           /* cluster position in the cut */
    int32_t visible;
    double p_cut, p_in, area;
    double est[3];       /* contribution / pdf */
    double reward;       /* |c| fed to Eq. 1 */
    double margin;       /* smallest distance of a deciding draw to its threshold */
} orc_sample_out;

typedef struct {
    const orc_tree* tree;
    const float* tri;      /* [N][9] input order */
    const float* emis;     /* [N][3] current radiance, input order */
    int nbox;
    const float* boxes;    /* [K][6] */
} orc_scene;

static double orc_min(double a, double b) { return a < b ? a : b; }

/* Two-level descent (reading of the in-cluster choice): from internal node g
 * the candidates are the children of g's children, a child that is a single
 * light standing for itself (2 to 4 candidates, in light order). Candidate i
 * has weight w_i = num_i / max(den_i, 1e-30) (binary32, its descent bound);
 * if all weights are 0 the candidates' powers are used, if those are 0 too
 * the choice is uniform. With the binary32 prefix sums P_i = w_0 + ... + w_i
 * (in order) and S = P_{k-1}, the chosen candidate is the first i with
 * u S < P_i, and its probability is (P_i - P_{i-1}) / S. */
static int orc_frontier(const orc_tree* t, int32_t g, int32_t cand[4])
{
    int64_t nl = t->n;
    int k = 0;
    int32_t kids[2] = {t->left[g], t->right[g]};
    for (int j = 0; j < 2; ++j) {
        int32_t x = kids[j];
        if (x >= nl - 1) {
            cand[k++] = x;
        } else {
            cand[k++] = t->left[x];
            cand[k++] = t->right[x];
        }
    }
    return k;
}

static void orc_frontier_weights(const orc_tree* t, const int32_t* cand, int k, const float x[3],
                                 const float n[3], float w[4], int* uniform)
{
    float sum = 0.0f;
    for (int i = 0; i < k; ++i) {
        float num, den;
        orc_importance32(REC(t, cand[i]), x, n, &num, &den);
        w[i] = num / fmaxf(den, 1e-30f);
        sum = sum + w[i];
    }
    *uniform = 0;
    if (!(sum > 0.0f)) {
        sum = 0.0f;
        for (int i = 0; i < k; ++i) {
            w[i] = REC(t, cand[i])[6];
            sum = sum + w[i];
        }
        if (!(sum > 0.0f)) *uniform = 1;
    }
}

/* descend from cut node `node` to a light; returns the light and multiplies
 * p_in; margin tracks the closest deciding draw. */
static int64_t orc_descend(const orc_scene* sc, int mode, int32_t node, const float x[3],
                           const float n[3], orc_stream* rs, double* p_in, double* margin)
{
    const orc_tree* t = sc->tree;
    int64_t nl = t->n;
    if (mode == ORC_MODE_UNIFORM) {
        uint32_t b = t->begin[node], e = t->end[node];
        uint32_t w = e - b;
        float u = orc_draw(rs, ORC_DRAW_UNIFORM);
        uint32_t u24 = (uint32_t)(u * 16777216.0f);
        uint32_t k = (uint32_t)(((uint64_t)u24 * (uint64_t)w) >> 24);
        *p_in = 1.0 / (double)w;
        return (int64_t)b + k;
    }
    *p_in = 1.0;
    uint32_t level = 0;
    if (mode == ORC_MODE_DESCENT2) {
        while (node < nl - 1) {
            int32_t cand[4];
            float w[4];
            int uniform;
            int k = orc_frontier(t, node, cand);
            orc_frontier_weights(t, cand, k, x, n, w, &uniform);
            float u = orc_draw(rs, ORC_DRAW_DESCENT + level);
            ++level;
            int pick = 0;
            if (uniform) {
                uint32_t u24 = (uint32_t)(u * 16777216.0f);
                pick = (int)(((uint64_t)u24 * (uint64_t)k) >> 24);
                *p_in *= 1.0 / (double)k;
            } else {
                float S = 0.0f, pre[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                for (int i = 0; i < k; ++i) {
                    S = S + w[i];
                    pre[i] = S;
                }
                pick = k - 1;
                for (int i = 0; i < k; ++i)
                    if ((double)u * (double)S < (double)pre[i]) { pick = i; break; }
                double lo = pick > 0 ? (double)pre[pick - 1] / (double)S : 0.0;
                double hi = (double)pre[pick] / (double)S;
                *margin = orc_min(*margin, orc_min(fabs((double)u - lo), fabs(hi - (double)u)));
                *p_in *= hi - lo;  /* the chosen interval of the binary32 prefix sums */
            }
            node = cand[pick];
        }
        return (int64_t)(node - (nl - 1));
    }
    while (node < nl - 1) {
        int32_t a = t->left[node], c = t->right[node];
        float wa, wc;
        orc_branch_weights(REC(t, a), REC(t, c), x, n, &wa, &wc);
        float s = wa + wc;
        float u = orc_draw(rs, ORC_DRAW_DESCENT + level);
        ++level;
        double ratio_left;
        int go_left;
        if (s > 0.0f) {
            go_left = (double)u * (double)s < (double)wa;
            ratio_left = (double)wa / ((double)wa + (double)wc);
        } else {
            go_left = u < 0.5f;
            ratio_left = 0.5;
        }
        *margin = orc_min(*margin, fabs((double)u - ratio_left));
        if (go_left) {
            *p_in *= ratio_left;
            node = a;
        } else {
            *p_in *= 1.0 - ratio_left;
            node = c;
        }
    }
    return (int64_t)(node - (nl - 1));
}

/* Light point, contribution, estimate, reward. */
static void orc_shade(const orc_scene* sc, int64_t l, const float x[3], const float n[3], float albedo,
                      orc_stream* rs, int reward_mode, orc_sample_out* o)
{
    const orc_tree* t = sc->tree;
    uint32_t li = t->perm[l];
    const float* v = sc->tri + (size_t)li * 9;
    const float* le = sc->emis + (size_t)li * 3;
    /* sample point (binary32: it decides the shadow test) */
    float ua = orc_draw(rs, ORC_DRAW_TRI_A), ub = orc_draw(rs, ORC_DRAW_TRI_B);
    float su = sqrtf(ua);
    float b0 = 1.0f - su, b1 = ub * su, b2 = su - b1;
    float y[3], org[3];
    for (int k = 0; k < 3; ++k) {
        y[k] = (b0 * v[k] + b1 * v[3 + k]) + b2 * v[6 + k];
        org[k] = x[k] + 1e-4f * n[k];
    }
    int occl = orc_occluded32(org, y, sc->nbox, sc->boxes);
    /* contribution in double */
    double e1[3], e2[3], nl[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = (double)v[3 + k] - v[k];
        e2[k] = (double)v[6 + k] - v[k];
    }
    nl[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nl[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nl[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double cl = sqrt(nl[0] * nl[0] + nl[1] * nl[1] + nl[2] * nl[2]);
    double area = 0.5 * cl;
    for (int k = 0; k < 3; ++k) nl[k] /= cl;
    double w[3] = {(double)y[0] - x[0], (double)y[1] - x[1], (double)y[2] - x[2]};
    double d2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double dist = sqrt(d2);
    for (int k = 0; k < 3; ++k) w[k] /= dist;
    double cx = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
    double cy = -(nl[0] * w[0] + nl[1] * w[1] + nl[2] * w[2]);
    if (cx < 0.0) cx = 0.0;
    if (cy < 0.0) cy = 0.0;
    double geo = occl ? 0.0 : cx * cy / d2;
    double f = (double)albedo / 3.14159265358979323846;
    double c[3] = {f * le[0] * geo, f * le[1] * geo, f * le[2] * geo};
    double pdf = o->p_cut * o->p_in / area;
    for (int k = 0; k < 3; ++k) o->est[k] = c[k] / pdf;
    o->visible = !occl;
    o->area = area;
    /* Eq. 1 reward |c|: luminance of the cluster-level estimate c / (p_in p_A)
       (reading), or of the light's own contribution c / p_A (literal). */
    double lum = orc_lum64(c[0], c[1], c[2]);
    o->reward = reward_mode == 0 ? lum * area / o->p_in : lum * area;
}

static void orc_one_sample(const orc_scene* sc, orc_grid* g, const float x[3], const float n[3],
                           float albedo, uint32_t level, uint64_t seed, uint32_t sample_id,
                           uint32_t frame, orc_sample_out* o)
{
    orc_stream rs;
    orc_stream_init(&rs, seed, sample_id, frame);
    float jit[5];
    for (int k = 0; k < 5; ++k) jit[k] = orc_draw(&rs, ORC_DRAW_JIT + (uint32_t)k);
    uint64_t key = orc_cell_key_level(g, level, x, n, jit);
    int64_t slot = orc_lookup_insert_level(g, level, key);
    const int32_t* cut = slot >= 0 ? g->cut + (size_t)slot * g->M : g->def_cut;
    const double* C = slot >= 0 ? g->C + (size_t)slot * g->M : g->def_C;
    uint32_t m = g->m;
    /* binary search over C: first s with C(s) > u * C(m-1) (Section 3.1) */
    float u = orc_draw(&rs, ORC_DRAW_CUT);
    double total = C[m - 1];
    double target = (double)u * total;
    uint32_t s = 0;
    while (s < m - 1 && !(C[s] > target)) ++s;
    double lo = s > 0 ? C[s - 1] : 0.0;
    o->slot = slot;
    o->s = (int32_t)s;
    o->p_cut = (C[s] - lo) / total;
    o->margin = orc_min(fabs(target - lo), fabs(C[s] - target)) / total;
    double p_in = 1.0;
    o->light = orc_descend(sc, (int)g->mode, cut[s], x, n, &rs, &p_in, &o->margin);
    o->p_in = p_in;
    orc_shade(sc, o->light, x, n, albedo, &rs, (int)g->reward_mode, o);
}

/* A whole pass: every point, spp samples (sample id = point * spp + j). The
 * grid is read and lazily extended; Q and C are not changed (C is rebuilt at
 * the end of the pass, Section 3). Outputs per sample and the per-point mean. */
int orc_sample_frame(const orc_tree* tree, const float* tri, const float* emis, int nbox,
                     const float* boxes, orc_grid* g, int64_t npts, const float* pos,
                     const float* nrm, const float* albedo, const float* footprint, uint64_t seed,
                     uint32_t frame, int spp, double* rgb, int64_t* out_light, int64_t* out_slot,
                     int32_t* out_s, double* out_reward, double* out_pcut, double* out_pin,
                     double* out_margin, int32_t* out_visible, int64_t first, int64_t count)
{
    orc_scene sc = {tree, tri, emis, nbox, boxes};
    if (count < 0) count = npts - first;
    for (int64_t i = first; i < first + count; ++i) {
        float x[3] = {pos[i], pos[npts + i], pos[2 * npts + i]};
        float n[3] = {nrm[i], nrm[npts + i], nrm[2 * npts + i]};
        uint32_t level = footprint ? orc_footprint_level(footprint[i], g->h, g->levels) : 0;
        double acc[3] = {0, 0, 0};
        for (int j = 0; j < spp; ++j) {
            uint32_t sid = (uint32_t)(i * spp + j);
            orc_sample_out o;
            memset(&o, 0, sizeof(o));
            orc_one_sample(&sc, g, x, n, albedo[i], level, seed, sid, frame, &o);
            for (int k = 0; k < 3; ++k) acc[k] += o.est[k];
            int64_t r = (i - first) * spp + j;
            if (out_light) out_light[r] = o.light;
            if (out_slot) out_slot[r] = o.slot;
            if (out_s) out_s[r] = o.s;
            if (out_reward) out_reward[r] = o.reward;
            if (out_pcut) out_pcut[r] = o.p_cut;
            if (out_pin) out_pin[r] = o.p_in;
            if (out_margin) out_margin[r] = o.margin;
            if (out_visible) out_visible[r] = o.visible;
        }
        for (int k = 0; k < 3; ++k) rgb[k * count + (i - first)] = acc[k] / spp;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 (Section 3): Q(s) := (1 - alpha) Q(s) + alpha |c_l|, applied to the */
/* records of a pass in sample order (reading: the paper does not fix the     */
/* order of the updates of one pass). Q is held in double during the pass and */
/* stored in the table precision when it ends; then C is rebuilt (Eq. 2) for  */
/* every touched cell.                                                       */
/* ------------------------------------------------------------------------ */
int orc_learn(orc_grid* g, int64_t nrec, const int64_t* slot, const int32_t* s, const double* reward,
              uint8_t* touched)
{
    double a = g->alpha;
    for (int64_t i = 0; i < nrec; ++i) {
        if (slot[i] < 0) continue;
        double* q = g->Q + (size_t)slot[i] * g->M + s[i];
        *q = (1.0 - a) * (*q) + a * reward[i];
        touched[slot[i]] = 1;
    }
    double* tmp = (double*)malloc(sizeof(double) * g->m);
    for (uint32_t c = 0; c < g->H; ++c) {
        if (!touched[c]) continue;
        double* q = g->Q + (size_t)c * g->M;
        for (uint32_t k = 0; k < g->m; ++k) q[k] = orc_round_storage(q[k], (int)g->precision);
        orc_cdf((int)g->m, q, g->eps, (int)g->precision, tmp);
        for (uint32_t k = 0; k < g->m; ++k) g->C[(size_t)c * g->M + k] = tmp[k];
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Split-collapse (Section 3, Fig. "TreeCuts", Section 3.1). The Q of an      */
/* internal node is the sum of the Q of the cut leaves below it. l_max is the */
/* leaf of largest Q among leaves that are not single lights; p_min the      */
/* parent of smallest Q among internal nodes whose two children are both cut  */
/* leaves (reading: collapsing any other parent would change the cut size;   */
/* with Q >= 0 a minimiser over all parents is always such a node). Ties go  */
/* to the smaller range begin. If Q(l_max) > T Q(p_min), l_max is replaced by */
/* its children and p_min's children by p_min. Decisions in binary32 on the  */
/* stored Q. New Q values (reading): l_max's Q times f = phi_a / (phi_a +    */
/* phi_c) and times 1 - f (children's stored binary32 power), p_min's Q the  */
/* sum of its children's; binary32 arithmetic like the decisions that later  */
/* read them, then rounded to the table precision.                          */
/* One step; returns 1 if the cut changed.                                  */
/* ------------------------------------------------------------------------ */
static int orc_split_collapse_step(const orc_tree* t, int m, int32_t* cut, double* q, double T, int precision)
{
    int lmax = -1;
    float qmax = 0.0f;
    for (int i = 0; i < m; ++i) {
        if (t->end[cut[i]] - t->begin[cut[i]] <= 1) continue;
        float v = (float)q[i];
        if (lmax < 0 || v > qmax) { lmax = i; qmax = v; }
    }
    int pmin = -1;
    float qmin = 0.0f;
    for (int i = 0; i + 1 < m; ++i) {
        int32_t pa = t->parent[cut[i]];
        if (pa < 0 || pa != t->parent[cut[i + 1]]) continue;
        float v = (float)q[i] + (float)q[i + 1];
        if (pmin < 0 || v < qmin) { pmin = i; qmin = v; }
    }
    if (!(lmax >= 0 && pmin >= 0 && lmax != pmin && lmax != pmin + 1 && qmax > (float)T * qmin)) return 0;
    int32_t nc[1024];
    double nq[1024];
    int k = 0;
    for (int i = 0; i < m; ++i) {
        if (i == lmax) {
            int32_t node = cut[i];
            int32_t a = t->left[node], c = t->right[node];
            float pa = REC(t, a)[6], pc = REC(t, c)[6];
            float sum = pa + pc;
            float fa = sum > 0.0f ? pa / sum : 0.5f;
            float qi = (float)q[i];
            nc[k] = a; nq[k] = (double)(qi * fa); ++k;
            nc[k] = c; nq[k] = (double)(qi * (1.0f - fa)); ++k;
        } else if (i == pmin) {
            nc[k] = t->parent[cut[i]]; nq[k] = (double)((float)q[i] + (float)q[i + 1]); ++k;
            ++i;
        } else {
            nc[k] = cut[i]; nq[k] = q[i]; ++k;
        }
    }
    for (int i = 0; i < m; ++i) {
        cut[i] = nc[i];
        q[i] = orc_round_storage(nq[i], precision);
    }
    return 1;
}

/* Split-collapse of one cell, repeated until a step changes nothing or      */
/* max_iter steps were taken (Section 3: the basic algorithm is one step;    */
/* the paper notes it may be repeated until no pair of nodes is touched).    */
/* Then Eq. 2. Returns the number of steps that changed the cut.            */
int orc_split_collapse_cell(const orc_tree* t, int m, int32_t* cut, double* q, double T, double eps,
                            int precision, int max_iter, double* c_out)
{
    int steps = 0;
    while (steps < max_iter && orc_split_collapse_step(t, m, cut, q, T, precision)) ++steps;
    orc_cdf(m, q, eps, precision, c_out);
    return steps;
}

/* ------------------------------------------------------------------------ */
/* Probability of choosing sorted light l at (x, n) from a cell's cut and C: */
/* p = p_cut(cluster containing l) * p_in(path from the cut node to l). The   */
/* sampler must return exactly this pdf (pin: "sample pdf = cut selection x  */
/* descent probability").                                                    */
/* ------------------------------------------------------------------------ */
double orc_light_pdf(const orc_tree* t, int mode, int m, const int32_t* cut, const double* C,
                     const float x[3], const float n[3], int64_t l)
{
    int64_t nl = t->n;
    int s = -1;
    for (int i = 0; i < m; ++i)
        if ((uint32_t)l >= t->begin[cut[i]] && (uint32_t)l < t->end[cut[i]]) { s = i; break; }
    if (s < 0) return 0.0;
    double lo = s > 0 ? C[s - 1] : 0.0;
    double p = (C[s] - lo) / C[m - 1];
    int32_t node = cut[s];
    if (mode == ORC_MODE_UNIFORM) return p / (double)(t->end[node] - t->begin[node]);
    if (mode == ORC_MODE_DESCENT2) {
        while (node < nl - 1) {
            int32_t cand[4];
            float w[4];
            int uniform;
            int k = orc_frontier(t, node, cand);
            orc_frontier_weights(t, cand, k, x, n, w, &uniform);
            int pick = -1;
            for (int i = 0; i < k; ++i)
                if ((uint32_t)l >= t->begin[cand[i]] && (uint32_t)l < t->end[cand[i]]) pick = i;
            if (uniform) {
                p *= 1.0 / (double)k;
            } else {
                float S = 0.0f, pre[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                for (int i = 0; i < k; ++i) {
                    S = S + w[i];
                    pre[i] = S;
                }
                double lo = pick > 0 ? (double)pre[pick - 1] / (double)S : 0.0;
                p *= (double)pre[pick] / (double)S - lo;
            }
            node = cand[pick];
        }
        return p;
    }
    while (node < nl - 1) {
        int32_t a = t->left[node], c = t->right[node];
        float wa, wc;
        orc_branch_weights(REC(t, a), REC(t, c), x, n, &wa, &wc);
        double ratio = ((double)wa + (double)wc) > 0.0 ? (double)wa / ((double)wa + (double)wc) : 0.5;
        if ((uint32_t)l < t->end[a]) { p *= ratio; node = a; }
        else { p *= 1.0 - ratio; node = c; }
    }
    return p;
}

/* ------------------------------------------------------------------------ */
/* Energy-based baseline (Section 4): lights sampled in proportion to their  */
/* emitted power by inversion of the global cdf over the sorted lights.      */
/* ------------------------------------------------------------------------ */
int orc_sample_power(const orc_tree* tree, const float* tri, const float* emis, int nbox,
                     const float* boxes, int64_t npts, const float* pos, const float* nrm,
                     const float* albedo, uint64_t seed, uint32_t frame, int spp, double* rgb,
                     int64_t* out_light, int64_t first, int64_t count)
{
    orc_scene sc = {tree, tri, emis, nbox, boxes};
    int64_t nl = tree->n;
    double* cdf = (double*)malloc(sizeof(double) * (size_t)nl);
    double acc = 0.0;
    for (int64_t l = 0; l < nl; ++l) {
        acc += tree->phi64[nl - 1 + l];
        cdf[l] = acc;
    }
    if (count < 0) count = npts - first;
    for (int64_t i = first; i < first + count; ++i) {
        float x[3] = {pos[i], pos[npts + i], pos[2 * npts + i]};
        float n[3] = {nrm[i], nrm[npts + i], nrm[2 * npts + i]};
        double sum[3] = {0, 0, 0};
        for (int j = 0; j < spp; ++j) {
            orc_stream rs;
            orc_stream_init(&rs, seed, (uint32_t)(i * spp + j), frame);
            float u = orc_draw(&rs, ORC_DRAW_CUT);
            double target = (double)u * acc;
            int64_t lo = 0, hi = nl - 1;
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (cdf[mid] > target) hi = mid; else lo = mid + 1;
            }
            orc_sample_out o;
            memset(&o, 0, sizeof(o));
            o.p_cut = tree->phi64[nl - 1 + lo] / acc;
            o.p_in = 1.0;
            orc_shade(&sc, lo, x, n, albedo[i], &rs, 0, &o);
            for (int k = 0; k < 3; ++k) sum[k] += o.est[k];
            if (out_light) out_light[(i - first) * spp + j] = lo;
        }
        for (int k = 0; k < 3; ++k) rgb[k * count + (i - first)] = sum[k] / spp;
    }
    free(cdf);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact direct lighting, the quantity every estimate above is unbiased for: */
/* L(x) = sum_i int_{tri i} (rho/pi) Le cos_x cos_l / r^2 V dA, by midpoint   */
/* quadrature on the 4^k congruent sub-triangles of each triangle, visibility */
/* in double with the same segment (x + 1e-4 n to y, t < 0.9999).            */
/* ------------------------------------------------------------------------ */
static int orc_occluded64(const double o[3], const double y[3], int nbox, const float* boxes)
{
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = y[k] - o[k];
    for (int b = 0; b < nbox; ++b) {
        const float* bx = boxes + (size_t)b * 6;
        double tn = 0.0, tf = 0.9999;
        int miss = 0;
        for (int k = 0; k < 3 && !miss; ++k) {
            if (d[k] == 0.0) {
                if (!(o[k] > bx[k] && o[k] < bx[3 + k])) miss = 1;
                continue;
            }
            double t0 = (bx[k] - o[k]) / d[k], t1 = (bx[3 + k] - o[k]) / d[k];
            if (t0 > t1) { double tmp = t0; t0 = t1; t1 = tmp; }
            if (t0 > tn) tn = t0;
            if (t1 < tf) tf = t1;
        }
        if (!miss && tn < tf) return 1;
    }
    return 0;
}

/* The two shadow tests as library entry points (tests compare them). */
int orc_shadow32(const float o[3], const float y[3], int nbox, const float* boxes)
{
    return orc_occluded32(o, y, nbox, boxes);
}
int orc_shadow64(const double o[3], const double y[3], int nbox, const float* boxes)
{
    return orc_occluded64(o, y, nbox, boxes);
}

static void orc_tri_quad(const double* a, const double* b, const double* c, int level, const double x[3],
                         const double n[3], const double nl[3], int nbox, const float* boxes,
                         int vis, double* acc)
{
    if (level == 0) {
        double y[3], e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            y[k] = (a[k] + b[k] + c[k]) / 3.0;
            e1[k] = b[k] - a[k];
            e2[k] = c[k] - a[k];
        }
        double cx = e1[1] * e2[2] - e1[2] * e2[1];
        double cy = e1[2] * e2[0] - e1[0] * e2[2];
        double cz = e1[0] * e2[1] - e1[1] * e2[0];
        double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
        double w[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
        double d2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        double dist = sqrt(d2);
        double ctx = (n[0] * w[0] + n[1] * w[1] + n[2] * w[2]) / dist;
        double ctl = -(nl[0] * w[0] + nl[1] * w[1] + nl[2] * w[2]) / dist;
        if (ctx <= 0.0 || ctl <= 0.0) return;
        if (vis) {
            double o[3] = {x[0] + 1e-4 * n[0], x[1] + 1e-4 * n[1], x[2] + 1e-4 * n[2]};
            if (orc_occluded64(o, y, nbox, boxes)) return;
        }
        *acc += ctx * ctl / d2 * area;
        return;
    }
    double ab[3], bc[3], ca[3];
    for (int k = 0; k < 3; ++k) {
        ab[k] = 0.5 * (a[k] + b[k]);
        bc[k] = 0.5 * (b[k] + c[k]);
        ca[k] = 0.5 * (c[k] + a[k]);
    }
    orc_tri_quad(a, ab, ca, level - 1, x, n, nl, nbox, boxes, vis, acc);
    orc_tri_quad(ab, b, bc, level - 1, x, n, nl, nbox, boxes, vis, acc);
    orc_tri_quad(ca, bc, c, level - 1, x, n, nl, nbox, boxes, vis, acc);
    orc_tri_quad(ab, bc, ca, level - 1, x, n, nl, nbox, boxes, vis, acc);
}

void orc_direct_bruteforce(const float x32[3], const float n32[3], float albedo, int64_t ntri,
                           const float* tri, const float* emis, int nbox, const float* boxes,
                           int level, double rgb[3])
{
    double x[3] = {x32[0], x32[1], x32[2]}, n[3] = {n32[0], n32[1], n32[2]};
    rgb[0] = rgb[1] = rgb[2] = 0.0;
    for (int64_t i = 0; i < ntri; ++i) {
        const float* v = tri + (size_t)i * 9;
        double a[3] = {v[0], v[1], v[2]}, b[3] = {v[3], v[4], v[5]}, c[3] = {v[6], v[7], v[8]};
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double nl[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
        double len = sqrt(nl[0] * nl[0] + nl[1] * nl[1] + nl[2] * nl[2]);
        for (int k = 0; k < 3; ++k) nl[k] /= len;
        double acc = 0.0;
        orc_tri_quad(a, b, c, level, x, n, nl, nbox, boxes, nbox > 0, &acc);
        for (int k = 0; k < 3; ++k) rgb[k] += emis[i * 3 + k] * acc;
    }
    double f = (double)albedo / 3.14159265358979323846;
    for (int k = 0; k < 3; ++k) rgb[k] *= f;
}

/* ------------------------------------------------------------------------ */
/* Path vertices of one diffuse bounce and their footprints (Section 3, first */
/* ingredient: cells sized from the ray footprint of each path vertex,       */
/* derived from its area pdf). Reading: from each shading point x with unit   */
/* normal n, one cosine-weighted direction (Malley: a uniform point (a, b) of */
/* the unit disk lifted to the hemisphere) is traced to the nearest face of   */
/* an occluder box or of the room's inside; the vertex y gets the footprint  */
/* f = (N_t p_A)^(-1/2), p_A = cos(theta_x) cos(theta_y) / (pi d^2) the area   */
/* density of y for one path, shared by the N_t paths that leave one tile.   */
/* The disk point comes from rejection: draws 2k, 2k + 1 of the point's      */
/* stream (Philox counter = (point, frame, draw / 4, 1)) give a = 2u - 1,    */
/* b = 2u' - 1, accepted at the first k < 16 with a^2 + b^2 < 1 (else a = b =  */
/* 0). Everything is binary32 with one correctly rounded operation per step  */
/* (the hit face is a decision). Only surfaces ahead (t > 1e-6) count; a ray */
/* from outside the room may find none and escapes: y = x + 1e-4 n, normal   */
/* 0 and footprint +inf (the coarsest level).                                */
/* ------------------------------------------------------------------------ */
#define ORC_BOUNCE_TRIES 16
#define ORC_BOUNCE_OFFSET 1e-4f
#define ORC_BOUNCE_TMIN 1e-6f
#define ORC_PI_F 3.14159265358979323846f

static void orc_bounce_one(const float x[3], const float n[3], int nbox, const float* boxes, const float room[6],
                           uint64_t seed, uint32_t point, uint32_t frame, float paths_per_tile, float y[3],
                           float ny[3], float* footprint)
{
    /* the disk point */
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {point, frame, 0, 1}, w[4];
    float a = 0.0f, b = 0.0f;
    for (int k = 0; k < ORC_BOUNCE_TRIES; ++k) {
        if ((k & 1) == 0) {  /* draws 2k .. 2k + 3 are the words of block k / 2 */
            ctr[2] = (uint32_t)(k >> 1);
            orc_philox4x32_10(ctr, key, w);
        }
        float ua = orc_u24(w[(2 * k) & 3]), ub = orc_u24(w[(2 * k + 1) & 3]);
        float ta = 2.0f * ua - 1.0f, tb = 2.0f * ub - 1.0f;
        if (ta * ta + tb * tb < 1.0f) {
            a = ta;
            b = tb;
            break;
        }
    }
    float s = a * a + b * b;
    float c = sqrtf(fmaxf(0.0f, 1.0f - s));               /* cos(theta_x) */

    /* tangent frame of n: u = normalise(n x t), v = n x u */
    float t0 = fabsf(n[0]) < 0.9f ? 1.0f : 0.0f, t2 = fabsf(n[0]) < 0.9f ? 0.0f : 1.0f;
    float u[3] = {n[1] * t2 - n[2] * 0.0f, n[2] * t0 - n[0] * t2, n[0] * 0.0f - n[1] * t0};
    float ul = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int k = 0; k < 3; ++k) u[k] = u[k] / ul;
    float v[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};

    float d[3], o[3], inv[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = (a * u[k] + b * v[k]) + c * n[k];
        o[k] = x[k] + ORC_BOUNCE_OFFSET * n[k];
        inv[k] = 1.0f / d[k];
    }

    /* leave the room through the first wall ahead (a point outside the room may have none) */
    float t_best = INFINITY;
    int axis = 0;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0f) continue;
        float wall = d[k] > 0.0f ? room[3 + k] : room[k];
        float t = (wall - o[k]) * inv[k];
        if (t > ORC_BOUNCE_TMIN && t < t_best) {
            t_best = t;
            axis = k;
        }
    }
    /* the nearest box face in front of it */
    for (int i = 0; i < nbox; ++i) {
        const float* bx = boxes + (size_t)i * 6;
        float tn = -INFINITY, tf = INFINITY;
        int ax = 0, miss = 0;
        for (int k = 0; k < 3; ++k) {
            if (d[k] == 0.0f) {  /* parallel to this slab: inside it or a miss */
                if (!(o[k] > bx[k] && o[k] < bx[3 + k])) miss = 1;
                continue;
            }
            float ta = (bx[k] - o[k]) * inv[k];
            float tb = (bx[3 + k] - o[k]) * inv[k];
            float lo = fminf(ta, tb), hi = fmaxf(ta, tb);
            if (lo > tn) {
                tn = lo;
                ax = k;
            }
            tf = fminf(tf, hi);
        }
        if (!miss && tn < tf && tn > ORC_BOUNCE_TMIN && tn < t_best) {
            t_best = tn;
            axis = ax;
        }
    }
    if (t_best == INFINITY) {  /* nothing ahead: the path escapes, no vertex */
        for (int k = 0; k < 3; ++k) {
            y[k] = o[k];
            ny[k] = 0.0f;
        }
        *footprint = INFINITY;
        return;
    }
    for (int k = 0; k < 3; ++k) {
        y[k] = o[k] + t_best * d[k];
        ny[k] = 0.0f;
    }
    ny[axis] = d[axis] > 0.0f ? -1.0f : 1.0f;               /* the face turned toward x */
    float cy = fabsf(d[axis]);                               /* cos(theta_y) */
    float q = (paths_per_tile * fmaxf(c, 1e-6f)) * fmaxf(cy, 1e-6f);
    *footprint = t_best * sqrtf(ORC_PI_F / q);               /* d sqrt(pi / (N_t cx cy)) */
}

/* Bounce vertices of P points: pos, nrm SoA [3][P] in, y, ny SoA [3][P] and
 * footprint [P] out; room [6] = min xyz, max xyz. */
void orc_bounce_vertices(int64_t npts, const float* pos, const float* nrm, int nbox, const float* boxes,
                         const float room[6], uint64_t seed, uint32_t frame, float paths_per_tile, float* y_out,
                         float* ny_out, float* fp_out)
{
    for (int64_t p = 0; p < npts; ++p) {
        float x[3] = {pos[p], pos[npts + p], pos[2 * npts + p]};
        float n[3] = {nrm[p], nrm[npts + p], nrm[2 * npts + p]};
        float y[3], ny[3], f;
        orc_bounce_one(x, n, nbox, boxes, room, seed, (uint32_t)p, frame, paths_per_tile, y, ny, &f);
        for (int k = 0; k < 3; ++k) {
            y_out[k * npts + p] = y[k];
            ny_out[k * npts + p] = ny[k];
        }
        fp_out[p] = f;
    }
}
