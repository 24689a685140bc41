/*
 * CPU oracle for exact DDM region matching.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library, and the CUDA library does not depend on it.
 *
 * What it computes (paper Section 3, "The Region Matching Problem"): given
 * subscription extents S_1..S_n and update extents U_1..U_m, d-dimensional
 * axis-parallel rectangles with closed sides, the list of all (i, j) with
 * S_i and U_j intersecting.  Ids are 0-based; the list is returned sorted
 * lexicographically by (i, j).
 *
 * Two independent routes to that list:
 *   oracle_bruteforce  Algorithm 2 (Brute-Force matching) extended to d
 *                      dimensions by the "logical and" of Section 3: every
 *                      pair is tested with Algorithm 1 in every dimension.
 *   oracle_sbm         Algorithm 4 (Sort-Based Matching) on dimension 0, the
 *                      other dimensions filtered per reported pair (Section 3,
 *                      d-dimensional reduction).
 *
 * Readings of points the paper leaves open (each is stated again where used):
 *   R1  "Sort T in non-decreasing order" does not say how equal coordinates
 *       are ordered.  Algorithm 1 treats intervals as closed, so two extents
 *       that only touch must be reported; the sweep does so only if, at equal
 *       coordinates, every lower endpoint comes before every upper endpoint.
 *       Further ties are broken by (subscription before update, then id),
 *       which makes the order total; it does not change the reported set.
 *   R2  Coordinates compare as IEEE-754 float32 values: -0 equals +0, +-inf
 *       are ordinary values.  NaN, or lo > hi in any dimension, is rejected.
 *   R3  The d > 1 filter applies Algorithm 1 to dimensions 1..d-1 of every
 *       pair the dimension-0 sweep reports.
 *
 * Return values: K >= 0 on success; ORACLE_EINVAL for invalid input;
 * ORACLE_ENOMEM when memory runs out.  Arrays are dimension-major:
 * sub_lo[k * n + i] is the lower bound of S_i along dimension k.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* ------------------------------------------------------------------------ */
/* Algorithm 1, Intersect-1D: closed intervals x and y overlap iff          */
/* x.low <= y.high and y.low <= x.high.                                     */
/* ------------------------------------------------------------------------ */
static int intersect_1d(float x_low, float x_high, float y_low, float y_high)
{
#if ORACLE_MUTANT == 3
    return x_low < y_high && y_low < x_high;           /* planted: open intervals */
#else
    return x_low <= y_high && y_low <= x_high;
#endif
}

/* Section 3: two d-rectangles overlap iff all their projections overlap.
 * Checks dimensions k0..d-1 of (S_i, U_j). */
static int intersect_dims(int k0, int d, int64_t n, int64_t m,
                          const float *sub_lo, const float *sub_hi,
                          const float *upd_lo, const float *upd_hi,
                          int64_t i, int64_t j)
{
#if ORACLE_MUTANT == 2
    d = d - 1;                                          /* planted: last dimension dropped */
#endif
    for (int k = k0; k < d; ++k) {
        if (!intersect_1d(sub_lo[k * n + i], sub_hi[k * n + i],
                          upd_lo[k * m + j], upd_hi[k * m + j]))
            return 0;
    }
    return 1;
}

/* R2: reject NaN and lo > hi (written so that a NaN fails the test). */
static int valid_extents(int d, int64_t count, const float *lo, const float *hi)
{
    for (int64_t e = 0; e < (int64_t)d * count; ++e)
        if (!(lo[e] <= hi[e]))
            return 0;
    return 1;
}

static int valid_input(int d, int64_t n, int64_t m, const float *sub_lo,
                       const float *sub_hi, const float *upd_lo, const float *upd_hi)
{
    if (d < 1 || n < 0 || m < 0)
        return 0;
    return valid_extents(d, n, sub_lo, sub_hi) && valid_extents(d, m, upd_lo, upd_hi);
}

/* ------------------------------------------------------------------------ */
/* The result list L: a growable array of (i, j) int32 pairs.               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t *pairs;   /* 2 * cap ints, or NULL when only counting */
    int64_t len, cap;
    int store, failed;
} pair_list;

static void list_add(pair_list *L, int64_t i, int64_t j)
{
    if (L->store) {
        if (L->len == L->cap) {
            int64_t cap = L->cap ? 2 * L->cap : 1024;
            int32_t *p = (int32_t *)realloc(L->pairs, (size_t)cap * 2 * sizeof(int32_t));
            if (!p) { L->failed = 1; return; }
            L->pairs = p;
            L->cap = cap;
        }
        L->pairs[2 * L->len] = (int32_t)i;
        L->pairs[2 * L->len + 1] = (int32_t)j;
    }
    L->len++;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Sort the list lexicographically: bucket by subscription id (counting sort),
 * then sort every bucket's update ids with qsort. */
static int sort_pairs(pair_list *L, int64_t n)
{
    if (!L->store || L->len == 0)
        return 0;
    int64_t *start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *upd = (int32_t *)malloc((size_t)L->len * sizeof(int32_t));
    if (!start || !upd) { free(start); free(upd); return ORACLE_ENOMEM; }
    for (int64_t k = 0; k < L->len; ++k)
        start[L->pairs[2 * k] + 1]++;
    for (int64_t i = 0; i < n; ++i)
        start[i + 1] += start[i];
    int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!fill) { free(start); free(upd); return ORACLE_ENOMEM; }
    memcpy(fill, start, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t k = 0; k < L->len; ++k)
        upd[fill[L->pairs[2 * k]]++] = L->pairs[2 * k + 1];
    for (int64_t i = 0; i < n; ++i) {
        int64_t a = start[i], b = start[i + 1];
        qsort(upd + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
        for (int64_t k = a; k < b; ++k) {
            L->pairs[2 * k] = (int32_t)i;
            L->pairs[2 * k + 1] = upd[k];
        }
    }
    free(fill);
    free(start);
    free(upd);
    return 0;
}

static int64_t finish(pair_list *L, int64_t n, int32_t **pairs_out)
{
    if (L->failed) { free(L->pairs); return ORACLE_ENOMEM; }
    int rc = sort_pairs(L, n);
    if (rc) { free(L->pairs); return rc; }
    if (pairs_out)
        *pairs_out = L->pairs;
    else
        free(L->pairs);
    return L->len;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, BruteForce: test every (S_i, U_j) pair, in every dimension. */
/* ------------------------------------------------------------------------ */
int64_t oracle_bruteforce(int d, int64_t n, int64_t m,
                          const float *sub_lo, const float *sub_hi,
                          const float *upd_lo, const float *upd_hi,
                          int32_t **pairs_out)
{
    if (!valid_input(d, n, m, sub_lo, sub_hi, upd_lo, upd_hi))
        return ORACLE_EINVAL;
    pair_list L = {0};
    L.store = pairs_out != NULL;
#if ORACLE_MUTANT == 5
    int64_t m_loop = m > 0 ? m - 1 : 0;                 /* planted: last update skipped */
#else
    int64_t m_loop = m;
#endif
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m_loop; ++j)
            if (intersect_dims(0, d, n, m, sub_lo, sub_hi, upd_lo, upd_hi, i, j))
                list_add(&L, i, j);
    return finish(&L, n, pairs_out);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 4, Sort-Based Matching, on dimension 0.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    float x;          /* coordinate of the endpoint along dimension 0 */
    uint8_t upper;    /* 0: lower bound, 1: upper bound */
    uint8_t update;   /* 0: belongs to a subscription, 1: to an update */
    int32_t id;       /* 0-based index of the owning extent */
} endpoint;

/* Non-decreasing coordinate; at equal coordinates lowers first (R1), then
 * subscriptions first, then by id. */
static int cmp_endpoint(const void *pa, const void *pb)
{
    const endpoint *a = (const endpoint *)pa, *b = (const endpoint *)pb;
    if (a->x < b->x) return -1;
    if (b->x < a->x) return 1;
#if ORACLE_MUTANT == 1
    /* planted: uppers of other extents first (an extent's own lower still first) */
    if (a->upper != b->upper && (a->update != b->update || a->id != b->id))
        return a->upper ? -1 : 1;
    if (a->upper != b->upper) return a->upper ? 1 : -1;
#else
    if (a->upper != b->upper) return a->upper ? 1 : -1;
#endif
    if (a->update != b->update) return a->update ? 1 : -1;
    return (a->id > b->id) - (a->id < b->id);
}

/* An active set (SubSet or UpdSet): members in a dense array, plus the slot
 * of each id, so that insertion and deletion take O(1). */
typedef struct {
    int32_t *member;
    int64_t *slot;
    int64_t size;
} active_set;

static int set_init(active_set *s, int64_t universe)
{
    s->member = (int32_t *)malloc((size_t)(universe > 0 ? universe : 1) * sizeof(int32_t));
    s->slot = (int64_t *)malloc((size_t)(universe > 0 ? universe : 1) * sizeof(int64_t));
    s->size = 0;
    return s->member && s->slot;
}

static void set_free(active_set *s) { free(s->member); free(s->slot); }

static void set_insert(active_set *s, int32_t id)
{
    s->slot[id] = s->size;
    s->member[s->size++] = id;
}

static void set_remove(active_set *s, int32_t id)
{
    int64_t k = s->slot[id];
    int32_t last = s->member[--s->size];
    s->member[k] = last;
    s->slot[last] = k;
}

/* Build T (every extent contributes its lower and upper endpoint along
 * dimension 0) and sort it.  Returns NULL when memory runs out. */
static endpoint *sorted_endpoints(int64_t n, int64_t m, const float *sub_lo,
                                  const float *sub_hi, const float *upd_lo,
                                  const float *upd_hi)
{
    int64_t E = 2 * (n + m);
    endpoint *T = (endpoint *)malloc((size_t)(E > 0 ? E : 1) * sizeof(endpoint));
    if (!T)
        return NULL;
    int64_t t = 0;
    for (int64_t i = 0; i < n; ++i) {
        T[t++] = (endpoint){sub_lo[i], 0, 0, (int32_t)i};
        T[t++] = (endpoint){sub_hi[i], 1, 0, (int32_t)i};
    }
    for (int64_t j = 0; j < m; ++j) {
        T[t++] = (endpoint){upd_lo[j], 0, 1, (int32_t)j};
        T[t++] = (endpoint){upd_hi[j], 1, 1, (int32_t)j};
    }
    qsort(T, (size_t)E, sizeof(endpoint), cmp_endpoint);
    return T;
}

int64_t oracle_sbm(int d, int64_t n, int64_t m,
                   const float *sub_lo, const float *sub_hi,
                   const float *upd_lo, const float *upd_hi,
                   int32_t **pairs_out)
{
    if (!valid_input(d, n, m, sub_lo, sub_hi, upd_lo, upd_hi))
        return ORACLE_EINVAL;
    endpoint *T = sorted_endpoints(n, m, sub_lo, sub_hi, upd_lo, upd_hi);
    active_set SubSet, UpdSet;
    int ok_s = set_init(&SubSet, n), ok_u = set_init(&UpdSet, m);
    if (!T || !ok_s || !ok_u) {
        free(T); set_free(&SubSet); set_free(&UpdSet);
        return ORACLE_ENOMEM;
    }
    pair_list L = {0};
    L.store = pairs_out != NULL;
    int64_t E = 2 * (n + m);
    for (int64_t t = 0; t < E; ++t) {
        const endpoint *p = &T[t];
        if (!p->update) {                               /* endpoint of S_i */
            if (!p->upper) {
                set_insert(&SubSet, p->id);
            } else {
                set_remove(&SubSet, p->id);
                for (int64_t k = 0; k < UpdSet.size; ++k)
                    if (intersect_dims(1, d, n, m, sub_lo, sub_hi, upd_lo, upd_hi,
                                       p->id, UpdSet.member[k]))
                        list_add(&L, p->id, UpdSet.member[k]);
            }
        } else {                                        /* endpoint of U_j */
            if (!p->upper) {
                set_insert(&UpdSet, p->id);
            } else {
                set_remove(&UpdSet, p->id);
                for (int64_t k = 0; k < SubSet.size; ++k) {
#if ORACLE_MUTANT == 4
                    int64_t i = p->id, j = SubSet.member[k];   /* planted: operands swapped */
                    if (i >= n || j >= m) continue;
#else
                    int64_t i = SubSet.member[k], j = p->id;
#endif
                    if (intersect_dims(1, d, n, m, sub_lo, sub_hi, upd_lo, upd_hi, i, j))
                        list_add(&L, i, j);
                }
            }
        }
    }
    free(T);
    set_free(&SubSet);
    set_free(&UpdSet);
    return finish(&L, n, pairs_out);
}

/* ------------------------------------------------------------------------ */
/* The sweep of Algorithm 4 made visible, for checking the stages of a      */
/* parallel implementation: the sorted order of T (kind: 0 S lower, 1 U     */
/* lower, 2 S upper, 3 U upper; id) and |SubSet|, |UpdSet| right after each */
/* endpoint is processed.  Dimension 0 only.  Returns 0 or an error code.   */
/* ------------------------------------------------------------------------ */
int64_t oracle_sweep_trace(int64_t n, int64_t m, const float *sub_lo,
                           const float *sub_hi, const float *upd_lo,
                           const float *upd_hi, uint8_t *kind_out, int32_t *id_out,
                           int64_t *subset_size, int64_t *updset_size)
{
    if (!valid_input(1, n, m, sub_lo, sub_hi, upd_lo, upd_hi))
        return ORACLE_EINVAL;
    endpoint *T = sorted_endpoints(n, m, sub_lo, sub_hi, upd_lo, upd_hi);
    if (!T)
        return ORACLE_ENOMEM;
    int64_t subs = 0, upds = 0;
    for (int64_t t = 0; t < 2 * (n + m); ++t) {
        const endpoint *p = &T[t];
        kind_out[t] = (uint8_t)(p->upper * 2 + p->update);
        id_out[t] = p->id;
        if (p->update)
            upds += p->upper ? -1 : 1;
        else
            subs += p->upper ? -1 : 1;
        subset_size[t] = subs;
        updset_size[t] = upds;
    }
    free(T);
    return 0;
}

void oracle_free(void *p) { free(p); }
