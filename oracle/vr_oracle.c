/*
 * vr_oracle.c -- plain, slow, obviously-correct CPU oracle for Vietoris-Rips
 * persistence barcodes over Z/2.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package smoke check and the CPU
 * baseline of the benchmark do.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * Every distance is handled as a double.  When the input distances come from
 * the single-precision formula (or_distances_f32) every value is an exact
 * float, so every comparison below is the same comparison the float path
 * makes; the double type only lets the same code also serve a float64
 * finite-difference oracle.
 *
 * What is computed, and where the dissertation (arXiv 2502.05063) defines it:
 *
 *   or_distances_f32   d(i,j) = sqrt(sum_k (x_ik - x_jk)^2), k ascending, one
 *                      rounding per operation (compile with -ffp-contract=off),
 *                      the distance matrix D of Sec. 5.1 (Def 5.1.1).
 *   or_enclosing_radius R = min_x max_y d(x,y), Sec. 5.2.12.
 *   or_plain           the definition: every simplex of dimension <= dmax+1
 *                      with diam <= threshold (eq. 5.3), ordered by the
 *                      simplex-wise refinement of Sec. 5.1.4 (diam asc, dim
 *                      asc, combinatorial index desc; index by eq. 5.6), the
 *                      Z/2 boundary matrix (Def 2.6.7), reduced by the
 *                      standard algorithm (Algorithm 2); pivots (low(j), j)
 *                      are the persistence pairs (Thm 3.2.20), zero columns
 *                      that are never a low are essential classes.
 *   or_reduce_explicit the bare Algorithm 2 on a caller-given sparse matrix
 *                      (for the worked example of Figs 4.1/4.2).
 *   or_cohom           the dual reduction of Sec. 5.2.4 (Prop 4.3.5): the
 *                      implicit coboundary matrix (Sec. 5.2.8) with columns in
 *                      reverse filtration order (Sec. 5.2.1), each column
 *                      reduced by the oblivious column reduction of
 *                      Algorithm 12, clearing (Sec. 5.2.3) behind a flag.
 *   or_apparent        apparent pairs straight from Def 5.3.4 (youngest facet
 *                      of the oldest cofacet), no lemma used.
 *   or_critical_edge   the edge of a simplex that attains its diameter; ties
 *                      go to the largest edge index C(u,2)+v (the paper is
 *                      silent; this is the reading used throughout).
 *
 * Pins that hold this file to the paper live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXV 10 /* vertices per simplex: dmax + 2 <= OR_MAXV */

typedef struct {
    int32_t dim;       /* homology dimension p of the class                  */
    int32_t pad;
    double birth;      /* diam of the birth simplex                          */
    double death;      /* diam of the death simplex, INFINITY if essential   */
    int64_t birth_cidx; /* combinatorial index of the birth p-simplex        */
    int64_t death_cidx; /* combinatorial index of the (p+1)-simplex, or -1   */
} or_pair;

void or_free(void *p) { free(p); }

/* ------------------------------------------------------------------ */
/* distances                                                           */
/* ------------------------------------------------------------------ */

/* Condensed lower triangle: entry (i,j), i>j, at i(i-1)/2 + j. */
static inline double dist(const double *D, int64_t i, int64_t j) {
    if (i == j) return 0.0;
    if (i < j) { int64_t t = i; i = j; j = t; }
    return D[i * (i - 1) / 2 + j];
}

void or_distances_f32(const float *pts, int64_t n, int32_t ambient, float *out) {
    for (int64_t i = 1; i < n; ++i)
        for (int64_t j = 0; j < i; ++j) {
            float acc = 0.0f;
            for (int32_t k = 0; k < ambient; ++k) {
                float diff = pts[i * ambient + k] - pts[j * ambient + k];
                float sq = diff * diff;
                acc = acc + sq;
            }
            out[i * (i - 1) / 2 + j] = sqrtf(acc);
        }
}

void or_distances_f64(const double *pts, int64_t n, int32_t ambient, double *out) {
    for (int64_t i = 1; i < n; ++i)
        for (int64_t j = 0; j < i; ++j) {
            double acc = 0.0;
            for (int32_t k = 0; k < ambient; ++k) {
                double diff = pts[i * ambient + k] - pts[j * ambient + k];
                acc = acc + diff * diff;
            }
            out[i * (i - 1) / 2 + j] = sqrt(acc);
        }
}

double or_enclosing_radius(const double *D, int64_t n) {
    double R = INFINITY;
    for (int64_t x = 0; x < n; ++x) {
        double m = 0.0;
        for (int64_t y = 0; y < n; ++y)
            if (y != x && dist(D, x, y) > m) m = dist(D, x, y);
        if (m < R) R = m;
    }
    return n > 0 ? R : 0.0;
}

/* ------------------------------------------------------------------ */
/* combinatorial number system, eq. 5.6                                */
/* ------------------------------------------------------------------ */

typedef struct { int64_t n; int K; uint64_t *t; } binom_t;

static int binom_init(binom_t *b, int64_t n, int K) {
    b->n = n; b->K = K;
    b->t = (uint64_t *)calloc((size_t)(n + 1) * (K + 1), sizeof(uint64_t));
    if (!b->t) return -1;
    for (int64_t v = 0; v <= n; ++v) {
        b->t[v * (K + 1)] = 1;
        for (int k = 1; k <= K; ++k) {
            if (v == 0) { b->t[k] = 0; continue; }
            uint64_t a = b->t[(v - 1) * (K + 1) + k - 1], c = b->t[(v - 1) * (K + 1) + k];
            b->t[v * (K + 1) + k] = (a > UINT64_MAX - c) ? UINT64_MAX : a + c;
        }
    }
    return 0;
}
static inline uint64_t C(const binom_t *b, int64_t v, int k) {
    if (k < 0 || v < 0) return 0;
    return b->t[v * (b->K + 1) + k];
}

/* vertices ascending v[0] < ... < v[q]:  cidx = sum_i C(v[i], i+1). */
static uint64_t cidx_of(const binom_t *b, const int32_t *v, int q) {
    uint64_t c = 0;
    for (int i = 0; i <= q; ++i) c += C(b, v[i], i + 1);
    return c;
}

/* inverse of cidx_of: peel the largest vertex first. */
static void vertices_of(const binom_t *b, uint64_t c, int q, int64_t n, int32_t *v) {
    int64_t top = n - 1;
    for (int i = q; i >= 0; --i) {
        int64_t x = top;
        while (C(b, x, i + 1) > c) --x;
        v[i] = (int32_t)x;
        c -= C(b, x, i + 1);
        top = x - 1;
    }
}

static double diam_of(const double *D, const int32_t *v, int q) {
    double m = 0.0;
    for (int i = 0; i <= q; ++i)
        for (int j = 0; j < i; ++j)
            if (dist(D, v[i], v[j]) > m) m = dist(D, v[i], v[j]);
    return m;
}

/* ------------------------------------------------------------------ */
/* growable arrays and a uint64 hash map                              */
/* ------------------------------------------------------------------ */

typedef struct { or_pair *a; int64_t n, cap; } pairvec;
static int pv_push(pairvec *pv, or_pair p) {
    if (pv->n == pv->cap) {
        int64_t nc = pv->cap ? pv->cap * 2 : 256;
        or_pair *na = (or_pair *)realloc(pv->a, nc * sizeof(or_pair));
        if (!na) return -1;
        pv->a = na; pv->cap = nc;
    }
    pv->a[pv->n++] = p;
    return 0;
}

typedef struct { uint64_t *k, *v; int64_t cap, n; } hmap;
#define HM_EMPTY UINT64_MAX
static inline uint64_t hm_hash(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33; return x;
}
static int hm_init(hmap *h, int64_t cap) {
    h->cap = 16; while (h->cap < cap) h->cap *= 2;
    h->n = 0;
    h->k = (uint64_t *)malloc(h->cap * sizeof(uint64_t));
    h->v = (uint64_t *)malloc(h->cap * sizeof(uint64_t));
    if (!h->k || !h->v) return -1;
    for (int64_t i = 0; i < h->cap; ++i) h->k[i] = HM_EMPTY;
    return 0;
}
static void hm_free(hmap *h) { free(h->k); free(h->v); }
static int hm_get(const hmap *h, uint64_t key, uint64_t *val) {
    int64_t i = (int64_t)(hm_hash(key) & (uint64_t)(h->cap - 1));
    while (h->k[i] != HM_EMPTY) {
        if (h->k[i] == key) { if (val) *val = h->v[i]; return 1; }
        i = (i + 1) & (h->cap - 1);
    }
    return 0;
}
static int hm_put(hmap *h, uint64_t key, uint64_t val);
static int hm_grow(hmap *h) {
    hmap g;
    if (hm_init(&g, h->cap * 2)) return -1;
    for (int64_t i = 0; i < h->cap; ++i)
        if (h->k[i] != HM_EMPTY) hm_put(&g, h->k[i], h->v[i]);
    hm_free(h);
    *h = g;
    return 0;
}
static int hm_put(hmap *h, uint64_t key, uint64_t val) {
    if (2 * (h->n + 1) > h->cap && hm_grow(h)) return -1;
    int64_t i = (int64_t)(hm_hash(key) & (uint64_t)(h->cap - 1));
    while (h->k[i] != HM_EMPTY && h->k[i] != key) i = (i + 1) & (h->cap - 1);
    if (h->k[i] == HM_EMPTY) h->n++;
    h->k[i] = key; h->v[i] = val;
    return 0;
}

/* ------------------------------------------------------------------ */
/* the Rips complex: all simplices up to dimension top, diam <= thr    */
/* (eq. 5.3), generated as cliques of the thr-graph                    */
/* ------------------------------------------------------------------ */

typedef struct {
    double diam;
    int32_t dim;
    int32_t v[OR_MAXV]; /* ascending */
    uint64_t cidx;
} simp;

typedef struct { simp *a; int64_t n, cap; } simpvec;
static int sv_push(simpvec *s, const simp *x) {
    if (s->n == s->cap) {
        int64_t nc = s->cap ? s->cap * 2 : 1024;
        simp *na = (simp *)realloc(s->a, nc * sizeof(simp));
        if (!na) return -1;
        s->a = na; s->cap = nc;
    }
    s->a[s->n++] = *x;
    return 0;
}

/* level[q] for q = 0..top; returns 0 on success */
static int build_levels(const double *D, int64_t n, int top, double thr,
                        const binom_t *b, simpvec *level) {
    for (int q = 0; q <= top; ++q) level[q].a = NULL, level[q].n = level[q].cap = 0;
    if (!(0.0 <= thr)) return 0;
    for (int64_t i = 0; i < n; ++i) {
        simp s; memset(&s, 0, sizeof s);
        s.diam = 0.0; s.dim = 0; s.v[0] = (int32_t)i; s.cidx = (uint64_t)i;
        if (sv_push(&level[0], &s)) return -1;
    }
    for (int q = 0; q < top; ++q) {
        for (int64_t a = 0; a < level[q].n; ++a) {
            simp s = level[q].a[a];
            for (int64_t w = s.v[q] + 1; w < n; ++w) {
                double m = s.diam;
                int ok = 1;
                for (int i = 0; i <= q; ++i) {
                    double d = dist(D, w, s.v[i]);
                    if (d > thr) { ok = 0; break; }
                    if (d > m) m = d;
                }
                if (!ok) continue;
                simp t = s;
                t.dim = q + 1; t.v[q + 1] = (int32_t)w; t.diam = m;
                t.cidx = cidx_of(b, t.v, q + 1);
                if (sv_push(&level[q + 1], &t)) return -1;
            }
        }
    }
    return 0;
}

/* simplex-wise refinement order of Sec. 5.1.4 */
static int filt_cmp(const void *pa, const void *pb) {
    const simp *a = (const simp *)pa, *b = (const simp *)pb;
    if (a->diam != b->diam) return a->diam < b->diam ? -1 : 1;
    if (a->dim != b->dim) return a->dim < b->dim ? -1 : 1;
    if (a->cidx != b->cidx) return a->cidx > b->cidx ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 on sparse Z/2 columns (sorted ascending row lists)      */
/* ------------------------------------------------------------------ */

typedef struct { int64_t *r; int64_t n, cap; } col;

static int col_xor(col *a, const col *b) { /* a <- a + b over Z/2 */
    int64_t *out = (int64_t *)malloc((size_t)(a->n + b->n + 1) * sizeof(int64_t));
    if (!out) return -1;
    int64_t i = 0, j = 0, k = 0;
    while (i < a->n && j < b->n) {
        if (a->r[i] < b->r[j]) out[k++] = a->r[i++];
        else if (a->r[i] > b->r[j]) out[k++] = b->r[j++];
        else { ++i; ++j; } /* 1 + 1 = 0 */
    }
    while (i < a->n) out[k++] = a->r[i++];
    while (j < b->n) out[k++] = b->r[j++];
    free(a->r);
    a->r = out; a->n = k; a->cap = a->n + b->n + 1;
    return 0;
}

/* cols[0..N-1]; L[row] <- column whose low is row, or -1 (Algorithm 2). */
static int reduce_std(col *cols, int64_t N, int64_t *L) {
    for (int64_t r = 0; r < N; ++r) L[r] = -1;
    for (int64_t j = 0; j < N; ++j) {
        while (cols[j].n > 0 && L[cols[j].r[cols[j].n - 1]] != -1)
            if (col_xor(&cols[j], &cols[L[cols[j].r[cols[j].n - 1]]])) return -1;
        if (cols[j].n > 0) L[cols[j].r[cols[j].n - 1]] = j;
    }
    return 0;
}

/* Bare Algorithm 2 on an explicit matrix given in CSC form (row lists
 * sorted ascending).  Writes low[j] (-1 for zero columns).               */
int64_t or_reduce_explicit(int64_t N, const int64_t *colptr, const int64_t *rows, int64_t *low) {
    col *cols = (col *)calloc((size_t)N, sizeof(col));
    int64_t *L = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    if (!cols || !L) return -1;
    for (int64_t j = 0; j < N; ++j) {
        int64_t m = colptr[j + 1] - colptr[j];
        cols[j].r = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
        memcpy(cols[j].r, rows + colptr[j], (size_t)m * sizeof(int64_t));
        cols[j].n = m; cols[j].cap = m + 1;
    }
    int rc = reduce_std(cols, N, L);
    for (int64_t j = 0; j < N; ++j) {
        low[j] = cols[j].n ? cols[j].r[cols[j].n - 1] : -1;
        free(cols[j].r);
    }
    free(cols); free(L);
    return rc ? -1 : 0;
}

typedef struct { uint64_t cidx; int64_t pos; } cpos;
static int cpos_cmp(const void *pa, const void *pb) {
    const cpos *a = (const cpos *)pa, *b = (const cpos *)pb;
    return a->cidx < b->cidx ? -1 : (a->cidx > b->cidx ? 1 : 0);
}
static int64_t cpos_find(const cpos *arr, int64_t m, uint64_t c) {
    int64_t lo = 0, hi = m - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (arr[mid].cidx == c) return arr[mid].pos;
        if (arr[mid].cidx < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* The definition (Algorithm 2 on the full boundary matrix).
 * Returns the number of pairs written to *out (caller frees with or_free),
 * or a negative value on error.  Pairs of every length are returned,
 * including zero-length ones; essential classes have death = INFINITY.   */
int64_t or_plain(const double *D, int64_t n, int32_t dmax, double thr, or_pair **out) {
    *out = NULL;
    if (n < 0 || dmax < 0 || dmax + 2 > OR_MAXV) return -2;
    int top = dmax + 1;
    binom_t b;
    if (binom_init(&b, n, top + 2)) return -1;
    simpvec level[OR_MAXV];
    if (build_levels(D, n, top, thr, &b, level)) return -1;
    int64_t N = 0;
    for (int q = 0; q <= top; ++q) N += level[q].n;
    simp *S = (simp *)malloc((size_t)(N > 0 ? N : 1) * sizeof(simp));
    int64_t k = 0;
    for (int q = 0; q <= top; ++q) {
        memcpy(S + k, level[q].a, (size_t)level[q].n * sizeof(simp));
        k += level[q].n;
        free(level[q].a);
    }
    qsort(S, (size_t)N, sizeof(simp), filt_cmp);

    /* position lookup per dimension */
    cpos *idx[OR_MAXV]; int64_t cnt[OR_MAXV] = {0};
    for (int q = 0; q <= top; ++q) idx[q] = (cpos *)malloc((size_t)(N > 0 ? N : 1) * sizeof(cpos));
    for (int64_t j = 0; j < N; ++j) {
        int q = S[j].dim;
        idx[q][cnt[q]].cidx = S[j].cidx; idx[q][cnt[q]].pos = j; cnt[q]++;
    }
    for (int q = 0; q <= top; ++q) qsort(idx[q], (size_t)cnt[q], sizeof(cpos), cpos_cmp);

    /* boundary matrix over Z/2 (Def 2.6.7, signs vanish) */
    col *cols = (col *)calloc((size_t)(N > 0 ? N : 1), sizeof(col));
    for (int64_t j = 0; j < N; ++j) {
        int q = S[j].dim;
        if (q == 0) continue;
        cols[j].r = (int64_t *)malloc((size_t)(q + 2) * sizeof(int64_t));
        cols[j].cap = q + 2;
        for (int m = 0; m <= q; ++m) {
            int32_t f[OR_MAXV]; int t = 0;
            for (int i = 0; i <= q; ++i) if (i != m) f[t++] = S[j].v[i];
            int64_t pos = cpos_find(idx[q - 1], cnt[q - 1], cidx_of(&b, f, q - 1));
            cols[j].r[cols[j].n++] = pos; /* facets of a clique are in K */
        }
        /* sort the q+1 rows ascending (insertion sort) */
        for (int64_t a = 1; a < cols[j].n; ++a) {
            int64_t x = cols[j].r[a], c = a - 1;
            while (c >= 0 && cols[j].r[c] > x) { cols[j].r[c + 1] = cols[j].r[c]; --c; }
            cols[j].r[c + 1] = x;
        }
    }
    int64_t *L = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    int rc = reduce_std(cols, N, L);

    pairvec pv = {0};
    if (!rc) {
        for (int64_t j = 0; j < N; ++j) {
            if (cols[j].n > 0) {
                int64_t lo = cols[j].r[cols[j].n - 1];
                or_pair p = {S[lo].dim, 0, S[lo].diam, S[j].diam, (int64_t)S[lo].cidx, (int64_t)S[j].cidx};
                pv_push(&pv, p);
            } else if (L[j] == -1 && S[j].dim <= dmax) {
                or_pair p = {S[j].dim, 0, S[j].diam, INFINITY, (int64_t)S[j].cidx, -1};
                pv_push(&pv, p);
            }
        }
    }
    for (int64_t j = 0; j < N; ++j) free(cols[j].r);
    free(cols); free(L); free(S); free(b.t);
    for (int q = 0; q <= top; ++q) free(idx[q]);
    if (rc) { free(pv.a); return -1; }
    *out = pv.a;
    return pv.n;
}

/* ------------------------------------------------------------------ */
/* cohomology: implicit coboundary, Algorithm 12                       */
/* ------------------------------------------------------------------ */

typedef struct { double diam; uint64_t cidx; } ent; /* a row of the coboundary matrix */

/* "a comes first in the filtration" (Sec. 5.1.4, equal dimension) */
static inline int ent_before(const ent *a, const ent *b) {
    return a->diam < b->diam || (a->diam == b->diam && a->cidx > b->cidx);
}
static int ent_cmp(const void *pa, const void *pb) {
    const ent *a = (const ent *)pa, *b = (const ent *)pb;
    if (ent_before(a, b)) return -1;
    if (ent_before(b, a)) return 1;
    return 0;
}

typedef struct { ent *e; int64_t n, cap; } entvec;
static int ev_push(entvec *v, ent x) {
    if (v->n == v->cap) {
        int64_t nc = v->cap ? v->cap * 2 : 64;
        ent *ne = (ent *)realloc(v->e, nc * sizeof(ent));
        if (!ne) return -1;
        v->e = ne; v->cap = nc;
    }
    v->e[v->n++] = x;
    return 0;
}

/* Cofacets of the p-simplex v[0..p] (ascending) with diam <= thr: add one
 * vertex w not in the simplex; diam(t) = max(diam(s), d(w, v_i)).         */
static int cofacets(const double *D, int64_t n, const binom_t *b, const int32_t *v, int p,
                    double sdiam, double thr, entvec *out) {
    out->n = 0;
    for (int64_t w = n - 1; w >= 0; --w) {
        int in = 0;
        for (int i = 0; i <= p; ++i) if (v[i] == w) in = 1;
        if (in) continue;
        double m = sdiam;
        for (int i = 0; i <= p; ++i) if (dist(D, w, v[i]) > m) m = dist(D, w, v[i]);
        if (m > thr) continue;
        int32_t t[OR_MAXV]; int k = 0, placed = 0;
        for (int i = 0; i <= p; ++i) {
            if (!placed && w < v[i]) { t[k++] = (int32_t)w; placed = 1; }
            t[k++] = v[i];
        }
        if (!placed) t[k++] = (int32_t)w;
        ent e = {m, cidx_of(b, t, p + 1)};
        if (ev_push(out, e)) return -1;
    }
    return 0;
}

static int ev_xor_sorted(entvec *a, const entvec *b, entvec *tmp) {
    tmp->n = 0;
    int64_t i = 0, j = 0;
    while (i < a->n && j < b->n) {
        if (ent_before(&a->e[i], &b->e[j])) { if (ev_push(tmp, a->e[i++])) return -1; }
        else if (ent_before(&b->e[j], &a->e[i])) { if (ev_push(tmp, b->e[j++])) return -1; }
        else { ++i; ++j; }
    }
    while (i < a->n) if (ev_push(tmp, a->e[i++])) return -1;
    while (j < b->n) if (ev_push(tmp, b->e[j++])) return -1;
    entvec s = *a; *a = *tmp; *tmp = s;
    return 0;
}

/* column order of the coboundary matrix: reverse filtration order */
static int cob_col_cmp(const void *pa, const void *pb) {
    const simp *a = (const simp *)pa, *b = (const simp *)pb;
    if (a->diam != b->diam) return a->diam > b->diam ? -1 : 1;
    if (a->cidx != b->cidx) return a->cidx < b->cidx ? -1 : 1;
    return 0;
}

/* The dual (cohomology) reduction, dims 0..dmax.  clearing != 0 drops the
 * p-columns that are death simplices of (p-1)-pairs before reducing.
 * stats (optional, 4*(dmax+1) int64): per dim {columns, additions,
 * pairs incl. zero-length, essential}.                                   */
int64_t or_cohom(const double *D, int64_t n, int32_t dmax, double thr, int32_t clearing,
                 or_pair **out, int64_t *stats) {
    *out = NULL;
    if (n < 0 || dmax < 0 || dmax + 2 > OR_MAXV) return -2;
    binom_t b;
    if (binom_init(&b, n, dmax + 3)) return -1;
    simpvec level[OR_MAXV];
    if (build_levels(D, n, dmax, thr, &b, level)) return -1;

    pairvec pv = {0};
    hmap prev_deaths; hm_init(&prev_deaths, 16);
    entvec W = {0}, A = {0}, T = {0};
    int err = 0;
    for (int p = 0; p <= dmax && !err; ++p) {
        simpvec *L = &level[p];
        qsort(L->a, (size_t)L->n, sizeof(simp), cob_col_cmp);
        hmap pivot_of; hm_init(&pivot_of, 1024); /* pivot cidx -> column cidx */
        hmap deaths; hm_init(&deaths, 1024);
        int64_t ncols = 0, nadd = 0, npairs = 0, ness = 0;
        for (int64_t j = 0; j < L->n && !err; ++j) {
            const simp *s = &L->a[j];
            int cleared = hm_get(&prev_deaths, s->cidx, NULL);
            if (clearing && cleared) continue;
            ncols++;
            if (cofacets(D, n, &b, s->v, p, s->diam, thr, &W)) { err = 1; break; }
            int sorted = 0;
            for (;;) {
                if (W.n == 0) break;
                int64_t best = 0; /* low = the row first in filtration order */
                if (sorted) best = 0;
                else for (int64_t i = 1; i < W.n; ++i) if (ent_before(&W.e[i], &W.e[best])) best = i;
                uint64_t owner;
                if (!hm_get(&pivot_of, W.e[best].cidx, &owner)) break;
                /* R[j] <- R[j] + D_owner (Algorithm 12, line 3) */
                if (!sorted) { qsort(W.e, (size_t)W.n, sizeof(ent), ent_cmp); sorted = 1; }
                int32_t ov[OR_MAXV];
                vertices_of(&b, owner, p, n, ov);
                if (cofacets(D, n, &b, ov, p, diam_of(D, ov, p), thr, &A)) { err = 1; break; }
                qsort(A.e, (size_t)A.n, sizeof(ent), ent_cmp);
                if (ev_xor_sorted(&W, &A, &T)) { err = 1; break; }
                nadd++;
            }
            if (err) break;
            if (W.n > 0) {
                int64_t best = 0;
                for (int64_t i = 1; i < W.n; ++i) if (ent_before(&W.e[i], &W.e[best])) best = i;
                ent piv = W.e[best];
                hm_put(&pivot_of, piv.cidx, s->cidx);
                hm_put(&deaths, piv.cidx, 1);
                or_pair pr = {p, 0, s->diam, piv.diam, (int64_t)s->cidx, (int64_t)piv.cidx};
                pv_push(&pv, pr);
                npairs++;
            } else if (!cleared) {
                or_pair pr = {p, 0, s->diam, INFINITY, (int64_t)s->cidx, -1};
                pv_push(&pv, pr);
                ness++;
            }
        }
        if (stats) {
            stats[4 * p + 0] = ncols; stats[4 * p + 1] = nadd;
            stats[4 * p + 2] = npairs; stats[4 * p + 3] = ness;
        }
        hm_free(&pivot_of);
        hm_free(&prev_deaths);
        prev_deaths = deaths;
    }
    hm_free(&prev_deaths);
    free(W.e); free(A.e); free(T.e);
    for (int q = 0; q <= dmax; ++q) free(level[q].a);
    free(b.t);
    if (err) { free(pv.a); return -1; }
    *out = pv.a;
    return pv.n;
}

/* ------------------------------------------------------------------ */
/* apparent pairs by Def 5.3.4                                         */
/* ------------------------------------------------------------------ */

/* For every p-simplex s of K (diam <= thr): t = oldest cofacet of s in K,
 * then s must be the youngest facet of t.  Writes (s, t) index pairs to
 * *out as 2*count uint64 values; returns count or negative on error.     */
int64_t or_apparent(const double *D, int64_t n, int32_t p, double thr, uint64_t **out) {
    *out = NULL;
    if (p < 0 || p + 2 > OR_MAXV) return -2;
    binom_t b;
    if (binom_init(&b, n, p + 3)) return -1;
    simpvec level[OR_MAXV];
    if (build_levels(D, n, p, thr, &b, level)) return -1;
    uint64_t *res = NULL; int64_t cnt = 0, cap = 0;
    entvec W = {0};
    for (int64_t j = 0; j < level[p].n; ++j) {
        const simp *s = &level[p].a[j];
        cofacets(D, n, &b, s->v, p, s->diam, thr, &W);
        if (W.n == 0) continue;
        int64_t best = 0;
        for (int64_t i = 1; i < W.n; ++i) if (ent_before(&W.e[i], &W.e[best])) best = i;
        ent t = W.e[best];
        int32_t tv[OR_MAXV];
        vertices_of(&b, t.cidx, p + 1, n, tv);
        /* youngest facet: last in filtration order (diam desc, then cidx asc) */
        ent young = {-1.0, 0};
        for (int m = 0; m <= p + 1; ++m) {
            int32_t f[OR_MAXV]; int k = 0;
            for (int i = 0; i <= p + 1; ++i) if (i != m) f[k++] = tv[i];
            ent e = {diam_of(D, f, p), cidx_of(&b, f, p)};
            if (young.diam < 0 || ent_before(&young, &e)) young = e;
        }
        if (young.cidx == s->cidx) {
            if (cnt == cap) { cap = cap ? 2 * cap : 1024; res = (uint64_t *)realloc(res, 2 * cap * sizeof(uint64_t)); }
            res[2 * cnt] = s->cidx; res[2 * cnt + 1] = t.cidx; cnt++;
        }
    }
    free(W.e);
    for (int q = 0; q <= p; ++q) free(level[q].a);
    free(b.t);
    *out = res;
    return cnt;
}

/* ------------------------------------------------------------------ */
/* critical edge and the simplex <-> index map                         */
/* ------------------------------------------------------------------ */

int32_t or_simplex_vertices(uint64_t cidx, int32_t q, int64_t n, int32_t *v) {
    if (q < 0 || q + 1 > OR_MAXV) return -2;
    binom_t b;
    if (binom_init(&b, n, q + 2)) return -1;
    vertices_of(&b, cidx, q, n, v);
    free(b.t);
    return 0;
}

uint64_t or_simplex_index(const int32_t *v_ascending, int32_t q, int64_t n) {
    binom_t b;
    if (binom_init(&b, n, q + 2)) return UINT64_MAX;
    uint64_t c = cidx_of(&b, v_ascending, q);
    free(b.t);
    return c;
}

/* Writes the edge (u, v), u > v, of the q-simplex that attains its diameter,
 * ties broken by the largest edge index C(u,2) + v.                      */
int32_t or_critical_edge(const double *D, int64_t n, uint64_t cidx, int32_t q, int32_t *uv) {
    int32_t v[OR_MAXV];
    if (or_simplex_vertices(cidx, q, n, v)) return -1;
    double dm = diam_of(D, v, q);
    int64_t bu = -1, bv = -1;
    for (int i = 0; i <= q; ++i)
        for (int j = 0; j < i; ++j) /* v[i] > v[j] */
            if (dist(D, v[i], v[j]) == dm) {
                int64_t e = (int64_t)v[i] * (v[i] - 1) / 2 + v[j];
                if (bu < 0 || e > bu * (bu - 1) / 2 + bv) { bu = v[i]; bv = v[j]; }
            }
    uv[0] = (int32_t)bu; uv[1] = (int32_t)bv;
    return 0;
}
