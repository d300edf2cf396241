/*
 * Slim Graph CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, single-threaded, deliberately slow restatement of the lossy
 * compression kernels of Slim Graph (Besta et al., arXiv 1912.08950) and of
 * the accuracy analytics used to judge them.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this file.  It shares no
 * code, header, table or constant generator with the CUDA library; it is
 * written from the paper and from the published definitions it relies on:
 *
 *   Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *   easy as 1, 2, 3", SC'11 (the counter-based generator replacing SG.rand).
 *
 * Every function below is a pure function of (graph, kernel, p, seed).
 * Graphs are symmetric CSR: off[n+1] (int64), col[2m] (uint32, rows sorted,
 * no self-loops, no duplicates), optional w[2m] (float32, equal on both arcs).
 *
 * Readings of the paper that this file fixes (each also cited in place):
 *  - randomness: one Philox4x32-10 draw per edge keyed by the canonical pair
 *    (lo < hi), per triangle keyed by its sorted vertex triple (a < b < c);
 *  - uniform sampling keeps an edge with probability p (Listing 1,
 *    random_uniform; Sec. 4.2.2);
 *  - spectral sparsification keeps (u,v) with probability
 *    min(1, Y / min(d_u, d_v)), Y = p ln n or p m / n, and gives kept edges
 *    weight 1 / p_uv (Sec. 4.2.1);
 *  - Triangle p-1-Reduction selects each triangle with probability p and
 *    deletes one uniformly chosen edge of it (Sec. 4.3, "SG.p is a
 *    probability of sampling a triangle"); all kernel instances see the
 *    triangles of the INPUT graph (one run_kernels pass, Listing 2), so the
 *    deleted set is the union over selected triangles;
 *  - the max-weight variant deletes the heaviest edge (Sec. 4.3; Sec. 6
 *    "Others": the MST weight is preserved), ties broken by endpoint pair;
 *  - Edge-Once TR considers edge-disjoint triangles only (Sec. 6, Edge-Once
 *    p-1-TR: no two edges deleted from one triangle, every edge considered at
 *    most once): selected triangles are scanned in increasing order of
 *    (r2, a, b, c); a triangle is accepted iff none of its edges was already
 *    considered; an accepted triangle marks its three edges considered and
 *    deletes its chosen edge;
 *  - Triangle p-2-Reduction (Sec. 4.3, x = 2) deletes two edges of each
 *    selected triangle chosen u.a.r., i.e. keeps the edge the draw r1 picks;
 *  - Min-Count TR (the technical-report variant behind "CT", Sec. 7) deletes
 *    the edge lying in the fewest triangles of the input, ties broken by the
 *    smaller endpoint pair; CT is Edge-Once with that choice;
 *  - PageRank (Table 1; output "P", a distribution) uses damping d, uniform
 *    teleport and uniform redistribution of dangling mass; KL divergence is
 *    sum_i P(i) log2(P(i)/Q(i)) (Sec. 5.2.3);
 *  - the single-vertex kernel low_degree (Listing 1; Sec. 4.4) deletes, in
 *    one pass over the input degrees, every vertex of degree 0 or 1 with its
 *    edges; the kept vertices are renumbered in increasing id order;
 *  - BFS critical edges (Sec. 5.3): for a root r, the tree edges plus the
 *    edges that could replace a tree edge, i.e. every edge joining BFS
 *    levels L and L + 1; the metric is |E~_cr| / |E_cr| with both sets taken
 *    from traversals of G and of the compressed graph from the same root;
 *  - reordered neighbours A_REN (Sec. 5.2.2): the edges {u,v} of G whose
 *    endpoint scores change relative order (sign of x_u - x_v differs from
 *    sign of y_u - y_v, compared in the scores' own float precision), as a
 *    fraction of m.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_EDGE 0x45444745u /* "EDGE" */
#define ORC_TAG_TRI 0x54524931u  /* "TRI1" */

enum {
    ORC_UNIFORM = 0,
    ORC_SPECTRAL_LOGN = 1,
    ORC_SPECTRAL_AVGDEG = 2,
    ORC_TR_RANDOM = 3,
    ORC_TR_MAXW = 4,
    ORC_TR_EO = 5,
    ORC_TR_EO_MAXW = 6,
    ORC_TR_P2 = 7,          /* Triangle p-2-Reduction: two edges of each selected triangle go */
    ORC_TR_MINCOUNT = 8,    /* Min-Count p-1-TR: the edge in the fewest triangles of G goes */
    ORC_TR_EO_MINCOUNT = 9  /* "CT": Edge-Once with the min-count choice */
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11): 10 rounds of a multiply/xor Feistel   */
/* network on four 32-bit words, with a Weyl-sequence key schedule.          */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t tag, uint32_t r[4])
{
    uint32_t ctr[4] = {a, b, c, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, r);
}

/* A probability p in [0,1] becomes the integer threshold floor(p * 2^32):   */
/* an event with probability p happens iff a uniform 32-bit draw is below it. */
uint64_t orc_threshold(double p)
{
    double t = floor(p * 4294967296.0);
    if (t >= 4294967296.0) return 4294967296ull;
    if (t <= 0.0) return 0;
    return (uint64_t)t;
}

/* Scaled spectral threshold floor(Y * 2^32), saturating at 2^64 - 1. */
static uint64_t scaled_threshold(double y)
{
    double t = floor(y * 4294967296.0);
    if (t >= 18446744073709551615.0) return UINT64_MAX;
    if (t <= 0.0) return 0;
    return (uint64_t)t;
}

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */
static int64_t find_arc(const int64_t *off, const uint32_t *col, uint32_t x, uint32_t y)
{
    int64_t lo = off[x], hi = off[x + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < y) lo = mid + 1; else hi = mid;
    }
    return (lo < off[x + 1] && col[lo] == y) ? lo : -1;
}

/* canonical edge id: the arc index of (lo -> hi) in the symmetric CSR */
static int64_t edge_id(const int64_t *off, const uint32_t *col, uint32_t x, uint32_t y)
{
    return x < y ? find_arc(off, col, x, y) : find_arc(off, col, y, x);
}

/* Write the output CSR: keep arc (x,y) iff del[edge_id(x,y)] == 0. */
static int64_t build_output(int64_t n, const int64_t *off, const uint32_t *col,
                            const float *wsrc, const uint8_t *del,
                            int64_t *off_out, uint32_t *col_out, float *w_out)
{
    int64_t k = 0;
    off_out[0] = 0;
    for (int64_t x = 0; x < n; ++x) {
        for (int64_t i = off[x]; i < off[x + 1]; ++i) {
            uint32_t y = col[i];
            int64_t e = (uint32_t)x < y ? i : find_arc(off, col, y, (uint32_t)x);
            if (!del[e]) {
                col_out[k] = y;
                if (w_out && wsrc) w_out[k] = wsrc[i];
                ++k;
            }
        }
        off_out[x + 1] = k;
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* triangles of G: canonical triples a < b < c, listed by the definition     */
/* {a,b}, {a,c}, {b,c} in E (merge of the sorted rows of a and b, c > b).    */
/* ------------------------------------------------------------------------ */
typedef void (*tri_fn)(uint32_t a, uint32_t b, uint32_t c, int64_t eab, int64_t eac,
                       int64_t ebc, void *ctx);

static void for_each_triangle(int64_t n, const int64_t *off, const uint32_t *col, tri_fn fn, void *ctx)
{
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t i = off[a]; i < off[a + 1]; ++i) {
            uint32_t b = col[i];
            if (b <= (uint32_t)a) continue;
            /* intersect N(a) and N(b), keep c > b */
            int64_t p = off[a], q = off[b];
            while (p < off[a + 1] && q < off[b + 1]) {
                uint32_t ca = col[p], cb = col[q];
                if (ca < cb) ++p;
                else if (cb < ca) ++q;
                else {
                    if (ca > b) fn((uint32_t)a, b, ca, i, p, q, ctx);
                    ++p; ++q;
                }
            }
        }
    }
}

static void count_cb(uint32_t a, uint32_t b, uint32_t c, int64_t e0, int64_t e1, int64_t e2, void *ctx)
{
    (void)a; (void)b; (void)c; (void)e0; (void)e1; (void)e2;
    ++*(int64_t *)ctx;
}

int64_t orc_triangle_count(int64_t n, const int64_t *off, const uint32_t *col)
{
    int64_t t = 0;
    for_each_triangle(n, off, col, count_cb, &t);
    return t;
}

typedef struct { uint32_t *out; int64_t k, cap; } list_ctx;

static void list_cb(uint32_t a, uint32_t b, uint32_t c, int64_t e0, int64_t e1, int64_t e2, void *vctx)
{
    (void)e0; (void)e1; (void)e2;
    list_ctx *L = (list_ctx *)vctx;
    if (L->k < L->cap) {
        L->out[3 * L->k] = a; L->out[3 * L->k + 1] = b; L->out[3 * L->k + 2] = c;
    }
    ++L->k;
}

/* lists triangles (a<b<c) in lexicographic order; returns the count */
int64_t orc_triangle_list(int64_t n, const int64_t *off, const uint32_t *col, uint32_t *out, int64_t cap)
{
    list_ctx L = {out, 0, cap};
    for_each_triangle(n, off, col, list_cb, &L);
    return L.k;
}

/* ------------------------------------------------------------------------ */
/* which edge of a triangle a kernel instance removes                       */
/* e0 = {a,b}, e1 = {a,c}, e2 = {b,c}                                       */
/* ------------------------------------------------------------------------ */
static int random_choice(uint32_t r1)
{
    /* uniform index in {0,1,2}: floor(r1 * 3 / 2^32) */
    return (int)(((uint64_t)r1 * 3u) >> 32);
}

/* heaviest edge under the strict order (w, lo, hi) */
static int maxw_choice(const float *w, const int64_t e[3], const uint32_t lo[3], const uint32_t hi[3])
{
    int best = 0;
    for (int k = 1; k < 3; ++k) {
        float wk = w[e[k]], wb = w[e[best]];
        int greater = (wk > wb) || (wk == wb && (lo[k] > lo[best] || (lo[k] == lo[best] && hi[k] > hi[best])));
        if (greater) best = k;
    }
    return best;
}

/* the edge in the fewest triangles under the order (count, lo, hi) */
static int mincount_choice(const int64_t *tcount, const int64_t e[3], const uint32_t lo[3], const uint32_t hi[3])
{
    int best = 0;
    for (int k = 1; k < 3; ++k) {
        int64_t ck = tcount[e[k]], cb = tcount[e[best]];
        int smaller = (ck < cb) || (ck == cb && (lo[k] < lo[best] || (lo[k] == lo[best] && hi[k] < hi[best])));
        if (smaller) best = k;
    }
    return best;
}

static void tcount_cb(uint32_t a, uint32_t b, uint32_t c, int64_t eab, int64_t eac, int64_t ebc, void *ctx)
{
    (void)a; (void)b; (void)c;
    int64_t *t = (int64_t *)ctx;
    ++t[eab]; ++t[eac]; ++t[ebc];
}

/* number of triangles of G through every edge, indexed by canonical edge id */
static int64_t *edge_triangle_counts(int64_t n, int64_t nnz, const int64_t *off, const uint32_t *col)
{
    int64_t *t = (int64_t *)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(int64_t));
    if (t) for_each_triangle(n, off, col, tcount_cb, t);
    return t;
}

typedef struct {
    uint64_t seed, tp;
    int mode;  /* 0 random, 1 max-weight, 2 two edges, 3 min-count */
    const float *w;
    const int64_t *tcount;
    uint8_t *del;
} union_ctx;

static void union_cb(uint32_t a, uint32_t b, uint32_t c, int64_t eab, int64_t eac, int64_t ebc, void *vctx)
{
    union_ctx *U = (union_ctx *)vctx;
    uint32_t r[4];
    draw(U->seed, a, b, c, ORC_TAG_TRI, r);
    if ((uint64_t)r[0] >= U->tp) return; /* triangle not selected */
    int64_t e[3] = {eab, eac, ebc};
    uint32_t lo[3] = {a, a, b}, hi[3] = {b, c, c};
    if (U->mode == 2) { /* x = 2: all but the edge the draw picks */
        int keep = random_choice(r[1]);
        for (int k = 0; k < 3; ++k) if (k != keep) U->del[e[k]] = 1;
        return;
    }
    int k = U->mode == 1 ? maxw_choice(U->w, e, lo, hi)
          : U->mode == 3 ? mincount_choice(U->tcount, e, lo, hi)
                         : random_choice(r[1]);
    U->del[e[k]] = 1; /* SG.del is idempotent */
}

/* Edge-Once: collect the selected triangles, sort, scan greedily.  A record
 * holds only the sort key (r2, a, b, c): the scan looks the three edges up
 * again and redraws r1, so that a scale-22 graph's billion selected
 * triangles fit in host memory (16 bytes each). */
typedef struct {
    uint32_t r2, a, b, c;
} sel_tri;

typedef struct {
    uint64_t seed, tp;
    sel_tri *v;
    int64_t k, cap;
    int oom;
} eo_ctx;

static void eo_collect_cb(uint32_t a, uint32_t b, uint32_t c, int64_t eab, int64_t eac, int64_t ebc, void *vctx)
{
    eo_ctx *E = (eo_ctx *)vctx;
    uint32_t r[4];
    draw(E->seed, a, b, c, ORC_TAG_TRI, r);
    if ((uint64_t)r[0] >= E->tp) return;
    if (E->k == E->cap) {
        int64_t ncap = E->cap ? 2 * E->cap : 1024;
        sel_tri *nv = (sel_tri *)realloc(E->v, (size_t)ncap * sizeof(sel_tri));
        if (!nv) { E->oom = 1; return; }
        E->v = nv; E->cap = ncap;
    }
    (void)eab; (void)eac; (void)ebc;
    sel_tri *t = &E->v[E->k++];
    t->r2 = r[2]; t->a = a; t->b = b; t->c = c;
}

static int sel_cmp(const void *x, const void *y)
{
    const sel_tri *s = (const sel_tri *)x, *t = (const sel_tri *)y;
    if (s->r2 != t->r2) return s->r2 < t->r2 ? -1 : 1;
    if (s->a != t->a) return s->a < t->a ? -1 : 1;
    if (s->b != t->b) return s->b < t->b ? -1 : 1;
    if (s->c != t->c) return s->c < t->c ? -1 : 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* compress(G, kernel, p, seed) -> H                                          */
/* Returns the number of arcs of H, or -1 on bad arguments, -2 if the graph  */
/* lacks the weights the kernel needs, -3 on allocation failure.             */
/* The caller sizes off_out[n+1], col_out[nnz], w_out[nnz] (w_out optional). */
/* If accepted_out is non-NULL (EO kernels), it receives one byte per arc:   */
/* 1 iff the edge belongs to an accepted (considered) triangle.              */
/* ------------------------------------------------------------------------ */
int64_t orc_compress(int64_t n, int64_t nnz, const int64_t *off, const uint32_t *col, const float *w,
                     int kernel, double p, uint64_t seed, int want_weights,
                     int64_t *off_out, uint32_t *col_out, float *w_out, uint8_t *accepted_out)
{
    if (!(p >= 0.0 && p <= 1.0)) return -1;
    if ((kernel == ORC_TR_MAXW || kernel == ORC_TR_EO_MAXW) && !w) return -2;
    if (kernel < ORC_UNIFORM || kernel > ORC_TR_EO_MINCOUNT) return -1;
    uint8_t *del = (uint8_t *)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
    if (!del) return -3;
    float *wnew = NULL;
    const float *wsrc = w;
    int64_t m = nnz / 2;

    if (kernel == ORC_UNIFORM) {
        /* random_uniform(E e): the edge stays with probability p */
        uint64_t tp = orc_threshold(p);
        for (int64_t x = 0; x < n; ++x)
            for (int64_t i = off[x]; i < off[x + 1]; ++i) {
                uint32_t y = col[i];
                if ((uint32_t)x > y) continue; /* one decision per undirected edge */
                uint32_t r[4];
                draw(seed, (uint32_t)x, y, 0, ORC_TAG_EDGE, r);
                if ((uint64_t)r[0] >= tp) del[i] = 1;
            }
    } else if (kernel == ORC_SPECTRAL_LOGN || kernel == ORC_SPECTRAL_AVGDEG) {
        /* spectral_sparsify(E e): stays with prob. min(1, Y / min(d_u, d_v)) */
        double Y = (kernel == ORC_SPECTRAL_LOGN) ? p * log((double)n)
                                                 : (n > 0 ? p * (double)m / (double)n : 0.0);
        uint64_t ty = scaled_threshold(Y);
        float yf = (float)Y;
        if (want_weights) {
            wnew = (float *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(float));
            if (!wnew) { free(del); return -3; }
        }
        for (int64_t x = 0; x < n; ++x)
            for (int64_t i = off[x]; i < off[x + 1]; ++i) {
                uint32_t y = col[i];
                uint32_t lo = (uint32_t)x < y ? (uint32_t)x : y;
                uint32_t hi = (uint32_t)x < y ? y : (uint32_t)x;
                uint64_t dx = (uint64_t)(off[x + 1] - off[x]);
                uint64_t dy = (uint64_t)(off[y + 1] - off[y]);
                uint64_t dmin = dx < dy ? dx : dy;
                uint32_t r[4];
                draw(seed, lo, hi, 0, ORC_TAG_EDGE, r);
                /* r/2^32 < Y/dmin, evaluated exactly in integers */
                int stays = (uint64_t)r[0] * dmin < ty;
                if ((uint32_t)x < y && !stays) del[i] = 1;
                if (wnew) {
                    /* W(u,v) = 1/p_uv: 1 when p_uv = 1, else dmin / Y */
                    if (dmin * 4294967296ull <= ty) wnew[i] = 1.0f;
                    else wnew[i] = (float)dmin / yf;
                }
            }
        wsrc = wnew;
    } else if (kernel == ORC_TR_RANDOM || kernel == ORC_TR_MAXW || kernel == ORC_TR_P2 ||
               kernel == ORC_TR_MINCOUNT) {
        int64_t *tc = NULL;
        if (kernel == ORC_TR_MINCOUNT) {
            tc = edge_triangle_counts(n, nnz, off, col);
            if (!tc) { free(del); return -3; }
        }
        union_ctx U = {seed, orc_threshold(p),
                       kernel == ORC_TR_MAXW ? 1 : kernel == ORC_TR_P2 ? 2 : kernel == ORC_TR_MINCOUNT ? 3 : 0,
                       w, tc, del};
        for_each_triangle(n, off, col, union_cb, &U);
        free(tc);
    } else { /* ORC_TR_EO, ORC_TR_EO_MAXW, ORC_TR_EO_MINCOUNT */
        eo_ctx E = {seed, orc_threshold(p), NULL, 0, 0, 0};
        for_each_triangle(n, off, col, eo_collect_cb, &E);
        if (E.oom) { free(E.v); free(del); return -3; }
        qsort(E.v, (size_t)E.k, sizeof(sel_tri), sel_cmp);
        uint8_t *considered = (uint8_t *)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
        int64_t *tc = kernel == ORC_TR_EO_MINCOUNT ? edge_triangle_counts(n, nnz, off, col) : NULL;
        if (!considered || (kernel == ORC_TR_EO_MINCOUNT && !tc)) { free(tc); free(considered); free(E.v); free(del); return -3; }
        for (int64_t s = 0; s < E.k; ++s) {
            const sel_tri *t = &E.v[s];
            /* the canonical ids of {a,b}, {a,c}, {b,c} */
            int64_t e[3];
            e[0] = find_arc(off, col, t->a, t->b);
            if (considered[e[0]]) continue;
            e[1] = find_arc(off, col, t->a, t->c);
            if (considered[e[1]]) continue;
            e[2] = find_arc(off, col, t->b, t->c);
            if (considered[e[2]]) continue;
            considered[e[0]] = considered[e[1]] = considered[e[2]] = 1;
            uint32_t lo[3] = {t->a, t->a, t->b}, hi[3] = {t->b, t->c, t->c};
            int k;
            if (kernel == ORC_TR_EO_MAXW) {
                k = maxw_choice(w, e, lo, hi);
            } else if (kernel == ORC_TR_EO_MINCOUNT) {
                k = mincount_choice(tc, e, lo, hi);
            } else {
                uint32_t r[4];
                draw(E.seed, t->a, t->b, t->c, ORC_TAG_TRI, r);
                k = random_choice(r[1]);
            }
            del[e[k]] = 1;
        }
        free(tc);
        if (accepted_out) {
            for (int64_t x = 0; x < n; ++x)
                for (int64_t i = off[x]; i < off[x + 1]; ++i)
                    accepted_out[i] = considered[edge_id(off, col, (uint32_t)x, col[i])];
        }
        free(considered);
        free(E.v);
    }

    int64_t k = build_output(n, off, col, wsrc, del, off_out, col_out, w_out);
    free(wnew);
    free(del);
    return k;
}

/* |N(x) ∩ N(y)| by a merge of the two sorted lists */
static int64_t common_count(const int64_t *off, const uint32_t *col, uint32_t x, uint32_t y)
{
    int64_t i = off[x], j = off[y], k = 0;
    while (i < off[x + 1] && j < off[y + 1]) {
        if (col[i] < col[j]) ++i;
        else if (col[j] < col[i]) ++j;
        else { ++k; ++i; ++j; }
    }
    return k;
}

/* Per-edge query of a union-semantics TR kernel on edge {x,y}: is it deleted?  */
/* Walks the triangles through {x,y} only, so it runs on graphs of any size.     */
int orc_tr_union_edge_deleted(int64_t n, const int64_t *off, const uint32_t *col, const float *w,
                              int kernel, double p, uint64_t seed, uint32_t x, uint32_t y)
{
    (void)n;
    uint64_t tp = orc_threshold(p);
    uint32_t lo = x < y ? x : y, hi = x < y ? y : x;
    int64_t p0 = off[lo], q0 = off[hi];
    while (p0 < off[lo + 1] && q0 < off[hi + 1]) {
        uint32_t ca = col[p0], cb = col[q0];
        if (ca < cb) { ++p0; continue; }
        if (cb < ca) { ++q0; continue; }
        uint32_t z = ca;
        ++p0; ++q0;
        uint32_t a, b, c;
        if (z < lo) { a = z; b = lo; c = hi; }
        else if (z < hi) { a = lo; b = z; c = hi; }
        else { a = lo; b = hi; c = z; }
        uint32_t r[4];
        draw(seed, a, b, c, ORC_TAG_TRI, r);
        if ((uint64_t)r[0] >= tp) continue;
        int k;
        uint32_t l3[3] = {a, a, b}, h3[3] = {b, c, c};
        if (kernel == ORC_TR_MAXW) {
            int64_t e[3] = {edge_id(off, col, a, b), edge_id(off, col, a, c), edge_id(off, col, b, c)};
            k = maxw_choice(w, e, l3, h3);
        } else if (kernel == ORC_TR_MINCOUNT) {
            /* triangle counts of the three edges: |N(x) ∩ N(y)| each */
            int64_t cnt[3] = {common_count(off, col, a, b), common_count(off, col, a, c),
                              common_count(off, col, b, c)};
            int64_t e[3] = {0, 1, 2};
            k = mincount_choice(cnt, e, l3, h3);
        } else {
            k = random_choice(r[1]);
        }
        uint32_t dl = (k == 2) ? b : a, dh = (k == 0) ? b : c;
        if (kernel == ORC_TR_P2) {
            if (!(dl == lo && dh == hi)) return 1; /* only the drawn edge stays */
        } else if (dl == lo && dh == hi) {
            return 1;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* analytics                                                                 */
/* ------------------------------------------------------------------------ */

/* PageRank, FP64: x0 = 1/n; x' = (1-d)/n + d (sum_{u in N(v)} x_u/d_u + D/n),  */
/* D = total rank on vertices of degree 0.  Returns ||x_T - x_{T-1}||_1.        */
double orc_pagerank(int64_t n, const int64_t *off, const uint32_t *col, double damping, int iters,
                    double *x_out)
{
    if (n == 0) return 0.0;
    double *x = x_out;
    double *y = (double *)malloc((size_t)n * sizeof(double));
    double *nx = (double *)malloc((size_t)n * sizeof(double));
    double resid = 0.0;
    for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
    for (int it = 0; it < iters; ++it) {
        double dangling = 0.0;
        for (int64_t u = 0; u < n; ++u) {
            int64_t du = off[u + 1] - off[u];
            if (du == 0) { dangling += x[u]; y[u] = 0.0; }
            else y[u] = x[u] / (double)du;
        }
        for (int64_t v = 0; v < n; ++v) {
            double s = 0.0;
            for (int64_t i = off[v]; i < off[v + 1]; ++i) s += y[col[i]];
            nx[v] = (1.0 - damping) / (double)n + damping * (s + dangling / (double)n);
        }
        resid = 0.0;
        for (int64_t v = 0; v < n; ++v) { resid += fabs(nx[v] - x[v]); x[v] = nx[v]; }
    }
    free(y);
    free(nx);
    return resid;
}

/* D_KL(P||Q) = sum_i P(i) log2(P(i)/Q(i)), both normalised to sum 1 first. */
double orc_kl_divergence(int64_t n, const double *P, const double *Q)
{
    double sp = 0.0, sq = 0.0, kl = 0.0;
    for (int64_t i = 0; i < n; ++i) { sp += P[i]; sq += Q[i]; }
    for (int64_t i = 0; i < n; ++i) {
        double pi = P[i] / sp, qi = Q[i] / sq;
        if (pi > 0.0) kl += pi * log2(pi / qi);
    }
    return kl;
}

static int64_t uf_find(int64_t *parent, int64_t v)
{
    while (parent[v] != v) {
        parent[v] = parent[parent[v]];
        v = parent[v];
    }
    return v;
}

/* number of connected components (isolated vertices count); labels optional */
int64_t orc_cc_count(int64_t n, const int64_t *off, const uint32_t *col, int64_t *labels_out)
{
    int64_t *parent = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) parent[v] = v;
    for (int64_t x = 0; x < n; ++x)
        for (int64_t i = off[x]; i < off[x + 1]; ++i) {
            int64_t a = uf_find(parent, x), b = uf_find(parent, col[i]);
            if (a != b) { if (a < b) parent[b] = a; else parent[a] = b; }
        }
    int64_t cc = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t r = uf_find(parent, v);
        if (r == v) ++cc;
        if (labels_out) labels_out[v] = r;
    }
    free(parent);
    return cc;
}

/* Kruskal: MST (forest) weight in exact integer units of 2^-24 when every  */
/* weight is k * 2^-24; returns the sum of round(w * 2^24).                 */
typedef struct { float w; uint32_t lo, hi; } wedge;

static int wedge_cmp(const void *x, const void *y)
{
    const wedge *s = (const wedge *)x, *t = (const wedge *)y;
    if (s->w != t->w) return s->w < t->w ? -1 : 1;
    if (s->lo != t->lo) return s->lo < t->lo ? -1 : 1;
    if (s->hi != t->hi) return s->hi < t->hi ? -1 : 1;
    return 0;
}

int64_t orc_mst_weight_units(int64_t n, const int64_t *off, const uint32_t *col, const float *w)
{
    int64_t m = 0;
    for (int64_t x = 0; x < n; ++x)
        for (int64_t i = off[x]; i < off[x + 1]; ++i) if ((uint32_t)x < col[i]) ++m;
    wedge *E = (wedge *)malloc((size_t)(m > 0 ? m : 1) * sizeof(wedge));
    int64_t k = 0;
    for (int64_t x = 0; x < n; ++x)
        for (int64_t i = off[x]; i < off[x + 1]; ++i)
            if ((uint32_t)x < col[i]) { E[k].w = w[i]; E[k].lo = (uint32_t)x; E[k].hi = col[i]; ++k; }
    qsort(E, (size_t)m, sizeof(wedge), wedge_cmp);
    int64_t *parent = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) parent[v] = v;
    int64_t total = 0;
    for (int64_t s = 0; s < m; ++s) {
        int64_t a = uf_find(parent, E[s].lo), b = uf_find(parent, E[s].hi);
        if (a == b) continue;
        if (a < b) parent[b] = a; else parent[a] = b;
        total += (int64_t)llround((double)E[s].w * 16777216.0);
    }
    free(parent);
    free(E);
    return total;
}

/* ------------------------------------------------------------------------ */
/* single-vertex kernel low_degree (Listing 1; Sec. 4.4)                     */
/* ------------------------------------------------------------------------ */
/* Keeps the vertices of input degree >= 2 and the edges among them.          */
/* new_id[v] = new index of a kept vertex, or -1.  Returns the kept vertex     */
/* count; off_out[n'+1], col_out (arcs with both ends kept, renumbered).       */
int64_t orc_low_degree(int64_t n, const int64_t *off, const uint32_t *col, int64_t *new_id,
                       int64_t *off_out, uint32_t *col_out, int64_t *nnz_out)
{
    int64_t kept = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = off[v + 1] - off[v];
        new_id[v] = (d == 0 || d == 1) ? -1 : kept++;
    }
    int64_t k = 0;
    off_out[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (new_id[v] < 0) continue;
        for (int64_t i = off[v]; i < off[v + 1]; ++i)
            if (new_id[col[i]] >= 0) col_out[k++] = (uint32_t)new_id[col[i]];
        off_out[new_id[v] + 1] = k;
    }
    *nnz_out = k;
    return kept;
}

/* ------------------------------------------------------------------------ */
/* BFS critical edges (Sec. 5.3)                                             */
/* ------------------------------------------------------------------------ */
/* BFS levels from root (-1 = unreached), by a plain FIFO queue.               */
void orc_bfs_levels(int64_t n, const int64_t *off, const uint32_t *col, int64_t root, int64_t *level)
{
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    if (root < 0 || root >= n) return;
    int64_t *queue = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t head = 0, tail = 0;
    level[root] = 0;
    queue[tail++] = root;
    while (head < tail) {
        int64_t x = queue[head++];
        for (int64_t i = off[x]; i < off[x + 1]; ++i) {
            uint32_t y = col[i];
            if (level[y] < 0) {
                level[y] = level[x] + 1;
                queue[tail++] = y;
            }
        }
    }
    free(queue);
}

/* |E_cr|: undirected edges {x,y} with level(y) = level(x) + 1 -- the tree   */
/* edges and every edge that could stand in for one.                          */
int64_t orc_critical_edges(int64_t n, const int64_t *off, const uint32_t *col, int64_t root)
{
    int64_t *level = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    orc_bfs_levels(n, off, col, root, level);
    int64_t cnt = 0;
    for (int64_t x = 0; x < n; ++x) {
        if (level[x] < 0) continue;
        for (int64_t i = off[x]; i < off[x + 1]; ++i)
            if (level[col[i]] == level[x] + 1) ++cnt;
    }
    free(level);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* reordered neighbours A_REN (Sec. 5.2.2)                                   */
/* ------------------------------------------------------------------------ */
static int fsign(float a, float b) { return (a > b) - (a < b); }

/* Number of undirected edges {u,v} of G with sign(x_u - x_v) != sign(y_u - y_v). */
int64_t orc_reordered_neighbours(int64_t n, const int64_t *off, const uint32_t *col, const float *x,
                                 const float *y)
{
    int64_t cnt = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t i = off[u]; i < off[u + 1]; ++i) {
            uint32_t v = col[i];
            if ((int64_t)v <= u) continue; /* each edge once */
            if (fsign(x[u], x[v]) != fsign(y[u], y[v])) ++cnt;
        }
    return cnt;
}

/* Triangles through every vertex (the per-vertex output "TC" of Table 1). */
static void vtc_cb(uint32_t a, uint32_t b, uint32_t c, int64_t eab, int64_t eac, int64_t ebc, void *ctx)
{
    (void)eab; (void)eac; (void)ebc;
    int64_t *t = (int64_t *)ctx;
    ++t[a]; ++t[b]; ++t[c];
}

void orc_vertex_triangle_counts(int64_t n, const int64_t *off, const uint32_t *col, int64_t *out)
{
    for (int64_t v = 0; v < n; ++v) out[v] = 0;
    for_each_triangle(n, off, col, vtc_cb, out);
}

static int isign(int64_t a, int64_t b) { return (a > b) - (a < b); }

/* A_REN count for integer scores (exact). */
int64_t orc_reordered_neighbours_i64(int64_t n, const int64_t *off, const uint32_t *col, const int64_t *x,
                                     const int64_t *y)
{
    int64_t cnt = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t i = off[u]; i < off[u + 1]; ++i) {
            uint32_t v = col[i];
            if ((int64_t)v <= u) continue;
            if (isign(x[u], x[v]) != isign(y[u], y[v])) ++cnt;
        }
    return cnt;
}
