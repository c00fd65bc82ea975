/*
 * CPU ORACLE for exact all-k clique counting with the Succinct Clique Tree
 * (Jain & Seshadhri, "The Power of Pivoting for Exact Clique Counting",
 * WSDM 2020).  TEST INFRASTRUCTURE ONLY: the library's tests, its smoke
 * check and the benchmark's CPU-baseline leg use this file; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * It is deliberately plain and sequential (an optional root-parallel mode
 * follows the paper's parallel variant for global counts, Sec. 4 "Parallel
 * version"):
 *   1. Degeneracy orientation (Lemma degen; Alg. 1 step 1): vertices are
 *      removed one at a time, always one of minimum remaining degree
 *      (bucket form of Matula and Beck, as laid out by Batagelj and
 *      Zaversnik 2003).  N+(v) = neighbours removed after v.
 *   2. For every vertex v, the root's child labelled N+(v) with the link
 *      (v, hold) (Alg. 1 step 3), explored depth first (Sec. 4, "Storage
 *      cost": one path at a time).
 *   3. At a node labelled S != {}: the subgraph induced on S (undirected
 *      adjacency, N(S,u) = N(u) cap S, Sec. 2), the pivot p maximising
 *      |N(S,p)| (Alg. 1 pivot step; ties: smallest vertex id), the pivot child
 *      N(S,p) with link (p, pivot), and for the non-neighbours v_1 < ... <
 *      v_l of p in S \ {p} the hold children N(S,v_i) \ {v_1..v_{i-1}} with
 *      links (v_i, hold) (Alg. 1 hold step; order: ascending id).
 *   4. At each leaf (S = {}), with h = |H(T)| and p = |P(T)|, the updates of
 *      Alg. 2: C_{h+i} += C(p,i); per vertex of H: c_{h+i} += C(p,i); per
 *      vertex of P: c_{h+1+i} += C(p-1,i); per edge HH: c_{h+i} += C(p,i);
 *      per edge PH: c_{h+1+i} += C(p-1,i); per edge PP: c_{h+2+i} +=
 *      C(p-2,i).
 *   5. Truncation to k <= kmax (Sec. 4, "Counting k-cliques for a specific
 *      k"): a branch whose hold count exceeds kmax is cut.
 * Counts are multi-limb unsigned integers (32-bit limbs, least significant
 * first) whose width the caller picks; any carry out of the top limb is
 * reported as an error, so results are exact or refused.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 3, ORC_EOVERFLOW = 4, ORC_ECAP = 7 };

/* ------------------------------------------------------------ integers */

static void big_add(uint32_t *dst, const uint32_t *src, int nl, int *ovf)
{
    uint64_t c = 0;
    for (int i = 0; i < nl; ++i) {
        c += (uint64_t)dst[i] + src[i];
        dst[i] = (uint32_t)c;
        c >>= 32;
    }
    if (c) *ovf = 1;
}

/* Pascal's rule: C(a,b) = C(a-1,b-1) + C(a-1,b), C(a,0) = C(a,a) = 1.
 * Layout: row a starts at a*(a+1)/2, entry b of row a at that + b. */
static uint32_t *binom_table(int amax, int nl, int *ovf)
{
    size_t rows = (size_t)amax + 1;
    uint32_t *t = (uint32_t *)calloc(rows * (rows + 1) / 2 * (size_t)nl, sizeof(uint32_t));
    if (!t) return NULL;
    for (int a = 0; a <= amax; ++a) {
        uint32_t *row = t + (size_t)a * (a + 1) / 2 * nl;
        row[0] = 1;
        row[(size_t)a * nl] = 1;
        if (a >= 2) {
            const uint32_t *prev = t + (size_t)(a - 1) * a / 2 * nl;
            for (int b = 1; b < a; ++b) {
                memcpy(row + (size_t)b * nl, prev + (size_t)(b - 1) * nl, nl * sizeof(uint32_t));
                big_add(row + (size_t)b * nl, prev + (size_t)b * nl, nl, ovf);
            }
        }
    }
    return t;
}

static const uint32_t *binom_at(const uint32_t *t, int a, int b, int nl)
{
    return t + ((size_t)a * (a + 1) / 2 + b) * nl;
}

/* ---------------------------------------------------------------- graph */

typedef struct {
    int64_t n, m;
    const int64_t *rp;
    const uint32_t *col;
    int64_t *up;      /* up[u]: number of edges (a,b), a<b, with a < u */
    uint32_t *rank;   /* removal index in the degeneracy order */
    int64_t *orp;     /* out-neighbourhoods N+(v), sorted by id */
    uint32_t *ocol;
    int alpha;
} graph;

static int row_find(const graph *g, uint32_t a, uint32_t b, int64_t *pos)
{
    int64_t lo = g->rp[a], hi = g->rp[a + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->col[mid] < b) lo = mid + 1; else hi = mid;
    }
    if (pos) *pos = lo;
    return lo < g->rp[a + 1] && g->col[lo] == b;
}

static int is_adj(const graph *g, uint32_t a, uint32_t b)
{
    if (g->rp[a + 1] - g->rp[a] > g->rp[b + 1] - g->rp[b]) { uint32_t t = a; a = b; b = t; }
    return row_find(g, a, b, NULL);
}

/* canonical edge id: rank of (min,max) in lexicographic order */
static int64_t edge_id(const graph *g, uint32_t a, uint32_t b)
{
    if (a > b) { uint32_t t = a; a = b; b = t; }
    int64_t pos, first;
    row_find(g, a, b, &pos);
    row_find(g, a, a, &first); /* first neighbour > a (no self-loops) */
    return g->up[a] + (pos - first);
}

/* Degeneracy order: repeatedly remove a vertex of minimum remaining degree.
 * Bucket layout after Batagelj-Zaversnik: `vert` lists vertices by current
 * degree, `bin[d]` is where degree-d vertices start, `pos[v]` is v's slot. */
static int degeneracy_order(graph *g, uint32_t *core)
{
    int64_t n = g->n;
    int64_t *deg = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint32_t *vert = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    int64_t md = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (!deg || !pos || !vert) break;
        deg[v] = g->rp[v + 1] - g->rp[v];
        if (deg[v] > md) md = deg[v];
    }
    int64_t *bin = (int64_t *)calloc((size_t)md + 2, sizeof(int64_t));
    if (!deg || !pos || !vert || !bin) { free(deg); free(pos); free(vert); free(bin); return ORC_ENOMEM; }
    for (int64_t v = 0; v < n; ++v) bin[deg[v]]++;
    int64_t start = 0;
    for (int64_t d = 0; d <= md; ++d) { int64_t c = bin[d]; bin[d] = start; start += c; }
    for (int64_t v = 0; v < n; ++v) { pos[v] = bin[deg[v]]; vert[pos[v]] = (uint32_t)v; bin[deg[v]]++; }
    for (int64_t d = md; d >= 1; --d) bin[d] = bin[d - 1];
    bin[0] = 0;
    int64_t alpha = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t v = vert[i];
        g->rank[v] = (uint32_t)i;
        if (core) core[v] = (uint32_t)deg[v];
        if (deg[v] > alpha) alpha = deg[v];
        for (int64_t e = g->rp[v]; e < g->rp[v + 1]; ++e) {
            uint32_t u = g->col[e];
            if (deg[u] > deg[v]) {
                int64_t du = deg[u], pu = pos[u], pw = bin[du];
                uint32_t w = vert[pw];
                if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    (void)alpha;
    free(deg); free(pos); free(vert); free(bin);
    return ORC_OK;
}

static int graph_init(graph *g, int64_t n, const int64_t *rp, const uint32_t *col)
{
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->rp = rp;
    g->col = col;
    g->m = rp[n] / 2;
    g->up = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    g->rank = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    g->orp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    g->ocol = (uint32_t *)malloc(((size_t)g->m + 1) * sizeof(uint32_t));
    if (!g->up || !g->rank || !g->orp || !g->ocol) return ORC_ENOMEM;
    g->up[0] = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t c = 0;
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) c += col[e] > u;
        g->up[u + 1] = g->up[u] + c;
    }
    int rc = degeneracy_order(g, NULL);
    if (rc) return rc;
    g->orp[0] = 0;
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e)
            if (g->rank[col[e]] > g->rank[v]) g->ocol[k++] = col[e];
        g->orp[v + 1] = k;
        if (k - g->orp[v] > g->alpha) g->alpha = (int)(k - g->orp[v]);
    }
    return ORC_OK;
}

/* The same graph with a caller's acyclic orientation instead of the
 * degeneracy order (any acyclic orientation counts every clique once, at its
 * first vertex): out-lists orow/ocol, each sorted ascending.  They must be an
 * orientation of the graph -- every edge in exactly one of its endpoints'
 * lists, nothing else -- and acyclic (Kahn's topological sort consumes every
 * vertex); else ORC_EINVAL.  rank[] becomes the topological position. */
static int graph_init_dag(graph *g, int64_t n, const int64_t *rp, const uint32_t *col, const int64_t *orow,
                          const uint32_t *ocol)
{
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->rp = rp;
    g->col = col;
    g->m = rp[n] / 2;
    g->up = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    g->rank = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    g->orp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    g->ocol = (uint32_t *)malloc(((size_t)g->m + 1) * sizeof(uint32_t));
    int64_t *indeg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    uint32_t *queue = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    int rc = ORC_OK;
    if (!g->up || !g->rank || !g->orp || !g->ocol || !indeg || !queue) rc = ORC_ENOMEM;
    if (!rc && (orow[0] != 0 || orow[n] != g->m)) rc = ORC_EINVAL;
    for (int64_t v = 0; !rc && v < n; ++v) {
        if (orow[v + 1] < orow[v]) { rc = ORC_EINVAL; break; }
        for (int64_t i = orow[v]; i < orow[v + 1]; ++i) {
            const uint32_t u = ocol[i];
            if ((uint64_t)u >= (uint64_t)n || (i > orow[v] && ocol[i - 1] >= u) || !row_find(g, (uint32_t)v, u, NULL)) {
                rc = ORC_EINVAL;
                break;
            }
            indeg[u]++;
        }
    }
    /* every edge in exactly one list: lists hold m entries in all, each a
     * neighbour, and no edge is in both of its endpoints' lists */
    for (int64_t v = 0; !rc && v < n; ++v)
        for (int64_t i = orow[v]; i < orow[v + 1] && !rc; ++i) {
            const uint32_t u = ocol[i];
            int64_t lo = orow[u], hi = orow[u + 1];
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (ocol[mid] < (uint32_t)v) lo = mid + 1; else hi = mid;
            }
            if (lo < orow[u + 1] && ocol[lo] == (uint32_t)v) rc = ORC_EINVAL;
        }
    if (!rc) {
        int64_t head = 0, tail = 0;
        for (int64_t v = 0; v < n; ++v) if (!indeg[v]) queue[tail++] = (uint32_t)v;
        while (head < tail) {
            const uint32_t v = queue[head];
            g->rank[v] = (uint32_t)head++;
            for (int64_t i = orow[v]; i < orow[v + 1]; ++i)
                if (--indeg[ocol[i]] == 0) queue[tail++] = ocol[i];
        }
        if (tail != n) rc = ORC_EINVAL; /* a cycle */
    }
    if (!rc) {
        g->up[0] = 0;
        for (int64_t u = 0; u < n; ++u) {
            int64_t c = 0;
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) c += col[e] > u;
            g->up[u + 1] = g->up[u] + c;
        }
        for (int64_t v = 0; v <= n; ++v) g->orp[v] = orow[v];
        for (int64_t i = 0; i < g->m; ++i) g->ocol[i] = ocol[i];
        for (int64_t v = 0; v < n; ++v)
            if (orow[v + 1] - orow[v] > g->alpha) g->alpha = (int)(orow[v + 1] - orow[v]);
    }
    free(indeg);
    free(queue);
    return rc;
}

static void graph_free(graph *g)
{
    free(g->up); free(g->rank); free(g->orp); free(g->ocol);
}

/* ------------------------------------------------------------- SCT walk */

typedef struct {
    const graph *g;
    int kmax, K, nl;
    const uint32_t *binom;
    uint32_t *C, *cv, *ce;   /* outputs (NULL = not wanted) */
    uint32_t *H, *P;         /* current path's hold / pivot vertices */
    int h, p;
    uint8_t *arena;          /* bump allocator for per-node scratch */
    size_t top, cap;
    int ovf, err;
    uint64_t nodes, leaves, sum_s;
    uint64_t chain;          /* nodes below the topmost clique labels (see visit) */
    int clq;                 /* the parent node's label is a clique */
    uint64_t *hist;          /* optional leaf histogram over (h, p) */
    int hdim;
    int32_t *paths;          /* optional leaf dump: h, p, H..., P... */
    int64_t plen, pcap;
} walker;

static void *walk_alloc(walker *w, size_t bytes)
{
    bytes = (bytes + 7) & ~(size_t)7;
    if (w->top + bytes > w->cap) { w->err = ORC_ENOMEM; return NULL; }
    void *p = w->arena + w->top;
    w->top += bytes;
    return p;
}

static void add_row(walker *w, uint32_t *cell0, int kfirst, int a)
{
    /* cell0[k] += C(a, k - kfirst) for k = kfirst .. kfirst + a (within K) */
    for (int i = 0; i <= a; ++i) {
        int k = kfirst + i;
        if (k > w->kmax) break;
        big_add(cell0 + (size_t)k * w->nl, binom_at(w->binom, a, i, w->nl), w->nl, &w->ovf);
    }
}

static void leaf(walker *w)
{
    int h = w->h, p = w->p, K = w->K, nl = w->nl;
    w->leaves++;
    if (w->hist && h < w->hdim && p < w->hdim) w->hist[(size_t)h * w->hdim + p]++;
    if (w->paths) {
        if (w->plen + 2 + h + p > w->pcap) { w->err = ORC_ECAP; return; }
        w->paths[w->plen++] = h;
        w->paths[w->plen++] = p;
        for (int i = 0; i < h; ++i) w->paths[w->plen++] = (int32_t)w->H[i];
        for (int i = 0; i < p; ++i) w->paths[w->plen++] = (int32_t)w->P[i];
    }
    /* Alg. 2: global counts */
    if (w->C) add_row(w, w->C, h, p);
    /* Alg. 2 step ht / pt: per-vertex counts */
    if (w->cv) {
        for (int i = 0; i < h; ++i) add_row(w, w->cv + (size_t)w->H[i] * K * nl, h, p);
        for (int i = 0; i < p; ++i) add_row(w, w->cv + (size_t)w->P[i] * K * nl, h + 1, p - 1);
    }
    /* Alg. 2 steps hht / pht / ppt: per-edge counts */
    if (w->ce) {
        const graph *g = w->g;
        for (int i = 0; i < h; ++i)
            for (int j = i + 1; j < h; ++j)
                add_row(w, w->ce + (size_t)edge_id(g, w->H[i], w->H[j]) * K * nl, h, p);
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < h; ++j)
                add_row(w, w->ce + (size_t)edge_id(g, w->P[i], w->H[j]) * K * nl, h + 1, p - 1);
        for (int i = 0; i < p; ++i)
            for (int j = i + 1; j < p; ++j)
                add_row(w, w->ce + (size_t)edge_id(g, w->P[i], w->P[j]) * K * nl, h + 2, p - 2);
    }
}

/* Node labelled S = {v[0] < ... < v[s-1]}; A is the s x s adjacency matrix of
 * the subgraph induced on S. */
static void visit(walker *w, const uint32_t *v, const uint8_t *A, int s)
{
    if (w->err) return;
    if (w->h > w->kmax) return; /* truncation: only cliques larger than kmax below */
    w->nodes++;
    if (s == 0) { leaf(w); return; }
    w->sum_s += (uint64_t)s;
    size_t mark = w->top;
    int *deg = (int *)walk_alloc(w, (size_t)s * sizeof(int));
    int *idx = (int *)walk_alloc(w, (size_t)s * sizeof(int));
    int *R = (int *)walk_alloc(w, (size_t)s * sizeof(int));
    uint32_t *cv = (uint32_t *)walk_alloc(w, (size_t)s * sizeof(uint32_t));
    uint8_t *cA = (uint8_t *)walk_alloc(w, (size_t)s * s);
    if (w->err) return;

    /* |N(S,u)| for every u in S; pivot = first maximum (smallest id) */
    int pi = 0;
    for (int i = 0; i < s; ++i) {
        deg[i] = 0;
        for (int j = 0; j < s; ++j) deg[i] += A[(size_t)i * s + j];
        if (deg[i] > deg[pi]) pi = i;
    }

    /* A nonempty label that is a clique has one continuation: each pivot is
     * adjacent to the rest, so its subtree is the chain of pivot children
     * S, S minus one member, ..., {} -- |S| nodes below S.  Count them at the
     * topmost such label of a path (statistics only). */
    int is_clique = 1;
    for (int i = 0; i < s; ++i) if (deg[i] != s - 1) { is_clique = 0; break; }
    if (is_clique && !w->clq) w->chain += (uint64_t)s;

    /* pivot child: N(S,p), link (p, pivot) */
    int cs = 0;
    for (int j = 0; j < s; ++j) if (A[(size_t)pi * s + j]) idx[cs++] = j;
    for (int a = 0; a < cs; ++a) {
        cv[a] = v[idx[a]];
        for (int b = 0; b < cs; ++b) cA[(size_t)a * cs + b] = A[(size_t)idx[a] * s + idx[b]];
    }
    w->P[w->p++] = v[pi];
    const int parent_clq = w->clq;
    w->clq = is_clique;
    visit(w, cv, cA, cs);
    w->clq = parent_clq;
    w->p--;

    /* non-neighbours of p in S \ {p}, ascending: v_1 < ... < v_l */
    int r = 0;
    for (int j = 0; j < s; ++j) if (j != pi && !A[(size_t)pi * s + j]) R[r++] = j;

    /* hold children: N(S,v_i) \ {v_1..v_{i-1}}, link (v_i, hold) */
    for (int t = 0; t < r && !w->err; ++t) {
        int vi = R[t];
        cs = 0;
        for (int j = 0; j < s; ++j) {
            if (!A[(size_t)vi * s + j]) continue;
            int earlier = 0;
            for (int q = 0; q < t; ++q) if (R[q] == j) { earlier = 1; break; }
            if (!earlier) idx[cs++] = j;
        }
        for (int a = 0; a < cs; ++a) {
            cv[a] = v[idx[a]];
            for (int b = 0; b < cs; ++b) cA[(size_t)a * cs + b] = A[(size_t)idx[a] * s + idx[b]];
        }
        w->H[w->h++] = v[vi];
        const int parent_clq = w->clq;
        w->clq = 0; /* a label with a hold child is not a clique */
        visit(w, cv, cA, cs);
        w->clq = parent_clq;
        w->h--;
    }
    w->top = mark;
}

/* Root's child for vertex r: label N+(r), link (r, hold) (Alg. 1 step 3). */
static void visit_root(walker *w, uint32_t r)
{
    const graph *g = w->g;
    int s = (int)(g->orp[r + 1] - g->orp[r]);
    const uint32_t *v = g->ocol + g->orp[r];
    size_t mark = w->top;
    uint8_t *A = (uint8_t *)walk_alloc(w, (size_t)s * s + 1);
    if (w->err) return;
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j)
            A[(size_t)i * s + j] = (uint8_t)(i != j && is_adj(g, v[i], v[j]));
    w->h = 0;
    w->p = 0;
    w->clq = 0;
    w->H[w->h++] = r;
    visit(w, v, A, s);
    w->top = mark;
}

static int walker_init(walker *w, const graph *g, int kmax, int nl, const uint32_t *binom)
{
    memset(w, 0, sizeof(*w));
    w->g = g;
    w->kmax = kmax;
    w->K = kmax + 1;
    w->nl = nl;
    w->binom = binom;
    size_t a = (size_t)g->alpha + 2;
    /* per level: 4 int arrays and an s x s matrix; s shrinks along a path */
    w->cap = a * a * a / 3 + a * a * 40 + 4096;
    w->arena = (uint8_t *)malloc(w->cap);
    w->H = (uint32_t *)malloc((a + 2) * sizeof(uint32_t));
    w->P = (uint32_t *)malloc((a + 2) * sizeof(uint32_t));
    if (!w->arena || !w->H || !w->P) return ORC_ENOMEM;
    return ORC_OK;
}

static void walker_free(walker *w)
{
    free(w->arena); free(w->H); free(w->P);
}

/* ------------------------------------------------------ threaded global */

typedef struct {
    walker w;
    const uint32_t *roots;
    int64_t nroots;
    int64_t *next;
} worker;

static void *worker_main(void *arg)
{
    worker *k = (worker *)arg;
    for (;;) {
        int64_t i0 = __atomic_fetch_add(k->next, 16, __ATOMIC_RELAXED);
        if (i0 >= k->nroots) break;
        int64_t i1 = i0 + 16 < k->nroots ? i0 + 16 : k->nroots;
        for (int64_t i = i0; i < i1 && !k->w.err; ++i)
            visit_root(&k->w, k->roots ? k->roots[i] : (uint32_t)i);
    }
    return NULL;
}

/* -------------------------------------------------------------- exports */

/* Degeneracy order and out-degree bound: rank[v] (removal index) and the
 * largest out-degree alpha of the resulting orientation. */
int orc_orient(int64_t n, const int64_t *rp, const uint32_t *col, uint32_t *rank, uint32_t *core,
               int32_t *alpha)
{
    graph g;
    int rc = graph_init(&g, n, rp, col);
    if (!rc) {
        if (rank) memcpy(rank, g.rank, (size_t)n * sizeof(uint32_t));
        if (alpha) *alpha = g.alpha;
        if (core) rc = degeneracy_order(&g, core);
    }
    graph_free(&g);
    return rc;
}

/*
 * Exact counts for k = 0..kmax (kmax < 0: all k), nl 32-bit limbs each.
 *   C  [kmax+1][nl]       global counts           (NULL: skip)
 *   cv [n][kmax+1][nl]    per-vertex counts       (NULL: skip)
 *   ce [m][kmax+1][nl]    per-edge counts         (NULL: skip; edge id =
 *                         rank of (min,max) in lexicographic order)
 * Output arrays must be zeroed by the caller.  roots/nroots restrict the walk
 * to the given root vertices (NULL: all).  nthreads > 1 is allowed only for
 * global counts (private arrays per thread, summed at the end).
 * stats[0..5] = nodes (excluding the tree's root), leaves, sum of |S| over
 * internal nodes, alpha, kmax used, and the nodes below the topmost clique
 * labels of the paths (the pivot chains that a walk closing clique labels
 * at once skips).  orow_in/ocol_in (NULL: the degeneracy order) give an
 * acyclic orientation to walk instead (see graph_init_dag).  hist (hdim x hdim) counts leaves by
 * (h, p).  Returns 0, or an ORC_* error (ORC_EOVERFLOW if nl is too small).
 */
int orc_count(int64_t n, const int64_t *rp, const uint32_t *col, int kmax, int nl, uint32_t *C,
              uint32_t *cv, uint32_t *ce, const uint32_t *roots, int64_t nroots, int nthreads,
              uint64_t *stats, uint64_t *hist, int hdim, const int64_t *orow_in, const uint32_t *ocol_in)
{
    if (n < 0 || nl < 1 || (nthreads > 1 && (cv || ce))) return ORC_EINVAL;
    graph g;
    int rc = orow_in ? graph_init_dag(&g, n, rp, col, orow_in, ocol_in) : graph_init(&g, n, rp, col);
    if (rc) { graph_free(&g); return rc; }
    if (kmax < 0) kmax = g.alpha + 1;
    if (!roots) nroots = n;
    int ovf = 0;
    uint32_t *binom = binom_table(g.alpha + 2, nl, &ovf);
    if (!binom) { graph_free(&g); return ORC_ENOMEM; }
    if (nthreads < 1) nthreads = 1;
    worker *wk = (worker *)calloc((size_t)nthreads, sizeof(worker));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int64_t next = 0;
    size_t Cw = (size_t)(kmax + 1) * nl;
    for (int t = 0; t < nthreads && !rc; ++t) {
        rc = walker_init(&wk[t].w, &g, kmax, nl, binom);
        wk[t].roots = roots;
        wk[t].nroots = nroots;
        wk[t].next = &next;
        if (C) {
            wk[t].w.C = (uint32_t *)calloc(Cw, sizeof(uint32_t));
            if (!wk[t].w.C) rc = ORC_ENOMEM;
        }
        wk[t].w.cv = cv;
        wk[t].w.ce = ce;
        if (hist) {
            wk[t].w.hist = (uint64_t *)calloc((size_t)hdim * hdim, sizeof(uint64_t));
            wk[t].w.hdim = hdim;
        }
    }
    if (!rc) {
        if (nthreads == 1) {
            worker_main(&wk[0]);
        } else {
            for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, worker_main, &wk[t]);
            for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
        }
    }
    uint64_t st[4] = {0, 0, 0, 0};
    for (int t = 0; t < nthreads; ++t) {
        walker *w = &wk[t].w;
        if (!rc && w->err) rc = w->err;
        if (w->ovf) ovf = 1;
        if (C && w->C)
            for (int k = 0; k <= kmax; ++k) big_add(C + (size_t)k * nl, w->C + (size_t)k * nl, nl, &ovf);
        st[0] += w->nodes;
        st[1] += w->leaves;
        st[2] += w->sum_s;
        st[3] += w->chain;
        if (hist && w->hist)
            for (size_t i = 0; i < (size_t)hdim * hdim; ++i) hist[i] += w->hist[i];
        free(w->C);
        free(w->hist);
        walker_free(w);
    }
    if (stats) {
        stats[0] = st[0];
        stats[1] = st[1];
        stats[2] = st[2];
        stats[3] = (uint64_t)g.alpha;
        stats[4] = (uint64_t)kmax;
        stats[5] = st[3];
    }
    free(wk);
    free(th);
    free(binom);
    graph_free(&g);
    if (!rc && ovf) rc = ORC_EOVERFLOW;
    return rc;
}

/* Leaf dump for tiny graphs: for every root-to-leaf path T, in walk order,
 * writes h, p, then the vertices of H(T), then those of P(T).  Returns the
 * number of int32 written, or -(error). */
int64_t orc_paths(int64_t n, const int64_t *rp, const uint32_t *col, int32_t *out, int64_t cap)
{
    graph g;
    int rc = graph_init(&g, n, rp, col);
    if (rc) { graph_free(&g); return -rc; }
    int ovf = 0;
    uint32_t *binom = binom_table(g.alpha + 2, 1, &ovf);
    walker w;
    rc = binom ? walker_init(&w, &g, g.alpha + 1, 1, binom) : ORC_ENOMEM;
    int64_t len = -1;
    if (!rc) {
        w.paths = out;
        w.pcap = cap;
        for (int64_t r = 0; r < n && !w.err; ++r) visit_root(&w, (uint32_t)r);
        len = w.err ? -(int64_t)w.err : w.plen;
        walker_free(&w);
    } else {
        len = -(int64_t)rc;
    }
    free(binom);
    graph_free(&g);
    return len;
}

/*
 * Triangles: the number of vertex triples that are pairwise adjacent, which
 * is C_3 of the k-clique counts (Sec. 2, k = 3).  Plain enumeration,
 * independent of the SCT code above: order the vertices by (degree, id),
 * keep for every vertex its neighbours later in that order (N+), and count
 * each triangle once, at its earliest vertex u, as a pair v -> w of N+(u)
 * with w in N+(v) (the "forward" algorithm of Schank and Wagner, 2005, with
 * a marker array over N+(u)).  Returns the count, or -1 for bad input or no
 * memory.
 */
static int later(const int64_t *rp, uint32_t a, uint32_t b)
{
    const int64_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
    return da < db || (da == db && a < b);
}

typedef struct {
    const int64_t *orow;
    const uint32_t *ocol;
    int64_t n, *next, count;
    uint8_t *mark;
} tri_worker;

static void *tri_main(void *arg)
{
    tri_worker *k = (tri_worker *)arg;
    for (;;) {
        const int64_t u0 = __atomic_fetch_add(k->next, 64, __ATOMIC_RELAXED);
        if (u0 >= k->n) break;
        const int64_t u1 = u0 + 64 < k->n ? u0 + 64 : k->n;
        for (int64_t u = u0; u < u1; ++u) {
            for (int64_t i = k->orow[u]; i < k->orow[u + 1]; ++i) k->mark[k->ocol[i]] = 1;
            for (int64_t i = k->orow[u]; i < k->orow[u + 1]; ++i) {
                const uint32_t v = k->ocol[i];
                for (int64_t j = k->orow[v]; j < k->orow[v + 1]; ++j) k->count += k->mark[k->ocol[j]];
            }
            for (int64_t i = k->orow[u]; i < k->orow[u + 1]; ++i) k->mark[k->ocol[i]] = 0;
        }
    }
    return NULL;
}

/* threads >= 1 split the vertices u in chunks of 64 (each thread its own
 * marker array and count, summed at the end). */
int64_t orc_triangles(int64_t n, const int64_t *rp, const uint32_t *col, int threads)
{
    if (n < 0 || (n > 0 && (!rp || !col)) || threads < 1) return -1;
    if (n == 0) return 0;
    int64_t *orow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint32_t *ocol = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
    tri_worker *wk = (tri_worker *)calloc((size_t)threads, sizeof(tri_worker));
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    int ok = orow && ocol && wk && th;
    for (int t = 0; ok && t < threads; ++t) ok = (wk[t].mark = (uint8_t *)calloc((size_t)n, 1)) != NULL;
    int64_t total = -1;
    if (ok) {
        orow[0] = 0;
        for (int64_t u = 0; u < n; ++u) {
            int64_t k = orow[u];
            for (int64_t i = rp[u]; i < rp[u + 1]; ++i)
                if (later(rp, (uint32_t)u, col[i])) ocol[k++] = col[i];
            orow[u + 1] = k;
        }
        int64_t next = 0;
        for (int t = 0; t < threads; ++t) {
            wk[t].orow = orow;
            wk[t].ocol = ocol;
            wk[t].n = n;
            wk[t].next = &next;
        }
        if (threads == 1) {
            tri_main(&wk[0]);
        } else {
            for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, tri_main, &wk[t]);
            for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
        }
        total = 0;
        for (int t = 0; t < threads; ++t) total += wk[t].count;
    }
    for (int t = 0; wk && t < threads; ++t) free(wk[t].mark);
    free(wk);
    free(th);
    free(orow);
    free(ocol);
    return total;
}
