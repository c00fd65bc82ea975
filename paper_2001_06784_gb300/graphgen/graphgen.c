/*
 * Seeded synthetic graph generators (host C).
 *
 * These stand in for the SNAP social and web networks the paper measures on
 * (Sec. 5, Tab. main): power-law Chung-Lu graphs, Erdos-Renyi graphs and
 * planted dense communities.  Everything here only produces inputs: a simple,
 * undirected graph in CSR form (Sec. "Problem Statement"), rows sorted, no
 * self-loops, no duplicate edges, every edge stored in both rows.  It holds
 * none of the clique-counting arithmetic and is shared, as an input source
 * only, by the CUDA library's tests and benchmarks and by the CPU oracle.
 *
 * Randomness: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), one sequential stream per generator call
 * seeded from (seed, salt).  Output depends only on the arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t state;
} gg_rng;

static uint64_t gg_next(gg_rng *r)
{
    uint64_t z = (r->state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void gg_seed(gg_rng *r, uint64_t seed, uint64_t salt)
{
    r->state = seed * 0xD1B54A32D192ED03ull + salt;
    (void)gg_next(r);
}

/* uniform double in [0, 1) with 53 random bits */
static double gg_unif(gg_rng *r) { return (double)(gg_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, k) (k > 0), by 128-bit multiply-shift */
static uint64_t gg_below(gg_rng *r, uint64_t k)
{
    return (uint64_t)(((unsigned __int128)gg_next(r) * k) >> 64);
}

/* ---------------------------------------------------------------- edge list */

typedef struct {
    int64_t n;
    uint64_t *keys; /* (min << 32) | max, min < max */
    int64_t len, cap;
    int64_t m;         /* after finish */
    int64_t *row_ptr;  /* after finish */
    uint32_t *col;     /* after finish */
    int64_t cl_m;      /* unique Chung-Lu edges drawn (last call) */
} gg_graph;

static int gg_push(gg_graph *g, uint32_t a, uint32_t b)
{
    if (a == b) return 0;
    if (a > b) { uint32_t t = a; a = b; b = t; }
    if (g->len == g->cap) {
        int64_t nc = g->cap ? g->cap * 2 : 1024;
        uint64_t *nk = (uint64_t *)realloc(g->keys, (size_t)nc * sizeof(uint64_t));
        if (!nk) return -1;
        g->keys = nk;
        g->cap = nc;
    }
    g->keys[g->len++] = ((uint64_t)a << 32) | b;
    return 0;
}

/* LSD radix sort of 64-bit keys with 16-bit digits, then in-place dedup.
 * Returns the number of unique keys, or -1 on allocation failure. */
static int64_t gg_sort_unique(uint64_t *a, int64_t len)
{
    if (len <= 1) return len;
    uint64_t *tmp = (uint64_t *)malloc((size_t)len * sizeof(uint64_t));
    int64_t *cnt = (int64_t *)malloc(65536 * sizeof(int64_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t maxk = 0;
    for (int64_t i = 0; i < len; ++i) if (a[i] > maxk) maxk = a[i];
    uint64_t *src = a, *dst = tmp;
    int passes = 0;
    for (int shift = 0; shift < 64 && (shift == 0 || (maxk >> shift)); shift += 16) {
        memset(cnt, 0, 65536 * sizeof(int64_t));
        for (int64_t i = 0; i < len; ++i) cnt[(src[i] >> shift) & 0xFFFF]++;
        int64_t s = 0;
        for (int d = 0; d < 65536; ++d) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (int64_t i = 0; i < len; ++i) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
        ++passes;
    }
    if (src != a) memcpy(a, src, (size_t)len * sizeof(uint64_t));
    free(tmp);
    free(cnt);
    int64_t u = 1;
    for (int64_t i = 1; i < len; ++i)
        if (a[i] != a[u - 1]) a[u++] = a[i];
    return u;
}

void *gg_begin(int64_t n)
{
    if (n < 0 || n > 0xFFFFFFFFll) return NULL;
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (g) g->n = n;
    return g;
}

void gg_free(void *h)
{
    gg_graph *g = (gg_graph *)h;
    if (!g) return;
    free(g->keys);
    free(g->row_ptr);
    free(g->col);
    free(g);
}

int gg_add_edge(void *h, uint32_t a, uint32_t b)
{
    gg_graph *g = (gg_graph *)h;
    if (a >= g->n || b >= g->n) return -2;
    return gg_push(g, a, b);
}

/* ------------------------------------------------------------- Erdos-Renyi */

/* G(n, p) with p = avg_deg / (n - 1): every pair independently, visited by
 * geometric skips over the pairs (w, v), w < v, in row order (Batagelj and
 * Brandes, "Efficient generation of large random networks", 2005). */
int gg_add_er(void *h, double avg_deg, uint64_t seed)
{
    gg_graph *g = (gg_graph *)h;
    int64_t n = g->n;
    if (n < 2 || avg_deg <= 0) return 0;
    double p = avg_deg / (double)(n - 1);
    if (p >= 1.0) {
        for (int64_t v = 1; v < n; ++v)
            for (int64_t w = 0; w < v; ++w)
                if (gg_push(g, (uint32_t)w, (uint32_t)v)) return -1;
        return 0;
    }
    gg_rng r;
    gg_seed(&r, seed, 0x45520001ull);
    double lq = log(1.0 - p);
    int64_t v = 1, w = -1;
    while (v < n) {
        double u = 1.0 - gg_unif(&r); /* (0, 1] */
        w += 1 + (int64_t)floor(log(u) / lq);
        while (w >= v && v < n) { w -= v; ++v; }
        if (v < n && gg_push(g, (uint32_t)w, (uint32_t)v)) return -1;
    }
    return 0;
}

/* -------------------------------------------------------------- Chung-Lu */

/* Power-law Chung-Lu graph with about m unique edges and degree exponent
 * beta > 1.  Weights w_i = c (i + i0)^(-1/(beta-1)), scaled so that they sum
 * to 2m; the offset i0 is the smallest for which the largest weight does not
 * exceed the structural cut-off sqrt(2m).  Endpoint pairs are drawn
 * independently in proportion to the weights (Walker/Vose alias table);
 * self-loops and repeats are dropped and draws continue until at least m
 * unique pairs exist. */
int gg_add_chung_lu(void *h, int64_t m, double beta, uint64_t seed)
{
    gg_graph *g = (gg_graph *)h;
    int64_t n = g->n;
    g->cl_m = 0;
    if (n < 2 || m <= 0) return 0;
    if (m > n * (n - 1) / 4) return -3; /* too dense for rejection drawing */
    double gam = 1.0 / (beta - 1.0);
    double cap = sqrt(2.0 * (double)m);
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *prob = (double *)malloc((size_t)n * sizeof(double));
    uint32_t *alias = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *stk = (uint32_t *)malloc((size_t)n * 2 * sizeof(uint32_t));
    uint64_t *keys = NULL;
    int rc = -1;
    if (!w || !prob || !alias || !stk) goto out;

    /* bisection for i0: max weight 2m * i0^-gam / sum_i (i+i0)^-gam <= cap */
    double lo = 1.0, hi = (double)n;
    for (int it = 0; it < 60; ++it) {
        double mid = 0.5 * (lo + hi), s = 0;
        for (int64_t i = 0; i < n; ++i) s += pow((double)i + mid, -gam);
        double w0 = 2.0 * (double)m * pow(mid, -gam) / s;
        if (w0 > cap) lo = mid; else hi = mid;
    }
    double s = 0;
    for (int64_t i = 0; i < n; ++i) { w[i] = pow((double)i + hi, -gam); s += w[i]; }

    /* Vose alias table over w / s */
    {
        uint32_t *small = stk, *large = stk + n;
        int64_t ns = 0, nl = 0;
        for (int64_t i = 0; i < n; ++i) {
            prob[i] = w[i] / s * (double)n;
            if (prob[i] < 1.0) small[ns++] = (uint32_t)i; else large[nl++] = (uint32_t)i;
        }
        while (ns && nl) {
            uint32_t a = small[--ns], b = large[--nl];
            alias[a] = b;
            prob[b] = (prob[b] + prob[a]) - 1.0;
            if (prob[b] < 1.0) small[ns++] = b; else large[nl++] = b;
        }
        while (nl) { uint32_t b = large[--nl]; prob[b] = 1.0; alias[b] = b; }
        while (ns) { uint32_t a = small[--ns]; prob[a] = 1.0; alias[a] = a; }
    }

    gg_rng r;
    gg_seed(&r, seed, 0x434C0001ull);
    int64_t have = 0, len = 0, cap_k = 0;
    int64_t want = m + m / 20 + 16;
    while (have < m) {
        int64_t need = len + want;
        if (need > cap_k) {
            uint64_t *nk = (uint64_t *)realloc(keys, (size_t)need * sizeof(uint64_t));
            if (!nk) goto out;
            keys = nk;
            cap_k = need;
        }
        for (int64_t t = 0; t < want; ++t) {
            uint32_t e[2];
            for (int j = 0; j < 2; ++j) {
                uint64_t i = gg_below(&r, (uint64_t)n);
                e[j] = gg_unif(&r) < prob[i] ? (uint32_t)i : alias[i];
            }
            if (e[0] == e[1]) continue;
            uint32_t a = e[0] < e[1] ? e[0] : e[1], b = e[0] < e[1] ? e[1] : e[0];
            keys[len++] = ((uint64_t)a << 32) | b;
        }
        len = gg_sort_unique(keys, len);
        if (len < 0) goto out;
        have = len;
        want = (m - have) + (m - have) / 2 + 16;
    }
    g->cl_m = have;
    for (int64_t i = 0; i < have; ++i)
        if (gg_push(g, (uint32_t)(keys[i] >> 32), (uint32_t)keys[i])) goto out;
    rc = 0;
out:
    free(w); free(prob); free(alias); free(stk); free(keys);
    return rc;
}

int64_t gg_last_chung_lu_edges(void *h) { return ((gg_graph *)h)->cl_m; }

/* --------------------------------------------------- planted communities */

/* `count` communities; each has a size drawn uniformly from [smin, smax], its
 * members are distinct vertices drawn uniformly, and each member pair is an
 * edge with probability rho (rho = 1 plants a clique).  Communities may
 * overlap one another and the background graph. */
int gg_add_planted(void *h, int64_t count, int smin, int smax, double rho, uint64_t seed)
{
    gg_graph *g = (gg_graph *)h;
    int64_t n = g->n;
    if (count <= 0) return 0;
    if (smin < 2 || smax < smin || smax > n) return -3;
    uint32_t *mem = (uint32_t *)malloc((size_t)smax * sizeof(uint32_t));
    if (!mem) return -1;
    gg_rng r;
    gg_seed(&r, seed, 0x504C0001ull);
    for (int64_t c = 0; c < count; ++c) {
        int s = smin + (int)gg_below(&r, (uint64_t)(smax - smin + 1));
        int k = 0;
        while (k < s) {
            uint32_t v = (uint32_t)gg_below(&r, (uint64_t)n);
            int dup = 0;
            for (int j = 0; j < k; ++j) if (mem[j] == v) { dup = 1; break; }
            if (!dup) mem[k++] = v;
        }
        for (int a = 0; a < s; ++a)
            for (int b = a + 1; b < s; ++b)
                if (rho >= 1.0 || gg_unif(&r) < rho)
                    if (gg_push(g, mem[a], mem[b])) { free(mem); return -1; }
    }
    free(mem);
    return 0;
}

/* ------------------------------------------------------------------- CSR */

/* Sort and deduplicate all edges and build the symmetric CSR.  Returns the
 * number of undirected edges m, or a negative value on failure. */
int64_t gg_finish(void *h)
{
    gg_graph *g = (gg_graph *)h;
    int64_t n = g->n;
    int64_t m = gg_sort_unique(g->keys, g->len);
    if (m < 0) return -1;
    g->len = m;
    g->m = m;
    g->row_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->col = (uint32_t *)malloc((size_t)(2 * m + 1) * sizeof(uint32_t));
    int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!g->row_ptr || !g->col || !fill) { free(fill); return -1; }
    for (int64_t i = 0; i < m; ++i) {
        g->row_ptr[(g->keys[i] >> 32) + 1]++;
        g->row_ptr[(g->keys[i] & 0xFFFFFFFFu) + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) g->row_ptr[v + 1] += g->row_ptr[v];
    memcpy(fill, g->row_ptr, ((size_t)n + 1) * sizeof(int64_t));
    /* keys are sorted by (a, b): appending in key order leaves every row
     * sorted (smaller neighbours arrive as second endpoints first). */
    for (int64_t i = 0; i < m; ++i) {
        uint32_t a = (uint32_t)(g->keys[i] >> 32), b = (uint32_t)g->keys[i];
        g->col[fill[a]++] = b;
        g->col[fill[b]++] = a;
    }
    free(fill);
    free(g->keys);
    g->keys = NULL;
    g->cap = 0;
    return m;
}

void gg_copy_csr(void *h, int64_t *row_ptr, uint32_t *col)
{
    gg_graph *g = (gg_graph *)h;
    memcpy(row_ptr, g->row_ptr, ((size_t)g->n + 1) * sizeof(int64_t));
    memcpy(col, g->col, (size_t)(2 * g->m) * sizeof(uint32_t));
}
