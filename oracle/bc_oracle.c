/*
 * bc_oracle.c -- plain CPU oracle for betweenness centrality (test infrastructure).
 *
 * This file is test infrastructure only.  It is called by the tests, by the smoke
 * check and by the benchmark's CPU-baseline leg; the CUDA library never links or
 * calls it, and it shares no code with the CUDA library.
 *
 * What it computes is the plain static definition, recomputed from scratch on the
 * current graph: the incremental method of the paper (Algorithm 3, Lemma 2, Lemma 4)
 * claims to reach exactly this state, so this is the oracle for it.
 *
 *   * d(s,t): Dijkstra from every source s (Section 2, Algorithm 7 step 3), in int64.
 *   * P_s(t) = { a : (a,t) in E and d(s,t) = d(s,a) + w(a,t) }         (Eq. 1)
 *   * sigma_ss = 1, sigma_st = sum over a in P_s(t) of sigma_sa, taken over the
 *     vertices in non-decreasing distance (Section 2; Algorithm 6 step 7), in uint64
 *     with every addition checked for overflow.
 *   * delta_s.(v) by Algorithm 1 (Accumulate-dependency): vertices are popped in
 *     non-increasing distance; each popped w pushes sigma_sv / sigma_sw * (1 +
 *     delta_s.(w)) to every v in P_s(w)  (Eq. 4); BC(w) += delta_s.(w) for w != s.
 *   * Undirected graphs are run on G_D (Section 3, "Undirected graphs": every edge
 *     {a,b} becomes (a,b) and (b,a)) and BC is halved, so that each unordered pair
 *     {s,t} is counted once (Eq. 3 summed over unordered pairs).
 *
 * Conventions (readings where the paper is silent):
 *   * unreachable t: d = INT64_MAX, sigma = 0, and the pair contributes nothing;
 *   * Delta[s][s] = 0 and Delta[s][t] = delta_s.(t) otherwise;
 *   * BC is the raw sum of Eq. 3 (no normalisation).
 *
 * Errors: ORACLE_ERR_OVERFLOW when a path count needs more than 64 bits,
 * ORACLE_ERR_DIST_OVERFLOW when a distance needs more than 63 bits, ORACLE_ERR_ARG
 * for a malformed graph (vertex out of range, self-loop, weight < 1, repeated edge).
 *
 * Threads: sources are split into contiguous blocks, one per thread; each thread
 * keeps a private BC vector and the vectors are added in thread order.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_OVERFLOW (-3)
#define ORACLE_ERR_DIST_OVERFLOW (-4)
#define ORACLE_ERR_OOM (-5)

#define INF INT64_MAX

typedef struct {
    int32_t n;
    int32_t *out_off, *out_dst; int64_t *out_w;   /* out-adjacency (CSR) */
    int32_t *in_off, *in_src;   int64_t *in_w;    /* in-adjacency (CSR)  */
} graph_t;

static void graph_free(graph_t *g) {
    free(g->out_off); free(g->out_dst); free(g->out_w);
    free(g->in_off); free(g->in_src); free(g->in_w);
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Build G (or G_D for an undirected graph) as out- and in-adjacency arrays. */
static int graph_build(graph_t *g, int32_t n, int32_t directed, int64_t m,
                       const int32_t *src, const int32_t *dst, const int64_t *w) {
    memset(g, 0, sizeof(*g));
    g->n = n;
    if (n < 0 || m < 0) return ORACLE_ERR_ARG;
    int64_t arcs = directed ? m : 2 * m;
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)(arcs > 0 ? arcs : 1));
    if (!keys) return ORACLE_ERR_OOM;
    for (int64_t i = 0; i < m; i++) {
        int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b || w[i] < 1) { free(keys); return ORACLE_ERR_ARG; }
        keys[directed ? i : 2 * i] = (int64_t)a * n + b;
        if (!directed) keys[2 * i + 1] = (int64_t)b * n + a;
    }
    qsort(keys, (size_t)arcs, sizeof(int64_t), cmp_i64);
    for (int64_t i = 1; i < arcs; i++)
        if (keys[i] == keys[i - 1]) { free(keys); return ORACLE_ERR_ARG; }
    free(keys);

    g->out_off = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->in_off = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->out_dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(arcs + 1));
    g->out_w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(arcs + 1));
    g->in_src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(arcs + 1));
    g->in_w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(arcs + 1));
    if (!g->out_off || !g->in_off || !g->out_dst || !g->out_w || !g->in_src || !g->in_w) {
        graph_free(g); return ORACLE_ERR_OOM;
    }
    for (int64_t i = 0; i < m; i++) {
        g->out_off[src[i] + 1]++; g->in_off[dst[i] + 1]++;
        if (!directed) { g->out_off[dst[i] + 1]++; g->in_off[src[i] + 1]++; }
    }
    for (int32_t v = 0; v < n; v++) { g->out_off[v + 1] += g->out_off[v]; g->in_off[v + 1] += g->in_off[v]; }
    int32_t *po = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *pi = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!po || !pi) { free(po); free(pi); graph_free(g); return ORACLE_ERR_OOM; }
    memcpy(po, g->out_off, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(pi, g->in_off, sizeof(int32_t) * ((size_t)n + 1));
    for (int64_t i = 0; i < m; i++) {
        int32_t a = src[i], b = dst[i];
        g->out_dst[po[a]] = b; g->out_w[po[a]++] = w[i];
        g->in_src[pi[b]] = a;  g->in_w[pi[b]++] = w[i];
        if (!directed) {
            g->out_dst[po[b]] = a; g->out_w[po[b]++] = w[i];
            g->in_src[pi[a]] = b;  g->in_w[pi[a]++] = w[i];
        }
    }
    free(po); free(pi);
    return ORACLE_OK;
}

/* ---- binary min-heap of (distance, vertex) with lazy deletion ---- */
typedef struct { int64_t d; int32_t v; } hitem;
typedef struct { hitem *a; int64_t size, cap; } heap_t;

static int heap_less(hitem x, hitem y) { return x.d < y.d || (x.d == y.d && x.v < y.v); }

static int heap_push(heap_t *h, int64_t d, int32_t v) {
    if (h->size == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 64;
        hitem *na = (hitem *)realloc(h->a, sizeof(hitem) * (size_t)nc);
        if (!na) return ORACLE_ERR_OOM;
        h->a = na; h->cap = nc;
    }
    int64_t i = h->size++;
    h->a[i].d = d; h->a[i].v = v;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_less(h->a[i], h->a[p])) break;
        hitem t = h->a[i]; h->a[i] = h->a[p]; h->a[p] = t; i = p;
    }
    return ORACLE_OK;
}

static hitem heap_pop(heap_t *h) {
    hitem top = h->a[0];
    h->a[0] = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < h->size && heap_less(h->a[l], h->a[b])) b = l;
        if (r < h->size && heap_less(h->a[r], h->a[b])) b = r;
        if (b == i) break;
        hitem t = h->a[i]; h->a[i] = h->a[b]; h->a[b] = t; i = b;
    }
    return top;
}

/* Per-thread work space for one source at a time. */
typedef struct {
    int64_t *d; uint64_t *sigma; double *delta;
    int32_t *order;      /* vertices in the order Dijkstra settles them */
    uint8_t *settled;
    heap_t heap;
} ws_t;

static int ws_init(ws_t *ws, int32_t n) {
    memset(ws, 0, sizeof(*ws));
    size_t k = (size_t)(n > 0 ? n : 1);
    ws->d = (int64_t *)malloc(sizeof(int64_t) * k);
    ws->sigma = (uint64_t *)malloc(sizeof(uint64_t) * k);
    ws->delta = (double *)malloc(sizeof(double) * k);
    ws->order = (int32_t *)malloc(sizeof(int32_t) * k);
    ws->settled = (uint8_t *)malloc(k);
    if (!ws->d || !ws->sigma || !ws->delta || !ws->order || !ws->settled) return ORACLE_ERR_OOM;
    return ORACLE_OK;
}

static void ws_free(ws_t *ws) {
    free(ws->d); free(ws->sigma); free(ws->delta); free(ws->order); free(ws->settled);
    free(ws->heap.a);
}

/*
 * One source of Brandes' algorithm (Algorithm 7 body):
 *   1. Dijkstra gives d(s,.) and the settle order (non-decreasing d);
 *   2. sigma from Eq. 1 predecessors in settle order;
 *   3. Algorithm 1 in reverse settle order gives delta_s.; bc[w] += delta_s.(w), w != s.
 * *nsettled receives the number of reachable vertices.
 */
static int brandes_source(const graph_t *g, int32_t s, ws_t *ws, double *bc, int32_t *nsettled) {
    const int32_t n = g->n;
    for (int32_t v = 0; v < n; v++) { ws->d[v] = INF; ws->sigma[v] = 0; ws->delta[v] = 0.0; ws->settled[v] = 0; }
    ws->heap.size = 0;
    ws->d[s] = 0;
    int rc = heap_push(&ws->heap, 0, s);
    if (rc) return rc;
    int32_t cnt = 0;
    while (ws->heap.size > 0) {
        hitem it = heap_pop(&ws->heap);
        int32_t a = it.v;
        if (ws->settled[a] || it.d != ws->d[a]) continue;   /* stale entry */
        ws->settled[a] = 1;
        ws->order[cnt++] = a;
        for (int32_t e = g->out_off[a]; e < g->out_off[a + 1]; e++) {
            int32_t b = g->out_dst[e];
            int64_t wt = g->out_w[e];
            if (ws->d[a] > INF - 1 - wt) return ORACLE_ERR_DIST_OVERFLOW;
            int64_t nd = ws->d[a] + wt;
            if (nd < ws->d[b]) {
                ws->d[b] = nd;
                rc = heap_push(&ws->heap, nd, b);
                if (rc) return rc;
            }
        }
    }
    /* sigma_st = sum of sigma_sa over a in P_s(t) (Eq. 1), in settle order. */
    ws->sigma[s] = 1;
    for (int32_t i = 1; i < cnt; i++) {
        int32_t t = ws->order[i];
        uint64_t acc = 0;
        for (int32_t e = g->in_off[t]; e < g->in_off[t + 1]; e++) {
            int32_t a = g->in_src[e];
            if (ws->d[a] != INF && ws->d[a] + g->in_w[e] == ws->d[t]) {
                if (__builtin_add_overflow(acc, ws->sigma[a], &acc)) return ORACLE_ERR_OVERFLOW;
            }
        }
        ws->sigma[t] = acc;
    }
    /* Algorithm 1: pop w in non-increasing d; push to every v in P_s(w) (Eq. 4). */
    for (int32_t i = cnt - 1; i >= 0; i--) {
        int32_t x = ws->order[i];
        for (int32_t e = g->in_off[x]; e < g->in_off[x + 1]; e++) {
            int32_t v = g->in_src[e];
            if (ws->d[v] != INF && ws->d[v] + g->in_w[e] == ws->d[x])
                ws->delta[v] += ((double)ws->sigma[v] / (double)ws->sigma[x]) * (1.0 + ws->delta[x]);
        }
        if (x != s && bc) bc[x] += ws->delta[x];
    }
    ws->delta[s] = 0.0;
    if (nsettled) *nsettled = cnt;
    return ORACLE_OK;
}

typedef struct {
    const graph_t *g;
    const int32_t *sources; int32_t nsrc;     /* NULL sources = all vertices */
    int32_t lo, hi;                           /* index range into sources */
    int64_t *D; uint64_t *SIG; double *DEL;   /* rows indexed by position in sources */
    double *bc;                               /* private BC (n) */
    int rc;
} job_t;

static void *run_job(void *p) {
    job_t *j = (job_t *)p;
    const int32_t n = j->g->n;
    ws_t ws;
    j->rc = ws_init(&ws, n);
    for (int32_t i = j->lo; i < j->hi && j->rc == ORACLE_OK; i++) {
        int32_t s = j->sources ? j->sources[i] : i;
        j->rc = brandes_source(j->g, s, &ws, j->bc, NULL);
        if (j->rc) break;
        size_t off = (size_t)i * (size_t)n;
        if (j->D) memcpy(j->D + off, ws.d, sizeof(int64_t) * (size_t)n);
        if (j->SIG) memcpy(j->SIG + off, ws.sigma, sizeof(uint64_t) * (size_t)n);
        if (j->DEL) memcpy(j->DEL + off, ws.delta, sizeof(double) * (size_t)n);
    }
    ws_free(&ws);
    return NULL;
}

/*
 * Static Brandes over the sources sources[0..nsrc) (all vertices when sources is NULL).
 * Row i of D / SIG / DEL (each optional, n entries per row) belongs to sources[i].
 * BC (optional, n doubles) receives the sum over these sources of delta_s.(v), v != s,
 * halved for an undirected graph -- with all sources this is Eq. 3.
 */
int oracle_brandes_sources(int32_t n, int32_t directed, int64_t m, const int32_t *src,
                           const int32_t *dst, const int64_t *w, int32_t nsrc,
                           const int32_t *sources, int64_t *D, uint64_t *SIG, double *DEL,
                           double *BC, int32_t nthreads) {
    graph_t g;
    int rc = graph_build(&g, n, directed, m, src, dst, w);
    if (rc) { graph_free(&g); return rc; }
    if (!sources) nsrc = n;
    for (int32_t i = 0; sources && i < nsrc; i++)
        if (sources[i] < 0 || sources[i] >= n) { graph_free(&g); return ORACLE_ERR_ARG; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nsrc) nthreads = nsrc > 0 ? nsrc : 1;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); graph_free(&g); return ORACLE_ERR_OOM; }
    for (int32_t t = 0; t < nthreads; t++) {
        jobs[t].g = &g; jobs[t].sources = sources; jobs[t].nsrc = nsrc;
        jobs[t].lo = (int32_t)((int64_t)nsrc * t / nthreads);
        jobs[t].hi = (int32_t)((int64_t)nsrc * (t + 1) / nthreads);
        jobs[t].D = D; jobs[t].SIG = SIG; jobs[t].DEL = DEL;
        jobs[t].bc = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        if (!jobs[t].bc) rc = ORACLE_ERR_OOM;
    }
    int started = 0;
    if (!rc) {
        for (int32_t t = 0; t < nthreads; t++) {
            if (pthread_create(&th[t], NULL, run_job, &jobs[t]) != 0) { rc = ORACLE_ERR_OOM; break; }
            started++;
        }
    }
    for (int32_t t = 0; t < started; t++) pthread_join(th[t], NULL);
    for (int32_t t = 0; t < nthreads && !rc; t++) if (jobs[t].rc) rc = jobs[t].rc;
    if (!rc && BC) {
        for (int32_t v = 0; v < n; v++) BC[v] = 0.0;
        for (int32_t t = 0; t < nthreads; t++)
            for (int32_t v = 0; v < n; v++) BC[v] += jobs[t].bc[v];
        if (!directed)
            for (int32_t v = 0; v < n; v++) BC[v] *= 0.5;
    }
    for (int32_t t = 0; t < nthreads; t++) free(jobs[t].bc);
    free(jobs); free(th);
    graph_free(&g);
    return rc;
}

/* Full static state: D, SIG, DEL are n*n row-major (each optional), BC is n. */
int oracle_brandes(int32_t n, int32_t directed, int64_t m, const int32_t *src, const int32_t *dst,
                   const int64_t *w, int64_t *D, uint64_t *SIG, double *DEL, double *BC,
                   int32_t nthreads) {
    return oracle_brandes_sources(n, directed, m, src, dst, w, n, NULL, D, SIG, DEL, BC, nthreads);
}
