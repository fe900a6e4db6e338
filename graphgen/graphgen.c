/*
 * graphgen.c - seeded synthetic graph inputs (RMAT and Erdos-Renyi) as CSR.
 *
 * This is input plumbing shared by the tests, the benchmark, the oracle and the
 * CUDA path. It holds none of the PageRank / partition-centric arithmetic: it
 * only draws edges, relabels nodes and lays the result out as a compressed
 * sparse row (CSR) out-adjacency with every row sorted ascending, duplicates
 * and self-loops removed.
 *
 * Randomness is counter based so the result does not depend on the number of
 * threads: every draw is SplitMix64's output function (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a
 * (seed, stream, counter) triple.
 *
 * RMAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each edge descends `scale`
 * levels of the adjacency matrix, picking quadrant (0,0) with probability a,
 * (0,1) with b, (1,0) with c and (1,1) with 1-a-b-c; quadrant row bits form the
 * source, column bits the destination. No noise is added.
 *
 * Relabelings: RANDOM applies a uniformly random permutation (Fisher-Yates);
 * BFS applies RANDOM first and then numbers nodes in breadth-first order from
 * the node of highest out-degree (ties to the lower ID), following out-edges in
 * CSR order; nodes the search never reaches follow in increasing ID order.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_RELABEL_NONE 0
#define GG_RELABEL_RANDOM 1
#define GG_RELABEL_BFS 2

/* ------------------------------------------------------------------ RNG */
static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
    uint64_t key = sm64_mix(seed * 0x9E3779B97F4A7C15ULL + stream + 1);
    return sm64_mix(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}
/* uniform integer in [0, bound) by the high half of a 64x64 product */
static inline uint64_t below(uint64_t r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

/* ------------------------------------------------------------- threads */
typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void* ctx; uint64_t lo, hi; } job_t;
static void* job_run(void* p) { job_t* j = (job_t*)p; j->fn(j->ctx, j->lo, j->hi); return NULL; }

static void parallel_for(int threads, uint64_t n, range_fn fn, void* ctx) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > n) threads = n ? (int)n : 1;
    pthread_t tid[256];
    job_t jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * (uint64_t)t / threads;
        jobs[t].hi = n * (uint64_t)(t + 1) / threads;
    }
    for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, job_run, &jobs[t]);
    job_run(&jobs[0]);
    for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
}

/* --------------------------------------------------------- edge drawing */
typedef struct {
    int scale; double a, ab, abc; uint64_t seed;
    uint32_t* src; uint32_t* dst;
} rmat_ctx;

static void rmat_range(void* p, uint64_t lo, uint64_t hi) {
    rmat_ctx* c = (rmat_ctx*)p;
    const uint64_t words = (uint64_t)(c->scale + 1) / 2;
    const double inv32 = 1.0 / 4294967296.0;
    for (uint64_t e = lo; e < hi; ++e) {
        uint32_t u = 0, v = 0;
        uint64_t w = 0;
        for (int l = 0; l < c->scale; ++l) {
            if ((l & 1) == 0) w = draw(c->seed, 1, e * words + (uint64_t)(l >> 1));
            double r = (double)((l & 1) ? (uint32_t)(w >> 32) : (uint32_t)w) * inv32;
            uint32_t bit = 1u << (c->scale - 1 - l);
            if (r < c->a) {
            } else if (r < c->ab) {
                v |= bit;
            } else if (r < c->abc) {
                u |= bit;
            } else {
                u |= bit; v |= bit;
            }
        }
        c->src[e] = u; c->dst[e] = v;
    }
}

typedef struct { uint64_t n, seed; uint32_t* src; uint32_t* dst; } er_ctx;
static void er_range(void* p, uint64_t lo, uint64_t hi) {
    er_ctx* c = (er_ctx*)p;
    for (uint64_t e = lo; e < hi; ++e) {
        c->src[e] = (uint32_t)below(draw(c->seed, 3, 2 * e), c->n);
        c->dst[e] = (uint32_t)below(draw(c->seed, 3, 2 * e + 1), c->n);
    }
}

/* ---------------------------------------------------------- relabeling */
static void random_permutation(uint32_t* perm, uint64_t n, uint64_t seed) {
    for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    for (uint64_t i = n; i > 1; --i) {
        uint64_t j = below(draw(seed, 2, i), i);
        uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
    }
}

typedef struct { const uint32_t* lab; uint32_t* src; uint32_t* dst; } relabel_ctx;
static void relabel_range(void* p, uint64_t lo, uint64_t hi) {
    relabel_ctx* c = (relabel_ctx*)p;
    for (uint64_t e = lo; e < hi; ++e) { c->src[e] = c->lab[c->src[e]]; c->dst[e] = c->lab[c->dst[e]]; }
}

/* --------------------------------------------------- edge list -> CSR */
typedef struct {
    const uint32_t* src; const uint32_t* dst;
    uint32_t* deg;           /* n, atomically incremented */
    uint64_t* cursor;        /* n */
    uint32_t* col;           /* M (unsorted rows) */
} fill_ctx;

static void count_range(void* p, uint64_t lo, uint64_t hi) {
    fill_ctx* c = (fill_ctx*)p;
    for (uint64_t e = lo; e < hi; ++e) __atomic_fetch_add(&c->deg[c->src[e]], 1u, __ATOMIC_RELAXED);
}
static void place_range(void* p, uint64_t lo, uint64_t hi) {
    fill_ctx* c = (fill_ctx*)p;
    for (uint64_t e = lo; e < hi; ++e) {
        uint64_t pos = __atomic_fetch_add(&c->cursor[c->src[e]], 1ull, __ATOMIC_RELAXED);
        c->col[pos] = c->dst[e];
    }
}

static int cmp_u32(const void* x, const void* y) {
    uint32_t a = *(const uint32_t*)x, b = *(const uint32_t*)y;
    return (a > b) - (a < b);
}
static void sort_u32(uint32_t* v, uint64_t len) {
    if (len < 2) return;
    if (len <= 24) {
        for (uint64_t i = 1; i < len; ++i) {
            uint32_t x = v[i]; uint64_t j = i;
            while (j > 0 && v[j - 1] > x) { v[j] = v[j - 1]; --j; }
            v[j] = x;
        }
    } else {
        qsort(v, len, sizeof(uint32_t), cmp_u32);
    }
}

typedef struct {
    const uint64_t* start; uint32_t* col; uint32_t* newdeg; int dedupe, drop_self;
} rowsort_ctx;
static void rowsort_range(void* p, uint64_t lo, uint64_t hi) {
    rowsort_ctx* c = (rowsort_ctx*)p;
    for (uint64_t u = lo; u < hi; ++u) {
        uint32_t* row = c->col + c->start[u];
        uint64_t len = c->start[u + 1] - c->start[u];
        sort_u32(row, len);
        uint64_t w = 0;
        for (uint64_t i = 0; i < len; ++i) {
            if (c->drop_self && row[i] == (uint32_t)u) continue;
            if (c->dedupe && w > 0 && row[w - 1] == row[i]) continue;
            row[w++] = row[i];
        }
        c->newdeg[u] = (uint32_t)w;
    }
}

typedef struct {
    const uint64_t* start; const uint32_t* col; const uint32_t* row_ptr; uint32_t* out;
} compact_ctx;
static void compact_range(void* p, uint64_t lo, uint64_t hi) {
    compact_ctx* c = (compact_ctx*)p;
    for (uint64_t u = lo; u < hi; ++u)
        memcpy(c->out + c->row_ptr[u], c->col + c->start[u],
               (size_t)(c->row_ptr[u + 1] - c->row_ptr[u]) * sizeof(uint32_t));
}

/* Builds a CSR from an edge list; src/dst are consumed (freed by caller).
 * Returns 0 on success, -1 on allocation failure, -2 if the result has 2^32 or
 * more edges. */
static int edges_to_csr(uint64_t n, uint64_t M, const uint32_t* src, const uint32_t* dst,
                        int dedupe, int drop_self, int threads,
                        uint32_t** row_ptr_out, uint32_t** col_out, uint64_t* m_out) {
    uint32_t* deg = (uint32_t*)calloc(n + 1, sizeof(uint32_t));
    uint64_t* start = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    uint64_t* cursor = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    uint32_t* col = (uint32_t*)malloc((M ? M : 1) * sizeof(uint32_t));
    if (!deg || !start || !cursor || !col) { free(deg); free(start); free(cursor); free(col); return -1; }
    fill_ctx fc = {src, dst, deg, cursor, col};
    parallel_for(threads, M, count_range, &fc);
    start[0] = 0;
    for (uint64_t u = 0; u < n; ++u) start[u + 1] = start[u] + deg[u];
    memcpy(cursor, start, (n + 1) * sizeof(uint64_t));
    parallel_for(threads, M, place_range, &fc);
    free(cursor);
    rowsort_ctx rc = {start, col, deg, dedupe, drop_self};
    parallel_for(threads, n, rowsort_range, &rc);
    uint64_t m = 0;
    for (uint64_t u = 0; u < n; ++u) m += deg[u];
    if (m >= 0xFFFFFFFFull) { free(deg); free(start); free(col); return -2; }
    uint32_t* row_ptr = (uint32_t*)malloc((n + 1) * sizeof(uint32_t));
    uint32_t* out = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    if (!row_ptr || !out) { free(deg); free(start); free(col); free(row_ptr); free(out); return -1; }
    row_ptr[0] = 0;
    for (uint64_t u = 0; u < n; ++u) row_ptr[u + 1] = row_ptr[u] + deg[u];
    compact_ctx cc = {start, col, row_ptr, out};
    parallel_for(threads, n, compact_range, &cc);
    free(deg); free(start); free(col);
    *row_ptr_out = row_ptr; *col_out = out; *m_out = m;
    return 0;
}

/* BFS numbering from the highest out-degree node over a CSR graph. */
static int bfs_labels(uint64_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t* lab) {
    const uint32_t NONE = 0xFFFFFFFFu;
    uint32_t* queue = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!queue) return -1;
    for (uint64_t u = 0; u < n; ++u) lab[u] = NONE;
    uint64_t best = 0;
    for (uint64_t u = 1; u < n; ++u)
        if (row_ptr[u + 1] - row_ptr[u] > row_ptr[best + 1] - row_ptr[best]) best = u;
    uint64_t next = 0, head = 0, tail = 0;
    if (n) { lab[best] = (uint32_t)next++; queue[tail++] = (uint32_t)best; }
    while (head < tail) {
        uint32_t u = queue[head++];
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t v = col[e];
            if (lab[v] == NONE) { lab[v] = (uint32_t)next++; queue[tail++] = v; }
        }
    }
    for (uint64_t u = 0; u < n; ++u)
        if (lab[u] == NONE) lab[u] = (uint32_t)next++;
    free(queue);
    return 0;
}

typedef struct { const uint32_t* row_ptr; const uint32_t* col; uint32_t* src; uint32_t* dst; } expand_ctx;
static void expand_range(void* p, uint64_t lo, uint64_t hi) {
    expand_ctx* c = (expand_ctx*)p;
    for (uint64_t u = lo; u < hi; ++u)
        for (uint32_t e = c->row_ptr[u]; e < c->row_ptr[u + 1]; ++e) { c->src[e] = (uint32_t)u; c->dst[e] = c->col[e]; }
}

/* Shared tail of both generators: relabel, build CSR, optionally BFS-relabel. */
static int finish(uint64_t n, uint64_t M, uint32_t* src, uint32_t* dst, int relabel, uint64_t seed,
                  int threads, uint32_t** row_ptr, uint32_t** col, uint64_t* m) {
    if (relabel != GG_RELABEL_NONE) {
        uint32_t* perm = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
        if (!perm) return -1;
        random_permutation(perm, n, seed + 1);
        relabel_ctx rc = {perm, src, dst};
        parallel_for(threads, M, relabel_range, &rc);
        free(perm);
    }
    int rc = edges_to_csr(n, M, src, dst, 1, 1, threads, row_ptr, col, m);
    if (rc || relabel != GG_RELABEL_BFS) return rc;
    uint32_t* lab = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!lab) return -1;
    if (bfs_labels(n, *row_ptr, *col, lab)) { free(lab); return -1; }
    expand_ctx ec = {*row_ptr, *col, src, dst};
    parallel_for(threads, n, expand_range, &ec);
    uint64_t m1 = *m;
    relabel_ctx lc = {lab, src, dst};
    parallel_for(threads, m1, relabel_range, &lc);
    free(lab);
    free(*row_ptr); free(*col);
    return edges_to_csr(n, m1, src, dst, 0, 0, threads, row_ptr, col, m);
}

/* ------------------------------------------------------------- exports */
int gg_rmat(int scale, double edge_factor, double a, double b, double c, uint64_t seed,
            int relabel, int threads, uint32_t** row_ptr, uint32_t** col, uint64_t* m) {
    if (scale < 1 || scale > 31 || edge_factor <= 0 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -3;
    uint64_t n = 1ull << scale;
    uint64_t M = (uint64_t)(edge_factor * (double)n);
    uint32_t* src = (uint32_t*)malloc((M ? M : 1) * sizeof(uint32_t));
    uint32_t* dst = (uint32_t*)malloc((M ? M : 1) * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
    rmat_ctx ctx = {scale, a, a + b, a + b + c, seed, src, dst};
    parallel_for(threads, M, rmat_range, &ctx);
    int rc = finish(n, M, src, dst, relabel, seed, threads, row_ptr, col, m);
    free(src); free(dst);
    return rc;
}

int gg_er(uint64_t n, double mean_degree, uint64_t seed, int relabel, int threads,
          uint32_t** row_ptr, uint32_t** col, uint64_t* m) {
    if (n < 1 || n >= 0x80000000ull || mean_degree < 0) return -3;
    uint64_t M = (uint64_t)(mean_degree * (double)n);
    uint32_t* src = (uint32_t*)malloc((M ? M : 1) * sizeof(uint32_t));
    uint32_t* dst = (uint32_t*)malloc((M ? M : 1) * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
    er_ctx ctx = {n, seed, src, dst};
    parallel_for(threads, M, er_range, &ctx);
    int rc = finish(n, M, src, dst, relabel, seed, threads, row_ptr, col, m);
    free(src); free(dst);
    return rc;
}

/* Uniform doubles in [0, 1) from stream 4: used for seeded rank vectors. */
void gg_uniform(uint64_t count, uint64_t seed, double* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = (double)(draw(seed, 4, i) >> 11) * (1.0 / 9007199254740992.0);
}

void gg_free(void* p) { free(p); }
