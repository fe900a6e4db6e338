/*
 * pcpm_oracle.c - plain, slow, sequential FP64 reference for PCPM PageRank.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline / reference arm may load this. The CUDA library
 * shares no code, header, table or helper with this file.
 *
 * What it computes, with the passage of Lakhotia, Kannan and Prasanna,
 * "Accelerating PageRank using Partition-Centric Processing" (arXiv 1709.07122)
 * that each function follows:
 *
 *   oracle_pull_step    Eq. 1 (Sec. 2.1) applied in the pull direction of
 *                       Algorithm 1 to a range of destination nodes, keeping
 *                       PR and the scaled vector SPR (Table 1: SPR(v) =
 *                       PR(v)/|N_o(v)|) apart. Dangling nodes (no out-edges)
 *                       are a reading: the paper is silent, so either their
 *                       mass is spread uniformly over all nodes (default) or
 *                       it leaks, as Eq. 1 literally does.
 *   oracle_pagerank     oracle_pull_step over all nodes, iterated.
 *   oracle_pull_step_mt oracle_pull_step over all nodes with the destination
 *                       range cut into `threads` contiguous pieces, one POSIX
 *                       thread each (every y[v] is computed exactly as in the
 *                       sequential step; only the order in which the pieces'
 *                       L1 sums are added differs). oracle_pagerank_mt
 *                       iterates it. They exist to time the oracle on all host
 *                       cores and to make full-size checks finish in seconds.
 *   oracle_png_count    first scan of the PNG construction (Sec. 3.3): for each
 *                       source partition p and destination partition p', the
 *                       number of nodes of p with at least one out-neighbour in
 *                       p' (|N_i^p(p')|, one update each, Sec. 3.2) and the
 *                       number of edges from p into p'.
 *   oracle_png_fill     offsets (Sec. 3.1: a partition's offset into a bin is
 *                       what all lower-ID partitions write there) and the second
 *                       PNG scan, which fills the bins: the source node of every
 *                       update in update-bin order, and the destination IDs with
 *                       the most significant bit set on the first ID of every
 *                       message (Sec. 3.2).
 *   oracle_scatter_gather  Algorithm 3 (scatter over the PNG) followed by the
 *                       branch-avoiding gather of Algorithm 4, in FP64, giving
 *                       the sum of SPR over in-neighbours for every node.
 *   oracle_png_fill_weights  weighted graphs (Sec. 3.5): the edge weights
 *                       stored beside the destination IDs, in bin order.
 *   oracle_spmv         y(v) = sum over in-edges (u, v) of w(u, v) * x(u), the
 *                       weighted product the extension computes, by its plain
 *                       definition over the edges.
 *   oracle_weighted_gather  Algorithm 3 then Algorithm 4 with the weights read
 *                       in the gather and applied to each update (Sec. 3.5).
 *
 * Partitions are index ranges [i*q, (i+1)*q) (Sec. 3.1); the last one may be
 * shorter. Inputs are a CSR out-adjacency (row_ptr[n+1], col[m]) whose rows are
 * sorted ascending.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MSB 0x80000000u
#define ID_MASK 0x7FFFFFFFu

/* In-neighbour lists N_i(v) from the out-adjacency: the sources of the edges
 * into v are in_src[in_start[v] .. in_start[v+1]), in increasing source order.
 * in_start has n+1 entries, in_src m. */
void oracle_in_adjacency(uint32_t n, const uint32_t* row_ptr, const uint32_t* col,
                         uint32_t* in_start, uint32_t* in_src) {
    memset(in_start, 0, ((size_t)n + 1) * sizeof(uint32_t));
    for (uint32_t u = 0; u < n; ++u)
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) in_start[col[e] + 1] += 1;
    for (uint32_t v = 0; v < n; ++v) in_start[v + 1] += in_start[v];
    uint32_t* fill = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    memcpy(fill, in_start, (size_t)n * sizeof(uint32_t));
    for (uint32_t u = 0; u < n; ++u)
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) in_src[fill[col[e]]++] = u;
    free(fill);
}

/* Mass sitting on dangling nodes (no out-edges). */
double oracle_dangling_mass(uint32_t n, const uint32_t* row_ptr, const double* x) {
    double dangling = 0.0;
    for (uint32_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] == row_ptr[u]) dangling += x[u];
    return dangling;
}

/* One application of Eq. 1 (pull direction, Algorithm 1) to the destination
 * nodes v in [v_begin, v_end):
 *   y[v] = (1-d)/n + d * (sum_{u in N_i(v)} x[u]/|N_o(u)| + dangling/n).
 * `dangling` is the mass handed back uniformly (0 for the leaking reading).
 * Returns sum over the range of |y[v] - x[v]|. */
double oracle_pull_step(uint32_t n, const uint32_t* row_ptr, const uint32_t* in_start,
                        const uint32_t* in_src, double d, double dangling,
                        uint32_t v_begin, uint32_t v_end, const double* x, double* y) {
    double r = 0.0;
    for (uint32_t v = v_begin; v < v_end; ++v) {
        double temp = 0.0; /* sum of SPR over in-neighbours */
        for (uint32_t j = in_start[v]; j < in_start[v + 1]; ++j) {
            uint32_t u = in_src[j];
            temp += x[u] / (double)(row_ptr[u + 1] - row_ptr[u]);
        }
        y[v] = (1.0 - d) / (double)n + d * (temp + dangling / (double)n);
        r += fabs(y[v] - x[v]);
    }
    return r;
}

struct pull_piece {
    uint32_t n;
    const uint32_t *row_ptr, *in_start, *in_src;
    double d, dangling;
    uint32_t v_begin, v_end;
    const double* x;
    double* y;
    double r;
};

static void* pull_piece_run(void* arg) {
    struct pull_piece* a = (struct pull_piece*)arg;
    a->r = oracle_pull_step(a->n, a->row_ptr, a->in_start, a->in_src, a->d, a->dangling, a->v_begin, a->v_end,
                            a->x, a->y);
    return NULL;
}

/* oracle_pull_step over the destinations [v_begin, v_end) on `threads`
 * threads (contiguous pieces of the range); the pieces' L1 sums are added in
 * range order. Returns the L1 change over the range. */
double oracle_pull_step_mt(uint32_t n, const uint32_t* row_ptr, const uint32_t* in_start, const uint32_t* in_src,
                           double d, double dangling, uint32_t v_begin, uint32_t v_end, const double* x, double* y,
                           int threads) {
    if (threads < 1) threads = 1;
    if (threads > 512) threads = 512;
    struct pull_piece pieces[512];
    pthread_t tid[512];
    int started[512];
    for (int i = 0; i < threads; ++i) {
        const uint64_t len = v_end > v_begin ? (uint64_t)(v_end - v_begin) : 0;
        struct pull_piece a = {n, row_ptr, in_start, in_src, d, dangling,
                               v_begin + (uint32_t)(len * i / threads), v_begin + (uint32_t)(len * (i + 1) / threads),
                               x, y, 0.0};
        pieces[i] = a;
    }
    for (int i = 1; i < threads; ++i) started[i] = pthread_create(&tid[i], NULL, pull_piece_run, &pieces[i]) == 0;
    pull_piece_run(&pieces[0]);
    double r = pieces[0].r;
    for (int i = 1; i < threads; ++i) {
        if (started[i]) pthread_join(tid[i], NULL);
        else pull_piece_run(&pieces[i]); /* run it here instead */
        r += pieces[i].r;
    }
    return r;
}

/* Eq. 1 iterated `iters` times from x0 (uniform 1/n when x0 is NULL), the
 * pull step on `threads` threads (oracle_pagerank: one).
 * x_hist, when not NULL, receives (iters+1) vectors of n doubles: x_0 .. x_iters.
 * resid[i-1] = sum_v |x_i(v) - x_{i-1}(v)|. Returns 0, or -1 on allocation failure. */
int oracle_pagerank_mt(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, double d,
                       int dangling_uniform, int iters, const double* x0,
                       double* x_hist, double* x_out, double* resid, int threads) {
    uint64_t m = row_ptr[n];
    uint32_t* in_start = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t* in_src = (uint32_t*)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    double* x = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* y = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    if (!in_start || !in_src || !x || !y) {
        free(in_start); free(in_src); free(x); free(y);
        return -1;
    }
    oracle_in_adjacency(n, row_ptr, col, in_start, in_src);
    for (uint32_t v = 0; v < n; ++v) x[v] = x0 ? x0[v] : 1.0 / (double)n;
    if (x_hist) memcpy(x_hist, x, (size_t)n * sizeof(double));
    for (int it = 1; it <= iters; ++it) {
        double dangling = dangling_uniform ? oracle_dangling_mass(n, row_ptr, x) : 0.0;
        double r = threads > 1 ? oracle_pull_step_mt(n, row_ptr, in_start, in_src, d, dangling, 0, n, x, y, threads)
                               : oracle_pull_step(n, row_ptr, in_start, in_src, d, dangling, 0, n, x, y);
        if (resid) resid[it - 1] = r;
        double* t = x; x = y; y = t;
        if (x_hist) memcpy(x_hist + (size_t)it * n, x, (size_t)n * sizeof(double));
    }
    if (x_out) memcpy(x_out, x, (size_t)n * sizeof(double));
    free(in_start); free(in_src); free(x); free(y);
    return 0;
}

int oracle_pagerank(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, double d,
                    int dangling_uniform, int iters, const double* x0,
                    double* x_hist, double* x_out, double* resid) {
    return oracle_pagerank_mt(n, row_ptr, col, d, dangling_uniform, iters, x0, x_hist, x_out, resid, 1);
}

/* First PNG scan. cnt_u and cnt_e are k*k arrays (row = source partition p,
 * column = destination partition p'), zeroed here. A node contributes one
 * update to p' for its first out-edge into p'; the other edges into p' are the
 * "unused" ones of Sec. 3.2 and only add destination IDs. */
void oracle_png_count(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t q,
                      uint32_t* cnt_u, uint32_t* cnt_e) {
    uint32_t k = (n + q - 1) / q;
    memset(cnt_u, 0, (size_t)k * k * sizeof(uint32_t));
    memset(cnt_e, 0, (size_t)k * k * sizeof(uint32_t));
    for (uint32_t p = 0; p < k; ++p) {
        uint32_t u_end = (p + 1) * (uint64_t)q < n ? (p + 1) * q : n;
        for (uint32_t u = p * q; u < u_end; ++u) {
            uint32_t prev_bin = UINT32_MAX;
            for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                uint32_t bin = col[e] / q;
                if (bin != prev_bin) { cnt_u[(size_t)p * k + bin] += 1; prev_bin = bin; }
                cnt_e[(size_t)p * k + bin] += 1;
            }
        }
    }
}

/* Offsets and the second PNG scan.
 *   off_u[p][p'] = sum over partitions p~ < p of cnt_u[p~][p']  (Sec. 3.1)
 *   bin_u[p']    = start of update_bins[p'] in one array holding all bins in
 *                  partition order; bin_u[k] = |E'|. off_e and bin_e likewise for
 *                  the destination-ID bins, bin_e[k] = m.
 *   src_idx[bin_u[p'] + off_u[p][p'] + j] = the j-th node of partition p (in ID
 *                  order) with an out-neighbour in p': the node whose value the
 *                  scatter inserts at that position.
 *   dest_ids       for each such node, its out-neighbours in p' in adjacency
 *                  order, the first with the MSB set.                        */
void oracle_png_fill(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t q,
                     const uint32_t* cnt_u, const uint32_t* cnt_e,
                     uint32_t* off_u, uint32_t* off_e, uint32_t* bin_u, uint32_t* bin_e,
                     uint32_t* src_idx, uint32_t* dest_ids) {
    uint32_t k = (n + q - 1) / q;
    /* Offsets: partitions write to every bin in the order of their IDs. */
    for (uint32_t pd = 0; pd < k; ++pd) {
        uint32_t su = 0, se = 0;
        for (uint32_t p = 0; p < k; ++p) {
            off_u[(size_t)p * k + pd] = su;
            off_e[(size_t)p * k + pd] = se;
            su += cnt_u[(size_t)p * k + pd];
            se += cnt_e[(size_t)p * k + pd];
        }
        bin_u[pd + 1] = su; /* bin sizes for now, prefix-summed below */
        bin_e[pd + 1] = se;
    }
    bin_u[0] = 0;
    bin_e[0] = 0;
    for (uint32_t pd = 0; pd < k; ++pd) {
        bin_u[pd + 1] += bin_u[pd];
        bin_e[pd + 1] += bin_e[pd];
    }
    /* Second scan: write cursors start at each partition's offsets. */
    uint32_t* cur_u = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
    uint32_t* cur_e = (uint32_t*)malloc((size_t)k * sizeof(uint32_t));
    for (uint32_t p = 0; p < k; ++p) {
        for (uint32_t pd = 0; pd < k; ++pd) {
            cur_u[pd] = bin_u[pd] + off_u[(size_t)p * k + pd];
            cur_e[pd] = bin_e[pd] + off_e[(size_t)p * k + pd];
        }
        uint32_t u_end = (p + 1) * (uint64_t)q < n ? (p + 1) * q : n;
        for (uint32_t u = p * q; u < u_end; ++u) {
            uint32_t prev_bin = UINT32_MAX;
            for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                uint32_t v = col[e];
                uint32_t bin = v / q;
                if (bin != prev_bin) {
                    src_idx[cur_u[bin]++] = u;
                    dest_ids[cur_e[bin]++] = v | MSB;
                    prev_bin = bin;
                } else {
                    dest_ids[cur_e[bin]++] = v;
                }
            }
        }
    }
    free(cur_u);
    free(cur_e);
}

/* Algorithm 3 then Algorithm 4 over the bins above, in FP64.
 * update[t] = spr[src_idx[t]]; then for every bin, walk its destination IDs,
 * advancing the update pointer by the MSB of each ID (branch avoidance). The
 * pointer starts one before the bin's first update, so the first (flagged) ID
 * reads the bin's first update. y[v] receives sum over in-neighbours u of spr[u]. */
void oracle_scatter_gather(uint32_t n, uint32_t k, const uint32_t* bin_u, const uint32_t* bin_e,
                           const uint32_t* src_idx, const uint32_t* dest_ids,
                           const double* spr, double* y) {
    uint32_t ne = bin_u[k];
    double* update = (double*)malloc((size_t)(ne ? ne : 1) * sizeof(double));
    for (uint32_t t = 0; t < ne; ++t) update[t] = spr[src_idx[t]]; /* scatter */
    for (uint32_t v = 0; v < n; ++v) y[v] = 0.0;
    for (uint32_t p = 0; p < k; ++p) { /* gather */
        int64_t update_ptr = (int64_t)bin_u[p] - 1;
        for (uint32_t j = bin_e[p]; j < bin_e[p + 1]; ++j) {
            uint32_t id = dest_ids[j];
            update_ptr += id >> 31;
            y[id & ID_MASK] += update[update_ptr];
        }
    }
    free(update);
}

/* Weighted graphs (Sec. 3.5): the weight of every edge goes to the position
 * its destination ID takes in the bins (the second PNG scan, same cursors).
 * weights[m] in CSR order; wbin[m] receives them in bin order. */
void oracle_png_fill_weights(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t q,
                             const uint32_t* off_e, const uint32_t* bin_e, const double* weights, double* wbin) {
    uint32_t k = (n + q - 1) / q;
    uint32_t* cur_e = (uint32_t*)malloc((size_t)(k ? k : 1) * sizeof(uint32_t));
    for (uint32_t p = 0; p < k; ++p) {
        for (uint32_t pd = 0; pd < k; ++pd) cur_e[pd] = bin_e[pd] + off_e[(size_t)p * k + pd];
        uint32_t u_end = (p + 1) * (uint64_t)q < n ? (p + 1) * q : n;
        for (uint32_t u = p * q; u < u_end; ++u)
            for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) wbin[cur_e[col[e] / q]++] = weights[e];
    }
    free(cur_e);
}

/* y(v) = sum over edges (u, v) of w(u, v) * x(u), in FP64, by the definition:
 * one pass over the out-adjacency. */
void oracle_spmv(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const double* weights,
                 const double* x, double* y) {
    memset(y, 0, (size_t)n * sizeof(double));
    for (uint32_t u = 0; u < n; ++u)
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) y[col[e]] += weights[e] * x[u];
}

/* Sec. 3.5, a non-square matrix A (n_rows x n_cols) in CSR:
 * y(c) = sum over the entries (r, c) of w * x(r), for c < n_cols. */
void oracle_spmv_rect(uint32_t n_rows, uint32_t n_cols, const uint32_t* row_ptr, const uint32_t* col,
                      const double* weights, const double* x, double* y) {
    memset(y, 0, (size_t)n_cols * sizeof(double));
    for (uint32_t r = 0; r < n_rows; ++r)
        for (uint32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) y[col[e]] += weights[e] * x[r];
}

/* Sec. 3.5 with Algorithms 3 and 4: update[t] = x[src_idx[t]]; the gather
 * walks each bin's IDs with the update pointer of Algorithm 4 and adds
 * weight * update to the destination. */
void oracle_weighted_gather(uint32_t n, uint32_t k, const uint32_t* bin_u, const uint32_t* bin_e,
                            const uint32_t* src_idx, const uint32_t* dest_ids, const double* wbin,
                            const double* x, double* y) {
    uint32_t ne = bin_u[k];
    double* update = (double*)malloc((size_t)(ne ? ne : 1) * sizeof(double));
    for (uint32_t t = 0; t < ne; ++t) update[t] = x[src_idx[t]];
    memset(y, 0, (size_t)n * sizeof(double));
    for (uint32_t pd = 0; pd < k; ++pd) {
        int64_t ptr = (int64_t)bin_u[pd] - 1;
        for (uint32_t j = bin_e[pd]; j < bin_e[pd + 1]; ++j) {
            ptr += dest_ids[j] >> 31;
            y[dest_ids[j] & ID_MASK] += wbin[j] * update[ptr];
        }
    }
    free(update);
}
