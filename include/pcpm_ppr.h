/* pcpm_ppr.h - batched personalized PageRank over a PNG (C ABI).
 *
 * Not among the paper's experiments; it extends Eq. 1 and the scatter-gather
 * of Eq. 2 / Algorithms 3-4 from one rank vector to a block of
 * PCPM_PPR_COLS columns. Column j has its own teleport distribution t_j,
 * uniform over a set S_j of seed nodes:
 *
 *   R'[:, j] = (1 - d) t_j + d (A^T (R[:, j] * w) + D_j t_j)
 *   w(u) = 1 / |N_o(u)| (0 if u is dangling),  D_j = sum of R[u, j] over dangling u
 *
 * so the mass of dangling nodes returns to the column's own teleport and
 * every column keeps summing to 1. Iterations start from R = T.
 *
 * Data path, per iteration, with the PNG of pcpm_build (any part_size):
 *   scatter  every update of the PNG (one per node u and destination
 *            partition, Sec. 3.2) becomes a 256-byte row: the 64 values
 *            R[u, :] / |N_o(u)|, written at its bin position;
 *   gather   every destination v sums the rows of its in-entries (the same
 *            rows Algorithm 4 reads for v, summed per v instead of in bin
 *            order), adds the teleport term and writes R'[v, :]; the L1
 *            change and the dangling mass of each column are reduced in FP64.
 * Ranks and rows are FP32.
 *
 * Layouts: rank blocks are node-major, n rows of PCPM_PPR_COLS floats
 * (row v = the 64 columns of node v, 256 bytes). Status codes are those of
 * pcpm.h. All device memory comes from the library's pool (pcpm.h).
 */
#ifndef PCPM_PPR_H
#define PCPM_PPR_H

#include <stdint.h>

#include "pcpm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PCPM_PPR_COLS 64

typedef struct pcpm_ppr pcpm_ppr;

/* Creates a solver for the PNG `png` (borrowed: it must outlive the solver)
 * and PCPM_PPR_COLS teleport columns.
 *   seed_ptr  host, PCPM_PPR_COLS + 1 entries: column j's seeds are
 *             seed_idx[seed_ptr[j] .. seed_ptr[j+1]); seed_ptr[0] = 0.
 *   seed_idx  host node IDs; every column has at least one seed, all < n and
 *             distinct within the column.
 *   stream    the stream the index build runs on; synchronised before return.
 *   out       host; receives the solver (free with pcpm_ppr_free).
 * PCPM_EINVAL for a bad argument (a null pointer, an empty column, a seed >= n
 * or repeated in its column); PCPM_ENOMEM / PCPM_ECUDA from the device. */
int pcpm_ppr_create(pcpm_png* png, const uint32_t* seed_ptr, const uint32_t* seed_idx, void* stream,
                    pcpm_ppr** out);

/* Resets R to the teleport block T and runs `iters` >= 0 iterations on
 * `stream`, recording each column's L1 change per iteration on the device.
 * Does not synchronise. PCPM_EINVAL for a bad d (not in [0, 1)) or iters. */
int pcpm_ppr_run(pcpm_ppr* ppr, float d, int iters, void* stream);

/* Copies the L1 changes of the last run to host `out`: iters rows of
 * PCPM_PPR_COLS doubles (row i = iteration i + 1). Synchronises the run's
 * stream. PCPM_EINVAL if iters exceeds the last run's count. */
int pcpm_ppr_residuals(pcpm_ppr* ppr, double* out, int iters);

/* Copies the current ranks (n rows of PCPM_PPR_COLS floats) to device `out`
 * on `stream`. */
int pcpm_ppr_ranks(pcpm_ppr* ppr, float* out, void* stream);

/* Sizes: device bytes held by the solver, and destinations whose in-entries
 * are summed in several pieces (more than 1024 entries). Either may be NULL. */
int pcpm_ppr_info(const pcpm_ppr* ppr, uint64_t* device_bytes, uint32_t* split_destinations);

/* Waits for the device, then releases the solver. NULL is a no-op. */
void pcpm_ppr_free(pcpm_ppr* ppr);

#ifdef __cplusplus
}
#endif
#endif /* PCPM_PPR_H */
