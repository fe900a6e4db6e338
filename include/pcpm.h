/*
 * pcpm.h - C ABI of the GB300 (sm_103a) Partition-Centric PageRank library.
 *
 * Method: Lakhotia, Kannan, Prasanna, "Accelerating PageRank using
 * Partition-Centric Processing" (arXiv 1709.07122). One PageRank iteration is
 * Eq. 1 of Sec. 2.1,
 *     PR_{i+1}(v) = (1-d)/|V| + d * sum_{u in N_i(v)} PR_i(u)/|N_o(u)|,
 * computed as the sparse product A^T * SPR of Eq. 2 (SPR(u) = PR(u)/|N_o(u)|,
 * Table 1) in two phases over index-range partitions of q nodes (Sec. 3.1):
 *   scatter (Algorithm 3): every node sends at most one update to each
 *     destination partition (Sec. 3.2), laid out by the Partition-Node Graph
 *     (PNG, Sec. 3.3) into contiguous per-partition bins at static offsets;
 *   gather (Algorithm 4) + apply (Algorithm 2, apply loop): every destination
 *     partition accumulates its bin; a destination ID with its most
 *     significant bit set starts the next update's message.
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA global-memory addresses on the current device;
 *     host pointers are ordinary CPU memory. Each argument says which.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is enqueued on it; calls return after enqueueing unless the
 *     entry point says it synchronises.
 *   - Return value: PCPM_OK (0), a positive informational code, or a negative
 *     error code (see pcpm_strerror). On error no output argument is written
 *     and no memory is leaked. Invalid arguments are rejected on the host
 *     before anything is launched.
 *   - A pcpm_png handle owns its device memory and one solver state; calls on
 *     the same handle must not run concurrently.
 *   - Dangling nodes (no out-edges): the paper does not say what happens to
 *     their rank. By default their mass is spread uniformly over all nodes
 *     (ranks keep summing to 1); PCPM_DANGLING_LEAK drops it, as Eq. 1 read
 *     literally does.
 */
#ifndef PCPM_H
#define PCPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define PCPM_OK 0
#define PCPM_NOT_CONVERGED 1   /* tol > 0 and max_iters reached first */
#define PCPM_EINVAL (-1)       /* bad argument (null, size or range) */
#define PCPM_ECUDA (-2)        /* a CUDA runtime call failed */
#define PCPM_ENOMEM (-3)       /* device or host allocation failed */
#define PCPM_ETIMEOUT (-4)     /* a bounded device-side wait gave up */
#define PCPM_EDEVICE (-5)      /* a device-side consistency check failed */
#define PCPM_EBADGRAPH (-6)    /* CSR invalid: column >= n or a row not sorted */
#define PCPM_ESCRATCH (-7)     /* input larger than the fixed no-allocation scratch */

/* ------------------------------------------------------------------ limits */
/* Node IDs keep their most significant bit free for the message flag
 * (Sec. 3.2), so n < 2^31. */
#define PCPM_MAX_NODES 0x7FFFFFFFu
/* One partition's FP32 accumulator lives in shared memory (<= 227 KB/CTA). */
#define PCPM_MAX_PART_SIZE 32768u
/* Weighted graphs stage each chunk's weights beside its IDs, which leaves
 * room for half the accumulator. */
#define PCPM_MAX_WEIGHTED_PART_SIZE 16384u
/* Bounded by the builder's per-warp counting tables in shared memory. */
#define PCPM_MAX_PARTITIONS 8192u

/* ------------------------------------------------------------------- flags */
#define PCPM_DANGLING_LEAK 0x1u /* drop dangling mass instead of spreading it */
/* Run every iteration as the paper's two phases: a scatter kernel (Algorithm
 * 3), then a gather + apply kernel (Algorithm 4 and the apply loop). Without
 * this flag an iteration is one fused kernel per partition: gather, apply, and
 * the scatter of that partition's new values into a second set of update bins
 * for the next iteration (a standalone scatter runs first when those bins do
 * not yet hold the current ranks). Both compute the same iteration. When a
 * bin is too large for one work unit (skewed graphs; it is then cut into
 * several units whose partial sums meet in global memory), iterations run in
 * the two-phase form whatever the flag says. */
#define PCPM_TWO_PHASE 0x2u
/* Delta iterations (not in the paper; meant for 16-bit update bins). After
 * the first iteration since pcpm_reset, each iteration scatters the change
 * of SPR since the previous iteration instead of SPR itself, and the apply
 * adds it to the current ranks, which Eq. 1 allows by linearity:
 *   PR_{i+1} = PR_i + d * (A^T (SPR_i - SPR_{i-1}) + (D_i - D_{i-1}) / n)
 * (D the dangling mass; 0 under PCPM_DANGLING_LEAK). The changes shrink as the
 * iteration converges, so the rounding of 16-bit bins shrinks with them
 * instead of leaving a floor; FP16 bins store each change times 2^E with
 * E = floor(log2(65504 / r)), r the last L1 change (which bounds every change
 * of SPR), and the gather divides by 2^E. With 16-bit bins every iteration of
 * such a solve, the first included, adds to each node's stored value what the
 * rounding of its previous one left out (error feedback, one FP32 per node),
 * so the stored values sum to the true ones up to the last rounding. The FP32
 * rounding of the ranks is not damped away as in the plain form: it adds up
 * over the iterations. Iterations run in the two-phase form. */
#define PCPM_DELTA 0x4u

/* Kernels timed by pcpm_iterate_timed, in this order. In fused mode the
 * standalone scatter runs only when needed and the gather phase includes the
 * next iteration's scatter. */
#define PCPM_PHASE_SCATTER 0
#define PCPM_PHASE_GATHER_APPLY 1
#define PCPM_PHASE_REDUCE 2
#define PCPM_NUM_PHASES 3

/* Storage type of the update bins (build option update_dtype). The paper
 * keeps one 4-byte value per update (Sec. 3.2, Eq. 5's d_v); 16-bit updates
 * halve the bins' part of the traffic at the cost of rounding every SPR
 * value once per iteration. Accumulation stays FP32 and the reductions FP64. */
#define PCPM_UPDATE_F32 0u  /* SPR(u) as float */
#define PCPM_UPDATE_F16 1u  /* IEEE binary16 of SPR(u) * 2^15, round to nearest even, saturating at 65504 */
#define PCPM_UPDATE_BF16 2u /* bfloat16 of SPR(u), round to nearest even */
/* log2 of the FP16 scale: SPR <= PR <= 1 while ranks sum to at most 1, so
 * SPR * 2^15 stays below FP16's largest finite value. */
#define PCPM_F16_SCALE_LOG2 15

typedef struct pcpm_png pcpm_png; /* opaque, device-resident */

typedef struct pcpm_png_info {
    uint32_t n;               /* |V| */
    uint32_t part_size;       /* q, nodes per partition (Sec. 3.1) */
    uint32_t num_partitions;  /* k = ceil(n / q) */
    uint32_t shard_part_lo;   /* destination partitions the handle gathers: [shard_part_lo, */
    uint64_t num_edges;       /* m = |E| (a shard: the edges into its partitions) */
    uint64_t num_updates;     /* |E'|: edges of the PNG = updates per iteration (Sec. 3.3) */
    double compression_ratio; /* r = |E| / |E'| (Sec. 4, Table params) */
    uint64_t device_bytes;    /* device memory held by the handle */
    int32_t iterations_done;  /* iterations applied since the last reset */
    uint32_t gather_units;    /* gather work units (bins, large ones cut) */
    uint32_t scatter_units;   /* scatter work units (source partitions, large ones cut) */
    uint32_t gather_cluster;  /* CTAs (one thread-block cluster) per gather unit */
    uint32_t fused_ok;        /* 1 if iterations can run fused (no bin was cut) */
    uint32_t canonical_gather; /* 1 if the gather decodes the canonical bins */
    uint32_t gather_runs;     /* 1 if the gather sums runs of IDs with the same destination in a
                                 register before one shared-memory add */
    uint64_t merged_adds;     /* IDs of the gather layout whose value joins the next ID's (same
                                 destination, same lane): shared-memory adds saved by register runs */
    uint32_t update_dtype;    /* PCPM_UPDATE_* of the update bins */
    uint32_t update_bytes;    /* bytes per update: 4 or 2 */
    uint32_t gather_windows;  /* 1 if the gather reads the window layout */
    uint32_t shard_part_hi;   /*  shard_part_hi); [0, k) unless built by pcpm_build_shard */
    uint64_t num_windows;     /* windows of the window layout */
} pcpm_png_info;

/* Tuning of the work decomposition; zero fields take the automatic choice.
 * Results do not depend on these, only speed. */
typedef struct pcpm_build_options {
    uint32_t gather_unit_chunks;  /* most 256-ID chunks one gather unit takes from a bin */
    uint32_t scatter_unit_groups; /* most 4-update groups one scatter unit writes */
    uint32_t gather_cluster;      /* CTAs per gather unit: 1, 2, 4 or 8 */
    uint32_t canonical_gather;    /* 1: gather straight from the canonical bins, decoding the
                                     message flags (Algorithm 4); 0: also build a gather copy of
                                     the destination IDs with explicit update offsets, ordered so
                                     concurrent shared-memory adds hit distinct banks */
    uint32_t gather_runs;         /* bank-spread layout only: 1 sums runs of equal destinations in a
                                     register before one shared-memory add, 2 adds every ID, 0 picks
                                     1 when at least m/16 IDs join a run */
    uint32_t update_dtype;        /* PCPM_UPDATE_F32 (0, default), PCPM_UPDATE_F16 or
                                     PCPM_UPDATE_BF16; 16-bit types need a gather copy of the IDs
                                     (canonical_gather = 0) */
    uint32_t gather_windows;      /* gather copy of the IDs (canonical_gather = 0): 0 or 1 the window
                                     layout, where every warp of a CTA owns a disjoint set of
                                     destinations and adds without atomics (4096-ID windows shared
                                     by the CTA); 2 the bank-spread layout of 256-ID chunks per warp
                                     with shared-memory atomics */
} pcpm_build_options;

/* Builds the Partition-Node Graph of Sec. 3.3 from a CSR out-adjacency:
 * partitions of `part_size` consecutive node IDs (Sec. 3.1); for every
 * (source partition p, destination partition p') the number of nodes of p with
 * an out-neighbour in p' (one update each, Sec. 3.2) and the number of edges
 * p -> p'; the write offsets of Sec. 3.1 (each partition writes into a bin after
 * all lower-ID partitions); and the bins themselves: in update order, the
 * source node of every update, and in destination-ID order, the out-neighbours
 * of that node in p' with the first one's MSB set (Sec. 3.2). Within a bin,
 * source partitions appear in ID order, nodes in ID order and destinations in
 * adjacency order.
 *
 *   row_ptr  device, uint32[n+1]; row_ptr[0] = 0, non-decreasing, row_ptr[n] = m.
 *   col_idx  device, uint32[m]; out-neighbours of node u in
 *            col_idx[row_ptr[u] .. row_ptr[u+1]), each < n, sorted
 *            non-decreasing within the row. Duplicates and self-loops are
 *            kept as ordinary edges. Both arrays are only read, and only
 *            during this call.
 *   n        1 <= n <= PCPM_MAX_NODES.    m  < 2^32 and equal to row_ptr[n].
 *   part_size  1 <= q <= PCPM_MAX_PART_SIZE and ceil(n/q) <= PCPM_MAX_PARTITIONS.
 *   out      host; receives the new handle (free with pcpm_free).
 * Synchronises `stream`. Returns PCPM_EBADGRAPH, and no handle, if a column is
 * >= n or a row is not sorted; PCPM_EINVAL if row_ptr[n] != m. */
int pcpm_build(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
               uint32_t part_size, void* stream, pcpm_png** out);

/* pcpm_build with tuning options (host struct, nullable = all automatic).
 * PCPM_EINVAL if gather_cluster is not 0, 1, 2, 4 or 8, gather_runs or gather_windows is above
 * 2, update_dtype is not a PCPM_UPDATE_* value, a 16-bit update_dtype comes with
 * canonical_gather, or gather_windows = 1 comes with canonical_gather. */
int pcpm_build_ex(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                  uint32_t part_size, const pcpm_build_options* options, void* stream,
                  pcpm_png** out);

/* Batched solves (not in the paper): many independent graphs, each with its
 * own handle, solved by one CUDA graph launch. pcpm_batch_create captures,
 * for every handle, pcpm_reset to the uniform start followed by `iters`
 * iterations (d, flags as in pcpm_iterate, no tolerance), each handle on one
 * of up to 32 graph branches so that small graphs run side by side; it
 * instantiates the graph once. pcpm_batch_launch runs the whole batch with
 * one cudaGraphLaunch on `stream` and leaves every handle as if that work had
 * been enqueued through pcpm_reset and pcpm_iterate (pcpm_ranks and
 * pcpm_residual_history then read the results).
 *   handles  host array of `count` distinct handles (PCPM_EINVAL otherwise),
 *            which must outlive the batch.
 * pcpm_batch_create synchronises the default stream if a handle's residual
 * history has to grow (it captures on private streams). The L1 changes reach
 * each handle's history at every launch, also after later pcpm_iterate calls
 * have grown it. pcpm_batch_free waits for the device before it releases
 * the batch's buffers. */
typedef struct pcpm_batch pcpm_batch;
int pcpm_batch_create(pcpm_png* const* handles, int count, float d, int iters, uint32_t flags,
                      pcpm_batch** out);
int pcpm_batch_launch(pcpm_batch* batch, void* stream);
void pcpm_batch_free(pcpm_batch* batch); /* NULL is a no-op */
/* The number of kernels one pcpm_batch_launch runs (the kernel nodes of its
 * CUDA graph) into *launches. When every handle has the window layout and no
 * weights, and the flags ask for two-phase or fused iterations (not delta
 * ones; fused only if every handle can fuse), each phase is a single launch
 * over the units of all graphs that share a part size, a gather cluster size
 * and a bin format: per such group 2 + 3 iters launches for two-phase
 * iterations (reset, its reduction, then scatter, gather, reduction per
 * iteration) or 3 + 2 iters for fused ones (one scatter, then gather with
 * the next scatter, and reduction per iteration), plus one copy of the
 * histories. Otherwise each handle's work is captured as pcpm_reset and
 * pcpm_iterate enqueue it. PCPM_EINVAL for NULL arguments. */
int pcpm_batch_kernel_launches(const pcpm_batch* batch, int* launches);

/* Weighted graphs and SpMV (Sec. 3.5): pcpm_build with an edge weight per
 * column index.
 *   weights  device, float[m], in CSR order (weight of col_idx[e] at e); only
 *            read during this call. Weights are stored beside the destination
 *            IDs in bin order and applied in the gather of pcpm_spmv.
 * Requires part_size <= PCPM_MAX_WEIGHTED_PART_SIZE, canonical_gather = 0 and
 * FP32 updates (PCPM_EINVAL otherwise). PageRank iterations on the handle
 * ignore the weights (PageRank of the unweighted graph). */
int pcpm_build_weighted(const uint32_t* row_ptr, const uint32_t* col_idx, const float* weights, uint32_t n,
                        uint64_t m, uint32_t part_size, const pcpm_build_options* options, void* stream,
                        pcpm_png** out);

/* ------------------------------------------------------ destination shards
 * One iteration split over several GPUs (one process each). Every partition of
 * destinations is gathered and applied independently of the others (Sec. 3.1:
 * bin p' receives all updates into partition p', and Algorithm 4 reads only
 * that bin), so each rank builds the bins of a contiguous range of destination
 * partitions and owns the ranks of their nodes. Its scatter (Algorithm 3) needs
 * the ranks of every source, so between iterations the ranks exchange their
 * owned slices of the new vector (an all-gather) and add two FP64 sums (an
 * all-reduce): the L1 change and the dangling mass. The exchange is the
 * caller's (NCCL or any collective library); these calls never wait on another
 * GPU and never read another GPU's memory.
 *
 * pcpm_dest_partition_counts: edges per destination partition of a device CSR
 * (col_idx device uint32[m]; counts host uint64[ceil(n/part_size)]).
 * Synchronises `stream`. PCPM_EBADGRAPH if a column is >= n.
 *
 * pcpm_shard_split (host only, no device work): cuts the k = ceil(n/part_size)
 * partitions into `nranks` contiguous ranges of near-equal weight, where
 * partition p weighs ids_per_part[p] plus its node count. part_lo (host,
 * nranks + 1 entries) receives the cuts: rank r takes [part_lo[r],
 * part_lo[r+1]), part_lo[0] = 0, part_lo[nranks] = k. Cut r is the partition
 * boundary b whose prefix weight is nearest r/nranks of the total (ties to
 * the lower b), moved as little as needed to leave every rank at least one
 * partition. PCPM_EINVAL if nranks is 0 or above k.
 *
 * pcpm_build_shard: pcpm_build_ex restricted to destination partitions
 * [part_lo, part_hi) (0 <= part_lo < part_hi <= k): the PNG of the edges into
 * nodes [part_lo*q, min(part_hi*q, n)) from every source node, with the
 * out-degrees of the whole CSR. Same CSR rules and errors as pcpm_build_ex
 * (a column >= n anywhere in the CSR gives PCPM_EBADGRAPH). pcpm_png_export of
 * a shard gives its bins: those of partitions in range equal the whole
 * graph's, the others are empty. A shard whose range is not all of [0, k)
 * rejects pcpm_reset, pcpm_iterate, pcpm_iterate_timed, pcpm_pagerank,
 * pcpm_spmv and batches (PCPM_EINVAL); it runs through the two calls below.
 * Any handle can run them, a whole-graph one as its own single shard.
 *
 * pcpm_shard_init: writes PR_0 to all n entries of pr_out (device float[n]):
 * pr_init (device float[n], nullable = uniform 1/n). sums (device double[2])
 * receives {0, dangling mass of PR_0 over the shard's own nodes}.
 *
 * pcpm_shard_step: one iteration of Eq. 1 for the shard's own nodes.
 *   pr_in   device float[n]: PR_i of every node (all shards' slices).
 *   sums    device double[2], read then written: on entry sums[1] must hold
 *           the whole graph's dangling mass of pr_in (the all-reduced sums of
 *           the previous call); on return sums = {sum over own nodes of
 *           |PR_{i+1}(v) - PR_i(v)|, dangling mass of PR_{i+1} over own nodes}.
 *   pr_out  device float[n], != pr_in: PR_{i+1} is written to the shard's own
 *           nodes only; other entries are left as they were.
 *   flags   PCPM_DANGLING_LEAK or 0 (iterations are always two-phase).
 * Enqueued on `stream`; does not synchronise. A bounded device wait that gave
 * up is reported by pcpm_sync_status. */
int pcpm_dest_partition_counts(const uint32_t* col_idx, uint64_t m, uint32_t n, uint32_t part_size,
                               uint64_t* counts, void* stream);
int pcpm_shard_split(const uint64_t* ids_per_part, uint32_t n, uint32_t part_size, uint32_t nranks,
                     uint32_t* part_lo);
int pcpm_build_shard(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                     uint32_t part_size, uint32_t part_lo, uint32_t part_hi, const pcpm_build_options* options,
                     void* stream, pcpm_png** out);
int pcpm_shard_init(pcpm_png* png, const float* pr_init, float* pr_out, double* sums, void* stream);
int pcpm_shard_step(pcpm_png* png, float d, uint32_t flags, const float* pr_in, float* pr_out, double* sums,
                    void* stream);

/* Waits for the handle's last stream and returns the device-side status of
 * its kernels since the last reset or shard init: PCPM_OK, PCPM_ETIMEOUT (a
 * bounded wait gave up) or PCPM_EDEVICE. */
int pcpm_sync_status(const pcpm_png* png);

/* Sparse matrix-vector product over the PNG (Sec. 3.5):
 *   y(v) = sum over edges (u, v) of w(u, v) * x(u)      (y = A^T_w x)
 * with w = 1 on an unweighted handle. One scatter of x (Algorithm 3, x
 * itself rather than x/outdeg) and one gather with the weights applied
 * (Algorithm 4), FP32 accumulation.
 *   x  device float[n], read;  y  device float[n], written.
 * Uses the handle's rank buffers: its solver state afterwards is undefined
 * (pcpm_reset before solving). Enqueued on `stream`; does not synchronise. */
int pcpm_spmv(pcpm_png* png, const float* x, float* y, void* stream);

/* Non-square matrices (Sec. 3.5): rows and columns are partitioned
 * separately; the scatter runs over the row partitions and the gather over
 * the column partitions. A is n_rows x n_cols in CSR (rows are the sources):
 *   row_ptr  device, uint32[n_rows + 1];  col_idx  device, uint32[m], each
 *            < n_cols, sorted within the row;  weights  device float[m] or
 *            NULL (all 1; then the PCPM_MAX_PART_SIZE limit applies, else
 *            PCPM_MAX_WEIGHTED_PART_SIZE).
 * Rows and columns share one range of n = max(n_rows, n_cols) IDs and the
 * part size q: k = ceil(n / q) partitions, of which the first ceil(n_rows / q)
 * hold sources and the first ceil(n_cols / q) are gathered. PCPM_EBADGRAPH if a
 * column is >= n_cols; other errors as pcpm_build_ex. The handle runs
 * pcpm_spmv_rect only (PageRank needs a square matrix).
 * pcpm_spmv_rect: y = A^T_w x, x device float[n_rows], y device float[n_cols],
 * one scatter and one gather (FP32 accumulation). Enqueued on `stream`. */
int pcpm_build_rect(const uint32_t* row_ptr, const uint32_t* col_idx, const float* weights, uint32_t n_rows,
                    uint32_t n_cols, uint64_t m, uint32_t part_size, const pcpm_build_options* options, void* stream,
                    pcpm_png** out);
int pcpm_spmv_rect(pcpm_png* png, const float* x, float* y, void* stream);

/* Test hook: the weights in canonical bin order, host float[m] (the position
 * of each weight matches pcpm_png_export's dest_ids). Synchronises.
 * PCPM_EINVAL for an unweighted handle. */
int pcpm_export_weights(const pcpm_png* png, float* wbin);

/* Releases the handle and all its device memory. NULL is a no-op. Waits for
 * all work on the device (as cudaFree does), then returns the memory to the
 * library's device-memory pool.
 *
 * Memory: handles, build temporaries and pcpm_pagerank_host's copies come
 * from one stream-ordered pool per device (cudaMemPool) that keeps freed
 * memory for the next build instead of returning it to the driver, so
 * repeated builds make no new driver allocations. */
void pcpm_free(pcpm_png* png);

/* Partition-size autotuner. The paper studies r, traffic and time against the
 * partition size (Sec. 5.3.2); the best size depends on the graph. This builds
 * the PNG of the device CSR for every candidate part size, resets it to the
 * uniform start, runs `warmup` untimed and then `iters` timed iterations
 * (pcpm_iterate_timed with d and flags on `stream`), and frees it.
 *   part_sizes     host, `count` >= 1 candidates.
 *   best_part_size host; receives the candidate with the least time per iteration.
 *   ms_per_iter    host, `count` floats, nullable: each candidate's time per
 *                  iteration, or -1 where the build rejected the size
 *                  (PCPM_EINVAL: above PCPM_MAX_PART_SIZE, or too many partitions).
 * PCPM_EINVAL if no candidate builds or an argument is bad; other errors from
 * the builds and iterations are returned as they occur. Synchronises. */
int pcpm_autotune(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                  const uint32_t* part_sizes, int count, float d, int warmup, int iters, uint32_t flags,
                  void* stream, uint32_t* best_part_size, float* ms_per_iter);

/* The autotuner over partition sizes and tile shapes: every partition size
 * with every build option set (the work decomposition: gather_unit_chunks,
 * scatter_unit_groups, gather_cluster, gather layout; results do not depend
 * on them, only speed), timed as in pcpm_autotune.
 *   options      host, `noptions` >= 1 option sets (NULL: one automatic set).
 *   best_option  host; receives the index of the fastest option set.
 *   ms_per_iter  host, count * noptions floats (row = partition size),
 *                nullable; -1 where the build rejected the combination. */
int pcpm_autotune_ex(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                     const uint32_t* part_sizes, int count, const pcpm_build_options* options, int noptions,
                     float d, int warmup, int iters, uint32_t flags, void* stream, uint32_t* best_part_size,
                     int* best_option, float* ms_per_iter);

/* Returns the memory that the library's pools hold but no live handle uses
 * to the driver (cudaMemPoolTrimTo 0 on every device the library used).
 * PCPM_ECUDA if a trim fails. */
int pcpm_release_cached_memory(void);

/* Sizes of the handle (host struct). */
int pcpm_png_get_info(const pcpm_png* png, pcpm_png_info* info);

/* Copies the PNG to host buffers; any pointer may be NULL to skip it.
 * Synchronises. Layout (k = num_partitions, row = source partition p,
 * column = destination partition p'):
 *   cnt_u[k*k]  updates p -> p'            cnt_e[k*k]  edges p -> p'
 *   off_u[k*k]  offset of p in update_bins[p'] (Sec. 3.1)  off_e[k*k] same for IDs
 *   bin_u[k+1]  start of update_bins[p'] in the concatenated bins; bin_u[k] = |E'|
 *   bin_e[k+1]  start of destID_bins[p'];                      bin_e[k] = m
 *   src_idx[|E'|]  source node of each update, in bin order
 *   dest_ids[m]    destination IDs in bin order, MSB = first of a message */
int pcpm_png_export(const pcpm_png* png, uint32_t* cnt_u, uint32_t* cnt_e, uint32_t* off_u,
                    uint32_t* off_e, uint32_t* bin_u, uint32_t* bin_e, uint32_t* src_idx,
                    uint32_t* dest_ids);

/* Starts a new solve: PR_0 = pr_init (device, float[n], read during the call;
 * NULL = uniform 1/n), SPR_0 = PR_0/|N_o| (0 for dangling nodes), and the
 * dangling mass of PR_0. Resets iterations_done to 0. */
int pcpm_reset(pcpm_png* png, const float* pr_init, void* stream);

/* Applies up to `iters` iterations of Eq. 1 to the handle's current ranks,
 * each one a scatter (Algorithm 3), a gather + apply (Algorithm 4 and the apply
 * loop of Algorithm 2) and an FP64 reduction of the L1 change
 * sum_v |PR_{i+1}(v) - PR_i(v)| and of the next dangling mass.
 *   d     damping factor, 0 <= d < 1.      iters >= 0.
 *   tol   > 0: stop after the first iteration whose L1 change is < tol;
 *         <= 0: run exactly `iters` iterations.
 *   flags PCPM_DANGLING_LEAK and/or PCPM_TWO_PHASE, or 0.
 *   iters_run, last_residual  host, nullable: iterations applied by this call
 *         and the L1 change of the last one (0 if none). If either is
 *         requested, or tol > 0, the call synchronises.
 * Returns PCPM_NOT_CONVERGED if tol > 0 was not reached. */
int pcpm_iterate(pcpm_png* png, float d, int iters, double tol, uint32_t flags, int* iters_run,
                 double* last_residual, void* stream);

/* Same as pcpm_iterate with tol <= 0, and also records CUDA events around
 * every kernel on `stream`. kernel_ms (host, PCPM_NUM_PHASES + 1 floats)
 * receives the total milliseconds spent in each phase over the `iters`
 * iterations, then the span from the event before the first kernel to the
 * event after the last one. Synchronises. */
int pcpm_iterate_timed(pcpm_png* png, float d, int iters, uint32_t flags, float* kernel_ms,
                       void* stream);

/* Copies the current ranks PR_i to pr_out (device, float[n], caller-owned). */
int pcpm_ranks(const pcpm_png* png, float* pr_out, void* stream);

/* L1 changes of the iterations since the last reset (host double[max_count]);
 * writes min(max_count, iterations_done) values and returns that count (or a
 * negative error). Synchronises. */
int pcpm_residual_history(const pcpm_png* png, double* out, int max_count);

/* pcpm_reset + pcpm_iterate + pcpm_ranks. pr_out (device, float[n]) receives
 * PR after the last iteration; pr_init as in pcpm_reset. Synchronises when
 * tol > 0 or when iters_run / final_residual are requested. */
int pcpm_pagerank(pcpm_png* png, float d, int max_iters, double tol, uint32_t flags,
                  const float* pr_init, float* pr_out, int* iters_run, double* final_residual,
                  void* stream);

/* End-to-end solve from host memory: copies the CSR (host row_ptr[n+1],
 * col_idx[m], rules of pcpm_build) to the device, builds the PNG, runs
 * pcpm_pagerank with a uniform start and copies the ranks to pr_out (host,
 * float[n]). Allocates and frees its own device memory; synchronises. */
int pcpm_pagerank_host(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                       uint32_t part_size, float d, int max_iters, double tol, uint32_t flags,
                       float* pr_out, int* iters_run, double* final_residual);

/* Test hooks. pcpm_scatter_only runs one scatter (Algorithm 3) of the current
 * ranks into the current update bins without advancing the solve.
 * pcpm_export_state copies the current state to host buffers (nullable):
 * pr[n], spr[n] (= pr/outdeg, recomputed on the device), updates (the current
 * update bins in bin order: |E'| values of the handle's update_dtype, so
 * |E'| * update_bytes bytes) and the dangling mass of pr. Synchronises. */
int pcpm_scatter_only(pcpm_png* png, void* stream);
int pcpm_export_state(const pcpm_png* png, float* pr, float* spr, void* updates, double* dangling);

/* Test hook for the bounded device-side waits (PCPM_ETIMEOUT). Sets, on the
 * current device and for every handle, the bound of the window-layout
 * gather's waits for work (a free ring stage for the producer, a filled one
 * for the consumers): `cycles` > 0 SM cycles; 0 restores the default (about
 * one second); < 0 makes those waits give up at once, as if what they wait for
 * never happened. A wait that gives up sets PCPM_ETIMEOUT in the handle's
 * state, stops the CTA's streaming and leaves that launch's ranks undefined;
 * the copies already in flight are still waited for with the default bound
 * before the CTA exits. pcpm_reset clears the status. Not for concurrent use
 * with other work on the device. */
int pcpm_test_wait_limit(long long cycles);

/* Allocation-free rank statistics. There is no counterpart in the paper: this
 * entry point exists for callers that cannot call cudaMalloc, such as code
 * running inside a custom memory pool or allocator callback that must not
 * re-enter the allocator, or a process whose device memory is fully reserved
 * before it starts. It allocates nothing: its scratch is a fixed array
 * compiled into the library (PCPM_NOALLOC_MAX_BLOCKS * 16 bytes = 1 MiB,
 * held on every GPU that loads the library until the process exits).
 *
 * Computes, in FP64, out[0] = sum_v |x(v) - y(v)| (the L1 change the solver
 * reports per iteration) and out[1] = sum of x(v) over nodes v without
 * out-edges (row_ptr[v+1] == row_ptr[v]; the dangling mass), summed in a
 * fixed order.
 *   x, y     device, float[n], caller-owned, read only.
 *   row_ptr  device, uint32[n+1] (the CSR row offsets of pcpm_build).
 *   out      device, double[2], caller-owned, written.
 *   n        1 <= n <= PCPM_NOALLOC_MAX_NODES; larger inputs return
 *            PCPM_ESCRATCH before anything is launched.
 * Enqueued on `stream`; does not synchronise. The first call on each device
 * looks up the scratch array's device address (with that device current) and
 * so should come before any stream capture. Every call on a device shares the
 * one scratch array: calls that may overlap on the GPU (different streams
 * without ordering) race and must be serialised by the caller. Each call
 * writes every scratch slot it reads, so nothing carries over between calls. */
#define PCPM_NOALLOC_MAX_BLOCKS 65536u
#define PCPM_NOALLOC_MAX_NODES (PCPM_NOALLOC_MAX_BLOCKS * 4096u)
int pcpm_rank_stats_noalloc(const float* x, const float* y, const uint32_t* row_ptr, uint32_t n,
                            double* out, void* stream);

/* Message for a status code (static string). */
const char* pcpm_strerror(int code);
/* Name of the CUDA runtime error behind the calling thread's last PCPM_ECUDA
 * (or PCPM_ENOMEM from an allocation), e.g. "cudaErrorInvalidValue";
 * "cudaSuccess" if none was recorded. */
const char* pcpm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PCPM_H */
