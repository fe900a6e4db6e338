// pcpm_internal.cuh - shared definitions of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pcpm.h"

namespace pcpm {

// ---------------------------------------------------------------- layout
// Destination IDs carry the message flag in bit 31 (Sec. 3.2).
constexpr uint32_t kMsb = 0x80000000u;
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr uint32_t kNoHub = 0xFFFFFFFFu;

// Builder: edges per warp tile (each tile lies inside one source partition).
constexpr uint32_t kTileEdges = 8192;
// Builder: a destination needs this many in-edges inside its bin before the
// gather keeps it in registers instead of shared-memory atomics.
constexpr uint32_t kHubMinInDegree = 64;
// Gather: destination IDs per chunk. Every chunk of the concatenated bins
// starts at a multiple of kChunk entries and has a precomputed update base
// (the number of flagged IDs before it), so any warp can decode any chunk.
constexpr uint32_t kChunk = 256;
// Gather: a chunk needs the updates [base-1, next base) (the first ID may
// continue the previous message), widened to 16-byte boundaries: at most
// kUpdSlot 4-byte updates, or 2 * kUpdSlot 2-byte ones (kChunk + 16 needed).
constexpr uint32_t kUpdSlot = kChunk + 8;
// Gather, bank-spread layout: one 32-bit word per destination ID holding an
// accumulator slot (16 bits), the offset of its update in the chunk's update
// slice (9 bits) and a run bit (the next ID of the same gather lane has the
// same slot). Slots below q are the partition's nodes. Padding words name one
// of kPadSlots spare slots after them (offset 0), which are never read. IDs
// of the bin's two hub destinations name slot q + kPadSlots + {0, 1}, which
// each warp moves to a private pair of slots, so hub adds from different
// warps never meet on one address; the pairs are added to the hubs' real
// slots once, after the warp's last chunk.
constexpr uint32_t kGwLocMask = 0xFFFFu;
constexpr uint32_t kGwUpdShift = 16;
constexpr uint32_t kGwUpdMask = 0x1FFu;
constexpr uint32_t kGwRunBit = 1u << 30;
constexpr uint32_t kPadSlots = 32;
static_assert(kUpdSlot <= kGwUpdMask + 1 && kChunk + 16 <= kGwUpdMask + 1, "update offsets must fit their field");
// Gather: warps per CTA and pipeline depth of each warp's private ring.
constexpr int kGatherWarps = 24;
constexpr int kGatherStages = 2;
constexpr uint32_t kHubSlots = 2 * kGatherWarps;
// Gather, window layout (the default): a bin's destination IDs are cut into
// windows of at most kWin consecutive IDs (whole windows of one bin per work
// unit). The window's update slice and its IDs reach shared memory by bulk
// copies into a ring that all kWinWarps consumer warps of the CTA share. Each
// consumer warp owns a set of accumulator slots: blocks of 32 consecutive
// nodes, dealt to warps as contiguous ranges balanced by in-degree, and a
// private slot for each of the bin's kWinHubs largest in-degree nodes (whose
// IDs are dealt to all warps in turn). A window's IDs are grouped by owner
// warp, so no two warps ever add into one slot and the adds need no atomics.
// Inside a group, IDs are sorted by (bank, slot, position) and dealt lane by
// lane: lane l takes a contiguous run of sorted positions, so equal slots sit
// in one lane (or in consecutive lanes, joined by a shuffle scan), and the
// lanes of one round hit rising banks. Each 32-bit word holds the slot (16
// bits), the offset of its update in the window's slice (13 bits) and an end
// bit (the next sorted ID of the group has another slot). A window starts
// with a header of kWinHdrWords words: the kWinWarps + 1 group offsets as
// 16-bit values.
constexpr uint32_t kWin = 4096;
constexpr int kWinWarps = 12;
constexpr uint32_t kWinHubs = 8;
constexpr uint32_t kWinHdrWords = 16;
constexpr uint32_t kWinStride = kWinHdrWords + kWin;  // words per window in the layout array
constexpr uint32_t kWinSlotMask = 0xFFFFu;
constexpr uint32_t kWinOffShift = 16;
constexpr uint32_t kWinOffMask = 0x1FFFu;
constexpr uint32_t kWinEndBit = 1u << 29;
static_assert(kWinWarps + 1 <= 2 * kWinHdrWords, "the header holds the group offsets as 16-bit values");
static_assert(kWin + 16 <= kWinOffMask + 1, "update offsets of a window must fit their field");
static_assert(PCPM_MAX_PART_SIZE + kWinWarps * kWinHubs <= kWinSlotMask + 1, "slots must fit their field");
// Update bin storage: PCPM_UPDATE_F32, _F16 (SPR * 2^15), _BF16.
constexpr int kUpdF32 = (int)PCPM_UPDATE_F32, kUpdF16 = (int)PCPM_UPDATE_F16, kUpdBF16 = (int)PCPM_UPDATE_BF16;
constexpr float kF16Scale = (float)(1 << PCPM_F16_SCALE_LOG2);
// Scatter: threads per CTA; bytes of each of a warp's two bulk-copy stages of
// source indices.
constexpr int kScatterThreads = 1024;
constexpr uint32_t kScatterStageBytes = 1488;
// Apply / reduce threads.
constexpr int kReduceThreads = 512;
// Largest thread-block cluster used for one bin.
constexpr int kMaxCluster = 8;
// Streams (graph branches) a batch capture spreads its solves over.
constexpr int kBatchStreams = 32;

// Upper bound for a device-side wait on an mbarrier, in SM clock cycles
// (about one second at 2 GHz). A wait that runs out sets kErrTimeout.
constexpr long long kWaitLimitCycles = 2000000000LL;

// Device error bits (DevState::err).
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;
constexpr int kErrBadGraph = 4;

// Solver scalars kept on the device.
struct DevState {
    double dangling;       // sum of PR over dangling nodes for the current ranks
    double residual;       // L1 change of the last iteration
    int stop;              // set once residual < tol (tol > 0)
    int iters_done;        // iterations applied since reset
    int err;               // kErr* bits
    int pad;
    double dangling_prev;  // the dangling mass of the ranks before the current ones
};

}  // namespace pcpm

// The handle behind the opaque ABI type.
struct pcpm_png {
    int device;
    int sms;
    uint32_t n, q, k;
    uint64_t m, ne;
    uint64_t nchunks;        // ceil(m / kChunk)
    // PNG
    uint32_t* dest;          // m destination IDs in bin order (padded to whole chunks)
    uint32_t* src;           // ne source IDs in bin order (padded)
    uint16_t* src16;         // the same as indices within their source partition (ne + 16)
    uint32_t* bin_u;         // k+1 starts of update bins
    uint32_t* bin_e;         // k+1 starts of destination-ID bins
    uint32_t* seg_u;         // k*k absolute start of segment (p, p') in the update array
    uint32_t* cnt_u;         // k*k updates p -> p'
    uint32_t* seg_e;         // k*k absolute start of segment (p, p') in the ID array
    uint32_t* cnt_e;         // k*k edges p -> p'
    uint32_t* chunk_base;    // nchunks+1: flagged IDs before each chunk
    uint32_t* hubs;          // 2k: per bin, local IDs of its two largest in-degrees (or kNoHub)
    // Bank-spread gather layout (unless the canonical bins are gathered
    // directly): every bin padded to whole kChunk-ID chunks; each chunk's IDs
    // permuted so that the IDs one warp adds at once fall in distinct
    // shared-memory banks as far as possible, in the word format of kGw*.
    int canonical_gather;    // 1: the gather decodes the canonical bins (MSB flags)
    int gather_runs;         // 1: the gather sums run-bit runs in a register
    int upd_dtype;           // kUpd*: storage of the update bins
    // Weighted graphs (Sec. 3.5): edge weights beside the destination IDs.
    int weighted;
    const float* weights_in; // caller's CSR-order weights, read during the build only
    float* wdest;            // m (padded like dest): weights in canonical bin order
    float* gweight;          // nichunks * kChunk: weights in the bank-spread layout's order
    uint32_t upd_bytes;      // 4 or 2
    uint64_t merged_adds;    // IDs with bit 30 set
    // Window layout (gather_windows = 1), see kWin: nwin windows, bin p's
    // windows [win_start[p], win_start[p+1]); window w's header and words at
    // wwords + w * kWinStride; wdesc[w] = (first update of its slice, slice
    // bytes, bytes of header + words to copy, IDs).
    int gather_windows;
    uint64_t nwin;
    uint32_t* win_start;     // k+1
    uint32_t* wwords;        // nwin * kWinStride
    float* wweight;          // weighted graphs: weights at their IDs' word positions
    uint4* wdesc;            // nwin
    uint32_t* whubs;         // k * kWinHubs: local IDs of each bin's hubs (or kNoHub)
    uint32_t* indeg;         // n: in-degree of every node in the handle's bins (window layout only)
    uint32_t* gdest;         // nichunks * kChunk words
    uint32_t* gslice_start;  // nichunks: first update of the chunk's slice (multiple of 4)
    uint32_t* gslice_bytes;  // nichunks: bytes of the slice (multiple of 16)
    uint32_t* ichunk_start;  // k+1: first chunk of each bin in gdest
    uint64_t nichunks;
    // Work units. A gather unit is a run of chunks of one bin (uint4: bin,
    // first chunk, end chunk, pieces of that bin); a scatter unit is a range of
    // 4-entry groups of one source partition (partition, first group, end
    // group, pieces). Large bins and partitions are cut into several units so
    // skewed graphs still spread over all SMs; orders list units largest first.
    uint4* gunits;
    uint32_t* gorder;
    uint32_t ngunits;
    uint4* sunits;
    uint32_t* sorder;
    uint32_t nsunits;
    int fused_ok;            // every bin is a single gather unit
    // Destination shard: the handle holds the bins of destination partitions
    // [plo, phi) only (all of [0, k) unless built by pcpm_build_shard), gathers
    // and applies those, and owns nodes [plo * q, min(phi * q, n)).
    uint32_t plo, phi;
    // Non-square matrix (pcpm_build_rect, Sec. 3.5): rows [0, n_rows) are the
    // sources, columns [0, n_cols) the destinations, over n = max of the two
    // IDs; the gather runs the column partitions only (phi = ceil(n_cols / q)).
    int rect;
    uint32_t n_rows, n_cols;
    float* gacc;             // n: partial sums of bins cut into several units
    uint32_t* bin_done;      // k: units of a cut bin that have flushed
    float* inv_deg;          // n: 1/|N_o(u)|, 0 for dangling nodes
    float* dq_err;           // 2n (16-bit update bins): rounding left out of each node's last stored value
                             // (delta solves), carried into its next one; read from half dq_cur, written to
                             // the other; zeroed by a reset
    int dq_cur;
    // solver state
    float* pr[2];            // ranks ping-pong
    int cur;                 // pr[cur] holds PR_i
    void* upd[2];            // update bins (padded, upd_dtype); upd[ucur] is the current one
    int ucur;
    int upd_valid;           // upd[ucur] holds the scatter of PR_i
    int cluster;             // CTAs per gather unit (a thread-block cluster)
    double* partials;        // 2 * partial_slots(): per-CTA (residual, dangling)
    int partial_count;       // CTAs that wrote partials for the pending reduce
    double* hist;            // residual history
    int hist_cap;
    pcpm::DevState* state;   // device scalars
    pcpm::DevState* state_host;  // pinned mirror
    int iters_done;
    uint64_t device_bytes;
    cudaStream_t last_stream;
    cudaStream_t alloc_stream;  // the build's stream: device memory is allocated in its order
};

namespace pcpm {

// Builder entry (png_build.cu). Fills every PNG field of `g` (n, q, k, m set by
// the caller); returns a PCPM_* status.
int build_png(pcpm_png* g, const uint32_t* row_ptr, const uint32_t* col, const pcpm_build_options& opt,
              cudaStream_t s);

// out[0..n] = exclusive scan of in[0..n), out[n] = total (png_build.cu);
// temporaries from the pool in s's order. A PCPM_* status.
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t s);

// Destination shards (png_build.cu). keep_counts: per row u, the columns in
// [vlo, vhi) (a warp per row), with kErrBadGraph in *err for a column >= n or
// a row whose offsets decrease or pass m. keep_copy: those columns in row
// order at out_ptr[u]. dest_counts: edges per destination partition (host
// uint64[k]), kErrBadGraph for a column >= n.
int shard_filter_csr(const uint32_t* row_ptr, const uint32_t* col, uint32_t n, uint64_t m, uint32_t vlo,
                     uint32_t vhi, uint32_t** rp_out, uint32_t** col_out, uint64_t* m_out, cudaStream_t s);
int compute_inv_deg(pcpm_png* g, const uint32_t* row_ptr, cudaStream_t s);
int dest_partition_counts(const uint32_t* col, uint64_t m, uint32_t n, uint32_t q, uint64_t* counts_host,
                          cudaStream_t s);

// Iteration kernels (pcpm_iter.cu).
int configure_kernels(pcpm_png* g);
int pull_sum(pcpm_png* g, const float* pr_like, float* out, cudaStream_t s);
// Records a failed CUDA call for pcpm_last_cuda_error (per thread).
void note_cuda_error(cudaError_t e);
// PCPM_OK if the last kernel launch on this thread succeeded, else records the
// error and returns PCPM_ECUDA.
int launch_status();
int launch_init(pcpm_png* g, const float* pr_init, cudaStream_t s);
// out[v] = x[v] for v < len, 0 for len <= v < n (a non-square matrix's rows).
int launch_copy_pad(const float* x, uint32_t len, float* out, uint32_t n, cudaStream_t s);
// init into `out` (n floats), with the dangling partial sums over nodes [lo, hi) only.
int launch_init_range(pcpm_png* g, const float* pr_init, float* out, uint32_t lo, uint32_t hi, cudaStream_t s);
// raw: stage x itself (SpMV) instead of x * (1/outdeg).
// delta: scatter the change of SPR since the previous ranks (PCPM_DELTA);
// feedback: 16-bit bins carry each node's rounding left-over (dq_err) into
// its next stored value (every iteration of a PCPM_DELTA solve).
int launch_scatter(pcpm_png* g, cudaStream_t s, bool raw = false, bool delta = false, bool feedback = false);
// Algorithm 3 for a 32-bit value per node, copied bit for bit: out[t] = x[src[t]]
// in the update bins' layout (FP32 update bins only; PCPM_EINVAL otherwise).
int launch_scatter_bits(pcpm_png* g, const void* x, void* out, cudaStream_t s);
// spmv: the weighted gather of a weighted handle (Sec. 3.5).
int launch_gather(pcpm_png* g, float d, uint32_t flags, bool fused, cudaStream_t s, bool spmv = false,
                  bool delta = false);
// Batched solves with one launch per phase over the units of all graphs
// (pcpm_batch_*) of each (part size, cluster size, bin format) group: usable
// when every handle has the window layout, no weights and the whole square
// graph, the iterations are not delta ones, and (fused iterations) every
// handle can fuse. batch_kernels_free wants the device idle.
struct BatchKernels;
bool batch_kernels_ok(pcpm_png* const* hs, int count, uint32_t flags);
bool batch_kernels_fused(const BatchKernels* b);
// hist: count x iters doubles, row i the L1 changes of hs[i].
int batch_kernels_create(pcpm_png* const* hs, int count, float d, uint32_t flags, double* hist, int iters,
                         cudaStream_t s, BatchKernels** out);
int batch_kernels_groups(const BatchKernels* b);
// group i recorded on streams[i % nstreams]: groups run side by side
int batch_kernels_record(BatchKernels* b, int iters, const cudaStream_t* streams, int nstreams);
void batch_kernels_free(BatchKernels* b);
// dst[i][t] = src[i * iters + t] for t < iters (dst: device table of count pointers).
int launch_hist_copy(const double* src, double* const* dst, int iters, int count, cudaStream_t s);
// The window gather's bound on waits for work (see pcpm_test_wait_limit).
int set_work_wait_limit(long long cycles);
// record = false: the L1 change goes to the device state only, not the history.
int launch_reduce(pcpm_png* g, double tol, int hist_slot, cudaStream_t s, bool record = true);
int launch_spr(pcpm_png* g, float* spr, cudaStream_t s);
size_t partial_slots(const pcpm_png* g);

// Device memory comes from one stream-ordered pool per device that keeps what
// is freed (release threshold unlimited), so a build after a free reuses it
// without new driver allocations; pcpm_release_cached_memory trims it.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);
// Device allocation of a handle's array (on g->alloc_stream), recording sizes.
cudaError_t dev_alloc(pcpm_png* g, void** p, size_t bytes);

}  // namespace pcpm
