// png_build.cu - device construction of the Partition-Node Graph (Sec. 3.3).
//
// The paper builds the PNG with two scans over each source partition's edges:
// the first counts, per destination partition p', the updates (one per node
// with a neighbour in p', Sec. 3.2) and the edges; a prefix sum turns the counts
// into write offsets (Sec. 3.1); the second scan fills the bins. Here the same
// two scans run as a stable counting sort of all edges keyed by destination
// partition:
//   tiles      every source partition's edge range is cut into tiles of
//              kTileEdges edges (one warp each), so a tile never straddles two
//              source partitions;
//   count      each warp counts edges and message starts per key p' over its
//              tile into warp-private shared-memory tables;
//   scan       column-wise exclusive scans of the [tile][p'] tables give every
//              tile its write cursor into every bin, and the column totals give
//              the bin starts. Because tiles follow CSR order, the cursor of the
//              first tile of partition p is exactly the Sec. 3.1 offset of p;
//   fill       each warp replays its tile, ranks equal keys inside a 32-edge
//              window with match/ballot, and writes destination IDs (first of a
//              message flagged) and, for message starts, the source node.
// The result is the canonical bin order: source partitions in ID order, nodes
// in ID order, destinations in adjacency order. Finally the per-chunk update
// bases used by the gather (number of flagged IDs before every kChunk-entry
// chunk), the two largest in-degrees of every bin (kept in registers by the
// gather), largest-first launch orders of bins and source partitions, and
// 1/outdegree are computed.
#include <algorithm>
#include <vector>

#include "pcpm_internal.cuh"

namespace pcpm {
namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// First index i in [lo, hi) with a[i] > x (hi if none); a is non-decreasing.
__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t x) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// v / q for v < 2^32 and q <= 2^15 without a division: with
// m = ceil(2^64 / q), v * m / 2^64 = v / q + e where 0 <= e < 2^-32, and the
// fraction of v / q is at most 1 - 1/q <= 1 - 2^-15, so the floor is exact.
struct DivQ {
    uint64_t m;  // 0 for q = 1
    uint32_t q;
    __device__ __forceinline__ uint32_t operator()(uint32_t v) const {
        return m ? (uint32_t)__umul64hi((uint64_t)v, m) : v;
    }
};
DivQ make_divq(uint32_t q) { return DivQ{q > 1 ? UINT64_MAX / q + 1 : 0, q}; }
static_assert(PCPM_MAX_PART_SIZE <= 32768, "DivQ needs q <= 2^15");

// Exclusive scan of one value per thread over a block of up to 1024 threads.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total, uint32_t* sh32) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh32[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? sh32[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh32[lane] = s;
    }
    __syncthreads();
    const uint32_t prefix = warp ? sh32[warp - 1] : 0;
    *total = sh32[nw - 1];
    __syncthreads();
    return prefix + x - v;
}

// --------------------------------------------------------- small scans
// out[0..N] = exclusive scan of in[0..N), out[N] = total. One block of 1024
// threads, N <= 1024 * kSmallScanItems.
constexpr int kSmallScanItems = 16;

__global__ void __launch_bounds__(1024) scan_small_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                          uint32_t N) {
    __shared__ uint32_t sh32[32];
    const uint32_t per = (N + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(N, threadIdx.x * per), hi = min(N, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += in[i];
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, &total, sh32);
    for (uint32_t i = lo; i < hi; ++i) {
        uint32_t x = in[i];
        out[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) out[N] = total;
}

// Large exclusive scan: block sums, a small scan of the sums, then the blocks.
constexpr uint32_t kScanBlockItems = 4096;  // 1024 threads x 4

__global__ void __launch_bounds__(1024) scan_block_sums_kernel(const uint32_t* __restrict__ in, uint32_t N,
                                                               uint32_t* __restrict__ sums) {
    const uint32_t base = blockIdx.x * kScanBlockItems + threadIdx.x * 4;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += (base + j < N) ? in[base + j] : 0;
    s = __reduce_add_sync(0xffffffffu, s);
    __shared__ uint32_t ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = ws[threadIdx.x];
        t = __reduce_add_sync(0xffffffffu, t);
        if (threadIdx.x == 0) sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) scan_block_apply_kernel(const uint32_t* __restrict__ in, uint32_t N,
                                                                const uint32_t* __restrict__ block_off,
                                                                uint32_t* __restrict__ out) {
    __shared__ uint32_t sh32[32];
    const uint32_t base = blockIdx.x * kScanBlockItems + threadIdx.x * 4;
    uint32_t x[4];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        x[j] = (base + j < N) ? in[base + j] : 0;
        s += x[j];
    }
    uint32_t total;
    uint32_t run = block_off[blockIdx.x] + block_exclusive_scan(s, &total, sh32);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < N) out[base + j] = run;
        run += x[j];
    }
}

// ---------------------------------------------------- CSR validation
__global__ void check_row_ptr_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, int* __restrict__ err) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        if (row_ptr[u] > row_ptr[u + 1]) atomicOr(err, kErrBadGraph);
}

// ------------------------------------------------------ partition tiles
__global__ void partition_tiles_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, uint32_t q, uint32_t k,
                                       uint32_t* __restrict__ tiles) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
        const uint32_t u0 = p * q, u1 = min(n, u0 + q);
        const uint32_t edges = row_ptr[u1] - row_ptr[u0];
        tiles[p] = (edges + kTileEdges - 1) / kTileEdges;
    }
}

// ------------------------------------------------ count / fill of tiles
// One warp per tile. kFill = false: per-tile counts of edges (tab_e) and of
// message starts (tab_u) for every destination partition. kFill = true: the
// tables hold scanned cursors; write the bins.
template <bool kFill>
__global__ void tile_kernel(const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col, uint32_t n,
                            uint32_t q, uint32_t k, const uint32_t* __restrict__ tile_start, uint32_t ntiles,
                            uint32_t* __restrict__ tab_e, uint32_t* __restrict__ tab_u,
                            const uint32_t* __restrict__ bin_e, const uint32_t* __restrict__ bin_u,
                            uint32_t* __restrict__ dest, uint32_t* __restrict__ src, int* __restrict__ err,
                            const float* __restrict__ weights = nullptr, float* __restrict__ wdest = nullptr) {
    extern __shared__ uint32_t sh[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    uint32_t* ce = sh + (size_t)warp * 2 * k;  // edges (count) / ID cursor (fill)
    uint32_t* cu = ce + k;                      // updates / update cursor
    const uint32_t lt = lanemask_lt();

    for (uint32_t t = blockIdx.x * wpc + warp; t < ntiles; t += gridDim.x * wpc) {
        const uint32_t p = upper_bound_u32(tile_start, 0, k + 1, t) - 1;
        const uint32_t u_begin = p * q, u_end = min(n, u_begin + q);
        const uint32_t e_begin = row_ptr[u_begin] + (t - tile_start[p]) * kTileEdges;
        const uint32_t e_end = (uint32_t)min((uint64_t)e_begin + kTileEdges, (uint64_t)row_ptr[u_end]);
        for (uint32_t j = lane; j < k; j += 32) {
            if (kFill) {
                ce[j] = bin_e[j] + tab_e[(size_t)t * k + j];
                cu[j] = bin_u[j] + tab_u[(size_t)t * k + j];
            } else {
                ce[j] = 0;
                cu[j] = 0;
            }
        }
        __syncwarp();
        // Rows covering the tile: the last row starting at or before an edge owns it.
        const uint32_t ulo = upper_bound_u32(row_ptr, u_begin, u_end + 1, e_begin) - 1;
        const uint32_t uhi = upper_bound_u32(row_ptr, ulo, u_end + 1, e_end - 1) - 1;
        uint32_t carry_v = (e_begin > row_ptr[ulo]) ? col[e_begin - 1] : 0;

        for (uint32_t w0 = e_begin; w0 < e_end; w0 += 32) {
            const uint32_t e = w0 + lane;
            bool valid = e < e_end;
            uint32_t u = 0, v = 0;
            if (valid) {
                u = upper_bound_u32(row_ptr, ulo, uhi + 1, e) - 1;
                v = col[e];
            }
            uint32_t prev_v = __shfl_up_sync(0xffffffffu, v, 1);
            if (lane == 0) prev_v = carry_v;
            carry_v = __shfl_sync(0xffffffffu, v, 31);
            uint32_t key = 0xffffffffu;
            bool start = false;
            if (valid) {
                const bool row_start = (e == row_ptr[u]);
                if (v >= n || (!row_start && prev_v > v)) {
                    atomicOr(err, kErrBadGraph);
                    valid = false;
                } else {
                    key = v / q;
                    start = row_start || (prev_v / q != key);
                }
            }
            const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
            const uint32_t smask = __ballot_sync(0xffffffffu, start);
            const uint32_t peers = __match_any_sync(0xffffffffu, key) & vmask;
            if (kFill && valid) {
                const uint32_t pos_e = ce[key] + __popc(peers & lt);
                dest[pos_e] = start ? (v | kMsb) : v;
                if (wdest) wdest[pos_e] = weights[e];  // Sec. 3.5: the weight beside its ID
                if (start) src[cu[key] + __popc(peers & smask & lt)] = u;
            }
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) {
                ce[key] += __popc(peers);
                cu[key] += __popc(peers & smask);
            }
            __syncwarp();
        }
        if (!kFill) {
            for (uint32_t j = lane; j < k; j += 32) {
                tab_e[(size_t)t * k + j] = ce[j];
                tab_u[(size_t)t * k + j] = cu[j];
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------ staged fill of tiles
// The fill of tile_kernel<true> writes every ID straight to its bin: with k
// bins and thousands of tiles in flight, the half-written sectors exceed L2
// and are evicted partial (read-modify-write in DRAM). This fill gives each
// tile one CTA and writes every (tile, bin) run in one piece instead:
//   stage    the tile's col and the local row of every edge (stage_tile: no
//            per-edge search);
//   count    each warp counts its 1/kFillWarps of the tile per key p' with
//            shared atomics (edges in the low, message starts in the high
//            half of one word);
//   scan     per key over warps, then over keys: each warp's cursor in the
//            tile's bin-ordered staging buffers;
//   rank     each warp replays its slice in order, ranks equal keys with
//            match/ballot and stages 16-bit local IDs (bit 15: message flag);
//   copy     one half-warp per bin copies the bin's run of the tile out.
// Same result as tile_kernel<true>: warps own consecutive slices and rank in
// edge order, so the sort stays stable. Local IDs fit 16 bits because
// q <= 32768; k <= kFillMaxK keeps the per-warp tables small.
constexpr int kFillWarps = 8;
constexpr uint32_t kFillSlice = kTileEdges / kFillWarps;
constexpr uint32_t kFillMaxK = 1024;
constexpr uint32_t kFillPerThread = kTileEdges / (kFillWarps * 32);
static_assert(kTileEdges % (kFillWarps * 32) == 0 && kFillPerThread == 32,
              "32 staged edges per thread: four 16-byte words of 2-byte row marks");
static_assert(PCPM_MAX_PART_SIZE <= 32768, "local IDs must fit 15 bits");

size_t fill_smem_bytes(uint32_t k, bool weighted) {
    return (size_t)kTileEdges * (sizeof(uint32_t) + 3 * sizeof(uint16_t) + (weighted ? sizeof(float) : 0)) +
           (size_t)(kFillWarps + 3) * k * sizeof(uint32_t) + sizeof(uint32_t);
}

// Exclusive max-scan of one value per thread over the block.
__device__ uint32_t block_exclusive_max(uint32_t v, uint32_t* sh32) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = max(x, y);
    }
    if (lane == 31) sh32[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? sh32[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s = max(s, y);
        }
        sh32[lane] = s;
    }
    __syncthreads();
    const uint32_t before = warp ? sh32[warp - 1] : 0;
    const uint32_t xl = __shfl_up_sync(0xffffffffu, x, 1);
    __syncthreads();
    return max(before, lane ? xl : 0u);
}

// (source partition, first row) of every tile: the row owning its first edge.
__global__ void tile_info_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, uint32_t q, uint32_t k,
                                 const uint32_t* __restrict__ tile_start, uint32_t ntiles,
                                 uint2* __restrict__ tile_info) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        const uint32_t p = upper_bound_u32(tile_start, 0, k + 1, t) - 1;
        const uint32_t u_begin = p * q, u_end = min(n, u_begin + q);
        const uint32_t e_begin = row_ptr[u_begin] + (t - tile_start[p]) * kTileEdges;
        tile_info[t] = make_uint2(p, upper_bound_u32(row_ptr, u_begin, u_end + 1, e_begin) - 1);
    }
}

// Stages a tile for the staged count and fill: scol = its col, rowof = the
// local row of every edge (each non-empty row marks its first edge in the
// tile; an edge belongs to the last row starting at or before it, and the
// marks rise with the position, so a max-scan carries them forward). Returns
// the tile's bounds. Whole block; ends with a barrier.
struct TileSpan {
    uint32_t p, ulo, u_begin, e_begin, e_end;
    bool first_starts_row;
};
__device__ TileSpan stage_tile(const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col, uint32_t n,
                               uint32_t q, const uint32_t* __restrict__ tile_start,
                               const uint2* __restrict__ tile_info, uint32_t ntiles, uint32_t t, uint32_t* scol,
                               uint16_t* rowof, uint32_t* sh32) {
    const uint32_t tid = threadIdx.x;
    const uint2 ti = tile_info[t];
    TileSpan sp;
    sp.p = ti.x;
    sp.ulo = ti.y;
    sp.u_begin = sp.p * q;
    const uint32_t u_end = min(n, sp.u_begin + q);
    sp.e_begin = row_ptr[sp.u_begin] + (t - tile_start[sp.p]) * kTileEdges;
    sp.e_end = (uint32_t)min((uint64_t)sp.e_begin + kTileEdges, (uint64_t)row_ptr[u_end]);
    sp.first_starts_row = sp.e_begin == row_ptr[sp.ulo];
    const uint32_t L = sp.e_end - sp.e_begin;
    // rows up to the next tile's first row (or the partition's last) cover the tile
    const uint32_t rhi = (t + 1 < ntiles && tile_start[sp.p + 1] > t + 1) ? tile_info[t + 1].y : u_end - 1;
    {
        uint32_t x[kFillPerThread];
#pragma unroll
        for (uint32_t j = 0; j < kFillPerThread; ++j) {
            const uint32_t i = j * blockDim.x + tid;
            x[j] = i < L ? __ldcs(col + sp.e_begin + i) : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < kFillPerThread; ++j) {
            const uint32_t i = j * blockDim.x + tid;
            scol[i] = x[j];
            rowof[i] = 0;
        }
    }
    __syncthreads();
    for (uint32_t r = sp.ulo + tid; r <= rhi; r += blockDim.x) {
        const uint32_t a = row_ptr[r], b = row_ptr[r + 1];
        if (b > a && b > sp.e_begin && a < sp.e_end)
            rowof[a > sp.e_begin ? a - sp.e_begin : 0] = (uint16_t)(r - sp.ulo);
    }
    __syncthreads();
    {
        // a thread's 32 consecutive marks as four 16-byte words (scalar 2-byte
        // accesses at a 64-byte stride would hit two banks per warp)
        uint4* mine = reinterpret_cast<uint4*>(rowof + tid * kFillPerThread);
        uint4 w[4];
        uint32_t mx = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            w[c] = mine[c];
            mx = max(mx, max(max(max(w[c].x & 0xFFFFu, w[c].x >> 16), max(w[c].y & 0xFFFFu, w[c].y >> 16)),
                             max(max(w[c].z & 0xFFFFu, w[c].z >> 16), max(w[c].w & 0xFFFFu, w[c].w >> 16))));
        }
        uint32_t run = block_exclusive_max(mx, sh32);
        auto carry2 = [&run](uint32_t x) {  // two marks, low half first
            const uint32_t lo = run = max(run, x & 0xFFFFu);
            const uint32_t hi = run = max(run, x >> 16);
            return lo | (hi << 16);
        };
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            w[c].x = carry2(w[c].x);
            w[c].y = carry2(w[c].y);
            w[c].z = carry2(w[c].z);
            w[c].w = carry2(w[c].w);
            mine[c] = w[c];
        }
    }
    __syncthreads();
    return sp;
}

// Count pass for k <= kFillMaxK: one CTA per tile counts edges and message
// starts per key p' with shared-memory atomics (one packed word per key:
// edges in the low, starts in the high half; counting needs no order) and
// writes the tile's row of tab_e and tab_u. Same tables as tile_kernel<false>.
__global__ void __launch_bounds__(kFillWarps * 32) count_staged_kernel(
    const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col, uint32_t n, DivQ div, uint32_t k,
    const uint32_t* __restrict__ tile_start, const uint2* __restrict__ tile_info, uint32_t ntiles,
    uint32_t* __restrict__ tab_e, uint32_t* __restrict__ tab_u, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ uint32_t sh32[32];
    uint32_t* scol = reinterpret_cast<uint32_t*>(fsm);
    uint16_t* rowof = reinterpret_cast<uint16_t*>(scol + kTileEdges);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(rowof + kTileEdges);  // k packed counters
    const uint32_t tid = threadIdx.x, q = div.q;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (uint32_t j = tid; j < k; j += blockDim.x) cnt[j] = 0;
        const TileSpan sp = stage_tile(row_ptr, col, n, q, tile_start, tile_info, ntiles, t, scol, rowof, sh32);
        const uint32_t L = sp.e_end - sp.e_begin;
        const uint32_t prev0 = (L && !sp.first_starts_row) ? col[sp.e_begin - 1] : 0u;
        for (uint32_t i = tid; i < L; i += blockDim.x) {
            const uint32_t v = scol[i], r = rowof[i];
            const bool row_start = i == 0 ? sp.first_starts_row : rowof[i - 1] != r;
            const uint32_t prev_v = i == 0 ? prev0 : scol[i - 1];
            if (v >= n || (!row_start && prev_v > v)) {
                atomicOr(err, kErrBadGraph);
                continue;
            }
            const uint32_t key = div(v);
            const bool start = row_start || prev_v < key * q;  // prev_v <= v in a row
            atomicAdd(&cnt[key], 1u | (start ? 0x10000u : 0u));
        }
        __syncthreads();
        for (uint32_t j = tid; j < k; j += blockDim.x) {
            const uint32_t c = cnt[j];
            tab_e[(size_t)t * k + j] = c & 0xFFFFu;
            tab_u[(size_t)t * k + j] = c >> 16;
        }
        __syncthreads();
    }
}

size_t count_smem_bytes(uint32_t k) {
    return (size_t)kTileEdges * (sizeof(uint32_t) + sizeof(uint16_t)) + (size_t)k * sizeof(uint32_t);
}

__global__ void __launch_bounds__(kFillWarps * 32) fill_staged_kernel(
    const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col, uint32_t n, DivQ div, uint32_t k,
    const uint32_t* __restrict__ tile_start, const uint2* __restrict__ tile_info, uint32_t ntiles,
    const uint32_t* __restrict__ tab_e, const uint32_t* __restrict__ tab_u, const uint32_t* __restrict__ bin_e,
    const uint32_t* __restrict__ bin_u, uint32_t* __restrict__ dest, uint32_t* __restrict__ src,
    int* __restrict__ err, const float* __restrict__ weights, float* __restrict__ wdest) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ uint32_t sh32[32];
    uint32_t* scol = reinterpret_cast<uint32_t*>(fsm);        // the tile's col
    uint16_t* rowof = reinterpret_cast<uint16_t*>(scol + kTileEdges);  // local row of each edge
    uint16_t* d16 = rowof + kTileEdges;                       // staged IDs, bin order
    uint16_t* s16 = d16 + kTileEdges;                         // staged sources, bin order
    float* wst = reinterpret_cast<float*>(s16 + kTileEdges);  // staged weights (weighted graphs)
    uint32_t* hist = reinterpret_cast<uint32_t*>(wst + (weights ? kTileEdges : 0));  // [warp][key]
    uint32_t* loff = hist + (size_t)kFillWarps * k;           // k + 1 run starts in the staging buffers
    uint32_t* gbe = loff + k + 1;                             // k: the tile's cursor in bin p' (IDs)
    uint32_t* gbu = gbe + k;                                  // k: the same for updates
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t q = div.q;

    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (uint32_t j = tid; j < kFillWarps * k; j += blockDim.x) hist[j] = 0;
        for (uint32_t j = tid; j < k; j += blockDim.x) {
            gbe[j] = bin_e[j] + tab_e[(size_t)t * k + j];
            gbu[j] = bin_u[j] + tab_u[(size_t)t * k + j];
        }
        const TileSpan sp = stage_tile(row_ptr, col, n, q, tile_start, tile_info, ntiles, t, scol, rowof, sh32);
        const uint32_t ulo = sp.ulo, u_begin = sp.u_begin, e_begin = sp.e_begin, L = sp.e_end - sp.e_begin;

        // One pass over the warp's slice; body(valid, i, v, local row, key,
        // start, peers, smask) runs once per 32 edges (warp-collective).
        const uint32_t s_lo = min(L, warp * kFillSlice), s_hi = min(L, s_lo + kFillSlice);
        const bool first_starts_row = sp.first_starts_row;
        auto walk = [&](auto&& body) {
            uint32_t carry = 0;
            if (s_lo > 0 && s_lo < s_hi) carry = scol[s_lo - 1];
            else if (s_lo == 0 && !first_starts_row) carry = col[e_begin - 1];
            for (uint32_t i0 = s_lo; i0 < s_hi; i0 += 32) {
                const uint32_t i = i0 + lane;
                bool valid = i < s_hi;
                uint32_t v = 0, r = 0;
                bool row_start = false;
                if (valid) {
                    v = scol[i];
                    r = rowof[i];
                    row_start = i == 0 ? first_starts_row : rowof[i - 1] != r;
                }
                uint32_t prev_v = __shfl_up_sync(0xffffffffu, v, 1);
                if (lane == 0) prev_v = carry;
                carry = __shfl_sync(0xffffffffu, v, 31);
                uint32_t key = 0xffffffffu;
                bool start = false;
                if (valid) {
                    if (v >= n || (!row_start && prev_v > v)) {
                        atomicOr(err, kErrBadGraph);
                        valid = false;
                    } else {
                        key = div(v);
                        start = row_start || prev_v < key * q;  // prev_v <= v in a row
                    }
                }
                const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
                const uint32_t smask = __ballot_sync(0xffffffffu, start);
                const uint32_t peers = __match_any_sync(0xffffffffu, key) & vmask;
                body(valid, i, v, r, key, start, peers, smask);
                __syncwarp();
            }
        };
        // count the warp's slice per key (no order needed: shared atomics)
        {
            const uint32_t prev0 = (L && !first_starts_row) ? col[e_begin - 1] : 0u;
            for (uint32_t i = s_lo + lane; i < s_hi; i += 32) {
                const uint32_t v = scol[i], r = rowof[i];
                const bool row_start = i == 0 ? first_starts_row : rowof[i - 1] != r;
                const uint32_t prev_v = i == 0 ? prev0 : scol[i - 1];
                if (v >= n || (!row_start && prev_v > v)) continue;  // reported by the rank pass
                const uint32_t key = div(v);
                const bool start = row_start || prev_v < key * q;
                atomicAdd(&hist[warp * k + key], 1u | (start ? 0x10000u : 0u));
            }
        }
        __syncthreads();
        // scan: per key over warps, then over keys (both halves at once: each
        // total is at most kTileEdges < 2^16)
        for (uint32_t j = tid; j < k; j += blockDim.x) {
            uint32_t run = 0;
            for (int w = 0; w < kFillWarps; ++w) {
                const uint32_t x = hist[w * k + j];
                hist[w * k + j] = run;
                run += x;
            }
            loff[j] = run;
        }
        __syncthreads();
        {
            const uint32_t per = (k + blockDim.x - 1) / blockDim.x;
            const uint32_t j0 = min(k, tid * per), j1 = min(k, j0 + per);
            uint32_t sum = 0;
            for (uint32_t j = j0; j < j1; ++j) sum += loff[j];
            uint32_t total;
            uint32_t run = block_exclusive_scan(sum, &total, sh32);
            for (uint32_t j = j0; j < j1; ++j) {
                const uint32_t x = loff[j];
                loff[j] = run;
                run += x;
            }
            if (tid == 0) loff[k] = total;
        }
        __syncthreads();
        for (uint32_t j = tid; j < k; j += blockDim.x) {
            const uint32_t b = loff[j];
            for (int w = 0; w < kFillWarps; ++w) hist[w * k + j] += b;
        }
        __syncthreads();
        // rank and stage
        walk([&](bool valid, uint32_t i, uint32_t v, uint32_t r, uint32_t key, bool start, uint32_t peers,
                 uint32_t smask) {
            if (valid) {
                const uint32_t c = hist[warp * k + key];
                const uint32_t pe = (c & 0xFFFFu) + __popc(peers & lt);
                d16[pe] = (uint16_t)((v - key * q) | (start ? 0x8000u : 0u));
                if (weights) wst[pe] = weights[e_begin + i];  // Sec. 3.5: the weight beside its ID
                if (start) s16[(c >> 16) + __popc(peers & smask & lt)] = (uint16_t)(ulo + r - u_begin);
            }
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1)
                hist[warp * k + key] += __popc(peers) | (__popc(peers & smask) << 16);
        });
        __syncthreads();
        // copy each bin's run out (a half-warp per bin: runs are short)
        const uint32_t hl = lane & 15;
        for (uint32_t j = 2 * warp + (lane >> 4); j < k; j += 2 * kFillWarps) {
            const uint32_t a = loff[j], b = loff[j + 1];
            const uint32_t ae = a & 0xFFFFu, be = b & 0xFFFFu, au = a >> 16, bu = b >> 16;
            const uint32_t ge = gbe[j], gu = gbu[j], vbase = j * q;
            for (uint32_t i = ae + hl; i < be; i += 16) {
                const uint32_t x = d16[i];
                dest[ge + (i - ae)] = (vbase + (x & 0x7FFFu)) | ((x & 0x8000u) ? kMsb : 0u);
                if (weights) wdest[ge + (i - ae)] = wst[i];
            }
            for (uint32_t i = au + hl; i < bu; i += 16) src[gu + (i - au)] = u_begin + s16[i];
        }
        __syncthreads();
    }
}

// ------------------------------------------------ column scans of tables
// A table is [nrows + 1][k]; rows are tiles. After the three kernels, row r
// holds the exclusive column prefix over rows < r and row nrows the totals.
constexpr uint32_t kColRows = 256;  // rows per block (multiple of 32)

__global__ void __launch_bounds__(1024) colscan_sums_kernel(const uint32_t* __restrict__ tab, uint32_t nrows,
                                                            uint32_t k, uint32_t* __restrict__ bsum) {
    __shared__ uint32_t red[32][33];
    const uint32_t tx = threadIdx.x, ty = threadIdx.y;
    const uint32_t key = blockIdx.x * 32 + tx;
    const uint32_t r0 = blockIdx.y * kColRows, r1 = min(nrows, r0 + kColRows);
    uint32_t s = 0;
    if (key < k)
        for (uint32_t r = r0 + ty; r < r1; r += 32) s += tab[(size_t)r * k + key];
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && key < k) {
        uint32_t t = 0;
        for (int i = 0; i < 32; ++i) t += red[i][tx];
        bsum[(size_t)blockIdx.y * k + key] = t;
    }
}

__global__ void colscan_blocks_kernel(uint32_t* __restrict__ bsum, uint32_t nb, uint32_t k,
                                      uint32_t* __restrict__ tab, uint32_t nrows, uint32_t* __restrict__ totals) {
    const uint32_t key = blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= k) return;
    uint32_t run = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        const uint32_t x = bsum[(size_t)b * k + key];
        bsum[(size_t)b * k + key] = run;
        run += x;
    }
    tab[(size_t)nrows * k + key] = run;
    totals[key] = run;
}

__global__ void __launch_bounds__(1024) colscan_apply_kernel(uint32_t* __restrict__ tab, uint32_t nrows, uint32_t k,
                                                             const uint32_t* __restrict__ boff) {
    __shared__ uint32_t sm[32][33];
    __shared__ uint32_t carry[32];
    const uint32_t tx = threadIdx.x, ty = threadIdx.y;
    const uint32_t key = blockIdx.x * 32 + tx;
    const uint32_t r0 = blockIdx.y * kColRows, r1 = min(nrows, r0 + kColRows);
    if (ty == 0) carry[tx] = key < k ? boff[(size_t)blockIdx.y * k + key] : 0;
    __syncthreads();
    for (uint32_t g = r0; g < r1; g += 32) {
        const uint32_t r = g + ty;
        const bool ok = key < k && r < r1;
        sm[ty][tx] = ok ? tab[(size_t)r * k + key] : 0;
        __syncthreads();
        // warp ty scans key column ty of this block over rows tx
        const uint32_t y = sm[tx][ty];
        uint32_t incl = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t z = __shfl_up_sync(0xffffffffu, incl, o);
            if (tx >= o) incl += z;
        }
        const uint32_t c = carry[ty];
        sm[tx][ty] = c + incl - y;
        __syncthreads();
        if (tx == 31) carry[ty] = c + incl;
        if (ok) tab[(size_t)r * k + key] = sm[ty][tx];
        __syncthreads();
    }
}

// --------------------------------------------------- segments and chunks
// seg_x[p][p'] = absolute start of the entries partition p writes into bin p';
// cnt_x[p][p'] = their number. Row tile_start[p] of a scanned table is the
// Sec. 3.1 offset of partition p (row ntiles = column totals).
__global__ void segments_kernel(const uint32_t* __restrict__ tab, const uint32_t* __restrict__ tile_start,
                                const uint32_t* __restrict__ bin, uint32_t k, uint32_t* __restrict__ seg,
                                uint32_t* __restrict__ cnt) {
    const uint64_t total = (uint64_t)k * k;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = (uint32_t)(i / k), pd = (uint32_t)(i % k);
        const uint32_t off = tab[(size_t)tile_start[p] * k + pd];
        const uint32_t nxt = tab[(size_t)tile_start[p + 1] * k + pd];
        seg[i] = bin[pd] + off;
        cnt[i] = nxt - off;
    }
}

// Flagged IDs per kChunk-entry chunk (one warp per chunk).
__global__ void chunk_flags_kernel(const uint32_t* __restrict__ dest, uint64_t m, uint64_t nchunks,
                                   uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t c = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < nchunks; c += warps) {
        uint32_t s = 0;
        for (uint32_t j = lane; j < kChunk; j += 32) {
            const uint64_t pos = c * kChunk + j;
            if (pos < m) s += dest[pos] >> 31;
        }
        s = __reduce_add_sync(0xffffffffu, s);
        if (lane == 0) cnt[c] = s;
    }
}

__global__ void inv_deg_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, float* __restrict__ inv) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const uint32_t deg = row_ptr[u + 1] - row_ptr[u];
        inv[u] = deg ? 1.0f / (float)deg : 0.0f;
    }
}

// ------------------------------------------------------ destination shards
// A destination shard keeps the edges into nodes [vlo, vhi). One warp per row
// decides with one predicate in both passes (a ballot per 32 columns), so the
// copy writes exactly the counted columns whatever the row's order; a row
// whose offsets decrease or pass m, or a column >= n, sets kErrBadGraph and
// keeps nothing of that row.
__device__ __forceinline__ bool shard_row(const uint32_t* row_ptr, uint32_t u, uint64_t m, uint32_t& lo,
                                          uint32_t& hi) {
    lo = row_ptr[u];
    hi = row_ptr[u + 1];
    return hi >= lo && hi <= m;
}

__global__ void shard_count_kernel(const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                                   uint32_t n, uint64_t m, uint32_t vlo, uint32_t vhi, uint32_t* __restrict__ cnt,
                                   int* __restrict__ err) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        uint32_t lo, hi, c = 0;
        bool bad = !shard_row(row_ptr, (uint32_t)u, m, lo, hi);
        if (!bad)
            for (uint32_t e = lo; e < hi; e += 32) {
                const uint32_t v = e + lane < hi ? col[e + lane] : vlo;
                bad |= __any_sync(0xffffffffu, e + lane < hi && v >= n);
                c += __popc(__ballot_sync(0xffffffffu, e + lane < hi && v >= vlo && v < vhi));
            }
        if (lane == 0) {
            cnt[u] = bad ? 0u : c;
            if (bad) atomicOr(err, kErrBadGraph);
        }
    }
}

__global__ void shard_copy_kernel(const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                                  uint32_t n, uint64_t m, uint32_t vlo, uint32_t vhi,
                                  const uint32_t* __restrict__ out_ptr, uint32_t* __restrict__ out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        uint32_t lo, hi;
        const uint32_t o0 = out_ptr[u], o1 = out_ptr[u + 1];
        if (!shard_row(row_ptr, (uint32_t)u, m, lo, hi) || o1 == o0) continue;
        uint32_t o = o0;
        for (uint32_t e = lo; e < hi; e += 32) {
            const uint32_t v = e + lane < hi ? col[e + lane] : vlo;
            const bool keep = e + lane < hi && v >= vlo && v < vhi && v < n;
            const uint32_t b = __ballot_sync(0xffffffffu, keep);
            const uint32_t at = o + __popc(b & ((1u << lane) - 1u));
            if (keep && at < o1) out[at] = v;
            o += __popc(b);
        }
    }
}

// Edges per destination partition: a shared-memory histogram per CTA (k <=
// PCPM_MAX_PARTITIONS counters), added to the global 64-bit counts once.
__global__ void __launch_bounds__(1024) dest_hist_kernel(const uint32_t* __restrict__ col, uint64_t m, uint32_t n,
                                                         DivQ div, uint32_t k,
                                                         unsigned long long* __restrict__ counts,
                                                         int* __restrict__ err) {
    __shared__ uint32_t h[PCPM_MAX_PARTITIONS];
    for (uint32_t p = threadIdx.x; p < k; p += blockDim.x) h[p] = 0;
    __syncthreads();
    bool bad = false;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = col[e];
        if (v >= n) bad = true;
        else atomicAdd(&h[div(v)], 1u);
    }
    if (bad) atomicOr(err, kErrBadGraph);
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < k; p += blockDim.x)
        if (h[p]) atomicAdd(&counts[p], (unsigned long long)h[p]);
}

// In-degree of every node.
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long x, unsigned long long* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    x = lane < nw ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
    __syncthreads();
    return x;
}

// Per destination partition p: local IDs of the two nodes with the largest
// in-degree (ties to the lower ID), kNoHub below kHubMinInDegree. The gather
// sums their updates in registers instead of contended shared-memory atomics.
// Every in-edge of a node of p lies in bin p, so the in-degrees are counted
// in shared memory from the bin's IDs (one CTA per bin).
__global__ void __launch_bounds__(1024) bin_hubs_kernel(const uint32_t* __restrict__ dest,
                                                        const uint32_t* __restrict__ bin_e, uint32_t n, uint32_t q,
                                                        uint32_t* __restrict__ hubs) {
    extern __shared__ uint32_t deg[];
    __shared__ unsigned long long sh[32];
    const uint32_t p = blockIdx.x, base = p * q, len = min(q, n - base);
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) deg[i] = 0;
    __syncthreads();
    const uint32_t e0 = bin_e[p], e1 = bin_e[p + 1];
    constexpr uint32_t kIlp = 4;
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += kIlp * blockDim.x) {
        uint32_t loc[kIlp];
#pragma unroll
        for (uint32_t j = 0; j < kIlp; ++j) {
            const uint32_t x = e + j * blockDim.x;
            loc[j] = x < e1 ? (__ldcs(dest + x) & kIdMask) - base : 0xFFFFFFFFu;
        }
#pragma unroll
        for (uint32_t j = 0; j < kIlp; ++j)
            if (loc[j] < len) atomicAdd(&deg[loc[j]], 1u);
    }
    __syncthreads();
    unsigned long long best = 0;
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
        best = max(best, ((unsigned long long)deg[i] << 32) | (0xFFFFFFFFu - i));
    const unsigned long long b1 = block_max_u64(best, sh);
    unsigned long long second = 0;
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        const unsigned long long key = ((unsigned long long)deg[i] << 32) | (0xFFFFFFFFu - i);
        if (key != b1) second = max(second, key);
    }
    const unsigned long long b2 = block_max_u64(second, sh);
    if (threadIdx.x == 0) {
        hubs[2 * p] = (b1 >> 32) >= kHubMinInDegree ? 0xFFFFFFFFu - (uint32_t)b1 : kNoHub;
        hubs[2 * p + 1] = (b2 >> 32) >= kHubMinInDegree ? 0xFFFFFFFFu - (uint32_t)b2 : kNoHub;
    }
}

// groups[p] = 4-entry groups the scatter of source partition p writes.
__global__ void src_groups_kernel(const uint32_t* __restrict__ seg_u, const uint32_t* __restrict__ cnt_u, uint32_t k,
                                  uint32_t* __restrict__ size) {
    const uint32_t p = blockIdx.x;
    uint32_t s = 0;
    for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) {
        const uint32_t a = seg_u[(size_t)p * k + j], c = cnt_u[(size_t)p * k + j];
        s += c ? ((a + c + 3) >> 2) - (a >> 2) : 0;
    }
    s = __reduce_add_sync(0xffffffffu, s);
    __shared__ uint32_t ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
        t = __reduce_add_sync(0xffffffffu, t);
        if (threadIdx.x == 0) size[p] = t;
    }
}

// order[rank] = p by decreasing size (ties to the lower index): the largest
// units are launched first so the last wave is made of small ones.
__global__ void order_kernel(const uint32_t* __restrict__ size, uint32_t k, uint32_t* __restrict__ order) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint32_t si = size[i];
        uint32_t rank = 0;
        for (uint32_t j = 0; j < k; ++j) {
            const uint32_t sj = size[j];
            rank += (sj > si) || (sj == si && j < i);
        }
        order[rank] = i;
    }
}

// ------------------------------------------------------------ work units
// Chunks of bin p: [first, first + count). Canonical layout: the globally
// aligned kChunk-entry chunks the bin overlaps; bank-spread layout: the bin's
// own padded chunks.
__device__ __forceinline__ void bin_chunks(const uint32_t* bin_e, const uint32_t* ichunk_start, uint32_t p,
                                           uint32_t& first, uint32_t& count) {
    if (ichunk_start) {
        first = ichunk_start[p];
        count = ichunk_start[p + 1] - first;
    } else {
        const uint32_t e0 = bin_e[p], e1 = bin_e[p + 1];
        first = e0 / kChunk;
        count = e1 > e0 ? (e1 - 1) / kChunk - first + 1 : 0;
    }
}

// pieces[p] = units of bin p: its chunks cut into runs of at most `per`
// (an empty bin still gets one unit for its apply). Bins outside the
// handle's destination shard [plo, phi) get none: no other node is applied.
__global__ void gather_pieces_kernel(const uint32_t* __restrict__ bin_e, const uint32_t* __restrict__ ichunk_start,
                                     uint32_t k, uint32_t per, uint32_t plo, uint32_t phi,
                                     uint32_t* __restrict__ pieces) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
        uint32_t first, nch;
        bin_chunks(bin_e, ichunk_start, p, first, nch);
        pieces[p] = (p < plo || p >= phi) ? 0u : nch ? (nch + per - 1) / per : 1u;
    }
}

__global__ void gather_units_kernel(const uint32_t* __restrict__ bin_e, const uint32_t* __restrict__ ichunk_start,
                                    const uint32_t* __restrict__ start, uint32_t k, uint32_t per, uint32_t nunits,
                                    uint4* __restrict__ units, uint32_t* __restrict__ sizes) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < nunits; u += gridDim.x * blockDim.x) {
        const uint32_t p = upper_bound_u32(start, 0, k + 1, u) - 1;
        uint32_t c0, nch;
        bin_chunks(bin_e, ichunk_start, p, c0, nch);
        const uint32_t idx = u - start[p];
        const uint32_t lo = c0 + min(nch, idx * per), hi = c0 + min(nch, (idx + 1) * per);
        units[u] = make_uint4(p, lo, hi, start[p + 1] - start[p]);
        sizes[u] = hi - lo;
    }
}

// ------------------------------------------------- bank-spread gather layout
__global__ void bin_chunk_counts_kernel(const uint32_t* __restrict__ bin_e, uint32_t k, uint32_t* __restrict__ cnt) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
        cnt[p] = (bin_e[p + 1] - bin_e[p] + kChunk - 1) / kChunk;
}

constexpr int kLayoutWarps = 8;
constexpr uint32_t kKeyHub = 32, kKeyPad = 33, kNumKeys = 34;

// One warp per padded chunk: the update index of every ID (flags before the
// chunk plus the inclusive count inside it, minus one), then a stable counting
// sort of the chunk's IDs by shared-memory bank of their destination (hub
// destinations, which the gather sums in per-warp slots, and padding sort
// last). Inside a group, IDs are ordered by slot. Sorted position s goes to
// round s % 8 and lane s / 8 of the gather's 8-round, 32-lane pass over the
// chunk: the 32 adds of a round come from every eighth sorted ID (distinct
// banks unless a bank holds more than eight of the chunk's IDs), and each
// lane's eight IDs are consecutive in sorted order, so repeated destinations
// meet in one lane.
__global__ void __launch_bounds__(kLayoutWarps * 32) gather_layout_kernel(
    const uint32_t* __restrict__ dest, const uint32_t* __restrict__ bin_e, const uint32_t* __restrict__ ichunk_start,
    uint32_t k, const uint32_t* __restrict__ chunk_base, const uint32_t* __restrict__ hubs, uint32_t q,
    uint64_t nichunks, uint32_t* __restrict__ gdest, uint32_t* __restrict__ slice_start,
    uint32_t* __restrict__ slice_bytes, uint32_t upd_bytes, unsigned long long* __restrict__ stats,
    const float* __restrict__ wdest = nullptr, float* __restrict__ gweight = nullptr) {
    __shared__ uint32_t keycnt[kLayoutWarps][kNumKeys + 2];
    __shared__ uint32_t sortbuf[kLayoutWarps][kChunk];
    __shared__ float sortw[kLayoutWarps][kChunk];  // weighted graphs: weights follow their IDs
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    uint32_t* cnt = keycnt[warp];
    uint32_t nmerged = 0;
    bool bad = false;
    uint32_t p = 0;  // the warp's chunks rise, so their bins do too
    for (uint64_t ic = blockIdx.x * (uint64_t)kLayoutWarps + warp; ic < nichunks;
         ic += (uint64_t)gridDim.x * kLayoutWarps) {
        {  // bin of chunk ic: the last p with ichunk_start[p] <= ic, galloping from the last one
            uint32_t step = 1;
            while (p + step < k && ichunk_start[p + step] <= (uint32_t)ic) {
                p += step;
                step <<= 1;
            }
            p = upper_bound_u32(ichunk_start, p, min(k, p + step), (uint32_t)ic) - 1;
        }
        const uint32_t P = bin_e[p] + ((uint32_t)ic - ichunk_start[p]) * kChunk;
        const uint32_t Pend = min(P + kChunk, bin_e[p + 1]);
        const uint32_t vbase = p * q, h0 = hubs[2 * p], h1 = hubs[2 * p + 1];
        // flagged IDs before P
        const uint32_t cbase = P & ~(kChunk - 1);
        uint32_t running = chunk_base[P / kChunk];
        for (uint32_t x = cbase; x < P; x += 32) {
            const uint32_t pos = x + lane;
            running += __popc(__ballot_sync(0xffffffffu, pos < P && (dest[pos] >> 31)));
        }
        uint32_t idx[kChunk / 32], loc[kChunk / 32], key[kChunk / 32];
#pragma unroll
        for (int r = 0; r < (int)(kChunk / 32); ++r) {
            const uint32_t pos = P + 32 * r + lane;
            const bool valid = pos < Pend;
            const uint32_t w = valid ? dest[pos] : 0u;
            const uint32_t b = __ballot_sync(0xffffffffu, valid && (w >> 31));
            idx[r] = running + __popc(b & (lt | (1u << lane))) - 1;
            running += __popc(b);
            loc[r] = (w & kIdMask) - vbase;
            key[r] = !valid ? kKeyPad : (loc[r] == h0 || loc[r] == h1) ? kKeyHub : (loc[r] & 31u);
        }
        const uint32_t n = Pend - P;
        const uint32_t u_first = __shfl_sync(0xffffffffu, idx[0], 0);
        uint32_t u_last = 0;
#pragma unroll
        for (int r = 0; r < (int)(kChunk / 32); ++r) {
            const uint32_t x = __shfl_sync(0xffffffffu, idx[r], (n - 1) & 31);
            if ((uint32_t)r == (n - 1) / 32) u_last = x;
        }
        // the chunk's update slice, widened to 16-byte boundaries
        const uint32_t align = 16u / upd_bytes, slot_max = min((kUpdSlot * 4u) / upd_bytes, kGwUpdMask + 1);
        const uint32_t us = u_first & ~(align - 1), ue = (u_last + align) & ~(align - 1);
        // counting sort by key, stable in (round, lane) order
        for (uint32_t j = lane; j < kNumKeys; j += 32) cnt[j] = 0;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < (int)(kChunk / 32); ++r) {
            const uint32_t peers = __match_any_sync(0xffffffffu, key[r]);
            if (lane == (uint32_t)(__ffs(peers) - 1)) cnt[key[r]] += __popc(peers);
            __syncwarp();
        }
        {  // exclusive scan of the counts: bank groups (one per lane), then hub and padding
            const uint32_t c = cnt[lane], c_hub = cnt[kKeyHub];
            uint32_t x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            const uint32_t banks = __shfl_sync(0xffffffffu, x, 31);
            __syncwarp();
            cnt[lane] = x - c;
            if (lane == 0) {
                cnt[kKeyHub] = banks;
                cnt[kKeyPad] = banks + c_hub;
            }
            static_assert(kKeyHub == 32 && kKeyPad == 33 && kNumKeys == 34, "32 bank groups, then hub and padding");
        }
        __syncwarp();
        // gather words staged by sorted position
        uint32_t* sorted = sortbuf[warp];
#pragma unroll
        for (int r = 0; r < (int)(kChunk / 32); ++r) {
            const uint32_t peers = __match_any_sync(0xffffffffu, key[r]);
            const uint32_t pos = cnt[key[r]] + __popc(peers & lt);
            __syncwarp();
            if (lane == (uint32_t)(__ffs(peers) - 1)) cnt[key[r]] += __popc(peers);
            __syncwarp();
            // padding: the pad slot of the lane that will hold it (distinct
            // banks within a round); hubs: the hub slot pair
            const uint32_t slot = key[r] == kKeyHub ? q + kPadSlots + (loc[r] == h1 ? 1u : 0u) : loc[r];
            sorted[pos] = key[r] == kKeyPad ? q + (pos >> 3) : (slot | ((idx[r] - us) << kGwUpdShift));
            if (gweight) sortw[warp][pos] = key[r] == kKeyPad ? 0.0f : wdest[P + 32 * r + lane];
            if (key[r] != kKeyPad && (loc[r] >= q || idx[r] - us >= slot_max)) bad = true;
        }
        __syncwarp();
        // cnt[j] now holds the end of group j; group j starts at cnt[j - 1].
        // Inside each bank group (one per lane), and in the hub group, order
        // IDs by slot, so equal destinations sit next to each other and the
        // gather sums them in a register before one shared-memory add. The
        // padding group is in slot order already.
        {
            const uint32_t grp = lane;
            const uint32_t g_end = cnt[grp], g_beg = grp ? cnt[grp - 1] : 0;
            for (uint32_t x = g_beg + 1; x < g_end; ++x) {
                const uint32_t w = sorted[x];
                const float wt = gweight ? sortw[warp][x] : 0.0f;
                uint32_t y = x;
                while (y > g_beg && (sorted[y - 1] & kGwLocMask) > (w & kGwLocMask)) {
                    sorted[y] = sorted[y - 1];
                    if (gweight) sortw[warp][y] = sortw[warp][y - 1];
                    --y;
                }
                sorted[y] = w;
                if (gweight) sortw[warp][y] = wt;
            }
        }
        __syncwarp();
        {  // the hub group holds two slots: a stable partition, first hub first
            const uint32_t hb = cnt[kKeyHub - 1], he = cnt[kKeyHub], hub0 = q + kPadSlots;
            uint32_t w[kChunk / 32], n0 = 0;
            float wt[kChunk / 32];
#pragma unroll
            for (int r = 0; r < (int)(kChunk / 32); ++r) {
                const uint32_t x = hb + 32 * r + lane;
                w[r] = x < he ? sorted[x] : 0u;
                wt[r] = (gweight && x < he) ? sortw[warp][x] : 0.0f;
                n0 += __popc(__ballot_sync(0xffffffffu, x < he && (w[r] & kGwLocMask) == hub0));
            }
            __syncwarp();
            uint32_t r0 = 0, r1 = 0;
#pragma unroll
            for (int r = 0; r < (int)(kChunk / 32); ++r) {
                const uint32_t x = hb + 32 * r + lane;
                const bool live = x < he, first = (w[r] & kGwLocMask) == hub0;
                const uint32_t b0 = __ballot_sync(0xffffffffu, live && first);
                const uint32_t b1 = __ballot_sync(0xffffffffu, live && !first);
                if (live) {
                    const uint32_t to = first ? hb + r0 + __popc(b0 & lt) : hb + n0 + r1 + __popc(b1 & lt);
                    sorted[to] = w[r];
                    if (gweight) sortw[warp][to] = wt[r];
                }
                r0 += __popc(b0);
                r1 += __popc(b1);
            }
        }
        __syncwarp();
        // Position s goes to round s % 8, lane s / 8 of the gather's pass.
        // The run bit marks an ID whose successor in the same lane has the
        // same slot (not a padding slot): the gather adds it to a register
        // run instead of shared memory.
        uint32_t* out = gdest + ic * kChunk;
        for (uint32_t sp = lane; sp < kChunk; sp += 32) {
            const uint32_t round = sp & 7u, slot_lane = sp >> 3;
            uint32_t w = sorted[sp];
            const uint32_t l = w & kGwLocMask;
            const bool pad = l >= q && l < q + kPadSlots;
            if (round != 7u && !pad && (sorted[sp + 1] & kGwLocMask) == l) w |= kGwRunBit;
            nmerged += __popc(__ballot_sync(0xffffffffu, (w & kGwRunBit) != 0));
            const uint32_t o = 128 * (round >> 2) + 4 * slot_lane + (round & 3u);
            out[o] = w;
            if (gweight) gweight[ic * kChunk + o] = sortw[warp][sp];
        }
        if (lane == 0) {
            slice_start[ic] = us;
            slice_bytes[ic] = (ue - us) * upd_bytes;
            if (ue - us > slot_max) bad = true;
        }
        __syncwarp();
    }
    // stats[0]: IDs with the run bit; stats[1]: nonzero if a word would
    // address outside the accumulator or the chunk's update slice (the gather
    // relies on this check instead of testing every ID).
    if (lane == 0 && nmerged) atomicAdd(&stats[0], (unsigned long long)nmerged);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicAdd(&stats[1], 1ull);
}

// ----------------------------------------------------- window gather layout
// One CTA per bin p (every in-edge of a node of p lies in bin p, so the bin's
// IDs give the in-degrees of p's nodes, counted in shared memory):
//   whubs[p * kWinHubs + h]  the kWinHubs largest in-degrees (at least
//       kHubMinInDegree; ties to the lower ID), largest first, else kNoHub.
//       The gather sums their IDs in per-warp slots, dealt to all warps.
//   bnd[p * (kWinWarps + 1) + w]  first 32-node block owned by gather warp w:
//       the blocks, weighed by the in-degrees of their non-hub nodes, are cut
//       into kWinWarps contiguous ranges of about equal weight (a block goes
//       to the warp whose share holds its midpoint); bnd[.. + kWinWarps] is the
//       block count.
__global__ void __launch_bounds__(1024) bin_owner_kernel(const uint32_t* __restrict__ dest,
                                                         const uint32_t* __restrict__ bin_e, uint32_t n, uint32_t q,
                                                         uint32_t* __restrict__ whubs, uint32_t* __restrict__ bnd,
                                                         uint32_t* __restrict__ indeg) {
    extern __shared__ uint32_t deg[];  // q in-degrees, then one weight per block
    __shared__ unsigned long long sh[32];
    __shared__ uint32_t sh32[32];
    __shared__ uint8_t own[1024];
    const uint32_t p = blockIdx.x, base = p * q, len = min(q, n - base);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) deg[i] = 0;
    __syncthreads();
    const uint32_t e0 = bin_e[p], e1 = bin_e[p + 1];
    constexpr uint32_t kIlp = 4;  // independent loads in flight per thread
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += kIlp * blockDim.x) {
        uint32_t loc[kIlp];
#pragma unroll
        for (uint32_t j = 0; j < kIlp; ++j) {
            const uint32_t x = e + j * blockDim.x;
            loc[j] = x < e1 ? (__ldcs(dest + x) & kIdMask) - base : 0xFFFFFFFFu;
        }
#pragma unroll
        for (uint32_t j = 0; j < kIlp; ++j)
            if (loc[j] < len) atomicAdd(&deg[loc[j]], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) indeg[base + i] = deg[i];  // kept by the handle
    for (uint32_t h = 0; h < kWinHubs; ++h) {
        unsigned long long best = 0;
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
            best = max(best, ((unsigned long long)deg[i] << 32) | (0xFFFFFFFFu - i));
        const unsigned long long b = block_max_u64(best, sh);
        const uint32_t hub = (b >> 32) >= kHubMinInDegree ? 0xFFFFFFFFu - (uint32_t)b : kNoHub;
        if (threadIdx.x == 0) {
            whubs[(size_t)p * kWinHubs + h] = hub;
            if (hub != kNoHub) deg[hub] = 0;  // its IDs go to every warp: no owner weight
        }
        __syncthreads();
    }
    const uint32_t nblk = (len + 31) / 32;
    uint32_t* wt = deg + ((q + 31) & ~31u);
    for (uint32_t b = warp; b < nblk; b += blockDim.x >> 5) {
        const uint32_t i = 32 * b + lane;
        const uint32_t x = __reduce_add_sync(0xffffffffu, i < len ? deg[i] : 0u);
        if (lane == 0) wt[b] = x;
    }
    __syncthreads();
    const uint32_t t = threadIdx.x;  // one block per thread (nblk <= 1024)
    const uint32_t w_t = t < nblk ? wt[t] : 0u;
    uint32_t total = 0;
    const uint32_t cum = block_exclusive_scan(w_t, &total, sh32);
    if (t < nblk) {
        const unsigned long long mid = ((2ull * cum + w_t) * kWinWarps) / (2ull * total ? 2ull * total : 1ull);
        const uint32_t o = total ? (uint32_t)(mid < (unsigned long long)kWinWarps ? mid : kWinWarps - 1)
                                 : (uint32_t)(((uint64_t)t * kWinWarps) / nblk);
        own[t] = (uint8_t)o;
    }
    __syncthreads();
    if (t <= (uint32_t)kWinWarps) {  // first block with owner >= t (owners never decrease)
        uint32_t lo = 0, hi = nblk;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (own[mid] < t) lo = mid + 1; else hi = mid;
        }
        bnd[(size_t)p * (kWinWarps + 1) + t] = t == (uint32_t)kWinWarps ? nblk : lo;
    }
}

// windows[p] = windows of bin p: ceil(IDs / kWin).
__global__ void bin_window_counts_kernel(const uint32_t* __restrict__ bin_e, uint32_t k, uint32_t* __restrict__ cnt) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
        cnt[p] = (bin_e[p + 1] - bin_e[p] + kWin - 1) / kWin;
}

constexpr int kWlThreads = 512;
constexpr int kWlWarps = kWlThreads / 32;
constexpr uint32_t kWlSpan = kWin / kWlWarps;   // consecutive items per warp
constexpr uint32_t kWlSteps = kWlSpan / 32;     // 32-item steps per warp
constexpr uint32_t kWlOwnerBuckets = 32 + kWinHubs;   // per owner: 32 banks, then one per hub
constexpr uint32_t kWlBuckets = kWinWarps * kWlOwnerBuckets;
constexpr uint32_t kWlSlotBins = (PCPM_MAX_PART_SIZE + kWinWarps * kWinHubs + 31) / 32;  // slot >> 5
constexpr uint32_t kWlMaxBins = kWlSlotBins > kWlBuckets ? kWlSlotBins : kWlBuckets;
static_assert(kWin <= 4096 && kWin % (32 * kWlWarps) == 0, "12-bit positions, whole steps per warp");

// Dynamic shared memory of window_layout_kernel.
constexpr size_t kWlSmemSk = 0;                                          // u32[kWin]
constexpr size_t kWlSmemTmp = kWlSmemSk + kWin * 4;                      // u32[kWin]
constexpr size_t kWlSmemOff = kWlSmemTmp + kWin * 4;                     // u16[kWin]
constexpr size_t kWlSmemCnt = kWlSmemOff + kWin * 2;                     // u16[kWlWarps][kWlMaxBins]
constexpr size_t kWlSmemStart = kWlSmemCnt + ((kWlWarps * kWlMaxBins * 2 + 15) & ~(size_t)15);  // u32[kWlMaxBins + 1]
constexpr size_t kWlSmemBytes = kWlSmemStart + (kWlMaxBins + 1) * 4;

// One stable counting-sort pass over the window's items. Each thread holds
// kWlSteps items in warp-major order (warp w, step i, lane l holds item
// w * kWlSpan + 32 i + l, and an item's index is its order):
// out[start(key) + items of the same key before it] = val. Keys >= kBins
// mark absent items. Per-warp ranks come from match_any, then each bin's
// counts are turned into prefixes over the warps and a block scan gives the
// bin starts.
template <uint32_t kBins>
__device__ __forceinline__ void stable_pass(const uint32_t (&key)[kWlSteps], const uint32_t (&val)[kWlSteps],
                                            uint32_t* out, uint16_t* wcnt, uint32_t* start, uint32_t* sh32) {
    static_assert(kBins <= kWlMaxBins, "bins");
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t lt = lanemask_lt();
    for (uint32_t x = t; x < kWlWarps * kBins; x += kWlThreads) wcnt[x] = 0;
    __syncthreads();
    uint16_t* mine = wcnt + warp * kBins;
    uint32_t rank[kWlSteps];
#pragma unroll
    for (uint32_t i = 0; i < kWlSteps; ++i) {
        const uint32_t k = key[i];
        const uint32_t peers = __match_any_sync(0xffffffffu, k);
        const uint32_t base = k < kBins ? (uint32_t)mine[k] : 0u;
        rank[i] = base + __popc(peers & lt);
        __syncwarp();
        if (k < kBins && lane == (uint32_t)(__ffs(peers) - 1)) mine[k] = (uint16_t)(base + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    constexpr uint32_t kPer = (kBins + kWlThreads - 1) / kWlThreads;
    uint32_t c[kPer], sum = 0;
#pragma unroll
    for (uint32_t j = 0; j < kPer; ++j) {
        const uint32_t b = kPer * t + j;
        uint32_t tot = 0;
        if (b < kBins)
            for (uint32_t w = 0; w < (uint32_t)kWlWarps; ++w) {
                const uint32_t x = wcnt[w * kBins + b];
                wcnt[w * kBins + b] = (uint16_t)tot;
                tot += x;
            }
        c[j] = tot;
        sum += tot;
    }
    uint32_t all = 0;
    uint32_t x = block_exclusive_scan(sum, &all, sh32);
#pragma unroll
    for (uint32_t j = 0; j < kPer; ++j) {
        const uint32_t b = kPer * t + j;
        if (b < kBins) start[b] = x;
        x += c[j];
    }
    if (t == 0) start[kBins] = all;
    __syncthreads();
#pragma unroll
    for (uint32_t i = 0; i < kWlSteps; ++i)
        if (key[i] < kBins) out[start[key[i]] + mine[key[i]] + rank[i]] = val[i];
    __syncthreads();
}

// One CTA per window of kWin consecutive IDs of one bin (each CTA takes a
// contiguous range of windows, so the bin's owner table is rebuilt only when
// the bin changes). Warp w reads IDs [w * kWlSpan, +kWlSpan) of the window in
// steps of 32; ballots give every ID its update index (flagged IDs before it,
// inclusive, minus one: Algorithm 4's pointer) and the hub IDs their rank.
// Every ID gets its owner warp and slot (the i-th hub ID of the window goes to
// warp i mod kWinWarps, slot q + warp * kWinHubs + hub). Two stable counting
// sorts, first by slot / 32 and then by bucket (per owner, the 32 banks of
// the slot, then one bucket per hub), leave every owner's group in (bank,
// slot, position) order with its hub IDs last. Group w's sorted position s
// goes to lane l, round r of that warp's pass: with R = ceil(N_w / 32)
// rounds, the first N_w - 32 (R - 1) lanes take R consecutive positions and
// the others R - 1, stored at r * 32 + l. The end bit marks the last position
// of a run of equal slots. The CTA checks every word against the partition
// and the update slice (stats[1]) and counts IDs whose run continues
// (stats[0]).
__global__ void __launch_bounds__(kWlThreads, 2) window_layout_kernel(
    const uint32_t* __restrict__ dest, const uint32_t* __restrict__ bin_e, const uint32_t* __restrict__ win_start,
    uint32_t k, const uint32_t* __restrict__ chunk_base, const uint32_t* __restrict__ whubs,
    const uint32_t* __restrict__ bnd, uint32_t n, uint32_t q, uint64_t nwin, uint32_t upd_bytes,
    uint32_t* __restrict__ words, uint4* __restrict__ desc, unsigned long long* __restrict__ stats,
    const float* __restrict__ wdest, float* __restrict__ wweight) {
    extern __shared__ __align__(16) unsigned char wl_smem[];
    uint32_t* s_sk = reinterpret_cast<uint32_t*>(wl_smem + kWlSmemSk);    // sorted: slot << 12 | position
    uint32_t* s_tmp = reinterpret_cast<uint32_t*>(wl_smem + kWlSmemTmp);  // after the first pass
    uint16_t* s_off = reinterpret_cast<uint16_t*>(wl_smem + kWlSmemOff);  // by position: offset in the slice
    uint16_t* s_wcnt = reinterpret_cast<uint16_t*>(wl_smem + kWlSmemCnt);
    uint32_t* s_start = reinterpret_cast<uint32_t*>(wl_smem + kWlSmemStart);
    __shared__ uint8_t s_own[1024];
    __shared__ uint32_t s_hub[kWinHubs];
    __shared__ uint32_t s_bnd[kWinWarps + 1];
    __shared__ uint32_t s_goff[kWinWarps + 1];
    __shared__ uint32_t s_wtot[kWlWarps][2];
    __shared__ uint32_t sh32[32];
    __shared__ uint32_t s_fb, s_first, s_last;
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t align = 16u / upd_bytes;
    const uint32_t slice_cap = kWin + 2 * align;
    uint32_t nbad = 0, nmerged = 0;
    const uint64_t per = (nwin + gridDim.x - 1) / gridDim.x;
    const uint64_t wb0 = blockIdx.x * per;
    const uint64_t wbeg = wb0 < nwin ? wb0 : nwin, wend = wbeg + per < nwin ? wbeg + per : nwin;
    uint32_t cached = 0xFFFFFFFFu;
    for (uint64_t win = wbeg; win < wend; ++win) {
        const uint32_t p = upper_bound_u32(win_start, 0, k + 1, (uint32_t)win) - 1;
        const uint32_t j = (uint32_t)win - win_start[p];
        const uint32_t P = bin_e[p] + j * kWin, Pend = min(P + kWin, bin_e[p + 1]);
        const uint32_t N = Pend - P;
        const uint32_t vbase = p * q, len = min(q, n - vbase);
        if (p != cached) {  // the bin's hubs and owner table
            if (t < kWinHubs) s_hub[t] = whubs[(size_t)p * kWinHubs + t];
            if (t <= (uint32_t)kWinWarps) s_bnd[t] = bnd[(size_t)p * (kWinWarps + 1) + t];
            __syncthreads();
            const uint32_t nblk = s_bnd[kWinWarps];
            for (uint32_t x = t; x < nblk; x += kWlThreads)
                s_own[x] = (uint8_t)(upper_bound_u32(s_bnd, 0, kWinWarps, x) - 1);
            cached = p;
        }
        if (warp == 0) {  // flagged IDs before P: the chunk's base plus the flags of its head
            const uint32_t cbase = P & ~(kChunk - 1);
            uint32_t run = chunk_base[P / kChunk];
            for (uint32_t x = cbase; x < P; x += 32) {
                const uint32_t pos = x + lane;
                run += __popc(__ballot_sync(0xffffffffu, pos < P && (dest[pos] >> 31)));
            }
            if (lane == 0) s_fb = run;
        }
        // this warp's IDs: flags (inclusive within the warp) and hub ranks
        uint32_t loc[kWlSteps], rel[kWlSteps], hx[kWlSteps];
        uint32_t frun = 0, hrun = 0;
#pragma unroll
        for (uint32_t i = 0; i < kWlSteps; ++i) {
            const uint32_t pos = warp * kWlSpan + 32 * i + lane;
            const bool valid = pos < N;
            const uint32_t id = valid ? dest[P + pos] : 0u;
            loc[i] = (id & kIdMask) - vbase;
            uint32_t h = kWinHubs;
#pragma unroll
            for (uint32_t hh = 0; hh < kWinHubs; ++hh)
                if (valid && loc[i] < len && loc[i] == s_hub[hh] && h == kWinHubs) h = hh;
            const uint32_t bf = __ballot_sync(0xffffffffu, valid && (id >> 31));
            const uint32_t bh = __ballot_sync(0xffffffffu, h < kWinHubs);
            rel[i] = frun + __popc(bf & (lt | (1u << lane)));
            hx[i] = h | ((hrun + __popc(bh & lt)) << 8);
            frun += __popc(bf);
            hrun += __popc(bh);
        }
        if (lane == 0) {
            s_wtot[warp][0] = frun;
            s_wtot[warp][1] = hrun;
        }
        __syncthreads();  // s_fb, s_own, warp totals
        uint32_t fbase = 0, hbase = 0;
        for (uint32_t w = 0; w < warp; ++w) {
            fbase += s_wtot[w][0];
            hbase += s_wtot[w][1];
        }
        const uint32_t fb0 = s_fb;  // the ID before P belongs to update fb0 - 1
        uint32_t key[kWlSteps], val[kWlSteps];
#pragma unroll
        for (uint32_t i = 0; i < kWlSteps; ++i) {
            const uint32_t pos = warp * kWlSpan + 32 * i + lane;
            const bool valid = pos < N;
            rel[i] += fbase;  // update index - (fb0 - 1)
            const uint32_t h = hx[i] & 0xFFu;
            uint32_t sl;
            if (h < kWinHubs) {
                sl = q + ((hbase + (hx[i] >> 8)) % kWinWarps) * kWinHubs + h;
            } else {
                const bool in = loc[i] < len;
                if (valid && !in) ++nbad;
                sl = in ? loc[i] : 0u;
            }
            if (pos == 0) s_first = fb0 - 1 + rel[i];
            if (valid && pos + 1 == N) s_last = fb0 - 1 + rel[i];
            key[i] = valid ? sl >> 5 : kWlSlotBins;
            val[i] = (sl << 12) | pos;
        }
        stable_pass<kWlSlotBins>(key, val, s_tmp, s_wcnt, s_start, sh32);
        const uint32_t us = N ? s_first & ~(align - 1) : 0u, ue = N ? (s_last + align) & ~(align - 1) : 0u;
        if (t == 0 && N && ue - us > slice_cap) ++nbad;
#pragma unroll
        for (uint32_t i = 0; i < kWlSteps; ++i) {
            const uint32_t pos = warp * kWlSpan + 32 * i + lane;
            if (pos < N) {
                const uint32_t off = fb0 - 1 + rel[i] - us;
                if (off >= slice_cap) ++nbad;
                s_off[pos] = (uint16_t)min(off, kWinOffMask);
            }
        }
        // second pass, in the first pass's order: by bucket
#pragma unroll
        for (uint32_t i = 0; i < kWlSteps; ++i) {
            const uint32_t item = warp * kWlSpan + 32 * i + lane;
            const bool valid = item < N;
            const uint32_t v = valid ? s_tmp[item] : 0u, sl = v >> 12;
            uint32_t b = kWlBuckets;
            if (valid)
                b = sl >= q ? ((sl - q) / kWinHubs) * kWlOwnerBuckets + 32 + (sl - q) % kWinHubs
                            : (uint32_t)s_own[sl >> 5] * kWlOwnerBuckets + (sl & 31u);
            key[i] = b;
            val[i] = v;
        }
        stable_pass<kWlBuckets>(key, val, s_sk, s_wcnt, s_start, sh32);
        if (t <= (uint32_t)kWinWarps) s_goff[t] = t < (uint32_t)kWinWarps ? s_start[kWlOwnerBuckets * t] : N;
        __syncthreads();
        // deal every group lane by lane: one (group, lane) pair per thread
        uint32_t* out = words + win * kWinStride;
        for (uint32_t pr = t; pr < (uint32_t)kWinWarps * 32; pr += kWlThreads) {
            const uint32_t w = pr >> 5, l = pr & 31;  // w is warp-uniform
            const uint32_t g0 = s_goff[w], Nw = s_goff[w + 1] - g0;
            if (Nw == 0) continue;
            const uint32_t R = (Nw + 31) / 32, longer = Nw - 32 * (R - 1);
            const uint32_t cnt = l < longer ? R : R - 1;
            const uint32_t st0 = l < longer ? l * R : longer * R + (l - longer) * (R - 1);
            for (uint32_t r = 0; r < cnt; ++r) {
                const uint32_t s = g0 + st0 + r;
                const uint32_t sk = s_sk[s], sl = sk >> 12, pos = sk & 4095u;
                const bool end = st0 + r + 1 == Nw || (s_sk[s + 1] >> 12) != sl;
                nmerged += end ? 0u : 1u;
                const uint32_t o = kWinHdrWords + g0 + r * 32 + l;
                out[o] = sl | ((uint32_t)s_off[pos] << kWinOffShift) | (end ? kWinEndBit : 0u);
                if (wweight) wweight[win * kWinStride + o] = wdest[P + pos];
            }
        }
        if (t < kWinHdrWords) {
            const uint32_t a0 = 2 * t, a1 = 2 * t + 1;
            const uint32_t v0 = a0 <= (uint32_t)kWinWarps ? s_goff[a0] : 0u;
            const uint32_t v1 = a1 <= (uint32_t)kWinWarps ? s_goff[a1] : 0u;
            out[t] = v0 | (v1 << 16);
        }
        if (t == 0) desc[win] = make_uint4(us, (ue - us) * upd_bytes, (kWinHdrWords + ((N + 3) & ~3u)) * 4u, N);
        __syncthreads();
    }
    nmerged = __reduce_add_sync(0xffffffffu, nmerged);
    nbad = __reduce_add_sync(0xffffffffu, nbad);
    if (lane == 0 && nmerged) atomicAdd(&stats[0], (unsigned long long)nmerged);
    if (lane == 0 && nbad) atomicAdd(&stats[1], (unsigned long long)nbad);
}

// src16[t] = src[t] - p q, p = src[t] / q: the index within its source
// partition.
__global__ void src_local_kernel(const uint32_t* __restrict__ src, uint64_t ne, DivQ divq,
                                 uint16_t* __restrict__ src16) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < ne; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = src[t];
        src16[t] = (uint16_t)(v - divq(v) * divq.q);
    }
}

__global__ void scatter_pieces_kernel(const uint32_t* __restrict__ groups, uint32_t k, uint32_t per,
                                      uint32_t* __restrict__ pieces) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
        pieces[p] = groups[p] ? (groups[p] + per - 1) / per : 1;
}

__global__ void scatter_units_kernel(const uint32_t* __restrict__ groups, const uint32_t* __restrict__ start,
                                     uint32_t k, uint32_t per, uint32_t nunits, uint4* __restrict__ units,
                                     uint32_t* __restrict__ sizes) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < nunits; u += gridDim.x * blockDim.x) {
        const uint32_t p = upper_bound_u32(start, 0, k + 1, u) - 1;
        const uint32_t idx = u - start[p];
        const uint32_t lo = min(groups[p], idx * per), hi = min(groups[p], (idx + 1) * per);
        units[u] = make_uint4(p, lo, hi, start[p + 1] - start[p]);
        sizes[u] = hi - lo;
    }
}

// Build temporaries, from the library's pool in the build stream's order.
struct TempBufs {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit TempBufs(cudaStream_t stream) : s(stream) {}
    ~TempBufs() {
        for (void* p : ptrs) pool_free(p, s);
    }
    template <class T>
    cudaError_t alloc(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = pool_alloc(&q, std::max<size_t>(count, 1) * sizeof(T), s);
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = (T*)q;
        }
        return e;
    }
};

#define BCK(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            note_cuda_error(e_);                                               \
            return e_ == cudaErrorMemoryAllocation ? PCPM_ENOMEM : PCPM_ECUDA; \
        }                                                                      \
    } while (0)

int grid_for(uint64_t work, int threads, int cap) {
    uint64_t b = (work + threads - 1) / threads;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, (uint64_t)cap));
}

// Exclusive scan of N values into out[0..N] (out[N] = total).
int scan_exclusive(const uint32_t* in, uint32_t* out, uint64_t N, TempBufs& tmp, cudaStream_t s) {
    if (N <= 1024ull * kSmallScanItems) {
        scan_small_kernel<<<1, 1024, 0, s>>>(in, out, (uint32_t)N);
        return launch_status();
    }
    const uint64_t nb = (N + kScanBlockItems - 1) / kScanBlockItems;
    if (nb > 1024ull * kSmallScanItems) return PCPM_EINVAL;
    uint32_t *sums = nullptr, *offs = nullptr;
    BCK(tmp.alloc(&sums, nb));
    BCK(tmp.alloc(&offs, nb + 1));
    scan_block_sums_kernel<<<(unsigned)nb, 1024, 0, s>>>(in, (uint32_t)N, sums);
    scan_small_kernel<<<1, 1024, 0, s>>>(sums, offs, (uint32_t)nb);
    scan_block_apply_kernel<<<(unsigned)nb, 1024, 0, s>>>(in, (uint32_t)N, offs, out);
    BCK(cudaMemcpyAsync(out + N, offs + nb, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    return launch_status();
}

int colscan(uint32_t* tab, uint32_t nrows, uint32_t k, uint32_t* totals, TempBufs& tmp, cudaStream_t s) {
    const uint32_t nb = std::max<uint32_t>(1, (nrows + kColRows - 1) / kColRows);
    uint32_t* bsum = nullptr;
    BCK(tmp.alloc(&bsum, (size_t)nb * k));
    dim3 blk(32, 32), grd((k + 31) / 32, nb);
    colscan_sums_kernel<<<grd, blk, 0, s>>>(tab, nrows, k, bsum);
    colscan_blocks_kernel<<<(k + 255) / 256, 256, 0, s>>>(bsum, nb, k, tab, nrows, totals);
    colscan_apply_kernel<<<grd, blk, 0, s>>>(tab, nrows, k, bsum);
    return launch_status();
}

int read_err(int* d_err, cudaStream_t s, int* h_err) {
    BCK(cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    return PCPM_OK;
}

}  // namespace

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t s) {
    TempBufs tmp(s);
    return scan_exclusive(in, out, n, tmp, s);
}

int shard_filter_csr(const uint32_t* row_ptr, const uint32_t* col, uint32_t n, uint64_t m, uint32_t vlo,
                     uint32_t vhi, uint32_t** rp_out, uint32_t** col_out, uint64_t* m_out, cudaStream_t s) {
    TempBufs tmp(s);
    uint32_t* cnt = nullptr;
    int* d_err = nullptr;
    BCK(tmp.alloc(&cnt, n));
    BCK(tmp.alloc(&d_err, 1));
    BCK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    uint32_t* rp = nullptr;
    BCK(pool_alloc((void**)&rp, ((size_t)n + 1) * sizeof(uint32_t), s));
    const int grid = grid_for((uint64_t)n * 32, 256, 152 * 16);
    shard_count_kernel<<<grid, 256, 0, s>>>(row_ptr, col, n, m, vlo, vhi, cnt, d_err);
    int rc = launch_status();
    if (rc == PCPM_OK) rc = scan_exclusive(cnt, rp, n, tmp, s);
    uint32_t total = 0;
    int h_err = 0;
    if (rc == PCPM_OK && cudaMemcpyAsync(&total, rp + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = PCPM_ECUDA;
    if (rc == PCPM_OK) rc = read_err(d_err, s, &h_err);
    if (rc == PCPM_OK && h_err) rc = PCPM_EBADGRAPH;
    uint32_t* c = nullptr;
    if (rc == PCPM_OK) {
        const cudaError_t e = pool_alloc((void**)&c, std::max<size_t>(total, 1) * sizeof(uint32_t), s);
        if (e != cudaSuccess) {
            note_cuda_error(e);
            rc = e == cudaErrorMemoryAllocation ? PCPM_ENOMEM : PCPM_ECUDA;
        }
    }
    if (rc == PCPM_OK) {
        shard_copy_kernel<<<grid, 256, 0, s>>>(row_ptr, col, n, m, vlo, vhi, rp, c);
        rc = launch_status();
    }
    if (rc != PCPM_OK) {
        pool_free(rp, s);
        pool_free(c, s);
        return rc;
    }
    *rp_out = rp;
    *col_out = c;
    *m_out = total;
    return PCPM_OK;
}

int compute_inv_deg(pcpm_png* g, const uint32_t* row_ptr, cudaStream_t s) {
    inv_deg_kernel<<<grid_for(g->n, 256, 4096), 256, 0, s>>>(row_ptr, g->n, g->inv_deg);
    return launch_status();
}

int dest_partition_counts(const uint32_t* col, uint64_t m, uint32_t n, uint32_t q, uint64_t* counts_host,
                          cudaStream_t s) {
    const uint32_t k = (uint32_t)(((uint64_t)n + q - 1) / q);
    TempBufs tmp(s);
    unsigned long long* counts = nullptr;
    int* d_err = nullptr;
    BCK(tmp.alloc(&counts, k));
    BCK(tmp.alloc(&d_err, 1));
    BCK(cudaMemsetAsync(counts, 0, (size_t)k * sizeof(unsigned long long), s));
    BCK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    if (m) {
        dest_hist_kernel<<<grid_for(m, 1024, 152 * 2), 1024, 0, s>>>(col, m, n, make_divq(q), k, counts, d_err);
        BCK(cudaGetLastError());
    }
    BCK(cudaMemcpyAsync(counts_host, counts, (size_t)k * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    int h_err = 0;
    const int rc = read_err(d_err, s, &h_err);
    if (rc != PCPM_OK) return rc;
    return h_err ? PCPM_EBADGRAPH : PCPM_OK;
}

int build_png(pcpm_png* g, const uint32_t* row_ptr, const uint32_t* col, const pcpm_build_options& opt,
              cudaStream_t s) {
    const uint32_t n = g->n, q = g->q, k = g->k;
    g->canonical_gather = opt.canonical_gather ? 1 : 0;
    const uint64_t m = g->m;
    TempBufs tmp(s);
    int* d_err = nullptr;
    BCK(tmp.alloc(&d_err, 1));
    BCK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    int h_err = 0;
    int rc;

    check_row_ptr_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(row_ptr, n, d_err);
    BCK(cudaGetLastError());
    if ((rc = read_err(d_err, s, &h_err)) != PCPM_OK) return rc;
    if (h_err) return PCPM_EBADGRAPH;

    // Tiles: kTileEdges edges of one source partition each.
    uint32_t *tiles = nullptr, *tile_start = nullptr;
    BCK(tmp.alloc(&tiles, k));
    BCK(tmp.alloc(&tile_start, k + 1));
    partition_tiles_kernel<<<grid_for(k, 256, 1024), 256, 0, s>>>(row_ptr, n, q, k, tiles);
    if ((rc = scan_exclusive(tiles, tile_start, k, tmp, s)) != PCPM_OK) return rc;
    uint32_t ntiles = 0;
    BCK(cudaMemcpyAsync(&ntiles, tile_start + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));

    // Count pass.
    uint32_t *tab_e = nullptr, *tab_u = nullptr;
    BCK(tmp.alloc(&tab_e, (size_t)(ntiles + 1) * k));
    BCK(tmp.alloc(&tab_u, (size_t)(ntiles + 1) * k));
    const int wpc = (int)std::max<uint32_t>(1, std::min<uint32_t>(8, 12288u / k));  // <= 96 KB of tables
    const size_t tile_smem = (size_t)wpc * 2 * k * sizeof(uint32_t);
    BCK(cudaFuncSetAttribute(tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem));
    BCK(cudaFuncSetAttribute(tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem));
    const int sms = g->sms;
    const int tile_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((ntiles + wpc - 1) / wpc, (uint64_t)sms * 16));
    // k <= kFillMaxK: one CTA per tile (staged count and fill), which needs
    // every tile's (source partition, first row); else one warp per tile
    const bool staged = k <= kFillMaxK;
    const DivQ divq = make_divq(q);
    uint2* tile_info = nullptr;
    BCK(tmp.alloc(&tile_info, std::max<uint32_t>(ntiles, 1)));
    auto staged_grid = [&](const void* f, size_t smem, int* grid) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kFillWarps * 32, smem);
        *grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, (uint64_t)sms * (uint64_t)std::max(per_sm, 1)));
        return e;
    };
    if (ntiles && staged) {
        tile_info_kernel<<<grid_for(ntiles, 256, 4096), 256, 0, s>>>(row_ptr, n, q, k, tile_start, ntiles, tile_info);
        const size_t cs = count_smem_bytes(k);
        int grid = 1;
        BCK(staged_grid((const void*)count_staged_kernel, cs, &grid));
        count_staged_kernel<<<grid, kFillWarps * 32, cs, s>>>(row_ptr, col, n, divq, k, tile_start, tile_info, ntiles,
                                                             tab_e, tab_u, d_err);
        BCK(cudaGetLastError());
    } else if (ntiles) {
        tile_kernel<false><<<tile_grid, wpc * 32, tile_smem, s>>>(row_ptr, col, n, q, k, tile_start, ntiles, tab_e,
                                                                 tab_u, nullptr, nullptr, nullptr, nullptr, d_err);
        BCK(cudaGetLastError());
    }
    if ((rc = read_err(d_err, s, &h_err)) != PCPM_OK) return rc;
    if (h_err) return PCPM_EBADGRAPH;

    // Scans: per-tile cursors, bin starts.
    uint32_t *tot_e = nullptr, *tot_u = nullptr;
    BCK(tmp.alloc(&tot_e, k));
    BCK(tmp.alloc(&tot_u, k));
    if (ntiles) {
        if ((rc = colscan(tab_e, ntiles, k, tot_e, tmp, s)) != PCPM_OK) return rc;
        if ((rc = colscan(tab_u, ntiles, k, tot_u, tmp, s)) != PCPM_OK) return rc;
    } else {
        BCK(cudaMemsetAsync(tab_e, 0, (size_t)k * sizeof(uint32_t), s));
        BCK(cudaMemsetAsync(tab_u, 0, (size_t)k * sizeof(uint32_t), s));
        BCK(cudaMemsetAsync(tot_e, 0, (size_t)k * sizeof(uint32_t), s));
        BCK(cudaMemsetAsync(tot_u, 0, (size_t)k * sizeof(uint32_t), s));
    }
    BCK(dev_alloc(g, (void**)&g->bin_e, (k + 1) * sizeof(uint32_t)));
    BCK(dev_alloc(g, (void**)&g->bin_u, (k + 1) * sizeof(uint32_t)));
    if ((rc = scan_exclusive(tot_e, g->bin_e, k, tmp, s)) != PCPM_OK) return rc;
    if ((rc = scan_exclusive(tot_u, g->bin_u, k, tmp, s)) != PCPM_OK) return rc;
    uint32_t ends[2] = {0, 0};
    BCK(cudaMemcpyAsync(&ends[0], g->bin_e + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(&ends[1], g->bin_u + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    if (ends[0] != m) return PCPM_EDEVICE;
    g->ne = ends[1];

    // Fill pass.
    g->nchunks = (m + kChunk - 1) / kChunk;
    const size_t dest_len = std::max<uint64_t>(g->nchunks, 1) * kChunk;
    BCK(dev_alloc(g, (void**)&g->dest, dest_len * sizeof(uint32_t)));
    BCK(cudaMemsetAsync(g->dest, 0, dest_len * sizeof(uint32_t), s));
    BCK(dev_alloc(g, (void**)&g->src, (g->ne + 4) * sizeof(uint32_t)));
    if (ntiles) {
        if (g->weighted) BCK(dev_alloc(g, (void**)&g->wdest, dest_len * sizeof(float)));
        if (staged) {
            const size_t fs = fill_smem_bytes(k, g->weighted != 0);
            int fill_grid = 1;
            BCK(staged_grid((const void*)fill_staged_kernel, fs, &fill_grid));
            fill_staged_kernel<<<fill_grid, kFillWarps * 32, fs, s>>>(row_ptr, col, n, divq, k, tile_start, tile_info,
                                                                     ntiles, tab_e, tab_u, g->bin_e, g->bin_u,
                                                                     g->dest, g->src, d_err, g->weights_in, g->wdest);
        } else {
            tile_kernel<true><<<tile_grid, wpc * 32, tile_smem, s>>>(row_ptr, col, n, q, k, tile_start, ntiles,
                                                                    tab_e, tab_u, g->bin_e, g->bin_u, g->dest,
                                                                    g->src, d_err, g->weights_in, g->wdest);
        }
        BCK(cudaGetLastError());
    }
    // 16-bit local source indices for the scatter (Sec. 3.3: u - p q fits
    // 16 bits for q <= 2^16), with room for copies rounded to 16 bytes
    BCK(dev_alloc(g, (void**)&g->src16, (g->ne + 16) * sizeof(uint16_t)));
    BCK(cudaMemsetAsync(g->src16, 0, (g->ne + 16) * sizeof(uint16_t), s));
    if (g->ne) {
        src_local_kernel<<<grid_for(g->ne, 256, sms * 8), 256, 0, s>>>(g->src, g->ne, divq, g->src16);
        BCK(cudaGetLastError());
    }

    // Segment table for the scatter (and offsets for export).
    const size_t kk = (size_t)k * k;
    BCK(dev_alloc(g, (void**)&g->seg_u, kk * sizeof(uint32_t)));
    BCK(dev_alloc(g, (void**)&g->cnt_u, kk * sizeof(uint32_t)));
    BCK(dev_alloc(g, (void**)&g->seg_e, kk * sizeof(uint32_t)));
    BCK(dev_alloc(g, (void**)&g->cnt_e, kk * sizeof(uint32_t)));
    segments_kernel<<<grid_for(kk, 256, 4096), 256, 0, s>>>(tab_u, tile_start, g->bin_u, k, g->seg_u, g->cnt_u);
    segments_kernel<<<grid_for(kk, 256, 4096), 256, 0, s>>>(tab_e, tile_start, g->bin_e, k, g->seg_e, g->cnt_e);
    BCK(cudaGetLastError());

    // Update base of every chunk of the destination-ID array.
    BCK(dev_alloc(g, (void**)&g->chunk_base, (g->nchunks + 1) * sizeof(uint32_t)));
    if (g->nchunks) {
        uint32_t* ccnt = nullptr;
        BCK(tmp.alloc(&ccnt, g->nchunks));
        chunk_flags_kernel<<<grid_for(g->nchunks * 32, 256, 8192), 256, 0, s>>>(g->dest, m, g->nchunks, ccnt);
        BCK(cudaGetLastError());
        if ((rc = scan_exclusive(ccnt, g->chunk_base, g->nchunks, tmp, s)) != PCPM_OK) return rc;
    } else {
        BCK(cudaMemsetAsync(g->chunk_base, 0, sizeof(uint32_t), s));
    }

    // Hubs per bin: the two largest in-degrees for the canonical and chunk
    // gathers; the window gather picks its own (bin_owner_kernel).
    g->gather_windows = !g->canonical_gather && opt.gather_windows != 2;
    BCK(dev_alloc(g, (void**)&g->hubs, 2 * (size_t)k * sizeof(uint32_t)));
    if (!g->gather_windows) {
        const size_t hub_smem = (size_t)q * sizeof(uint32_t);
        BCK(cudaFuncSetAttribute(bin_hubs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hub_smem));
        bin_hubs_kernel<<<k, 1024, hub_smem, s>>>(g->dest, g->bin_e, n, q, g->hubs);
        BCK(cudaGetLastError());
    } else {
        BCK(cudaMemsetAsync(g->hubs, 0xFF, 2 * (size_t)k * sizeof(uint32_t), s));
    }

    // Work units, largest first. Gather: runs of at most `gper` chunks, at
    // least q/64 chunks (so a unit's flush of q partial sums stays small next
    // to its work) and about nchunks/(2*SMs). Scatter: runs of at most `sper`
    // groups, at least q (a unit stages the partition's q values once).
    uint32_t *pieces = nullptr, *start = nullptr, *sizes = nullptr, *groups = nullptr, *gstart = nullptr;
    BCK(tmp.alloc(&pieces, k));
    BCK(tmp.alloc(&start, k + 1));
    BCK(tmp.alloc(&groups, k));
    BCK(tmp.alloc(&gstart, k + 1));
    const uint32_t* ichunks = nullptr;
    uint64_t gchunks = g->nchunks;
    uint32_t gper_default = (uint32_t)std::max<uint64_t>((q + 63) / 64, (gchunks + 2 * sms - 1) / (2 * sms));
    if (g->gather_windows) {
        // Window layout: owners and hubs per bin, then the windows.
        uint32_t *bnd = nullptr, *wc = nullptr;
        BCK(tmp.alloc(&bnd, (size_t)k * (kWinWarps + 1)));
        BCK(tmp.alloc(&wc, k));
        BCK(dev_alloc(g, (void**)&g->whubs, (size_t)k * kWinHubs * sizeof(uint32_t)));
        const size_t own_smem = ((size_t)((q + 31) & ~31u) + 1024) * sizeof(uint32_t);
        BCK(cudaFuncSetAttribute(bin_owner_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)own_smem));
        BCK(dev_alloc(g, (void**)&g->indeg, (size_t)n * sizeof(uint32_t)));
        bin_owner_kernel<<<k, 1024, own_smem, s>>>(g->dest, g->bin_e, n, q, g->whubs, bnd, g->indeg);
        BCK(cudaGetLastError());
        BCK(dev_alloc(g, (void**)&g->win_start, (k + 1) * sizeof(uint32_t)));
        bin_window_counts_kernel<<<grid_for(k, 256, 64), 256, 0, s>>>(g->bin_e, k, wc);
        if ((rc = scan_exclusive(wc, g->win_start, k, tmp, s)) != PCPM_OK) return rc;
        uint32_t nw = 0;
        BCK(cudaMemcpyAsync(&nw, g->win_start + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        g->nwin = nw;
        BCK(dev_alloc(g, (void**)&g->wwords, std::max<uint64_t>(nw, 1) * kWinStride * sizeof(uint32_t)));
        BCK(dev_alloc(g, (void**)&g->wdesc, std::max<uint64_t>(nw, 1) * sizeof(uint4)));
        if (g->weighted) BCK(dev_alloc(g, (void**)&g->wweight, std::max<uint64_t>(nw, 1) * kWinStride * sizeof(float)));
        unsigned long long* lstats = nullptr;
        BCK(tmp.alloc(&lstats, 2));
        BCK(cudaMemsetAsync(lstats, 0, 2 * sizeof(*lstats), s));
        if (nw) {
            BCK(cudaFuncSetAttribute(window_layout_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kWlSmemBytes));
            window_layout_kernel<<<(unsigned)std::min<uint64_t>(nw, (uint64_t)sms * 8), kWlThreads, kWlSmemBytes, s>>>(
                g->dest, g->bin_e, g->win_start, k, g->chunk_base, g->whubs, bnd, n, q, nw, g->upd_bytes, g->wwords,
                g->wdesc, lstats, g->wdest, g->wweight);
            BCK(cudaGetLastError());
        }
        unsigned long long hstats[2] = {0, 0};
        BCK(cudaMemcpyAsync(hstats, lstats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        if (hstats[1]) return PCPM_EDEVICE;
        g->merged_adds = hstats[0];
        g->gather_runs = 1;
        ichunks = g->win_start;
        gchunks = nw;
        // in windows: the chunk-based defaults divided by kWin / kChunk
        gper_default = (uint32_t)std::max<uint64_t>((q + 1023) / 1024, (gchunks + 2 * sms - 1) / (2 * sms));
    } else if (!g->canonical_gather) {
        // Bank-spread gather layout.
        uint32_t* cc = nullptr;
        BCK(tmp.alloc(&cc, k));
        BCK(dev_alloc(g, (void**)&g->ichunk_start, (k + 1) * sizeof(uint32_t)));
        bin_chunk_counts_kernel<<<grid_for(k, 256, 64), 256, 0, s>>>(g->bin_e, k, cc);
        if ((rc = scan_exclusive(cc, g->ichunk_start, k, tmp, s)) != PCPM_OK) return rc;
        uint32_t nic = 0;
        BCK(cudaMemcpyAsync(&nic, g->ichunk_start + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        g->nichunks = nic;
        BCK(dev_alloc(g, (void**)&g->gdest, std::max<uint64_t>(nic, 1) * kChunk * sizeof(uint32_t)));
        BCK(dev_alloc(g, (void**)&g->gslice_start, std::max<uint64_t>(nic, 1) * sizeof(uint32_t)));
        BCK(dev_alloc(g, (void**)&g->gslice_bytes, std::max<uint64_t>(nic, 1) * sizeof(uint32_t)));
        unsigned long long* lstats = nullptr;
        BCK(tmp.alloc(&lstats, 2));
        BCK(cudaMemsetAsync(lstats, 0, 2 * sizeof(*lstats), s));
        if (nic) {
            if (g->weighted) BCK(dev_alloc(g, (void**)&g->gweight, (size_t)nic * kChunk * sizeof(float)));
            gather_layout_kernel<<<grid_for((uint64_t)nic * 32, kLayoutWarps * 32, sms * 8), kLayoutWarps * 32, 0, s>>>(
                g->dest, g->bin_e, g->ichunk_start, k, g->chunk_base, g->hubs, q, nic, g->gdest, g->gslice_start,
                g->gslice_bytes, g->upd_bytes, lstats, g->wdest, g->gweight);
            BCK(cudaGetLastError());
        }
        unsigned long long hstats[2] = {0, 0};
        BCK(cudaMemcpyAsync(hstats, lstats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        if (hstats[1]) return PCPM_EDEVICE;
        const unsigned long long nmerged = hstats[0];
        g->merged_adds = nmerged;
        // Register runs cost a few instructions per ID; they pay once runs
        // are common (hot destinations), where they also remove same-address
        // conflicts.
        g->gather_runs = opt.gather_runs == 1 || (opt.gather_runs == 0 && nmerged * 16 >= g->m);
        ichunks = g->ichunk_start;
        gchunks = nic;
    }

    const uint32_t gper = !opt.gather_unit_chunks ? gper_default
                          : g->gather_windows     ? (opt.gather_unit_chunks + kWin / kChunk - 1) / (kWin / kChunk)
                                                  : opt.gather_unit_chunks;
    gather_pieces_kernel<<<grid_for(k, 256, 64), 256, 0, s>>>(g->bin_e, ichunks, k, gper, g->plo, g->phi, pieces);
    if ((rc = scan_exclusive(pieces, start, k, tmp, s)) != PCPM_OK) return rc;
    src_groups_kernel<<<k, 256, 0, s>>>(g->seg_u, g->cnt_u, k, groups);
    if ((rc = scan_exclusive(groups, gstart, k, tmp, s)) != PCPM_OK) return rc;
    uint32_t totals[2] = {0, 0};
    BCK(cudaMemcpyAsync(&totals[0], start + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(&totals[1], gstart + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    g->ngunits = totals[0];
    // The fused iteration scatters every source partition's next updates; a
    // destination shard gets other shards' ranks only between iterations.
    g->fused_ok = g->ngunits == k && g->plo == 0 && g->phi == k;
    BCK(tmp.alloc(&sizes, std::max<uint32_t>(g->ngunits, k) + 1));
    BCK(dev_alloc(g, (void**)&g->gunits, (size_t)g->ngunits * sizeof(uint4)));
    BCK(dev_alloc(g, (void**)&g->gorder, (size_t)g->ngunits * sizeof(uint32_t)));
    gather_units_kernel<<<grid_for(g->ngunits, 256, 1024), 256, 0, s>>>(g->bin_e, ichunks, start, k, gper,
                                                                        g->ngunits, g->gunits, sizes);
    order_kernel<<<grid_for(g->ngunits, 128, 1024), 128, 0, s>>>(sizes, g->ngunits, g->gorder);
    BCK(cudaGetLastError());
    const uint32_t sper = opt.scatter_unit_groups
                              ? opt.scatter_unit_groups
                              : (uint32_t)std::max<uint64_t>(q, ((uint64_t)totals[1] + 2 * sms - 1) / (2 * sms));
    scatter_pieces_kernel<<<grid_for(k, 256, 64), 256, 0, s>>>(groups, k, sper, pieces);
    if ((rc = scan_exclusive(pieces, start, k, tmp, s)) != PCPM_OK) return rc;
    BCK(cudaMemcpyAsync(&totals[0], start + k, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    g->nsunits = totals[0];
    uint32_t* ssizes = nullptr;
    BCK(tmp.alloc(&ssizes, g->nsunits + 1));
    BCK(dev_alloc(g, (void**)&g->sunits, (size_t)g->nsunits * sizeof(uint4)));
    BCK(dev_alloc(g, (void**)&g->sorder, (size_t)g->nsunits * sizeof(uint32_t)));
    scatter_units_kernel<<<grid_for(g->nsunits, 256, 1024), 256, 0, s>>>(groups, start, k, sper, g->nsunits,
                                                                         g->sunits, ssizes);
    order_kernel<<<grid_for(g->nsunits, 128, 1024), 128, 0, s>>>(ssizes, g->nsunits, g->sorder);
    BCK(cudaGetLastError());

    BCK(dev_alloc(g, (void**)&g->inv_deg, (size_t)n * sizeof(float)));
    inv_deg_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(row_ptr, n, g->inv_deg);
    BCK(cudaGetLastError());
    if ((rc = read_err(d_err, s, &h_err)) != PCPM_OK) return rc;
    if (h_err) return PCPM_EDEVICE;
    return PCPM_OK;
}

}  // namespace pcpm
