// ppr.cu - batched personalized PageRank over a PNG (PCPM_PPR_COLS columns).
//
// The PNG's updates (one per node u and destination partition, Sec. 3.2)
// become 256-byte rows of the 64 column values R[u, :] / |N_o(u)|; each
// destination v then sums the rows of its in-entries (Algorithm 4's rows for
// v) and applies the personalized form of Eq. 1:
//   R'[v, j] = d * sum + (1 - d + d * D_j) * t_j[v]
// with D_j the dangling mass of column j. Two indexes are built once from the
// canonical bins:
//   by source       upos[uptr[u] .. uptr[u+1]) = positions of u's update
//                   rows, so the scatter reads each rank row once, in order,
//                   and writes whole rows;
//   by destination  uidx[colptr[v] .. colptr[v+1]) = the update row of each
//                   in-entry of v (the position of the message it belongs to:
//                   the number of flagged IDs up to it, minus one).
// A half-warp (16 lanes, one float4 each) handles one row, so a warp keeps two
// nodes in flight. Destinations with more than kPieceEntries in-entries are
// summed in pieces (FP32 atomics into a scratch row), then finalised apart.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "pcpm_internal.cuh"
#include "pcpm_ppr.h"

namespace pcpm {
namespace {

constexpr int kCols = PCPM_PPR_COLS;
static_assert(kCols == 64, "16 lanes x float4 per row");
constexpr uint32_t kPieceEntries = 1024;
constexpr int kPprThreads = 256;
constexpr unsigned kAll = 0xffffffffu;
constexpr int kSlots = 2 * kCols;  // per block: L1 change, then dangling mass, per column

#define PCK(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            note_cuda_error(e_);                                               \
            return e_ == cudaErrorMemoryAllocation ? PCPM_ENOMEM : PCPM_ECUDA; \
        }                                                                      \
    } while (0)

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4_stream(float* p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 scale4(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ void add_comp(float4& a, uint32_t i, float v) {
    if (i == 0) a.x += v;
    else if (i == 1) a.y += v;
    else if (i == 2) a.z += v;
    else a.w += v;
}

// ------------------------------------------------------------ index build
__global__ void count_keys_kernel(const uint32_t* __restrict__ key, uint64_t len, uint32_t mask,
                                  uint32_t* __restrict__ cnt) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < len; i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[key[i] & mask], 1u);
}

// upos: the positions t of the update rows of each source node (src[t] = u).
__global__ void fill_by_source_kernel(const uint32_t* __restrict__ src, uint64_t ne, uint32_t* __restrict__ cursor,
                                      uint32_t* __restrict__ upos) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < ne; t += (uint64_t)gridDim.x * blockDim.x)
        upos[atomicAdd(&cursor[src[t]], 1u)] = (uint32_t)t;
}

// uidx: for every destination entry j, the update row of its message
// (flagged IDs up to and including j, minus one), grouped by destination.
// One warp per kChunk-entry chunk; chunk_base[c] = flagged IDs before it.
__global__ void fill_by_destination_kernel(const uint32_t* __restrict__ dest, uint64_t m,
                                           const uint32_t* __restrict__ chunk_base, uint64_t nchunks,
                                           uint32_t* __restrict__ cursor, uint32_t* __restrict__ uidx) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t le;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(le));
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = w0; c < nchunks; c += nw) {
        uint32_t base = chunk_base[c];
        for (uint32_t r = 0; r < kChunk / 32; ++r) {
            const uint64_t pos = c * kChunk + 32 * r + lane;
            const bool valid = pos < m;
            const uint32_t w = valid ? dest[pos] : 0u;
            const uint32_t b = __ballot_sync(kAll, valid && (w >> 31));
            if (valid) uidx[atomicAdd(&cursor[w & kIdMask], 1u)] = base + __popc(b & le) - 1u;
            base += __popc(b);
        }
    }
}

// ------------------------------------------------------------ iteration
// R[s, j] = 1 / |S_j| for every seed entry; dangling seeds give D_j of R = T.
__global__ void seed_init_kernel(const uint32_t* __restrict__ snode, const uint32_t* __restrict__ scol,
                                 const float* __restrict__ sw, uint32_t nseeds, const float* __restrict__ inv_deg,
                                 float* __restrict__ r, double* __restrict__ dang) {
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nseeds; e += gridDim.x * blockDim.x) {
        const uint32_t v = snode[e], j = scol[e];
        r[(size_t)v * kCols + j] = sw[e];
        if (inv_deg[v] == 0.0f) atomicAdd(&dang[j], (double)sw[e]);
    }
}

// Scatter: row t of `upd` = R[u, :] * (1/|N_o(u)|) for every update t of u.
__global__ void __launch_bounds__(kPprThreads) ppr_scatter_kernel(const float* __restrict__ r,
                                                                   const float* __restrict__ inv_deg,
                                                                   const uint32_t* __restrict__ uptr,
                                                                   const uint32_t* __restrict__ upos, uint32_t n,
                                                                   float* __restrict__ upd) {
    const uint32_t lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t vb = 2 * gw; vb < n; vb += 2 * nw) {  // warp-uniform
        const uint64_t u = vb + half;
        const bool live = u < n;
        uint32_t beg = 0, end = 0;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live) {
            beg = uptr[u];
            end = uptr[u + 1];
            if (end > beg) x = scale4(ld4(r + u * kCols + 4 * hl), inv_deg[u]);
        }
        const uint32_t nb = (end - beg + 15) / 16;
        const uint32_t nmax = max(nb, __shfl_xor_sync(kAll, nb, 16));
        for (uint32_t it = 0; it < nmax; ++it) {
            const uint32_t e0 = beg + 16 * it;
            const uint32_t tl = e0 + hl < end ? upos[e0 + hl] : 0u;
#pragma unroll
            for (uint32_t i = 0; i < 16; ++i) {
                const uint32_t t = __shfl_sync(kAll, tl, i, 16);
                if (e0 + i < end) st4_stream(upd + (size_t)t * kCols + 4 * hl, x);
            }
        }
    }
}

// Sum of the update rows uidx[beg .. end) (16 lanes, columns 4 hl .. 4 hl + 3);
// warp-uniform trip count (both halves call it together).
__device__ __forceinline__ float4 sum_rows(const float* __restrict__ upd, const uint32_t* __restrict__ uidx,
                                           uint32_t beg, uint32_t end, uint32_t hl) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t nb = (end - beg + 15) / 16;
    const uint32_t nmax = max(nb, __shfl_xor_sync(kAll, nb, 16));
    for (uint32_t it = 0; it < nmax; ++it) {
        const uint32_t e0 = beg + 16 * it;
        const uint32_t tl = e0 + hl < end ? uidx[e0 + hl] : 0u;
        float4 x[16];
#pragma unroll
        for (uint32_t i = 0; i < 16; ++i) {
            const uint32_t t = __shfl_sync(kAll, tl, i, 16);
            x[i] = e0 + i < end ? ld4(upd + (size_t)t * kCols + 4 * hl) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (uint32_t i = 0; i < 16; ++i) acc = add4(acc, x[i]);
    }
    return acc;
}

// The apply of node v: R'[v] = d * sum + (1 - d + d * D_j) t_j[v]; adds its
// L1 change and (dangling v) its mass to the lane's column partials.
__device__ __forceinline__ void finish_row(uint32_t v, float4 sum, float d, const float* __restrict__ r_old,
                                           float* __restrict__ r_new, const float* __restrict__ inv_deg,
                                           const uint32_t* __restrict__ nsp, const uint32_t* __restrict__ nscol,
                                           const float* __restrict__ nsw, const double* __restrict__ dang,
                                           uint32_t hl, float4& res, float4& dg) {
    float4 y = scale4(sum, d);
    for (uint32_t e = nsp[v]; e < nsp[v + 1]; ++e) {  // v's seed entries (rare)
        const uint32_t j = nscol[e];
        if (j / 4 == hl) add_comp(y, j & 3u, (1.0f - d + d * (float)dang[j]) * nsw[e]);
    }
    const float4 o = ld4(r_old + (size_t)v * kCols + 4 * hl);
    res.x += fabsf(y.x - o.x);
    res.y += fabsf(y.y - o.y);
    res.z += fabsf(y.z - o.z);
    res.w += fabsf(y.w - o.w);
    if (inv_deg[v] == 0.0f) dg = add4(dg, y);
    *reinterpret_cast<float4*>(r_new + (size_t)v * kCols + 4 * hl) = y;
}

// Column partials of the block (FP64): slots [0, 64) L1 change, [64, 128) dangling mass.
__device__ void block_partials(float4 res, float4 dg, double* __restrict__ out) {
    __shared__ double sh[kPprThreads / 32][kSlots];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, hl = lane & 15;
    // the two halves hold the same columns
    res.x += __shfl_xor_sync(kAll, res.x, 16);
    res.y += __shfl_xor_sync(kAll, res.y, 16);
    res.z += __shfl_xor_sync(kAll, res.z, 16);
    res.w += __shfl_xor_sync(kAll, res.w, 16);
    dg.x += __shfl_xor_sync(kAll, dg.x, 16);
    dg.y += __shfl_xor_sync(kAll, dg.y, 16);
    dg.z += __shfl_xor_sync(kAll, dg.z, 16);
    dg.w += __shfl_xor_sync(kAll, dg.w, 16);
    if (lane < 16) {
        sh[warp][4 * hl] = res.x;
        sh[warp][4 * hl + 1] = res.y;
        sh[warp][4 * hl + 2] = res.z;
        sh[warp][4 * hl + 3] = res.w;
        sh[warp][kCols + 4 * hl] = dg.x;
        sh[warp][kCols + 4 * hl + 1] = dg.y;
        sh[warp][kCols + 4 * hl + 2] = dg.z;
        sh[warp][kCols + 4 * hl + 3] = dg.w;
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < (uint32_t)kSlots; c += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kPprThreads / 32; ++w) s += sh[w][c];
        out[(size_t)blockIdx.x * kSlots + c] = s;
    }
}

// Per-destination flags: summed in pieces (not here), has seed entries.
constexpr uint8_t kFlagSplit = 1, kFlagSeed = 2;

// Gather + apply of the destinations that are not split. Half-warp h walks the
// contiguous destinations [vrange[h], vrange[h+1]) (balanced by entries on the
// host) as a pipeline: while the rows of v are summed, the next column
// pointer, the first 16 entry indices of v + 1, its old rank row and its
// flags are already in flight, so a destination costs about one memory round.
__global__ void __launch_bounds__(kPprThreads) ppr_gather_kernel(
    const float* __restrict__ upd, const uint32_t* __restrict__ colptr, const uint32_t* __restrict__ uidx,
    const uint8_t* __restrict__ vflag, const uint32_t* __restrict__ vrange, uint32_t nhalves, float d,
    const float* __restrict__ r_old, float* __restrict__ r_new, const float* __restrict__ inv_deg,
    const uint32_t* __restrict__ nsp, const uint32_t* __restrict__ nscol, const float* __restrict__ nsw,
    const double* __restrict__ dang, double* __restrict__ partials) {
    const uint32_t lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const uint32_t h = 2 * ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) + half;
    const uint32_t va = h < nhalves ? vrange[h] : 0u, vb = h < nhalves ? vrange[h + 1] : 0u;
    const uint32_t nv = vb - va;
    const uint32_t nvmax = max(nv, __shfl_xor_sync(kAll, nv, 16));
    float4 res = make_float4(0.f, 0.f, 0.f, 0.f), dg = res;
    // pipeline registers for the destination of the coming step
    uint32_t b0 = 0, e0 = 0, tl = 0, fl = 0;
    float inv = 0.f;
    float4 ro = make_float4(0.f, 0.f, 0.f, 0.f);
    auto prefetch = [&](uint32_t v, uint32_t b, uint32_t e) {  // v < vb
        fl = vflag[v];
        inv = inv_deg[v];
        ro = ld4(r_old + (size_t)v * kCols + 4 * hl);
        tl = (!(fl & kFlagSplit) && b + hl < e) ? uidx[b + hl] : 0u;
    };
    if (nv) {
        b0 = colptr[va];
        e0 = colptr[va + 1];
        prefetch(va, b0, e0);
    }
    for (uint32_t step = 0; step < nvmax; ++step) {  // warp-uniform
        const bool live = step < nv;
        const uint32_t v = va + step;
        const uint32_t b = b0, fv = fl, tv = tl;
        const bool split = (fv & kFlagSplit) != 0;
        const uint32_t e = split ? b : e0;
        const float iv = inv;
        const float4 rov = ro;
        // issue the next destination's loads before this one's rows
        if (live && step + 1 < nv) {
            b0 = e0;
            e0 = colptr[v + 2];
            prefetch(v + 1, b0, e0);
        }
        // rows of v: the first 16 indices are in tv; each later chunk's
        // indices load while the previous chunk's rows are in flight
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t nb = live ? (e - b + 15) / 16 : 0u;
        const uint32_t nbmax = max(nb, __shfl_xor_sync(kAll, nb, 16));
        uint32_t tc = tv;
        for (uint32_t it = 0; it < nbmax; ++it) {
            const uint32_t c0 = b + 16 * it;
            float4 x[16];
#pragma unroll
            for (uint32_t i = 0; i < 16; ++i) {
                const uint32_t t = __shfl_sync(kAll, tc, i, 16);
                x[i] = (live && c0 + i < e) ? ld4(upd + (size_t)t * kCols + 4 * hl) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            tc = (live && c0 + 16 + hl < e) ? uidx[c0 + 16 + hl] : 0u;
#pragma unroll
            for (uint32_t i = 0; i < 16; ++i) acc = add4(acc, x[i]);
        }
        if (live && !split) {
            float4 y = scale4(acc, d);
            if (fv & kFlagSeed)
                for (uint32_t q = nsp[v]; q < nsp[v + 1]; ++q) {
                    const uint32_t j = nscol[q];
                    if (j / 4 == hl) add_comp(y, j & 3u, (1.0f - d + d * (float)dang[j]) * nsw[q]);
                }
            res.x += fabsf(y.x - rov.x);
            res.y += fabsf(y.y - rov.y);
            res.z += fabsf(y.z - rov.z);
            res.w += fabsf(y.w - rov.w);
            if (iv == 0.0f) dg = add4(dg, y);
            *reinterpret_cast<float4*>(r_new + (size_t)v * kCols + 4 * hl) = y;
        }
    }
    block_partials(res, dg, partials);
}

// Pieces of the split destinations: (v, first entry, end entry, scratch row).
__global__ void __launch_bounds__(kPprThreads) ppr_pieces_kernel(const float* __restrict__ upd,
                                                                  const uint32_t* __restrict__ uidx,
                                                                  const uint4* __restrict__ pieces,
                                                                  uint32_t npieces, float* __restrict__ scratch) {
    const uint32_t lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t pb = 2 * gw; pb < npieces; pb += 2 * nw) {
        const uint64_t pi = pb + half;
        uint4 pc = make_uint4(0, 0, 0, 0);
        if (pi < npieces) pc = pieces[pi];
        const float4 s = sum_rows(upd, uidx, pc.y, pc.z, hl);
        if (pi < npieces) {
            float* row = scratch + (size_t)pc.w * kCols + 4 * hl;
            atomicAdd(row, s.x);
            atomicAdd(row + 1, s.y);
            atomicAdd(row + 2, s.z);
            atomicAdd(row + 3, s.w);
        }
    }
}

// Apply of the split destinations from their scratch rows (cleared after use).
__global__ void __launch_bounds__(kPprThreads) ppr_split_apply_kernel(
    const uint32_t* __restrict__ split, uint32_t nsplit, float* __restrict__ scratch, float d,
    const float* __restrict__ r_old, float* __restrict__ r_new, const float* __restrict__ inv_deg,
    const uint32_t* __restrict__ nsp, const uint32_t* __restrict__ nscol, const float* __restrict__ nsw,
    const double* __restrict__ dang, double* __restrict__ partials) {
    const uint32_t lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    float4 res = make_float4(0.f, 0.f, 0.f, 0.f), dg = res;
    for (uint64_t hb = 2 * gw; hb < nsplit; hb += 2 * nw) {
        const uint64_t h = hb + half;
        if (h < nsplit) {
            float* row = scratch + (size_t)h * kCols + 4 * hl;
            const float4 s = *reinterpret_cast<const float4*>(row);
            *reinterpret_cast<float4*>(row) = make_float4(0.f, 0.f, 0.f, 0.f);
            finish_row(split[h], s, d, r_old, r_new, inv_deg, nsp, nscol, nsw, dang, hl, res, dg);
        }
    }
    block_partials(res, dg, partials);
}

// Column sums of the partials: the iteration's L1 change per column into
// hist, and the new dangling mass per column for the next iteration.
constexpr int kReduceSplit = 8;  // threads per slot
__global__ void __launch_bounds__(kSlots * kReduceSplit) ppr_reduce_kernel(const double* __restrict__ partials,
                                                                           uint32_t nblocks,
                                                                           double* __restrict__ hist,
                                                                           double* __restrict__ dang) {
    __shared__ double sh[kReduceSplit][kSlots];
    const uint32_t c = threadIdx.x % kSlots, part = threadIdx.x / kSlots;
    double s = 0.0;
    for (uint32_t b = part; b < nblocks; b += kReduceSplit) s += partials[(size_t)b * kSlots + c];
    sh[part][c] = s;
    __syncthreads();
    if (part == 0) {
        for (int p = 1; p < kReduceSplit; ++p) s += sh[p][c];
        if (c < (uint32_t)kCols) hist[c] = s;
        else dang[c - kCols] = s;
    }
}

int grid_blocks(int sms) { return std::max(1, sms * 8); }

}  // namespace
}  // namespace pcpm

using namespace pcpm;

struct pcpm_ppr {
    pcpm_png* png;
    uint32_t n, nseeds, nsplit, npieces;
    uint64_t m, ne;
    uint32_t *uptr, *upos, *colptr, *uidx;
    uint8_t* vflag;      // per destination: kFlagSplit, kFlagSeed
    uint32_t* vrange;    // gather: destination range of every half-warp
    uint32_t nhalves;
    uint32_t* split;     // destinations summed in pieces
    uint4* pieces;       // (v, first entry, end entry, scratch row)
    float* scratch;      // nsplit rows
    uint32_t *snode, *scol, *nsp, *nscol;
    float *sw, *nsw;
    float* r[2];
    int cur;
    float* upd;          // ne rows
    double* dang;        // kCols: dangling mass of r[cur]
    double* partials;
    uint32_t gather_blocks, split_blocks;
    double* hist;
    int hist_cap, last_iters;
    uint64_t device_bytes;
    cudaStream_t alloc_stream, last_stream;
};

namespace {

cudaError_t ppr_alloc(pcpm_ppr* h, void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    const cudaError_t e = pool_alloc(p, bytes, h->alloc_stream);
    if (e == cudaSuccess) h->device_bytes += bytes;
    return e;
}

void ppr_release(pcpm_ppr* h) {
    if (!h) return;
    void* ptrs[] = {h->uptr, h->upos, h->colptr, h->uidx, h->vflag, h->vrange, h->split, h->pieces, h->scratch, h->snode, h->scol,
                    h->nsp, h->nscol, h->sw, h->nsw, h->r[0], h->r[1], h->upd, h->dang, h->partials, h->hist};
    for (void* p : ptrs) pool_free(p, h->last_stream);
    delete h;
}

int ppr_build(pcpm_ppr* h, const std::vector<uint32_t>& seed_node, const std::vector<uint32_t>& seed_col,
              const std::vector<float>& seed_w, cudaStream_t s) {
    pcpm_png* g = h->png;
    const uint32_t n = h->n;
    const int grid = grid_blocks(g->sms);
    // by source: upos
    PCK(ppr_alloc(h, (void**)&h->uptr, ((size_t)n + 1) * sizeof(uint32_t)));
    PCK(ppr_alloc(h, (void**)&h->upos, std::max<uint64_t>(h->ne, 1) * sizeof(uint32_t)));
    struct Scratch {  // a build temporary, returned to the pool in s's order on every path
        uint32_t* p = nullptr;
        cudaStream_t s;
        ~Scratch() { pool_free(p, s); }
    } cnt{nullptr, s};
    PCK(pool_alloc((void**)&cnt.p, ((size_t)n + 1) * sizeof(uint32_t), s));
    int rc = PCPM_OK;
    PCK(cudaMemsetAsync(cnt.p, 0, (size_t)n * sizeof(uint32_t), s));
    if (h->ne) count_keys_kernel<<<grid, 256, 0, s>>>(g->src, h->ne, 0xFFFFFFFFu, cnt.p);
    if ((rc = exclusive_scan_u32(cnt.p, h->uptr, n, s)) != PCPM_OK) return rc;
    PCK(cudaMemcpyAsync(cnt.p, h->uptr, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    if (h->ne) fill_by_source_kernel<<<grid, 256, 0, s>>>(g->src, h->ne, cnt.p, h->upos);
    // by destination: uidx
    PCK(ppr_alloc(h, (void**)&h->colptr, ((size_t)n + 1) * sizeof(uint32_t)));
    PCK(ppr_alloc(h, (void**)&h->uidx, std::max<uint64_t>(h->m, 1) * sizeof(uint32_t)));
    PCK(cudaMemsetAsync(cnt.p, 0, (size_t)n * sizeof(uint32_t), s));
    if (h->m) count_keys_kernel<<<grid, 256, 0, s>>>(g->dest, h->m, kIdMask, cnt.p);
    if ((rc = exclusive_scan_u32(cnt.p, h->colptr, n, s)) != PCPM_OK) return rc;
    PCK(cudaMemcpyAsync(cnt.p, h->colptr, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    if (h->m)
        fill_by_destination_kernel<<<grid, 256, 0, s>>>(g->dest, h->m, g->chunk_base, g->nchunks, cnt.p, h->uidx);
    if ((rc = launch_status()) != PCPM_OK) return rc;
    // destinations split into pieces (found on the host from colptr)
    std::vector<uint32_t> cp((size_t)n + 1);
    PCK(cudaMemcpyAsync(cp.data(), h->colptr, ((size_t)n + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    std::vector<uint32_t> split;
    std::vector<uint4> pieces;
    for (uint32_t v = 0; v < n; ++v) {
        const uint32_t b = cp[v], e = cp[v + 1];
        if (e - b <= kPieceEntries) continue;
        const uint32_t row = (uint32_t)split.size();
        split.push_back(v);
        for (uint32_t x = b; x < e; x += kPieceEntries) pieces.push_back(make_uint4(v, x, std::min(e, x + kPieceEntries), row));
    }
    h->nsplit = (uint32_t)split.size();
    h->npieces = (uint32_t)pieces.size();
    PCK(ppr_alloc(h, (void**)&h->split, std::max<size_t>(split.size(), 1) * sizeof(uint32_t)));
    PCK(ppr_alloc(h, (void**)&h->pieces, std::max<size_t>(pieces.size(), 1) * sizeof(uint4)));
    PCK(ppr_alloc(h, (void**)&h->scratch, std::max<size_t>(split.size(), 1) * kCols * sizeof(float)));
    if (!split.empty())
        PCK(cudaMemcpyAsync(h->split, split.data(), split.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    if (!pieces.empty())
        PCK(cudaMemcpyAsync(h->pieces, pieces.data(), pieces.size() * sizeof(uint4), cudaMemcpyHostToDevice, s));
    PCK(cudaMemsetAsync(h->scratch, 0, std::max<size_t>(split.size(), 1) * kCols * sizeof(float), s));
    // seeds: entries (node, column, weight) and the same grouped by node
    const uint32_t S = h->nseeds;
    std::vector<uint32_t> order(S), nsp((size_t)n + 1, 0), nscol(S);
    std::vector<float> nsw(S);
    for (uint32_t e = 0; e < S; ++e) ++nsp[seed_node[e] + 1];
    for (uint32_t v = 0; v < n; ++v) nsp[v + 1] += nsp[v];
    {
        std::vector<uint32_t> cur(nsp.begin(), nsp.end() - 1);
        for (uint32_t e = 0; e < S; ++e) {
            const uint32_t at = cur[seed_node[e]]++;
            nscol[at] = seed_col[e];
            nsw[at] = seed_w[e];
        }
    }
    PCK(ppr_alloc(h, (void**)&h->snode, S * sizeof(uint32_t)));
    PCK(ppr_alloc(h, (void**)&h->scol, S * sizeof(uint32_t)));
    PCK(ppr_alloc(h, (void**)&h->sw, S * sizeof(float)));
    PCK(ppr_alloc(h, (void**)&h->nsp, ((size_t)n + 1) * sizeof(uint32_t)));
    PCK(ppr_alloc(h, (void**)&h->nscol, S * sizeof(uint32_t)));
    PCK(ppr_alloc(h, (void**)&h->nsw, S * sizeof(float)));
    PCK(cudaMemcpyAsync(h->snode, seed_node.data(), S * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(h->scol, seed_col.data(), S * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(h->sw, seed_w.data(), S * sizeof(float), cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(h->nsp, nsp.data(), ((size_t)n + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(h->nscol, nscol.data(), S * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(h->nsw, nsw.data(), S * sizeof(float), cudaMemcpyHostToDevice, s));
    // per-destination flags; gather ranges balanced by entries (+8 per destination)
    {
        std::vector<uint8_t> flag(n, 0);
        for (uint32_t v : split) flag[v] |= kFlagSplit;
        for (uint32_t v = 0; v < n; ++v)
            if (nsp[v + 1] > nsp[v]) flag[v] |= kFlagSeed;
        int per_sm = 0;
        PCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ppr_gather_kernel, kPprThreads, 0));
        h->gather_blocks = (uint32_t)std::max(1, per_sm * g->sms);
        h->nhalves = h->gather_blocks * (kPprThreads / 16);
        std::vector<uint64_t> cost((size_t)n + 1, 0);
        for (uint32_t v = 0; v < n; ++v)
            cost[v + 1] = cost[v] + 8 + ((flag[v] & kFlagSplit) ? 0 : (uint64_t)(cp[v + 1] - cp[v]));
        std::vector<uint32_t> vr((size_t)h->nhalves + 1);
        for (uint32_t i = 0; i <= h->nhalves; ++i) {
            const uint64_t target = cost[n] * i / h->nhalves;
            vr[i] = (uint32_t)(std::lower_bound(cost.begin(), cost.end(), target) - cost.begin());
            vr[i] = std::min(vr[i], n);
        }
        vr[0] = 0;
        vr[h->nhalves] = n;
        PCK(ppr_alloc(h, (void**)&h->vflag, std::max<size_t>(n, 1)));
        PCK(ppr_alloc(h, (void**)&h->vrange, ((size_t)h->nhalves + 1) * sizeof(uint32_t)));
        PCK(cudaMemcpyAsync(h->vflag, flag.data(), n, cudaMemcpyHostToDevice, s));
        PCK(cudaMemcpyAsync(h->vrange, vr.data(), ((size_t)h->nhalves + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice,
                            s));
        PCK(cudaStreamSynchronize(s));  // the host vectors leave scope
    }
    // iteration state
    const size_t rows = (size_t)n * kCols * sizeof(float);
    PCK(ppr_alloc(h, (void**)&h->r[0], rows));
    PCK(ppr_alloc(h, (void**)&h->r[1], rows));
    PCK(ppr_alloc(h, (void**)&h->upd, std::max<uint64_t>(h->ne, 1) * kCols * sizeof(float)));
    PCK(ppr_alloc(h, (void**)&h->dang, kCols * sizeof(double)));
    h->split_blocks = (uint32_t)std::max(1, std::min(grid, (int)((h->nsplit + 15) / 16)));
    PCK(ppr_alloc(h, (void**)&h->partials, (size_t)(h->gather_blocks + h->split_blocks) * kSlots * sizeof(double)));
    h->hist_cap = 64;
    PCK(ppr_alloc(h, (void**)&h->hist, (size_t)h->hist_cap * kCols * sizeof(double)));
    PCK(cudaStreamSynchronize(s));
    return PCPM_OK;
}

}  // namespace

extern "C" {

int pcpm_ppr_create(pcpm_png* png, const uint32_t* seed_ptr, const uint32_t* seed_idx, void* stream,
                    pcpm_ppr** out) {
    if (!png || !seed_ptr || !out || png->weighted) return PCPM_EINVAL;
    if (seed_ptr[0] != 0) return PCPM_EINVAL;
    const uint32_t n = png->n;
    std::vector<uint32_t> node, col;
    std::vector<float> w;
    for (int j = 0; j < kCols; ++j) {
        const uint32_t b = seed_ptr[j], e = seed_ptr[j + 1];
        if (e <= b || !seed_idx) return PCPM_EINVAL;
        std::vector<uint32_t> s(seed_idx + b, seed_idx + e);
        std::sort(s.begin(), s.end());
        if (s.back() >= n || std::adjacent_find(s.begin(), s.end()) != s.end()) return PCPM_EINVAL;
        for (uint32_t v : s) {
            node.push_back(v);
            col.push_back((uint32_t)j);
            w.push_back(1.0f / (float)(e - b));
        }
    }
    pcpm_ppr* h = new (std::nothrow) pcpm_ppr;
    if (!h) return PCPM_ENOMEM;
    std::memset(h, 0, sizeof(*h));
    h->png = png;
    h->n = n;
    h->m = png->m;
    h->ne = png->ne;
    h->nseeds = (uint32_t)node.size();
    h->alloc_stream = h->last_stream = (cudaStream_t)stream;
    const int rc = ppr_build(h, node, col, w, (cudaStream_t)stream);
    if (rc != PCPM_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaGetLastError();
        ppr_release(h);
        return rc;
    }
    *out = h;
    return PCPM_OK;
}

int pcpm_ppr_run(pcpm_ppr* h, float d, int iters, void* stream) {
    if (!h || iters < 0 || !(d >= 0.0f && d < 1.0f)) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    if (iters > h->hist_cap) {
        double* nh = nullptr;
        PCK(pool_alloc((void**)&nh, (size_t)iters * kCols * sizeof(double), s));
        pool_free(h->hist, s);
        h->device_bytes += (size_t)(iters - h->hist_cap) * kCols * sizeof(double);
        h->hist = nh;
        h->hist_cap = iters;
    }
    pcpm_png* g = h->png;
    const uint32_t n = h->n;
    // R = T and its dangling mass
    h->cur = 0;
    PCK(cudaMemsetAsync(h->r[0], 0, (size_t)n * kCols * sizeof(float), s));
    PCK(cudaMemsetAsync(h->dang, 0, kCols * sizeof(double), s));
    seed_init_kernel<<<std::max(1u, (h->nseeds + 255) / 256), 256, 0, s>>>(h->snode, h->scol, h->sw, h->nseeds,
                                                                         g->inv_deg, h->r[0], h->dang);
    if (launch_status() != PCPM_OK) return PCPM_ECUDA;
    for (int i = 0; i < iters; ++i) {
        const float* ro = h->r[h->cur];
        float* rn = h->r[h->cur ^ 1];
        ppr_scatter_kernel<<<h->gather_blocks, kPprThreads, 0, s>>>(ro, g->inv_deg, h->uptr, h->upos, n, h->upd);
        ppr_gather_kernel<<<h->gather_blocks, kPprThreads, 0, s>>>(h->upd, h->colptr, h->uidx, h->vflag,
                                                                   h->vrange, h->nhalves, d, ro, rn, g->inv_deg,
                                                                   h->nsp, h->nscol, h->nsw, h->dang, h->partials);
        uint32_t nb = h->gather_blocks;
        if (h->nsplit) {
            ppr_pieces_kernel<<<h->gather_blocks, kPprThreads, 0, s>>>(h->upd, h->uidx, h->pieces, h->npieces,
                                                                       h->scratch);
            ppr_split_apply_kernel<<<h->split_blocks, kPprThreads, 0, s>>>(
                h->split, h->nsplit, h->scratch, d, ro, rn, g->inv_deg, h->nsp, h->nscol, h->nsw, h->dang,
                h->partials + (size_t)h->gather_blocks * kSlots);
            nb += h->split_blocks;
        }
        ppr_reduce_kernel<<<1, kSlots * kReduceSplit, 0, s>>>(h->partials, nb, h->hist + (size_t)i * kCols, h->dang);
        if (launch_status() != PCPM_OK) return PCPM_ECUDA;
        h->cur ^= 1;
    }
    h->last_iters = iters;
    return PCPM_OK;
}

int pcpm_ppr_residuals(pcpm_ppr* h, double* out, int iters) {
    if (!h || iters < 0 || iters > h->last_iters || (iters > 0 && !out)) return PCPM_EINVAL;
    PCK(cudaStreamSynchronize(h->last_stream));
    if (iters) PCK(cudaMemcpy(out, h->hist, (size_t)iters * kCols * sizeof(double), cudaMemcpyDeviceToHost));
    return PCPM_OK;
}

int pcpm_ppr_ranks(pcpm_ppr* h, float* out, void* stream) {
    if (!h || !out) return PCPM_EINVAL;
    PCK(cudaMemcpyAsync(out, h->r[h->cur], (size_t)h->n * kCols * sizeof(float), cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream));
    return PCPM_OK;
}

int pcpm_ppr_info(const pcpm_ppr* h, uint64_t* device_bytes, uint32_t* split_destinations) {
    if (!h) return PCPM_EINVAL;
    if (device_bytes) *device_bytes = h->device_bytes;
    if (split_destinations) *split_destinations = h->nsplit;
    return PCPM_OK;
}

void pcpm_ppr_free(pcpm_ppr* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    cudaGetLastError();
    ppr_release(h);
}

}  // extern "C"
