// pcpm_api.cu - the extern "C" boundary: argument checks, handle lifetime,
// the iteration loop and host-side copies. All arithmetic of the method runs
// in the kernels of png_build.cu and pcpm_iter.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "pcpm_internal.cuh"

namespace pcpm {


namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t pool_for_current_device(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pool_for_current_device(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, s);
}

void pool_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

cudaError_t dev_alloc(pcpm_png* g, void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    cudaError_t e = pool_alloc(p, bytes, g->alloc_stream);
    if (e == cudaSuccess) g->device_bytes += bytes;
    return e;
}

thread_local cudaError_t g_last_cuda_error = cudaSuccess;

void note_cuda_error(cudaError_t e) { g_last_cuda_error = e; }

int launch_status() {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return PCPM_OK;
    note_cuda_error(e);
    return PCPM_ECUDA;
}

namespace {

#define CK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            note_cuda_error(e_);                                                  \
            return e_ == cudaErrorMemoryAllocation ? PCPM_ENOMEM : PCPM_ECUDA;    \
        }                                                                         \
    } while (0)

#define RC(call)                          \
    do {                                  \
        int r_ = (call);                  \
        if (r_ != PCPM_OK) return r_;     \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void release(pcpm_png* g) {
    if (!g) return;
    void* ptrs[] = {g->dest, g->src, g->src16, g->bin_u, g->bin_e, g->seg_u, g->cnt_u, g->seg_e, g->cnt_e,
                    g->chunk_base, g->hubs, g->gdest, g->gslice_start, g->gslice_bytes, g->ichunk_start,
                    g->gunits, g->gorder, g->sunits, g->sorder, g->gacc,
                    g->bin_done, g->inv_deg, g->pr[0], g->pr[1], g->upd[0], g->upd[1], g->partials,
                    g->hist, g->state, g->wdest, g->gweight, g->win_start, g->wwords, g->wweight, g->wdesc,
                    g->whubs, g->indeg, g->dq_err};
    // the caller has waited for every use of the handle's memory
    for (void* p : ptrs) pool_free(p, g->last_stream);
    if (g->state_host) cudaFreeHost(g->state_host);
    delete g;
}

int alloc_state(pcpm_png* g) {
    const uint32_t n = g->n;
    const cudaStream_t s = g->alloc_stream;
    CK(dev_alloc(g, (void**)&g->pr[0], (size_t)n * sizeof(float)));
    CK(dev_alloc(g, (void**)&g->pr[1], (size_t)n * sizeof(float)));
    // Update bins: two buffers (the fused iteration gathers one and scatters
    // the next), padded so a chunk's update slice may round up past the end.
    // 16 spare entries: 16-byte update groups and slices never leave the buffer.
    const size_t ubytes = (g->ne + 16) * g->upd_bytes;
    CK(dev_alloc(g, (void**)&g->upd[0], ubytes));
    CK(dev_alloc(g, (void**)&g->upd[1], ubytes));
    CK(cudaMemsetAsync(g->upd[0], 0, ubytes, s));
    CK(cudaMemsetAsync(g->upd[1], 0, ubytes, s));
    CK(dev_alloc(g, (void**)&g->partials, 2 * partial_slots(g) * sizeof(double)));
    CK(dev_alloc(g, (void**)&g->gacc, (size_t)n * sizeof(float)));
    CK(dev_alloc(g, (void**)&g->bin_done, (size_t)g->k * sizeof(uint32_t)));
    if (g->upd_bytes == 2) {  // the rounding carried between delta iterations
        CK(dev_alloc(g, (void**)&g->dq_err, (size_t)2 * n * sizeof(float)));
        CK(cudaMemsetAsync(g->dq_err, 0, (size_t)2 * n * sizeof(float), s));
    }
    CK(cudaMemsetAsync(g->gacc, 0, (size_t)n * sizeof(float), s));
    CK(cudaMemsetAsync(g->bin_done, 0, (size_t)g->k * sizeof(uint32_t), s));
    g->hist_cap = 1024;
    CK(dev_alloc(g, (void**)&g->hist, (size_t)g->hist_cap * sizeof(double)));
    CK(dev_alloc(g, (void**)&g->state, sizeof(DevState)));
    CK(cudaMallocHost((void**)&g->state_host, sizeof(DevState)));
    std::memset(g->state_host, 0, sizeof(DevState));
    CK(cudaMemsetAsync(g->state, 0, sizeof(DevState), s));
    return PCPM_OK;
}

int ensure_hist(pcpm_png* g, int needed, cudaStream_t s) {
    if (needed <= g->hist_cap) return PCPM_OK;
    int cap = g->hist_cap;
    while (cap < needed) cap *= 2;
    double* h = nullptr;
    CK(pool_alloc((void**)&h, (size_t)cap * sizeof(double), s));
    cudaError_t e = cudaMemcpyAsync(h, g->hist, (size_t)g->hist_cap * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        pool_free(h, s);
        note_cuda_error(e);
        return PCPM_ECUDA;
    }
    pool_free(g->hist, s);
    g->device_bytes += (size_t)(cap - g->hist_cap) * sizeof(double);
    g->hist = h;
    g->hist_cap = cap;
    return PCPM_OK;
}

int check_device_err(const DevState& st) {
    if (st.err & kErrTimeout) return PCPM_ETIMEOUT;
    if (st.err) return PCPM_EDEVICE;
    return PCPM_OK;
}

int sync_state(pcpm_png* g, cudaStream_t s) {
    CK(cudaMemcpyAsync(g->state_host, g->state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return check_device_err(*g->state_host);
}

// Launches iterations [0, iters) with optional event records around kernels.
// Two-phase: scatter, gather + apply, reduce (the paper's phases). Fused: the
// gather kernel also scatters the next iteration's updates into the other
// buffer, so a standalone scatter runs only when no valid bins exist yet.
int run_iterations(pcpm_png* g, float d, int iters, double tol, uint32_t flags, cudaStream_t s,
                   std::vector<cudaEvent_t>* ev) {
    RC(ensure_hist(g, g->iters_done + iters, s));
    const bool fused = !(flags & (PCPM_TWO_PHASE | PCPM_DELTA)) && g->fused_ok;
    for (int i = 0; i < iters; ++i) {
        // the delta form needs the ranks before the current ones: from the
        // second iteration since the reset on
        const bool delta = (flags & PCPM_DELTA) && g->iters_done + i >= 1;
        if (ev) CK(cudaEventRecord((*ev)[4 * i], s));
        if (!fused || !g->upd_valid) RC(launch_scatter(g, s, false, delta, (flags & PCPM_DELTA) != 0));
        if (ev) CK(cudaEventRecord((*ev)[4 * i + 1], s));
        RC(launch_gather(g, d, flags, fused, s, false, delta));
        if (ev) CK(cudaEventRecord((*ev)[4 * i + 2], s));
        RC(launch_reduce(g, tol, g->iters_done + i, s));
        if (ev) CK(cudaEventRecord((*ev)[4 * i + 3], s));
        g->cur ^= 1;
        if (fused) {
            g->ucur ^= 1;
            g->upd_valid = 1;
        } else {
            g->upd_valid = 0;
        }
    }
    return PCPM_OK;
}

int iterate_impl(pcpm_png* g, float d, int iters, double tol, uint32_t flags, int* iters_run, double* last_residual,
                 cudaStream_t s) {
    g->last_stream = s;
    CK(cudaMemsetAsync(&g->state->stop, 0, sizeof(int), s));
    const int start_done = g->iters_done;
    const int start_cur = g->cur;
    const int start_ucur = g->ucur;
    const int start_dq = g->dq_cur;
    const int start_valid = g->upd_valid;
    const bool need_sync = tol > 0.0 || iters_run || last_residual;
    if (tol > 0.0) {
        // Batches of iterations; kernels after convergence return at once.
        const int batch = 8;
        int launched = 0;
        while (launched < iters) {
            const int b = std::min(batch, iters - launched);
            RC(run_iterations(g, d, b, tol, flags, s, nullptr));
            g->iters_done += b;  // provisional, corrected below
            launched += b;
            RC(sync_state(g, s));
            if (g->state_host->stop) break;
        }
    } else {
        RC(run_iterations(g, d, iters, tol, flags, s, nullptr));
        g->iters_done += iters;
        if (need_sync) RC(sync_state(g, s));
    }
    if (need_sync) {
        const int done = g->state_host->iters_done - start_done;
        g->iters_done = g->state_host->iters_done;
        g->cur = start_cur ^ (done & 1);
        if ((flags & PCPM_DELTA) && g->dq_err) g->dq_cur = start_dq ^ (done & 1);  // one scatter per iteration
        if (!(flags & (PCPM_TWO_PHASE | PCPM_DELTA)) && g->fused_ok) {
            g->ucur = start_ucur ^ (done & 1);
            g->upd_valid = done > 0 ? 1 : start_valid;
        } else if (done > 0) {
            g->upd_valid = 0;
        }
        if (iters_run) *iters_run = done;
        if (last_residual) *last_residual = done > 0 ? g->state_host->residual : 0.0;
        if (tol > 0.0 && !g->state_host->stop) return PCPM_NOT_CONVERGED;
    }
    return PCPM_OK;
}

bool bad_damping(float d) { return !(d >= 0.0f && d < 1.0f); }

// A handle that gathers only some destination partitions computes part of an
// iteration; it is driven by pcpm_shard_init / pcpm_shard_step only. A
// non-square matrix has no PageRank; it is driven by pcpm_spmv_rect only.
bool partial_shard(const pcpm_png* g) { return g->plo != 0 || g->phi != g->k || g->rect; }

constexpr uint32_t kAllFlags = PCPM_DANGLING_LEAK | PCPM_TWO_PHASE | PCPM_DELTA;

}  // namespace

// out(v) = sum over in-edges u -> v of pr_like(u) / outdeg(u): one PCPM pass,
// the scatter of pr_like * (1/outdeg) and a gather applied with d = 1 and no
// dangling term, so the apply returns the bare sum. Leaves the handle after
// that pass (callers reset before solving).
int pull_sum(pcpm_png* g, const float* pr_like, float* out, cudaStream_t s) {
    if (partial_shard(g)) return PCPM_EINVAL;
    g->last_stream = s;
    CK(cudaMemsetAsync(g->state, 0, sizeof(DevState), s));
    CK(cudaMemsetAsync(g->gacc, 0, (size_t)g->n * sizeof(float), s));
    CK(cudaMemsetAsync(g->bin_done, 0, (size_t)g->k * sizeof(uint32_t), s));
    g->cur = 0;
    g->iters_done = 0;
    g->upd_valid = 0;
    RC(launch_init(g, pr_like, s));
    RC(run_iterations(g, 1.0f, 1, 0.0, PCPM_TWO_PHASE | PCPM_DANGLING_LEAK, s, nullptr));
    g->iters_done = 1;
    CK(cudaMemcpyAsync(out, g->pr[g->cur], (size_t)g->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return PCPM_OK;
}

}  // namespace pcpm

using namespace pcpm;

extern "C" {

int pcpm_build(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m, uint32_t part_size,
               void* stream, pcpm_png** out) {
    return pcpm_build_ex(row_ptr, col_idx, n, m, part_size, nullptr, stream, out);
}

namespace {
// shard: build only the bins of destination partitions [part_lo, part_hi)
// from the edges into them (pcpm_build_shard).
int build_impl(const uint32_t* row_ptr, const uint32_t* col_idx, const float* weights, uint32_t n, uint64_t m,
               uint32_t part_size, const pcpm_build_options* options, void* stream, pcpm_png** out,
               bool shard = false, uint32_t part_lo = 0, uint32_t part_hi = 0, uint32_t rect_rows = 0,
               uint32_t rect_cols = 0) {
    if (!out || !row_ptr || n == 0 || n > PCPM_MAX_NODES || part_size == 0 || part_size > PCPM_MAX_PART_SIZE)
        return PCPM_EINVAL;
    pcpm_build_options opt = {};
    if (options) opt = *options;
    if (weights) {
        if (part_size > PCPM_MAX_WEIGHTED_PART_SIZE || opt.canonical_gather || opt.update_dtype != PCPM_UPDATE_F32)
            return PCPM_EINVAL;
        if (m > 0 && !is_device_ptr(weights)) return PCPM_EINVAL;
    }
    if (opt.gather_cluster != 0 && opt.gather_cluster != 1 && opt.gather_cluster != 2 && opt.gather_cluster != 4 &&
        opt.gather_cluster != 8)
        return PCPM_EINVAL;
    if (opt.gather_runs > 2 || opt.gather_windows > 2) return PCPM_EINVAL;
    if (opt.gather_windows == 1 && opt.canonical_gather) return PCPM_EINVAL;
    if (opt.update_dtype > PCPM_UPDATE_BF16) return PCPM_EINVAL;
    if (opt.update_dtype != PCPM_UPDATE_F32 && opt.canonical_gather) return PCPM_EINVAL;
    if (m > 0xFFFFFF00ull) return PCPM_EINVAL;
    const uint64_t k = ((uint64_t)n + part_size - 1) / part_size;
    if (k > PCPM_MAX_PARTITIONS) return PCPM_EINVAL;
    if (shard && (weights || part_lo >= part_hi || part_hi > k)) return PCPM_EINVAL;
    if (!is_device_ptr(row_ptr)) return PCPM_EINVAL;
    if (m > 0 && !is_device_ptr(col_idx)) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t ends[2] = {1, 0};
    CK(cudaMemcpyAsync(&ends[0], row_ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&ends[1], row_ptr + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] != m) return PCPM_EINVAL;

    pcpm_png* g = new (std::nothrow) pcpm_png;
    if (!g) return PCPM_ENOMEM;
    std::memset(g, 0, sizeof(*g));
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return PCPM_ECUDA;
    }
    g->n = n;
    g->q = part_size;
    g->k = (uint32_t)k;
    g->m = m;
    g->last_stream = s;
    g->alloc_stream = s;
    g->cluster = (int)opt.gather_cluster;
    g->upd_dtype = (int)opt.update_dtype;
    g->upd_bytes = opt.update_dtype == PCPM_UPDATE_F32 ? 4u : 2u;
    g->weighted = weights ? 1 : 0;
    g->weights_in = weights;
    g->plo = shard ? part_lo : 0;
    g->phi = shard ? part_hi : (uint32_t)k;
    if (rect_cols) {  // gather the column partitions only
        g->rect = 1;
        g->n_rows = rect_rows;
        g->n_cols = rect_cols;
        g->phi = (rect_cols + part_size - 1) / part_size;
    }
    int rc = PCPM_OK;
    if (cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) rc = PCPM_ECUDA;
    if (shard) {
        // the shard's own CSR: every source row, only the edges into its nodes
        uint32_t *rp = nullptr, *cl = nullptr;
        uint64_t ms = 0;
        const uint32_t vlo = part_lo * part_size;
        const uint32_t vhi = (uint32_t)std::min<uint64_t>((uint64_t)part_hi * part_size, n);
        if (rc == PCPM_OK) rc = shard_filter_csr(row_ptr, col_idx ? col_idx : row_ptr, n, m, vlo, vhi, &rp, &cl, &ms, s);
        if (rc == PCPM_OK) {
            g->m = ms;
            rc = build_png(g, rp, cl, opt, s);
        }
        // out-degrees (1/|N_o(u)|) are those of the whole graph
        if (rc == PCPM_OK) rc = compute_inv_deg(g, row_ptr, s);
        pool_free(rp, s);
        pool_free(cl, s);
    } else if (rc == PCPM_OK) {
        rc = build_png(g, row_ptr, col_idx ? col_idx : row_ptr, opt, s);
    }
    if (rc == PCPM_OK) rc = alloc_state(g);
    if (rc == PCPM_OK) rc = configure_kernels(g);
    if (rc == PCPM_OK) {
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = PCPM_ECUDA;
    }
    g->weights_in = nullptr;  // read during the build only
    if (rc != PCPM_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        release(g);
        return rc;
    }
    *out = g;
    return PCPM_OK;
}
}  // namespace

int pcpm_build_ex(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m, uint32_t part_size,
                  const pcpm_build_options* options, void* stream, pcpm_png** out) {
    return build_impl(row_ptr, col_idx, nullptr, n, m, part_size, options, stream, out);
}

int pcpm_build_weighted(const uint32_t* row_ptr, const uint32_t* col_idx, const float* weights, uint32_t n,
                        uint64_t m, uint32_t part_size, const pcpm_build_options* options, void* stream,
                        pcpm_png** out) {
    if (!weights) return PCPM_EINVAL;
    return build_impl(row_ptr, col_idx, weights, n, m, part_size, options, stream, out);
}

// ----------------------------------------------------- non-square matrices
namespace pcpm_rect {
__global__ void extend_rows_kernel(const uint32_t* __restrict__ row_ptr, uint32_t rows, uint32_t n,
                                   uint32_t* __restrict__ out) {
    const uint32_t end = row_ptr[rows];
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x)
        out[v] = v <= rows ? row_ptr[v] : end;
}
}  // namespace pcpm_rect

int pcpm_build_rect(const uint32_t* row_ptr, const uint32_t* col_idx, const float* weights, uint32_t n_rows,
                    uint32_t n_cols, uint64_t m, uint32_t part_size, const pcpm_build_options* options, void* stream,
                    pcpm_png** out) {
    if (!out || !row_ptr || n_rows == 0 || n_cols == 0 || part_size == 0 || part_size > PCPM_MAX_PART_SIZE)
        return PCPM_EINVAL;
    const uint32_t n = std::max(n_rows, n_cols);
    if (n > PCPM_MAX_NODES || ((uint64_t)n + part_size - 1) / part_size > PCPM_MAX_PARTITIONS || m > 0xFFFFFF00ull)
        return PCPM_EINVAL;
    if (!is_device_ptr(row_ptr) || (m > 0 && !is_device_ptr(col_idx))) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // every column index below n_cols (the build itself checks < n)
    if (m > 0) {
        std::vector<uint64_t> counts(((uint64_t)n_cols + part_size - 1) / part_size);
        RC(dest_partition_counts(col_idx, m, n_cols, part_size, counts.data(), s));
    }
    if (n_cols <= n_rows)
        return build_impl(row_ptr, col_idx, weights, n, m, part_size, options, stream, out, false, 0, 0, n_rows,
                          n_cols);
    // more columns than rows: rows n_rows .. n-1 are empty
    uint32_t* rp = nullptr;
    CK(pool_alloc((void**)&rp, ((size_t)n + 1) * sizeof(uint32_t), s));
    pcpm_rect::extend_rows_kernel<<<(int)std::min<uint64_t>(4096, ((uint64_t)n + 256) / 256), 256, 0, s>>>(row_ptr, n_rows, n,
                                                                                                 rp);
    int rc = launch_status();
    if (rc == PCPM_OK)
        rc = build_impl(rp, col_idx, weights, n, m, part_size, options, stream, out, false, 0, 0, n_rows, n_cols);
    cudaStreamSynchronize(s);
    pool_free(rp, s);
    return rc;
}

int pcpm_spmv_rect(pcpm_png* g, const float* x, float* y, void* stream) {
    if (!g || !g->rect || !is_device_ptr(x) || !is_device_ptr(y)) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    CK(cudaMemsetAsync(g->state, 0, sizeof(DevState), s));
    CK(cudaMemsetAsync(g->gacc, 0, (size_t)g->n * sizeof(float), s));
    CK(cudaMemsetAsync(g->bin_done, 0, (size_t)g->k * sizeof(uint32_t), s));
    g->cur = 0;
    g->iters_done = 0;
    g->upd_valid = 0;
    RC(launch_copy_pad(x, g->n_rows, g->pr[0], g->n, s));  // x on the rows, 0 past them
    RC(launch_scatter(g, s, /*raw=*/true));                // update[t] = x[src[t]], the row partitions
    RC(launch_gather(g, 1.0f, PCPM_DANGLING_LEAK, /*fused=*/false, s, /*spmv=*/true));  // the column partitions
    CK(cudaMemcpyAsync(y, g->pr[1], (size_t)g->n_cols * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return PCPM_OK;
}

// ------------------------------------------------------- destination shards
int pcpm_build_shard(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m, uint32_t part_size,
                     uint32_t part_lo, uint32_t part_hi, const pcpm_build_options* options, void* stream,
                     pcpm_png** out) {
    return build_impl(row_ptr, col_idx, nullptr, n, m, part_size, options, stream, out, true, part_lo, part_hi);
}

int pcpm_dest_partition_counts(const uint32_t* col_idx, uint64_t m, uint32_t n, uint32_t part_size,
                               uint64_t* counts, void* stream) {
    if (!counts || n == 0 || n > PCPM_MAX_NODES || part_size == 0 || part_size > PCPM_MAX_PART_SIZE ||
        m > 0xFFFFFF00ull)
        return PCPM_EINVAL;
    if (((uint64_t)n + part_size - 1) / part_size > PCPM_MAX_PARTITIONS) return PCPM_EINVAL;
    if (m > 0 && !is_device_ptr(col_idx)) return PCPM_EINVAL;
    return dest_partition_counts(col_idx, m, n, part_size, counts, (cudaStream_t)stream);
}

int pcpm_shard_split(const uint64_t* ids_per_part, uint32_t n, uint32_t part_size, uint32_t nranks,
                     uint32_t* part_lo) {
    if (!ids_per_part || !part_lo || n == 0 || part_size == 0 || nranks == 0) return PCPM_EINVAL;
    const uint64_t k = ((uint64_t)n + part_size - 1) / part_size;
    if (nranks > k) return PCPM_EINVAL;
    // w(p) = destination IDs of bin p + nodes of p: the gather's streamed IDs
    // plus the apply's per-node work (an edgeless graph splits by nodes).
    std::vector<uint64_t> pre(k + 1, 0);
    for (uint64_t p = 0; p < k; ++p) {
        const uint64_t nodes = std::min<uint64_t>(part_size, (uint64_t)n - p * part_size);
        pre[p + 1] = pre[p] + ids_per_part[p] + nodes;
    }
    const uint64_t W = pre[k];
    part_lo[0] = 0;
    for (uint32_t r = 1; r < nranks; ++r) {
        // the cut nearest r/nranks of the total weight, leaving at least one
        // partition to this rank and to each later one
        const long double t = (long double)W * r / nranks;
        uint64_t b = std::lower_bound(pre.begin(), pre.end(), (uint64_t)std::ceil(t)) - pre.begin();
        if (b > 0 && (t - (long double)pre[b - 1]) <= ((long double)pre[std::min<uint64_t>(b, k)] - t)) --b;
        const uint64_t lo = (uint64_t)part_lo[r - 1] + 1, hi = k - (nranks - r);
        part_lo[r] = (uint32_t)std::min(std::max(b, lo), hi);
    }
    part_lo[nranks] = (uint32_t)k;
    return PCPM_OK;
}

int pcpm_shard_init(pcpm_png* g, const float* pr_init, float* pr_out, double* sums, void* stream) {
    if (!g || g->rect || !is_device_ptr(pr_out) || !is_device_ptr(sums)) return PCPM_EINVAL;
    if (pr_init && !is_device_ptr(pr_init)) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    const uint32_t vlo = g->plo * g->q, vhi = (uint32_t)std::min<uint64_t>((uint64_t)g->phi * g->q, g->n);
    CK(cudaMemsetAsync(g->state, 0, sizeof(DevState), s));
    CK(cudaMemsetAsync(g->gacc, 0, (size_t)g->n * sizeof(float), s));
    CK(cudaMemsetAsync(g->bin_done, 0, (size_t)g->k * sizeof(uint32_t), s));
    g->iters_done = 0;
    g->upd_valid = 0;
    RC(launch_init_range(g, pr_init, pr_out, vlo, vhi, s));
    RC(launch_reduce(g, 0.0, -1, s));
    CK(cudaMemsetAsync(sums, 0, sizeof(double), s));
    CK(cudaMemcpyAsync(sums + 1, &g->state->dangling, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return PCPM_OK;
}

int pcpm_shard_step(pcpm_png* g, float d, uint32_t flags, const float* pr_in, float* pr_out, double* sums,
                    void* stream) {
    if (!g || g->rect || bad_damping(d) || (flags & ~kAllFlags) || (flags & PCPM_DELTA)) return PCPM_EINVAL;
    if (!is_device_ptr(pr_in) || !is_device_ptr(pr_out) || !is_device_ptr(sums) || pr_in == pr_out)
        return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    // the whole graph's dangling mass of pr_in, as the caller summed it
    CK(cudaMemcpyAsync(&g->state->dangling, sums + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(&g->state->stop, 0, sizeof(int), s));
    float* const saved[2] = {g->pr[0], g->pr[1]};
    const int saved_cur = g->cur;
    g->pr[0] = const_cast<float*>(pr_in);  // only read by the scatter and the apply
    g->pr[1] = pr_out;
    g->cur = 0;
    int rc = launch_scatter(g, s);
    if (rc == PCPM_OK) rc = launch_gather(g, d, flags | PCPM_TWO_PHASE, /*fused=*/false, s);
    if (rc == PCPM_OK) rc = launch_reduce(g, 0.0, 0, s, /*record=*/false);
    g->pr[0] = saved[0];
    g->pr[1] = saved[1];
    g->cur = saved_cur;
    g->upd_valid = 0;
    if (rc != PCPM_OK) return rc;
    g->iters_done += 1;
    CK(cudaMemcpyAsync(sums, &g->state->residual, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(sums + 1, &g->state->dangling, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return PCPM_OK;
}

int pcpm_sync_status(const pcpm_png* g) {
    if (!g) return PCPM_EINVAL;
    CK(cudaStreamSynchronize(g->last_stream));
    DevState st;
    CK(cudaMemcpy(&st, g->state, sizeof(DevState), cudaMemcpyDeviceToHost));
    return check_device_err(st);
}

int pcpm_spmv(pcpm_png* g, const float* x, float* y, void* stream) {
    if (!g || partial_shard(g) || !is_device_ptr(x) || !is_device_ptr(y)) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    CK(cudaMemsetAsync(g->state, 0, sizeof(DevState), s));
    CK(cudaMemsetAsync(g->gacc, 0, (size_t)g->n * sizeof(float), s));
    CK(cudaMemsetAsync(g->bin_done, 0, (size_t)g->k * sizeof(uint32_t), s));
    g->cur = 0;
    g->iters_done = 0;
    g->upd_valid = 0;
    RC(launch_init(g, x, s));                     // pr[0] = x
    RC(launch_scatter(g, s, /*raw=*/true));       // update[t] = x[src[t]] (Algorithm 3 without 1/outdeg)
    RC(launch_gather(g, 1.0f, PCPM_DANGLING_LEAK, /*fused=*/false, s, /*spmv=*/true));
    CK(cudaMemcpyAsync(y, g->pr[1], (size_t)g->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return PCPM_OK;
}

// ------------------------------------------------------------------ batches
// The captured work writes each handle's L1 changes into the batch's own
// history rows; the graph's last kernel copies them to the handles' history
// buffers through a device table of pointers, refreshed at launch when a
// handle's history has grown (moved) since the capture.
struct pcpm_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    pcpm::BatchKernels* kernels = nullptr;  // one launch per phase over all graphs, else per-handle work
    double* hist = nullptr;                 // count x iters
    double** hist_dst = nullptr;            // count device pointers
    std::vector<double*> hist_dst_host;
    int iters = 0;
    // each handle's host-side solver state right after the captured work
    struct After {
        pcpm_png* g;
        int cur, ucur, upd_valid, iters_done, dq_cur;
    };
    std::vector<After> after;
};

int pcpm_batch_create(pcpm_png* const* handles, int count, float d, int iters, uint32_t flags, pcpm_batch** out) {
    if (!handles || count < 1 || iters < 1 || bad_damping(d) || (flags & ~kAllFlags) || !out) return PCPM_EINVAL;
    std::set<const pcpm_png*> seen;
    for (int i = 0; i < count; ++i)
        if (!handles[i] || partial_shard(handles[i]) || !seen.insert(handles[i]).second)
            return PCPM_EINVAL;  // no handle twice, no destination shard
    // history room for the batch's iterations (grows outside the capture)
    for (int i = 0; i < count; ++i) RC(ensure_hist(handles[i], iters, (cudaStream_t)0));
    pcpm_batch* b = new (std::nothrow) pcpm_batch;
    if (!b) return PCPM_ENOMEM;
    b->iters = iters;
    const int nb = std::min(count, kBatchStreams);
    std::vector<cudaStream_t> streams(nb, nullptr);
    std::vector<cudaEvent_t> joins(nb, nullptr);
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    int rc = PCPM_OK;
    bool capturing = false;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess) {
            note_cuda_error(e);
            if (rc == PCPM_OK) rc = e == cudaErrorMemoryAllocation ? PCPM_ENOMEM : PCPM_ECUDA;
        }
        return rc == PCPM_OK;
    };
    if (ok(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking)))
        ok(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    if (rc == PCPM_OK && ok(pool_alloc((void**)&b->hist, (size_t)count * iters * sizeof(double), origin)) &&
        ok(pool_alloc((void**)&b->hist_dst, (size_t)count * sizeof(double*), origin))) {
        for (int i = 0; i < count; ++i) b->hist_dst_host.push_back(handles[i]->hist);
        if (ok(cudaMemcpyAsync(b->hist_dst, b->hist_dst_host.data(), (size_t)count * sizeof(double*),
                               cudaMemcpyHostToDevice, origin)))
            ok(cudaStreamSynchronize(origin));
    }
    const bool one_launch = rc == PCPM_OK && batch_kernels_ok(handles, count, flags);
    if (one_launch) rc = batch_kernels_create(handles, count, d, flags, b->hist, iters, origin, &b->kernels);
    for (int j = 0; j < nb && rc == PCPM_OK; ++j)
        if (ok(cudaStreamCreateWithFlags(&streams[j], cudaStreamNonBlocking)))
            ok(cudaEventCreateWithFlags(&joins[j], cudaEventDisableTiming));
    if (rc == PCPM_OK) capturing = ok(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
    if (rc == PCPM_OK && ok(cudaEventRecord(fork, origin)))
        for (int j = 0; j < nb && rc == PCPM_OK; ++j) ok(cudaStreamWaitEvent(streams[j], fork, 0));
    if (one_launch && rc == PCPM_OK) {
        // each (part size, cluster size) group on its own branch
        rc = batch_kernels_record(b->kernels, iters, streams.data(),
                                  std::max(1, std::min(nb, batch_kernels_groups(b->kernels))));
        const bool fused = batch_kernels_fused(b->kernels);
        for (int i = 0; i < count && rc == PCPM_OK; ++i) {
            pcpm_png* g = handles[i];
            // as pcpm_reset then `iters` iterations leave it
            b->after.push_back({g, iters & 1, fused ? g->ucur ^ (iters & 1) : g->ucur, fused ? 1 : 0, iters, 0});
        }
    } else if (rc == PCPM_OK) {
        // handle i on branch i % nb: independent graphs run side by side
        for (int i = 0; i < count && rc == PCPM_OK; ++i) {
            pcpm_png* g = handles[i];
            cudaStream_t s = streams[i % nb];
            double* const own_hist = g->hist;
            const int own_cap = g->hist_cap;
            g->hist = b->hist + (size_t)i * iters;  // the captured reductions write the batch's rows
            g->hist_cap = iters;
            rc = pcpm_reset(g, nullptr, s);
            if (rc == PCPM_OK) rc = run_iterations(g, d, iters, 0.0, flags, s, nullptr);
            g->hist = own_hist;
            g->hist_cap = own_cap;
            if (rc == PCPM_OK) {
                g->iters_done = iters;
                b->after.push_back({g, g->cur, g->ucur, g->upd_valid, g->iters_done, g->dq_cur});
            }
        }
    }
    for (int j = 0; j < nb && rc == PCPM_OK; ++j)
        if (ok(cudaEventRecord(joins[j], streams[j]))) ok(cudaStreamWaitEvent(origin, joins[j], 0));
    if (rc == PCPM_OK) rc = launch_hist_copy(b->hist, b->hist_dst, iters, count, origin);
    if (capturing) {
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(origin, &graph);
        if (rc == PCPM_OK && e == cudaSuccess) {
            b->graph = graph;
            ok(cudaGraphInstantiate(&b->exec, graph, 0));
        } else {
            if (e != cudaSuccess) note_cuda_error(e);
            if (graph) cudaGraphDestroy(graph);
            if (rc == PCPM_OK) rc = PCPM_ECUDA;
        }
    }
    cudaGetLastError();
    for (int j = 0; j < nb; ++j) {
        if (joins[j]) cudaEventDestroy(joins[j]);
        if (streams[j]) cudaStreamDestroy(streams[j]);
    }
    if (fork) cudaEventDestroy(fork);
    if (origin) {
        cudaStreamSynchronize(origin);
        cudaStreamDestroy(origin);
    }
    for (int i = 0; i < count; ++i) handles[i]->last_stream = nullptr;
    if (rc != PCPM_OK) {
        pcpm_batch_free(b);
        return rc;
    }
    *out = b;
    return PCPM_OK;
}

int pcpm_batch_launch(pcpm_batch* b, void* stream) {
    if (!b || !b->exec) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    bool moved = false;
    for (size_t i = 0; i < b->after.size(); ++i) {
        pcpm_png* g = b->after[i].g;
        RC(ensure_hist(g, b->iters, s));
        if (g->hist != b->hist_dst_host[i]) {
            b->hist_dst_host[i] = g->hist;
            moved = true;
        }
    }
    if (moved)
        CK(cudaMemcpyAsync(b->hist_dst, b->hist_dst_host.data(), b->hist_dst_host.size() * sizeof(double*),
                           cudaMemcpyHostToDevice, s));
    CK(cudaGraphLaunch(b->exec, s));
    for (const auto& a : b->after) {
        a.g->cur = a.cur;
        a.g->ucur = a.ucur;
        a.g->upd_valid = a.upd_valid;
        a.g->iters_done = a.iters_done;
        a.g->dq_cur = a.dq_cur;
        a.g->last_stream = s;
    }
    return PCPM_OK;
}

int pcpm_batch_kernel_launches(const pcpm_batch* b, int* launches) {
    if (!b || !b->graph || !launches) return PCPM_EINVAL;
    size_t count = 0;
    CK(cudaGraphGetNodes(b->graph, nullptr, &count));
    std::vector<cudaGraphNode_t> nodes(count);
    if (count) CK(cudaGraphGetNodes(b->graph, nodes.data(), &count));
    int k = 0;
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(node, &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *launches = k;
    return PCPM_OK;
}

void pcpm_batch_free(pcpm_batch* b) {
    if (!b) return;
    // the batch's buffers return to the pool only once no launch can still use them
    cudaDeviceSynchronize();
    cudaGetLastError();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    pcpm::batch_kernels_free(b->kernels);
    if (b->hist) pool_free(b->hist, nullptr);
    if (b->hist_dst) pool_free(b->hist_dst, nullptr);
    delete b;
}

int pcpm_export_weights(const pcpm_png* g, float* wbin) {
    if (!g || !wbin || !g->weighted) return PCPM_EINVAL;
    CK(cudaStreamSynchronize(g->last_stream));
    if (g->m) CK(cudaMemcpy(wbin, g->wdest, g->m * sizeof(float), cudaMemcpyDeviceToHost));
    return PCPM_OK;
}

void pcpm_free(pcpm_png* png) {
    if (!png) return;
    // the handle's memory returns to the pool only once no stream can still use it
    cudaDeviceSynchronize();
    cudaGetLastError();
    release(png);
}

int pcpm_autotune(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                  const uint32_t* part_sizes, int count, float d, int warmup, int iters, uint32_t flags,
                  void* stream, uint32_t* best_part_size, float* ms_per_iter) {
    if (!best_part_size) return PCPM_EINVAL;
    int best_opt = 0;
    return pcpm_autotune_ex(row_ptr, col_idx, n, m, part_sizes, count, nullptr, 1, d, warmup, iters, flags, stream,
                            best_part_size, &best_opt, ms_per_iter);
}

int pcpm_autotune_ex(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                     const uint32_t* part_sizes, int count, const pcpm_build_options* options, int noptions,
                     float d, int warmup, int iters, uint32_t flags, void* stream, uint32_t* best_part_size,
                     int* best_option, float* ms_per_iter) {
    if (!part_sizes || count < 1 || noptions < 1 || !best_part_size || !best_option || warmup < 0 || iters < 1 ||
        bad_damping(d) || (flags & ~kAllFlags))
        return PCPM_EINVAL;
    float best = -1.0f;
    for (int i = 0; i < count; ++i) {
        for (int j = 0; j < noptions; ++j) {
            float* slot = ms_per_iter ? ms_per_iter + (size_t)i * noptions + j : nullptr;
            if (slot) *slot = -1.0f;
            pcpm_png* g = nullptr;
            int rc = pcpm_build_ex(row_ptr, col_idx, n, m, part_sizes[i], options ? options + j : nullptr, stream, &g);
            if (rc == PCPM_EINVAL) continue;  // this partition size or tile shape does not apply
            if (rc != PCPM_OK) return rc;
            float kms[PCPM_NUM_PHASES + 1] = {};
            rc = pcpm_reset(g, nullptr, stream);
            if (rc == PCPM_OK && warmup > 0) rc = pcpm_iterate(g, d, warmup, 0.0, flags, nullptr, nullptr, stream);
            if (rc == PCPM_OK) rc = pcpm_iterate_timed(g, d, iters, flags, kms, stream);
            pcpm_free(g);
            if (rc != PCPM_OK) return rc;
            const float ms = kms[PCPM_NUM_PHASES] / (float)iters;
            if (slot) *slot = ms;
            if (best < 0.0f || ms < best) {
                best = ms;
                *best_part_size = part_sizes[i];
                *best_option = j;
            }
        }
    }
    return best < 0.0f ? PCPM_EINVAL : PCPM_OK;
}

int pcpm_release_cached_memory(void) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (int dev = 0; dev < kMaxDevices; ++dev) {
        if (!g_pools[dev]) continue;
        const cudaError_t e = cudaMemPoolTrimTo(g_pools[dev], 0);
        if (e != cudaSuccess) {
            note_cuda_error(e);
            return PCPM_ECUDA;
        }
    }
    return PCPM_OK;
}

int pcpm_png_get_info(const pcpm_png* g, pcpm_png_info* info) {
    if (!g || !info) return PCPM_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->part_size = g->q;
    info->num_partitions = g->k;
    info->num_edges = g->m;
    info->num_updates = g->ne;
    info->compression_ratio = g->ne ? (double)g->m / (double)g->ne : 0.0;
    info->device_bytes = g->device_bytes;
    info->iterations_done = g->iters_done;
    info->gather_units = g->ngunits;
    info->scatter_units = g->nsunits;
    info->gather_cluster = (uint32_t)g->cluster;
    info->fused_ok = (uint32_t)g->fused_ok;
    info->canonical_gather = (uint32_t)g->canonical_gather;
    info->gather_runs = (uint32_t)g->gather_runs;
    info->merged_adds = g->merged_adds;
    info->update_dtype = (uint32_t)g->upd_dtype;
    info->update_bytes = g->upd_bytes;
    info->gather_windows = (uint32_t)g->gather_windows;
    info->shard_part_lo = g->plo;
    info->shard_part_hi = g->phi;
    info->num_windows = g->nwin;
    return PCPM_OK;
}

int pcpm_png_export(const pcpm_png* g, uint32_t* cnt_u, uint32_t* cnt_e, uint32_t* off_u, uint32_t* off_e,
                    uint32_t* bin_u, uint32_t* bin_e, uint32_t* src_idx, uint32_t* dest_ids) {
    if (!g) return PCPM_EINVAL;
    CK(cudaStreamSynchronize(g->last_stream));
    const size_t kk = (size_t)g->k * g->k;
    std::vector<uint32_t> hb_u(g->k + 1), hb_e(g->k + 1);
    CK(cudaMemcpy(hb_u.data(), g->bin_u, (g->k + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hb_e.data(), g->bin_e, (g->k + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (cnt_u) CK(cudaMemcpy(cnt_u, g->cnt_u, kk * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (cnt_e) CK(cudaMemcpy(cnt_e, g->cnt_e, kk * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (off_u || off_e) {
        std::vector<uint32_t> seg(kk);
        if (off_u) {
            CK(cudaMemcpy(seg.data(), g->seg_u, kk * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < kk; ++i) off_u[i] = seg[i] - hb_u[i % g->k];
        }
        if (off_e) {
            CK(cudaMemcpy(seg.data(), g->seg_e, kk * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < kk; ++i) off_e[i] = seg[i] - hb_e[i % g->k];
        }
    }
    if (bin_u) std::memcpy(bin_u, hb_u.data(), (g->k + 1) * sizeof(uint32_t));
    if (bin_e) std::memcpy(bin_e, hb_e.data(), (g->k + 1) * sizeof(uint32_t));
    if (src_idx && g->ne) CK(cudaMemcpy(src_idx, g->src, g->ne * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (dest_ids && g->m) CK(cudaMemcpy(dest_ids, g->dest, g->m * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return PCPM_OK;
}

int pcpm_reset(pcpm_png* g, const float* pr_init, void* stream) {
    if (!g || partial_shard(g)) return PCPM_EINVAL;
    if (pr_init && !is_device_ptr(pr_init)) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    CK(cudaMemsetAsync(g->state, 0, sizeof(DevState), s));
    if (g->dq_err) CK(cudaMemsetAsync(g->dq_err, 0, (size_t)2 * g->n * sizeof(float), s));
    g->dq_cur = 0;
    CK(cudaMemsetAsync(g->gacc, 0, (size_t)g->n * sizeof(float), s));
    CK(cudaMemsetAsync(g->bin_done, 0, (size_t)g->k * sizeof(uint32_t), s));
    g->cur = 0;
    g->iters_done = 0;
    g->upd_valid = 0;
    RC(launch_init(g, pr_init, s));
    RC(launch_reduce(g, 0.0, -1, s));
    return PCPM_OK;
}

int pcpm_iterate(pcpm_png* g, float d, int iters, double tol, uint32_t flags, int* iters_run, double* last_residual,
                 void* stream) {
    if (!g || partial_shard(g) || iters < 0 || bad_damping(d) || (flags & ~kAllFlags)) return PCPM_EINVAL;
    return iterate_impl(g, d, iters, tol, flags, iters_run, last_residual, (cudaStream_t)stream);
}

int pcpm_iterate_timed(pcpm_png* g, float d, int iters, uint32_t flags, float* kernel_ms, void* stream) {
    if (!g || partial_shard(g) || iters < 0 || bad_damping(d) || !kernel_ms || (flags & ~kAllFlags))
        return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    std::vector<cudaEvent_t> ev((size_t)4 * iters);
    int rc = PCPM_OK;
    size_t made = 0;
    for (; made < ev.size(); ++made)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) {
            rc = PCPM_ECUDA;
            break;
        }
    if (rc == PCPM_OK && cudaMemsetAsync(&g->state->stop, 0, sizeof(int), s) != cudaSuccess) rc = PCPM_ECUDA;
    if (rc == PCPM_OK) rc = run_iterations(g, d, iters, 0.0, flags, s, &ev);
    if (rc == PCPM_OK) {
        g->iters_done += iters;
        rc = sync_state(g, s);
    }
    if (rc == PCPM_OK) {
        for (int p = 0; p <= PCPM_NUM_PHASES; ++p) kernel_ms[p] = 0.0f;
        if (iters > 0 && cudaEventElapsedTime(&kernel_ms[PCPM_NUM_PHASES], ev[0], ev[4 * iters - 1]) != cudaSuccess)
            rc = PCPM_ECUDA;
        for (int i = 0; i < iters && rc == PCPM_OK; ++i)
            for (int p = 0; p < PCPM_NUM_PHASES; ++p) {
                float ms = 0.0f;
                if (cudaEventElapsedTime(&ms, ev[4 * i + p], ev[4 * i + p + 1]) != cudaSuccess) rc = PCPM_ECUDA;
                kernel_ms[p] += ms;
            }
    }
    for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

int pcpm_ranks(const pcpm_png* g, float* pr_out, void* stream) {
    if (!g || !is_device_ptr(pr_out)) return PCPM_EINVAL;
    CK(cudaMemcpyAsync(pr_out, g->pr[g->cur], (size_t)g->n * sizeof(float), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return PCPM_OK;
}

int pcpm_residual_history(const pcpm_png* g, double* out, int max_count) {
    if (!g || !out || max_count < 0) return PCPM_EINVAL;
    CK(cudaStreamSynchronize(g->last_stream));
    const int count = std::min(max_count, std::min(g->iters_done, g->hist_cap));
    if (count > 0) CK(cudaMemcpy(out, g->hist, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost));
    return count;
}

int pcpm_pagerank(pcpm_png* g, float d, int max_iters, double tol, uint32_t flags, const float* pr_init,
                  float* pr_out, int* iters_run, double* final_residual, void* stream) {
    if (!g || partial_shard(g) || max_iters < 0 || bad_damping(d) || (flags & ~kAllFlags)) return PCPM_EINVAL;
    if (!is_device_ptr(pr_out)) return PCPM_EINVAL;
    if (pr_init && !is_device_ptr(pr_init)) return PCPM_EINVAL;
    RC(pcpm_reset(g, pr_init, stream));
    const int rc = iterate_impl(g, d, max_iters, tol, flags, iters_run, final_residual, (cudaStream_t)stream);
    if (rc < 0) return rc;
    RC(pcpm_ranks(g, pr_out, stream));
    return rc;
}

int pcpm_pagerank_host(const uint32_t* row_ptr, const uint32_t* col_idx, uint32_t n, uint64_t m,
                       uint32_t part_size, float d, int max_iters, double tol, uint32_t flags, float* pr_out,
                       int* iters_run, double* final_residual) {
    if (!row_ptr || !pr_out || (m > 0 && !col_idx) || n == 0 || n > PCPM_MAX_NODES || m > 0xFFFFFF00ull)
        return PCPM_EINVAL;
    if (max_iters < 0 || bad_damping(d) || (flags & ~kAllFlags)) return PCPM_EINVAL;
    uint32_t *d_rp = nullptr, *d_col = nullptr;
    float* d_pr = nullptr;
    pcpm_png* g = nullptr;
    int rc = PCPM_OK;
    cudaStream_t s = nullptr;
    auto fail = [&](cudaError_t e) { return e == cudaErrorMemoryAllocation ? PCPM_ENOMEM : PCPM_ECUDA; };
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = pool_alloc((void**)&d_rp, ((size_t)n + 1) * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = pool_alloc((void**)&d_col, std::max<size_t>(m, 1) * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = pool_alloc((void**)&d_pr, (size_t)n * sizeof(float), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_rp, row_ptr, ((size_t)n + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && m)
        e = cudaMemcpyAsync(d_col, col_idx, (size_t)m * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = fail(e);
    if (rc == PCPM_OK) rc = pcpm_build(d_rp, d_col, n, m, part_size, s, &g);
    if (rc == PCPM_OK) rc = pcpm_pagerank(g, d, max_iters, tol, flags, nullptr, d_pr, iters_run, final_residual, s);
    if (rc >= 0) {
        e = cudaMemcpyAsync(pr_out, d_pr, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(e);
    }
    if (s) cudaStreamSynchronize(s);
    if (g) pcpm_free(g);
    pool_free(d_rp, s);
    pool_free(d_col, s);
    pool_free(d_pr, s);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    return rc;
}

int pcpm_scatter_only(pcpm_png* g, void* stream) {
    if (!g) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    CK(cudaMemsetAsync(&g->state->stop, 0, sizeof(int), s));
    RC(launch_scatter(g, s));
    g->upd_valid = 1;
    return PCPM_OK;
}

int pcpm_export_state(const pcpm_png* g, float* pr, float* spr, void* updates, double* dangling) {
    if (!g) return PCPM_EINVAL;
    CK(cudaStreamSynchronize(g->last_stream));
    if (pr) CK(cudaMemcpy(pr, g->pr[g->cur], (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost));
    if (spr) {
        float* tmp = nullptr;
        CK(cudaMalloc((void**)&tmp, (size_t)g->n * sizeof(float)));
        int rc = launch_spr(const_cast<pcpm_png*>(g), tmp, g->last_stream);
        cudaError_t e = cudaStreamSynchronize(g->last_stream);
        if (rc == PCPM_OK && e == cudaSuccess)
            e = cudaMemcpy(spr, tmp, (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost);
        cudaFree(tmp);
        if (rc != PCPM_OK) return rc;
        if (e != cudaSuccess) return PCPM_ECUDA;
    }
    if (updates && g->ne) CK(cudaMemcpy(updates, g->upd[g->ucur], g->ne * g->upd_bytes, cudaMemcpyDeviceToHost));
    if (dangling) {
        DevState st;
        CK(cudaMemcpy(&st, g->state, sizeof(DevState), cudaMemcpyDeviceToHost));
        *dangling = st.dangling;
        const int rc = check_device_err(st);
        if (rc != PCPM_OK) return rc;
    }
    return PCPM_OK;
}

int pcpm_test_wait_limit(long long cycles) { return set_work_wait_limit(cycles); }

const char* pcpm_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda_error); }

const char* pcpm_strerror(int code) {
    switch (code) {
        case PCPM_OK: return "success";
        case PCPM_NOT_CONVERGED: return "tolerance not reached within max_iters";
        case PCPM_EINVAL: return "invalid argument";
        case PCPM_ECUDA: return "CUDA runtime error";
        case PCPM_ENOMEM: return "out of memory";
        case PCPM_ETIMEOUT: return "bounded device wait timed out";
        case PCPM_EDEVICE: return "device-side consistency check failed";
        case PCPM_EBADGRAPH: return "invalid CSR: column out of range or row not sorted";
        case PCPM_ESCRATCH: return "input larger than the fixed no-allocation scratch (PCPM_NOALLOC_MAX_NODES)";
        default: return "unknown status code";
    }
}

}  // extern "C"
