// pcpm_noalloc.cu - an entry point that allocates no memory.
//
// pcpm_rank_stats_noalloc computes the two FP64 sums the solver reduces every
// iteration - the L1 change sum_v |x(v) - y(v)| and the dangling mass
// sum over nodes without out-edges of x(v) - for rank vectors the caller
// owns. It is the reduction of pcpm_iter.cu with its per-block partial sums
// kept in a fixed array compiled into this library instead of memory
// allocated per handle, for callers that cannot call cudaMalloc (for example
// code running inside a memory pool or allocator hook that must not re-enter
// the allocator, or a process whose device memory is fully reserved up
// front).
#include <mutex>

#include "pcpm_internal.cuh"

namespace pcpm {
namespace {

constexpr int kNoAllocThreads = 512;
constexpr uint32_t kNoAllocNodesPerBlock = 4096;  // 8 nodes per thread
constexpr int kMaxDevices = 64;

// Per-block (L1 change, dangling mass) partial sums. Every GPU that loads the
// library holds these PCPM_NOALLOC_MAX_BLOCKS * 16 bytes (1 MiB) until exit.
static __device__ __align__(256) double g_noalloc_partials[2 * PCPM_NOALLOC_MAX_BLOCKS];

__device__ __forceinline__ void block_sum2_na(double& a, double& b) {
    __shared__ double sa[kNoAllocThreads / 32], sb[kNoAllocThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        a = lane < kNoAllocThreads / 32 ? sa[lane] : 0.0;
        b = lane < kNoAllocThreads / 32 ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Block b covers nodes [b * kNoAllocNodesPerBlock, +kNoAllocNodesPerBlock) and
// writes its own two slots, so every slot a call reads was written by it.
__global__ void __launch_bounds__(kNoAllocThreads) stats_partials_kernel(const float* __restrict__ x,
                                                                         const float* __restrict__ y,
                                                                         const uint32_t* __restrict__ row_ptr,
                                                                         uint32_t n, double* __restrict__ partials) {
    const uint64_t lo = (uint64_t)blockIdx.x * kNoAllocNodesPerBlock;
    const uint64_t hi = lo + kNoAllocNodesPerBlock < n ? lo + kNoAllocNodesPerBlock : n;
    double l1 = 0.0, dang = 0.0;
    for (uint64_t v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const float xv = x[v];
        l1 += fabs((double)xv - (double)y[v]);
        if (row_ptr[v + 1] == row_ptr[v]) dang += (double)xv;
    }
    block_sum2_na(l1, dang);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = l1;
        partials[2 * blockIdx.x + 1] = dang;
    }
}

// Sums the partials in a fixed order (deterministic) into out[0..1].
__global__ void __launch_bounds__(kNoAllocThreads) stats_final_kernel(const double* __restrict__ partials, int count,
                                                                      double* __restrict__ out) {
    double l1 = 0.0, dang = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        l1 += partials[2 * i];
        dang += partials[2 * i + 1];
    }
    block_sum2_na(l1, dang);
    if (threadIdx.x == 0) {
        out[0] = l1;
        out[1] = dang;
    }
}

std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};

// Device address of the partials array on the current device, looked up
// once per device (the symbol's host-side name is not a device address).
int partials_address(double** out) {
    int dev = 0;
    if (const cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) {
        note_cuda_error(e);
        return PCPM_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        note_cuda_error(cudaErrorInvalidDevice);
        return PCPM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            note_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            return PCPM_ECUDA;
        }
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return PCPM_OK;
}

// Launches f<<<blocks, kNoAllocThreads, 0, s>>>(args...) and returns this
// launch's own status: an error some earlier call left pending is neither
// cleared nor blamed on this one.
template <class... Params, class... Args>
int launch(void (*f)(Params...), unsigned blocks, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kNoAllocThreads);
    cfg.stream = s;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, f, args...);
    if (e == cudaSuccess) return PCPM_OK;
    note_cuda_error(e);
    return PCPM_ECUDA;
}

}  // namespace
}  // namespace pcpm

extern "C" int pcpm_rank_stats_noalloc(const float* x, const float* y, const uint32_t* row_ptr, uint32_t n,
                                       double* out, void* stream) {
    if (!x || !y || !row_ptr || !out || n == 0) return PCPM_EINVAL;
    const uint64_t blocks = ((uint64_t)n + pcpm::kNoAllocNodesPerBlock - 1) / pcpm::kNoAllocNodesPerBlock;
    if (blocks > PCPM_NOALLOC_MAX_BLOCKS) return PCPM_ESCRATCH;
    double* partials = nullptr;
    int rc = pcpm::partials_address(&partials);
    if (rc != PCPM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = pcpm::launch(pcpm::stats_partials_kernel, (unsigned)blocks, s, x, y, row_ptr, n, partials);
    if (rc != PCPM_OK) return rc;
    return pcpm::launch(pcpm::stats_final_kernel, 1u, s, (const double*)partials, (int)blocks, out);
}
