// warmstart.cu - learned warm start: node features, a 5-64-64-1 network's
// inference and training kernels, Adam, and the initial rank vector. The
// degree features are in-edge sums computed as PCPM passes over the handle
// (scatter and gather of Algorithms 3 and 4, applied with d = 1).
//
// Not in the paper: power iteration (Eq. 1) starts from 1/n there. Here a
// per-node network predicts log(n * PR*(v)) and the iteration may start from
// the softmax of the prediction; it reaches the same fixed point.
//
// Training works on tiles of kTile nodes per CTA. Each thread runs one node's
// forward pass, keeping h1 and h2 in shared memory rows padded to kRow floats
// (distinct banks for the per-thread row accesses); the weight gradients are
// then tile-wide sums (dW2 = dz2^T h1 over the tile, dW1 = dz1^T x^) that the
// CTA's threads split by output entry and add to the global gradient once.
#include <cuda_bf16.h>

#include "pcpm_internal.cuh"
#include "pcpm_warmstart.h"

namespace pcpm {
namespace {

constexpr int F = PCPM_WS_FEATURES;
constexpr int H = PCPM_WS_HIDDEN;
constexpr int P = PCPM_WS_PARAMS;
constexpr int OFF_MU = 0, OFF_IS = F, OFF_W1 = 2 * F, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H,
              OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H;
static_assert(OFF_B3 + 1 == P, "parameter layout");
static_assert(OFF_W1 == PCPM_WS_TRAINABLE_OFFSET, "parameter layout");

constexpr int kPredictThreads = 256;
constexpr int kTile = 256;     // nodes per training CTA (one per thread)
constexpr int kRow = H + 1;    // padded shared-memory row

// ------------------------------------------------------------- features
// The vectors whose in-edge sums give the degree features: the PCPM pass of
// pull_sum divides by outdeg(u), so x(u) * outdeg(u) yields sum_u x(u) over
// in-edges: x = 1 (in-degree), x = indeg(u), x = outdeg(u).
__global__ void degree_vector_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, const float* __restrict__ x,
                                     int power, float* __restrict__ out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float dout = (float)(row_ptr[v + 1] - row_ptr[v]);
        out[v] = x ? x[v] * dout : (power == 2 ? dout * dout : dout);
    }
}

__global__ void features_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, const float* __restrict__ indeg,
                                const float* __restrict__ s_in, const float* __restrict__ s_out,
                                const float* __restrict__ pr1, float* __restrict__ feat) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        float* f = feat + (size_t)v * F;
        f[0] = log1pf(indeg[v]);
        f[1] = log1pf((float)(row_ptr[v + 1] - row_ptr[v]));
        f[2] = log1pf(s_in[v]);
        f[3] = log1pf(s_out[v]);
        f[4] = logf((float)n * pr1[v]);
    }
}

__global__ void targets_kernel(const float* __restrict__ pr, uint32_t n, float* __restrict__ target) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        target[v] = (float)log((double)n * (double)pr[v]);
}

// ------------------------------------------------------------- network
// Loads the parameters into shared memory; with kBf16, W1..b3 rounded to
// bfloat16 (nearest even) and widened back.
template <bool kBf16>
__device__ void load_params(const float* __restrict__ params, float* w) {
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float x = params[i];
        w[i] = (kBf16 && i >= OFF_W1) ? __bfloat162float(__float2bfloat16_rn(x)) : x;
    }
    __syncthreads();
}

__device__ __forceinline__ void standardise(const float* __restrict__ feat, uint64_t v, const float* w, float* xh) {
#pragma unroll
    for (int f = 0; f < F; ++f) xh[f] = (feat[v * F + f] - w[OFF_MU + f]) * w[OFF_IS + f];
}

__device__ __forceinline__ void layer1(const float* w, const float* xh, float* h1) {
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float s = w[OFF_B1 + j];
#pragma unroll
        for (int f = 0; f < F; ++f) s = fmaf(w[OFF_W1 + j * F + f], xh[f], s);
        h1[j] = fmaxf(s, 0.0f);
    }
}

// Inference keeps W2 at a 16-byte-aligned shared offset (the flat layout puts
// it at float 394): entries from W2 on move up by kShift floats.
constexpr int kShift = 2;
static_assert((OFF_W2 + kShift) % 4 == 0, "W2 rows must start on 16-byte boundaries");

__global__ void __launch_bounds__(kPredictThreads) predict_kernel(const float* __restrict__ params,
                                                                  const float* __restrict__ feat, uint32_t n,
                                                                  float* __restrict__ out) {
    __shared__ __align__(16) float w[P + kShift];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float x = params[i];
        w[i < OFF_W2 ? i : i + kShift] = i >= OFF_W1 ? __bfloat162float(__float2bfloat16_rn(x)) : x;
    }
    __syncthreads();
    const float* w2 = w + OFF_W2 + kShift;
    const float* b2 = w2 + H * H;
    const float* w3 = b2 + H;
    const float b3 = w3[H];
    // two nodes per thread: every 16-byte weight load feeds eight FMAs
    const uint64_t stride = 2ull * gridDim.x * blockDim.x;
#pragma unroll 1
    for (uint64_t v0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) * 2; v0 < n; v0 += stride) {
        asm volatile("" ::: "memory");  // weights stay in shared memory, not in registers across nodes
        const bool two = v0 + 1 < n;
        float xa[F], xb[F], ha[H], hb[H];
        standardise(feat, v0, w, xa);
        if (two) standardise(feat, v0 + 1, w, xb);
        else {
#pragma unroll
            for (int f = 0; f < F; ++f) xb[f] = 0.0f;
        }
        layer1(w, xa, ha);
        layer1(w, xb, hb);
        float ya = b3, yb = b3;
#pragma unroll 1
        for (int j = 0; j < H; ++j) {
            float sa = b2[j], sb = sa;
            const float4* row = reinterpret_cast<const float4*>(w2 + j * H);
#pragma unroll
            for (int i4 = 0; i4 < H / 4; ++i4) {
                const float4 q = row[i4];
                sa = fmaf(q.x, ha[4 * i4], sa);
                sa = fmaf(q.y, ha[4 * i4 + 1], sa);
                sa = fmaf(q.z, ha[4 * i4 + 2], sa);
                sa = fmaf(q.w, ha[4 * i4 + 3], sa);
                sb = fmaf(q.x, hb[4 * i4], sb);
                sb = fmaf(q.y, hb[4 * i4 + 1], sb);
                sb = fmaf(q.z, hb[4 * i4 + 2], sb);
                sb = fmaf(q.w, hb[4 * i4 + 3], sb);
            }
            ya = fmaf(w3[j], fmaxf(sa, 0.0f), ya);
            yb = fmaf(w3[j], fmaxf(sb, 0.0f), yb);
        }
        out[v0] = ya;
        if (two) out[v0 + 1] = yb;
    }
}

// Forward and backward over tiles of kTile nodes; adds the tile's gradient
// to grad and its squared-error sum to loss.
__global__ void __launch_bounds__(kTile) loss_grad_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ feat,
                                                          const float* __restrict__ target, uint32_t n,
                                                          float inv_n, float* __restrict__ grad,
                                                          double* __restrict__ loss) {
    extern __shared__ __align__(16) float sm[];
    float* w = sm;                        // P
    float* s_h1 = w + P;                  // kTile x kRow: h1, then dz1
    float* s_h2 = s_h1 + kTile * kRow;    // kTile x kRow: h2, then dz2
    float* s_xh = s_h2 + kTile * kRow;    // kTile x F
    float* s_dy = s_xh + kTile * F;       // kTile
    __shared__ double red[kTile / 32];
    load_params<false>(params, w);
    const int t = threadIdx.x;
    for (uint64_t base = (uint64_t)blockIdx.x * kTile; base < n; base += (uint64_t)gridDim.x * kTile) {
        const uint64_t v = base + t;
        const bool live = v < n;
        // forward: one node per thread
        float xh[F], h1[H];
        if (live) {
            standardise(feat, v, w, xh);
        } else {
#pragma unroll
            for (int f = 0; f < F; ++f) xh[f] = 0.0f;
        }
        layer1(w, xh, h1);
        float y = w[OFF_B3];
#pragma unroll 1
        for (int j = 0; j < H; ++j) {
            float s = w[OFF_B2 + j];
#pragma unroll
            for (int i = 0; i < H; ++i) s = fmaf(w[OFF_W2 + j * H + i], h1[i], s);
            const float h2 = fmaxf(s, 0.0f);
            s_h2[t * kRow + j] = h2;
            y = fmaf(w[OFF_W3 + j], h2, y);
        }
#pragma unroll
        for (int i = 0; i < H; ++i) s_h1[t * kRow + i] = h1[i];
#pragma unroll
        for (int f = 0; f < F; ++f) s_xh[t * F + f] = xh[f];
        const float r = live ? y - target[v] : 0.0f;
        const float dy = 2.0f * r * inv_n;
        s_dy[t] = dy;
        double sq = (double)r * (double)r;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
        if ((t & 31) == 0) red[t >> 5] = sq;
        __syncthreads();
        if (t == 0) {
            double s = 0.0;
            for (int i = 0; i < kTile / 32; ++i) s += red[i];
            atomicAdd(loss, s * (double)inv_n);
        }
        // output layer: dw3[j] = sum_t dy h2[t][j], db3 = sum_t dy
        if (t < H) {
            float s = 0.0f;
            for (int u = 0; u < kTile; ++u) s = fmaf(s_dy[u], s_h2[u * kRow + t], s);
            atomicAdd(&grad[OFF_W3 + t], s);
        } else if (t == H) {
            float s = 0.0f;
            for (int u = 0; u < kTile; ++u) s += s_dy[u];
            atomicAdd(&grad[OFF_B3], s);
        }
        __syncthreads();
        // dz2 = dy * w3 * [h2 > 0], in place of h2 (own row)
        for (int j = 0; j < H; ++j) {
            const float h2 = s_h2[t * kRow + j];
            s_h2[t * kRow + j] = h2 > 0.0f ? dy * w[OFF_W3 + j] : 0.0f;
        }
        __syncthreads();
        // dW2[j][i] = sum_t dz2[t][j] h1[t][i]; db2[j] = sum_t dz2[t][j]
        for (int o = t; o < H * H + H; o += kTile) {
            float s = 0.0f;
            if (o < H * H) {
                const int j = o / H, i = o % H;
                for (int u = 0; u < kTile; ++u) s = fmaf(s_h2[u * kRow + j], s_h1[u * kRow + i], s);
                atomicAdd(&grad[OFF_W2 + o], s);
            } else {
                const int j = o - H * H;
                for (int u = 0; u < kTile; ++u) s += s_h2[u * kRow + j];
                atomicAdd(&grad[OFF_B2 + j], s);
            }
        }
        __syncthreads();
        // dz1[i] = (sum_j W2[j][i] dz2[j]) * [h1[i] > 0], in place of h1 (own row)
        {
            float dz1[H];
#pragma unroll
            for (int i = 0; i < H; ++i) dz1[i] = 0.0f;
#pragma unroll 1
            for (int j = 0; j < H; ++j) {
                const float g = s_h2[t * kRow + j];
#pragma unroll
                for (int i = 0; i < H; ++i) dz1[i] = fmaf(w[OFF_W2 + j * H + i], g, dz1[i]);
            }
#pragma unroll
            for (int i = 0; i < H; ++i) s_h1[t * kRow + i] = h1[i] > 0.0f ? dz1[i] : 0.0f;
        }
        __syncthreads();
        // dW1[j][f] = sum_t dz1[t][j] x^[t][f]; db1[j] = sum_t dz1[t][j]
        for (int o = t; o < H * F + H; o += kTile) {
            float s = 0.0f;
            if (o < H * F) {
                const int j = o / F, f = o % F;
                for (int u = 0; u < kTile; ++u) s = fmaf(s_h1[u * kRow + j], s_xh[u * F + f], s);
                atomicAdd(&grad[OFF_W1 + o], s);
            } else {
                const int j = o - H * F;
                for (int u = 0; u < kTile; ++u) s += s_h1[u * kRow + j];
                atomicAdd(&grad[OFF_B1 + j], s);
            }
        }
        __syncthreads();
    }
}

__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr, float beta1, float beta2, float eps, float c1,
                            float c2) {
    for (int i = OFF_W1 + blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = beta1 * m[i] + (1.0f - beta1) * g;
        const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
        m[i] = mi;
        v[i] = vi;
        params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ------------------------------------------------------------ warm start
__global__ void exp_sum_kernel(const float* __restrict__ pred, uint32_t n, double* __restrict__ sum) {
    double s = 0.0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        s += (double)expf(fminf(fmaxf(pred[v], -80.0f), 80.0f));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, s);
}

__global__ void normalise_kernel(const float* __restrict__ pred, uint32_t n, const double* __restrict__ sum,
                                 float* __restrict__ pr) {
    const double inv = 1.0 / *sum;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        pr[v] = (float)((double)expf(fminf(fmaxf(pred[v], -80.0f), 80.0f)) * inv);
}

int grid_for_n(uint64_t work, int threads) {
    return (int)std::min<uint64_t>(std::max<uint64_t>((work + threads - 1) / threads, 1), 152ull * 32);
}

bool is_dev(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t train_smem() { return (size_t)(P + 2 * kTile * kRow + kTile * F + kTile) * sizeof(float); }

}  // namespace
}  // namespace pcpm

using namespace pcpm;

extern "C" int pcpm_ws_features(pcpm_png* png, const uint32_t* row_ptr, const uint32_t* col, float* features,
                                void* stream) {
    pcpm_png_info info;
    if (!png || pcpm_png_get_info(png, &info) != PCPM_OK) return PCPM_EINVAL;
    if (!is_dev(row_ptr) || !is_dev(features) || (info.num_edges > 0 && !is_dev(col))) return PCPM_EINVAL;
    const uint32_t n = info.n;
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: a staging vector and four sums (in-degree, the two 2-hop sums, PR_1)
    float* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, (size_t)5 * n * sizeof(float), s) != cudaSuccess) {
        cudaGetLastError();
        return PCPM_ENOMEM;
    }
    float *x = buf, *indeg = buf + (size_t)n, *s_in = buf + 2 * (size_t)n, *s_out = buf + 3 * (size_t)n,
          *pr1 = buf + 4 * (size_t)n;
    const int grid = grid_for_n(n, 256);
    int rc = PCPM_OK;
    // in-degree: sum of 1 over in-edges
    degree_vector_kernel<<<grid, 256, 0, s>>>(row_ptr, n, nullptr, 1, x);
    if (rc == PCPM_OK) rc = pull_sum(png, x, indeg, s);
    // sum of indeg(u) over in-edges
    if (rc == PCPM_OK) degree_vector_kernel<<<grid, 256, 0, s>>>(row_ptr, n, indeg, 1, x);
    if (rc == PCPM_OK) rc = pull_sum(png, x, s_in, s);
    // sum of outdeg(u) over in-edges
    if (rc == PCPM_OK) degree_vector_kernel<<<grid, 256, 0, s>>>(row_ptr, n, nullptr, 2, x);
    if (rc == PCPM_OK) rc = pull_sum(png, x, s_out, s);
    // PR_1: one Eq. 1 step from the uniform start
    if (rc == PCPM_OK) rc = pcpm_reset(png, nullptr, stream);
    if (rc == PCPM_OK) rc = pcpm_iterate(png, 0.85f, 1, 0.0, PCPM_TWO_PHASE, nullptr, nullptr, stream);
    if (rc == PCPM_OK) rc = pcpm_ranks(png, pr1, stream);
    if (rc == PCPM_OK) {
        features_kernel<<<grid, 256, 0, s>>>(row_ptr, n, indeg, s_in, s_out, pr1, features);
        if (cudaGetLastError() != cudaSuccess) rc = PCPM_ECUDA;
    }
    cudaFreeAsync(buf, s);
    if (rc == PCPM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = PCPM_ECUDA;
    return rc;
}

extern "C" int pcpm_ws_targets(const float* pr, uint32_t n, float* target, void* stream) {
    if (!pr || !target) return PCPM_EINVAL;
    if (n == 0) return PCPM_OK;
    targets_kernel<<<grid_for_n(n, 256), 256, 0, (cudaStream_t)stream>>>(pr, n, target);
    return cudaGetLastError() == cudaSuccess ? PCPM_OK : PCPM_ECUDA;
}

extern "C" int pcpm_ws_predict(const float* params, const float* features, uint32_t n, float* out, void* stream) {
    if (!params || !features || !out) return PCPM_EINVAL;
    if (n == 0) return PCPM_OK;
    predict_kernel<<<grid_for_n(n, kPredictThreads), kPredictThreads, 0, (cudaStream_t)stream>>>(params, features,
                                                                                                  n, out);
    return cudaGetLastError() == cudaSuccess ? PCPM_OK : PCPM_ECUDA;
}

extern "C" int pcpm_ws_loss_grad(const float* params, const float* features, const float* target, uint32_t n,
                                 float* grad, double* loss, void* stream) {
    if (!params || !features || !target || !grad || !loss || n == 0) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(loss_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem()) !=
            cudaSuccess)
            return PCPM_ECUDA;
        attr_set = true;
    }
    if (cudaMemsetAsync(grad, 0, P * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess)
        return PCPM_ECUDA;
    const int blocks = (int)std::min<uint64_t>(((uint64_t)n + kTile - 1) / kTile, 152ull * 8);
    loss_grad_kernel<<<blocks, kTile, train_smem(), s>>>(params, features, target, n, 1.0f / (float)n, grad, loss);
    return cudaGetLastError() == cudaSuccess ? PCPM_OK : PCPM_ECUDA;
}

extern "C" int pcpm_ws_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                            float beta2, float eps, void* stream) {
    if (!params || !grad || !m || !v || step < 1) return PCPM_EINVAL;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    adam_kernel<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, lr, beta1, beta2, eps, c1,
                                                                    c2);
    return cudaGetLastError() == cudaSuccess ? PCPM_OK : PCPM_ECUDA;
}

extern "C" int pcpm_ws_init_ranks(const float* pred, uint32_t n, float* pr, void* stream) {
    if (!pred || !pr || n == 0) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double* sum = nullptr;
    if (cudaMallocAsync((void**)&sum, sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return PCPM_ENOMEM;
    }
    int rc = PCPM_OK;
    if (cudaMemsetAsync(sum, 0, sizeof(double), s) != cudaSuccess) rc = PCPM_ECUDA;
    if (rc == PCPM_OK) {
        exp_sum_kernel<<<grid_for_n(n, 256), 256, 0, s>>>(pred, n, sum);
        normalise_kernel<<<grid_for_n(n, 256), 256, 0, s>>>(pred, n, sum, pr);
        if (cudaGetLastError() != cudaSuccess) rc = PCPM_ECUDA;
    }
    cudaFreeAsync(sum, s);
    if (rc == PCPM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = PCPM_ECUDA;
    return rc;
}
