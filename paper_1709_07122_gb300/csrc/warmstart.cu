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

#include <algorithm>
#include <mutex>

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

constexpr int kTile = 256;     // nodes per training CTA (one per thread)
constexpr int kRow = H + 1;    // padded shared-memory row

// ------------------------------------------------------------- features
// Exact in-edge sums over the canonical bins, one CTA per destination bin p
// (every in-edge of a node of p lies in bin p): acc[v - p q] += val for every
// destination ID v of the bin, with val = 1 (kMode 0: the in-degree), indeg(u)
// (1) or outdeg(u) (2) of the ID's source u, or (3) the ID's update value
// vals[idx] (a per-source value already scattered into the update bins by
// Algorithm 3, so it is read in bin order instead of at random). The source
// is that of the ID's
// update: Algorithm 4's update index, the flagged IDs up to and including the
// ID minus one, found from the chunk's precomputed base and a ballot per 32
// IDs. Unsigned 32-bit shared-memory atomics; a sum that passes 2^32 sets
// kErrBounds in *err.
constexpr int kDegThreads = 512;

// L2 policies: the bins stream through once (evict first), the degree tables
// are read at random and should stay in L2 (evict last).
__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_hint(const uint32_t* p, uint64_t policy) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(policy));
    return v;
}

template <int kMode>
__global__ void __launch_bounds__(kDegThreads) bin_degree_kernel(
    const uint32_t* __restrict__ dest, const uint32_t* __restrict__ src, const uint32_t* __restrict__ bin_e,
    const uint32_t* __restrict__ chunk_base, uint32_t n, uint32_t q, const uint32_t* __restrict__ row_ptr,
    const uint32_t* __restrict__ indeg, uint32_t* __restrict__ out, int* __restrict__ err,
    const uint32_t* __restrict__ vals = nullptr) {
    extern __shared__ uint32_t acc[];
    const uint32_t p = blockIdx.x;
    const uint32_t v0 = p * q, len = min(q, n - v0);
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) acc[i] = 0u;
    __syncthreads();
    const uint32_t e0 = bin_e[p], e1 = bin_e[p + 1];
    bool over = false;
    if (e1 > e0) {
        const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const uint32_t c0 = e0 / kChunk, c1 = (e1 - 1) / kChunk;
        constexpr uint32_t kR = kChunk / 32;  // rounds of 32 IDs per chunk
        constexpr uint32_t kC = 4;            // chunks per warp step
        const uint64_t stream = l2_policy_first(), keep = l2_policy_last();
        for (uint32_t cb = c0 + kC * warp; cb <= c1; cb += kC * nw) {
            // all loads of a step are issued before any is used: the IDs,
            // then the sources of the in-bin IDs, then their degrees
            uint32_t id[kC * kR], idx[kC * kR];
#pragma unroll
            for (uint32_t i = 0; i < kC * kR; ++i) {
                const uint32_t e = (cb + i / kR) * kChunk + (i % kR) * 32 + lane;
                id[i] = (cb + i / kR <= c1 && e < e1) ? ld_hint(dest + e, stream) : 0u;
            }
#pragma unroll
            for (uint32_t ci = 0; ci < kC; ++ci) {
                uint32_t base = cb + ci <= c1 ? chunk_base[cb + ci] : 0u;
#pragma unroll
                for (uint32_t r = 0; r < kR; ++r) {
                    const uint32_t i = ci * kR + r;
                    const uint32_t fl = __ballot_sync(0xffffffffu, (id[i] & kMsb) != 0u);
                    idx[i] = base + __popc(fl & ((2u << lane) - 1u)) - 1u;
                    base += __popc(fl);
                    const uint32_t e = (cb + ci) * kChunk + r * 32 + lane;
                    if (cb + ci > c1 || e < e0 || e >= e1 || (id[i] & kIdMask) - v0 >= len)
                        id[i] = kNoHub;  // not this bin's
                }
            }
            uint32_t val[kC * kR];
            if (kMode == 3) {  // the ID's update holds the value (scattered by source partition)
#pragma unroll
                for (uint32_t i = 0; i < kC * kR; ++i) val[i] = id[i] != kNoHub ? ld_hint(vals + idx[i], stream) : 0u;
            } else if (kMode != 0) {
                uint32_t u[kC * kR];
#pragma unroll
                for (uint32_t i = 0; i < kC * kR; ++i) u[i] = id[i] != kNoHub ? ld_hint(src + idx[i], stream) : 0u;
#pragma unroll
                for (uint32_t i = 0; i < kC * kR; ++i)
                    val[i] = id[i] == kNoHub ? 0u
                             : kMode == 1    ? ld_hint(indeg + u[i], keep)
                                             : ld_hint(row_ptr + u[i] + 1, keep) - ld_hint(row_ptr + u[i], keep);
            }
#pragma unroll
            for (uint32_t i = 0; i < kC * kR; ++i) {
                if (id[i] != kNoHub) {
                    const uint32_t add = kMode == 0 ? 1u : val[i];
                    const uint32_t old = atomicAdd(&acc[(id[i] & kIdMask) - v0], add);
                    over |= old + add < old;
                }
            }
        }
    }
    if (over) atomicOr(err, kErrBounds);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) out[v0 + i] = acc[i];
}

__global__ void degree_u32_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, uint32_t* __restrict__ out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = row_ptr[v + 1] - row_ptr[v];
}

__global__ void features_kernel(const uint32_t* __restrict__ row_ptr, uint32_t n, const uint32_t* __restrict__ sums,
                                const float* __restrict__ pr1, float* __restrict__ feat) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        float* f = feat + (size_t)v * F;
        f[0] = log1pf((float)sums[v]);
        f[1] = log1pf((float)(row_ptr[v + 1] - row_ptr[v]));
        f[2] = log1pf((float)sums[(size_t)n + v]);
        f[3] = log1pf((float)sums[2 * (size_t)n + v]);
        f[4] = logf((float)n * pr1[v]);
    }
}

// FP64 moments of the feature columns, accumulated: m[0] += rows, m[1 + f] +=
// sum of x_f, m[6 + f] += sum of x_f^2.
constexpr int kMomThreads = 256;
__global__ void __launch_bounds__(kMomThreads) moments_kernel(const float* __restrict__ feat, uint32_t n,
                                                              double* __restrict__ m) {
    double s[F], s2[F];
#pragma unroll
    for (int f = 0; f < F; ++f) s[f] = s2[f] = 0.0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const double x = (double)feat[(size_t)v * F + f];
            s[f] += x;
            s2[f] += x * x;
        }
    }
    __shared__ double sh[kMomThreads / 32][2 * F];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < F; ++f) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s[f] += __shfl_down_sync(0xffffffffu, s[f], o);
            s2[f] += __shfl_down_sync(0xffffffffu, s2[f], o);
        }
        if (lane == 0) {
            sh[warp][f] = s[f];
            sh[warp][F + f] = s2[f];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * F) {
        double t = 0.0;
        for (int w = 0; w < kMomThreads / 32; ++w) t += sh[w][threadIdx.x];
        atomicAdd(&m[1 + threadIdx.x], t);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&m[0], (double)n);
}

// mu = mean, inv_sigma = 1 / max(population std, 1e-6) into params[0, 10).
__global__ void standardisation_kernel(const double* __restrict__ m, float* __restrict__ params) {
    const int f = threadIdx.x;
    if (f < F) {
        const double rows = m[0] > 0.0 ? m[0] : 1.0;
        const double mean = m[1 + f] / rows;
        const double var = fmax(m[1 + F + f] / rows - mean * mean, 0.0);
        params[OFF_MU + f] = (float)mean;
        params[OFF_IS + f] = (float)(1.0 / fmax(sqrt(var), 1e-6));
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

// ------------------------------------------------------------ inference
// One warp per tile of 16 nodes, both hidden layers on the tensor cores:
// mma.sync m16n8k16 with BF16 operands and FP32 accumulation. The weights are
// BF16 by definition (rounded once, nearest even) and stay in registers as B
// fragments for the whole kernel; the standardised inputs (K = 5, padded to
// 16) and h1 are rounded to BF16 (relative 2^-9) for the products. Biases,
// ReLU and the output dot product with w3 are FP32.
//
// Fragment layouts (PTX ISA, mma.m16n8k16, g = lane / 4, t = lane % 4):
//   A (16 x 16, row-major), 4 registers of two BF16: (row g, k 2t..2t+1),
//     (row g+8, k 2t..2t+1), (row g, k 2t+8..2t+9), (row g+8, k 2t+8..2t+9);
//   B (16 x 8), 2 registers: (k 2t..2t+1, n g), (k 2t+8..2t+9, n g);
//   C (16 x 8, FP32), 4 values: (row g, n 2t..2t+1), (row g+8, n 2t..2t+1).
// The C fragments of output columns 16k .. 16k+15 (two n-tiles) are exactly
// the A fragment of input columns 16k .. 16k+15 of the next layer, so h1 goes
// from layer 1 to layer 2 without leaving the registers.
constexpr int kPredictWarps = 8;
constexpr int kPredictGroup = 4;  // tiles per warp step: the next step's loads are in flight meanwhile

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void __launch_bounds__(kPredictWarps * 32) predict_kernel(const float* __restrict__ params,
                                                                     const float* __restrict__ feat, uint32_t n,
                                                                     float* __restrict__ out) {
    __shared__ float sb1[H], sb2[H], sw3[H];
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        sb1[i] = bf16r(params[OFF_B1 + i]);
        sb2[i] = bf16r(params[OFF_B2 + i]);
        sw3[i] = bf16r(params[OFF_W3 + i]);
    }
    const uint32_t lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // B fragments: layer 1 (K = 5 padded to 16: only k = 2t, 2t+1 < 5 are
    // nonzero), layer 2 (4 k-tiles x 8 n-tiles)
    uint32_t bw1[8], bw2[4][8][2];
#pragma unroll
    for (int jt = 0; jt < 8; ++jt) {
        const int nn = 8 * jt + g;
        const float x0 = 2 * t < F ? params[OFF_W1 + nn * F + 2 * t] : 0.0f;
        const float x1 = 2 * t + 1 < F ? params[OFF_W1 + nn * F + 2 * t + 1] : 0.0f;
        bw1[jt] = bf16x2_bits(__floats2bfloat162_rn(x0, x1));
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const float* r = params + OFF_W2 + nn * H + 16 * kt + 2 * t;
            bw2[kt][jt][0] = bf16x2_bits(__floats2bfloat162_rn(r[0], r[1]));
            bw2[kt][jt][1] = bf16x2_bits(__floats2bfloat162_rn(r[8], r[9]));
        }
    }
    float mu[2], is[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int f = 2 * t + c;
        mu[c] = f < F ? params[OFF_MU + f] : 0.0f;
        is[c] = f < F ? params[OFF_IS + f] : 0.0f;
    }
    const float b3 = bf16r(params[OFF_B3]);
    __syncthreads();
    const uint64_t warps = (uint64_t)gridDim.x * kPredictWarps;
    const uint64_t ntiles = ((uint64_t)n + 15) / 16;
    const uint64_t ngroups = (ntiles + kPredictGroup - 1) / kPredictGroup;
    // features of a group of tiles: per tile rows g and g + 8, columns 2t and
    // 2t + 1 (< F). A warp works on groups of kPredictGroup tiles and loads
    // the next group's features while it computes this one.
    auto load_x = [&](uint64_t grp, float (&x)[kPredictGroup][4]) {
#pragma unroll
        for (int tt = 0; tt < kPredictGroup; ++tt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint64_t v = (grp * kPredictGroup + tt) * 16 + g + 8 * (i >> 1);
                const int f = 2 * t + (i & 1);
                x[tt][i] = (grp < ngroups && v < n && f < F) ? __ldg(feat + v * F + f) : 0.0f;
            }
    };
    uint64_t grp = (uint64_t)blockIdx.x * kPredictWarps + (threadIdx.x >> 5);
    float xn[kPredictGroup][4];
    load_x(grp, xn);
#pragma unroll 1
    for (; grp < ngroups; grp += warps) {
        float xg[kPredictGroup][4];
#pragma unroll
        for (int tt = 0; tt < kPredictGroup; ++tt)
#pragma unroll
            for (int i = 0; i < 4; ++i) xg[tt][i] = xn[tt][i];
        load_x(grp + warps, xn);  // the next group's loads overlap this group
#pragma unroll
        for (int tt = 0; tt < kPredictGroup; ++tt) {
            const uint64_t tile = grp * kPredictGroup + tt;
            if (tile >= ntiles) break;
            const float* x = xg[tt];
            // layer 1: 8 n-tiles; A has k = 2t, 2t+1 only (k >= 8 are zero)
            const uint32_t a0 = bf16x2_bits(__floats2bfloat162_rn((x[0] - mu[0]) * is[0], (x[1] - mu[1]) * is[1]));
            const uint32_t a1 = bf16x2_bits(__floats2bfloat162_rn((x[2] - mu[0]) * is[0], (x[3] - mu[1]) * is[1]));
            uint32_t a2[4][4];
#pragma unroll
            for (int jt = 0; jt < 8; ++jt) {
                float c1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                mma_bf16_16816(c1, a0, a1, 0u, 0u, bw1[jt], 0u);
                // h1 = relu(c1 + b1) as the A fragments of layer 2
                const int col = 8 * jt + 2 * t, kt = jt >> 1, half = jt & 1;
                const float bb0 = sb1[col], bb1 = sb1[col + 1];
                a2[kt][2 * half] =
                    bf16x2_bits(__floats2bfloat162_rn(fmaxf(c1[0] + bb0, 0.0f), fmaxf(c1[1] + bb1, 0.0f)));
                a2[kt][2 * half + 1] =
                    bf16x2_bits(__floats2bfloat162_rn(fmaxf(c1[2] + bb0, 0.0f), fmaxf(c1[3] + bb1, 0.0f)));
            }
            // layer 2 and the output dot product, one n-tile at a time
            float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
            for (int jt = 0; jt < 8; ++jt) {
                float c2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int kt = 0; kt < 4; ++kt)
                    mma_bf16_16816(c2, a2[kt][0], a2[kt][1], a2[kt][2], a2[kt][3], bw2[kt][jt][0], bw2[kt][jt][1]);
                const int col = 8 * jt + 2 * t;
                const float bb0 = sb2[col], bb1 = sb2[col + 1], w0 = sw3[col], w1 = sw3[col + 1];
                y0 = fmaf(w0, fmaxf(c2[0] + bb0, 0.0f), y0);
                y0 = fmaf(w1, fmaxf(c2[1] + bb1, 0.0f), y0);
                y1 = fmaf(w0, fmaxf(c2[2] + bb0, 0.0f), y1);
                y1 = fmaf(w1, fmaxf(c2[3] + bb1, 0.0f), y1);
            }
            // the four lanes of a row group hold disjoint columns
            y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
            y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
            y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
            y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
            if (t == 0) {
                const uint64_t v = tile * 16 + g;
                if (v < n) out[v] = y0 + b3;
                if (v + 8 < n) out[v + 8] = y1 + b3;
            }
        }
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
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {  // one FP64 atomic per block
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        atomicAdd(sum, t);
    }
}

__global__ void normalise_kernel(const float* __restrict__ pred, uint32_t n, const double* __restrict__ sum,
                                 float* __restrict__ pr) {
    const float inv = (float)(1.0 / *sum);
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        pr[v] = expf(fminf(fmaxf(pred[v], -80.0f), 80.0f)) * inv;
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

namespace pcpm {
namespace {
// The three exact in-edge sums of a whole-graph handle into sums[3][n].
int degree_sums(pcpm_png* g, const uint32_t* row_ptr, uint32_t* sums, cudaStream_t s) {
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        const size_t smem = PCPM_MAX_PART_SIZE * sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(bin_degree_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bin_degree_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bin_degree_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bin_degree_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);

        attr_err = e;
    });
    if (attr_err != cudaSuccess) {
        note_cuda_error(attr_err);
        return PCPM_ECUDA;
    }
    const uint32_t n = g->n;
    const size_t smem = (size_t)g->q * sizeof(uint32_t);
    int* err = &g->state->err;
    // the solver's scalars start over (the scatter runs only while no
    // tolerance has stopped the solve)
    if (cudaMemsetAsync(g->state, 0, sizeof(DevState), s) != cudaSuccess) return PCPM_ECUDA;
    if (g->indeg) {  // the window-layout build kept the in-degrees
        if (cudaMemcpyAsync(sums, g->indeg, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return PCPM_ECUDA;
    } else {
        bin_degree_kernel<0><<<g->k, kDegThreads, smem, s>>>(g->dest, g->src, g->bin_e, g->chunk_base, n, g->q,
                                                              row_ptr, nullptr, sums, err);
    }
    if (g->upd_dtype == (int)PCPM_UPDATE_F32) {
        // Scatter indeg(u) and outdeg(u) into the two update buffers
        // (Algorithm 3 on 32-bit values, copied bit for bit), then sum them
        // from the bins in bin order instead of reading the degrees at random.
        // The solver's update bins are overwritten.
        degree_u32_kernel<<<grid_for_n(n, 256), 256, 0, s>>>(row_ptr, n, sums + 2 * (size_t)n);
        int rc = launch_status();
        if (rc == PCPM_OK) rc = launch_scatter_bits(g, sums, g->upd[0], s);
        if (rc == PCPM_OK) rc = launch_scatter_bits(g, sums + 2 * (size_t)n, g->upd[1], s);
        g->upd_valid = 0;
        if (rc != PCPM_OK) return rc;
        bin_degree_kernel<3><<<g->k, kDegThreads, smem, s>>>(g->dest, g->src, g->bin_e, g->chunk_base, n, g->q,
                                                              row_ptr, nullptr, sums + n, err,
                                                              static_cast<const uint32_t*>(g->upd[0]));
        bin_degree_kernel<3><<<g->k, kDegThreads, smem, s>>>(g->dest, g->src, g->bin_e, g->chunk_base, n, g->q,
                                                              row_ptr, nullptr, sums + 2 * (size_t)n, err,
                                                              static_cast<const uint32_t*>(g->upd[1]));
        return launch_status();
    }
    bin_degree_kernel<1><<<g->k, kDegThreads, smem, s>>>(g->dest, g->src, g->bin_e, g->chunk_base, n, g->q, row_ptr,
                                                          sums, sums + n, err);
    bin_degree_kernel<2><<<g->k, kDegThreads, smem, s>>>(g->dest, g->src, g->bin_e, g->chunk_base, n, g->q, row_ptr,
                                                          nullptr, sums + 2 * (size_t)n, err);
    return launch_status();
}

int check_state_err(pcpm_png* g, cudaStream_t s) {
    int h = 0;
    if (cudaMemcpyAsync(&h, &g->state->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PCPM_ECUDA;
    return h ? PCPM_EDEVICE : PCPM_OK;
}

bool whole_graph(const pcpm_png* g) { return g->plo == 0 && g->phi == g->k; }
}  // namespace
}  // namespace pcpm

extern "C" int pcpm_ws_degree_sums(pcpm_png* png, const uint32_t* row_ptr, uint32_t* sums, void* stream) {
    if (!png || !whole_graph(png) || !is_dev(row_ptr) || !is_dev(sums)) return PCPM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    png->last_stream = s;
    int rc = degree_sums(png, row_ptr, sums, s);
    if (rc == PCPM_OK) rc = check_state_err(png, s);
    return rc;
}

extern "C" int pcpm_ws_features(pcpm_png* png, const uint32_t* row_ptr, const uint32_t* col, float* features,
                                void* stream) {
    (void)col;
    if (!png || !whole_graph(png) || !is_dev(row_ptr) || !is_dev(features)) return PCPM_EINVAL;
    const uint32_t n = png->n;
    cudaStream_t s = (cudaStream_t)stream;
    png->last_stream = s;
    // scratch from the library's pool: the three sums (uint32) and PR_1
    uint32_t* sums = nullptr;
    if (pool_alloc((void**)&sums, (size_t)4 * n * sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return PCPM_ENOMEM;
    }
    float* pr1 = reinterpret_cast<float*>(sums + 3 * (size_t)n);
    int rc = degree_sums(png, row_ptr, sums, s);
    // overflow of a sum is reported at the end (the reset below clears the
    // handle's status, so it is read first, on the stream)
    int* h_err = nullptr;
    if (rc == PCPM_OK && cudaMallocHost((void**)&h_err, sizeof(int)) != cudaSuccess) rc = PCPM_ENOMEM;
    if (rc == PCPM_OK && cudaMemcpyAsync(h_err, &png->state->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = PCPM_ECUDA;
    // PR_1: one Eq. 1 step from the uniform start
    if (rc == PCPM_OK) rc = pcpm_reset(png, nullptr, stream);
    if (rc == PCPM_OK) rc = pcpm_iterate(png, 0.85f, 1, 0.0, PCPM_TWO_PHASE, nullptr, nullptr, stream);
    if (rc == PCPM_OK) rc = pcpm_ranks(png, pr1, stream);
    if (rc == PCPM_OK) {
        features_kernel<<<grid_for_n(n, 256), 256, 0, s>>>(row_ptr, n, sums, pr1, features);
        if (cudaGetLastError() != cudaSuccess) rc = PCPM_ECUDA;
    }
    pool_free(sums, s);
    if (rc == PCPM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = PCPM_ECUDA;
    if (rc == PCPM_OK && *h_err) rc = PCPM_EDEVICE;
    if (h_err) cudaFreeHost(h_err);
    return rc;
}

extern "C" int pcpm_ws_feature_moments(const float* features, uint32_t n, double* moments, void* stream) {
    if (!is_dev(features) || !is_dev(moments) || n == 0) return PCPM_EINVAL;
    moments_kernel<<<grid_for_n(n, kMomThreads), kMomThreads, 0, (cudaStream_t)stream>>>(features, n, moments);
    return cudaGetLastError() == cudaSuccess ? PCPM_OK : PCPM_ECUDA;
}

extern "C" int pcpm_ws_standardisation(const double* moments, float* params, void* stream) {
    if (!is_dev(moments) || !is_dev(params)) return PCPM_EINVAL;
    standardisation_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(moments, params);
    return cudaGetLastError() == cudaSuccess ? PCPM_OK : PCPM_ECUDA;
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
    const uint64_t tiles = ((uint64_t)n + 15) / 16;
    const uint64_t groups = (tiles + kPredictGroup - 1) / kPredictGroup;
    const int blocks = (int)std::min<uint64_t>((groups + kPredictWarps - 1) / kPredictWarps, 152ull * 2);
    predict_kernel<<<blocks, kPredictWarps * 32, 0, (cudaStream_t)stream>>>(params, features, n, out);
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
    if (pool_alloc((void**)&sum, sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return PCPM_ENOMEM;
    }
    int rc = PCPM_OK;
    if (cudaMemsetAsync(sum, 0, sizeof(double), s) != cudaSuccess) rc = PCPM_ECUDA;
    if (rc == PCPM_OK) {
        exp_sum_kernel<<<std::min(grid_for_n(n, 256), 152 * 4), 256, 0, s>>>(pred, n, sum);
        normalise_kernel<<<std::min(grid_for_n(n, 256), 152 * 8), 256, 0, s>>>(pred, n, sum, pr);
        if (cudaGetLastError() != cudaSuccess) rc = PCPM_ECUDA;
    }
    pool_free(sum, s);
    return rc;
}
