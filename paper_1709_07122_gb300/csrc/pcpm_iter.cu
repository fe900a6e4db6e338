// pcpm_iter.cu - one PCPM PageRank iteration on sm_103a.
//
// Scatter (Algorithm 3 over the PNG): one CTA per source partition p, largest
// first. The partition's slice of SPR = PR/outdeg (q floats) is staged in shared
// memory - the paper's cached vertex data of p - and, for every destination
// partition p', the segment of update_bins[p'] that p owns (static offsets,
// Sec. 3.1) is filled: update[t] = SPR[src[t]]. The k segments are walked as one
// flattened range of 4-entry groups so every thread has equal work; source IDs
// stream in and updates stream out as 16-byte vectors, several groups in flight
// per thread.
//
// Gather + apply (Algorithm 4 and the apply loop of Algorithm 2): a thread-block
// cluster of S CTAs per destination partition p', largest bins first. Every CTA
// holds a full q-float accumulator in shared memory and takes a contiguous 1/S
// of the bin's chunks, split again into one contiguous run per warp. Each warp
// streams its chunks with cp.async.bulk (TMA, non-tensor form) into a private
// kGatherStages-deep ring: the chunk's kChunk destination IDs and the slice of
// the update bin they refer to, both landing on one mbarrier; the per-chunk
// update bases come from the builder. Branch avoidance (Algorithm 4) becomes
// warp arithmetic: the update of an ID is the chunk's base plus the inclusive
// count of flagged IDs before it, from ballots. The bin's two largest in-degree
// destinations are summed in registers instead of contended atomics. Then the
// cluster synchronises, each CTA adds the S partial sums of its 1/S of the
// partition over distributed shared memory and applies
//   PR'(v) = (1-d)/n + d*(acc(v) + D/n)
// writing PR' and FP64 partial sums of |PR' - PR| and of PR' over dangling
// nodes. In the fused form the same cluster then assembles SPR' = PR'/outdeg for
// the whole partition in shared memory and scatters it into the other update
// buffer for the next iteration: gather, apply and the next scatter of one
// partition in one launch, without writing SPR to memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "pcpm_internal.cuh"

namespace pcpm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Nodes per thread in flight in the apply loop.
constexpr int kApplyIlp = 8;
// Groups of four nodes per thread in flight in the vectorised apply (and in
// the apply of a bin cut into several units, done by one CTA).
constexpr int kApplyVec = 4;
constexpr int kApplyVecCut = 2;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ------------------------------------------------------------ mbarrier / TMA
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later bulk copies (async proxy) into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// L2 eviction-priority policies for bulk copies.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Bulk copy global -> shared completing on an mbarrier, with an L2 eviction
// policy. Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                               uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Prefetch [p, p + n floats) into L2 (whole 16-byte blocks inside the range).
__device__ __forceinline__ void prefetch_l2(const float* p, uint32_t n, uint64_t policy) {
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = (uintptr_t)(p + n) & ~(uintptr_t)15;
    if (e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(a), "r"((uint32_t)(e - a)),
                     "l"(policy)
                     : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the given phase parity, for at most kWaitLimitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitLimitCycles) return false;
    return true;
}

// The bound of the window gather's waits for work (a stage to fill, a
// window to consume), in SM cycles: kWaitLimitCycles unless a test shortens it
// (pcpm_test_wait_limit); negative: give up without waiting. Waits that drain
// copies still in flight always keep kWaitLimitCycles, so no copy can land
// after its CTA has exited.
__device__ long long g_work_wait_limit = kWaitLimitCycles;

__device__ __forceinline__ bool mbar_wait_work(uint64_t* bar, uint32_t parity, long long limit) {
    if (limit < 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// ------------------------------------------------------------------- cluster
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of `p` (this CTA's shared memory) in the shared memory of CTA `rank`.
__device__ __forceinline__ uint32_t map_rank(const void* p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_addr(p)), "r"(rank));
    return a;
}

__device__ __forceinline__ float ld_cluster_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ float4 ld_cluster_f32x4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_f32x4(uint32_t addr, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// Copies cnt floats from this CTA's src to dst in the shared memory of CTA
// `target` (both 16-byte aligned): distributed-shared-memory stores, which
// need no round trip, where a remote load would wait for one.
__device__ __forceinline__ void push_range(const float* src, float* dst, uint32_t cnt, uint32_t target) {
    const uint32_t c4 = cnt >> 2;
    for (uint32_t i = threadIdx.x; i < c4; i += blockDim.x)
        st_cluster_f32x4(map_rank(dst + 4 * i, target), reinterpret_cast<const float4*>(src)[i]);
    for (uint32_t i = (c4 << 2) + threadIdx.x; i < cnt; i += blockDim.x) st_cluster_f32(map_rank(dst + i, target), src[i]);
}

// ------------------------------------------------------------ global memory
__device__ __forceinline__ void st_stream_f4(float* p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Vector FP32 reduction into global memory (p 16-byte aligned).
__device__ __forceinline__ void red_add_v4(float* p, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void st_stream_u2(void* p, uint32_t a, uint32_t b) {
    asm volatile("st.global.cs.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b) : "memory");
}

// ------------------------------------------------------------ update bins
// One update as stored (PCPM_UPDATE_*): the FP32 SPR value, IEEE binary16 of
// SPR * 2^15 (saturating at the largest finite half) or bfloat16 of SPR, both
// rounded to nearest even. The gather adds the stored values in FP32 and
// multiplies the sum by acc_scale.
template <int kUpd>
struct Upd;
template <>
struct Upd<kUpdF32> {
    using T = float;
    static constexpr float acc_scale = 1.0f;
    __device__ static float load(const T* p, uint32_t i) { return p[i]; }
    __device__ static T from(float x) { return x; }
    // the value whose from() is q, in the units from() takes
    __device__ static float back(T q) { return q; }
    __device__ static void store4(T* p, uint32_t e, float a, float b, float c, float d) {
        st_stream_f4(p + e, make_float4(a, b, c, d));
    }
};
template <>
struct Upd<kUpdF16> {
    using T = __half;
    static constexpr float acc_scale = 1.0f / kF16Scale;
    __device__ static float load(const T* p, uint32_t i) { return __half2float(p[i]); }
    __device__ static T from(float x) { return __float2half_rn(fmaxf(fminf(x * kF16Scale, 65504.0f), -65504.0f)); }
    __device__ static float back(T q) { return __half2float(q) * (1.0f / kF16Scale); }
    __device__ static void store4(T* p, uint32_t e, float a, float b, float c, float d) {
        st_stream_u2(p + e, (uint32_t)__half_as_ushort(from(a)) | ((uint32_t)__half_as_ushort(from(b)) << 16),
                     (uint32_t)__half_as_ushort(from(c)) | ((uint32_t)__half_as_ushort(from(d)) << 16));
    }
};
template <>
struct Upd<kUpdBF16> {
    using T = __nv_bfloat16;
    static constexpr float acc_scale = 1.0f;
    __device__ static float load(const T* p, uint32_t i) { return __bfloat162float(p[i]); }
    __device__ static T from(float x) { return __float2bfloat16_rn(x); }
    __device__ static float back(T q) { return __bfloat162float(q); }
    __device__ static void store4(T* p, uint32_t e, float a, float b, float c, float d) {
        st_stream_u2(p + e,
                     (uint32_t)__bfloat16_as_ushort(from(a)) | ((uint32_t)__bfloat16_as_ushort(from(b)) << 16),
                     (uint32_t)__bfloat16_as_ushort(from(c)) | ((uint32_t)__bfloat16_as_ushort(from(d)) << 16));
    }
};

// Delta iterations (PCPM_DELTA): the bins carry the change of SPR since the
// previous iteration, bounded by the last L1 change r (|dSPR(u)| <=
// |dPR(u)| <= r). FP16 bins rescale it by 2^E, E = floor(log2(65504 / r)),
// so the largest possible change maps to the top of the FP16 range and the
// shrinking changes keep their relative precision; FP32 and BF16 bins need no
// scale. delta_stage_scale multiplies the change before Upd::from (which
// itself multiplies FP16 values by 2^15); the gather's sums are multiplied by
// delta_acc_scale (instead of Upd::acc_scale).
template <int kUpd>
__device__ __forceinline__ int delta_exponent(const DevState* st) {
    if (kUpd != kUpdF16) return 0;
    const double r = st->residual;
    if (!(r > 0.0)) return 100;  // no change to carry
    return max(-100, min(100, (int)floor(log2(65504.0 / r))));
}
template <int kUpd>
__device__ __forceinline__ float delta_stage_scale(const DevState* st) {
    return kUpd == kUpdF16 ? ldexpf(1.0f, delta_exponent<kUpd>(st) - PCPM_F16_SCALE_LOG2) : 1.0f;
}
template <int kUpd>
__device__ __forceinline__ float delta_acc_scale(const DevState* st) {
    return kUpd == kUpdF16 ? ldexpf(1.0f, -delta_exponent<kUpd>(st)) : 1.0f;
}

// Deterministic block sum of two doubles; result valid in thread 0. `scratch`
// is 2 * kThreads / 32 doubles of shared memory.
template <int kThreads>
__device__ __forceinline__ void block_sum2(double& a, double& b, double* scratch) {
    double* sa = scratch;
    double* sb = scratch + kThreads / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(kFull, a, o);
        b += __shfl_down_sync(kFull, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        a = lane < kThreads / 32 ? sa[lane] : 0.0;
        b = lane < kThreads / 32 ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(kFull, a, o);
            b += __shfl_down_sync(kFull, b, o);
        }
    }
}

template <int kThreads>
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double scratch[2 * kThreads / 32];
    block_sum2<kThreads>(a, b, scratch);
}

// ------------------------------------------------------------ scatter body
// 4-entry groups of a segment [a, a + c): the aligned groups that overlap it.
__device__ __forceinline__ uint32_t seg_groups(uint32_t a, uint32_t c) {
    return c ? ((a + c + 3) >> 2) - (a >> 2) : 0;
}

// gpre[j] = groups of segments < j, gpre[k] = total (whole block). With
// dsh: dsh[j] = segrow[j] / 4 - gpre[j] (mod 2^32), so the flattened group f
// of segment j starts at entry 4 * (f + dsh[j]) of the update array, and
// emsk[j] = lo | hi << 2: the entries of the segment's first group start at
// lo, those of its last group end before hi (1..4).
__device__ void segment_groups_prefix(const uint32_t* __restrict__ segrow, const uint32_t* __restrict__ cntrow,
                                      uint32_t k, uint32_t* gpre, uint32_t* sh32, uint32_t* dsh = nullptr,
                                      uint8_t* emsk = nullptr) {
    const uint32_t per = (k + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(k, threadIdx.x * per), hi = min(k, lo + per);
    uint32_t s = 0;
    for (uint32_t j = lo; j < hi; ++j) s += seg_groups(segrow[j], cntrow[j]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh32[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nw ? sh32[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        sh32[lane] = t;
    }
    __syncthreads();
    uint32_t run = (warp ? sh32[warp - 1] : 0) + x - s;
    for (uint32_t j = lo; j < hi; ++j) {
        const uint32_t a = segrow[j], c = cntrow[j];
        gpre[j] = run;
        if (dsh) {
            dsh[j] = (a >> 2) - run;
            emsk[j] = (uint8_t)((a & 3u) | ((((a + c - 1u) & 3u) + 1u) << 2));
        }
        run += seg_groups(a, c);
    }
    if (threadIdx.x == 0) gpre[k] = sh32[nw - 1];
    __syncthreads();
}

// Last segment j >= from with gpre[j] <= f (gpre non-decreasing, gpre[from]
// <= f < gpre[k]): galloping forward, then bisection, O(log distance).
__device__ __forceinline__ uint32_t segment_at(const uint32_t* gpre, uint32_t k, uint32_t from, uint32_t f) {
    uint32_t lo = from, step = 1;
    while (lo + step < k && gpre[lo + step] <= f) {
        lo += step;
        step <<= 1;
    }
    uint32_t hi = lo + step < k ? lo + step : k;
    while (lo + 1 < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (gpre[mid] <= f) lo = mid; else hi = mid;
    }
    return lo;
}


// ------------------------------------------------------------------ init
// PR_0 = pr_init (or 1/n) on all n nodes; the dangling mass of nodes [lo, hi)
// into the FP64 partials (a destination shard sums only the nodes it owns).
__global__ void __launch_bounds__(kReduceThreads) init_kernel(uint32_t n, const float* __restrict__ pr_init,
                                                              const float* __restrict__ inv_deg, float* __restrict__ pr,
                                                              double* __restrict__ partials, uint32_t lo,
                                                              uint32_t hi) {
    const float uniform = (float)(1.0 / (double)n);
    double dang = 0.0, zero = 0.0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const float x = pr_init ? pr_init[v] : uniform;
        pr[v] = x;
        if (inv_deg[v] == 0.0f && v >= lo && v < hi) dang += (double)x;
    }
    block_sum2<kReduceThreads>(zero, dang);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = 0.0;
        partials[2 * blockIdx.x + 1] = dang;
    }
}

__global__ void spr_kernel(uint32_t n, const float* __restrict__ pr, const float* __restrict__ inv_deg,
                           float* __restrict__ spr) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        spr[v] = pr[v] * inv_deg[v];
}

// Algorithm 3 for the groups [f_lo, f_hi) of one source partition's
// flattened segment list: update[t] = sspr[src[t] - base], stored as
// Upd<kUpd>. The source indices are fed through bulk copies into shared
// memory: each warp owns two stages of up to stage_bytes / 16 groups, so a
// whole stage of loads is in flight while the warp works on the other,
// without holding them in registers. A stage holds a contiguous range of the
// flattened group index: whole segments while they fit (not contiguous in
// src: one copy each), else a piece of one segment. The segment tables gpre,
// dsh and emsk (see segment_groups_prefix) are in shared memory, so the loop
// reads no other table. `prologue` runs (on every thread) once the first
// stages are in flight and before any is read, followed by a block barrier:
// the scatter kernel fills sspr there. The barriers `bars` (two per warp) must
// be initialised and visible to the block.
//
// kIdx16: src holds 16-bit local indices src[t] - base (Sec. 3.3 allows them
// for q <= 2^16), so a group is 8 bytes. A bulk copy must start and end on
// 16-byte boundaries: every piece is copied from the even group at or below
// its first group to the even group above its last, and each lane keeps, for
// the piece of segment sg + lane, the offset from a group's global index to
// its position in the stage (a stage holds at most 32 pieces).
template <int kUpd, bool kIdx16, class Prologue>
__device__ void scatter_groups_staged(const float* sspr, uint32_t base, uint32_t len, const uint32_t* gpre,
                                      const uint32_t* dsh, const uint8_t* emsk, uint32_t k,
                                      const void* __restrict__ src_raw,
                                      void* __restrict__ upd_raw, uint32_t f_lo, uint32_t f_hi, int* err,
                                      unsigned char* stages, uint32_t stage_bytes, uint64_t* bars,
                                      Prologue prologue) {
    using U = Upd<kUpd>;
    typename U::T* upd = reinterpret_cast<typename U::T*>(upd_raw);
    const uint32_t* src = static_cast<const uint32_t*>(src_raw);
    const uint16_t* src16 = static_cast<const uint16_t*>(src_raw);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t span = f_hi - f_lo;
    const uint32_t w_lo = f_lo + (uint32_t)((uint64_t)span * warp / nw);
    const uint32_t w_hi = f_lo + (uint32_t)((uint64_t)span * (warp + 1) / nw);
    const uint32_t cap = stage_bytes / (kIdx16 ? 8 : 16);  // groups (16-bit: 8-byte units) per stage
    unsigned char* wst = stages + (size_t)warp * 2 * stage_bytes;
    uint64_t* wb = bars + 2 * warp;
    const uint64_t policy = policy_evict_first();
    // per slot (warp-uniform): groups, first flattened group, its segment
    uint32_t n0 = 0, n1 = 0, fb0 = 0, fb1 = 0, sg0 = 0, sg1 = 0, ph0 = 0, ph1 = 0;
    // kIdx16, per slot: one piece (warp-uniform), and per lane the stage
    // offset of the piece of segment sg + lane (group f of segment j sits at
    // 8-byte unit f + dsh[j] + off)
    bool one0 = true, one1 = true;
    uint32_t off0 = 0, off1 = 0;
    uint32_t pf = w_lo, ppd = 0;
    auto issue16 = [&](int slot) -> bool {  // warp-collective
        if (pf >= w_hi) return false;
        ppd = segment_at(gpre, k, ppd, pf);  // gpre[ppd] <= pf < gpre[ppd + 1]
        unsigned char* dst = wst + (size_t)slot * stage_bytes;
        const uint32_t lim = min(w_hi, pf + cap - 2);  // two units for the rounding of one piece
        uint32_t f_end, off;
        bool one;
        if (gpre[ppd + 1] >= lim) {  // a piece of one segment fills the stage
            one = true;
            f_end = lim;
            const uint32_t dd = dsh[ppd];
            const uint32_t a0 = (pf + dd) & ~1u, a1 = (lim + dd + 1) & ~1u;
            if (lane == 0) {
                mbar_arrive_expect_tx(&wb[slot], (a1 - a0) * 8u);
                bulk_load_hint(dst, src16 + (size_t)a0 * 4, (a1 - a0) * 8u, &wb[slot], policy);
            }
            off = 0u - a0;
        } else {  // the rest of segment ppd, then whole segments while they fit (at most 32 pieces)
            one = false;
            const uint32_t j = ppd + lane;
            uint32_t units = 0, a0 = 0;
            if (j < k) {
                const uint32_t fs = max(pf, gpre[j]), fe = gpre[j + 1];
                if (fe > fs) {
                    a0 = (fs + dsh[j]) & ~1u;
                    units = ((fe + dsh[j] + 1) & ~1u) - a0;
                }
            }
            uint32_t incl = units;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= (uint32_t)o) incl += y;
            }
            // a prefix of the lanes: incl, gpre[j + 1] and j all rise with the lane
            const uint32_t c = __popc(__ballot_sync(kFull, j < k && incl <= cap && gpre[j + 1] <= w_hi));
            f_end = gpre[ppd + c];  // c >= 1: the first piece is under lim - pf + 2 <= cap units
            const uint32_t total = __shfl_sync(kFull, incl, c - 1);
            if (lane == 0) mbar_arrive_expect_tx(&wb[slot], total * 8u);
            __syncwarp();
            const uint32_t excl = incl - units;
            if (lane < c && units)
                bulk_load_hint(dst + (size_t)excl * 8u, src16 + (size_t)a0 * 4, units * 8u, &wb[slot], policy);
            off = excl - a0;
        }
        if (slot) { n1 = f_end - pf; fb1 = pf; sg1 = ppd; one1 = one; off1 = off; }
        else { n0 = f_end - pf; fb0 = pf; sg0 = ppd; one0 = one; off0 = off; }
        pf = f_end;
        return true;
    };
    auto issue = [&](int slot) -> bool {  // warp-collective
        if constexpr (kIdx16) return issue16(slot);
        if (pf >= w_hi) return false;
        ppd = segment_at(gpre, k, ppd, pf);  // gpre[ppd] <= pf < gpre[ppd + 1]
        // The stage holds a piece of one segment that alone fills it (the
        // common case: one copy), or else whole segments while they fit,
        // found 32 at a time (one copy each: they are not contiguous in src).
        const uint32_t lim = min(w_hi, pf + cap);
        unsigned char* dst = wst + (size_t)slot * stage_bytes;
        uint32_t f_end = lim;
        if (gpre[ppd + 1] >= lim) {
            if (lane == 0) {
                mbar_arrive_expect_tx(&wb[slot], (lim - pf) * 16u);
                bulk_load_hint(dst, src + ((pf + dsh[ppd]) << 2), (lim - pf) * 16u, &wb[slot], policy);
            }
        } else {
            for (uint32_t j0 = ppd;; j0 += 32) {
                const uint32_t j = j0 + lane;
                const uint32_t c = __popc(__ballot_sync(kFull, j < k && gpre[j + 1] <= lim));  // a prefix
                if (c) f_end = gpre[j0 + c];
                if (c < 32) break;
            }
            if (lane == 0) mbar_arrive_expect_tx(&wb[slot], (f_end - pf) * 16u);
            __syncwarp();
            // the pieces [max(pf, gpre[j]), min(gpre[j+1], f_end)) tile [pf, f_end)
            for (uint32_t j0 = ppd; j0 < k && gpre[j0] < f_end; j0 += 32) {
                const uint32_t j = j0 + lane;
                if (j < k) {
                    const uint32_t fs = max(pf, gpre[j]), fe = min(gpre[j + 1], f_end);
                    if (fs < fe)
                        bulk_load_hint(dst + (size_t)(fs - pf) * 16u, src + ((fs + dsh[j]) << 2), (fe - fs) * 16u,
                                       &wb[slot], policy);
                }
            }
        }
        if (slot) { n1 = f_end - pf; fb1 = pf; sg1 = ppd; } else { n0 = f_end - pf; fb0 = pf; sg0 = ppd; }
        pf = f_end;
        return true;
    };
    bool has0 = issue(0), has1 = issue(1), ok = true;
    prologue();
    __syncthreads();
    auto consume = [&](int slot) -> bool {  // false: nothing left, or a wait timed out
        const bool has = slot ? has1 : has0;
        if (!has) return false;
        ok = __all_sync(kFull, mbar_wait_bounded(&wb[slot], slot ? ph1 : ph0));
        if (!ok) return false;
        if (slot) ph1 ^= 1u; else ph0 ^= 1u;
        const uint32_t n = slot ? n1 : n0, fb = slot ? fb1 : fb0;
        uint32_t pd = slot ? sg1 : sg0;
        const uint4* ids = reinterpret_cast<const uint4*>(wst + (size_t)slot * stage_bytes);
        if constexpr (kIdx16) {
            const uint2* ids16 = reinterpret_cast<const uint2*>(wst + (size_t)slot * stage_bytes);
            const uint32_t off = slot ? off1 : off0;
            // one group of four local indices: as put below
            auto put16 = [&](uint32_t f, uint32_t u, uint32_t dd, uint32_t glo, uint32_t ghi, uint32_t em) {
                const uint32_t e = (f + dd) << 2;
                const uint2 w = ids16[u];
                const uint32_t i0 = w.x & 0xFFFFu, i1 = w.x >> 16, i2 = w.y & 0xFFFFu, i3 = w.y >> 16;
                if (f != glo && f + 1 != ghi) {
                    if (i0 < len && i1 < len && i2 < len && i3 < len)
                        U::store4(upd, e, sspr[i0], sspr[i1], sspr[i2], sspr[i3]);
                    else
                        atomicOr(err, kErrBounds);
                } else {
                    const uint32_t jlo = f == glo ? (em & 3u) : 0u, jhi = f + 1 == ghi ? (em >> 2) : 4u;
                    const uint32_t v[4] = {i0, i1, i2, i3};
#pragma unroll
                    for (uint32_t jj = 0; jj < 4; ++jj) {
                        if (jj >= jlo && jj < jhi) {
                            if (v[jj] < len) upd[e + jj] = U::from(sspr[v[jj]]); else atomicOr(err, kErrBounds);
                        }
                    }
                }
            };
            if (slot ? one1 : one0) {  // one piece: the same segment and offset for every group
                const uint32_t glo = gpre[pd], ghi = gpre[pd + 1], dd = dsh[pd], em = emsk[pd];
                for (uint32_t g = lane; g < n; g += 32) put16(fb + g, fb + g + dd + off, dd, glo, ghi, em);
            } else {
                uint32_t hint = pd;
                for (uint32_t g0 = 0; g0 < n; g0 += 32) {  // uniform trips: the offsets come by shuffle
                    const uint32_t g = g0 + lane, f = fb + g;
                    const bool act = g < n;
                    if (act) hint = segment_at(gpre, k, hint, f);
                    const uint32_t o = __shfl_sync(kFull, off, act ? hint - pd : 0u);
                    if (act) put16(f, f + dsh[hint] + o, dsh[hint], gpre[hint], gpre[hint + 1], emsk[hint]);
                }
            }
            __syncwarp();  // every lane is done with the slot before it is refilled
            if (slot) has1 = issue(1); else has0 = issue(0);
            return true;
        }
        // one group: interior groups lie inside their segment; a segment's
        // first or last group holds its entries [jlo, jhi) only
        auto put = [&](uint32_t f, uint32_t g, uint32_t dd, uint32_t glo, uint32_t ghi, uint32_t em) {
            const uint32_t e = (f + dd) << 2;
            const uint4 id = ids[g];
            if (f != glo && f + 1 != ghi) {
                const uint32_t i0 = id.x - base, i1 = id.y - base, i2 = id.z - base, i3 = id.w - base;
                if (i0 < len && i1 < len && i2 < len && i3 < len)
                    U::store4(upd, e, sspr[i0], sspr[i1], sspr[i2], sspr[i3]);
                else
                    atomicOr(err, kErrBounds);
            } else {
                const uint32_t jlo = f == glo ? (em & 3u) : 0u, jhi = f + 1 == ghi ? (em >> 2) : 4u;
                const uint32_t v[4] = {id.x, id.y, id.z, id.w};
#pragma unroll
                for (uint32_t jj = 0; jj < 4; ++jj) {
                    if (jj >= jlo && jj < jhi) {
                        const uint32_t i = v[jj] - base;
                        if (i < len) upd[e + jj] = U::from(sspr[i]); else atomicOr(err, kErrBounds);
                    }
                }
            }
        };
        if (fb + n <= gpre[pd + 1]) {  // inside one segment (the common case): no per-group search
            const uint32_t glo = gpre[pd], ghi = gpre[pd + 1], dd = dsh[pd], em = emsk[pd];
            for (uint32_t g = lane; g < n; g += 32) put(fb + g, g, dd, glo, ghi, em);
        } else {
            for (uint32_t g = lane; g < n; g += 32) {
                const uint32_t f = fb + g;
                pd = segment_at(gpre, k, pd, f);
                put(f, g, dsh[pd], gpre[pd], gpre[pd + 1], emsk[pd]);
            }
        }
        __syncwarp();  // every lane is done with the slot before it is refilled
        if (slot) has1 = issue(1); else has0 = issue(0);
        return true;
    };
    while (consume(0) && consume(1)) {
    }
    if (!ok) {
        // a copy did not land in time: record it and wait (bounded) for the
        // copies still in flight before the shared memory is released
        if (lane == 0) atomicOr(err, kErrTimeout);
        if (has0) (void)mbar_wait_bounded(&wb[0], ph0);
        if (has1) (void)mbar_wait_bounded(&wb[1], ph1);
    }
}

// --------------------------------------------------------------- scatter
// Bytes of the staged scatter's segment tables in shared memory: gpre (k + 1
// group starts), dsh (k offsets) and emsk (k bytes), each rounded to 128
// bytes so the stages after them stay aligned.
__host__ __device__ constexpr size_t scatter_gpre_bytes(uint32_t k) {
    return (((size_t)k + 1) * sizeof(uint32_t) + 127) & ~(size_t)127;
}
__host__ __device__ constexpr size_t scatter_dsh_bytes(uint32_t k) {
    return (((size_t)k) * sizeof(uint32_t) + 127) & ~(size_t)127;
}
__host__ __device__ constexpr size_t scatter_table_bytes(uint32_t k) {
    return scatter_gpre_bytes(k) + scatter_dsh_bytes(k) + (((size_t)k + 127) & ~(size_t)127);
}
// The scatter kernel's stage bytes: kScatterStageBytes, smaller where the
// partition and its tables leave less room in the CTA's shared memory.
constexpr size_t kScatterSmemBudget = 232448 - 1024;
__host__ __device__ constexpr uint32_t scatter_stage_bytes(uint32_t q, uint32_t k) {
    const size_t fit = ((kScatterSmemBudget - (size_t)((q + 3) & ~3u) * sizeof(float) - scatter_table_bytes(k)) /
                        (2 * (kScatterThreads / 32))) & ~(size_t)15;
    return fit < kScatterStageBytes ? (uint32_t)fit : kScatterStageBytes;
}
template <int kUpd>
__device__ __forceinline__ void scatter_body(
    uint32_t n, uint32_t q, uint32_t k, const float* __restrict__ pr, const float* __restrict__ inv_deg,
    const uint32_t* __restrict__ src, const uint16_t* __restrict__ src16, const uint32_t* __restrict__ seg_u,
    const uint32_t* __restrict__ cnt_u,
    const uint4* __restrict__ units, const uint32_t* __restrict__ order, void* __restrict__ upd,
    const DevState* __restrict__ st, int* __restrict__ err, const float* __restrict__ pr_prev,
    const float* __restrict__ dq_in, float* __restrict__ dq_out, uint32_t upos) {
    if (st->stop) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint32_t sh32[32];
    __shared__ __align__(8) uint64_t bars[2 * (kScatterThreads / 32)];
    // delta form: the change of SPR since pr_prev, scaled for the bins' format
    const float dsc = pr_prev ? delta_stage_scale<kUpd>(st) : 1.0f;
    float* sspr = reinterpret_cast<float*>(smraw);
    const size_t gpre_off = (size_t)((q + 3) & ~3u) * sizeof(float);
    uint32_t* gpre = reinterpret_cast<uint32_t*>(smraw + gpre_off);
    uint32_t* dsh = reinterpret_cast<uint32_t*>(smraw + gpre_off + scatter_gpre_bytes(k));
    uint8_t* emsk = smraw + gpre_off + scatter_gpre_bytes(k) + scatter_dsh_bytes(k);
    unsigned char* stages = smraw + gpre_off + scatter_table_bytes(k);
    const uint4 unit = units[order[upos]];  // (partition, first group, end group, pieces)
    const uint32_t p = unit.x;
    const uint32_t base = p * q, len = min(q, n - base);
    const uint32_t* segrow = seg_u + (size_t)p * k;
    const uint32_t* cntrow = cnt_u + (size_t)p * k;
    if (threadIdx.x < 2 * (kScatterThreads / 32)) mbar_init(&bars[threadIdx.x], 1);
    fence_mbar_init();
    segment_groups_prefix(segrow, cntrow, k, gpre, sh32, dsh, emsk);  // ends with __syncthreads
    // While the first stages of source indices load: SPR of the partition,
    // staged in shared memory (x itself when inv_deg is null: the SpMV of
    // weighted graphs scatters the vector unscaled), two independent 16-byte
    // loads of each array in flight per thread.
    auto stage_spr = [&] {
        constexpr int kIlp = 2;
        if (dq_in) {
            // error feedback (16-bit bins in a delta solve): SPR, or from the
            // second iteration on its change, plus what the rounding of this
            // node's previous stored value left out, rounded to the bins'
            // format here (every update of the node carries the same value);
            // what this rounding leaves out goes into the next change, so the
            // stored values sum to the true ones up to the last rounding
            // instead of piling up. Every unit of the partition computes the
            // same values from dq_in; its first unit alone writes dq_out.
            using U = Upd<kUpd>;
            const bool writer = unit.y == 0;
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
                const float x = pr_prev ? pr[base + i] - pr_prev[base + i] : pr[base + i];
                const float v = x * inv_deg[base + i] + dq_in[base + i];
                const float sq = U::back(U::from(v * dsc));  // what the stores below will write
                sspr[i] = sq;
                if (writer) dq_out[base + i] = v - sq / dsc;
            }
        } else if (pr_prev) {  // delta form: (PR - PR_prev) / outdeg, scaled
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
                sspr[i] = (pr[base + i] - pr_prev[base + i]) * inv_deg[base + i] * dsc;
        } else if ((base & 3) == 0) {
            const uint32_t v4 = len >> 2;
            const float4* pr4 = reinterpret_cast<const float4*>(pr + base);
            const float4* in4 = reinterpret_cast<const float4*>(inv_deg ? inv_deg + base : pr + base);
            for (uint32_t i0 = threadIdx.x; i0 < v4; i0 += kIlp * blockDim.x) {
                float4 x[kIlp], w[kIlp];
#pragma unroll
                for (int j = 0; j < kIlp; ++j) {
                    const uint32_t i = i0 + j * blockDim.x;
                    if (i < v4) {
                        x[j] = __ldg(pr4 + i);
                        w[j] = inv_deg ? __ldg(in4 + i) : make_float4(1.f, 1.f, 1.f, 1.f);
                    }
                }
#pragma unroll
                for (int j = 0; j < kIlp; ++j) {
                    const uint32_t i = i0 + j * blockDim.x;
                    if (i < v4)
                        reinterpret_cast<float4*>(sspr)[i] =
                            inv_deg ? make_float4(x[j].x * w[j].x, x[j].y * w[j].y, x[j].z * w[j].z, x[j].w * w[j].w)
                                    : x[j];  // unscaled: a bit-for-bit copy
                }
            }
            for (uint32_t i = (v4 << 2) + threadIdx.x; i < len; i += blockDim.x)
                sspr[i] = inv_deg ? pr[base + i] * inv_deg[base + i] : pr[base + i];
        } else {
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x)
                sspr[i] = inv_deg ? pr[base + i] * inv_deg[base + i] : pr[base + i];
        }
    };
    // 16-bit local indices with FP32 bins, where they save time; with 16-bit
    // bins the 32-bit ones measured faster
    constexpr bool kIdx16 = kUpd == kUpdF32;
    scatter_groups_staged<kUpd, kIdx16>(sspr, base, len, gpre, dsh, emsk, k,
                                        kIdx16 ? static_cast<const void*>(src16) : static_cast<const void*>(src), upd,
                                        unit.y, min(unit.z, gpre[k]), err, stages, scatter_stage_bytes(q, k), bars,
                                        stage_spr);
}

template <int kUpd>
__global__ void __launch_bounds__(kScatterThreads, 1) scatter_kernel(
    uint32_t n, uint32_t q, uint32_t k, const float* __restrict__ pr, const float* __restrict__ inv_deg,
    const uint32_t* __restrict__ src, const uint16_t* __restrict__ src16, const uint32_t* __restrict__ seg_u,
    const uint32_t* __restrict__ cnt_u,
    const uint4* __restrict__ units, const uint32_t* __restrict__ order, void* __restrict__ upd,
    const DevState* __restrict__ st, int* __restrict__ err, const float* __restrict__ pr_prev,
    const float* __restrict__ dq_in, float* __restrict__ dq_out) {
    scatter_body<kUpd>(n, q, k, pr, inv_deg, src, src16, seg_u, cnt_u, units, order, upd, st, err, pr_prev, dq_in,
                       dq_out, blockIdx.x);
}

// The scatter of one graph of a batch (its bins in any format).
struct ScatterArgs {
    uint32_t n, q, k;
    const float* pr;
    const float* inv_deg;
    const uint32_t* src;
    const uint16_t* src16;
    const uint32_t* seg_u;
    const uint32_t* cnt_u;
    const uint4* units;
    const uint32_t* order;
    void* upd;
    const DevState* st;
    int* err;
};

// Many graphs in one launch: block b takes item b (graph, position of the
// unit in that graph's order).
template <int kUpd>
__global__ void __launch_bounds__(kScatterThreads, 1) scatter_batch_kernel(const ScatterArgs* __restrict__ tab,
                                                                          const uint2* __restrict__ items) {
    const uint2 it = items[blockIdx.x];
    const ScatterArgs a = tab[it.x];
    scatter_body<kUpd>(a.n, a.q, a.k, a.pr, a.inv_deg, a.src, a.src16, a.seg_u, a.cnt_u, a.units, a.order, a.upd,
                       a.st, a.err, nullptr, nullptr, nullptr, it.y);
}

// ---------------------------------------------------------- gather+apply
struct GatherArgs {
    uint32_t n, q, k;
    const uint32_t* dest;
    const uint32_t* bin_e;
    const uint32_t* chunk_base;
    const uint32_t* gdest;
    const uint32_t* slice_start;
    const uint32_t* slice_bytes;
    const uint4* units;
    const uint32_t* order;
    const uint32_t* hubs;
    float* gacc;
    uint32_t* bin_done;
    const void* upd_in;
    const float* gweight;  // weighted gather (kW): weights in the layout's order
    // window layout
    const uint32_t* wwords;
    const float* wweight;
    const uint4* wdesc;
    const uint32_t* whubs;
    const float* pr_in;
    const float* inv_deg;
    float* pr_out;
    double* partials;
    const DevState* st;
    int* err;
    float d;
    int uniform_dangling;
    int delta;  // PR' = PR + d (A^T dSPR + dD / n): the bins hold changes (PCPM_DELTA)
    // fused scatter of the next iteration
    const uint32_t* src;
    const uint32_t* seg_u;
    const uint32_t* cnt_u;
    void* upd_out;
};

constexpr uint32_t kIdSlotBytes = kChunk * sizeof(uint32_t);
constexpr uint32_t kUpdSlotBytes = kUpdSlot * sizeof(float);
// Shared-memory layout of the gather: per warp kGatherStages ring slots of
// [IDs | weights (weighted graphs) | update slice], then the mbarriers, the
// per-slot metadata and the accumulator.
template <bool kW>
struct Ring {
    static constexpr uint32_t kWOff = kIdSlotBytes;
    static constexpr uint32_t kUpdOff = kIdSlotBytes + (kW ? kChunk * sizeof(float) : 0);
    static constexpr uint32_t kStage = kUpdOff + kUpdSlotBytes;
    static constexpr size_t kBytes = (size_t)kGatherWarps * kGatherStages * kStage;
    static constexpr size_t kBar = (size_t)kGatherWarps * kGatherStages * sizeof(uint64_t);
    static constexpr size_t kMeta = (size_t)kGatherWarps * kGatherStages * 2 * sizeof(uint32_t);
    static constexpr size_t kAcc = kBytes + kBar + kMeta;
    static_assert(kStage % 16 == 0, "ring slots must stay 16-byte aligned");
    static_assert(kAcc % 16 == 0, "accumulator must be 16-byte aligned");
};
// The block sum after the apply borrows the ring's last bytes (idle by then;
// pushed partial sums stay below them).
constexpr size_t kSumScratchBytes = 2 * kGatherWarps * sizeof(double);

// After the accumulation: merge the S CTAs' partial sums of the partition
// over distributed shared memory, apply PR' = (1-d)/n + d*(acc + D/n), write
// the FP64 (L1 change, dangling mass) partials and, in the fused form, scatter
// the partition's SPR' for the next iteration. `ring` (ring_bytes) is idle
// shared memory for the merge and the block sum; the fused scatter takes
// 2 * kThreads / 32 mbarriers at `sbars` and its tables and stages from
// `sarea` (sarea_bytes), both inside idle memory.
template <bool kFused, int kUpd, int kThreads>
__device__ __forceinline__ void gather_finish(const GatherArgs& a, unsigned char* ring, size_t ring_bytes,
                                              uint64_t* sbars, unsigned char* sarea, size_t sarea_bytes, float* acc,
                                              uint32_t* sh32, uint32_t S, uint32_t rank, uint32_t pd,
                                              uint32_t npieces, uint32_t vbase, uint32_t len, uint32_t pslot) {
    using U = Upd<kUpd>;
    constexpr size_t kSumScratch = 2 * (kThreads / 32) * sizeof(double);
    cluster_sync();  // every CTA of the cluster has finished its accumulator

    // This CTA owns nodes [lo, hi) of the partition (multiples of 4). The
    // other CTAs push their partial sums for that range into this CTA's ring
    // memory, idle now, so the merge below reads local shared memory only.
    const uint32_t per = (((len + S - 1) / S) + 3) & ~3u;
    const uint32_t lo = min(len, rank * per), hi = min(len, lo + per);
    float* stage = reinterpret_cast<float*>(ring);
    const bool push = (size_t)(S - 1) * per * sizeof(float) <= ring_bytes - kSumScratch;
    if (push && S > 1) {
        for (uint32_t t = 0; t < S; ++t) {
            if (t == rank) continue;
            const uint32_t tlo = min(len, t * per), thi = min(len, tlo + per);
            push_range(acc + tlo, stage + (size_t)(rank < t ? rank : rank - 1) * per, thi - tlo, t);
        }
        cluster_sync();
    }
    // Sum of the S partial sums of node i in [lo, hi), in a fixed order.
    auto merged = [&](uint32_t i) -> float {
        float s = 0.0f;
        if (push) {
            s = acc[i];
            for (uint32_t q = 0; q + 1 < S; ++q) s += stage[(size_t)q * per + (i - lo)];
        } else {
            for (uint32_t r = 0; r < S; ++r) s += ld_cluster_f32(map_rank(acc + i, r));
        }
        return s;
    };
    // The same for nodes i .. i+3 (i - lo a multiple of 4).
    auto merged4 = [&](uint32_t i) -> float4 {
        if (!push) return make_float4(merged(i), merged(i + 1), merged(i + 2), merged(i + 3));
        float4 s = *reinterpret_cast<const float4*>(acc + i);
        for (uint32_t q = 0; q + 1 < S; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(stage + (size_t)q * per + (i - lo));
            s.x += t.x;
            s.y += t.y;
            s.z += t.z;
            s.w += t.w;
        }
        return s;
    };

    const double D = a.uniform_dangling ? a.st->dangling : 0.0;
    // delta form: PR' = PR + d * (acc + (D - D_prev) / n), acc the sum of the
    // changes of SPR (their scale removed)
    const double Dd = a.uniform_dangling ? a.st->dangling - a.st->dangling_prev : 0.0;
    const float cst = a.delta ? (float)((double)a.d * Dd / (double)a.n)
                              : (float)((1.0 - (double)a.d) / (double)a.n + (double)a.d * D / (double)a.n);
    // exact: the scales are powers of two
    const float d_acc = a.d * (a.delta ? delta_acc_scale<kUpd>(a.st) : U::acc_scale);
    const float keep = a.delta ? 1.0f : 0.0f;  // the delta form adds the old rank
    // Per-thread partial sums of at most len / blockDim terms in FP32 (FP64
    // arithmetic is slow on this part); thread and block totals in FP64.
    float res_f = 0.0f, dg_f = 0.0f;
    // Apply to one node: PR', residual and dangling terms, SPR' for the fused scatter.
    auto apply1 = [&](uint32_t i, float s, float old, float inv) -> float {
        const float x = fmaf(keep, old, fmaf(d_acc, s, cst));
        if (kFused) acc[i] = x * inv;
        res_f += fabsf(x - old);
        if (inv == 0.0f) dg_f += x;
        return x;
    };
    // Nodes [lo, vec_end) go four at a time with 16-byte loads and stores
    // (the partition starts on a 16-byte boundary), kApplyVec groups of
    // four in flight per thread; the rest one at a time.
    const uint32_t vec_end = (npieces == 1 && (vbase & 3u) == 0) ? lo + ((hi - lo) & ~3u) : lo;
    for (uint32_t i0 = lo + 4 * threadIdx.x; i0 < vec_end; i0 += 4 * kApplyVec * blockDim.x) {
        float4 o[kApplyVec], w[kApplyVec], s[kApplyVec];
#pragma unroll
        for (int j = 0; j < kApplyVec; ++j) {
            const uint32_t i = i0 + 4 * j * blockDim.x;
            if (i < vec_end) {
                o[j] = __ldg(reinterpret_cast<const float4*>(a.pr_in + vbase + i));
                w[j] = __ldg(reinterpret_cast<const float4*>(a.inv_deg + vbase + i));
                s[j] = merged4(i);
            }
        }
#pragma unroll
        for (int j = 0; j < kApplyVec; ++j) {
            const uint32_t i = i0 + 4 * j * blockDim.x;
            if (i < vec_end) {
                float4 x;
                x.x = apply1(i, s[j].x, o[j].x, w[j].x);
                x.y = apply1(i + 1, s[j].y, o[j].y, w[j].y);
                x.z = apply1(i + 2, s[j].z, o[j].z, w[j].z);
                x.w = apply1(i + 3, s[j].w, o[j].w, w[j].w);
                *reinterpret_cast<float4*>(a.pr_out + vbase + i) = x;
            }
        }
    }
    if (npieces == 1) {
        // The remaining nodes: kApplyIlp independent nodes per thread per
        // round, their loads in flight together.
        for (uint32_t i0 = vec_end + threadIdx.x; i0 < hi; i0 += kApplyIlp * blockDim.x) {
            float s[kApplyIlp], old[kApplyIlp], inv[kApplyIlp];
#pragma unroll
            for (int j = 0; j < kApplyIlp; ++j) {
                const uint32_t i = i0 + j * blockDim.x;
                s[j] = 0.0f;
                old[j] = 0.0f;
                inv[j] = 1.0f;
                if (i < hi) {
                    old[j] = a.pr_in[vbase + i];
                    inv[j] = a.inv_deg[vbase + i];
                    s[j] = merged(i);
                }
            }
#pragma unroll
            for (int j = 0; j < kApplyIlp; ++j) {
                const uint32_t i = i0 + j * blockDim.x;
                if (i < hi) a.pr_out[vbase + i] = apply1(i, s[j], old[j], inv[j]);
            }
        }
    } else {
        // The bin is cut into several units: add this unit's sums to the
        // global partial sums; the last CTA to arrive applies the partition.
        uint32_t& last = sh32[0];
        const bool aligned = (vbase & 3u) == 0;
        const uint32_t gv_end = aligned ? lo + ((hi - lo) & ~3u) : lo;
        for (uint32_t i = lo + 4 * threadIdx.x; i < gv_end; i += 4 * blockDim.x) {
            const float4 s = merged4(i);
            if (s.x != 0.0f || s.y != 0.0f || s.z != 0.0f || s.w != 0.0f) red_add_v4(a.gacc + vbase + i, s);
        }
        for (uint32_t i = gv_end + threadIdx.x; i < hi; i += blockDim.x) {
            const float s = merged(i);
            if (s != 0.0f) atomicAdd(&a.gacc[vbase + i], s);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(&a.bin_done[pd], 1u) == npieces * S - 1 ? 1u : 0u;
        __syncthreads();
        if (last) {
            __threadfence();
            // The whole partition from the global sums: four nodes at a time
            // where the partition starts on a 16-byte boundary, then the rest.
            const uint32_t av_end = aligned ? (len & ~3u) : 0;
            for (uint32_t i0 = 4 * threadIdx.x; i0 < av_end; i0 += 4 * kApplyVecCut * blockDim.x) {
                float4 o[kApplyVecCut], w[kApplyVecCut], s[kApplyVecCut];
#pragma unroll
                for (int j = 0; j < kApplyVecCut; ++j) {
                    const uint32_t i = i0 + 4 * j * blockDim.x;
                    if (i < av_end) {
                        s[j] = __ldcg(reinterpret_cast<const float4*>(a.gacc + vbase + i));
                        o[j] = __ldg(reinterpret_cast<const float4*>(a.pr_in + vbase + i));
                        w[j] = __ldg(reinterpret_cast<const float4*>(a.inv_deg + vbase + i));
                    }
                }
#pragma unroll
                for (int j = 0; j < kApplyVecCut; ++j) {
                    const uint32_t i = i0 + 4 * j * blockDim.x;
                    if (i < av_end) {
                        float4 x;
                        x.x = apply1(i, s[j].x, o[j].x, w[j].x);
                        x.y = apply1(i + 1, s[j].y, o[j].y, w[j].y);
                        x.z = apply1(i + 2, s[j].z, o[j].z, w[j].z);
                        x.w = apply1(i + 3, s[j].w, o[j].w, w[j].w);
                        *reinterpret_cast<float4*>(a.gacc + vbase + i) = make_float4(0.f, 0.f, 0.f, 0.f);
                        *reinterpret_cast<float4*>(a.pr_out + vbase + i) = x;
                    }
                }
            }
            for (uint32_t i0 = av_end + threadIdx.x; i0 < len; i0 += kApplyIlp * blockDim.x) {
                float s[kApplyIlp], old[kApplyIlp], inv[kApplyIlp];
#pragma unroll
                for (int j = 0; j < kApplyIlp; ++j) {
                    const uint32_t i = i0 + j * blockDim.x;
                    s[j] = 0.0f;
                    old[j] = 0.0f;
                    inv[j] = 1.0f;
                    if (i < len) {
                        s[j] = __ldcg(&a.gacc[vbase + i]);
                        old[j] = a.pr_in[vbase + i];
                        inv[j] = a.inv_deg[vbase + i];
                    }
                }
#pragma unroll
                for (int j = 0; j < kApplyIlp; ++j) {
                    const uint32_t i = i0 + j * blockDim.x;
                    if (i < len) {
                        const float x = fmaf(keep, old[j], fmaf(d_acc, s[j], cst));
                        a.gacc[vbase + i] = 0.0f;
                        a.pr_out[vbase + i] = x;
                        res_f += fabsf(x - old[j]);
                        if (inv[j] == 0.0f) dg_f += x;
                    }
                }
            }
            if (threadIdx.x == 0) a.bin_done[pd] = 0;
        }
    }
    double res = (double)res_f, dg = (double)dg_f;
    block_sum2<kThreads>(res, dg, reinterpret_cast<double*>(ring + ring_bytes - kSumScratch));
    if (threadIdx.x == 0) {
        a.partials[2 * pslot] = res;
        a.partials[2 * pslot + 1] = dg;
    }

    if constexpr (kFused) {
        if (npieces != 1) {  // the host runs cut bins in two-phase form only
            if (threadIdx.x == 0) atomicOr(a.err, kErrBounds);
            cluster_sync();
            return;
        }
        // Fused scatter of the next iteration: assemble SPR' of the whole
        // partition in every CTA's shared memory (each pushes its range to
        // the others), then write 1/S of the partition's update segments.
        __syncthreads();
        if (push) {
            for (uint32_t t = 0; t < S; ++t)
                if (t != rank) push_range(acc + lo, acc + lo, hi - lo, t);
            cluster_sync();
        } else {
            cluster_sync();
            for (uint32_t r = 0; r < S; ++r) {
                if (r == rank) continue;
                const uint32_t rlo = min(len, r * per), rhi = min(len, rlo + per);
                const uint32_t q4 = (rhi - rlo) >> 2;
                for (uint32_t i = threadIdx.x; i < q4; i += blockDim.x)
                    reinterpret_cast<float4*>(acc + rlo)[i] = ld_cluster_f32x4(map_rank(acc + rlo + 4 * i, r));
                for (uint32_t i = rlo + (q4 << 2) + threadIdx.x; i < rhi; i += blockDim.x)
                    acc[i] = ld_cluster_f32(map_rank(acc + i, r));
            }
            cluster_sync();  // no CTA reads another's shared memory after this point
        }
        uint32_t* gpre = reinterpret_cast<uint32_t*>(sarea);
        const uint32_t* segrow = a.seg_u + (size_t)pd * a.k;
        const uint32_t* cntrow = a.cnt_u + (size_t)pd * a.k;
        constexpr int kWarps = kThreads / 32;
        if (threadIdx.x < 2 * kWarps) mbar_init(&sbars[threadIdx.x], 1);
        fence_mbar_init();
        fence_proxy_async_smem();  // the block sum's scratch becomes a bulk-copy target
        uint32_t* dsh = reinterpret_cast<uint32_t*>(sarea + scatter_gpre_bytes(a.k));
        uint8_t* emsk = sarea + scatter_gpre_bytes(a.k) + scatter_dsh_bytes(a.k);
        segment_groups_prefix(segrow, cntrow, a.k, gpre, sh32, dsh, emsk);  // ends with __syncthreads
        const uint32_t G = gpre[a.k];
        const uint32_t f_lo = (uint32_t)((uint64_t)G * rank / S);
        const uint32_t f_hi = (uint32_t)((uint64_t)G * (rank + 1) / S);
        // stages: the scatter area after the segment table
        const size_t st_off = scatter_table_bytes(a.k);
        const uint32_t stage_bytes = (uint32_t)(((sarea_bytes - st_off) / (2 * kWarps)) & ~(size_t)15);
        scatter_groups_staged<kUpd, false>(acc, vbase, len, gpre, dsh, emsk, a.k, a.src, a.upd_out, f_lo, f_hi, a.err,
                                    sarea + st_off, stage_bytes, sbars, [] {});
    } else {
        if (!push) cluster_sync();  // remote loads of this CTA's shared memory are done
    }
}

// kFused: also scatter the next iteration; kCanon: decode the canonical bins;
// kRuns: sum run-bit runs of the bank-spread layout in a register; kUpd: the
// update bins' storage (canonical bins: FP32 only); kW: multiply every update
// by its edge's weight (weighted graphs, Sec. 3.5).
template <bool kFused, bool kCanon, bool kRuns, int kUpd, bool kW = false>
__global__ void __launch_bounds__(kGatherWarps * 32, 1) gather_kernel(const GatherArgs a) {
    using U = Upd<kUpd>;
    using R = Ring<kW>;
    static_assert(!kCanon || kUpd == kUpdF32, "the canonical gather reads FP32 updates");
    static_assert(!kW || (!kCanon && !kFused), "the weighted gather is a two-phase, bank-spread gather");
    if (a.st->stop) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint32_t sh32[32];
    unsigned char* ring = smraw;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + R::kBytes);
    uint32_t* meta = reinterpret_cast<uint32_t*>(smraw + R::kBytes + R::kBar);
    float* acc = reinterpret_cast<float*>(smraw + R::kAcc);

    const uint32_t S = cluster_size(), rank = cluster_rank();
    const uint4 unit = a.units[a.order[blockIdx.x / S]];  // (bin, first chunk, end chunk, pieces of the bin)
    const uint32_t pd = unit.x, npieces = unit.w;
    const uint32_t vbase = pd * a.q, len = min(a.q, a.n - vbase);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (uint32_t i = threadIdx.x; i < (len + 3) / 4; i += blockDim.x)
        reinterpret_cast<float4*>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x < kHubSlots) acc[a.q + kPadSlots + threadIdx.x] = 0.0f;
    if (threadIdx.x < kGatherWarps * kGatherStages) mbar_init(&bars[threadIdx.x], 1);
    fence_mbar_init();
    __syncthreads();

    // The apply at the end of the unit reads PR_old and 1/outdeg of this CTA's
    // share of the partition: have them in L2 by then.
    if (threadIdx.x == 0 && npieces == 1) {
        const uint32_t per0 = (((len + S - 1) / S) + 3) & ~3u;
        const uint32_t lo0 = min(len, rank * per0), hi0 = min(len, lo0 + per0);
        const uint64_t keep = policy_evict_last();
        prefetch_l2(a.pr_in + vbase + lo0, hi0 - lo0, keep);
        prefetch_l2(a.inv_deg + vbase + lo0, hi0 - lo0, keep);
    }
    const uint32_t h0 = a.hubs[2 * pd], h1 = a.hubs[2 * pd + 1];
    float hub0 = 0.0f, hub1 = 0.0f;  // canonical layout: hub sums in registers
    // bank-spread layout: hub slot pair of the words, and this warp's pair
    const uint32_t hub_slot = a.q + kPadSlots, hub_off = 2u * (uint32_t)warp;
    const uint32_t E0 = a.bin_e[pd], E1 = a.bin_e[pd + 1];
    if (unit.z > unit.y) {
        const uint32_t c_first = unit.y;
        const uint32_t nch = unit.z - unit.y;
        const uint32_t gw = rank * kGatherWarps + warp, GW = S * kGatherWarps;
        const uint32_t wc0 = c_first + (uint32_t)((uint64_t)nch * gw / GW);
        const uint32_t nmine = c_first + (uint32_t)((uint64_t)nch * (gw + 1) / GW) - wc0;
        unsigned char* wring = ring + (size_t)warp * kGatherStages * R::kStage;
        uint64_t* wbar = bars + warp * kGatherStages;
        uint32_t* wmeta = meta + warp * kGatherStages * 2;
        const uint32_t lt = lanemask_lt();
        const uint64_t stream_policy = policy_evict_first();  // each chunk is read once

        // Per-chunk values of this warp's run, 32 per register table, loaded
        // two tables ahead: the canonical layout's update bases (entry j+1
        // bounds chunk j's slice), or the bank-spread layout's slice start and
        // size.
        auto load_a = [&](uint32_t t) -> uint32_t {
            const uint32_t j = 32 * t + lane;
            if constexpr (kCanon) return j <= nmine ? a.chunk_base[wc0 + j] : 0u;
            else return j < nmine ? a.slice_start[wc0 + j] : 0u;
        };
        auto load_b = [&](uint32_t t) -> uint32_t {
            const uint32_t j = 32 * t + lane;
            if constexpr (kCanon) return 0u;
            else return j < nmine ? a.slice_bytes[wc0 + j] : 0u;
        };
        uint32_t tb = 0, t0 = load_a(0), t1 = load_a(1), t2 = load_a(2);
        uint32_t s0 = load_b(0), s1 = load_b(1), s2 = load_b(2);
        auto pick = [&](uint32_t x0, uint32_t x1, uint32_t j) -> uint32_t {  // warp-collective
            const uint32_t y0 = __shfl_sync(kFull, x0, j & 31);
            const uint32_t y1 = __shfl_sync(kFull, x1, j & 31);
            return (j >> 5) == tb ? y0 : y1;
        };
        auto issue = [&](uint32_t j) {  // warp-collective
            if (((j + 1) >> 5) > tb + 1) {
                ++tb;
                t0 = t1;
                t1 = t2;
                t2 = load_a(tb + 2);
                s0 = s1;
                s1 = s2;
                s2 = load_b(tb + 2);
            }
            uint32_t us, ubytes, fb = 0;
            if constexpr (kCanon) {
                const uint32_t cb0 = pick(t0, t1, j), cb1 = pick(t0, t1, j + 1);
                us = (cb0 > 0 ? cb0 - 1 : 0) & ~3u;
                ubytes = (((cb1 + 3) & ~3u) - us) * (uint32_t)sizeof(float);
                fb = cb0;
            } else {
                us = pick(t0, t1, j);
                ubytes = pick(s0, s1, j);
            }
            if (lane == 0) {
                const uint32_t slot = j % kGatherStages;
                unsigned char* dst = wring + (size_t)slot * R::kStage;
                if constexpr (kCanon) {
                    wmeta[2 * slot] = fb;
                    wmeta[2 * slot + 1] = us;
                }
                const uint32_t* ids = (kCanon ? a.dest : a.gdest) + (size_t)(wc0 + j) * kChunk;
                mbar_arrive_expect_tx(&wbar[slot], kIdSlotBytes + (kW ? kChunk * 4u : 0u) + ubytes);
                bulk_load_hint(dst, ids, kIdSlotBytes, &wbar[slot], stream_policy);
                if constexpr (kW)
                    bulk_load_hint(dst + R::kWOff, a.gweight + (size_t)(wc0 + j) * kChunk, kChunk * 4u, &wbar[slot],
                                   stream_policy);
                if (ubytes)
                    bulk_load_hint(dst + R::kUpdOff, static_cast<const typename U::T*>(a.upd_in) + us, ubytes,
                                   &wbar[slot], stream_policy);
            }
        };

        const uint32_t pre = nmine < (uint32_t)kGatherStages ? nmine : (uint32_t)kGatherStages;
        for (uint32_t j = 0; j < pre; ++j) issue(j);
        uint32_t issued = pre;
        uint32_t j = 0;
        bool ok = true;
        for (; j < nmine; ++j) {
            const uint32_t slot = j % kGatherStages;
            ok = __all_sync(kFull, mbar_wait_bounded(&wbar[slot], (j / kGatherStages) & 1u));
            if (!ok) break;
            const unsigned char* stage = wring + (size_t)slot * R::kStage;
            const uint32_t* ids_s = reinterpret_cast<const uint32_t*>(stage);
            const typename U::T* ups = reinterpret_cast<const typename U::T*>(stage + R::kUpdOff);
            constexpr int kPer = kChunk / 32;  // IDs per lane
            // All loads of the chunk first (IDs, then update values), then the
            // adds: eight independent shared-memory operations per lane.
            uint32_t id[kPer], uo[kPer], valid = 0, cont = 0;
#pragma unroll
            for (int h = 0; h < kPer / 4; ++h) {
                const uint4 v4 = *reinterpret_cast<const uint4*>(ids_s + h * 128 + lane * 4);
                id[4 * h] = v4.x;
                id[4 * h + 1] = v4.y;
                id[4 * h + 2] = v4.z;
                id[4 * h + 3] = v4.w;
            }
            if constexpr (kCanon) {
                // Algorithm 4's update pointer as warp arithmetic: the update
                // of an ID is the inclusive count of flagged IDs up to it - 1.
                uint32_t fbase = wmeta[2 * slot];
                const uint32_t us = wmeta[2 * slot + 1];
                const uint32_t cstart = (wc0 + j) * kChunk;
#pragma unroll
                for (int h = 0; h < kPer / 4; ++h) {
                    uint32_t f[4], b[4], before = 0, total = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        f[q] = id[4 * h + q] >> 31;
                        b[q] = __ballot_sync(kFull, f[q]);
                        before += __popc(b[q] & lt);
                        total += __popc(b[q]);
                    }
                    uint32_t u = fbase + before - 1 - us;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        u += f[q];
                        uo[4 * h + q] = u;
                        id[4 * h + q] = (id[4 * h + q] & kIdMask) - vbase;
                    }
                    fbase += total;
                }
                // Only a bin's first and last chunk hold IDs of other bins.
                if (cstart >= E0 && cstart + kChunk <= E1) {
                    valid = (1u << kPer) - 1u;
                } else {
#pragma unroll
                    for (int h = 0; h < kPer / 4; ++h)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t pos = cstart + h * 128 + lane * 4 + q;
                            valid |= (pos >= E0 && pos < E1) ? 1u << (4 * h + q) : 0u;
                        }
                }
            } else {
                // Bank-spread layout: local destination and update offset are
                // stored in the word, padding names a spare accumulator slot,
                // and the build checked every word against the accumulator
                // and the slice, so no ID needs a test here.
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    if constexpr (kRuns) cont |= (id[q] & kGwRunBit) ? 1u << q : 0u;
                    uo[q] = (id[q] >> kGwUpdShift) & kGwUpdMask;
                    id[q] &= kGwLocMask;
                }
            }
            float val[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) val[q] = U::load(ups, (!kCanon || (valid >> q & 1u)) ? uo[q] : 0u);
            if constexpr (kW) {
                // the weight of each ID sits at the ID's position (Sec. 3.5)
                const float* wts = reinterpret_cast<const float*>(stage + R::kWOff);
#pragma unroll
                for (int h = 0; h < kPer / 4; ++h) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wts + h * 128 + lane * 4);
                    val[4 * h] *= w4.x;
                    val[4 * h + 1] *= w4.y;
                    val[4 * h + 2] *= w4.z;
                    val[4 * h + 3] *= w4.w;
                }
            }
            [[maybe_unused]] float run = 0.0f;  // kRuns: sum of a run of equal destinations in this lane
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const uint32_t loc = id[q];
                if constexpr (kCanon) {
                    const bool ok_q = (valid >> q & 1u) != 0;
                    const bool is0 = ok_q && loc == h0, is1 = ok_q && loc == h1;
                    hub0 += is0 ? val[q] : 0.0f;
                    hub1 += is1 ? val[q] : 0.0f;
                    if (ok_q && !is0 && !is1) {
                        if (loc < len) atomicAdd(&acc[loc], val[q]);
                        else atomicOr(a.err, kErrBounds);
                    }
                } else {
                    // hub slots move to this warp's private pair
                    const uint32_t slot = loc + (loc >= hub_slot ? hub_off : 0u);
                    if constexpr (kRuns) {
                        // one shared-memory add per run of equal slots
                        run += val[q];
                        if (!(cont >> q & 1u)) {
                            atomicAdd(&acc[slot], run);
                            run = 0.0f;
                        }
                    } else {
                        atomicAdd(&acc[slot], val[q]);
                    }
                }
            }
            __syncwarp();
            if (issued < nmine) {
                issue(issued);
                ++issued;
            }
        }
        if (!ok) {
            // A copy did not land in time: record it, then wait (bounded) for
            // every copy still in flight before shared memory is reused.
            if (lane == 0) atomicOr(a.err, kErrTimeout);
            for (uint32_t jj = j; jj < issued; ++jj)
                (void)mbar_wait_bounded(&wbar[jj % kGatherStages], (jj / kGatherStages) & 1u);
        }
    }
    // The two hubs' sums: registers (canonical layout) or this warp's slot
    // pair (bank-spread layout, complete after the loop's last __syncwarp).
    if constexpr (kCanon) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hub0 += __shfl_xor_sync(kFull, hub0, o);
            hub1 += __shfl_xor_sync(kFull, hub1, o);
        }
    } else {
        __syncwarp();
        hub0 = acc[hub_slot + hub_off];
        hub1 = acc[hub_slot + hub_off + 1];
    }
    if (lane == 0) {
        if (h0 < len) atomicAdd(&acc[h0], hub0);
        if (h1 < len) atomicAdd(&acc[h1], hub1);
    }
    static_assert(R::kMeta >= 2 * kGatherWarps * sizeof(uint64_t), "two stage barriers per warp for the fused scatter");
    static_assert(R::kBytes >= scatter_table_bytes(PCPM_MAX_PARTITIONS) + 2 * kGatherWarps * 16 * 16,
                  "the fused scatter's stages must hold at least 16 groups beside the largest segment tables");
    gather_finish<kFused, kUpd, kGatherWarps * 32>(a, ring, R::kBytes, reinterpret_cast<uint64_t*>(meta), ring,
                                                   R::kBytes, acc, sh32, S, rank, pd, npieces, vbase, len, blockIdx.x);
}


// ------------------------------------------------- gather+apply, window layout
// Shared memory of the window gather: kStages ring stages of [header + IDs |
// weights (weighted graphs) | update slice], the full and empty mbarriers of
// each stage, then the accumulator (q slots and kWinWarps * kWinHubs hub
// slots).
template <int kUpd, bool kW>
struct WinRing {
    using T = typename Upd<kUpd>::T;
    static constexpr uint32_t kWordBytes = kWinStride * sizeof(uint32_t);
    static constexpr uint32_t kWOff = kWordBytes;
    static constexpr uint32_t kUpdOff = kWordBytes * (kW ? 2u : 1u);
    static constexpr uint32_t kUpdCap = kWin + 2 * (16 / (uint32_t)sizeof(T));
    static constexpr uint32_t kStage = kUpdOff + ((kUpdCap * (uint32_t)sizeof(T) + 15u) & ~15u);
    // as many stages as fit beside the largest accumulator (and 1 KB of
    // static shared memory), at most 8
    static constexpr size_t kBudget =
        232448 - 1024 - 128 -
        (size_t)((kW ? PCPM_MAX_WEIGHTED_PART_SIZE : PCPM_MAX_PART_SIZE) + kWinWarps * kWinHubs) * sizeof(float);
    static constexpr int kStages = (int)(kBudget / kStage < 8 ? kBudget / kStage : 8);
    static_assert(kStages >= 2, "the ring needs two stages");
    static constexpr size_t kBytes = (size_t)kStages * kStage;
    static constexpr size_t kAcc = kBytes + 128;  // 2 * kStages mbarriers
    static_assert(kStage % 16 == 0 && kWordBytes % 16 == 0, "stage areas must stay 16-byte aligned");
    static_assert(2 * kStages * sizeof(uint64_t) <= 128, "barrier area");
};
constexpr int kWinThreads = (kWinWarps + 1) * 32;  // consumer warps and one producer warp
constexpr size_t kWinScatterBars = 512;            // fused scatter: 2 mbarriers per warp at the ring's start
static_assert(2 * (kWinThreads / 32) * sizeof(uint64_t) <= kWinScatterBars, "scatter barriers");

// Gather + apply over the window layout (see kWin). A cluster of S CTAs takes
// one gather unit (a run of windows of one bin); each CTA a contiguous share
// of its windows. Warp kWinWarps produces: one lane issues, per window, the
// bulk copies of its words (and weights) and update slice into the next ring
// stage once every consumer warp has released it. Consumer warp w takes group
// w of every window: lane l walks its run of the group's sorted positions,
// summing the values of equal slots in a register and adding each finished
// run into the accumulator with a plain load and store (the slot belongs to
// this warp alone, and its run ends in this lane alone). A lane's unfinished
// last run (its slot continues in the next lane) is added with one
// shared-memory atomic after the warp's plain adds, so at most one atomic per
// lane and window remains of the one per ID of a racing layout. Then the hub
// slots of all warps are summed into the hubs in warp order, and
// gather_finish merges, applies and (fused) scatters.
// uslot: the unit's position in a.order; pslot: this CTA's pair of FP64
// partial sums in a.partials.
template <bool kFused, int kUpd, bool kW>
__device__ __forceinline__ void gather_win_body(const GatherArgs& a, uint32_t uslot, uint32_t pslot) {
    using U = Upd<kUpd>;
    using R = WinRing<kUpd, kW>;
    using T = typename U::T;
    static_assert(!kW || !kFused, "the weighted gather is two-phase");
    if (a.st->stop) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint32_t sh32[32];
    unsigned char* ring = smraw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smraw + R::kBytes);
    uint64_t* empty = full + R::kStages;
    float* acc = reinterpret_cast<float*>(smraw + R::kAcc);

    const uint32_t S = cluster_size(), rank = cluster_rank();
    const uint4 unit = a.units[a.order[uslot]];  // (bin, first window, end window, pieces of the bin)
    const uint32_t pd = unit.x, npieces = unit.w;
    const uint32_t vbase = pd * a.q, len = min(a.q, a.n - vbase);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (uint32_t i = threadIdx.x; i < (len + 3) / 4; i += blockDim.x)
        reinterpret_cast<float4*>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t i = threadIdx.x; i < kWinWarps * kWinHubs; i += blockDim.x) acc[a.q + i] = 0.0f;
    if (threadIdx.x < R::kStages) {
        mbar_init(&full[threadIdx.x], 1);
        mbar_init(&empty[threadIdx.x], kWinWarps);
    }
    fence_mbar_init();
    __syncthreads();
    if (threadIdx.x == 0 && npieces == 1) {  // PR_old and 1/outdeg of this CTA's share, for the apply
        const uint32_t per0 = (((len + S - 1) / S) + 3) & ~3u;
        const uint32_t lo0 = min(len, rank * per0), hi0 = min(len, lo0 + per0);
        const uint64_t keep = policy_evict_last();
        prefetch_l2(a.pr_in + vbase + lo0, hi0 - lo0, keep);
        prefetch_l2(a.inv_deg + vbase + lo0, hi0 - lo0, keep);
    }
    const uint32_t nwu = unit.z - unit.y;
    const uint32_t w0 = unit.y + (uint32_t)((uint64_t)nwu * rank / S);
    const uint32_t nmine = unit.y + (uint32_t)((uint64_t)nwu * (rank + 1) / S) - w0;
    const long long work_limit = g_work_wait_limit;

    if (warp == (uint32_t)kWinWarps) {
        if (lane == 0) {  // producer
            const uint64_t policy = policy_evict_first();  // every window is read once
            // The next window's descriptor loads while the producer waits for
            // a free stage, so no global-memory latency sits between a stage's
            // release and its refill.
            uint4 next = nmine ? a.wdesc[w0] : make_uint4(0u, 0u, 0u, 0u);
            uint32_t j = 0;
            bool ok = true;
            for (; j < nmine; ++j) {
                const uint4 dsc = next;  // (slice start, slice bytes, word bytes, IDs)
                if (j + 1 < nmine) next = a.wdesc[w0 + j + 1];
                const uint32_t s = j % R::kStages;
                if (j >= (uint32_t)R::kStages && !mbar_wait_work(&empty[s], ((j / R::kStages) - 1) & 1u, work_limit)) {
                    ok = false;
                    break;
                }
                unsigned char* st = ring + (size_t)s * R::kStage;
                mbar_arrive_expect_tx(&full[s], dsc.z * (kW ? 2u : 1u) + dsc.y);
                bulk_load_hint(st, a.wwords + (size_t)(w0 + j) * kWinStride, dsc.z, &full[s], policy);
                if constexpr (kW)
                    bulk_load_hint(st + R::kWOff, a.wweight + (size_t)(w0 + j) * kWinStride, dsc.z, &full[s], policy);
                if (dsc.y)
                    bulk_load_hint(st + R::kUpdOff, static_cast<const T*>(a.upd_in) + dsc.x, dsc.y, &full[s], policy);
            }
            // a stage that was not released in time is recorded; either way
            // the last window issued into each stage has landed (bounded wait)
            // before this warp reaches the merge: consumers that gave up no
            // longer wait for them, and no copy may land after the CTA exits
            if (!ok) atomicOr(a.err, kErrTimeout);
            for (uint32_t jj = j > (uint32_t)R::kStages ? j - R::kStages : 0u; jj < j; ++jj)
                (void)mbar_wait_bounded(&full[jj % R::kStages], (jj / R::kStages) & 1u);
        }
        __syncwarp();
    } else {
        for (uint32_t j = 0; j < nmine; ++j) {
            const uint32_t s = j % R::kStages;
            if (!__all_sync(kFull, mbar_wait_work(&full[s], (j / R::kStages) & 1u, work_limit))) {
                if (lane == 0) atomicOr(a.err, kErrTimeout);
                break;
            }
            const unsigned char* st = ring + (size_t)s * R::kStage;
            const uint16_t* hdr = reinterpret_cast<const uint16_t*>(st);
            const uint32_t g0 = hdr[warp], nw = hdr[warp + 1] - g0;
            if (nw) {
                const uint32_t* wd = reinterpret_cast<const uint32_t*>(st) + kWinHdrWords + g0;
                const T* ups = reinterpret_cast<const T*>(st + R::kUpdOff);
                const uint32_t rounds = (nw + 31) >> 5, longer = nw - 32 * (rounds - 1);
                const uint32_t cnt = lane < longer ? rounds : rounds - 1;
                float run = 0.0f;
                uint32_t last = kWinEndBit;  // word of the lane's last ID (none: no unfinished run)
                constexpr uint32_t kU = 3;
                for (uint32_t r0 = 0; r0 < rounds; r0 += kU) {
                    uint32_t wv[kU];
                    float v[kU];
#pragma unroll
                    for (uint32_t i = 0; i < kU; ++i) wv[i] = r0 + i < cnt ? wd[(r0 + i) * 32 + lane] : 0u;
#pragma unroll
                    for (uint32_t i = 0; i < kU; ++i) {
                        v[i] = r0 + i < cnt ? U::load(ups, (wv[i] >> kWinOffShift) & kWinOffMask) : 0.0f;
                        if constexpr (kW) {
                            const float* wts = reinterpret_cast<const float*>(st + R::kWOff) + kWinHdrWords + g0;
                            if (r0 + i < cnt) v[i] *= wts[(r0 + i) * 32 + lane];
                        }
                    }
                    // The runs that finish in this batch have distinct slots
                    // (a slot's run ends once per group), so their
                    // accumulator loads are all issued before any store.
                    float old[kU];
#pragma unroll
                    for (uint32_t i = 0; i < kU; ++i)
                        old[i] = (r0 + i < cnt && (wv[i] & kWinEndBit)) ? acc[wv[i] & kWinSlotMask] : 0.0f;
#pragma unroll
                    for (uint32_t i = 0; i < kU; ++i) {
                        if (r0 + i < cnt) {
                            run += v[i];
                            last = wv[i];
                            if (wv[i] & kWinEndBit) {  // a finished run: this lane alone adds it
                                old[i] += run;
                                run = 0.0f;
                            }
                        }
                    }
#pragma unroll
                    for (uint32_t i = 0; i < kU; ++i)
                        if (r0 + i < cnt && (wv[i] & kWinEndBit)) acc[wv[i] & kWinSlotMask] = old[i];
                }
                // A run that continues in the next lane: no run of the group
                // ends on its slot in this lane, but one lane finishes it with
                // a plain add above and others may hold parts too, so the
                // parts are added atomically, after the warp's plain adds.
                __syncwarp();
                if (!(last & kWinEndBit)) atomicAdd(&acc[last & kWinSlotMask], run);
            }
            __syncwarp();  // every lane is done with the stage and its adds
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    // hub slots of every warp into the hubs, in warp order
    if (threadIdx.x < kWinHubs) {
        const uint32_t h = a.whubs[(size_t)pd * kWinHubs + threadIdx.x];
        if (h < len) {
            float sum = 0.0f;
            for (uint32_t w = 0; w < (uint32_t)kWinWarps; ++w) sum += acc[a.q + w * kWinHubs + threadIdx.x];
            acc[h] += sum;
        }
    }
    static_assert(R::kBytes >= kWinScatterBars + scatter_table_bytes(PCPM_MAX_PARTITIONS) + 2 * (kWinThreads / 32) * 16 * 16,
                  "the fused scatter's stages must hold at least 16 groups beside the largest segment tables");
    gather_finish<kFused, kUpd, kWinThreads>(a, ring, R::kBytes, reinterpret_cast<uint64_t*>(ring),
                                             ring + kWinScatterBars, R::kBytes - kWinScatterBars, acc, sh32, S, rank,
                                             pd, npieces, vbase, len, pslot);
}

template <bool kFused, int kUpd, bool kW>
__global__ void __launch_bounds__(kWinThreads, 1) gather_win_kernel(const GatherArgs a) {
    gather_win_body<kFused, kUpd, kW>(a, blockIdx.x / cluster_size(), blockIdx.x);
}

// Many graphs in one launch (batched solves): item b / S of `items` names a
// graph (its arguments in tab) and one of its gather units; the CTA's partial
// sums go to that graph's slot unit * S + rank, as in its own launch.
template <bool kFused, int kUpd>
__global__ void __launch_bounds__(kWinThreads, 1) gather_win_batch_kernel(const GatherArgs* __restrict__ tab,
                                                                          const uint2* __restrict__ items) {
    const uint32_t S = cluster_size();
    const uint2 it = items[blockIdx.x / S];
    const GatherArgs a = tab[it.x];
    gather_win_body<kFused, kUpd, false>(a, it.y, it.y * S + cluster_rank());
}

// ---------------------------------------------------------------- reduce
__device__ __forceinline__ void reduce_body(const double* __restrict__ partials, int count, DevState* __restrict__ st,
                                            double* __restrict__ hist, int hist_slot, double tol);

__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(const double* __restrict__ partials, int count,
                                                                DevState* __restrict__ st, double* __restrict__ hist,
                                                                int hist_slot, double tol) {
    reduce_body(partials, count, st, hist, hist_slot, tol);
}

// The reduction of one graph of a batch; block b takes graph b.
struct ReduceArgs {
    const double* partials;
    int count;
    DevState* st;
    double* hist;
};
__global__ void __launch_bounds__(kReduceThreads) reduce_batch_kernel(const ReduceArgs* __restrict__ tab,
                                                                      int hist_slot) {
    const ReduceArgs a = tab[blockIdx.x];
    reduce_body(a.partials, a.count, a.st, a.hist, hist_slot, 0.0);
}

// A batch's reset, graph blockIdx.y: PR_0 = 1/n, the dangling mass of PR_0
// into the partials of its first gridDim.x blocks, the solver scalars zeroed,
// and the cut bins' global sums and counters cleared.
struct InitArgs {
    uint32_t n, k;
    const float* inv_deg;
    float* pr;
    double* partials;
    DevState* st;
    float* gacc;
    uint32_t* bin_done;
};
__global__ void __launch_bounds__(kReduceThreads) init_batch_kernel(const InitArgs* __restrict__ tab) {
    const InitArgs a = tab[blockIdx.y];
    const float uniform = (float)(1.0 / (double)a.n);
    double dang = 0.0, zero = 0.0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x) {
        a.pr[v] = uniform;
        a.gacc[v] = 0.0f;
        if (a.inv_deg[v] == 0.0f) dang += (double)uniform;
    }
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < a.k; p += gridDim.x * blockDim.x) a.bin_done[p] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->dangling = 0.0;
        a.st->residual = 0.0;
        a.st->stop = 0;
        a.st->iters_done = 0;
        a.st->err = 0;
        a.st->dangling_prev = 0.0;
    }
    block_sum2<kReduceThreads>(zero, dang);
    if (threadIdx.x == 0) {
        a.partials[2 * blockIdx.x] = 0.0;
        a.partials[2 * blockIdx.x + 1] = dang;
    }
}

__device__ __forceinline__ void reduce_body(const double* __restrict__ partials, int count, DevState* __restrict__ st,
                                            double* __restrict__ hist, int hist_slot, double tol) {
    if (st->stop) return;
    double r = 0.0, dg = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        r += partials[2 * i];
        dg += partials[2 * i + 1];
    }
    block_sum2<kReduceThreads>(r, dg);
    if (threadIdx.x == 0) {
        st->dangling_prev = st->dangling;
        st->dangling = dg;
        if (hist_slot >= 0) {
            st->residual = r;
            if (hist) hist[hist_slot] = r;
            st->iters_done += 1;
            if (tol > 0.0 && r < tol) st->stop = 1;
        }
    }
}

constexpr int kInitBlocks = 1024;

using GatherFn = void (*)(const GatherArgs);

// The gather instantiation for a layout and update type (the canonical bins
// hold FP32 updates only).
template <bool kFused>
GatherFn pick_gather(bool canonical, bool runs, int upd) {
    if (canonical) return gather_kernel<kFused, true, false, kUpdF32>;
    switch (upd) {
        case kUpdF16:
            return runs ? gather_kernel<kFused, false, true, kUpdF16> : gather_kernel<kFused, false, false, kUpdF16>;
        case kUpdBF16:
            return runs ? gather_kernel<kFused, false, true, kUpdBF16> : gather_kernel<kFused, false, false, kUpdBF16>;
        default:
            return runs ? gather_kernel<kFused, false, true, kUpdF32> : gather_kernel<kFused, false, false, kUpdF32>;
    }
}

template <bool kFused>
GatherFn pick_gather_win(int upd, bool weighted) {
    if (weighted) return gather_win_kernel<false, kUpdF32, true>;
    switch (upd) {
        case kUpdF16: return gather_win_kernel<kFused, kUpdF16, false>;
        case kUpdBF16: return gather_win_kernel<kFused, kUpdBF16, false>;
        default: return gather_win_kernel<kFused, kUpdF32, false>;
    }
}

// The window gather's shared memory: ring, barriers, q accumulator slots and
// the hub slots of every warp.
template <int kUpd, bool kW>
size_t gather_win_smem_bytes(uint32_t q) {
    return WinRing<kUpd, kW>::kAcc + (size_t)(((q + 3) & ~3u) + kWinWarps * kWinHubs) * sizeof(float);
}
size_t win_smem_bytes(uint32_t q, int upd, bool weighted) {
    if (weighted) return gather_win_smem_bytes<kUpdF32, true>(q);
    return upd == kUpdF32 ? gather_win_smem_bytes<kUpdF32, false>(q) : gather_win_smem_bytes<kUpdF16, false>(q);
}
static_assert(WinRing<kUpdF16, false>::kBytes == WinRing<kUpdBF16, false>::kBytes, "16-bit rings alike");

// The accumulator holds q real slots, kPadSlots for the layout's padding and
// kHubSlots (a pair per warp) for the hubs.
template <bool kW = false>
size_t gather_smem_bytes(uint32_t q) {
    return Ring<kW>::kAcc + (size_t)(((q + 3) & ~3u) + kPadSlots + kHubSlots) * sizeof(float);
}
static_assert(scatter_stage_bytes(PCPM_MAX_PART_SIZE, PCPM_MAX_PARTITIONS) >= 16 * 16,
              "the scatter's stages must hold at least 16 groups at the largest partition size and count");
size_t scatter_smem_bytes(uint32_t q, uint32_t k) {
    return (size_t)((q + 3) & ~3u) * sizeof(float) + scatter_table_bytes(k) +
           (size_t)2 * (kScatterThreads / 32) * scatter_stage_bytes(q, k);
}

}  // namespace

size_t partial_slots(const pcpm_png* g) {
    return std::max<size_t>((size_t)g->ngunits * kMaxCluster, (size_t)kInitBlocks);
}

// Picks the cluster size for the gather and sets shared-memory limits.
// The dynamic shared-memory limit is a property of the kernel, shared by every
// handle: only ever raise it, so a handle built later with a smaller q does
// not lower the limit an earlier handle's launches need.
std::mutex g_smem_attr_mutex;

cudaError_t raise_smem_limit(const void* f, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_smem_attr_mutex);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int configure_kernels(pcpm_png* g) {
    const size_t gs = gather_smem_bytes(g->q), ss = scatter_smem_bytes(g->q, g->k);
    const void* gathers[] = {
        (const void*)gather_kernel<false, true, false, kUpdF32>, (const void*)gather_kernel<true, true, false, kUpdF32>,
        (const void*)pick_gather<false>(false, false, kUpdF32), (const void*)pick_gather<true>(false, false, kUpdF32),
        (const void*)pick_gather<false>(false, true, kUpdF32),  (const void*)pick_gather<true>(false, true, kUpdF32),
        (const void*)pick_gather<false>(false, false, kUpdF16), (const void*)pick_gather<true>(false, false, kUpdF16),
        (const void*)pick_gather<false>(false, true, kUpdF16),  (const void*)pick_gather<true>(false, true, kUpdF16),
        (const void*)pick_gather<false>(false, false, kUpdBF16), (const void*)pick_gather<true>(false, false, kUpdBF16),
        (const void*)pick_gather<false>(false, true, kUpdBF16), (const void*)pick_gather<true>(false, true, kUpdBF16)};
    for (const void* f : gathers)
        if (const cudaError_t e = raise_smem_limit(f, gs); e != cudaSuccess) {
            note_cuda_error(e);
            return PCPM_ECUDA;
        }
    if (g->weighted) {  // weighted handles have q <= PCPM_MAX_WEIGHTED_PART_SIZE
        const size_t gw = gather_smem_bytes<true>(g->q);
        const void* wg[] = {(const void*)gather_kernel<false, false, false, kUpdF32, true>,
                            (const void*)gather_kernel<false, false, true, kUpdF32, true>};
        for (const void* f : wg)
            if (const cudaError_t e = raise_smem_limit(f, gw); e != cudaSuccess) {
                note_cuda_error(e);
                return PCPM_ECUDA;
            }
    }
    if (g->gather_windows) {
        const size_t ws = win_smem_bytes(g->q, g->upd_dtype, false);
        const void* wins[] = {(const void*)pick_gather_win<false>(g->upd_dtype, false),
                              (const void*)pick_gather_win<true>(g->upd_dtype, false)};
        for (const void* f : wins)
            if (const cudaError_t e = raise_smem_limit(f, ws); e != cudaSuccess) {
                note_cuda_error(e);
                return PCPM_ECUDA;
            }
        if (g->weighted)
            if (const cudaError_t e = raise_smem_limit((const void*)pick_gather_win<false>(kUpdF32, true),
                                                       win_smem_bytes(g->q, kUpdF32, true));
                e != cudaSuccess) {
                note_cuda_error(e);
                return PCPM_ECUDA;
            }
    }
    const void* scatters[] = {(const void*)scatter_kernel<kUpdF32>, (const void*)scatter_kernel<kUpdF16>,
                              (const void*)scatter_kernel<kUpdBF16>};
    for (const void* f : scatters)
        if (const cudaError_t e = raise_smem_limit(f, ss); e != cudaSuccess) {
            note_cuda_error(e);
            return PCPM_ECUDA;
        }
    // Two CTAs per gather unit unless the build options ask otherwise (two
    // measured best at k = 512 against one and four); smaller if the device
    // cannot co-schedule that many.
    const int want = g->cluster ? g->cluster : 2;
    for (int S = want; S >= 1; S /= 2) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = S;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(g->ngunits * S);
        cfg.blockDim = dim3(g->gather_windows ? kWinThreads : kGatherWarps * 32);
        cfg.dynamicSmemBytes = g->gather_windows ? win_smem_bytes(g->q, g->upd_dtype, false) : gs;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        const GatherFn probe = g->gather_windows ? pick_gather_win<true>(g->upd_dtype, false)
                                                 : gather_kernel<true, false, false, kUpdF32>;
        if (cudaOccupancyMaxActiveClusters(&clusters, probe, &cfg) == cudaSuccess && clusters > 0) {
            g->cluster = S;
            return PCPM_OK;
        }
        cudaGetLastError();
    }
    return PCPM_ECUDA;
}

int launch_init_range(pcpm_png* g, const float* pr_init, float* out, uint32_t lo, uint32_t hi, cudaStream_t s) {
    const int blocks = (int)std::min<uint64_t>(kInitBlocks, (g->n + kReduceThreads - 1) / kReduceThreads);
    init_kernel<<<blocks, kReduceThreads, 0, s>>>(g->n, pr_init, g->inv_deg, out, g->partials, lo, hi);
    g->partial_count = blocks;
    return launch_status();
}

__global__ void copy_pad_kernel(const float* __restrict__ x, uint32_t len, float* __restrict__ out, uint32_t n) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = v < len ? x[v] : 0.0f;
}

int launch_copy_pad(const float* x, uint32_t len, float* out, uint32_t n, cudaStream_t s) {
    copy_pad_kernel<<<(int)std::min<uint64_t>(4096, ((uint64_t)n + 255) / 256), 256, 0, s>>>(x, len, out, n);
    return launch_status();
}

int launch_init(pcpm_png* g, const float* pr_init, cudaStream_t s) {
    return launch_init_range(g, pr_init, g->pr[g->cur], 0, g->n, s);
}

int launch_spr(pcpm_png* g, float* spr, cudaStream_t s) {
    spr_kernel<<<(int)std::min<uint64_t>(4096, (g->n + 255) / 256), 256, 0, s>>>(g->n, g->pr[g->cur], g->inv_deg,
                                                                                  spr);
    return launch_status();
}

int launch_scatter(pcpm_png* g, cudaStream_t s, bool raw, bool delta, bool feedback) {
    feedback = feedback && g->dq_err && !raw;
    const size_t smem = scatter_smem_bytes(g->q, g->k);
    void (*f)(uint32_t, uint32_t, uint32_t, const float*, const float*, const uint32_t*, const uint16_t*,
              const uint32_t*,
              const uint32_t*, const uint4*, const uint32_t*, void*, const DevState*, int*, const float*,
              const float*, float*) =
        g->upd_dtype == kUpdF16 ? scatter_kernel<kUpdF16>
        : g->upd_dtype == kUpdBF16 ? scatter_kernel<kUpdBF16>
                                   : scatter_kernel<kUpdF32>;
    f<<<g->nsunits, kScatterThreads, smem, s>>>(g->n, g->q, g->k, g->pr[g->cur], raw ? nullptr : g->inv_deg, g->src,
                                               g->src16,
                                               g->seg_u,
                                               g->cnt_u, g->sunits, g->sorder, g->upd[g->ucur], g->state,
                                               &g->state->err, delta ? g->pr[g->cur ^ 1] : nullptr,
                                               feedback ? g->dq_err + (size_t)g->dq_cur * g->n : nullptr,
                                               feedback ? g->dq_err + (size_t)(g->dq_cur ^ 1) * g->n : nullptr);
    if (feedback) g->dq_cur ^= 1;
    return launch_status();
}

int launch_scatter_bits(pcpm_png* g, const void* x, void* out, cudaStream_t s) {
    if (g->upd_dtype != kUpdF32) return PCPM_EINVAL;
    scatter_kernel<kUpdF32><<<g->nsunits, kScatterThreads, scatter_smem_bytes(g->q, g->k), s>>>(
        g->n, g->q, g->k, static_cast<const float*>(x), nullptr, g->src, g->src16, g->seg_u, g->cnt_u, g->sunits,
        g->sorder,
        out, g->state, &g->state->err, nullptr, nullptr, nullptr);
    return launch_status();
}

namespace {
// The gather's arguments for the handle's ranks pr[cur] -> pr[cur ^ 1].
GatherArgs gather_args(pcpm_png* g, float d, uint32_t flags, bool delta, int cur, int ucur) {
    GatherArgs a;
    a.delta = delta ? 1 : 0;
    a.gweight = g->gweight;
    a.n = g->n;
    a.q = g->q;
    a.k = g->k;
    a.dest = g->dest;
    a.bin_e = g->bin_e;
    a.chunk_base = g->chunk_base;
    a.gdest = g->gdest;
    a.slice_start = g->gslice_start;
    a.slice_bytes = g->gslice_bytes;
    a.units = g->gunits;
    a.order = g->gorder;
    a.hubs = g->hubs;
    a.gacc = g->gacc;
    a.bin_done = g->bin_done;
    a.upd_in = g->upd[ucur];
    a.pr_in = g->pr[cur];
    a.inv_deg = g->inv_deg;
    a.pr_out = g->pr[cur ^ 1];
    a.partials = g->partials;
    a.st = g->state;
    a.err = &g->state->err;
    a.d = d;
    a.uniform_dangling = (flags & PCPM_DANGLING_LEAK) ? 0 : 1;
    a.src = g->src;
    a.seg_u = g->seg_u;
    a.cnt_u = g->cnt_u;
    a.upd_out = g->upd[ucur ^ 1];
    a.wwords = g->wwords;
    a.wweight = g->wweight;
    a.wdesc = g->wdesc;
    a.whubs = g->whubs;
    return a;
}
}  // namespace

int launch_gather(pcpm_png* g, float d, uint32_t flags, bool fused, cudaStream_t s, bool spmv, bool delta) {
    const bool weighted = spmv && g->weighted;  // only SpMV applies the weights
    const GatherArgs a = gather_args(g, d, flags, delta, g->cur, g->ucur);

    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g->cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(g->ngunits * g->cluster);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    GatherFn f;
    if (g->gather_windows) {
        cfg.blockDim = dim3(kWinThreads);
        cfg.dynamicSmemBytes = win_smem_bytes(g->q, weighted ? kUpdF32 : g->upd_dtype, weighted);
        f = weighted ? pick_gather_win<false>(kUpdF32, true)
            : fused  ? pick_gather_win<true>(g->upd_dtype, false)
                     : pick_gather_win<false>(g->upd_dtype, false);
    } else {
        cfg.blockDim = dim3(kGatherWarps * 32);
        cfg.dynamicSmemBytes = weighted ? gather_smem_bytes<true>(g->q) : gather_smem_bytes(g->q);
        f = weighted ? (g->gather_runs ? gather_kernel<false, false, true, kUpdF32, true>
                                       : gather_kernel<false, false, false, kUpdF32, true>)
            : fused  ? pick_gather<true>(g->canonical_gather != 0, g->gather_runs != 0, g->upd_dtype)
                     : pick_gather<false>(g->canonical_gather != 0, g->gather_runs != 0, g->upd_dtype);
    }
    e = cudaLaunchKernelEx(&cfg, f, a);
    g->partial_count = (int)(g->ngunits * g->cluster);
    if (e != cudaSuccess) note_cuda_error(e);
    return e == cudaSuccess ? PCPM_OK : PCPM_ECUDA;
}

int set_work_wait_limit(long long cycles) {
    const long long v = cycles == 0 ? kWaitLimitCycles : cycles;
    const cudaError_t e = cudaMemcpyToSymbol(g_work_wait_limit, &v, sizeof(v));
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return PCPM_ECUDA;
    }
    return PCPM_OK;
}

int launch_reduce(pcpm_png* g, double tol, int hist_slot, cudaStream_t s, bool record) {
    reduce_kernel<<<1, kReduceThreads, 0, s>>>(g->partials, g->partial_count, g->state, record ? g->hist : nullptr,
                                               hist_slot, tol);
    return launch_status();
}

}  // namespace pcpm

// ------------------------------------------------------------ batch kernels
namespace pcpm {

struct BatchKernels {
    struct Group {
        int count = 0;
        int S = 1;
        int upd = kUpdF32;
        size_t gsmem = 0, ssmem = 0;
        GatherArgs* gtab = nullptr;   // [2][count]: from pr[0] and from pr[1]
        ScatterArgs* stab = nullptr;  // [2][count]
        ReduceArgs* rtab = nullptr;   // [count] after an iteration
        ReduceArgs* rtab0 = nullptr;  // [count] after the reset (init partials)
        InitArgs* itab = nullptr;     // [count]
        uint2* gitems = nullptr;
        uint32_t ngitems = 0;
        uint2* sitems = nullptr;
        uint32_t nsitems = 0;
        int init_blocks = 1;
    };
    std::vector<Group> groups;
    std::vector<void*> allocs;
    bool fused = false;  // gather + apply + next scatter per iteration
};

bool batch_kernels_ok(pcpm_png* const* hs, int count, uint32_t flags) {
    if ((flags & PCPM_DELTA) || count > 65535) return false;
    const bool fused = !(flags & PCPM_TWO_PHASE);
    for (int i = 0; i < count; ++i) {
        const pcpm_png* g = hs[i];
        if (!g->gather_windows || g->weighted || g->rect || g->plo != 0 || g->phi != g->k || (fused && !g->fused_ok))
            return false;
    }
    return true;
}

bool batch_kernels_fused(const BatchKernels* b) { return b->fused; }

namespace {
using BatchGatherFn = void (*)(const GatherArgs*, const uint2*);
using BatchScatterFn = void (*)(const ScatterArgs*, const uint2*);
template <bool kFused>
BatchGatherFn pick_batch_gather(int upd) {
    return upd == kUpdF16    ? gather_win_batch_kernel<kFused, kUpdF16>
           : upd == kUpdBF16 ? gather_win_batch_kernel<kFused, kUpdBF16>
                             : gather_win_batch_kernel<kFused, kUpdF32>;
}
BatchScatterFn pick_batch_scatter(int upd) {
    return upd == kUpdF16    ? scatter_batch_kernel<kUpdF16>
           : upd == kUpdBF16 ? scatter_batch_kernel<kUpdBF16>
                             : scatter_batch_kernel<kUpdF32>;
}
}  // namespace

void batch_kernels_free(BatchKernels* b) {
    if (!b) return;
    for (void* p : b->allocs) pool_free(p, nullptr);
    delete b;
}

namespace {
template <class T>
int upload(BatchKernels* b, const std::vector<T>& host, T** dev, cudaStream_t s) {
    void* p = nullptr;
    cudaError_t e = pool_alloc(&p, std::max<size_t>(host.size(), 1) * sizeof(T), s);
    if (e == cudaSuccess) {
        b->allocs.push_back(p);
        if (!host.empty()) e = cudaMemcpyAsync(p, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? PCPM_ENOMEM : PCPM_ECUDA;
    }
    *dev = static_cast<T*>(p);
    return PCPM_OK;
}

// (graph, position in its order) of every unit, largest first
int batch_items(const std::vector<pcpm_png*>& gs, bool gather, std::vector<uint2>& items, cudaStream_t s) {
    std::vector<std::pair<uint32_t, uint2>> all;
    for (size_t j = 0; j < gs.size(); ++j) {
        pcpm_png* g = gs[j];
        const uint32_t nu = gather ? g->ngunits : g->nsunits;
        std::vector<uint4> units(nu);
        std::vector<uint32_t> order(nu);
        cudaError_t e = cudaMemcpyAsync(units.data(), gather ? g->gunits : g->sunits, nu * sizeof(uint4),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(order.data(), gather ? g->gorder : g->sorder, nu * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            note_cuda_error(e);
            return PCPM_ECUDA;
        }
        for (uint32_t r = 0; r < nu; ++r) {
            const uint4 u = units[order[r]];
            all.push_back({u.z - u.y, make_uint2((uint32_t)j, r)});
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    items.clear();
    for (const auto& x : all) items.push_back(x.second);
    return PCPM_OK;
}
}  // namespace

int batch_kernels_create(pcpm_png* const* hs, int count, float d, uint32_t flags, double* hist, int iters,
                         cudaStream_t s, BatchKernels** out) {
    BatchKernels* b = new (std::nothrow) BatchKernels;
    if (!b) return PCPM_ENOMEM;
    b->fused = !(flags & PCPM_TWO_PHASE);
    // one group per (part size, cluster size, bin format): the launch's
    // shared memory follows q, its cluster dimension the handle's CTAs per
    // gather unit, its instantiation the bins' format
    std::vector<uint3> keys;
    for (int i = 0; i < count; ++i) {
        const uint3 key = make_uint3(hs[i]->q, (uint32_t)hs[i]->cluster, (uint32_t)hs[i]->upd_dtype);
        if (std::find_if(keys.begin(), keys.end(), [&](const uint3& x) {
                return x.x == key.x && x.y == key.y && x.z == key.z;
            }) == keys.end())
            keys.push_back(key);
    }
    int rc = PCPM_OK;
    for (const auto& key : keys) {
        const uint32_t q = key.x;
        std::vector<pcpm_png*> gs;
        std::vector<int> idx;  // position in hs: the graph's history rows
        for (int i = 0; i < count; ++i)
            if (hs[i]->q == q && (uint32_t)hs[i]->cluster == key.y && (uint32_t)hs[i]->upd_dtype == key.z) {
                gs.push_back(hs[i]);
                idx.push_back(i);
            }
        BatchKernels::Group G;
        G.count = (int)gs.size();
        G.S = gs[0]->cluster;
        G.upd = gs[0]->upd_dtype;
        G.gsmem = win_smem_bytes(q, G.upd, false);
        uint32_t nmax = 0;
        std::vector<GatherArgs> gt(2 * gs.size());
        std::vector<ScatterArgs> st(2 * gs.size());
        std::vector<ReduceArgs> rt(gs.size()), rt0(gs.size());
        std::vector<InitArgs> it(gs.size());
        for (size_t j = 0; j < gs.size(); ++j) {
            pcpm_png* g = gs[j];
            G.ssmem = std::max(G.ssmem, scatter_smem_bytes(q, g->k));
            nmax = std::max(nmax, g->n);
            for (int c = 0; c < 2; ++c) {
                // iteration i reads pr[i & 1]; the fused form also swaps the
                // update buffers every iteration
                const int u = b->fused ? g->ucur ^ c : g->ucur;
                gt[c * gs.size() + j] = gather_args(g, d, flags, false, c, u);
                ScatterArgs& a = st[c * gs.size() + j];
                a = ScatterArgs{g->n, g->q, g->k, g->pr[c], g->inv_deg, g->src, g->src16, g->seg_u, g->cnt_u, g->sunits,
                                g->sorder, g->upd[u], g->state, &g->state->err};
            }
            rt[j] = ReduceArgs{g->partials, (int)(g->ngunits * g->cluster), g->state, hist + (size_t)idx[j] * iters};
            it[j] = InitArgs{g->n, g->k, g->inv_deg, g->pr[0], g->partials, g->state, g->gacc, g->bin_done};
        }
        G.init_blocks = (int)std::min<uint64_t>(kInitBlocks, ((uint64_t)nmax + kReduceThreads - 1) / kReduceThreads);
        for (size_t j = 0; j < gs.size(); ++j) rt0[j] = ReduceArgs{gs[j]->partials, G.init_blocks, gs[j]->state, nullptr};
        std::vector<uint2> gi, si;
        if (rc == PCPM_OK) rc = batch_items(gs, true, gi, s);
        if (rc == PCPM_OK) rc = batch_items(gs, false, si, s);
        if (rc == PCPM_OK) rc = upload(b, gt, &G.gtab, s);
        if (rc == PCPM_OK) rc = upload(b, st, &G.stab, s);
        if (rc == PCPM_OK) rc = upload(b, rt, &G.rtab, s);
        if (rc == PCPM_OK) rc = upload(b, rt0, &G.rtab0, s);
        if (rc == PCPM_OK) rc = upload(b, it, &G.itab, s);
        if (rc == PCPM_OK) rc = upload(b, gi, &G.gitems, s);
        if (rc == PCPM_OK) rc = upload(b, si, &G.sitems, s);
        G.ngitems = (uint32_t)gi.size();
        G.nsitems = (uint32_t)si.size();
        if (rc == PCPM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = PCPM_ECUDA;  // host tables go out of scope
        if (rc == PCPM_OK) {
            const void* gf = b->fused ? (const void*)pick_batch_gather<true>(G.upd)
                                      : (const void*)pick_batch_gather<false>(G.upd);
            cudaError_t e = raise_smem_limit(gf, G.gsmem);
            if (e == cudaSuccess) e = raise_smem_limit((const void*)pick_batch_scatter(G.upd), G.ssmem);
            if (e != cudaSuccess) {
                note_cuda_error(e);
                rc = PCPM_ECUDA;
            }
        }
        if (rc != PCPM_OK) break;
        b->groups.push_back(G);
    }
    if (rc != PCPM_OK) {
        cudaStreamSynchronize(s);
        batch_kernels_free(b);
        return rc;
    }
    *out = b;
    return PCPM_OK;
}

int batch_kernels_groups(const BatchKernels* b) { return (int)b->groups.size(); }

// The reset and `iters` iterations of every graph, one launch per phase and
// group; group i on streams[i % nstreams]. Two-phase: scatter, gather,
// reduce per iteration. Fused: one scatter, then gather (with the next
// iteration's scatter) and reduce per iteration.
int batch_kernels_record(BatchKernels* b, int iters, const cudaStream_t* streams, int nstreams) {
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const auto& G = b->groups[gi];
        cudaStream_t s = streams[gi % nstreams];
        init_batch_kernel<<<dim3(G.init_blocks, G.count), kReduceThreads, 0, s>>>(G.itab);
        reduce_batch_kernel<<<G.count, kReduceThreads, 0, s>>>(G.rtab0, -1);
        const BatchScatterFn sf = pick_batch_scatter(G.upd);
        const BatchGatherFn gf = b->fused ? pick_batch_gather<true>(G.upd) : pick_batch_gather<false>(G.upd);
        for (int i = 0; i < iters; ++i) {
            const int c = i & 1;
            if (G.nsitems && (!b->fused || i == 0))
                sf<<<G.nsitems, kScatterThreads, G.ssmem, s>>>(G.stab + (size_t)c * G.count, G.sitems);
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = G.S;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(G.ngitems * G.S);
            cfg.blockDim = dim3(kWinThreads);
            cfg.dynamicSmemBytes = G.gsmem;
            cfg.stream = s;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const cudaError_t e =
                G.ngitems ? cudaLaunchKernelEx(&cfg, gf, (const GatherArgs*)(G.gtab + (size_t)c * G.count),
                                               (const uint2*)G.gitems)
                          : cudaSuccess;
            if (e != cudaSuccess) {
                note_cuda_error(e);
                return PCPM_ECUDA;
            }
            reduce_batch_kernel<<<G.count, kReduceThreads, 0, s>>>(G.rtab, i);
        }
        const int rc = launch_status();
        if (rc != PCPM_OK) return rc;
    }
    return PCPM_OK;
}

}  // namespace pcpm

namespace pcpm {
namespace {
// Row i of the batch's history (iters values) to dst[i].
__global__ void hist_copy_kernel(const double* __restrict__ src, double* const* __restrict__ dst, int iters,
                                 int count) {
    for (int i = blockIdx.x; i < count; i += gridDim.x)
        for (int t = threadIdx.x; t < iters; t += blockDim.x) dst[i][t] = src[(size_t)i * iters + t];
}
}  // namespace

int launch_hist_copy(const double* src, double* const* dst, int iters, int count, cudaStream_t s) {
    hist_copy_kernel<<<std::min(count, 1024), 128, 0, s>>>(src, dst, iters, count);
    return launch_status();
}
}  // namespace pcpm
