// Device helpers of the sampled-gradient kernels: Philox4x64-10 draws,
// randi, the elementwise losses, BF16 row loads and the status word.
//
// Written for sm_103a.  Shares nothing with any other implementation of the
// same conventions; the conventions themselves are stated in include/gcp.h.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/gcp.h"

namespace gcpk {

constexpr int kMaxModes = GCP_MAX_MODES;

// Philox tags (the third counter word)
constexpr uint64_t kTagUniform = 0, kTagNonzero = 1, kTagZeroCandidate = 2, kTagSemiZero = 3, kTagObserved = 4;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies, key bumped by
// the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U64x4 {
    uint64_t w[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kMul0 = 0xD2E7470EE14C6C93ull;
    constexpr uint64_t kMul1 = 0xCA5A826395121157ull;
    constexpr uint64_t kWeyl0 = 0x9E3779B97F4A7C15ull;
    constexpr uint64_t kWeyl1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(kMul0, c0), lo0 = kMul0 * c0;
        const uint64_t hi1 = __umul64hi(kMul1, c2), lo1 = kMul1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    return U64x4{{c0, c1, c2, c3}};
}

// randi(n), 0-based: the high word of word * n.
__device__ __forceinline__ uint32_t randi32(uint64_t word, uint64_t n)
{
    return static_cast<uint32_t>(__umul64hi(word, n));
}
__device__ __forceinline__ uint64_t randi64(uint64_t word, uint64_t n) { return __umul64hi(word, n); }

// The D mode indices of draw j in one sampling stream.
template <int D>
__device__ __forceinline__ void draw_index(const uint32_t* __restrict__ dims, uint64_t seed, uint64_t problem,
                                           uint64_t stream, uint64_t tag, uint64_t j, int d_rt,
                                           uint32_t (&ix)[D])
{
    if constexpr (D <= 4) {
        const U64x4 b = philox4x64_10(j, stream, tag, 0, seed, problem);
#pragma unroll
        for (int k = 0; k < D; ++k) ix[k] = randi32(b.w[k], dims[k]);
    } else {
        U64x4 b = philox4x64_10(j, stream, tag, 0, seed, problem);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k == 4 && d_rt > 4) b = philox4x64_10(j, stream, tag, 1, seed, problem);
            ix[k] = k < d_rt ? randi32(b.w[k & 3], dims[k]) : 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Losses: f(x,m) and g(x,m) = df/dm, FP32.
// ---------------------------------------------------------------------------
constexpr float kMEps = 1e-10f;  // odds/identity-link losses are evaluated at m + kMEps

__device__ __forceinline__ float loss_g(int loss, float x, float m)
{
    switch (loss) {
    case GCP_LOSS_GAUSSIAN: return 2.0f * (m - x);
    case GCP_LOSS_BERNOULLI_LOGIT: return 1.0f / (1.0f + expf(-m)) - x;
    case GCP_LOSS_POISSON_LOG: return expf(m) - x;
    case GCP_LOSS_BERNOULLI_ODDS: {
        const float mp = m + kMEps;
        return 1.0f / (mp + 1.0f) - x / mp;
    }
    case GCP_LOSS_POISSON_IDENTITY: return 1.0f - x / (m + kMEps);
    case GCP_LOSS_GAMMA: {
        const float mp = m + kMEps;
        return -x / (mp * mp) + 1.0f / mp;
    }
    default: {  // GCP_LOSS_BETA_HALF
        const float mp = m + kMEps;
        const float r = rsqrtf(mp);
        return r - x * r / mp;
    }
    }
}

__device__ __forceinline__ float loss_f(int loss, float x, float m)
{
    switch (loss) {
    case GCP_LOSS_GAUSSIAN: {
        const float r = x - m;
        return r * r;
    }
    case GCP_LOSS_BERNOULLI_LOGIT: return fmaxf(m, 0.0f) + log1pf(expf(-fabsf(m))) - x * m;
    case GCP_LOSS_POISSON_LOG: return expf(m) - x * m;
    case GCP_LOSS_BERNOULLI_ODDS: {
        const float mp = m + kMEps;
        return log1pf(mp) - x * logf(mp);
    }
    case GCP_LOSS_POISSON_IDENTITY: {
        const float mp = m + kMEps;
        return mp - x * logf(mp);
    }
    case GCP_LOSS_GAMMA: {
        const float mp = m + kMEps;
        return x / mp + logf(mp);
    }
    default: {  // GCP_LOSS_BETA_HALF
        const float mp = m + kMEps;
        return 2.0f * sqrtf(mp) + 2.0f * x * rsqrtf(mp);
    }
    }
}

// y of a drawn entry: the semi-stratified nonzero subtracts the x = 0 term
// (Alg. 3).  For the log-link losses the m-dependent parts of g(x,m) and
// g(0,m) are identical and cancel exactly: g(x,m) - g(0,m) = -2x (Gaussian)
// or -x (Bernoulli-logit, Poisson-log); that difference is taken in closed
// form, without evaluating the link twice and subtracting in FP32.
__device__ __forceinline__ float entry_y(int loss, int cls, float x, float m, float w)
{
    if (cls == GCP_CLS_SEMI_NZ) {
        switch (loss) {
        case GCP_LOSS_GAUSSIAN: return w * (-2.0f * x);
        case GCP_LOSS_BERNOULLI_LOGIT:
        case GCP_LOSS_POISSON_LOG: return w * -x;
        default: return w * (loss_g(loss, x, m) - loss_g(loss, 0.0f, m));
        }
    }
    return w * loss_g(loss, x, m);
}

// The F-hat term of a drawn entry, with the same closed forms for the
// semi-stratified nonzero: f(x,m) - f(0,m) = x^2 - 2xm (Gaussian) or -xm
// (Bernoulli-logit, Poisson-log).
__device__ __forceinline__ float entry_f(int loss, int cls, float x, float m, float w)
{
    if (cls == GCP_CLS_SEMI_NZ) {
        switch (loss) {
        case GCP_LOSS_GAUSSIAN: return w * (x * x - 2.0f * x * m);
        case GCP_LOSS_BERNOULLI_LOGIT:
        case GCP_LOSS_POISSON_LOG: return w * -(x * m);
        default: return w * (loss_f(loss, x, m) - loss_f(loss, 0.0f, m));
        }
    }
    return w * loss_f(loss, x, m);
}

// ---------------------------------------------------------------------------
// Row loads: 4 consecutive factor entries as float4 from FP32 (16 B) or
// BF16 (8 B) storage.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 load4(const float* __restrict__ p)
{
    return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ float4 load4(const __nv_bfloat16* __restrict__ p)
{
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    float4 out;
    out.x = __uint_as_float(raw.x << 16);
    out.y = __uint_as_float(raw.x & 0xFFFF0000u);
    out.z = __uint_as_float(raw.y << 16);
    out.w = __uint_as_float(raw.y & 0xFFFF0000u);
    return out;
}

// G_k(i, cols) += v: one 16-byte reduction performed at L2 (red, no value
// returned to the thread; relaxed, GPU scope).  Needs a 16-byte aligned address.
__device__ __forceinline__ void red_add4(float* p, const float4 v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Asynchronous global -> shared copies (cp.async): a thread's own copies are
// complete and visible to it after cp_async_wait_all().
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src)
{
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
}

// 4 factor entries staged in shared memory: float4 (FP32 rows) or 4 BF16 (8 bytes).
__device__ __forceinline__ float4 staged4(const float4* p) { return *p; }
__device__ __forceinline__ float4 staged4(const uint2* p)
{
    const uint2 raw = *p;
    float4 out;
    out.x = __uint_as_float(raw.x << 16);
    out.y = __uint_as_float(raw.x & 0xFFFF0000u);
    out.z = __uint_as_float(raw.y << 16);
    out.w = __uint_as_float(raw.y & 0xFFFF0000u);
    return out;
}

__device__ __forceinline__ float4 mul4(float4 a, float4 b)
{
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 scale4(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
__device__ __forceinline__ float sum4(float4 a) { return (a.x + a.y) + (a.z + a.w); }
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

// Sum of reps replica chunks r[0], r[stride], ... (each then zeroed), added
// in replica order, in rounds of 16: every load of a round is issued before
// any is used, so a fold costs one round trip to L2 per 16 replicas.
__device__ __forceinline__ float4 fold_replicas(float4* r, uint32_t reps, uint64_t stride)
{
    constexpr int kWide = 16;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 acc = zero;
#pragma unroll 1
    for (uint32_t q0 = 0; q0 < reps; q0 += kWide) {
        float4 v[kWide];
#pragma unroll
        for (int q = 0; q < kWide; ++q) v[q] = q0 + q < reps ? r[(q0 + q) * stride] : zero;
#pragma unroll
        for (int q = 0; q < kWide; ++q) acc = add4(acc, v[q]);
#pragma unroll
        for (int q = 0; q < kWide; ++q)
            if (q0 + q < reps) r[(q0 + q) * stride] = zero;
    }
    return acc;
}

// Cluster barrier halves (all threads of every block of the cluster): arrive
// releases this thread's earlier memory accesses, wait acquires everyone's.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialization attribute may begin while its predecessor in the
// stream is still running; pdl_wait() blocks until that predecessor has
// completed and its writes are visible (a no-op after a normal launch), and
// pdl_trigger() lets the successor begin launching.  Every kernel of the path
// calls pdl_wait() before pdl_trigger(), so when a kernel starts, the kernel
// two launches before it has completed.  Every kernel calls pdl_wait() before
// its first global-memory access, with two exceptions, both reading only
// data written at least two launches back: the gradient kernel's early
// descriptors (the data tensor, the handle's nonzero tables) and the fused
// Adam step's first element (A, B, C, alpha and the done flag).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Sticky status word: keep the first error.
__device__ __forceinline__ void set_status(int32_t* status, int32_t code)
{
    if (status) atomicCAS(status, 0, code);
}

}  // namespace gcpk
