// The elementwise Adam step of Alg. 4 on the float4 chunks of all modes,
// with the replica slabs of the gradient folded in, as device functions (the
// Adam kernels of gcp_adam.cu).
//
// Layout: kParts lanes per float4 element; lane p of an element's group adds
// replicas p, p + kParts, ... (all its loads in flight at once) and zeroes
// them, the group sums its partials with shuffles in a fixed order, and lane
// 0 applies the update to A, B, C (and the BF16 copy) and zeroes G.
#pragma once

#include <cuda_bf16.h>

#include "gcp_device.cuh"
#include "gcp_kernels.cuh"

namespace gcpk {

constexpr int kParts = 4;

__device__ __forceinline__ int mode_of(const ModeTable& mt, int64_t i4)
{
    int k = 0;
#pragma unroll
    for (int l = 1; l < GCP_MAX_MODES; ++l)
        if (l < mt.d && i4 >= mt.off4[l]) k = l;
    return k;
}

__device__ __forceinline__ void store_bf16x4(uint16_t* dst, float4 v)
{
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v.x), b1 = __float2bfloat16_rn(v.y);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(v.z), b3 = __float2bfloat16_rn(v.w);
    uint2 packed;
    packed.x = static_cast<uint32_t>(__bfloat16_as_ushort(b0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(b1)) << 16);
    packed.y = static_cast<uint32_t>(__bfloat16_as_ushort(b2)) | (static_cast<uint32_t>(__bfloat16_as_ushort(b3)) << 16);
    *reinterpret_cast<uint2*>(dst) = packed;
}

// One entry of the Adam step with the bias corrections given as reciprocals
// (ic1 = 1 / (1 - beta1^n), ic2 = 1 / (1 - beta2^n)).  The step bh / den is
// taken with the hardware reciprocal square root (eps inside the root) or
// the fast division (eps outside): a few FP32 ulps of the step, far below
// the FP32 rounding of the factor itself for any alpha < 1.
__device__ __forceinline__ float adam_one(float& a, float& b, float& c, float g, float beta1, float beta2,
                                          float ic1, float ic2, float eps, float alpha, float lower, bool inside)
{
    b = beta1 * b + (1.0f - beta1) * g;
    c = beta2 * c + (1.0f - beta2) * (g * g);
    const float bh = b * ic1;
    const float ch = c * ic2;
    const float step = inside ? bh * rsqrtf(ch + eps) : __fdividef(bh, sqrtf(ch) + eps);
    a = fmaxf(a - alpha * step, lower);
    return a;
}

// 1 / (1 - beta^n) = 1 / -expm1(n log1p(beta - 1)): accurate to a few FP32
// ulps even for beta near 1 and small n, where 1 - powf(beta, n) would cancel.
__device__ __forceinline__ float inv_bias_correction(float beta, float n)
{
    return 1.0f / -expm1f(n * log1pf(beta - 1.0f));
}

// An element's mode, position and its A, B, C (lane 0 of the group only).
struct AdamElem {
    int k;
    uint32_t loc;
    float4 A4, B4, C4;
};

__device__ __forceinline__ void adam_prepare(const AdamArgs& a, uint32_t i4, uint32_t total4, uint32_t part,
                                             AdamElem& e)
{
    e.k = 0;
    e.loc = 0;
    e.A4 = e.B4 = e.C4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i4 >= total4) return;
    const ModeTable& mt = a.mt;
    e.k = mode_of(mt, i4);
    e.loc = i4 - static_cast<uint32_t>(mt.off4[e.k]);
    if (part == 0) {
        e.A4 = reinterpret_cast<const float4*>(mt.A[e.k])[e.loc];
        e.B4 = reinterpret_cast<const float4*>(mt.B[e.k])[e.loc];
        e.C4 = reinterpret_cast<const float4*>(mt.C[e.k])[e.loc];
    }
}

// Folds, updates and clears element e.  Every lane of the warp calls it
// together (the group sum uses full-warp shuffles); live says whether the
// lane's element exists.
__device__ __forceinline__ void adam_finish(const AdamArgs& a, bool live, uint32_t part, AdamElem& e, float ic1,
                                            float ic2, float alpha, int done)
{
    const ModeTable& mt = a.mt;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 g = acc;
    if (live) {
        if (part == 0) g = reinterpret_cast<const float4*>(mt.G[e.k])[e.loc];
        const uint32_t reps = a.reps[e.k] > 1 ? a.reps[e.k] : 0;
        float4* r = reinterpret_cast<float4*>(a.R[e.k]) + e.loc;
        const uint64_t rs = a.rep_stride4[e.k];
        constexpr int kWide = 8;  // per lane: replicas part, part + kParts, ... (up to 32 in flight per group)
        float4 v[kWide];
#pragma unroll
        for (int q = 0; q < kWide; ++q) {
            const uint32_t rep = part + static_cast<uint32_t>(q) * kParts;
            v[q] = rep < reps ? r[rep * rs] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < kWide; ++q) acc = add4(acc, v[q]);
#pragma unroll
        for (int q = 0; q < kWide; ++q) {
            const uint32_t rep = part + static_cast<uint32_t>(q) * kParts;
            if (rep < reps) r[rep * rs] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (uint32_t rep = part + kWide * kParts; rep < reps; rep += kParts) {
            acc = add4(acc, r[rep * rs]);
            r[rep * rs] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // the group's partial sums: lane 0 ends with ((p0 + p1) + (p2 + p3))
#pragma unroll
    for (int off = 1; off < kParts; off <<= 1) {
        acc.x += __shfl_xor_sync(0xFFFFFFFFu, acc.x, off);
        acc.y += __shfl_xor_sync(0xFFFFFFFFu, acc.y, off);
        acc.z += __shfl_xor_sync(0xFFFFFFFFu, acc.z, off);
        acc.w += __shfl_xor_sync(0xFFFFFFFFu, acc.w, off);
    }
    if (!live || part != 0) return;
    g = add4(g, acc);
    const uint32_t ld4 = static_cast<uint32_t>(mt.ld) / 4;
    const int col = static_cast<int>((e.loc % ld4) * 4);
    const bool inside = a.eps_inside_sqrt != 0;
    if (!done && col < mt.rank) {
        const int ncol = mt.rank - col;  // columns of this chunk below rank
        float4& A4 = e.A4;
        float4& B4 = e.B4;
        float4& C4 = e.C4;
        adam_one(A4.x, B4.x, C4.x, g.x, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
        if (ncol > 1) adam_one(A4.y, B4.y, C4.y, g.y, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
        if (ncol > 2) adam_one(A4.z, B4.z, C4.z, g.z, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
        if (ncol > 3) adam_one(A4.w, B4.w, C4.w, g.w, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
        reinterpret_cast<float4*>(mt.A[e.k])[e.loc] = A4;
        reinterpret_cast<float4*>(mt.B[e.k])[e.loc] = B4;
        reinterpret_cast<float4*>(mt.C[e.k])[e.loc] = C4;
        if (mt.Abf[e.k]) store_bf16x4(mt.Abf[e.k] + static_cast<size_t>(e.loc) * 4, A4);
    }
    reinterpret_cast<float4*>(mt.G[e.k])[e.loc] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// The step over all elements for the threads [gthread0 .. gthread0 + nthreads)
// of a launch (kParts per element, a warp-uniform trip count), with the
// calling thread's first element already prepared in `first`.  t, alpha and
// done are the step's scalars (t already advanced for this step).
__device__ __forceinline__ void adam_elements(const AdamArgs& a, uint32_t gthread, uint32_t nthreads,
                                              AdamElem& first, int64_t t, float alpha, int done)
{
    const uint32_t total4 = static_cast<uint32_t>(a.mt.off4[a.mt.d]);
    const float n = static_cast<float>(t);
    const float ic1 = inv_bias_correction(a.beta1, n);
    const float ic2 = inv_bias_correction(a.beta2, n);
    const uint32_t part = gthread % kParts;
    const uint32_t stride = nthreads / kParts;
    const uint32_t i0 = gthread / kParts;
    const uint32_t w0 = (gthread & ~31u) / kParts;
    for (uint32_t w4 = w0, i4 = i0; w4 < total4; w4 += stride, i4 += stride) {
        if (i4 != i0) adam_prepare(a, i4, total4, part, first);
        adam_finish(a, i4 < total4, part, first, ic1, ic2, alpha, done);
    }
}

}  // namespace gcpk
