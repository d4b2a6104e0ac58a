// Batched form: many independent GCP-Adam problems (uneven shapes, ranks and
// losses) advanced together.  Each step is one launch for all problems:
//   batch_fused_kernel -- a whole iteration (gradient and Adam step) of every
//                         problem in one persistent launch, or, in two:
//   batch_grad_kernel  -- the fused sampled gradient (Alg. 1) of every problem;
//                         warps take 32 consecutive draws of one problem at a
//                         time from the flattened table of all problems' draws;
//   batch_adam_kernel  -- Adam with projection (Alg. 4) over every problem's
//                         parameters;
//   batch_loss_kernel  -- every problem's fixed-sample F-hat (FP64 sums);
//   batch_epoch_kernel -- every problem's epoch accept / revert.
// The per-problem arithmetic is that of the single-problem kernels; lanes per
// draw and chunks per lane are chosen per problem from its rank at run time.
// A mode whose rows each receive many updates per iteration spreads them over
// replica slabs (warp u adds into replica u mod R), which the Adam kernel
// folds into G and clears, as the single-problem gcp_iteration does.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "gcp_adam_phase.cuh"
#include "gcp_device.cuh"
#include "gcp_kernels.cuh"

namespace gcpk {

constexpr int kBatchMaxD = 4;

struct BatchDesc {
    int32_t d, ld, rank, loss;
    int32_t L, NC, bf16, pad;
    uint32_t dims[kBatchMaxD];
    uint64_t strides[kBatchMaxD];
    const float* X;
    const void* Ag[kBatchMaxD];  // gather source (FP32 master or BF16 copy)
    float* A[kBatchMaxD];
    uint16_t* Abf[kBatchMaxD];
    float* G[kBatchMaxD];
    float* B[kBatchMaxD];
    float* C[kBatchMaxD];
    float* SA[kBatchMaxD];
    float* SB[kBatchMaxD];
    float* SC[kBatchMaxD];
    float* R[kBatchMaxD];          // replica slabs of mode k (reps[k] > 1), kept zero between iterations
    uint32_t reps[kBatchMaxD];
    uint64_t rep_stride[kBatchMaxD];  // floats between replicas: n_k * ld
    int64_t off4[kBatchMaxD + 1];  // float4 prefix of the problem's modes
    uint64_t seed, problem;
    int64_t s;
    float w;  // omega / s
    float beta1, beta2, eps, lower;
    int32_t eps_inside, kappa;
    float nu;
    int64_t tau;
    gcp_adam_state* st;
    const int32_t* lidx[kBatchMaxD];
    const float* lx;
    const float* lw;
    const int8_t* lcls;
    int64_t n_est;
};

struct BatchArgs {
    const BatchDesc* desc;
    int32_t count;
    int32_t begin;                  // epoch kernel: 1 = begin (snapshot only)
    const int64_t* work_begin;      // prefix of 32-draw warp batches, count + 1
    const int64_t* param_begin4;    // prefix of float4 parameter chunks, count + 1
    const int64_t* est_block_begin; // prefix of loss-estimate blocks, count + 1
    double* partials;
    unsigned int* ticket;
    // the one-launch iteration (batch_fused_kernel): every problem's gradient
    // batches, then every problem's Adam chunks, taken in that order from one queue
    const int64_t* adam_begin;      // prefix of Adam chunks, count + 1
    unsigned int* grad_done;        // per problem: gradient batches finished (zero between launches)
    unsigned int* adam_done;        // per problem: Adam chunks finished (zero between launches)
    unsigned long long* queue;      // [0] next item, [1] warps finished (zero between launches)
};

__device__ __forceinline__ int find_problem(const int64_t* prefix, int count, int64_t u)
{
    int lo = 0, hi = count;  // prefix[lo] <= u < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool batch_last_block(unsigned int* ticket)
{
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    return is_last != 0;
}

// 4 consecutive factor entries of row `row` of mode k, from the problem's gather storage
__device__ __forceinline__ float4 brow(const BatchDesc& P, int k, uint32_t row, int col)
{
    const size_t off = static_cast<size_t>(row) * P.ld + col;
    if (P.bf16) return load4(static_cast<const __nv_bfloat16*>(P.Ag[k]) + off);
    return load4(static_cast<const float*>(P.Ag[k]) + off);
}

// One batch of 32 consecutive draws of one problem (warp item u of the
// flattened table of all problems' draws): Alg. 1's draws, the model values,
// y, and the sampled MTTKRP into G (or the replica slabs).  The whole warp calls it.
__device__ __forceinline__ void batch_grad_item(const BatchArgs& a, const int64_t* s_work, int64_t u, int lane)
{
    constexpr unsigned kFull = 0xFFFFFFFFu;
    const int pb = find_problem(s_work, a.count, u);
    const BatchDesc& P = a.desc[pb];
    const int d = P.d, L = P.L, NC = P.NC, rank = P.rank, ld = P.ld;
    const int64_t j = (u - s_work[pb]) * 32 + lane;
    const uint64_t stream = static_cast<uint64_t>(*reinterpret_cast<const volatile int64_t*>(&P.st->iter));
    // this lane's draw (Alg. 1): i_k = randi(n_k), x = X(i), weight omega / s
    const bool mine = j < P.s;
    uint32_t ix[kBatchMaxD] = {0u, 0u, 0u, 0u};
    float x = 0.0f;
    if (mine) {
        const U64x4 blk = philox4x64_10(static_cast<uint64_t>(j), stream, kTagUniform, 0, P.seed, P.problem);
        uint64_t lin = 0;
#pragma unroll
        for (int k = 0; k < kBatchMaxD; ++k) {
            if (k < d) {
                ix[k] = randi32(blk.w[k], P.dims[k]);
                lin += static_cast<uint64_t>(ix[k]) * P.strides[k];
            }
        }
        x = __ldg(P.X + lin);
    }
    const int gl = lane & (L - 1), gbase = lane & ~(L - 1);
    // this batch's destination of each mode: G_k, or replica u mod R of its slabs
    float* dst[kBatchMaxD];
#pragma unroll
    for (int k = 0; k < kBatchMaxD; ++k)
        dst[k] = (k < d && P.reps[k] > 1)
                     ? P.R[k] + static_cast<size_t>(static_cast<uint32_t>(u) % P.reps[k]) * P.rep_stride[k]
                     : P.G[k];
    for (int b = 0; b < L; ++b) {
        const int src = gbase + b;
        uint32_t jx[kBatchMaxD];
#pragma unroll
        for (int k = 0; k < kBatchMaxD; ++k) jx[k] = __shfl_sync(kFull, ix[k], src);
        const float xb = __shfl_sync(kFull, x, src);
        const bool vb = __shfl_sync(kFull, static_cast<int>(mine), src) != 0;
        float part = 0.0f;
        for (int c = 0; c < NC; ++c) {
            const int col = (gl * NC + c) * 4;
            if (!vb || col >= rank) continue;
            float4 prod = brow(P, 0, jx[0], col);
#pragma unroll
            for (int k = 1; k < kBatchMaxD; ++k)
                if (k < d) prod = mul4(prod, brow(P, k, jx[k], col));
            part += sum4(prod);
        }
        for (int off = L >> 1; off > 0; off >>= 1) part += __shfl_xor_sync(kFull, part, off);
        if (!vb) continue;  // no shuffles below this point
        const float y = P.w * loss_g(P.loss, xb, part);
        for (int c = 0; c < NC; ++c) {
            const int col = (gl * NC + c) * 4;
            if (col >= rank) continue;
            float4 rc[kBatchMaxD];
#pragma unroll
            for (int k = 0; k < kBatchMaxD; ++k)
                rc[k] = k < d ? brow(P, k, jx[k], col) : make_float4(1.f, 1.f, 1.f, 1.f);
            float4 pre[kBatchMaxD], suf[kBatchMaxD];
            pre[0] = make_float4(y, y, y, y);
#pragma unroll
            for (int k = 1; k < kBatchMaxD; ++k) pre[k] = mul4(pre[k - 1], rc[k - 1]);
            suf[kBatchMaxD - 1] = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
            for (int k = kBatchMaxD - 2; k >= 0; --k) suf[k] = mul4(suf[k + 1], rc[k + 1]);
#pragma unroll
            for (int k = 0; k < kBatchMaxD; ++k) {
                if (k >= d) continue;
                red_add4(dst[k] + static_cast<size_t>(jx[k]) * ld + col, mul4(pre[k], suf[k]));
            }
        }
    }
}

__global__ void __launch_bounds__(256, 4) batch_grad_kernel(const BatchArgs a)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ int64_t s_work[];
    for (int i = threadIdx.x; i <= a.count; i += blockDim.x) s_work[i] = a.work_begin[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t W = s_work[a.count];
    const int64_t warp_global = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t u = warp_global; u < W; u += nwarps) batch_grad_item(a, s_work, u, lane);
}

__device__ __forceinline__ void bstore_bf16x4(uint16_t* dst, float4 v)
{
    uint2 packed;
    packed.x = static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v.x))) |
               (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v.y))) << 16);
    packed.y = static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v.z))) |
               (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(v.w))) << 16);
    *reinterpret_cast<uint2*>(dst) = packed;
}

__device__ __forceinline__ int mode_in_problem(const BatchDesc& P, int64_t loc4)
{
    int k = 0;
#pragma unroll
    for (int l = 1; l < kBatchMaxD; ++l)
        if (l < P.d && loc4 >= P.off4[l]) k = l;
    return k;
}

// The Adam step (Alg. 4) of float4 element p4 of problem P's parameters:
// its gradient (with the replica slabs folded in, in order, and cleared),
// moments, update, projection and BF16 copy, then G = 0.  G and the slabs
// are read past L1 (they were written at L2 by reductions of this launch or
// the one before).
__device__ __forceinline__ void batch_adam_element(const BatchDesc& P, int64_t p4, float ic1, float ic2, float alpha,
                                                   bool done)
{
    const int k = mode_in_problem(P, p4);
    const int64_t loc = p4 - P.off4[k];
    const int col = static_cast<int>((loc * 4) % P.ld);
    float4* g4 = reinterpret_cast<float4*>(P.G[k]) + loc;
    float4 g = __ldcg(g4);
    if (P.reps[k] > 1) {  // fold the replica slabs of this mode in order, leaving them zero
        // the first kWide loads are all issued before any is added or cleared
        constexpr int kWide = 16;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        float4* r = reinterpret_cast<float4*>(P.R[k]) + loc;
        const uint64_t rs = P.rep_stride[k] / 4;
        const uint32_t reps = P.reps[k];
        float4 v[kWide];
#pragma unroll
        for (int q = 0; q < kWide; ++q) v[q] = static_cast<uint32_t>(q) < reps ? __ldcg(r + q * rs) : zero;
        float4 acc = zero;
#pragma unroll
        for (int q = 0; q < kWide; ++q) acc = add4(acc, v[q]);
#pragma unroll
        for (int q = 0; q < kWide; ++q)
            if (static_cast<uint32_t>(q) < reps) r[q * rs] = zero;
        for (uint32_t q = kWide; q < reps; ++q) {
            acc = add4(acc, __ldcg(r + q * rs));
            r[q * rs] = zero;
        }
        g = add4(g, acc);
    }
    if (!done && col < P.rank) {
        float4* a4p = reinterpret_cast<float4*>(P.A[k]) + loc;
        float4* b4p = reinterpret_cast<float4*>(P.B[k]) + loc;
        float4* c4p = reinterpret_cast<float4*>(P.C[k]) + loc;
        float4 A4 = *a4p, B4 = *b4p, C4 = *c4p;
        const bool inside = P.eps_inside != 0;
        const int ncol = P.rank - col;
        adam_one(A4.x, B4.x, C4.x, g.x, P.beta1, P.beta2, ic1, ic2, P.eps, alpha, P.lower, inside);
        if (ncol > 1) adam_one(A4.y, B4.y, C4.y, g.y, P.beta1, P.beta2, ic1, ic2, P.eps, alpha, P.lower, inside);
        if (ncol > 2) adam_one(A4.z, B4.z, C4.z, g.z, P.beta1, P.beta2, ic1, ic2, P.eps, alpha, P.lower, inside);
        if (ncol > 3) adam_one(A4.w, B4.w, C4.w, g.w, P.beta1, P.beta2, ic1, ic2, P.eps, alpha, P.lower, inside);
        *a4p = A4;
        *b4p = B4;
        *c4p = C4;
        if (P.Abf[k]) bstore_bf16x4(P.Abf[k] + loc * 4, A4);
    }
    *g4 = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Adam of every problem: per-problem bias corrections, learning rate and
// done flag are read once per block into shared memory.
__global__ void __launch_bounds__(256, 3) batch_adam_kernel(const BatchArgs a)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ int64_t s_param[];  // count + 1 prefixes, then 4 floats per problem
    float* s_prob = reinterpret_cast<float*>(s_param + a.count + 1);
    for (int i = threadIdx.x; i <= a.count; i += blockDim.x) s_param[i] = a.param_begin4[i];
    for (int b = threadIdx.x; b < a.count; b += blockDim.x) {
        const BatchDesc& P = a.desc[b];
        const float n = static_cast<float>(P.st->t + 1);
        s_prob[4 * b + 0] = inv_bias_correction(P.beta1, n);
        s_prob[4 * b + 1] = inv_bias_correction(P.beta2, n);
        s_prob[4 * b + 2] = P.st->alpha;
        s_prob[4 * b + 3] = P.st->done ? 1.0f : 0.0f;
    }
    __syncthreads();
    const int64_t total4 = s_param[a.count];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i4 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i4 < total4; i4 += stride) {
        const int pb = find_problem(s_param, a.count, i4);
        batch_adam_element(a.desc[pb], i4 - s_param[pb], s_prob[4 * pb], s_prob[4 * pb + 1], s_prob[4 * pb + 2],
                           s_prob[4 * pb + 3] != 0.0f);
    }
    if (batch_last_block(a.ticket)) {  // every problem's step count, one thread per problem
        for (int b = threadIdx.x; b < a.count; b += blockDim.x) {
            gcp_adam_state* st = a.desc[b].st;
            if (!st->done) st->t += 1;
            st->iter += 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *a.ticket = 0u;
            __threadfence();
        }
    }
}

// One launch for a whole iteration of every problem (gradient and Adam step).
// Warps take items from one queue in order, kClaim at a time: first every
// problem's gradient batches (as batch_grad_kernel), then every problem's
// Adam chunks of kAdamChunk float4 elements (4 per lane).  A warp holding an
// Adam chunk of problem b waits until all of b's gradient batches are done;
// those were all claimed before any Adam chunk, by warps that work their
// gradient batches without waiting (a warp's later claims only ever hold later
// items), so the wait ends.
// The wait is bounded: after kBatchSpinLimit polls the warp records
// GCP_ERR_TIMEOUT in the problem's state and skips the chunk.  The problem's
// last Adam chunk advances its t and iter and clears its counters; the last
// warp to leave clears the queue.
// Release / acquire ordering at device scope: a warp's reductions are made
// visible before its count of finished batches (release), and a waiting warp
// sees them after reading the count (acquire).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

constexpr int kAdamChunk = 128;
constexpr int kBatchSpinLimit = 1 << 21;
constexpr int kClaim = 1;  // queue items a warp claims at a time (more made the tail longer: measured)

__global__ void __launch_bounds__(256, 3) batch_fused_kernel(const BatchArgs a)
{
    pdl_wait();
    pdl_trigger();
    constexpr unsigned kFull = 0xFFFFFFFFu;
    extern __shared__ int64_t s_pre[];  // gradient batch prefix (count + 1), then Adam chunk prefix (count + 1)
    int64_t* s_work = s_pre;
    int64_t* s_adam = s_pre + a.count + 1;
    for (int i = threadIdx.x; i <= a.count; i += blockDim.x) {
        s_work[i] = a.work_begin[i];
        s_adam[i] = a.adam_begin[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t W = s_work[a.count];
    const int64_t total = W + s_adam[a.count];
    // items are claimed kClaim at a time, the next claim in flight while this one is worked
    unsigned long long got = 0ull;
    if (lane == 0) got = atomicAdd(&a.queue[0], static_cast<unsigned long long>(kClaim));
    int64_t claim = static_cast<int64_t>(__shfl_sync(kFull, got, 0));
    while (claim < total) {
        unsigned long long next = 0ull;
        if (lane == 0) next = atomicAdd(&a.queue[0], static_cast<unsigned long long>(kClaim));
        for (int64_t item = claim; item < claim + kClaim && item < total; ++item) {
            if (item < W) {
                batch_grad_item(a, s_work, item, lane);
                __syncwarp();
                if (lane == 0) {
                    fence_acq_rel_gpu();
                    atomicAdd(&a.grad_done[find_problem(s_work, a.count, item)], 1u);
                }
                continue;
            }
            const int64_t ai = item - W;
            const int pb = find_problem(s_adam, a.count, ai);
            const BatchDesc& P = a.desc[pb];
            int ok = 1;
            if (lane == 0) {
                const unsigned need = static_cast<unsigned>(s_work[pb + 1] - s_work[pb]);
                int spins = 0;
                while (*reinterpret_cast<volatile unsigned*>(&a.grad_done[pb]) < need) {
                    if (++spins > kBatchSpinLimit) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                fence_acq_rel_gpu();
            }
            ok = __shfl_sync(kFull, ok, 0);
            __syncwarp();
            if (ok) {
                const float n = static_cast<float>(P.st->t + 1);
                const float ic1 = inv_bias_correction(P.beta1, n), ic2 = inv_bias_correction(P.beta2, n);
                const float alpha = P.st->alpha;
                const bool done = P.st->done != 0;
                const int64_t c0 = (ai - s_adam[pb]) * kAdamChunk;
                const int64_t n4 = P.off4[P.d];
#pragma unroll 1
                for (int i = 0; i < kAdamChunk / 32; ++i) {
                    const int64_t p4 = c0 + i * 32 + lane;
                    if (p4 < n4) batch_adam_element(P, p4, ic1, ic2, alpha, done);
                }
            } else if (lane == 0) {
                atomicCAS(&P.st->status, 0, static_cast<int32_t>(GCP_ERR_TIMEOUT));
            }
            __syncwarp();
            if (lane == 0) {
                fence_acq_rel_gpu();
                const unsigned chunks = static_cast<unsigned>(s_adam[pb + 1] - s_adam[pb]);
                if (atomicAdd(&a.adam_done[pb], 1u) + 1u == chunks) {  // the problem's last Adam chunk
                    gcp_adam_state* st = P.st;
                    if (!st->done) st->t += 1;
                    st->iter += 1;
                    a.grad_done[pb] = 0u;
                    a.adam_done[pb] = 0u;
                    fence_acq_rel_gpu();
                }
            }
        }
        claim = static_cast<int64_t>(__shfl_sync(kFull, next, 0));
    }
    if (lane == 0) {  // the last warp to leave clears the queue for the next launch
        const unsigned long long warps = static_cast<unsigned long long>(gridDim.x) * (blockDim.x >> 5);
        if (atomicAdd(&a.queue[1], 1ull) + 1ull == warps) {
            a.queue[0] = 0ull;
            a.queue[1] = 0ull;
            fence_acq_rel_gpu();
        }
    }
}

// gcp_batch_grad on its own: every problem's replica slabs folded into G (and
// cleared); gcp_batch_iteration folds them inside the Adam kernel instead.
__global__ void __launch_bounds__(256) batch_fold_kernel(const BatchArgs a)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ int64_t s_param[];
    for (int i = threadIdx.x; i <= a.count; i += blockDim.x) s_param[i] = a.param_begin4[i];
    __syncthreads();
    const int64_t total4 = s_param[a.count];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i4 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i4 < total4; i4 += stride) {
        const int pb = find_problem(s_param, a.count, i4);
        const BatchDesc& P = a.desc[pb];
        const int64_t p4 = i4 - s_param[pb];
        const int k = mode_in_problem(P, p4);
        if (P.reps[k] <= 1) continue;
        const int64_t loc = p4 - P.off4[k];
        float4* g4 = reinterpret_cast<float4*>(P.G[k]) + loc;
        *g4 = add4(*g4, fold_replicas(reinterpret_cast<float4*>(P.R[k]) + loc, P.reps[k], P.rep_stride[k] / 4));
    }
}

// Every problem's F-hat: blocks [est_block_begin[b], est_block_begin[b+1])
// serve problem b; the last block to finish sums each problem's partials in
// block order.
__global__ void __launch_bounds__(256) batch_loss_kernel(const BatchArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ double warp_sums[8];
    const int pb = find_problem(a.est_block_begin, a.count, blockIdx.x);
    const BatchDesc& P = a.desc[pb];
    const int64_t first = a.est_block_begin[pb], nblk = a.est_block_begin[pb + 1] - first;
    const int64_t lb = blockIdx.x - first;
    double acc = 0.0;
    for (int64_t e = lb * blockDim.x + threadIdx.x; e < P.n_est; e += nblk * blockDim.x) {
        uint32_t ix[kBatchMaxD] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < kBatchMaxD; ++k)
            if (k < P.d) ix[k] = static_cast<uint32_t>(__ldg(P.lidx[k] + e));
        float m = 0.0f;
        for (int col = 0; col < P.rank; col += 4) {
            float4 prod = brow(P, 0, ix[0], col);
#pragma unroll
            for (int k = 1; k < kBatchMaxD; ++k)
                if (k < P.d) prod = mul4(prod, brow(P, k, ix[k], col));
            m += sum4(prod);
        }
        acc += static_cast<double>(entry_f(P.loss, __ldg(P.lcls + e), __ldg(P.lx + e), m, __ldg(P.lw + e)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double blk = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) blk += warp_sums[w];
        a.partials[blockIdx.x] = blk;
    }
    if (batch_last_block(a.ticket)) {
        __threadfence();
        const volatile double* p = a.partials;
        for (int b = threadIdx.x; b < a.count; b += blockDim.x) {
            double total = 0.0;
            for (int64_t q = a.est_block_begin[b]; q < a.est_block_begin[b + 1]; ++q) total += p[q];
            a.desc[b].st->F = total;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *a.ticket = 0u;
            __threadfence();
        }
    }
}

// Every problem's epoch begin (snapshot) or end (accept or revert).
__global__ void __launch_bounds__(256) batch_epoch_kernel(const BatchArgs a)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ int64_t s_param[];
    int* s_fail = reinterpret_cast<int*>(s_param + a.count + 1);
    for (int i = threadIdx.x; i <= a.count; i += blockDim.x) s_param[i] = a.param_begin4[i];
    for (int b = threadIdx.x; b < a.count; b += blockDim.x) {
        const gcp_adam_state* st = a.desc[b].st;
        s_fail[b] = a.begin ? 0 : !(st->F <= st->F_old);
    }
    __syncthreads();
    const int64_t total4 = s_param[a.count];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i4 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i4 < total4; i4 += stride) {
        const int pb = find_problem(s_param, a.count, i4);
        const BatchDesc& P = a.desc[pb];
        const int64_t p4 = i4 - s_param[pb];
        const int k = mode_in_problem(P, p4);
        const int64_t loc = p4 - P.off4[k];
        float4* A4 = reinterpret_cast<float4*>(P.A[k]) + loc;
        float4* B4 = reinterpret_cast<float4*>(P.B[k]) + loc;
        float4* C4 = reinterpret_cast<float4*>(P.C[k]) + loc;
        float4* SA4 = reinterpret_cast<float4*>(P.SA[k]) + loc;
        float4* SB4 = reinterpret_cast<float4*>(P.SB[k]) + loc;
        float4* SC4 = reinterpret_cast<float4*>(P.SC[k]) + loc;
        if (s_fail[pb]) {
            const float4 sa = *SA4;
            *A4 = sa;
            *B4 = *SB4;
            *C4 = *SC4;
            if (P.Abf[k]) bstore_bf16x4(P.Abf[k] + loc * 4, sa);
        } else {
            *SA4 = *A4;
            *SB4 = *B4;
            *SC4 = *C4;
        }
    }
    if (batch_last_block(a.ticket) && threadIdx.x == 0) {
        for (int b = 0; b < a.count; ++b) {
            const BatchDesc& P = a.desc[b];
            gcp_adam_state* st = P.st;
            if (a.begin) {
                st->F_old = st->F;
            } else if (s_fail[b]) {
                if (!isfinite(st->F)) atomicCAS(&st->status, 0, static_cast<int32_t>(GCP_ERR_NONFINITE));
                st->F = st->F_old;
                st->t -= P.tau;
                st->alpha *= P.nu;
                st->bad += 1;
                st->done = st->bad > P.kappa ? 1 : 0;
            } else {
                st->F_old = st->F;
            }
        }
        *a.ticket = 0u;
        __threadfence();
    }
}

}  // namespace gcpk

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace gcpk;

struct gcp_batch {
    int32_t count = 0;
    BatchDesc* d_desc = nullptr;
    int64_t* d_work = nullptr;
    int64_t* d_param = nullptr;
    int64_t* d_est = nullptr;
    double* d_partials = nullptr;
    unsigned int* d_ticket = nullptr;
    float* d_rep = nullptr;  // every problem's replica slabs
    int64_t total_work = 0, total_param4 = 0, est_blocks = 0;
    int num_sms = 1;
    int block = 0, grid = 0;
    int64_t* d_adam = nullptr;            // prefix of Adam chunks (the one-launch iteration)
    unsigned int* d_done = nullptr;       // per problem: gradient batches done, then Adam chunks done
    unsigned long long* d_queue = nullptr;  // the one-launch iteration's queue: next item, warps finished
    int64_t total_adam = 0;
    std::vector<BatchDesc> host_desc;  // the uploaded table, for reshaping
    int chunks_per_lane = 1, replica_target = 64, max_replicas = 32;
};

namespace {

constexpr int kBatchMaxProblems = 1024;
constexpr int kBatchEstBlocksPerProblem = 32;
// replica slabs: a mode whose rows receive more than kBatchRepTarget updates
// per iteration on average gets ceil(updates / kBatchRepTarget) slabs, at most
// kBatchMaxReps (the single-problem defaults)
constexpr double kBatchRepTarget = 64.0;
constexpr int64_t kBatchMaxReps = 32;

bool al(const void* p, size_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) == 0; }

gcp_status to_status(cudaError_t e)
{
    if (e == cudaSuccess) return GCP_OK;
    return e == cudaErrorMemoryAllocation ? GCP_ERR_NO_MEMORY : GCP_ERR_CUDA;
}

// Lanes per draw and float4 chunks per lane of a rank-r problem: a lane takes
// up to cpl chunks of a row, and the lanes per draw are the power of two that
// covers the rest (at most 32); more chunks per lane, more draws per warp step.
void lanes_chunks(int rank, int cpl, int32_t* L_out, int32_t* NC_out)
{
    const int chunks = (rank + 3) / 4;
    const int per = (chunks + cpl - 1) / cpl;
    int L = 1;
    while (L < per && L < 32) L <<= 1;
    *L_out = L;
    *NC_out = (chunks + L - 1) / L;
}

// Replica slabs of mode k: ceil(updates per row / target), at most max_reps.
int64_t replicas_for(const BatchDesc& d, int k, int target, int max_reps)
{
    const double hits = static_cast<double>(d.s) / static_cast<double>(d.dims[k]);
    return std::max<int64_t>(1, std::min<int64_t>(static_cast<int64_t>(std::ceil(hits / target)), max_reps));
}

gcp_status fill_desc(const gcp_batch_problem& p, BatchDesc* o)
{
    const gcp_tensor& X = p.X;
    const gcp_factors& F = p.F;
    if (X.sparse || X.d < 2 || X.d > kBatchMaxD || !X.vals || X.weights) return GCP_ERR_INVALID_ARG;
    if (F.rank < 1 || F.rank > 256 || F.ld < F.rank || F.ld % 4 != 0) return GCP_ERR_INVALID_ARG;
    if (p.loss < GCP_LOSS_GAUSSIAN || p.loss > GCP_LOSS_BETA_HALF) return GCP_ERR_INVALID_ARG;
    if (p.S.kind != GCP_SAMPLER_UNIFORM || p.S.q < 0 || p.S.q > (int64_t(1) << 40)) return GCP_ERR_INVALID_ARG;
    if (!al(p.state, 8)) return GCP_ERR_INVALID_ARG;
    if (!(p.adam.beta1 >= 0.f && p.adam.beta1 < 1.f && p.adam.beta2 >= 0.f && p.adam.beta2 < 1.f)) return GCP_ERR_INVALID_ARG;
    if (p.est.n < 0 || (p.est.n > 0 && (!p.est.x || !p.est.w || !p.est.cls))) return GCP_ERR_INVALID_ARG;
    *o = BatchDesc{};
    o->d = X.d;
    o->ld = F.ld;
    o->rank = F.rank;
    o->loss = p.loss;
    lanes_chunks(F.rank, 1, &o->L, &o->NC);
    o->bf16 = F.bf16 ? 1 : 0;
    double omega = 1.0;
    uint64_t stride = 1;
    for (int k = X.d - 1; k >= 0; --k) {
        if (X.dims[k] < 1 || X.dims[k] >= (int64_t(1) << 31)) return GCP_ERR_INVALID_ARG;
        o->dims[k] = static_cast<uint32_t>(X.dims[k]);
        o->strides[k] = stride;
        stride *= static_cast<uint64_t>(X.dims[k]);
    }
    for (int k = 0; k < X.d; ++k) omega *= static_cast<double>(X.dims[k]);
    o->X = X.vals;
    o->off4[0] = 0;
    for (int k = 0; k < X.d; ++k) {
        if (!al(F.A[k], 16) || !al(p.G[k], 16) || !al(p.B[k], 16) || !al(p.C[k], 16) || !al(p.SA[k], 16) ||
            !al(p.SB[k], 16) || !al(p.SC[k], 16))
            return GCP_ERR_INVALID_ARG;
        if (F.bf16 && !al(F.A_bf16[k], 8)) return GCP_ERR_INVALID_ARG;
        if (F.A_bf16[k] && !al(F.A_bf16[k], 8)) return GCP_ERR_INVALID_ARG;
        if (p.est.n > 0 && !p.est.idx[k]) return GCP_ERR_INVALID_ARG;
        o->Ag[k] = F.bf16 ? static_cast<const void*>(F.A_bf16[k]) : static_cast<const void*>(F.A[k]);
        o->A[k] = F.A[k];
        o->Abf[k] = F.A_bf16[k];
        o->G[k] = p.G[k];
        o->B[k] = p.B[k];
        o->C[k] = p.C[k];
        o->SA[k] = p.SA[k];
        o->SB[k] = p.SB[k];
        o->SC[k] = p.SC[k];
        o->off4[k + 1] = o->off4[k] + X.dims[k] * F.ld / 4;
        o->lidx[k] = p.est.idx[k];
    }
    o->seed = p.S.seed;
    o->problem = p.S.problem;
    o->s = p.S.q;
    o->w = p.S.q > 0 ? static_cast<float>(omega / static_cast<double>(p.S.q)) : 0.0f;
    o->beta1 = p.adam.beta1;
    o->beta2 = p.adam.beta2;
    o->eps = p.adam.eps;
    o->lower = p.adam.lower;
    o->eps_inside = p.adam.eps_inside_sqrt;
    o->kappa = p.epoch.kappa;
    o->nu = p.epoch.nu;
    o->tau = p.epoch.tau;
    o->st = p.state;
    o->lx = p.est.x;
    o->lw = p.est.w;
    o->lcls = p.est.cls;
    o->n_est = p.est.n;
    return GCP_OK;
}

BatchArgs batch_args(const gcp_batch* b, int begin)
{
    BatchArgs a{};
    a.desc = b->d_desc;
    a.count = b->count;
    a.begin = begin;
    a.work_begin = b->d_work;
    a.param_begin4 = b->d_param;
    a.est_block_begin = b->d_est;
    a.partials = b->d_partials;
    a.ticket = b->d_ticket;
    a.adam_begin = b->d_adam;
    a.grad_done = b->d_done;
    a.adam_done = b->d_done + b->count;
    a.queue = b->d_queue;
    return a;
}

int elementwise_blocks(const gcp_batch* b)
{
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((b->total_param4 + 255) / 256, int64_t(b->num_sms) * 8)));
}

}  // namespace

extern "C" {

gcp_status gcp_batch_create(gcp_batch** out, const gcp_batch_problem* problems, int32_t count, gcp_stream_t stream)
{
    if (!out || !problems || count < 1 || count > kBatchMaxProblems) return GCP_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<BatchDesc> desc(count);
    std::vector<int64_t> work(count + 1, 0), param(count + 1, 0), est(count + 1, 0), adam(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        gcp_status st = fill_desc(problems[i], &desc[i]);
        if (st != GCP_OK) return st;
        work[i + 1] = work[i] + (desc[i].s + 31) / 32;
        param[i + 1] = param[i] + desc[i].off4[desc[i].d];
        adam[i + 1] = adam[i] + (desc[i].off4[desc[i].d] + kAdamChunk - 1) / kAdamChunk;
        const int64_t nb = std::max<int64_t>(1, std::min<int64_t>((desc[i].n_est + 255) / 256, kBatchEstBlocksPerProblem));
        est[i + 1] = est[i] + nb;
    }
    // replica slabs per problem and mode, one workspace for all (offsets filled after allocation)
    std::vector<int64_t> rep_off(static_cast<size_t>(count) * kBatchMaxD, -1);
    int64_t rep_floats = 0;
    for (int i = 0; i < count; ++i) {
        for (int k = 0; k < desc[i].d; ++k) {
            const int64_t r = replicas_for(desc[i], k, static_cast<int>(kBatchRepTarget), static_cast<int>(kBatchMaxReps));
            desc[i].reps[k] = static_cast<uint32_t>(r);
            desc[i].rep_stride[k] = static_cast<uint64_t>(desc[i].dims[k]) * desc[i].ld;
            if (r > 1) {
                rep_off[static_cast<size_t>(i) * kBatchMaxD + k] = rep_floats;
                rep_floats += r * static_cast<int64_t>(desc[i].rep_stride[k]);
            }
        }
    }
    gcp_batch* b = new (std::nothrow) gcp_batch();
    if (!b) return GCP_ERR_NO_MEMORY;
    b->count = count;
    b->total_work = work[count];
    b->total_param4 = param[count];
    b->est_blocks = est[count];
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->num_sms < 1) b->num_sms = 1;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err) {
        gcp_batch_destroy(b);
        return to_status(err);
    };
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_desc), sizeof(BatchDesc) * count)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_work), sizeof(int64_t) * (count + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_param), sizeof(int64_t) * (count + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_est), sizeof(int64_t) * (count + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_partials), sizeof(double) * b->est_blocks)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_ticket), sizeof(unsigned int))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_adam), sizeof(int64_t) * (count + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_done), sizeof(unsigned int) * 2 * count)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_queue), sizeof(unsigned long long) * 2)) != cudaSuccess) return fail(e);
    b->total_adam = adam[count];
    if (rep_floats > 0) {
        if ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_rep), sizeof(float) * rep_floats)) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(b->d_rep, 0, sizeof(float) * rep_floats, s)) != cudaSuccess) return fail(e);
    }
    for (int i = 0; i < count; ++i)
        for (int k = 0; k < desc[i].d; ++k) {
            const int64_t off = rep_off[static_cast<size_t>(i) * kBatchMaxD + k];
            desc[i].R[k] = off >= 0 ? b->d_rep + off : nullptr;
        }
    if ((e = cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemcpyAsync(b->d_work, work.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemcpyAsync(b->d_param, param.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemcpyAsync(b->d_est, est.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned int), s)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(b->d_adam, adam.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned int) * 2 * count, s)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long) * 2, s)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
    b->host_desc = desc;
    *out = b;
    return GCP_OK;
}

gcp_status gcp_batch_set_shape(gcp_batch* b, int32_t chunks_per_lane, int32_t replica_target, int32_t max_replicas,
                               gcp_stream_t stream)
{
    if (!b || chunks_per_lane < 0 || chunks_per_lane > 8 || replica_target < 0 || max_replicas < 0 ||
        max_replicas > 1024)
        return GCP_ERR_INVALID_ARG;
    const int cpl = chunks_per_lane > 0 ? chunks_per_lane : 1;
    const int target = replica_target > 0 ? replica_target : static_cast<int>(kBatchRepTarget);
    const int maxr = max_replicas > 0 ? max_replicas : static_cast<int>(kBatchMaxReps);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<BatchDesc> desc = b->host_desc;
    std::vector<int64_t> rep_off(desc.size() * kBatchMaxD, -1);
    int64_t rep_floats = 0;
    for (size_t i = 0; i < desc.size(); ++i) {
        lanes_chunks(desc[i].rank, cpl, &desc[i].L, &desc[i].NC);
        for (int k = 0; k < desc[i].d; ++k) {
            const int64_t r = replicas_for(desc[i], k, target, maxr);
            desc[i].reps[k] = static_cast<uint32_t>(r);
            if (r > 1) {
                rep_off[i * kBatchMaxD + k] = rep_floats;
                rep_floats += r * static_cast<int64_t>(desc[i].rep_stride[k]);
            }
        }
    }
    // new replica slabs (zeroed) once the stream has finished with the old ones
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return to_status(e);
    float* rep = nullptr;
    if (rep_floats > 0) {
        if ((e = cudaMalloc(reinterpret_cast<void**>(&rep), sizeof(float) * rep_floats)) != cudaSuccess)
            return to_status(e);
        if ((e = cudaMemsetAsync(rep, 0, sizeof(float) * rep_floats, s)) != cudaSuccess) {
            cudaFree(rep);
            return to_status(e);
        }
    }
    for (size_t i = 0; i < desc.size(); ++i)
        for (int k = 0; k < desc[i].d; ++k) {
            const int64_t off = rep_off[i * kBatchMaxD + k];
            desc[i].R[k] = off >= 0 ? rep + off : nullptr;
        }
    if ((e = cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(BatchDesc) * desc.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        cudaFree(rep);
        return to_status(e);
    }
    cudaFree(b->d_rep);
    b->d_rep = rep;
    b->host_desc = desc;
    b->chunks_per_lane = cpl;
    b->replica_target = target;
    b->max_replicas = maxr;
    return GCP_OK;
}

gcp_status gcp_batch_get_shape(gcp_batch* b, int32_t problem, int32_t* lanes, int32_t* chunks, int32_t* replicas)
{
    if (!b || problem < 0 || problem >= b->count || !lanes || !chunks || !replicas) return GCP_ERR_INVALID_ARG;
    const BatchDesc& d = b->host_desc[static_cast<size_t>(problem)];
    *lanes = d.L;
    *chunks = d.NC;
    for (int k = 0; k < kBatchMaxD; ++k) replicas[k] = k < d.d ? static_cast<int32_t>(d.reps[k]) : 0;
    return GCP_OK;
}

gcp_status gcp_batch_destroy(gcp_batch* b)
{
    if (!b) return GCP_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    cudaFree(b->d_desc);
    cudaFree(b->d_work);
    cudaFree(b->d_param);
    cudaFree(b->d_est);
    cudaFree(b->d_partials);
    cudaFree(b->d_ticket);
    cudaFree(b->d_rep);
    cudaFree(b->d_adam);
    cudaFree(b->d_done);
    cudaFree(b->d_queue);
    delete b;
    return GCP_OK;
}

gcp_status gcp_batch_set_tuning(gcp_batch* b, int32_t block, int32_t grid_blocks)
{
    if (!b || block < 0 || block > 256 || block % 32 != 0 || grid_blocks < 0) return GCP_ERR_INVALID_ARG;
    b->block = block;
    b->grid = grid_blocks;
    return GCP_OK;
}

// The gradient kernel alone: replicated modes are left in their slabs.
static gcp_status batch_grad_launch(gcp_batch* b, gcp_stream_t stream)
{
    if (!b) return GCP_ERR_INVALID_ARG;
    if (b->total_work == 0) return GCP_OK;
    const int block = b->block > 0 ? b->block : 256;
    const size_t smem = sizeof(int64_t) * (b->count + 1);
    int bps = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_grad_kernel, block, smem);
    const int64_t warps_per_block = block / 32;
    const int64_t want = (b->total_work + warps_per_block - 1) / warps_per_block;
    const int grid = b->grid > 0 ? b->grid
                                 : static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(b->num_sms) * std::max(bps, 1))));
    return to_status(launch_pdl(batch_grad_kernel, dim3(grid), dim3(block), smem, reinterpret_cast<cudaStream_t>(stream),
                                batch_args(b, 0)));
}

gcp_status gcp_batch_grad(gcp_batch* b, gcp_stream_t stream)
{
    gcp_status st = batch_grad_launch(b, stream);
    if (st != GCP_OK || !b->d_rep) return st;
    const size_t smem = sizeof(int64_t) * (b->count + 1);
    return to_status(launch_pdl(batch_fold_kernel, dim3(elementwise_blocks(b)), dim3(256), smem,
                                reinterpret_cast<cudaStream_t>(stream), batch_args(b, 0)));
}

gcp_status gcp_batch_adam_step(gcp_batch* b, gcp_stream_t stream)
{
    if (!b) return GCP_ERR_INVALID_ARG;
    const size_t smem = sizeof(int64_t) * (b->count + 1) + sizeof(float) * 4 * b->count;
    return to_status(launch_pdl(batch_adam_kernel, dim3(elementwise_blocks(b)), dim3(256), smem,
                                reinterpret_cast<cudaStream_t>(stream), batch_args(b, 0)));
}

gcp_status gcp_batch_iteration(gcp_batch* b, gcp_stream_t stream)
{
    gcp_status st = batch_grad_launch(b, stream);  // the Adam kernel folds the replica slabs
    if (st != GCP_OK) return st;
    return gcp_batch_adam_step(b, stream);
}

gcp_status gcp_batch_iteration_fused(gcp_batch* b, gcp_stream_t stream)
{
    if (!b) return GCP_ERR_INVALID_ARG;
    const int block = 256;
    const size_t smem = sizeof(int64_t) * 2 * (b->count + 1);
    int bps = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_fused_kernel, block, smem);
    const int64_t items = b->total_work + b->total_adam;
    const int64_t want = std::max<int64_t>(1, (items + block / 32 - 1) / (block / 32));
    const int grid = static_cast<int>(std::min<int64_t>(want, int64_t(b->num_sms) * std::max(bps, 1)));
    return to_status(launch_pdl(batch_fused_kernel, dim3(grid), dim3(block), smem,
                                reinterpret_cast<cudaStream_t>(stream), batch_args(b, 0)));
}

gcp_status gcp_batch_loss_est(gcp_batch* b, gcp_stream_t stream)
{
    if (!b) return GCP_ERR_INVALID_ARG;
    return to_status(launch_pdl(batch_loss_kernel, dim3(static_cast<unsigned>(b->est_blocks)), dim3(256), 0,
                                reinterpret_cast<cudaStream_t>(stream), batch_args(b, 0)));
}

static gcp_status batch_epoch(gcp_batch* b, int begin, gcp_stream_t stream)
{
    if (!b) return GCP_ERR_INVALID_ARG;
    const size_t smem = sizeof(int64_t) * (b->count + 1) + sizeof(int) * b->count;
    return to_status(launch_pdl(batch_epoch_kernel, dim3(elementwise_blocks(b)), dim3(256), smem,
                                reinterpret_cast<cudaStream_t>(stream), batch_args(b, begin)));
}

gcp_status gcp_batch_epoch_begin(gcp_batch* b, gcp_stream_t stream) { return batch_epoch(b, 1, stream); }
gcp_status gcp_batch_epoch_end(gcp_batch* b, gcp_stream_t stream) { return batch_epoch(b, 0, stream); }

}  // extern "C"
