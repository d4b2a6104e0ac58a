// Adam with projection and the epoch logic of Alg. 4, with the optimizer
// state (F-hat, F-hat_old, t, iteration, alpha, failed epochs) kept in device
// memory so that whole epochs can be replayed from a CUDA graph.
//
// Scalars that every block reads at its start are changed only after all
// blocks have read them: by block 0 after a cluster barrier (small grids) or
// by the last block to finish (a completion ticket).
#include <cuda_bf16.h>

#include <algorithm>

#include "gcp_adam_phase.cuh"
#include "gcp_device.cuh"
#include "gcp_kernels.cuh"

namespace gcpk {

// Completion ticket: returns true in exactly one thread of the last block.
__device__ __forceinline__ bool last_block_done(unsigned int* ticket)
{
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    return is_last && threadIdx.x == 0;
}

// One launch of the Adam step.  Every thread reads the step's scalars (t,
// alpha, done) itself, then issues the loads of its element -- the gradient,
// its replica slabs, A, B, C -- before using any, so an element costs one
// round trip to L2.  kSync says how t and iter advance:
//   kTicket:   after every block has read t, by the last block to finish;
//   kCluster:  a grid of at most 8 blocks launched as one thread-block
//              cluster; each thread arrives at the cluster barrier right after
//              its reads, block 0 waits and writes.
enum AdamSync { kTicket = 0, kCluster = 1 };

template <int kSync>
__global__ void __launch_bounds__(256) adam_kernel(const AdamArgs a)
{
    pdl_wait();
    pdl_trigger();
    const int64_t t0 = a.st->t;
    const float alpha = a.st->alpha;
    const int done = a.st->done;
    if constexpr (kSync == kCluster) cluster_arrive();
    const float n = static_cast<float>(t0 + 1);
    const float ic1 = inv_bias_correction(a.beta1, n);
    const float ic2 = inv_bias_correction(a.beta2, n);
    const ModeTable& mt = a.mt;
    // 32-bit element indices: the host keeps the factor set below 2^31 float4 chunks
    const uint32_t total4 = static_cast<uint32_t>(mt.off4[mt.d]);
    const uint32_t ld4 = static_cast<uint32_t>(mt.ld) / 4;
    const uint32_t stride = gridDim.x * blockDim.x;
    const bool inside = a.eps_inside_sqrt != 0;
    for (uint32_t i4 = blockIdx.x * blockDim.x + threadIdx.x; i4 < total4; i4 += stride) {
        const int k = mode_of(mt, i4);
        const uint32_t loc = i4 - static_cast<uint32_t>(mt.off4[k]);
        const int col = static_cast<int>((loc % ld4) * 4);
        float4* g4 = reinterpret_cast<float4*>(mt.G[k]) + loc;
        float4* a4p = reinterpret_cast<float4*>(mt.A[k]) + loc;
        float4* b4p = reinterpret_cast<float4*>(mt.B[k]) + loc;
        float4* c4p = reinterpret_cast<float4*>(mt.C[k]) + loc;
        float4 g = *g4;
        float4 A4 = *a4p, B4 = *b4p, C4 = *c4p;
        if (a.reps[k] > 1)  // fold the replica slabs of this mode, leaving them zero
            g = add4(g, fold_replicas(reinterpret_cast<float4*>(a.R[k]) + loc, a.reps[k], a.rep_stride4[k]));
        if (!done && col < mt.rank) {
            const int live = mt.rank - col;  // columns of this chunk below rank
            adam_one(A4.x, B4.x, C4.x, g.x, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
            if (live > 1) adam_one(A4.y, B4.y, C4.y, g.y, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
            if (live > 2) adam_one(A4.z, B4.z, C4.z, g.z, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
            if (live > 3) adam_one(A4.w, B4.w, C4.w, g.w, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
            *a4p = A4;
            *b4p = B4;
            *c4p = C4;
            if (mt.Abf[k]) store_bf16x4(mt.Abf[k] + static_cast<size_t>(loc) * 4, A4);
        }
        *g4 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (kSync == kCluster) {
        cluster_wait();
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (!done) a.st->t = t0 + 1;
            a.st->iter += 1;
        }
    } else if (last_block_done(&a.st->ticket)) {
        if (!a.st->done) a.st->t += 1;
        a.st->iter += 1;
        a.st->ticket = 0u;
        __threadfence();
    }
}

// Grids of up to 8 blocks run as one cluster (rounded up to 1, 2, 4 or 8 blocks).
cudaError_t launch_adam(const AdamArgs& a, int grid, cudaStream_t s)
{
    if (grid > 8) return launch_pdl(adam_kernel<kTicket>, dim3(grid), dim3(256), 0, s, a);
    int c = 1;
    while (c < grid) c <<= 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = static_cast<unsigned>(c);
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, adam_kernel<kCluster>, a);
}

// The step after a gradient kernel that advanced t (gcp_iteration), with
// the replica fold split over kParts lanes per float4 element (the layout of
// adam_elements), spread thinly (64 threads per block) over many SMs.  No
// block waits for another: t was advanced by the gradient kernel; block 0
// advances iter, which no Adam block reads.
//
// The first element's mode, addresses and A, B, C, and the scalars alpha and
// done, were last written two launches back or earlier (the previous
// iteration's Adam step, an epoch kernel), which had completed before this
// iteration's gradient kernel passed its wait; they are read before this
// kernel's wait, with the kernel parameters.  G and the replicas come from the
// gradient kernel and are read after it.
__global__ void __launch_bounds__(64) adam_split_kernel(const AdamArgs a)
{
    const uint32_t total4 = static_cast<uint32_t>(a.mt.off4[a.mt.d]);
    const uint32_t gthread = blockIdx.x * blockDim.x + threadIdx.x;
    AdamElem e;
    adam_prepare(a, gthread / kParts, total4, gthread % kParts, e);
    const float alpha = a.st->alpha;
    const int done = a.st->done;
    pdl_wait();
    pdl_trigger();
    adam_elements(a, gthread, gridDim.x * blockDim.x, e, a.st->t, alpha, done);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->iter += 1;
}

// The same step for large factor sets (bandwidth-bound): every thread takes
// kStreamU float4 elements per round, a block's threads adjacent elements
// (coalesced), with the loads of all of them -- A, B, C, then G -- issued
// before any is used; the first round's A, B, C before the dependency wait,
// so that blocks made resident while the gradient kernel drains already
// stream them.  Replicated modes fold their slabs in the thread that owns
// the element.  t was advanced by the gradient kernel; block 0 advances
// iter, which no Adam block reads.
constexpr int kStreamU = 4;
constexpr int kStreamBlock = 256;

__global__ void __launch_bounds__(kStreamBlock, 2) adam_stream_kernel(const AdamArgs a)
{
    const ModeTable& mt = a.mt;
    const uint32_t total4 = static_cast<uint32_t>(mt.off4[mt.d]);
    const uint32_t ld4 = static_cast<uint32_t>(mt.ld) / 4;
    const uint32_t round = gridDim.x * kStreamBlock * kStreamU;
    int k[kStreamU];
    uint32_t loc[kStreamU];
    float4 g[kStreamU], A4[kStreamU], B4[kStreamU], C4[kStreamU];
    // an element's mode and position and its A, B, C: the first round's are
    // loaded before the dependency wait -- A, B, C and the scalars alpha and
    // done were last written two launches back or earlier (the previous
    // iteration's Adam step, an epoch kernel), complete before the gradient
    // kernel that precedes this one passed its own wait
    auto prepare = [&](uint32_t base) {
#pragma unroll
        for (int u = 0; u < kStreamU; ++u) {
            const uint32_t i4 = base + static_cast<uint32_t>(u) * kStreamBlock;
            k[u] = 0;
            loc[u] = 0;
            A4[u] = B4[u] = C4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i4 < total4) {
                k[u] = mode_of(mt, i4);
                loc[u] = i4 - static_cast<uint32_t>(mt.off4[k[u]]);
                A4[u] = reinterpret_cast<const float4*>(mt.A[k[u]])[loc[u]];
                B4[u] = reinterpret_cast<const float4*>(mt.B[k[u]])[loc[u]];
                C4[u] = reinterpret_cast<const float4*>(mt.C[k[u]])[loc[u]];
            }
        }
    };
    const uint32_t base0 = blockIdx.x * kStreamBlock * kStreamU + threadIdx.x;
    prepare(base0);
    const float alpha = a.st->alpha;
    const int done = a.st->done;
    pdl_wait();
    pdl_trigger();
    const float n = static_cast<float>(a.st->t);  // advanced by the gradient kernel
    const float ic1 = inv_bias_correction(a.beta1, n);
    const float ic2 = inv_bias_correction(a.beta2, n);
    const bool inside = a.eps_inside_sqrt != 0;
    for (uint32_t base = base0; base < total4; base += round) {
        if (base != base0) prepare(base);
#pragma unroll
        for (int u = 0; u < kStreamU; ++u) {
            const uint32_t i4 = base + static_cast<uint32_t>(u) * kStreamBlock;
            g[u] = i4 < total4 ? reinterpret_cast<const float4*>(mt.G[k[u]])[loc[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kStreamU; ++u) {
            const uint32_t i4 = base + static_cast<uint32_t>(u) * kStreamBlock;
            if (i4 >= total4) continue;
            if (a.reps[k[u]] > 1) {  // fold the replica slabs of this mode in order, leaving them zero
                // (replicated modes are short, so few elements take this path)
                float4* r = reinterpret_cast<float4*>(a.R[k[u]]) + loc[u];
                const uint64_t rs = a.rep_stride4[k[u]];
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (uint32_t q = 0; q < a.reps[k[u]]; ++q) {
                    acc = add4(acc, r[q * rs]);
                    r[q * rs] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                g[u] = add4(g[u], acc);
            }
            const int col = static_cast<int>((loc[u] % ld4) * 4);
            if (!done && col < mt.rank) {
                const int live = mt.rank - col;  // columns of this chunk below rank
                adam_one(A4[u].x, B4[u].x, C4[u].x, g[u].x, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
                if (live > 1)
                    adam_one(A4[u].y, B4[u].y, C4[u].y, g[u].y, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
                if (live > 2)
                    adam_one(A4[u].z, B4[u].z, C4[u].z, g[u].z, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
                if (live > 3)
                    adam_one(A4[u].w, B4[u].w, C4[u].w, g[u].w, a.beta1, a.beta2, ic1, ic2, a.eps, alpha, a.lower, inside);
                reinterpret_cast<float4*>(mt.A[k[u]])[loc[u]] = A4[u];
                reinterpret_cast<float4*>(mt.B[k[u]])[loc[u]] = B4[u];
                reinterpret_cast<float4*>(mt.C[k[u]])[loc[u]] = C4[u];
                if (mt.Abf[k[u]]) store_bf16x4(mt.Abf[k[u]] + static_cast<size_t>(loc[u]) * 4, A4[u]);
            }
            reinterpret_cast<float4*>(mt.G[k[u]])[loc[u]] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->iter += 1;
}

// Factor sets of at least this many float4 elements take the streaming
// kernel (bandwidth-bound); smaller ones the split kernel (latency-bound,
// many replica slabs to fold).
constexpr int64_t kStreamMin4 = 1 << 18;

cudaError_t launch_adam_advanced(const AdamArgs& a, int num_sms, cudaStream_t s)
{
    const int64_t total4 = a.mt.off4[a.mt.d];
    if (total4 >= kStreamMin4) {
        const int64_t per_block = int64_t(kStreamBlock) * kStreamU;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((total4 + per_block - 1) / per_block,
                                                                    int64_t(num_sms) * 8));
        return launch_pdl(adam_stream_kernel, dim3(static_cast<unsigned>(grid)), dim3(kStreamBlock), 0, s, a);
    }
    const int64_t threads = total4 * kParts;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((threads + 63) / 64, int64_t(num_sms) * 32));
    return launch_pdl(adam_split_kernel, dim3(static_cast<unsigned>(grid)), dim3(64), 0, s, a);
}

// epoch_begin (snapshot) and epoch_end (accept or revert)
__global__ void __launch_bounds__(256) epoch_kernel(const EpochArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        const double F = a.st->F, Fo = a.st->F_old;
        s_fail = a.begin ? 0 : !(F <= Fo);  // an increase or a non-finite estimate fails
    }
    __syncthreads();
    const ModeTable& mt = a.mt;
    const int64_t total4 = mt.off4[mt.d];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i4 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i4 < total4; i4 += stride) {
        const int k = mode_of(mt, i4);
        const int64_t loc = i4 - mt.off4[k];
        float4* A4 = reinterpret_cast<float4*>(mt.A[k]) + loc;
        float4* B4 = reinterpret_cast<float4*>(mt.B[k]) + loc;
        float4* C4 = reinterpret_cast<float4*>(mt.C[k]) + loc;
        float4* SA4 = reinterpret_cast<float4*>(mt.SA[k]) + loc;
        float4* SB4 = reinterpret_cast<float4*>(mt.SB[k]) + loc;
        float4* SC4 = reinterpret_cast<float4*>(mt.SC[k]) + loc;
        if (s_fail) {
            const float4 sa = *SA4;
            *A4 = sa;
            *B4 = *SB4;
            *C4 = *SC4;
            if (mt.Abf[k]) store_bf16x4(mt.Abf[k] + loc * 4, sa);
        } else {
            *SA4 = *A4;
            *SB4 = *B4;
            *SC4 = *C4;
        }
    }
    if (last_block_done(&a.st->ticket)) {
        gcp_adam_state* st = a.st;
        if (a.begin) {
            st->F_old = st->F;
        } else if (s_fail) {
            if (!isfinite(st->F)) atomicCAS(&st->status, 0, static_cast<int32_t>(GCP_ERR_NONFINITE));
            st->F = st->F_old;
            st->t -= a.tau;
            st->alpha *= a.nu;
            st->bad += 1;
            st->done = st->bad > a.kappa ? 1 : 0;
        } else {
            st->F_old = st->F;
        }
        st->ticket = 0u;
        __threadfence();
    }
}

cudaError_t launch_epoch(const EpochArgs& a, int grid, cudaStream_t s)
{
    return launch_pdl(epoch_kernel, dim3(grid), dim3(256), 0, s, a);
}

__global__ void state_init_kernel(gcp_adam_state* st, float alpha)
{
    st->F = 0.0;
    st->F_old = 0.0;
    st->t = 0;
    st->iter = 0;
    st->alpha = alpha;
    st->bad = 0;
    st->done = 0;
    st->status = 0;
    st->ticket = 0u;
    st->reserved[0] = st->reserved[1] = st->reserved[2] = 0u;
}

cudaError_t launch_state_init(gcp_adam_state* st, float alpha, cudaStream_t s)
{
    state_init_kernel<<<1, 1, 0, s>>>(st, alpha);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) to_bf16_kernel(const ModeTable mt)
{
    pdl_wait();
    pdl_trigger();
    const int64_t total4 = mt.off4[mt.d];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i4 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i4 < total4; i4 += stride) {
        const int k = mode_of(mt, i4);
        const int64_t loc = i4 - mt.off4[k];
        if (mt.Abf[k]) store_bf16x4(mt.Abf[k] + loc * 4, reinterpret_cast<const float4*>(mt.A[k])[loc]);
    }
}

cudaError_t launch_to_bf16(const ModeTable& mt, int grid, cudaStream_t s)
{
    return launch_pdl(to_bf16_kernel, dim3(grid), dim3(256), 0, s, mt);
}

}  // namespace gcpk
