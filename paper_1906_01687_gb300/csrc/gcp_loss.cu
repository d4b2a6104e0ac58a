// Fixed-sample loss estimate F-hat (Eqs. (5.1)-(5.2); the semi-stratified
// form subtracts f(0, m) at the nonzeros like Alg. 3's gradient).  Each term
// is computed in FP32; terms are summed in FP64: per thread in a fixed
// grid-stride order, then per block, then the last block to finish adds the
// block partials (thread i the partials i, i + blockDim, ... in order, then a
// fixed shuffle and warp tree).  The result is therefore the same on every
// launch with the same list and grid.
#include <type_traits>

#include "gcp_draw.cuh"

namespace gcpk {

template <int D, bool BF16>
__global__ void __launch_bounds__(256) loss_kernel(const LossArgs a)
{
    pdl_wait();
    pdl_trigger();
    using T = std::conditional_t<BF16, __nv_bfloat16, float>;
    __shared__ double warp_sums[8];
    __shared__ int is_last;
    const int d = D <= 4 ? D : a.dr.d;
    double acc = 0.0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < a.dr.n_total; e += stride) {
        Draw<D> o;
        make_draw<D>(a.dr, e, 0, o);
        float m = 0.0f;
        for (int col = 0; col < a.rank; col += 4) {
            float4 prod = load4(static_cast<const T*>(a.A[0]) + static_cast<size_t>(o.ix[0]) * a.ld + col);
#pragma unroll
            for (int k = 1; k < D; ++k)
                if (k < d) prod = mul4(prod, load4(static_cast<const T*>(a.A[k]) + static_cast<size_t>(o.ix[k]) * a.ld + col));
            m += sum4(prod);
        }
        acc += static_cast<double>(entry_f(a.loss, o.cls, o.x, m, o.w));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double block = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) block += warp_sums[w];
        a.partials[blockIdx.x] = block;
        __threadfence();
        const unsigned prev = atomicAdd(a.ticket, 1u);
        is_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;  // block-uniform
    __threadfence();
    const volatile double* p = a.partials;
    double part = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) part += p[b];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, off);
    __syncthreads();  // warp_sums is reused
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double total = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) total += warp_sums[w];
        *a.out = total;
        *a.ticket = 0u;
    }
}

cudaError_t launch_loss(const LossArgs& a, bool bf16, int grid, int block, cudaStream_t s)
{
    const int d = a.dr.d;
    const dim3 g(grid), b(block);
    if (d == 3) return bf16 ? launch_pdl(loss_kernel<3, true>, g, b, 0, s, a) : launch_pdl(loss_kernel<3, false>, g, b, 0, s, a);
    if (d == 4) return bf16 ? launch_pdl(loss_kernel<4, true>, g, b, 0, s, a) : launch_pdl(loss_kernel<4, false>, g, b, 0, s, a);
    return bf16 ? launch_pdl(loss_kernel<8, true>, g, b, 0, s, a) : launch_pdl(loss_kernel<8, false>, g, b, 0, s, a);
}

}  // namespace gcpk
