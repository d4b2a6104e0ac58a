// Host-side dispatch of the fused sampled-gradient kernel instantiations.
#include "gcp_device.cuh"
#include "gcp_kernels.cuh"

namespace gcpk {

const void* grad_kernel_ptr_d3(int L, int NC, bool bf16, int layout);
const void* grad_kernel_ptr_d4(int L, int NC, bool bf16, int layout);
const void* grad_kernel_ptr_d8(int L, int NC, bool bf16, int layout);
const void* grad_kernel_ptr_d3z(int L, int NC, bool bf16);
const void* grad_kernel_ptr_d4z(int L, int NC, bool bf16);
const void* grad_kernel_ptr_d3c(int L, int NC, bool bf16);
const void* grad_kernel_ptr_d4c(int L, int NC, bool bf16);
const void* grad_kernel_ptr_d3zc(int L, int NC, bool bf16);
const void* grad_kernel_ptr_d4zc(int L, int NC, bool bf16);

static const void* grad_ptr(int D, int L, int NC, bool bf16, int layout)
{
    if (layout >= 3) {  // the group-walk variants (3 or 4 modes)
        if (D != 3 && D != 4) return nullptr;
        switch (layout) {
        case 3: return D == 3 ? grad_kernel_ptr_d3z(L, NC, bf16) : grad_kernel_ptr_d4z(L, NC, bf16);
        case 4: return D == 3 ? grad_kernel_ptr_d3c(L, NC, bf16) : grad_kernel_ptr_d4c(L, NC, bf16);
        case 5: return D == 3 ? grad_kernel_ptr_d3zc(L, NC, bf16) : grad_kernel_ptr_d4zc(L, NC, bf16);
        default: return nullptr;
        }
    }
    switch (D) {
    case 3: return grad_kernel_ptr_d3(L, NC, bf16, layout);
    case 4: return grad_kernel_ptr_d4(L, NC, bf16, layout);
    case 8: return grad_kernel_ptr_d8(L, NC, bf16, layout);
    default: return nullptr;
    }
}

bool grad_has_config(int D, int L, int NC, int layout) { return grad_ptr(D, L, NC, false, layout) != nullptr; }

cudaError_t grad_occupancy(int D, int L, int NC, bool bf16, int layout, int block, size_t smem, int* blocks_per_sm)
{
    const void* f = grad_ptr(D, L, NC, bf16, layout);
    if (!f) return cudaErrorInvalidValue;
    // the default dynamic allowance is 48 KB less the kernel's static shared
    // memory, so any sizeable request raises it explicitly
    if (smem >= 16 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
}

cudaError_t launch_grad(const GradArgs& a, int D, int L, int NC, bool bf16, int layout, int grid, int block,
                        size_t smem, cudaStream_t s)
{
    const void* f = grad_ptr(D, L, NC, bf16, layout);
    if (!f) return cudaErrorInvalidValue;
    // the default dynamic allowance is 48 KB less the kernel's static shared
    // memory, so any sizeable request raises it explicitly
    if (smem >= 16 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    void* args[] = {const_cast<GradArgs*>(&a)};
    return launch_pdl_ptr(f, dim3(grid), dim3(block), smem, s, args);
}

__global__ void __launch_bounds__(256) fold_kernel(const FoldArgs a)
{
    pdl_wait();
    pdl_trigger();
    const int64_t total4 = a.off4[a.nmodes];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i4 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i4 < total4; i4 += stride) {
        int m = 0;
#pragma unroll
        for (int l = 1; l < GCP_MAX_MODES; ++l)
            if (l < a.nmodes && i4 >= a.off4[l]) m = l;
        const int64_t loc = i4 - a.off4[m];
        float4* g = reinterpret_cast<float4*>(a.G[m]) + loc;
        float4* r = reinterpret_cast<float4*>(a.R[m]) + loc;
        *g = add4(*g, fold_replicas(r, a.reps[m], a.rep_stride4[m]));
    }
}

cudaError_t launch_fold(const FoldArgs& a, int grid, cudaStream_t s)
{
    return launch_pdl(fold_kernel, dim3(grid), dim3(256), 0, s, a);
}

}  // namespace gcpk
