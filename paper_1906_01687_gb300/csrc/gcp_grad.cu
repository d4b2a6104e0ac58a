// Host-side dispatch of the fused sampled-gradient kernel instantiations.
#include "gcp_kernels.cuh"

namespace gcpk {

const void* grad_kernel_ptr_d3(int L, int NC, bool bf16);
const void* grad_kernel_ptr_d4(int L, int NC, bool bf16);
const void* grad_kernel_ptr_d8(int L, int NC, bool bf16);

static const void* grad_ptr(int D, int L, int NC, bool bf16)
{
    switch (D) {
    case 3: return grad_kernel_ptr_d3(L, NC, bf16);
    case 4: return grad_kernel_ptr_d4(L, NC, bf16);
    case 8: return grad_kernel_ptr_d8(L, NC, bf16);
    default: return nullptr;
    }
}

bool grad_has_config(int D, int L, int NC) { return grad_ptr(D, L, NC, false) != nullptr; }

cudaError_t grad_occupancy(int D, int L, int NC, bool bf16, int block, size_t smem, int* blocks_per_sm)
{
    const void* f = grad_ptr(D, L, NC, bf16);
    if (!f) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
}

cudaError_t launch_grad(const GradArgs& a, int D, int L, int NC, bool bf16, int grid, int block, size_t smem,
                        cudaStream_t s)
{
    const void* f = grad_ptr(D, L, NC, bf16);
    if (!f) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    void* args[] = {const_cast<GradArgs*>(&a)};
    return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace gcpk
