// Instantiations of the fused sampled-gradient kernel for 4 modes.
#include "gcp_grad_impl.cuh"

namespace gcpk {
const void* grad_kernel_ptr_d4(int L, int NC, bool bf16, int layout)
{
    return bf16 ? grad_kernel_ptr<4, true>(L, NC, layout) : grad_kernel_ptr<4, false>(L, NC, layout);
}
}  // namespace gcpk
