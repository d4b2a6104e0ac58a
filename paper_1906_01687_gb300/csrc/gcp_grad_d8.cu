// Instantiations of the fused sampled-gradient kernel for 2 to 8 modes (runtime d).
#include "gcp_grad_impl.cuh"

namespace gcpk {
const void* grad_kernel_ptr_d8(int L, int NC, bool bf16, int layout)
{
    return bf16 ? grad_kernel_ptr<8, true>(L, NC, layout) : grad_kernel_ptr<8, false>(L, NC, layout);
}
}  // namespace gcpk
