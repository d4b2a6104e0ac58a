// Instantiations of the fused sampled-gradient kernel for 4 modes with
// warp-level pre-reduction of same-address updates (layout 4).
#include "gcp_grad_impl.cuh"

namespace gcpk {
const void* grad_kernel_ptr_d4c(int L, int NC, bool bf16)
{
    return bf16 ? grad_kernel_ptr_variant<4, true, 4>(L, NC) : grad_kernel_ptr_variant<4, false, 4>(L, NC);
}
}  // namespace gcpk
