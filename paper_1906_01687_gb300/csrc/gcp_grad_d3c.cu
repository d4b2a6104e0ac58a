// Instantiations of the fused sampled-gradient kernel for 3 modes with
// warp-level pre-reduction of same-address updates (layout 4).
#include "gcp_grad_impl.cuh"

namespace gcpk {
const void* grad_kernel_ptr_d3c(int L, int NC, bool bf16)
{
    return bf16 ? grad_kernel_ptr_variant<3, true, 4>(L, NC) : grad_kernel_ptr_variant<3, false, 4>(L, NC);
}
}  // namespace gcpk
