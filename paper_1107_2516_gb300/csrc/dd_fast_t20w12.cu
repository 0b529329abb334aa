// Kernel 2 instantiation: 20 samples x 4 DM trials per thread, 12 warps per block.
#include "dd_fast_impl.cuh"

namespace dd {

cudaError_t fast_launch_t20w12(dd_dtype t, const FastLaunch &a, cudaStream_t s)
{
    return fast_launch_cfg<20, 12>(t, a, s);
}

cudaError_t fast_prepare_t20w12(size_t optin) { return fast_prepare_cfg<20, 12>(optin); }

cudaError_t batch_launch_t20w12(const BatchLaunch &b, int grid, size_t smem, cudaStream_t s)
{
    return batch_launch_cfg<20, 12>(b, grid, smem, s);
}

}  // namespace dd
