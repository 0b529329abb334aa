// Kernel 2 instantiation: 36 samples x 4 DM trials per thread, 8 warps per block.
#include "dd_fast_impl.cuh"

namespace dd {

cudaError_t fast_launch_t36w8(dd_dtype t, const FastLaunch &a, cudaStream_t s)
{
    return fast_launch_cfg<36, 8>(t, a, s);
}

cudaError_t fast_prepare_t36w8(size_t optin) { return fast_prepare_cfg<36, 8>(optin); }

cudaError_t batch_launch_t36w8(const BatchLaunch &b, int grid, size_t smem, cudaStream_t s)
{
    return batch_launch_cfg<36, 8>(b, grid, smem, s);
}

}  // namespace dd
