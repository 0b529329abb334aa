// Kernel 5 instantiation (its one compiled shape, three input types).
#include "dd_share_impl.cuh"

namespace dd {

cudaError_t share_launch(dd_dtype t, const ShareLaunch &a, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    switch (t) {
    case DD_F32: share_kernel<float, false, kShTI, kShDR, kShNW, kShCS, kShNP><<<grid, kShNW * 32, a.smem, s>>>(a); break;
    case DD_F16: share_kernel<__half, false, kShTI, kShDR, kShNW, kShCS, kShNP><<<grid, kShNW * 32, a.smem, s>>>(a); break;
    case DD_U8: share_kernel<uint8_t, true, kShTI, kShDR, kShNW, kShCS, kShNP><<<grid, kShNW * 32, a.smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t share_prepare(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)share_kernel<float, false, kShTI, kShDR, kShNW, kShCS, kShNP>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_kernel<__half, false, kShTI, kShDR, kShNW, kShCS, kShNP>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_kernel<uint8_t, true, kShTI, kShDR, kShNW, kShCS, kShNP>, optin);
    return e;
}

}  // namespace dd
