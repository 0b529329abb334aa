// Kernel 5 instantiations (its compiled shapes, three input types).
#include "dd_share_impl.cuh"

namespace dd {

template <int TI, int MINB>
static cudaError_t share_launch_cfg(dd_dtype t, const ShareLaunch &a, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    switch (t) {
    case DD_F32: share_kernel<float, false, TI, kShDR, kShNW, kShCS, kShNP, MINB><<<grid, kShNW * 32, a.smem, s>>>(a); break;
    case DD_F16: share_kernel<__half, false, TI, kShDR, kShNW, kShCS, kShNP, MINB><<<grid, kShNW * 32, a.smem, s>>>(a); break;
    case DD_U8: share_kernel<uint8_t, true, TI, kShDR, kShNW, kShCS, kShNP, MINB><<<grid, kShNW * 32, a.smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int TI, int MINB>
static cudaError_t share_prepare_cfg(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)share_kernel<float, false, TI, kShDR, kShNW, kShCS, kShNP, MINB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_kernel<__half, false, TI, kShDR, kShNW, kShCS, kShNP, MINB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_kernel<uint8_t, true, TI, kShDR, kShNW, kShCS, kShNP, MINB>, optin);
    return e;
}

cudaError_t share_launch(int k, dd_dtype t, const ShareLaunch &a, cudaStream_t s)
{
    return k == 0 ? share_launch_cfg<kShareCfg[0].ti, kShareCfg[0].minb>(t, a, s)
                  : share_launch_cfg<kShareCfg[1].ti, kShareCfg[1].minb>(t, a, s);
}

cudaError_t share_prepare(int k, size_t optin)
{
    return k == 0 ? share_prepare_cfg<kShareCfg[0].ti, kShareCfg[0].minb>(optin)
                  : share_prepare_cfg<kShareCfg[1].ti, kShareCfg[1].minb>(optin);
}

}  // namespace dd
