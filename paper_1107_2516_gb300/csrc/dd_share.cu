// Kernel 5 instantiations (its compiled shapes, three input types).
#include "dd_share_impl.cuh"

namespace dd {

template <int TI, int DR, int NW, int MINB, int NS>
static cudaError_t share_launch_cfg(dd_dtype t, const ShareLaunch &a, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    switch (t) {
    case DD_F32: share_kernel<float, false, TI, DR, NW, kShCS, kShNP, NS, MINB><<<grid, NW * 32, a.smem, s>>>(a); break;
    case DD_F16: share_kernel<__half, false, TI, DR, NW, kShCS, kShNP, NS, MINB><<<grid, NW * 32, a.smem, s>>>(a); break;
    case DD_U8: share_kernel<uint8_t, true, TI, DR, NW, kShCS, kShNP, NS, MINB><<<grid, NW * 32, a.smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int TI, int DR, int NW, int MINB, int NS>
static cudaError_t share_prepare_cfg(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)share_kernel<float, false, TI, DR, NW, kShCS, kShNP, NS, MINB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_kernel<__half, false, TI, DR, NW, kShCS, kShNP, NS, MINB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_kernel<uint8_t, true, TI, DR, NW, kShCS, kShNP, NS, MINB>, optin);
    return e;
}

#define DD_SHARE_CFG(k) kShareCfg[k].ti, kShareCfg[k].dr, kShareCfg[k].nw, kShareCfg[k].minb, kShareCfg[k].ns
static_assert(kNumShareCfg == 3, "one case per compiled shape");

cudaError_t share_launch(int k, dd_dtype t, const ShareLaunch &a, cudaStream_t s)
{
    switch (k) {
    case 0: return share_launch_cfg<DD_SHARE_CFG(0)>(t, a, s);
    case 1: return share_launch_cfg<DD_SHARE_CFG(1)>(t, a, s);
    default: return share_launch_cfg<DD_SHARE_CFG(2)>(t, a, s);
    }
}

cudaError_t share_prepare(int k, size_t optin)
{
    switch (k) {
    case 0: return share_prepare_cfg<DD_SHARE_CFG(0)>(optin);
    case 1: return share_prepare_cfg<DD_SHARE_CFG(1)>(optin);
    default: return share_prepare_cfg<DD_SHARE_CFG(2)>(optin);
    }
}

}  // namespace dd
