// Kernel 4 instantiation of tile configuration kTmemCfg[0].
#include "dd_tmem_impl.cuh"

namespace dd {

cudaError_t tmem_launch_c0(dd_dtype t, const TmemLaunch &a, cudaStream_t s)
{
    return tmem_launch_cfg<kTmemCfg[0].n, kTmemCfg[0].dbw, kTmemCfg[0].nw, kTmemCfg[0].tpw>(t, a, s);
}

cudaError_t tmem_prepare_c0(size_t optin)
{
    return tmem_prepare_cfg<kTmemCfg[0].n, kTmemCfg[0].dbw, kTmemCfg[0].nw, kTmemCfg[0].tpw>(optin);
}

}  // namespace dd
