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

// The warp-specialised shape: PW stage-1 warps + NW stage-2 warps per block.
template <int TI, int DR, int NW, int NS, int PW, int PB>
static cudaError_t share_ws_launch_cfg(dd_dtype t, const ShareLaunch &a, cudaStream_t s)
{
    const unsigned grid = (unsigned)(a.ntile * a.nblk);
    constexpr int kThreads = (NW + PW) * 32;
    switch (t) {
    case DD_F32: share_ws_kernel<float, false, TI, DR, NW, PW, kShCS, kShNP, NS, PB><<<grid, kThreads, a.smem, s>>>(a); break;
    case DD_F16: share_ws_kernel<__half, false, TI, DR, NW, PW, kShCS, kShNP, NS, PB><<<grid, kThreads, a.smem, s>>>(a); break;
    case DD_U8: share_ws_kernel<uint8_t, true, TI, DR, NW, PW, kShCS, kShNP, NS, PB><<<grid, kThreads, a.smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int TI, int DR, int NW, int NS, int PW, int PB>
static cudaError_t share_ws_prepare_cfg(size_t optin)
{
    cudaError_t e = allow_max_dynamic_smem((const void *)share_ws_kernel<float, false, TI, DR, NW, PW, kShCS, kShNP, NS, PB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_ws_kernel<__half, false, TI, DR, NW, PW, kShCS, kShNP, NS, PB>, optin);
    if (e == cudaSuccess)
        e = allow_max_dynamic_smem((const void *)share_ws_kernel<uint8_t, true, TI, DR, NW, PW, kShCS, kShNP, NS, PB>, optin);
    return e;
}

template <int TI, int DR, int NW, int NS, int PW, int PB>
static bool share_ws_regs_ok_cfg()
{
    using Regs = WsRegs<NW, PW>;
    if (!Regs::kSplit) return true;
    const void *fn[3] = {(const void *)share_ws_kernel<float, false, TI, DR, NW, PW, kShCS, kShNP, NS, PB>,
                         (const void *)share_ws_kernel<__half, false, TI, DR, NW, PW, kShCS, kShNP, NS, PB>,
                         (const void *)share_ws_kernel<uint8_t, true, TI, DR, NW, PW, kShCS, kShNP, NS, PB>};
    for (const void *f : fn) {
        cudaFuncAttributes at{};
        if (cudaFuncGetAttributes(&at, f) != cudaSuccess || at.numRegs < Regs::kNeed) return false;
    }
    return true;
}

#define DD_SHARE_CFG(k) kShareCfg[k].ti, kShareCfg[k].dr, kShareCfg[k].nw, kShareCfg[k].minb, kShareCfg[k].ns
#define DD_SHARE_WS_CFG(k) kShareCfg[k].ti, kShareCfg[k].dr, kShareCfg[k].nw, kShareCfg[k].ns, kShareCfg[k].pw, kShareCfg[k].pb
static_assert(kNumShareCfg == 4, "one case per compiled shape");
static_assert(kShareCfg[0].pw == 0 && kShareCfg[1].pw == 0 && kShareCfg[2].pw == 0 && kShareCfg[3].pw > 0,
              "shapes 0-2 are the one-barrier kernel, shape 3 the warp-specialised one");

cudaError_t share_launch(int k, dd_dtype t, const ShareLaunch &a, cudaStream_t s)
{
    switch (k) {
    case 0: return share_launch_cfg<DD_SHARE_CFG(0)>(t, a, s);
    case 1: return share_launch_cfg<DD_SHARE_CFG(1)>(t, a, s);
    case 2: return share_launch_cfg<DD_SHARE_CFG(2)>(t, a, s);
    default: return share_ws_launch_cfg<DD_SHARE_WS_CFG(3)>(t, a, s);
    }
}

cudaError_t share_prepare(int k, size_t optin)
{
    switch (k) {
    case 0: return share_prepare_cfg<DD_SHARE_CFG(0)>(optin);
    case 1: return share_prepare_cfg<DD_SHARE_CFG(1)>(optin);
    case 2: return share_prepare_cfg<DD_SHARE_CFG(2)>(optin);
    default: return share_ws_prepare_cfg<DD_SHARE_WS_CFG(3)>(optin);
    }
}

bool share_regs_ok(int k)
{
    switch (k) {
    case 3: return share_ws_regs_ok_cfg<DD_SHARE_WS_CFG(3)>();
    default: return true;
    }
}

// Mixed persistent batch: kernel 5 shape 0 with kernel 3 shape 2.
constexpr ShareShape kMS = kShareCfg[kMixedShare];
constexpr LaneShape kML = kLaneCfg[kMixedLane];
static_assert(kMS.ti == kML.ti && kMS.dr == kML.dr && kMS.nw == kML.nw && kMS.minb == kML.minb,
              "the mixed batch's kernel 3 and kernel 5 shapes must share the block geometry");

cudaError_t mixed_batch_launch(const LaneBatchLaunch &b, int sms, size_t smem, cudaStream_t s)
{
    mixed_batch_kernel<kMS.ti, kMS.dr, kMS.nw, kShCS, kShNP, kMS.ns, kMS.minb><<<sms * kMS.minb, kMS.nw * 32, smem, s>>>(b);
    return cudaGetLastError();
}

int mixed_batch_occupancy(size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, mixed_batch_kernel<kMS.ti, kMS.dr, kMS.nw, kShCS, kShNP, kMS.ns, kMS.minb>, kMS.nw * 32, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t mixed_batch_prepare(size_t optin)
{
    return allow_max_dynamic_smem((const void *)mixed_batch_kernel<kMS.ti, kMS.dr, kMS.nw, kShCS, kShNP, kMS.ns, kMS.minb>,
                                  optin);
}

}  // namespace dd
