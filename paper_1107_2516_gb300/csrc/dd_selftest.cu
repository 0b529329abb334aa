// Self-test of the failure path every staged kernel relies on: the bounded
// mbarrier wait (dd_fast_impl.cuh) that gives up, records DD_ERR_TIMEOUT and
// lets the kernel return instead of spinning forever when an input copy never
// completes.  One block arms an mbarrier for 16 bytes; with issue_copy it then
// issues the 16-byte bulk copy that completes it, without it nothing arrives
// and the wait runs out after limit_ns.  Nothing is left in flight either way.
#include "dd_fast_impl.cuh"

namespace dd {

__global__ void wait_selftest_kernel(const int4 *src, int *err, uint64_t limit_ns, int issue_copy)
{
    __shared__ __align__(16) int4 buf;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_arrive_tx(&bar, (uint32_t)sizeof(int4));
    if (issue_copy) bulk_g2s(&buf, src, (uint32_t)sizeof(int4), &bar);
    if (mbar_wait(&bar, 0, err, limit_ns) && buf.x != src->x) atomicExch(err, DD_ERR_ARG);
}

}  // namespace dd

using namespace dd;

extern "C" int dd_wait_selftest(int64_t limit_ns, int32_t issue_copy, int32_t *device_status)
{
    if (limit_ns < 1 || limit_ns > (int64_t)kWaitLimitNs || !device_status)
        return set_error(DD_ERR_ARG, "limit_ns must be in 1..%llu and device_status non-NULL",
                         (unsigned long long)kWaitLimitNs);
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(int4));
    if (e != cudaSuccess) return cuda_fail(e, "self-test buffer");
    int4 *src = reinterpret_cast<int4 *>(d) + 1;
    const int4 pat = make_int4(0x5a5a0001, 2, 3, 4);
    e = cudaMemset(d, 0, sizeof(int4));
    if (e == cudaSuccess) e = cudaMemcpy(src, &pat, sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32>>>(src, d, (uint64_t)limit_ns, issue_copy ? 1 : 0);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    *device_status = h;
    if (h == DD_ERR_TIMEOUT) return set_error(DD_ERR_TIMEOUT, "bounded wait gave up after %lld ns", (long long)limit_ns);
    if (h) return set_error(h, "wait self-test: copied data differs");
    return DD_OK;
}
