// Diagnostics (C ABI dinr_selftest_timeout): the bounded-wait path of the
// tensor-core kernels, exercised without any fault. One warp waits on an
// mbarrier that nothing arrives on, with the same wait primitive and error
// flag protocol as the persistent kernels but a caller-given limit; it gives
// up, records the timeout code and returns, and the host reports it as it
// reports a real timeout, leaving the context usable.
#include "context.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kSelftestCode = 99;

__global__ void k_wait_selftest(int *err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    dinr::tc::mbar_init(&bar, 1);
    dinr::tc::fence_mbar_init();
  }
  __syncwarp();
  const bool ok = dinr::tc::mbar_wait_for(&bar, 0, err, kSelftestCode, limit_ns);
  (void)__all_sync(0xffffffffu, ok);
}

}  // namespace

dinr_status dinr_selftest_timeout(dinr_ctx *c, int64_t limit_ns) {
  if (!c) return DINR_ERR_ARG;
  if (c->failed) return DINR_ERR_CUDA;
  if (limit_ns < 1000000 || limit_ns > 4000000000LL)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "limit must be in [1 ms, 4 s]");
  int *flag = c->d_flag + 3;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), c->st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, c->st>>>(flag, (unsigned long long)limit_ns);
    e = cudaGetLastError();
  }
  int code = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&code, flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
  if (code != 0)
    return (dinr_status)dinr_fail(c, DINR_ERR_TIMEOUT,
                                  "a kernel gave up waiting (code %d, self-test)", code);
  return DINR_OK;
}
