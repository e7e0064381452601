// libmam: self-test of the bounded device waits.
//
// Every spin wait of the column kernels (an mbarrier phase that the bulk
// copies complete) is bounded by %globaltimer: when the bound runs out the
// kernel records an error and returns instead of hanging, and the host then
// reports MAM_ERR_TIMEOUT.  This entry point exercises that path without a
// fault: one warp waits, through the same helper, on an mbarrier phase that
// expects two arrivals and receives none, so the wait must run out.
#include "mam_device.cuh"
#include "mam_handle.h"

namespace mam {
namespace {

__global__ void wait_timeout_kernel(unsigned long long limit_ns, int* timed_out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);  // two arrivals expected, none will come
    fence_mbar_init();
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
  if (__all_sync(0xffffffffu, !ok) && threadIdx.x == 0) *timed_out = 1;
}

}  // namespace
}  // namespace mam

extern "C" mam_status mam_selftest_wait_timeout(int32_t limit_us) {
  using namespace mam;
  if (limit_us < 1 || limit_us > 2000000)
    return fail(nullptr, MAM_ERR_INVALID_ARG, "limit_us must be in 1..2000000");
  int* flag = nullptr;
  cudaError_t e = cudaMalloc(&flag, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, MAM_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  int v = 0;
  e = cudaMemset(flag, 0, sizeof(int));
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32>>>(1000ull * (unsigned long long)limit_us, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(flag);
  if (e != cudaSuccess) return fail(nullptr, MAM_ERR_CUDA, cudaGetErrorString(e));
  if (v != 1) return fail(nullptr, MAM_ERR_STATE, "the bounded wait did not run out");
  return fail(nullptr, MAM_ERR_TIMEOUT, "device wait ran out of its bound (self-test)");
}
