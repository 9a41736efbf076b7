// Self-test of the bounded device waits: a kernel waits on an mbarrier that
// nothing will complete, with the same helper (and error word) the Schur
// kernels use for their bulk-copy waits, and must give up and report instead
// of hanging.  No GPU fault is involved.
#include <cuda_runtime.h>

#include "../../include/ddel.h"
#include "ddel_device.cuh"

namespace ddel {
namespace {

__global__ void wait_selftest_kernel(uint32_t limit, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival; none comes
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar, 0, limit));
  if (!ok && threadIdx.x == 0) atomicExch(err, kErrTimeout);
}

}  // namespace
}  // namespace ddel

extern "C" int ddel_selftest_wait_timeout(unsigned int poll_limit, int* status) {
  using namespace ddel;
  if (!status || poll_limit == 0 || poll_limit > kWaitLimit) return DDEL_EINVAL;
  int* d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) return DDEL_ENOMEM;
  int h = 0;
  cudaError_t e = cudaMemset(d_err, 0, sizeof(int));
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32>>>(poll_limit, d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_err);
  if (e != cudaSuccess) return DDEL_ECUDA;
  *status = h == kErrTimeout ? DDEL_ETIMEOUT : DDEL_OK;
  return DDEL_OK;
}
