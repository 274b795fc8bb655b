// Self-test of the bounded device-side waits of the tensor-core kernels.
//
// Every mbarrier wait of the mode-product kernels goes through mbar_wait
// (b3_kernel.cuh): it polls the barrier, reads %globaltimer every 64 polls and
// gives up after kTimeoutNs, raising the CTA's abort flag and recording its
// code in the device error word that the host turns into FCGLE_ERR_TIMEOUT.
// This kernel runs that same function on an mbarrier nothing ever arrives on,
// so the wait can only end by its time limit; the host then checks the code it
// left and that the context still runs work.  No fault, trap or endless loop
// is involved: the only way out is the wait's own bound.
#include <cuda_runtime.h>

#include <stdexcept>
#include <string>

#include "b3_kernel.cuh"
#include "common.h"
#include "selftest.h"

namespace fcgle {
namespace {

__global__ void bounded_wait_selftest_kernel(int* err, int code, int* done) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  const uint32_t b = b3::smem_u32(&bar);
  b3::mbar_init(b, 1);   // one arrival completes phase 0; none is ever made
  abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const bool completed = b3::mbar_wait(b, 0, &abort_flag, err, code);
  *done = completed ? 1 : 2;   // 2: gave up at the time limit, as it must
}

__global__ void selftest_followup_kernel(int* done) { *done += 10; }

}  // namespace

int bounded_wait_selftest(cudaStream_t st) {
  int* dev = nullptr;
  FCGLE_CUDA(cudaMalloc(&dev, 2 * sizeof(int)));
  int host[2] = {0, 0};
  try {
    FCGLE_CUDA(cudaMemsetAsync(dev, 0, 2 * sizeof(int), st));
    bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(dev, kSelftestWaitCode, dev + 1);
    FCGLE_CUDA(cudaGetLastError());
    // a second kernel on the same stream: the context must still run work
    selftest_followup_kernel<<<1, 1, 0, st>>>(dev + 1);
    FCGLE_CUDA(cudaGetLastError());
    FCGLE_CUDA(cudaMemcpyAsync(host, dev, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    FCGLE_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    cudaFree(dev);
    throw;
  }
  FCGLE_CUDA(cudaFree(dev));
  // the wait gave up (2), the follow-up ran (+10), and the error word holds the code
  if (host[1] != 12) throw std::runtime_error("bounded-wait self-test: unexpected completion state " +
                                              std::to_string(host[1]));
  return host[0];
}

}  // namespace fcgle
