// Discrete L2 norm of a user-layout tensor without any device allocation.
//
// The handle-based fcgle_norm packs the tensor into a preallocated internal
// buffer of the handle and reduces it there; obtaining a handle allocates
// about fifteen state-sized buffers.  This variant reads the tensor in place
// and keeps its partial sums in a fixed scratch array that lives in the
// library's own static device memory, so it needs no handle and allocates
// nothing on the device.
//
//   ||u||_h = sqrt(h_1 ... h_d * sum_j |u_j|^2),  h_mu = (b_mu - a_mu) / (n_mu + 1)
//
// Reduction: the N complex entries are cut into fixed chunks of kChunk
// entries; one block sums one chunk (each thread a fixed strided subset, then
// a fixed tree), writing one FP64 partial per chunk; a second single-block
// kernel sums the partials in a fixed order.  The chunking does not depend on
// the GPU, so the result is bitwise reproducible.  Every partial slot and the
// result slot are written before they are read: nothing has to start at zero.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.h"
#include "engine.h"
#include "norm_static.h"

namespace fcgle {
namespace {

constexpr int kThreads1 = 256;
constexpr int kThreads2 = 1024;

// partial sums, then the final sum in the last slot
static __device__ __align__(256) double g_norm_scratch[kNormStaticMaxPartials + 1];

template <typename R>
__global__ void __launch_bounds__(kThreads1) norm_partials_kernel(const R* __restrict__ x, unsigned long long nreal,
                                                                  double* __restrict__ part) {
  const unsigned long long base = (unsigned long long)blockIdx.x * (2ull * kNormStaticChunk);
  unsigned long long end = base + 2ull * kNormStaticChunk;
  if (end > nreal) end = nreal;
  double acc = 0.0;
  for (unsigned long long q = base + threadIdx.x; q < end; q += kThreads1) {
    const double v = (double)x[q];
    acc = fma(v, v, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[kThreads1 / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = lane < kThreads1 / 32 ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[blockIdx.x] = acc;
  }
}

__global__ void __launch_bounds__(kThreads2) norm_final_kernel(const double* __restrict__ part, int np,
                                                               double* __restrict__ out) {
  double acc = 0.0;
  for (int q = threadIdx.x; q < np; q += kThreads2) acc += part[q];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[kThreads2 / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = red[lane];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) *out = acc;
  }
}

// address of g_norm_scratch per device, looked up once per device
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {};

}  // namespace

double norm_static_sumsq(const void* u, bool fp64, unsigned long long n_complex, cudaStream_t st) {
  const unsigned long long nchunks = (n_complex + kNormStaticChunk - 1) / kNormStaticChunk;
  if (nchunks > (unsigned long long)kNormStaticMaxPartials)
    throw InvalidArg("tensor has " + std::to_string(n_complex) + " entries; the allocation-free norm handles at most " +
                     std::to_string(kNormStaticMaxEntries) + " (" + std::to_string(kNormStaticMaxPartials) +
                     " chunks of " + std::to_string(kNormStaticChunk) + ")");
  int dev = 0;
  FCGLE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Unsupported("device ordinal beyond the library's table");
  // the scratch used is the current device's: the stream and the tensor must be on it too
  int sdev = dev;
  if (st) FCGLE_CUDA(cudaStreamGetDevice(st, &sdev));
  if (sdev != dev)
    throw InvalidArg("the stream belongs to device " + std::to_string(sdev) + " but device " + std::to_string(dev) +
                     " is current");
  cudaPointerAttributes pa;
  FCGLE_CUDA(cudaPointerGetAttributes(&pa, u));
  if (pa.type == cudaMemoryTypeUnregistered) throw InvalidArg("u is not memory known to CUDA");
  if (pa.type == cudaMemoryTypeDevice && pa.device != dev)
    throw InvalidArg("u lives on device " + std::to_string(pa.device) + " but device " + std::to_string(dev) +
                     " is current");
  // One scratch array per device and process: calls that overlapped on one
  // device would race on it, so the whole call (which ends with a stream
  // synchronisation) holds this lock.
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    FCGLE_CUDA(cudaGetSymbolAddress(&p, g_norm_scratch));
    g_scratch[dev] = static_cast<double*>(p);
  }
  double* part = g_scratch[dev];
  const int np = (int)nchunks;
  const unsigned long long nreal = 2ull * n_complex;
  if (fp64)
    norm_partials_kernel<double><<<np, kThreads1, 0, st>>>(static_cast<const double*>(u), nreal, part);
  else
    norm_partials_kernel<float><<<np, kThreads1, 0, st>>>(static_cast<const float*>(u), nreal, part);
  FCGLE_CUDA(cudaGetLastError());
  norm_final_kernel<<<1, kThreads2, 0, st>>>(part, np, part + kNormStaticMaxPartials);
  FCGLE_CUDA(cudaGetLastError());
  double h = 0.0;
  FCGLE_CUDA(cudaMemcpyAsync(&h, part + kNormStaticMaxPartials, sizeof(double), cudaMemcpyDeviceToHost, st));
  FCGLE_CUDA(cudaStreamSynchronize(st));
  return h;
}

}  // namespace fcgle
