// Allocation-free discrete L2 norm (scratch in static device memory).
#pragma once

#include <cuda_runtime.h>

namespace fcgle {

// one FP64 partial sum per chunk of kNormStaticChunk complex entries
constexpr int kNormStaticChunk = 8192;
constexpr int kNormStaticMaxPartials = 32768;   // 256 KB of scratch
constexpr unsigned long long kNormStaticMaxEntries =
    (unsigned long long)kNormStaticChunk * kNormStaticMaxPartials;   // 2^28 complex entries

// sum_j |u_j|^2 over n_complex interleaved complex entries (complex128 if
// fp64, else complex64) on stream st; synchronises st.  Throws InvalidArg
// beyond kNormStaticMaxEntries.
double norm_static_sumsq(const void* u, bool fp64, unsigned long long n_complex, cudaStream_t st);

}  // namespace fcgle
