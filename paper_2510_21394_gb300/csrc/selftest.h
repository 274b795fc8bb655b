// Self-test of the bounded device-side waits (selftest.cu).
#pragma once

#include <cuda_runtime.h>

namespace fcgle {

// the code the self-test's wait records when it gives up
constexpr int kSelftestWaitCode = 99;

// Runs one wait on an mbarrier that never completes, through the kernels' own
// bounded wait, then a follow-up kernel on the same stream; synchronises st.
// Returns the code left in the device error word (kSelftestWaitCode when the
// wait gave up at its limit).  Throws if the wait completed or the follow-up
// did not run.
int bounded_wait_selftest(cudaStream_t st);

}  // namespace fcgle
