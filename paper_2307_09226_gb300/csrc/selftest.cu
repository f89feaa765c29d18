// Failure-detection self test.  Every device-side wait in the library is bounded: it
// polls an mbarrier phase, reads %globaltimer, and after its limit records
// kStatusTimeout in the context's status word and returns, so that a stuck wait never
// hangs the GPU and the host learns of it from rsim_sync_status().  This kernel runs that
// same bounded wait on a barrier phase that nothing completes, so a test can make the
// limit run out on purpose and check the status and that the context still works.
#include "rsim_internal.h"

namespace rsim {
namespace {

__global__ void wait_timeout_selftest(unsigned* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init_single(&bar);
  __syncthreads();
  // no thread arrives and no copy completes a transaction: phase 0 never completes
  const bool done = wait_phase_bounded(&bar, 0, limit_ns);
  if (!done && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned* status, unsigned long long limit_ns, cudaStream_t st) {
  wait_timeout_selftest<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

}  // namespace rsim
