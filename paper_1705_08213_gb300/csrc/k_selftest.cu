// Self-test of the bounded waits that every pipeline of the library uses
// (mbar_wait_bounded): a wait that nothing can complete must give up after its
// time limit, record CCC_ETIMEOUT in the status word and return, leaving the
// CUDA context usable.
#include "ccc_dev.cuh"
#include "ccc_launch.h"

namespace ccc {
namespace {

// One CTA: thread 0 waits for phase 0 of an mbarrier with an arrival count of
// one that no thread arrives on; the other threads wait for it at the final
// barrier.  The wait ends by its time limit (device global timer).
__global__ void k_wait_selftest(int32_t *status, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_bounded(smem_u32(&bar), 0, status, &abort_flag, limit_ns);
  __syncthreads();
}

}  // namespace

int launch_wait_selftest(int32_t *status, uint64_t limit_ns, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(status, limit_ns);
  return note_launch();
}

}  // namespace ccc
