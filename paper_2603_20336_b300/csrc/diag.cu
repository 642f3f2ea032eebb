// Self-test of the bounded-wait mechanism every pipelined kernel relies on:
// one warp waits, with the same mbar_wait as the scoring kernels, on an
// mbarrier that nothing arrives on.  The wait gives up after `budget` SM cycles,
// records GEM_ERR_TIMEOUT in the workspace's status word and the kernel
// returns, so the context stays usable.
#include "internal.h"
#include "ptx.cuh"

namespace gem {
namespace {

__global__ void wait_selftest_kernel(int* status, long long budget) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  __syncwarp();
  // nothing arrives on `bar`: phase 0 never completes
  mbar_wait(&bar, 0, status, &abort_flag, budget);
}

}  // namespace

gem_status launch_wait_selftest(int* status, long long budget, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(status, budget);
  GEM_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return GEM_OK;
}

}  // namespace gem
