// selftest.cu -- failure-detection self-test of the bounded device waits
// (ndg_selftest_timeout): one CTA waits on an mbarrier that nothing ever
// completes, with the same wait helpers as the tensor-core kernels.  When
// the bound runs out the CTA records NDG_ERR_TIMEOUT in the workspace status
// word and returns, so the context stays usable; nothing faults or traps.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "tcgen05.cuh"

namespace ndg {

// which = 0: the sleeping warp wait (warp_wait: lane 0 polls with the
// suspend-time hint, kSleepLimit polls); which = 1: the spinning wait of the
// kernels' final drain (mbar_wait_bounded, kWaitLimit polls).
__global__ void selftest_wait_kernel(int* status, int which) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // one arrival expected; none is ever made
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    bool ok;
    if (which == 0) {
      ok = warp_wait(&bar, 0, &abort_flag);
    } else {
      int r = 1;
      if (threadIdx.x == 0) r = mbar_wait_bounded(&bar, 0, kWaitLimit) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, r, 0) != 0;
    }
    if (!ok && threadIdx.x == 0 && status) set_status(status, NDG_ERR_TIMEOUT);
  }
}

int launch_selftest_wait(int* status, int which, cudaStream_t s) {
  selftest_wait_kernel<<<1, 64, 0, s>>>(status, which);
  return 1;
}

}  // namespace ndg
