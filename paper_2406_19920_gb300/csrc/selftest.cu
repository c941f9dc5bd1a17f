// selftest.cu -- ibm_selftest_timeout: the bounded-wait path without a fault.
//
// One CTA allocates tensor memory and waits on an mbarrier that nothing
// completes, with the same bounded wait (mbar_wait_ns) the tensor-core and
// bulk-copy kernels use.  The wait gives up after the requested time, ORs
// kErrTimeout into the plan's error word, the warp frees the tensor memory
// and the kernel returns; the context stays usable.
#include "plan.h"
#include "tc.cuh"
#include "tma.cuh"

namespace ibm {

__global__ void k_selftest_timeout(int *err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) tc_alloc(&tbase, 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  // nothing arrives on bar: every thread's wait runs out
  mbar_wait_ns(&bar, 0, threadIdx.x == 0 ? err : nullptr, limit_ns);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tc_dealloc(tmem, 32);
  }
}

}  // namespace ibm

using namespace ibm;

extern "C" int ibm_selftest_timeout(ibm_plan plan, double limit_ms, void *stream) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_selftest_timeout: NULL plan");
  if (!(limit_ms > 0) || !(limit_ms <= 5000))
    return set_error(IBM_ERR_ARG, "ibm_selftest_timeout: limit_ms must be in (0, 5000]");
  k_selftest_timeout<<<1, 64, 0, (cudaStream_t)stream>>>(plan->derr, (unsigned long long)(limit_ms * 1e6));
  IBM_CUDA_TRY(cudaGetLastError());
  return IBM_OK;
}
