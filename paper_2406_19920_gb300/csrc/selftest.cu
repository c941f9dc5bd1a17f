// selftest.cu -- ibm_selftest_timeout: the bounded-wait paths without a fault.
//
// One CTA runs a wait that cannot complete, with the same bounded wait
// (mbar_wait, kWaitLimitNs unless a limit is given) every kernel of the
// library uses, and takes the same way out:
//   IBM_SELFTEST_TENSOR_MEMORY: the CTA holds tensor memory and waits on an
//     mbarrier that nothing arrives on (the tensor-core kernels' wait on an
//     MMA commit); after the wait gives up the warp frees the tensor memory.
//   IBM_SELFTEST_BULK_COPY: thread 0 announces twice the bytes it copies
//     and issues one in-bounds 16-byte bulk copy (the tile kernels' wait on
//     their cp.async.bulk rows); the copy lands but the barrier's
//     transaction count never drains.  After the wait gives up the CTA
//     waits once more, bounded, for copies in flight, as the tile kernels do.
// Either way the wait ORs kErrTimeout into the plan's error word and the
// kernel returns; the context stays usable.
#include "plan.h"
#include "tc.cuh"
#include "tma.cuh"

namespace ibm {

__global__ void k_selftest_timeout(int *err, const double *src, int path, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ __align__(16) double landing[2];
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (path == IBM_SELFTEST_BULK_COPY) {
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&bar, 32u);  // twice the 16 bytes copied below
      bulk_g2s(landing, src, 16u, &bar);
    }
    if (!__syncthreads_and(mbar_wait(&bar, 0, threadIdx.x == 0 ? err : nullptr, limit_ns)))
      mbar_wait(&bar, 0, nullptr, limit_ns);
    return;
  }
  if (threadIdx.x < 32) tc_alloc(&tbase, 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  // nothing arrives on bar: every thread's wait runs out
  mbar_wait(&bar, 0, threadIdx.x == 0 ? err : nullptr, limit_ns);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tc_dealloc(tmem, 32);
  }
}

}  // namespace ibm

using namespace ibm;

extern "C" int ibm_selftest_timeout(ibm_plan plan, int path, double limit_ms, void *stream) {
  if (!plan) return set_error(IBM_ERR_ARG, "ibm_selftest_timeout: NULL plan");
  if (path != IBM_SELFTEST_TENSOR_MEMORY && path != IBM_SELFTEST_BULK_COPY)
    return set_error(IBM_ERR_ARG, "ibm_selftest_timeout: path %d", path);
  if (!(limit_ms > 0) || !(limit_ms <= 5000))
    return set_error(IBM_ERR_ARG, "ibm_selftest_timeout: limit_ms must be in (0, 5000]");
  k_selftest_timeout<<<1, 64, 0, (cudaStream_t)stream>>>(plan->derr, plan->dsc, path,
                                                         (unsigned long long)(limit_ms * 1e6));
  IBM_CUDA_TRY(cudaGetLastError());
  return IBM_OK;
}
