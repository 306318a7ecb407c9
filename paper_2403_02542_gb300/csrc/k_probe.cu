// Check of the bounded mbarrier wait that every tensor-core pipeline uses.
//
// One thread initialises an mbarrier that nothing ever arrives on and waits
// for its first phase with the pipelines' wait helper, bounded by a
// caller-chosen number of cycles.  When the wait gives up the kernel raises
// bit 128 of the context's tensor-core error flag, as a pipeline stage that
// timed out does, and returns; afqmc_sync then reports the timeout.  No copy,
// MMA or TMEM allocation is involved, so nothing is left in flight.
#include "internal.cuh"
#include "tc_common.cuh"

namespace afq {
namespace {

constexpr int kProbeFlag = 128;

__global__ void wait_probe_kernel(int* err, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) atomicOr(err, kProbeFlag);
}

}  // namespace
}  // namespace afq

using namespace afq;

extern "C" afqmc_status afqmc_wait_probe(afqmc_ctx* c, long long limit_cycles) {
  if (!c) return AFQMC_EINVAL;
  if (limit_cycles < 1 || limit_cycles > kTcWaitCycles) return AFQMC_EINVAL;
  if (!c->tc.ok || !c->tc.err) return AFQMC_ENOTSUP;
  wait_probe_kernel<<<1, 32, 0, c->stream>>>(static_cast<int*>(c->tc.err), limit_cycles);
  c->launches += 1;
  return cudaGetLastError() == cudaSuccess ? AFQMC_OK : AFQMC_ECUDA;
}
