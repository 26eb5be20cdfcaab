// Failure-detection diagnostic: the library's bounded wait (ptx.cuh) on an
// mbarrier that nothing arrives on.  The wait gives up after its limit, the
// block records a timeout in a status word and returns normally, exactly as
// the folds do when a producer never delivers; the context stays usable.

#include "ptx.cuh"
#include "srw_internal.h"

namespace srw {
namespace {

__global__ void wait_timeout_kernel(unsigned long long limit_ns, unsigned* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned abort_flag;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    abort_flag = 0u;
    ptx::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !ptx::mbar_wait(&bar, 0, &abort_flag, limit_ns)) atomicOr(status, kStatusTimeout);
  __syncthreads();
}

}  // namespace
}  // namespace srw

extern "C" srw_status srw_diag_wait_timeout(unsigned limit_us) {
  if (limit_us < 1 || limit_us > 1000000) return SRW_EINVAL;
  unsigned* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) return SRW_ENOMEM;
  unsigned st = 0;
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned));
  if (e == cudaSuccess) {
    srw::wait_timeout_kernel<<<1, 32>>>((unsigned long long)limit_us * 1000ull, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&st, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return SRW_ECUDA;
  return (st & srw::kStatusTimeout) ? SRW_ETIMEOUT : SRW_OK;
}
