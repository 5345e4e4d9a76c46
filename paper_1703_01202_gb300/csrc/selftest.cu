// Self-test of the failure detection in the library's TMA copy rings: every
// mbarrier wait there is bounded (mbar_wait_bounded gives up after a cycle
// limit, the caller records PFC_ETIMEOUT, drains its own copies and returns),
// so a copy that never lands ends the kernel with an error status instead of
// a hung GPU.  This kernel exercises that wait on a barrier with no copy in
// flight: with no arrival its phase never completes and the wait must run out.
#include <cuda_runtime.h>

#include "../../include/pfc.h"
#include "pfc_internal.cuh"
#include "pfc_tma.cuh"

namespace pfc {
namespace {

__global__ void k_wait_selftest(int arrive, long long limit, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(&bar);
    *status = mbar_wait_bounded(&bar, 0u, limit) ? PFC_OK : PFC_ETIMEOUT;
  }
}

}  // namespace
}  // namespace pfc

extern "C" int pfc_wait_selftest(int arrive, long long limit_cycles, int* dev_status, void* cuda_stream) {
  if (!dev_status || (arrive != 0 && arrive != 1) || limit_cycles < 1 || limit_cycles > pfc::kWaitCycles)
    return PFC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  pfc::k_wait_selftest<<<1, 32, 0, st>>>(arrive, limit_cycles, dev_status);
  pfc::count_launches(1);
  if (cudaGetLastError() != cudaSuccess) return PFC_ECUDA;
  int h = PFC_ECUDA;
  if (cudaMemcpyAsync(&h, dev_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PFC_ECUDA;
  return h;
}
