// rid_selftest.cu -- the library's bounded device waits, made to run out.
//
// Every device-side wait of the library gives up after kWaitLimitNs of the
// GPU's global timer, records kErrTimeout in the device state and lets its
// kernel exit.  This covers the grid barrier of the cooperative LUPP panel and
// the mbarrier waits of the tensor-core kernels.  A stuck wait therefore ends
// the call with ID_ERR_TIMEOUT, and the CUDA context stays usable.
// id_selftest_timeout runs one wait of each kind that nothing can satisfy.  It
// uses the same helpers as the kernels, so the timeout path itself is tested.
#include <cuda_runtime.h>
#include <stdint.h>

#include "randid.h"
#include "rid_common.cuh"
#include "rid_tc_common.cuh"

namespace rid {
namespace {

// One block adds one arrival; the target asks for two, so the counter never
// reaches it and the barrier can only time out.
__global__ void k_unsatisfied_grid_barrier(DevState* st) { grid_barrier(&st->bar[0], 2u, st); }

// An mbarrier that expects one arrival, which never comes: phase 0 never
// completes and the wait can only time out.  Nothing asynchronous was issued
// on it, so the block may exit at once.
__global__ void k_unsatisfied_mbarrier(DevState* st) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tcx::mbar_init(&bar, 1);
    tcx::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) tcx::mbar_wait(&bar, 0, st);
}

}  // namespace
}  // namespace rid

extern "C" int id_selftest_timeout(int which, void* ws, size_t ws_bytes, void* stream) {
  if (which != 0 && which != 1) return -1;
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) % 256) != 0 || ws_bytes < sizeof(rid::DevState))
    return ID_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rid::DevState* st = static_cast<rid::DevState*>(ws);
  if (cudaMemsetAsync(st, 0, sizeof(rid::DevState), s) != cudaSuccess) return ID_ERR_CUDA;
  if (which == 0)
    rid::k_unsatisfied_grid_barrier<<<1, 32, 0, s>>>(st);
  else
    rid::k_unsatisfied_mbarrier<<<1, 32, 0, s>>>(st);
  if (cudaGetLastError() != cudaSuccess) return ID_ERR_CUDA;
  rid::DevState h;
  if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ID_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ID_ERR_CUDA;
  return (h.err & rid::kErrTimeout) ? ID_ERR_TIMEOUT : ID_OK;
}
