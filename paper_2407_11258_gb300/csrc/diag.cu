// Diagnostic: the bounded device wait that every mbarrier wait of the library goes through
// (mbar_wait_for in ptx.cuh), exercised on its own. One thread initialises an mbarrier with an arrival
// count of one and waits for its first phase with a wall-clock budget. With `arrive` set it arrives
// first, so the wait succeeds at once; without, nothing ever arrives, the budget runs out, the kernel
// records the timeout in the status word and returns. No TMA copy or MMA is issued, so nothing is in
// flight when it gives up. The host maps the status to LNOCC_ETIMEOUT, as it does after the
// contraction kernels.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "ptx.cuh"

namespace lnocc {
namespace {

__global__ void k_bounded_wait(int arrive, unsigned long long budget_ns, int* status, unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_barrier_init();
  if (arrive) mbar_arrive(&bar);
  const unsigned long long t0 = globaltimer();
  const bool ok = mbar_wait_for(&bar, 0, budget_ns);
  *waited_ns = globaltimer() - t0;
  if (!ok) atomicExch(status, kDevTimeoutMma);
}

}  // namespace
}  // namespace lnocc

extern "C" int lnocc_debug_wait(int arrive, long long budget_ns, long long* waited_ns, void* stream) {
  using namespace lnocc;
  set_error("");
  if (budget_ns < 0 || budget_ns > 2000000000LL) {
    set_error("lnocc_debug_wait: budget must be in [0, 2e9] ns");
    return LNOCC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* d = nullptr;
  count_alloc();
  LN_CUDA(cudaMalloc(&d, 16));
  int* status = static_cast<int*>(d);
  unsigned long long* dw = reinterpret_cast<unsigned long long*>(static_cast<char*>(d) + 8);
  int hst = 0;
  unsigned long long hw = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, 16, s);
  if (e == cudaSuccess) {
    count_launch();
    k_bounded_wait<<<1, 32, 0, s>>>(arrive ? 1 : 0, static_cast<unsigned long long>(budget_ns), status, dw);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hw, dw, sizeof(hw), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error(std::string("lnocc_debug_wait: ") + cudaGetErrorString(e));
    return LNOCC_ECUDA;
  }
  if (waited_ns) *waited_ns = static_cast<long long>(hw);
  if (hst != 0) {
    set_error("lnocc_debug_wait: device wait timed out");
    return LNOCC_ETIMEOUT;
  }
  return LNOCC_OK;
}
