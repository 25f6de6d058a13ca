// lnocc_gemm_noalloc: the contraction engine's C = A B^T without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed device-memory budget handed out
// by another allocator (a memory pool or arena that owns all free memory), and code that must not
// synchronize the device (cudaMalloc / cudaFree can wait for outstanding work). For them this entry
// point keeps its working memory -- the packed operands and the device status word -- in a
// file-scope __device__ array that lives as long as the library is loaded on each GPU.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace lnocc {
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB on every GPU that loads the library
constexpr size_t kStatusBytes = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array per device (the host-side symbol is only a stand-in).
void* g_scratch_addr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error(std::string("lnocc_gemm_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return LNOCC_ECUDA;
  }
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("lnocc_gemm_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return LNOCC_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return LNOCC_OK;
}

}  // namespace
}  // namespace lnocc

extern "C" int lnocc_gemm_noalloc(int precision, int M, int N, int K, const double* A, const double* B, double* C,
                                  void* stream) {
  using namespace lnocc;
  set_error("");
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C ||
      (precision != LNOCC_PREC_FP64 && precision != LNOCC_PREC_MIXED)) {
    set_error("lnocc_gemm_noalloc: bad arguments");
    return LNOCC_EINVAL;
  }
  const bool bf = precision == LNOCC_PREC_MIXED;
  const size_t Kp = static_cast<size_t>(round_up(K, 64));
  const size_t esz = bf ? 4 : 8;  // BF16 hi + lo, or FP64
  const size_t bytesA = (static_cast<size_t>(M) * Kp * esz + 255) / 256 * 256;
  const size_t bytesB = static_cast<size_t>(N) * Kp * esz;
  if (kStatusBytes + bytesA + bytesB > kNoAllocBytes) {
    set_error("lnocc_gemm_noalloc: (M + N) * roundup(K, 64) packed operands exceed the 32 MiB scratch (" +
              std::to_string(kStatusBytes + bytesA + bytesB) + " bytes needed)");
    return LNOCC_EINVAL;
  }
  unsigned char* base = nullptr;
  const int st0 = scratch_for_current_device(&base);
  if (st0 != LNOCC_OK) return st0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* dstatus = reinterpret_cast<int*>(base);
  Packed PA, PB;
  PA.bf16 = PB.bf16 = bf;
  PA.p = base + kStatusBytes;
  PB.p = base + kStatusBytes + bytesA;
  // the status word must start at zero; the packed operands are fully rewritten by the packing kernels
  LN_CUDA(cudaMemsetAsync(dstatus, 0, sizeof(int), s));
  const Ax one{1, 0};
  pack(view(A, one, one, Ax{M, K}, one, one, Ax{K, 1}), PA, s);
  pack(view(B, one, one, Ax{N, K}, one, one, Ax{K, 1}), PB, s);
  // no split-K here: its partials would need workspace of their own; and no tile timing by the
  // autotuner (its mode 2 allocates a scratch output and synchronizes): table lookups only
  const SplitWs saved = split_ws();
  split_ws() = SplitWs{};
  const bool timing = autotune_timing_allowed();
  autotune_timing_allowed() = false;
  gemm(PA, PB, M, N, K, out_rowmajor(C, N), s, dstatus);
  autotune_timing_allowed() = timing;
  split_ws() = saved;
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("lnocc_gemm_noalloc: ") + cudaGetErrorString(e));
    return LNOCC_ECUDA;
  }
  if (st != 0) {
    set_error("lnocc_gemm_noalloc: device wait timed out");
    return LNOCC_ETIMEOUT;
  }
  return LNOCC_OK;
}
