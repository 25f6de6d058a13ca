// Local-Hamiltonian integrals from k-point DF factors (Eq. 27a), reduced to the real Gamma-point form the
// fragment solver takes (lnocc_build_ints):
//   V_pqrs = sum_q sum_P L^P_pq(q) L^P_rs(-q).
// For real orbitals the factors satisfy L_pq(q) = L_qp(q) and L(-q) = conj L(q), so a pair (q, -q) adds
// L_pq(q) conj L_rs(q) + conj L_pq(q) L_rs(q) = 2 (Re L_pq Re L_rs + Im L_pq Im L_rs), and a self-conjugate
// q (q = -q) is real and adds L_pq L_rs. The real factors B~ are therefore sqrt(2) Re L(q) and
// sqrt(2) Im L(q) for one q of each pair and Re L(q) for each self-conjugate q: N_k * naux auxiliary
// functions, with sum_Q B~_Qpq B~_Qrs = V_pqrs exactly, at half the work of complex contractions.
// The input symmetries are checked on the device first (max-reductions): factors that do not belong to
// real orbitals are rejected.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace lnocc {
namespace {

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* a, double x) {
  // non-negative doubles order like their bit patterns
  atomicMax(a, static_cast<unsigned long long>(__double_as_longlong(x)));
}

// out[0] = max |L|, out[1] = max |L(-q) - conj L(q)|, out[2] = max |L_pr(q) - L_rp(q)|
__global__ void k_kpt_check(const double2* __restrict__ L, const int* __restrict__ qneg, int nk, long long per_q,
                            int n, unsigned long long* __restrict__ out) {
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  const long long tot = per_q * nk;
  const long long nn = 1LL * n * n;
  for (long long x = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; x < tot;
       x += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(x / per_q);
    const long long r = x % per_q;
    const long long blk = r / nn;
    const int p = static_cast<int>((r % nn) / n), s = static_cast<int>(r % n);
    const double2 a = L[x];
    const double2 b = L[static_cast<long long>(qneg[q]) * per_q + r];
    const double2 t = L[static_cast<long long>(q) * per_q + blk * nn + static_cast<long long>(s) * n + p];
    m0 = fmax(m0, hypot(a.x, a.y));
    m1 = fmax(m1, hypot(b.x - a.x, b.y + a.y));
    m2 = fmax(m2, hypot(a.x - t.x, a.y - t.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if (threadIdx.x % 32 == 0) {
    atomic_max_nonneg(out, m0);
    atomic_max_nonneg(out + 1, m1);
    atomic_max_nonneg(out + 2, m2);
  }
}

struct OutBlock {
  int q, imag;
  double scale;
};

// B~[b * per_q + r] = scale_b * (Re or Im) L[q_b][r] for output blocks b (r runs over (P, p, r))
__global__ void k_kpt_real(const double2* __restrict__ L, const OutBlock* __restrict__ blocks, int nblocks,
                           long long per_q, double* __restrict__ B) {
  const long long tot = per_q * nblocks;
  for (long long x = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; x < tot;
       x += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(x / per_q);
    const long long r = x % per_q;
    const OutBlock ob = blocks[b];
    const double2 z = L[static_cast<long long>(ob.q) * per_q + r];
    B[x] = ob.scale * (ob.imag ? z.y : z.x);
  }
}

}  // namespace
}  // namespace lnocc

extern "C" int lnocc_kpoint_df(int nk, int naux, int n, const double* L, const int* qneg, double* B_out,
                               double* sym_err, void* stream) {
  using namespace lnocc;
  set_error("");
  if (nk < 1 || naux < 1 || n < 1 || !L || !qneg || !B_out || 1LL * naux * n * n > (1LL << 40)) {
    set_error("lnocc_kpoint_df: bad arguments");
    return LNOCC_EINVAL;
  }
  for (int q = 0; q < nk; ++q) {
    if (qneg[q] < 0 || qneg[q] >= nk || qneg[qneg[q]] != q) {
      set_error("lnocc_kpoint_df: qneg must be an involution of [0, nk)");
      return LNOCC_EINVAL;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long per_q = 1LL * naux * n * n;
  std::vector<OutBlock> hb;
  for (int q = 0; q < nk; ++q) {
    if (qneg[q] == q) {
      hb.push_back(OutBlock{q, 0, 1.0});
    } else if (q < qneg[q]) {
      hb.push_back(OutBlock{q, 0, std::sqrt(2.0)});
      hb.push_back(OutBlock{q, 1, std::sqrt(2.0)});
    }
  }
  // each output block is naux auxiliary functions (one q, real or imaginary part): rows (Q, p, r) of B~
  const std::vector<OutBlock>& rows = hb;
  // one allocation: 64 bytes of maxima, the -q map, then the block table at a 16-byte boundary
  const size_t q_bytes = (sizeof(int) * nk + 15) / 16 * 16;
  void* d = nullptr;
  count_alloc();
  LN_CUDA(cudaMalloc(&d, 64 + q_bytes + sizeof(OutBlock) * rows.size()));
  unsigned long long* dmax = static_cast<unsigned long long*>(d);
  int* dq = reinterpret_cast<int*>(static_cast<char*>(d) + 64);
  OutBlock* drows = reinterpret_cast<OutBlock*>(static_cast<char*>(d) + 64 + q_bytes);
  cudaError_t e = cudaMemsetAsync(dmax, 0, 64, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dq, qneg, sizeof(int) * nk, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(drows, rows.data(), sizeof(OutBlock) * rows.size(), cudaMemcpyHostToDevice, s);
  unsigned long long hm[3] = {0, 0, 0};
  if (e == cudaSuccess) {
    const double2* Lz = reinterpret_cast<const double2*>(L);
    const long long tot = per_q * nk;
    const int grid = static_cast<int>(std::max(1LL, std::min<long long>((tot + 255) / 256, 152LL * 16)));
    count_launch();
    k_kpt_check<<<grid, 256, 0, s>>>(Lz, dq, nk, per_q, n, dmax);
    e = cudaMemcpyAsync(hm, dmax, sizeof(hm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    cudaFree(d);
    set_error(std::string("lnocc_kpoint_df: ") + cudaGetErrorString(e));
    return LNOCC_ECUDA;
  }
  double mx[3];
  for (int k = 0; k < 3; ++k) {
    long long bits = static_cast<long long>(hm[k]);
    std::memcpy(&mx[k], &bits, sizeof(double));
  }
  const double err = std::max(mx[1], mx[2]);
  if (sym_err) *sym_err = mx[0] > 0 ? err / mx[0] : 0.0;
  if (err > 1e-10 * mx[0]) {
    cudaFree(d);
    set_error("lnocc_kpoint_df: factors lack the symmetries of real orbitals (L_pq(q) = L_qp(q), L(-q) = conj L(q))");
    return LNOCC_EINVAL;
  }
  const long long tot = per_q * static_cast<long long>(rows.size());
  const int grid = static_cast<int>(std::max(1LL, std::min<long long>((tot + 255) / 256, 152LL * 16)));
  count_launch();
  k_kpt_real<<<grid, 256, 0, s>>>(reinterpret_cast<const double2*>(L), drows, static_cast<int>(rows.size()), per_q,
                                  B_out);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error(std::string("lnocc_kpoint_df: ") + cudaGetErrorString(e));
    return LNOCC_ECUDA;
  }
  return LNOCC_OK;
}
