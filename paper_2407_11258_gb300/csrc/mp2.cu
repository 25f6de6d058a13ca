// Full-system MP2 correlation energy for the composite correction of Eq. 17:
//   Delta E_c,MP2 = E_c,MP2 - sum_F E_c,MP2^(F),
// where E_c,MP2 is the canonical closed-shell MP2 energy of the whole system (first-order amplitudes of
// Eq. 21 in the canonical basis) and the fragment terms are the MP2 fragment energies that
// lnocc_fragment_energy returns (Eq. 12-13 with t1 = 0 and the first-order amplitudes).
//
//   E_c,MP2 = sum_ijab (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b),  (ia|jb) = sum_Q B_Qia B_Qjb.
//
// The ov block of the DF factors is packed once as a K = naux operand with rows (i, a). Occupied rows are
// taken in chunks [i0, i0 + ni): one contraction gives X[(i, a)][(j, b)] = (ia|jb) for j < i0 + ni only
// (the pair energy of (i, j) equals that of (j, i), so pairs j > i are skipped and j < i counts twice),
// and a tile-pair kernel reduces each (i, j) block: for a v x v block M_ab = (ia|jb) with symmetric
// denominators D_ab = D_ba, the 32 x 32 tile pair (A, B), A < B, holds M_AB and M_BA and contributes
// sum (2 M_ab^2 + 2 M_ba^2 - 2 M_ab M_ba) / D_ab; a diagonal tile contributes sum M_ab (2 M_ab - M_ba) / D_ab.
// Block partials (FP64) are summed in a fixed order: the result does not depend on timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.h"

namespace lnocc {
namespace {

constexpr int kTile = 32;

// One block per (tile pair, j, i - i0); partial sums to part[blockIdx linear].
__global__ void __launch_bounds__(256) k_mp2_pairs(const double* __restrict__ X, long long ldx, int i0, int ni, int o,
                                                   int v, const double* __restrict__ eps, double* __restrict__ part) {
  __shared__ double P[kTile][kTile + 1];
  __shared__ double Q[kTile][kTile + 1];
  __shared__ double red[8];
  const int T = (v + kTile - 1) / kTile;
  const int j = blockIdx.y, ii = blockIdx.z, i = i0 + ii;
  const long long blk = (static_cast<long long>(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  double acc = 0.0;
  if (j <= i) {
    // tile pair index -> (ta, tb), ta <= tb, row-major over the upper triangle
    int p = blockIdx.x, ta = 0;
    while (p >= T - ta) {
      p -= T - ta;
      ++ta;
    }
    const int tb = ta + p;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;  // 32 x 8 threads
    const double* Mrow = X + static_cast<long long>(ii) * v * ldx + static_cast<long long>(j) * v;
    // P[r][c] = M[ta*32 + r][tb*32 + c],  Q[r][c] = M[tb*32 + r][ta*32 + c]  (coalesced along c)
    for (int r = ty; r < kTile; r += 8) {
      const int a = ta * kTile + r, b = tb * kTile + tx;
      P[r][tx] = (a < v && b < v) ? Mrow[static_cast<long long>(a) * ldx + b] : 0.0;
      const int a2 = tb * kTile + r, b2 = ta * kTile + tx;
      Q[r][tx] = (a2 < v && b2 < v) ? Mrow[static_cast<long long>(a2) * ldx + b2] : 0.0;
    }
    __syncthreads();
    const double eij = eps[i] + eps[j];
    for (int r = ty; r < kTile; r += 8) {
      const int a = ta * kTile + r, b = tb * kTile + tx;
      if (a >= v || b >= v) continue;
      const double D = eij - eps[o + a] - eps[o + b];
      const double mab = P[r][tx];
      if (ta == tb) {
        const double mba = P[tx][r];
        acc += mab * (2.0 * mab - mba) / D;
      } else {
        const double mba = Q[tx][r];
        acc += (2.0 * mab * mab + 2.0 * mba * mba - 2.0 * mab * mba) / D;
      }
    }
    if (j < i) acc *= 2.0;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    part[blk] = s;
  }
}

// out[0] += sum of part[0 .. n) in a fixed order (one block)
__global__ void k_mp2_sum(const double* __restrict__ part, long long n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) t += red[w];
    out[0] += t;
  }
}

struct Mp2Plan {
  size_t status, packed, X, part, total;
  int ni;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

Mp2Plan mp2_plan(bool bf, int o, int v, int N) {
  Mp2Plan p{};
  const size_t Kp = static_cast<size_t>(round_up(N, 64));
  const size_t ov = static_cast<size_t>(o) * v;
  // X chunk: ni * v rows of o * v FP64 columns, at most 512 MB (at least one occupied row)
  const size_t row_bytes = ov * v * 8;
  p.ni = static_cast<int>(std::max<size_t>(1, std::min<size_t>(o, (size_t(512) << 20) / std::max<size_t>(row_bytes, 1))));
  const int T = (v + kTile - 1) / kTile;
  p.status = 256;
  p.packed = align256(ov * Kp * (bf ? 4 : 8));
  p.X = align256(static_cast<size_t>(p.ni) * row_bytes);
  p.part = align256(static_cast<size_t>(T) * (T + 1) / 2 * o * p.ni * 8 + 8);
  p.total = p.status + p.packed + p.X + p.part;
  return p;
}

}  // namespace
}  // namespace lnocc

extern "C" int lnocc_mp2_workspace_bytes(int precision, int nocc, int nvir, int naux, long long* bytes) {
  using namespace lnocc;
  set_error("");
  if (!bytes || nocc < 1 || nvir < 1 || naux < 1 ||
      (precision != LNOCC_PREC_FP64 && precision != LNOCC_PREC_MIXED)) {
    set_error("lnocc_mp2_workspace_bytes: bad arguments");
    return LNOCC_EINVAL;
  }
  *bytes = static_cast<long long>(mp2_plan(precision == LNOCC_PREC_MIXED, nocc, nvir, naux).total);
  return LNOCC_OK;
}

extern "C" int lnocc_mp2_energy(int precision, int nocc, int nvir, int naux, const double* eps, const double* B_ov,
                                void* workspace, long long workspace_bytes, double* e_mp2, void* stream) {
  using namespace lnocc;
  set_error("");
  if (nocc < 1 || nvir < 1 || naux < 1 || !eps || !B_ov || !e_mp2 ||
      (precision != LNOCC_PREC_FP64 && precision != LNOCC_PREC_MIXED) ||
      static_cast<long long>(nocc) * nvir > (1LL << 30)) {
    set_error("lnocc_mp2_energy: bad arguments");
    return LNOCC_EINVAL;
  }
  const bool bf = precision == LNOCC_PREC_MIXED;
  const Mp2Plan plan = mp2_plan(bf, nocc, nvir, naux);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = static_cast<unsigned char*>(workspace);
  bool own = false;
  if (base) {
    if (workspace_bytes < static_cast<long long>(plan.total)) {
      set_error("lnocc_mp2_energy: workspace smaller than lnocc_mp2_workspace_bytes (" +
                std::to_string(plan.total) + " bytes)");
      return LNOCC_EINVAL;
    }
  } else {
    count_alloc();
    if (cudaMalloc(&base, plan.total) != cudaSuccess) {
      cudaGetLastError();
      set_error("lnocc_mp2_energy: device allocation failed");
      return LNOCC_ENOMEM;
    }
    own = true;
  }
  int* dstatus = reinterpret_cast<int*>(base);
  double* dres = reinterpret_cast<double*>(base + 128);
  Packed PA;
  PA.bf16 = bf;
  PA.rows = nocc * nvir;
  PA.Kp = round_up(naux, 64);
  PA.p = base + plan.status;
  double* X = reinterpret_cast<double*>(base + plan.status + plan.packed);
  double* part = reinterpret_cast<double*>(base + plan.status + plan.packed + plan.X);
  const int o = nocc, v = nvir, N = naux;
  const long long ov = 1LL * o * v;
  int st = LNOCC_OK;
  cudaError_t e = cudaMemsetAsync(base, 0, 256, s);  // status word and result start at zero
  if (e == cudaSuccess) {
    // rows (i, a), K = Q: element (r, Q) = B_ov[Q][i][a]
    pack(view(B_ov, kOne, Ax{o, v}, Ax{v, 1}, kOne, kOne, Ax{N, ov}), PA, s);
    const SplitWs saved = split_ws();
    split_ws() = SplitWs{};  // no split-K: its partials would need workspace beyond the plan
    const int T = (v + kTile - 1) / kTile;
    for (int i0 = 0; i0 < o; i0 += plan.ni) {
      const int ni = std::min(plan.ni, o - i0);
      const int ncols = (i0 + ni) * v;  // pairs j <= i only
      gemm_off(PA, i0 * v, PA, 0, ni * v, ncols, N, out_rowmajor(X, ncols), s, dstatus);
      dim3 grid(T * (T + 1) / 2, i0 + ni, ni);
      count_launch(2);
      k_mp2_pairs<<<grid, 256, 0, s>>>(X, ncols, i0, ni, o, v, eps, part);
      k_mp2_sum<<<1, 1024, 0, s>>>(part, static_cast<long long>(grid.x) * grid.y * grid.z, dres);
    }
    split_ws() = saved;
    int hst = 0;
    e = cudaMemcpyAsync(&hst, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(e_mp2, dres, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && hst != 0) {
      set_error("lnocc_mp2_energy: device wait timed out");
      st = LNOCC_ETIMEOUT;
    }
  }
  if (e != cudaSuccess) {
    set_error(std::string("lnocc_mp2_energy: ") + cudaGetErrorString(e));
    st = LNOCC_ECUDA;
  }
  if (own) cudaFree(base);
  return st;
}
