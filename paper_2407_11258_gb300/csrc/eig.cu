// Symmetric eigendecomposition in FP64 on the device: parallel cyclic Jacobi.
//
// A sweep visits every pair (p, q) once in m - 1 rounds of the round-robin ("circle") schedule over
// m = n rounded up to even players: in round r, pair 0 is (m - 1, r) and pair k >= 1 is
// ((r + k) mod (m - 1), (r - k) mod (m - 1)). The m / 2 pairs of one round are disjoint, so their plane
// rotations commute: one kernel computes the angles that zero every A_pq of the round, a second applies
// A <- J^T A J as independent 2 x 2 blocks (rows of pair P, columns of pair Q) and V <- V J. A player
// index >= n (odd n) is a bye. Rotation angles follow the classical form: theta = (A_qq - A_pp) / 2A_pq,
// t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1 / sqrt(1 + t^2), s = t c, which gives
// A'_pp = A_pp - t A_pq, A'_qq = A_qq + t A_pq, A'_pq = 0. After each sweep the off-diagonal norm is read
// back; the host stops when it is below 1e-15 of the Frobenius norm (Jacobi converges quadratically) or
// after 60 sweeps. Eigenvalues are then sorted (single-block bitonic sort) with their vectors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "internal.h"

namespace lnocc {
namespace {

__device__ __forceinline__ void jac_pair(int r, int k, int m, int* p, int* q) {
  const int m1 = m - 1;
  if (k == 0) {
    *p = m1;
    *q = r;
  } else {
    *p = (r + k) % m1;
    *q = (r - k + m1) % m1;
  }
}

__global__ void k_jac_angles(const double* __restrict__ A, int n, int m, int r, double2* __restrict__ cs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m / 2) return;
  int p, q;
  jac_pair(r, k, m, &p, &q);
  double c = 1.0, s = 0.0;
  if (p < n && q < n) {
    const double apq = A[static_cast<long long>(p) * n + q];
    const double app = A[static_cast<long long>(p) * n + p], aqq = A[static_cast<long long>(q) * n + q];
    // skip a rotation whose off-diagonal element is negligible against its diagonal pair
    if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
      const double th = (aqq - app) / (2.0 * apq);
      const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      c = 1.0 / sqrt(t * t + 1.0);
      s = t * c;
    }
  }
  cs[k] = make_double2(c, s);
}

// Work items: (m/2)^2 blocks of A, then n * (m/2) row-pairs of V.
__global__ void k_jac_rotate(double* __restrict__ A, double* __restrict__ V, int n, int m, int r,
                             const double2* __restrict__ cs) {
  const long long h = m / 2;
  const long long nA = h * h, nV = static_cast<long long>(n) * h;
  for (long long w = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; w < nA + nV;
       w += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (w < nA) {
      const int kP = static_cast<int>(w / h), kQ = static_cast<int>(w % h);
      int p1, q1, p2, q2;
      jac_pair(r, kP, m, &p1, &q1);
      jac_pair(r, kQ, m, &p2, &q2);
      const double2 g1 = cs[kP], g2 = cs[kQ];
      const bool r1 = p1 < n, r2 = q1 < n, c1 = p2 < n, c2 = q2 < n;  // byes are absent rows / columns
      const double a = (r1 && c1) ? A[static_cast<long long>(p1) * n + p2] : 0.0;
      const double b = (r1 && c2) ? A[static_cast<long long>(p1) * n + q2] : 0.0;
      const double cc = (r2 && c1) ? A[static_cast<long long>(q1) * n + p2] : 0.0;
      const double d = (r2 && c2) ? A[static_cast<long long>(q1) * n + q2] : 0.0;
      // rows: p <- c row_p - s row_q, q <- s row_p + c row_q
      const double a1 = g1.x * a - g1.y * cc, b1 = g1.x * b - g1.y * d;
      const double c1v = g1.y * a + g1.x * cc, d1 = g1.y * b + g1.x * d;
      // columns: p <- c col_p - s col_q, q <- s col_p + c col_q
      double a2 = g2.x * a1 - g2.y * b1, b2 = g2.y * a1 + g2.x * b1;
      double c2v = g2.x * c1v - g2.y * d1, d2 = g2.y * c1v + g2.x * d1;
      if (kP == kQ) b2 = c2v = 0.0;  // the element this rotation annihilates
      if (r1 && c1) A[static_cast<long long>(p1) * n + p2] = a2;
      if (r1 && c2) A[static_cast<long long>(p1) * n + q2] = b2;
      if (r2 && c1) A[static_cast<long long>(q1) * n + p2] = c2v;
      if (r2 && c2) A[static_cast<long long>(q1) * n + q2] = d2;
    } else {
      const long long x = w - nA;
      const int i = static_cast<int>(x / h), k = static_cast<int>(x % h);
      int p, q;
      jac_pair(r, k, m, &p, &q);
      if (p >= n || q >= n) continue;
      const double2 g = cs[k];
      double* row = V + static_cast<long long>(i) * n;
      const double vp = row[p], vq = row[q];
      row[p] = g.x * vp - g.y * vq;
      row[q] = g.y * vp + g.x * vq;
    }
  }
}

// out[0] = sum of squares of the off-diagonal elements, out[1] = of all elements (one block, fixed order)
__global__ void k_jac_norms(const double* __restrict__ A, int n, double* __restrict__ out) {
  __shared__ double red[2][32];
  double off = 0.0, all = 0.0;
  const long long nn = static_cast<long long>(n) * n;
  for (long long idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const double x = A[idx];
    all += x * x;
    if (idx / n != idx % n) off += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    all += __shfl_xor_sync(0xffffffffu, all, o);
  }
  if (threadIdx.x % 32 == 0) {
    red[0][threadIdx.x / 32] = off;
    red[1][threadIdx.x / 32] = all;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    out[0] = s0;
    out[1] = s1;
  }
}

__global__ void k_identity(double* V, int n) {
  const long long nn = static_cast<long long>(n) * n;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < nn;
       idx += static_cast<long long>(gridDim.x) * blockDim.x)
    V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

// Eigenvalues (diagonal of A) sorted with a bitonic sort in one block of 1024 threads; `order[k]` is
// the column of V holding the k-th value (decreasing when `desc`, else increasing; ties by index).
constexpr int kSortMax = 8192;
__global__ void __launch_bounds__(1024) k_eig_sort(const double* __restrict__ A, int n, int desc,
                                                   double* __restrict__ w, int* __restrict__ order) {
  extern __shared__ unsigned char sm[];
  int P = 1;
  while (P < n) P <<= 1;
  double* key = reinterpret_cast<double*>(sm);
  int* idx = reinterpret_cast<int*>(key + P);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const double x = i < n ? A[static_cast<long long>(i) * n + i] : 0.0;
    // pad entries sort last in either direction
    key[i] = i < n ? (desc ? -x : x) : INFINITY;
    idx[i] = i;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const bool gt = key[i] > key[j] || (key[i] == key[j] && idx[i] > idx[j]);
          if (gt == up) {
            const double tk = key[i];
            key[i] = key[j];
            key[j] = tk;
            const int ti = idx[i];
            idx[i] = idx[j];
            idx[j] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    w[i] = desc ? -key[i] : key[i];
    order[i] = idx[i];
  }
}

// out[:, k] = V[:, order[k]] for k < ncols (n x ncols output, row-major, leading dimension ldo)
__global__ void k_gather_cols(const double* __restrict__ V, int n, const int* __restrict__ order, int ncols,
                              double* __restrict__ out, int ldo) {
  const long long tot = static_cast<long long>(n) * ncols;
  for (long long x = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; x < tot;
       x += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(x / ncols), k = static_cast<int>(x % ncols);
    out[static_cast<long long>(i) * ldo + k] = V[static_cast<long long>(i) * n + order[k]];
  }
}

int grid_of(long long work, int threads) {
  return static_cast<int>(std::max(1LL, std::min<long long>((work + threads - 1) / threads, 152LL * 32)));
}

}  // namespace

// A [n][n] symmetric (destroyed); on return w [n] holds the eigenvalues (decreasing when desc, else
// increasing), order [n] their columns in V, and V [n][n] the eigenvectors as columns (A V = V diag).
// Device pointers; `scratch` holds at least 16 doubles + m/2 double2. Synchronizes `s` once per sweep.
int sym_eig(double* A, double* V, double* w, int* order, int n, bool desc, double* scratch, cudaStream_t s,
            int* sweeps_out) {
  if (n < 1 || n > kSortMax) {
    set_error("eigendecomposition: size must be in [1, " + std::to_string(kSortMax) + "]");
    return LNOCC_EINVAL;
  }
  const int m = n + (n & 1);
  double* norms = scratch;
  double2* cs = reinterpret_cast<double2*>(scratch + 16);
  count_launch();
  k_identity<<<grid_of(1LL * n * n, 256), 256, 0, s>>>(V, n);
  int sweep = 0;
  double h[2] = {0.0, 0.0};
  if (n > 1) {
    const long long work = 1LL * (m / 2) * (m / 2) + 1LL * n * (m / 2);
    for (sweep = 0; sweep < 60; ++sweep) {
      count_launch();
      k_jac_norms<<<1, 1024, 0, s>>>(A, n, norms);
      LN_CUDA(cudaMemcpyAsync(h, norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      LN_CUDA(cudaStreamSynchronize(s));
      if (!std::isfinite(h[1])) {
        set_error("eigendecomposition: non-finite matrix");
        return LNOCC_ENUMERIC;
      }
      if (h[0] <= 1e-30 * h[1] || h[0] == 0.0) break;
      for (int r = 0; r < m - 1; ++r) {
        count_launch(2);
        k_jac_angles<<<grid_of(m / 2, 128), 128, 0, s>>>(A, n, m, r, cs);
        k_jac_rotate<<<grid_of(work, 256), 256, 0, s>>>(A, V, n, m, r, cs);
      }
    }
    if (sweep == 60) {
      set_error("eigendecomposition: Jacobi sweeps did not converge");
      return LNOCC_ENOCONV;
    }
  }
  int P = 1;
  while (P < n) P <<= 1;
  const size_t smem = static_cast<size_t>(P) * (sizeof(double) + sizeof(int));
  if (smem > 48 * 1024) {
    static bool attr_set = false;
    if (!attr_set) {
      LN_CUDA(cudaFuncSetAttribute(k_eig_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr_set = true;
    }
  }
  count_launch();
  k_eig_sort<<<1, 1024, smem, s>>>(A, n, desc ? 1 : 0, w, order);
  if (sweeps_out) *sweeps_out = sweep;
  LN_CUDA(cudaGetLastError());
  return LNOCC_OK;
}

void gather_cols(const double* V, int n, const int* order, int ncols, double* out, int ldo, cudaStream_t s) {
  if (ncols < 1) return;
  count_launch();
  k_gather_cols<<<grid_of(1LL * n * ncols, 256), 256, 0, s>>>(V, n, order, ncols, out, ldo);
}

}  // namespace lnocc
