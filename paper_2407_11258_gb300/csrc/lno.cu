// Local active space of a fragment (Sec. II.C and II.E), on the device:
//   lnocc_lno_internal   -- Eq. 18-19: internal orbitals of one block from the SVD of U^(F), semi-canonical
//   lnocc_lno_densities  -- Eq. 20 (LNO) or Eq. 28 (CBNO): MP2 density blocks from the MP1 amplitudes of
//                           Eq. 21 with the DF integrals of Eq. 22 (Gamma point, real orbitals)
//   lnocc_lno_select     -- Eq. 24-26: the density projected onto the external space, diagonalised, LNOs with
//                           |lambda| >= eta
//   lnocc_active_space   -- the semi-canonical active space and its DF factors (Eq. 27 at the Gamma point):
//                           the input of lnocc_build_ints
//
// Densities (amplitudes T = t^(1) with T[iF][a][j][b] = t_{iF a j b}, t_{i a kF b} = T[kF][b][i][a]):
//   LNO  D_vir = sum_iF 2 A A^T + 2 B B^T - A B^T - B A^T,  A[a][(j,c)] = T[iF][a][j][c], B[a][(j,c)] = T[iF][c][j][a]
//        D_occ = sum_kF 4 C C^T - C C'^T - C' C^T,          C[i][(b,a)] = T[kF][b][i][a], C'[i][(b,a)] = T[kF][a][i][b]
//   CBNO D_occ = 4 C C^T - C C'^T - C' C^T with C[i][(aF,k,bF)] = t_{i aF k bF}, C'[i][(aF,k,bF)] = t_{i bF k aF}
//        D_vir = 4 A A^T - A A'^T - A' A^T with A[a][(iF,jF,c)] = t_{iF a jF c}, A'[a][(iF,jF,c)] = t_{iF c jF a}
// The products are tensor-core (or FP64) contractions of packed strided views of T (the contraction engine
// packs any strided view); the cross terms are formed once (alpha = -2) and the result symmetrised, which
// equals the symmetric sum above because A A^T and B B^T are symmetric.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace lnocc {

int sym_eig(double* A, double* V, double* w, int* order, int n, bool desc, double* scratch, cudaStream_t s,
            int* sweeps_out);
void gather_cols(const double* V, int n, const int* order, int ncols, double* out, int ldo, cudaStream_t s);

namespace {

int grid1(long long work, int threads = 256) {
  return static_cast<int>(std::max(1LL, std::min<long long>((work + threads - 1) / threads, 152LL * 32)));
}
#define GSTRIDE(i, total)                                                                          \
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < (total); \
       i += static_cast<long long>(gridDim.x) * blockDim.x)

// Device allocations of one call, freed when the call returns.
struct Arena {
  std::vector<void*> ptrs;
  bool failed = false;
  void* get(size_t bytes) {
    void* p = nullptr;
    count_alloc();
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    return p;
  }
  template <typename T>
  T* get_n(long long n) { return static_cast<T*>(get(static_cast<size_t>(std::max(n, 1LL)) * sizeof(T))); }
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// C = alpha A B^T + beta C for strided views (packed into two scratch operands of the call's precision)
struct Engine {
  Arena& ar;
  bool bf;
  cudaStream_t s;
  int* dstatus;
  Packed PA, PB;
  size_t capA = 0, capB = 0;
  bool grow(Packed& P, size_t& cap, size_t need) {
    if (need <= cap) return true;
    P.p = ar.get(need);
    cap = P.p ? need : 0;
    return P.p != nullptr;
  }
  bool run(const View& a, const View& b, const OutMap& c) {
    PA.bf16 = PB.bf16 = bf;
    const size_t esz = bf ? 4 : 8;
    const size_t na = static_cast<size_t>(a.rows()) * round_up(std::max(a.K(), 1), 64) * esz;
    const size_t nb = static_cast<size_t>(b.rows()) * round_up(std::max(b.K(), 1), 64) * esz;
    if (!grow(PA, capA, na) || !grow(PB, capB, nb)) return false;
    pack(a, PA, s);
    pack(b, PB, s);
    gemm(PA, PB, a.rows(), b.rows(), a.K(), c, s, dstatus);
    return true;
  }
  // C = alpha A A^T + beta C (one packed operand)
  bool run_sym(const View& a, const OutMap& c) {
    PA.bf16 = bf;
    const size_t na = static_cast<size_t>(a.rows()) * round_up(std::max(a.K(), 1), 64) * (bf ? 4 : 8);
    if (!grow(PA, capA, na)) return false;
    pack(a, PA, s);
    gemm(PA, PA, a.rows(), a.rows(), a.K(), c, s, dstatus);
    return true;
  }
};

inline Ax A_(int n, long long s) { return Ax{n, s}; }

// G[k][l] = sum_i U[i][k] U[i][l]   (one block per (k, l))
__global__ void k_gram(const double* __restrict__ U, int n, int nlo, double* __restrict__ G) {
  __shared__ double red[8];
  const int k = blockIdx.x / nlo, l = blockIdx.x % nlo;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += U[static_cast<long long>(i) * nlo + k] * U[static_cast<long long>(i) * nlo + l];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) t += red[w];
    G[blockIdx.x] = t;
  }
}

// W[i][k] = sum_l U[i][l] Vg[l][order[k]] / sigma_k   for k < nint   (sigma_k = sqrt(w[k]))
__global__ void k_left_vectors(const double* __restrict__ U, int n, int nlo, const double* __restrict__ Vg,
                               const int* __restrict__ order, const double* __restrict__ w, int nint,
                               double* __restrict__ W) {
  GSTRIDE(x, 1LL * n * nint) {
    const int i = static_cast<int>(x / nint), k = static_cast<int>(x % nint);
    double acc = 0.0;
    for (int l = 0; l < nlo; ++l) acc += U[static_cast<long long>(i) * nlo + l] * Vg[static_cast<long long>(l) * nlo + order[k]];
    W[x] = acc / sqrt(w[k]);
  }
}

// F[k][l] = sum_i W[i][k] e[i] W[i][l]   (one block per (k, l)); W is [n][m]
__global__ void k_fock_block(const double* __restrict__ W, int n, int m, const double* __restrict__ e,
                             double* __restrict__ F) {
  __shared__ double red[8];
  const int k = blockIdx.x / m, l = blockIdx.x % m;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    acc += W[static_cast<long long>(i) * m + k] * e[i] * W[static_cast<long long>(i) * m + l];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w2 = 0; w2 < static_cast<int>(blockDim.x / 32); ++w2) t += red[w2];
    F[blockIdx.x] = t;
  }
}

// out[i][k] (leading dimension ldo) = sum_l W[i][l] R[l][order[k]], k < m   (W [n][m], R [m][m])
__global__ void k_rotate_cols(const double* __restrict__ W, int n, int m, const double* __restrict__ R,
                              const int* __restrict__ order, double* __restrict__ out, int ldo) {
  GSTRIDE(x, 1LL * n * m) {
    const int i = static_cast<int>(x / m), k = static_cast<int>(x % m);
    double acc = 0.0;
    for (int l = 0; l < m; ++l) acc += W[static_cast<long long>(i) * m + l] * R[static_cast<long long>(l) * m + order[k]];
    out[static_cast<long long>(i) * ldo + k] = acc;
  }
}

__global__ void k_zero(double* p, long long n) {
  GSTRIDE(x, n) p[x] = 0.0;
}

// Bt[Q][a] = sum_i W[i][col] B_ov[Q][i][a]   (W leading dimension ldw)
__global__ void k_occ_transform(const double* __restrict__ Bov, int N, int o, int v, const double* __restrict__ W,
                                int ldw, int col, double* __restrict__ Bt) {
  GSTRIDE(x, 1LL * N * v) {
    const long long Q = x / v;
    const int a = static_cast<int>(x % v);
    const double* b = Bov + Q * o * v + a;
    double acc = 0.0;
    for (int i = 0; i < o; ++i) acc += W[static_cast<long long>(i) * ldw + col] * b[static_cast<long long>(i) * v];
    Bt[x] = acc;
  }
}

// L[Q][i][k] = sum_a B_ov[Q][i][a] Wv[a][k]   (k < nk; Wv leading dimension ldw)
__global__ void k_vir_transform(const double* __restrict__ Bov, long long NO, int v, const double* __restrict__ Wv,
                                int ldw, int nk, double* __restrict__ L) {
  GSTRIDE(x, NO * nk) {
    const long long r = x / nk;
    const int k = static_cast<int>(x % nk);
    const double* b = Bov + r * v;
    double acc = 0.0;
    for (int a = 0; a < v; ++a) acc += b[a] * Wv[static_cast<long long>(a) * ldw + k];
    L[x] = acc;
  }
}

// T[a][j][b] = X[a][j][b] / (fi + e_j - e_a - e_b)   (LNO amplitudes of one internal occupied orbital)
__global__ void k_mp1_one(double* __restrict__ X, int o, int v, const double* __restrict__ eps, double fi) {
  const long long ov = 1LL * o * v;
  GSTRIDE(x, 1LL * v * ov) {
    const int a = static_cast<int>(x / ov);
    const int j = static_cast<int>((x % ov) / v), b = static_cast<int>(x % v);
    X[x] /= fi + eps[j] - eps[o + a] - eps[o + b];
  }
}

// t[p][x][q][y] /= (d1[p] + d1[q] - d2[x] - d2[y]) for a [n1][n2][n1][n2] array (CBNO amplitudes)
__global__ void k_mp1_pairs(double* __restrict__ X, int n1, int n2, const double* __restrict__ d1,
                            const double* __restrict__ d2) {
  const long long m = 1LL * n1 * n2;
  GSTRIDE(x, m * m) {
    const long long r = x / m, c = x % m;
    const int p = static_cast<int>(r / n2), xx = static_cast<int>(r % n2);
    const int q = static_cast<int>(c / n2), y = static_cast<int>(c % n2);
    X[x] /= d1[p] + d1[q] - d2[xx] - d2[y];
  }
}

// D <- (D + D^T) / 2
__global__ void k_symmetrize(double* D, int n) {
  GSTRIDE(x, 1LL * n * n) {
    const int i = static_cast<int>(x / n), j = static_cast<int>(x % n);
    if (i < j) {
      const double s = 0.5 * (D[x] + D[static_cast<long long>(j) * n + i]);
      D[x] = s;
      D[static_cast<long long>(j) * n + i] = s;
    }
  }
}

// Y[i][k] = sum_j D[i][j] W[j][k]  (D [n][n], W [n][m]); one thread per output
__global__ void k_mul_nm(const double* __restrict__ D, const double* __restrict__ W, int n, int m, double* __restrict__ Y) {
  GSTRIDE(x, 1LL * n * m) {
    const int i = static_cast<int>(x / m), k = static_cast<int>(x % m);
    const double* d = D + static_cast<long long>(i) * n;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += d[j] * W[static_cast<long long>(j) * m + k];
    Y[x] = acc;
  }
}

// Z[j][k] = sum_l X[l][j] W[l][k]  (X [n][n], W [n][m]): X^T W
__global__ void k_mul_tn(const double* __restrict__ X, const double* __restrict__ W, int n, int m, double* __restrict__ Z) {
  GSTRIDE(x, 1LL * n * m) {
    const int j = static_cast<int>(x / m), k = static_cast<int>(x % m);
    double acc = 0.0;
    for (int l = 0; l < n; ++l) acc += X[static_cast<long long>(l) * n + j] * W[static_cast<long long>(l) * m + k];
    Z[x] = acc;
  }
}

// out[i][j] = X[i][j] - sum_k Y[i][k] W[j][k]  (X, out [n][n]; Y, W [n][m]); out may alias X
__global__ void k_sub_outer(const double* X, const double* __restrict__ Y, const double* __restrict__ W, int n, int m,
                            double* out) {
  GSTRIDE(x, 1LL * n * n) {
    const int i = static_cast<int>(x / n), j = static_cast<int>(x % n);
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc += Y[static_cast<long long>(i) * m + k] * W[static_cast<long long>(j) * m + k];
    out[x] = X[x] - acc;
  }
}

// keep |w[k]| >= eta in the sorted order: korder[c] = order[k], lam[c] = w[k]; count to *cnt (one thread)
__global__ void k_select(const double* __restrict__ w, const int* __restrict__ order, int n, double eta,
                         int* __restrict__ korder, double* __restrict__ lam, int* __restrict__ cnt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int c = 0;
  for (int k = 0; k < n; ++k) {
    if (fabs(w[k]) >= eta) {
      korder[c] = order[k];
      lam[c] = w[k];
      ++c;
    }
  }
  for (int k = c; k < n; ++k) lam[k] = 0.0;
  *cnt = c;
}

// out[i][k] = V[i][korder[k]] for k < *cnt, 0 for the remaining columns (out [n][n])
__global__ void k_gather_kept(const double* __restrict__ V, int n, const int* __restrict__ korder,
                              const int* __restrict__ cnt, double* __restrict__ out) {
  const int c = *cnt;
  GSTRIDE(x, 1LL * n * n) {
    const int i = static_cast<int>(x / n), k = static_cast<int>(x % n);
    out[x] = k < c ? V[static_cast<long long>(i) * n + korder[k]] : 0.0;
  }
}

// C_F (n x nF) block diagonal from Co [o][no] and Cv [v][nv]
__global__ void k_block_diag(const double* __restrict__ Co, int o, int no, const double* __restrict__ Cv, int v,
                             int nv, double* __restrict__ CF) {
  const int n = o + v, nF = no + nv;
  GSTRIDE(x, 1LL * n * nF) {
    const int p = static_cast<int>(x / nF), t = static_cast<int>(x % nF);
    double val = 0.0;
    if (p < o && t < no) val = Co[static_cast<long long>(p) * no + t];
    if (p >= o && t >= no) val = Cv[static_cast<long long>(p - o) * nv + (t - no)];
    CF[x] = val;
  }
}

int finish(cudaStream_t s, int* dstatus, const char* who) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, dstatus, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(who) + ": " + cudaGetErrorString(e));
    return LNOCC_ECUDA;
  }
  if (st != 0) {
    set_error(std::string(who) + ": device wait timed out");
    return LNOCC_ETIMEOUT;
  }
  return LNOCC_OK;
}

struct SplitScope {  // split-K partials for long-K / small-output contractions, for the call's duration
  SplitWs saved;
  SplitScope(Arena& ar) : saved(split_ws()) {
    double* ws = ar.get_n<double>(1LL << 22);
    split_ws() = ws ? SplitWs{ws, size_t(1) << 22} : SplitWs{};
  }
  ~SplitScope() { split_ws() = saved; }
};

// Semi-canonical internal space of one block; W_out [n][ldo] (first nint columns), f_out [nint] ascending.
int internal_block(int n, int nlo, const double* U, const double* e, double sv_tol, double* W_out, int ldo,
                   double* f_out, int* nint_out, Arena& ar, cudaStream_t s) {
  double* G = ar.get_n<double>(1LL * nlo * nlo);
  double* Vg = ar.get_n<double>(1LL * nlo * nlo);
  double* w = ar.get_n<double>(nlo);
  int* ord = ar.get_n<int>(nlo);
  double* scr = ar.get_n<double>(16 + 2LL * nlo + 8);
  if (ar.failed) {
    set_error("lnocc_lno_internal: device allocation failed");
    return LNOCC_ENOMEM;
  }
  count_launch();
  k_gram<<<nlo * nlo, 256, 0, s>>>(U, n, nlo, G);
  int st = sym_eig(G, Vg, w, ord, nlo, true, scr, s, nullptr);
  if (st) return st;
  std::vector<double> hw(nlo);
  LN_CUDA(cudaMemcpyAsync(hw.data(), w, nlo * sizeof(double), cudaMemcpyDeviceToHost, s));
  LN_CUDA(cudaStreamSynchronize(s));
  // singular values sigma_k = sqrt(w_k); zero below sv_tol relative to the largest
  const double smax = std::sqrt(std::max(hw[0], 0.0));
  int nint = 0;
  for (int k = 0; k < nlo; ++k)
    if (hw[k] > 0.0 && std::sqrt(hw[k]) > sv_tol * smax) ++nint;
  *nint_out = nint;
  count_launch();
  k_zero<<<grid1(1LL * n * ldo), 256, 0, s>>>(W_out, 1LL * n * ldo);
  if (nint == 0) return LNOCC_OK;
  double* W = ar.get_n<double>(1LL * n * nint);
  double* F = ar.get_n<double>(1LL * nint * nint);
  double* R = ar.get_n<double>(1LL * nint * nint);
  int* ord2 = ar.get_n<int>(nint);
  if (ar.failed) {
    set_error("lnocc_lno_internal: device allocation failed");
    return LNOCC_ENOMEM;
  }
  count_launch(2);
  k_left_vectors<<<grid1(1LL * n * nint), 256, 0, s>>>(U, n, nlo, Vg, ord, w, nint, W);
  k_fock_block<<<nint * nint, 256, 0, s>>>(W, n, nint, e, F);
  st = sym_eig(F, R, f_out, ord2, nint, false, scr, s, nullptr);
  if (st) return st;
  count_launch();
  k_rotate_cols<<<grid1(1LL * n * nint), 256, 0, s>>>(W, n, nint, R, ord2, W_out, ldo);
  return LNOCC_OK;
}

}  // namespace
}  // namespace lnocc

using namespace lnocc;

extern "C" int lnocc_lno_internal(int n, int nlo, const double* U, const double* e, double sv_tol, double* W_int,
                                  double* f_int, int* n_int, void* stream) {
  set_error("");
  if (n < 1 || nlo < 1 || nlo > 256 || !U || !e || !W_int || !f_int || !n_int || !(sv_tol > 0.0) || sv_tol >= 1.0) {
    set_error("lnocc_lno_internal: bad arguments (1 <= nlo <= 256, 0 < sv_tol < 1)");
    return LNOCC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar;
  int st = internal_block(n, nlo, U, e, sv_tol, W_int, nlo, f_int, n_int, ar, s);
  if (st) return st;
  LN_CUDA(cudaStreamSynchronize(s));
  LN_CUDA(cudaGetLastError());
  return LNOCC_OK;
}

extern "C" int lnocc_lno_densities(int precision, int kind, int nocc, int nvir, int naux, const double* eps,
                                   const double* B_ov, int n_io, const double* W_occ, const double* f_occ, int n_iv,
                                   const double* W_vir, const double* f_vir, double* D_occ, double* D_vir,
                                   void* stream) {
  set_error("");
  const bool bad_common = nocc < 1 || nvir < 1 || naux < 1 || !eps || !B_ov || !D_occ || !D_vir ||
                          (precision != LNOCC_PREC_FP64 && precision != LNOCC_PREC_MIXED) || n_io < 1 || !W_occ ||
                          !f_occ || n_io > nocc || n_iv < 0 || n_iv > nvir || (n_iv > 0 && (!W_vir || !f_vir));
  if (bad_common || (kind != LNOCC_LNO_MP2 && kind != LNOCC_LNO_CBNO) ||
      1LL * nvir * nvir > (1LL << 31) - 64 || 1LL * nocc * nvir > (1LL << 30)) {
    set_error("lnocc_lno_densities: bad arguments");
    return LNOCC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool bf = precision == LNOCC_PREC_MIXED;
  const int o = nocc, v = nvir, N = naux;
  const long long ov = 1LL * o * v, vv = 1LL * v * v;
  Arena ar;
  int* dstatus = ar.get_n<int>(4);
  if (!dstatus) {
    set_error("lnocc_lno_densities: device allocation failed");
    return LNOCC_ENOMEM;
  }
  LN_CUDA(cudaMemsetAsync(dstatus, 0, 16, s));
  SplitScope split(ar);
  Engine eng{ar, bf, s, dstatus};
  count_launch(2);
  k_zero<<<grid1(1LL * o * o), 256, 0, s>>>(D_occ, 1LL * o * o);
  k_zero<<<grid1(vv), 256, 0, s>>>(D_vir, vv);
  bool ok = true;
  if (kind == LNOCC_LNO_MP2) {
    // B_ov packed once as rows (j, b), K = Q
    Packed PBov;
    PBov.bf16 = bf;
    PBov.p = ar.get(static_cast<size_t>(ov) * round_up(N, 64) * (bf ? 4 : 8));
    double* Bt = ar.get_n<double>(1LL * N * v);
    double* X = ar.get_n<double>(vv * o);
    std::vector<double> hf(n_io);
    if (ar.failed) {
      set_error("lnocc_lno_densities: device allocation failed");
      return LNOCC_ENOMEM;
    }
    LN_CUDA(cudaMemcpyAsync(hf.data(), f_occ, n_io * sizeof(double), cudaMemcpyDeviceToHost, s));
    LN_CUDA(cudaStreamSynchronize(s));
    pack(view(B_ov, kOne, A_(o, v), A_(v, 1), kOne, kOne, A_(N, ov)), PBov, s);
    for (int k = 0; k < n_io && ok; ++k) {
      count_launch();
      k_occ_transform<<<grid1(1LL * N * v), 256, 0, s>>>(B_ov, N, o, v, W_occ, n_io, k, Bt);
      // X[a][(j,b)] = sum_Q Bt[Q][a] B_ov[Q][j][b]
      {
        Packed& PA = eng.PA;
        PA.bf16 = bf;
        if (!eng.grow(PA, eng.capA, static_cast<size_t>(v) * round_up(N, 64) * (bf ? 4 : 8))) { ok = false; break; }
        pack(view(Bt, kOne, kOne, A_(v, 1), kOne, kOne, A_(N, v)), PA, s);
        gemm(PA, PBov, v, static_cast<int>(ov), N, out_rowmajor(X, ov), s, dstatus);
      }
      count_launch();
      k_mp1_one<<<grid1(vv * o), 256, 0, s>>>(X, o, v, eps, hf[k]);
      // virtual block: A[a][(j,c)] = T[a][j][c], B[a][(j,c)] = T[c][j][a]
      const View Av = view(X, kOne, kOne, A_(v, ov), kOne, A_(o, v), A_(v, 1));
      const View Bv = view(X, kOne, kOne, A_(v, 1), kOne, A_(o, v), A_(v, ov));
      ok = ok && eng.run_sym(Av, out_rowmajor(D_vir, v, 2.0, 1.0));
      ok = ok && eng.run_sym(Bv, out_rowmajor(D_vir, v, 2.0, 1.0));
      ok = ok && eng.run(Av, Bv, out_rowmajor(D_vir, v, -2.0, 1.0));
      // occupied block: C[i][(b,a)] = T[b][i][a], C'[i][(b,a)] = T[a][i][b]
      const View Cv = view(X, kOne, kOne, A_(o, v), kOne, A_(v, ov), A_(v, 1));
      const View Cpv = view(X, kOne, kOne, A_(o, v), kOne, A_(v, 1), A_(v, ov));
      ok = ok && eng.run_sym(Cv, out_rowmajor(D_occ, o, 4.0, 1.0));
      ok = ok && eng.run(Cv, Cpv, out_rowmajor(D_occ, o, -2.0, 1.0));
    }
  } else {
    // virtual block: both occupied internal. L'[Q][iF][a], then t[iF][a][jF][c]
    {
      const long long m = 1LL * n_io * v;
      double* Lp = ar.get_n<double>(1LL * N * m);
      double* Vo = ar.get_n<double>(m * m);
      double* Bt = ar.get_n<double>(1LL * N * v);
      if (ar.failed) {
        set_error("lnocc_lno_densities: device allocation failed");
        return LNOCC_ENOMEM;
      }
      for (int k = 0; k < n_io; ++k) {
        // Lp[Q][k][a] = sum_i Wo[i][k] B[Q][i][a] (one internal orbital at a time, then into place)
        count_launch();
        k_occ_transform<<<grid1(1LL * N * v), 256, 0, s>>>(B_ov, N, o, v, W_occ, n_io, k, Bt);
        LN_CUDA(cudaMemcpy2DAsync(Lp + 1LL * k * v, m * 8, Bt, v * 8, v * 8, N, cudaMemcpyDeviceToDevice, s));
      }
      const View Lv = view(Lp, kOne, kOne, A_(static_cast<int>(m), 1), kOne, kOne, A_(N, m));
      ok = ok && eng.run(Lv, Lv, out_rowmajor(Vo, m));
      count_launch();
      k_mp1_pairs<<<grid1(m * m), 256, 0, s>>>(Vo, n_io, v, f_occ, eps + o);
      // A[a][(iF,jF,c)] = t[iF][a][jF][c]; A'[a][(iF,jF,c)] = t[iF][c][jF][a]
      const View Aw = view(Vo, kOne, kOne, A_(v, m), A_(n_io, v * m), A_(n_io, v), A_(v, 1));
      const View Apw = view(Vo, kOne, kOne, A_(v, 1), A_(n_io, v * m), A_(n_io, v), A_(v, m));
      ok = ok && eng.run_sym(Aw, out_rowmajor(D_vir, v, 4.0, 1.0));
      ok = ok && eng.run(Aw, Apw, out_rowmajor(D_vir, v, -2.0, 1.0));
    }
    // occupied block: both virtuals internal. L[Q][i][aF], then t[i][aF][k][bF]
    if (n_iv > 0 && ok) {
      const long long m = 1LL * o * n_iv;
      double* L = ar.get_n<double>(1LL * N * m);
      double* Vv = ar.get_n<double>(m * m);
      if (ar.failed) {
        set_error("lnocc_lno_densities: device allocation failed");
        return LNOCC_ENOMEM;
      }
      count_launch();
      k_vir_transform<<<grid1(1LL * N * o * n_iv), 256, 0, s>>>(B_ov, 1LL * N * o, v, W_vir, n_iv, n_iv, L);
      const View Lv = view(L, kOne, kOne, A_(static_cast<int>(m), 1), kOne, kOne, A_(N, m));
      ok = ok && eng.run(Lv, Lv, out_rowmajor(Vv, m));
      count_launch();
      k_mp1_pairs<<<grid1(m * m), 256, 0, s>>>(Vv, o, n_iv, eps, f_vir);
      // C[i][(aF,k,bF)] = t[i][aF][k][bF]; C'[i][(aF,k,bF)] = t[i][bF][k][aF]
      const View Cw = view(Vv, kOne, kOne, A_(o, n_iv * m), A_(n_iv, m), A_(o, n_iv), A_(n_iv, 1));
      const View Cpw = view(Vv, kOne, kOne, A_(o, n_iv * m), A_(n_iv, 1), A_(o, n_iv), A_(n_iv, m));
      ok = ok && eng.run_sym(Cw, out_rowmajor(D_occ, o, 4.0, 1.0));
      ok = ok && eng.run(Cw, Cpw, out_rowmajor(D_occ, o, -2.0, 1.0));
    }
  }
  if (!ok) {
    set_error("lnocc_lno_densities: device allocation failed");
    cudaStreamSynchronize(s);
    return LNOCC_ENOMEM;
  }
  count_launch(2);
  k_symmetrize<<<grid1(1LL * o * o), 256, 0, s>>>(D_occ, o);
  k_symmetrize<<<grid1(vv), 256, 0, s>>>(D_vir, v);
  return finish(s, dstatus, "lnocc_lno_densities");
}

extern "C" int lnocc_lno_select(int n, const double* D, int n_int, const double* W_int, double eta, double* C,
                                double* lambda, int* n_keep, void* stream) {
  set_error("");
  if (n < 1 || n > 8192 || !D || !C || !lambda || !n_keep || n_int < 0 || n_int > n || (n_int > 0 && !W_int) ||
      !(eta >= 0.0)) {
    set_error("lnocc_lno_select: bad arguments (1 <= n <= 8192, 0 <= n_int <= n, eta >= 0)");
    return LNOCC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar;
  const long long nn = 1LL * n * n;
  double* A = ar.get_n<double>(nn);
  double* V = ar.get_n<double>(nn);
  double* w = ar.get_n<double>(n);
  int* ord = ar.get_n<int>(n);
  int* kord = ar.get_n<int>(n);
  int* cnt = ar.get_n<int>(1);
  double* scr = ar.get_n<double>(16 + 2LL * n + 8);
  double* Y = n_int > 0 ? ar.get_n<double>(1LL * n * n_int) : nullptr;
  if (ar.failed) {
    set_error("lnocc_lno_select: device allocation failed");
    return LNOCC_ENOMEM;
  }
  LN_CUDA(cudaMemcpyAsync(A, D, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (n_int > 0) {
    // external projection A = P D P with P = 1 - W W^T (Eq. 24 with W_bar W_bar^T = P):
    //   A1 = D P = D - (D W) W^T,   A = P A1 = A1 - W (A1^T W)^T
    count_launch(4);
    k_mul_nm<<<grid1(1LL * n * n_int), 256, 0, s>>>(A, W_int, n, n_int, Y);
    k_sub_outer<<<grid1(nn), 256, 0, s>>>(A, Y, W_int, n, n_int, A);
    k_mul_tn<<<grid1(1LL * n * n_int), 256, 0, s>>>(A, W_int, n, n_int, Y);
    k_sub_outer<<<grid1(nn), 256, 0, s>>>(A, W_int, Y, n, n_int, A);
  }
  count_launch();
  k_symmetrize<<<grid1(nn), 256, 0, s>>>(A, n);
  int st = sym_eig(A, V, w, ord, n, true, scr, s, nullptr);
  if (st) return st;
  count_launch(2);
  k_select<<<1, 32, 0, s>>>(w, ord, n, eta, kord, lambda, cnt);
  k_gather_kept<<<grid1(nn), 256, 0, s>>>(V, n, kord, cnt, C);
  int hc = 0;
  LN_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  LN_CUDA(cudaStreamSynchronize(s));
  LN_CUDA(cudaGetLastError());
  *n_keep = hc;
  return LNOCC_OK;
}

extern "C" int lnocc_active_space(int precision, int nocc, int nvir, int naux, const double* eps, const double* B,
                                  int no_F, const double* C_occ, int nv_F, const double* C_vir, double* eps_F,
                                  double* B_F, double* C_F, void* stream) {
  set_error("");
  if (nocc < 1 || nvir < 1 || naux < 1 || !eps || !B || no_F < 1 || no_F > nocc || nv_F < 1 || nv_F > nvir || !C_occ ||
      !C_vir || !eps_F || !B_F || (precision != LNOCC_PREC_FP64 && precision != LNOCC_PREC_MIXED) ||
      1LL * naux * (nocc + nvir) > (1LL << 31) - 1) {
    set_error("lnocc_active_space: bad arguments");
    return LNOCC_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int o = nocc, v = nvir, n = o + v, nF = no_F + nv_F, N = naux;
  Arena ar;
  int* dstatus = ar.get_n<int>(4);
  double* Fo = ar.get_n<double>(1LL * no_F * no_F);
  double* Ro = ar.get_n<double>(1LL * no_F * no_F);
  double* Fv = ar.get_n<double>(1LL * nv_F * nv_F);
  double* Rv = ar.get_n<double>(1LL * nv_F * nv_F);
  int* oo_ = ar.get_n<int>(no_F);
  int* ov_ = ar.get_n<int>(nv_F);
  double* Co = ar.get_n<double>(1LL * o * no_F);
  double* Cv = ar.get_n<double>(1LL * v * nv_F);
  double* CF = ar.get_n<double>(1LL * n * nF);
  const int nq_h = static_cast<int>(std::max(1LL, std::min<long long>(N, (1LL << 27) / std::max(1LL * n * round_up(n, 64), 1LL))));
  double* H = ar.get_n<double>(1LL * nq_h * n * nF);
  double* scr = ar.get_n<double>(16 + 2LL * std::max(no_F, nv_F) + 8);
  if (ar.failed) {
    set_error("lnocc_active_space: device allocation failed");
    return LNOCC_ENOMEM;
  }
  LN_CUDA(cudaMemsetAsync(dstatus, 0, 16, s));
  // semi-canonical active blocks: diagonalise C^T diag(e) C inside each block (energies increasing)
  count_launch(2);
  k_fock_block<<<no_F * no_F, 256, 0, s>>>(C_occ, o, no_F, eps, Fo);
  k_fock_block<<<nv_F * nv_F, 256, 0, s>>>(C_vir, v, nv_F, eps + o, Fv);
  int st = sym_eig(Fo, Ro, eps_F, oo_, no_F, false, scr, s, nullptr);
  if (st) return st;
  st = sym_eig(Fv, Rv, eps_F + no_F, ov_, nv_F, false, scr, s, nullptr);
  if (st) return st;
  count_launch(3);
  k_rotate_cols<<<grid1(1LL * o * no_F), 256, 0, s>>>(C_occ, o, no_F, Ro, oo_, Co, no_F);
  k_rotate_cols<<<grid1(1LL * v * nv_F), 256, 0, s>>>(C_vir, v, nv_F, Rv, ov_, Cv, nv_F);
  k_block_diag<<<grid1(1LL * n * nF), 256, 0, s>>>(Co, o, no_F, Cv, v, nv_F, CF);
  SplitScope split(ar);
  Engine eng{ar, precision == LNOCC_PREC_MIXED, s, dstatus};
  // per block of auxiliary indices Q (bounded packed operands):
  // H[Q][p][t] = sum_q B[Q][p][q] C_F[q][t]: rows (Q, p), K q; columns t (rows of C_F^T)
  // B_F[Q][s][t] = sum_p C_F[p][s] H[Q][p][t]: rows s, K p; columns (Q, t), K p
  const View CFt = view(CF, kOne, kOne, A_(nF, 1), kOne, kOne, A_(n, nF));
  const long long per_q = 1LL * n * round_up(n, 64);
  const int nq = static_cast<int>(std::max(1LL, std::min<long long>(N, (1LL << 27) / std::max(per_q, 1LL))));
  bool ok = true;
  for (int q0 = 0; q0 < N && ok; q0 += nq) {
    const int bq = std::min(nq, N - q0);
    const View Bv = view(B + 1LL * q0 * n * n, kOne, kOne, A_(bq * n, n), kOne, kOne, A_(n, 1));
    ok = eng.run(Bv, CFt, out_rowmajor(H, nF));
    const View Hv = view(H, kOne, A_(bq, 1LL * n * nF), A_(nF, 1), kOne, kOne, A_(n, nF));
    OutMap om{B_F + 1LL * q0 * nF * nF, 0, nF, 1LL * nF * nF, 1, 1 << 30, nF, 1.0, 0.0};
    ok = ok && eng.run(CFt, Hv, om);
  }
  if (ok && C_F) LN_CUDA(cudaMemcpyAsync(C_F, CF, 1LL * n * nF * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (!ok) {
    set_error("lnocc_active_space: device allocation failed");
    cudaStreamSynchronize(s);
    return LNOCC_ENOMEM;
  }
  return finish(s, dstatus, "lnocc_active_space");
}
