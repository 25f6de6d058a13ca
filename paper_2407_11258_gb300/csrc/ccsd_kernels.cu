// FP64 element-wise and reduction kernels of the CCSD iteration: tau / u builders, the packed
// +/- operands and the unpacking of the particle-particle ladder, residual assembly with the
// amplitude update (t += R / D, D from the orbital energies), deterministic energy and
// dot-product reductions (warp shuffles, fixed-order second pass) and the DIIS solve.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ccsd_kernels.h"
#include "ptx.cuh"

namespace lnocc {

namespace {
constexpr int kThreads = 256;
inline int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return static_cast<int>(b < 152LL * 32 ? (b > 0 ? b : 1) : 152LL * 32);
}
#define GRID_STRIDE(idx, total)                                                                          \
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < (total); \
       idx += static_cast<long long>(gridDim.x) * blockDim.x)

__device__ __forceinline__ int tri_le(int i, int j) { return j * (j + 1) / 2 + i; }  // i <= j
__device__ __forceinline__ int tri_lt(int i, int j) { return j * (j - 1) / 2 + i; }  // i <  j

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block sum (fixed order within the block); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double x) {
  __shared__ double sh[32];
  x = warp_sum(x);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) sh[w] = x;
  __syncthreads();
  double y = 0.0;
  if (w == 0) {
    y = (l < static_cast<int>(blockDim.x / 32)) ? sh[l] : 0.0;
    y = warp_sum(y);
  }
  __syncthreads();
  return y;
}

__device__ __forceinline__ void block_sum_store(double x, double* out) {
  const double y = block_sum(x);
  if (threadIdx.x == 0) out[blockIdx.x] = y;
}
}  // namespace

// ---------------------------------------------------------------------------------------------
__global__ void k_tau(const double* t1, const double* t2, double* tau, int o, int v) {
  const long long total = static_cast<long long>(o) * o * v * v;
  GRID_STRIDE(idx, total) {
    const int b = idx % v, a = (idx / v) % v, j = (idx / (v * v)) % o, i = idx / (static_cast<long long>(v) * v * o);
    tau[idx] = (t2 ? t2[idx] : 0.0) + t1[i * v + a] * t1[j * v + b];
  }
}

__global__ void k_u(const double* t2, double* u, int o, int v) {
  const long long total = static_cast<long long>(o) * o * v * v;
  const long long vv = static_cast<long long>(v) * v;
  GRID_STRIDE(idx, total) {
    const long long ab = idx % vv;
    const int j = (idx / vv) % o, i = idx / (vv * o);
    u[idx] = 2.0 * t2[idx] - t2[(static_cast<long long>(j) * o + i) * vv + ab];
  }
}

// B+[ij][cd] = w_cd (t_ij^cd + t_ij^dc) / 2 for i<=j, c<=d (w = 1/2 on c = d);
// B-[ij][cd] = (t_ij^cd - t_ij^dc) / 2 for i<j, c<d.
template <bool BF16>
__global__ void k_ladder_ops(const double* t2, void* Bp, void* Bm, int o, int v, int Kpp, int Kpm, long long plane_p,
                             long long plane_m) {
  const long long vv = static_cast<long long>(v) * v;
  const long long total = static_cast<long long>(o) * o * vv;
  GRID_STRIDE(idx, total) {
    const int d = idx % v, c = (idx / v) % v, j = (idx / vv) % o, i = idx / (vv * o);
    if (i > j || c > d) continue;
    const double x = t2[idx];
    const double y = t2[(static_cast<long long>(i) * o + j) * vv + static_cast<long long>(d) * v + c];
    const double sp = (c == d ? 0.25 : 0.5) * (x + y);
    const long long pp = static_cast<long long>(tri_le(i, j)) * Kpp + tri_le(c, d);
    if (BF16) {
      __nv_bfloat16 hi, lo;
      split_bf16(sp, hi, lo);
      static_cast<__nv_bfloat16*>(Bp)[pp] = hi;
      static_cast<__nv_bfloat16*>(Bp)[pp + plane_p] = lo;
    } else {
      static_cast<double*>(Bp)[pp] = sp;
    }
    if (i < j && c < d) {
      const double sm = 0.5 * (x - y);
      const long long pm = static_cast<long long>(tri_lt(i, j)) * Kpm + tri_lt(c, d);
      if (BF16) {
        __nv_bfloat16 hi, lo;
        split_bf16(sm, hi, lo);
        static_cast<__nv_bfloat16*>(Bm)[pm] = hi;
        static_cast<__nv_bfloat16*>(Bm)[pm + plane_m] = lo;
      } else {
        static_cast<double*>(Bm)[pm] = sm;
      }
    }
  }
}

// R[i][j][a][b] += L+[ab][ij] + sgn(b-a) sgn(j-i) L-[ab][ij]
__global__ void k_ladder_unpack(const double* Lp, const double* Lm, double* R, int o, int v, int ldp, int ldm) {
  const long long vv = static_cast<long long>(v) * v;
  const long long total = static_cast<long long>(o) * o * vv;
  GRID_STRIDE(idx, total) {
    const int b = idx % v, a = (idx / v) % v, j = (idx / vv) % o, i = idx / (vv * o);
    const int a0 = min(a, b), b0 = max(a, b), i0 = min(i, j), j0 = max(i, j);
    double L = Lp[static_cast<long long>(tri_le(a0, b0)) * ldp + tri_le(i0, j0)];
    if (a != b && i != j) {
      const double s = ((b > a) == (j > i)) ? 1.0 : -1.0;
      L += s * Lm[static_cast<long long>(tri_lt(a0, b0)) * ldm + tri_lt(i0, j0)];
    }
    R[idx] += L;
  }
}

// Doubles residual R = Rsym + S + S^(ij)(ab) + P[C2] and update t2n = t2 + R / D.
// C2_aibj = -1/2 Cp[j,b,i,a] - Cp[i,b,j,a] (Cp[(j,b),(i,a)] = sum_kc t_kj^bc X_kiac).
// The three operands read with (a, b) exchanged -- S[j][i][b][a], Cp[(j,b)(i,a)], Cp[(i,b)(j,a)] -- go
// through 32 x 32 shared-memory tiles so that every global access is coalesced. Blocks walk the
// (i, j, a-tile, b-tile) tiles grid-stride; the per-block partial of sum d^2 is in a fixed order.
__global__ void k_assemble(const double* __restrict__ Rsym, const double* __restrict__ S, const double* __restrict__ Cp,
                           const double* __restrict__ t2, const double* __restrict__ eps, double* __restrict__ t2n,
                           double* __restrict__ err, double* __restrict__ part, int o, int v) {
  __shared__ double TS[32][33], T1[32][33], T2[32][33];  // [b_local][a_local]
  const long long vv = static_cast<long long>(v) * v, ov = static_cast<long long>(o) * v;
  const int nt = (v + 31) / 32;
  const long long ntiles = static_cast<long long>(o) * o * nt * nt;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  double acc = 0.0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int bt = static_cast<int>(t % nt), at = static_cast<int>((t / nt) % nt);
    const int ij = static_cast<int>(t / (static_cast<long long>(nt) * nt)), j = ij % o, i = ij / o;
    const int a0 = 32 * at, b0 = 32 * bt;
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int b = b0 + r, a = a0 + tx;
      const bool ok = a < v && b < v;
      TS[r][tx] = ok ? S[(static_cast<long long>(j) * o + i) * vv + static_cast<long long>(b) * v + a] : 0.0;
      T1[r][tx] = ok ? Cp[(static_cast<long long>(j) * v + b) * ov + static_cast<long long>(i) * v + a] : 0.0;
      T2[r][tx] = ok ? Cp[(static_cast<long long>(i) * v + b) * ov + static_cast<long long>(j) * v + a] : 0.0;
    }
    __syncthreads();
    const double ei_j = eps[i] + eps[j];
    for (int r = ty; r < 32; r += 8) {
      const int a = a0 + r, b = b0 + tx;
      if (a >= v || b >= v) continue;
      const long long idx = (static_cast<long long>(i) * o + j) * vv + static_cast<long long>(a) * v + b;
      const double c2 = -0.5 * T1[tx][r] - T2[tx][r] -
                        0.5 * Cp[(static_cast<long long>(i) * v + a) * ov + static_cast<long long>(j) * v + b] -
                        Cp[(static_cast<long long>(j) * v + a) * ov + static_cast<long long>(i) * v + b];
      const double R = Rsym[idx] + S[idx] + TS[tx][r] + c2;
      const double D = ei_j - eps[o + a] - eps[o + b];
      const double d = R / D;
      t2n[idx] = t2[idx] + d;
      err[idx] = d;
      acc += d * d;
    }
  }
  block_sum_store(acc, part);
}

// Singles: R1[i][a] += F_vo[a][i]; t1n = t1 + R1 / (e_i - e_a)
__global__ void k_update_t1(const double* R1, const double* Fvo, const double* t1, const double* eps, double* t1n,
                            double* err, double* part, int o, int v) {
  double acc = 0.0;
  GRID_STRIDE(idx, static_cast<long long>(o) * v) {
    const int a = idx % v, i = idx / v;
    const double R = R1[idx] + Fvo[a * o + i];
    const double d = R / (eps[i] - eps[o + a]);
    t1n[idx] = t1[idx] + d;
    err[idx] = d;
    acc += d * d;
  }
  block_sum_store(acc, part);
}

// E = sum_ijab (t_ij^ab + t_i^a t_j^b)(2(ia|jb) - (ib|ja)); OVOV[i][a][j][b] = (ia|jb)
// Lpair[i][j][a][b] = 2(ia|jb) - (ib|ja) (k_pair_L): both streams read in the same order (coalesced)
__global__ void k_energy(const double* t1, const double* t2, const double* Lpair, double* part, int o, int v) {
  const long long vv = static_cast<long long>(v) * v;
  const long long total = static_cast<long long>(o) * o * vv;
  double acc = 0.0;
  GRID_STRIDE(idx, total) {
    const int b = idx % v, a = (idx / v) % v, j = (idx / vv) % o, i = idx / (vv * o);
    const double tau = t2[idx] + (t1 ? t1[i * v + a] * t1[j * v + b] : 0.0);
    acc += tau * Lpair[idx];
  }
  block_sum_store(acc, part);
}

// Fixed-order final sum of `n` partials into out[0].
__global__ void k_finish_sum(const double* part, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  block_sum_store(acc, out);
}

// t2mp2[i][j][a][b] = (ia|jb) / (e_i + e_j - e_a - e_b)
__global__ void k_mp2_amps(const double* ovov, const double* eps, double* t2, int o, int v) {
  const long long vv = static_cast<long long>(v) * v;
  const long long total = static_cast<long long>(o) * o * vv;
  GRID_STRIDE(idx, total) {
    const int b = idx % v, a = (idx / v) % v, j = (idx / vv) % o, i = idx / (vv * o);
    const double iajb = ovov[((static_cast<long long>(i) * v + a) * o + j) * v + b];
    t2[idx] = iajb / (eps[i] + eps[j] - eps[o + a] - eps[o + b]);
  }
}

// dots[k] partials: sum_x e_new[x] * e_all[k][x] for k < m, one block row per k.
// DIIS bookkeeping lives on the device so that one CUDA graph serves every iteration:
// ctr[0] = vectors pushed so far (cnt); the new vector goes to slot cnt % mmax and the subspace then
// holds min(cnt + 1, mmax) vectors. k_diis_solve advances ctr[0] and records that count in ctr[1].
__device__ __forceinline__ int diis_slot(const int* ctr, int mmax) { return ctr[0] % mmax; }
__device__ __forceinline__ int diis_nvec(const int* ctr, int mmax) { return min(ctr[0] + 1, mmax); }

__global__ void k_diis_push(const double* __restrict__ x, const double* __restrict__ e, double* __restrict__ xs,
                            double* __restrict__ es, long long len, int mmax, const int* __restrict__ ctr) {
  const long long off = static_cast<long long>(diis_slot(ctr, mmax)) * len;
  GRID_STRIDE(idx, len) {
    xs[off + idx] = x[idx];
    es[off + idx] = e[idx];
  }
}
__global__ void k_dots(const double* e_new, const double* e_all, long long len, int mmax, const int* ctr,
                       double* part, int nblk) {
  const int k = blockIdx.y;
  if (k >= diis_nvec(ctr, mmax)) return;
  double acc = 0.0;
  for (long long x = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; x < len;
       x += static_cast<long long>(gridDim.x) * blockDim.x)
    acc += e_new[x] * e_all[k * len + x];
  block_sum_store(acc, part + static_cast<long long>(k) * nblk);
}
__global__ void k_finish_dots(const double* part, int nblk, const int* ctr, double* G, int mmax) {
  const int k = blockIdx.x;
  if (k >= diis_nvec(ctr, mmax)) return;
  const int slot = diis_slot(ctr, mmax);
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[static_cast<long long>(k) * nblk + i];
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) {
    G[slot * mmax + k] = tot;
    G[k * mmax + slot] = tot;
  }
}
__global__ void k_diis_solve(const double* G, int mmax, int* ctr, double* coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = diis_nvec(ctr, mmax), newest = diis_slot(ctr, mmax);
  ctr[0] += 1;
  ctr[1] = m;
  double A[9][10];
  const int n = m + 1;
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(G[i * mmax + i]));
  if (!(scale > 0.0)) scale = 1.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i][j] = G[i * mmax + j] / scale;
    A[i][m] = -1.0;
    A[i][n] = 0.0;
  }
  for (int j = 0; j < m; ++j) A[m][j] = -1.0;
  A[m][m] = 0.0;
  A[m][n] = -1.0;
  bool ok = true;
  for (int c = 0; c < n && ok; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (!(fabs(A[p][c]) > 1e-300)) {
      ok = false;
      break;
    }
    if (p != c)
      for (int k = 0; k <= n; ++k) {
        const double t = A[c][k];
        A[c][k] = A[p][k];
        A[p][k] = t;
      }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r][c] / A[c][c];
      for (int k = c; k <= n; ++k) A[r][k] -= f * A[c][k];
    }
  }
  double sum = 0.0;
  if (ok)
    for (int i = 0; i < m; ++i) {
      coef[i] = A[i][n] / A[i][i];
      if (!isfinite(coef[i])) ok = false;
      sum += coef[i];
    }
  if (!ok || !(fabs(sum - 1.0) < 1e-6)) {
    for (int i = 0; i < m; ++i) coef[i] = (i == newest) ? 1.0 : 0.0;
  }
}

// out[x] = sum_k coef[k] * vecs[k][x]
__global__ void k_extrapolate(const double* vecs, const double* coef, const int* ctr, long long len, double* out) {
  const int m = ctr[1];
  GRID_STRIDE(x, len) {
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc += coef[k] * vecs[k * len + x];
    out[x] = acc;
  }
}

// E[i][i'] = sum_x tau[i][x] L[i'][x] over x = (j,a,b): one block per (i,i'), FP64, fixed order.
__global__ void k_pair_dots(const double* __restrict__ tau, const double* __restrict__ L, int o, long long K,
                            double* __restrict__ E) {
  const int i = blockIdx.x / o, ip = blockIdx.x % o;
  const double* a = tau + i * K;
  const double* b = L + ip * K;
  double acc = 0.0;
  for (long long x = threadIdx.x; x < K; x += blockDim.x) acc += a[x] * b[x];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) E[blockIdx.x] = t;
}

// E_frag = sum_alpha sum_ii' U[i][alpha] E[i][i'] U[i'][alpha]   (one block)
__global__ void k_project(const double* E, const double* U, int o, int nlo, double* out) {
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < o * o * nlo; idx += blockDim.x) {
    const int al = idx % nlo, ip = (idx / nlo) % o, i = idx / (nlo * o);
    acc += U[i * nlo + al] * E[i * o + ip] * U[ip * nlo + al];
  }
  block_sum_store(acc, out);
}

// Lpair[i'][j][a][b] = 2(i'a|jb) - (i'b|ja)
__global__ void k_pair_L(const double* ovov, double* L, int o, int v) {
  const long long vv = static_cast<long long>(v) * v;
  const long long total = static_cast<long long>(o) * o * vv;
  GRID_STRIDE(idx, total) {
    const int b = idx % v, a = (idx / v) % v, j = (idx / vv) % o, i = idx / (vv * o);
    L[idx] = 2.0 * ovov[((static_cast<long long>(i) * v + a) * o + j) * v + b] -
             ovov[((static_cast<long long>(i) * v + b) * o + j) * v + a];
  }
}

// V+/-[ab][cd] from G[a][c][b][d] = (ac|bd) for rows with a in [a0, a0 + na):
//   V+ = (ac|bd) + (ad|bc) (a<=b, c<=d),  V- = (ac|bd) - (ad|bc) (a<b, c<d)
// V+-[ab][cd] from G[al][c][b][d] = (a0+al c|b d): for fixed (al, b) the v x v slice M[c][d] is combined
// with its transpose, M[c][d] +- M[d][c]. One block per (al, b, 32 x 32 tile pair (cb <= db)): both tiles
// are read coalesced into shared memory, and the packed rows (c fastest for fixed d, as tri_le(c, d)
// runs) are written coalesced.
__device__ __forceinline__ void split_bf16g(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) { split_bf16(x, hi, lo); }
__device__ __forceinline__ void split_bf16g(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

template <bool BF16, typename TG>
__global__ void k_pack_vvvv(const TG* __restrict__ G, int a0, int v, void* Vp, void* Vm, int Kpp, int Kpm,
                            long long plane_p, long long plane_m) {
  __shared__ TG T1[32][33], T2[32][33];  // T1[c][d] = M[cb+c][db+d], T2[d][c] = M[db+d][cb+c]
  const int al = blockIdx.z, b = blockIdx.y, a = a0 + al;
  if (a > b) return;
  // tile pair index -> (cb, db) with cb <= db over T = ceil(v / 32) tiles
  int tp = blockIdx.x, cbt = 0;
  const int T = (v + 31) / 32;
  while (tp >= T - cbt) {
    tp -= T - cbt;
    ++cbt;
  }
  const int cb = 32 * cbt, db = 32 * (cbt + tp);
  const long long vv = static_cast<long long>(v) * v;
  const TG* Mb = G + (static_cast<long long>(al) * v * vv + b * static_cast<long long>(v));  // M[c][d] = Mb[c*vv + d]
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int c1 = cb + r, d1 = db + tx;
    T1[r][tx] = (c1 < v && d1 < v) ? Mb[c1 * vv + d1] : TG(0);
    const int d2 = db + r, c2 = cb + tx;
    T2[r][tx] = (d2 < v && c2 < v) ? Mb[d2 * vv + c2] : TG(0);
  }
  __syncthreads();
  const long long rowp = static_cast<long long>(tri_le(a, b)) * Kpp;
  const long long rowm = a < b ? static_cast<long long>(tri_lt(a, b)) * Kpm : -1;
  for (int r = ty; r < 32; r += 8) {
    const int d = db + r, c = cb + tx;
    if (d >= v || c >= v || c > d) continue;
    // FP32 G (mixed path): sums and the BF16 split in FP32; FP64 G: FP64
    const TG acbd = T1[tx][r], adbc = T2[r][tx];
    const TG xp = acbd + adbc;
    const long long pp = rowp + tri_le(c, d);
    if (BF16) {
      __nv_bfloat16 hi, lo;
      split_bf16g(xp, hi, lo);
      static_cast<__nv_bfloat16*>(Vp)[pp] = hi;
      static_cast<__nv_bfloat16*>(Vp)[pp + plane_p] = lo;
    } else {
      static_cast<double*>(Vp)[pp] = xp;
    }
    if (rowm >= 0 && c < d) {
      const TG xm = acbd - adbc;
      const long long pm = rowm + tri_lt(c, d);
      if (BF16) {
        __nv_bfloat16 hi, lo;
        split_bf16g(xm, hi, lo);
        static_cast<__nv_bfloat16*>(Vm)[pm] = hi;
        static_cast<__nv_bfloat16*>(Vm)[pm + plane_m] = lo;
      } else {
        static_cast<double*>(Vm)[pm] = xm;
      }
    }
  }
}

// Dense n x n dressing matrices: X = 1 - T, Y = 1 + T with T[o+a][i] = t_i^a.
__global__ void k_dress_mats(const double* t1, double* X, double* Y, int o, int v) {
  const int n = o + v;
  GRID_STRIDE(idx, static_cast<long long>(n) * n) {
    const int q = idx % n, p = idx / n;
    double t = (p >= o && q < o) ? t1[q * v + (p - o)] : 0.0;
    const double d = (p == q) ? 1.0 : 0.0;
    X[idx] = d - t;
    Y[idx] = d + t;
  }
}

// T1-transformed one-electron part h^ = (1 - T) h (1 + T), T[o+a][i] = t_i^a, in two steps:
//   g_kq  = h_kq + [q occ] sum_c h_k,c t_q^c                    (occupied rows k of h (1 + T))
//   h^_pq = h_pq + [q occ] sum_c h_p,c t_q^c - [p vir] sum_k t_k^p g_kq
__global__ void k_hhat_rows(const double* __restrict__ h, const double* __restrict__ t1, double* __restrict__ g, int o,
                            int v) {
  const int n = o + v;
  GRID_STRIDE(idx, static_cast<long long>(o) * n) {
    const int q = idx % n, k2 = idx / n;
    double r = h[k2 * n + q];
    if (q < o)
      for (int c = 0; c < v; ++c) r += h[k2 * n + o + c] * t1[q * v + c];
    g[idx] = r;
  }
}
__global__ void k_hhat(const double* __restrict__ h, const double* __restrict__ t1, const double* __restrict__ g,
                       double* __restrict__ out, int o, int v) {
  const int n = o + v;
  GRID_STRIDE(idx, static_cast<long long>(n) * n) {
    const int q = idx % n, p = idx / n;
    double r = h[idx];
    if (q < o)
      for (int c = 0; c < v; ++c) r += h[p * n + o + c] * t1[q * v + c];
    if (p >= o)
      for (int k2 = 0; k2 < o; ++k2) r -= t1[k2 * v + (p - o)] * g[k2 * n + q];
    out[idx] = r;
  }
}

// xq[Q] = sum_k Boo[Q][k][k]
__global__ void k_trace_oo(const double* Boo, int naux, int o, double* xq) {
  GRID_STRIDE(Q, naux) {
    double s = 0.0;
    for (int k = 0; k < o; ++k) s += Boo[(static_cast<long long>(Q) * o + k) * o + k];
    xq[Q] = s;
  }
}

// dst[p*ld + q] += alpha * sum_Q B[Q*qstride + p*rstride + q] x[Q]
// Block of 32 (p,q) x 8 Q-lanes: each lane sums every 8th Q, then a fixed-order reduction over the lanes.
__global__ void k_coulomb(const double* B, long long qstride, int rows, int cols, long long rstride, const double* x,
                          int naux, double alpha, double* dst, long long ld) {
  __shared__ double part[8][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const long long total = static_cast<long long>(rows) * cols;
  const long long idx = static_cast<long long>(blockIdx.x) * 32 + tx;
  double acc = 0.0;
  if (idx < total) {
    const int q = static_cast<int>(idx % cols), p = static_cast<int>(idx / cols);
    const double* b = B + p * rstride + q;
#pragma unroll 4
    for (int Q = ty; Q < naux; Q += 8) acc += b[Q * qstride] * x[Q];
  }
  part[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && idx < total) {
    double s = 0.0;
    for (int l = 0; l < 8; ++l) s += part[l][tx];
    const int q = static_cast<int>(idx % cols), p = static_cast<int>(idx / cols);
    dst[p * ld + q] += alpha * s;
  }
}

// NaN / Inf scan; flag[0] = 1 if any
__global__ void k_finite(const double* x, long long n, int* flag) {
  GRID_STRIDE(i, n) {
    if (!isfinite(x[i])) atomicExch(flag, 1);
  }
}

// E2 occupied part, S[i][j][ab] -= sum_k t2[i][k][ab] F[k][j] (nocc <= 32): a contraction of length
// nocc is bound by the traffic of t2 and S, so it runs as one streaming pass with FP32 products and
// sums (relative error ~1e-7, below the BF16x3 contractions of the mixed path) instead of a padded GEMM.
template <int MAXO>
__global__ void k_e2_occ(const double* __restrict__ t2, const double* __restrict__ F, double* __restrict__ S, int o,
                         long long vv) {
  __shared__ float Fs[32][33];
  for (int x = threadIdx.x; x < 32 * 32; x += blockDim.x) {
    const int k = x / 32, j = x % 32;
    Fs[k][j] = (k < o && j < o) ? static_cast<float>(F[k * o + j]) : 0.f;
  }
  __syncthreads();
  const long long total = static_cast<long long>(o) * vv;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long i = e / vv, ab = e % vv;
    float t[MAXO];
#pragma unroll
    for (int k = 0; k < MAXO; ++k) t[k] = k < o ? f64_to_f32_fields(t2[(i * o + k) * vv + ab]) : 0.f;
    for (int j = 0; j < o; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < MAXO; ++k) acc = fmaf(t[k], Fs[k][j], acc);
      S[(i * o + j) * vv + ab] -= f32_to_f64_fields(acc);
    }
  }
}

// T1 dressing of the virtual-virtual DF block in one pass over B_vv (mixed path, nocc <= 32): per row
// (Q, a), with t1 and B_ov[Q] staged in shared memory,
//   B^_vv[Q][a][c] = B_vv[Q][a][c] - sum_k t_k^a B_ov[Q][k][c]
//   B^_vo[Q][a][i] += sum_c B_vv[Q][a][c] t_i^c
// Both corrections are length-o / length-v dot products on data read once, so the pass is bound by the
// traffic of B_vv (read) and B^_vv (written); products, sums and the difference in FP32 (relative
// error ~1e-7; every consumer of B^_vv on the mixed path splits it into BF16 hi/lo, 16 bits), the
// conversions through the IEEE fields (no FP64-pipe work per element), the dressed factors stored as
// FP64. One warp per row; the v-sums end in a fixed-order warp butterfly.
template <int MAXO>
__global__ void __launch_bounds__(256, 2) k_dress_vv(const double* __restrict__ Bvv, const double* __restrict__ Bov,
                           const double* __restrict__ t1, double* __restrict__ Bvv_h, double* __restrict__ Bvo_h,
                           int o, int v) {
  // Rows of B_vv[Q] in chunks of kRows: each thread owns columns c (it keeps B_ov[Q][k][c] for its
  // column in registers) and reads the chunk's kRows values of its column with all loads in flight;
  // the chunk is kept (FP32) in shared memory for the B^_vo sums, one (a, k) per thread. Row strides of
  // v + 1 floats keep the column-wise reads of t1 free of bank conflicts.
  constexpr int kRows = 16;
  extern __shared__ float dsm[];
  const int vp = v + 1;
  float* ts = dsm;              // t1[k][c], row stride vp
  float* xs = dsm + MAXO * vp;  // the chunk's rows of B_vv[Q] (FP32), row stride vp
  const int Q = blockIdx.x;
  const long long ov = static_cast<long long>(o) * v, vv = static_cast<long long>(v) * v;
  // rows k >= nocc are zero (the unrolled k loops below read all MAXO rows)
  for (int x = threadIdx.x; x < MAXO * v; x += blockDim.x) {
    const int k = x / v, c = x % v;
    ts[k * vp + c] = k < o ? f64_to_f32_fields(t1[x]) : 0.f;
  }
  __syncthreads();
  const double* Bq = Bvv + Q * vv;
  double* Hq = Bvv_h + Q * vv;
  for (int a0 = 0; a0 < v; a0 += kRows) {
    const int nr = min(kRows, v - a0);
    for (int c = threadIdx.x; c < v; c += blockDim.x) {
      float bk[MAXO];
#pragma unroll
      for (int k = 0; k < MAXO; ++k) bk[k] = k < o ? f64_to_f32_fields(Bov[Q * ov + 1LL * k * v + c]) : 0.f;
      double xr[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) xr[r] = r < nr ? Bq[1LL * (a0 + r) * v + c] : 0.0;
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        if (r < nr) {
          const float xf = f64_to_f32_fields(xr[r]);
          float corr = 0.f;
#pragma unroll
          for (int k = 0; k < MAXO; ++k) corr = fmaf(ts[k * vp + a0 + r], bk[k], corr);  // t_k^a B_ov[Q][k][c]
          Hq[1LL * (a0 + r) * v + c] = f32_to_f64_fields(xf - corr);
          xs[r * vp + c] = xf;
        }
      }
    }
    __syncthreads();
    // B^_vo[Q][a][k] += sum_c B_vv[Q][a][c] t_k^c for the chunk's rows (fixed summation order over c)
    for (int e = threadIdx.x; e < nr * o; e += blockDim.x) {
      const int r = e / o, k = e % o;
      const float* xr = xs + r * vp;
      const float* tk = ts + k * vp;
      float acc = 0.f;
      for (int c = 0; c < v; ++c) acc = fmaf(xr[c], tk[c], acc);
      Bvo_h[Q * ov + 1LL * (a0 + r) * o + k] += static_cast<double>(acc);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// launch wrappers
void launch_tau(const double* t1, const double* t2, double* tau, int o, int v, cudaStream_t s) {
  count_launch();
  k_tau<<<grid_for(1LL * o * o * v * v), kThreads, 0, s>>>(t1, t2, tau, o, v);
}
void launch_u(const double* t2, double* u, int o, int v, cudaStream_t s) {
  count_launch();
  k_u<<<grid_for(1LL * o * o * v * v), kThreads, 0, s>>>(t2, u, o, v);
}
void launch_ladder_ops(const double* t2, Packed& Bp, Packed& Bm, int o, int v, cudaStream_t s) {
  const long long pp = 1LL * Bp.rows * Bp.Kp, pm = 1LL * Bm.rows * Bm.Kp;
  count_launch();
  if (Bp.bf16)
    k_ladder_ops<true><<<grid_for(1LL * o * o * v * v), kThreads, 0, s>>>(t2, Bp.p, Bm.p, o, v, Bp.Kp, Bm.Kp, pp, pm);
  else
    k_ladder_ops<false>
        <<<grid_for(1LL * o * o * v * v), kThreads, 0, s>>>(t2, Bp.p, Bm.p, o, v, Bp.Kp, Bm.Kp, pp, pm);
}
void launch_ladder_unpack(const double* Lp, const double* Lm, double* R, int o, int v, int ldp, int ldm,
                          cudaStream_t s) {
  count_launch();
  k_ladder_unpack<<<grid_for(1LL * o * o * v * v), kThreads, 0, s>>>(Lp, Lm, R, o, v, ldp, ldm);
}
int launch_assemble(const double* Rsym, const double* S, const double* Cp, const double* t2, const double* eps,
                    double* t2n, double* err, double* part, int o, int v, cudaStream_t s) {
  const int nt = (v + 31) / 32;
  const int g = static_cast<int>(std::min<long long>(1LL * o * o * nt * nt, 152LL * 8));
  count_launch();
  k_assemble<<<g, kThreads, 0, s>>>(Rsym, S, Cp, t2, eps, t2n, err, part, o, v);
  return g;
}
int launch_update_t1(const double* R1, const double* Fvo, const double* t1, const double* eps, double* t1n,
                     double* err, double* part, int o, int v, cudaStream_t s) {
  const int g = grid_for(1LL * o * v);
  count_launch();
  k_update_t1<<<g, kThreads, 0, s>>>(R1, Fvo, t1, eps, t1n, err, part, o, v);
  return g;
}
int launch_energy(const double* t1, const double* t2, const double* Lpair, double* part, int o, int v,
                  cudaStream_t s) {
  const int g = grid_for(1LL * o * o * v * v);
  count_launch();
  k_energy<<<g, kThreads, 0, s>>>(t1, t2, Lpair, part, o, v);
  return g;
}
void launch_finish_sum(const double* part, int n, double* out, cudaStream_t s) {
  count_launch();
  k_finish_sum<<<1, 1024, 0, s>>>(part, n, out);
}
void launch_mp2_amps(const double* ovov, const double* eps, double* t2, int o, int v, cudaStream_t s) {
  count_launch();
  k_mp2_amps<<<grid_for(1LL * o * o * v * v), kThreads, 0, s>>>(ovov, eps, t2, o, v);
}
void launch_diis_step(const double* x_new, const double* e_new, double* xs, double* es, long long len, int mmax,
                      int* ctr, double* part, double* G, double* coef, double* out, cudaStream_t s) {
  const int nblk = 152;
  count_launch(5);
  k_diis_push<<<grid_for(len), kThreads, 0, s>>>(x_new, e_new, xs, es, len, mmax, ctr);
  k_dots<<<dim3(nblk, mmax), kThreads, 0, s>>>(e_new, es, len, mmax, ctr, part, nblk);
  k_finish_dots<<<mmax, kThreads, 0, s>>>(part, nblk, ctr, G, mmax);
  k_diis_solve<<<1, 32, 0, s>>>(G, mmax, ctr, coef);
  k_extrapolate<<<grid_for(len), kThreads, 0, s>>>(xs, coef, ctr, len, out);
}
void launch_project(const double* E, const double* U, int o, int nlo, double* out, cudaStream_t s) {
  count_launch();
  k_project<<<1, 256, 0, s>>>(E, U, o, nlo, out);
}
void launch_pair_dots(const double* tau, const double* L, int o, long long K, double* E, cudaStream_t s) {
  count_launch();
  k_pair_dots<<<o * o, 512, 0, s>>>(tau, L, o, K, E);
}
void launch_pair_L(const double* ovov, double* L, int o, int v, cudaStream_t s) {
  count_launch();
  k_pair_L<<<grid_for(1LL * o * o * v * v), kThreads, 0, s>>>(ovov, L, o, v);
}
void launch_pack_vvvv(const void* G, bool g32, int a0, int na, int v, Packed& Vp, Packed& Vm, cudaStream_t s) {
  const long long pp = 1LL * Vp.rows * Vp.Kp, pm = 1LL * Vm.rows * Vm.Kp;
  const int T = (v + 31) / 32;
  dim3 grid(T * (T + 1) / 2, v, na);
  count_launch();
  if (Vp.bf16 && g32)
    k_pack_vvvv<true, float><<<grid, 256, 0, s>>>(static_cast<const float*>(G), a0, v, Vp.p, Vm.p, Vp.Kp, Vm.Kp, pp, pm);
  else if (Vp.bf16)
    k_pack_vvvv<true, double><<<grid, 256, 0, s>>>(static_cast<const double*>(G), a0, v, Vp.p, Vm.p, Vp.Kp, Vm.Kp, pp,
                                                   pm);
  else
    k_pack_vvvv<false, double><<<grid, 256, 0, s>>>(static_cast<const double*>(G), a0, v, Vp.p, Vm.p, Vp.Kp, Vm.Kp, pp,
                                                    pm);
}
void launch_dress_mats(const double* t1, double* X, double* Y, int o, int v, cudaStream_t s) {
  count_launch();
  k_dress_mats<<<grid_for(1LL * (o + v) * (o + v)), kThreads, 0, s>>>(t1, X, Y, o, v);
}
void launch_hhat(const double* h, const double* t1, double* g, double* out, int o, int v, cudaStream_t s) {
  count_launch(2);
  k_hhat_rows<<<grid_for(1LL * o * (o + v)), kThreads, 0, s>>>(h, t1, g, o, v);
  k_hhat<<<grid_for(1LL * (o + v) * (o + v)), kThreads, 0, s>>>(h, t1, g, out, o, v);
}
void launch_trace_oo(const double* Boo, int naux, int o, double* xq, cudaStream_t s) {
  count_launch();
  k_trace_oo<<<grid_for(naux), kThreads, 0, s>>>(Boo, naux, o, xq);
}
void launch_coulomb(const double* B, long long qstride, int rows, int cols, long long rstride, const double* x,
                    int naux, double alpha, double* dst, long long ld, cudaStream_t s) {
  count_launch();
  k_coulomb<<<static_cast<int>((1LL * rows * cols + 31) / 32), 256, 0, s>>>(B, qstride, rows, cols, rstride, x, naux,
                                                                          alpha, dst, ld);
}
void launch_dress_vv(const double* Bvv, const double* Bov, const double* t1, double* Bvv_h, double* Bvo_h, int naux,
                     int o, int v, cudaStream_t s) {
  static std::once_flag once;  // the attribute is process-wide: set it once, to the largest size used
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_dress_vv<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (16 + 16) * 851 * 4);
    cudaFuncSetAttribute(k_dress_vv<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (32 + 16) * 851 * 4);
  });
  count_launch();
  // t1 (MAXO rows) and one chunk of 16 rows of B_vv[Q], row stride v + 1
  if (o <= 16) {
    const size_t sm = (16 + 16) * static_cast<size_t>(v + 1) * 4;
    k_dress_vv<16><<<naux, 256, sm, s>>>(Bvv, Bov, t1, Bvv_h, Bvo_h, o, v);
  } else {
    const size_t sm = (32 + 16) * static_cast<size_t>(v + 1) * 4;
    k_dress_vv<32><<<naux, 256, sm, s>>>(Bvv, Bov, t1, Bvv_h, Bvo_h, o, v);
  }
}
void launch_e2_occ(const double* t2, const double* F, double* S, int o, int v, cudaStream_t s) {
  count_launch();
  if (o <= 16)
    k_e2_occ<16><<<grid_for(1LL * o * v * v), kThreads, 0, s>>>(t2, F, S, o, 1LL * v * v);
  else
    k_e2_occ<32><<<grid_for(1LL * o * v * v), kThreads, 0, s>>>(t2, F, S, o, 1LL * v * v);
}
void launch_finite(const double* x, long long n, int* flag, cudaStream_t s) {
  count_launch();
  k_finite<<<grid_for(n), kThreads, 0, s>>>(x, n, flag);
}

}  // namespace lnocc
