// LNO-(T): W and V intermediates of the supplementary Sec. S1 and the projected (T) pair energy of
// Eq. 10, summed as E^(F) = sum_alpha sum_ii' U_i,alpha E_ii',(T) U_i',alpha (Eq. 9).
//
// Loop structure ("virtual-outer"): for each pair b <= c and every a <= b the block
// W^{abc}_{ijk} over all occupied (i,j,k) is formed. Because W and V are invariant under a
// simultaneous permutation of (i,a), (j,b), (k,c), the block of the sorted triple a<=b<=c yields
// W^{pi(abc)} for every ordering pi by permuting (i,j,k), so each distinct virtual triple is formed
// once (2 o^3 v^4 + 2 o^4 v^3 flops in the contractions), and the projection over (i, i') stays
// local to the block.
//
// For a fixed (b, c) the six d-terms and six l-terms of W are GEMMs over d (or l) whose rows run
// over a and one occupied index:
//   G_i  rows (a,i), cols (k,j): (ai|bd) t_kj^cd + (ai|cd) t_jk^bd - t_il^ab (ck|jl) - t_il^ac (bj|kl)
//   G_j  rows (a,j), cols (k,i): (bj|ad) t_ki^cd - t_jl^ba (ck|il)
//   G_k  rows (a,k), cols (j,i): (ck|ad) t_ji^bd - t_kl^ca (bj|il)
//   G_4  rows (a,i,k), cols j  : t_ik^ad (bj|cd) - (ai|kl) t_jl^bc
//   G_6  rows (a,i,j), cols k  : t_ij^ad (ck|bd) - (ai|jl) t_kl^cb
// all accumulated into W[a][i][j][k]; a block energy kernel then applies V = W + (ai|bj) t_k^c +
// (ai|ck) t_j^b + (bj|ck) t_i^a, w = W / sqrt(-Delta), v = V / sqrt(-Delta) and the contraction
// -1/3 sum (4 w^abc + w^bca + w^cab)(v^abc - v^cba) for every distinct ordering of (a, b, c).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ccsd_kernels.h"
#include "fragment.h"
#include "internal.h"

namespace lnocc {

static inline Ax A_(int n, long long s) { return Ax{n, s}; }

namespace {

// Position permutations of three slots, listed as (p1, p2, p3) in 0-based slots.
__constant__ int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Block energy. One CTA per (pair, a) with a <= b; threads over (j, k).
// W: [slot][a][i][j][k]; out: per block {canonical, projected} partials (FP64).
__global__ void k_t_energy(const double* __restrict__ W, long long slot_stride, const int* __restrict__ pb,
                           const int* __restrict__ pc, int pair0, int o, int v, const double* __restrict__ eps,
                           const double* __restrict__ t1, const double* __restrict__ ovov,
                           const double* __restrict__ U, int nlo, double* __restrict__ out) {
  const int slot = blockIdx.y;
  const int a = blockIdx.x;
  const int b = pb[pair0 + slot], c = pc[pair0 + slot];
  const long long oblk = 1LL * o * o * o;
  const long long blk_id = (1LL * (pair0 + slot)) * v + a;
  if (a > b) {
    if (threadIdx.x == 0) {
      out[2 * blk_id] = 0.0;
      out[2 * blk_id + 1] = 0.0;
    }
    return;
  }
  const double* Wb = W + slot * slot_stride + a * oblk;
  const int x[3] = {a, b, c};
  const double ex = eps[o + a] + eps[o + b] + eps[o + c];
  const long long ov = 1LL * o * v;
  auto widx = [&](int y0, int y1, int y2) { return (1LL * y0 * o + y1) * o + y2; };
  // w and v of the block at occupied (y0, y1, y2)
  auto wv = [&](int y0, int y1, int y2, double& w, double& vv) {
    const double Wv = Wb[widx(y0, y1, y2)];
    const double Vv = Wv + ovov[(1LL * y0 * v + a) * ov + 1LL * y1 * v + b] * t1[y2 * v + c] +
                      ovov[(1LL * y0 * v + a) * ov + 1LL * y2 * v + c] * t1[y1 * v + b] +
                      ovov[(1LL * y1 * v + b) * ov + 1LL * y2 * v + c] * t1[y0 * v + a];
    const double s = 1.0 / sqrt(ex - eps[y0] - eps[y1] - eps[y2]);
    w = Wv * s;
    vv = Vv * s;
  };
  double e_can = 0.0, e_frag = 0.0;
  for (int jk = threadIdx.x; jk < o * o; jk += blockDim.x) {
    const int j = jk / o, k = jk % o;
    for (int pi = 0; pi < 6; ++pi) {
      const int p0 = kPerm[pi][0], p1 = kPerm[pi][1], p2 = kPerm[pi][2];
      // skip orderings already counted (equal labels)
      bool dup = false;
      for (int q = 0; q < pi && !dup; ++q)
        dup = x[kPerm[q][0]] == x[p0] && x[kPerm[q][1]] == x[p1] && x[kPerm[q][2]] == x[p2];
      if (dup) continue;
      // ordering T = (x[p0], x[p1], x[p2]); W^T_{ijk} = W^{abc}_y with y[p0]=i, y[p1]=j, y[p2]=k
      double zs[32], ys[32];
      for (int i = 0; i < o; ++i) {
        int y[3];
        double w0, w1, w2, v0, v3, dummy;
        y[p0] = i; y[p1] = j; y[p2] = k;        // T
        wv(y[0], y[1], y[2], w0, v0);
        y[p1] = i; y[p2] = j; y[p0] = k;        // T o c   = (t2, t3, t1): slots (p1, p2, p0)
        wv(y[0], y[1], y[2], w1, dummy);
        y[p2] = i; y[p0] = j; y[p1] = k;        // T o c^2 = (t3, t1, t2): slots (p2, p0, p1)
        wv(y[0], y[1], y[2], w2, dummy);
        y[p2] = i; y[p1] = j; y[p0] = k;        // (t3, t2, t1): slots (p2, p1, p0)
        wv(y[0], y[1], y[2], dummy, v3);
        const double z = 4.0 * w0 + w1 + w2;
        const double yy = v0 - v3;
        e_can += z * yy;
        if (i < 32) {
          zs[i] = z;
          ys[i] = yy;
        }
      }
      for (int al = 0; al < nlo; ++al) {
        double zu = 0.0, yu = 0.0;
        for (int i = 0; i < o && i < 32; ++i) {
          zu += U[i * nlo + al] * zs[i];
          yu += U[i * nlo + al] * ys[i];
        }
        e_frag += zu * yu;
      }
    }
  }
  // block reduction (fixed order)
  __shared__ double sh[2][32];
  for (int off = 16; off > 0; off >>= 1) {
    e_can += __shfl_xor_sync(0xffffffffu, e_can, off);
    e_frag += __shfl_xor_sync(0xffffffffu, e_frag, off);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) {
    sh[0][w] = e_can;
    sh[1][w] = e_frag;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < static_cast<int>(blockDim.x / 32); ++q) {
      s0 += sh[0][q];
      s1 += sh[1][q];
    }
    out[2 * blk_id] = -s0 / 3.0;
    out[2 * blk_id + 1] = -s1 / 3.0;
  }
}

// Sum of the per-block partials in a fixed order: out[0] canonical, out[1] projected.
__global__ void k_t_finish(const double* part, long long nblk, double* out) {
  __shared__ double sh[2][32];
  double s0 = 0.0, s1 = 0.0;
  for (long long i = threadIdx.x; i < nblk; i += blockDim.x) {
    s0 += part[2 * i];
    s1 += part[2 * i + 1];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) {
    sh[0][w] = s0;
    sh[1][w] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int q = 0; q < static_cast<int>(blockDim.x / 32); ++q) {
      a0 += sh[0][q];
      a1 += sh[1][q];
    }
    out[0] = a0;
    out[1] = a1;
  }
}

// dst row (y, a, i) <- src row (a, y, i) of a packed [planes][rows][Kp] operand (rows = v*v*o)
template <typename T>
__global__ void k_swap_outer_rows(const T* src, T* dst, int v, int o, int Kp, int planes) {
  const long long rows = 1LL * v * v * o;
  const long long total = rows * Kp * planes;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = idx % Kp;
    const long long r = (idx / Kp) % rows;
    const long long pl = idx / (Kp * rows);
    const int i = r % o, a = (r / o) % v, y = r / (1LL * o * v);
    const long long sr = (1LL * a * v + y) * o + i;
    dst[(pl * rows + r) * Kp + k] = src[(pl * rows + sr) * Kp + k];
  }
}

}  // namespace

// A packed operand restricted to a row range (FP64: pointer offset; BF16: the kernel needs the
// full plane stride, so the GEMM gets the row offset explicitly).
struct Sub {
  const Packed* P;
  int row0, rows;
};

int Frag::triples(int nlo, const double* U, double* e_full, double* e_frag) {
  const long long oo = 1LL * o * o, vv = 1LL * v * v, ov = 1LL * o * v, ooo = oo * o;
  const bool bf = mixed;
  cudaMemsetAsync(dstatus, 0, 16 * 4, s);
  const double* t1 = xcur;
  const double* t2 = xcur + ov;

  // ---- operands (packed once per call)
  std::vector<void*> mine;
  auto tmp_alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mine.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    for (void* p : mine) cudaFree(p);
  };
  auto mk = [&](int rows, int K) -> Packed {
    Packed P;
    P.rows = rows;
    P.Kp = round_up(std::max(K, 1), 64);
    P.bf16 = bf;
    P.p = tmp_alloc(static_cast<size_t>(rows) * P.Kp * (bf ? 4 : 8));
    if (P.p) cudaMemsetAsync(P.p, 0, static_cast<size_t>(rows) * P.Kp * (bf ? 4 : 8), s);
    return P;
  };
  Packed X1 = mk(static_cast<int>(vv * o), v), X2 = mk(static_cast<int>(vv * o), v);
  Packed Tv = mk(static_cast<int>(v * oo), v), TvT = mk(static_cast<int>(v * oo), v);
  Packed T2x = mk(static_cast<int>(vv * o), o), T2y = mk(static_cast<int>(vv * o), o);
  Packed O1 = mk(static_cast<int>(v * oo), o), O1T = mk(static_cast<int>(v * oo), o);
  double* ovoo = static_cast<double*>(tmp_alloc(ooo * v * 8));
  if (!X1.p || !X2.p || !Tv.p || !TvT.p || !T2x.p || !T2y.p || !O1.p || !O1T.p || !ovoo) {
    cleanup();
    set_error("lnocc_triples: device allocation failed (operands)");
    return LNOCC_ENOMEM;
  }
  // amplitudes: Tv[z][r][q][d] = t_rq^zd, TvT[z][k][j][d] = t_jk^zd,
  // T2x[x][a][i][l] = -t_il^ax, T2y[c][a][k][l] = -t_kl^ca (the l-terms enter W with a minus sign)
  pack(view(t2, A_(v, v), A_(o, o * vv), A_(o, vv), kOne, kOne, A_(v, 1)), Tv, s);
  pack(view(t2, A_(v, v), A_(o, vv), A_(o, o * vv), kOne, kOne, A_(v, 1)), TvT, s);
  pack(view(t2, A_(v, 1), A_(v, v), A_(o, o * vv), kOne, kOne, A_(o, vv), -1.0), T2x, s);
  pack(view(t2, A_(v, v), A_(v, 1), A_(o, o * vv), kOne, kOne, A_(o, vv), -1.0), T2y, s);
  // (kz|jl) -> O1[z][k][j][l] = (zk|jl), O1T[z][k][j][l] = (zj|kl)
  contract(view(Bov, kOne, kOne, A_(static_cast<int>(ov), 1), kOne, kOne, A_(N, ov)),
           view(Boo, kOne, kOne, A_(static_cast<int>(oo), 1), kOne, kOne, A_(N, oo)), out_rowmajor(ovoo, oo), true);
  pack(view(ovoo, A_(v, oo), A_(o, v * oo), A_(o, o), kOne, kOne, A_(o, 1)), O1, s);
  pack(view(ovoo, A_(v, oo), A_(o, o), A_(o, v * oo), kOne, kOne, A_(o, 1)), O1T, s);
  // (jb|ad) -> X2[b][a][j][d], in chunks of b; X1[y][a][i][d] = (ai|yd) = X2[a][y][i][d]
  {
    Packed PBvv = mk(static_cast<int>(vv), N);
    if (!PBvv.p) {
      cleanup();
      set_error("lnocc_triples: device allocation failed (B_vv)");
      return LNOCC_ENOMEM;
    }
    pack(view(Bvv, kOne, kOne, A_(static_cast<int>(vv), 1), kOne, kOne, A_(N, vv)), PBvv, s);
    const int bc = static_cast<int>(std::max(1LL, std::min<long long>(v, (1LL << 26) / (o * vv))));
    double* tmp = static_cast<double*>(tmp_alloc(static_cast<size_t>(bc) * o * vv * 8));
    if (!tmp) {
      cleanup();
      set_error("lnocc_triples: device allocation failed (ovvv chunk)");
      return LNOCC_ENOMEM;
    }
    const bool keep = mixed;
    mixed = bf;
    for (int b0 = 0; b0 < v; b0 += bc) {
      const int nb = std::min(bc, v - b0);
      contract_packed_b(view(Bov + b0, kOne, A_(o, v), A_(nb, 1), kOne, kOne, A_(N, ov)), PBvv, static_cast<int>(vv),
                        out_rowmajor(tmp, vv));
      pack_rows(view(tmp, A_(nb, vv), A_(v, v), A_(o, nb * vv), kOne, kOne, A_(v, 1)), X2, b0 * v * o, s);
    }
    mixed = keep;
    const long long tot = static_cast<long long>(X2.rows) * X2.Kp * (bf ? 2 : 1);
    const int blocks = static_cast<int>(std::min<long long>((tot + 255) / 256, 152LL * 32));
    if (bf)
      k_swap_outer_rows<unsigned short><<<blocks, 256, 0, s>>>(static_cast<const unsigned short*>(X2.p),
                                                                 static_cast<unsigned short*>(X1.p), v, o, X2.Kp, 2);
    else
      k_swap_outer_rows<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(X2.p), static_cast<double*>(X1.p), v,
                                                       o, X2.Kp, 1);
  }

  // ---- pairs b <= c
  std::vector<int> hb, hc;
  for (int c = 0; c < v; ++c)
    for (int b = 0; b <= c; ++b) {
      hb.push_back(b);
      hc.push_back(c);
    }
  const int npair = static_cast<int>(hb.size());
  int* dpb = static_cast<int*>(tmp_alloc(npair * 4));
  int* dpc = static_cast<int*>(tmp_alloc(npair * 4));
  double* tpart = static_cast<double*>(tmp_alloc(static_cast<size_t>(npair) * v * 2 * 8));
  const long long slot_stride = v * ooo;
  const int P = static_cast<int>(std::max(1LL, std::min<long long>(npair, (1LL << 26) / slot_stride)));
  double* W = static_cast<double*>(tmp_alloc(static_cast<size_t>(P) * slot_stride * 8));
  double* dU = nullptr;
  if (nlo > 0) dU = const_cast<double*>(U);
  if (!dpb || !dpc || !tpart || !W) {
    cleanup();
    set_error("lnocc_triples: device allocation failed (W chunk)");
    return LNOCC_ENOMEM;
  }
  cudaMemcpyAsync(dpb, hb.data(), npair * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dpc, hc.data(), npair * 4, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);

  const int o2 = static_cast<int>(oo);
  for (int p0 = 0; p0 < npair; p0 += P) {
    const int np = std::min(P, npair - p0);
    for (int q = 0; q < np; ++q) {
      const int b = hb[p0 + q], c = hc[p0 + q];
      double* Wz = W + q * slot_stride;
      const int Ma = (b + 1) * o;        // rows (a <= b, p)
      const int Ma2 = (b + 1) * o2;      // rows (a <= b, p, q)
      const int xb = b * v * o, xc = c * v * o;  // row offsets of the y = b / y = c slices of X1, X2, T2x, T2y
      // G_i: rows (a,i), cols (k,j)  -> W[a][i][j][k]
      const OutMap Gi{Wz, ooo, oo, 1, o, o, o, 1.0, 0.0};
      OutMap Gi1 = Gi;
      Gi1.beta = 1.0;
      gemm_off(X1, xb, Tv, c * o2, Ma, o2, v, Gi, s, dstatus);
      gemm_off(X1, xc, TvT, b * o2, Ma, o2, v, Gi1, s, dstatus);
      gemm_off(T2x, xb, O1, c * o2, Ma, o2, o, Gi1, s, dstatus);
      gemm_off(T2x, xc, O1T, b * o2, Ma, o2, o, Gi1, s, dstatus);
      // G_j: rows (a,j), cols (k,i)
      const OutMap Gj{Wz, ooo, o, 1, oo, o, o, 1.0, 1.0};
      gemm_off(X2, xb, Tv, c * o2, Ma, o2, v, Gj, s, dstatus);
      gemm_off(T2y, xb, O1, c * o2, Ma, o2, o, Gj, s, dstatus);
      // G_k: rows (a,k), cols (j,i)
      const OutMap Gk{Wz, ooo, 1, o, oo, o, o, 1.0, 1.0};
      gemm_off(X2, xc, Tv, b * o2, Ma, o2, v, Gk, s, dstatus);
      gemm_off(T2y, xc, O1, b * o2, Ma, o2, o, Gk, s, dstatus);
      // G_4: rows (a,i,k), cols j ; G_6: rows (a,i,j), cols k
      const OutMap G4{Wz, oo, 1, 0, o, o, 1 << 30, 1.0, 1.0};
      const OutMap G6{Wz, oo, o, 0, 1, o, 1 << 30, 1.0, 1.0};
      gemm_off(Tv, 0, X1, xc + b * o, Ma2, o, v, G4, s, dstatus);
      gemm_off(O1, 0, T2x, xc + b * o, Ma2, o, o, G4, s, dstatus);
      gemm_off(Tv, 0, X1, xb + c * o, Ma2, o, v, G6, s, dstatus);
      gemm_off(O1, 0, T2x, xb + c * o, Ma2, o, o, G6, s, dstatus);
    }
    k_t_energy<<<dim3(v, np), 128, 0, s>>>(W, slot_stride, dpb, dpc, p0, o, v, eps, t1, ovov, dU, nlo, tpart);
  }
  k_t_finish<<<1, 1024, 0, s>>>(tpart, 1LL * npair * v, scal + 4);
  cudaMemcpyAsync(h_scal + 4, scal + 4, 16, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  const int st = check_device();
  if (e_full) *e_full = h_scal[4];
  if (e_frag) *e_frag = nlo > 0 ? h_scal[5] : 0.0;
  cleanup();
  if (st == LNOCC_OK && !std::isfinite(h_scal[4])) {
    set_error("non-finite (T) energy");
    return LNOCC_ENUMERIC;
  }
  return st;
}

}  // namespace lnocc
