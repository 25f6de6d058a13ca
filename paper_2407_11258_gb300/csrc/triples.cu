// LNO-(T): W and V intermediates of the supplementary Sec. S1 and the projected (T) pair energy of
// Eq. 16, summed as E^(F) = sum_alpha sum_ii' U_i,alpha E_ii',(T) U_i',alpha (Eq. 15).
//
// Loop structure ("virtual-outer"): for each pair b <= c and every a <= b the block
// W^{abc}_{ijk} over all occupied (i,j,k) is formed. Because W and V are invariant under a
// simultaneous permutation of (i,a), (j,b), (k,c), the block of the sorted triple a<=b<=c yields
// W^{pi(abc)} for every ordering pi by permuting (i,j,k), so each distinct virtual triple is formed
// once (2 o^3 v^4 + 2 o^4 v^3 flops in the contractions), and the projection over (i, i') stays
// local to the block.
//
// Within a slab of fixed b (virtual c >= b in chunks of up to 768 MB of W, a <= b) each of the six
// permutation terms is one GEMM over K = v + o: the d-part (K = v) and the l-part (K = o) operands are
// packed side by side along K (listed per fixed (b, c); rows run over a and one or two occupied indices):
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
#include <mutex>
#include <string>
#include <vector>

#include "ccsd_kernels.h"
#include "fragment.h"
#include "internal.h"

namespace lnocc {

static inline Ax A_(int n, long long s) { return Ax{n, s}; }

namespace {

// Position permutations of three slots, listed as (p1, p2, p3) in 0-based slots.
__constant__ int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Compensated FP32 summation for the FP32 block-energy kernels: a running sum s and the sum c of the
// rounding errors of its additions, each error obtained exactly by Knuth's TwoSum (TAOCP vol. 2,
// 4.2.2), cascaded as in the Sum2 algorithm of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 1955
// (2005)). s + c is as accurate as a sum formed in twice the FP32 precision (error about
// u|S| + (n u)^2 sum|x_i|, u = 2^-24), which keeps the block partials as accurate as the FP64 sums
// they replace without FP64-pipe work (the part's FP64 rate is a small fraction of its FP32 rate).
// The _rn intrinsics keep the compiler from fusing or reordering the error terms.
struct CSum {
  float s, c;
};
__device__ __forceinline__ void csum_add(CSum& a, float x) {
  const float t = __fadd_rn(a.s, x);
  const float bp = __fsub_rn(t, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  a.s = t;
  a.c = __fadd_rn(a.c, err);
}
__device__ __forceinline__ void csum_merge(CSum& a, const CSum& b) {
  csum_add(a, b.s);
  a.c = __fadd_rn(a.c, b.c);
}
// Block result {canonical, projected} of two compensated sums: warp trees, then warp 0 over the warps'
// sums, in a fixed order; thread 0 writes -(s + c) / 3 in FP64 (the 1/3 of the six orderings).
__device__ __forceinline__ void csum_block_out(CSum e0, CSum e1, double* out, long long blk_id) {
  __shared__ float4 sh[32];
  for (int off = 16; off > 0; off >>= 1) {
    CSum o0, o1;
    o0.s = __shfl_xor_sync(0xffffffffu, e0.s, off);
    o0.c = __shfl_xor_sync(0xffffffffu, e0.c, off);
    o1.s = __shfl_xor_sync(0xffffffffu, e1.s, off);
    o1.c = __shfl_xor_sync(0xffffffffu, e1.c, off);
    csum_merge(e0, o0);
    csum_merge(e1, o1);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) sh[w] = make_float4(e0.s, e0.c, e1.s, e1.c);
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum a0{0.f, 0.f}, a1{0.f, 0.f};
    for (int q = 0; q < static_cast<int>(blockDim.x / 32); ++q) {
      const float4 t = sh[q];
      csum_merge(a0, CSum{t.x, t.y});
      csum_merge(a1, CSum{t.z, t.w});
    }
    out[2 * blk_id] = -(static_cast<double>(a0.s) + static_cast<double>(a0.c)) / 3.0;
    out[2 * blk_id + 1] = -(static_cast<double>(a1.s) + static_cast<double>(a1.c)) / 3.0;
  }
}

// Block energy, generic form: one CTA per (pair, a) with a <= b; threads over (j, k). Any nocc and any
// number of LOs: the projected i-sums are kept for up to kLoChunk LOs at a time, and for more LOs the
// i loop is repeated per chunk (the canonical part is accumulated in the first pass only). W is FP64
// (plain path) or FP32 (mixed path); the arithmetic here is FP64 on both.
// W: [slot][a][i][k][j]; out: per block {canonical, projected} partials (FP64).
constexpr int kLoChunk = 8;

template <typename TW>
__global__ void k_t_energy(const TW* __restrict__ W, long long slot_stride, int b, int c0, int o, int v,
                           const double* __restrict__ eps, const double* __restrict__ t1,
                           const double* __restrict__ ovov, const double* __restrict__ U, int nlo,
                           double* __restrict__ out) {
  const int slot = blockIdx.y;
  const int a = blockIdx.x;
  const int c = c0 + slot;
  const long long oblk = 1LL * o * o * o;
  const long long blk_id = static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
  const TW* Wb = W + slot * slot_stride + a * oblk;
  const int x[3] = {a, b, c};
  const double ex = eps[o + a] + eps[o + b] + eps[o + c];
  const long long ov = 1LL * o * v;
  auto widx = [&](int y0, int y1, int y2) { return (1LL * y0 * o + y2) * o + y1; };  // W stored [a][i][k][j]
  // w and v of the block at occupied (y0, y1, y2)
  auto wv = [&](int y0, int y1, int y2, double& w, double& vv) {
    const double Wv = static_cast<double>(Wb[widx(y0, y1, y2)]);
    const double Vv = Wv + ovov[(1LL * y0 * v + a) * ov + 1LL * y1 * v + b] * t1[y2 * v + c] +
                      ovov[(1LL * y0 * v + a) * ov + 1LL * y2 * v + c] * t1[y1 * v + b] +
                      ovov[(1LL * y1 * v + b) * ov + 1LL * y2 * v + c] * t1[y0 * v + a];
    const double s = 1.0 / sqrt(ex - eps[y0] - eps[y1] - eps[y2]);
    w = Wv * s;
    vv = Vv * s;
  };
  double e_can = 0.0, e_frag = 0.0;
  const int nchunk = nlo > 0 ? (nlo + kLoChunk - 1) / kLoChunk : 1;
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
      for (int ch = 0; ch < nchunk; ++ch) {
        const int al0 = ch * kLoChunk;
        const int nal = nlo > 0 ? min(kLoChunk, nlo - al0) : 0;
        double zu[kLoChunk], yu[kLoChunk];
#pragma unroll
        for (int q = 0; q < kLoChunk; ++q) zu[q] = yu[q] = 0.0;
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
          if (ch == 0) e_can += z * yy;
#pragma unroll
          for (int q = 0; q < kLoChunk; ++q) {
            if (q < nal) {
              const double u = U[i * nlo + al0 + q];
              zu[q] += u * z;
              yu[q] += u * yy;
            }
          }
        }
#pragma unroll
        for (int q = 0; q < kLoChunk; ++q)
          if (q < nal) e_frag += zu[q] * yu[q];
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

// Staged block energy: one CTA per (pair, a), a <= b. w = W s and v = (W + disconnected) s are formed once
// per block in shared memory (Real = float on the mixed path, double on the FP64 path), with
// s = 1/sqrt(-Delta) and -Delta = d_i + d_j + d_k, d_m = (e_a + e_b + e_c)/3 - e_m > 0 evaluated in FP64
// (a sum of positive terms: no cancellation when it is rounded to Real). Threads then run over (j, k)
// and every distinct ordering of (a, b, c); the i-sums are accumulated in Real and the block sum in FP64.
// VFLY: only w is staged and v = w + disc s is recomputed where it is read (the slices, t1 columns and
// d_m are in shared memory already); half the shared memory, for blocks too large to stage both.
// Launched for the FP64 path; the mixed path runs k_t_energy_f32 (w and v staged) or k_t_energy_vfly
// (w staged) below.
template <typename TW, typename Real, int NLO, bool VFLY>
__global__ void k_t_energy_staged(const TW* __restrict__ W, long long slot_stride, int b, int c0, int o, int v,
                                  const double* __restrict__ eps, const double* __restrict__ t1,
                                  const double* __restrict__ ovov, const double* __restrict__ U, int nlo_rt,
                                  double* __restrict__ out) {
  // NLO: number of fragment LO columns of U, fixed at compile time (0 = canonical energy only);
  // U is zero-padded to NLO columns by the host, so nlo_rt (the caller's count) is not needed here
  (void)nlo_rt;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int slot = blockIdx.y, a = blockIdx.x;
  const int c = c0 + slot;
  const long long blk_id = static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
  const int o2 = o * o, o3 = o2 * o;
  // shared-memory blocks w and v use padded strides (S0 = o(o+1)+1, S1 = o+1, S2 = 1, all odd for
  // even o) so that the permuted reads of the orderings below spread over the banks
  const int S1 = o + 1, S0 = o * S1 + 1;
  const int blk = o * S0;
  Real* sw = reinterpret_cast<Real*>(smraw);
  Real* sv = sw + blk;
  const int P1 = o + 1, o2p = o * P1;  // o x o slices padded to odd row stride
  Real* Sab = VFLY ? sv : sv + blk;  // (y0 a|y1 b)
  Real* Sac = Sab + o2p;    // (y0 a|y2 c)
  Real* Sbc = Sac + o2p;    // (y1 b|y2 c)
  Real* ta = Sbc + o2p;     // t1[y][a], t1[y][b], t1[y][c]
  Real* tb = ta + o;
  Real* tc = tb + o;
  Real* dm = tc + o;        // d_m
  Real* Us = dm + o;        // U[i][alpha]
  const long long ov = 1LL * o * v;
  const double ex3 = (eps[o + a] + eps[o + b] + eps[o + c]) / 3.0;
  for (int idx = threadIdx.x; idx < o2; idx += blockDim.x) {
    const int p = idx / o, q = idx % o;
    Sab[p * P1 + q] = static_cast<Real>(ovov[(1LL * p * v + a) * ov + 1LL * q * v + b]);
    Sac[p * P1 + q] = static_cast<Real>(ovov[(1LL * p * v + a) * ov + 1LL * q * v + c]);
    Sbc[p * P1 + q] = static_cast<Real>(ovov[(1LL * p * v + b) * ov + 1LL * q * v + c]);
  }
  for (int y = threadIdx.x; y < o; y += blockDim.x) {
    ta[y] = static_cast<Real>(t1[y * v + a]);
    tb[y] = static_cast<Real>(t1[y * v + b]);
    tc[y] = static_cast<Real>(t1[y * v + c]);
    dm[y] = static_cast<Real>(ex3 - eps[y]);
  }
  for (int idx = threadIdx.x; idx < o * NLO; idx += blockDim.x) Us[idx] = static_cast<Real>(U[idx]);
  __syncthreads();
  const TW* Wb = W + slot * slot_stride + static_cast<long long>(a) * o3;
  // W is stored [i][k][j] (j fastest): read it in that order (coalesced)
  // (y0, y2, y1) of idx advance by the fixed stride blockDim.x with carries: no division in the loop
  const int st = blockDim.x, d1 = st % o, d2 = (st / o) % o, d0 = st / o2;
  int y1 = threadIdx.x % o, y2 = (threadIdx.x / o) % o, y0 = threadIdx.x / o2;
  for (int idx = threadIdx.x; idx < o3; idx += st) {
    const Real Wv = static_cast<Real>(Wb[idx]);
    const Real disc = Sab[y0 * P1 + y1] * tc[y2] + Sac[y0 * P1 + y2] * tb[y1] + Sbc[y1 * P1 + y2] * ta[y0];
    const Real d = dm[y0] + dm[y1] + dm[y2];
    Real sc;
    if (sizeof(Real) == 4)
      sc = static_cast<Real>(rsqrtf(static_cast<float>(d)));
    else
      sc = static_cast<Real>(1.0 / sqrt(static_cast<double>(d)));
    const int sidx = y0 * S0 + y1 * S1 + y2;
    sw[sidx] = Wv * sc;
    if (!VFLY) sv[sidx] = (Wv + disc) * sc;
    y1 += d1;
    int cy = y1 >= o;
    y1 -= cy ? o : 0;
    y2 += d2 + cy;
    cy = y2 >= o;
    y2 -= cy ? o : 0;
    y0 += d0 + cy;
  }
  __syncthreads();
  // The six placements of (i, j, k) into the slots of W^{abc}_y: placement q puts i in slot PM[q][0],
  // j in PM[q][1], k in PM[q][2]. For ordering (p0, p1, p2) of the virtual labels, the four W values it
  // needs -- T, T o c, T o c^2 and the reversal -- are the placements (p0,p1,p2), (p1,p2,p0), (p2,p0,p1)
  // and (p2,p1,p0). Each thread loads the six w (and v) placements once per i and evaluates every
  // distinct ordering from registers. With the loops fully unrolled every index is a compile-time choice.
  constexpr int PM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int x0 = a, x1 = b, x2 = c;
  auto X = [&](int p) { return p == 0 ? x0 : (p == 1 ? x1 : x2); };
  auto SS = [&](int p) { return p == 0 ? S0 : (p == 1 ? S1 : 1); };
  bool act[6];  // orderings with distinct label sequences (equal labels repeat an ordering)
#pragma unroll
  for (int pi = 0; pi < 6; ++pi) {
    bool dup = false;
#pragma unroll
    for (int q = 0; q < pi; ++q)
      dup = dup || (X(PM[q][0]) == X(PM[pi][0]) && X(PM[q][1]) == X(PM[pi][1]) && X(PM[q][2]) == X(PM[pi][2]));
    act[pi] = !dup;
  }
  // per-thread partials in FP64: FP32 (Real = float) sums run over one (j, k) only (6 nocc terms)
  double r_can = 0, r_frag = 0;
  for (int jk = threadIdx.x; jk < o2; jk += blockDim.x) {
    const int j = jk / o, k = jk % o;
    int off[6], si[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      off[q] = j * SS(PM[q][1]) + k * SS(PM[q][2]);
      si[q] = SS(PM[q][0]);
    }
    Real acc = 0, zu[6][NLO > 0 ? NLO : 1], yu[6][NLO > 0 ? NLO : 1];
#pragma unroll
    for (int pi = 0; pi < 6; ++pi)
#pragma unroll
      for (int al = 0; al < NLO; ++al) zu[pi][al] = yu[pi][al] = 0;
    for (int i = 0; i < o; ++i) {
      Real wq[6], vq[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        wq[q] = sw[off[q]];
        if (!VFLY) {
          vq[q] = sv[off[q]];
        } else {
          // v = w + disc s at this placement (slices, t1 columns and d_m are staged)
          const int y0 = PM[q][0] == 0 ? i : (PM[q][1] == 0 ? j : k);
          const int y1 = PM[q][0] == 1 ? i : (PM[q][1] == 1 ? j : k);
          const int y2 = PM[q][0] == 2 ? i : (PM[q][1] == 2 ? j : k);
          const Real dd = Sab[y0 * P1 + y1] * tc[y2] + Sac[y0 * P1 + y2] * tb[y1] + Sbc[y1 * P1 + y2] * ta[y0];
          const Real d = dm[y0] + dm[y1] + dm[y2];
          Real sc;
          if (sizeof(Real) == 4)
            sc = static_cast<Real>(rsqrtf(static_cast<float>(d)));
          else
            sc = static_cast<Real>(1.0 / sqrt(static_cast<double>(d)));
          vq[q] = wq[q] + dd * sc;
        }
        off[q] += si[q];
      }
#pragma unroll
      for (int pi = 0; pi < 6; ++pi) {
        if (!act[pi]) continue;
        const int p0 = PM[pi][0], p1 = PM[pi][1], p2 = PM[pi][2];
        auto idx = [&](int s0, int s1) {  // placement index of the tuple (s0, s1, 3 - s0 - s1)
          return s0 == 0 ? (s1 == 1 ? 0 : 1) : (s0 == 1 ? (s1 == 0 ? 2 : 3) : (s1 == 0 ? 4 : 5));
        };
        const Real z = 4 * wq[idx(p0, p1)] + wq[idx(p1, p2)] + wq[idx(p2, p0)];
        const Real y = vq[idx(p0, p1)] - vq[idx(p2, p1)];
        acc += z * y;
#pragma unroll
        for (int al = 0; al < NLO; ++al) {
          zu[pi][al] += Us[i * NLO + al] * z;
          yu[pi][al] += Us[i * NLO + al] * y;
        }
      }
    }
    r_can += acc;
#pragma unroll
    for (int pi = 0; pi < 6; ++pi)
#pragma unroll
      for (int al = 0; al < NLO; ++al) r_frag += zu[pi][al] * yu[pi][al];
  }
  double e_can = static_cast<double>(r_can), e_frag = static_cast<double>(r_frag);
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

// Block energy of the mixed path with w and v both staged (FP32 W): the same quantities and orderings
// as k_t_energy_staged with Real = float and both w and v staged (the form it replaced on this path),
// with the data movement reworked and the partials across (j, k) summed in compensated FP32 (CSum)
// instead of FP64:
//  * the staging pass issues eight independent W loads per thread before it uses any of them;
//  * w and v of one (y0, y1, y2) sit side by side, so a placement is one 8-byte shared-memory load;
//  * the projected i-sums of z and y for one LO form a pair updated by one packed FP32 FMA, with
//    U[i][alpha] duplicated into both halves of a pair in shared memory.
// OC > 0: compiled for nocc = OC (constant strides and trip counts); OC = 0: any nocc (o_in).
template <int NLO, int OC>
__global__ void __launch_bounds__(256, NLO <= 2 ? 4 : 2)
    k_t_energy_f32(const float* __restrict__ W, long long slot_stride, int b, int c0, int o_in, int v,
                   const double* __restrict__ eps, const double* __restrict__ t1, const float* __restrict__ ovT,
                   const double* __restrict__ U, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int o = OC > 0 ? OC : o_in;
  const int slot = blockIdx.y, a = blockIdx.x;
  const int c = c0 + slot;
  const long long blk_id = static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
  const int o2 = o * o, o3 = o2 * o;
  const int S1 = o + 1, S0 = o * S1 + 1;  // padded strides of the staged block (odd for even o)
  const int blk = o * S0;
  float2* swv = reinterpret_cast<float2*>(smraw);  // (w, v) at y0 * S0 + y1 * S1 + y2
  float* fs = reinterpret_cast<float*>(smraw) + 2 * blk;
  const int P1 = o + 1, o2p = o * P1;
  float* Sab = fs;  // (y0 a|y1 b)
  float* Sac = Sab + o2p;
  float* Sbc = Sac + o2p;
  float* ta = Sbc + o2p;
  float* tb = ta + o;
  float* tc = tb + o;
  float* dm = tc + o;
  // U pairs (U[i][al], U[i][al]), 16-byte aligned for 128-bit loads
  const int uoff = (2 * blk + 3 * o2p + 4 * o + 3) & ~3;
  float* U2 = reinterpret_cast<float*>(smraw) + uoff;
  // (pa|qb) etc. from the FP32 copy ovT[x][y][p][q] = (px|qy): o^2 consecutive floats per slice
  const float* oab = ovT + (1LL * a * v + b) * o2;
  const float* oac = ovT + (1LL * a * v + c) * o2;
  const float* obc = ovT + (1LL * b * v + c) * o2;
  for (int idx = threadIdx.x; idx < o2; idx += blockDim.x) {
    const int p = idx / o, q = idx % o;
    Sab[p * P1 + q] = oab[idx];
    Sac[p * P1 + q] = oac[idx];
    Sbc[p * P1 + q] = obc[idx];
  }
  for (int y = threadIdx.x; y < o; y += blockDim.x) {
    const double ex3 = (eps[o + a] + eps[o + b] + eps[o + c]) / 3.0;  // FP64 in these o threads only
    ta[y] = static_cast<float>(t1[y * v + a]);
    tb[y] = static_cast<float>(t1[y * v + b]);
    tc[y] = static_cast<float>(t1[y * v + c]);
    dm[y] = static_cast<float>(ex3 - eps[y]);
  }
  for (int idx = threadIdx.x; idx < o * NLO; idx += blockDim.x) {
    const float u = static_cast<float>(U[idx]);
    U2[2 * idx] = u;
    U2[2 * idx + 1] = u;
  }
  __syncthreads();
  const float* Wb = W + slot * slot_stride + static_cast<long long>(a) * o3;
  // W is stored [i][k][j] (j fastest). Each thread owns pairs (j, k) = (y1, y2) (consecutive threads:
  // consecutive j, so every load instruction reads a contiguous row of W) and walks i = y0 with eight
  // loads in flight; the terms that depend on (j, k) only (t1 of b and c, (bj|ck), d_j + d_k) stay in
  // registers across the walk.
  constexpr int kLoads = 8;
  for (int jk = threadIdx.x; jk < o2; jk += blockDim.x) {
    const int y1 = jk % o, y2 = jk / o;
    const float tcv = tc[y2], tbv = tb[y1], sbc = Sbc[y1 * P1 + y2], d12 = dm[y1] + dm[y2];
    const float* wp = Wb + jk;
    float2* dst = swv + y1 * S1 + y2;
    for (int i0 = 0; i0 < o; i0 += kLoads) {
      float wr[kLoads];
#pragma unroll
      for (int u = 0; u < kLoads; ++u) wr[u] = i0 + u < o ? wp[static_cast<long long>(i0 + u) * o2] : 0.f;
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const int y0 = i0 + u;
        if (y0 < o) {
          const float disc = Sab[y0 * P1 + y1] * tcv + Sac[y0 * P1 + y2] * tbv + sbc * ta[y0];
          const float sc = rsqrtf(dm[y0] + d12);
          dst[y0 * S0] = make_float2(wr[u] * sc, (wr[u] + disc) * sc);
        }
      }
    }
  }
  __syncthreads();
  // placements and orderings as in k_t_energy_staged
  constexpr int PM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int x0 = a, x1 = b, x2 = c;
  auto X = [&](int p) { return p == 0 ? x0 : (p == 1 ? x1 : x2); };
  auto SS = [&](int p) { return p == 0 ? S0 : (p == 1 ? S1 : 1); };
  const bool distinct = a < b && b < c;
  bool act[6];
#pragma unroll
  for (int pi = 0; pi < 6; ++pi) {
    bool dup = false;
    if (!distinct) {
#pragma unroll
      for (int q = 0; q < pi; ++q)
        dup = dup || (X(PM[q][0]) == X(PM[pi][0]) && X(PM[q][1]) == X(PM[pi][1]) && X(PM[q][2]) == X(PM[pi][2]));
    }
    act[pi] = !dup;
  }
  constexpr int NL = NLO > 0 ? NLO : 1;
  // FP32 sums run over one (j, k) only; partials across (j, k) in compensated FP32 (CSum)
  CSum r_can{0.f, 0.f}, r_frag{0.f, 0.f};
  for (int jk = threadIdx.x; jk < o2; jk += blockDim.x) {
    const int j = jk / o, k = jk % o;
    int off[6], si[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      off[q] = j * SS(PM[q][1]) + k * SS(PM[q][2]);
      si[q] = SS(PM[q][0]);
    }
    float acc = 0.f;
    if (distinct) {
      // a < b < c: all six orderings are distinct. With w_q, v_q the six placements (q = 0, 3, 4 the
      // cyclic ones, 1, 2, 5 the others), ordering q has z_q = 3 w_q + S (S the sum of w over q's class)
      // and y_q = v_q - v_r with r = rev(q) the placement of the reversed slots (0<->5, 3<->1, 4<->2,
      // always of the other class), so y_r = -y_q. Each pair then contributes
      // (z_q - z_r) y_q = (3 (w_q - w_r) + S_cyc - S_oth) y_q to the canonical sum, and, since the
      // i-sums of y_r are minus those of y_q, (sum_i U (z_q - z_r)) (sum_i U y_q) to the projected one:
      // three products per (i, j, k) instead of six, the same quantities.
      float2 zp[3][NL];  // (sum_i U (z_q - z_r), sum_i U y_q) per pair and LO
#pragma unroll
      for (int h = 0; h < 3; ++h)
#pragma unroll
        for (int al = 0; al < NL; ++al) zp[h][al] = make_float2(0.f, 0.f);
#pragma unroll (OC > 0 ? OC : 2)
      for (int i = 0; i < o; ++i) {
        float2 p[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          p[q] = swv[off[q]];
          off[q] += si[q];
        }
        const float dS = (p[0].x + p[3].x + p[4].x) - (p[1].x + p[2].x + p[5].x);
        const float2 d0 = make_float2(fmaf(3.f, p[0].x - p[5].x, dS), p[0].y - p[5].y);
        const float2 d1 = make_float2(fmaf(3.f, p[3].x - p[1].x, dS), p[3].y - p[1].y);
        const float2 d2 = make_float2(fmaf(3.f, p[4].x - p[2].x, dS), p[4].y - p[2].y);
        acc = fmaf(d0.x, d0.y, acc);
        acc = fmaf(d1.x, d1.y, acc);
        acc = fmaf(d2.x, d2.y, acc);
        if constexpr (NLO > 0) {
          float2 u2[NL];
          if constexpr (NLO == 1) {
            u2[0] = reinterpret_cast<const float2*>(U2)[i];
          } else {
#pragma unroll
            for (int h = 0; h < NLO / 2; ++h) {
              const float4 t = reinterpret_cast<const float4*>(U2)[i * (NLO / 2) + h];
              u2[2 * h] = make_float2(t.x, t.y);
              u2[2 * h + 1] = make_float2(t.z, t.w);
            }
          }
#pragma unroll
          for (int al = 0; al < NLO; ++al) {
            zp[0][al] = __ffma2_rn(u2[al], d0, zp[0][al]);
            zp[1][al] = __ffma2_rn(u2[al], d1, zp[1][al]);
            zp[2][al] = __ffma2_rn(u2[al], d2, zp[2][al]);
          }
        }
      }
      csum_add(r_can, acc);
      float f = 0.f;
#pragma unroll
      for (int h = 0; h < 3; ++h)
#pragma unroll
        for (int al = 0; al < NLO; ++al) f += zp[h][al].x * zp[h][al].y;
      csum_add(r_frag, f);
      continue;
    }
    float2 zy[6][NL];  // (sum_i U z, sum_i U y) per ordering and LO
#pragma unroll
    for (int pi = 0; pi < 6; ++pi)
#pragma unroll
      for (int al = 0; al < NL; ++al) zy[pi][al] = make_float2(0.f, 0.f);
    for (int i = 0; i < o; ++i) {
      float2 p[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        p[q] = swv[off[q]];
        off[q] += si[q];
      }
      float2 u2[NL];
      if constexpr (NLO == 1) {
        u2[0] = reinterpret_cast<const float2*>(U2)[i];
      } else if constexpr (NLO > 1) {
#pragma unroll
        for (int h = 0; h < NLO / 2; ++h) {
          const float4 t = reinterpret_cast<const float4*>(U2)[i * (NLO / 2) + h];
          u2[2 * h] = make_float2(t.x, t.y);
          u2[2 * h + 1] = make_float2(t.z, t.w);
        }
      }
#pragma unroll
      for (int pi = 0; pi < 6; ++pi) {
        if (!act[pi]) continue;
        const int p0 = PM[pi][0], p1 = PM[pi][1], p2 = PM[pi][2];
        auto idx = [&](int s0, int s1) {
          return s0 == 0 ? (s1 == 1 ? 0 : 1) : (s0 == 1 ? (s1 == 0 ? 2 : 3) : (s1 == 0 ? 4 : 5));
        };
        const float z = 4 * p[idx(p0, p1)].x + p[idx(p1, p2)].x + p[idx(p2, p0)].x;
        const float y = p[idx(p0, p1)].y - p[idx(p2, p1)].y;
        acc += z * y;
        const float2 zyv = make_float2(z, y);
#pragma unroll
        for (int al = 0; al < NLO; ++al) zy[pi][al] = __ffma2_rn(u2[al], zyv, zy[pi][al]);
      }
    }
    csum_add(r_can, acc);
    float f = 0.f;
#pragma unroll
    for (int pi = 0; pi < 6; ++pi)
#pragma unroll
      for (int al = 0; al < NLO; ++al) f += zy[pi][al].x * zy[pi][al].y;
    csum_add(r_frag, f);
  }
  csum_block_out(r_can, r_frag, out, blk_id);
}

// Block energy of the mixed path when only w fits in shared memory (nocc 29..35 at 200 KB): w = W s is
// staged, v = w + disc s is formed where it is read. s depends on the unordered triple (i, j, k), so one
// rsqrt per (i, j, k) serves all six placements; of the fifteen slice / t1 values the six placements'
// disconnected terms need at fixed (j, k), the ones that do not involve i stay in registers across the
// i walk. Orderings are paired as in k_t_energy_f32 when a < b < c. 512 threads per block (two (j, k)
// pairs per thread at nocc 32) with NLO <= 2, 256 above.
template <int NLO>
__global__ void __launch_bounds__(NLO <= 2 ? 512 : 256, 1)
    k_t_energy_vfly(const float* __restrict__ W, long long slot_stride, int b, int c0, int o, int v,
                    const double* __restrict__ eps, const double* __restrict__ t1, const float* __restrict__ ovT,
                    const double* __restrict__ U, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int slot = blockIdx.y, a = blockIdx.x;
  const int c = c0 + slot;
  const long long blk_id = static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x;
  const int o2 = o * o, o3 = o2 * o;
  const int S1 = o + 1, S0 = o * S1 + 1;
  const int blk = o * S0;
  float* sw = reinterpret_cast<float*>(smraw);  // w at y0 * S0 + y1 * S1 + y2
  float* fs = sw + blk;
  const int P1 = o + 1, o2p = o * P1;
  float* Sab = fs;  // (y0 a|y1 b)
  float* Sac = Sab + o2p;
  float* Sbc = Sac + o2p;
  float* ta = Sbc + o2p;
  float* tb = ta + o;
  float* tc = tb + o;
  float* dm = tc + o;
  const int uoff = (blk + 3 * o2p + 4 * o + 3) & ~3;
  float* U2 = sw + uoff;  // (U[i][al], U[i][al]) pairs
  const float* oab = ovT + (1LL * a * v + b) * o2;
  const float* oac = ovT + (1LL * a * v + c) * o2;
  const float* obc = ovT + (1LL * b * v + c) * o2;
  for (int idx = threadIdx.x; idx < o2; idx += blockDim.x) {
    const int p = idx / o, q = idx % o;
    Sab[p * P1 + q] = oab[idx];
    Sac[p * P1 + q] = oac[idx];
    Sbc[p * P1 + q] = obc[idx];
  }
  for (int y = threadIdx.x; y < o; y += blockDim.x) {
    const double ex3 = (eps[o + a] + eps[o + b] + eps[o + c]) / 3.0;  // FP64 in these o threads only
    ta[y] = static_cast<float>(t1[y * v + a]);
    tb[y] = static_cast<float>(t1[y * v + b]);
    tc[y] = static_cast<float>(t1[y * v + c]);
    dm[y] = static_cast<float>(ex3 - eps[y]);
  }
  for (int idx = threadIdx.x; idx < o * NLO; idx += blockDim.x) {
    const float u = static_cast<float>(U[idx]);
    U2[2 * idx] = u;
    U2[2 * idx + 1] = u;
  }
  __syncthreads();
  const float* Wb = W + slot * slot_stride + static_cast<long long>(a) * o3;
  // staging: thread-owned (j, k) pairs walking i, as in k_t_energy_f32 (w only)
  constexpr int kLoads = 8;
  for (int jk = threadIdx.x; jk < o2; jk += blockDim.x) {
    const int y1 = jk % o, y2 = jk / o;
    const float d12 = dm[y1] + dm[y2];
    const float* wp = Wb + jk;
    float* dst = sw + y1 * S1 + y2;
    for (int i0 = 0; i0 < o; i0 += kLoads) {
      float wr[kLoads];
#pragma unroll
      for (int u = 0; u < kLoads; ++u) wr[u] = i0 + u < o ? wp[static_cast<long long>(i0 + u) * o2] : 0.f;
#pragma unroll
      for (int u = 0; u < kLoads; ++u)
        if (i0 + u < o) dst[(i0 + u) * S0] = wr[u] * rsqrtf(dm[i0 + u] + d12);
    }
  }
  __syncthreads();
  constexpr int PM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int x0 = a, x1 = b, x2 = c;
  auto X = [&](int p) { return p == 0 ? x0 : (p == 1 ? x1 : x2); };
  auto SS = [&](int p) { return p == 0 ? S0 : (p == 1 ? S1 : 1); };
  const bool distinct = a < b && b < c;
  bool act[6];
#pragma unroll
  for (int pi = 0; pi < 6; ++pi) {
    bool dup = false;
    if (!distinct) {
#pragma unroll
      for (int q = 0; q < pi; ++q)
        dup = dup || (X(PM[q][0]) == X(PM[pi][0]) && X(PM[q][1]) == X(PM[pi][1]) && X(PM[q][2]) == X(PM[pi][2]));
    }
    act[pi] = !dup;
  }
  constexpr int NL = NLO > 0 ? NLO : 1;
  // FP32 sums over one (j, k); partials across (j, k) in compensated FP32 (CSum)
  CSum r_can{0.f, 0.f}, r_frag{0.f, 0.f};
  for (int jk = threadIdx.x; jk < o2; jk += blockDim.x) {
    const int j = jk / o, k = jk % o;
    int off[6], si[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      off[q] = j * SS(PM[q][1]) + k * SS(PM[q][2]);
      si[q] = SS(PM[q][0]);
    }
    // (j, k)-only factors of the disconnected terms d(y0,y1,y2) = Sab[y0][y1] tc[y2] + Sac[y0][y2] tb[y1]
    // + Sbc[y1][y2] ta[y0] of the placements (i,j,k), (i,k,j), (j,i,k), (k,i,j), (j,k,i), (k,j,i)
    const float sbc_jk = Sbc[j * P1 + k], sbc_kj = Sbc[k * P1 + j], sac_jk = Sac[j * P1 + k],
                sac_kj = Sac[k * P1 + j], sab_jk = Sab[j * P1 + k], sab_kj = Sab[k * P1 + j];
    const float taj = ta[j], tak = ta[k], tbj = tb[j], tbk = tb[k], tcj = tc[j], tck = tc[k];
    const float djk = dm[j] + dm[k];
    float acc = 0.f;
    float2 zy[6][NL];
#pragma unroll
    for (int h = 0; h < 6; ++h)
#pragma unroll
      for (int al = 0; al < NL; ++al) zy[h][al] = make_float2(0.f, 0.f);
    for (int i = 0; i < o; ++i) {
      float w[6], vv[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        w[q] = sw[off[q]];
        off[q] += si[q];
      }
      const float s = rsqrtf(dm[i] + djk);
      const float sab_ij = Sab[i * P1 + j], sab_ji = Sab[j * P1 + i], sab_ik = Sab[i * P1 + k],
                  sab_ki = Sab[k * P1 + i];
      const float sac_ij = Sac[i * P1 + j], sac_ji = Sac[j * P1 + i], sac_ik = Sac[i * P1 + k],
                  sac_ki = Sac[k * P1 + i];
      const float sbc_ij = Sbc[i * P1 + j], sbc_ji = Sbc[j * P1 + i], sbc_ik = Sbc[i * P1 + k],
                  sbc_ki = Sbc[k * P1 + i];
      const float tai = ta[i], tbi = tb[i], tci = tc[i];
      vv[0] = w[0] + (sab_ij * tck + sac_ik * tbj + sbc_jk * tai) * s;  // (i, j, k)
      vv[1] = w[1] + (sab_ik * tcj + sac_ij * tbk + sbc_kj * tai) * s;  // (i, k, j)
      vv[2] = w[2] + (sab_ji * tck + sac_jk * tbi + sbc_ik * taj) * s;  // (j, i, k)
      vv[3] = w[3] + (sab_ki * tcj + sac_kj * tbi + sbc_ij * tak) * s;  // (k, i, j)
      vv[4] = w[4] + (sab_jk * tci + sac_ji * tbk + sbc_ki * taj) * s;  // (j, k, i)
      vv[5] = w[5] + (sab_kj * tci + sac_ki * tbj + sbc_ji * tak) * s;  // (k, j, i)
      float2 u2[NL];
      if constexpr (NLO == 1) {
        u2[0] = reinterpret_cast<const float2*>(U2)[i];
      } else if constexpr (NLO > 1) {
#pragma unroll
        for (int h = 0; h < NLO / 2; ++h) {
          const float4 t = reinterpret_cast<const float4*>(U2)[i * (NLO / 2) + h];
          u2[2 * h] = make_float2(t.x, t.y);
          u2[2 * h + 1] = make_float2(t.z, t.w);
        }
      }
      if (distinct) {
        // pairs (0, 5), (3, 1), (4, 2): (z_q - z_r, y_q), see k_t_energy_f32
        const float dS = (w[0] + w[3] + w[4]) - (w[1] + w[2] + w[5]);
        const float2 d0 = make_float2(fmaf(3.f, w[0] - w[5], dS), vv[0] - vv[5]);
        const float2 d1 = make_float2(fmaf(3.f, w[3] - w[1], dS), vv[3] - vv[1]);
        const float2 d2 = make_float2(fmaf(3.f, w[4] - w[2], dS), vv[4] - vv[2]);
        acc = fmaf(d0.x, d0.y, acc);
        acc = fmaf(d1.x, d1.y, acc);
        acc = fmaf(d2.x, d2.y, acc);
#pragma unroll
        for (int al = 0; al < NLO; ++al) {
          zy[0][al] = __ffma2_rn(u2[al], d0, zy[0][al]);
          zy[1][al] = __ffma2_rn(u2[al], d1, zy[1][al]);
          zy[2][al] = __ffma2_rn(u2[al], d2, zy[2][al]);
        }
      } else {
#pragma unroll
        for (int pi = 0; pi < 6; ++pi) {
          if (!act[pi]) continue;
          const int p0 = PM[pi][0], p1 = PM[pi][1], p2 = PM[pi][2];
          auto idx = [&](int s0, int s1) {
            return s0 == 0 ? (s1 == 1 ? 0 : 1) : (s0 == 1 ? (s1 == 0 ? 2 : 3) : (s1 == 0 ? 4 : 5));
          };
          const float z = 4 * w[idx(p0, p1)] + w[idx(p1, p2)] + w[idx(p2, p0)];
          const float y = vv[idx(p0, p1)] - vv[idx(p2, p1)];
          acc += z * y;
          const float2 zyv = make_float2(z, y);
#pragma unroll
          for (int al = 0; al < NLO; ++al) zy[pi][al] = __ffma2_rn(u2[al], zyv, zy[pi][al]);
        }
      }
    }
    csum_add(r_can, acc);
    float f = 0.f;
#pragma unroll
    for (int pi = 0; pi < 6; ++pi)
#pragma unroll
      for (int al = 0; al < NLO; ++al) f += zy[pi][al].x * zy[pi][al].y;
    csum_add(r_frag, f);
  }
  csum_block_out(r_can, r_frag, out, blk_id);
}

// Per-c tables of the batched (T) terms, one entry per (b, c >= b) in b-major order (the order of the
// chunk plan: entry (b, c) at b v - b (b - 1) / 2 + c - b). For W chunks of ncmax(b) = max(1, welems /
// ((b + 1) o^3)) values of c, c sits at position q = (c - b) mod ncmax(b) of its chunk. bat: sigma5
// (rows (c, a, k) of XT2 against rows (b, i, j) of TOT); bat12: sigma1 (rows (b, a, i) of XT1 against rows
// (c, k, j) of TO) then sigma2 (rows (c, a, i) of XT1 against rows (b, k, j) of TOT) into one accumulator.
__global__ void k_batch_tables(int o, int v, long long welems, BatchEntry* __restrict__ bat,
                               BatchEntry* __restrict__ bat12) {
  const long long oo = 1LL * o * o, ooo = oo * o;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < v; b += gridDim.x * blockDim.x) {
    const long long slab = 1LL * (b + 1) * ooo;
    const long long ncmax = welems / slab > 1 ? welems / slab : 1;
    const long long base = 1LL * b * v - 1LL * b * (b - 1) / 2;
    const int Ma = (b + 1) * o;
    const int brow = b * static_cast<int>(oo);
    for (int c = b; c < v; ++c) {
      const long long q = (c - b) % ncmax;
      const int arow = c * v * o;
      bat[base + c - b] = BatchEntry{arow, brow, Ma, arow, brow, 0, q * slab};
      bat12[base + c - b] = BatchEntry{b * v * o, c * static_cast<int>(oo), Ma, arow, brow, 0, q * slab};
    }
  }
}

// FP32 copy of (ia|jb) in the order the block energy reads it: ovT[a][b][i][j] = (ia|jb).
__global__ void k_ovov_t(const double* __restrict__ ovov, float* __restrict__ ovT, int o, int v) {
  const long long ov = 1LL * o * v, n = ov * ov, oo = 1LL * o * o;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < n;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(idx % v), j = static_cast<int>((idx / v) % o);
    const int a = static_cast<int>((idx / ov) % v), i = static_cast<int>(idx / (ov * v));
    ovT[(1LL * a * v + b) * oo + 1LL * i * o + j] = static_cast<float>(ovov[idx]);
  }
}

// Sum of the per-block partials in a fixed order: out[0] canonical, out[1] projected.
// Block g sums partials [g * chunk, min((g + 1) * chunk, nblk)) into out[2g], out[2g + 1] (the first of
// two fixed-order passes; one 1024-thread block alone took about 1.3 ms for the 2.3e6 block partials
// of a diamond-like call).
__global__ void k_t_finish_part(const double* part, long long nblk, long long chunk, double* out) {
  __shared__ double sh[2][32];
  double s0 = 0.0, s1 = 0.0;
  const long long i0 = blockIdx.x * chunk, i1 = min(nblk, i0 + chunk);
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
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
    out[2 * blockIdx.x] = a0;
    out[2 * blockIdx.x + 1] = a1;
  }
}

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

// dst row (y, a, i) <- src row (a, y, i) of a packed [planes][rows][Kp] operand (rows = v*v*o): one
// warp per row, 16-byte copies (a packed row is a multiple of 128 bytes)
__global__ void k_swap_outer_rows(const uint4* __restrict__ src, uint4* __restrict__ dst, int v, int o, int nvec,
                                  int planes) {
  const long long rows = 1LL * v * v * o;
  const int lane = threadIdx.x % 32;
  const long long nw = static_cast<long long>(gridDim.x) * blockDim.x / 32;
  for (long long w = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) / 32; w < rows * planes;
       w += nw) {
    const long long r = w % rows, pl = w / rows;
    const int i = static_cast<int>(r % o);
    const long long q = r / o;
    const int a = static_cast<int>(q % v);
    const long long y = q / v;
    const long long sr = (1LL * a * v + y) * o + i;
    const uint4* s = src + (pl * rows + sr) * nvec;
    uint4* d = dst + (pl * rows + r) * nvec;
    for (int e = lane; e < nvec; e += 32) d[e] = s[e];
  }
}

}  // namespace

// Device temporaries of one lnocc_triples call, in allocation order. Every size here is what the call
// asks for; with a caller workspace attached the call carves them from it in this order (256-byte
// aligned), so lnocc_workspace_bytes and the call agree by construction.
TriplesPlan triples_plan(int o, int v, int N, bool bf, int chunk_mb) {
  TriplesPlan p{};
  const long long oo = 1LL * o * o, vv = 1LL * v * v, ooo = oo * o;
  const size_t esz = bf ? 4 : 8;
  auto packed = [&](long long rows, int K) { return static_cast<size_t>(rows) * round_up(std::max(K, 1), 64) * esz; };
  const int Kt = v + o;
  p.xt = packed(vv * o, Kt);
  p.to = packed(v * oo, Kt);
  p.ovoo = static_cast<size_t>(ooo * v * 8);
  p.pbvv = packed(vv, N);
  p.bc = static_cast<int>(std::max(1LL, std::min<long long>(v, (1LL << 26) / (o * vv))));
  p.ovvv_chunk = static_cast<size_t>(p.bc) * o * vv * 8;
  // W chunk: up to chunk_mb (fewer, larger contraction launches measured faster than chunks that fit
  // L2), but never more than the largest slab (b + 1)(v - b) o^3 needs, and at least one c of a slab
  long long max_slab = 0;
  for (int bb = 0; bb < v; ++bb) max_slab = std::max(max_slab, 1LL * (bb + 1) * (v - bb) * ooo);
  const long long cmb = chunk_mb > 0 ? chunk_mb : 768;
  p.welems = std::max<long long>(std::min<long long>((cmb << 20) / static_cast<long long>(esz), max_slab), v * ooo);
  p.w = static_cast<size_t>(p.welems) * esz;
  p.nblk = 0;
  for (int b = 0; b < v; ++b) p.nblk += 1LL * (b + 1) * (v - b);
  p.tpart = static_cast<size_t>(p.nblk + 256) * 2 * 8;  // block partials, then 256 first-pass sums
  p.batch = sizeof(BatchEntry) * static_cast<size_t>(std::max(1LL, vv / 2 + v));  // one entry per (b, c >= b)
  p.u = static_cast<size_t>(o) * 8 * 8;  // U padded to at most 8 LOs
  p.ovt = bf ? static_cast<size_t>(vv * oo) * 4 : 0;  // FP32 (ia|jb) in block-energy order (mixed)
  auto al = [](size_t x) { return (std::max<size_t>(x, 256) + 255) / 256 * 256; };
  p.total = 2 * al(p.xt) + 2 * al(p.to) + al(p.ovoo) + al(p.pbvv) + al(p.ovvv_chunk) + al(p.w) + al(p.tpart) +
            2 * al(p.batch) + al(p.u) + (bf ? al(p.ovt) : 0);
  return p;
}

int Frag::triples(int nlo, const double* U, double* e_full, double* e_frag, double* e_dev, int* st_dev) {
  const long long oo = 1LL * o * o, vv = 1LL * v * v, ov = 1LL * o * v, ooo = oo * o;
  const bool bf = mixed;
  // device-output mode: enqueue only (no host synchronisation, no event timing, no allocation, no
  // tile timing), so that the call can be captured into a CUDA graph; the energies and the device
  // status word are copied to the caller's device memory at the end of the stream's work
  const bool dev_out = e_dev != nullptr;
  const TriplesPlan tp = triples_plan(o, v, N, bf, opts.triples_chunk_mb);
  if (ws_ext && ws_ext_bytes < tp.total) {
    set_error("lnocc_triples: attached workspace smaller than lnocc_workspace_bytes (" + std::to_string(tp.total) +
              " bytes)");
    return LNOCC_EINVAL;
  }
  if (dev_out && !ws_ext) {
    set_error("lnocc_triples_device: attach a workspace first (lnocc_frag_set_workspace)");
    return LNOCC_EINVAL;
  }
  struct TimingGuard {  // no tile timing (it synchronises and allocates) in device-output mode
    bool saved, active;
    explicit TimingGuard(bool on) : saved(autotune_timing_allowed()), active(on) {
      if (active) autotune_timing_allowed() = false;
    }
    ~TimingGuard() {
      if (active) autotune_timing_allowed() = saved;
    }
  } timing_guard(dev_out);
  cudaMemsetAsync(dstatus, 0, 16 * 4, s);
  const double* t1 = xcur;
  const double* t2 = xcur + ov;
  cudaEvent_t ev_call0 = nullptr, ev_call1 = nullptr;
  if (!dev_out) {
    cudaEventCreate(&ev_call0);
    cudaEventCreate(&ev_call1);
    cudaEventRecord(ev_call0, s);
  }
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gev;  // around each chunk's contraction launches

  // ---- operands (packed once per call)
  std::vector<void*> mine;
  size_t ws_used = 0;
  // temporaries: carved in plan order from the caller's workspace when one is attached (no device
  // allocation), else allocated in the fragment's memory mode and freed before returning
  auto tmp_alloc = [&](size_t bytes) -> void* {
    bytes = (std::max<size_t>(bytes, 256) + 255) / 256 * 256;
    if (ws_ext) {
      if (ws_used + bytes > ws_ext_bytes) return nullptr;
      void* p = static_cast<unsigned char*>(ws_ext) + ws_used;
      ws_used += bytes;
      return p;
    }
    void* p = dev_alloc(bytes);
    if (p) mine.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    if (!dev_out) cudaStreamSynchronize(s);
    for (void* p : mine) dev_free(p);
    if (ev_call0) cudaEventDestroy(ev_call0);
    if (ev_call1) cudaEventDestroy(ev_call1);
    ev_call0 = ev_call1 = nullptr;
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
  // Each (T) term is d-part (K = v) + l-part (K = o): the two operands of a side share one packed row
  // space, so they are packed side by side along K (columns [0, v) and [v, v + o)) and every term is a
  // single contraction of length v + o (no second, mostly padded, K segment).
  //   XT1[x][a][i] = [ (ai|xd) | -t_il^ax ],   XT2[c][a][k] = [ (kc|ad) | -t_kl^ca ]
  //   TO[z][r][q]  = [ t_rq^zd | (zr|ql) ],     TOT[z][k][j] = [ t_jk^zd | (zj|kl) ]
  const int Kt = v + o;
  Packed XT1 = mk(static_cast<int>(vv * o), Kt), XT2 = mk(static_cast<int>(vv * o), Kt);
  Packed TO = mk(static_cast<int>(v * oo), Kt), TOT = mk(static_cast<int>(v * oo), Kt);
  double* ovoo = static_cast<double*>(tmp_alloc(ooo * v * 8));
  const double* dU = nlo > 0 ? U : nullptr;
  if (!XT1.p || !XT2.p || !TO.p || !TOT.p || !ovoo) {
    cleanup();
    set_error("lnocc_triples: device allocation failed (operands)");
    return LNOCC_ENOMEM;
  }
  const int wl = XT1.Kp - v;  // width of the l-part columns, zero padding included
  // amplitudes: TO[z][r][q][d] = t_rq^zd, TOT[z][k][j][d] = t_jk^zd (columns [0, v))
  pack_cols(view(t2, A_(v, v), A_(o, o * vv), A_(o, vv), kOne, kOne, A_(v, 1)), TO, 0, 0, v, s);
  pack_cols(view(t2, A_(v, v), A_(o, vv), A_(o, o * vv), kOne, kOne, A_(v, 1)), TOT, 0, 0, v, s);
  // (kz|jl) -> TO[z][k][j][v + l] = (zk|jl), TOT[z][k][j][v + l] = (zj|kl)
  contract(view(Bov, kOne, kOne, A_(static_cast<int>(ov), 1), kOne, kOne, A_(N, ov)),
           view(Boo, kOne, kOne, A_(static_cast<int>(oo), 1), kOne, kOne, A_(N, oo)), out_rowmajor(ovoo, oo), true);
  pack_cols(view(ovoo, A_(v, oo), A_(o, v * oo), A_(o, o), kOne, kOne, A_(o, 1)), TO, 0, v, wl, s);
  pack_cols(view(ovoo, A_(v, oo), A_(o, o), A_(o, v * oo), kOne, kOne, A_(o, 1)), TOT, 0, v, wl, s);
  // (jb|ad) -> XT2[b][a][j][d], in chunks of b; XT1[y][a][i][d] = (ai|yd) = XT2[a][y][i][d]
  {
    Packed PBvv = mk(static_cast<int>(vv), N);
    if (!PBvv.p) {
      cleanup();
      set_error("lnocc_triples: device allocation failed (B_vv)");
      return LNOCC_ENOMEM;
    }
    pack(view(Bvv, kOne, kOne, A_(static_cast<int>(vv), 1), kOne, kOne, A_(N, vv)), PBvv, s);
    const int bc = tp.bc;
    double* tmp = static_cast<double*>(tmp_alloc(tp.ovvv_chunk));
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
      pack_cols(view(tmp, A_(nb, vv), A_(v, v), A_(o, nb * vv), kOne, kOne, A_(v, 1)), XT2, b0 * v * o, 0, v, s);
    }
    mixed = keep;
    const int planes = bf ? 2 : 1;
    const int nvec = XT2.Kp * (bf ? 2 : 8) / 16;
    const long long nrows = static_cast<long long>(XT2.rows) * planes;
    const int blocks = static_cast<int>(std::min<long long>((nrows + 7) / 8, 152LL * 16));
    count_launch();
    k_swap_outer_rows<<<blocks, 256, 0, s>>>(static_cast<const uint4*>(XT2.p), static_cast<uint4*>(XT1.p), v, o,
                                             nvec, planes);
  }
  // l-parts (after the row swap, which copies whole rows): XT1[x][a][i][v + l] = -t_il^ax,
  // XT2[c][a][k][v + l] = -t_kl^ca (the l-terms enter W with a minus sign)
  pack_cols(view(t2, A_(v, 1), A_(v, v), A_(o, o * vv), kOne, kOne, A_(o, vv), -1.0), XT1, 0, v, wl, s);
  pack_cols(view(t2, A_(v, v), A_(v, 1), A_(o, o * vv), kOne, kOne, A_(o, vv), -1.0), XT2, 0, v, wl, s);

  // ---- slabs of fixed b: virtual c in [b, v) in chunks, a in [0, b]; W_chunk[c - c0][a][i][j][k]
  const size_t wsz = bf ? 4 : 8;
  const long long welems = tp.welems;
  void* W = tmp_alloc(tp.w);
  const long long nblk_total = tp.nblk;
  double* tpart = static_cast<double*>(tmp_alloc(tp.tpart));
  // chunk plan and the per-c batch tables of the sigma2 / sigma5 terms (uploaded once)
  struct Chunk {
    int b, c0, nc;
    long long tab, part;
  };
  std::vector<Chunk> plan;
  long long ntab = 0;  // entries of the per-c tables: one per (b, c >= b), b-major
  {
    long long part = 0;
    for (int b = 0; b < v; ++b) {
      const long long slab = 1LL * (b + 1) * ooo;  // W elements per c
      const int ncmax = static_cast<int>(std::max(1LL, welems / slab));
      for (int c0 = b; c0 < v; c0 += ncmax) {
        const int nc = std::min(ncmax, v - c0);
        plan.push_back(Chunk{b, c0, nc, ntab, part});
        ntab += nc;
        part += 1LL * (b + 1) * nc;
      }
    }
  }
  BatchEntry* dbat = static_cast<BatchEntry*>(tmp_alloc(tp.batch));
  BatchEntry* dbat12 = static_cast<BatchEntry*>(tmp_alloc(tp.batch));
  if (sizeof(BatchEntry) * static_cast<size_t>(ntab) > tp.batch) {
    cleanup();
    set_error("lnocc_triples: internal error (launch tables larger than planned)");
    return LNOCC_EINVAL;
  }
  if (!W || !tpart || !dbat || !dbat12) {
    cleanup();
    set_error("lnocc_triples: device allocation failed (W chunk)");
    return LNOCC_ENOMEM;
  }
  count_launch();
  k_batch_tables<<<(v + 127) / 128, 128, 0, s>>>(o, v, welems, dbat, dbat12);

  const long long sblk = 1LL * o * (1LL * o * (o + 1) + 1);  // padded w / v block of the energy kernel
  // slices, t1 columns, d_m and U (up to 8 LOs, duplicated into pairs, plus 16-byte alignment)
  const long long small_smem = (3LL * o * (o + 1) + 4LL * o + 16LL * o + 4) * wsz;
  const bool staged_full = 2LL * sblk * wsz + small_smem <= 200LL * 1024;
  const bool staged = (staged_full || sblk * wsz + small_smem <= 200LL * 1024) && nlo <= 8;
  // (the staged kernel reads U padded to its compile-time LO count)
  const size_t esmem = (staged_full ? 2 : 1) * sblk * wsz + static_cast<size_t>(small_smem);
  // the energy kernel is compiled for 0, 1, 2, 4 or 8 LOs; U is zero-padded to the next size
  // (the generic kernel, used when the staged ones are not, reads U as given: any nlo)
  const int nlo_t = nlo == 0 ? 0 : nlo <= 1 ? 1 : nlo <= 2 ? 2 : nlo <= 4 ? 4 : 8;
  double* dUp = nullptr;
  if (staged && nlo_t > 0) {
    dUp = static_cast<double*>(tmp_alloc(tp.u));
    if (!dUp) {
      cleanup();
      set_error("lnocc_triples: device allocation failed (U)");
      return LNOCC_ENOMEM;
    }
    cudaMemsetAsync(dUp, 0, static_cast<size_t>(o) * nlo_t * 8, s);
    cudaMemcpy2DAsync(dUp, nlo_t * 8, U, nlo * 8, nlo * 8, o, cudaMemcpyDeviceToDevice, s);
  }
  float* ovT = nullptr;  // k_t_energy_f32 / k_t_energy_vfly read (ia|jb) from this FP32 copy
  if (bf && staged) {
    ovT = static_cast<float*>(tmp_alloc(tp.ovt));
    if (!ovT) {
      cleanup();
      set_error("lnocc_triples: device allocation failed (ovT)");
      return LNOCC_ENOMEM;
    }
    count_launch();
    k_ovov_t<<<1216, 256, 0, s>>>(ovov, ovT, o, v);
  }
  auto energy_launch = [&](const void* Wp, long long Sc, int b, int c0, int na, int nc, double* part) {
    dim3 grid(na, nc);
    count_launch();
    // FP32 W with w and v staged: k_t_energy_f32; otherwise the generic staged kernel
#define LN_F(K)                                                                                          \
  do {                                                                                                   \
    if (staged_full)                                                                                     \
      if (o == 16)                                                                                       \
        k_t_energy_f32<K, 16><<<grid, 256, esmem, s>>>(static_cast<const float*>(Wp), Sc, b, c0, o, v, eps, \
                                                       t1, ovT, dUp, part);                              \
      else                                                                                               \
        k_t_energy_f32<K, 0><<<grid, 256, esmem, s>>>(static_cast<const float*>(Wp), Sc, b, c0, o, v, eps,  \
                                                      t1, ovT, dUp, part);                               \
    else                                                                                                 \
      k_t_energy_vfly<K><<<grid, K <= 2 ? 512 : 256, esmem, s>>>(static_cast<const float*>(Wp), Sc, b, c0, o, \
                                                                 v, eps, t1, ovT, dUp, part);            \
  } while (0)
#define LN_D(K)                                                                                          \
  do {                                                                                                   \
    if (staged_full)                                                                                     \
      k_t_energy_staged<double, double, K, false><<<grid, 256, esmem, s>>>(static_cast<const double*>(Wp), Sc, \
                                                                           b, c0, o, v, eps, t1, ovov,   \
                                                                           dUp, nlo_t, part);            \
    else                                                                                                 \
      k_t_energy_staged<double, double, K, true><<<grid, 256, esmem, s>>>(static_cast<const double*>(Wp), Sc, \
                                                                          b, c0, o, v, eps, t1, ovov, dUp, \
                                                                          nlo_t, part);                  \
  } while (0)
    if (bf) {
      switch (nlo_t) {
        case 0: LN_F(0); break;
        case 1: LN_F(1); break;
        case 2: LN_F(2); break;
        case 4: LN_F(4); break;
        default: LN_F(8); break;
      }
    } else {
      switch (nlo_t) {
        case 0: LN_D(0); break;
        case 1: LN_D(1); break;
        case 2: LN_D(2); break;
        case 4: LN_D(4); break;
        default: LN_D(8); break;
      }
    }
#undef LN_F
#undef LN_D
  };
  if (staged) {
    // The attribute is per kernel and process-wide: set it once to the largest size the staged
    // kernel is ever launched with (the 200 KB cap above), so that concurrent calls on fragments of
    // other sizes never lower it under one another's launches.
    static std::once_flag once;
    std::call_once(once, [] {
      auto attr = [](const void* fn) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      };
      attr(reinterpret_cast<const void*>(k_t_energy_f32<0, 0>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<0, 16>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<1, 0>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<1, 16>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<2, 0>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<2, 16>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<4, 0>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<4, 16>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<8, 0>));
      attr(reinterpret_cast<const void*>(k_t_energy_f32<8, 16>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 0, false>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 1, false>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 2, false>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 4, false>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 8, false>));
      attr(reinterpret_cast<const void*>(k_t_energy_vfly<0>));
      attr(reinterpret_cast<const void*>(k_t_energy_vfly<1>));
      attr(reinterpret_cast<const void*>(k_t_energy_vfly<2>));
      attr(reinterpret_cast<const void*>(k_t_energy_vfly<4>));
      attr(reinterpret_cast<const void*>(k_t_energy_vfly<8>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 0, true>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 1, true>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 2, true>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 4, true>));
      attr(reinterpret_cast<const void*>(k_t_energy_staged<double, double, 8, true>));
    });
  }
  auto omap = [&](double beta) {
    OutMap m{bf ? nullptr : static_cast<double*>(W), 0, 0, 0, 0, 1 << 30, 1 << 30, 1.0, beta};
    if (bf) m.dst32 = static_cast<float*>(W);
    return m;
  };
  const int o2 = static_cast<int>(oo);
  // grouped launches (two per chunk instead of five) where 128-row tiles hold whole a values (kind 1)
  // and a (y, z) plane is one (nocc 16) or four (nocc 32) 256-column accumulator tiles
  const bool grouped = bf && (o == 16 || o == 32) && opts.triples_kernel != LNOCC_TK_PER_TERM;
  const Packed* ops_a[4] = {&XT1, &TO, &XT2, &TOT};
  const Packed* ops_b[4] = {&TO, &XT2, &TO, &XT1};
  const int box_ab[4] = {128, 256, 128, 256};
  // tuning passes (t_max_chunks > 0) visit about t_max_chunks chunks spread over the plan
  const size_t chunk_stride = t_max_chunks > 0 ? std::max<size_t>(1, plan.size() / t_max_chunks) : 1;
  size_t chunk_idx = 0;
  for (const Chunk& ch : plan) {
    if (chunk_idx++ % chunk_stride != 0) continue;
    const int b = ch.b, c0 = ch.c0, nc = ch.nc;
    const int na = b + 1, Ma = na * o, Ma2 = na * o2;
    const long long Sc = 1LL * na * ooo;  // W stride of c
    const int xb = b * v * o;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!dev_out) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
    }
    // W layout [c - c0][a][i][k][j]; each term is one contraction over K = v + o (d-part, then l-part).
    if (grouped) {
      // launch 1, per (c, 128-row tile of (a, x)): sigma1 + sigma2 stored, then sigma3 and sigma5 added
      // (the output maps of the per-term launches below, restricted to one c)
      GrpSpec g{};
      g.kind = 1;
      g.Ma = Ma;
      g.mt = (Ma + 127) / 128;
      g.nkb = XT1.Kp / 64;
      g.c0 = c0;
      g.nc = nc;
      g.cblk = 256 / o;
      g.ncol = o2 / 256;
      g.b = b;
      g.bvo = xb;
      g.vo = v * o;
      g.oo = o2;
      g.o = o;
      g.Sc = Sc;
      g.nreg = nc * g.mt;
      OutMap ca[3] = {omap(0.0), omap(1.0), omap(1.0)};
      ca[0].sm1 = ooo; ca[0].sm0 = oo; ca[0].mdiv = o; ca[0].sn1 = o; ca[0].sn0 = 1; ca[0].ndiv = o;   // (a,i) x (k,j)
      ca[1].sm1 = ooo; ca[1].sm0 = 1; ca[1].mdiv = o; ca[1].sn1 = o; ca[1].sn0 = oo; ca[1].ndiv = o;   // (a,j) x (k,i)
      ca[2].sm1 = ooo; ca[2].sm0 = o; ca[2].mdiv = o; ca[2].sn1 = oo; ca[2].sn0 = 1; ca[2].ndiv = o;   // (a,k) x (i,j)
      gemm_grouped(ops_a, box_ab, g, ca, 3, s, dstatus);
      // launch 2, per (128-row tile of (a, x, y), block of 256 / o values of c): sigma4 and sigma6 added
      GrpSpec h = g;
      h.kind = 2;
      h.Ma = Ma2;
      h.mt = (Ma2 + 127) / 128;
      h.nreg = h.mt * ((nc + g.cblk - 1) / g.cblk);
      OutMap cb[2] = {omap(1.0), omap(1.0)};
      cb[0].sm2 = ooo; cb[0].sm1 = oo; cb[0].sm0 = o; cb[0].mdiv = o; cb[0].mdiv1 = o;   // (a,i,k) x (c,j)
      cb[0].sn1 = Sc; cb[0].sn0 = 1; cb[0].ndiv = o;
      cb[1].sm2 = ooo; cb[1].sm1 = oo; cb[1].sm0 = 1; cb[1].mdiv = o; cb[1].mdiv1 = o;   // (a,i,j) x (c,k)
      cb[1].sn1 = Sc; cb[1].sn0 = o; cb[1].ndiv = o;
      gemm_grouped(ops_b, box_ab, h, cb, 2, s, dstatus);
    } else {
    // sigma1 + sigma2 (batched over c, two K segments into one accumulator; first writer of W):
    // rows (a,i), cols (k,j): (ai|bd) t_kj^cd - t_il^ab (ck|jl) + (ai|cd) t_jk^bd - t_il^ac (bj|kl)
    {
      OutMap m = omap(0.0);
      m.sm1 = ooo; m.sm0 = oo; m.mdiv = o;
      m.sn1 = o; m.sn0 = 1; m.ndiv = o;
      gemm2_batched(XT1, TO, &XT1, &TOT, dbat12 + ch.tab, nc, Ma, o2, Kt, Kt, m, s, dstatus);
    }
    // sigma3: rows (a,j), cols (c,k,i): (bj|ad) t_ki^cd - t_jl^ba (ck|il)
    {
      OutMap m = omap(1.0);
      m.sm1 = ooo; m.sm0 = 1; m.mdiv = o;
      m.sn2 = Sc; m.sn1 = o; m.sn0 = oo; m.ndiv = o; m.ndiv1 = o;
      gemm_off(XT2, xb, TO, c0 * o2, Ma, nc * o2, Kt, m, s, dstatus);
    }
    // sigma4: rows (a,i,k), cols (c,j): t_ik^ad (bj|cd) - (ai|kl) t_jl^bc
    {
      OutMap m = omap(1.0);
      m.sm2 = ooo; m.sm1 = oo; m.sm0 = o; m.mdiv = o; m.mdiv1 = o;
      m.sn1 = Sc; m.sn0 = 1; m.ndiv = o;
      gemm_off(TO, 0, XT2, xb + c0 * o, Ma2, nc * o, Kt, m, s, dstatus);
    }
    // sigma6: rows (a,i,j), cols (c,k): t_ij^ad (ck|bd) - (ai|jl) t_kl^cb
    {
      OutMap m = omap(1.0);
      m.sm2 = ooo; m.sm1 = oo; m.sm0 = 1; m.mdiv = o; m.mdiv1 = o;
      m.sn1 = Sc; m.sn0 = o; m.ndiv = o;
      gemm_off(TO, 0, XT1, xb + c0 * o, Ma2, nc * o, Kt, m, s, dstatus);
    }
    // sigma5 (batched over c): rows (a,k), cols (i,j): (ck|ad) t_ji^bd - t_kl^ca (bj|il)
    // (TOT[b][i][j] = [t_ji^bd | (bj|il)]: j runs fastest in the columns)
    {
      OutMap m = omap(1.0);
      m.sm1 = ooo; m.sm0 = o; m.mdiv = o;
      m.sn1 = oo; m.sn0 = 1; m.ndiv = o;
      gemm_batched(XT2, TOT, dbat + ch.tab, nc, Ma, o2, Kt, m, s, dstatus);
    }
    }
    if (!dev_out) {
      cudaEventRecord(e1, s);
      gev.emplace_back(e0, e1);
    }
    if (staged) {
      energy_launch(W, Sc, b, c0, na, nc, tpart + 2 * ch.part);
    } else {
      count_launch();
      if (bf)
        k_t_energy<float><<<dim3(na, nc), 128, 0, s>>>(static_cast<const float*>(W), Sc, b, c0, o, v, eps, t1, ovov,
                                                       dU, nlo, tpart + 2 * ch.part);
      else
        k_t_energy<double><<<dim3(na, nc), 128, 0, s>>>(static_cast<const double*>(W), Sc, b, c0, o, v, eps, t1,
                                                        ovov, dU, nlo, tpart + 2 * ch.part);
    }
  }
  {
    constexpr int kParts = 256;  // first-pass blocks; their sums sit after the nblk block partials
    const long long chunk = (nblk_total + kParts - 1) / kParts;
    count_launch(2);
    k_t_finish_part<<<kParts, 1024, 0, s>>>(tpart, nblk_total, chunk, tpart + 2 * nblk_total);
    k_t_finish<<<1, 1024, 0, s>>>(tpart + 2 * nblk_total, kParts, scal + 4);
  }
  if (dev_out) {
    // E_T and E_T^(F) (zero without LOs: the kernels sum no projected terms then) and the status word
    cudaMemcpyAsync(e_dev, scal + 4, 16, cudaMemcpyDeviceToDevice, s);
    if (st_dev) cudaMemcpyAsync(st_dev, dstatus, 4, cudaMemcpyDeviceToDevice, s);
    cleanup();
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
      set_error(std::string("lnocc_triples_device: ") + cudaGetErrorString(ce));
      return LNOCC_ECUDA;
    }
    return LNOCC_OK;
  }
  cudaMemcpyAsync(h_scal + 4, scal + 4, 16, cudaMemcpyDeviceToHost, s);
  cudaEventRecord(ev_call1, s);
  cudaStreamSynchronize(s);
  {
    float ms = 0.f;
    t_gemm_ms = 0.0;
    for (auto& pr : gev) {
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      t_gemm_ms += ms;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    cudaEventElapsedTime(&ms, ev_call0, ev_call1);
    t_triples_ms = ms;
  }
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
