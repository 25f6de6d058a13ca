// Learned T2 initial guess: a per-amplitude MLP correction to the first-order (MP2) amplitudes.
//
//   t_ij^ab(guess) = t_ij^ab(MP2) + s_out * g(x),  x = standardised features of the amplitude
//   features: [t_MP2, e_i, e_j, e_a, e_b, D, (ia|jb), (ib|ja)], D = e_i + e_j - e_a - e_b, taken at the
//   canonical member of {(i,j,a,b), (j,i,b,a)} (i < j, or i == j and a <= b) so the guess keeps
//   t_ij^ab = t_ji^ba; g: 8 -> 128 -> 128 -> 1 with SiLU, parameters W1[128][8], b1, W2[128][128],
//   b2, w3, b3 (row-major, output index first).
//
// Kernels: feature extraction from a fragment's MP2 amplitudes and integrals; FP32 training (forward,
// backward, Adam; also compiled in FP64 for gradient checks) with deterministic fixed-order
// reductions; and the fused inference kernel that evaluates the guess for all o^2 v^2 amplitudes:
// features and layer 1 on the CUDA cores, layer 2 as a 128 x 128 x 128 BF16 tcgen05 MMA per tile of
// 128 amplitudes (operands in shared memory, FP32 accumulator in TMEM), layer 3 in the TMEM epilogue.
// The paper has no learned component: its CCSD starts from MP2 amplitudes (Eq. 21).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fragment.h"
#include "internal.h"
#include "ptx.cuh"

namespace lnocc {

constexpr int kH = 128, kF = 8;
constexpr int kOffW1 = 0, kOffB1 = kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH,
              kOffB3 = kOffW3 + kH, kNParams = kOffB3 + 1;

struct Mlp {
  float* p = nullptr;  // parameters (device, FP32 master copy)
  float* m = nullptr;  // Adam first moment
  float* v = nullptr;  // Adam second moment
  double* norm = nullptr;  // device [17]: mu[8], sd[8], s_out
  double h_norm[17];
  long long step = 0;
  // training workspace (grown on demand)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* gbuf = nullptr;  // gradient [P] (FP64)
  double* lbuf = nullptr;  // loss
};

namespace {

// fast SiLU of the inference kernel: the hardware exponential and division approximations (errors of
// a few ulp of FP32, far below the BF16 rounding applied to the hidden layer)
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.f + __expf(-z)); }
template <typename R>
__device__ __forceinline__ R silu_r(R z) { return z / (R(1) + exp(-z)); }
template <typename R>
__device__ __forceinline__ R dsilu_r(R z) {
  const R s = R(1) / (R(1) + exp(-z));
  return s * (R(1) + z * (R(1) - s));
}

// canonical member and the raw features of flat amplitude index e = ((i*o + j)*v + a)*v + b
__device__ __forceinline__ void amp_features(long long e, int o, int v, const double* __restrict__ t2mp2,
                                             const double* __restrict__ eps, const double* __restrict__ ovov,
                                             double (&f)[kF], double& t_own) {
  int b = static_cast<int>(e % v);
  long long r = e / v;
  int a = static_cast<int>(r % v);
  r /= v;
  int j = static_cast<int>(r % o), i = static_cast<int>(r / o);
  t_own = t2mp2[e];
  if (i > j || (i == j && a > b)) {
    const int ti = i, ta = a;
    i = j;
    j = ti;
    a = b;
    b = ta;
  }
  const long long ov = static_cast<long long>(o) * v;
  const double iajb = ovov[(static_cast<long long>(i) * v + a) * ov + static_cast<long long>(j) * v + b];
  const double ibja = ovov[(static_cast<long long>(i) * v + b) * ov + static_cast<long long>(j) * v + a];
  const double ei = eps[i], ej = eps[j], ea = eps[o + a], eb = eps[o + b];
  const double D = ei + ej - ea - eb;
  f[0] = iajb / D;
  f[1] = ei;
  f[2] = ej;
  f[3] = ea;
  f[4] = eb;
  f[5] = D;
  f[6] = iajb;
  f[7] = ibja;
}

__global__ void k_mlp_samples(const long long* __restrict__ idx, int n, int o, int v, const double* __restrict__ t2mp2,
                              const double* __restrict__ eps, const double* __restrict__ ovov,
                              const double* __restrict__ t2conv, float* __restrict__ X, float* __restrict__ dt) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const long long e = idx[s];
    double f[kF], t0;
    amp_features(e, o, v, t2mp2, eps, ovov, f, t0);
#pragma unroll
    for (int k = 0; k < kF; ++k) X[static_cast<long long>(s) * kF + k] = static_cast<float>(f[k]);
    if (dt) dt[s] = static_cast<float>(t2conv[e] - t0);
  }
}

// ---------------------------------------------------------------- deterministic block reductions
template <typename R>
__device__ R block_sum_r(R x) {
  __shared__ R red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  R t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : R(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// mean / std of the 8 features and rms of dt: partials per block, then one block sums them in order
__global__ void k_norm_partials(const float* __restrict__ X, const float* __restrict__ dt, int n,
                                double* __restrict__ part) {
  double s[2 * kF + 1];
#pragma unroll
  for (int k = 0; k < 2 * kF + 1; ++k) s[k] = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < kF; ++k) {
      const double x = X[static_cast<long long>(q) * kF + k];
      s[k] += x;
      s[kF + k] += x * x;
    }
    const double d = dt[q];
    s[2 * kF] += d * d;
  }
  for (int k = 0; k < 2 * kF + 1; ++k) {
    const double t = block_sum_r(s[k]);
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = t;
  }
}
__global__ void k_norm_finish(const double* __restrict__ part, int nblk, int n, double* __restrict__ norm) {
  double s[2 * kF + 1];
  for (int k = 0; k < 2 * kF + 1; ++k) {
    double acc = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[k * nblk + b];
    s[k] = block_sum_r(acc);
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < kF; ++k) {
      const double mu = s[k] / n;
      const double var = fmax(s[kF + k] / n - mu * mu, 0.0);
      norm[k] = mu;
      norm[kF + k] = var > 0 ? sqrt(var) : 1.0;
    }
    const double so = sqrt(s[2 * kF] / n);
    norm[2 * kF] = so > 0 ? so : 1.0;
  }
}

// ---------------------------------------------------------------- training (Real = float or double)
// layer 1 forward: Z1[n][H], H1 = silu(Z1), x standardised
template <typename R>
__global__ void k_fwd1(const float* __restrict__ X, int n, const R* __restrict__ prm, const double* __restrict__ norm,
                       R* __restrict__ Xs, R* __restrict__ Z1, R* __restrict__ H1) {
  const long long total = static_cast<long long>(n) * kH;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int s = static_cast<int>(e / kH), k = static_cast<int>(e % kH);
    R z = static_cast<R>(prm[kOffB1 + k]);
#pragma unroll
    for (int f = 0; f < kF; ++f) {
      const R x = static_cast<R>((static_cast<double>(X[static_cast<long long>(s) * kF + f]) - norm[f]) / norm[kF + f]);
      z += static_cast<R>(prm[kOffW1 + k * kF + f]) * x;
      if (k == 0) Xs[static_cast<long long>(s) * kF + f] = x;
    }
    Z1[e] = z;
    H1[e] = silu_r(z);
  }
}

// C[m][c] = sum_k A(m, k) B(c, k), A(m,k) = A[m*sam + k*sak], B(c,k) = B[c*sbc + k*sbk]; tiles of 32 x 32,
// K in chunks of 32; split over K into gridDim.z fixed ranges writing partials ws[z][M][Nc]
template <typename R>
__global__ void k_small_gemm(const R* __restrict__ A, long long sam, long long sak, const R* __restrict__ B,
                             long long sbc, long long sbk, int M, int Nc, int K, int kper, R* __restrict__ ws) {
  __shared__ R As[32][33], Bs[32][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 256 threads: 8 rows of 32
  const int m0 = blockIdx.x * 32, c0 = blockIdx.y * 32, z = blockIdx.z;
  const int k_begin = z * kper, k_end = min(K, k_begin + kper);
  R acc[4] = {0, 0, 0, 0};
  for (int k0 = k_begin; k0 < k_end; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int k = k0 + tx;
      As[r][tx] = (m0 + r < M && k < k_end) ? A[(m0 + r) * sam + k * sak] : R(0);
      Bs[r][tx] = (c0 + r < Nc && k < k_end) ? B[(c0 + r) * sbc + k * sbk] : R(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const R b = Bs[tx][kk];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][kk] * b;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = m0 + ty + 8 * q, c = c0 + tx;
    if (m < M && c < Nc) ws[(static_cast<long long>(z) * M + m) * Nc + c] = acc[q];
  }
}
template <typename R>
__global__ void k_sum_splits(const R* __restrict__ ws, int splits, long long MN, R* __restrict__ out) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < MN;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    R acc = 0;
    for (int z = 0; z < splits; ++z) acc += ws[z * MN + e];
    out[e] = acc;
  }
}

// layer 2 bias + silu, output and loss pieces: Z2 += b2; H2 = silu(Z2); y = w3.H2 + b3; dy = 2(y - t)/n
template <typename R>
__global__ void k_fwd3(int n, const R* __restrict__ prm, const double* __restrict__ norm, R* __restrict__ Z2,
                       R* __restrict__ H2, const float* __restrict__ dt, R* __restrict__ y, R* __restrict__ dy,
                       double* __restrict__ lpart) {
  double lsum = 0;
  for (int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; s < n; s += gridDim.x * (blockDim.x / 32)) {
    const int l = threadIdx.x % 32;
    R acc = 0;
    for (int k = l; k < kH; k += 32) {
      const R z = Z2[static_cast<long long>(s) * kH + k] + static_cast<R>(prm[kOffB2 + k]);
      Z2[static_cast<long long>(s) * kH + k] = z;
      const R h = silu_r(z);
      H2[static_cast<long long>(s) * kH + k] = h;
      acc += static_cast<R>(prm[kOffW3 + k]) * h;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (l == 0) {
      const R yy = acc + static_cast<R>(prm[kOffB3]);
      y[s] = yy;
      if (dt) {
        const R t = static_cast<R>(static_cast<double>(dt[s]) / norm[2 * kF]);
        const R d = yy - t;
        dy[s] = R(2) * d / static_cast<R>(n);
        lsum += static_cast<double>(d) * static_cast<double>(d);
      }
    }
  }
  const double t = block_sum_r(lsum);
  if (threadIdx.x == 0 && lpart) lpart[blockIdx.x] = t;
}

// dZ2 = dy * w3 * dsilu(Z2) (in place over Z2); also dw3 pieces need H2, taken by the GEMM driver
template <typename R>
__global__ void k_bwd2(int n, const R* __restrict__ prm, const R* __restrict__ dy, R* __restrict__ Z2) {
  const long long total = static_cast<long long>(n) * kH;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int s = static_cast<int>(e / kH), k = static_cast<int>(e % kH);
    Z2[e] = dy[s] * static_cast<R>(prm[kOffW3 + k]) * dsilu_r(Z2[e]);
  }
}
// dZ1 = dH1 * dsilu(Z1) (in place over dH1)
template <typename R>
__global__ void k_bwd1(long long total, const R* __restrict__ Z1, R* __restrict__ dH1) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    dH1[e] *= dsilu_r(Z1[e]);
}
// column sums of Mtx[n][cols] in fixed order (partials per block, then per column)
template <typename R>
__global__ void k_colsum_part(const R* __restrict__ Mtx, int n, int cols, int rows_per, R* __restrict__ part) {
  const int c = threadIdx.x;
  if (c >= cols) return;
  const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
  R acc = 0;
  for (int r = r0; r < r1; ++r) acc += Mtx[static_cast<long long>(r) * cols + c];
  part[static_cast<long long>(blockIdx.x) * cols + c] = acc;
}
template <typename R>
__global__ void k_colsum_finish(const R* __restrict__ part, int nblk, int cols, R* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  R acc = 0;
  for (int b = 0; b < nblk; ++b) acc += part[static_cast<long long>(b) * cols + c];
  out[c] = acc;
}
template <typename P, typename R>
__global__ void k_convert(const P* __restrict__ src, int n, R* __restrict__ dst) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    dst[k] = static_cast<R>(src[k]);
}
template <typename R>
__global__ void k_copy_grad(const R* __restrict__ src, long long n, double* __restrict__ dst) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[e] = static_cast<double>(src[e]);
}
__global__ void k_loss_finish(const double* __restrict__ part, int nblk, int n, double* __restrict__ out) {
  double acc = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[b];
  const double t = block_sum_r(acc);
  if (threadIdx.x == 0) out[0] = t / n;
}

// Adam (Kingma & Ba): bias-corrected moments; FP32 state, FP64 gradient input
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const double* __restrict__ g, int np, float lr, float b1, float b2, float epsv, float c1,
                       float c2) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    const float gk = static_cast<float>(g[k]);
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + epsv);
  }
}

// ---------------------------------------------------------------- fused inference (tcgen05 BF16)
constexpr int kTileBytes = 128 * 128 * 2;  // one 128 x 128 BF16 operand, two 64-column swizzle atoms
constexpr int kInferSmem = 2 * kTileBytes + (kH * kF + 3 * kH + 1) * 4 + 64 + 1024;

// byte offset of element (row r, column k) of a 128 x 128 BF16 K-major operand stored as two
// 128B-swizzled atoms of 64 columns (the layout the SW128 shared-memory descriptor describes)
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  const int atom = k >> 6, chunk = (k & 63) >> 3, within = k & 7;
  return atom * (128 * 128) + r * 128 + (((chunk ^ (r & 7)) << 4)) + within * 2;
}

__global__ void __launch_bounds__(128) k_mlp_infer(int o, int v, const double* __restrict__ t2mp2,
                                                   const double* __restrict__ eps, const double* __restrict__ ovov,
                                                   const float* __restrict__ prm, const double* __restrict__ norm,
                                                   double* __restrict__ out, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = sm;
  unsigned char* sB = sm + kTileBytes;
  float* sW1 = reinterpret_cast<float*>(sm + 2 * kTileBytes);
  float* sb1 = sW1 + kH * kF;
  float* sb2 = sb1 + kH;
  float* sw3 = sb2 + kH;
  float* sb3 = sw3 + kH;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb3 + 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

  for (int k = tid; k < kH * kF; k += blockDim.x) sW1[k] = prm[kOffW1 + k];
  for (int k = tid; k < kH; k += blockDim.x) {
    sb1[k] = prm[kOffB1 + k];
    sb2[k] = prm[kOffB2 + k];
    sw3[k] = prm[kOffW3 + k];
  }
  if (tid == 0) sb3[0] = prm[kOffB3];
  // W2 as the B operand: row n = output unit, K = input unit
  for (int e = tid; e < kH * kH; e += blockDim.x) {
    const int n = e / kH, k = e % kH;
    *reinterpret_cast<__nv_bfloat16*>(sB + sw128_off(n, k)) = __float2bfloat16_rn(prm[kOffW2 + e]);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tslot, 128);
  float mu[kF], isd[kF];
#pragma unroll
  for (int f = 0; f < kF; ++f) {
    mu[f] = static_cast<float>(norm[f]);
    isd[f] = static_cast<float>(1.0 / norm[kF + f]);
  }
  const double s_out = norm[2 * kF];
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = idesc_bf16_f32(128, 128);
  const long long total = static_cast<long long>(o) * o * v * v;
  const long long ntiles = (total + 127) / 128;
  uint32_t phase = 0;
  bool ok = true;
  for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    const long long e = t * 128 + tid;
    double t_own = 0.0;
    // ---- features and layer 1 (one amplitude per thread) -> BF16 row of A
    {
      double fd[kF];
      float x[kF];
      if (e < total) {
        amp_features(e, o, v, t2mp2, eps, ovov, fd, t_own);
#pragma unroll
        for (int f = 0; f < kF; ++f) x[f] = (static_cast<float>(fd[f]) - mu[f]) * isd[f];
      } else {
#pragma unroll
        for (int f = 0; f < kF; ++f) x[f] = 0.f;
      }
#pragma unroll 1
      for (int c = 0; c < kH; c += 8) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          float z0 = sb1[c + q], z1 = sb1[c + q + 1];
#pragma unroll
          for (int f = 0; f < kF; ++f) {
            z0 = fmaf(sW1[(c + q) * kF + f], x[f], z0);
            z1 = fmaf(sW1[(c + q + 1) * kF + f], x[f], z1);
          }
          w[q / 2] = static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(silu_f(z0)))) |
                     (static_cast<uint32_t>(__bfloat16_as_ushort(__float2bfloat16_rn(silu_f(z1)))) << 16);
        }
        *reinterpret_cast<uint4*>(sA + sw128_off(tid, c)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    fence_proxy_async();  // generic-proxy smem writes -> visible to the tensor core
    tc_fence_before();
    __syncthreads();
    // ---- layer 2: one thread issues the 8 K=16 MMAs of the 128 x 128 x 128 tile
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kb = 0; kb < 2; ++kb)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = kb * (128 * 128) + kk * 32;
          mma_bf16(tmem, sdesc_sw128(smem_u32(sA) + off), sdesc_sw128(smem_u32(sB) + off), idesc,
                   (kb | kk) != 0 ? 1u : 0u);
        }
      mma_commit(bar);
    }
    const bool waited = mbar_wait(bar, phase);
    if (!waited && lane == 0) atomicExch(status, 3);
    ok = __syncthreads_and(waited) != 0;  // every thread leaves the tile loop together
    phase ^= 1;
    tc_fence_after();
    // ---- layer 3 in the epilogue: row tid of the accumulator lives in TMEM lane tid
    if (ok) {
      float acc = 0.f;
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < kH; c0 += 32) {
        float z[32];
        tmem_ld32(taddr + c0, z);
#pragma unroll
        for (int q = 0; q < 32; ++q) acc = fmaf(sw3[c0 + q], silu_f(z[q] + sb2[c0 + q]), acc);
      }
      if (e < total) out[e] = t_own + s_out * static_cast<double>(acc + sb3[0]);
    }
    tc_fence_before();
    __syncthreads();  // A and the accumulator are reused by the next tile
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

int grid_of(long long n, int threads) {
  return static_cast<int>(std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152LL * 16)));
}

// ---------------------------------------------------------------- training / gradient pass driver
struct TrainWs {
  int n, splits, lblk;
  size_t bytes;
};
template <typename R>
TrainWs train_ws(int n) {
  TrainWs w;
  w.n = n;
  w.splits = std::max(1, std::min(64, (n + 1023) / 1024));
  w.lblk = std::max(1, std::min(512, (n + 7) / 8));
  const size_t nh = static_cast<size_t>(n) * kH;
  w.bytes = sizeof(R) * (static_cast<size_t>(n) * kF + 5 * nh + 2 * static_cast<size_t>(n) + 2 * kNParams +
                         static_cast<size_t>(w.splits) * kH * kH + 256 * kH) +
            sizeof(double) * 520 + 256;
  return w;
}

template <typename R>
void small_gemm(const R* A, long long sam, long long sak, const R* B, long long sbc, long long sbk, int M, int Nc,
                int K, int splits, R* out, R* part, cudaStream_t s) {
  const int kper = splits > 1 ? ((K + splits - 1) / splits + 31) / 32 * 32 : K;
  const int nz = splits > 1 ? (K + kper - 1) / kper : 1;
  dim3 grid((M + 31) / 32, (Nc + 31) / 32, nz);
  count_launch();
  k_small_gemm<R><<<grid, 256, 0, s>>>(A, sam, sak, B, sbc, sbk, M, Nc, K, kper, nz > 1 ? part : out);
  if (nz > 1) {
    count_launch();
    k_sum_splits<R><<<grid_of(static_cast<long long>(M) * Nc, 256), 256, 0, s>>>(part, nz,
                                                                               static_cast<long long>(M) * Nc, out);
  }
}
template <typename R>
void colsum(const R* Mtx, int n, int cols, R* out, R* cpart, cudaStream_t s) {
  const int nblk = std::max(1, std::min(256, n));
  const int rows_per = (n + nblk - 1) / nblk;
  count_launch(2);
  k_colsum_part<R><<<nblk, 128, 0, s>>>(Mtx, n, cols, rows_per, cpart);
  k_colsum_finish<R><<<1, 128, 0, s>>>(cpart, nblk, cols, out);
}

// Forward (and with dt, the loss and the backward pass) over n samples in precision R. Parameters are
// converted to R first. y (device, n values in R) is written when y_out is set; the FP64 gradient
// goes to g and the loss to lossd.
template <typename R, typename P>
void mlp_pass(const P* prm, const double* norm, int n, const float* X, const float* dt, void* ws, double* y_out,
              double* g, double* lossd, cudaStream_t s) {
  const TrainWs w = train_ws<R>(n);
  const size_t nh = static_cast<size_t>(n) * kH;
  R* Xs = static_cast<R*>(ws);
  R* Z1 = Xs + static_cast<size_t>(n) * kF;
  R* H1 = Z1 + nh;
  R* Z2 = H1 + nh;
  R* H2 = Z2 + nh;
  R* dH1 = H2 + nh;
  R* y = dH1 + nh;
  R* dy = y + n;
  R* pr = dy + n;
  R* gR = pr + kNParams;
  R* part = gR + kNParams;
  R* cpart = part + static_cast<size_t>(w.splits) * kH * kH;
  double* lpart = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(cpart + 256 * kH) + 15) & ~uintptr_t(15));
  count_launch(2);
  k_convert<P, R><<<grid_of(kNParams, 256), 256, 0, s>>>(prm, kNParams, pr);
  k_fwd1<R><<<grid_of(static_cast<long long>(nh), 256), 256, 0, s>>>(X, n, pr, norm, Xs, Z1, H1);
  // Z2[s][k] = sum_l H1[s][l] W2[k][l]
  small_gemm<R>(H1, kH, 1, pr + kOffW2, kH, 1, n, kH, kH, 1, Z2, part, s);
  count_launch();
  k_fwd3<R><<<w.lblk, 256, 0, s>>>(n, pr, norm, Z2, H2, dt, y, dy, dt ? lpart : nullptr);
  if (y_out) {
    count_launch();
    k_copy_grad<R><<<grid_of(n, 256), 256, 0, s>>>(y, n, y_out);
  }
  if (!dt) return;
  count_launch();
  k_loss_finish<<<1, 256, 0, s>>>(lpart, w.lblk, n, lossd);
  // output layer: dw3[k] = sum_s dy[s] H2[s][k], db3 = sum_s dy[s]
  small_gemm<R>(H2, 1, kH, dy, 0, 1, kH, 1, n, w.splits, gR + kOffW3, part, s);
  colsum<R>(dy, n, 1, gR + kOffB3, cpart, s);
  // dZ2 = dy w3 silu'(Z2) (over Z2); dW2[k][l] = sum_s dZ2[s][k] H1[s][l]; db2 = column sums of dZ2
  count_launch();
  k_bwd2<R><<<grid_of(static_cast<long long>(nh), 256), 256, 0, s>>>(n, pr, dy, Z2);
  small_gemm<R>(Z2, 1, kH, H1, 1, kH, kH, kH, n, w.splits, gR + kOffW2, part, s);
  colsum<R>(Z2, n, kH, gR + kOffB2, cpart, s);
  // dH1[s][l] = sum_k dZ2[s][k] W2[k][l]; dZ1 = dH1 silu'(Z1)
  small_gemm<R>(Z2, kH, 1, pr + kOffW2, 1, kH, n, kH, kH, 1, dH1, part, s);
  count_launch();
  k_bwd1<R><<<grid_of(static_cast<long long>(nh), 256), 256, 0, s>>>(static_cast<long long>(nh), Z1, dH1);
  // dW1[k][f] = sum_s dZ1[s][k] x[s][f]; db1 = column sums of dZ1
  small_gemm<R>(dH1, 1, kH, Xs, 1, kF, kH, kF, n, w.splits, gR + kOffW1, part, s);
  colsum<R>(dH1, n, kH, gR + kOffB1, cpart, s);
  count_launch();
  k_copy_grad<R><<<grid_of(kNParams, 256), 256, 0, s>>>(gR, kNParams, g);
}

int ensure_ws(Mlp& m, size_t bytes) {
  if (m.ws_bytes >= bytes) return LNOCC_OK;
  if (m.ws) cudaFree(m.ws);
  m.ws = nullptr;
  m.ws_bytes = 0;
  count_alloc();
  if (cudaMalloc(&m.ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("lnocc_mlp: device allocation failed (workspace)");
    return LNOCC_ENOMEM;
  }
  m.ws_bytes = bytes;
  return LNOCC_OK;
}

}  // namespace

// learned guess into t2_out (device [o][o][v][v]); used by lnocc_mlp_guess and the MLP guess mode
int mlp_guess(const Mlp& m, int o, int v, const double* t2mp2, const double* eps, const double* ovov,
              double* t2_out, int* dstatus, cudaStream_t s) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem);
  });
  const long long total = static_cast<long long>(o) * o * v * v;
  const long long ntiles = (total + 127) / 128;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = static_cast<int>(std::min<long long>(ntiles, 3LL * nsm));
  count_launch();
  k_mlp_infer<<<grid, 128, kInferSmem, s>>>(o, v, t2mp2, eps, ovov, m.p, m.norm, t2_out, dstatus);
  LN_CUDA(cudaGetLastError());
  return LNOCC_OK;
}

}  // namespace lnocc

struct lnocc_mlp {
  lnocc::Mlp m;
};

using lnocc::Mlp;

extern "C" {

int lnocc_mlp_nparams(void) { return lnocc::kNParams; }

int lnocc_mlp_create(const float* params, lnocc_mlp** out) {
  lnocc::set_error("");
  if (!params || !out) {
    lnocc::set_error("lnocc_mlp_create: bad arguments");
    return LNOCC_EINVAL;
  }
  *out = nullptr;
  lnocc_mlp* h = new (std::nothrow) lnocc_mlp;
  if (!h) return LNOCC_ENOMEM;
  Mlp& m = h->m;
  const size_t pb = sizeof(float) * lnocc::kNParams;
  lnocc::count_alloc(6);
  if (cudaMalloc(&m.p, pb) != cudaSuccess || cudaMalloc(&m.m, pb) != cudaSuccess ||
      cudaMalloc(&m.v, pb) != cudaSuccess || cudaMalloc(&m.norm, 17 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&m.gbuf, sizeof(double) * lnocc::kNParams) != cudaSuccess ||
      cudaMalloc(&m.lbuf, sizeof(double) * 2) != cudaSuccess) {
    cudaGetLastError();
    lnocc_mlp_free(h);
    lnocc::set_error("lnocc_mlp_create: device allocation failed");
    return LNOCC_ENOMEM;
  }
  for (int k = 0; k < 8; ++k) {
    m.h_norm[k] = 0.0;
    m.h_norm[8 + k] = 1.0;
  }
  m.h_norm[16] = 1.0;
  LN_CUDA(cudaMemcpy(m.p, params, pb, cudaMemcpyHostToDevice));
  LN_CUDA(cudaMemset(m.m, 0, pb));
  LN_CUDA(cudaMemset(m.v, 0, pb));
  LN_CUDA(cudaMemcpy(m.norm, m.h_norm, sizeof(m.h_norm), cudaMemcpyHostToDevice));
  *out = h;
  return LNOCC_OK;
}

int lnocc_mlp_free(lnocc_mlp* h) {
  if (!h) return LNOCC_OK;
  Mlp& m = h->m;
  for (void* p : {static_cast<void*>(m.p), static_cast<void*>(m.m), static_cast<void*>(m.v),
                  static_cast<void*>(m.norm), m.ws, static_cast<void*>(m.gbuf), static_cast<void*>(m.lbuf)})
    if (p) cudaFree(p);
  delete h;
  return LNOCC_OK;
}

int lnocc_mlp_get(const lnocc_mlp* h, float* params, double* norm) {
  lnocc::set_error("");
  if (!h) return LNOCC_EINVAL;
  if (params) LN_CUDA(cudaMemcpy(params, h->m.p, sizeof(float) * lnocc::kNParams, cudaMemcpyDeviceToHost));
  if (norm) LN_CUDA(cudaMemcpy(norm, h->m.norm, 17 * sizeof(double), cudaMemcpyDeviceToHost));
  return LNOCC_OK;
}

int lnocc_mlp_set_norm(lnocc_mlp* h, const double* norm) {
  lnocc::set_error("");
  if (!h || !norm) return LNOCC_EINVAL;
  for (int k = 0; k < 8; ++k)
    if (!(norm[8 + k] > 0)) {
      lnocc::set_error("lnocc_mlp_set_norm: standard deviations must be positive");
      return LNOCC_EINVAL;
    }
  if (!(norm[16] > 0)) {
    lnocc::set_error("lnocc_mlp_set_norm: output scale must be positive");
    return LNOCC_EINVAL;
  }
  std::memcpy(h->m.h_norm, norm, sizeof(h->m.h_norm));
  LN_CUDA(cudaMemcpy(h->m.norm, norm, 17 * sizeof(double), cudaMemcpyHostToDevice));
  return LNOCC_OK;
}

int lnocc_mlp_samples(const lnocc_frag* f, int n, const long long* idx, float* X, float* dt, void* stream) {
  lnocc::set_error("");
  if (!f || n < 0 || (n > 0 && (!idx || !X))) {
    lnocc::set_error("lnocc_mlp_samples: bad arguments");
    return LNOCC_EINVAL;
  }
  const lnocc::Frag& fr = f->f;
  if (dt && !fr.have_amps) {
    lnocc::set_error("lnocc_mlp_samples: targets need converged amplitudes (call lnocc_ccsd first)");
    return LNOCC_EINVAL;
  }
  if (n == 0) return LNOCC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lnocc::count_launch();
  lnocc::k_mlp_samples<<<lnocc::grid_of(n, 256), 256, 0, s>>>(idx, n, fr.o, fr.v, fr.t2mp2, fr.eps, fr.ovov,
                                                              fr.xcur + static_cast<long long>(fr.o) * fr.v, X, dt);
  LN_CUDA(cudaGetLastError());
  return LNOCC_OK;
}

int lnocc_mlp_fit_norm(lnocc_mlp* h, int n, const float* X, const float* dt, void* stream) {
  lnocc::set_error("");
  if (!h || n < 2 || !X || !dt) {
    lnocc::set_error("lnocc_mlp_fit_norm: bad arguments");
    return LNOCC_EINVAL;
  }
  Mlp& m = h->m;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblk = 256;
  const int st = lnocc::ensure_ws(m, sizeof(double) * 17 * nblk);
  if (st != LNOCC_OK) return st;
  lnocc::count_launch(2);
  lnocc::k_norm_partials<<<nblk, 256, 0, s>>>(X, dt, n, static_cast<double*>(m.ws));
  lnocc::k_norm_finish<<<1, 256, 0, s>>>(static_cast<double*>(m.ws), nblk, n, m.norm);
  LN_CUDA(cudaMemcpyAsync(m.h_norm, m.norm, sizeof(m.h_norm), cudaMemcpyDeviceToHost, s));
  LN_CUDA(cudaStreamSynchronize(s));
  return LNOCC_OK;
}

int lnocc_mlp_forward(const lnocc_mlp* h, int precision, int n, const float* X, double* y, void* stream) {
  lnocc::set_error("");
  if (!h || n < 1 || !X || !y || (precision != LNOCC_PREC_FP64 && precision != LNOCC_PREC_MIXED)) {
    lnocc::set_error("lnocc_mlp_forward: bad arguments");
    return LNOCC_EINVAL;
  }
  Mlp& m = const_cast<Mlp&>(h->m);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == LNOCC_PREC_FP64) {
    const int st = lnocc::ensure_ws(m, lnocc::train_ws<double>(n).bytes);
    if (st != LNOCC_OK) return st;
    lnocc::mlp_pass<double, float>(m.p, m.norm, n, X, nullptr, m.ws, y, nullptr, nullptr, s);
  } else {
    const int st = lnocc::ensure_ws(m, lnocc::train_ws<float>(n).bytes);
    if (st != LNOCC_OK) return st;
    lnocc::mlp_pass<float, float>(m.p, m.norm, n, X, nullptr, m.ws, y, nullptr, nullptr, s);
  }
  LN_CUDA(cudaStreamSynchronize(s));
  LN_CUDA(cudaGetLastError());
  return LNOCC_OK;
}

int lnocc_mlp_grad(const lnocc_mlp* h, int precision, int n, const float* X, const float* dt, double* grad,
                   double* loss, void* stream) {
  lnocc::set_error("");
  if (!h || n < 1 || !X || !dt || !grad || (precision != LNOCC_PREC_FP64 && precision != LNOCC_PREC_MIXED)) {
    lnocc::set_error("lnocc_mlp_grad: bad arguments");
    return LNOCC_EINVAL;
  }
  Mlp& m = const_cast<Mlp&>(h->m);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == LNOCC_PREC_FP64) {
    const int st = lnocc::ensure_ws(m, lnocc::train_ws<double>(n).bytes);
    if (st != LNOCC_OK) return st;
    lnocc::mlp_pass<double, float>(m.p, m.norm, n, X, dt, m.ws, nullptr, grad, m.lbuf, s);
  } else {
    const int st = lnocc::ensure_ws(m, lnocc::train_ws<float>(n).bytes);
    if (st != LNOCC_OK) return st;
    lnocc::mlp_pass<float, float>(m.p, m.norm, n, X, dt, m.ws, nullptr, grad, m.lbuf, s);
  }
  double l = 0;
  LN_CUDA(cudaMemcpyAsync(&l, m.lbuf, sizeof(double), cudaMemcpyDeviceToHost, s));
  LN_CUDA(cudaStreamSynchronize(s));
  LN_CUDA(cudaGetLastError());
  if (loss) *loss = l;
  return LNOCC_OK;
}

int lnocc_mlp_train_step(lnocc_mlp* h, int n, const float* X, const float* dt, float lr, double* loss,
                         void* stream) {
  lnocc::set_error("");
  if (!h || n < 1 || !X || !dt || !(lr > 0)) {
    lnocc::set_error("lnocc_mlp_train_step: bad arguments");
    return LNOCC_EINVAL;
  }
  Mlp& m = h->m;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int st = lnocc::ensure_ws(m, lnocc::train_ws<float>(n).bytes);
  if (st != LNOCC_OK) return st;
  lnocc::mlp_pass<float, float>(m.p, m.norm, n, X, dt, m.ws, nullptr, m.gbuf, m.lbuf, s);
  m.step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, static_cast<float>(m.step)), c2 = 1.f - std::pow(b2, static_cast<float>(m.step));
  lnocc::count_launch();
  lnocc::k_adam<<<lnocc::grid_of(lnocc::kNParams, 256), 256, 0, s>>>(m.p, m.m, m.v, m.gbuf, lnocc::kNParams, lr, b1,
                                                                     b2, 1e-8f, c1, c2);
  if (loss) {
    LN_CUDA(cudaMemcpyAsync(loss, m.lbuf, sizeof(double), cudaMemcpyDeviceToHost, s));
    LN_CUDA(cudaStreamSynchronize(s));
  }
  LN_CUDA(cudaGetLastError());
  return LNOCC_OK;
}

int lnocc_mlp_guess(lnocc_frag* f, const lnocc_mlp* h, double* t2_out, void* stream) {
  lnocc::set_error("");
  if (!f || !h || !t2_out) {
    lnocc::set_error("lnocc_mlp_guess: bad arguments");
    return LNOCC_EINVAL;
  }
  lnocc::Frag& fr = f->f;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LN_CUDA(cudaMemsetAsync(fr.dstatus, 0, 4, s));
  const int st = lnocc::mlp_guess(h->m, fr.o, fr.v, fr.t2mp2, fr.eps, fr.ovov, t2_out, fr.dstatus, s);
  if (st != LNOCC_OK) return st;
  const int s2 = fr.check_device();
  return s2;
}

int lnocc_frag_set_mlp(lnocc_frag* f, const lnocc_mlp* h) {
  if (!f) return LNOCC_EINVAL;
  f->f.mlp = h ? &h->m : nullptr;
  return LNOCC_OK;
}

}  // extern "C"
