// Contraction engine: operand packing (strided FP64 view -> K-major FP64 or BF16 hi/lo planes),
// an FP64 SIMT GEMM (the plain FP64 path) and a tcgen05 BF16x3 GEMM with FP32 accumulation in
// TMEM, TMA-staged operands and an FP64 strided epilogue (the mixed path).
//
// Both GEMMs compute C(m, n) = sum_k A(m, k) B(n, k) with A, B K-major (rows x Kp), K padded to
// a multiple of 64 with zeros, and write alpha*C + beta*dst through an OutMap.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace lnocc {

GemmStats& gemm_stats() {
  static thread_local GemmStats s;
  return s;
}

std::atomic<long long>& launch_counter() {
  static std::atomic<long long> n{0};
  return n;
}
std::atomic<long long>& alloc_counter() {
  static std::atomic<long long> n{0};
  return n;
}
long long& thread_launch_counter() {
  static thread_local long long n = 0;
  return n;
}

// ------------------------------------------------------------------------------------------------
// Packing
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ long long view_roff(const View& v, int r) {
  const int r0 = r % v.R0, rr = r / v.R0;
  const int r1 = rr % v.R1, r2 = rr / v.R1;
  return r2 * v.sr2 + r1 * v.sr1 + r0 * v.sr0;
}
__device__ __forceinline__ long long view_koff(const View& v, int k) {
  const int k0 = k % v.K0, kk = k / v.K0;
  const int k1 = kk % v.K1, k2 = kk / v.K1;
  return k2 * v.sk2 + k1 * v.sk1 + k0 * v.sk0;
}
__device__ __forceinline__ long long view_off(const View& v, long long r, int k) {
  return view_roff(v, static_cast<int>(r)) + view_koff(v, k);
}

// Store scale * x: BF16 hi/lo planes (x truncated to FP32 through its fields and the scale applied in
// FP32: the values keep ~16 bits anyway) or FP64.
template <bool BF16>
__device__ __forceinline__ void put(void* out, long long idx, long long plane, double x, double scale) {
  if (BF16) {
    __nv_bfloat16 hi, lo;
    const float xf = f64_to_f32_fields(x) * static_cast<float>(scale);
    hi = __float2bfloat16_rn(xf);
    lo = __float2bfloat16_rn(xf - __bfloat162float(hi));
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
    o[idx] = hi;
    o[idx + plane] = lo;
  } else {
    static_cast<double*>(out)[idx] = scale * x;
  }
}

// Row-major pack (K index contiguous or nearly so in the source): one warp per (row, 256-wide K chunk).
// Writes columns [0, Kw) of rows [0, rows(v)) at `out` (row stride ld, plane stride `plane` elements);
// columns at or beyond K(v) are zero.
template <bool BF16>
__global__ void k_pack(View v, void* out, int Kw, int ld, long long plane) {
  const int K = v.K2 * v.K1 * v.K0;
  const int rows = v.R2 * v.R1 * v.R0;
  const int lane = threadIdx.x % 32;
  const long long warp = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) / 32;
  const long long nwarp = static_cast<long long>(gridDim.x) * blockDim.x / 32;
  const int nchunk = (Kw + 255) / 256;
  const long long items = static_cast<long long>(rows) * nchunk;
  const bool kflat = (v.K1 == 1 && v.K2 == 1);
  for (long long it = warp; it < items; it += nwarp) {
    const int r = static_cast<int>(it / nchunk), ch = static_cast<int>(it % nchunk);
    const double* src = v.src + view_roff(v, r);
    const long long base = static_cast<long long>(r) * ld;
    const int kend = min(Kw, (ch + 1) * 256);
    // all eight loads of the lane first (independent, in flight together), then the stores
    double x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = ch * 256 + lane + 32 * t;
      x[t] = (k < K && k < kend) ? src[kflat ? static_cast<long long>(k) * v.sk0 : view_koff(v, k)] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = ch * 256 + lane + 32 * t;
      if (k < kend) put<BF16>(out, base + k, plane, x[t], v.scale);
    }
  }
}

// The same for K contiguous in the source (K1 = K2 = 1, sk0 = 1) with every row start 16-byte aligned
// and an even destination offset: each lane moves two consecutive k (one 16-byte load, one 4-byte store
// per BF16 plane), 512 columns per warp item.
__global__ void k_pack2_bf16(View v, __nv_bfloat16* out, int Kw, int ld, long long plane) {
  const int K = v.K0;
  const int rows = v.R2 * v.R1 * v.R0;
  const int lane = threadIdx.x % 32;
  const long long warp = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) / 32;
  const long long nwarp = static_cast<long long>(gridDim.x) * blockDim.x / 32;
  const int nchunk = (Kw + 511) / 512;
  const long long items = static_cast<long long>(rows) * nchunk;
  const float sc = static_cast<float>(v.scale);
  for (long long it = warp; it < items; it += nwarp) {
    const int r = static_cast<int>(it / nchunk), ch = static_cast<int>(it % nchunk);
    const double* src = v.src + view_roff(v, r);
    const long long base = static_cast<long long>(r) * ld;
    const int kend = min(Kw, (ch + 1) * 512);
    double2 x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = ch * 512 + 2 * (lane + 32 * t);
      if (k + 1 < K) {
        x[t] = *reinterpret_cast<const double2*>(src + k);
      } else {
        x[t].x = k < K ? src[k] : 0.0;
        x[t].y = 0.0;
      }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = ch * 512 + 2 * (lane + 32 * t);
      if (k < kend) {
        const float f0 = f64_to_f32_fields(x[t].x) * sc, f1 = f64_to_f32_fields(x[t].y) * sc;
        const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(f0 - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(f1 - __bfloat162float(h1));
        // kend is even (Kw is a multiple of 64 or an even width), so k + 1 < kend here
        *reinterpret_cast<__nv_bfloat162*>(out + base + k) = __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162*>(out + base + k + plane) = __halves2bfloat162(l0, l1);
      }
    }
  }
}

// Transposing pack for sources whose rows are contiguous (sr0 == 1) and K is strided:
// 32 x 32 tiles through shared memory so that both the reads and the writes are coalesced.
// Blocks walk the 32 x 32 tiles grid-stride (few, long-lived blocks); a tile wholly beyond K is
// written as zeros without reading.
template <bool BF16, bool PAIRS>
__global__ void k_pack_t(View v, void* out, int Kw, int ld, long long plane) {
  __shared__ double tile[32][33];
  const int K = v.K2 * v.K1 * v.K0;
  const int rows = v.R2 * v.R1 * v.R0;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  const int nrt = (rows + 31) / 32, nkt = (Kw + 31) / 32;
  const long long ntiles = static_cast<long long>(nrt) * nkt;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int rb = static_cast<int>(t / nkt) * 32, kb = static_cast<int>(t % nkt) * 32;
    if (kb < K) {
      double x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + tx, k = kb + ty + 8 * q;
        x[q] = (r < rows && k < K) ? v.src[view_off(v, r, k)] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) tile[ty + 8 * q][tx] = x[q];
      __syncthreads();
      if constexpr (PAIRS) {
        // BF16 with even widths and offsets: each thread writes two k of one row per plane (4 bytes)
        const float sc = static_cast<float>(v.scale);
        __nv_bfloat16* o16 = static_cast<__nv_bfloat16*>(out);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int p = threadIdx.x + 256 * q, rl = p / 16, kl = 2 * (p % 16);
          const int r = rb + rl, k = kb + kl;
          if (r < rows && k < Kw) {
            const float f0 = f64_to_f32_fields(tile[kl][rl]) * sc, f1 = f64_to_f32_fields(tile[kl + 1][rl]) * sc;
            const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(f0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(f1 - __bfloat162float(h1));
            const long long idx = static_cast<long long>(r) * ld + k;
            *reinterpret_cast<__nv_bfloat162*>(o16 + idx) = __halves2bfloat162(h0, h1);
            *reinterpret_cast<__nv_bfloat162*>(o16 + idx + plane) = __halves2bfloat162(l0, l1);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = rb + ty + 8 * q, k = kb + tx;
          if (r < rows && k < Kw)
            put<BF16>(out, static_cast<long long>(r) * ld + k, plane, tile[tx][ty + 8 * q], v.scale);
        }
      }
      __syncthreads();
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = rb + ty + 8 * q, k = kb + tx;
        if (r < rows && k < Kw) put<BF16>(out, static_cast<long long>(r) * ld + k, plane, 0.0, 1.0);
      }
    }
  }
}

static void launch_pack(const View& v, void* out, int Kw, int ld, long long plane, bool bf16, cudaStream_t s) {
  const int rows = v.rows();
  const bool transpose = v.sr0 == 1 && v.R0 >= 32 && (v.sk0 != 1);
  count_launch();
  if (transpose) {
    const long long tiles = static_cast<long long>((rows + 31) / 32) * ((Kw + 31) / 32);
    const int grid = static_cast<int>(std::min<long long>(tiles, 152LL * 8));
    const bool pairs = bf16 && Kw % 2 == 0 && ld % 2 == 0 && plane % 2 == 0 &&
                       (reinterpret_cast<uintptr_t>(out) & 3) == 0;
    if (pairs)
      k_pack_t<true, true><<<grid, 256, 0, s>>>(v, out, Kw, ld, plane);
    else if (bf16)
      k_pack_t<true, false><<<grid, 256, 0, s>>>(v, out, Kw, ld, plane);
    else
      k_pack_t<false, false><<<grid, 256, 0, s>>>(v, out, Kw, ld, plane);
  } else if (bf16 && v.K1 == 1 && v.K2 == 1 && v.sk0 == 1 && Kw % 2 == 0 && ld % 2 == 0 && plane % 2 == 0 &&
             (reinterpret_cast<uintptr_t>(out) & 3) == 0 && (reinterpret_cast<uintptr_t>(v.src) & 15) == 0 &&
             v.sr0 % 2 == 0 && v.sr1 % 2 == 0 && v.sr2 % 2 == 0) {
    // K contiguous, every row start 16-byte aligned (even strides from an aligned base), destination
    // pairs 4-byte aligned
    const long long items = static_cast<long long>(rows) * ((Kw + 511) / 512);
    const int blocks = static_cast<int>(std::min<long long>((items + 7) / 8, 152LL * 32));
    k_pack2_bf16<<<std::max(blocks, 1), 256, 0, s>>>(v, static_cast<__nv_bfloat16*>(out), Kw, ld, plane);
  } else {
    const long long items = static_cast<long long>(rows) * ((Kw + 255) / 256);
    const int blocks = static_cast<int>(std::min<long long>((items + 7) / 8, 152LL * 32));
    if (bf16)
      k_pack<true><<<std::max(blocks, 1), 256, 0, s>>>(v, out, Kw, ld, plane);
    else
      k_pack<false><<<std::max(blocks, 1), 256, 0, s>>>(v, out, Kw, ld, plane);
  }
}

void pack(const View& v, Packed& out, cudaStream_t s) {
  out.rows = v.rows();
  out.Kp = round_up(std::max(v.K(), 1), 64);
  const long long total = static_cast<long long>(out.rows) * out.Kp;
  launch_pack(v, out.p, out.Kp, out.Kp, total, out.bf16, s);
}

// Pack a view into rows [row0, row0 + v.rows()) of an existing packed operand `full`.
void pack_rows(const View& v, Packed& full, int row0, cudaStream_t s) {
  pack_cols(v, full, row0, 0, full.Kp, s);
}

// Pack a view into rows [row0, row0 + v.rows()) and columns [col0, col0 + width) of `full` (columns
// at or beyond the view's K are written as zeros): lets two operands share one K dimension.
void pack_cols(const View& v, Packed& full, int row0, int col0, int width, cudaStream_t s) {
  const long long plane = static_cast<long long>(full.rows) * full.Kp;
  const size_t off = static_cast<size_t>(row0) * full.Kp + col0;
  void* base = full.bf16 ? static_cast<void*>(static_cast<__nv_bfloat16*>(full.p) + off)
                         : static_cast<void*>(static_cast<double*>(full.p) + off);
  launch_pack(v, base, width, full.Kp, plane, full.bf16, s);
}

__global__ void k_permute(View v, double* dst, double beta) {
  const int K = v.K2 * v.K1 * v.K0;
  const long long total = static_cast<long long>(v.R2) * v.R1 * v.R0 * K;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(idx % K);
    const long long r = idx / K;
    const double x = v.scale * v.src[view_off(v, r, k)];
    dst[idx] = beta != 0.0 ? x + beta * dst[idx] : x;
  }
}

void permute(const View& v, double* dst, double beta, cudaStream_t s) {
  const long long total = static_cast<long long>(v.rows()) * v.K();
  if (total <= 0) return;
  const int threads = 256;
  const int blocks = static_cast<int>(std::min<long long>((total + threads - 1) / threads, 152LL * 32));
  count_launch();
  k_permute<<<blocks, threads, 0, s>>>(v, dst, beta);
}

__device__ __forceinline__ long long out_moff(const OutMap& C, int m) {
  const int m0 = m % C.mdiv, mm = m / C.mdiv;
  const int m1 = mm % C.mdiv1, m2 = mm / C.mdiv1;
  return m2 * C.sm2 + m1 * C.sm1 + static_cast<long long>(m0) * C.sm0;
}
__device__ __forceinline__ long long out_noff(const OutMap& C, int n) {
  const int n0 = n % C.ndiv, nn = n / C.ndiv;
  const int n1 = nn % C.ndiv1, n2 = nn / C.ndiv1;
  return n2 * C.sn2 + n1 * C.sn1 + static_cast<long long>(n0) * C.sn0;
}

__device__ __forceinline__ void store_at(const OutMap& C, long long off, double acc) {
  if (C.dst32) {
    float r = static_cast<float>(C.alpha * acc);
    if (C.beta != 0.0) r += static_cast<float>(C.beta) * C.dst32[off];
    C.dst32[off] = r;
  } else {
    double r = C.alpha * acc;
    if (C.beta != 0.0) r += C.beta * C.dst[off];
    C.dst[off] = r;
  }
}

// Epilogue store of an FP32 accumulator: the scaling is done in FP32 (alpha, beta are small exact
// constants); an FP64 destination gets one FP64 add for beta = 1 and none for beta = 0.
__device__ __forceinline__ void store_at_f(const OutMap& C, long long off, float v, float alpha, float beta) {
  const float a = alpha * v;
  if (C.dst32) {
    C.dst32[off] = (beta != 0.f) ? fmaf(beta, C.dst32[off], a) : a;
  } else {
    double r = static_cast<double>(a);
    if (C.beta == 1.0)
      r += C.dst[off];
    else if (C.beta != 0.0)
      r += C.beta * C.dst[off];
    C.dst[off] = r;
  }
}

__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
// four consecutive floats in one reduction (p 16-byte aligned): a quarter of the L2 atomic operations
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Sixteen epilogue stores. beta = 1 accumulates with fire-and-forget reductions (each element is
// touched once per launch, so launches on one stream still add in a fixed order); other beta values
// load all old values first (independent loads in flight together), then store.
__device__ __forceinline__ void store16(const OutMap& C, const long long (&off)[16], const bool (&ok)[16],
                                        const float (&v)[16], float alpha, float beta) {
  if (C.dst32) {
    if (beta == 1.f) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (ok[j]) red_add(C.dst32 + off[j], alpha * v[j]);
      return;
    }
    float old[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) old[j] = (beta != 0.f && ok[j]) ? C.dst32[off[j]] : 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (ok[j]) C.dst32[off[j]] = fmaf(beta, old[j], alpha * v[j]);
  } else {
    if (C.beta == 1.0) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (ok[j]) red_add(C.dst + off[j], static_cast<double>(alpha * v[j]));
      return;
    }
    double old[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) old[j] = (C.beta != 0.0 && ok[j]) ? C.dst[off[j]] : 0.0;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (ok[j]) {
        double r = static_cast<double>(alpha * v[j]);
        if (C.beta != 0.0) r += C.beta * old[j];
        C.dst[off[j]] = r;
      }
  }
}

__device__ __forceinline__ void store_out(const OutMap& C, int m, int n, double acc, long long base = 0) {
  store_at(C, base + out_moff(C, m) + out_noff(C, n), acc);
}

// ------------------------------------------------------------------------------------------------
// FP64 SIMT GEMM: 64x64 tile, 16-wide K steps, 256 threads with 4x4 outputs each.
// ------------------------------------------------------------------------------------------------
// SYM: C = A A^T (B == A, M == N): only tiles on or above the diagonal run, and off-diagonal tiles
// also store their mirror image, which halves the work of a symmetric product.
template <bool SYM>
__global__ void __launch_bounds__(256) k_gemm_f64(const double* __restrict__ A, const double* __restrict__ B,
                                                  int M, int N, int Kp, OutMap C, int ksplit, double* ws,
                                                  const BatchEntry* __restrict__ batch, int seg) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  if (SYM && blockIdx.x > blockIdx.y) return;
  long long cbase = 0;
  int kbeg = blockIdx.z * ksplit, kend = min(Kp, kbeg + ksplit);
  if (batch) {  // one problem per blockIdx.z; no split-K
    const BatchEntry be = batch[blockIdx.z];
    if (m0 >= be.M) return;
    A += static_cast<long long>(seg ? be.a_row1 : be.a_row0) * Kp;
    B += static_cast<long long>(seg ? be.b_row1 : be.b_row0) * Kp;
    M = be.M;
    cbase = be.cbase;
    kbeg = 0;
    kend = Kp;
  }
  double acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int r = e / 16, k = e % 16;
      const int m = m0 + r, n = n0 + r;
      As[k][r] = (m < M) ? A[static_cast<long long>(m) * Kp + k0 + k] : 0.0;
      Bs[k][r] = (n < N) ? B[static_cast<long long>(n) * Kp + k0 + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (ws) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < M && n < N) ws[(static_cast<long long>(blockIdx.z) * M + m) * N + n] = acc[i][j];
      }
    return;
  }
  // load every old value first, then store (independent loads in flight together)
  long long off[4][4];
  double old[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      off[i][j] = (m < M && n < N) ? cbase + out_moff(C, m) + out_noff(C, n) : -1;
      old[i][j] = 0.0;
      if (off[i][j] >= 0 && C.beta != 0.0) old[i][j] = C.dst32 ? C.dst32[off[i][j]] : C.dst[off[i][j]];
    }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (off[i][j] >= 0) {
        const double r = C.alpha * acc[i][j] + C.beta * old[i][j];
        if (C.dst32)
          C.dst32[off[i][j]] = static_cast<float>(r);
        else
          C.dst[off[i][j]] = r;
      }
  if (SYM && blockIdx.x != blockIdx.y) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < M && n < N) store_out(C, n, m, acc[i][j]);
      }
  }
}

// Fixed-order sum of split-K partials ws[split][M][N], then the OutMap store.
__global__ void k_splitk_reduce(const double* __restrict__ ws, int splits, int M, int N, OutMap C) {
  const long long total = static_cast<long long>(M) * N;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += ws[z * total + idx];
    store_out(C, static_cast<int>(idx / N), static_cast<int>(idx % N), acc);
  }
}

SplitWs& split_ws() {
  static thread_local SplitWs w;
  return w;
}

// Number of K splits: enough CTAs to cover the SMs twice, at least 4 K blocks per split, and the
// partials must fit the workspace.
static int choose_splits(long long tiles, int nkb, long long MN) {
  if (tiles >= 76 || nkb < 8) return 1;
  long long s = (304 + tiles - 1) / tiles;
  s = std::min<long long>(s, nkb / 4);
  const SplitWs& w = split_ws();
  if (!w.p) return 1;
  s = std::min<long long>(s, static_cast<long long>(w.cap / std::max<long long>(MN, 1)));
  if (s < 2) return 1;
  const int per = (nkb + static_cast<int>(s) - 1) / static_cast<int>(s);
  return (nkb + per - 1) / per;  // no empty split
}

static void splitk_reduce(int splits, int M, int N, const OutMap& C, cudaStream_t s) {
  const long long total = static_cast<long long>(M) * N;
  const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 152LL * 8));
  count_launch();
  k_splitk_reduce<<<blocks, 256, 0, s>>>(split_ws().p, splits, M, N, C);
}

void gemm_f64(const Packed& A, const Packed& B, int M, int N, int K, const OutMap& C, cudaStream_t s) {
  (void)K;
  const long long tiles = static_cast<long long>((N + 63) / 64) * ((M + 63) / 64);
  const int nk16 = A.Kp / 16;
  const int splits = choose_splits(tiles, nk16 / 4, static_cast<long long>(M) * N);
  const int per = splits > 1 ? ((nk16 + splits - 1) / splits) * 16 : A.Kp;
  const int nsplit = splits > 1 ? (A.Kp + per - 1) / per : 1;
  dim3 grid((M + 63) / 64, (N + 63) / 64, nsplit);
  count_launch();
  k_gemm_f64<false><<<grid, 256, 0, s>>>(static_cast<const double*>(A.p), static_cast<const double*>(B.p), M, N, A.Kp, C,
                                  per, nsplit > 1 ? split_ws().p : nullptr, nullptr, 0);
  if (nsplit > 1) splitk_reduce(nsplit, M, N, C, s);
}

void gemm_f64_sym(const Packed& A, int M, const OutMap& C, cudaStream_t s) {
  if (M <= 0) return;
  GemmStats& st = gemm_stats();
  st.launches++;
  st.flops += 1.0 * M * M * A.Kp;  // half of 2 M^2 K
  dim3 grid((M + 63) / 64, (M + 63) / 64, 1);
  count_launch();
  k_gemm_f64<true><<<grid, 256, 0, s>>>(static_cast<const double*>(A.p), static_cast<const double*>(A.p), M, M, A.Kp,
                                        C, A.Kp, nullptr, nullptr, 0);
}

// ------------------------------------------------------------------------------------------------
// tcgen05 BF16x3 GEMM.
//   CTA tile 128 x BN, K blocks of 64 (one 128-byte swizzled row per operand row and plane).
//   warp 0 lane 0: TMA producer; warp 1 lane 0: MMA issuer; warp 2: TMEM owner; all 4 warps: epilogue.
//   Per K block: 4 K=16 steps x 3 products (hi*hi, hi*lo, lo*hi) into one FP32 TMEM accumulator.
// ------------------------------------------------------------------------------------------------
// BK_ = 64: 128-byte swizzled K blocks; 32: 64-byte swizzled K blocks, half the stage size (the grouped
// (T) launches: four stages at BN = 256 instead of two).
template <int BN, int BK_ = 64>
struct TcCfg {
  static constexpr int BM = 128;
  static constexpr int BK = BK_;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  // epilogue scratch: the transpose tiles of 4 warps, or per warp BN column offsets + BN/4 flags
  // (BN = 256, the grouped (T) launches: two 4 KB W boxes per warp)
  static constexpr int EPI_BYTES0 = 4 * 32 * 17 * 4 > 4 * (BN * 8 + BN / 4) ? 4 * 32 * 17 * 4 : 4 * (BN * 8 + BN / 4);
  static constexpr int EPI_BYTES = BN == 256 && EPI_BYTES0 < 32768 ? 32768 : EPI_BYTES0;
  // as many stages (up to 4) as fit in the 227 KB of shared memory a CTA may hold beside the epilogue
  // scratch, the 1 KB alignment slack and the barriers
  static constexpr int STAGE_ROOM = 232448 - EPI_BYTES - 1024 - 256;
  static constexpr int STAGES = STAGE_ROOM / STAGE_BYTES > 4 ? 4 : STAGE_ROOM / STAGE_BYTES;
  static constexpr int ACC_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  static constexpr int TMEM_COLS = 2 * ACC_COLS;  // two accumulators: MMA of tile t+1 overlaps epilogue of t
  static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static_assert(STAGES >= 2 && SMEM <= 232448, "pipeline does not fit the shared memory of one CTA");
};

// Arguments of one tcgen05 GEMM launch. Two K segments: C = A0 B0^T (nkb0 blocks) + A1 B1^T (nkb1 blocks)
// accumulate into the same TMEM tile; rows of segment s start at a_row[s] / b_row[s] (or come from the
// batch table, one problem per z). Split-K (kb_per < nkb0, ws != null) only with one segment.
struct TcArgs {
  int M, N, nkb0, nkb1;
  int a_row0, b_row0, a_row1, b_row1;
  int kb_per;
  int tiles_m, tiles_n, tiles_z;
  OutMap C;
  float alpha_f, beta_f;  // FP32 copies of C.alpha / C.beta for the epilogue
  int* status;
  double* ws;
  const BatchEntry* batch;
  GrpSpec g;              // grouped (T) launch when g.kind != 0 (tiles decoded from the spec)
  OutMap Cg[3];           // output maps of the grouped launch's terms
};

// Per-tile problem description, computed identically by every role.
struct TileInfo {
  bool valid;
  int m0, n0, z, M, kb0, nkbA;
  int a_row0, b_row0, a_row1, b_row1;
  long long cbase;
  int nkb1, N;                 // second-segment K blocks and valid columns of this tile
  int ma0, mb0, ma1, mb1;      // tensor maps (0..3 = tA0, tB0, tA1, tB1) of the two segments
  int omap, cz, ct;            // grouped launches: term (output map), region's W chunk c, column tile
};

// Grouped (T) launch: regions of one W chunk, each computed by one CTA as 3 (kind 1) or 2 (kind 2)
// consecutive tiles that cover the same W elements; CTA b takes regions b, b + grid, ... Tile w of the
// CTA's sequence is term w % terms of region blockIdx.x + (w / terms) * gridDim.x.
//   kind 1 (maps: 0 = XT1 [A], 1 = TO [B], 2 = XT2 [A], 3 = TOT [B]); region (c, 128-row tile of (a, x)):
//     term 0: sigma1 + sigma2 (store), term 1: sigma3, term 2: sigma5 (reductions)
//   kind 2 (maps: 0 = TO [A], 1 = XT2 [B], 3 = XT1 [B]); region (128-row tile of (a, i, x), block of c):
//     term 0: sigma4, term 1: sigma6 (reductions)
// Every epilogue warp owns the same W elements in all terms of a region (its 32 rows are 2 whole a
// values (kind 1) or 2 whole i values of one a (kind 2)), so the ordering of a region's store before
// its reductions is the warp's own (a wait on its bulk groups), with no barrier across warps.
__device__ __forceinline__ bool grp_tile(const GrpSpec& g, int w, TileInfo& ti) {
  // kind 1: 3 terms x ncol column tiles of 256 per region (all tiles of a term before the next term)
  const int per = g.kind == 1 ? 3 * g.ncol : 2;
  const int r = blockIdx.x + (w / per) * gridDim.x;
  if (r >= g.nreg) return false;
  const int q = w % per;
  const int term = g.kind == 1 ? q / g.ncol : q;
  const int ct = g.kind == 1 ? q % g.ncol : 0;
  ti.valid = true;
  ti.n0 = ct * 256;
  ti.ct = ct;
  ti.z = 0;
  ti.kb0 = 0;
  ti.nkbA = g.nkb;
  ti.nkb1 = 0;
  ti.omap = term;
  ti.ma1 = 0;
  ti.mb1 = 1;
  ti.a_row1 = ti.b_row1 = 0;
  if (g.kind == 1) {
    const int cl = r / g.mt, c = g.c0 + cl;
    ti.m0 = (r % g.mt) * 128;
    ti.M = g.Ma;
    ti.N = g.oo;
    ti.cbase = cl * g.Sc;
    ti.cz = cl;
    // B rows: the (y, z) plane of c (TO) or b (TOT); the producer adds n0 = 256 ct for the column tile
    const int bc = c * g.oo, bb = g.b * g.oo;
    if (term == 0) {
      ti.ma0 = 0; ti.a_row0 = g.bvo;          ti.mb0 = 1; ti.b_row0 = bc;
      ti.ma1 = 0; ti.a_row1 = c * g.vo;       ti.mb1 = 3; ti.b_row1 = bb;
      ti.nkb1 = g.nkb;
    } else if (term == 1) {
      ti.ma0 = 2; ti.a_row0 = g.bvo;          ti.mb0 = 1; ti.b_row0 = bc;
    } else {
      ti.ma0 = 2; ti.a_row0 = c * g.vo;       ti.mb0 = 3; ti.b_row0 = bb;
    }
  } else {
    const int cb = r / g.mt, cs = g.c0 + cb * g.cblk;
    ti.m0 = (r % g.mt) * 128;
    ti.M = g.Ma;
    ti.N = min(g.cblk, g.c0 + g.nc - cs) * g.o;
    ti.cbase = static_cast<long long>(cs - g.c0) * g.Sc;
    ti.cz = cs - g.c0;
    ti.ma0 = 0; ti.a_row0 = 0;
    ti.mb0 = term == 0 ? 1 : 3; ti.b_row0 = g.bvo + cs * g.o;
  }
  return true;
}

template <int BN>
__device__ __forceinline__ TileInfo tile_info(const TcArgs& p, int t) {
  TileInfo ti;
  const int tm = t % p.tiles_m, tn = (t / p.tiles_m) % p.tiles_n, z = t / (p.tiles_m * p.tiles_n);
  ti.m0 = tm * 128;
  ti.n0 = tn * BN;
  ti.z = z;
  ti.M = p.M;
  ti.a_row0 = p.a_row0;
  ti.b_row0 = p.b_row0;
  ti.a_row1 = p.a_row1;
  ti.b_row1 = p.b_row1;
  ti.cbase = 0;
  ti.kb0 = z * p.kb_per;
  ti.nkbA = min(p.nkb0 - ti.kb0, p.kb_per);
  if (p.batch) {
    const BatchEntry be = p.batch[z];
    ti.M = be.M;
    ti.a_row0 = be.a_row0;
    ti.b_row0 = be.b_row0;
    ti.a_row1 = be.a_row1;
    ti.b_row1 = be.b_row1;
    ti.cbase = be.cbase;
    ti.kb0 = 0;
    ti.nkbA = p.nkb0;
  }
  ti.nkb1 = p.nkb1;
  ti.N = p.N;
  ti.ma0 = 0;
  ti.mb0 = 1;
  ti.ma1 = 2;
  ti.mb1 = 3;
  ti.omap = 0;
  ti.cz = 0;
  ti.ct = 0;
  ti.valid = ti.m0 < ti.M && ti.nkbA + p.nkb1 > 0;
  return ti;
}

// Tile w of this CTA's sequence: 1 = a tile to process, 0 = an empty slot, -1 = the end.
template <int BN>
__device__ __forceinline__ int get_tile(const TcArgs& p, int w, TileInfo& ti) {
  if (p.g.kind != 0) return grp_tile(p.g, w, ti) ? 1 : -1;
  const int t = blockIdx.x + w * gridDim.x;
  if (t >= p.tiles_m * p.tiles_n * p.tiles_z) return -1;
  ti = tile_info<BN>(p, t);
  return ti.valid ? 1 : 0;
}

__device__ __forceinline__ const CUtensorMap* pick_map(int id, const CUtensorMap* m0, const CUtensorMap* m1,
                                                       const CUtensorMap* m2, const CUtensorMap* m3) {
  return id == 0 ? m0 : id == 1 ? m1 : id == 2 ? m2 : m3;
}

// Epilogue of a grouped (T) tile (nocc = 16; W chunk viewed as the 5-D tensor {j, k, i, a, c}, j fastest).
// This warp's 32 accumulator rows are sent 32 columns at a time: the 32 x 32 block is written into a
// 4 KB shared box in W order (64-byte swizzle: byte x holds logical byte x ^ (((x >> 7) & 3) << 4)) and
// one lane issues a TMA store (term 0 of kind 1) or a TMA reduce-add (every other term) of the box.
// Two boxes per warp alternate; a box is rewritten once the copy issued from it two steps before has
// read it. Boxes (j, k, i, a, c) and the thread -> element maps (row r = 16 hi + lo, column n):
//   kind 1, term 0 (sigma1 + sigma2): rows (a, i), cols (k, j); box {16, 2, 16, 2, 1} at (0, 2cc, 0, a0, c)
//   kind 1, term 1 (sigma3):          rows (a, j), cols (k, i); the same box
//   kind 1, term 2 (sigma5):          rows (a, k), cols (i, j); box {16, 16, 2, 2, 1} at (0, 0, 2cc, a0, c)
//   kind 2, term 0 (sigma4):          rows (a, i, k), cols (c, j); box {16, 16, 2, 1, 2} at (0, 0, i0, a0, c + 2cc)
//   kind 2, term 1 (sigma6):          rows (a, i, j), cols (c, k); the same box
template <int BN>
__device__ __forceinline__ void grp_epilogue(const TcArgs& p, const TileInfo& ti, const CUtensorMap* tW0,
                                             const CUtensorMap* tW1, uint32_t acc, uint32_t sbox, int ew, int lane,
                                             int& nbox) {
  constexpr int O = 16;
  const GrpSpec& g = p.g;
  const int term = ti.omap;
  const int mb = ti.m0 + ew * 32;  // first accumulator row of this warp
  const int hi = lane >> 4, lo = lane & 15;
  const int a0 = g.kind == 1 ? mb / O : mb / (O * O);
  const int i0 = g.kind == 1 ? 0 : (mb / O) % O;
  if (a0 > g.b) return;  // rows past the slab (a > b): nothing to write
  const bool vec = (g.kind == 1 && term != 1) || (g.kind == 2 && term == 0);
  // per-thread swizzle terms: 16-byte chunk t of a 64-byte row, or word j of it
  const int x = vec ? (g.kind == 1 && term == 0 ? lane & 3 : (lo >> 1) & 3) : 0;
  uint32_t off4[4], jx[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    off4[t] = static_cast<uint32_t>((t ^ x) << 4);
    jx[t] = static_cast<uint32_t>(4 * (lo ^ (t << 2)));
  }
#pragma unroll 1
  for (int cc = 0; cc < BN / 32; ++cc) {
    if (g.kind == 2 && ti.cz + 2 * cc >= g.nc) break;  // c past the chunk: the rest of the block is empty
    float v[32];
    tmem_ld32(acc + cc * 32, v);
    const uint32_t buf = sbox + (nbox & 1) * 4096;
    if (lane == 0) bulk_wait_read1();
    __syncwarp();
    if (g.kind == 1 && term == 0) {
      const uint32_t base = buf + lane * 128;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        st_shared_v4(base + (q >> 2) * 64 + off4[q & 3], v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if (g.kind == 1 && term == 1) {
      const uint32_t base = buf + hi * 2048;
#pragma unroll
      for (int col = 0; col < 32; ++col) {
        const int kp = col >> 4, i = col & 15;
        st_shared_f32(base + i * 128 + kp * 64 + jx[i & 3], v[col]);
      }
    } else if (vec) {
      // kind 1 term 2: thread (a', k), columns (i', j); kind 2 term 0: thread (i', k), columns (c', j)
      const uint32_t base = buf + (g.kind == 1 ? hi * 2048 : hi * 1024) + lo * 64;
      const uint32_t step = g.kind == 1 ? 1024 : 2048;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          st_shared_v4(base + h * step + off4[q], v[16 * h + 4 * q], v[16 * h + 4 * q + 1], v[16 * h + 4 * q + 2],
                       v[16 * h + 4 * q + 3]);
    } else {
      // kind 2 term 1: thread (i', j), columns (c', k)
      const uint32_t base = buf + hi * 1024;
#pragma unroll
      for (int col = 0; col < 32; ++col) {
        const int cp = col >> 4, k = col & 15;
        st_shared_f32(base + cp * 2048 + k * 64 + jx[(k >> 1) & 3], v[col]);
      }
    }
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
      if (g.kind == 1) {
        if (term == 0) {
          tma_store_5d(tW0, buf, 0, 2 * cc, 0, a0, ti.cz);
        } else {
          if (term == 1 && cc == 0) bulk_wait_all();  // the region's stores are performed first
          if (term == 1)
            tma_reduce_add_5d(tW0, buf, 0, 2 * cc, 0, a0, ti.cz);
          else
            tma_reduce_add_5d(tW1, buf, 0, 0, 2 * cc, a0, ti.cz);
        }
      } else {
        tma_reduce_add_5d(tW0, buf, 0, 0, i0, a0, ti.cz + 2 * cc);
      }
      bulk_commit();
    }
    ++nbox;
  }
}

// The same at nocc = 32: W viewed as {j, k, i, a, c} with 32 per occupied axis, every box 32 x 32 FP32
// with 128-byte rows under the 128-byte swizzle (byte x holds logical byte x ^ (((x >> 7) & 7) << 4)).
// A warp's 32 rows are one whole a (kind 1) or one whole i of one a (kind 2); chunk cc of column tile
// ct is one value of the column's outer index:
//   kind 1, term 0 (sigma1 + sigma2): rows (a, i), cols (k, j), k = 8 ct + cc; box [i][j] at (0, k, 0, a0, c)
//   kind 1, term 1 (sigma3):          rows (a, j), cols (k, i), same k;          box [i][j], same place
//   kind 1, term 2 (sigma5):          rows (a, k), cols (i, j), i = 8 ct + cc;  box [k][j] at (0, 0, i, a0, c)
//   kind 2, term 0 (sigma4):          rows (a, i, k), cols (c, j), c = cz + cc; box [k][j] at (0, 0, i0, a0, c)
//   kind 2, term 1 (sigma6):          rows (a, i, j), cols (c, k), same c;       box [k][j], same place
// A "row" term (thread = box row) stores 8 16-byte chunks per thread, a "column" term (thread = box
// column: sigma3, sigma6) 32 scalars; the swizzle keeps both free of bank conflicts.
template <int BN>
__device__ __forceinline__ void grp_epilogue32(const TcArgs& p, const TileInfo& ti, const CUtensorMap* tW0,
                                               const CUtensorMap* tW1, uint32_t acc, uint32_t sbox, int ew,
                                               int lane, int& nbox) {
  constexpr int O = 32;
  const GrpSpec& g = p.g;
  const int term = ti.omap;
  const int mb = ti.m0 + ew * 32;
  const int a0 = g.kind == 1 ? mb / O : mb / (O * O);
  const int i0 = g.kind == 1 ? 0 : (mb / O) % O;
  if (a0 > g.b) return;
  const bool col_term = term == 1;  // sigma3 (kind 1) and sigma6 (kind 2)
  const uint32_t x = static_cast<uint32_t>(lane & 7);
#pragma unroll 1
  for (int cc = 0; cc < BN / 32; ++cc) {
    if (g.kind == 2 && ti.cz + cc >= g.nc) break;  // c past the chunk
    float v[32];
    tmem_ld32(acc + cc * 32, v);
    const uint32_t buf = sbox + (nbox & 1) * 4096;
    if (lane == 0) bulk_wait_read1();
    __syncwarp();
    if (!col_term) {
      const uint32_t base = buf + lane * 128;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        st_shared_v4(base + ((static_cast<uint32_t>(q) ^ x) << 4), v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
      // column `lane` of the box: row r holds the accumulator column r
      const uint32_t jc = static_cast<uint32_t>(lane >> 2), jw = static_cast<uint32_t>(lane & 3) * 4;
#pragma unroll
      for (int r = 0; r < 32; ++r)
        st_shared_f32(buf + r * 128 + ((jc ^ static_cast<uint32_t>(r & 7)) << 4) + jw, v[r]);
    }
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
      if (g.kind == 1) {
        const int kk = 8 * ti.ct + cc;
        if (term == 0) {
          tma_store_5d(tW0, buf, 0, kk, 0, a0, ti.cz);
        } else {
          if (term == 1 && ti.ct == 0 && cc == 0) bulk_wait_all();  // the region's stores are performed first
          if (term == 1)
            tma_reduce_add_5d(tW0, buf, 0, kk, 0, a0, ti.cz);
          else
            tma_reduce_add_5d(tW1, buf, 0, 0, kk, a0, ti.cz);
        }
      } else {
        tma_reduce_add_5d(tW0, buf, 0, 0, i0, a0, ti.cz + cc);
      }
      bulk_commit();
    }
    ++nbox;
  }
}

// Persistent warp-specialized GEMM: warp 0 lane 0 = TMA producer, warp 1 lane 0 = MMA issuer,
// warp 2 = TMEM owner, warps 4..7 = epilogue (lanes 32*(w-4) .. +31 of the accumulator).
template <int BN, int BK = 64>
__global__ void __launch_bounds__(256, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tB0,
              const __grid_constant__ CUtensorMap tA1, const __grid_constant__ CUtensorMap tB1,
              const __grid_constant__ CUtensorMap tW0, const __grid_constant__ CUtensorMap tW1, const TcArgs p) {
  using Cfg = TcCfg<BN, BK>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* epi = reinterpret_cast<float*>(smem + S * Cfg::STAGE_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::STAGE_BYTES + Cfg::EPI_BYTES);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;   // [2] MMA -> epilogue
  uint64_t* acce = accf + 2;    // [2] epilogue -> MMA
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acce + 2);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const OutMap& C = p.C;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    fence_barrier_init();
    prefetch_tensormap(&tA0);
    prefetch_tensormap(&tB0);
    if (p.nkb1 > 0 || p.g.kind != 0) {
      prefetch_tensormap(&tA1);
      prefetch_tensormap(&tB1);
    }
  }
  if (warp == 2) tmem_alloc(tmem_holder, Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int g = 0;  // global K-block counter across tiles (stage / phase)
    bool ok = true;
    for (int w = 0; ok; ++w) {
      TileInfo ti;
      const int gt = get_tile<BN>(p, w, ti);
      if (gt < 0) break;
      if (gt == 0) continue;
      const int nkb = ti.nkbA + ti.nkb1;
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int s = g % S;
        if (g >= S && !mbar_wait(&empty[s], ((g / S) - 1) & 1)) {
          atomicExch(p.status, kDevTimeoutProducer);
          ok = false;
          break;
        }
        uint8_t* st = smem + s * Cfg::STAGE_BYTES;
        mbar_arrive_expect_tx(&full[s], Cfg::STAGE_BYTES);
        const bool seg0 = kb < ti.nkbA;
        const CUtensorMap* ta = pick_map(seg0 ? ti.ma0 : ti.ma1, &tA0, &tB0, &tA1, &tB1);
        const CUtensorMap* tb = pick_map(seg0 ? ti.mb0 : ti.mb1, &tA0, &tB0, &tA1, &tB1);
        const int kc = (seg0 ? ti.kb0 + kb : kb - ti.nkbA) * Cfg::BK;
        const int ar = (seg0 ? ti.a_row0 : ti.a_row1) + ti.m0, br = (seg0 ? ti.b_row0 : ti.b_row1) + ti.n0;
        tma_load_3d(st, ta, &full[s], kc, ar, 0);
        tma_load_3d(st + Cfg::A_BYTES, ta, &full[s], kc, ar, 1);
        tma_load_3d(st + 2 * Cfg::A_BYTES, tb, &full[s], kc, br, 0);
        tma_load_3d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, tb, &full[s], kc, br, 1);
      }
    }
    // let the copies in flight land before the CTA retires
    for (int q = (g > S ? g - S : 0); q < g; ++q) mbar_wait(&full[q % S], (q / S) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(Cfg::BM, BN);
    int g = 0, it = 0;
    bool ok = true;
    for (int w = 0; ok; ++w) {
      TileInfo ti;
      const int gt = get_tile<BN>(p, w, ti);
      if (gt < 0) break;
      if (gt == 0) continue;
      const int buf = it & 1;
      if (it >= 2 && !mbar_wait(&acce[buf], ((it / 2) - 1) & 1)) {
        atomicExch(p.status, kDevTimeoutMma);
        break;
      }
      tc_fence_after();
      const uint32_t acc = tmem + buf * Cfg::ACC_COLS;
      const int nkb = ti.nkbA + ti.nkb1;
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int s = g % S;
        if (!mbar_wait(&full[s], (g / S) & 1)) {
          atomicExch(p.status, kDevTimeoutMma);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_hi = smem_u32(smem + s * Cfg::STAGE_BYTES);
        const uint32_t a_lo = a_hi + Cfg::A_BYTES;
        const uint32_t b_hi = a_lo + Cfg::A_BYTES;
        const uint32_t b_lo = b_hi + Cfg::B_BYTES;
#pragma unroll
        for (int kk = 0; kk < Cfg::BK / 16; ++kk) {
          const uint32_t off = kk * 32;  // 16 bf16 = 32 bytes along K inside the swizzle atom
          auto sd = [](uint32_t a) { return BK == 64 ? sdesc_sw128(a) : sdesc_sw64(a); };
          const uint64_t dah = sd(a_hi + off), dal = sd(a_lo + off);
          const uint64_t dbh = sd(b_hi + off), dbl = sd(b_lo + off);
          mma_bf16(acc, dah, dbh, idesc, (kb | kk) != 0 ? 1u : 0u);
          mma_bf16(acc, dah, dbl, idesc, 1u);
          mma_bf16(acc, dal, dbh, idesc, 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&accf[buf]);
      ++it;
    }
  } else if (warp >= 4) {
    // ---------------- epilogue warps
    const int ew = warp - 4;  // TMEM lane quadrant
    const bool colmajor = !p.ws && (C.sn0 == 1 || C.sn0 == -1);
    // FP32 destination with beta 0 or 1: direct row writes with per-tile column offsets (below)
    const bool f32_direct = !p.ws && C.dst32 && (p.beta_f == 1.f || p.beta_f == 0.f);
    float* tile = epi + ew * (32 * 17);
    int it = 0, nbox = 0;
    for (int w = 0;; ++w) {
      TileInfo ti;
      const int gt = get_tile<BN>(p, w, ti);
      if (gt < 0) break;
      if (gt == 0) continue;
      const int buf = it & 1;
      if (!mbar_wait(&accf[buf], (it / 2) & 1)) {
        if (lane == 0) atomicExch(p.status, kDevTimeoutEpilogue);
        break;
      }
      tc_fence_after();
      const uint32_t acc = tmem + buf * Cfg::ACC_COLS + (static_cast<uint32_t>(ew * 32) << 16);
      const int M = ti.M;
      const bool grp = p.g.kind != 0;
      const OutMap& C = grp ? p.Cg[ti.omap] : p.C;
      if (grp) {
        // W boxes: 2 x 4 KB per epilogue warp in the epilogue scratch (1024-byte aligned)
        if (p.g.o == 32)
          grp_epilogue32<BN>(p, ti, &tW0, &tW1, acc, smem_u32(epi) + ew * 8192, ew, lane, nbox);
        else
          grp_epilogue<BN>(p, ti, &tW0, &tW1, acc, smem_u32(epi) + ew * 8192, ew, lane, nbox);
      } else if (f32_direct) {
        // FP32 destination, beta 0 or 1 (the (T) W terms). Each epilogue warp computes the column
        // offsets of the tile once into its own shared-memory slot, with a flag per group of 4 columns
        // that are consecutive and 16-byte aligned in the destination (warp-local: no barrier across
        // warps). Each thread then writes its own accumulator row straight from the TMEM load: one
        // 4-wide store / reduction per flagged group, scalar otherwise (with unit row stride the lanes
        // of a warp still cover consecutive addresses).
        long long* colo = reinterpret_cast<long long*>(epi) + ew * BN;
        uint8_t* qok = reinterpret_cast<uint8_t*>(reinterpret_cast<long long*>(epi) + 4 * BN) + ew * (BN / 4);
        __syncwarp();  // the previous tile's offsets are no longer read
        for (int q = lane; q < BN / 4; q += 32) {
          long long co[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int n = ti.n0 + 4 * q + k;
            co[k] = n < ti.N ? out_noff(C, n) : -1;
            colo[4 * q + k] = co[k];
          }
          qok[q] = co[0] >= 0 && co[3] >= 0 && co[1] == co[0] + 1 && co[2] == co[0] + 2 && co[3] == co[0] + 3 &&
                   (co[0] & 3) == 0;
        }
        __syncwarp();
        const int m = ti.m0 + ew * 32 + lane;
        const bool mvalid = m < ti.M;
        const long long rowoff = mvalid ? ti.cbase + out_moff(C, m) : 0;
        float* rowp = C.dst32 + rowoff;
        const bool rowv4 = mvalid && (reinterpret_cast<uintptr_t>(rowp) & 15) == 0;
        const float al = grp ? static_cast<float>(C.alpha) : p.alpha_f;
        const bool acc_mode = (grp ? static_cast<float>(C.beta) : p.beta_f) == 1.f;
        // 16 accumulator columns starting at c0 (values v) to the destination row
        auto emit16 = [&](const float* v, int c0) {
#pragma unroll
          for (int g4 = 0; g4 < 4; ++g4) {
            const int q = (c0 >> 2) + g4;
            if (rowv4 && qok[q]) {
              float* d = rowp + colo[4 * q];
              const float a0 = al * v[4 * g4], a1 = al * v[4 * g4 + 1], a2 = al * v[4 * g4 + 2], a3 = al * v[4 * g4 + 3];
              if (acc_mode)
                red_add4(d, a0, a1, a2, a3);
              else
                *reinterpret_cast<float4*>(d) = make_float4(a0, a1, a2, a3);
            } else {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const long long co = colo[4 * q + k];
                if (co < 0) continue;
                if (acc_mode)
                  red_add(rowp + co, al * v[4 * g4 + k]);
                else
                  rowp[co] = al * v[4 * g4 + k];
              }
            }
          }
        };
        // 32 columns per TMEM load (one wait per 32 columns instead of per 16); a 16-column tail for BN = 144
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
          if (c0 + 32 <= BN) {
            float v[32];
            tmem_ld32(acc + c0, v);
            if (!mvalid) continue;
            emit16(v, c0);
            emit16(v + 16, c0 + 16);
          } else {
            float v[16];
            tmem_ld16(acc + c0, v);
            if (!mvalid) continue;
            emit16(v, c0);
          }
        }
      } else if (p.ws) {  // split-K partials, FP64 row-major [z][M][N]
        const int m = ti.m0 + ew * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
          float v[16];
          tmem_ld16(acc + c0, v);
          if (m < M)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = ti.n0 + c0 + j;
              if (n < p.N) p.ws[(static_cast<long long>(ti.z) * M + m) * p.N + n] = static_cast<double>(v[j]);
            }
        }
      } else if (!colmajor) {
        // one row per thread; column offsets advance incrementally (no division per element).
        // Each 16-column chunk loads all old values before storing (independent loads, no aliasing stall).
        const int m = ti.m0 + ew * 32 + lane;
        const long long moff = ti.cbase + (m < M ? out_moff(C, m) : 0);
        int n = ti.n0;
        int d0 = n % C.ndiv, q = n / C.ndiv, d1 = q % C.ndiv1, d2 = q / C.ndiv1;
        long long noff = d2 * C.sn2 + d1 * C.sn1 + static_cast<long long>(d0) * C.sn0;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
          float v[16];
          tmem_ld16(acc + c0, v);
          long long offs[16];
          bool ok[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            offs[j] = moff + noff;
            ok[j] = m < M && n < p.N;
            ++n;
            noff += C.sn0;
            if (++d0 == C.ndiv) {
              d0 = 0;
              noff += C.sn1 - static_cast<long long>(C.ndiv) * C.sn0;
              if (++d1 == C.ndiv1) {
                d1 = 0;
                noff += C.sn2 - static_cast<long long>(C.ndiv1) * C.sn1;
              }
            }
          }
          store16(C, offs, ok, v, p.alpha_f, p.beta_f);
        }
      } else {
        // columns contiguous in the destination: transpose 32 x 16 blocks through shared memory so that
        // consecutive lanes store consecutive columns; row offsets computed once per tile
        const int jl = lane % 16, rh = lane / 16;
        long long moffs[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int m = ti.m0 + ew * 32 + rh + 2 * r;
          moffs[r] = m < M ? ti.cbase + out_moff(C, m) : -1;
        }
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
          float v[16];
          tmem_ld16(acc + c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) tile[lane * 17 + j] = v[j];
          __syncwarp();
          const int n = ti.n0 + c0 + jl;
          const long long noff = (n < p.N) ? out_noff(C, n) : 0;
          long long offs[16];
          bool ok[16];
          float w[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            offs[r] = moffs[r] + noff;
            ok[r] = moffs[r] >= 0 && n < p.N;
            w[r] = tile[(rh + 2 * r) * 17 + jl];
          }
          store16(C, offs, ok, w, p.alpha_f, p.beta_f);
          __syncwarp();
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[buf]);
      ++it;
    }
    if (p.g.kind != 0 && lane == 0) bulk_wait_all();  // W boxes read and written before the CTA retires
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

static int num_sms() {
  static std::atomic<int> n{0};
  int v = n.load(std::memory_order_relaxed);
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 148;
    n.store(v, std::memory_order_relaxed);
  }
  return v;
}

// ---- host side: tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Operand [2][rows][Kp] bf16 as a 3-D tensor {Kp, rows, 2}; box {64, box_rows, 1}, 128-byte swizzle.
static bool make_map(CUtensorMap* map, const Packed& P, int box_rows, int bk = 64) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(P.Kp), static_cast<cuuint64_t>(P.rows), 2};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(P.Kp) * 2,
                           static_cast<cuuint64_t>(P.Kp) * 2 * static_cast<cuuint64_t>(P.rows)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(bk), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, P.p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int BK = 64>
static void set_smem_attr() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_gemm_tc<BN, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN, BK>::SMEM);
  });
}

// One launch: segment 1 is used when A1 != nullptr.
template <int BN>
static void launch_tc(const Packed& A0, const Packed& B0, const Packed* A1, const Packed* B1, TcArgs args,
                      int gridM, int nbatch, cudaStream_t s) {
  using Cfg = TcCfg<BN>;
  set_smem_attr<BN>();
  CUtensorMap ta0, tb0, ta1, tb1;
  if (!make_map(&ta0, A0, Cfg::BM) || !make_map(&tb0, B0, BN) ||
      (A1 && (!make_map(&ta1, *A1, Cfg::BM) || !make_map(&tb1, *B1, BN)))) {
    set_error("cuTensorMapEncodeTiled failed");
    return;
  }
  if (!A1) {
    ta1 = ta0;
    tb1 = tb0;
  }
  int splits = 1;
  if (!A1 && !args.batch) {
    const long long tiles = static_cast<long long>((args.N + BN - 1) / BN) * gridM;
    splits = choose_splits(tiles, args.nkb0, static_cast<long long>(args.M) * args.N);
  }
  args.kb_per = (args.nkb0 + splits - 1) / splits;
  args.ws = splits > 1 ? split_ws().p : nullptr;
  args.tiles_m = gridM;
  args.tiles_n = (args.N + BN - 1) / BN;
  args.tiles_z = args.batch ? nbatch : splits;
  args.alpha_f = static_cast<float>(args.C.alpha);
  args.beta_f = static_cast<float>(args.C.beta);
  const long long ntiles = static_cast<long long>(args.tiles_m) * args.tiles_n * args.tiles_z;
  const int grid = static_cast<int>(std::min<long long>(ntiles, num_sms()));
  count_launch();
  k_gemm_tc<BN><<<grid, 256, Cfg::SMEM, s>>>(ta0, tb0, ta1, tb1, ta0, ta0, args);
  if (splits > 1) splitk_reduce(splits, args.M, args.N, args.C, s);
}

static int heuristic_bn(int N) {
  return N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : N <= 144 ? 144 : N <= 192 ? 192 : 256;
}

static void launch_bn(int bn, const Packed& A0, const Packed& B0, const Packed* A1, const Packed* B1,
                      const TcArgs& a, int gridM, int nbatch, cudaStream_t s) {
  switch (bn) {
    case 32: launch_tc<32>(A0, B0, A1, B1, a, gridM, nbatch, s); break;
    case 64: launch_tc<64>(A0, B0, A1, B1, a, gridM, nbatch, s); break;
    case 128: launch_tc<128>(A0, B0, A1, B1, a, gridM, nbatch, s); break;
    case 144: launch_tc<144>(A0, B0, A1, B1, a, gridM, nbatch, s); break;
    case 192: launch_tc<192>(A0, B0, A1, B1, a, gridM, nbatch, s); break;
    default: launch_tc<256>(A0, B0, A1, B1, a, gridM, nbatch, s); break;
  }
}

// ---- tile autotuner ------------------------------------------------------------------------------
// The N-width of the CTA tile (BN) decides the number of tiles (wave quantisation over the SMs), how
// often each A tile is re-read, the TMEM columns and the pipeline depth. The fixed rule above takes
// the narrowest BN that covers N; the tuner instead times every candidate on the real operands and
// keeps the fastest per shape bucket (M and the K-block count in octaves, N in half-octaves, one or
// two K segments). Timed runs write to a scratch copy of the output footprint with beta = 0,
// so the call's real output is written once, by the chosen configuration, afterwards. Batched
// (per-entry table) launches always use the fixed rule.
namespace {
struct TuneKey {
  int seg, mb, nb, kb;
  bool operator<(const TuneKey& o) const {
    return seg != o.seg ? seg < o.seg : mb != o.mb ? mb < o.mb : nb != o.nb ? nb < o.nb : kb < o.kb;
  }
};
struct Tuner {
  std::mutex mu;
  std::map<TuneKey, int> table;
  std::atomic<int> mode{0};
  long long hits = 0, misses = 0, tuned = 0;
};
Tuner& tuner() {
  static Tuner t;
  return t;
}
int octave(long long x) { return static_cast<int>(std::floor(std::log2(static_cast<double>(std::max(x, 1LL))))); }
int half_octave(long long x) { return static_cast<int>(std::floor(2.0 * std::log2(static_cast<double>(std::max(x, 1LL))))); }
TuneKey make_key(bool seg2, int M, int N, int nkb) { return TuneKey{seg2 ? 2 : 1, octave(M), half_octave(N), octave(nkb)}; }

// element range [lo, hi] that an OutMap touches for m < M, n < N (host mirror of out_moff / out_noff)
void out_extent(const OutMap& C, int M, int N, long long* lo, long long* hi) {
  auto moff = [&](int m) {
    const int m0 = m % C.mdiv, mm = m / C.mdiv;
    return (mm / C.mdiv1) * C.sm2 + (mm % C.mdiv1) * C.sm1 + static_cast<long long>(m0) * C.sm0;
  };
  auto noff = [&](int n) {
    const int n0 = n % C.ndiv, nn = n / C.ndiv;
    return (nn / C.ndiv1) * C.sn2 + (nn % C.ndiv1) * C.sn1 + static_cast<long long>(n0) * C.sn0;
  };
  long long mlo = LLONG_MAX, mhi = LLONG_MIN, nlo = LLONG_MAX, nhi = LLONG_MIN;
  for (int m = 0; m < M; ++m) {
    const long long x = moff(m);
    mlo = std::min(mlo, x);
    mhi = std::max(mhi, x);
  }
  for (int n = 0; n < N; ++n) {
    const long long x = noff(n);
    nlo = std::min(nlo, x);
    nhi = std::max(nhi, x);
  }
  *lo = mlo + nlo;
  *hi = mhi + nhi;
}
}  // namespace

bool& autotune_timing_allowed() {
  static thread_local bool allowed = true;
  return allowed;
}

int autotune_mode(int mode) {
  const int prev = tuner().mode.load();
  if (mode >= 0) tuner().mode.store(mode);
  return prev;
}
void autotune_stats(long long out[4]) {
  Tuner& T = tuner();
  std::lock_guard<std::mutex> lk(T.mu);
  out[0] = static_cast<long long>(T.table.size());
  out[1] = T.hits;
  out[2] = T.misses;
  out[3] = T.tuned;
}
bool autotune_save(const char* path) {
  Tuner& T = tuner();
  std::lock_guard<std::mutex> lk(T.mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return false;
  std::fprintf(f, "# lnocc tile table: seg mbucket nbucket kbucket BN\n");
  for (const auto& kv : T.table)
    std::fprintf(f, "%d %d %d %d %d\n", kv.first.seg, kv.first.mb, kv.first.nb, kv.first.kb, kv.second);
  return std::fclose(f) == 0;
}
bool autotune_load(const char* path) {
  Tuner& T = tuner();
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  std::map<TuneKey, int> t;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    TuneKey k{};
    int bn = 0;
    if (std::sscanf(line, "%d %d %d %d %d", &k.seg, &k.mb, &k.nb, &k.kb, &bn) != 5) continue;
    if (bn != 32 && bn != 64 && bn != 128 && bn != 144 && bn != 192 && bn != 256) continue;
    t[k] = bn;
  }
  std::fclose(f);
  std::lock_guard<std::mutex> lk(T.mu);
  for (const auto& kv : t) T.table[kv.first] = kv.second;
  return true;
}

static int tune_bn(const Packed& A0, const Packed& B0, const Packed* A1, const Packed* B1, const TcArgs& a,
                   int gridM, cudaStream_t s, int fallback) {
  long long lo = 0, hi = 0;
  out_extent(a.C, a.M, a.N, &lo, &hi);
  if (lo < 0 || hi < lo) return fallback;
  const size_t esz = a.C.dst32 ? 4 : 8;
  void* scratch = nullptr;
  count_alloc();
  if (cudaMalloc(&scratch, static_cast<size_t>(hi + 1) * esz) != cudaSuccess) {
    cudaGetLastError();
    return fallback;
  }
  TcArgs t = a;
  t.C.beta = 0.0;
  if (a.C.dst32) t.C.dst32 = static_cast<float*>(scratch);
  else t.C.dst = static_cast<double*>(scratch);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = fallback;
  float best_ms = 1e30f;
  for (int bn : {32, 64, 128, 144, 192, 256}) {
    if (bn != fallback && (bn / 2 >= std::max(a.N, 32) || (bn == 32 && a.N > 64))) continue;
    launch_bn(bn, A0, B0, A1, B1, t, gridM, 1, s);  // warm-up (TMA descriptors, caches)
    float ms_min = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, s);
      launch_bn(bn, A0, B0, A1, B1, t, gridM, 1, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_min = std::min(ms_min, ms);
    }
    if (ms_min < best_ms * 0.98f || (bn == fallback && ms_min <= best_ms)) {
      best_ms = ms_min;
      best = bn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(scratch);
  return best;
}

static void dispatch_tc(const Packed& A0, const Packed& B0, const Packed* A1, const Packed* B1, const TcArgs& a,
                        int gridM, int nbatch, cudaStream_t s) {
  int bn = heuristic_bn(a.N);
  Tuner& T = tuner();
  const int mode = T.mode.load(std::memory_order_relaxed);
  if (mode != 0 && !a.batch) {
    const TuneKey key = make_key(A1 != nullptr, a.M, a.N, a.nkb0 + a.nkb1);
    bool found = false;
    {
      std::lock_guard<std::mutex> lk(T.mu);
      auto it = T.table.find(key);
      if (it != T.table.end()) {
        bn = it->second;
        found = true;
        T.hits++;
      } else {
        T.misses++;
      }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!found && mode == 2 && autotune_timing_allowed() && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      bn = tune_bn(A0, B0, A1, B1, a, gridM, s, bn);
      std::lock_guard<std::mutex> lk(T.mu);
      T.table[key] = bn;
      T.tuned++;
    }
  }
  launch_bn(bn, A0, B0, A1, B1, a, gridM, nbatch, s);
}

static TcArgs tc_args(int M, int N, int nkb0, int nkb1, const OutMap& C, int* dstatus) {
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.nkb0 = nkb0;
  a.nkb1 = nkb1;
  a.kb_per = nkb0;
  a.C = C;
  a.status = dstatus;
  return a;
}

// The FP32 W chunk [c][a][i][k][j] as the 5-D tensor {j, k, i, a, c}; boxes 64-byte swizzled at nocc 16
// (rows of 16 floats), 128-byte swizzled at nocc 32 (rows of 32 floats).
static bool make_wmap(CUtensorMap* map, float* W, const GrpSpec& g, const cuuint32_t box[5]) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t o = static_cast<cuuint64_t>(g.o);
  cuuint64_t dims[5] = {o, o, o, static_cast<cuuint64_t>(g.b + 1), static_cast<cuuint64_t>(g.nc)};
  cuuint64_t strides[4] = {o * 4, o * o * 4, o * o * o * 4, static_cast<cuuint64_t>(g.Sc) * 4};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, W, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            g.o == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void gemm_grouped(const Packed* const ops[4], const int box_rows[4], const GrpSpec& g, const OutMap* Cg, int ncg,
                  cudaStream_t s, int* dstatus) {
  if (g.nreg <= 0) return;
  if ((g.o != 16 && g.o != 32) || g.oo != g.o * g.o || g.ncol != g.oo / 256 || g.cblk != 256 / g.o ||
      (g.kind != 1 && g.kind != 2) || !Cg[0].dst32) {
    set_error("gemm_grouped: nocc 16 or 32 and an FP32 W chunk only");
    return;
  }
  // K-block width: 32 at nocc 32 (four pipeline stages of 48 KB at BN = 256; measured 8.13 -> 7.78 s of
  // contractions at 32/480/1600), 64 at nocc 16 (two stages of 96 KB; its 256-long K measured faster
  // with the wider blocks: 73 vs 83 ms at 16/240/960)
  const int gbk = g.o == 32 ? 32 : 64;
  if (gbk == 32)
    set_smem_attr<256, 32>();
  else
    set_smem_attr<256, 64>();
  CUtensorMap m[4];
  for (int k = 0; k < 4; ++k) {
    if (ops[k]->Kp % gbk != 0 || !make_map(&m[k], *ops[k], box_rows[k], gbk)) {
      set_error("cuTensorMapEncodeTiled failed");
      return;
    }
  }
  CUtensorMap w0, w1;
  // boxes (j, k, i, a, c) of the epilogue's 32 x 32 blocks (see grp_epilogue / grp_epilogue32)
  const cuuint32_t box16_a0[5] = {16, 2, 16, 2, 1}, box16_a1[5] = {16, 16, 2, 2, 1}, box16_b[5] = {16, 16, 2, 1, 2};
  const cuuint32_t box32_a0[5] = {32, 1, 32, 1, 1}, box32_a1[5] = {32, 32, 1, 1, 1}, box32_b[5] = {32, 32, 1, 1, 1};
  const cuuint32_t* b0 = g.o == 16 ? (g.kind == 1 ? box16_a0 : box16_b) : (g.kind == 1 ? box32_a0 : box32_b);
  const cuuint32_t* b1 = g.o == 16 ? (g.kind == 1 ? box16_a1 : box16_b) : (g.kind == 1 ? box32_a1 : box32_b);
  if (!make_wmap(&w0, Cg[0].dst32, g, b0) || !make_wmap(&w1, Cg[0].dst32, g, b1)) {
    set_error("cuTensorMapEncodeTiled failed (W chunk)");
    return;
  }
  TcArgs a{};
  a.M = g.Ma;
  a.N = 256;
  a.nkb0 = ops[0]->Kp / gbk;
  a.kb_per = a.nkb0;
  a.tiles_m = a.tiles_n = a.tiles_z = 1;
  a.status = dstatus;
  a.g = g;
  a.g.nkb = ops[0]->Kp / gbk;  // K blocks of one term in this launch's block width
  for (int k = 0; k < ncg && k < 3; ++k) a.Cg[k] = Cg[k];
  a.C = Cg[0];
  a.alpha_f = 1.f;
  a.beta_f = 0.f;
  GemmStats& st = gemm_stats();
  st.launches++;
  // useful flops: kind 1 = sigma1, sigma2, sigma3, sigma5 over (a, x) x (y, z) per c; kind 2 = sigma4,
  // sigma6 over (a, x, y) x (c, z)
  st.flops += g.kind == 1 ? 2.0 * g.Ma * g.oo * (64.0 * g.nkb) * 4 * g.nc
                          : 2.0 * g.Ma * (1.0 * g.nc * g.o) * (64.0 * g.nkb) * 2;
  const int grid = static_cast<int>(std::min<long long>(g.nreg, num_sms()));
  count_launch();
  static_assert(TcCfg<256, 32>::STAGES == 4 && TcCfg<256, 64>::STAGES == 2, "grouped launch pipelines");
  if (gbk == 32)
    k_gemm_tc<256, 32><<<grid, 256, TcCfg<256, 32>::SMEM, s>>>(m[0], m[1], m[2], m[3], w0, w1, a);
  else
    k_gemm_tc<256, 64><<<grid, 256, TcCfg<256, 64>::SMEM, s>>>(m[0], m[1], m[2], m[3], w0, w1, a);
}

void gemm_tc(const Packed& A, int a_row0, const Packed& B, int b_row0, int M, int N, const OutMap& C,
             cudaStream_t s, int* dstatus) {
  TcArgs a = tc_args(M, N, A.Kp / 64, 0, C, dstatus);
  a.a_row0 = a_row0;
  a.b_row0 = b_row0;
  dispatch_tc(A, B, nullptr, nullptr, a, (M + 127) / 128, 1, s);
}

void gemm_batched(const Packed& A, const Packed& B, const BatchEntry* dbatch, int nbatch, int maxM, int N, int K,
                  const OutMap& C, cudaStream_t s, int* dstatus) {
  gemm2_batched(A, B, nullptr, nullptr, dbatch, nbatch, maxM, N, K, 0, C, s, dstatus);
}

void gemm2_batched(const Packed& A0, const Packed& B0, const Packed* A1, const Packed* B1, const BatchEntry* dbatch,
                   int nbatch, int maxM, int N, int K0, int K1, const OutMap& C, cudaStream_t s, int* dstatus) {
  if (nbatch <= 0 || maxM <= 0 || N <= 0) return;
  GemmStats& st = gemm_stats();
  st.launches++;
  st.flops += 2.0 * maxM * N * (K0 + K1) * nbatch * 0.5;  // rows shrink along the batch; counted as half
  if (A0.bf16) {
    TcArgs a = tc_args(maxM, N, A0.Kp / 64, A1 ? A1->Kp / 64 : 0, C, dstatus);
    a.batch = dbatch;
    dispatch_tc(A0, B0, A1, B1, a, (maxM + 127) / 128, nbatch, s);
  } else {
    dim3 grid((maxM + 63) / 64, (N + 63) / 64, nbatch);
    count_launch();
    k_gemm_f64<false><<<grid, 256, 0, s>>>(static_cast<const double*>(A0.p), static_cast<const double*>(B0.p), maxM, N,
                                    A0.Kp, C, A0.Kp, nullptr, dbatch, 0);
    if (A1) {
      OutMap C1 = C;
      C1.beta = 1.0;
      count_launch();
      k_gemm_f64<false><<<grid, 256, 0, s>>>(static_cast<const double*>(A1->p), static_cast<const double*>(B1->p), maxM, N,
                                      A1->Kp, C1, A1->Kp, nullptr, dbatch, 1);
    }
  }
}

void gemm2_off(const Packed& A0, int a0, const Packed& B0, int b0, int K0, const Packed& A1, int a1, const Packed& B1,
               int b1, int K1, int M, int N, const OutMap& C, cudaStream_t s, int* dstatus) {
  if (M <= 0 || N <= 0) return;
  GemmStats& st = gemm_stats();
  st.launches++;
  st.flops += 2.0 * M * N * (K0 + K1);
  if (A0.bf16) {
    TcArgs a = tc_args(M, N, A0.Kp / 64, A1.Kp / 64, C, dstatus);
    a.a_row0 = a0;
    a.b_row0 = b0;
    a.a_row1 = a1;
    a.b_row1 = b1;
    dispatch_tc(A0, B0, &A1, &B1, a, (M + 127) / 128, 1, s);
  } else {
    gemm_off(A0, a0, B0, b0, M, N, K0, C, s, dstatus);
    OutMap C1 = C;
    C1.beta = 1.0;
    gemm_off(A1, a1, B1, b1, M, N, K1, C1, s, dstatus);
  }
}

void gemm_off(const Packed& A, int a_row0, const Packed& B, int b_row0, int M, int N, int K, const OutMap& C,
              cudaStream_t s, int* dstatus) {
  if (M <= 0 || N <= 0) return;
  GemmStats& st = gemm_stats();
  st.launches++;
  st.flops += 2.0 * M * N * K;
  if (A.bf16) {
    gemm_tc(A, a_row0, B, b_row0, M, N, C, s, dstatus);
  } else {
    Packed a = A, b = B;
    a.p = static_cast<double*>(A.p) + static_cast<size_t>(a_row0) * A.Kp;
    b.p = static_cast<double*>(B.p) + static_cast<size_t>(b_row0) * B.Kp;
    gemm_f64(a, b, M, N, K, C, s);
  }
}

void gemm(const Packed& A, const Packed& B, int M, int N, int K, const OutMap& C, cudaStream_t s, int* dstatus) {
  gemm_off(A, 0, B, 0, M, N, K, C, s, dstatus);
}

}  // namespace lnocc
