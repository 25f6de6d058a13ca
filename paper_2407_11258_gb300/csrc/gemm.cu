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
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace lnocc {

GemmStats& gemm_stats() {
  static GemmStats s;
  return s;
}

long long& launch_counter() {
  static long long n = 0;
  return n;
}

// ------------------------------------------------------------------------------------------------
// Packing
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ long long view_off(const View& v, long long r, int k) {
  const long long r0 = r % v.R0, rr = r / v.R0;
  const long long r1 = rr % v.R1, r2 = rr / v.R1;
  const int k0 = k % v.K0, kk = k / v.K0;
  const int k1 = kk % v.K1, k2 = kk / v.K1;
  return r2 * v.sr2 + r1 * v.sr1 + r0 * v.sr0 + k2 * v.sk2 + k1 * v.sk1 + k0 * v.sk0;
}

// Writes rows [0, rows(v)) of a packed operand at `out` (plane stride `plane` elements).
template <bool BF16>
__global__ void k_pack(View v, void* out, int Kp, long long plane) {
  const int K = v.K2 * v.K1 * v.K0;
  const long long total = static_cast<long long>(v.R2) * v.R1 * v.R0 * Kp;
  for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(idx % Kp);
    const long long r = idx / Kp;
    double x = 0.0;
    if (k < K) x = v.scale * v.src[view_off(v, r, k)];
    if (BF16) {
      __nv_bfloat16 hi, lo;
      split_bf16(x, hi, lo);
      __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
      o[idx] = hi;
      o[idx + plane] = lo;
    } else {
      static_cast<double*>(out)[idx] = x;
    }
  }
}

void pack(const View& v, Packed& out, cudaStream_t s) {
  out.rows = v.rows();
  out.Kp = round_up(std::max(v.K(), 1), 64);
  const long long total = static_cast<long long>(out.rows) * out.Kp;
  const int threads = 256;
  const int blocks = static_cast<int>(std::min<long long>((total + threads - 1) / threads, 152LL * 32));
  count_launch();
  if (out.bf16)
    k_pack<true><<<blocks, threads, 0, s>>>(v, out.p, out.Kp, total);
  else
    k_pack<false><<<blocks, threads, 0, s>>>(v, out.p, out.Kp, total);
}

// Pack a view into rows [row0, row0 + v.rows()) of an existing packed operand `full`.
void pack_rows(const View& v, Packed& full, int row0, cudaStream_t s) {
  const long long total = static_cast<long long>(v.rows()) * full.Kp;
  const int threads = 256;
  const int blocks = static_cast<int>(std::min<long long>((total + threads - 1) / threads, 152LL * 32));
  const long long plane = static_cast<long long>(full.rows) * full.Kp;
  const size_t off = static_cast<size_t>(row0) * full.Kp;
  count_launch();
  if (full.bf16)
    k_pack<true><<<blocks, threads, 0, s>>>(v, static_cast<__nv_bfloat16*>(full.p) + off, full.Kp, plane);
  else
    k_pack<false><<<blocks, threads, 0, s>>>(v, static_cast<double*>(full.p) + off, full.Kp, plane);
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

__device__ __forceinline__ void store_out(const OutMap& C, int m, int n, double acc, long long base = 0) {
  const long long off = base + static_cast<long long>(m / C.mdiv) * C.sm1 +
                        static_cast<long long>(m % C.mdiv) * C.sm0 + static_cast<long long>(n / C.ndiv) * C.sn1 +
                        static_cast<long long>(n % C.ndiv) * C.sn0;
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

// ------------------------------------------------------------------------------------------------
// FP64 SIMT GEMM: 64x64 tile, 16-wide K steps, 256 threads with 4x4 outputs each.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gemm_f64(const double* __restrict__ A, const double* __restrict__ B,
                                                  int M, int N, int Kp, OutMap C, int ksplit, double* ws,
                                                  const BatchEntry* __restrict__ batch) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  long long cbase = 0;
  int kbeg = blockIdx.z * ksplit, kend = min(Kp, kbeg + ksplit);
  if (batch) {  // one problem per blockIdx.z; no split-K
    const BatchEntry be = batch[blockIdx.z];
    if (m0 >= be.M) return;
    A += static_cast<long long>(be.a_row0) * Kp;
    B += static_cast<long long>(be.b_row0) * Kp;
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
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) {
        if (ws)
          ws[(static_cast<long long>(blockIdx.z) * M + m) * N + n] = acc[i][j];
        else
          store_out(C, m, n, acc[i][j], cbase);
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
  static SplitWs w;
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
  dim3 grid((N + 63) / 64, (M + 63) / 64, nsplit);
  count_launch();
  k_gemm_f64<<<grid, 256, 0, s>>>(static_cast<const double*>(A.p), static_cast<const double*>(B.p), M, N, A.Kp, C,
                                  per, nsplit > 1 ? split_ws().p : nullptr, nullptr);
  if (nsplit > 1) splitk_reduce(nsplit, M, N, C, s);
}

// ------------------------------------------------------------------------------------------------
// tcgen05 BF16x3 GEMM.
//   CTA tile 128 x BN, K blocks of 64 (one 128-byte swizzled row per operand row and plane).
//   warp 0 lane 0: TMA producer; warp 1 lane 0: MMA issuer; warp 2: TMEM owner; all 4 warps: epilogue.
//   Per K block: 4 K=16 steps x 3 products (hi*hi, hi*lo, lo*hi) into one FP32 TMEM accumulator.
// ------------------------------------------------------------------------------------------------
template <int BN>
struct TcCfg {
  static constexpr int BM = 128;
  static constexpr int BK = 64;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int STAGES = (200 * 1024) / STAGE_BYTES > 4 ? 4 : (200 * 1024) / STAGE_BYTES;
  static constexpr int TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
};

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int M, int N,
              int nkb_total, OutMap C, int* status, int a_row0, int b_row0, int kb_per, double* ws,
              const BatchEntry* __restrict__ batch) {
  using Cfg = TcCfg<BN>;
  int kb0 = blockIdx.z * kb_per;
  int nkb = min(nkb_total - kb0, kb_per);
  long long cbase = 0;
  if (batch) {  // one problem per blockIdx.z (rows [a_row0, a_row0 + M) of A); no split-K
    const BatchEntry be = batch[blockIdx.z];
    if (static_cast<int>(blockIdx.y) * Cfg::BM >= be.M) return;
    a_row0 = be.a_row0;
    b_row0 = be.b_row0;
    M = be.M;
    cbase = be.cbase;
    kb0 = 0;
    nkb = nkb_total;
  }
  constexpr int S = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::STAGE_BYTES);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.y * Cfg::BM, n0 = blockIdx.x * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    fence_barrier_init();
    prefetch_tensormap(&tA);
    prefetch_tensormap(&tB);
  }
  if (warp == 2) tmem_alloc(tmem_holder, Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (kb >= S && !mbar_wait(&empty[s], ((kb / S) - 1) & 1)) {
        atomicExch(status, kDevTimeoutProducer);
        ok = false;
        break;
      }
      uint8_t* st = smem + s * Cfg::STAGE_BYTES;
      mbar_arrive_expect_tx(&full[s], Cfg::STAGE_BYTES);
      const int kc = (kb0 + kb) * Cfg::BK;
      tma_load_3d(st, &tA, &full[s], kc, a_row0 + m0, 0);
      tma_load_3d(st + Cfg::A_BYTES, &tA, &full[s], kc, a_row0 + m0, 1);
      tma_load_3d(st + 2 * Cfg::A_BYTES, &tB, &full[s], kc, b_row0 + n0, 0);
      tma_load_3d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, &tB, &full[s], kc, b_row0 + n0, 1);
      ++issued;
    }
    if (!ok) {  // let the copies already in flight land before the CTA retires
      for (int kb = (issued > S ? issued - S : 0); kb < issued; ++kb) mbar_wait(&full[kb % S], (kb / S) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(Cfg::BM, BN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (!mbar_wait(&full[s], (kb / S) & 1)) {
        atomicExch(status, kDevTimeoutMma);
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
        const uint64_t dah = sdesc_sw128(a_hi + off), dal = sdesc_sw128(a_lo + off);
        const uint64_t dbh = sdesc_sw128(b_hi + off), dbl = sdesc_sw128(b_lo + off);
        mma_bf16(tmem, dah, dbh, idesc, (kb | kk) != 0 ? 1u : 0u);
        mma_bf16(tmem, dah, dbl, idesc, 1u);
        mma_bf16(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(accf);
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> registers -> FP64 destination
  if (!mbar_wait(accf, 0)) {
    if (lane == 0) atomicExch(status, kDevTimeoutEpilogue);
  } else {
    tc_fence_after();
    const int row = warp * 32 + lane;
    const int m = m0 + row;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < N) {
            if (ws)
              ws[(static_cast<long long>(blockIdx.z) * M + m) * N + n] = static_cast<double>(v[j]);
            else
              store_out(C, m, n, static_cast<double>(v[j]), cbase);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, Cfg::TMEM_COLS);
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
static bool make_map(CUtensorMap* map, const Packed& P, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(P.Kp), static_cast<cuuint64_t>(P.rows), 2};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(P.Kp) * 2,
                           static_cast<cuuint64_t>(P.Kp) * 2 * static_cast<cuuint64_t>(P.rows)};
  cuuint32_t box[3] = {64, static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, P.p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
static void launch_tc(const Packed& A, int a_row0, const Packed& B, int b_row0, int M, int N, const OutMap& C,
                      cudaStream_t s, int* dstatus) {
  using Cfg = TcCfg<BN>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    attr = true;
  }
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, Cfg::BM) || !make_map(&tb, B, BN)) {
    set_error("cuTensorMapEncodeTiled failed");
    return;
  }
  const long long tiles = static_cast<long long>((N + BN - 1) / BN) * ((M + Cfg::BM - 1) / Cfg::BM);
  const int nkb = A.Kp / 64;
  const int splits = choose_splits(tiles, nkb, static_cast<long long>(M) * N);
  const int per = (nkb + splits - 1) / splits;
  dim3 grid((N + BN - 1) / BN, (M + Cfg::BM - 1) / Cfg::BM, splits);
  count_launch();
  k_gemm_tc<BN><<<grid, 128, Cfg::SMEM, s>>>(ta, tb, M, N, nkb, C, dstatus, a_row0, b_row0, per,
                                              splits > 1 ? split_ws().p : nullptr, nullptr);
  if (splits > 1) splitk_reduce(splits, M, N, C, s);
}

template <int BN>
static void launch_tc_batched(const Packed& A, const Packed& B, const BatchEntry* dbatch, int nbatch, int maxM, int N,
                              const OutMap& C, cudaStream_t s, int* dstatus) {
  using Cfg = TcCfg<BN>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    attr = true;
  }
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, Cfg::BM) || !make_map(&tb, B, BN)) {
    set_error("cuTensorMapEncodeTiled failed");
    return;
  }
  dim3 grid((N + BN - 1) / BN, (maxM + Cfg::BM - 1) / Cfg::BM, nbatch);
  count_launch();
  k_gemm_tc<BN><<<grid, 128, Cfg::SMEM, s>>>(ta, tb, maxM, N, A.Kp / 64, C, dstatus, 0, 0, A.Kp / 64, nullptr,
                                              dbatch);
}

void gemm_batched(const Packed& A, const Packed& B, const BatchEntry* dbatch, int nbatch, int maxM, int N, int K,
                  const OutMap& C, cudaStream_t s, int* dstatus) {
  if (nbatch <= 0 || maxM <= 0 || N <= 0) return;
  GemmStats& st = gemm_stats();
  st.launches++;
  st.flops += 2.0 * maxM * N * K * nbatch * 0.5;  // rows shrink along the batch; counted as half
  if (A.bf16) {
    if (N <= 32)
      launch_tc_batched<32>(A, B, dbatch, nbatch, maxM, N, C, s, dstatus);
    else if (N <= 64)
      launch_tc_batched<64>(A, B, dbatch, nbatch, maxM, N, C, s, dstatus);
    else if (N <= 128)
      launch_tc_batched<128>(A, B, dbatch, nbatch, maxM, N, C, s, dstatus);
    else if (N <= 144)
      launch_tc_batched<144>(A, B, dbatch, nbatch, maxM, N, C, s, dstatus);
    else if (N <= 192)
      launch_tc_batched<192>(A, B, dbatch, nbatch, maxM, N, C, s, dstatus);
    else
      launch_tc_batched<256>(A, B, dbatch, nbatch, maxM, N, C, s, dstatus);
  } else {
    dim3 grid((N + 63) / 64, (maxM + 63) / 64, nbatch);
    count_launch();
    k_gemm_f64<<<grid, 256, 0, s>>>(static_cast<const double*>(A.p), static_cast<const double*>(B.p), maxM, N, A.Kp,
                                    C, A.Kp, nullptr, dbatch);
  }
}

void gemm_tc(const Packed& A, int a_row0, const Packed& B, int b_row0, int M, int N, const OutMap& C,
             cudaStream_t s, int* dstatus) {
  // N tile: the smallest of {32, 64, 128, 144, 192, 256} that covers N (larger N tiles at 256)
  if (N <= 32)
    launch_tc<32>(A, a_row0, B, b_row0, M, N, C, s, dstatus);
  else if (N <= 64)
    launch_tc<64>(A, a_row0, B, b_row0, M, N, C, s, dstatus);
  else if (N <= 128)
    launch_tc<128>(A, a_row0, B, b_row0, M, N, C, s, dstatus);
  else if (N <= 144)
    launch_tc<144>(A, a_row0, B, b_row0, M, N, C, s, dstatus);
  else if (N <= 192)
    launch_tc<192>(A, a_row0, B, b_row0, M, N, C, s, dstatus);
  else
    launch_tc<256>(A, a_row0, B, b_row0, M, N, C, s, dstatus);
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
