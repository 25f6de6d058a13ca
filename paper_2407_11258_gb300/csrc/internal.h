// Internal (host-side) interfaces shared by the translation units of liblnocc.
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lnocc.h"

namespace lnocc {

// Device-side error codes written to the status word (host reads it after a sync).
enum DevErr : int {
  kDevOk = 0,
  kDevTimeoutProducer = 1,
  kDevTimeoutMma = 2,
  kDevTimeoutEpilogue = 3,
  kDevBadShape = 4,
};

// Destination of a contraction: C(m, n) with m = (m2, m1, m0), n = (n2, n1, n0),
//   m0 = m % mdiv, m1 = (m / mdiv) % mdiv1, m2 = m / (mdiv * mdiv1)   (same for n)
//   dst[m2*sm2 + m1*sm1 + m0*sm0 + n2*sn2 + n1*sn1 + n0*sn0] = alpha * C + beta * dst (beta = 0 overwrites).
// The two-level form {dst, sm1, sm0, sn1, sn0, mdiv, ndiv, alpha, beta} leaves the outer levels unused.
// When dst32 is set the destination is FP32 instead (dst unused).
struct OutMap {
  double* dst;
  long long sm1, sm0, sn1, sn0;
  int mdiv, ndiv;
  double alpha, beta;
  float* dst32 = nullptr;
  long long sm2 = 0, sn2 = 0;
  int mdiv1 = 1 << 30, ndiv1 = 1 << 30;
};

inline OutMap out_rowmajor(double* dst, long long ldc, double alpha = 1.0, double beta = 0.0) {
  return OutMap{dst, 0, ldc, 0, 1, 1 << 30, 1 << 30, alpha, beta};
}

// One problem of a batched GEMM: rows [a_row0, a_row0 + M) of A against rows [b_row0, b_row0 + N) of B,
// destination offset cbase (elements) added to the OutMap.
struct BatchEntry {
  int a_row0, b_row0, M, a_row1, b_row1, pad;
  long long cbase;
};

// A strided FP64 view used as a K-major operand: row r = (r2, r1, r0), column k = (k2, k1, k0)
// (last index fastest); element (r, k) sits at
//   src[r2*sr2 + r1*sr1 + r0*sr0 + k2*sk2 + k1*sk1 + k0*sk0] * scale.
struct View {
  const double* src;
  int R2, R1, R0, K2, K1, K0;
  long long sr2, sr1, sr0, sk2, sk1, sk0;
  double scale;
  int rows() const { return R2 * R1 * R0; }
  int K() const { return K2 * K1 * K0; }
};

// Helpers to build views: rows(dim, stride) lists from outermost to innermost.
struct Ax {
  int n;
  long long s;
};
inline View view(const double* p, Ax r2, Ax r1, Ax r0, Ax k2, Ax k1, Ax k0, double scale = 1.0) {
  return View{p, r2.n, r1.n, r0.n, k2.n, k1.n, k0.n, r2.s, r1.s, r0.s, k2.s, k1.s, k0.s, scale};
}
constexpr Ax kOne{1, 0};

// A packed operand: FP64 [rows][Kp] or BF16 [2][rows][Kp] (hi plane, lo plane).
struct Packed {
  void* p = nullptr;
  int rows = 0, Kp = 0;
  bool bf16 = false;
};

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---- kernels (launch wrappers); all enqueue on `s` and do not synchronize
void pack(const View& v, Packed& out, cudaStream_t s);
void pack_rows(const View& v, Packed& full, int row0, cudaStream_t s);
void pack_cols(const View& v, Packed& full, int row0, int col0, int width, cudaStream_t s);
// dst[r*K + k] = view(r, k) + beta * dst[r*K + k]   (FP64, no padding)
void permute(const View& v, double* dst, double beta, cudaStream_t s);
void gemm_f64(const Packed& A, const Packed& B, int M, int N, int K, const OutMap& C, cudaStream_t s);
// C = A A^T in FP64 with the symmetric half computed once and mirrored (A FP64-packed, M rows)
void gemm_f64_sym(const Packed& A, int M, const OutMap& C, cudaStream_t s);
void gemm_tc(const Packed& A, int a_row0, const Packed& B, int b_row0, int M, int N, const OutMap& C,
             cudaStream_t s, int* dstatus);
// rows [a_row0, a_row0 + M) of A against rows [b_row0, b_row0 + N) of B
void gemm_off(const Packed& A, int a_row0, const Packed& B, int b_row0, int M, int N, int K, const OutMap& C,
              cudaStream_t s, int* dstatus);
void gemm_batched(const Packed& A, const Packed& B, const BatchEntry* dbatch, int nbatch, int maxM, int N, int K,
                  const OutMap& C, cudaStream_t s, int* dstatus);
// Two K segments accumulated in one pass: C = A0 B0^T (K0) + A1 B1^T (K1); batched rows from the table.
void gemm2_batched(const Packed& A0, const Packed& B0, const Packed* A1, const Packed* B1, const BatchEntry* dbatch,
                   int nbatch, int maxM, int N, int K0, int K1, const OutMap& C, cudaStream_t s, int* dstatus);
void gemm2_off(const Packed& A0, int a0, const Packed& B0, int b0, int K0, const Packed& A1, int a1, const Packed& B1,
               int b1, int K1, int M, int N, const OutMap& C, cudaStream_t s, int* dstatus);
// dispatch on A.bf16
void gemm(const Packed& A, const Packed& B, int M, int N, int K, const OutMap& C, cudaStream_t s,
          int* dstatus);

// A grouped (T) launch (see grp_tile in gemm.cu): kind 1 = sigma1 + sigma2, sigma3, sigma5 per region
// (c, 128-row tile of (a, x)); kind 2 = sigma4, sigma6 per region (128-row tile of (a, i, x), block of
// cblk c values). Rows: A operands start at the given bases; W chunk offsets advance by Sc per c.
struct GrpSpec {
  int kind;          // 0: not a grouped launch
  int nreg;          // regions
  int mt;            // 128-row tiles per c (kind 1) or per c block (kind 2)
  int Ma;            // valid rows of the problem: (b + 1) o (kind 1) or (b + 1) o^2 (kind 2)
  int nkb;           // K blocks of one term (Kp / 64)
  int c0, nc, cblk;  // the chunk's first c, its number of c, c values per column block (kind 2)
  int ncol;          // kind 1: 256-column tiles per term (o^2 / 256: 1 at nocc 16, 4 at nocc 32)
  int b, bvo, vo, oo, o;  // slab b, b v o, v o, o^2, o
  long long Sc;      // W elements per c in the chunk
};
// Grouped (T) contraction on BF16 hi/lo operands ops[0..3] (box rows 128 for A roles, 256 for B roles)
// with output maps Cg[0..ncg) (alpha 1; beta 0 for the first term of a region, 1 for the others).
void gemm_grouped(const Packed* const ops[4], const int box_rows[4], const GrpSpec& g, const OutMap* Cg, int ncg,
                  cudaStream_t s, int* dstatus);

// Workspace for split-K partials (FP64 elements), provided by the caller of the contraction engine.
// Per host thread: each thread drives its own fragment and stream.
struct SplitWs {
  double* p = nullptr;
  size_t cap = 0;
};
SplitWs& split_ws();

struct GemmStats {
  long long launches = 0;
  double flops = 0.0;
};
GemmStats& gemm_stats();  // per host thread
// Library-wide count of kernel launches issued by the host wrappers (monotonic, all threads), and the
// calling thread's own count (used to count the kernels a captured CUDA graph holds).
std::atomic<long long>& launch_counter();
long long& thread_launch_counter();
// Library-wide count of device allocations made by the library (monotonic, all threads).
std::atomic<long long>& alloc_counter();
inline void count_alloc(long long n = 1) { alloc_counter().fetch_add(n, std::memory_order_relaxed); }
inline void count_launch(long long n = 1) {
  launch_counter().fetch_add(n, std::memory_order_relaxed);
  thread_launch_counter() += n;
}

// Tile autotuner of the tcgen05 GEMM (gemm.cu). mode 0: fixed BN rule; 1: use the table (fixed rule
// on a miss); 2: time the candidates for shapes missing from the table (synchronous; not while the
// stream is being captured). autotune_mode(-1) only reads the mode.
int autotune_mode(int mode);
// Per host thread: false keeps the tuner from timing candidates on this thread (mode 2 then acts as
// mode 1). Timing allocates a scratch output and synchronizes, which callers that must not allocate
// or synchronize cannot allow.
bool& autotune_timing_allowed();
// The library-wide stream-ordered pool of the current device (created on first use, keeps freed memory;
// nullptr if the device cannot create one).
cudaMemPool_t cached_pool();
void autotune_stats(long long out[4]);  // entries, hits, misses, shapes tuned
bool autotune_save(const char* path);
bool autotune_load(const char* path);

void set_error(const std::string& msg);

}  // namespace lnocc

#define LN_CUDA(call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      lnocc::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      return LNOCC_ECUDA;                                                                     \
    }                                                                                         \
  } while (0)
