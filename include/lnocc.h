/*
 * lnocc -- fragment CCSD(T) in a local-natural-orbital active space on one GB300 GPU (sm_103a).
 *
 * The operations follow Ye & Berkelbach, "Periodic Local Coupled-Cluster Theory for Insulators and
 * Metals" (arXiv 2407.11258):
 *   - the fragment Hamiltonian is given by its semi-canonical orbital energies (the diagonal of the
 *     fragment Fock matrix f^(F), Eq. 8) and density-fitted integrals (pq|rs) = sum_Q B_Qpq B_Qrs
 *     (Eq. 15a, Gamma-point real form);
 *   - CCSD is solved in the active space (Sec. II.B, Eq. 7);
 *   - correlation energies are projected onto the fragment's localized occupied orbitals: the CCSD
 *     pair matrix E_ii' (Eq. 7) and the (T) pair matrix E_ii',(T) (Eq. 10, intermediates of the
 *     supplementary Sec. S1), contracted as E^(F) = sum_{alpha in F} sum_ii' U_i,alpha E_ii' U_i',alpha
 *     (Eq. 6 and Eq. 9).
 *
 * Conventions for every entry point
 *   - Return value: LNOCC_OK (0) or one of the LNOCC_E* codes below; the message of the last failure on
 *     the calling thread is available from lnocc_last_error().
 *   - Array arguments are DEVICE pointers to FP64, C-contiguous, owned by the caller. The library never
 *     frees them and copies whatever it keeps. Energies are returned through HOST pointers.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is enqueued on it; calls that
 *     return energies synchronize that stream before returning.
 *   - Orbital order: occupied first (nocc), then virtual (nvir); n = nocc + nvir.
 *   - Amplitudes: t1[i][a] = t_i^a (nocc x nvir); t2[i][j][a][b] = t_ij^ab (nocc^2 x nvir^2), which is
 *     the paper's t_iajb (virtual a pairs with occupied i, b with j); t_ij^ab = t_ji^ba.
 *   - The library allocates device memory only inside lnocc_build_ints (held by the handle).
 */
#ifndef LNOCC_H
#define LNOCC_H

#ifdef __cplusplus
extern "C" {
#endif

#define LNOCC_OK 0
#define LNOCC_EINVAL 1   /* bad argument (size, pointer, option) */
#define LNOCC_ENOMEM 2   /* device allocation failed */
#define LNOCC_ENOCONV 3  /* CCSD did not converge within max_iter (last energy is still returned) */
#define LNOCC_ENUMERIC 4 /* NaN/Inf in a residual or energy, or a non-positive denominator */
#define LNOCC_ETIMEOUT 5 /* a bounded device-side wait ran out; results are invalid */
#define LNOCC_ECUDA 6    /* a CUDA runtime call failed */

#define LNOCC_PREC_FP64 0  /* every contraction in FP64 (plain GPU path) */
#define LNOCC_PREC_MIXED 1 /* contractions as BF16x3 products with FP32 accumulation (tcgen05) */

#define LNOCC_GUESS_MP2 0   /* t1 = 0, t2 = first-order amplitudes (Eq. 11, canonical form) */
#define LNOCC_GUESS_GIVEN 1 /* start from t1_in / t2_in (restart / checkpoint resume) */

#define LNOCC_FAULT_NAN_INPUT 1 /* fault injection (host side): poison one element of the B copy */
#define LNOCC_FAULT_ZERO_DIIS 2 /* fault injection: run without DIIS extrapolation */

typedef struct lnocc_frag lnocc_frag; /* opaque: integrals, amplitudes and workspace of one fragment */

typedef struct lnocc_opts {
  int precision;      /* LNOCC_PREC_FP64 or LNOCC_PREC_MIXED */
  int max_iter;       /* CCSD iteration cap (default 100) */
  int diis_space;     /* Pulay DIIS vectors, 0..8 (default 8) */
  int n_refine;       /* mixed only: CCSD iterations with an FP64 residual after mixed convergence */
  double conv_rms;    /* convergence: rms of the doubles update |R/D| below this (default 1e-8) */
  double conv_energy; /* convergence: |E_k - E_k-1| below this (default 1e-10 Eh) */
  int fault_inject;   /* LNOCC_FAULT_* bitmask, 0 in production */
  int verbose;        /* 1: print one line per iteration to stderr */
  int reserved[6];
} lnocc_opts;

typedef struct lnocc_info {
  int nocc, nvir, naux, precision;
  int n_iter;              /* CCSD iterations of the last lnocc_ccsd call */
  int converged;           /* 1 when the last solve met both thresholds */
  double e_mp2;            /* MP2 correlation energy (iteration 0) */
  double e_ccsd;           /* CCSD correlation energy of the last solve */
  double last_rms;         /* rms doubles update of the last iteration */
  double model_flops_ccsd; /* 2 o^2 v^4 + 16 o^3 v^3 + 2 o^4 v^2 per iteration, times n_iter */
  double model_flops_t;    /* 6 o^3 v^4 + 6 o^4 v^3 */
  double exec_flops;       /* contraction flops issued since build (BF16x3 counted once per product) */
  long long gemm_launches; /* contraction kernel launches since build */
  long long device_bytes;  /* device memory held by the handle */
  long long kernel_launches; /* library-wide count of kernel launches so far (monotonic) */
  double t_triples_gemm_ms;  /* last lnocc_triples: device time of its contraction launches (CUDA events) */
  double t_triples_ms;       /* last lnocc_triples: device time of the whole call (CUDA events) */
} lnocc_info;

/* Fill `opts` with the defaults listed above (precision = LNOCC_PREC_MIXED). */
void lnocc_default_opts(lnocc_opts* opts);

/*
 * lnocc_build_ints -- integral assembly for one fragment (Sec. II.D item 2, Eq. 15a at the Gamma point).
 *   nocc, nvir, naux : active occupied, virtual and auxiliary dimensions (nocc >= 1, nvir >= 1, naux >= 1).
 *   eps  [n]         : orbital energies (the fragment Fock diagonal); every virtual must lie above every
 *                      occupied (else LNOCC_ENUMERIC: the (T) denominators of Sec. S1 need -Delta > 0).
 *   B    [naux][n][n]: real DF factors, symmetric in the last two indices; (pq|rs) = sum_Q B_Qpq B_Qrs.
 *   opts             : may be NULL for defaults; copied.
 *   out              : receives the new handle (free with lnocc_free_fragment).
 * Slices B, assembles the constant ERI blocks the solver needs -- (ia|jb), (ij|ab)-type blocks, the
 * (ia|bc) block and the packed (ac|bd) +/- combinations of the particle-particle ladder -- in FP64 or
 * as BF16 hi/lo pairs, and allocates all workspace. Synchronizes `stream`.
 */
int lnocc_build_ints(int nocc, int nvir, int naux, const double* eps, const double* B, const lnocc_opts* opts,
                     void* stream, lnocc_frag** out);

/*
 * lnocc_ccsd -- closed-shell CCSD amplitude equations in the fragment active space (Sec. II.B, Eq. 7;
 * the paper solves canonical CCSD with H^(F); the spin-adapted equations are the T1-transformed
 * closed-shell form of Koch et al., Chem. Phys. Lett. 228, 233 (1994)).
 *   t1_in [o][v], t2_in [o][o][v][v] : starting amplitudes when guess_mode == LNOCC_GUESS_GIVEN, else
 *                                      ignored (may be NULL).
 *   t1_out, t2_out                    : optional (NULL allowed) copies of the converged amplitudes.
 *   e_corr (host)                     : E_c = sum_ijab tau_ij^ab [2(ia|jb) - (ib|ja)], tau = t2 + t1 t1
 *                                       (Eq. 5; the printed minus sign is read as +).
 *   n_iter (host, may be NULL)        : iterations taken.
 * The converged amplitudes stay in the handle for lnocc_triples / lnocc_fragment_energy. The same
 * convergence test applies to every guess mode. Returns LNOCC_ENOCONV (with the last energy) when
 * max_iter is reached, LNOCC_ENUMERIC on NaN/Inf.
 */
int lnocc_ccsd(lnocc_frag* f, const double* t1_in, const double* t2_in, int guess_mode, double* t1_out,
               double* t2_out, double* e_corr, int* n_iter, void* stream);

/*
 * lnocc_fragment_energy -- projected CCSD and MP2 fragment energies (Eq. 6-7).
 *   nlo, U_frag [nocc][nlo] : the fragment's LO coefficients in the occupied space (columns alpha in F).
 *   e_ccsd_frag (host)      : sum_alpha sum_ii' U_i,alpha E_ii' U_i',alpha with the CCSD pair matrix
 *                             E_ii' = sum_jab tau_ij^ab [2(i'a|jb) - (i'b|ja)] of the last lnocc_ccsd.
 *   e_mp2_frag (host)       : the same contraction with the first-order amplitudes (t1 = 0).
 * Either output may be NULL. Requires a preceding successful lnocc_ccsd for e_ccsd_frag.
 */
int lnocc_fragment_energy(lnocc_frag* f, int nlo, const double* U_frag, double* e_ccsd_frag, double* e_mp2_frag,
                          void* stream);

/*
 * lnocc_triples -- LNO-(T) energy (Eq. 9-10 with the intermediates W, V, w, v of supplementary Sec. S1)
 * from the amplitudes of the last lnocc_ccsd.
 *   nlo, U_frag [nocc][nlo] : fragment LO coefficients; U_frag == NULL (or nlo == 0) skips projection.
 *   e_t_full (host)         : canonical (T) energy, the trace of the (T) pair matrix (full active space).
 *   e_t_frag (host)         : sum_alpha sum_ii' U_i,alpha E_ii',(T) U_i',alpha (may be NULL).
 * FP64 precision: FP64 contractions. Mixed precision: W and V contractions as BF16x3/FP32 on tensor
 * cores, denominators, square roots, products and the energy sum in FP64.
 */
int lnocc_triples(lnocc_frag* f, int nlo, const double* U_frag, double* e_t_full, double* e_t_frag,
                  void* stream);

/*
 * lnocc_debug_gemm -- diagnostic: C[M][N] = A[M][K] B[N][K]^T through the library's contraction engine
 * (operand packing + FP64 SIMT GEMM, or BF16x3 tcgen05 GEMM with FP32 accumulation). Device pointers,
 * row-major FP64. Allocates its own temporaries and synchronizes `stream`. Not part of the method; it
 * lets the contraction kernels be checked on their own.
 */
int lnocc_debug_gemm(int precision, int M, int N, int K, const double* A, const double* B, double* C, void* stream);

/*
 * lnocc_gemm_noalloc -- C[M][N] = A[M][K] B[N][K]^T like lnocc_debug_gemm, but without allocating device
 * memory. The paper has no counterpart: this serves callers that cannot call cudaMalloc -- code running
 * under a fixed device-memory budget owned by another allocator, or code that must not synchronize the
 * device, which cudaMalloc / cudaFree can do.
 *   Working memory is a file-scope __device__ array of 32 MiB that every GPU loading the library holds until
 *   the process exits; the packed operands need (M + N) * roundup(K, 64) * (8 bytes FP64 | 4 bytes mixed)
 *   plus 256 bytes, and larger requests return LNOCC_EINVAL before any device work.
 *   The first call on a device looks up that array's device address (cudaGetSymbolAddress, with the device
 *   current); make that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents: calls that overlap on the GPU (other
 *   streams, other host threads) race on it. The call synchronizes `stream` before it returns.
 *   Device pointers, row-major FP64; precision LNOCC_PREC_FP64 or LNOCC_PREC_MIXED.
 */
int lnocc_gemm_noalloc(int precision, int M, int N, int K, const double* A, const double* B, double* C, void* stream);

/* Copy the handle's bookkeeping (energies, iteration count, flop counters) into *info. */
int lnocc_frag_info(const lnocc_frag* f, lnocc_info* info);

/* Release everything the handle holds (safe on NULL). */
int lnocc_free_fragment(lnocc_frag* f);

/* Message of the last failing call on this thread ("" when none). */
const char* lnocc_last_error(void);

/* Library version string. */
const char* lnocc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LNOCC_H */
