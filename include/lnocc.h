/*
 * lnocc -- fragment CCSD(T) in a local-natural-orbital active space on one GB300 GPU (sm_103a).
 *
 * The operations follow Ye & Berkelbach, "Periodic Local Coupled-Cluster Theory for Insulators and
 * Metals" (arXiv 2407.11258):
 *   - the fragment Hamiltonian is given by its semi-canonical orbital energies (the diagonal of the
 *     fragment Fock matrix f^(F), Eq. 11) and density-fitted integrals (pq|rs) = sum_Q B_Qpq B_Qrs
 *     (Eq. 27a, Gamma-point real form);
 *   - CCSD is solved in the active space (Sec. II.B, Eq. 10-11);
 *   - correlation energies are projected onto the fragment's localized occupied orbitals: the CCSD
 *     pair matrix E_ii' (Eq. 13) and the (T) pair matrix E_ii',(T) (Eq. 16, intermediates of the
 *     supplementary Sec. S1), contracted as E^(F) = sum_{alpha in F} sum_ii' U_i,alpha E_ii' U_i',alpha
 *     (Eq. 12 and Eq. 15).
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
 *   - Device memory is allocated by lnocc_build_ints (held by the handle until lnocc_free_fragment).
 *     lnocc_ccsd and lnocc_fragment_energy allocate nothing. lnocc_triples needs temporaries of
 *     lnocc_workspace_bytes(...) bytes: from a workspace the caller attached with lnocc_frag_set_workspace
 *     (then it allocates nothing), else it allocates and frees them itself within the call. The other
 *     allocating calls say so (the diagnostic GEMM, the batch runtime, MLP handles, autotuner mode 2).
 *     A handle's allocations come from the library's cached stream-ordered pool (opts.memory, default
 *     LNOCC_MEM_CACHED), which keeps freed memory for later handles; lnocc_trim_pool returns it.
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

#define LNOCC_GUESS_MP2 0   /* t1 = 0, t2 = first-order amplitudes (Eq. 21, canonical form) */
#define LNOCC_GUESS_GIVEN 1 /* start from t1_in / t2_in (restart / checkpoint resume) */
#define LNOCC_GUESS_MLP 2   /* t1 = 0, t2 = learned guess of the model attached by lnocc_frag_set_mlp */

/* (T) contraction launches on the mixed path. PER_TERM: one launch per W term (sigma1 + sigma2, sigma3,
 * sigma4, sigma6, sigma5) per chunk. GROUPED: two launches per chunk; the first runs sigma1 + sigma2,
 * sigma3 and sigma5 of one (c, 128-row tile of (a, x)) block back to back in one CTA (the block stays
 * in L2 between its store and its two reductions), the second sigma4 and sigma6. GROUPED needs
 * nocc = 16 or 32 (128 rows hold whole a values; the (y, z) plane is one or four 256-column
 * accumulator tiles); AUTO takes it there and PER_TERM elsewhere, and GROUPED falls back to PER_TERM
 * for other nocc. */
#define LNOCC_TK_AUTO 0
#define LNOCC_TK_PER_TERM 1
#define LNOCC_TK_GROUPED 2

/* Device memory of a handle (and of its lnocc_triples temporaries). CACHED: stream-ordered allocations
 * from one library-wide pool per device that keeps freed memory for later handles (no cudaMalloc /
 * cudaFree, and no device synchronisation, once the pool holds enough; lnocc_trim_pool returns the
 * unused part to the device). DIRECT: cudaMalloc / cudaFree per buffer. */
#define LNOCC_MEM_CACHED 0
#define LNOCC_MEM_DIRECT 1

#define LNOCC_FAULT_NAN_INPUT 1 /* fault injection (host side): poison one element of the B copy */
#define LNOCC_FAULT_ZERO_DIIS 2 /* fault injection: run without DIIS extrapolation */

typedef struct lnocc_frag lnocc_frag; /* opaque: integrals, amplitudes and workspace of one fragment */

typedef struct lnocc_opts {
  int precision;      /* LNOCC_PREC_FP64 or LNOCC_PREC_MIXED */
  int max_iter;       /* CCSD iteration cap (default 100) */
  int diis_space;     /* Pulay DIIS vectors, 0..8 (default 8) */
  int n_refine;       /* mixed only: at most this many FP64-residual CCSD iterations, run only when the
                         mixed solve reaches its noise floor with an energy spread above 1e-7 Eh (they
                         continue from the lowest-rms amplitudes until rms < conv_rms and
                         |dE| < max(conv_energy, 1e-8) Eh); 0 (default):
                         such a solve returns LNOCC_ENOCONV with the energy of those amplitudes. Needs
                         the FP64 operands, built by lnocc_build_ints when n_refine > 0 */
  double conv_rms;    /* convergence: rms of the doubles update |R/D| below this (default 1e-8) */
  double conv_energy; /* convergence: |E_k - E_k-1| below this (default 1e-10 Eh) */
  int fault_inject;   /* LNOCC_FAULT_* bitmask, 0 in production */
  int verbose;        /* 1: print one line per iteration to stderr */
  int graph;          /* 1 (default): after the first iteration, replay each CCSD iteration from a CUDA
                         graph captured once per fragment (same kernels, same results; fewer host launches) */
  int triples_chunk_mb; /* bound on the W chunk of lnocc_triples in MB (0, the default: 768); part of the
                           workspace size that lnocc_workspace_bytes reports */
  int triples_kernel;   /* (T) contraction launches on the mixed path: LNOCC_TK_AUTO (0, the default),
                           LNOCC_TK_PER_TERM or LNOCC_TK_GROUPED (same W, same energy) */
  int memory;           /* LNOCC_MEM_CACHED (0, the default) or LNOCC_MEM_DIRECT (see their definitions) */
  int reserved[2];
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
  long long device_allocs;   /* library-wide count of device allocations made so far (monotonic) */
  double floor_spread;       /* mixed: CCSD energy spread (Eh) over the last iterations when the noise floor
                                was reached (0 if the FP64 thresholds were met first) */
  int n_refined;             /* mixed: FP64-residual iterations the last solve ran (see opts.n_refine) */
  int diis_restarts;         /* mixed: DIIS subspace restarts from the lowest-rms amplitudes */
} lnocc_info;

/* Fill `opts` with the defaults listed above (precision = LNOCC_PREC_MIXED). */
void lnocc_default_opts(lnocc_opts* opts);

/*
 * lnocc_build_ints -- integral assembly for one fragment (Sec. II.D item 2, Eq. 27a at the Gamma point).
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
 * lnocc_ccsd -- closed-shell CCSD amplitude equations in the fragment active space (Sec. II.B, Eq. 10-11;
 * the paper solves canonical CCSD with H^(F); the spin-adapted equations are the T1-transformed
 * closed-shell form of Koch et al., Chem. Phys. Lett. 228, 233 (1994)).
 *   t1_in [o][v], t2_in [o][o][v][v] : starting amplitudes when guess_mode == LNOCC_GUESS_GIVEN, else
 *                                      ignored (may be NULL).
 *   t1_out, t2_out                    : optional (NULL allowed) copies of the converged amplitudes.
 *   e_corr (host)                     : E_c = sum_ijab tau_ij^ab [2(ia|jb) - (ib|ja)], tau = t2 + t1 t1
 *                                       (Eq. 7; the printed minus sign is read as +).
 *   n_iter (host, may be NULL)        : iterations taken.
 * The converged amplitudes stay in the handle for lnocc_triples / lnocc_fragment_energy. The same
 * convergence test applies to every guess mode. Returns LNOCC_ENOCONV (with the last energy) when
 * max_iter is reached, LNOCC_ENUMERIC on NaN/Inf.
 * LNOCC_GUESS_MLP falls back to the MP2 guess when the learned guess has a non-finite element, and
 * repeats the solve from the MP2 guess when the run from the learned guess ends in ENOCONV or
 * ENUMERIC (n_iter then counts both runs).
 */
int lnocc_ccsd(lnocc_frag* f, const double* t1_in, const double* t2_in, int guess_mode, double* t1_out,
               double* t2_out, double* e_corr, int* n_iter, void* stream);

/*
 * lnocc_fragment_energy -- projected CCSD and MP2 fragment energies (Eq. 12-13).
 *   nlo, U_frag [nocc][nlo] : the fragment's LO coefficients in the occupied space (columns alpha in F).
 *   e_ccsd_frag (host)      : sum_alpha sum_ii' U_i,alpha E_ii' U_i',alpha with the CCSD pair matrix
 *                             E_ii' = sum_jab tau_ij^ab [2(i'a|jb) - (i'b|ja)] of the last lnocc_ccsd.
 *   e_mp2_frag (host)       : the same contraction with the first-order amplitudes (t1 = 0).
 * Either output may be NULL. Requires a preceding successful lnocc_ccsd for e_ccsd_frag.
 */
int lnocc_fragment_energy(lnocc_frag* f, int nlo, const double* U_frag, double* e_ccsd_frag, double* e_mp2_frag,
                          void* stream);

/*
 * lnocc_triples -- LNO-(T) energy (Eq. 15-16 with the intermediates W, V, w, v of supplementary Sec. S1)
 * from the amplitudes of the last lnocc_ccsd.
 *   nlo, U_frag [nocc][nlo] : fragment LO coefficients; U_frag == NULL (or nlo == 0) skips projection.
 *   e_t_full (host)         : canonical (T) energy, the trace of the (T) pair matrix (full active space).
 *   e_t_frag (host)         : sum_alpha sum_ii' U_i,alpha E_ii',(T) U_i',alpha (may be NULL).
 * FP64 precision: FP64 contractions and energy arithmetic. Mixed precision: the W contractions as
 * BF16x3/FP32 on tensor cores; the denominators' terms formed in FP64, the scaled w and v, their
 * products and the i-sums in FP32; a block's partials summed in compensated FP32 (the rounding error
 * of every addition carried alongside, both converted to FP64 once per block) by the staged kernels,
 * in FP64 by the generic one; the sums over blocks and the total in FP64.
 * Any nocc and any number of LOs (up to 8 LOs and while a block of the (T) energy fits shared memory the
 * staged energy kernels run; otherwise a generic kernel that stages nothing).
 * Temporaries (the packed (T) operands, a W chunk of at most opts.triples_chunk_mb or one b-slab, the
 * per-block partial sums, the launch tables and the padded U) come from the attached workspace
 * (lnocc_frag_set_workspace; LNOCC_EINVAL if it is smaller than lnocc_workspace_bytes), or else are
 * allocated in the fragment's memory mode and freed before the call returns (LNOCC_ENOMEM when they do
 * not fit). Synchronizes `stream`.
 */
int lnocc_triples(lnocc_frag* f, int nlo, const double* U_frag, double* e_t_full, double* e_t_frag,
                  void* stream);

/*
 * Graph-capturable forms (device-pointer outputs). They enqueue the same work on `stream` as
 * lnocc_fragment_energy / lnocc_triples and return without synchronising: no host-side wait, no
 * timing events, no device allocation, no tile timing. The results are written to DEVICE memory when
 * the stream reaches them, so either call may be captured into a CUDA graph (stream capture) and
 * replayed; the handle's amplitudes are read when the work runs.
 *   lnocc_fragment_energy_device: e_dev[0] = E_CCSD^(F), e_dev[1] = E_MP2^(F) (Eq. 12-13).
 *   lnocc_triples_device: needs a workspace attached with lnocc_frag_set_workspace (LNOCC_EINVAL
 *     otherwise); e_dev[0] = E_(T), e_dev[1] = E_(T)^(F) (0 when U_frag is NULL); status_dev (device
 *     int, may be NULL) receives the device status word of the call: 0, or a nonzero code when a bounded
 *     wait of a contraction kernel ran out (the host-synchronous call reports that as LNOCC_ETIMEOUT).
 * Argument errors are reported at enqueue time as by the synchronous calls; a non-finite energy is
 * not checked (it is in e_dev).
 */
int lnocc_fragment_energy_device(lnocc_frag* f, int nlo, const double* U_frag, double* e_dev, void* stream);
int lnocc_triples_device(lnocc_frag* f, int nlo, const double* U_frag, double* e_dev, int* status_dev,
                         void* stream);

/*
 * lnocc_workspace_bytes -- device scratch that lnocc_triples needs for a fragment of these sizes
 * (Sec. II.D's (T) step: packed W/V operands, the W chunk and the block partial sums), for the precision
 * and opts->triples_chunk_mb of `opts` (NULL: defaults). *bytes receives the size.
 */
int lnocc_workspace_bytes(int nocc, int nvir, int naux, const lnocc_opts* opts, long long* bytes);

/*
 * lnocc_frag_set_workspace -- attach caller-owned device memory (at least lnocc_workspace_bytes bytes for
 * the fragment's sizes and options, else LNOCC_EINVAL) from which lnocc_triples takes its temporaries, so
 * that no call after lnocc_build_ints allocates. The caller keeps ownership; the memory must stay valid
 * while attached and must not be used by other work during lnocc_triples. NULL detaches.
 */
int lnocc_frag_set_workspace(lnocc_frag* f, void* workspace, long long workspace_bytes);

/*
 * lnocc_debug_gemm -- diagnostic: C[M][N] = A[M][K] B[N][K]^T through the library's contraction engine
 * (operand packing + FP64 SIMT GEMM, or BF16x3 tcgen05 GEMM with FP32 accumulation). Device pointers,
 * row-major FP64. Allocates its own temporaries and synchronizes `stream`. Not part of the method; it
 * lets the contraction kernels be checked on their own.
 */
int lnocc_debug_gemm(int precision, int M, int N, int K, const double* A, const double* B, double* C, void* stream);

/*
 * lnocc_debug_wait -- diagnostic of the bounded device wait that every mbarrier wait in the library uses:
 * a one-thread kernel waits for the first phase of an mbarrier with a wall-clock budget of budget_ns
 * (0 .. 2e9 ns; the library's own waits use 2 s). arrive != 0 arrives first (the wait succeeds: LNOCC_OK);
 * arrive == 0 lets nothing arrive, the budget runs out and the call returns LNOCC_ETIMEOUT with the context
 * intact. *waited_ns (host, may be NULL) receives the time the kernel spent waiting. Not part of the
 * method (the paper has no device code); allocates 16 bytes and synchronizes `stream`.
 */
int lnocc_debug_wait(int arrive, long long budget_ns, long long* waited_ns, void* stream);

/*
 * lnocc_gemm_noalloc -- C[M][N] = A[M][K] B[N][K]^T like lnocc_debug_gemm, but without allocating device
 * memory. The paper has no counterpart: this serves callers that cannot call cudaMalloc -- code running
 * under a fixed device-memory budget owned by another allocator, or code that must not synchronize the
 * device, which cudaMalloc / cudaFree can do.
 *   Working memory is a file-scope __device__ array of 32 MiB that every GPU loading the library holds until
 *   the process exits; the packed operands need (M + N) * roundup(K, 64) * (8 bytes FP64 | 4 bytes mixed)
 *   plus 256 bytes, and larger requests return LNOCC_EINVAL before any device work.
 *   The first call on a device looks up that array's device address (cudaGetSymbolAddress, with the device
 *   current); make that first call before any stream capture. With CUDA's default lazy module loading the
 *   array is only placed in device memory at that first call, so make it before another allocator claims
 *   the free memory (from then on the array stays put).
 *   The tile autotuner only looks its table up here: in mode 2 (lnocc_autotune) a table miss falls back
 *   to the fixed rule instead of timing candidates, which would allocate and synchronize.
 *   All calls share the array and it keeps the last call's contents: calls that overlap on the GPU (other
 *   streams, other host threads) race on it. The call synchronizes `stream` before it returns.
 *   Device pointers, row-major FP64; precision LNOCC_PREC_FP64 or LNOCC_PREC_MIXED.
 */
int lnocc_gemm_noalloc(int precision, int M, int N, int K, const double* A, const double* B, double* C, void* stream);

/*
 * lnocc_mp2_energy -- canonical closed-shell MP2 correlation energy of the whole system, the first term of
 * the MP2 composite correction (Eq. 17): Delta E_c,MP2 = E_c,MP2 - sum_F E_c,MP2^(F), whose fragment terms
 * are the e_mp2_frag of lnocc_fragment_energy (Eq. 12-13 with the first-order amplitudes of Eq. 21).
 *   E_c,MP2 = sum_ijab (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b), (ia|jb) = sum_Q B_Qia B_Qjb.
 *   precision          : LNOCC_PREC_FP64 (FP64 contraction) or LNOCC_PREC_MIXED ((ia|jb) as BF16x3 products
 *                        with FP32 accumulation); denominators, products and sums in FP64 on both.
 *   nocc, nvir, naux   : the system's occupied, virtual and auxiliary dimensions (nocc * nvir <= 2^30).
 *   eps [nocc + nvir]  : canonical orbital energies (device), occupied first; every virtual above every occupied.
 *   B_ov [naux][nocc][nvir] : the occupied-virtual block of the DF factors (device).
 *   workspace, workspace_bytes : caller-owned device scratch of at least lnocc_mp2_workspace_bytes(...) bytes,
 *                        or NULL (the call then allocates and frees its own); LNOCC_EINVAL when too small.
 *   e_mp2 (host)       : the energy (Eh).
 * The sum over blocks is taken in a fixed order (repeatable bit for bit). Synchronizes `stream`.
 */
int lnocc_mp2_workspace_bytes(int precision, int nocc, int nvir, int naux, long long* bytes);
int lnocc_mp2_energy(int precision, int nocc, int nvir, int naux, const double* eps, const double* B_ov,
                     void* workspace, long long workspace_bytes, double* e_mp2, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Local active space of a fragment (Sec. II.C; CBNOs of Sec. II.E). For a fragment F with LO coefficients
 * U^(F) in the canonical occupied (and, for LOs that overlap the virtual space, virtual) orbitals of the
 * system: the internal orbitals (Eq. 18-19), the MP2 densities that rank the external orbitals (Eq. 20 or
 * Eq. 28, from the MP1 amplitudes of Eq. 21 with the DF integrals of Eq. 22 at the Gamma point), the LNOs
 * kept by the thresholds of Eq. 24-26, and the semi-canonical active space with its DF factors, which is
 * the input of lnocc_build_ints. Real orbitals; all arrays are device FP64, row-major. Each call allocates
 * its own temporaries and synchronizes `stream`.
 * ---------------------------------------------------------------------------------------------- */
#define LNOCC_LNO_MP2 0  /* Eq. 20: one occupied index of the MP2 density restricted to the internal space */
#define LNOCC_LNO_CBNO 1 /* Eq. 28: both virtual (occupied block) / both occupied (virtual block) internal */

/*
 * lnocc_lno_internal -- Eq. 18-19 for one block (occupied or virtual): the left singular vectors of
 * U [n][nlo] with singular value above sv_tol times the largest (0 < sv_tol < 1; 1e-10 is a good choice)
 * span the internal space; they are returned semi-canonical: the block Fock matrix (diagonal e [n] in
 * the canonical basis) is diagonalised inside the internal space, f_int [nlo] receives its eigenvalues
 * in increasing order (first *n_int used) and W_int [n][nlo] the orbitals as columns (first *n_int used,
 * the rest zero). 1 <= nlo <= 256. *n_int (host) is the internal dimension.
 */
int lnocc_lno_internal(int n, int nlo, const double* U, const double* e, double sv_tol, double* W_int, double* f_int,
                       int* n_int, void* stream);

/*
 * lnocc_lno_densities -- the occupied block D_occ [nocc][nocc] and virtual block D_vir [nvir][nvir] of the
 * MP2 density used to rank the external orbitals of fragment F:
 *   kind LNOCC_LNO_MP2 (Eq. 20):  D_ij = 2 sum_kF sum_ab t_{iakFb} (2 t_{jakFb} - t_{jbkFa}),
 *     D_ab = sum_iF sum_jc 2 (t_{iFajc} t_{iFbjc} + t_{iFcja} t_{iFcjb}) - (t_{iFcja} t_{iFbjc} + t_{iFajc} t_{iFcjb});
 *   kind LNOCC_LNO_CBNO (Eq. 28): D_ij = 2 sum_{aF bF} sum_k t_{iaFkbF} (2 t_{jaFkbF} - t_{jbFkaF}),
 *     D_ab = 2 sum_{iF jF} sum_c t_{iFajFc} (2 t_{iFbjFc} - t_{iFcjFb}) (n_iv = 0 gives D_occ = 0);
 * with t_{pa qb} = (pa|qb) / (f_p + f_q - f_a - f_b), (ia|jb) = sum_Q B_Qia B_Qjb, canonical energies eps
 * [nocc + nvir] for canonical orbitals and f_occ / f_vir for the internal ones W_occ [nocc][n_io] /
 * W_vir [nvir][n_iv] (semi-canonical, as lnocc_lno_internal returns them, leading dimension n_io / n_iv).
 *   B_ov [naux][nocc][nvir] : the system's occupied-virtual DF block.
 *   precision : LNOCC_PREC_MIXED contracts as BF16x3 products with FP32 accumulation, LNOCC_PREC_FP64 in FP64;
 *               amplitudes, denominators and the outputs are FP64. Both blocks are returned symmetric.
 */
int lnocc_lno_densities(int precision, int kind, int nocc, int nvir, int naux, const double* eps, const double* B_ov,
                        int n_io, const double* W_occ, const double* f_occ, int n_iv, const double* W_vir,
                        const double* f_vir, double* D_occ, double* D_vir, void* stream);

/*
 * lnocc_lno_select -- Eq. 24-26: the density D [n][n] restricted to the external space (the complement of
 * the n_int columns of W_int [n][n_int], orthonormal; n_int = 0 keeps the whole space) is diagonalised and the
 * eigenpairs with |lambda| >= eta are kept, in decreasing order of lambda: C [n][n] receives the LNOs as its
 * first *n_keep columns (the rest zero) and lambda [n] their eigenvalues (the rest zero). The projection is
 * P D P with P = 1 - W_int W_int^T, whose eigenvectors of non-zero eigenvalue are the W_bar X of Eq. 25.
 * 1 <= n <= 8192; FP64 Jacobi eigendecomposition on the device.
 */
int lnocc_lno_select(int n, const double* D, int n_int, const double* W_int, double eta, double* C, double* lambda,
                     int* n_keep, void* stream);

/*
 * lnocc_active_space -- the fragment's active space in semi-canonical form and its DF factors: the occupied
 * orbitals C_occ [nocc][no_F] and virtual orbitals C_vir [nvir][nv_F] (orthonormal columns, e.g. internal and
 * kept LNOs) are rotated so that the Fock matrix (diagonal eps [nocc + nvir] in the canonical basis) is
 * diagonal inside each block; eps_F [no_F + nv_F] receives the orbital energies (occupied, then virtual,
 * each increasing) and B_F [naux][nF][nF] (nF = no_F + nv_F) the DF factors C_F^T B[Q] C_F of the system's
 * B [naux][n][n] (the Gamma-point real form of Eq. 27). C_F [n][nF] (may be NULL) receives the rotated
 * orbitals (block diagonal: occupied rows and columns first); a fragment's LO matrix in the active occupied
 * basis is then C_F[:nocc, :no_F]^T U^(F). precision as for lnocc_lno_densities.
 */
int lnocc_active_space(int precision, int nocc, int nvir, int naux, const double* eps, const double* B, int no_F,
                       const double* C_occ, int nv_F, const double* C_vir, double* eps_F, double* B_F, double* C_F,
                       void* stream);

/*
 * lnocc_kpoint_df -- integrals of the local Hamiltonian from k-point DF factors (Eq. 27a),
 * V_pqrs = sum_q sum_P L^P_pq(q) L^P_rs(-q), reduced to the real form (pq|rs) = sum_Q B_Qpq B_Qrs that
 * lnocc_build_ints takes.
 *   L [nk][naux][n][n] : complex factors (device, interleaved real/imaginary FP64) of the nk momentum
 *                        transfers q in the basis of the n active orbitals (real orbitals: L_pq(q) = L_qp(q),
 *                        L(-q) = conj L(q); checked, LNOCC_EINVAL beyond 1e-10 of max |L|).
 *   qneg [nk] (host)   : index of -q for each q (an involution).
 *   B_out [nk * naux][n][n] (device) : sqrt(2) Re L(q) and sqrt(2) Im L(q) for one q of each pair (q, -q),
 *                        Re L(q) for each self-conjugate q, in increasing q: sum_Q B_Qpq B_Qrs equals V_pqrs.
 *   sym_err (host, may be NULL) : the largest symmetry deviation relative to max |L|.
 * Allocates a small table and synchronizes `stream`.
 */
int lnocc_kpoint_df(int nk, int naux, int n, const double* L, const int* qneg, double* B_out, double* sym_err,
                    void* stream);

/* ------------------------------------------------------------------------------------------------
 * Batched fragments.
 *
 * The total correlation energy is a sum of fragment contributions (Eq. ecorr_cc, Sec. 2.2) and each
 * fragment's local CCSD(T) uses only that fragment's active-space integrals, so the fragments of a
 * calculation are independent problems. lnocc_solve_batch runs many of them -- of uneven
 * (nocc, nvir, naux) -- on one GPU: longest-processing-time-first order on a flop cost model,
 * `workers` concurrent pipelines (one host thread and one stream each) admitted under a device-memory
 * budget, one stream-ordered memory pool for all fragment buffers, and each fragment's CCSD iterations
 * replayed from a captured CUDA graph (opts->graph). Every fragment goes through exactly the same
 * build / CCSD / fragment-energy / (T) code as the single-fragment calls with the same opts, so its
 * energies equal those of lnocc_build_ints + lnocc_ccsd + lnocc_fragment_energy + lnocc_triples.
 * ---------------------------------------------------------------------------------------------- */
#define LNOCC_ORDER_LPT 0   /* longest processing time first (default) */
#define LNOCC_ORDER_INPUT 1 /* the order of items[] */

typedef struct lnocc_batch_item {
  int nocc, nvir, naux; /* sizes of this fragment's active space */
  int nlo;              /* columns of U_frag (0: canonical energies only, no projection) */
  const double* eps;    /* device [nocc+nvir], occupied then virtual, every virtual above every occupied */
  const double* B;      /* device [naux][n][n], symmetric in (p, q) */
  const double* U_frag; /* device [nocc][nlo] fragment LO coefficients, or NULL when nlo == 0 */
} lnocc_batch_item;

typedef struct lnocc_batch_opts {
  int workers;          /* concurrent fragment pipelines, 1..16 (0: 3) */
  int triples;          /* 1 (default): (T) after CCSD */
  int order;            /* LNOCC_ORDER_* */
  int autotune;         /* 0: tiles as the library's autotune mode says (lnocc_autotune); 1: first time the
                           GEMM tile candidates on up to 5 representative fragments (cost quantiles), then
                           use the table for the batch; 2: use the loaded table only */
  double mem_budget_gb; /* device memory the batch may hold at once, 1e9 bytes (0: 90% of free memory) */
  int reserved[8];
} lnocc_batch_opts;

typedef struct lnocc_batch_result {
  int status;           /* LNOCC_* of this fragment; ENOCONV keeps the last energies */
  int n_iter;           /* CCSD iterations */
  int worker;           /* pipeline that solved it */
  int order;            /* position in which it was started */
  double e_mp2, e_ccsd, e_mp2_frag, e_ccsd_frag, e_t, e_t_frag; /* Eh; *_frag are 0 when nlo == 0 */
  double t_start_ms, t_end_ms; /* host wall clock since the start of the batch */
  double model_flops;   /* (2o^2v^4 + 16o^3v^3 + 2o^4v^2) n_iter + (6o^3v^4 + 6o^4v^3) when (T) ran */
  long long device_bytes; /* device memory held by the fragment handle */
  double cost_estimate;   /* the scheduler's cost model (flops): LPT starts fragments in decreasing order */
  long long bytes_estimate; /* the scheduler's device-memory estimate used for admission */
} lnocc_batch_result;

/* Defaults: workers 0 (auto), triples 1, LPT order, autotune 0, memory budget 0 (auto). */
void lnocc_default_batch_opts(lnocc_batch_opts* b);

/*
 * lnocc_solve_batch -- solve nfrag independent fragments; returns when all are done.
 *   items   : host array of nfrag descriptions (device pointers inside; they must stay valid and
 *             unchanged until the call returns; work on `stream` that produces them is waited for).
 *   opts    : per-fragment options as for lnocc_build_ints (NULL: defaults).
 *   bopts   : scheduling options (NULL: defaults).
 *   results : host array of nfrag results, written by the call.
 *   Returns LNOCC_OK when every fragment converged, LNOCC_ENOCONV when some did not (their results
 *   say so), else the status of a failing fragment (lnocc_last_error names it). The call allocates
 *   its own device memory (a pool released on return) and host threads.
 */
int lnocc_solve_batch(int nfrag, const lnocc_batch_item* items, const lnocc_opts* opts, const lnocc_batch_opts* bopts,
                      lnocc_batch_result* results, void* stream);

/*
 * Tile autotuner of the tensor-core GEMM (library-wide, all fragments; no counterpart in the paper).
 * The CTA tile width BN (32..256) of every tcgen05 contraction is picked per shape bucket
 * (M and K blocks in octaves, N in half-octaves, one or two K segments).
 *   mode 0 (default): fixed rule (narrowest BN covering N);
 *   mode 1: table lookup, fixed rule on a miss;
 *   mode 2: like 1, but a miss first times every candidate on the call's own operands (into scratch,
 *           synchronously on the call's stream) and stores the winner. Use from one thread at a time.
 * lnocc_autotune sets the mode (mode < 0: only read it) and returns the previous one in *prev_mode.
 * The table persists as a text file (lnocc_autotune_save / _load; load merges).
 */
int lnocc_autotune(int mode, int* prev_mode);
int lnocc_autotune_save(const char* path);
int lnocc_autotune_load(const char* path);
/* entries in the table, lookups that hit / missed, shapes timed so far */
int lnocc_autotune_stats(long long* entries, long long* hits, long long* misses, long long* tuned);

/* ------------------------------------------------------------------------------------------------
 * Learned T2 initial guess (no counterpart in the paper, whose CCSD starts from the MP2 amplitudes of
 * Eq. 21): t_ij^ab = t_ij^ab(MP2) + s_out g(x_ijab), g an MLP 8 -> 128 -> 128 -> 1 with SiLU on the
 * standardised features x = [t_MP2, e_i, e_j, e_a, e_b, D_ij^ab, (ia|jb), (ib|ja)] of the canonical
 * member of {(i,j,a,b), (j,i,b,a)} (i < j, or i == j and a <= b). Training: mean squared error of g
 * against (t_converged - t_MP2) / s_out, Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Parameter vector (float, lnocc_mlp_nparams() = 17793 values): W1[128][8], b1[128], W2[128][128],
 * b2[128], w3[128], b3[1], row-major with the output index first. Standardisation ("norm", 17 doubles):
 * feature means [8], standard deviations [8], s_out.
 * ---------------------------------------------------------------------------------------------- */
typedef struct lnocc_mlp lnocc_mlp; /* opaque: parameters, Adam state and workspace on the device */

int lnocc_mlp_nparams(void);
/* New model from host parameters (float[nparams]); norm starts as mean 0, deviation 1, s_out 1. */
int lnocc_mlp_create(const float* params, lnocc_mlp** out);
int lnocc_mlp_free(lnocc_mlp* m);
/* Copy parameters (host float[nparams]) and / or norm (host double[17]) out; either may be NULL. */
int lnocc_mlp_get(const lnocc_mlp* m, float* params, double* norm);
/* Set the standardisation (host double[17]; deviations and s_out must be positive). */
int lnocc_mlp_set_norm(lnocc_mlp* m, const double* norm);
/*
 * Training samples of a solved fragment: for n flat amplitude indices idx (device int64,
 * ((i*o + j)*v + a)*v + b), the raw features X (device float[n][8]) and, when dt != NULL, the targets
 * dt = t_converged - t_MP2 (device float[n]; needs a previous lnocc_ccsd on f).
 */
int lnocc_mlp_samples(const lnocc_frag* f, int n, const long long* idx, float* X, float* dt, void* stream);
/* Standardisation from samples: feature means / deviations and s_out = rms(dt) (device reductions). */
int lnocc_mlp_fit_norm(lnocc_mlp* m, int n, const float* X, const float* dt, void* stream);
/* One Adam step on the minibatch (X, dt): forward, backward and update on the device (FP32); the
 * batch loss before the step goes to *loss (host, may be NULL). */
int lnocc_mlp_train_step(lnocc_mlp* m, int n, const float* X, const float* dt, float lr, double* loss, void* stream);
/* Network output y[n] (device double) for raw features X; precision LNOCC_PREC_FP64 runs the FP64
 * build of the training kernels, LNOCC_PREC_MIXED the FP32 one (checks). */
int lnocc_mlp_forward(const lnocc_mlp* m, int precision, int n, const float* X, double* y, void* stream);
/* Loss gradient (device double[nparams]) and loss (host) on (X, dt) without updating (checks). */
int lnocc_mlp_grad(const lnocc_mlp* m, int precision, int n, const float* X, const float* dt, double* grad,
                   double* loss, void* stream);
/* The learned guess of a built fragment into t2_out (device double[o][o][v][v]); layer 2 runs as a
 * BF16 tcgen05 MMA with FP32 accumulation. */
int lnocc_mlp_guess(lnocc_frag* f, const lnocc_mlp* m, double* t2_out, void* stream);
/* Attach (or detach with NULL) the model used by LNOCC_GUESS_MLP; the model must outlive its use. */
int lnocc_frag_set_mlp(lnocc_frag* f, const lnocc_mlp* m);

/* Copy the handle's bookkeeping (energies, iteration count, flop counters) into *info. */
int lnocc_frag_info(const lnocc_frag* f, lnocc_info* info);

/* Release everything the handle holds (safe on NULL). With LNOCC_MEM_CACHED its device memory goes back
 * to the library's pool (stream-ordered on the handle's stream), not to the device. */
int lnocc_free_fragment(lnocc_frag* f);

/* Return the unused memory of the library's cached pool on the current device to the device (after
 * synchronising the device). Handles still alive keep theirs. Returns LNOCC_OK or LNOCC_ECUDA. */
int lnocc_trim_pool(void);

/* Message of the last failing call on this thread ("" when none). */
const char* lnocc_last_error(void);

/* Library version string. */
const char* lnocc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LNOCC_H */
