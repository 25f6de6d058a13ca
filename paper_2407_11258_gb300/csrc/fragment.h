// The fragment handle behind `lnocc_frag`: integrals, amplitudes and workspace on the device.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "internal.h"

namespace lnocc {

struct Mlp;  // learned T2 guess model (mlp.cu)
// learned guess t2_out[i][j][a][b] = t_MP2 + s_out g(features) over all o^2 v^2 amplitudes (mlp.cu)
int mlp_guess(const Mlp& m, int o, int v, const double* t2mp2, const double* eps, const double* ovov, double* t2_out,
              int* dstatus, cudaStream_t s);

// Constant packed operands of the CCSD iteration for one precision.
struct Consts {
  Packed kl_cd;  // (kc|ld): rows (k,l), K (c,d)          -> Y_ij^kl
  Packed kc_ld;  // (kd|lc): rows (k,c), K (l,d)          -> C2 intermediate
  Packed L;      // 2(ld|kc) - (lc|kd): rows (k,c), K (l,d) -> D2 intermediate
  Packed c_kld;  // (ld|kc): rows c, K (k,l,d)            -> E2 virtual Fock term
  Packed kb_cd;  // (kc|bd): rows (k,b), K (c,d)          -> Z_ij^kb
  Packed Vp, Vm; // packed (ac|bd) +- (ad|bc)             -> particle-particle ladder
  Packed Bp_t, Bm_t;  // per-iteration packed t+- operands of the ladder
  Packed PBov;        // B_ov as rows (i,a), K = Q (constant)
  Packed PBoo, PBvo, PBvv;  // per-iteration T1-transformed DF factors as rows (p,q), K = Q
  bool built = false;
};

// Sizes (bytes) of the device temporaries of one lnocc_triples call (triples.cu).
struct TriplesPlan {
  size_t xt, to, ovoo, pbvv, ovvv_chunk, w, tpart, batch, u, ovt, total;
  long long welems, nblk;
  int bc;
};
TriplesPlan triples_plan(int o, int v, int N, bool bf, int chunk_mb);
// Elements (FP64-sized) of each of the two packing scratch buffers of a fragment (ccsd.cu).
long long packing_scratch_elems(int o, int v, int N);

struct Frag {
  int o = 0, v = 0, N = 0, n = 0;
  lnocc_opts opts{};
  bool mixed = true;
  cudaStream_t s = nullptr;

  // allocation bookkeeping. With `pool` set (the batch runtime), device memory comes from that
  // stream-ordered pool on stream `s` and is returned with cudaFreeAsync (no device-wide
  // synchronisation); otherwise cudaMalloc / cudaFree.
  std::vector<void*> allocs;
  long long device_bytes = 0;
  bool oom = false;
  bool scratch_overflow = false;
  cudaMemPool_t pool = nullptr;
  bool pool_cached = false;  // `pool` is the library-wide cached pool (the caller's stream, not a batch's)
  double* h_ext = nullptr;  // caller-owned pinned host buffer (16 doubles) used instead of cudaMallocHost
  void* ws_ext = nullptr;  // caller-owned workspace for the (T) temporaries (lnocc_frag_set_workspace)
  size_t ws_ext_bytes = 0;
  void* alloc(size_t bytes, bool zero = false);
  void* dev_alloc(size_t bytes);  // raw allocation in the fragment's memory mode (not tracked)
  void dev_free(void* p);
  Packed alloc_packed(int rows, int K, bool bf16);
  ~Frag();

  // inputs and constant integrals (FP64)
  double *eps = nullptr, *Boo = nullptr, *Bov = nullptr, *Bvv = nullptr, *h = nullptr;
  double *ovov = nullptr, *Lpair = nullptr, *t2mp2 = nullptr;
  Consts cst[2];  // [0] FP64, [1] BF16 hi/lo
  Consts& C() { return cst[mixed ? 1 : 0]; }
  int np_o = 0, nm_o = 0, np_v = 0, nm_v = 0;

  // amplitudes: x = [t1 (o*v) | t2 (o*o*v*v)]
  double *xcur = nullptr, *xnew = nullptr, *enew = nullptr;
  double* xbest = nullptr;  // mixed: amplitudes of the lowest-rms iteration
  // per-iteration work
  double *Boo_h = nullptr, *Bvo_h = nullptr, *Bvv_h = nullptr;
  double *Xm = nullptr, *Ym = nullptr, *hh = nullptr, *tmpn = nullptr, *Fh = nullptr, *xq = nullptr;
  double *tau = nullptr, *u = nullptr, *Rsym = nullptr, *S = nullptr, *Cp = nullptr, *Xk = nullptr, *Yk = nullptr;
  double *Z = nullptr, *Wb = nullptr, *Wy = nullptr, *R1 = nullptr, *Mtmp = nullptr, *Gooov = nullptr;
  double *Fvv2 = nullptr, *Foo2 = nullptr, *Eii = nullptr, *Lp_out = nullptr, *Lm_out = nullptr;
  void *scrA = nullptr, *scrB = nullptr;
  size_t scr_bytes = 0;
  double* splitk = nullptr;  // split-K partials workspace
  size_t splitk_cap = 0;
  void use_workspace() { split_ws() = SplitWs{splitk, splitk_cap}; }
  // DIIS (subspace counters on the device: dctr[0] vectors pushed, dctr[1] vectors in use)
  int dm = 0;
  double *dvec = nullptr, *derr = nullptr, *G = nullptr, *coef = nullptr, *dpart = nullptr;
  int* dctr = nullptr;
  // One CCSD iteration (residual, DIIS step, energy, copy of the convergence scalars to the host)
  // captured as a CUDA graph on a private stream and replayed on `s`.
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long graph_kernels = 0;
  bool graph_failed = false;
  void step(bool fp64_residual, bool use_diis);
  int launch_step(bool fp64_residual, bool use_diis, bool use_graph);
  // reductions / status
  double *part = nullptr, *scal = nullptr, *h_scal = nullptr;
  int* dstatus = nullptr;

  // results
  double e_mp2 = 0.0, e_ccsd = 0.0, last_rms = 0.0;
  double floor_spread = 0.0;  // mixed: energy spread over the window at the noise floor
  int n_refined = 0, diis_restarts = 0;
  int n_iter = 0;
  bool converged = false, have_amps = false;
  double flops_t = 0.0;
  double t_gemm_ms = 0.0, t_triples_ms = 0.0;  // device times of the last lnocc_triples
  long long t_max_chunks = -1;  // > 0: run only ~this many W chunks spread over the (T) plan (autotuning; energy invalid)

  // optional per-step timing (environment LNOCC_PROFILE=1): events between named marks
  bool prof = false;
  std::vector<std::pair<std::string, cudaEvent_t>> marks;
  std::map<std::string, double> prof_ms;
  void mark(const char* name);
  void prof_flush();
  void prof_print(const char* title);

  // learned guess (LNOCC_GUESS_MLP): the attached model, and what the last solve used
  const Mlp* mlp = nullptr;
  bool mlp_used = false, mlp_fallback = false;
  int solve_with_fallback(int guess, const double* t1_in, const double* t2_in);

  int build(const double* eps_in, const double* B_in);
  int build_consts(bool bf);
  int check_device();
  void contract(const View& a, const View& b, const OutMap& c, bool force_fp64 = false);
  void contract_packed_b(const View& a, const Packed& PB, int N, const OutMap& c);
  void pack_df();  // T1-transformed DF factors -> packed [pq][Q] operands of the current precision
  void iterate(bool fp64_residual);
  double energy_of(const double* x);
  int solve(int guess, const double* t1_in, const double* t2_in);
  // e_dev (device, 2 doubles) set: enqueue only, results copied there (graph-capturable forms)
  int fragment_energy(int nlo, const double* U, double* e_ccsd_frag, double* e_mp2_frag, double* e_dev = nullptr);
  int triples(int nlo, const double* U, double* e_full, double* e_frag, double* e_dev = nullptr,
              int* st_dev = nullptr);
};

}  // namespace lnocc

struct lnocc_frag {
  lnocc::Frag f;
};
