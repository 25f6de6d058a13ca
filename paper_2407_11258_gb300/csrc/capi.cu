// extern "C" boundary of liblnocc (declared in include/lnocc.h).
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "fragment.h"
#include "internal.h"

namespace lnocc {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace lnocc

using lnocc::Frag;

namespace lnocc {
cudaMemPool_t cached_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t p = nullptr;
  if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  unsigned long long keep = ~0ULL;  // keep freed memory for later handles
  cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = p;
  return p;
}
}  // namespace lnocc

extern "C" {

void lnocc_default_opts(lnocc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = LNOCC_PREC_MIXED;
  o->max_iter = 100;
  o->diis_space = 8;
  o->n_refine = 0;
  o->conv_rms = 1e-8;
  o->conv_energy = 1e-10;
  o->fault_inject = 0;
  o->verbose = 0;
  o->graph = 1;
}

const char* lnocc_last_error(void) { return lnocc::g_last_error.c_str(); }

const char* lnocc_version(void) { return "lnocc 0.1 (sm_103a)"; }

int lnocc_build_ints(int nocc, int nvir, int naux, const double* eps, const double* B, const lnocc_opts* opts,
                     void* stream, lnocc_frag** out) {
  lnocc::set_error("");
  if (!out || !eps || !B || nocc < 1 || nvir < 1 || naux < 1) {
    lnocc::set_error("lnocc_build_ints: bad arguments");
    return LNOCC_EINVAL;
  }
  *out = nullptr;
  lnocc_opts o;
  lnocc_default_opts(&o);
  if (opts) o = *opts;
  if ((o.precision != LNOCC_PREC_FP64 && o.precision != LNOCC_PREC_MIXED) || o.max_iter < 0 || o.diis_space < 0 ||
      o.diis_space > 8 || o.n_refine < 0 || (o.graph != 0 && o.graph != 1) || !(o.conv_rms > 0) || !(o.conv_energy > 0) ||
      o.triples_chunk_mb < 0 || o.triples_kernel < LNOCC_TK_AUTO || o.triples_kernel > LNOCC_TK_GROUPED ||
      (o.memory != LNOCC_MEM_CACHED && o.memory != LNOCC_MEM_DIRECT)) {
    lnocc::set_error("lnocc_build_ints: bad options");
    return LNOCC_EINVAL;
  }
  lnocc_frag* h = new (std::nothrow) lnocc_frag;
  if (!h) return LNOCC_ENOMEM;
  Frag& f = h->f;
  f.o = nocc;
  f.v = nvir;
  f.N = naux;
  f.n = nocc + nvir;
  f.opts = o;
  f.mixed = (o.precision == LNOCC_PREC_MIXED);
  f.s = static_cast<cudaStream_t>(stream);
  if (o.memory == LNOCC_MEM_CACHED) {
    f.pool = lnocc::cached_pool();
    f.pool_cached = f.pool != nullptr;
  }
  const char* pe = std::getenv("LNOCC_PROFILE");
  f.prof = pe && pe[0] == '1';
  lnocc::gemm_stats() = lnocc::GemmStats{};
  const int st = f.build(eps, B);
  if (st != LNOCC_OK) {
    delete h;
    return st;
  }
  *out = h;
  return LNOCC_OK;
}

int lnocc_ccsd(lnocc_frag* h, const double* t1_in, const double* t2_in, int guess_mode, double* t1_out,
               double* t2_out, double* e_corr, int* n_iter, void* stream) {
  lnocc::set_error("");
  if (!h || (guess_mode != LNOCC_GUESS_MP2 && guess_mode != LNOCC_GUESS_GIVEN && guess_mode != LNOCC_GUESS_MLP)) {
    lnocc::set_error("lnocc_ccsd: bad arguments");
    return LNOCC_EINVAL;
  }
  Frag& f = h->f;
  f.s = static_cast<cudaStream_t>(stream);
  f.use_workspace();
  const int st = f.solve_with_fallback(guess_mode, t1_in, t2_in);
  const long long ov = 1LL * f.o * f.v;
  if (f.have_amps) {
    if (t1_out) cudaMemcpyAsync(t1_out, f.xcur, ov * 8, cudaMemcpyDeviceToDevice, f.s);
    if (t2_out) cudaMemcpyAsync(t2_out, f.xcur + ov, ov * ov * 8, cudaMemcpyDeviceToDevice, f.s);
    if (t1_out || t2_out) cudaStreamSynchronize(f.s);
  }
  if (e_corr) *e_corr = f.e_ccsd;
  if (n_iter) *n_iter = f.n_iter;
  return st;
}

int lnocc_fragment_energy(lnocc_frag* h, int nlo, const double* U_frag, double* e_ccsd_frag, double* e_mp2_frag,
                          void* stream) {
  lnocc::set_error("");
  if (!h || nlo < 1 || !U_frag) {
    lnocc::set_error("lnocc_fragment_energy: bad arguments");
    return LNOCC_EINVAL;
  }
  h->f.s = static_cast<cudaStream_t>(stream);
  h->f.use_workspace();
  return h->f.fragment_energy(nlo, U_frag, e_ccsd_frag, e_mp2_frag);
}

int lnocc_triples(lnocc_frag* h, int nlo, const double* U_frag, double* e_t_full, double* e_t_frag, void* stream) {
  lnocc::set_error("");
  if (!h || (U_frag && nlo < 1)) {
    lnocc::set_error("lnocc_triples: bad arguments");
    return LNOCC_EINVAL;
  }
  if (!h->f.have_amps) {
    lnocc::set_error("lnocc_triples: no CCSD amplitudes (call lnocc_ccsd first)");
    return LNOCC_EINVAL;
  }
  h->f.s = static_cast<cudaStream_t>(stream);
  h->f.use_workspace();
  return h->f.triples(U_frag ? nlo : 0, U_frag, e_t_full, e_t_frag);
}

int lnocc_fragment_energy_device(lnocc_frag* h, int nlo, const double* U_frag, double* e_dev, void* stream) {
  lnocc::set_error("");
  if (!h || nlo < 1 || !U_frag || !e_dev) {
    lnocc::set_error("lnocc_fragment_energy_device: bad arguments");
    return LNOCC_EINVAL;
  }
  h->f.s = static_cast<cudaStream_t>(stream);
  h->f.use_workspace();
  return h->f.fragment_energy(nlo, U_frag, nullptr, nullptr, e_dev);
}

int lnocc_triples_device(lnocc_frag* h, int nlo, const double* U_frag, double* e_dev, int* status_dev, void* stream) {
  lnocc::set_error("");
  if (!h || (U_frag && nlo < 1) || !e_dev) {
    lnocc::set_error("lnocc_triples_device: bad arguments");
    return LNOCC_EINVAL;
  }
  if (!h->f.have_amps) {
    lnocc::set_error("lnocc_triples_device: no CCSD amplitudes (call lnocc_ccsd first)");
    return LNOCC_EINVAL;
  }
  h->f.s = static_cast<cudaStream_t>(stream);
  h->f.use_workspace();
  return h->f.triples(U_frag ? nlo : 0, U_frag, nullptr, nullptr, e_dev, status_dev);
}

int lnocc_workspace_bytes(int nocc, int nvir, int naux, const lnocc_opts* opts, long long* bytes) {
  lnocc::set_error("");
  lnocc_opts o;
  lnocc_default_opts(&o);
  if (opts) o = *opts;
  if (!bytes || nocc < 1 || nvir < 1 || naux < 1 || o.triples_chunk_mb < 0 ||
      (o.precision != LNOCC_PREC_FP64 && o.precision != LNOCC_PREC_MIXED)) {
    lnocc::set_error("lnocc_workspace_bytes: bad arguments");
    return LNOCC_EINVAL;
  }
  *bytes = static_cast<long long>(
      lnocc::triples_plan(nocc, nvir, naux, o.precision == LNOCC_PREC_MIXED, o.triples_chunk_mb).total);
  return LNOCC_OK;
}

int lnocc_frag_set_workspace(lnocc_frag* h, void* workspace, long long workspace_bytes) {
  lnocc::set_error("");
  if (!h) {
    lnocc::set_error("lnocc_frag_set_workspace: bad arguments");
    return LNOCC_EINVAL;
  }
  Frag& f = h->f;
  if (workspace) {
    const size_t need = lnocc::triples_plan(f.o, f.v, f.N, f.mixed, f.opts.triples_chunk_mb).total;
    if (workspace_bytes < 0 || static_cast<size_t>(workspace_bytes) < need) {
      lnocc::set_error("lnocc_frag_set_workspace: workspace smaller than lnocc_workspace_bytes (" +
                       std::to_string(need) + " bytes)");
      return LNOCC_EINVAL;
    }
  }
  f.ws_ext = workspace;
  f.ws_ext_bytes = workspace ? static_cast<size_t>(workspace_bytes) : 0;
  return LNOCC_OK;
}

int lnocc_frag_info(const lnocc_frag* h, lnocc_info* info) {
  if (!h || !info) return LNOCC_EINVAL;
  const Frag& f = h->f;
  const double o = f.o, v = f.v;
  info->nocc = f.o;
  info->nvir = f.v;
  info->naux = f.N;
  info->precision = f.mixed ? LNOCC_PREC_MIXED : LNOCC_PREC_FP64;
  info->n_iter = f.n_iter;
  info->converged = f.converged ? 1 : 0;
  info->e_mp2 = f.e_mp2;
  info->e_ccsd = f.e_ccsd;
  info->last_rms = f.last_rms;
  info->model_flops_ccsd = (2 * o * o * v * v * v * v + 16 * o * o * o * v * v * v + 2 * o * o * o * o * v * v) * f.n_iter;
  info->model_flops_t = 6 * o * o * o * v * v * v * v + 6 * o * o * o * o * v * v * v;
  info->exec_flops = lnocc::gemm_stats().flops;
  info->gemm_launches = lnocc::gemm_stats().launches;
  info->device_bytes = f.device_bytes;
  info->kernel_launches = lnocc::launch_counter().load();
  info->t_triples_gemm_ms = f.t_gemm_ms;
  info->t_triples_ms = f.t_triples_ms;
  info->device_allocs = lnocc::alloc_counter().load();
  info->floor_spread = f.floor_spread;
  info->n_refined = f.n_refined;
  info->diis_restarts = f.diis_restarts;
  return LNOCC_OK;
}

int lnocc_debug_gemm(int precision, int M, int N, int K, const double* A, const double* B, double* C, void* stream) {
  lnocc::set_error("");
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return LNOCC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool bf = precision == LNOCC_PREC_MIXED;
  lnocc::Packed PA, PB;
  PA.bf16 = PB.bf16 = bf;
  const int Kp = lnocc::round_up(K, 64);
  int* dstatus = nullptr;
  lnocc::count_alloc(4);
  LN_CUDA(cudaMalloc(&PA.p, static_cast<size_t>(M) * Kp * (bf ? 4 : 8)));
  LN_CUDA(cudaMalloc(&PB.p, static_cast<size_t>(N) * Kp * (bf ? 4 : 8)));
  LN_CUDA(cudaMalloc(&dstatus, 16));
  LN_CUDA(cudaMemsetAsync(dstatus, 0, 16, s));
  double* ws = nullptr;
  LN_CUDA(cudaMalloc(&ws, (1u << 22) * sizeof(double)));
  lnocc::split_ws() = lnocc::SplitWs{ws, 1u << 22};
  const lnocc::Ax one{1, 0};
  lnocc::pack(lnocc::view(A, one, one, lnocc::Ax{M, K}, one, one, lnocc::Ax{K, 1}), PA, s);
  lnocc::pack(lnocc::view(B, one, one, lnocc::Ax{N, K}, one, one, lnocc::Ax{K, 1}), PB, s);
  lnocc::gemm(PA, PB, M, N, K, lnocc::out_rowmajor(C, N), s, dstatus);
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, dstatus, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(PA.p);
  cudaFree(PB.p);
  cudaFree(dstatus);
  cudaFree(ws);
  lnocc::split_ws() = lnocc::SplitWs{};
  if (e != cudaSuccess) {
    lnocc::set_error(std::string("lnocc_debug_gemm: ") + cudaGetErrorString(e));
    return LNOCC_ECUDA;
  }
  if (st != 0) {
    lnocc::set_error("lnocc_debug_gemm: device wait timed out");
    return LNOCC_ETIMEOUT;
  }
  return LNOCC_OK;
}

int lnocc_autotune(int mode, int* prev_mode) {
  lnocc::set_error("");
  if (mode > 2) {
    lnocc::set_error("lnocc_autotune: mode must be 0, 1 or 2");
    return LNOCC_EINVAL;
  }
  const int prev = lnocc::autotune_mode(mode < 0 ? -1 : mode);
  if (prev_mode) *prev_mode = prev;
  return LNOCC_OK;
}

int lnocc_autotune_save(const char* path) {
  lnocc::set_error("");
  if (!path || !lnocc::autotune_save(path)) {
    lnocc::set_error("lnocc_autotune_save: cannot write the table");
    return LNOCC_EINVAL;
  }
  return LNOCC_OK;
}

int lnocc_autotune_load(const char* path) {
  lnocc::set_error("");
  if (!path || !lnocc::autotune_load(path)) {
    lnocc::set_error("lnocc_autotune_load: cannot read the table");
    return LNOCC_EINVAL;
  }
  return LNOCC_OK;
}

int lnocc_autotune_stats(long long* entries, long long* hits, long long* misses, long long* tuned) {
  long long s[4];
  lnocc::autotune_stats(s);
  if (entries) *entries = s[0];
  if (hits) *hits = s[1];
  if (misses) *misses = s[2];
  if (tuned) *tuned = s[3];
  return LNOCC_OK;
}

int lnocc_free_fragment(lnocc_frag* h) {
  if (h && lnocc::split_ws().p == h->f.splitk) lnocc::split_ws() = lnocc::SplitWs{};
  delete h;
  return LNOCC_OK;
}

int lnocc_trim_pool(void) {
  cudaMemPool_t p = lnocc::cached_pool();
  if (!p) return LNOCC_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(p, 0) != cudaSuccess) {
    lnocc::set_error(std::string("lnocc_trim_pool: ") + cudaGetErrorString(cudaGetLastError()));
    return LNOCC_ECUDA;
  }
  return LNOCC_OK;
}

}  // extern "C"
