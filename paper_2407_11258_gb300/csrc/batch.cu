// Batched solve of many uneven fragments: lnocc_solve_batch.
//
// The fragments of one LNO calculation are independent (each fragment's CCSD(T) uses only its own
// integrals, Sec. 2.2), so a batch is a scheduling problem: keep the GPU full with fragments whose
// sizes span two orders of magnitude in cost while staying inside device memory.
//
//   * order: longest processing time first (LPT) on a cost model (CCSD iterations x per-iteration
//     flops + (T) flops); a fragment's iteration count is estimated from its HOMO-LUMO gap.
//   * pipelines: `workers` host threads, each with its own non-blocking stream, pinned scalar buffer
//     and split-K workspace, take the next fragment in LPT order whose estimated device footprint fits
//     the memory budget that remains (first fit in LPT order; a worker waits when none fits).
//   * memory: every fragment allocates from one stream-ordered memory pool owned by the batch, so
//     building and freeing fragments never synchronises the device and freed memory is reused at once.
//   * each pipeline runs build -> CCSD (iterations replayed from a captured CUDA graph) -> fragment
//     energies -> (T), with the contraction tiles taken from the autotuner's table when one is loaded.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "fragment.h"
#include "internal.h"

namespace lnocc {
namespace {

double per_iter_flops(double o, double v) {
  return 2 * o * o * v * v * v * v + 16 * o * o * o * v * v * v + 2 * o * o * o * o * v * v;
}
double triples_flops(double o, double v) { return 6 * o * o * o * v * v * v * v + 6 * o * o * o * o * v * v * v; }

// CCSD iterations to convergence, estimated from the HOMO-LUMO gap (Eh): small-gap fragments need
// more iterations (the amplitude update is damped by 1/D).
double iter_estimate(double gap) {
  if (!(gap > 0)) return 40.0;
  return std::min(60.0, 10.0 + 1.6 / std::sqrt(gap));
}

long long kp(long long k) { return (std::max(k, 1LL) + 63) / 64 * 64; }

}  // namespace

// Device bytes of one fragment handle at its peak (build transients and the (T) operands included),
// from the allocation plan of Frag::build / build_consts / triples.
long long estimate_fragment_bytes(int o_, int v_, int N_, bool mixed, int n_refine, int diis, bool do_t,
                                  int chunk_mb) {
  const long long o = o_, v = v_, N = N_, n = o + v, oo = o * o, vv = v * v, ov = o * v;
  const long long L = ov + oo * vv;
  const long long np_o = o * (o + 1) / 2, nm_o = std::max(1LL, o * (o - 1) / 2);
  const long long np_v = v * (v + 1) / 2, nm_v = std::max(1LL, v * (v - 1) / 2);
  long long b = 0;
  b += 8 * (n + N * oo + 2 * N * ov + 2 * N * vv + 6 * n * n + 2 * ov * ov + N);
  b += 8 * ((mixed ? 4 : 3) * L + 8 * oo * vv + 2 * oo * ov + 2 * oo * oo + N * ov + ov + vv + 2 * oo);
  b += 8 * (np_v * np_o + nm_v * nm_o + N * ov);
  b += 8 * 2 * std::min(diis, 8) * L;
  const long long cap = packing_scratch_elems(o_, v_, N_);
  b += 2 * 8 * cap + 8 * (1LL << 22);
  auto consts = [&](long long esz) {
    long long c = np_o * kp(np_v) + nm_o * kp(nm_v) + (2 * ov + oo + vv) * kp(N) + oo * kp(vv) + 2 * ov * kp(ov) +
                  v * kp(oo * v) + ov * kp(vv) + np_v * kp(np_v) + nm_v * kp(nm_v);
    c *= esz;
    const long long per_k = v * vv;
    const long long kc = std::max(1LL, std::min(o, (1LL << 27) / per_k));
    const long long ac = std::max(1LL, std::min(v, (1LL << 27) / per_k));
    return c + 8 * (kc + ac) * per_k + esz * vv * kp(N);  // build transients
  };
  b += consts(mixed ? 4 : 8);
  if (mixed && n_refine > 0) b += consts(8);
  if (do_t) b += static_cast<long long>(triples_plan(o_, v_, N_, mixed, chunk_mb).total);
  return b + b / 16 + (64LL << 20);
}

}  // namespace lnocc

using lnocc::Frag;

namespace {

struct Job {
  int idx;
  double cost;
  long long bytes;
};

struct Shared {
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Job> pending;  // in schedule order
  long long in_use = 0, budget = 0;
  int running = 0, started = 0;
  std::string first_error;
};

}  // namespace

extern "C" {

void lnocc_default_batch_opts(lnocc_batch_opts* b) {
  if (!b) return;
  std::memset(b, 0, sizeof(*b));
  b->workers = 0;
  b->triples = 1;
  b->order = LNOCC_ORDER_LPT;
  b->autotune = 0;
  b->mem_budget_gb = 0.0;
}

int lnocc_solve_batch(int nfrag, const lnocc_batch_item* items, const lnocc_opts* opts,
                      const lnocc_batch_opts* bopts, lnocc_batch_result* results, void* stream) {
  using namespace lnocc;
  set_error("");
  if (nfrag < 0 || (nfrag > 0 && (!items || !results))) {
    set_error("lnocc_solve_batch: bad arguments");
    return LNOCC_EINVAL;
  }
  lnocc_batch_opts bo;
  lnocc_default_batch_opts(&bo);
  if (bopts) bo = *bopts;
  lnocc_opts o;
  lnocc_default_opts(&o);
  if (opts) o = *opts;
  if (bo.workers < 0 || bo.workers > 16 || (bo.order != LNOCC_ORDER_LPT && bo.order != LNOCC_ORDER_INPUT) ||
      bo.mem_budget_gb < 0 || bo.autotune < 0 || bo.autotune > 2) {
    set_error("lnocc_solve_batch: bad batch options");
    return LNOCC_EINVAL;
  }
  for (int f = 0; f < nfrag; ++f) {
    const lnocc_batch_item& it = items[f];
    if (it.nocc < 1 || it.nvir < 1 || it.naux < 1 || !it.eps || !it.B || it.nlo < 0 || (it.nlo > 0 && !it.U_frag)) {
      set_error("lnocc_solve_batch: bad item " + std::to_string(f));
      return LNOCC_EINVAL;
    }
  }
  if (nfrag == 0) return LNOCC_OK;
  int dev = 0;
  LN_CUDA(cudaGetDevice(&dev));
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  // inputs produced on the caller's stream must be complete before the pipelines read them
  LN_CUDA(cudaStreamSynchronize(user));

  // ---- cost model and schedule
  Shared sh;
  const bool mixed = o.precision == LNOCC_PREC_MIXED;
  for (int f = 0; f < nfrag; ++f) {
    const lnocc_batch_item& it = items[f];
    double gap = 1.0;
    {
      double pair[2];
      LN_CUDA(cudaMemcpy(pair, it.eps + it.nocc - 1, 2 * sizeof(double), cudaMemcpyDeviceToHost));
      gap = pair[1] - pair[0];
    }
    const double cost = iter_estimate(gap) * per_iter_flops(it.nocc, it.nvir) +
                        (bo.triples ? triples_flops(it.nocc, it.nvir) : 0.0) +
                        2.0 * it.naux * (it.nocc + it.nvir) * double(it.nvir) * it.nvir * it.nvir;
    const long long bytes =
        estimate_fragment_bytes(it.nocc, it.nvir, it.naux, mixed, o.n_refine, o.diis_space, bo.triples != 0,
                                o.triples_chunk_mb);
    sh.pending.push_back(Job{f, cost, bytes});
  }
  if (bo.order == LNOCC_ORDER_LPT)
    std::stable_sort(sh.pending.begin(), sh.pending.end(), [](const Job& a, const Job& b) { return a.cost > b.cost; });
  size_t free_b = 0, total_b = 0;
  LN_CUDA(cudaMemGetInfo(&free_b, &total_b));
  sh.budget = bo.mem_budget_gb > 0 ? static_cast<long long>(bo.mem_budget_gb * 1e9)
                                   : static_cast<long long>(0.9 * static_cast<double>(free_b));
  int workers = bo.workers;
  if (workers == 0) workers = 3;
  workers = std::min(workers, nfrag);

  // ---- shared stream-ordered pool (kept until the batch ends)
  cudaMemPool_t pool = nullptr;
  {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    LN_CUDA(cudaMemPoolCreate(&pool, &props));
    unsigned long long keep = ~0ULL;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  // per-worker streams and pinned scalar buffers, created before any work starts
  std::vector<cudaStream_t> streams(workers, nullptr);
  double* hbuf = nullptr;
  LN_CUDA(cudaMallocHost(&hbuf, sizeof(double) * 16 * workers));
  for (int w = 0; w < workers; ++w) LN_CUDA(cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking));

  // ---- tile autotuning on representative fragments (cost quantiles), one at a time on stream 0
  const int prev_mode = autotune_mode(-1);
  if (bo.autotune == 1) {
    std::vector<Job> byc = sh.pending;
    std::sort(byc.begin(), byc.end(), [](const Job& a, const Job& b) { return a.cost < b.cost; });
    std::vector<int> reps;
    for (double q : {0.0, 0.25, 0.5, 0.75, 1.0}) {
      const int k = byc[static_cast<size_t>(std::lround(q * (byc.size() - 1)))].idx;
      if (std::find(reps.begin(), reps.end(), k) == reps.end()) reps.push_back(k);
    }
    autotune_mode(2);
    for (int k : reps) {
      const lnocc_batch_item& it = items[k];
      lnocc_frag* h = new (std::nothrow) lnocc_frag;
      if (!h) break;
      Frag& fr = h->f;
      fr.o = it.nocc;
      fr.v = it.nvir;
      fr.N = it.naux;
      fr.n = it.nocc + it.nvir;
      fr.opts = o;
      fr.opts.max_iter = 2;
      fr.opts.graph = 0;
      fr.mixed = mixed;
      fr.s = streams[0];
      fr.pool = pool;
      fr.h_ext = hbuf;
      if (fr.build(it.eps, it.B) == LNOCC_OK) {
        fr.use_workspace();
        fr.solve(LNOCC_GUESS_MP2, nullptr, nullptr);
        if (bo.triples) {
          fr.t_max_chunks = 6;
          double e1 = 0, e2 = 0;
          fr.triples(0, nullptr, &e1, &e2);
        }
      }
      delete h;
      split_ws() = SplitWs{};
      cudaStreamSynchronize(streams[0]);
    }
    cudaGetLastError();
    set_error("");
  }
  if (bo.autotune >= 1) autotune_mode(1);

  const auto t0 = std::chrono::steady_clock::now();
  auto now_ms = [&]() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  for (int f = 0; f < nfrag; ++f) {
    std::memset(&results[f], 0, sizeof(results[f]));
    results[f].status = LNOCC_EINVAL;
    results[f].worker = -1;
    results[f].order = -1;
  }
  for (const Job& j : sh.pending) {
    results[j.idx].cost_estimate = j.cost;
    results[j.idx].bytes_estimate = j.bytes;
  }

  auto run_one = [&](int w, const Job& job) {
    const lnocc_batch_item& it = items[job.idx];
    lnocc_batch_result& r = results[job.idx];
    r.worker = w;
    r.t_start_ms = now_ms();
    lnocc_frag* h = new (std::nothrow) lnocc_frag;
    if (!h) {
      r.status = LNOCC_ENOMEM;
      return;
    }
    Frag& fr = h->f;
    fr.o = it.nocc;
    fr.v = it.nvir;
    fr.N = it.naux;
    fr.n = it.nocc + it.nvir;
    fr.opts = o;
    fr.mixed = mixed;
    fr.s = streams[w];
    fr.pool = pool;
    fr.h_ext = hbuf + 16 * w;
    gemm_stats() = GemmStats{};
    int st = fr.build(it.eps, it.B);
    r.e_mp2 = fr.e_mp2;
    if (st == LNOCC_OK) {
      fr.use_workspace();
      st = fr.solve(LNOCC_GUESS_MP2, nullptr, nullptr);
      r.n_iter = fr.n_iter;
      r.e_ccsd = fr.e_ccsd;
      r.model_flops = per_iter_flops(it.nocc, it.nvir) * fr.n_iter;
      if ((st == LNOCC_OK || st == LNOCC_ENOCONV) && it.nlo > 0) {
        const int s2 = fr.fragment_energy(it.nlo, it.U_frag, &r.e_ccsd_frag, &r.e_mp2_frag);
        if (s2 != LNOCC_OK) st = s2;
      }
      if ((st == LNOCC_OK || st == LNOCC_ENOCONV) && bo.triples) {
        const int s3 = fr.triples(it.nlo, it.nlo > 0 ? it.U_frag : nullptr, &r.e_t, &r.e_t_frag);
        if (s3 != LNOCC_OK) st = s3;
        r.model_flops += triples_flops(it.nocc, it.nvir);
      }
    }
    r.device_bytes = fr.device_bytes;
    r.status = st;
    if (st != LNOCC_OK && st != LNOCC_ENOCONV) {
      std::lock_guard<std::mutex> lk(sh.mu);
      if (sh.first_error.empty())
        sh.first_error = "fragment " + std::to_string(job.idx) + ": " + std::string(lnocc_last_error());
    }
    delete h;  // frees into the pool on this worker's stream
    cudaStreamSynchronize(streams[w]);
    r.t_end_ms = now_ms();
  };

  auto worker = [&](int w) {
    cudaSetDevice(dev);
    split_ws() = SplitWs{};
    for (;;) {
      Job job{};
      {
        std::unique_lock<std::mutex> lk(sh.mu);
        for (;;) {
          if (sh.pending.empty()) return;
          auto pick = sh.pending.end();
          for (auto p = sh.pending.begin(); p != sh.pending.end(); ++p)
            if (p->bytes <= sh.budget - sh.in_use) {
              pick = p;
              break;
            }
          // nothing fits: with nothing else running, try the head anyway (it may still fit in practice)
          if (pick == sh.pending.end() && sh.running == 0) pick = sh.pending.begin();
          if (pick != sh.pending.end()) {
            job = *pick;
            sh.pending.erase(pick);
            sh.in_use += job.bytes;
            sh.running++;
            results[job.idx].order = sh.started++;
            break;
          }
          sh.cv.wait(lk);
        }
      }
      run_one(w, job);
      {
        std::lock_guard<std::mutex> lk(sh.mu);
        sh.in_use -= job.bytes;
        sh.running--;
      }
      sh.cv.notify_all();
    }
  };

  std::vector<std::thread> threads;
  for (int w = 0; w < workers; ++w) threads.emplace_back(worker, w);
  for (auto& t : threads) t.join();

  for (int w = 0; w < workers; ++w) {
    cudaStreamSynchronize(streams[w]);
    cudaStreamDestroy(streams[w]);
  }
  cudaFreeHost(hbuf);
  cudaMemPoolDestroy(pool);
  autotune_mode(prev_mode);
  int worst = LNOCC_OK;
  for (int f = 0; f < nfrag; ++f)
    if (results[f].status != LNOCC_OK && results[f].status != LNOCC_ENOCONV) worst = results[f].status;
  if (!sh.first_error.empty()) set_error(sh.first_error);
  if (worst == LNOCC_OK)
    for (int f = 0; f < nfrag; ++f)
      if (results[f].status == LNOCC_ENOCONV) {
        set_error("fragment " + std::to_string(f) + " did not converge");
        worst = LNOCC_ENOCONV;
        break;
      }
  return worst;
}

}  // extern "C"
