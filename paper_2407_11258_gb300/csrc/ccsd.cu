// Fragment CCSD driver: integral assembly (lnocc_build_ints), the CCSD iteration (lnocc_ccsd) and
// the projected fragment energies (lnocc_fragment_energy).
//
// Equations: closed-shell CCSD in T1-transformed form (Koch et al., Chem. Phys. Lett. 228, 233
// (1994)), with density-fitted integrals (pq|rs) = sum_Q B_Qpq B_Qrs (Eq. 27a, Gamma-point form).
// The T1 amplitudes are folded into the DF factors, B^ = (1 - T) B (1 + T); every dressed
// integral block is then a contraction over Q. The particle-particle ladder is the exception: it
// uses the undressed (ac|bd), assembled once in symmetric / antisymmetric packed form
//   V+-[ab][cd] = (ac|bd) +- (ad|bc)   (a<=b, c<=d),
// and the T1 part of the dressing is restored with the (kc|bd) and (kc|ld) contractions Z and Y.
// The doubles residual is R = Rsym + S + S^T + P[C2] with
//   Rsym = g^_aibj + sum_cd (ac|bd) t_ij^cd + sum_kl tau_kl^ab (g^_kilj + Y_ij^kl)      (P-symmetric)
//   S    = -sum_k t_k^a Z_ij^kb + D2 + E2                                              (pre-P)
// and the update t += R / D uses D = e_i + e_j - e_a - e_b in FP64 (likewise for t1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ccsd_kernels.h"
#include "fragment.h"
#include "internal.h"

namespace lnocc {

static inline Ax A(int n, long long s) { return Ax{n, s}; }

void* Frag::dev_alloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  count_alloc();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void Frag::dev_free(void* p) {
  if (!p) return;
  if (pool)
    cudaFreeAsync(p, s);
  else
    cudaFree(p);
}
void* Frag::alloc(size_t bytes, bool zero) {
  if (bytes == 0) bytes = 256;
  void* p = dev_alloc(bytes);
  if (!p) {
    oom = true;
    return nullptr;
  }
  if (zero) cudaMemsetAsync(p, 0, bytes, s);
  allocs.push_back(p);
  device_bytes += static_cast<long long>(bytes);
  return p;
}

void Frag::mark(const char* name) {
  if (!prof) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, s);
  marks.emplace_back(name, e);
}

void Frag::prof_flush() {
  if (!prof || marks.empty()) return;
  cudaEventSynchronize(marks.back().second);
  for (size_t i = 1; i < marks.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, marks[i - 1].second, marks[i].second);
    prof_ms[marks[i].first] += ms;
  }
  for (auto& m : marks) cudaEventDestroy(m.second);
  marks.clear();
}

void Frag::prof_print(const char* title) {
  if (!prof) return;
  prof_flush();
  double tot = 0.0;
  for (auto& kv : prof_ms) tot += kv.second;
  std::fprintf(stderr, "lnocc profile (%s): total %.3f ms\n", title, tot);
  std::vector<std::pair<double, std::string>> v;
  for (auto& kv : prof_ms) v.emplace_back(kv.second, kv.first);
  std::sort(v.rbegin(), v.rend());
  for (auto& p : v) std::fprintf(stderr, "  %-14s %10.3f ms  %5.1f%%\n", p.second.c_str(), p.first, 100.0 * p.first / tot);
  prof_ms.clear();
}

Frag::~Frag() {
  for (auto& m : marks) cudaEventDestroy(m.second);
  if (gexec) cudaGraphExecDestroy(gexec);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (pool_cached && !allocs.empty()) {
    // the caller's stream of the last call orders the frees; if it is gone, wait for the device and
    // free on the legacy stream
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      cudaDeviceSynchronize();
      s = nullptr;
    }
  }
  for (void* p : allocs) dev_free(p);
  if (h_scal && h_scal != h_ext) cudaFreeHost(h_scal);
}

Packed Frag::alloc_packed(int rows, int K, bool bf16) {
  Packed P;
  P.rows = rows;
  P.Kp = round_up(std::max(K, 1), 64);
  P.bf16 = bf16;
  P.p = alloc(static_cast<size_t>(rows) * P.Kp * (bf16 ? 4 : 8), true);
  return P;
}

// Pack both operands into scratch and run C = A B^T through the precision's GEMM.
void Frag::contract(const View& a, const View& b, const OutMap& c, bool force_fp64) {
  Packed PA, PB;
  PA.p = scrA;
  PB.p = scrB;
  PA.bf16 = PB.bf16 = mixed && !force_fp64;
  const size_t ea = static_cast<size_t>(a.rows()) * round_up(std::max(a.K(), 1), 64) * (PA.bf16 ? 4 : 8);
  const size_t eb = static_cast<size_t>(b.rows()) * round_up(std::max(b.K(), 1), 64) * (PB.bf16 ? 4 : 8);
  if (ea > scr_bytes || eb > scr_bytes) {
    scratch_overflow = true;
    return;
  }
  pack(a, PA, s);
  pack(b, PB, s);
  gemm(PA, PB, a.rows(), b.rows(), a.K(), c, s, dstatus);
}

void Frag::contract_packed_b(const View& a, const Packed& PB, int N, const OutMap& c) {
  Packed PA;
  PA.p = scrA;
  PA.bf16 = PB.bf16;
  const size_t ea = static_cast<size_t>(a.rows()) * round_up(std::max(a.K(), 1), 64) * (PA.bf16 ? 4 : 8);
  if (ea > scr_bytes) {
    scratch_overflow = true;
    return;
  }
  pack(a, PA, s);
  gemm(PA, PB, a.rows(), N, a.K(), c, s, dstatus);
}

// ------------------------------------------------------------------------------------------------
// Integral assembly
// ------------------------------------------------------------------------------------------------
// Elements of each packing scratch buffer: the largest packed operand (rows x K rounded up to 64) of any
// contraction that goes through Frag::contract / contract_packed_b, for either ordering of nocc and nvir.
long long packing_scratch_elems(int o_, int v_, int N_) {
  const long long o = o_, v = v_, N = N_, n = o + v, oo = o * o, vv = v * v, ov = o * v;
  auto Kp = [](long long k) { return static_cast<long long>(round_up(static_cast<int>(std::max(k, 1LL)), 64)); };
  long long cap = 0;
  cap = std::max(cap, 1LL * N * o * Kp(v));
  cap = std::max(cap, 1LL * N * v * Kp(v));
  cap = std::max(cap, 1LL * N * v * Kp(o));
  cap = std::max(cap, 1LL * n * Kp(n));
  cap = std::max(cap, 1LL * v * Kp(1LL * N * o));
  cap = std::max(cap, 1LL * vv * Kp(N));
  cap = std::max(cap, 1LL * ov * Kp(N));
  cap = std::max(cap, 1LL * N * Kp(ov));
  cap = std::max(cap, 1LL * ov * Kp(ov));
  cap = std::max(cap, 1LL * v * Kp(1LL * N * v));
  cap = std::max(cap, 1LL * v * Kp(oo * v));
  cap = std::max(cap, 1LL * oo * Kp(vv));
  cap = std::max(cap, 1LL * oo * v * Kp(o));
  cap = std::max(cap, 1LL * vv * Kp(oo));
  cap = std::max(cap, 1LL * oo * v * Kp(v));
  cap = std::max(cap, 1LL * o * vv * Kp(o));
  // operands whose size grows with nocc (the largest when nocc > nvir)
  cap = std::max(cap, 1LL * N * o * Kp(o));   // B^_oo rows (Q, k), K i
  cap = std::max(cap, 1LL * n * Kp(1LL * N * o));  // core Hamiltonian exchange, rows p, K (Q, k)
  cap = std::max(cap, 1LL * oo * Kp(oo));     // hole-hole ladder W_kl^ij
  cap = std::max(cap, 1LL * o * Kp(1LL * N * v));  // B_ov rows i, K (Q, a); Mtmp
  cap = std::max(cap, 1LL * o * Kp(oo * v));  // g^_kilc rows i, K (k, l, c)
  cap = std::max(cap, 1LL * oo * Kp(N));      // (T): B_oo rows (j, l), K Q
  cap = std::max(cap, 1LL * oo * v * Kp(o));
  return cap;
}

int Frag::build(const double* eps_in, const double* B_in) {
  const long long n2 = 1LL * n * n, oo = 1LL * o * o, vv = 1LL * v * v, ov = 1LL * o * v;
  eps = static_cast<double*>(alloc(n * 8));
  Boo = static_cast<double*>(alloc(N * oo * 8));
  Bov = static_cast<double*>(alloc(N * ov * 8));
  Bvv = static_cast<double*>(alloc(N * vv * 8));
  h = static_cast<double*>(alloc(n2 * 8));
  ovov = static_cast<double*>(alloc(ov * ov * 8));
  Lpair = static_cast<double*>(alloc(ov * ov * 8));
  // per-iteration FP64 buffers
  const long long L = ov + oo * vv;
  xcur = static_cast<double*>(alloc(L * 8, true));
  xnew = static_cast<double*>(alloc(L * 8, true));
  enew = static_cast<double*>(alloc(L * 8, true));
  if (mixed) xbest = static_cast<double*>(alloc(L * 8, true));
  t2mp2 = static_cast<double*>(alloc(oo * vv * 8));
  Boo_h = static_cast<double*>(alloc(N * oo * 8));
  Bvo_h = static_cast<double*>(alloc(N * ov * 8));
  Bvv_h = static_cast<double*>(alloc(N * vv * 8));
  Xm = static_cast<double*>(alloc(n2 * 8));
  Ym = static_cast<double*>(alloc(n2 * 8));
  hh = static_cast<double*>(alloc(n2 * 8));
  tmpn = static_cast<double*>(alloc(n2 * 8));
  Fh = static_cast<double*>(alloc(n2 * 8));
  xq = static_cast<double*>(alloc(std::max(N, 1) * 8));
  tau = static_cast<double*>(alloc(oo * vv * 8));
  u = static_cast<double*>(alloc(oo * vv * 8));
  Rsym = static_cast<double*>(alloc(oo * vv * 8));
  S = static_cast<double*>(alloc(oo * vv * 8));
  Cp = static_cast<double*>(alloc(oo * vv * 8));
  Xk = static_cast<double*>(alloc(oo * vv * 8));
  Yk = static_cast<double*>(alloc(oo * vv * 8));
  Z = static_cast<double*>(alloc(oo * ov * 8));
  Wb = static_cast<double*>(alloc(oo * oo * 8));
  R1 = static_cast<double*>(alloc(ov * 8));
  Mtmp = static_cast<double*>(alloc(1LL * N * ov * 8));
  Gooov = static_cast<double*>(alloc(oo * ov * 8));
  Fvv2 = static_cast<double*>(alloc(vv * 8));
  Foo2 = static_cast<double*>(alloc(oo * 8));
  Eii = static_cast<double*>(alloc(oo * 8));
  np_o = o * (o + 1) / 2;
  nm_o = o * (o - 1) / 2;
  np_v = v * (v + 1) / 2;
  nm_v = v * (v - 1) / 2;
  Lp_out = static_cast<double*>(alloc(1LL * np_v * np_o * 8));
  Lm_out = static_cast<double*>(alloc(1LL * std::max(nm_v, 1) * std::max(nm_o, 1) * 8));
  Wy = static_cast<double*>(alloc(oo * oo * 8));
  // DIIS
  dm = std::max(0, std::min(opts.diis_space, 8));
  if (dm > 0) {
    dvec = static_cast<double*>(alloc(dm * L * 8, true));
    derr = static_cast<double*>(alloc(dm * L * 8, true));
  }
  G = static_cast<double*>(alloc(64 * 8, true));
  dctr = static_cast<int*>(alloc(16, true));
  coef = static_cast<double*>(alloc(8 * 8, true));
  dpart = static_cast<double*>(alloc(8 * 152 * 8, true));
  part = static_cast<double*>(alloc(152 * 32 * 8 * 4, true));
  scal = static_cast<double*>(alloc(16 * 8, true));
  dstatus = static_cast<int*>(alloc(16 * 4, true));
  if (h_ext) {
    h_scal = h_ext;
  } else if (cudaMallocHost(&h_scal, 16 * 8) != cudaSuccess) {
    h_scal = nullptr;
    oom = true;
  }
  const long long cap = packing_scratch_elems(o, v, N);
  scr_bytes = static_cast<size_t>(cap) * 8;
  scrA = alloc(scr_bytes);
  scrB = alloc(scr_bytes);
  splitk_cap = 1ull << 22;
  splitk = static_cast<double*>(alloc(splitk_cap * 8));
  use_workspace();
  if (oom) {
    set_error("device allocation failed in lnocc_build_ints");
    return LNOCC_ENOMEM;
  }

  // ---- slices of B (FP64 copies owned by the handle)
  LN_CUDA(cudaMemcpyAsync(eps, eps_in, n * 8, cudaMemcpyDeviceToDevice, s));
  permute(view(B_in, kOne, A(N, n2), A(o, n), kOne, kOne, A(o, 1)), Boo, 0.0, s);
  permute(view(B_in + o, kOne, A(N, n2), A(o, n), kOne, kOne, A(v, 1)), Bov, 0.0, s);
  permute(view(B_in + o * n + o, kOne, A(N, n2), A(v, n), kOne, kOne, A(v, 1)), Bvv, 0.0, s);
  if (opts.fault_inject & LNOCC_FAULT_NAN_INPUT) {
    const double nanv = std::nan("");
    LN_CUDA(cudaMemcpyAsync(Bov, &nanv, 8, cudaMemcpyHostToDevice, s));
  }

  // ---- core Hamiltonian h = f - sum_k [2(pq|kk) - (pk|kq)] (FP64)
  {
    std::vector<double> he(n2, 0.0);
    std::vector<double> eh(n);
    LN_CUDA(cudaMemcpyAsync(eh.data(), eps_in, n * 8, cudaMemcpyDeviceToHost, s));
    LN_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < o; ++i)
      for (int a = 0; a < v; ++a)
        if (!(eh[o + a] > eh[i])) {
          set_error("every virtual orbital energy must lie above every occupied one");
          return LNOCC_ENUMERIC;
        }
    for (int p = 0; p < n; ++p) he[p * n + p] = eh[p];
    LN_CUDA(cudaMemcpyAsync(h, he.data(), n2 * 8, cudaMemcpyHostToDevice, s));
    // x0[Q] = sum_k B_Qkk ; J: h -= 2 sum_Q B_Qpq x0_Q ; K: h += sum_{Q,k} B_Qpk B_Qkq
    launch_trace_oo(Boo, N, o, xq, s);
    launch_coulomb(B_in, n2, n, n, n, xq, N, -2.0, h, n, s);
    contract(view(B_in, kOne, kOne, A(n, n), kOne, A(N, n2), A(o, 1)),
             view(B_in, kOne, kOne, A(n, 1), kOne, A(N, n2), A(o, n)), out_rowmajor(h, n, 1.0, 1.0), true);
  }

  // ---- (ia|jb) = sum_Q B_Qia B_Qjb  (FP64 always: it feeds the energies)
  {  // symmetric in (ia) <-> (jb): the FP64 product computes one triangle of tiles and mirrors it
    Packed PA;
    PA.p = scrA;
    PA.bf16 = false;
    const View vb = view(Bov, kOne, kOne, A(static_cast<int>(ov), 1), kOne, kOne, A(N, ov));
    if (static_cast<size_t>(vb.rows()) * round_up(std::max(vb.K(), 1), 64) * 8 > scr_bytes) {
      scratch_overflow = true;
    } else {
      pack(vb, PA, s);
      gemm_f64_sym(PA, static_cast<int>(ov), out_rowmajor(ovov, ov), s);
    }
  }
  launch_pair_L(ovov, Lpair, o, v, s);
  launch_mp2_amps(ovov, eps, t2mp2, o, v, s);

  // ---- constant operands of the iteration, packed once per precision in use
  {
    const int st = build_consts(mixed);
    if (st != LNOCC_OK) return st;
    if (mixed && opts.n_refine > 0) {
      const int st2 = build_consts(false);
      if (st2 != LNOCC_OK) return st2;
    }
  }
  if (oom || scratch_overflow) {
    set_error(oom ? "device allocation failed" : "internal: packing scratch too small");
    return oom ? LNOCC_ENOMEM : LNOCC_EINVAL;
  }
  // MP2 energy (iteration 0)
  {
    const int g = launch_energy(nullptr, t2mp2, Lpair, part, o, v, s);
    launch_finish_sum(part, g, scal, s);
    LN_CUDA(cudaMemcpyAsync(h_scal, scal, 8, cudaMemcpyDeviceToHost, s));
    LN_CUDA(cudaStreamSynchronize(s));
    e_mp2 = h_scal[0];
  }
  return check_device();
}

// Constant packed operands of the iteration for one precision (bf = BF16 hi/lo, else FP64).
int Frag::build_consts(bool bf) {
  const long long oo = 1LL * o * o, vv = 1LL * v * v, ov = 1LL * o * v;
  Consts& c = cst[bf ? 1 : 0];
  const bool keep = mixed;
  mixed = bf;  // contract_packed_b follows the operand precision
  c.Bp_t = alloc_packed(np_o, np_v, bf);
  c.Bm_t = alloc_packed(std::max(nm_o, 1), std::max(nm_v, 1), bf);
  c.PBov = alloc_packed(static_cast<int>(ov), N, bf);
  c.PBoo = alloc_packed(static_cast<int>(oo), N, bf);
  c.PBvo = alloc_packed(static_cast<int>(ov), N, bf);
  c.PBvv = alloc_packed(static_cast<int>(vv), N, bf);
  if (c.PBov.p) pack(view(Bov, kOne, kOne, A(static_cast<int>(ov), 1), kOne, kOne, A(N, ov)), c.PBov, s);
  // (kc|ld) as rows (k,l), K (c,d)                       [Y_ij^kl]
  c.kl_cd = alloc_packed(static_cast<int>(oo), static_cast<int>(vv), bf);
  pack(view(ovov, kOne, A(o, ov * v), A(o, v), kOne, A(v, ov), A(v, 1)), c.kl_cd, s);
  // (kd|lc) as rows (k,c), K (l,d)                       [C2 intermediate]
  c.kc_ld = alloc_packed(static_cast<int>(ov), static_cast<int>(ov), bf);
  pack(view(ovov, kOne, A(o, ov * v), A(v, 1), kOne, A(o, v), A(v, ov)), c.kc_ld, s);
  // L_ldkc = 2(ld|kc) - (lc|kd) as rows (k,c), K (l,d)   [D2 intermediate]
  {
    double* Ltmp = Cp;  // borrow: [k][c][l][d]
    permute(view(ovov, kOne, A(o, v), A(v, 1), kOne, A(o, ov * v), A(v, ov), 2.0), Ltmp, 0.0, s);
    permute(view(ovov, kOne, A(o, v), A(v, ov), kOne, A(o, ov * v), A(v, 1), -1.0), Ltmp, 1.0, s);
    c.L = alloc_packed(static_cast<int>(ov), static_cast<int>(ov), bf);
    pack(view(Ltmp, kOne, kOne, A(static_cast<int>(ov), ov), kOne, kOne, A(static_cast<int>(ov), 1)), c.L, s);
  }
  // (kd|lc) as rows c, K (k,l,d)                          [E2: F_vv']
  c.c_kld = alloc_packed(v, static_cast<int>(oo * v), bf);
  pack(view(ovov, kOne, kOne, A(v, 1), A(o, v), A(o, ov * v), A(v, ov)), c.c_kld, s);

  // (ov|vv): (kc|bd) as rows (k,b), K (c,d)               [Z_ij^kb]
  {
    c.kb_cd = alloc_packed(static_cast<int>(ov), static_cast<int>(vv), bf);
    // B_vv packed once as rows (b,d), K = Q
    Packed PBvv = alloc_packed(static_cast<int>(vv), N, bf);
    pack(view(Bvv, kOne, kOne, A(static_cast<int>(vv), 1), kOne, kOne, A(N, vv)), PBvv, s);
    // chunks of k: G[k][c][b][d] (FP64 temp) -> packed rows (k,b), K (c,d)
    const long long per_k = v * vv;
    int kc = static_cast<int>(std::max(1LL, std::min<long long>(o, (1LL << 27) / per_k)));
    double* tmp = static_cast<double*>(alloc(static_cast<size_t>(kc) * per_k * 8));
    if (!tmp) {
      set_error("device allocation failed (ovvv chunk)");
      return LNOCC_ENOMEM;
    }
    for (int k0 = 0; k0 < o; k0 += kc) {
      const int nk = std::min(kc, o - k0);
      contract_packed_b(view(Bov + k0 * v, kOne, kOne, A(nk * v, 1), kOne, kOne, A(N, ov)), PBvv,
                        static_cast<int>(vv), out_rowmajor(tmp, vv));
      // tmp[k][c][b][d] -> rows (k0+k, b), K (c, d) of the packed operand
      pack_rows(view(tmp, kOne, A(nk, per_k), A(v, v), kOne, A(v, vv), A(v, 1)), c.kb_cd, k0 * v, s);
    }
    // ---- packed ladder integrals V+- from G[a][c][b][d] = (ac|bd), chunks of a
    c.Vp = alloc_packed(np_v, np_v, bf);
    c.Vm = alloc_packed(std::max(nm_v, 1), std::max(nm_v, 1), bf);
    // G chunks in FP32 on the mixed path (V+- are then split to BF16 hi/lo: FP32 carries more bits
    // than they keep), FP64 on the FP64 path; chunks of a of about 1 GB
    const size_t gsz = bf ? 4 : 8;
    int ac = static_cast<int>(std::max(1LL, std::min<long long>(v, (1LL << 30) / (per_k * static_cast<long long>(gsz)))));
    void* gtmp = alloc(static_cast<size_t>(ac) * per_k * gsz);
    if (!gtmp || oom) {
      set_error("device allocation failed (vvvv chunk)");
      return LNOCC_ENOMEM;
    }
    for (int a0 = 0; a0 < v; a0 += ac) {
      const int na = std::min(ac, v - a0);
      OutMap gm = out_rowmajor(bf ? nullptr : static_cast<double*>(gtmp), vv);
      if (bf) gm.dst32 = static_cast<float*>(gtmp);
      contract_packed_b(view(Bvv + static_cast<long long>(a0) * v, kOne, kOne, A(na * v, 1), kOne, kOne, A(N, vv)),
                        PBvv, static_cast<int>(vv), gm);
      launch_pack_vvvv(gtmp, bf, a0, na, v, c.Vp, c.Vm, s);
    }
    if (!pool) LN_CUDA(cudaStreamSynchronize(s));
    // the chunk temporaries are released right away
    for (void* p : {static_cast<void*>(tmp), gtmp, PBvv.p}) {
      dev_free(p);
      allocs.erase(std::find(allocs.begin(), allocs.end(), p));
    }
    device_bytes -= static_cast<long long>(kc) * per_k * 8 + static_cast<long long>(ac) * per_k * static_cast<long long>(gsz) +
                    static_cast<long long>(vv) * round_up(N, 64) * (bf ? 4 : 8);
  }
  mixed = keep;
  c.built = !oom;
  return oom ? LNOCC_ENOMEM : LNOCC_OK;
}

int Frag::check_device() {
  LN_CUDA(cudaGetLastError());
  int st[1] = {0};
  LN_CUDA(cudaMemcpyAsync(st, dstatus, 4, cudaMemcpyDeviceToHost, s));
  LN_CUDA(cudaStreamSynchronize(s));
  if (st[0] != 0) {
    set_error("device wait timed out (code " + std::to_string(st[0]) + ")");
    return LNOCC_ETIMEOUT;
  }
  if (scratch_overflow) {
    set_error("internal: packing scratch too small");
    return LNOCC_EINVAL;
  }
  return LNOCC_OK;
}

void Frag::pack_df() {
  const long long oo = 1LL * o * o, vv = 1LL * v * v, ov = 1LL * o * v;
  Consts& c = C();
  pack(view(Boo_h, kOne, kOne, A(static_cast<int>(oo), 1), kOne, kOne, A(N, oo)), c.PBoo, s);
  pack(view(Bvo_h, kOne, kOne, A(static_cast<int>(ov), 1), kOne, kOne, A(N, ov)), c.PBvo, s);
  pack(view(Bvv_h, kOne, kOne, A(static_cast<int>(vv), 1), kOne, kOne, A(N, vv)), c.PBvv, s);
}

// ------------------------------------------------------------------------------------------------
// One CCSD residual + Jacobi update: reads t1 = x, t2 = x + ov; writes xnew (t + R/D) and enew (R/D).
// Returns the rms of the update in *rms (device scalar scal[1]).
// ------------------------------------------------------------------------------------------------
void Frag::iterate(bool fp64_residual) {
  const bool keep_mixed = mixed;
  if (fp64_residual) mixed = false;  // refinement iterations: every contraction in FP64
  const long long n2 = 1LL * n * n, oo = 1LL * o * o, vv = 1LL * v * v, ov = 1LL * o * v, ovv = ov * v;
  const double* t1 = xcur;
  const double* t2 = xcur + ov;

  mark("start");
  // ---- T1-transformed DF factors
  // B^_oo[Q][k][i] = B_oo + sum_c B_ov[Q][k][c] t_i^c
  cudaMemcpyAsync(Boo_h, Boo, N * oo * 8, cudaMemcpyDeviceToDevice, s);
  contract(view(Bov, kOne, kOne, A(static_cast<int>(N * o), v), kOne, kOne, A(v, 1)),
           view(t1, kOne, kOne, A(o, v), kOne, kOne, A(v, 1)), out_rowmajor(Boo_h, o, 1.0, 1.0));
  // B^_vo[Q][a][i] = B_ov[Q][i][a] + sum_c B_vv[Q][a][c] t_i^c - sum_k t_k^a B^_oo[Q][k][i]
  permute(view(Bov, kOne, A(N, ov), A(v, 1), kOne, kOne, A(o, v)), Bvo_h, 0.0, s);
  // mixed path: B^_vv and the B_vv t1 part of B^_vo in one streaming pass over B_vv
  const bool fused_vv = mixed && o <= 32 && v <= 850;
  if (fused_vv) {
    launch_dress_vv(Bvv, Bov, t1, Bvv_h, Bvo_h, N, o, v, s);
  } else {
    contract(view(Bvv, kOne, kOne, A(static_cast<int>(N * v), v), kOne, kOne, A(v, 1)),
             view(t1, kOne, kOne, A(o, v), kOne, kOne, A(v, 1)), out_rowmajor(Bvo_h, o, 1.0, 1.0));
  }
  contract(view(t1, kOne, kOne, A(v, 1), kOne, kOne, A(o, v)),
           view(Boo_h, kOne, A(N, oo), A(o, 1), kOne, kOne, A(o, o)),
           OutMap{Bvo_h, 0, o, ov, 1, 1 << 30, o, -1.0, 1.0});
  // B^_vv[Q][a][c] = B_vv - sum_k t_k^a B_ov[Q][k][c]
  if (!fused_vv) {
    cudaMemcpyAsync(Bvv_h, Bvv, N * vv * 8, cudaMemcpyDeviceToDevice, s);
    contract(view(t1, kOne, kOne, A(v, 1), kOne, kOne, A(o, v)),
             view(Bov, kOne, A(N, ov), A(v, 1), kOne, kOne, A(o, v)), OutMap{Bvv_h, 0, v, vv, 1, 1 << 30, v, -1.0, 1.0});
  }

  pack_df();
  const Consts& K = C();
  mark("dress");
  // ---- T1-transformed Fock matrix F^ = (1-T) h (1+T) + sum_Q [2 B^_Qpq x_Q - sum_k B^_Qpk B^_Qkq]
  launch_hhat(h, t1, tmpn, Fh, o, v, s);
  launch_trace_oo(Boo_h, N, o, xq, s);
  // Coulomb part, block by block (F^ laid out n x n: oo | ov / vo | vv)
  auto coul = [&](const double* Bblk, int rows, int cols, long long qstride, double* dst, long long ld) {
    launch_coulomb(Bblk, qstride, rows, cols, cols, xq, N, 2.0, dst, ld, s);
  };
  coul(Boo_h, o, o, oo, Fh, n);
  coul(Bov, o, v, ov, Fh + o, n);
  coul(Bvo_h, v, o, ov, Fh + o * n, n);
  coul(Bvv_h, v, v, vv, Fh + o * n + o, n);
  // exchange part: F_pq -= sum_{Q,k} B^_Qpk B^_Qkq
  {
    // oo: B^_oo[Q][p][k] B^_oo[Q][k][q]
    contract(view(Boo_h, kOne, kOne, A(o, o), kOne, A(N, oo), A(o, 1)),
             view(Boo_h, kOne, kOne, A(o, 1), kOne, A(N, oo), A(o, o)), out_rowmajor(Fh, n, -1.0, 1.0));
    // ov: B^_oo[Q][p][k] B_ov[Q][k][c]
    contract(view(Boo_h, kOne, kOne, A(o, o), kOne, A(N, oo), A(o, 1)),
             view(Bov, kOne, kOne, A(v, 1), kOne, A(N, ov), A(o, v)), out_rowmajor(Fh + o, n, -1.0, 1.0));
    // vo: B^_vo[Q][a][k] B^_oo[Q][k][i]
    contract(view(Bvo_h, kOne, kOne, A(v, o), kOne, A(N, ov), A(o, 1)),
             view(Boo_h, kOne, kOne, A(o, 1), kOne, A(N, oo), A(o, o)), out_rowmajor(Fh + o * n, n, -1.0, 1.0));
    // vv: B^_vo[Q][a][k] B_ov[Q][k][c]
    contract(view(Bvo_h, kOne, kOne, A(v, o), kOne, A(N, ov), A(o, 1)),
             view(Bov, kOne, kOne, A(v, 1), kOne, A(N, ov), A(o, v)), out_rowmajor(Fh + o * n + o, n, -1.0, 1.0));
  }

  mark("fock");
  // ---- amplitude-derived arrays
  launch_tau(t1, nullptr, tau, o, v, s);  // t1 (x) t1
  launch_u(t2, u, o, v, s);

  mark("tau_u");
  // ---- Rsym = g^_aibj : (a,i) x (b,j) over Q, written to [i][j][a][b]
  gemm(K.PBvo, K.PBvo, static_cast<int>(ov), static_cast<int>(ov), N, OutMap{Rsym, v, o * vv, 1, vv, o, o, 1.0, 0.0},
       s, dstatus);
  mark("g_aibj");
  // particle-particle ladder with the packed undressed integrals
  launch_ladder_ops(t2, C().Bp_t, C().Bm_t, o, v, s);
  gemm(C().Vp, C().Bp_t, np_v, np_o, np_v, out_rowmajor(Lp_out, np_o), s, dstatus);
  if (nm_v > 0 && nm_o > 0)
    gemm(C().Vm, C().Bm_t, nm_v, nm_o, nm_v, out_rowmajor(Lm_out, nm_o), s, dstatus);
  else cudaMemsetAsync(Lm_out, 0, 8, s);
  launch_ladder_unpack(Lp_out, Lm_out, Rsym, o, v, np_o, std::max(nm_o, 1), s);
  mark("ladder");
  // Wy[i][j][k][l] = Y_ij^kl = sum_cd (kc|ld) t_ij^cd ; Wb = g^_kilj + Y_ij^kl
  contract_packed_b(view(t2, kOne, kOne, A(static_cast<int>(oo), vv), kOne, kOne, A(static_cast<int>(vv), 1)),
                    C().kl_cd, static_cast<int>(oo), out_rowmajor(Wy, oo));
  gemm(K.PBoo, K.PBoo, static_cast<int>(oo), static_cast<int>(oo), N, OutMap{Wb, o, oo * o, 1, oo, o, o, 1.0, 0.0}, s,
       dstatus);
  permute(view(Wy, kOne, kOne, A(static_cast<int>(oo), oo), kOne, kOne, A(static_cast<int>(oo), 1)), Wb, 1.0, s);
  mark("Y_Wb");
  // Rsym += sum_kl t_kl^ab Wb_ij^kl + sum_kl t_k^a t_l^b Y_ij^kl   (tau holds t1 (x) t1 here)
  contract(view(Wb, kOne, kOne, A(static_cast<int>(oo), oo), kOne, kOne, A(static_cast<int>(oo), 1)),
           view(t2, kOne, kOne, A(static_cast<int>(vv), 1), kOne, kOne, A(static_cast<int>(oo), vv)),
           out_rowmajor(Rsym, vv, 1.0, 1.0));
  contract(view(Wy, kOne, kOne, A(static_cast<int>(oo), oo), kOne, kOne, A(static_cast<int>(oo), 1)),
           view(tau, kOne, kOne, A(static_cast<int>(vv), 1), kOne, kOne, A(static_cast<int>(oo), vv)),
           out_rowmajor(Rsym, vv, 1.0, 1.0));

  mark("hh_ladder");
  // ---- S (pre-P part)
  // Z_ij^kb = sum_cd (kc|bd) t_ij^cd ; S[i][j][a][b] = -sum_k t_k^a Z_ij^kb
  contract_packed_b(view(t2, kOne, kOne, A(static_cast<int>(oo), vv), kOne, kOne, A(static_cast<int>(vv), 1)),
                    C().kb_cd, static_cast<int>(ov), out_rowmajor(Z, ov));
  mark("Z");
  contract(view(Z, kOne, A(static_cast<int>(oo), ov), A(v, 1), kOne, kOne, A(o, v)),
           view(t1, kOne, kOne, A(v, 1), kOne, kOne, A(o, v)), OutMap{S, vv, 1, 0, v, v, 1 << 30, -1.0, 0.0});
  mark("ZT");
  // E2: Fvv'_bc = F^_bc - sum_kld u_kl^bd (ld|kc); S += sum_c t_ij^ac Fvv'_bc
  permute(view(Fh + o * n + o, kOne, kOne, A(v, n), kOne, kOne, A(v, 1)), Fvv2, 0.0, s);
  contract_packed_b(view(u, kOne, kOne, A(v, v), kOne, A(static_cast<int>(oo), vv), A(v, 1)), C().c_kld, v,
                    out_rowmajor(Fvv2, v, -1.0, 1.0));
  mark("Fvv");
  contract(view(t2, kOne, kOne, A(static_cast<int>(oo * v), v), kOne, kOne, A(v, 1)),
           view(Fvv2, kOne, kOne, A(v, v), kOne, kOne, A(v, 1)), out_rowmajor(S, v, 1.0, 1.0));
  mark("E2a");
  // Foo'_kj = F^_kj + sum_lcd u_lj^cd (kd|lc); S -= sum_k t_ik^ab Foo'_kj
  permute(view(Fh, kOne, kOne, A(o, n), kOne, kOne, A(o, 1)), Foo2, 0.0, s);
  // Mtmp[Q][d][i] = sum_kc B_Qkc u_ki^cd (shared with the singles term A1);
  // sum_lcd u_lj^cd (kd|lc) = sum_{Q,d} B_Qkd Mtmp[Q][d][j]
  // (u rows taken as (i, d) with d contiguous so that the operand pack reads coalesced; the output
  // columns (i, d) land at Mtmp[Q][d][i])
  contract(view(Bov, kOne, kOne, A(N, ov), kOne, kOne, A(static_cast<int>(ov), 1)),
           view(u, kOne, A(o, vv), A(v, 1), kOne, A(o, o * vv), A(v, v)),
           OutMap{Mtmp, 0, ov, 1, o, 1 << 30, v, 1.0, 0.0});
  contract(view(Bov, kOne, kOne, A(o, v), kOne, A(N, ov), A(v, 1)),
           view(Mtmp, kOne, kOne, A(o, 1), kOne, A(N, ov), A(v, o)), out_rowmajor(Foo2, o, 1.0, 1.0));
  mark("Foo");
  if (mixed && o <= 32)
    launch_e2_occ(t2, Foo2, S, o, v, s);  // length-o contraction: one streaming pass
  else
    contract(view(t2, kOne, A(o, o * vv), A(static_cast<int>(vv), 1), kOne, kOne, A(o, vv)),
             view(Foo2, kOne, kOne, A(o, 1), kOne, kOne, A(o, o)),
             OutMap{S, o * vv, 1, 0, vv, static_cast<int>(vv), 1 << 30, -1.0, 1.0});
  mark("E2b");
  // C2 intermediate X_kiac = g^_kiac - 1/2 sum_dl t_li^ad (kd|lc), stored [k][i][a][c]
  gemm(K.PBoo, K.PBvv, static_cast<int>(oo), static_cast<int>(vv), N, out_rowmajor(Xk, vv), s, dstatus);
  contract_packed_b(view(t2, kOne, A(o, vv), A(v, v), kOne, A(o, o * vv), A(v, 1)), C().kc_ld, static_cast<int>(ov),
                    OutMap{Xk, vv, v, o * vv, 1, v, v, -0.5, 1.0});
  mark("X");
  // Cp[(j,b),(i,a)] = sum_kc t_kj^bc X_kiac
  contract(view(t2, kOne, A(o, vv), A(v, v), kOne, A(o, o * vv), A(v, 1)),
           view(Xk, kOne, A(o, vv), A(v, v), kOne, A(o, o * vv), A(v, 1)), out_rowmajor(Cp, ov));
  mark("Cp");
  // D2 intermediate Y[i][a][k][c] = 2 g^_aikc - g^_kiac + 1/2 sum_dl u_il^ad L_ldkc
  gemm(K.PBvo, K.PBov, static_cast<int>(ov), static_cast<int>(ov), N, OutMap{Yk, ov, ovv, 0, 1, o, 1 << 30, 2.0, 0.0},
       s, dstatus);
  gemm(K.PBoo, K.PBvv, static_cast<int>(oo), static_cast<int>(vv), N, OutMap{Yk, v, ovv, ov, 1, o, v, -1.0, 1.0}, s,
       dstatus);
  contract_packed_b(view(u, kOne, A(o, o * vv), A(v, v), kOne, A(o, vv), A(v, 1)), C().L, static_cast<int>(ov),
                    out_rowmajor(Yk, ov, 0.5, 1.0));
  mark("Yint");
  // S += 1/2 sum_kc u_jk^bc Y_aikc  -> rows (j,b), cols (i,a)
  contract(view(u, kOne, A(o, o * vv), A(v, v), kOne, A(o, vv), A(v, 1)),
           view(Yk, kOne, kOne, A(static_cast<int>(ov), ov), kOne, kOne, A(static_cast<int>(ov), 1)),
           OutMap{S, vv, 1, o * vv, v, v, v, 0.5, 1.0});

  mark("D2");
  // ---- singles residual R1[i][a]
  // A1 via DF: R1 += sum_{Q,d} B^_Qad Mtmp[Q][d][i]
  contract(view(Bvv_h, kOne, kOne, A(v, v), kOne, A(N, vv), A(v, 1)),
           view(Mtmp, kOne, kOne, A(o, 1), kOne, A(N, ov), A(v, o)), OutMap{R1, 0, 1, 0, v, 1 << 30, 1 << 30, 1.0, 0.0});
  mark("A1");
  // B1: R1 -= sum_klc u_kl^ac g^_kilc ; g^_kilc stored [i][k][l][c]
  gemm(K.PBoo, K.PBov, static_cast<int>(oo), static_cast<int>(ov), N, OutMap{Gooov, ov, o * ov, 0, 1, o, 1 << 30, 1.0, 0.0},
       s, dstatus);
  contract(view(u, kOne, kOne, A(v, v), kOne, A(static_cast<int>(oo), vv), A(v, 1)),
           view(Gooov, kOne, kOne, A(o, o * ov), kOne, kOne, A(static_cast<int>(o * ov), 1)),
           OutMap{R1, 0, 1, 0, v, 1 << 30, 1 << 30, -1.0, 1.0});
  mark("B1");
  // C1: R1 += sum_kc u_ik^ac F^_kc
  contract(view(u, kOne, A(o, o * vv), A(v, v), kOne, A(o, vv), A(v, 1)),
           view(Fh + o, kOne, kOne, A(1, 0), kOne, A(o, n), A(v, 1)), out_rowmajor(R1, 1, 1.0, 1.0));

  mark("C1");
  // ---- update: t2n = t2 + R/D, t1n = t1 + (R1 + F^_ai)/D1; rms of the update
  const int g2 = launch_assemble(Rsym, S, Cp, t2, eps, xnew + ov, enew + ov, part, o, v, s);
  // F^_vo as [a][i] (row stride n) -> compact copy
  permute(view(Fh + o * n, kOne, kOne, A(v, n), kOne, kOne, A(o, 1)), tmpn, 0.0, s);
  const int g1 = launch_update_t1(R1, tmpn, t1, eps, xnew, enew, part + g2, o, v, s);
  launch_finish_sum(part, g1 + g2, scal + 1, s);
  mark("update");
  mixed = keep_mixed;
  (void)n2;
}

double Frag::energy_of(const double* x) {
  const int g = launch_energy(x, x + 1LL * o * v, Lpair, part, o, v, s);
  launch_finish_sum(part, g, scal, s);
  return 0.0;
}

// ------------------------------------------------------------------------------------------------
// One CCSD iteration on stream s: residual and update, DIIS extrapolation into xcur, the energy of
// xcur and the copy of (energy, squared update norm) to the pinned host buffer h_scal.
void Frag::step(bool fp64_residual, bool use_diis) {
  const long long L = 1LL * o * v + 1LL * o * o * v * v;
  iterate(fp64_residual);
  if (use_diis)
    launch_diis_step(xnew, enew, dvec, derr, L, dm, dctr, dpart, G, coef, xcur, s);
  else
    cudaMemcpyAsync(xcur, xnew, L * 8, cudaMemcpyDeviceToDevice, s);
  energy_of(xcur);
  mark("diis_energy");
  cudaMemcpyAsync(h_scal, scal, 16, cudaMemcpyDeviceToHost, s);
}

// Runs step() eagerly, or through the captured graph. The graph holds the FP64/mixed residual of the
// fragment's own precision only (FP64 refinement iterations always run eagerly). Capture happens on a
// private stream in thread-local mode, so other host threads may allocate meanwhile; if capture or
// instantiation fails the solve continues eagerly.
int Frag::launch_step(bool fp64_residual, bool use_diis, bool use_graph) {
  if (!use_graph || fp64_residual || prof || graph_failed) {
    step(fp64_residual, use_diis);
    return LNOCC_OK;
  }
  if (!gexec) {
    if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      graph_failed = true;
      step(fp64_residual, use_diis);
      return LNOCC_OK;
    }
    cudaStream_t user = s;
    s = cap_stream;
    const long long n0 = thread_launch_counter();
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      step(false, use_diis);
      ok = cudaStreamEndCapture(s, &g) == cudaSuccess && g;
    }
    s = user;
    graph_kernels = thread_launch_counter() - n0;
    // nothing ran during capture: take the captured launches back out of the counters
    launch_counter().fetch_sub(graph_kernels, std::memory_order_relaxed);
    thread_launch_counter() -= graph_kernels;
    if (ok) ok = cudaGraphInstantiate(&gexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      gexec = nullptr;
      graph_failed = true;
      step(fp64_residual, use_diis);
      return LNOCC_OK;
    }
  }
  LN_CUDA(cudaGraphLaunch(gexec, s));
  count_launch(graph_kernels);
  return LNOCC_OK;
}

// The learned guess only changes where the iterations start: a solve from it that fails to converge
// or turns non-finite is repeated from the MP2 guess (same convergence test), and the iterations of
// both attempts are counted.
int Frag::solve_with_fallback(int guess, const double* t1_in, const double* t2_in) {
  mlp_used = mlp_fallback = false;
  const int st = solve(guess, t1_in, t2_in);
  if (guess != LNOCC_GUESS_MLP || st == LNOCC_OK || (st != LNOCC_ENOCONV && st != LNOCC_ENUMERIC)) return st;
  const int first = n_iter;
  mlp_fallback = true;
  const int st2 = solve(LNOCC_GUESS_MP2, nullptr, nullptr);
  n_iter += first;
  return st2;
}

int Frag::solve(int guess, const double* t1_in, const double* t2_in) {
  const long long ov = 1LL * o * v, L = ov + 1LL * o * o * v * v;
  cudaMemsetAsync(dstatus, 0, 16 * 4, s);
  if (guess == LNOCC_GUESS_GIVEN) {
    if (!t1_in || !t2_in) {
      set_error("LNOCC_GUESS_GIVEN needs t1_in and t2_in");
      return LNOCC_EINVAL;
    }
    LN_CUDA(cudaMemcpyAsync(xcur, t1_in, ov * 8, cudaMemcpyDeviceToDevice, s));
    LN_CUDA(cudaMemcpyAsync(xcur + ov, t2_in, (L - ov) * 8, cudaMemcpyDeviceToDevice, s));
  } else if (guess == LNOCC_GUESS_MLP) {
    if (!mlp) {
      set_error("LNOCC_GUESS_MLP needs a model attached with lnocc_frag_set_mlp");
      return LNOCC_EINVAL;
    }
    // t1 = 0, t2 = learned guess; a guess with any non-finite element is replaced by the MP2 guess
    LN_CUDA(cudaMemsetAsync(xcur, 0, ov * 8, s));
    const int st = mlp_guess(*mlp, o, v, t2mp2, eps, ovov, xcur + ov, dstatus, s);
    if (st != LNOCC_OK) return st;
    launch_finite(xcur + ov, L - ov, dstatus + 1, s);
    int flag[2] = {0, 0};
    LN_CUDA(cudaMemcpyAsync(flag, dstatus, 8, cudaMemcpyDeviceToHost, s));
    LN_CUDA(cudaStreamSynchronize(s));
    if (flag[0] != 0) {
      set_error("learned-guess kernel: device wait timed out");
      return LNOCC_ETIMEOUT;
    }
    mlp_used = flag[1] == 0;
    mlp_fallback = !mlp_used;
    if (!mlp_used) {
      LN_CUDA(cudaMemsetAsync(dstatus, 0, 16 * 4, s));
      LN_CUDA(cudaMemcpyAsync(xcur + ov, t2mp2, (L - ov) * 8, cudaMemcpyDeviceToDevice, s));
    }
  } else {
    LN_CUDA(cudaMemsetAsync(xcur, 0, ov * 8, s));
    LN_CUDA(cudaMemcpyAsync(xcur + ov, t2mp2, (L - ov) * 8, cudaMemcpyDeviceToDevice, s));
  }
  energy_of(xcur);
  LN_CUDA(cudaMemcpyAsync(h_scal, scal, 8, cudaMemcpyDeviceToHost, s));
  LN_CUDA(cudaStreamSynchronize(s));
  double e_old = h_scal[0];
  converged = false;
  n_iter = 0;
  floor_spread = 0.0;
  n_refined = 0;
  diis_restarts = 0;
  const bool use_diis = dm > 0 && !(opts.fault_inject & LNOCC_FAULT_ZERO_DIIS);
  LN_CUDA(cudaMemsetAsync(dctr, 0, 16, s));
  int refine_left = mixed ? opts.n_refine : 0;
  bool refining = false;
  const double tol_r = opts.conv_rms, tol_e = opts.conv_energy;
  // Mixed path: BF16x3 residuals carry rounding noise, so the update stalls at a noise floor (rms
  // ~1e-10..1e-7) instead of reaching the FP64 thresholds, and near it DIIS can extrapolate the noise
  // into growing excursions. The solver therefore keeps the amplitudes of the lowest-rms step (xbest),
  // restarts DIIS from them when the rms grows 100-fold past that best, and declares the floor reached
  // when the best rms has not improved by 20% for kFloorWin iterations (or rms has stopped falling and
  // the energy moves by < 1e-7). At the floor the energy spread over the window decides: below 1e-7 Eh
  // the solve is converged; otherwise FP64-residual iterations (at most n_refine) continue from xbest
  // until rms < conv_rms and |dE| < max(conv_energy, 1e-8), and with n_refine = 0 the call reports
  // ENOCONV with the energy of xbest.
  constexpr int kFloorWin = 6;
  constexpr double kSpreadTol = 1e-7;
  double best_rms = INFINITY, anchor_rms = INFINITY, e_best = e_old;
  int best_it = 0;
  std::vector<double> hist_rms, hist_de, hist_e;
  bool stop_noconv = false;
  for (int it = 1; it <= opts.max_iter; ++it) {
    // the first iteration runs eagerly (first launches set kernel attributes); later ones replay a
    // captured graph of the same launches when opts.graph is set
    const int st_step = launch_step(refining, use_diis, opts.graph != 0 && it >= 2);
    if (st_step != LNOCC_OK) return st_step;
    LN_CUDA(cudaStreamSynchronize(s));
    LN_CUDA(cudaGetLastError());
    prof_flush();
    const double e = h_scal[0];
    const double rms = std::sqrt(h_scal[1] / static_cast<double>(L));
    n_iter = it;
    last_rms = rms;
    if (opts.verbose)
      std::fprintf(stderr, "lnocc ccsd it %3d  E = %.14f  dE = %.3e  rms = %.3e%s\n", it, e, e - e_old, rms,
                   refining ? "  (fp64 residual)" : "");
    if (!std::isfinite(e) || !std::isfinite(rms)) {
      e_ccsd = e;
      set_error("non-finite CCSD energy or residual");
      return LNOCC_ENUMERIC;
    }
    const bool mixed_now = mixed && !refining;
    // energy threshold: conv_energy on the FP64 path; at least 1e-8 Eh for mixed and refinement
    // iterations (a refinement from a noisy start settles to ~1e-9 rms with 1e-9..1e-8 Eh energy
    // steps, well inside the 1e-6 Eh budget)
    const double te = mixed ? std::max(tol_e, 1e-8) : tol_e;
    hist_rms.push_back(rms);
    hist_de.push_back(std::fabs(e - e_old));
    hist_e.push_back(e);
    e_old = e;
    if (refining) --refine_left;
    bool conv = rms < tol_r && hist_de.back() < te;
    if (mixed_now && !conv) {
      if (rms < best_rms) {
        if (rms < 0.8 * anchor_rms) {  // a 20% gain over the rms of the last marked improvement
          anchor_rms = rms;
          best_it = it;
        }
        best_rms = rms;
        e_best = e;
        LN_CUDA(cudaMemcpyAsync(xbest, xcur, L * 8, cudaMemcpyDeviceToDevice, s));
      } else if (use_diis && best_rms < 1e-4 && rms > 100.0 * best_rms && diis_restarts < 4) {
        // DIIS excursion: restart the subspace from the best amplitudes
        ++diis_restarts;
        LN_CUDA(cudaMemcpyAsync(xcur, xbest, L * 8, cudaMemcpyDeviceToDevice, s));
        LN_CUDA(cudaMemsetAsync(dctr, 0, 16, s));
        e_old = e_best;
        best_it = it;
        anchor_rms = best_rms;
        continue;
      }
      bool floor = best_rms < 1e-5 && it - best_it >= kFloorWin;
      if (!floor && hist_rms.size() >= 6) {
        const double best_before = *std::min_element(hist_rms.begin(), hist_rms.end() - 4);
        const double best_recent = *std::min_element(hist_rms.end() - 4, hist_rms.end());
        const double de_recent = *std::max_element(hist_de.end() - 4, hist_de.end());
        floor = best_recent > 0.8 * best_before && de_recent < kSpreadTol && rms < 1e-5;
      }
      if (floor) {
        const size_t w = std::min<size_t>(kFloorWin, hist_e.size());
        const auto mm = std::minmax_element(hist_e.end() - w, hist_e.end());
        floor_spread = *mm.second - *mm.first;
        if (floor_spread < kSpreadTol) {
          conv = true;
        } else {
          // too noisy to meet the energy tolerance: continue from the best amplitudes
          LN_CUDA(cudaMemcpyAsync(xcur, xbest, L * 8, cudaMemcpyDeviceToDevice, s));
          e_old = e_best;
          if (refine_left > 0) {
            refining = true;
            LN_CUDA(cudaMemsetAsync(dctr, 0, 16, s));
            continue;
          }
          stop_noconv = true;
          break;
        }
      }
    }
    if (refining) ++n_refined;
    if (conv) {
      converged = true;
      break;
    }
    if (refining && refine_left <= 0) break;
  }
  if (stop_noconv || (mixed && !converged && !refining && best_rms < INFINITY && xbest)) {
    // not converged on the mixed path: leave the best amplitudes (and their energy) as the result
    LN_CUDA(cudaMemcpyAsync(xcur, xbest, L * 8, cudaMemcpyDeviceToDevice, s));
    e_old = e_best;
  }
  e_ccsd = e_old;
  have_amps = true;
  prof_print("ccsd");
  const int st = check_device();
  if (st != LNOCC_OK) return st;
  if (!converged) {
    if (stop_noconv)
      set_error(("CCSD (mixed) stopped at its noise floor with an energy spread of " + std::to_string(floor_spread) +
                 " Eh over its last iterations, above 1e-7 Eh: set opts.n_refine for FP64-residual refinement")
                    .c_str());
    else if (n_refined > 0 && n_iter < opts.max_iter)
      set_error("CCSD FP64 refinement did not converge within opts.n_refine iterations");
    else
      set_error("CCSD did not converge within max_iter");
    return LNOCC_ENOCONV;
  }
  return LNOCC_OK;
}

// Pair matrix E_ii' = sum_jab tau_ij^ab L[i'][j][a][b] (FP64), then the LO projection.
int Frag::fragment_energy(int nlo, const double* U, double* e_ccsd_frag, double* e_mp2_frag, double* e_dev) {
  const long long ov = 1LL * o * v;
  const long long kk = ov * v;  // (j,a,b)
  auto pair_and_project = [&](const double* t1, const double* t2, double* out_host, double* out_dev) -> int {
    if (t1) {
      launch_tau(t1, t2, tau, o, v, s);
    } else {
      LN_CUDA(cudaMemcpyAsync(tau, t2, 1LL * o * o * v * v * 8, cudaMemcpyDeviceToDevice, s));
    }
    launch_pair_dots(tau, Lpair, o, kk, Eii, s);
    launch_project(Eii, U, o, nlo, scal + 2, s);
    if (out_dev) {
      LN_CUDA(cudaMemcpyAsync(out_dev, scal + 2, 8, cudaMemcpyDeviceToDevice, s));
      return LNOCC_OK;
    }
    LN_CUDA(cudaMemcpyAsync(h_scal + 2, scal + 2, 8, cudaMemcpyDeviceToHost, s));
    LN_CUDA(cudaStreamSynchronize(s));
    *out_host = h_scal[2];
    return LNOCC_OK;
  };
  if (e_dev) {
    if (!have_amps) {
      set_error("lnocc_fragment_energy_device: no CCSD amplitudes (call lnocc_ccsd first)");
      return LNOCC_EINVAL;
    }
    const int st = pair_and_project(xcur, xcur + ov, nullptr, e_dev);
    if (st) return st;
    return pair_and_project(nullptr, t2mp2, nullptr, e_dev + 1);
  }
  if (e_ccsd_frag) {
    if (!have_amps) {
      set_error("lnocc_fragment_energy: no CCSD amplitudes (call lnocc_ccsd first)");
      return LNOCC_EINVAL;
    }
    const int st = pair_and_project(xcur, xcur + ov, e_ccsd_frag, nullptr);
    if (st) return st;
  }
  if (e_mp2_frag) {
    const int st = pair_and_project(nullptr, t2mp2, e_mp2_frag, nullptr);
    if (st) return st;
  }
  return check_device();
}

}  // namespace lnocc
