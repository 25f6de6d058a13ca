// Launch wrappers of the FP64 element-wise / reduction kernels (ccsd_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace lnocc {
void launch_tau(const double* t1, const double* t2, double* tau, int o, int v, cudaStream_t s);
void launch_u(const double* t2, double* u, int o, int v, cudaStream_t s);
void launch_ladder_ops(const double* t2, Packed& Bp, Packed& Bm, int o, int v, cudaStream_t s);
void launch_ladder_unpack(const double* Lp, const double* Lm, double* R, int o, int v, int ldp, int ldm,
                          cudaStream_t s);
int launch_assemble(const double* Rsym, const double* S, const double* Cp, const double* t2, const double* eps,
                    double* t2n, double* err, double* part, int o, int v, cudaStream_t s);
int launch_update_t1(const double* R1, const double* Fvo, const double* t1, const double* eps, double* t1n,
                     double* err, double* part, int o, int v, cudaStream_t s);
// E = sum tau_ij^ab Lpair[i][j][a][b], Lpair = 2(ia|jb) - (ib|ja); returns the number of partials
int launch_energy(const double* t1, const double* t2, const double* Lpair, double* part, int o, int v,
                  cudaStream_t s);
void launch_finish_sum(const double* part, int n, double* out, cudaStream_t s);
void launch_mp2_amps(const double* ovov, const double* eps, double* t2, int o, int v, cudaStream_t s);
// One Pulay DIIS step with the subspace bookkeeping in device memory (ctr[2], zero before the first
// step): push (x_new, e_new) into slot ctr[0] % mmax, update the overlap matrix G, solve for the
// coefficients and write the extrapolated vector to out.
void launch_diis_step(const double* x_new, const double* e_new, double* xs, double* es, long long len, int mmax,
                      int* ctr, double* part, double* G, double* coef, double* out, cudaStream_t s);
void launch_project(const double* E, const double* U, int o, int nlo, double* out, cudaStream_t s);
void launch_pair_dots(const double* tau, const double* L, int o, long long K, double* E, cudaStream_t s);
void launch_pair_L(const double* ovov, double* L, int o, int v, cudaStream_t s);
// G[al][c][b][d] = (a0+al c|b d), FP32 (g32) or FP64 -> packed V+- rows (a <= b)
void launch_pack_vvvv(const void* G, bool g32, int a0, int na, int v, Packed& Vp, Packed& Vm, cudaStream_t s);
void launch_dress_mats(const double* t1, double* X, double* Y, int o, int v, cudaStream_t s);
void launch_hhat(const double* h, const double* t1, double* g, double* out, int o, int v, cudaStream_t s);
void launch_trace_oo(const double* Boo, int naux, int o, double* xq, cudaStream_t s);
void launch_coulomb(const double* B, long long qstride, int rows, int cols, long long rstride, const double* x,
                    int naux, double alpha, double* dst, long long ld, cudaStream_t s);
void launch_finite(const double* x, long long n, int* flag, cudaStream_t s);
// B^_vv = B_vv - t1^T B_ov and B^_vo += B_vv t1^T in one pass over B_vv (nocc <= 32, 2*MAXO*v*4 bytes of
// shared memory, v <= 1700 for MAXO = 16 / 850 for 32); FP32 products and sums, FP64 results
void launch_dress_vv(const double* Bvv, const double* Bov, const double* t1, double* Bvv_h, double* Bvo_h, int naux,
                     int o, int v, cudaStream_t s);
// S[i][j][a][b] -= sum_k t2[i][k][a][b] F[k][j], nocc <= 32, FP32 products and sums
void launch_e2_occ(const double* t2, const double* F, double* S, int o, int v, cudaStream_t s);
}  // namespace lnocc
