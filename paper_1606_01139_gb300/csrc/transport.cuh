// Kernels of T(E) and its adjoint (see transport.cu).
#pragma once

#include "swi_internal.cuh"

namespace swi {

void launch_wbuild(const double2* MR, const double2* ML, int n, double2* R, double2* L, double2* W, cudaStream_t s,
                   long long* launches);
void launch_transmission(const double2* W, const double2* eps, int n, const double* E, int nE, double* T,
                         double* dTdE, cudaStream_t s, long long* launches);
void launch_gradM(const double2* R, const double2* L, const double2* eps, int n, const double* E, const double* w,
                  int nE, double2* M, cudaStream_t s, long long* launches);
// FP32 contractions (transport_f32.cu).  Projections over the rows [lo, hi) of
// each absorber: part holds proj_f32_chunks(n, hiR - loR) + proj_f32_chunks(n,
// hiL - loL) matrices of n x n complex64; writes R, L, W (complex128) and the
// complex64 copies R32, L32.
int proj_f32_chunks(int n, long long rows);
void launch_proj_f32(const double2* U, int ldu, int n, const double* gR, long long loR, long long hiR,
                     const double* gL, long long loL, long long hiL, float2* part, double2* R, double2* L,
                     double2* W, float2* R32, float2* L32, cudaStream_t s, long long* launches);
// out[r] = 2 Re sum_ac U_ra M_ac U_rc with M = sum_e w_e D_e R conj(D_e) L^T D_e;
// gt: nE x n complex64 scratch (the energy table), M: n x n complex64 scratch
void launch_grad_f32(const float2* R32, const float2* L32, const double2* eps, int n, const double* E,
                     const double* w, int nE, float2* gt, float2* M, const double2* U, int ldu, long long N,
                     double* out, cudaStream_t s, long long* launches);
void launch_rowdot(const double2* X, int ldx, const double2* U, int ldu, int n, int N, double* out, cudaStream_t s,
                   long long* launches);

}  // namespace swi
