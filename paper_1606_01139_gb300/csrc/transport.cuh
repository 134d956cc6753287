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
void launch_rowdot(const double2* X, int ldx, const double2* U, int ldu, int n, int N, double* out, cudaStream_t s,
                   long long* launches);

}  // namespace swi
