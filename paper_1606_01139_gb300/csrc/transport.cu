// Transmission T(E) = Tr{G Gamma_R G^dagger Gamma_L} through the spectral Green's
// function G(E) = sum_k U_k U_k^T / (E - eps_k) (Section 1), and its adjoint.
//
//   R = U^T Gamma_R conj(U),  L = U^T Gamma_L conj(U)   (Hermitian, n x n)
//   W = R o L,  g_ek = 1/(E_e - eps_k),  T_e = sum_kl g_ek W_kl conj(g_el)
//   dT_e/dE_e = -2 Re sum_kl g_ek^2 W_kl conj(g_el)
//   dL/dV(r) = 2 Re sum_ac U_ra M_ac U_rc,  M = sum_e w_e D_e R conj(D_e) L^T D_e
// (dG = G dV G for a real diagonal dV; D_e = diag(g_e)).
//
// R and L come from the tall-skinny Gram kernel (M_R = U^H Gamma_R U, R = M_R^T);
// M is an n x n x n contraction per energy; U M is a row GEMM followed by a
// row-wise bilinear dot.
#include "swi_internal.cuh"
#include "transport.cuh"

namespace swi {

namespace {

// W[k][l] = R_kl L_kl with R = MR^T, L = ML^T  ->  W[k][l] = MR[l][k] * ML[l][k]
__global__ void wbuild_kernel(const double2* __restrict__ MR, const double2* __restrict__ ML, int n,
                              double2* __restrict__ R, double2* __restrict__ L, double2* __restrict__ W) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int k = (int)(t / n), l = (int)(t % n);
  const double2 r = MR[(long long)l * n + k];
  const double2 q = ML[(long long)l * n + k];
  R[t] = r;
  L[t] = q;
  W[t] = cmul(r, q);
}

// one CTA per energy: T_e and dT_e/dE_e
__global__ void transmission_kernel(const double2* __restrict__ W, const double2* __restrict__ eps, int n,
                                    const double* __restrict__ E, double* __restrict__ T,
                                    double* __restrict__ dTdE) {
  extern __shared__ double2 sg[];  // g[n]
  __shared__ double red[2][32];
  const int e = blockIdx.x;
  const double En = E[e];
  for (int k = threadIdx.x; k < n; k += blockDim.x) sg[k] = cdiv(make_double2(1.0, 0.0), csub(make_double2(En, 0.0), eps[k]));
  __syncthreads();
  double tsum = 0.0, dsum = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double2 x = make_double2(0.0, 0.0);
    const double2* Wk = W + (long long)k * n;
    for (int l = 0; l < n; ++l) {
      const double2 g = sg[l];
      // x += W_kl conj(g_l)
      const double2 w = Wk[l];
      x.x = fma(w.x, g.x, fma(w.y, g.y, x.x));
      x.y = fma(w.y, g.x, fma(-w.x, g.y, x.y));
    }
    const double2 gk = sg[k];
    const double2 t1 = cmul(gk, x);
    tsum += t1.x;
    dsum += cmul(gk, t1).x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  }
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) {
    red[0][w] = tsum;
    red[1][w] = dsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      a += red[0][q];
      b += red[1][q];
    }
    T[e] = a;
    if (dTdE) dTdE[e] = -2.0 * b;
  }
}

// M[a][c] = sum_e w_e g_ea g_ec sum_l R[a][l] conj(g_el) L[c][l]
constexpr int kMT = 32, kLC = 16;
__global__ void __launch_bounds__(256) gradM_kernel(const double2* __restrict__ R, const double2* __restrict__ L,
                                                    const double2* __restrict__ eps, int n,
                                                    const double* __restrict__ E, const double* __restrict__ wts,
                                                    int nE, double2* __restrict__ M) {
  __shared__ double2 sr[kMT][kLC + 1];
  __shared__ double2 sl[kMT][kLC + 1];
  const int a0 = blockIdx.y * kMT, c0 = blockIdx.x * kMT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 macc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) macc[i][j] = make_double2(0.0, 0.0);
  for (int e = 0; e < nE; ++e) {
    const double En = E[e];
    const double we = wts[e];
    if (we == 0.0) continue;
    double2 acc[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
    for (int l0 = 0; l0 < n; l0 += kLC) {
      for (int q = threadIdx.x; q < kMT * kLC; q += 256) {
        const int rr = q / kLC, ll = q % kLC;
        const int a = a0 + rr, c = c0 + rr, l = l0 + ll;
        sr[rr][ll] = (a < n && l < n) ? R[(long long)a * n + l] : make_double2(0.0, 0.0);
        double2 v = make_double2(0.0, 0.0);
        if (c < n && l < n) {
          const double2 g = cdiv(make_double2(1.0, 0.0), csub(make_double2(En, 0.0), eps[l]));
          v = cmul(L[(long long)c * n + l], cconj(g));
        }
        sl[rr][ll] = v;
      }
      __syncthreads();
#pragma unroll
      for (int ll = 0; ll < kLC; ++ll) {
        const double2 r0 = sr[ty * 2][ll], r1 = sr[ty * 2 + 1][ll];
        const double2 q0 = sl[tx * 2][ll], q1 = sl[tx * 2 + 1][ll];
        cfma(acc[0][0], r0, q0);
        cfma(acc[0][1], r0, q1);
        cfma(acc[1][0], r1, q0);
        cfma(acc[1][1], r1, q1);
      }
      __syncthreads();
    }
    for (int i = 0; i < 2; ++i) {
      const int a = a0 + ty * 2 + i;
      if (a >= n) continue;
      const double2 ga = cdiv(make_double2(1.0, 0.0), csub(make_double2(En, 0.0), eps[a]));
      for (int j = 0; j < 2; ++j) {
        const int c = c0 + tx * 2 + j;
        if (c >= n) continue;
        const double2 gc = cdiv(make_double2(1.0, 0.0), csub(make_double2(En, 0.0), eps[c]));
        const double2 f = cscale(cmul(ga, gc), we);
        cfma(macc[i][j], f, acc[i][j]);
      }
    }
  }
  for (int i = 0; i < 2; ++i) {
    const int a = a0 + ty * 2 + i;
    if (a >= n) continue;
    for (int j = 0; j < 2; ++j) {
      const int c = c0 + tx * 2 + j;
      if (c < n) M[(long long)a * n + c] = macc[i][j];
    }
  }
}

// out[r] = 2 Re sum_c X[r][c] U[r][c]   (one warp per row)
__global__ void rowdot_kernel(const double2* __restrict__ X, int ldx, const double2* __restrict__ U, int ldu, int n,
                              int N, double* __restrict__ out) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= N) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) {
    const double2 x = X[warp * ldx + c], u = U[warp * ldu + c];
    s = fma(x.x, u.x, fma(-x.y, u.y, s));
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[warp] = 2.0 * s;
}

}  // namespace

void launch_wbuild(const double2* MR, const double2* ML, int n, double2* R, double2* L, double2* W, cudaStream_t s,
                   long long* launches) {
  const long long nn = (long long)n * n;
  if (nn == 0) return;
  wbuild_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(MR, ML, n, R, L, W);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_transmission(const double2* W, const double2* eps, int n, const double* E, int nE, double* T,
                         double* dTdE, cudaStream_t s, long long* launches) {
  if (nE <= 0) return;
  const size_t smem = sizeof(double2) * (size_t)(n > 0 ? n : 1);
  if (smem > 48 * 1024) SWI_CUDA_TRY(cudaFuncSetAttribute(transmission_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  transmission_kernel<<<nE, 256, smem, s>>>(W, eps, n, E, T, dTdE);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_gradM(const double2* R, const double2* L, const double2* eps, int n, const double* E, const double* w,
                  int nE, double2* M, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  dim3 grid((n + kMT - 1) / kMT, (n + kMT - 1) / kMT);
  gradM_kernel<<<grid, 256, 0, s>>>(R, L, eps, n, E, w, nE, M);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_rowdot(const double2* X, int ldx, const double2* U, int ldu, int n, int N, double* out, cudaStream_t s,
                   long long* launches) {
  const long long threads = (long long)N * 32;
  rowdot_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(X, ldx, U, ldu, n, N, out);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
