// T(E) and its adjoint with FP32 contractions (FP32 products, FP32
// accumulation): the reduced-precision form of the transport step of Section 1.
//
//   M_R = U^H Gamma_R U,  M_L = U^H Gamma_L U   (n x n Hermitian; R = M_R^T, L = M_L^T)
//   M   = sum_e w_e D_e R conj(D_e) L^T D_e      (D_e = diag(g_e), g_ek = 1/(E_e - eps_k))
//   dL/dV(r) = 2 Re sum_ac U_ra M_ac U_rc
//
// The three contractions are register-tiled products on the FP32 pipes: a
// 64 x 64 output tile per CTA, 256 threads of 4 x 4 outputs each, operands
// staged through shared memory 16 deep.  U stays in complex128 in HBM and is
// rounded to complex64 as it is staged.
//  - projections: only the upper output tiles are formed (the lower ones are
//    their conjugates), over the rows where Gamma is an FP32 normal number
//    (the other rows add exact zeros in FP32, or subnormal amounts below
//    2^-126 |U_ra||U_rc|), split over row chunks whose partial sums are added
//    in FP64.  Each thread sums 256-row blocks in FP32 and adds the block sums
//    into a second FP32 accumulator, so the accumulation error grows with
//    256 + (rows per chunk)/256 instead of the chunk length.
//  - adjoint M: per energy, the tile of R conj(D_e) L^T over l, then scaled by
//    w_e g_ea g_ec into the tile of M (the energy table g_e in FP32).
//  - dL/dV: per 64-row block of U, (U M) tile by tile, each tile contracted
//    with the same rows of U at once, so U M is never stored.
#include <algorithm>
#include <cfloat>

#include "swi_internal.cuh"
#include "transport.cuh"

namespace swi {

namespace {

constexpr int kT = 64;    // output tile edge
constexpr int kK = 16;    // contraction depth of one shared-memory stage
constexpr int kThr = 256; // 16 x 16 threads, 4 x 4 outputs each (rows ty + 16 i, columns tx + 16 j)
constexpr int kInner = 16;  // stages (of kK rows) summed before the block sum is added (projections)

__device__ __forceinline__ float2 f2(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 f2zero() { return make_float2(0.f, 0.f); }
// acc += a b
__device__ __forceinline__ void fcfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) b
__device__ __forceinline__ void fcfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
__device__ __forceinline__ float2 fcmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// part[s][a][c] = sum over the rows of chunk s of gamma_r conj(U_ra) U_rc, for
// the upper tile pairs (ta <= tc): blockIdx.x enumerates them row by row of
// tiles, blockIdx.y the chunks of rch rows of [lo, hi).
__global__ void __launch_bounds__(kThr) proj_f32_kernel(const double2* __restrict__ U, int ldu, int n,
                                                        const double* __restrict__ gam, long long lo, long long hi,
                                                        long long rch, int ntile, float2* __restrict__ part) {
  __shared__ float2 sa[kK][kT];  // sa[k][col] = gamma_r U[r][a0 + col], r = row k of the stage
  __shared__ float2 sc[kK][kT];  // sc[k][col] = U[r][c0 + col]
  int t = blockIdx.x, ta = 0;
  while (t >= ntile - ta) {
    t -= ntile - ta;
    ++ta;
  }
  const int tc = ta + t;
  const int a0 = ta * kT, c0 = tc * kT;
  const long long rb = lo + (long long)blockIdx.y * rch;
  const long long re = min(hi, rb + rch);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 acc[4][4], tot[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = tot[i][j] = f2zero();
  int stage = 0;
  for (long long r0 = rb; r0 < re; r0 += kK) {
    for (int q = threadIdx.x; q < kK * kT; q += kThr) {
      const int k = q / kT, col = q % kT;  // column fastest: coalesced rows of U
      const long long r = r0 + k;
      float2 va = f2zero(), vc = f2zero();
      if (r < re) {
        const double2* Ur = U + r * (long long)ldu;
        if (a0 + col < n) {
          const float g = (float)gam[r];
          const float2 u = f2(Ur[a0 + col]);
          va = make_float2(g * u.x, g * u.y);
        }
        if (c0 + col < n) vc = f2(Ur[c0 + col]);
      }
      sa[k][col] = va;
      sc[k][col] = vc;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      float2 xa[4], xc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xa[i] = sa[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) xc[j] = sc[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) fcfmac(acc[i][j], xa[i], xc[j]);
    }
    __syncthreads();
    if (++stage == kInner) {
      stage = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          tot[i][j].x += acc[i][j].x;
          tot[i][j].y += acc[i][j].y;
          acc[i][j] = f2zero();
        }
    }
  }
  float2* P = part + (size_t)blockIdx.y * n * n;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty + 16 * i;
    if (a >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < n) P[(size_t)a * n + c] = make_float2(tot[i][j].x + acc[i][j].x, tot[i][j].y + acc[i][j].y);
    }
  }
}

// M[a][c] from the chunk partials: the upper tiles directly, a lower tile as the
// conjugate of its mirror (FP64 sum over the chunks)
__device__ __forceinline__ double2 sum_parts(const float2* __restrict__ part, int ks, int n, int a, int c) {
  const bool up = (a / kT) <= (c / kT);
  const int i = up ? a : c, j = up ? c : a;
  double sx = 0.0, sy = 0.0;
  for (int s = 0; s < ks; ++s) {
    const float2 v = part[(size_t)s * n * n + (size_t)i * n + j];
    sx += v.x;
    sy += v.y;
  }
  return make_double2(sx, up ? sy : -sy);
}

// R[k][l] = M_R[l][k], L[k][l] = M_L[l][k], W = R o L; complex128 and complex64 copies
__global__ void proj_reduce_f32_kernel(const float2* __restrict__ partR, int kR, const float2* __restrict__ partL,
                                       int kL, int n, double2* __restrict__ R, double2* __restrict__ L,
                                       double2* __restrict__ W, float2* __restrict__ R32, float2* __restrict__ L32) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int k = (int)(t / n), l = (int)(t % n);
  const double2 r = sum_parts(partR, kR, n, l, k);
  const double2 q = sum_parts(partL, kL, n, l, k);
  R[t] = r;
  L[t] = q;
  W[t] = cmul(r, q);
  R32[t] = f2(r);
  L32[t] = f2(q);
}

// gt[e][l] = 1/(E_e - eps_l), formed in FP64 and rounded to complex64
__global__ void gtab_kernel(const double2* __restrict__ eps, int n, const double* __restrict__ E, int nE,
                            float2* __restrict__ gt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nE * n) return;
  const int e = (int)(t / n), l = (int)(t % n);
  gt[t] = f2(cdiv(make_double2(1.0, 0.0), csub(make_double2(E[e], 0.0), eps[l])));
}

// M[a][c] = sum_e w_e g_ea g_ec sum_l R[a][l] conj(g_el) L[c][l]
__global__ void __launch_bounds__(kThr) gradM_f32_kernel(const float2* __restrict__ R, const float2* __restrict__ L,
                                                         const float2* __restrict__ gt, const double* __restrict__ wts,
                                                         int n, int nE, float2* __restrict__ M) {
  __shared__ float2 sr[kK][kT + 1];  // sr[l][row] = R[a0 + row][l0 + l]
  __shared__ float2 sl[kK][kT + 1];  // sl[l][row] = conj(g_e,l0+l) L[c0 + row][l0 + l]
  const int a0 = blockIdx.y * kT, c0 = blockIdx.x * kT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float2 macc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) macc[i][j] = f2zero();
  for (int e = 0; e < nE; ++e) {
    const float we = (float)wts[e];
    if (we == 0.f) continue;  // the same for every thread of the block
    const float2* g = gt + (size_t)e * n;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = f2zero();
    for (int l0 = 0; l0 < n; l0 += kK) {
      for (int q = threadIdx.x; q < kK * kT; q += kThr) {
        const int ll = q % kK, row = q / kK;  // 16 consecutive l of one row
        const int l = l0 + ll, a = a0 + row, c = c0 + row;
        sr[ll][row] = (a < n && l < n) ? R[(size_t)a * n + l] : f2zero();
        float2 v = f2zero();
        if (c < n && l < n) {
          const float2 gl = g[l];
          v = fcmul(make_float2(gl.x, -gl.y), L[(size_t)c * n + l]);
        }
        sl[ll][row] = v;
      }
      __syncthreads();
#pragma unroll
      for (int ll = 0; ll < kK; ++ll) {
        float2 xr[4], xl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xr[i] = sr[ll][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) xl[j] = sl[ll][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) fcfma(acc[i][j], xr[i], xl[j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int a = a0 + ty + 16 * i;
      if (a >= n) continue;
      const float2 ga = g[a];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + tx + 16 * j;
        if (c >= n) continue;
        const float2 f = fcmul(ga, g[c]);
        fcfma(macc[i][j], make_float2(we * f.x, we * f.y), acc[i][j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty + 16 * i;
    if (a >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < n) M[(size_t)a * n + c] = macc[i][j];
    }
  }
}

// out[r] = 2 Re sum_{a,c} U_ra M_ac U_rc for the 64 rows r0 .. r0 + 63 of a block
__global__ void __launch_bounds__(kThr) rowquad_f32_kernel(const double2* __restrict__ U, int ldu,
                                                           const float2* __restrict__ M, int n, long long N,
                                                           double* __restrict__ out) {
  __shared__ float2 su[kK][kT + 1];  // su[a][row] = U[r0 + row][a0 + a]
  __shared__ float2 sm[kK][kT];      // sm[a][col] = M[a0 + a][c0 + col]
  const long long r0 = (long long)blockIdx.x * kT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float prow[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c0 = 0; c0 < n; c0 += kT) {
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = f2zero();
    for (int a0 = 0; a0 < n; a0 += kK) {
      for (int q = threadIdx.x; q < kK * kT; q += kThr) {
        {
          const int aa = q % kK, row = q / kK;  // 16 consecutive columns of one row of U
          const long long r = r0 + row;
          const int a = a0 + aa;
          su[aa][row] = (r < N && a < n) ? f2(U[r * ldu + a]) : f2zero();
        }
        {
          const int col = q % kT, ab = q / kT;  // 64 consecutive columns of one row of M
          const int a = a0 + ab, c = c0 + col;
          sm[ab][col] = (a < n && c < n) ? M[(size_t)a * n + c] : f2zero();
        }
      }
      __syncthreads();
#pragma unroll
      for (int aa = 0; aa < kK; ++aa) {
        float2 xu[4], xm[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xu[i] = su[aa][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) xm[j] = sm[aa][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) fcfma(acc[i][j], xu[i], xm[j]);
      }
      __syncthreads();
    }
    // contract the tile of U M with U[r][c0 + col] at once
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long r = r0 + ty + 16 * i;
      if (r >= N) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + tx + 16 * j;
        if (c >= n) continue;
        const float2 u = f2(U[r * ldu + c]);
        prow[i] = fmaf(acc[i][j].x, u.x, fmaf(-acc[i][j].y, u.y, prow[i]));
      }
    }
  }
  // sum over the 16 column lanes (tx) of each half-warp
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) prow[i] += __shfl_xor_sync(0xffffffffu, prow[i], o);
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long r = r0 + ty + 16 * i;
      if (r < N) out[r] = 2.0 * (double)prow[i];
    }
  }
}

struct ProjSplit {
  long long rch;  // rows per chunk (a multiple of kK)
  int chunks;
};

ProjSplit proj_split(int n, long long rows) {
  if (rows <= 0 || n <= 0) return ProjSplit{0, 0};
  const int nt = (n + kT - 1) / kT;
  const long long pairs = (long long)nt * (nt + 1) / 2;
  long long k = (2 * 152 + pairs - 1) / pairs;  // about two CTAs per SM over the tile pairs
  k = std::min<long long>(k, (rows + 255) / 256);  // chunks of at least ~256 rows
  k = std::min<long long>(k, 64);
  k = std::max<long long>(k, 1);
  long long rch = (rows + k - 1) / k;
  rch = (rch + kK - 1) / kK * kK;
  return ProjSplit{rch, (int)((rows + rch - 1) / rch)};
}

}  // namespace

int proj_f32_chunks(int n, long long rows) { return proj_split(n, rows).chunks; }

void launch_proj_f32(const double2* U, int ldu, int n, const double* gR, long long loR, long long hiR,
                     const double* gL, long long loL, long long hiL, float2* part, double2* R, double2* L,
                     double2* W, float2* R32, float2* L32, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  const int nt = (n + kT - 1) / kT;
  const long long pairs = (long long)nt * (nt + 1) / 2;
  const ProjSplit sR = proj_split(n, hiR - loR), sL = proj_split(n, hiL - loL);
  float2* pR = part;
  float2* pL = part + (size_t)sR.chunks * n * n;
  if (sR.chunks > 0) {
    proj_f32_kernel<<<dim3((unsigned)pairs, (unsigned)sR.chunks), kThr, 0, s>>>(U, ldu, n, gR, loR, hiR, sR.rch, nt,
                                                                                pR);
    SWI_CHECK_LAUNCH();
    if (launches) ++*launches;
  }
  if (sL.chunks > 0) {
    proj_f32_kernel<<<dim3((unsigned)pairs, (unsigned)sL.chunks), kThr, 0, s>>>(U, ldu, n, gL, loL, hiL, sL.rch, nt,
                                                                                pL);
    SWI_CHECK_LAUNCH();
    if (launches) ++*launches;
  }
  const long long nn = (long long)n * n;
  proj_reduce_f32_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(pR, sR.chunks, pL, sL.chunks, n, R, L, W, R32,
                                                                        L32);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_grad_f32(const float2* R32, const float2* L32, const double2* eps, int n, const double* E,
                     const double* w, int nE, float2* gt, float2* M, const double2* U, int ldu, long long N,
                     double* out, cudaStream_t s, long long* launches) {
  if (n <= 0 || N <= 0) return;
  const long long ne = (long long)nE * n;
  if (ne > 0) {
    gtab_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(eps, n, E, nE, gt);
    SWI_CHECK_LAUNCH();
    if (launches) ++*launches;
  }
  const unsigned nt = (unsigned)((n + kT - 1) / kT);
  gradM_f32_kernel<<<dim3(nt, nt), kThr, 0, s>>>(R32, L32, gt, w, n, nE, M);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
  rowquad_f32_kernel<<<(unsigned)((N + kT - 1) / kT), kThr, 0, s>>>(U, ldu, M, n, N, out);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
