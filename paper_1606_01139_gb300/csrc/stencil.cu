// Shifted stencil Y = (A - sigma_col) X for blocks of complex128 vectors.
//
// A = -1/2 nabla^2_FD + V - i Gamma (Eq. 1) applied matrix-free, as H_KS is in
// the paper (a matrix-vector product formula, never stored, Section 1); the
// per-column real shift sigma gives the shifted operator of Eq. (3).  The
// kinetic term is the radius-6 (12th-order) central second difference on each
// axis.  Ghost values: odd reflection (u[-1] = u[n] = 0, u[-1-k] = -u[-1+k],
// u[n+k] = -u[n-k]) or zero padding.
//
// Layout: X, Y are [N][ld] with the column (vector) index innermost, so the
// b columns of one grid point are contiguous and a warp reads whole points.
// FP64 on GB300 is ALU-bound (two DFMA per SM clock), so the kernel minimises
// FP64 operations (paired neighbours share one multiply) rather than traffic;
// neighbours come through L1/L2.
#include "swi_internal.cuh"

namespace swi {

namespace {

template <int BC>
__device__ __forceinline__ double2 fetch_axis(const double2* __restrict__ X, long long row0, long long stride,
                                              int i, int jj, int n, int ld, int c) {
  // value at axis index jj (row row0 is axis index i)
  if (jj >= 0 && jj < n) {
    const double2 v = __ldg(X + (row0 + (long long)(jj - i) * stride) * ld + c);
    return v;
  }
  if (BC == SWI_BC_ZERO) return make_double2(0.0, 0.0);
  int src;
  if (jj <= -2) {
    src = -2 - jj;
  } else if (jj >= n + 1) {
    src = 2 * n - jj;
  } else {
    return make_double2(0.0, 0.0);
  }
  const double2 v = __ldg(X + (row0 + (long long)(src - i) * stride) * ld + c);
  return make_double2(-v.x, -v.y);
}

template <int BC>
__device__ __forceinline__ void axis_sum(double2& acc, const double2* __restrict__ X, long long row, long long stride,
                                         int i, int n, int ld, int c, const double* cm) {
  if (i >= 6 && i + 6 < n) {
#pragma unroll
    for (int m = 1; m <= 6; ++m) {
      const double2 a = __ldg(X + (row - m * stride) * ld + c);
      const double2 b = __ldg(X + (row + m * stride) * ld + c);
      acc.x = fma(cm[m], a.x + b.x, acc.x);
      acc.y = fma(cm[m], a.y + b.y, acc.y);
    }
  } else {
#pragma unroll
    for (int m = 1; m <= 6; ++m) {
      const double2 a = fetch_axis<BC>(X, row, stride, i, i - m, n, ld, c);
      const double2 b = fetch_axis<BC>(X, row, stride, i, i + m, n, ld, c);
      acc.x = fma(cm[m], a.x + b.x, acc.x);
      acc.y = fma(cm[m], a.y + b.y, acc.y);
    }
  }
}

template <int BC>
__global__ void __launch_bounds__(256) stencil_f64_kernel(const __grid_constant__ StencilParams P,
                                                          const __grid_constant__ StencilBatch batch,
                                                          const double* __restrict__ sigma, int zchunk) {
  const StencilBlock& B = batch.blk[blockIdx.z];
  const int nc = B.ncols;
  const int plane = P.nx * P.ny;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)plane * nc) return;
  const int c = (int)(t % nc);
  const int pt = (int)(t / nc);
  const int i = pt % P.nx;
  const int j = pt / P.nx;
  const int z0 = blockIdx.y * zchunk;
  const int z1 = min(P.nz, z0 + zchunk);
  const double sig = sigma[B.sigma_off + c];
  const double cdiag = 3.0 * P.cm[0];
  double cm[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) cm[m] = P.cm[m];
  for (int k = z0; k < z1; ++k) {
    const long long row = (long long)k * plane + pt;
    const double2 x0 = __ldg(B.X + row * B.ldx + c);
    const double d = cdiag + __ldg(P.V + row) - sig;
    const double g = __ldg(P.G + row);
    double2 acc;
    // (V - sigma + 3 c0) x - i Gamma x
    acc.x = fma(d, x0.x, g * x0.y);
    acc.y = fma(d, x0.y, -g * x0.x);
    axis_sum<BC>(acc, B.X, row, 1, i, P.nx, B.ldx, c, cm);
    axis_sum<BC>(acc, B.X, row, P.nx, j, P.ny, B.ldx, c, cm);
    axis_sum<BC>(acc, B.X, row, plane, k, P.nz, B.ldx, c, cm);
    B.Y[row * B.ldy + c] = acc;
  }
}

}  // namespace

void launch_stencil(const StencilParams& P, const StencilBatch& batch, const double* sigma_dev, cudaStream_t s,
                    long long* launches) {
  if (batch.n <= 0) return;
  int maxc = 0;
  for (int q = 0; q < batch.n; ++q) maxc = batch.blk[q].ncols > maxc ? batch.blk[q].ncols : maxc;
  const long long work = (long long)P.nx * P.ny * maxc;
  const int threads = 256;
  const int gx = (int)((work + threads - 1) / threads);
  // z chunk: enough CTAs to fill the GPU a few times over
  int zchunk = 8;
  while (zchunk > 1 && (long long)gx * ((P.nz + zchunk - 1) / zchunk) * batch.n < 4 * 152) zchunk /= 2;
  dim3 grid(gx, (P.nz + zchunk - 1) / zchunk, batch.n);
  if (P.bc == SWI_BC_ZERO)
    stencil_f64_kernel<SWI_BC_ZERO><<<grid, threads, 0, s>>>(P, batch, sigma_dev, zchunk);
  else
    stencil_f64_kernel<SWI_BC_ODD><<<grid, threads, 0, s>>>(P, batch, sigma_dev, zchunk);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
