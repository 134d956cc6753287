// Shifted stencil Y = (A - sigma_col) X on complex128 vectors, in
// double-single arithmetic: the operator of Eq. 1 applied matrix-free and
// shifted as in Eq. 3, for the Krylov loop of the double-single solver.  Native
// FP64 caps the stencil at GB300's FP64 rate (two DFMA per SM clock, ~0.22
// TB/s of vectors); here every input value is split once into (hi, lo) floats
// from its bit fields when it is staged, and each of the 37 terms is an exact
// FMA product accumulated with TwoSum, on the FP32 pipes (~2^-48 relative per
// term).  Tiling as in the complex64 kernel: a 16 x 8 tile of (x, y) points x 4
// columns per CTA marching along z, the 12 z-neighbours of a point in a
// register queue, the x and y neighbours from the current plane staged with a
// cross-shaped halo in shared memory (ghosts by odd reflection or zero).
// Layout: X, Y are [N][ld] complex128, column index innermost.
#include <algorithm>

#include "ds.cuh"
#include "swi_internal.cuh"

namespace swi {

namespace {

constexpr int kTX = 16, kTY = 8, kNC = 4, kR = 6;
constexpr int kThreadsDs = kTX * kTY * kNC;
constexpr int kSX = kTX + 2 * kR, kSY = kTY + 2 * kR;
constexpr int kSlotsA = kTY * kSX * kNC, kSlotsB = 2 * kR * kTX * kNC;
constexpr int kSlots = kSlotsA + kSlotsB;
constexpr int kSlotsPerThread = (kSlots + kThreadsDs - 1) / kThreadsDs;

struct __align__(16) dsc {  // complex double-single
  float rh, rl, ih, il;
};

__device__ __forceinline__ dsc to_dsc(double2 v, float sgn) {
  dsc r;
  ds::split_bits(v.x, r.rh, r.rl);
  ds::split_bits(v.y, r.ih, r.il);
  r.rh *= sgn;
  r.rl *= sgn;
  r.ih *= sgn;
  r.il *= sgn;
  return r;
}

template <int BC>
__device__ __forceinline__ bool ghost_src(int j, int n, int& src, float& sgn) {
  if (j >= 0 && j < n) {
    src = j;
    sgn = 1.f;
    return true;
  }
  if (BC == SWI_BC_ZERO) return false;
  if (j <= -2) {
    src = -2 - j;
  } else if (j >= n + 1) {
    src = 2 * n - j;
  } else {
    return false;
  }
  if (src < 0 || src >= n) return false;
  sgn = -1.f;
  return true;
}

template <int BC>
__device__ __forceinline__ dsc load_z(const double2* __restrict__ X, long long pt_col, long long plane_ld, int z,
                                      int nz) {
  int src;
  float sgn;
  if (!ghost_src<BC>(z, nz, src, sgn)) return dsc{0.f, 0.f, 0.f, 0.f};
  return to_dsc(__ldg(X + pt_col + (long long)src * plane_ld), sgn);
}

// acc += c * (x), c a double-single real weight, x a double-single complex value
__device__ __forceinline__ void cfma(float (&acc)[4], float ch, float cl, const dsc& x) {
  ds::fma_acc(acc[0], acc[1], ch, cl, x.rh, x.rl);
  ds::fma_acc(acc[2], acc[3], ch, cl, x.ih, x.il);
}

template <int BC>
__global__ void __launch_bounds__(kThreadsDs, 1)
    stencil_ds_kernel(const __grid_constant__ StencilParams P, const __grid_constant__ StencilBatch batch,
                      const double* __restrict__ sigma, int zchunk) {
  __shared__ dsc s[kSY][kSX][kNC];
  const StencilBlock& B = batch.blk[blockIdx.z % batch.n];
  const int zc = blockIdx.z / batch.n;  // z chunk
  const int ncols = B.ncols, ldx = B.ldx;
  const double2* __restrict__ X = B.X;
  const int cc = threadIdx.x % kNC;
  const int tx = (threadIdx.x / kNC) % kTX;
  const int ty = threadIdx.x / (kNC * kTX);
  const int tiles_x = (P.nx + kTX - 1) / kTX;
  const int x0 = (blockIdx.x % tiles_x) * kTX, y0 = (blockIdx.x / tiles_x) * kTY;
  const int c0 = blockIdx.y * kNC;
  if (c0 >= ncols) return;
  const int x = x0 + tx, y = y0 + ty, c = c0 + cc;
  const bool mine = x < P.nx && y < P.ny && c < ncols;
  const int z0 = zc * zchunk, z1 = min(P.nz, z0 + zchunk);
  const long long plane = (long long)P.nx * P.ny;
  const long long plane_ld = plane * ldx;
  const long long pt_col = ((long long)y * P.nx + x) * ldx + c;
  float cmh[kR + 1], cml[kR + 1];
#pragma unroll
  for (int m = 0; m <= kR; ++m) ds::split_bits(P.cm[m], cmh[m], cml[m]);
  const double sig = mine ? sigma[B.sigma_off + c] : 0.0;
  const double cdiag = 3.0 * P.cm[0];

  int soff[kSlotsPerThread], sidx[kSlotsPerThread];
  float ssg[kSlotsPerThread];
#pragma unroll
  for (int k = 0; k < kSlotsPerThread; ++k) {
    const int e = threadIdx.x + k * kThreadsDs;
    int sc, sx, sy;
    if (e < kSlotsA) {
      sc = e % kNC;
      sx = (e / kNC) % kSX;
      sy = kR + e / (kNC * kSX);
    } else {
      const int f = e - kSlotsA;
      sc = f % kNC;
      sx = kR + (f / kNC) % kTX;
      const int r = f / (kNC * kTX);
      sy = r < kR ? r : r + kTY;
    }
    sidx[k] = -1;
    soff[k] = 0;
    ssg[k] = 0.f;
    if (e < kSlots) {
      sidx[k] = (sy * kSX + sx) * kNC + sc;
      int srcx, srcy;
      float sgx, sgy;
      const int gc = c0 + sc;
      if (gc < ncols && ghost_src<BC>(x0 + sx - kR, P.nx, srcx, sgx) && ghost_src<BC>(y0 + sy - kR, P.ny, srcy, sgy)) {
        soff[k] = (srcy * P.nx + srcx) * ldx + gc;
        ssg[k] = sgx * sgy;
      }
    }
  }
  dsc* sflat = &s[0][0][0];

  dsc q[2 * kR + 1];
#pragma unroll
  for (int k = 0; k < 2 * kR + 1; ++k)
    q[k] = mine ? load_z<BC>(X, pt_col, plane_ld, z0 - kR + k, P.nz) : dsc{0.f, 0.f, 0.f, 0.f};

  double2 pre[kSlotsPerThread];
#pragma unroll
  for (int k = 0; k < kSlotsPerThread; ++k)
    pre[k] = ssg[k] != 0.f ? __ldg(X + (long long)z0 * plane_ld + soff[k]) : make_double2(0.0, 0.0);
#pragma unroll
  for (int k = 0; k < kSlotsPerThread; ++k)
    if (sidx[k] >= 0) sflat[sidx[k]] = to_dsc(pre[k], ssg[k]);
  __syncthreads();

  for (int z = z0; z < z1; ++z) {
    const dsc nq = mine ? load_z<BC>(X, pt_col, plane_ld, z + kR + 1, P.nz) : dsc{0.f, 0.f, 0.f, 0.f};
    const bool more = z + 1 < z1;
#pragma unroll
    for (int k = 0; k < kSlotsPerThread; ++k)
      pre[k] = (more && ssg[k] != 0.f) ? __ldg(X + (long long)(z + 1) * plane_ld + soff[k]) : make_double2(0.0, 0.0);
    if (mine) {
      const long long row = (long long)z * plane + (long long)y * P.nx + x;
      float dh, dl, gh, gl;
      ds::split_bits(cdiag + __ldg(P.V + row) - sig, dh, dl);  // two FP64 adds per output
      ds::split_bits(__ldg(P.G + row), gh, gl);
      const dsc& x0v = q[kR];
      // (d - i g) x: re = d xr + g xi, im = d xi - g xr
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      ds::fma_acc(acc[0], acc[1], dh, dl, x0v.rh, x0v.rl);
      ds::fma_acc(acc[0], acc[1], gh, gl, x0v.ih, x0v.il);
      ds::fma_acc(acc[2], acc[3], dh, dl, x0v.ih, x0v.il);
      ds::fma_acc(acc[2], acc[3], -gh, -gl, x0v.rh, x0v.rl);
#pragma unroll
      for (int m = 1; m <= kR; ++m) {
        cfma(acc, cmh[m], cml[m], s[kR + ty][kR + tx - m][cc]);
        cfma(acc, cmh[m], cml[m], s[kR + ty][kR + tx + m][cc]);
        cfma(acc, cmh[m], cml[m], s[kR + ty - m][kR + tx][cc]);
        cfma(acc, cmh[m], cml[m], s[kR + ty + m][kR + tx][cc]);
        cfma(acc, cmh[m], cml[m], q[kR - m]);
        cfma(acc, cmh[m], cml[m], q[kR + m]);
      }
      if (B.out_ds) {
        const ds::df re = ds::two_sum(acc[0], acc[1]), im = ds::two_sum(acc[2], acc[3]);
        reinterpret_cast<float4*>(B.Y)[row * B.ldy + c] = make_float4(re.h, re.l, im.h, im.l);
      } else {
        B.Y[row * B.ldy + c] = make_double2((double)acc[0] + (double)acc[1], (double)acc[2] + (double)acc[3]);
      }
    }
#pragma unroll
    for (int k = 0; k < 2 * kR; ++k) q[k] = q[k + 1];
    q[2 * kR] = nq;
    __syncthreads();
    if (more) {
#pragma unroll
      for (int k = 0; k < kSlotsPerThread; ++k)
        if (sidx[k] >= 0) sflat[sidx[k]] = to_dsc(pre[k], ssg[k]);
    }
    __syncthreads();
  }
}

}  // namespace

void launch_stencil_ds(const StencilParams& P, const StencilBatch& batch, const double* sigma_dev, cudaStream_t s,
                       long long* launches) {
  if (batch.n <= 0) return;
  int maxc = 0;
  for (int q = 0; q < batch.n; ++q) maxc = batch.blk[q].ncols > maxc ? batch.blk[q].ncols : maxc;
  const int tiles = ((P.nx + kTX - 1) / kTX) * ((P.ny + kTY - 1) / kTY);
  const int cgroups = (maxc + kNC - 1) / kNC;
  // z chunks: a few CTAs per SM in total, each chunk at least 16 planes deep
  int nzc = (2 * 152 + tiles * cgroups * batch.n - 1) / (tiles * cgroups * batch.n);
  nzc = std::max(1, std::min(nzc, (P.nz + 15) / 16));
  const int zchunk = (P.nz + nzc - 1) / nzc;
  const int nz_chunks = (P.nz + zchunk - 1) / zchunk;
  dim3 grid(tiles, cgroups, batch.n * nz_chunks);
  if (P.bc == SWI_BC_ZERO)
    stencil_ds_kernel<SWI_BC_ZERO><<<grid, kThreadsDs, 0, s>>>(P, batch, sigma_dev, zchunk);
  else
    stencil_ds_kernel<SWI_BC_ODD><<<grid, kThreadsDs, 0, s>>>(P, batch, sigma_dev, zchunk);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
