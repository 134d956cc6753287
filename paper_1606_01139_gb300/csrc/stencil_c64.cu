// Shifted stencil Y = (A - sigma_col) X on complex64 vectors with FP32
// arithmetic (Eq. 1 applied matrix-free, shifted as in Eq. 3): the form for
// blocks whose rows are not 16-byte aligned (an odd column count); the
// TMA-staged kernel of stencil_c64_tma.cu serves the rest.  Each CTA owns a
// 16 x 8 tile of (x, y) points and 4 columns and marches along z.  The 12
// z-neighbours of a point live in a register queue (one new plane per step,
// prefetched a step ahead); the x and y neighbours come from the current plane,
// staged into shared memory with a 6-point cross-shaped halo (ghosts by odd
// reflection or zero, as in the FP64 kernel), the next plane's staging loads
// issued before this plane's arithmetic.  Layout: X, Y are [N][ld] complex64
// (float2), column index innermost.
#include <algorithm>

#include "swi_internal.cuh"

namespace swi {

namespace {

constexpr int kTX = 16, kTY = 8, kNC = 4, kR = 6;
constexpr int kThreadsC64 = kTX * kTY * kNC;
constexpr int kSX = kTX + 2 * kR, kSY = kTY + 2 * kR;

// value of column c at axis index j of a line whose in-range extent is n
// (odd reflection about the planes -1 and n, or zero)
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
  if (src < 0 || src >= n) return false;  // reflection beyond the far side: a zero ghost
  sgn = -1.f;
  return true;
}

template <int BC>
__device__ __forceinline__ float2 load_z(const float2* __restrict__ X, long long pt_col, long long plane_ld, int z,
                                         int nz) {
  int src;
  float sgn;
  if (!ghost_src<BC>(z, nz, src, sgn)) return make_float2(0.f, 0.f);
  const float2 v = __ldg(X + pt_col + (long long)src * plane_ld);
  return make_float2(sgn * v.x, sgn * v.y);
}

// Staging slots of the cross-shaped halo: the kTY tile rows over the full
// staged width, then the 2 kR halo rows over the tile's width; kNC columns each.
constexpr int kSlotsA = kTY * kSX * kNC, kSlotsB = 2 * kR * kTX * kNC;
constexpr int kSlots = kSlotsA + kSlotsB;
constexpr int kSlotsPerThread = (kSlots + kThreadsC64 - 1) / kThreadsC64;

template <int BC>
__global__ void __launch_bounds__(kThreadsC64, 1)
    stencil_c64_kernel(const __grid_constant__ StencilC64Params P, const float2* __restrict__ X, int ldx,
                       float2* __restrict__ Y, int ldy, int ncols, const float* __restrict__ sigma, int zchunk) {
  __shared__ float2 s[kSY][kSX][kNC];
  const int cc = threadIdx.x % kNC;
  const int tx = (threadIdx.x / kNC) % kTX;
  const int ty = threadIdx.x / (kNC * kTX);
  const int tiles_x = (P.nx + kTX - 1) / kTX;
  const int x0 = (blockIdx.x % tiles_x) * kTX, y0 = (blockIdx.x / tiles_x) * kTY;
  const int c0 = blockIdx.y * kNC;
  const int x = x0 + tx, y = y0 + ty, c = c0 + cc;
  const bool mine = x < P.nx && y < P.ny && c < ncols;
  const int z0 = blockIdx.z * zchunk, z1 = min(P.nz, z0 + zchunk);
  const long long plane = (long long)P.nx * P.ny;
  const long long plane_ld = plane * ldx;
  const long long pt_col = ((long long)y * P.nx + x) * ldx + c;
  float cm[kR + 1];
#pragma unroll
  for (int m = 0; m <= kR; ++m) cm[m] = P.cm[m];
  const float sig = mine ? sigma[c] : 0.f;

  // this thread's staging slots: smem index, source offset within a plane and
  // sign (0: a zero ghost or an unused slot)
  int soff[kSlotsPerThread], sidx[kSlotsPerThread];
  float ssg[kSlotsPerThread];
#pragma unroll
  for (int k = 0; k < kSlotsPerThread; ++k) {
    const int e = threadIdx.x + k * kThreadsC64;
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
  float2* sflat = &s[0][0][0];

  // z queue: q[k] = X at z - 6 + k, k = 0..12
  float2 q[2 * kR + 1];
#pragma unroll
  for (int k = 0; k < 2 * kR + 1; ++k)
    q[k] = mine ? load_z<BC>(X, pt_col, plane_ld, z0 - kR + k, P.nz) : make_float2(0.f, 0.f);
  const long long prow = (long long)y * P.nx + x;  // point index within a plane

  // stage plane z0
  float2 preA[kSlotsPerThread], preB[kSlotsPerThread];
#pragma unroll
  for (int k = 0; k < kSlotsPerThread; ++k)
    preA[k] = ssg[k] != 0.f ? __ldg(X + (long long)z0 * plane_ld + soff[k]) : make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < kSlotsPerThread; ++k)
    if (sidx[k] >= 0) sflat[sidx[k]] = make_float2(ssg[k] * preA[k].x, ssg[k] * preA[k].y);
  // loads two steps ahead, alternating between the A and B register sets:
  // staging values of plane z+1 / z+2, queue entries for planes z+7 / z+8,
  // V and Gamma of planes z / z+1
#pragma unroll
  for (int k = 0; k < kSlotsPerThread; ++k)
    preA[k] = (z0 + 1 < z1 && ssg[k] != 0.f) ? __ldg(X + (long long)(z0 + 1) * plane_ld + soff[k])
                                             : make_float2(0.f, 0.f);
  float2 nqA = mine ? load_z<BC>(X, pt_col, plane_ld, z0 + kR + 1, P.nz) : make_float2(0.f, 0.f), nqB;
  float vA = mine ? __ldg(P.V + (long long)z0 * plane + prow) : 0.f, gA = mine ? __ldg(P.G + (long long)z0 * plane + prow) : 0.f;
  float vB = 0.f, gB = 0.f;
  __syncthreads();

  auto step = [&](const int z, float2 (&pcur)[kSlotsPerThread], float2 (&pnxt)[kSlotsPerThread], float2& qcur,
                  float2& qnxt, float& vcur, float& gcur, float& vnxt, float& gnxt) {
    const bool more2 = z + 2 < z1;
#pragma unroll
    for (int k = 0; k < kSlotsPerThread; ++k)
      pnxt[k] = (more2 && ssg[k] != 0.f) ? __ldg(X + (long long)(z + 2) * plane_ld + soff[k]) : make_float2(0.f, 0.f);
    qnxt = mine ? load_z<BC>(X, pt_col, plane_ld, z + kR + 2, P.nz) : make_float2(0.f, 0.f);
    if (mine && z + 1 < z1) {
      vnxt = __ldg(P.V + (long long)(z + 1) * plane + prow);
      gnxt = __ldg(P.G + (long long)(z + 1) * plane + prow);
    }
    if (mine) {
      const float d = 3.f * cm[0] + vcur - sig;
      const float g = gcur;
      const float2 x0v = q[kR];
      float ar = fmaf(d, x0v.x, g * x0v.y);
      float ai = fmaf(d, x0v.y, -g * x0v.x);
#pragma unroll
      for (int m = 1; m <= kR; ++m) {
        const float2 a = s[kR + ty][kR + tx - m][cc], b = s[kR + ty][kR + tx + m][cc];
        const float2 u = s[kR + ty - m][kR + tx][cc], w = s[kR + ty + m][kR + tx][cc];
        const float2 lo = q[kR - m], hi = q[kR + m];
        ar = fmaf(cm[m], (a.x + b.x) + (u.x + w.x) + (lo.x + hi.x), ar);
        ai = fmaf(cm[m], (a.y + b.y) + (u.y + w.y) + (lo.y + hi.y), ai);
      }
      Y[((long long)z * plane + prow) * ldy + c] = make_float2(ar, ai);
    }
#pragma unroll
    for (int k = 0; k < 2 * kR; ++k) q[k] = q[k + 1];
    q[2 * kR] = qcur;
    __syncthreads();  // every read of plane z is done
    if (z + 1 < z1) {
#pragma unroll
      for (int k = 0; k < kSlotsPerThread; ++k)
        if (sidx[k] >= 0) sflat[sidx[k]] = make_float2(ssg[k] * pcur[k].x, ssg[k] * pcur[k].y);
    }
    __syncthreads();
  };
  int z = z0;
  for (; z + 1 < z1; z += 2) {
    step(z, preA, preB, nqA, nqB, vA, gA, vB, gB);
    step(z + 1, preB, preA, nqB, nqA, vB, gB, vA, gA);
  }
  if (z < z1) step(z, preA, preB, nqA, nqB, vA, gA, vB, gB);
}

}  // namespace

void launch_stencil_c64(const StencilC64Params& P, const float2* X, int ldx, float2* Y, int ldy, int ncols,
                        const float* sigma_dev, cudaStream_t s, long long* launches) {
  if (ncols <= 0) return;
  if (P.VG != nullptr && stencil_c64_tma_ok(X, ldx)) {  // TMA-staged form (stencil_c64_tma.cu) for 16-byte aligned rows
    launch_stencil_c64_tma(P, X, ldx, Y, ldy, ncols, sigma_dev, s, launches);
    return;
  }
  const int tiles = ((P.nx + kTX - 1) / kTX) * ((P.ny + kTY - 1) / kTY);
  const int cgroups = (ncols + kNC - 1) / kNC;
  // z chunks: a CTA per SM or more, each chunk at least 16 planes deep so the
  // 12-plane queue prologue stays a small fraction of the reads
  int nzc = (152 + tiles * cgroups - 1) / (tiles * cgroups);
  nzc = std::max(1, std::min(nzc, (P.nz + 15) / 16));
  const int zchunk = (P.nz + nzc - 1) / nzc;
  dim3 grid(tiles, cgroups, (P.nz + zchunk - 1) / zchunk);
  if (P.bc == SWI_BC_ZERO)
    stencil_c64_kernel<SWI_BC_ZERO><<<grid, kThreadsC64, 0, s>>>(P, X, ldx, Y, ldy, ncols, sigma_dev, zchunk);
  else
    stencil_c64_kernel<SWI_BC_ODD><<<grid, kThreadsC64, 0, s>>>(P, X, ldx, Y, ldy, ncols, sigma_dev, zchunk);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
