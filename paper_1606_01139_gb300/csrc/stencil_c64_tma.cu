// Shifted stencil Y = (A - sigma_col) X on complex64 vectors (Eq. 1 applied
// matrix-free, shifted as in Eq. 3), staged by the tensor memory accelerator.
//
// The kernel is HBM-bound (16 bytes of vectors per output against ~40 packed
// FP32 instructions), so it is organised for traffic:
//  - a block owns a 32 x 8 tile of (x, y) points and a group of 4 columns
//    (32 bytes, one sector per point) and marches along z;
//  - the 4 column groups of a tile are adjacent in the grid, so they run
//    together and read every 128-byte row of a 16-column block once from DRAM;
//  - plane z of the tile with its 6-point halo (a 44 x 20 x 4 box) arrives in
//    shared memory by one cp.async.bulk.tensor load, three planes in flight in
//    a ring of stages, each completed on an mbarrier;
//  - each thread computes two points stacked in y for one column: the
//    y-neighbours of the pair come from one 14-value strip (19 shared loads
//    per output instead of 24), the 12 z-neighbours from a register queue
//    filled by loads two planes ahead (512 threads, 16 warps per SM);
//  - the arithmetic is packed FP32x2 (re, im together).
// Ghost points: the tensor map fills out-of-range coordinates with zeros (the
// zero rule, and the planes -1 and n of the odd rule); odd-reflection ghosts
// further out are written into the staged box from their mirror points.
// Every mbarrier wait is bounded: on timeout the block records an error flag,
// drains its copies in flight (again bounded) and returns.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "swi_internal.cuh"

namespace swi {

namespace {

constexpr int kTX = 32, kTY = 8, kR = 6, kNC = 4;
constexpr int kBX = kTX + 2 * kR, kBY = kTY + 2 * kR;  // staged box (44 x 20 points)
constexpr int kStages = 3;
constexpr int kThreads = kTX * (kTY / 2) * kNC;  // 512: two points (y, y + 1) per thread
constexpr int kStageFloats = kBY * kBX * kNC * 2;       // 7040 floats = 28,160 bytes
constexpr unsigned kStageBytes = kStageFloats * 4;
constexpr long long kSpinLimit = 1LL << 26;  // ~ seconds of polling: a lost copy, not a slow one

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// true once the phase with the given parity has completed; false after kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_4d(float* dst, const CUtensorMap* map, unsigned long long* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// source index and sign of axis index j on a line of n points (odd reflection
// about the planes -1 and n, or zero); false for a zero ghost
template <int BC>
__device__ __forceinline__ bool ghost_src(int j, int n, int& src, float& sgn) {
  if (j >= 0 && j < n) {
    src = j;
    sgn = 1.f;
    return true;
  }
  if (BC == SWI_BC_ZERO) return false;
  if (j <= -2) src = -2 - j;
  else if (j >= n + 1) src = 2 * n - j;
  else return false;
  if (src < 0 || src >= n) return false;
  sgn = -1.f;
  return true;
}

template <int BC>
__device__ __forceinline__ float2 load_z(const float2* __restrict__ X, long long pt_col, long long plane_ld, int z,
                                         int nz, bool ok) {
  int src;
  float sgn;
  if (!ok || !ghost_src<BC>(z, nz, src, sgn)) return make_float2(0.f, 0.f);
  const float2 v = __ldg(X + pt_col + (long long)src * plane_ld);
  return make_float2(sgn * v.x, sgn * v.y);
}

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

}  // namespace

// set by a block whose mbarrier wait gave up (read and cleared by the host)
__device__ int g_stencil_tma_err = 0;

namespace {

template <int BC>
__global__ void __launch_bounds__(kThreads, 1)
    stencil_c64_tma_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ StencilC64Params P,
                           const float2* __restrict__ X, int ldx, float2* __restrict__ Y, int ldy, int ncols,
                           const float* __restrict__ sigma, int zchunk, int cgroups, int tiles_x) {
  extern __shared__ __align__(128) float stage_mem[];
  __shared__ __align__(8) unsigned long long bar[kStages];
  __shared__ unsigned s_ghost[kBY * kBX];  // cell | mirror cell << 16 (box cells < 2^16)
  __shared__ int s_nghost;
  const int tid = threadIdx.x;
  const int cc = tid % kNC;
  const int px = (tid / kNC) % kTX;
  const int py = tid / (kNC * kTX);
  const int g = blockIdx.x % cgroups;
  const int tile = blockIdx.x / cgroups;
  const int x0 = (tile % tiles_x) * kTX, y0 = (tile / tiles_x) * kTY;
  const int c0 = g * kNC, c = c0 + cc;
  const int z0 = blockIdx.y * zchunk, z1 = min(P.nz, z0 + zchunk);
  const int xa = x0 + px, ya = y0 + 2 * py;  // the pair's first point
  const long long plane = (long long)P.nx * P.ny;
  const long long plane_ld = plane * ldx;
  const bool colok = c < ncols;
  bool ok[2][1];
  long long ptc[2][1];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 1; ++dx) {
      ok[dy][dx] = colok && xa + dx < P.nx && ya + dy < P.ny;  // dx = 0: one point per row
      ptc[dy][dx] = ((long long)(ya + dy) * P.nx + (xa + dx)) * ldx + c;
    }
  float cm[kR + 1];
#pragma unroll
  for (int m = 0; m <= kR; ++m) cm[m] = P.cm[m];
  const float sig = colok ? sigma[c] : 0.f;
  const float dcen = 3.f * cm[0] - sig;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_nghost = 0;
  }
  __syncthreads();
  // odd-reflection ghosts inside the staged box (the same cells every plane):
  // a list of (cell, mirror cell, sign) built once per block
  const bool fixup = BC == SWI_BC_ODD && (x0 < kR || y0 < kR || x0 + kTX + kR > P.nx || y0 + kTY + kR > P.ny);
  if (fixup) {
    for (int e = tid; e < kBY * kBX; e += kThreads) {
      const int bx = e % kBX, by = e / kBX;
      const int gx = x0 - kR + bx, gy = y0 - kR + by;
      const bool gxin = gx >= 0 && gx < P.nx, gyin = gy >= 0 && gy < P.ny;
      if (gxin == gyin) continue;  // interior cells, and corners (never read)
      int sx, sy;
      float f;
      int src = -1;
      if (!gxin) {
        if (ghost_src<BC>(gx, P.nx, sx, f)) src = by * kBX + (sx - x0 + kR);
      } else if (ghost_src<BC>(gy, P.ny, sy, f)) {
        src = (sy - y0 + kR) * kBX + bx;
      }
      if (src >= 0) s_ghost[atomicAdd(&s_nghost, 1)] = (unsigned)e | ((unsigned)src << 16);
    }
    __syncthreads();
  }
  const int nghost = fixup ? s_nghost : 0;
  // prologue: planes z0, z0 + 1 in flight
  auto issue = [&](int z) {
    const int s = (z - z0) % kStages;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], kStageBytes);
    tma_load_4d(stage_mem + s * kStageFloats, &tmap, &bar[s], 2 * c0, x0 - kR, y0 - kR, z);
  };
  if (tid == 0) {
    for (int z = z0; z < min(z1, z0 + kStages - 1); ++z) issue(z);
  }

  // z queues of the two points, a ring of 13 planes: plane z0 - 6 + k in slot k
  // (mod 13); the z loop is unrolled by 13 so every slot index is a constant
  float2 q[2][1][2 * kR + 1];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 1; ++dx)
#pragma unroll
      for (int k = 0; k < 2 * kR + 1; ++k) q[dy][dx][k] = load_z<BC>(X, ptc[dy][dx], plane_ld, z0 - kR + k, P.nz, ok[dy][dx]);

  float vnext[2][1], gnext[2][1];
  float2 nq1[2][1];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy) nq1[dy][0] = load_z<BC>(X, ptc[dy][0], plane_ld, z0 + kR + 1, P.nz, ok[dy][0]);
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 1; ++dx) {
      const long long pi = (long long)z0 * plane + (long long)(ya + dy) * P.nx + (xa + dx);
      vnext[dy][dx] = ok[dy][dx] ? __ldg(P.V + pi) : 0.f;
      gnext[dy][dx] = ok[dy][dx] ? __ldg(P.G + pi) : 0.f;
    }

  bool bad = false;
  int zs = z0;
  for (int zb = z0; zb < z1 && !bad; zb += 2 * kR + 1) {
#pragma unroll
    for (int j = 0; j < 2 * kR + 1; ++j) {
      zs = zb + j;
      if (zs >= z1) break;
      const int s = (zs - z0) % kStages;
      const unsigned parity = (unsigned)(((zs - z0) / kStages) & 1);
      // queue entries two planes ahead and the local potential one plane ahead,
      // loaded before the wait
      float vv[2][1], gg[2][1];
      float2 nq[2][1];
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 1; ++dx) {
          nq[dy][dx] = nq1[dy][dx];
          nq1[dy][dx] = load_z<BC>(X, ptc[dy][dx], plane_ld, zs + kR + 2, P.nz, ok[dy][dx]);
          vv[dy][dx] = vnext[dy][dx];
          gg[dy][dx] = gnext[dy][dx];
          const long long pi = (long long)(zs + 1) * plane + (long long)(ya + dy) * P.nx + (xa + dx);
          const bool ld = ok[dy][dx] && zs + 1 < z1;
          vnext[dy][dx] = ld ? __ldg(P.V + pi) : 0.f;
          gnext[dy][dx] = ld ? __ldg(P.G + pi) : 0.f;
        }
      if (tid == 0 && zs + kStages - 1 < z1) issue(zs + kStages - 1);
      const bool landed = mbar_wait(&bar[s], parity);
      if (__syncthreads_or(!landed)) {  // one decision for the whole block
        bad = true;
        break;
      }
      float2* S2 = reinterpret_cast<float2*>(stage_mem + s * kStageFloats);  // [kBY][kBX][kNC]
      if (nghost > 0) {  // -(mirror point) into every ghost cell of the box, all columns
        for (int e = tid; e < nghost * kNC; e += kThreads) {
          const unsigned gcell = s_ghost[e / kNC];
          const int col = e % kNC;
          const float2 u = S2[(gcell >> 16) * kNC + col];
          S2[(gcell & 0xffffu) * kNC + col] = make_float2(-u.x, -u.y);
        }
        __syncthreads();
      }
      constexpr int Q = 2 * kR + 1;
      float2 acc[2][1];
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 1; ++dx) {
          const float2 u = q[dy][dx][(kR + j) % Q];
          const float d = dcen + vv[dy][dx], gm = gg[dy][dx];
          acc[dy][dx] = make_float2(fmaf(d, u.x, gm * u.y), fmaf(d, u.y, -gm * u.x));
        }
      // x neighbours of each point (13 values of its row)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float2* row = S2 + ((2 * py + dy + kR) * kBX + px) * kNC + cc;
#pragma unroll
        for (int m = 1; m <= kR; ++m)
          acc[dy][0] = __ffma2_rn(make_float2(cm[m], cm[m]), f2add(row[(kR - m) * kNC], row[(kR + m) * kNC]), acc[dy][0]);
      }
      // y strip of the pair (14 values), together with the z queues
      {
        float2 sy[2 * kR + 2];
        const float2* colp = S2 + ((2 * py) * kBX + px + kR) * kNC + cc;
#pragma unroll
        for (int k = 0; k < 2 * kR + 2; ++k) sy[k] = colp[k * kBX * kNC];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int m = 1; m <= kR; ++m) {
            const float2 t = f2add(f2add(sy[dy + kR - m], sy[dy + kR + m]),
                                   f2add(q[dy][0][(kR - m + j) % Q], q[dy][0][(kR + m + j) % Q]));
            acc[dy][0] = __ffma2_rn(make_float2(cm[m], cm[m]), t, acc[dy][0]);
          }
      }
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 1; ++dx) {
          if (ok[dy][dx]) Y[((long long)zs * plane + (long long)(ya + dy) * P.nx + (xa + dx)) * ldy + c] = acc[dy][dx];
          q[dy][dx][j % Q] = nq[dy][dx];  // plane zs + 7 replaces plane zs - 6
        }
      __syncthreads();  // stage s is free for the copy issued next step
    }
  }
  if (bad) {
    if (tid == 0) {
      atomicExch(&g_stencil_tma_err, 1);
      // drain the copies still in flight into this block's shared memory (bounded)
      for (int z = zs; z < min(z1, zs + kStages); ++z)
        mbar_wait(&bar[(z - z0) % kStages], (unsigned)(((z - z0) / kStages) & 1));
    }
    __syncthreads();
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

}  // namespace

bool stencil_c64_tma_ok(const float2* X, int ldx) {
  // the tensor map needs 16-byte aligned rows (even column counts) and base
  return ldx % 2 == 0 && (reinterpret_cast<unsigned long long>(X) & 15ull) == 0 && encode_fn() != nullptr;
}

int stencil_c64_tma_error(bool clear) {
  int v = 0;
  SWI_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_stencil_tma_err, sizeof(int)));
  if (clear && v) {
    const int z = 0;
    SWI_CUDA_TRY(cudaMemcpyToSymbol(g_stencil_tma_err, &z, sizeof(int)));
  }
  return v;
}

void launch_stencil_c64_tma(const StencilC64Params& P, const float2* X, int ldx, float2* Y, int ldy, int ncols,
                            const float* sigma_dev, cudaStream_t s, long long* launches) {
  if (ncols <= 0) return;
  if (!stencil_c64_tma_ok(X, ldx)) throw Error{SWI_EINVAL, "TMA stencil: needs an even leading dimension"};
  CUtensorMap map;
  const cuuint64_t dims[4] = {(cuuint64_t)2 * ldx, (cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz};
  const cuuint64_t strides[3] = {(cuuint64_t)8 * ldx, (cuuint64_t)8 * ldx * P.nx,
                                 (cuuint64_t)8 * ldx * P.nx * P.ny};
  const cuuint32_t box[4] = {2 * kNC, kBX, kBY, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2*>(X), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{SWI_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
  const int tiles_x = (P.nx + kTX - 1) / kTX, tiles_y = (P.ny + kTY - 1) / kTY;
  const int cgroups = (ncols + kNC - 1) / kNC;
  const int blocks_xy = tiles_x * tiles_y * cgroups;
  // about one block per SM; each z chunk at least 16 planes deep
  int nzc = std::max(1, (152 + blocks_xy / 2) / blocks_xy);
  nzc = std::max(1, std::min(nzc, P.nz / 16));
  const int zchunk = (P.nz + nzc - 1) / nzc;
  const dim3 grid(blocks_xy, (P.nz + zchunk - 1) / zchunk);
  const size_t smem = (size_t)kStages * kStageBytes;
  if (P.bc == SWI_BC_ZERO) {
    SWI_CUDA_TRY(cudaFuncSetAttribute(stencil_c64_tma_kernel<SWI_BC_ZERO>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    stencil_c64_tma_kernel<SWI_BC_ZERO><<<grid, kThreads, smem, s>>>(map, P, X, ldx, Y, ldy, ncols, sigma_dev, zchunk,
                                                                     cgroups, tiles_x);
  } else {
    SWI_CUDA_TRY(cudaFuncSetAttribute(stencil_c64_tma_kernel<SWI_BC_ODD>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    stencil_c64_tma_kernel<SWI_BC_ODD><<<grid, kThreads, smem, s>>>(map, P, X, ldx, Y, ldy, ncols, sigma_dev, zchunk,
                                                                    cgroups, tiles_x);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
