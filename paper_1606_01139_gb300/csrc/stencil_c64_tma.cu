// Shifted stencil Y = (A - sigma_col) X on complex64 vectors (Eq. 1 applied
// matrix-free, shifted as in Eq. 3), staged by the tensor memory accelerator.
//
// The kernel is HBM-bound (16 bytes of vectors per output against ~40 packed
// FP32 instructions), so it is organised for traffic and latency:
//  - a block owns a 32 x 8 tile of (x, y) points and a group of 4 columns
//    (32 bytes, one sector per point) and marches along z;
//  - the 4 column groups of a tile are adjacent in the grid, so they run
//    together and read every 128-byte row of a 16-column block once from DRAM;
//  - plane j of the tile with its 6-point halo (a 44 x 20 x 4 box), and the
//    plane's (V, Gamma) pairs of the tile, arrive in shared memory by
//    cp.async.bulk.tensor loads, three planes in flight in a ring of four
//    stages, each completed on an mbarrier; nothing else is read from global
//    memory inside the loop;
//  - the z direction is a forward sweep: when plane j lands, its value at a
//    point is added (times the stencil weight) into the 13 pending outputs
//    j - 6 .. j + 6 of that point, kept in a register ring; plane j's own
//    output receives its x and y terms and the diagonal, and output j - 6 is
//    then complete and stored.  The sweep runs over planes z0 - 6 .. z1 + 5
//    of the block's z range (ghost planes by reflection or zero);
//  - each thread computes two points stacked in y for one column (the y
//    neighbours of the pair come from one 14-value strip); the arithmetic is
//    packed FP32x2 (re, im together).
// Ghost points: the tensor map fills out-of-range coordinates with zeros (the
// zero rule, and the planes -1 and n of the odd rule); odd-reflection ghosts
// further out are written into the staged box from their mirror points, and
// reflected z planes are loaded from their mirror plane with a sign.
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
constexpr int kStages = 4;
constexpr int kThreads = kTX * (kTY / 2) * kNC;  // 512: two points (y, y + 1) per thread
constexpr int kBoxFloats = kBY * kBX * kNC * 2;    // 7040 floats = 28,160 bytes
constexpr int kVGFloats = kTY * kTX * 2;           // (V, Gamma) of the tile: 2,048 bytes
constexpr int kStageFloats = kBoxFloats + kVGFloats;  // 30,208 bytes (a multiple of 128)
constexpr unsigned kStageBytes = kStageFloats * 4;
constexpr int kQ = 2 * kR + 1;  // pending outputs per point
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

__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, unsigned long long* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
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

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

}  // namespace

// set by a block whose mbarrier wait gave up (read and cleared by the host)
__device__ int g_stencil_tma_err = 0;

namespace {

template <int BC>
__global__ void __launch_bounds__(kThreads, 1)
    stencil_c64_tma_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap vgmap,
                           const __grid_constant__ StencilC64Params P, float2* __restrict__ Y, int ldy, int ncols,
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
  const bool colok = c < ncols;
  bool ok[2];
  long long pto[2];  // (point index within a plane) * ldy + c
#pragma unroll
  for (int dy = 0; dy < 2; ++dy) {
    ok[dy] = colok && xa < P.nx && ya + dy < P.ny;
    pto[dy] = ((long long)(ya + dy) * P.nx + xa) * ldy + c;
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
  // a list of (cell, mirror cell) built once per block
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
  // the sweep: source planes j = z0 - 6 + t, t < ns
  const int js = z0 - kR, ns = (z1 - z0) + 2 * kR;
  // plane j is loaded from plane zsrc(j) with sign sgn(j) (zsrc = -1: a zero plane)
  auto src_plane = [&](int j, float& sgn) -> int {
    int zs;
    if (!ghost_src<BC>(j, P.nz, zs, sgn)) {
      sgn = 0.f;
      return -1;
    }
    return zs;
  };
  auto issue = [&](int t) {
    const int s = t % kStages;
    const int j = js + t;
    float sg;
    const int zsrc = src_plane(j, sg);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], kStageBytes);
    float* st = stage_mem + s * kStageFloats;
    tma_load_4d(st, &tmap, &bar[s], 2 * c0, x0 - kR, y0 - kR, zsrc);
    tma_load_3d(st + kBoxFloats, &vgmap, &bar[s], 2 * x0, y0, (j >= z0 && j < z1) ? j : -1);
  };
  if (tid == 0) {
    for (int t = 0; t < min(ns, kStages - 1); ++t) issue(t);
  }

  float2 acc[2][kQ];  // pending outputs: plane js + t' in slot t' mod 13
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int k = 0; k < kQ; ++k) acc[dy][k] = make_float2(0.f, 0.f);

  bool bad = false;
  int tlast = 0;
  for (int tb = 0; tb < ns && !bad; tb += kQ) {
#pragma unroll
    for (int u = 0; u < kQ; ++u) {
      const int t = tb + u;
      if (t >= ns) break;
      tlast = t;
      const int j = js + t;
      const int s = t % kStages;
      const unsigned parity = (unsigned)((t / kStages) & 1);
      if (tid == 0 && t + kStages - 1 < ns) issue(t + kStages - 1);
      const bool landed = mbar_wait(&bar[s], parity);
      if (__syncthreads_or(!landed)) {  // one decision for the whole block
        bad = true;
        break;
      }
      float2* S2 = reinterpret_cast<float2*>(stage_mem + s * kStageFloats);  // [kBY][kBX][kNC]
      const float2* VG = reinterpret_cast<const float2*>(stage_mem + s * kStageFloats + kBoxFloats);  // [kTY][kTX]
      const bool real = j >= z0 && j < z1;  // an output plane of this block (uniform)
      if (real && nghost > 0) {  // -(mirror point) into every ghost cell of the box, all columns
        for (int e = tid; e < nghost * kNC; e += kThreads) {
          const unsigned gcell = s_ghost[e / kNC];
          const int col = e % kNC;
          const float2 v = S2[(gcell >> 16) * kNC + col];
          S2[(gcell & 0xffffu) * kNC + col] = make_float2(-v.x, -v.y);
        }
        __syncthreads();
      }
      float sg;
      src_plane(j, sg);
      // the y strip of the pair (14 values); its entries 6 and 7 are the pair's own values
      float2 sy[2 * kR + 2];
      {
        const float2* colp = S2 + ((2 * py) * kBX + px + kR) * kNC + cc;
#pragma unroll
        for (int k = 0; k < 2 * kR + 2; ++k) sy[k] = colp[k * kBX * kNC];
      }
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float2 uc = make_float2(sg * sy[dy + kR].x, sg * sy[dy + kR].y);
        // z terms: plane j into the pending outputs j - 6 .. j + 6 (not j itself)
#pragma unroll
        for (int m = 1; m <= kR; ++m) {
          const float2 w = make_float2(cm[m], cm[m]);
          acc[dy][(u + kQ - m) % kQ] = __ffma2_rn(w, uc, acc[dy][(u + kQ - m) % kQ]);
          acc[dy][(u + m) % kQ] = __ffma2_rn(w, uc, acc[dy][(u + m) % kQ]);
        }
      }
      if (real) {
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const float2 uc = sy[dy + kR];
          const float2 vg = VG[(2 * py + dy) * kTX + px];
          const float d = dcen + vg.x, gm = vg.y;
          float2 a = acc[dy][u % kQ];
          a.x += fmaf(d, uc.x, gm * uc.y);
          a.y += fmaf(d, uc.y, -gm * uc.x);
          // x neighbours (13 values of the point's row) and y neighbours (the strip)
          const float2* row = S2 + ((2 * py + dy + kR) * kBX + px) * kNC + cc;
#pragma unroll
          for (int m = 1; m <= kR; ++m) {
            const float2 t2 = f2add(f2add(row[(kR - m) * kNC], row[(kR + m) * kNC]),
                                    f2add(sy[dy + kR - m], sy[dy + kR + m]));
            a = __ffma2_rn(make_float2(cm[m], cm[m]), t2, a);
          }
          acc[dy][u % kQ] = a;
        }
      }
      // output j - 6 is complete
      const int o = j - kR;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int so = (u + kQ - kR) % kQ;
        if (o >= z0 && ok[dy]) Y[(long long)o * plane * ldy + pto[dy]] = acc[dy][so];
        acc[dy][so] = make_float2(0.f, 0.f);
      }
      __syncthreads();  // stage s is free for the copy issued next step
    }
  }
  if (bad) {
    if (tid == 0) {
      atomicExch(&g_stencil_tma_err, 1);
      // drain the copies still in flight into this block's shared memory (bounded)
      for (int t = tlast; t < min(ns, tlast + kStages); ++t)
        mbar_wait(&bar[t % kStages], (unsigned)((t / kStages) & 1));
    }
    __syncthreads();
  }
}

__global__ void pack_vg_kernel(const float* __restrict__ V, const float* __restrict__ G, int nx, int ny, int nz,
                               int nxp, float2* __restrict__ VG) {
  const long long total = (long long)nxp * ny * nz;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % nxp);
    const long long row = e / nxp;  // z * ny + y
    VG[e] = x < nx ? make_float2(V[row * nx + x], G[row * nx + x]) : make_float2(0.f, 0.f);
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

void launch_pack_vg(const float* V, const float* G, int nx, int ny, int nz, float2* VG, cudaStream_t s) {
  const int nxp = nx + (nx & 1);
  const long long total = (long long)nxp * ny * nz;
  pack_vg_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(V, G, nx, ny, nz, nxp, VG);
  SWI_CHECK_LAUNCH();
}

void launch_stencil_c64_tma(const StencilC64Params& P, const float2* X, int ldx, float2* Y, int ldy, int ncols,
                            const float* sigma_dev, cudaStream_t s, long long* launches) {
  if (ncols <= 0) return;
  if (!stencil_c64_tma_ok(X, ldx) || P.VG == nullptr)
    throw Error{SWI_EINVAL, "TMA stencil: needs an even leading dimension and the packed (V, Gamma) planes"};
  const int nxp = P.nx + (P.nx & 1);
  CUtensorMap map, vgmap;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)2 * ldx, (cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz};
    const cuuint64_t strides[3] = {(cuuint64_t)8 * ldx, (cuuint64_t)8 * ldx * P.nx,
                                   (cuuint64_t)8 * ldx * P.nx * P.ny};
    const cuuint32_t box[4] = {2 * kNC, kBX, kBY, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2*>(X), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{SWI_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
  }
  {
    // (V, Gamma) pairs, rows of nxp points (16-byte row pitch); box = the tile
    const cuuint64_t dims[3] = {(cuuint64_t)2 * nxp, (cuuint64_t)P.ny, (cuuint64_t)P.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)8 * nxp, (cuuint64_t)8 * nxp * P.ny};
    const cuuint32_t box[3] = {2 * kTX, kTY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode_fn()(&vgmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(P.VG), dims,
                                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{SWI_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
  }
  const int tiles_x = (P.nx + kTX - 1) / kTX, tiles_y = (P.ny + kTY - 1) / kTY;
  const int cgroups = (ncols + kNC - 1) / kNC;
  const int blocks_xy = tiles_x * tiles_y * cgroups;
  // about one block per SM; each z chunk at least 24 planes deep (the sweep
  // reads 12 planes beyond its chunk)
  int nzc = std::max(1, (152 + blocks_xy / 2) / blocks_xy);
  nzc = std::max(1, std::min(nzc, P.nz / 24));
  const int zchunk = (P.nz + nzc - 1) / nzc;
  const dim3 grid(blocks_xy, (P.nz + zchunk - 1) / zchunk);
  const size_t smem = (size_t)kStages * kStageBytes;
  if (P.bc == SWI_BC_ZERO) {
    SWI_CUDA_TRY(cudaFuncSetAttribute(stencil_c64_tma_kernel<SWI_BC_ZERO>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    stencil_c64_tma_kernel<SWI_BC_ZERO><<<grid, kThreads, smem, s>>>(map, vgmap, P, Y, ldy, ncols, sigma_dev, zchunk,
                                                                     cgroups, tiles_x);
  } else {
    SWI_CUDA_TRY(cudaFuncSetAttribute(stencil_c64_tma_kernel<SWI_BC_ODD>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    stencil_c64_tma_kernel<SWI_BC_ODD><<<grid, kThreads, smem, s>>>(map, vgmap, P, Y, ldy, ncols, sigma_dev, zchunk,
                                                                    cgroups, tiles_x);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
