// Complex64 helpers of the single-vector Krylov loop: the in-place restart
// rotation of a complex64 basis (FP32 products), conversions between complex64
// and complex128 blocks, column copies and the counter-based random start
// vectors.  The Gram-Schmidt passes themselves are in krylov_sv.cu.
#include <algorithm>

#include "swi_internal.cuh"

namespace swi {

namespace {

// In-place rotation Q[r, 0:k] = Q[r, 0:m] Z32 (Z32 [m][ldz] complex64), a tile of
// kRotRows rows per block: the whole input rows are staged in shared memory
// before any output is written, so no block reads what another one writes.
constexpr int kRotRows = 16;
constexpr int kRotThreads = 256;

__global__ void __launch_bounds__(kRotThreads) rotate_inplace_kernel(float2* __restrict__ Q, int ldq, int N, int m,
                                                                     const float2* __restrict__ Z, int ldz, int k) {
  extern __shared__ float2 qs[];  // [kRotRows][m]
  const int r0 = blockIdx.x * kRotRows;
  const int rows = min(kRotRows, N - r0);
  for (int e = threadIdx.x; e < rows * m; e += kRotThreads) {
    const int rr = e / m, i = e % m;
    qs[rr * m + i] = Q[(long long)(r0 + rr) * ldq + i];
  }
  __syncthreads();
  // thread -> (column j, row group): each thread accumulates rows rr, rr + 4, ...
  for (int j0 = 0; j0 < k; j0 += kRotThreads / 4) {
    const int j = j0 + (threadIdx.x >> 2);
    const int rg = threadIdx.x & 3;
    float2 acc[kRotRows / 4];
#pragma unroll
    for (int t = 0; t < kRotRows / 4; ++t) acc[t] = make_float2(0.f, 0.f);
    if (j < k) {
      for (int i = 0; i < m; ++i) {
        const float2 z = __ldg(Z + (long long)i * ldz + j);
#pragma unroll
        for (int t = 0; t < kRotRows / 4; ++t) {
          const float2 q = qs[(rg + 4 * t) * m + i];
          acc[t].x = fmaf(q.x, z.x, fmaf(-q.y, z.y, acc[t].x));
          acc[t].y = fmaf(q.x, z.y, fmaf(q.y, z.x, acc[t].y));
        }
      }
    }
    if (j < k) {
#pragma unroll
      for (int t = 0; t < kRotRows / 4; ++t) {
        const int rr = rg + 4 * t;
        if (rr < rows) Q[(long long)(r0 + rr) * ldq + j] = acc[t];
      }
    }
  }
}

__global__ void z_to_c64_kernel(const double2* __restrict__ Z, int ldz, int m, int k, float2* __restrict__ Z32,
                                int ld32) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int i = e / k, j = e % k;
  const double2 z = Z[(long long)i * ldz + j];
  Z32[(long long)i * ld32 + j] = make_float2((float)z.x, (float)z.y);
}

__global__ void widen_kernel(const float2* __restrict__ src, int lds, double2* __restrict__ dst, int ldd, int rows,
                             int cols) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const long long r = e / cols;
  const int c = (int)(e % cols);
  const float2 v = src[r * lds + c];
  dst[r * ldd + c] = make_double2(v.x, v.y);
}

__global__ void narrow_kernel(const double2* __restrict__ src, int lds, float2* __restrict__ dst, int ldd, int rows,
                              int cols) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const long long r = e / cols;
  const int c = (int)(e % cols);
  const double2 v = src[r * lds + c];
  dst[r * ldd + c] = make_float2((float)v.x, (float)v.y);
}

__global__ void copy_col_c64_kernel(const float2* __restrict__ src, int lds, float2* __restrict__ dst, int ldd,
                                    int rows) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x)
    dst[r * ldd] = src[r * lds];
}

// counter-based generator (splitmix64 finaliser of seed and index), uniform in (-1, 1)
__device__ __forceinline__ float hash_unit(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

__global__ void random_col_c64_kernel(float2* __restrict__ dst, int ld, int rows, unsigned long long seed) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x)
    dst[r * ld] = make_float2(hash_unit(seed, 2 * r), hash_unit(seed, 2 * r + 1));
}

}  // namespace

void launch_c64_rotate_inplace(float2* Q, int ldq, int N, int m, const float2* Z32, int ldz, int k, cudaStream_t s,
                               long long* launches) {
  if (k <= 0) return;
  if (k > m || m > ldq) throw Error{SWI_ECUDA, "internal: rotation sizes out of range"};
  const size_t smem = (size_t)kRotRows * m * sizeof(float2);
  if (smem > 200 * 1024) throw Error{SWI_EINVAL, "rotation: basis too large for one shared-memory tile"};
  SWI_CUDA_TRY(cudaFuncSetAttribute(rotate_inplace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  rotate_inplace_kernel<<<(N + kRotRows - 1) / kRotRows, kRotThreads, smem, s>>>(Q, ldq, N, m, Z32, ldz, k);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_z_to_c64(const double2* Z, int ldz, int m, int k, float2* Z32, int ld32, cudaStream_t s,
                     long long* launches) {
  if (m * k <= 0) return;
  z_to_c64_kernel<<<(m * k + 255) / 256, 256, 0, s>>>(Z, ldz, m, k, Z32, ld32);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_widen(const float2* src, int lds, double2* dst, int ldd, int rows, int cols, cudaStream_t s,
                  long long* launches) {
  const long long n = (long long)rows * cols;
  if (n <= 0) return;
  widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_narrow(const double2* src, int lds, float2* dst, int ldd, int rows, int cols, cudaStream_t s,
                   long long* launches) {
  const long long n = (long long)rows * cols;
  if (n <= 0) return;
  narrow_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_copy_col_c64(const float2* src, int lds, float2* dst, int ldd, int rows, cudaStream_t s,
                         long long* launches) {
  copy_col_c64_kernel<<<std::min((rows + 255) / 256, 1024), 256, 0, s>>>(src, lds, dst, ldd, rows);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_random_col_c64(float2* dst, int ld, int rows, unsigned long long seed, cudaStream_t s,
                           long long* launches) {
  random_col_c64_kernel<<<std::min((rows + 255) / 256, 1024), 256, 0, s>>>(dst, ld, rows, seed);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
