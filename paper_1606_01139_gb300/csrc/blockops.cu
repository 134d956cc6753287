// Tall-skinny products over the grid rows, batched over windows.
//
// These are the dense contractions of the Krylov loop: the block
// orthogonalisation C = Q^H W, W -= Q C (the Arnoldi inner products and
// updates that ARPACK performs, whose O(N n_r^2) cost Section 1 attributes to
// orthogonalisation and subspace rotations), the thick-restart rotation Q Z,
// the Gram matrices of the Cholesky-QR and of Algorithm 2, and the
// Gamma-weighted projections of T(E).
//
// In FP64 these kernels are bound by the FP64 pipe (two DFMA per SM clock on
// GB300), not by HBM: they are register-blocked smem GEMMs that keep the DFMA
// pipe fed; the row (N) dimension is split across CTAs and reduced in a fixed
// order so results are deterministic.
#include "swi_internal.cuh"

#include <chrono>

namespace swi {

double now_seconds() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

namespace {

constexpr int kRowStage = 16;  // rows staged in shared memory per step

// One CTA computes a TI x TJ tile of op(X)^H diag(w) Y over a chunk of rows.
// 256 threads as 16 x 16; thread (ty, tx) owns rows ty*RI.. and cols tx*RJ..
__device__ __forceinline__ long long job_offset(const GramBatch& batch, int q, int nchunks) {
  long long off = 0;
  for (int p = 0; p < q; ++p) off += (long long)nchunks * batch.job[p].nx * batch.job[p].ny;
  return off;
}

template <int TI, int TJ, bool BILINEAR>
__global__ void __launch_bounds__(256) gram_partial_kernel(const __grid_constant__ GramBatch batch, int N,
                                                           const double* __restrict__ w, int rows_per_chunk,
                                                           double2* __restrict__ work) {
  constexpr int RI = TI / 16, RJ = TJ / 16;
  __shared__ double2 sx[kRowStage][TI];
  __shared__ double2 sy[kRowStage][TJ];
  const GramJob& J = batch.job[blockIdx.z];
  const int tiles_j = (J.ny + TJ - 1) / TJ;
  const int tiles_i = (J.nx + TI - 1) / TI;
  if ((int)blockIdx.y >= tiles_i * tiles_j) return;
  const int ti0 = (blockIdx.y / tiles_j) * TI;
  const int tj0 = (blockIdx.y % tiles_j) * TJ;
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(N, r0 + rows_per_chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[RI][RJ];
#pragma unroll
  for (int a = 0; a < RI; ++a)
#pragma unroll
    for (int b = 0; b < RJ; ++b) acc[a][b] = make_double2(0.0, 0.0);

  for (int rb = r0; rb < r1; rb += kRowStage) {
    // stage rows [rb, rb + kRowStage)
    for (int e = threadIdx.x; e < kRowStage * TI; e += 256) {
      const int rr = e / TI, cc = e % TI;
      const int r = rb + rr, col = ti0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (r < r1 && col < J.nx) {
        v = __ldg(J.X + (long long)r * J.ldx + col);
        if (!BILINEAR) v.y = -v.y;  // conj for the Hermitian product
      }
      sx[rr][cc] = v;
    }
    for (int e = threadIdx.x; e < kRowStage * TJ; e += 256) {
      const int rr = e / TJ, cc = e % TJ;
      const int r = rb + rr, col = tj0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (r < r1 && col < J.ny) {
        v = __ldg(J.Y + (long long)r * J.ldy + col);
        if (w) {
          const double s = __ldg(w + r);
          v.x *= s;
          v.y *= s;
        }
      }
      sy[rr][cc] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kRowStage; ++rr) {
      double2 xa[RI], yb[RJ];
#pragma unroll
      for (int a = 0; a < RI; ++a) xa[a] = sx[rr][ty * RI + a];
#pragma unroll
      for (int b = 0; b < RJ; ++b) yb[b] = sy[rr][tx * RJ + b];
#pragma unroll
      for (int a = 0; a < RI; ++a)
#pragma unroll
        for (int b = 0; b < RJ; ++b) cfma(acc[a][b], xa[a], yb[b]);
    }
    __syncthreads();
  }
  // partial tile -> work[job_off + chunk * nx * ny + i * ny + j]
  double2* out = work + job_offset(batch, blockIdx.z, gridDim.x) + (long long)blockIdx.x * J.nx * J.ny;
#pragma unroll
  for (int a = 0; a < RI; ++a) {
    const int i = ti0 + ty * RI + a;
    if (i >= J.nx) continue;
#pragma unroll
    for (int b = 0; b < RJ; ++b) {
      const int j = tj0 + tx * RJ + b;
      if (j < J.ny) out[(long long)i * J.ny + j] = acc[a][b];
    }
  }
}

__global__ void gram_reduce_kernel(const __grid_constant__ GramBatch batch, int nchunks,
                                   const double2* __restrict__ work) {
  const GramJob& J = batch.job[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= J.nx * J.ny) return;
  const double2* src = work + job_offset(batch, blockIdx.y, nchunks);
  double2 s = make_double2(0.0, 0.0);
  for (int c = 0; c < nchunks; ++c) s = cadd(s, src[(long long)c * J.nx * J.ny + e]);
  const int i = e / J.ny, j = e % J.ny;
  double2* dst = J.C + (long long)i * J.ldc + j;
  if (J.accumulate) s = cadd(s, *dst);
  *dst = s;
}

// Out tile (RN rows x TJ cols) = beta*Yin + X[rows, 0:k] * M[0:k, cols]
template <int RN, int TJ>
__global__ void __launch_bounds__(256) rowgemm_kernel(const __grid_constant__ RowGemmBatch batch, int N) {
  constexpr int KC = 16;
  constexpr int RR = RN / 16, RJ = TJ / 16;
  __shared__ double2 sa[RN][KC + 1];
  __shared__ double2 sb[KC][TJ];
  const RowGemmJob& J = batch.job[blockIdx.z];
  const int c0 = blockIdx.y * TJ;
  if (c0 >= J.ncols) return;
  const int r0 = blockIdx.x * RN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[RR][RJ];
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RJ; ++b) acc[a][b] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < J.k; k0 += KC) {
    for (int e = threadIdx.x; e < RN * KC; e += 256) {
      const int rr = e / KC, kk = e % KC;
      const int r = r0 + rr, k = k0 + kk;
      sa[rr][kk] = (r < N && k < J.k) ? __ldg(J.X + (long long)r * J.ldx + k) : make_double2(0.0, 0.0);
    }
    for (int e = threadIdx.x; e < KC * TJ; e += 256) {
      const int kk = e / TJ, cc = e % TJ;
      const int k = k0 + kk, c = c0 + cc;
      sb[kk][cc] = (k < J.k && c < J.ncols) ? __ldg(J.M + (long long)k * J.ldm + c) : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double2 xa[RR], yb[RJ];
#pragma unroll
      for (int a = 0; a < RR; ++a) xa[a] = sa[ty * RR + a][kk];
#pragma unroll
      for (int b = 0; b < RJ; ++b) yb[b] = sb[kk][tx * RJ + b];
#pragma unroll
      for (int a = 0; a < RR; ++a)
#pragma unroll
        for (int b = 0; b < RJ; ++b) cfma(acc[a][b], xa[a], yb[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < RR; ++a) {
    const int r = r0 + ty * RR + a;
    if (r >= N) continue;
#pragma unroll
    for (int b = 0; b < RJ; ++b) {
      const int c = c0 + tx * RJ + b;
      if (c >= J.ncols) continue;
      double2 v = cscale(acc[a][b], J.alpha);
      if (J.Yin) {
        const double2 y = J.Yin[(long long)r * J.ldy + c];
        v.x = fma(J.beta, y.x, v.x);
        v.y = fma(J.beta, y.y, v.y);
      }
      J.Out[(long long)r * J.ldo + c] = v;
    }
  }
}

__global__ void colnorm_partial_kernel(const double2* __restrict__ X, int ldx, const double2* __restrict__ Y, int ldy,
                                       const double2* __restrict__ theta, int ncols, int N, int rows_per_chunk,
                                       double* __restrict__ work) {
  // blockDim.x = 256 threads cover columns cyclically; each chunk of rows per CTA
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(N, r0 + rows_per_chunk);
  for (int c = threadIdx.x + blockIdx.y * blockDim.x; c < ncols; c += blockDim.x * gridDim.y) {
    const double2 th = theta ? theta[c] : make_double2(0.0, 0.0);
    double s = 0.0;
    for (int r = r0; r < r1; ++r) {
      double2 y = Y[(long long)r * ldy + c];
      if (theta) {
        const double2 x = X[(long long)r * ldx + c];
        y = csub(y, cmul(th, x));
      }
      s = fma(y.x, y.x, fma(y.y, y.y, s));
    }
    work[(long long)blockIdx.x * ncols + c] = s;
  }
}

__global__ void colnorm_reduce_kernel(const double* __restrict__ work, int nchunks, int ncols, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int q = 0; q < nchunks; ++q) s += work[(long long)q * ncols + c];
  out[c] = sqrt(s);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  // SplitMix64 (Steele, Lea, Flood 2014): counter-based, one 64-bit output per counter.
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void random_block_kernel(double2* X, int ld, int c0, int ncols, int N, unsigned long long seed) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * ncols) return;
  const long long r = t / ncols;
  const int c = (int)(t % ncols);
  const unsigned long long ctr = (unsigned long long)(r * 4096 + (c0 + c)) * 2ull;
  const unsigned long long a = splitmix64(seed * 0x632BE59BD9B4E019ull + ctr);
  const unsigned long long b = splitmix64(seed * 0x632BE59BD9B4E019ull + ctr + 1);
  const double inv = 1.0 / 9007199254740992.0;  // 2^-53
  X[r * ld + c0 + c] = make_double2((double)(a >> 11) * inv - 0.5, (double)(b >> 11) * inv - 0.5);
}

__global__ void copy_block_kernel(const double2* __restrict__ src, int lds, double2* __restrict__ dst, int ldd, int rows,
                                  int cols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)rows * cols) return;
  const long long r = t / cols;
  const int c = (int)(t % cols);
  dst[r * ldd + c] = src[r * lds + c];
}

// dst[:, q] = src[:, idx[q]], q < n
__global__ void gather_cols_kernel(const double2* __restrict__ src, int lds, const int* __restrict__ idx, int n,
                                   double2* __restrict__ dst, int ldd, int rows) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)rows * n) return;
  const long long r = t / n;
  const int q = (int)(t % n);
  dst[r * ldd + q] = src[r * lds + idx[q]];
}

// Y[:, q] -= eps[q] X[:, q], q < n (complex eps)
__global__ void sub_diag_kernel(double2* __restrict__ Y, int ldy, const double2* __restrict__ X, int ldx,
                                const double2* __restrict__ eps, int n, int rows) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)rows * n) return;
  const long long r = t / n;
  const int q = (int)(t % n);
  const double2 x = X[r * ldx + q], e = eps[q];
  double2 y = Y[r * ldy + q];
  y.x -= e.x * x.x - e.y * x.y;
  y.y -= e.x * x.y + e.y * x.x;
  Y[r * ldy + q] = y;
}

}  // namespace

void launch_gather_cols(const double2* src, int lds, const int* idx, int n, double2* dst, int ldd, int rows,
                        cudaStream_t s, long long* launches) {
  const long long t = (long long)rows * n;
  if (t == 0) return;
  gather_cols_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(src, lds, idx, n, dst, ldd, rows);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_sub_diag(double2* Y, int ldy, const double2* X, int ldx, const double2* eps, int n, int rows,
                     cudaStream_t s, long long* launches) {
  const long long t = (long long)rows * n;
  if (t == 0) return;
  sub_diag_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(Y, ldy, X, ldx, eps, n, rows);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_gram(const GramBatch& b, int N, const double* w, int bilinear, double2* work, size_t work_elems,
                 cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  int maxnx = 0, maxny = 0;
  long long per_chunk = 0;
  for (int q = 0; q < b.n; ++q) {
    maxnx = b.job[q].nx > maxnx ? b.job[q].nx : maxnx;
    maxny = b.job[q].ny > maxny ? b.job[q].ny : maxny;
    per_chunk += (long long)b.job[q].nx * b.job[q].ny;
  }
  const bool narrow = maxny <= 16;
  const int TI = narrow ? 64 : 32, TJ = narrow ? 16 : 32;
  const int tiles = ((maxnx + TI - 1) / TI) * ((maxny + TJ - 1) / TJ);
  // chunks: enough CTAs to cover the SMs ~4x, bounded by the workspace
  int nchunks = (4 * 152 + tiles * b.n - 1) / (tiles * b.n);
  const int max_by_rows = (N + 255) / 256;
  if (nchunks > max_by_rows) nchunks = max_by_rows;
  if (nchunks < 1) nchunks = 1;
  while (nchunks > 1 && (size_t)nchunks * per_chunk > work_elems) --nchunks;
  if ((size_t)per_chunk > work_elems) throw Error{SWI_ENOMEM, "gram workspace too small"};
  int rows_per_chunk = (N + nchunks - 1) / nchunks;
  rows_per_chunk = (rows_per_chunk + kRowStage - 1) / kRowStage * kRowStage;
  nchunks = (N + rows_per_chunk - 1) / rows_per_chunk;
  dim3 grid(nchunks, tiles, b.n);
  if (narrow) {
    if (bilinear)
      gram_partial_kernel<64, 16, true><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
    else
      gram_partial_kernel<64, 16, false><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
  } else {
    if (bilinear)
      gram_partial_kernel<32, 32, true><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
    else
      gram_partial_kernel<32, 32, false><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
  }
  SWI_CHECK_LAUNCH();
  const int maxe = maxnx * maxny;
  gram_reduce_kernel<<<dim3((maxe + 255) / 256, b.n), 256, 0, s>>>(b, nchunks, work);
  SWI_CHECK_LAUNCH();
  if (launches) *launches += 2;
}

void launch_rowgemm(const RowGemmBatch& b, int N, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  int maxc = 0;
  for (int q = 0; q < b.n; ++q) maxc = b.job[q].ncols > maxc ? b.job[q].ncols : maxc;
  if (maxc <= 16) {
    dim3 grid((N + 63) / 64, 1, b.n);
    rowgemm_kernel<64, 16><<<grid, 256, 0, s>>>(b, N);
  } else {
    dim3 grid((N + 31) / 32, (maxc + 31) / 32, b.n);
    rowgemm_kernel<32, 32><<<grid, 256, 0, s>>>(b, N);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_colnorm_resid(const double2* X, int ldx, const double2* Y, int ldy, const double2* theta, int ncols,
                          int N, double* out, double* work, size_t work_elems, cudaStream_t s, long long* launches) {
  int nchunks = 4 * 152;
  if (nchunks > N) nchunks = N;
  while (nchunks > 1 && (size_t)nchunks * ncols > work_elems) nchunks /= 2;
  const int rows_per_chunk = (N + nchunks - 1) / nchunks;
  nchunks = (N + rows_per_chunk - 1) / rows_per_chunk;
  const int gy = (ncols + 255) / 256;
  colnorm_partial_kernel<<<dim3(nchunks, gy), 256, 0, s>>>(X, ldx, Y, ldy, theta, ncols, N, rows_per_chunk, work);
  SWI_CHECK_LAUNCH();
  colnorm_reduce_kernel<<<(ncols + 255) / 256, 256, 0, s>>>(work, nchunks, ncols, out);
  SWI_CHECK_LAUNCH();
  if (launches) *launches += 2;
}

void launch_random_block(double2* X, int ld, int c0, int ncols, int N, unsigned long long seed, cudaStream_t s,
                         long long* launches) {
  const long long n = (long long)N * ncols;
  random_block_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, ld, c0, ncols, N, seed);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_copy_block(const double2* src, int lds, double2* dst, int ldd, int rows, int cols, cudaStream_t s,
                       long long* launches) {
  const long long n = (long long)rows * cols;
  if (n == 0) return;
  copy_block_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
