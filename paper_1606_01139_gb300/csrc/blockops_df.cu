// FP64-class tall-skinny products on the FP32 pipes (double-single arithmetic).
//
// GB300 executes FP64 at 1/70 of its FP32 rate, so the FP64 Gram and update
// products of the Krylov loop (C = Q^H W, W -= Q C, the Cholesky-QR Grams and
// the restart rotations) run here in double-single arithmetic: every FP64
// operand is split once into an unevaluated sum hi + lo of two floats while it
// is staged in shared memory, each product is formed exactly with FMA
// (a_hi b_hi + its rounding error + the cross terms), and the running sum is
// kept as an FP32 head accumulated with TwoSum (Knuth) plus an FP32 tail that
// collects the rounding errors.  The result is returned in FP64.  Per product
// term the relative error is ~2^-48; a dot product of K terms is accurate to
// ~K 2^-48, i.e. ~1e-13 for the bases used here, and every reduction across
// CTAs is done in FP64 in a fixed order.
#include "swi_internal.cuh"

namespace swi {

namespace {

constexpr int kRowStage = 16;

struct f2c {  // complex double-single: re = (rh, rl), im = (ih, il)
  float rh, rl, ih, il;
};

// x = hi + lo from the bit fields of x, on the integer and FP32 pipes (GB300's
// FP64 pipe is the scarce one): hi is x rounded to 24 significant bits, lo the
// signed 29-bit remainder rounded to a float, so |x - hi - lo| <= 2^-48 |x| as
// with the FP64 split.  Magnitudes below 2^-74 (where the remainder would leave
// the float range) and near the top of the float range take the FP64 route.
__device__ __forceinline__ void split1(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int top = (unsigned int)(b >> 32);
  const unsigned int sgn = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7ff);
  if (e >= 949 && e <= 1149) {
    const unsigned int up = (unsigned int)(b >> 28) & 1u;  // round half up on the first dropped bit
    const unsigned int fb = ((unsigned int)(e - 896) << 23 | ((unsigned int)(b >> 29) & 0x7fffffu)) + up;
    hi = __uint_as_float(sgn | fb);
    const int rem = (int)((unsigned int)b & 0x1fffffffu) - (int)(up << 29);  // x - hi in units of 2^(e-1075)
    const float t = (float)rem * __uint_as_float((unsigned int)(e - 948) << 23);
    lo = sgn ? -t : t;
  } else {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
}

__device__ __forceinline__ f2c split(double2 v) {
  f2c r;
  split1(v.x, r.rh, r.rl);
  split1(v.y, r.ih, r.il);
  return r;
}

// (s, e) += a * b exactly up to the tail: a, b double-single reals.
__device__ __forceinline__ void dsfma(float& s, float& e, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float pe = fmaf(ah, bh, -p);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  const float t = s + p;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (p - bp);
  s = t;
  e += err + pe;
}

struct acc2 {  // complex accumulator: (re head, re tail, im head, im tail)
  float rs, re, is, ie;
};

// acc += a * b
__device__ __forceinline__ void cmac(acc2& c, const f2c& a, const f2c& b) {
  dsfma(c.rs, c.re, a.rh, a.rl, b.rh, b.rl);
  dsfma(c.rs, c.re, -a.ih, -a.il, b.ih, b.il);
  dsfma(c.is, c.ie, a.rh, a.rl, b.ih, b.il);
  dsfma(c.is, c.ie, a.ih, a.il, b.rh, b.rl);
}

__device__ __forceinline__ double2 acc_value(const acc2& c) {
  return make_double2((double)c.rs + (double)c.re, (double)c.is + (double)c.ie);
}

__device__ __forceinline__ long long job_offset(const GramBatch& batch, int q, int nchunks) {
  long long off = 0;
  for (int p = 0; p < q; ++p) off += (long long)nchunks * batch.job[p].nx * batch.job[p].ny;
  return off;
}

template <int TI, int TJ, bool BILINEAR>
__global__ void __launch_bounds__(256) gram_df_kernel(const __grid_constant__ GramBatch batch, int N,
                                                      const double* __restrict__ w, int rows_per_chunk,
                                                      double2* __restrict__ work) {
  constexpr int RI = TI / 16, RJ = TJ / 16;
  __shared__ f2c sx[kRowStage][TI];
  __shared__ f2c sy[kRowStage][TJ];
  const GramJob& J = batch.job[blockIdx.z];
  const int tiles_j = (J.ny + TJ - 1) / TJ;
  const int tiles_i = (J.nx + TI - 1) / TI;
  if ((int)blockIdx.y >= tiles_i * tiles_j) return;
  const int ti0 = (blockIdx.y / tiles_j) * TI;
  const int tj0 = (blockIdx.y % tiles_j) * TJ;
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(N, r0 + rows_per_chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  acc2 acc[RI][RJ];
#pragma unroll
  for (int a = 0; a < RI; ++a)
#pragma unroll
    for (int b = 0; b < RJ; ++b) acc[a][b] = acc2{0.f, 0.f, 0.f, 0.f};

  for (int rb = r0; rb < r1; rb += kRowStage) {
    for (int e = threadIdx.x; e < kRowStage * TI; e += 256) {
      const int rr = e / TI, cc = e % TI;
      const int r = rb + rr, col = ti0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (r < r1 && col < J.nx) {
        v = __ldg(J.X + (long long)r * J.ldx + col);
        if (!BILINEAR) v.y = -v.y;
      }
      sx[rr][cc] = split(v);
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
      sy[rr][cc] = split(v);
    }
    __syncthreads();
#pragma unroll 2
    for (int rr = 0; rr < kRowStage; ++rr) {
      f2c xa[RI], yb[RJ];
#pragma unroll
      for (int a = 0; a < RI; ++a) xa[a] = sx[rr][ty * RI + a];
#pragma unroll
      for (int b = 0; b < RJ; ++b) yb[b] = sy[rr][tx * RJ + b];
#pragma unroll
      for (int a = 0; a < RI; ++a)
#pragma unroll
        for (int b = 0; b < RJ; ++b) cmac(acc[a][b], xa[a], yb[b]);
    }
    __syncthreads();
  }
  double2* out = work + job_offset(batch, blockIdx.z, gridDim.x) + (long long)blockIdx.x * J.nx * J.ny;
#pragma unroll
  for (int a = 0; a < RI; ++a) {
    const int i = ti0 + ty * RI + a;
    if (i >= J.nx) continue;
#pragma unroll
    for (int b = 0; b < RJ; ++b) {
      const int j = tj0 + tx * RJ + b;
      if (j < J.ny) out[(long long)i * J.ny + j] = acc_value(acc[a][b]);
    }
  }
}

__global__ void gram_df_reduce_kernel(const __grid_constant__ GramBatch batch, int nchunks,
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

template <int RN, int TJ>
__global__ void __launch_bounds__(256) rowgemm_df_kernel(const __grid_constant__ RowGemmBatch batch, int N) {
  constexpr int KC = 16;
  constexpr int RR = RN / 16, RJ = TJ / 16;
  __shared__ f2c sa[RN][KC + 1];
  __shared__ f2c sb[KC][TJ];
  const RowGemmJob& J = batch.job[blockIdx.z];
  const int c0 = blockIdx.y * TJ;
  if (c0 >= J.ncols) return;
  const int r0 = blockIdx.x * RN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  acc2 acc[RR][RJ];
#pragma unroll
  for (int a = 0; a < RR; ++a)
#pragma unroll
    for (int b = 0; b < RJ; ++b) acc[a][b] = acc2{0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < J.k; k0 += KC) {
    for (int e = threadIdx.x; e < RN * KC; e += 256) {
      const int rr = e / KC, kk = e % KC;
      const int r = r0 + rr, k = k0 + kk;
      sa[rr][kk] = split((r < N && k < J.k) ? __ldg(J.X + (long long)r * J.ldx + k) : make_double2(0.0, 0.0));
    }
    for (int e = threadIdx.x; e < KC * TJ; e += 256) {
      const int kk = e / TJ, cc = e % TJ;
      const int k = k0 + kk, c = c0 + cc;
      sb[kk][cc] = split((k < J.k && c < J.ncols) ? __ldg(J.M + (long long)k * J.ldm + c) : make_double2(0.0, 0.0));
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      f2c xa[RR], yb[RJ];
#pragma unroll
      for (int a = 0; a < RR; ++a) xa[a] = sa[ty * RR + a][kk];
#pragma unroll
      for (int b = 0; b < RJ; ++b) yb[b] = sb[kk][tx * RJ + b];
#pragma unroll
      for (int a = 0; a < RR; ++a)
#pragma unroll
        for (int b = 0; b < RJ; ++b) cmac(acc[a][b], xa[a], yb[b]);
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
      double2 v = cscale(acc_value(acc[a][b]), J.alpha);
      if (J.Yin) {
        const double2 y = J.Yin[(long long)r * J.ldy + c];
        v.x = fma(J.beta, y.x, v.x);
        v.y = fma(J.beta, y.y, v.y);
      }
      J.Out[(long long)r * J.ldo + c] = v;
    }
  }
}

}  // namespace

void launch_gram_df(const GramBatch& b, int N, const double* w, int bilinear, double2* work, size_t work_elems,
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
  // chunks of at most 1024 rows keep the tails of the FP32 sums small; FP64 across chunks
  int nchunks = (4 * 152 + tiles * b.n - 1) / (tiles * b.n);
  const int min_chunks = (N + 1023) / 1024;
  if (nchunks < min_chunks) nchunks = min_chunks;
  const int max_by_rows = (N + 255) / 256;
  if (nchunks > max_by_rows) nchunks = max_by_rows;
  if (nchunks < 1) nchunks = 1;
  while (nchunks > 1 && (size_t)nchunks * per_chunk > work_elems) --nchunks;
  if ((size_t)nchunks * per_chunk > work_elems) throw Error{SWI_ENOMEM, "gram workspace too small"};
  int rows_per_chunk = (N + nchunks - 1) / nchunks;
  rows_per_chunk = (rows_per_chunk + kRowStage - 1) / kRowStage * kRowStage;
  nchunks = (N + rows_per_chunk - 1) / rows_per_chunk;
  dim3 grid(nchunks, tiles, b.n);
  if (narrow) {
    if (bilinear)
      gram_df_kernel<64, 16, true><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
    else
      gram_df_kernel<64, 16, false><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
  } else {
    if (bilinear)
      gram_df_kernel<32, 32, true><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
    else
      gram_df_kernel<32, 32, false><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
  }
  SWI_CHECK_LAUNCH();
  const int maxe = maxnx * maxny;
  gram_df_reduce_kernel<<<dim3((maxe + 255) / 256, b.n), 256, 0, s>>>(b, nchunks, work);
  SWI_CHECK_LAUNCH();
  if (launches) *launches += 2;
}

void launch_rowgemm_df(const RowGemmBatch& b, int N, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  int maxc = 0;
  for (int q = 0; q < b.n; ++q) maxc = b.job[q].ncols > maxc ? b.job[q].ncols : maxc;
  if (maxc <= 16) {
    dim3 grid((N + 63) / 64, 1, b.n);
    rowgemm_df_kernel<64, 16><<<grid, 256, 0, s>>>(b, N);
  } else {
    dim3 grid((N + 31) / 32, (maxc + 31) / 32, b.n);
    rowgemm_df_kernel<32, 32><<<grid, 256, 0, s>>>(b, N);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
