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
#include <atomic>
#include <algorithm>

#include "ds.cuh"
#include "swi_internal.cuh"

namespace swi {

namespace {

constexpr int kRowStage = 16;

struct f2c {  // complex double-single: re = (rh, rl), im = (ih, il)
  float rh, rl, ih, il;
};

__device__ __forceinline__ void split1(double x, float& hi, float& lo) { ds::split_bits(x, hi, lo); }

__device__ __forceinline__ f2c split(double2 v) {
  f2c r;
  split1(v.x, r.rh, r.rl);
  split1(v.y, r.ih, r.il);
  return r;
}

__device__ __forceinline__ void dsfma(float& s, float& e, float ah, float al, float bh, float bl) {
  ds::fma_acc(s, e, ah, al, bh, bl);
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

// ---------------------------------------------------------------------------
// C = X^H Y on the tensor cores, exactly to ~2^-48: each FP64 operand is cut
// into seven 7-bit digits relative to the largest exponent of its column over a
// 32-row chunk (an error-free split: x = sign * 2^(e-49) * sum_k D_k 2^(7(6-k))),
// the digit products are formed by bf16 MMAs (digits <= 128 are exact in bf16)
// with FP32 accumulation, which stays exact because every accumulator sums at
// most 7 digit pairs x 2 products x 32 rows of values < 2^14 (< 2^23), and the
// 34 digit pairs s + u <= 7 (the rest weigh < 2^-55 of the chunk maxima) are
// combined in double-single arithmetic.  (The splitting-and-exact-products scheme is the
// one of Ozaki, Ogita, Oishi and Rump for accurate matrix products.)
// Tile: 64 columns of X x 16 columns of Y per CTA of 8 warps; warp (wm, wn)
// owns the 16 x 8 block (16 wm, 8 wn).
namespace oz {
constexpr int kTI = 64, kTJ = 16, kKC = 32, kDig = 7;  // digit pairs kept: s + u <= 7
constexpr int kRow = kKC + 8;  // padded row of a digit plane (bf16): conflict-free fragment loads
constexpr int kWords = kRow / 2;
constexpr size_t kSmem = sizeof(unsigned) * (size_t)kDig * 2 * (kTI + kTJ) * kWords;

// F = round(|x| 2^(1071 - emax)) < 2^49 (+1 at the top edge), emax the largest
// exponent field of the column; 0 for zeros and magnitudes below 2^-60 of it
__device__ __forceinline__ unsigned long long fixed49(double x, int emax, unsigned& sign16) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  sign16 = (unsigned)(b >> 48) & 0x8000u;
  const int sh = emax - e + 4;
  if (e == 0 || sh >= 60) return 0ull;
  const unsigned long long m53 = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  return (m53 + (1ull << (sh - 1))) >> sh;
}

// the float value of a digit d <= 128 (exact), from the 2^23 offset trick
__device__ __forceinline__ unsigned digit_float(unsigned d) {
  return __float_as_uint(__uint_as_float(0x4B000000u | d) - 8388608.0f);
}

// seven 7-bit digits of two reals (rows r, r+1 of one column), packed as bf16
// pairs: word k holds digit k of x0 in its low half and of x1 in its high half
__device__ __forceinline__ void digits2(double x0, double x1, int emax, unsigned (&w)[kDig]) {
  unsigned s0, s1;
  const unsigned long long F0 = fixed49(x0, emax, s0), F1 = fixed49(x1, emax, s1);
  const unsigned a0 = (unsigned)(F0 >> 21), b0 = (unsigned)F0 & 0x1FFFFFu;
  const unsigned a1 = (unsigned)(F1 >> 21), b1 = (unsigned)F1 & 0x1FFFFFu;
  const unsigned sg = s0 | (s1 << 16);
  const unsigned d0[kDig] = {a0 >> 21, (a0 >> 14) & 127u, (a0 >> 7) & 127u, a0 & 127u, b0 >> 14, (b0 >> 7) & 127u,
                             b0 & 127u};
  const unsigned d1[kDig] = {a1 >> 21, (a1 >> 14) & 127u, (a1 >> 7) & 127u, a1 & 127u, b1 >> 14, (b1 >> 7) & 127u,
                             b1 & 127u};
#pragma unroll
  for (int k = 0; k < kDig; ++k) w[k] = __byte_perm(digit_float(d0[k]), digit_float(d1[k]), 0x7632) | sg;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int efield(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
}
// The digit-pair products of one 32-row chunk on the tensor cores, in two
// passes over the pair weights d = s + u (7..4, then 3..0: fewer live
// accumulators, and the double-single sums take the small terms first), then
// the exact integer sums scaled into the warp's double-single accumulators.
// A digit planes: [kDig][2][64][kWords] (row m, k pairs), B: [kDig][2][16][kWords]
// (column n, k pairs); ema / emb: exponent fields of the A rows / B columns.
__device__ __forceinline__ void mma_flush(const unsigned* adig, const unsigned* bdig, const int* ema,
                                          const int* emb, int wm, int wn, int g, int t, float (&ohi)[2][4],
                                          float (&olo)[2][4]) {
    // 3) digit-pair products on the tensor cores, in two passes over the pair
  // weights d = s + u (7..4, then 3..0: fewer live accumulators, and the
  // double-single sums take the small terms first)
  const int i_a = 16 * wm + g, i_b = i_a + 8, j_a = 8 * wn + 2 * t, j_b = j_a + 1;
  const int es[4] = {ema[i_a] + emb[j_a], ema[i_a] + emb[j_b], ema[i_b] + emb[j_a], ema[i_b] + emb[j_b]};
#pragma unroll
  for (int half = 1; half >= 0; --half) {
    const int dlo = 4 * half;
    float acc[4][2][4];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[d][c][e] = 0.f;
#pragma unroll 1  // unrolled, the fragment loads of both k steps stay live and spill at 128 registers
    for (int ks = 0; ks < kKC / 16; ++ks) {
      const int kw = ks * 8 + t;  // word of k = 16 ks + 2 t
      unsigned bre[kDig][2], bim[kDig][2];
#pragma unroll
      for (int d = 0; d < kDig; ++d) {
        const unsigned* br = bdig + ((d * 2 + 0) * kTJ + 8 * wn + g) * kWords + kw;
        const unsigned* bi = bdig + ((d * 2 + 1) * kTJ + 8 * wn + g) * kWords + kw;
        bre[d][0] = br[0];
        bre[d][1] = br[4];
        bim[d][0] = bi[0];
        bim[d][1] = bi[4];
      }
#pragma unroll
      for (int s = 0; s < kDig; ++s) {
        if (s > dlo + 3) continue;
        unsigned are[4], aim[4], ain[4];
        const unsigned* ar = adig + ((s * 2 + 0) * kTI + 16 * wm + g) * kWords + kw;
        const unsigned* ai = adig + ((s * 2 + 1) * kTI + 16 * wm + g) * kWords + kw;
        are[0] = ar[0];
        are[1] = ar[8 * kWords];
        are[2] = ar[4];
        are[3] = ar[8 * kWords + 4];
        aim[0] = ai[0];
        aim[1] = ai[8 * kWords];
        aim[2] = ai[4];
        aim[3] = ai[8 * kWords + 4];
#pragma unroll
        for (int q = 0; q < 4; ++q) ain[q] = aim[q] ^ 0x80008000u;
        // Re += a c - b d, Im += a d + b c; consecutive MMAs go to different accumulators
#pragma unroll
        for (int u = 0; u < kDig; ++u)
          if (s + u >= dlo && s + u < dlo + 4) mma_bf16(acc[s + u - dlo][0], are, bre[u][0], bre[u][1]);
#pragma unroll
        for (int u = 0; u < kDig; ++u)
          if (s + u >= dlo && s + u < dlo + 4) mma_bf16(acc[s + u - dlo][1], are, bim[u][0], bim[u][1]);
#pragma unroll
        for (int u = 0; u < kDig; ++u)
          if (s + u >= dlo && s + u < dlo + 4) mma_bf16(acc[s + u - dlo][0], ain, bim[u][0], bim[u][1]);
#pragma unroll
        for (int u = 0; u < kDig; ++u)
          if (s + u >= dlo && s + u < dlo + 4) mma_bf16(acc[s + u - dlo][1], aim, bre[u][0], bre[u][1]);
      }
    }
    // 4) exact integer sums -> scaled, accumulated in double-single
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int dd = 3; dd >= 0; --dd) {
        // weight 2^(ex + ey - 14 - 7d), ex = emax - 1022, as a float built from its exponent
        // field (weights below 2^-126 of the unit are dropped: beyond double-single reach)
        const int ex2 = es[e] - 2058 - 7 * (dlo + dd);
        const float wgt = ex2 >= -126 ? __int_as_float((min(ex2, 127) + 127) << 23) : 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float v = acc[dd][c][e] * wgt;
          const float s1 = ohi[c][e] + v;
          const float bb = s1 - ohi[c][e];
          olo[c][e] += (ohi[c][e] - (s1 - bb)) + (v - bb);
          ohi[c][e] = s1;
        }
      }
  }
}
}  // namespace oz

__global__ void __launch_bounds__(256, 2) gram_oz_kernel(const __grid_constant__ GramBatch batch, int N,
                                                      int rows_per_chunk, double2* __restrict__ work) {
  using namespace oz;
  extern __shared__ __align__(16) unsigned oz_smem[];
  unsigned* adig = oz_smem;                                  // [kDig][2][kTI][kWords]
  unsigned* bdig = oz_smem + (size_t)kDig * 2 * kTI * kWords;  // [kDig][2][kTJ][kWords]
  __shared__ int emx[kTI], emy[kTJ];
  const GramJob& J = batch.job[blockIdx.z];
  const int tiles_i = (J.nx + kTI - 1) / kTI;
  if ((int)blockIdx.y >= tiles_i) return;
  const int ti0 = blockIdx.y * kTI;
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(N, r0 + rows_per_chunk);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;
  const int g = lane >> 2, t = lane & 3;
  // loader roles: X column li (of the tile), rows 2 lr, 2 lr + 1 (+8 k); Y column yj, rows 2 yr, 2 yr + 1.
  // The four lanes of one column are adjacent: their digit-plane stores fall in
  // distinct banks, and the column's exponent is combined by shuffles.
  const int li = tid >> 2, lr = tid & 3;
  const int yj = tid % kTJ, yr = tid / kTJ;   // yr in 0..15
  float ohi[2][4], olo[2][4];  // double-single running sums (re, im) of the warp's C fragment
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) ohi[c][e] = olo[c][e] = 0.f;

  // operands of one chunk into registers (X conjugated)
  auto load = [&](int rb, double2 (&xv)[4][2], double2 (&yv)[2]) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = rb + 2 * lr + h + 8 * k, col = ti0 + li;
        double2 v = make_double2(0.0, 0.0);
        if (r < r1 && col < J.nx) {
          v = __ldg(J.X + (long long)r * J.ldx + col);
          v.y = __longlong_as_double(__double_as_longlong(v.y) ^ (long long)0x8000000000000000ull);  // conj, no FP64 op
        }
        xv[k][h] = v;
      }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = rb + 2 * yr + h;
      double2 v = make_double2(0.0, 0.0);
      if (r < r1 && yj < J.ny) v = __ldg(J.Y + (long long)r * J.ldy + yj);
      yv[h] = v;
    }
  };
  double2 xv[4][2], yv[2];
  for (int rb = r0; rb < r1; rb += kKC) {
    load(rb, xv, yv);
    // 1) exponent fields of the chunk's columns into shared memory
    int ex_loc = 0, ey_loc = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) ex_loc = max(ex_loc, max(efield(xv[k][h].x), efield(xv[k][h].y)));
#pragma unroll
    for (int h = 0; h < 2; ++h) ey_loc = max(ey_loc, max(efield(yv[h].x), efield(yv[h].y)));
    ex_loc = max(ex_loc, __shfl_xor_sync(0xffffffffu, ex_loc, 1));
    ex_loc = max(ex_loc, __shfl_xor_sync(0xffffffffu, ex_loc, 2));
    if (tid < kTJ) emy[tid] = 0;
    __syncthreads();
    if (lr == 0) emx[li] = ex_loc;
    atomicMax(&emy[yj], ey_loc);
    __syncthreads();
    // 2) digit planes: A = conj(X)^T rows li, Y columns yj; rows paired in one 32-bit word
    {
      const int em = emx[li];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        unsigned wr[kDig], wi[kDig];
        digits2(xv[k][0].x, xv[k][1].x, em, wr);
        digits2(xv[k][0].y, xv[k][1].y, em, wi);
        const int w = lr + 4 * k;  // word index of rows (2 lr + 8 k, +1)
#pragma unroll
        for (int d = 0; d < kDig; ++d) {
          adig[((d * 2 + 0) * kTI + li) * kWords + w] = wr[d];
          adig[((d * 2 + 1) * kTI + li) * kWords + w] = wi[d];
        }
      }
      const int fm = emy[yj];
      unsigned wr[kDig], wi[kDig];
      digits2(yv[0].x, yv[1].x, fm, wr);
      digits2(yv[0].y, yv[1].y, fm, wi);
#pragma unroll
      for (int d = 0; d < kDig; ++d) {
        bdig[((d * 2 + 0) * kTJ + yj) * kWords + yr] = wr[d];
        bdig[((d * 2 + 1) * kTJ + yj) * kWords + yr] = wi[d];
      }
    }
    __syncthreads();
    oz::mma_flush(adig, bdig, emx, emy, wm, wn, g, t, ohi, olo);
    __syncthreads();  // digit planes and exponents are rewritten by the next chunk
  }
  // partial sums of this row range -> work[chunk][i][j] (FP64)
  double2* out = work + job_offset(batch, blockIdx.z, gridDim.x) + (long long)blockIdx.x * J.nx * J.ny;
  const int i_a = ti0 + 16 * wm + g, j_a = 8 * wn + 2 * t;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = i_a + ((e & 2) ? 8 : 0), j = j_a + (e & 1);
    if (i < J.nx && j < J.ny)
      out[(long long)i * J.ny + j] = make_double2((double)ohi[0][e] + (double)olo[0][e],
                                                  (double)ohi[1][e] + (double)olo[1][e]);
  }
}

// Out = alpha X M (+ beta Yin) on the tensor cores with the same exact digit
// split, for the wide products of the thick restart (Q Z, M with more than 16
// columns): each digit of X is reused against 16 columns of M.  Exponents: per
// row of X and per column of M over each 32-wide slice of the contraction.
// Tile: 64 rows x 16 columns per CTA of 8 warps.
__global__ void __launch_bounds__(256, 2) rowgemm_oz_kernel(const __grid_constant__ RowGemmBatch batch, int N) {
  using namespace oz;
  extern __shared__ __align__(16) unsigned oz_smem[];
  unsigned* adig = oz_smem;                                    // [kDig][2][64][kWords]
  unsigned* bdig = oz_smem + (size_t)kDig * 2 * kTI * kWords;  // [kDig][2][16][kWords]
  __shared__ int emr[kTI], emc[kTJ];
  const RowGemmJob& J = batch.job[blockIdx.z];
  const int r0 = blockIdx.x * kTI, c0 = blockIdx.y * kTJ;
  if (c0 >= J.ncols) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;
  const int g = lane >> 2, t = lane & 3;
  // loader roles: X row ar with k pairs 2 kq + 8 j (j < 4); M column bc with k pair 2 bk
  const int ar = tid >> 2, kq = tid & 3;
  const int bc = tid % kTJ, bk = tid / kTJ;
  float ohi[2][4], olo[2][4];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) ohi[c][e] = olo[c][e] = 0.f;
  for (int kb = 0; kb < J.k; kb += kKC) {
    double2 xa[4][2], mb[2];
    const int row = r0 + ar;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = kb + 2 * kq + 8 * j + h;
        xa[j][h] = (row < N && k < J.k) ? __ldg(J.X + (long long)row * J.ldx + k) : make_double2(0.0, 0.0);
      }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = kb + 2 * bk + h, col = c0 + bc;
      mb[h] = (k < J.k && col < J.ncols) ? __ldg(J.M + (long long)k * J.ldm + col) : make_double2(0.0, 0.0);
    }
    int ea = 0, eb = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) ea = max(ea, max(efield(xa[j][h].x), efield(xa[j][h].y)));
#pragma unroll
    for (int h = 0; h < 2; ++h) eb = max(eb, max(efield(mb[h].x), efield(mb[h].y)));
    // the four lanes of a row are adjacent: combine them by shuffles
    ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, 1));
    ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, 2));
    if (tid < kTJ) emc[tid] = 0;
    __syncthreads();
    if (kq == 0) emr[ar] = ea;
    atomicMax(&emc[bc], eb);
    __syncthreads();
    {
      const int em = emr[ar];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        unsigned wr[kDig], wi[kDig];
        digits2(xa[j][0].x, xa[j][1].x, em, wr);
        digits2(xa[j][0].y, xa[j][1].y, em, wi);
        const int w = kq + 4 * j;  // word of k = 2 kq + 8 j
#pragma unroll
        for (int d = 0; d < kDig; ++d) {
          adig[((d * 2 + 0) * kTI + ar) * kWords + w] = wr[d];
          adig[((d * 2 + 1) * kTI + ar) * kWords + w] = wi[d];
        }
      }
      const int fm = emc[bc];
      unsigned wr[kDig], wi[kDig];
      digits2(mb[0].x, mb[1].x, fm, wr);
      digits2(mb[0].y, mb[1].y, fm, wi);
#pragma unroll
      for (int d = 0; d < kDig; ++d) {
        bdig[((d * 2 + 0) * kTJ + bc) * kWords + bk] = wr[d];
        bdig[((d * 2 + 1) * kTJ + bc) * kWords + bk] = wi[d];
      }
    }
    __syncthreads();
    mma_flush(adig, bdig, emr, emc, wm, wn, g, t, ohi, olo);
    __syncthreads();
  }
  const int i_a = r0 + 16 * wm + g, j_a = c0 + 8 * wn + 2 * t;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int r = i_a + ((e & 2) ? 8 : 0), c = j_a + (e & 1);
    if (r < N && c < J.ncols) {
      double2 v = make_double2(J.alpha * ((double)ohi[0][e] + (double)olo[0][e]),
                               J.alpha * ((double)ohi[1][e] + (double)olo[1][e]));
      if (J.Yin) {
        const double2 y = J.Yin[(long long)r * J.ldy + c];
        v.x = fma(J.beta, y.x, v.x);
        v.y = fma(J.beta, y.y, v.y);
      }
      J.Out[(long long)r * J.ldo + c] = v;
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

// The dynamic shared-memory limit of a kernel is a per-device setting: set it
// once for each device this process launches on (bit d of `done`; devices
// past 63 set it on every call).
template <class K>
void set_smem_attr_once(K kernel, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  SWI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 64 && ((done.load() >> dev) & 1ull)) return;
  SWI_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  if (dev < 64) done.fetch_or(1ull << dev);
}

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
  // Hermitian Grams against a block of at most 16 columns (the block
  // Gram-Schmidt projections): tensor cores with the exact digit split
  bool tensor = !w && !bilinear && maxny <= 16 && maxnx > 16;
  if (tensor) {
    static std::atomic<unsigned long long> attr{0};  // devices whose attribute is set (solves may run on several host threads)
    set_smem_attr_once(gram_oz_kernel, (int)oz::kSmem, attr);
    const int tiles_i = (maxnx + oz::kTI - 1) / oz::kTI;
    int nch = (32 * 152 + tiles_i * b.n - 1) / (tiles_i * b.n);
    nch = std::max(1, std::min(nch, (N + oz::kKC - 1) / oz::kKC));
    while (nch > 1 && (size_t)nch * per_chunk > work_elems) --nch;
    if ((size_t)nch * per_chunk > work_elems) throw Error{SWI_ENOMEM, "gram workspace too small"};
    int rpc = (N + nch - 1) / nch;
    rpc = (rpc + oz::kKC - 1) / oz::kKC * oz::kKC;
    nch = (N + rpc - 1) / rpc;
    gram_oz_kernel<<<dim3(nch, tiles_i, b.n), 256, oz::kSmem, s>>>(b, N, rpc, work);
    SWI_CHECK_LAUNCH();
    const int maxe = maxnx * maxny;
    gram_df_reduce_kernel<<<dim3((maxe + 255) / 256, b.n), 256, 0, s>>>(b, nch, work);
    SWI_CHECK_LAUNCH();
    if (launches) *launches += 2;
    return;
  }
  // tile shapes: 16 x 16 for the b x b Grams of Cholesky-QR, 64 x 16 for
  // Q^H W with a block of at most 16 columns, 32 x 32 otherwise (128 x 16,
  // eight accumulators per thread, measured slower: fewer resident warps)
  const int shape = (maxny <= 16) ? (maxnx <= 16 ? 0 : 1) : 2;
  const int TI = shape == 0 ? 16 : (shape == 1 ? 64 : 32), TJ = shape == 2 ? 32 : 16;
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
  if (shape == 0) {
    if (bilinear)
      gram_df_kernel<16, 16, true><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
    else
      gram_df_kernel<16, 16, false><<<grid, 256, 0, s>>>(b, N, w, rows_per_chunk, work);
  } else if (shape == 1) {
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
  int maxk = 0;
  for (int q = 0; q < b.n; ++q) maxk = b.job[q].k > maxk ? b.job[q].k : maxk;
  if (maxc <= 16 && maxk <= 32) {
    dim3 grid((N + 63) / 64, 1, b.n);
    rowgemm_df_kernel<64, 16><<<grid, 256, 0, s>>>(b, N);
  } else {
    // long contractions (the Gram-Schmidt update W -= Q C, the restart rotation
    // Q Z): tensor cores with the exact digit split
    static std::atomic<unsigned long long> attr{0};  // devices whose attribute is set (solves may run on several host threads)
    set_smem_attr_once(rowgemm_oz_kernel, (int)oz::kSmem, attr);
    dim3 grid((N + oz::kTI - 1) / oz::kTI, (maxc + oz::kTJ - 1) / oz::kTJ, b.n);
    rowgemm_oz_kernel<<<grid, 256, oz::kSmem, s>>>(b, N);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
