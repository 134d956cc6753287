// Projected eigenproblem of a thick restart in double-single arithmetic.
//
// Same steps as the FP64 kernel in dense.cu -- Householder reduction to
// Hessenberg form, single-shift QR with Wilkinson shifts to the complex Schur
// form H = Z T Z^H, selection of the kept Ritz values (smallest |theta|, the
// 'SM' rule on the shifted operator of Eq. 3), reordering by adjacent Givens
// swaps, eigenvectors of the kept block and residual estimates ||B Z_k s|| --
// but every operation runs on the FP32 pipes in double-single form (about 48
// significant bits).  The chase is a long chain of dependent operations; on
// GB300 a dependent FP64 operation costs about as much as a whole warp's FP64
// issue, so this form is several times faster while keeping Z unitary and
// Z^H H Z = T to ~1e-14 relative.  Inputs and outputs stay FP64.
#include <cfloat>

#include "ds.cuh"
#include "swi_internal.cuh"

namespace swi {

namespace {

using namespace ds;

constexpr int kThreads = 256;
// deflation and tie tolerances relative to double-single precision
constexpr float kDeflate = 4e-15f;

struct RotD {
  df c;
  dc s;
};

__device__ __forceinline__ df dfz() { return df{0.f, 0.f}; }

// G = [[c, s], [-conj(s), c]], G [x; y] = [r; 0]; inputs scaled by a power of
// two first so the squares stay in float range.
__device__ RotD make_rot_ds(dc x, dc y) {
  RotD g;
  float mx = fmaxf(fmaxf(fabsf(x.re.h), fabsf(x.im.h)), fmaxf(fabsf(y.re.h), fabsf(y.im.h)));
  if (mx == 0.f) {
    g.c = df{1.f, 0.f};
    g.s = czero();
    return g;
  }
  int e;
  frexpf(mx, &e);
  x = dc{ldexp_(x.re, -e), ldexp_(x.im, -e)};
  y = dc{ldexp_(y.re, -e), ldexp_(y.im, -e)};
  const df ax2 = cabs2(x), ay2 = cabs2(y);
  if (ay2.h == 0.f) {
    g.c = df{1.f, 0.f};
    g.s = czero();
  } else if (ax2.h == 0.f) {
    const df t = rsqrt(ay2);
    g.c = dfz();
    g.s = dc{mul(y.re, t), neg(mul(y.im, t))};
  } else {
    const df t = rsqrt(mul(ax2, add(ax2, ay2)));  // 1 / (|x| r)
    g.c = mul(ax2, t);
    const dc xcy = dc{add(mul(x.re, y.re), mul(x.im, y.im)), sub(mul(x.im, y.re), mul(x.re, y.im))};
    g.s = cscale(xcy, t);
  }
  return g;
}

// rows (h1, h2) <- (c h1 + s h2, c h2 - conj(s) h1)
__device__ __forceinline__ void rot_rows(dc& h1, dc& h2, const RotD& g) {
  const dc a = h1, b = h2;
  h1 = cadd(cscale(a, g.c), cmul(g.s, b));
  h2 = csub(cscale(b, g.c), cmulc_l(g.s, a));
}
// cols (a1, a2) <- (c a1 + conj(s) a2, c a2 - s a1)
__device__ __forceinline__ void rot_cols(dc& a1, dc& a2, const RotD& g) {
  const dc a = a1, b = a2;
  a1 = cadd(cscale(a, g.c), cmulc_l(g.s, b));
  a2 = csub(cscale(b, g.c), cmul(g.s, a));
}

__device__ float block_reduce_sumf(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;
}

// double-single reduction (sum of df over the block)
__device__ df block_reduce_df(df v, df* red) {
  for (int o = 16; o > 0; o >>= 1) {
    df u;
    u.h = __shfl_xor_sync(0xffffffffu, v.h, o);
    u.l = __shfl_xor_sync(0xffffffffu, v.l, o);
    v = add(v, u);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  df s = dfz();
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = add(s, red[q]);
  __syncthreads();
  return s;
}

#define HD(i, j) Hd[(long long)(i) * ld + (j)]
#define ZD(i, j) Zd[(long long)(i) * ld + (j)]

__global__ void __launch_bounds__(kThreads) schur_ds_kernel(const __grid_constant__ SchurBatch batch) {
  const SchurJob& J = batch.job[blockIdx.x];
  dc* Hd = reinterpret_cast<dc*>(J.Hw);
  dc* Zd = reinterpret_cast<dc*>(J.Zw);
  const int m = J.m, ld = J.ld;
  __shared__ df red[kThreads / 32];
  __shared__ dc sv[1024];
  __shared__ RotD srot;
  __shared__ int s_flag;
  __shared__ int s_sel[1024];
  const int tid = threadIdx.x;
  if (m > 1024) {
    if (tid == 0) J.ordinfo[2] = 3;
    return;
  }
  // load H, Z = I
  for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    HD(i, j) = cfrom(J.H[(long long)i * ld + j]);
    ZD(i, j) = dc{df{i == j ? 1.f : 0.f, 0.f}, dfz()};
  }
  __syncthreads();

  // ---------------- Householder reduction to Hessenberg form
  for (int c = 0; c + 2 < m; ++c) {
    df part = dfz();
    for (int i = c + 2 + tid; i < m; i += blockDim.x) part = add(part, cabs2(HD(i, c)));
    const df tail2 = block_reduce_df(part, red);
    if (tail2.h == 0.f) continue;
    const dc x0 = HD(c + 1, c);
    const df ax02 = cabs2(x0);
    const df xn = sqrt_(add(tail2, ax02));
    dc ph;
    if (ax02.h > 0.f) {
      const df r = rsqrt(ax02);
      ph = dc{mul(x0.re, r), mul(x0.im, r)};
    } else {
      ph = dc{df{1.f, 0.f}, dfz()};
    }
    const dc alpha = dc{neg(mul(ph.re, xn)), neg(mul(ph.im, xn))};
    for (int i = c + 1 + tid; i < m; i += blockDim.x) sv[i] = (i == c + 1) ? csub(x0, alpha) : HD(i, c);
    __syncthreads();
    const df vn2 = add(cabs2(csub(x0, alpha)), tail2);
    const df tau = div(df{2.f, 0.f}, vn2);
    for (int j = c + 1 + tid; j < m; j += blockDim.x) {
      dc w = czero();
      for (int i = c + 1; i < m; ++i) w = cadd(w, cmulc_l(sv[i], HD(i, j)));
      w = cscale(w, tau);
      for (int i = c + 1; i < m; ++i) HD(i, j) = csub(HD(i, j), cmul(sv[i], w));
    }
    __syncthreads();
    for (int i = c + 1 + tid; i < m; i += blockDim.x) HD(i, c) = (i == c + 1) ? alpha : czero();
    for (int i = tid; i < m; i += blockDim.x) {
      dc u = czero();
      for (int j = c + 1; j < m; ++j) u = cadd(u, cmul(HD(i, j), sv[j]));
      u = cscale(u, tau);
      for (int j = c + 1; j < m; ++j) HD(i, j) = csub(HD(i, j), cmul(u, cconj(sv[j])));
      dc uz = czero();
      for (int j = c + 1; j < m; ++j) uz = cadd(uz, cmul(ZD(i, j), sv[j]));
      uz = cscale(uz, tau);
      for (int j = c + 1; j < m; ++j) ZD(i, j) = csub(ZD(i, j), cmul(uz, cconj(sv[j])));
    }
    __syncthreads();
  }

  // ---------------- single-shift QR to the complex Schur form (full T and Z)
  int status = 0;
  long long n_upd = 0;  // counted by thread 0
  {
    int ihi = m - 1, its = 0, total_its = 0;
    const int max_its = 60 * m + 100;
    while (ihi > 0) {
      int l = ihi;
      while (l > 0) {
        float tst = cabs1f(HD(l - 1, l - 1)) + cabs1f(HD(l, l));
        if (tst == 0.f) tst = 1.f;
        if (cabs1f(HD(l, l - 1)) <= kDeflate * tst) break;
        --l;
      }
      __syncthreads();
      if (l > 0 && tid == 0) HD(l, l - 1) = czero();
      if (l == ihi) {
        __syncthreads();
        --ihi;
        its = 0;
        continue;
      }
      ++its;
      if (++total_its > max_its) {
        status = 1;
        break;
      }
      dc mu;
      if (its % 10 == 0) {
        const dc hs = HD(ihi, ihi - 1);
        mu = cadd(HD(ihi, ihi), dc{df{0.75f * fabsf(approx(hs.re)), 0.f}, dfz()});
      } else {
        // Wilkinson shift, once per iteration, evaluated in FP64
        const double2 a = cto(HD(ihi - 1, ihi - 1)), bq = cto(HD(ihi - 1, ihi)), cq = cto(HD(ihi, ihi - 1)),
                      d = cto(HD(ihi, ihi));
        const double2 tr2 = swi::cscale(swi::csub(a, d), 0.5);
        const double2 bc = swi::cmul(bq, cq);
        const double2 disc = csqrt_p(swi::cadd(swi::cmul(tr2, tr2), bc));
        const double2 r1 = swi::cadd(tr2, disc), r2 = swi::csub(tr2, disc);
        const double2 den = swi::cabs(r1) >= swi::cabs(r2) ? r1 : r2;
        const double2 m64 = swi::cabs(den) > 0.0 ? swi::csub(d, swi::cdiv(bc, den)) : d;
        mu = cfrom(m64);
      }
      __syncthreads();
      for (int k = l; k < ihi; ++k) {
        if (tid == 0) {
          dc x, y;
          if (k == l) {
            x = csub(HD(l, l), mu);
            y = HD(l + 1, l);
          } else {
            x = HD(k, k - 1);
            y = HD(k + 1, k - 1);
          }
          srot = make_rot_ds(x, y);
          n_upd += (m - ((k == l) ? l : k - 1)) + (min(k + 2, ihi) + 1) + m;
        }
        __syncthreads();
        const RotD g = srot;
        const int c0 = (k == l) ? l : k - 1;
        const int r1 = min(k + 2, ihi) + 1;
        for (int j = c0 + tid; j < m; j += blockDim.x) {
          if (j == k || j == k + 1) continue;
          rot_rows(HD(k, j), HD(k + 1, j), g);
          if (j == k - 1) HD(k + 1, k - 1) = czero();
        }
        for (int i = tid; i < r1; i += blockDim.x) {
          if (i == k || i == k + 1) continue;
          rot_cols(HD(i, k), HD(i, k + 1), g);
        }
        for (int i = tid; i < m; i += blockDim.x) rot_cols(ZD(i, k), ZD(i, k + 1), g);
        if (tid == 0) {
          dc a = HD(k, k), b = HD(k, k + 1), cc = HD(k + 1, k), d = HD(k + 1, k + 1);
          rot_rows(a, cc, g);
          rot_rows(b, d, g);
          rot_cols(a, b, g);
          rot_cols(cc, d, g);
          HD(k, k) = a;
          HD(k, k + 1) = b;
          HD(k + 1, k) = cc;
          HD(k + 1, k + 1) = d;
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    if (i > j) HD(i, j) = czero();
  }
  __syncthreads();

  // ---------------- selection: rank by (|theta|, Re, Im, index) in FP64 of the diagonal
  for (int i = tid; i < m; i += blockDim.x) {
    const double2 ti = cto(HD(i, i));
    const double ai = hypot(ti.x, ti.y);
    int rank = 0;
    for (int q = 0; q < m; ++q) {
      if (q == i) continue;
      const double2 tq = cto(HD(q, q));
      const double aq = hypot(tq.x, tq.y);
      const bool less = aq < ai || (aq == ai && (tq.x < ti.x || (tq.x == ti.x && (tq.y < ti.y || (tq.y == ti.y && q < i)))));
      rank += less ? 1 : 0;
    }
    s_sel[i] = rank;
  }
  __syncthreads();
  if (tid == 0) {
    int k = J.keep < m ? J.keep : m;
    while (k < m - 1 && k < J.kmax) {
      double a_in = -1.0, a_out = -1.0;
      for (int q = 0; q < m; ++q) {
        const double2 tq = cto(HD(q, q));
        if (s_sel[q] == k - 1) a_in = hypot(tq.x, tq.y);
        if (s_sel[q] == k) a_out = hypot(tq.x, tq.y);
      }
      if (a_out - a_in <= 1e-10 * fmax(1.0, a_in)) ++k;
      else break;
    }
    s_flag = k;
  }
  __syncthreads();
  const int kk = s_flag;
  for (int i = tid; i < m; i += blockDim.x) s_sel[i] = (s_sel[i] < kk) ? 1 : 0;
  __syncthreads();
  {
    int ks = 0;
    for (int pos = 0; pos < m; ++pos) {
      if (!s_sel[pos]) continue;
      for (int q = pos - 1; q >= ks; --q) {
        if (tid == 0) {
          srot = make_rot_ds(HD(q, q + 1), csub(HD(q + 1, q + 1), HD(q, q)));
          n_upd += (m - q - 2) + q + m;
        }
        __syncthreads();
        const RotD g = srot;
        for (int j = q + 2 + tid; j < m; j += blockDim.x) rot_rows(HD(q, j), HD(q + 1, j), g);
        for (int i = tid; i < q; i += blockDim.x) rot_cols(HD(i, q), HD(i, q + 1), g);
        for (int i = tid; i < m; i += blockDim.x) rot_cols(ZD(i, q), ZD(i, q + 1), g);
        if (tid == 0) {
          const dc t11 = HD(q, q);
          HD(q, q) = HD(q + 1, q + 1);
          HD(q + 1, q + 1) = t11;
          HD(q + 1, q) = czero();
          const int f = s_sel[q];
          s_sel[q] = s_sel[q + 1];
          s_sel[q + 1] = f;
        }
        __syncthreads();
      }
      ++ks;
    }
  }
  __syncthreads();

  // ---------------- outputs in FP64: T into H, Z, theta, then S, Bz, residuals
  for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    J.H[(long long)i * ld + j] = cto(HD(i, j));
    J.Z[(long long)i * ld + j] = cto(ZD(i, j));
  }
  __syncthreads();
  double2* H = J.H;
  double2* Z = J.Z;
  for (int i = tid; i < m; i += blockDim.x) J.theta[i] = H[(long long)i * ld + i];
  for (int e = tid; e < J.b * kk; e += blockDim.x) {
    const int r = e / kk, l = e % kk;
    double2 bz = make_double2(0.0, 0.0);
    for (int q = 0; q < m; ++q) cfma(bz, J.B[(long long)r * ld + q], Z[(long long)q * ld + l]);
    J.Bz[(long long)r * ld + l] = bz;
  }
  __syncthreads();
  // eigenvectors of T[0:kk, 0:kk] (column i of S), unit 2-norm, FP64 back substitution
  for (int i = tid; i < kk; i += blockDim.x) {
    const double2 lam = H[(long long)i * ld + i];
    const double smin = fmax(1e-14 * swi::cabs(lam), 1e-290);
    double2* s = J.S;
    for (int l = i + 1; l < kk; ++l) s[(long long)l * ld + i] = make_double2(0.0, 0.0);
    s[(long long)i * ld + i] = make_double2(1.0, 0.0);
    for (int jj = i - 1; jj >= 0; --jj) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = jj + 1; l <= i; ++l) cfma(acc, H[(long long)jj * ld + l], s[(long long)l * ld + i]);
      double2 den = swi::csub(H[(long long)jj * ld + jj], lam);
      if (swi::cabs(den) < smin) den = make_double2(smin, 0.0);
      s[(long long)jj * ld + i] = swi::cdiv(make_double2(-acc.x, -acc.y), den);
    }
    double nrm = 0.0;
    for (int l = 0; l <= i; ++l) nrm += swi::cabs2(s[(long long)l * ld + i]);
    nrm = 1.0 / sqrt(nrm);
    for (int l = 0; l <= i; ++l) s[(long long)l * ld + i] = swi::cscale(s[(long long)l * ld + i], nrm);
  }
  __syncthreads();
  for (int i = tid; i < kk; i += blockDim.x) {
    double r2 = 0.0;
    for (int r = 0; r < J.b; ++r) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l <= i; ++l) cfma(acc, J.Bz[(long long)r * ld + l], J.S[(long long)l * ld + i]);
      r2 += swi::cabs2(acc);
    }
    J.resid[i] = sqrt(r2);
  }
  __syncthreads();
  if (tid == 0) {
    int nconv = 0;
    for (int i = 0; i < kk; ++i) {
      const double ai = swi::cabs(H[(long long)i * ld + i]);
      int rank = 0;
      for (int q = 0; q < kk; ++q) {
        const double aq = swi::cabs(H[(long long)q * ld + q]);
        if (aq < ai || (aq == ai && q < i)) ++rank;
      }
      if (rank < J.nwant && J.resid[i] <= J.tol_abs) ++nconv;
    }
    J.ordinfo[0] = kk;
    J.ordinfo[1] = nconv;
    J.ordinfo[2] = status;
    J.ordinfo[3] = (int)(n_upd >> 10);  // Givens pair updates / 1024 (work accounting)
  }
}

#undef HD
#undef ZD

}  // namespace

void launch_schur_ds_batch(const SchurBatch& b, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  schur_ds_kernel<<<b.n, kThreads, 0, s>>>(b);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
