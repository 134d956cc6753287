// Small dense FP64 kernels of the Krylov loop, one CTA per window.
//
// * Cholesky of the b x b Gram matrix and the inverse of its factor
//   (block QR of each new Krylov block by Cholesky-QR).
// * The projected eigenproblem of a thick restart: complex Schur form of the
//   m x m projected matrix H (Householder Hessenberg reduction, then
//   single-shift QR with Wilkinson shifts and deflation), selection of the
//   Ritz values closest to the shift (ARPACK's 'SM' rule on the shifted
//   operator of Eq. 3), reordering of the selected ones to the leading block,
//   Ritz vectors of the leading block and their residual estimates
//   ||B Z_k s|| from the Krylov relation A Q = Q H + V B.
//
// All matrices live in global memory (they are L1/L2 resident); every loop is
// bounded and a failure is reported through a status word, never by trapping.
#include "swi_internal.cuh"

#include <cfloat>

namespace swi {

namespace {

constexpr int kDenseThreads = 256;

__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }

// --------------------------------------------------------------------------- Cholesky
__global__ void chol_kernel(const __grid_constant__ CholBatch batch, int b, int* status) {
  __shared__ double2 sG[32][33];
  __shared__ double2 sR[32][33];
  __shared__ int bad;
  const int job = blockIdx.x;
  const double2* G = batch.G[job];
  double2* R = batch.R[job];
  double2* Ri = batch.Rinv[job];
  const int t = threadIdx.x;  // one warp
  for (int e = t; e < b * b; e += 32) {
    sG[e / b][e % b] = G[e];
    sR[e / b][e % b] = make_double2(0.0, 0.0);
  }
  if (t == 0) bad = 0;
  __syncwarp();
  double tr = 0.0;
  for (int i = 0; i < b; ++i) tr += sG[i][i].x;
  for (int k = 0; k < b; ++k) {
    // diagonal
    double d = sG[k][k].x;
    for (int i = 0; i < k; ++i) d -= cabs2(sR[i][k]);
    if (!(d > 1e-28 * tr)) {
      if (t == 0) bad = 1;
      d = fmax(d, 1e-300);
      d = fmax(d, 1e-28 * tr + 1e-300);
    }
    const double rkk = sqrt(d);
    __syncwarp();
    if (t == 0) sR[k][k] = make_double2(rkk, 0.0);
    // row k, columns j > k
    for (int j = k + 1 + t; j < b; j += 32) {
      double2 s = sG[k][j];
      for (int i = 0; i < k; ++i) {
        const double2 a = sR[i][k], c = sR[i][j];
        // s -= conj(a) * c
        s.x -= a.x * c.x + a.y * c.y;
        s.y -= a.x * c.y - a.y * c.x;
      }
      sR[k][j] = make_double2(s.x / rkk, s.y / rkk);
    }
    __syncwarp();
  }
  // inverse of the upper-triangular R: column j by back substitution (lane j)
  for (int j = t; j < b; j += 32) {
    double2 x[32];
    for (int i = 0; i < b; ++i) x[i] = make_double2(0.0, 0.0);
    x[j] = cdiv(make_double2(1.0, 0.0), sR[j][j]);
    for (int i = j - 1; i >= 0; --i) {
      double2 s = make_double2(0.0, 0.0);
      for (int l = i + 1; l <= j; ++l) cfma(s, sR[i][l], x[l]);
      x[i] = cdiv(make_double2(-s.x, -s.y), sR[i][i]);
    }
    for (int i = 0; i < b; ++i) Ri[i * b + j] = x[i];
  }
  for (int e = t; e < b * b; e += 32) R[e] = sR[e / b][e % b];
  if (t == 0 && status) status[job] = bad;
}

// --------------------------------------------------------------------------- Schur
struct Rot {
  double c;
  double2 s;
};

// G = [[c, s], [-conj(s), c]] with G [x; y] = [r; 0]
// c = |x|/r, s = x conj(y)/(|x| r), r = sqrt(|x|^2 + |y|^2); one reciprocal square
// root on the serial path (FP64 latency on GB300 is long, so the chain is kept short).
__device__ __forceinline__ Rot make_rot(double2 x, double2 y) {
  Rot g;
  const double ax2 = x.x * x.x + x.y * x.y, ay2 = y.x * y.x + y.y * y.y;
  if (ay2 == 0.0) {
    g.c = 1.0;
    g.s = make_double2(0.0, 0.0);
  } else if (ax2 == 0.0) {
    const double t = rsqrt(ay2);
    g.c = 0.0;
    g.s = make_double2(y.x * t, -y.y * t);  // conj(y)/|y|
  } else {
    const double t = rsqrt(ax2 * (ax2 + ay2));  // 1 / (|x| r)
    g.c = ax2 * t;
    g.s = make_double2((x.x * y.x + x.y * y.y) * t, (x.y * y.x - x.x * y.y) * t);
  }
  return g;
}

// rows (h1, h2) <- (c h1 + s h2, -conj(s) h1 + c h2)
__device__ __forceinline__ void rot_rows(double2& h1, double2& h2, const Rot& g) {
  const double2 a = h1, b = h2;
  h1 = make_double2(g.c * a.x + (g.s.x * b.x - g.s.y * b.y), g.c * a.y + (g.s.x * b.y + g.s.y * b.x));
  // -conj(s) a = -(s.x a.x + s.y a.y) - i (s.x a.y - s.y a.x)
  h2 = make_double2(g.c * b.x - (g.s.x * a.x + g.s.y * a.y), g.c * b.y - (g.s.x * a.y - g.s.y * a.x));
}
// cols (a1, a2) <- (c a1 + conj(s) a2, -s a1 + c a2)
__device__ __forceinline__ void rot_cols(double2& a1, double2& a2, const Rot& g) {
  const double2 a = a1, b = a2;
  a1 = make_double2(g.c * a.x + (g.s.x * b.x + g.s.y * b.y), g.c * a.y + (g.s.x * b.y - g.s.y * b.x));
  a2 = make_double2(g.c * b.x - (g.s.x * a.x - g.s.y * a.y), g.c * b.y - (g.s.x * a.y + g.s.y * a.x));
}

#define HH(i, j) H[(long long)(i) * ld + (j)]
#define ZZ(i, j) Z[(long long)(i) * ld + (j)]

__device__ double block_reduce_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(kDenseThreads) schur_kernel(const __grid_constant__ SchurBatch batch) {
  const SchurJob& J = batch.job[blockIdx.x];
  double2* H = J.H;
  double2* Z = J.Z;
  const int m = J.m, ld = J.ld;
  __shared__ double red[kDenseThreads / 32];
  __shared__ double2 sv[1024];  // Householder vector (m <= 1024)
  __shared__ Rot srot;
  __shared__ int s_flag;
  const int tid = threadIdx.x;

  if (m > 1024) {
    if (tid == 0) J.ordinfo[2] = 3;
    return;
  }
  // Z = I
  for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    ZZ(i, j) = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();

  // ---------------- Householder reduction to upper Hessenberg form
  for (int c = 0; c + 2 < m; ++c) {
    // x = H[c+1:m, c]
    double part = 0.0;
    for (int i = c + 2 + tid; i < m; i += blockDim.x) part += cabs2(HH(i, c));
    const double tail2 = block_reduce_sum(part, red);
    if (tail2 == 0.0) continue;
    const double2 x0 = HH(c + 1, c);
    const double ax0 = cabs(x0);
    const double xn = sqrt(tail2 + ax0 * ax0);
    const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
    const double2 alpha = make_double2(-ph.x * xn, -ph.y * xn);
    // v = x - alpha e1 ; tau = 2 / (v^H v)
    for (int i = c + 1 + tid; i < m; i += blockDim.x) sv[i] = (i == c + 1) ? csub(x0, alpha) : HH(i, c);
    __syncthreads();
    const double vn2 = cabs2(csub(x0, alpha)) + tail2;
    const double tau = 2.0 / vn2;
    // left: H[c+1:m, c+1:m] -= tau v (v^H H)
    for (int j = c + 1 + tid; j < m; j += blockDim.x) {
      double2 wsum = make_double2(0.0, 0.0);
      for (int i = c + 1; i < m; ++i) cfmac(wsum, sv[i], HH(i, j));
      wsum = cscale(wsum, tau);
      for (int i = c + 1; i < m; ++i) {
        const double2 t = cmul(sv[i], wsum);
        HH(i, j) = csub(HH(i, j), t);
      }
    }
    __syncthreads();
    // column c itself becomes (alpha, 0, ..., 0)
    for (int i = c + 1 + tid; i < m; i += blockDim.x) HH(i, c) = (i == c + 1) ? alpha : make_double2(0.0, 0.0);
    // right: H[0:m, c+1:m] -= tau (H v) v^H ; Z likewise
    for (int i = tid; i < m; i += blockDim.x) {
      double2 u = make_double2(0.0, 0.0);
      for (int j = c + 1; j < m; ++j) cfma(u, HH(i, j), sv[j]);
      u = cscale(u, tau);
      for (int j = c + 1; j < m; ++j) HH(i, j) = csub(HH(i, j), cmulc(u, sv[j]));
      double2 uz = make_double2(0.0, 0.0);
      for (int j = c + 1; j < m; ++j) cfma(uz, ZZ(i, j), sv[j]);
      uz = cscale(uz, tau);
      for (int j = c + 1; j < m; ++j) ZZ(i, j) = csub(ZZ(i, j), cmulc(uz, sv[j]));
    }
    __syncthreads();
  }

  // ---------------- shifted QR iteration to complex Schur form (full T, Z)
  int status = 0;
  {
    int ihi = m - 1;
    int its = 0;
    const int max_its = 60 * m + 100;
    int total_its = 0;
    // a subdiagonal entry is negligible below DBL_EPSILON times its diagonal
    // neighbours or times the largest entry of H (wanted Ritz values of
    // A - sigma lie near zero)
    double hmax = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) hmax = fmax(hmax, cabs1(HH(i, j)));
    while (ihi > 0) {
      // deflation search (all threads read the same values)
      int l = ihi;
      while (l > 0) {
        const double2 sub = HH(l, l - 1);
        double tst = cabs1(HH(l - 1, l - 1)) + cabs1(HH(l, l));
        if (tst == 0.0) tst = 1.0;
        if (cabs1(sub) <= DBL_EPSILON * fmax(tst, hmax)) break;
        --l;
      }
      __syncthreads();
      if (l > 0) {
        if (tid == 0) HH(l, l - 1) = make_double2(0.0, 0.0);
      }
      if (l == ihi) {
        __syncthreads();
        --ihi;
        its = 0;
        continue;
      }
      ++its;
      ++total_its;
      if (total_its > max_its) {
        status = 1;
        break;
      }
      double2 mu;
      if (its % 10 == 0) {
        // exceptional shift
        const double2 hs = HH(ihi, ihi - 1);
        mu = cadd(HH(ihi, ihi), make_double2(0.75 * fabs(hs.x), 0.0));
      } else {
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to H[ihi][ihi]
        const double2 a = HH(ihi - 1, ihi - 1), bq = HH(ihi - 1, ihi), cq = HH(ihi, ihi - 1), d = HH(ihi, ihi);
        const double2 tr2 = cscale(csub(a, d), 0.5);
        const double2 disc = csqrt_p(cadd(cmul(tr2, tr2), cmul(bq, cq)));
        const double2 r1 = cadd(tr2, disc), r2 = csub(tr2, disc);
        const double2 den = cabs(r1) >= cabs(r2) ? r1 : r2;
        const double2 bc = cmul(bq, cq);
        mu = (cabs(den) > 0.0) ? csub(d, cdiv(bc, den)) : d;
      }
      __syncthreads();
      // QR sweep on the active block [l, ihi]
      for (int k = l; k < ihi; ++k) {
        if (tid == 0) {
          double2 x, y;
          if (k == l) {
            x = csub(HH(l, l), mu);
            y = HH(l + 1, l);
          } else {
            x = HH(k, k - 1);
            y = HH(k + 1, k - 1);
          }
          srot = make_rot(x, y);
        }
        __syncthreads();
        const Rot g = srot;
        const int c0 = (k == l) ? l : k - 1;
        const int r1 = min(k + 2, ihi) + 1;
        // H <- G H G^H: rows (k, k+1) and columns (k, k+1) touch disjoint entries
        // except the 2x2 block, which thread 0 updates with both; one barrier.
        for (int j = c0 + tid; j < m; j += blockDim.x) {
          if (j == k || j == k + 1) continue;
          rot_rows(HH(k, j), HH(k + 1, j), g);
          if (j == k - 1) HH(k + 1, k - 1) = make_double2(0.0, 0.0);  // the chased bulge
        }
        for (int i = tid; i < r1; i += blockDim.x) {
          if (i == k || i == k + 1) continue;
          rot_cols(HH(i, k), HH(i, k + 1), g);
        }
        for (int i = tid; i < m; i += blockDim.x) rot_cols(ZZ(i, k), ZZ(i, k + 1), g);
        if (tid == 0) {
          double2 a = HH(k, k), b = HH(k, k + 1), c = HH(k + 1, k), d = HH(k + 1, k + 1);
          rot_rows(a, c, g);
          rot_rows(b, d, g);
          rot_cols(a, b, g);
          rot_cols(c, d, g);
          HH(k, k) = a;
          HH(k, k + 1) = b;
          HH(k + 1, k) = c;
          HH(k + 1, k + 1) = d;
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  // clean strictly-lower part (rounding residue below the subdiagonal is zero by construction)
  for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    if (i > j) HH(i, j) = make_double2(0.0, 0.0);
  }
  __syncthreads();

  // ---------------- select the 'keep' Ritz values closest to the shift (smallest |theta - i sig_im|)
  // rank by (|theta|, Re, Im, index)
  __shared__ int s_sel[1024];
  for (int i = tid; i < m; i += blockDim.x) {
    const double2 ti = HH(i, i);
    const double ai = cabs(make_double2(ti.x, ti.y - J.sig_im));
    int rank = 0;
    for (int q = 0; q < m; ++q) {
      if (q == i) continue;
      const double2 tq = HH(q, q);
      const double aq = cabs(make_double2(tq.x, tq.y - J.sig_im));
      bool less = aq < ai || (aq == ai && (tq.x < ti.x || (tq.x == ti.x && (tq.y < ti.y || (tq.y == ti.y && q < i)))));
      rank += less ? 1 : 0;
    }
    s_sel[i] = rank;
  }
  __syncthreads();
  // keep = J.keep, extended over a cluster that straddles the cut
  if (tid == 0) {
    int k = J.keep < m ? J.keep : m;
    // |theta| of the element with rank k-1 and rank k
    while (k < m - 1 && k < J.kmax) {
      double a_in = -1.0, a_out = -1.0;
      for (int q = 0; q < m; ++q) {
        if (s_sel[q] == k - 1) a_in = cabs(make_double2(HH(q, q).x, HH(q, q).y - J.sig_im));
        if (s_sel[q] == k) a_out = cabs(make_double2(HH(q, q).x, HH(q, q).y - J.sig_im));
      }
      if (a_out - a_in <= 1e-10 * fmax(1.0, a_in)) ++k;
      else break;
    }
    s_flag = k;
  }
  __syncthreads();
  const int kk = s_flag;
  // selected flag: rank < kk ; reorder selected to the top by adjacent swaps
  for (int i = tid; i < m; i += blockDim.x) s_sel[i] = (s_sel[i] < kk) ? 1 : 0;
  __syncthreads();
  {
    int ks = 0;
    for (int pos = 0; pos < m; ++pos) {
      if (!s_sel[pos]) continue;
      // move from pos to ks
      for (int q = pos - 1; q >= ks; --q) {
        // swap diagonal entries q, q+1
        if (tid == 0) {
          const double2 t11 = HH(q, q), t22 = HH(q + 1, q + 1);
          srot = make_rot(HH(q, q + 1), csub(t22, t11));
        }
        __syncthreads();
        const Rot g = srot;
        for (int j = q + 2 + tid; j < m; j += blockDim.x) rot_rows(HH(q, j), HH(q + 1, j), g);
        for (int i = tid; i < q; i += blockDim.x) rot_cols(HH(i, q), HH(i, q + 1), g);
        for (int i = tid; i < m; i += blockDim.x) rot_cols(ZZ(i, q), ZZ(i, q + 1), g);
        // the 2x2 block {q, q+1}^2 is disjoint from the loops above
        if (tid == 0) {
          const double2 t11 = HH(q, q);
          HH(q, q) = HH(q + 1, q + 1);
          HH(q + 1, q + 1) = t11;
          HH(q + 1, q) = make_double2(0.0, 0.0);
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

  // ---------------- outputs
  for (int i = tid; i < m; i += blockDim.x) J.theta[i] = HH(i, i);
  // Bz = B Z[:, 0:kk]
  for (int e = tid; e < J.b * kk; e += blockDim.x) {
    const int r = e / kk, l = e % kk;
    double2 bz = make_double2(0.0, 0.0);
    for (int q = 0; q < m; ++q) cfma(bz, J.B[(long long)r * ld + q], ZZ(q, l));
    J.Bz[(long long)r * ld + l] = bz;
  }
  // eigenvectors of T[0:kk, 0:kk] (column i in S), unit 2-norm
  const double smlnum = 1e-290;
  for (int i = tid; i < kk; i += blockDim.x) {
    const double2 lam = HH(i, i);
    const double smin = fmax(DBL_EPSILON * cabs(lam), smlnum);
    double2* s = J.S;  // column i: S[l*ld + i]
    for (int l = i + 1; l < kk; ++l) s[(long long)l * ld + i] = make_double2(0.0, 0.0);
    s[(long long)i * ld + i] = make_double2(1.0, 0.0);
    for (int jj = i - 1; jj >= 0; --jj) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = jj + 1; l <= i; ++l) cfma(acc, HH(jj, l), s[(long long)l * ld + i]);
      double2 den = csub(HH(jj, jj), lam);
      if (cabs(den) < smin) den = make_double2(smin, 0.0);
      s[(long long)jj * ld + i] = cdiv(make_double2(-acc.x, -acc.y), den);
    }
    double nrm = 0.0;
    for (int l = 0; l <= i; ++l) nrm += cabs2(s[(long long)l * ld + i]);
    nrm = 1.0 / sqrt(nrm);
    for (int l = 0; l <= i; ++l) s[(long long)l * ld + i] = cscale(s[(long long)l * ld + i], nrm);
  }
  __syncthreads();
  // residual estimate ||B Z_k s_i|| (the Ritz vector's residual through A Q = Q H + V B)
  for (int i = tid; i < kk; i += blockDim.x) {
    double r2 = 0.0;
    for (int r = 0; r < J.b; ++r) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l <= i; ++l) cfma(acc, J.Bz[(long long)r * ld + l], J.S[(long long)l * ld + i]);
      r2 += cabs2(acc);
    }
    J.resid[i] = sqrt(r2);
  }
  __syncthreads();
  if (tid == 0) {
    // wanted = the nwant smallest |theta| among the kept
    int nconv = 0;
    for (int i = 0; i < kk; ++i) {
      const double ai = cabs(make_double2(HH(i, i).x, HH(i, i).y - J.sig_im));
      int rank = 0;
      for (int q = 0; q < kk; ++q) {
        const double aq = cabs(make_double2(HH(q, q).x, HH(q, q).y - J.sig_im));
        if (aq < ai || (aq == ai && q < i)) ++rank;
      }
      if (rank < J.nwant && J.resid[i] <= J.tol_abs) ++nconv;
    }
    J.ordinfo[0] = kk;
    J.ordinfo[1] = nconv;
    J.ordinfo[2] = status;
  }
}

#undef HH
#undef ZZ

__global__ void ritz_kernel(const __grid_constant__ RitzBatch batch) {
  const RitzJob& J = batch.job[blockIdx.x];
  const int kk = J.ordinfo[0];
  __shared__ int widx[1024];
  const int tid = threadIdx.x;
  // wanted = nwant smallest |theta| among the leading kk, then ordered by (Re, Im)
  for (int i = tid; i < kk; i += blockDim.x) {
    const double2 ti = J.theta[i];
    const double ai = cabs(make_double2(ti.x, ti.y - J.sig_im));
    int rank = 0;
    for (int q = 0; q < kk; ++q) {
      const double aq = cabs(make_double2(J.theta[q].x, J.theta[q].y - J.sig_im));
      if (aq < ai || (aq == ai && q < i)) ++rank;
    }
    widx[i] = rank < J.nwant ? 1 : 0;
  }
  __syncthreads();
  // position among wanted by (Re, Im, index)
  for (int i = tid; i < kk; i += blockDim.x) {
    if (!widx[i]) continue;
    const double2 ti = J.theta[i];
    int pos = 0;
    for (int q = 0; q < kk; ++q) {
      if (q == i || !widx[q]) continue;
      const double2 tq = J.theta[q];
      if (tq.x < ti.x || (tq.x == ti.x && (tq.y < ti.y || (tq.y == ti.y && q < i)))) ++pos;
    }
    J.eps[pos] = make_double2(ti.x + J.sigma, ti.y);
    J.res_out[pos] = J.resid[i];
    // Yw[:, pos] = Z[:, 0:kk] s_i
    for (int r = 0; r < J.m; ++r) {
      double2 acc = make_double2(0.0, 0.0);
      for (int l = 0; l <= i; ++l) cfma(acc, J.Z[(long long)r * J.ld + l], J.S[(long long)l * J.ld + i]);
      J.Yw[(long long)r * J.ldy + pos] = acc;
    }
  }
}

// H = S^-1 K for m x m complex matrices (row-major, leading dimension ld) by
// Gauss-Jordan elimination with partial pivoting, one CTA; S is overwritten.
// status: 0, or 1 + the column at which no nonzero pivot was left.
__global__ void small_solve_kernel(double2* __restrict__ S, double2* __restrict__ H, int m, int ld, int* status) {
  __shared__ double2 f[1024];
  __shared__ int piv;
  const int tid = threadIdx.x;
  if (tid == 0) *status = 0;
  for (int c = 0; c < m; ++c) {
    if (tid == 0) {
      int p = c;
      double best = -1.0;
      for (int r = c; r < m; ++r) {
        const double a = cabs(S[(long long)r * ld + c]);
        if (a > best) {
          best = a;
          p = r;
        }
      }
      piv = best > 0.0 ? p : -1;
      if (piv < 0) *status = 1 + c;
    }
    __syncthreads();
    if (piv < 0) return;
    if (piv != c) {  // swap rows c and piv of [S | H]
      for (int j = tid; j < 2 * m; j += blockDim.x) {
        double2* X = j < m ? S : H;
        const int jj = j < m ? j : j - m;
        const double2 t = X[(long long)c * ld + jj];
        X[(long long)c * ld + jj] = X[(long long)piv * ld + jj];
        X[(long long)piv * ld + jj] = t;
      }
    }
    __syncthreads();
    // scale row c by 1 / S[c][c]
    const double2 inv = cdiv(make_double2(1.0, 0.0), S[(long long)c * ld + c]);
    __syncthreads();
    for (int j = tid; j < 2 * m; j += blockDim.x) {
      double2* X = j < m ? S : H;
      const int jj = j < m ? j : j - m;
      X[(long long)c * ld + jj] = cmul(X[(long long)c * ld + jj], inv);
    }
    __syncthreads();
    for (int r = tid; r < m; r += blockDim.x) f[r] = S[(long long)r * ld + c];
    __syncthreads();
    // eliminate column c from every other row
    for (int e = tid; e < m * 2 * m; e += blockDim.x) {
      const int r = e / (2 * m), j = e % (2 * m);
      if (r == c) continue;
      double2* X = j < m ? S : H;
      const int jj = j < m ? j : j - m;
      const double2 t = cmul(f[r], X[(long long)c * ld + jj]);
      X[(long long)r * ld + jj] = csub(X[(long long)r * ld + jj], t);
    }
    __syncthreads();
  }
}

__global__ void hupdate_kernel(const __grid_constant__ HUpdBatch batch) {
  const HUpdJob& J = batch.job[blockIdx.x];
  const int p = J.p, b = J.b, ld = J.ld;
  // new column block of H
  for (int e = threadIdx.x; e < (p + b) * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    J.H[(long long)i * ld + p + j] = cadd(J.C1[e], J.C2[e]);
  }
  // old coupling rows become H[p:p+b, 0:p]
  for (int e = threadIdx.x; e < b * p; e += blockDim.x) {
    const int i = e / p, j = e % p;
    J.H[(long long)(p + i) * ld + j] = J.Bm[(long long)i * ld + j];
  }
  __syncthreads();
  // B = [0, R2 R1]
  for (int e = threadIdx.x; e < b * (p + b); e += blockDim.x) {
    const int i = e / (p + b), j = e % (p + b);
    double2 v = make_double2(0.0, 0.0);
    if (j >= p) {
      const int jj = j - p;
      for (int l = 0; l < b; ++l) cfma(v, J.R2[i * b + l], J.R1[l * b + jj]);
    }
    J.Bm[(long long)i * ld + j] = v;
  }
}

__global__ void zext_kernel(const __grid_constant__ ZextBatch batch) {
  const ZextJob& J = batch.job[blockIdx.y];
  const int rows = J.m + J.b, cols = J.k + J.b;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)rows * cols) return;
  const int i = (int)(t / cols), j = (int)(t % cols);
  double2 v = make_double2(0.0, 0.0);
  if (i < J.m && j < J.k) v = J.Z[(long long)i * J.ldz + j];
  else if (i >= J.m && j >= J.k && (i - J.m) == (j - J.k)) v = make_double2(1.0, 0.0);
  J.Zext[(long long)i * J.ldo + j] = v;
}

}  // namespace

void launch_hupdate_batch(const HUpdBatch& b, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  hupdate_kernel<<<b.n, 256, 0, s>>>(b);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_zext_batch(const ZextBatch& b, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  int maxe = 0;
  for (int q = 0; q < b.n; ++q) {
    const int e = (b.job[q].m + b.job[q].b) * (b.job[q].k + b.job[q].b);
    maxe = e > maxe ? e : maxe;
  }
  zext_kernel<<<dim3((maxe + 255) / 256, b.n), 256, 0, s>>>(b);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_ritz_batch(const RitzBatch& b, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  ritz_kernel<<<b.n, kDenseThreads, 0, s>>>(b);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_chol_batch(const CholBatch& cb, int b, int* status, cudaStream_t s, long long* launches) {
  if (cb.n <= 0) return;
  chol_kernel<<<cb.n, 32, 0, s>>>(cb, b, status);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_small_solve(double2* S, double2* H, int m, int ld, int* status, cudaStream_t s, long long* launches) {
  if (m <= 0) return;
  if (m > 1024 || ld < m) throw Error{SWI_EINVAL, "small solve: size out of range"};
  small_solve_kernel<<<1, kDenseThreads, 0, s>>>(S, H, m, ld, status);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_schur_batch(const SchurBatch& b, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  schur_kernel<<<b.n, kDenseThreads, 0, s>>>(b);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
