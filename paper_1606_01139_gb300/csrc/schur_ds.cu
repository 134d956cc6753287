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

constexpr int kThreads = 512;
// Warp 0 runs the serial chain of the QR and reordering sweeps; the element
// owners live in the warps that do not share its scheduler (warps 4, 8, 12 of
// the 16 share warp 0's), 12 warps or 384 owners.
constexpr int kMaxOwners = 384;
// The register-owner sweeps run for orders up to kOwnerPathMaxM; restart
// matrices of order 240-384 (deflations inside the active window) exhausted
// the QR iteration limit in that path, so larger orders take the plain sweep.
constexpr int kOwnerPathMaxM = 224;
static_assert(kOwnerPathMaxM <= kMaxOwners, "every row and column of the sweep needs an owner thread");
__device__ __forceinline__ int owner_index(int tid) {
  const int w = tid >> 5;
  if ((w & 3) == 0) return -1;
  return (w - 1 - (w >> 2)) * 32 + (tid & 31);
}
// deflation and tie tolerances relative to double-single precision: a
// subdiagonal entry is negligible below kDeflate times its two diagonal
// neighbours, or below kDeflateAbs times the largest entry of H (the wanted
// Ritz values of A - sigma lie near zero, where the first test alone would ask
// for more than double-single rounding can give)
constexpr float kDeflate = 4e-15f;
constexpr float kDeflateAbs = 1e-14f;

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
  // 2^(127 - E), E the biased exponent of mx: brings mx into [1, 2)
  const int be = min(max((__float_as_int(mx) >> 23) & 0xff, 1), 253);
  const float sc = __int_as_float((254 - be) << 23);
  x = dc{df{x.re.h * sc, x.re.l * sc}, df{x.im.h * sc, x.im.l * sc}};
  y = dc{df{y.re.h * sc, y.re.l * sc}, df{y.im.h * sc, y.im.l * sc}};
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
// Z is kept transposed in the work array: the column rotations then touch
// consecutive addresses across the threads that own its rows.
#define ZD(i, j) Zd[(long long)(j) * ld + (i)]

__global__ void __launch_bounds__(kThreads) schur_ds_kernel(const __grid_constant__ SchurBatch batch) {
  const SchurJob& J = batch.job[blockIdx.x];
  dc* Hd = reinterpret_cast<dc*>(J.Hw);
  dc* Zd = reinterpret_cast<dc*>(J.Zw);
  const int m = J.m, ld = J.ld;
  __shared__ df red[kThreads / 32];
  __shared__ dc sv[1024];
  __shared__ RotD srot;
  __shared__ RotD s_rot2[2];
  __shared__ dc s_hand[2][4];
  __shared__ int s_flag;
  __shared__ int s_l;
  __shared__ dc s_mu;
  __shared__ int s_sel[1024];
  const int tid = threadIdx.x;
  if (m > 1024) {
    if (tid == 0) J.ordinfo[2] = 3;
    return;
  }
  // load H, Z = I, and the largest |Re| + |Im| of H
  __shared__ unsigned s_hmax;
  if (tid == 0) s_hmax = 0u;
  __syncthreads();
  {
    float hm = 0.f;
    for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
      const int i = (int)(e / m), j = (int)(e % m);
      const double2 h = J.H[(long long)i * ld + j];
      HD(i, j) = cfrom(h);
      ZD(i, j) = dc{df{i == j ? 1.f : 0.f, 0.f}, dfz()};
      hm = fmaxf(hm, (float)(fabs(h.x) + fabs(h.y)));
    }
    atomicMax(&s_hmax, __float_as_uint(hm));  // non-negative floats order as their bit patterns
  }
  __syncthreads();
  const float defl_abs = kDeflateAbs * __uint_as_float(s_hmax);

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
    // H <- P H: thread pairs share a column (even/odd rows, two partial sums
    // each), combined by a shuffle; the pair then updates its halves.
    for (int t = tid; t < 2 * (m - c - 1); t += blockDim.x) {
      const int j = c + 1 + (t >> 1), h = t & 1;
      dc w0 = czero(), w1 = czero();
      int i = c + 1 + h;
      for (; i + 2 < m; i += 4) {
        const dc x0 = HD(i, j), x1 = HD(i + 2, j);
        w0 = cadd(w0, cmulc_l(sv[i], x0));
        w1 = cadd(w1, cmulc_l(sv[i + 2], x1));
      }
      if (i < m) w0 = cadd(w0, cmulc_l(sv[i], HD(i, j)));
      dc w = cadd(w0, w1);
      const unsigned msk = 3u << (threadIdx.x & 30);  // the two lanes of the pair
      dc o;
      o.re.h = __shfl_xor_sync(msk, w.re.h, 1);
      o.re.l = __shfl_xor_sync(msk, w.re.l, 1);
      o.im.h = __shfl_xor_sync(msk, w.im.h, 1);
      o.im.l = __shfl_xor_sync(msk, w.im.l, 1);
      w = cscale(cadd(w, o), tau);
      for (int r = c + 1 + h; r < m; r += 2) HD(r, j) = csub(HD(r, j), cmul(sv[r], w));
    }
    __syncthreads();
    for (int i = c + 1 + tid; i < m; i += blockDim.x) HD(i, c) = (i == c + 1) ? alpha : czero();
    // H <- H P and Z <- Z P: one thread per row of H and per row of Z
    for (int t = tid; t < 2 * m; t += blockDim.x) {
      const bool isz = t >= m;
      dc* row = isz ? &ZD(t - m, 0) : &HD(t, 0);
      const long long st = isz ? ld : 1;
      dc u0 = czero(), u1 = czero();
      int j = c + 1;
      for (; j + 1 < m; j += 2) {
        const dc x0 = row[j * st], x1 = row[(j + 1) * st];
        u0 = cadd(u0, cmul(x0, sv[j]));
        u1 = cadd(u1, cmul(x1, sv[j + 1]));
      }
      if (j < m) u0 = cadd(u0, cmul(row[j * st], sv[j]));
      const dc u = cscale(cadd(u0, u1), tau);
      for (j = c + 1; j < m; ++j) row[j * st] = csub(row[j * st], cmul(u, cconj(sv[j])));
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
      // l = the largest index <= ihi with a negligible subdiagonal (0 if none),
      // every subdiagonal tested at once
      if (tid == 0) s_l = 0;
      __syncthreads();
      for (int i = tid + 1; i <= ihi; i += blockDim.x) {
        float tst = cabs1f(HD(i - 1, i - 1)) + cabs1f(HD(i, i));
        if (tst == 0.f) tst = 1.f;
        if (cabs1f(HD(i, i - 1)) <= fmaxf(kDeflate * tst, defl_abs)) atomicMax(&s_l, i);
      }
      __syncthreads();
      const int l = s_l;
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
      if (tid == 0) {  // the shift, formed once and shared
        dc mu;
        if (its % 10 == 0) {
          const dc hs = HD(ihi, ihi - 1);
          mu = cadd(HD(ihi, ihi), dc{df{0.75f * fabsf(approx(hs.re)), 0.f}, dfz()});
        } else {
          // Wilkinson shift, evaluated in FP64
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
        s_mu = mu;
      }
      __syncthreads();
      const dc mu = s_mu;
      if (m <= kOwnerPathMaxM) {
        // One barrier per rotation.  Warp 0 chases the bulge: at step k its
        // lanes 0-6 each form one half-rotation h = c u + w v (w = +-s or
        // +-conj(s)) of the 2x2 block {k, k+1}, of row k+2 (the new bulge) and
        // of column k-1; lanes 0-3 then apply the column rotation to the 2x2
        // block and every lane forms the next rotation from H[k+1][k] and the
        // bulge.  Owner q (owner_index) holds column q (left updates, rows k, k+1), row q
        // (right updates, columns k, k+1) and row q of Z, with its pair in
        // registers and the next-but-one element prefetched.  Hand-offs through
        // double-buffered shared slots, written at step k and read at k+1:
        // [0] H[k+1][k+2] (owner of column k+2 -> lanes 1, 3), [1] H[k][k+1]
        // (lane 3 -> owner of row k, which joins the right updates), [2]
        // H[k][k+2] and [3] H[k][k+3] (owners of columns k+2, k+3 -> owner of
        // row k).  Diagonal and subdiagonal entries ahead of the bulge come from
        // a copy in shared memory taken before the sweep.
        dc* sdg = sv;        // H[i][i]
        dc* ssb = sv + 512;  // H[i+1][i]
        for (int i = l + tid; i <= ihi; i += blockDim.x) {
          sdg[i] = HD(i, i);
          if (i < ihi) ssb[i] = HD(i + 1, i);
        }
        const int q = owner_index(tid);
        const bool owner = q >= 0 && q < m;
        const int ln = tid & 31;
        dc lt = czero(), lb = czero(), rl = czero(), rr = czero(), zl = czero(), zr = czero();
        dc pl0 = czero(), pl1 = czero(), pr0 = czero(), pr1 = czero(), pz0 = czero(), pz1 = czero();
        dc pu = czero(), pv = czero();
        // half-rotation coefficient signs: w = (sr Re s, si Im s)
        float sr1 = 1.f, si1 = 1.f, sr2 = 1.f, si2 = 1.f;
        if (ln <= 1) sr1 = -1.f;
        if (ln == 4 || ln == 5) si1 = -1.f;
        if (ln == 5) sr1 = -1.f;
        if (ln == 0 || ln == 2) si2 = -1.f;
        if (ln == 1 || ln == 3) { sr2 = -1.f; si2 = -1.f; }
        if (owner) {
          const bool m2 = l + 2 < m;
          if (q >= l + 2) {
            lt = HD(l, q);
            lb = HD(l + 1, q);
            if (m2) pl0 = HD(l + 2, q);
          }
          if (q < l) {
            rl = HD(q, l);
            rr = HD(q, l + 1);
            if (m2) pr0 = HD(q, l + 2);
          }
          zl = ZD(q, l);
          zr = ZD(q, l + 1);
          if (m2) pz0 = ZD(q, l + 2);
        }
        if (tid < 32) {
          const dc a = HD(l, l), b = HD(l, l + 1), c = HD(l + 1, l), d = HD(l + 1, l + 1);
          const dc f0 = (l + 2 <= ihi) ? HD(l + 2, l + 1) : czero();
          if (ln == 0) { pu = c; pv = a; }
          if (ln == 1) { pu = d; pv = b; }
          if (ln == 2) { pu = a; pv = c; }
          if (ln == 3) { pu = b; pv = d; }
          if (ln == 4) pv = f0;
          if (ln == 5) pu = f0;
          const RotD g0 = make_rot_ds(csub(a, mu), c);
          if (ln == 0) s_rot2[l & 1] = g0;
        }
        __syncthreads();
        // one step; (pa, pb) are the prefetch slots consumed / refilled
        auto step = [&](const int k, dc& pla, dc& plb, dc& pra, dc& prb, dc& pza, dc& pzb) {
          const RotD g = s_rot2[k & 1];
          const int par = k & 1;
          if (tid < 32) {
            if (ln == 0) n_upd += (m - ((k == l) ? l : k - 1)) + (min(k + 2, ihi) + 1) + m;
            if (k > l) {
              const dc hb = s_hand[par ^ 1][0];  // H[k][k+1]
              if (ln == 1) pv = hb;
              if (ln == 3) pu = hb;
            }
            // lane-dependent selections above and below: reconverge the warp
            // before each stretch of arithmetic so that it issues once for all lanes
            __syncwarp();
            const dc w1 = dc{df{sr1 * g.s.re.h, sr1 * g.s.re.l}, df{si1 * g.s.im.h, si1 * g.s.im.l}};
            const dc h1 = cadd(cscale(pu, g.c), cmul(w1, pv));
            dc o;
            o.re.h = __shfl_xor_sync(0xffffffffu, h1.re.h, 1);
            o.re.l = __shfl_xor_sync(0xffffffffu, h1.re.l, 1);
            o.im.h = __shfl_xor_sync(0xffffffffu, h1.im.h, 1);
            o.im.l = __shfl_xor_sync(0xffffffffu, h1.im.l, 1);
            const dc w2 = dc{df{sr2 * g.s.re.h, sr2 * g.s.re.l}, df{si2 * g.s.im.h, si2 * g.s.im.l}};
            const dc h2 = cadd(cscale(h1, g.c), cmul(w2, o));
            dc cpp, ep;  // H[k+1][k] and the bulge H[k+2][k], broadcast
            cpp.re.h = __shfl_sync(0xffffffffu, h2.re.h, 0);
            cpp.re.l = __shfl_sync(0xffffffffu, h2.re.l, 0);
            cpp.im.h = __shfl_sync(0xffffffffu, h2.im.h, 0);
            cpp.im.l = __shfl_sync(0xffffffffu, h2.im.l, 0);
            ep.re.h = __shfl_sync(0xffffffffu, h1.re.h, 4);
            ep.re.l = __shfl_sync(0xffffffffu, h1.re.l, 4);
            ep.im.h = __shfl_sync(0xffffffffu, h1.im.h, 4);
            ep.im.l = __shfl_sync(0xffffffffu, h1.im.l, 4);
            // lanes 0, 2 need H[k+2][k+1] (lane 5) and H[k+1][k+1] (lane 1)
            const int src_u = (ln == 0) ? 5 : 1, src_v = (ln == 0) ? 1 : 5;
            dc nu, nv;
            nu.re.h = __shfl_sync(0xffffffffu, (ln == 5) ? h1.re.h : h2.re.h, src_u);
            nu.re.l = __shfl_sync(0xffffffffu, (ln == 5) ? h1.re.l : h2.re.l, src_u);
            nu.im.h = __shfl_sync(0xffffffffu, (ln == 5) ? h1.im.h : h2.im.h, src_u);
            nu.im.l = __shfl_sync(0xffffffffu, (ln == 5) ? h1.im.l : h2.im.l, src_u);
            nv.re.h = __shfl_sync(0xffffffffu, (ln == 5) ? h1.re.h : h2.re.h, src_v);
            nv.re.l = __shfl_sync(0xffffffffu, (ln == 5) ? h1.re.l : h2.re.l, src_v);
            nv.im.h = __shfl_sync(0xffffffffu, (ln == 5) ? h1.im.h : h2.im.h, src_v);
            nv.im.l = __shfl_sync(0xffffffffu, (ln == 5) ? h1.im.l : h2.im.l, src_v);
            {
              // lane 0: H[k+1][k], 1: H[k+1][k+1], 2: H[k][k], 3: H[k][k+1],
              // 4, 5: H[k+2][k], H[k+2][k+1], 6: H[k][k-1] (and H[k+1][k-1] = 0)
              int r = -1, cc = 0;
              if (ln == 0) { r = k + 1; cc = k; }
              if (ln == 1) { r = k + 1; cc = k + 1; }
              if (ln == 2) { r = k; cc = k; }
              if (ln == 3) { r = k; cc = k + 1; }
              if (ln == 4 && k + 2 <= ihi) { r = k + 2; cc = k; }
              if (ln == 5 && k + 2 <= ihi) { r = k + 2; cc = k + 1; }
              if (ln == 6 && k > l) { r = k; cc = k - 1; }
              if (ln == 7 && k > l) { r = k + 1; cc = k - 1; }
              const dc val = (ln <= 3) ? h2 : ((ln == 7) ? czero() : h1);
              if (r >= 0) HD(r, cc) = val;
              if (ln == 3) s_hand[par][1] = h2;
            }
            __syncwarp();
            if (k + 1 < ihi) {
              const RotD gn = make_rot_ds(cpp, ep);
              if (ln == 0) s_rot2[par ^ 1] = gn;
              const dc dg = sdg[k + 2];
              const dc sb = (k + 3 <= ihi) ? ssb[k + 2] : czero();
              if (ln == 0 || ln == 2) { pu = nu; pv = nv; }
              if (ln == 1) pu = dg;
              if (ln == 3) pv = dg;
              if (ln == 4) { pu = czero(); pv = sb; }
              if (ln == 5) { pu = sb; pv = czero(); }
              if (ln == 6) { pu = cpp; pv = ep; }
            }
            __syncwarp();
          } else if (owner) {
            const bool m3 = k + 3 < m;
            if (q >= k + 2) {  // left: rows k, k+1 of column q
              if (m3 && q >= k + 4) plb = HD(k + 3, q);
              rot_rows(lt, lb, g);
              HD(k, q) = lt;  // final for this sweep; H[k+1][q] stays in a register
              if (q == k + 2) {
                s_hand[par][0] = lb;  // H[k+1][k+2] for warp 0
                s_hand[par][2] = lt;  // H[k][k+2] for the owner of row k
              }
              if (q == k + 3) s_hand[par][3] = lt;  // H[k][k+3] for the owner of row k
              lt = lb;
              lb = pla;
            }
            if (q < k) {  // right: columns k, k+1 of row q
              if (q == k - 1 && k > l) {
                rl = s_hand[par ^ 1][1];
                rr = s_hand[par ^ 1][2];
                pra = s_hand[par ^ 1][3];
              }
              if (m3) prb = HD(q, k + 3);
              rot_cols(rl, rr, g);
              HD(q, k) = rl;
              rl = rr;
              rr = pra;
            }
            if (m3) pzb = ZD(q, k + 3);
            rot_cols(zl, zr, g);  // Z: columns k, k+1 of row q
            ZD(q, k) = zl;
            zl = zr;
            zr = pza;
          }
          __syncthreads();
        };
        int k = l;
        for (; k + 1 < ihi; k += 2) {
          step(k, pl0, pl1, pr0, pr1, pz0, pz1);
          step(k + 1, pl1, pl0, pr1, pr0, pz1, pz0);
        }
        if (k < ihi) step(k, pl0, pl1, pr0, pr1, pz0, pz1);
        if (owner) {  // the elements still held in registers
          if (q >= ihi + 1) HD(ihi, q) = lt;
          if (q < ihi - 1) HD(q, ihi) = rl;
          ZD(q, ihi) = zl;
        }
      } else
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

  // ---------------- selection: rank by (|theta - i sig_im|, Re, Im, index) in FP64 of the diagonal
  for (int i = tid; i < m; i += blockDim.x) {
    const double2 ti = cto(HD(i, i));
    const double ai = hypot(ti.x, ti.y - J.sig_im);
    int rank = 0;
    for (int q = 0; q < m; ++q) {
      if (q == i) continue;
      const double2 tq = cto(HD(q, q));
      const double aq = hypot(tq.x, tq.y - J.sig_im);
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
        if (s_sel[q] == k - 1) a_in = hypot(tq.x, tq.y - J.sig_im);
        if (s_sel[q] == k) a_out = hypot(tq.x, tq.y - J.sig_im);
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
  if (m <= kOwnerPathMaxM) {
    // Each selected eigenvalue lambda moves up from pos to ks by adjacent swaps
    // q = pos-1, ..., ks, one barrier per swap.  The rotation of swap q comes
    // from (T[q][q+1], lambda - T[q][q]); the next one needs T[q-1][q] after
    // the column update of row q-1, so thread 0 updates row q-1 itself and
    // forms the next rotation at once.  Owner i (owner_index) holds column i (rows q, q+1),
    // row i (columns q, q+1) for i < q-1 and row i of Z, with its pair in
    // registers.  Hand-offs: T[q-1][q+1] (thread 0 -> the owner of column q+1,
    // which joins next swap) and T[q-2][q] (owner of row q-2 -> thread 0).
    const int i = owner_index(tid);
    const bool owner = i >= 0 && i < m;
    int ks = 0;
    for (int pos = 0; pos < m; ++pos) {
      if (!s_sel[pos]) continue;
      if (pos > ks) {
        const int q0 = pos - 1;
        dc lt = czero(), lb = czero(), rl = czero(), rr = czero(), zl = czero(), zr = czero();
        dc lam = czero(), tqq = czero(), a1 = czero(), a2 = czero();
        if (owner) {
          if (i >= q0 + 2) {
            lt = HD(q0, i);
            lb = HD(q0 + 1, i);
          }
          if (i < q0 - 1) {
            rl = HD(i, q0);
            rr = HD(i, q0 + 1);
          }
          zl = ZD(i, q0);
          zr = ZD(i, q0 + 1);
        }
        if (tid == 0) {
          lam = HD(pos, pos);
          tqq = HD(q0, q0);
          if (q0 >= 1) {
            a1 = HD(q0 - 1, q0);
            a2 = HD(q0 - 1, q0 + 1);
          }
          s_rot2[q0 & 1] = make_rot_ds(HD(q0, q0 + 1), csub(lam, tqq));
        }
        __syncthreads();
        for (int q = q0; q >= ks; --q) {
          const RotD g = s_rot2[q & 1];
          const int par = q & 1;
          if (tid == 0) {
            dc n_tqq = czero(), n_a1 = czero();
            if (q - 1 >= ks) {
              n_tqq = HD(q - 1, q - 1);
              if (q >= 2) n_a1 = HD(q - 2, q - 1);
            }
            n_upd += (m - q - 2) + q + m;
            if (q < q0 && q >= 1) a2 = s_hand[par ^ 1][1];  // T[q-1][q+1], from the owner of row q-1
            if (q >= 1) {
              rot_cols(a1, a2, g);  // row q-1, columns q, q+1
              HD(q - 1, q) = a1;
              HD(q - 1, q + 1) = a2;
              s_hand[par][0] = a2;
            }
            HD(q, q) = lam;
            HD(q + 1, q + 1) = tqq;
            HD(q + 1, q) = czero();
            if (q - 1 >= ks) {
              s_rot2[par ^ 1] = make_rot_ds(a1, csub(lam, n_tqq));
              tqq = n_tqq;
              a1 = n_a1;
            }
          } else if (owner) {
            const dc n_lt = (i >= q + 2 && q >= 1) ? HD(q - 1, i) : czero();
            const dc n_rl = (i < q - 2) ? HD(i, q - 1) : czero();
            const dc n_zl = (q >= 1) ? ZD(i, q - 1) : czero();
            if (i == q + 1) lb = HD(q, q + 1);  // joins the row updates next swap
            if (i >= q + 2) {  // rows q, q+1 of column i
              if (i == q + 2 && q < q0) lt = s_hand[par ^ 1][0];
              rot_rows(lt, lb, g);
              HD(q + 1, i) = lb;  // final for this bubble; T[q][i] stays in a register
              lb = lt;
              lt = n_lt;
            }
            if (i < q - 1) {  // columns q, q+1 of row i
              rot_cols(rl, rr, g);
              HD(i, q + 1) = rr;
              if (i == q - 2) s_hand[par][1] = rl;  // T[q-2][q] for thread 0
              rr = rl;
              rl = n_rl;
            }
            rot_cols(zl, zr, g);
            ZD(i, q + 1) = zr;
            zr = zl;
            zl = n_zl;
          }
          __syncthreads();
        }
        if (owner) {  // the elements still held in registers
          if (i >= ks + 2) HD(ks, i) = lb;
          if (i < ks - 1) HD(i, ks) = rr;
          ZD(i, ks) = zr;
        }
        if (tid == 0) {
          s_sel[ks] = 1;
          s_sel[pos] = 0;
        }
        __syncthreads();
      }
      ++ks;
    }
  } else {
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
      const double2 ti = H[(long long)i * ld + i];
      const double ai = swi::cabs(make_double2(ti.x, ti.y - J.sig_im));
      int rank = 0;
      for (int q = 0; q < kk; ++q) {
        const double2 tq = H[(long long)q * ld + q];
        const double aq = swi::cabs(make_double2(tq.x, tq.y - J.sig_im));
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
