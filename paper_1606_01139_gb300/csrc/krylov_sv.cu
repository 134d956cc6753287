// Gram-Schmidt passes of the single-vector Krylov loop (Section 2.1: one new
// vector per window and step, as in the implicitly restarted Arnoldi method the
// paper runs), batched over the windows of one solve; the same passes serve
// windows that add a block of nb = 2 vectors per step (a template parameter:
// each pass still streams the basis once, for both new vectors).
//
// Every window keeps its basis row-major, Q [N][ld] (a grid point's basis
// coefficients are contiguous), so each pass of classical Gram-Schmidt against
// the new vectors w streams the basis once.  Classical Gram-Schmidt twice is
// three passes: the Gram (FP32 products of the heads), the update fused with
// the second Gram (the accurate pass), and the update by the second pass's
// small coefficients (FP32 products).  Two element types share the kernels
// through an arithmetic policy:
//  - complex64 with FP32 arithmetic (the reduced-precision form);
//  - complex128 in double-single arithmetic: every FP64 operand split into a
//    float head and tail from its bit fields, products exact up to their
//    tails (FMA), sums TwoSum-compensated, ~2^-46 relative per term (GB300's
//    FP64 rate would cap these passes near a third of the HBM bandwidth); the
//    new vectors themselves are kept in split form while they are
//    orthogonalised.
//
//  sv_gram_kernel:   part[chunk][i][b] = sum_{rows of chunk} conj(Q[r, i]) w[r, b]
//                    (a block per 32-column slab and row chunk, one column per lane)
//  sv_update_kernel: w[r, :] -= Q[r, :] c (a warp per row), then the next
//                    Gram's partials: one pass over Q for both (double-single)
//  sv_update_fast_kernel: w[r, :] -= Q[r, :] c for the second pass's small
//                    coefficients (FP32 products of the heads)
//  sv_wgram_kernel:  part[chunk][a][b] = sum_{rows of chunk} conj(w[r, a]) w[r, b]
//  sv_reduce_kernel: FP64 sums of the chunk partials, added into columns of H;
//                    for w^H w the Cholesky factor of the block (Cholesky-QR)
// Chunks hold at most 1024 rows: the per-lane FP32 (or double-single) partial
// sums stay short, chunks are combined in FP64.
#include <algorithm>

#include "ds.cuh"
#include "swi_internal.cuh"

namespace swi {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ----------------------------------------------------------------- arithmetic policies
// w^H w entries are accumulated in double-single (heads and error terms of the
// real and imaginary parts) by lane 0 of a warp, on the FP32 pipe
struct Gds {
  float rh, re, ih, ie;
};
__device__ __forceinline__ void gds_acc(Gds& a, float xrh, float xrl, float xih, float xil, float yrh, float yrl,
                                        float yih, float yil) {  // a += conj(x) y
  ds::fma_acc(a.rh, a.re, xrh, xrl, yrh, yrl);
  ds::fma_acc(a.rh, a.re, xih, xil, yih, yil);
  ds::fma_acc(a.ih, a.ie, xrh, xrl, yih, yil);
  ds::fma_acc(a.ih, a.ie, -xih, -xil, yrh, yrl);
}

struct PolC64 {
  using T = float2;   // basis element
  using A = float2;   // accumulator
  using S = float2;   // an element prepared for products (no split in FP32)
  __device__ static S split(T v) { return v; }
  __device__ static S bcast0(S v) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, 0), __shfl_sync(0xffffffffu, v.y, 0));
  }
  __device__ static void conj_mac_s(A& a, S q, S w) { conj_mac(a, q, w); }
  __device__ static void mac_s(A& a, S q, S c) { mac(a, q, c); }
  __device__ static A zero() { return make_float2(0.f, 0.f); }
  // a += conj(q) * w
  __device__ static void conj_mac(A& a, T q, T w) {
    a.x = fmaf(q.x, w.x, fmaf(q.y, w.y, a.x));
    a.y = fmaf(q.x, w.y, fmaf(-q.y, w.x, a.y));
  }
  // a += q * c
  __device__ static void mac(A& a, T q, T c) {
    a.x = fmaf(q.x, c.x, fmaf(-q.y, c.y, a.x));
    a.y = fmaf(q.x, c.y, fmaf(q.y, c.x, a.y));
  }
  __device__ static A add(A a, A b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static A shfl_xor(A a, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
  }
  __device__ static double2 to_d(A a) { return make_double2(a.x, a.y); }
  __device__ static T from_c(double2 c) { return make_float2((float)c.x, (float)c.y); }
  // the new vectors w: complex64, like the basis
  using W = float2;
  __device__ static S wload(W v) { return v; }
  __device__ static W wstore(S v) { return v; }
  __device__ static S wsub(S w, A d) { return make_float2(w.x - d.x, w.y - d.y); }
  __device__ static void gacc(Gds& g, S x, S y) { gds_acc(g, x.x, 0.f, x.y, 0.f, y.x, 0.f, y.y, 0.f); }
  __device__ static double2 wto_d(W v) { return make_double2(v.x, v.y); }
  __device__ static W wfrom_d(double2 v) { return make_float2((float)v.x, (float)v.y); }
  // the FP32 passes: the same arithmetic
  using F = float2;
  __device__ static F fzero() { return make_float2(0.f, 0.f); }
  __device__ static void fconj_mac(F& a, T q, S w) { conj_mac(a, q, w); }
  __device__ static F fadd(F a, F b) { return add(a, b); }
  __device__ static F fshfl_xor(F a, int o) { return shfl_xor(a, o); }
  __device__ static double2 fto_d(F a) { return to_d(a); }
  __device__ static A fto_A(F a) { return a; }
  __device__ static float2 head2(T c) { return c; }
  __device__ static void fmac2(F& a, T q, float2 c) { mac(a, q, c); }
};

// x = hi + lo from the bit fields alone (integer and FP32 pipes only): hi is x
// rounded to 24 significant bits, lo the remainder rounded to a float.  Values
// below 2^-74 split to (0, 0) and magnitudes are capped at 2^126: the basis
// entries, new vectors and coefficients of the loop lie far inside that range,
// and no FP64 instruction is issued (a predicated FP64 fallback would occupy
// GB300's narrow FP64 pipe on every element).
__device__ __forceinline__ float hi_fast(double x) {  // the head of split_fast alone
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int top = (unsigned int)(b >> 32);
  const int e0 = (int)((top >> 20) & 0x7ff);
  const int e = min(max(e0, 949), 1149);
  const unsigned int fb =
      ((unsigned int)(e - 896) << 23 | ((unsigned int)(b >> 29) & 0x7fffffu)) + ((unsigned int)(b >> 28) & 1u);
  return e0 < 949 ? 0.f : __uint_as_float((top & 0x80000000u) | fb);
}

__device__ __forceinline__ void split_fast(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int top = (unsigned int)(b >> 32);
  const unsigned int sgn = top & 0x80000000u;
  const int e0 = (int)((top >> 20) & 0x7ff);
  const bool small = e0 < 949;
  const int e = min(max(e0, 949), 1149);
  const unsigned int up = (unsigned int)(b >> 28) & 1u;
  const unsigned int fb = ((unsigned int)(e - 896) << 23 | ((unsigned int)(b >> 29) & 0x7fffffu)) + up;
  const int rem = (int)((unsigned int)b & 0x1fffffffu) - (int)(up << 29);
  const float t = (float)rem * __uint_as_float((unsigned int)(e - 948) << 23);
  hi = small ? 0.f : __uint_as_float(sgn | fb);
  lo = small ? 0.f : (sgn ? -t : t);
}

struct PolDs {
  using T = double2;
  struct A {
    float rh, re, ih, ie;
  };
  struct S {  // heads and tails of the real and imaginary parts
    float rh, rl, ih, il;
  };
  __device__ static S split(T v) {
    S o;
    split_fast(v.x, o.rh, o.rl);
    split_fast(v.y, o.ih, o.il);
    return o;
  }
  __device__ static S bcast0(S v) {
    return S{__shfl_sync(0xffffffffu, v.rh, 0), __shfl_sync(0xffffffffu, v.rl, 0), __shfl_sync(0xffffffffu, v.ih, 0),
             __shfl_sync(0xffffffffu, v.il, 0)};
  }
  // a += conj(q) * w
  __device__ static void conj_mac_s(A& a, const S& q, const S& w) {
    ds::fma_acc(a.rh, a.re, q.rh, q.rl, w.rh, w.rl);
    ds::fma_acc(a.rh, a.re, q.ih, q.il, w.ih, w.il);
    ds::fma_acc(a.ih, a.ie, q.rh, q.rl, w.ih, w.il);
    ds::fma_acc(a.ih, a.ie, -q.ih, -q.il, w.rh, w.rl);
  }
  // a += q * c
  __device__ static void mac_s(A& a, const S& q, const S& c) {
    ds::fma_acc(a.rh, a.re, q.rh, q.rl, c.rh, c.rl);
    ds::fma_acc(a.rh, a.re, -q.ih, -q.il, c.ih, c.il);
    ds::fma_acc(a.ih, a.ie, q.rh, q.rl, c.ih, c.il);
    ds::fma_acc(a.ih, a.ie, q.ih, q.il, c.rh, c.rl);
  }
  __device__ static A zero() { return A{0.f, 0.f, 0.f, 0.f}; }
  __device__ static A add(A a, A b) {
    const ds::df r = ds::two_sum(a.rh, b.rh);
    const ds::df i = ds::two_sum(a.ih, b.ih);
    return A{r.h, r.l + a.re + b.re, i.h, i.l + a.ie + b.ie};
  }
  __device__ static A shfl_xor(A a, int o) {
    return A{__shfl_xor_sync(0xffffffffu, a.rh, o), __shfl_xor_sync(0xffffffffu, a.re, o),
             __shfl_xor_sync(0xffffffffu, a.ih, o), __shfl_xor_sync(0xffffffffu, a.ie, o)};
  }
  __device__ static double2 to_d(A a) { return make_double2((double)a.rh + (double)a.re, (double)a.ih + (double)a.ie); }
  __device__ static T from_c(double2 c) { return c; }
  // the new vectors w: kept in split form (heads and tails as floats) while
  // they are orthogonalised, so that forming w - Q c takes no FP64 instruction
  using W = float4;
  __device__ static S wload(W v) { return S{v.x, v.y, v.z, v.w}; }
  __device__ static W wstore(S v) { return make_float4(v.rh, v.rl, v.ih, v.il); }
  __device__ static S wsub(S w, A d) {  // w - d, renormalised to head + tail
    const ds::df r = ds::add(ds::df{w.rh, w.rl}, ds::df{-d.rh, -d.re});
    const ds::df i = ds::add(ds::df{w.ih, w.il}, ds::df{-d.ih, -d.ie});
    return S{r.h, r.l, i.h, i.l};
  }
  __device__ static void gacc(Gds& g, S x, S y) { gds_acc(g, x.rh, x.rl, x.ih, x.il, y.rh, y.rl, y.ih, y.il); }
  __device__ static double2 wto_d(W v) { return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w); }
  __device__ static W wfrom_d(double2 v) {
    S o;
    split_fast(v.x, o.rh, o.rl);
    split_fast(v.y, o.ih, o.il);
    return wstore(o);
  }
  // the FP32 passes: products of the heads in FP32 (the first Gram of
  // classical Gram-Schmidt twice, and the update by the second pass's small
  // coefficients, need no more)
  using F = float2;
  __device__ static F fzero() { return make_float2(0.f, 0.f); }
  __device__ static void fconj_mac(F& a, T q, const S& w) {  // a += conj(q) w
    const float qr = hi_fast(q.x), qi = hi_fast(q.y);
    a.x = fmaf(qr, w.rh, fmaf(qi, w.ih, a.x));
    a.y = fmaf(qr, w.ih, fmaf(-qi, w.rh, a.y));
  }
  __device__ static F fadd(F a, F b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static F fshfl_xor(F a, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
  }
  __device__ static double2 fto_d(F a) { return make_double2(a.x, a.y); }
  __device__ static A fto_A(F a) { return A{a.x, 0.f, a.y, 0.f}; }
  __device__ static float2 head2(T c) { return make_float2(hi_fast(c.x), hi_fast(c.y)); }
  __device__ static void fmac2(F& a, T q, float2 c) {  // a += q c, FP32 products of the heads
    const float qr = hi_fast(q.x), qi = hi_fast(q.y);
    a.x = fmaf(qr, c.x, fmaf(-qi, c.y, a.x));
    a.y = fmaf(qr, c.y, fmaf(qi, c.x, a.y));
  }
};

// ----------------------------------------------------------------- Gram pass
template <class Pol, int NB, bool FAST>
__global__ void __launch_bounds__(kThreads) sv_gram_kernel(const __grid_constant__ SvBatch batch, int N, int rpc) {
  using T = typename Pol::T;
  using A = typename Pol::A;
  const SvJob& J = batch.job[blockIdx.z];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y * 32 + lane;
  if (blockIdx.y * 32 >= J.ncols) return;  // this job has fewer slabs (uniform over the block)
  using Wt = typename Pol::W;
  const T* __restrict__ Q = static_cast<const T*>(J.Q);
  const Wt* __restrict__ w = static_cast<const Wt*>(J.w);
  const int r0 = blockIdx.x * rpc, r1 = min(N, r0 + rpc);
  const bool on = col < J.ncols;
  __shared__ double2 red[kWarps][NB][32];
  int r = r0 + warp;
  if constexpr (FAST) {
    // four rows per iteration, their loads issued together (memory-level
    // parallelism), two interleaved accumulators per column of w
    typename Pol::F a0[NB], a1[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) a0[b] = a1[b] = Pol::fzero();
    for (; r + 3 * kWarps < r1; r += 4 * kWarps) {
      T q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = on ? __ldg(Q + (long long)(r + u * kWarps) * J.ldq + col) : T{};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int b = 0; b < NB; ++b)
          Pol::fconj_mac((u & 1) ? a1[b] : a0[b], q[u], Pol::wload(w[(long long)(r + u * kWarps) * J.ldw + b]));
    }
    for (; r < r1; r += kWarps) {
      const T q0 = on ? __ldg(Q + (long long)r * J.ldq + col) : T{};
#pragma unroll
      for (int b = 0; b < NB; ++b) Pol::fconj_mac(a0[b], q0, Pol::wload(w[(long long)r * J.ldw + b]));
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) red[warp][b][lane] = Pol::fto_d(Pol::fadd(a0[b], a1[b]));
  } else {
    A a0[NB], a1[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) a0[b] = a1[b] = Pol::zero();
    for (; r + kWarps < r1; r += 2 * kWarps) {
      const T q0 = on ? __ldg(Q + (long long)r * J.ldq + col) : T{};
      const T q1 = on ? __ldg(Q + (long long)(r + kWarps) * J.ldq + col) : T{};
      const auto s0 = Pol::split(q0), s1 = Pol::split(q1);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        Pol::conj_mac_s(a0[b], s0, Pol::wload(w[(long long)r * J.ldw + b]));
        Pol::conj_mac_s(a1[b], s1, Pol::wload(w[(long long)(r + kWarps) * J.ldw + b]));
      }
    }
    if (r < r1) {
      const auto s0 = Pol::split(on ? __ldg(Q + (long long)r * J.ldq + col) : T{});
#pragma unroll
      for (int b = 0; b < NB; ++b) Pol::conj_mac_s(a0[b], s0, Pol::wload(w[(long long)r * J.ldw + b]));
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) red[warp][b][lane] = Pol::to_d(Pol::add(a0[b], a1[b]));
  }
  __syncthreads();
  if (warp == 0 && on) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < kWarps; ++k) {
        s.x += red[k][b][lane].x;
        s.y += red[k][b][lane].y;
      }
      J.part[(long long)blockIdx.x * J.ldp + col * NB + b] = s;
    }
  }
}

// ----------------------------------------------------------------- update fused with the second Gram
// The accurate pass: w[r, :] -= Q[r, :] c, then the partials of Q^H w, in
// double-single.  A warp per row; lane l holds basis columns l, l + 32, ...
// (NT of them); the row's values are read twice (the second read hits L1)
// rather than held in registers, which keeps two blocks on an SM.
template <class Pol, int NT, int NB>
__global__ void __launch_bounds__(kThreads, (NT <= 8) ? 2 : 1) sv_update_kernel(const __grid_constant__ SvBatch batch, int N, int rpc) {
  using T = typename Pol::T;
  using A = typename Pol::A;
  using Sp = typename Pol::S;
  // shared: the coefficients c in split form, then the cross-warp partials
  extern __shared__ double2 sh[];
  const SvJob& J = batch.job[blockIdx.y];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncols = J.ncols;
  Sp* cs = reinterpret_cast<Sp*>(sh);
  double2* red = sh + (size_t)ncols * NB;
  // stored vector-major (cs[b * ncols + i]): a warp's lanes read consecutive
  // 16-byte entries, without bank conflicts
  for (int e = threadIdx.x; e < ncols * NB; e += kThreads) cs[(e % NB) * ncols + e / NB] = Pol::split(Pol::from_c(J.c[e]));
  __syncthreads();
  using Wt = typename Pol::W;
  const T* __restrict__ Q = static_cast<const T*>(J.Q);
  Wt* w = static_cast<Wt*>(J.w);
  const int r0 = blockIdx.x * rpc, r1 = min(N, r0 + rpc);
  A acc[NT][NB];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[t][b] = Pol::zero();
  for (int r = r0 + warp; r < r1; r += kWarps) {
    // Q[r, :] c, two interleaved accumulators per new vector (independent chains)
    A d[NB], d1[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) d[b] = d1[b] = Pol::zero();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      if (i < ncols) {
        const Sp qs = Pol::split(__ldg(Q + (long long)r * J.ldq + i));
#pragma unroll
        for (int b = 0; b < NB; ++b) Pol::mac_s((t & 1) ? d1[b] : d[b], qs, cs[b * ncols + i]);
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      d[b] = Pol::add(d[b], d1[b]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d[b] = Pol::add(d[b], Pol::shfl_xor(d[b], o));
    }
    // the row's new values are formed by lane 0 alone (FP32 instructions
    // only, in split form) and broadcast
    Sp ws[NB]{};
    if (lane == 0) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        ws[b] = Pol::wsub(Pol::wload(w[(long long)r * J.ldw + b]), d[b]);
        w[(long long)r * J.ldw + b] = Pol::wstore(ws[b]);
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) ws[b] = Pol::bcast0(ws[b]);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      if (i < ncols) {
        const Sp qs = Pol::split(__ldg(Q + (long long)r * J.ldq + i));
#pragma unroll
        for (int b = 0; b < NB; ++b) Pol::conj_mac_s(acc[t][b], qs, ws[b]);
      }
    }
  }
  double2* out = J.part + (long long)blockIdx.x * J.ldp;
  // cross-warp sums, one 32-column slab at a time: red [kWarps][NB][32]
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if (32 * t >= ncols) break;  // uniform over the block
#pragma unroll
    for (int b = 0; b < NB; ++b) red[(warp * NB + b) * 32 + lane] = Pol::to_d(acc[t][b]);
    __syncthreads();
    if (threadIdx.x < 32 * NB) {
      const int b = threadIdx.x >> 5, l = threadIdx.x & 31, i = l + 32 * t;
      if (i < ncols) {
        double2 s = make_double2(0.0, 0.0);
        for (int k = 0; k < kWarps; ++k) {
          s.x += red[(k * NB + b) * 32 + l].x;
          s.y += red[(k * NB + b) * 32 + l].y;
        }
        out[i * NB + b] = s;
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------- the second update (FP32 products)
// w[r, :] -= Q[r, :] c for the second pass's small coefficients: products of
// the basis heads in FP32, the row's new value formed in split form by lane 0;
// a warp per row, few registers so that four blocks share an SM.
template <class Pol, int NT, int NB>
__global__ void __launch_bounds__(kThreads, (NT <= 8) ? 4 : ((NT <= 12) ? 2 : 1)) sv_update_fast_kernel(const __grid_constant__ SvBatch batch, int N,
                                                                      int rpc) {
  using T = typename Pol::T;
  using F = typename Pol::F;
  using Sp = typename Pol::S;
  using Wt = typename Pol::W;
  extern __shared__ double2 sh[];
  const SvJob& J = batch.job[blockIdx.y];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncols = J.ncols;
  // the coefficients' heads, [NB][ncols] (8 bytes per entry: conflict-free reads)
  float2* cs = reinterpret_cast<float2*>(sh);
  for (int e = threadIdx.x; e < ncols * NB; e += kThreads) cs[(e % NB) * ncols + e / NB] = Pol::head2(Pol::from_c(J.c[e]));
  __syncthreads();
  const T* __restrict__ Q = static_cast<const T*>(J.Q);
  Wt* w = static_cast<Wt*>(J.w);
  const int r0 = blockIdx.x * rpc, r1 = min(N, r0 + rpc);
  constexpr int kRows = 1;
  for (int r = r0 + warp; r < r1; r += kRows * kWarps) {
    const int rb = r + kWarps;
    const bool two = kRows == 2 && rb < r1;
    T qa[NT], qb[kRows == 2 ? NT : 1];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      qa[t] = i < ncols ? __ldg(Q + (long long)r * J.ldq + i) : T{};
      if (kRows == 2) qb[kRows == 2 ? t : 0] = (two && i < ncols) ? __ldg(Q + (long long)rb * J.ldq + i) : T{};
    }
    F fa[NB], fb[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) fa[b] = fb[b] = Pol::fzero();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      if (i < ncols)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const float2 cv = cs[b * ncols + i];
          Pol::fmac2(fa[b], qa[t], cv);
          if (kRows == 2) Pol::fmac2(fb[b], qb[kRows == 2 ? t : 0], cv);
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        fa[b] = Pol::fadd(fa[b], Pol::fshfl_xor(fa[b], o));
        fb[b] = Pol::fadd(fb[b], Pol::fshfl_xor(fb[b], o));
      }
    if (lane == 0) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        w[(long long)r * J.ldw + b] = Pol::wstore(Pol::wsub(Pol::wload(w[(long long)r * J.ldw + b]), Pol::fto_A(fa[b])));
        if (two)
          w[(long long)rb * J.ldw + b] =
              Pol::wstore(Pol::wsub(Pol::wload(w[(long long)rb * J.ldw + b]), Pol::fto_A(fb[b])));
      }
    }
  }
}

// ----------------------------------------------------------------- w^H w of the new block
// A block per row chunk and job, a thread per row (strided): double-single
// products on every lane, FP64 sums across the block.
template <class Pol, int NB>
__global__ void __launch_bounds__(kThreads) sv_wgram_kernel(const __grid_constant__ SvBatch batch, int N, int rpc) {
  using Wt = typename Pol::W;
  const SvJob& J = batch.job[blockIdx.y];
  const Wt* __restrict__ w = static_cast<const Wt*>(J.w);
  const int r0 = blockIdx.x * rpc, r1 = min(N, r0 + rpc);
  Gds g[NB * NB];
#pragma unroll
  for (int e = 0; e < NB * NB; ++e) g[e] = Gds{0.f, 0.f, 0.f, 0.f};
  for (int r = r0 + threadIdx.x; r < r1; r += kThreads) {
    typename Pol::S v[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) v[b] = Pol::wload(w[(long long)r * J.ldw + b]);
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) Pol::gacc(g[a * NB + b], v[a], v[b]);
  }
  __shared__ double2 red[NB * NB][kThreads];
#pragma unroll
  for (int e = 0; e < NB * NB; ++e)
    red[e][threadIdx.x] = make_double2((double)g[e].rh + (double)g[e].re, (double)g[e].ih + (double)g[e].ie);
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
#pragma unroll
      for (int e = 0; e < NB * NB; ++e) {
        red[e][threadIdx.x].x += red[e][threadIdx.x + st].x;
        red[e][threadIdx.x].y += red[e][threadIdx.x + st].y;
      }
    __syncthreads();
  }
  if (threadIdx.x < NB * NB) J.part[(long long)blockIdx.x * J.ldp + threadIdx.x] = red[threadIdx.x][0];
}

// ----------------------------------------------------------------- chunk reduction
// A block per 32 entries and job; 32 lanes per entry step through the chunks
// (independent loads in flight), then combine in shared memory.
constexpr int kRedLanes = 32;

// upper Cholesky factor R of the Hermitian nb x nb matrix G (G = R^H R), its
// inverse, and whether a pivot fell below 1e-14 of its diagonal entry
__device__ bool chol_small(const double2* G, int nb, double2* R, double2* Ri) {
  bool bad = false;
  for (int e = 0; e < 4; ++e) R[e] = Ri[e] = make_double2(0.0, 0.0);
  const double g00 = G[0].x;
  if (!(g00 > 0.0)) return true;
  const double r00 = sqrt(g00);
  R[0] = make_double2(r00, 0.0);
  Ri[0] = make_double2(1.0 / r00, 0.0);
  if (nb == 1) return false;
  const double2 r01 = make_double2(G[1].x / r00, G[1].y / r00);
  const double d = G[3].x - (r01.x * r01.x + r01.y * r01.y);
  if (!(d > 1e-14 * G[3].x)) {
    bad = true;
  }
  const double r11 = d > 0.0 ? sqrt(d) : 0.0;
  R[1] = r01;
  R[3] = make_double2(r11, 0.0);
  if (r11 > 0.0) {
    Ri[1] = make_double2(-r01.x / (r00 * r11), -r01.y / (r00 * r11));
    Ri[3] = make_double2(1.0 / r11, 0.0);
  }
  return bad;
}

__global__ void __launch_bounds__(32 * kRedLanes) sv_reduce_kernel(const __grid_constant__ SvReduceBatch batch) {
  const SvReduceJob& J = batch.job[blockIdx.y];
  const int cl = threadIdx.x & 31, k = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + cl;
  const int nent = J.mode == 0 ? J.ncols * J.nb : J.nb * J.nb;
  if (blockIdx.x * 32 >= nent) return;  // uniform over the block
  double2 a0 = make_double2(0.0, 0.0), a1 = a0;
  if (i < nent) {
    int ch = k;
    for (; ch + kRedLanes < J.nchunks; ch += 2 * kRedLanes) {
      const double2 v0 = J.part[(long long)ch * J.ldp + i];
      const double2 v1 = J.part[(long long)(ch + kRedLanes) * J.ldp + i];
      a0.x += v0.x;
      a0.y += v0.y;
      a1.x += v1.x;
      a1.y += v1.y;
    }
    if (ch < J.nchunks) {
      const double2 v0 = J.part[(long long)ch * J.ldp + i];
      a0.x += v0.x;
      a0.y += v0.y;
    }
  }
  __shared__ double2 red[kRedLanes][32];
  __shared__ double2 fin[4];
  red[k][cl] = make_double2(a0.x + a1.x, a0.y + a1.y);
  __syncthreads();
  if (k == 0 && i < nent) {
    double2 s = make_double2(0.0, 0.0);
#pragma unroll 8
    for (int q = 0; q < kRedLanes; ++q) {
      s.x += red[q][cl].x;
      s.y += red[q][cl].y;
    }
    if (J.mode == 0) {
      if (J.C) J.C[i] = s;
      if (J.H) {
        double2* h = J.H + (long long)(i / J.nb) * J.ldh + i % J.nb;
        *h = make_double2(h->x + s.x, h->y + s.y);
      }
    } else {
      fin[i] = s;
    }
  }
  if (J.mode == 0) return;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double2 R[4], Ri[4];
  const bool bad = chol_small(fin, J.nb, R, Ri);
  const int nb = J.nb;
  if (J.mode == 1) {
    for (int e = 0; e < nb * nb; ++e) {
      J.r[e] = Ri[e];
      J.r[4 + e] = R[e];
    }
    if (nb == 1 && J.H) J.H[0] = R[0];
  } else {
    // R = R2 R1 (both upper triangular, nb = 2)
    const double2* R1 = J.r + 4;
    for (int e = 0; e < 4; ++e) J.r[e] = Ri[e];
    if (J.H) {
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          double2 s = make_double2(0.0, 0.0);
          for (int q = 0; q < 2; ++q) {
            const double2 x = R[a * 2 + q], y = R1[q * 2 + b];
            s.x += x.x * y.x - x.y * y.y;
            s.y += x.x * y.y + x.y * y.x;
          }
          J.H[(long long)a * J.ldh + b] = s;
        }
    }
  }
  if (bad) J.r[8] = make_double2(1.0, 0.0);
}

// ----------------------------------------------------------------- normalisation
template <class Pol, int NB>
__global__ void sv_normalize_kernel(const __grid_constant__ SvNormBatch batch, int N) {
  using T = typename Pol::T;
  using Wt = typename Pol::W;
  const SvNormJob& J = batch.job[blockIdx.y];
  double2 r[NB * NB];
#pragma unroll
  for (int e = 0; e < NB * NB; ++e) r[e] = J.r[e];
  const Wt* w = static_cast<const Wt*>(J.w);
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < N;
       row += (long long)gridDim.x * blockDim.x) {
    double2 v[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) v[a] = Pol::wto_d(w[row * J.ldw + a]);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        re += v[a].x * r[a * NB + b].x - v[a].y * r[a * NB + b].y;
        im += v[a].x * r[a * NB + b].y + v[a].y * r[a * NB + b].x;
      }
      if (J.out_w) {
        static_cast<Wt*>(J.dst1)[row * J.ld1 + b] = Pol::wfrom_d(make_double2(re, im));
      } else {
        T o;
        o.x = (decltype(o.x))re;
        o.y = (decltype(o.y))im;
        static_cast<T*>(J.dst1)[row * J.ld1 + b] = o;
        if (J.dst2) static_cast<T*>(J.dst2)[row * J.ld2 + b] = o;
      }
    }
  }
}

// FUSE: the accurate pass (update + second Gram), else the FP32 second update
template <class Pol, int NT, int NB, bool FUSE>
void launch_update_nt(const SvBatch& b, int N, int rpc, int maxcols, cudaStream_t s) {
  const int nchunks = (N + rpc - 1) / rpc;
  if constexpr (!FUSE) {
    const size_t smem = sizeof(double2) * (size_t)maxcols * NB;
    if (smem > 48 * 1024)
      SWI_CUDA_TRY(cudaFuncSetAttribute(sv_update_fast_kernel<Pol, NT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    sv_update_fast_kernel<Pol, NT, NB><<<dim3(nchunks, b.n), kThreads, smem, s>>>(b, N, rpc);
  } else {
    const size_t smem = sizeof(double2) * ((size_t)maxcols * NB + (size_t)kWarps * NB * 32);
    if (smem > 48 * 1024)
      SWI_CUDA_TRY(cudaFuncSetAttribute(sv_update_kernel<Pol, NT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    sv_update_kernel<Pol, NT, NB><<<dim3(nchunks, b.n), kThreads, smem, s>>>(b, N, rpc);
  }
}

template <class Pol, int NB, bool FUSE>
void launch_update(const SvBatch& b, int N, int rpc, int maxcols, cudaStream_t s) {
  if (maxcols <= 64) launch_update_nt<Pol, 2, NB, FUSE>(b, N, rpc, maxcols, s);
  else if (maxcols <= 128) launch_update_nt<Pol, 4, NB, FUSE>(b, N, rpc, maxcols, s);
  else if (maxcols <= 256) launch_update_nt<Pol, 8, NB, FUSE>(b, N, rpc, maxcols, s);
  else if (maxcols <= 384) launch_update_nt<Pol, 12, NB, FUSE>(b, N, rpc, maxcols, s);
  else if (maxcols <= 512) launch_update_nt<Pol, 16, NB, FUSE>(b, N, rpc, maxcols, s);
  else if constexpr (NB == 1) launch_update_nt<Pol, 32, NB, FUSE>(b, N, rpc, maxcols, s);
  else throw Error{SWI_EINVAL, "Gram-Schmidt pass: at most 512 basis columns with 2-vector blocks"};
}

template <class Pol, int NB>
void launch_pass_nb(const SvBatch& b, int mode, int N, int rpc, int maxcols, cudaStream_t s) {
  const int nchunks = (N + rpc - 1) / rpc;
  if (mode == SV_GRAM) {
    const dim3 grid(nchunks, (maxcols + 31) / 32, b.n);
    sv_gram_kernel<Pol, NB, true><<<grid, kThreads, 0, s>>>(b, N, rpc);
  } else if (mode == SV_UPDATE_GRAM) {
    launch_update<Pol, NB, true>(b, N, rpc, maxcols, s);
  } else if (mode == SV_UPDATE) {
    launch_update<Pol, NB, false>(b, N, rpc, maxcols, s);
  } else {
    sv_wgram_kernel<Pol, NB><<<dim3(nchunks, b.n), kThreads, 0, s>>>(b, N, rpc);
  }
}

}  // namespace

int sv_rows_per_chunk(int N, int njobs) {
  // enough row chunks for about eight blocks per SM over the jobs, at most
  // 1024 rows per chunk (the bound on the per-lane partial sums)
  const long long target = 8LL * 152;
  long long per = (long long)N * std::max(njobs, 1) / target;
  per = std::max<long long>(256, std::min<long long>(1024, per));
  return (int)((per + 7) / 8 * 8);
}

void launch_sv_pass(const SvBatch& b, int mode, bool ds, int nb, int N, int rpc, cudaStream_t s,
                    long long* launches) {
  if (b.n <= 0) return;
  if (nb != 1 && nb != 2) throw Error{SWI_EINVAL, "Gram-Schmidt pass: blocks of 1 or 2 vectors"};
  int maxcols = 0;
  for (int q = 0; q < b.n; ++q) {
    const int nc = b.job[q].ncols;
    if (nc > 1024 || (mode != SV_WGRAM && nc < 1))
      throw Error{SWI_EINVAL, "Gram-Schmidt pass: 1..1024 basis columns"};
    maxcols = std::max(maxcols, nc);
  }
  if (rpc < 8 || rpc > 1024) throw Error{SWI_EINVAL, "Gram-Schmidt pass: rows per chunk out of range"};
  if (ds) {
    if (nb == 1) launch_pass_nb<PolDs, 1>(b, mode, N, rpc, maxcols, s);
    else launch_pass_nb<PolDs, 2>(b, mode, N, rpc, maxcols, s);
  } else {
    if (nb == 1) launch_pass_nb<PolC64, 1>(b, mode, N, rpc, maxcols, s);
    else launch_pass_nb<PolC64, 2>(b, mode, N, rpc, maxcols, s);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_sv_reduce(const SvReduceBatch& b, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  int maxent = 1;
  for (int q = 0; q < b.n; ++q) {
    const SvReduceJob& J = b.job[q];
    if (J.nb != 1 && J.nb != 2) throw Error{SWI_EINVAL, "chunk reduction: blocks of 1 or 2 vectors"};
    if (J.mode != 0 && J.r == nullptr) throw Error{SWI_EINVAL, "chunk reduction: Cholesky output missing"};
    if (J.mode == 2 && J.nb != 2) throw Error{SWI_EINVAL, "chunk reduction: second Cholesky pass needs nb = 2"};
    maxent = std::max(maxent, J.mode == 0 ? J.ncols * J.nb : J.nb * J.nb);
  }
  sv_reduce_kernel<<<dim3((maxent + 31) / 32, b.n), 32 * kRedLanes, 0, s>>>(b);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_sv_normalize(const SvNormBatch& b, bool ds, int nb, int N, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  if (nb != 1 && nb != 2) throw Error{SWI_EINVAL, "normalisation: blocks of 1 or 2 vectors"};
  const int blocks = std::min((N + 255) / 256, 1024);
  const dim3 grid(blocks, b.n);
  if (ds) {
    if (nb == 1) sv_normalize_kernel<PolDs, 1><<<grid, 256, 0, s>>>(b, N);
    else sv_normalize_kernel<PolDs, 2><<<grid, 256, 0, s>>>(b, N);
  } else {
    if (nb == 1) sv_normalize_kernel<PolC64, 1><<<grid, 256, 0, s>>>(b, N);
    else sv_normalize_kernel<PolC64, 2><<<grid, 256, 0, s>>>(b, N);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
