// Gram-Schmidt passes of the single-vector Krylov loop (Section 2.1: one new
// vector per window and step, as in the implicitly restarted Arnoldi method the
// paper runs), batched over the windows of one solve.
//
// Every window keeps its basis row-major, Q [N][ld] (a grid point's basis
// coefficients are contiguous), so each pass of classical Gram-Schmidt against
// the single new vector w streams the basis once (HBM-bound).  Two element
// types share the kernels through an arithmetic policy:
//  - complex64 with FP32 arithmetic (the reduced-precision form);
//  - complex128 in double-single arithmetic: every FP64 operand split into a
//    float head and tail from its bit fields, products exact up to their
//    tails (FMA), sums TwoSum-compensated, ~2^-46 relative per term (GB300's
//    FP64 rate would cap these passes near a third of the HBM bandwidth).
//
//  sv_gram_kernel:   part[chunk][i] = sum_{rows of chunk} conj(Q[r, i]) w[r]
//                    (a block per 32-column slab and row chunk, one column per lane)
//  sv_update_kernel: w[r] -= Q[r, :] c (a warp per row), then either the next
//                    Gram's partials (FUSE_GRAM, the row's values reused from
//                    registers: one read of Q for both passes) or ||w||^2
//  sv_reduce_kernel: FP64 sums of the chunk partials, added into a column of H
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
struct PolC64 {
  using T = float2;   // basis element
  using A = float2;   // accumulator
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
  __device__ static T sub(T w, A d) { return make_float2(w.x - d.x, w.y - d.y); }
  __device__ static T from_c(double2 c) { return make_float2((float)c.x, (float)c.y); }
  __device__ static double abs2(T w) { return (double)w.x * w.x + (double)w.y * w.y; }
};

struct PolDs {
  using T = double2;
  struct A {
    float rh, re, ih, ie;
  };
  __device__ static A zero() { return A{0.f, 0.f, 0.f, 0.f}; }
  __device__ static void conj_mac(A& a, T q, T w) {
    float qrh, qrl, qih, qil, wrh, wrl, wih, wil;
    ds::split_bits(q.x, qrh, qrl);
    ds::split_bits(q.y, qih, qil);
    ds::split_bits(w.x, wrh, wrl);
    ds::split_bits(w.y, wih, wil);
    ds::fma_acc(a.rh, a.re, qrh, qrl, wrh, wrl);
    ds::fma_acc(a.rh, a.re, qih, qil, wih, wil);
    ds::fma_acc(a.ih, a.ie, qrh, qrl, wih, wil);
    ds::fma_acc(a.ih, a.ie, -qih, -qil, wrh, wrl);
  }
  __device__ static void mac(A& a, T q, T c) {
    float qrh, qrl, qih, qil, crh, crl, cih, cil;
    ds::split_bits(q.x, qrh, qrl);
    ds::split_bits(q.y, qih, qil);
    ds::split_bits(c.x, crh, crl);
    ds::split_bits(c.y, cih, cil);
    ds::fma_acc(a.rh, a.re, qrh, qrl, crh, crl);
    ds::fma_acc(a.rh, a.re, -qih, -qil, cih, cil);
    ds::fma_acc(a.ih, a.ie, qrh, qrl, cih, cil);
    ds::fma_acc(a.ih, a.ie, qih, qil, crh, crl);
  }
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
  __device__ static T sub(T w, A d) {
    const double2 dd = to_d(d);
    return make_double2(w.x - dd.x, w.y - dd.y);
  }
  __device__ static T from_c(double2 c) { return c; }
  __device__ static double abs2(T w) { return fma(w.x, w.x, w.y * w.y); }
};

// ----------------------------------------------------------------- Gram pass
template <class Pol>
__global__ void __launch_bounds__(kThreads) sv_gram_kernel(const __grid_constant__ SvBatch batch, int N, int rpc) {
  using T = typename Pol::T;
  using A = typename Pol::A;
  const SvJob& J = batch.job[blockIdx.z];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y * 32 + lane;
  if (blockIdx.y * 32 >= J.ncols) return;  // this job has fewer slabs (uniform over the block)
  const T* __restrict__ Q = static_cast<const T*>(J.Q);
  const T* __restrict__ w = static_cast<const T*>(J.w);
  const int r0 = blockIdx.x * rpc, r1 = min(N, r0 + rpc);
  const bool on = col < J.ncols;
  // two interleaved accumulators per lane for instruction-level parallelism
  A a0 = Pol::zero(), a1 = Pol::zero();
  int r = r0 + warp;
  for (; r + kWarps < r1; r += 2 * kWarps) {
    const T q0 = on ? __ldg(Q + (long long)r * J.ldq + col) : T{};
    const T q1 = on ? __ldg(Q + (long long)(r + kWarps) * J.ldq + col) : T{};
    const T w0 = w[(long long)r * J.ldw], w1 = w[(long long)(r + kWarps) * J.ldw];
    Pol::conj_mac(a0, q0, w0);
    Pol::conj_mac(a1, q1, w1);
  }
  if (r < r1) {
    const T q0 = on ? __ldg(Q + (long long)r * J.ldq + col) : T{};
    Pol::conj_mac(a0, q0, w[(long long)r * J.ldw]);
  }
  __shared__ double2 red[kWarps][32];
  red[warp][lane] = Pol::to_d(Pol::add(a0, a1));
  __syncthreads();
  if (warp == 0 && on) {
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      s.x += red[k][lane].x;
      s.y += red[k][lane].y;
    }
    J.part[(long long)blockIdx.x * J.ldp + col] = s;
  }
}

// ----------------------------------------------------------------- update pass (+ Gram or norm)
// A warp per row; lane l holds columns l, l + 32, ... (NT of them, the row's
// values kept in registers for the fused Gram).
template <class Pol, int NT, bool FUSE_GRAM>
__global__ void __launch_bounds__(kThreads) sv_update_kernel(const __grid_constant__ SvBatch batch, int N, int rpc) {
  using T = typename Pol::T;
  using A = typename Pol::A;
  extern __shared__ double2 sh[];  // Gram partials [kWarps][ncols], then the coefficients c [ncols]
  const SvJob& J = batch.job[blockIdx.y];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncols = J.ncols;
  double2* red = sh;
  T* cs = reinterpret_cast<T*>(sh + (FUSE_GRAM ? kWarps * ncols : kWarps));
  for (int i = threadIdx.x; i < ncols; i += kThreads) cs[i] = Pol::from_c(J.c[i]);
  __syncthreads();
  const T* __restrict__ Q = static_cast<const T*>(J.Q);
  T* w = static_cast<T*>(J.w);
  const int r0 = blockIdx.x * rpc, r1 = min(N, r0 + rpc);
  A acc[FUSE_GRAM ? NT : 1];
#pragma unroll
  for (int t = 0; t < (FUSE_GRAM ? NT : 1); ++t) acc[t] = Pol::zero();
  double nrm = 0.0;
  for (int r = r0 + warp; r < r1; r += kWarps) {
    T q[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      q[t] = i < ncols ? __ldg(Q + (long long)r * J.ldq + i) : T{};
    }
    A d = Pol::zero();
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      if (i < ncols) Pol::mac(d, q[t], cs[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = Pol::add(d, Pol::shfl_xor(d, o));
    const T wv = Pol::sub(w[(long long)r * J.ldw], d);
    if (lane == 0) w[(long long)r * J.ldw] = wv;
    if (FUSE_GRAM) {
#pragma unroll
      for (int t = 0; t < NT; ++t) Pol::conj_mac(acc[FUSE_GRAM ? t : 0], q[t], wv);
    } else {
      nrm += Pol::abs2(wv);
    }
  }
  double2* out = J.part + (long long)blockIdx.x * J.ldp;
  if (!FUSE_GRAM) {
    if (lane == 0) red[warp] = make_double2(nrm, 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < kWarps; ++k) s += red[k].x;
      out[0] = make_double2(s, 0.0);
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int i = lane + 32 * t;
    if (i < ncols) red[warp * ncols + i] = Pol::to_d(acc[FUSE_GRAM ? t : 0]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ncols; i += kThreads) {
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < kWarps; ++k) {
      s.x += red[k * ncols + i].x;
      s.y += red[k * ncols + i].y;
    }
    out[i] = s;
  }
}

// ----------------------------------------------------------------- chunk reduction
// A block per 32 columns and job; 8 lanes per column step through the chunks
// (independent loads in flight), then combine in shared memory.
__global__ void sv_reduce_kernel(const __grid_constant__ SvReduceBatch batch) {
  const SvReduceJob& J = batch.job[blockIdx.y];
  const int cl = threadIdx.x & 31, k = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + cl;
  const int ncols = J.mode == 1 ? 1 : J.ncols;
  if (blockIdx.x * 32 >= ncols) return;
  double2 a = make_double2(0.0, 0.0);
  if (i < ncols)
    for (int ch = k; ch < J.nchunks; ch += 8) {
      const double2 v = J.part[(long long)ch * J.ldp + i];
      a.x += v.x;
      a.y += v.y;
    }
  __shared__ double2 red[8][32];
  red[k][cl] = a;
  __syncthreads();
  if (k != 0 || i >= ncols) return;
  double2 s = make_double2(0.0, 0.0);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    s.x += red[q][cl].x;
    s.y += red[q][cl].y;
  }
  if (J.mode == 1) {
    const double beta = sqrt(s.x);
    if (J.H) J.H[0] = make_double2(beta, 0.0);
    if (J.invb) *J.invb = beta > 0.0 ? 1.0 / beta : 0.0;
    return;
  }
  if (J.C) J.C[i] = s;
  if (J.H) {
    double2* h = J.H + (long long)i * J.ldh;
    *h = make_double2(h->x + s.x, h->y + s.y);
  }
}

// ----------------------------------------------------------------- normalisation
template <class T>
__global__ void sv_normalize_kernel(const __grid_constant__ SvNormBatch batch, int N) {
  const SvNormJob& J = batch.job[blockIdx.y];
  const double s = *J.invb;
  const T* w = static_cast<const T*>(J.w);
  T* d1 = static_cast<T*>(J.dst1);
  T* d2 = static_cast<T*>(J.dst2);
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    const T v = w[r * J.ldw];
    T o;
    o.x = (decltype(v.x))(v.x * s);
    o.y = (decltype(v.y))(v.y * s);
    d1[r * J.ld1] = o;
    if (d2) d2[r * J.ld2] = o;
  }
}

template <class Pol, int NT, bool FUSE>
void launch_update_nt(const SvBatch& b, int N, int rpc, int maxcols, cudaStream_t s) {
  const int nchunks = (N + rpc - 1) / rpc;
  const size_t smem = sizeof(double2) * ((FUSE ? (size_t)kWarps * maxcols : kWarps) + maxcols);
  if (smem > 48 * 1024)
    SWI_CUDA_TRY(cudaFuncSetAttribute(sv_update_kernel<Pol, NT, FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  sv_update_kernel<Pol, NT, FUSE><<<dim3(nchunks, b.n), kThreads, smem, s>>>(b, N, rpc);
}

template <class Pol, bool FUSE>
void launch_update(const SvBatch& b, int N, int rpc, int maxcols, cudaStream_t s) {
  if (maxcols <= 64) launch_update_nt<Pol, 2, FUSE>(b, N, rpc, maxcols, s);
  else if (maxcols <= 128) launch_update_nt<Pol, 4, FUSE>(b, N, rpc, maxcols, s);
  else if (maxcols <= 256) launch_update_nt<Pol, 8, FUSE>(b, N, rpc, maxcols, s);
  else if (maxcols <= 512) launch_update_nt<Pol, 16, FUSE>(b, N, rpc, maxcols, s);
  else launch_update_nt<Pol, 32, FUSE>(b, N, rpc, maxcols, s);
}

}  // namespace

int sv_rows_per_chunk(int N, int njobs) {
  // enough row chunks for about eight blocks per SM over the jobs, at most
  // 1024 rows per chunk (the bound on the per-lane partial sums)
  const long long target = 8LL * 152;
  long long per = (long long)N * std::max(njobs, 1) / target;
  per = std::max<long long>(64, std::min<long long>(1024, per));
  return (int)((per + 7) / 8 * 8);
}

void launch_sv_pass(const SvBatch& b, int mode, bool ds, int N, int rpc, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  int maxcols = 0;
  for (int q = 0; q < b.n; ++q) {
    if (b.job[q].ncols > 1024 || b.job[q].ncols < 1) throw Error{SWI_EINVAL, "Gram-Schmidt pass: 1..1024 columns"};
    maxcols = std::max(maxcols, b.job[q].ncols);
  }
  if (rpc < 8 || rpc > 1024) throw Error{SWI_EINVAL, "Gram-Schmidt pass: rows per chunk out of range"};
  const int nchunks = (N + rpc - 1) / rpc;
  if (mode == SV_GRAM) {
    const dim3 grid(nchunks, (maxcols + 31) / 32, b.n);
    if (ds) sv_gram_kernel<PolDs><<<grid, kThreads, 0, s>>>(b, N, rpc);
    else sv_gram_kernel<PolC64><<<grid, kThreads, 0, s>>>(b, N, rpc);
  } else if (mode == SV_UPDATE_GRAM) {
    if (ds) launch_update<PolDs, true>(b, N, rpc, maxcols, s);
    else launch_update<PolC64, true>(b, N, rpc, maxcols, s);
  } else {
    if (ds) launch_update<PolDs, false>(b, N, rpc, maxcols, s);
    else launch_update<PolC64, false>(b, N, rpc, maxcols, s);
  }
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_sv_reduce(const SvReduceBatch& b, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  int maxcols = 1;
  for (int q = 0; q < b.n; ++q) maxcols = std::max(maxcols, b.job[q].mode == 1 ? 1 : b.job[q].ncols);
  sv_reduce_kernel<<<dim3((maxcols + 31) / 32, b.n), 256, 0, s>>>(b);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

void launch_sv_normalize(const SvNormBatch& b, bool ds, int N, cudaStream_t s, long long* launches) {
  if (b.n <= 0) return;
  const int blocks = std::min((N + 255) / 256, 1024);
  if (ds) sv_normalize_kernel<double2><<<dim3(blocks, b.n), 256, 0, s>>>(b, N);
  else sv_normalize_kernel<float2><<<dim3(blocks, b.n), 256, 0, s>>>(b, N);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
