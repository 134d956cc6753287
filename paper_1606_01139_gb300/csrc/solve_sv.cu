// The windowed solve with single-vector windows (block width 1) or windows
// of 2-vector blocks.
//
// Each window j runs the Krylov-Schur iteration on the shifted, never-inverted
// operator A - sigma_j (Eq. 3) with the 'SM' selection: the exact-shift thick
// restart that ARPACK's implicitly restarted Arnoldi method performs (Section
// 2.1), nb = 1 or 2 new basis vectors per window and step.  A single starting
// vector spans only one vector of each eigenspace, so eigenvalues of
// multiplicity two (a wire whose cross-section and potential share a symmetry)
// need nb = 2 to converge both partners.  All windows step in lockstep: one
// stencil launch applies A - sigma_j to the newest vectors of every window,
// and each Gram-Schmidt pass (classical, twice) is one launch over all windows
// that streams every basis once; a 2-vector block is then orthonormalised by
// Cholesky-QR, twice.  A window whose basis is full runs its projected
// eigenproblem (schur_ds.cu) on a stream of its own while the others keep
// expanding, then rotates its basis to the kept Schur vectors.
//
// Two arithmetics share this driver:
//  - complex128 bases, double-single products and stencil (krylov_sv.cu,
//    stencil_ds.cu): the FP64 method, pairs to FP64-class residuals;
//  - complex64 bases, FP32 products and stencil (krylov_sv.cu, krylov_c64.cu,
//    stencil_c64_tma.cu): the reduced-precision form of SWI_PREC_MIXED
//    contexts, whose pairs are widened to complex128 for the merge and checked
//    by the same FP64 residuals (their accuracy is that of FP32 arithmetic, so
//    Algorithm 2's equal-eigenvalue and redundancy tests default to 1e-5 and
//    1e-2 there).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "host.cuh"
#include "merge.cuh"
#include "swi_internal.cuh"

namespace swi {
namespace host {

namespace {

template <bool DS>
struct SV {
  using T = std::conditional_t<DS, double2, float2>;
  using Sig = std::conditional_t<DS, double, float>;
};

template <bool DS>
struct SvWin {
  using T = typename SV<DS>::T;
  double sigma = 0.0;  // the shift the stencil applies (rounded to FP32 in the complex64 form)
  double sig_im = 0.0; // imaginary part of a complex shift (applied by the selection only)
  int nreq = 0, m = 0, keep = 0, ldq = 0, ldh = 0, col = 0;
  int p = 0;  // the newest block is basis columns [p, p + nb) (the ones expanded next)
  DevMem Q, H, Z, S, Bz, theta, resid, Yw, eps_w, res_w, Hw, Zw, C1, C2, Z32, rinv, part;  // part: FP64 chunk partials
  DevMem Hsave;          // the projected matrix of the Schur step in flight (for a retry in FP64)
  bool retry = false;    // the double-single step gave up; the FP64 step runs on the saved matrix
  int schur_retries = 0;
  bool done = false, failed = false;
  long long matvecs = 0;
  int restarts = 0, nconv = 0;
};

// H <- [[T_kk, 0], [Bz, 0]]: keep the leading kk x kk Schur block, put the nb
// coupling rows Bz = B Z[:, 0:kk] ([nb][ldh]) below it, clear the rest of the
// (n x n) array.
__global__ void restart_h_kernel(double2* H, int ldh, int n, int kk, int nb, const double2* Bz) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (i < kk && j < kk) return;
  H[(long long)i * ldh + j] =
      (i >= kk && i < kk + nb && j < kk) ? Bz[(long long)(i - kk) * ldh + j] : make_double2(0.0, 0.0);
}

void launch_restart_h(double2* H, int ldh, int n, int kk, int nb, const double2* Bz, cudaStream_t s,
                      long long* launches) {
  const long long e = (long long)n * n;
  restart_h_kernel<<<(unsigned)((e + 255) / 256), 256, 0, s>>>(H, ldh, n, kk, nb, Bz);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

// a random start vector in the split form of the double-single loop (heads and
// tails of the real and imaginary parts as floats)
__global__ void random_col_ds_kernel(float4* __restrict__ dst, int ld, int rows, unsigned long long seed) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (2 * r + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    unsigned long long y = seed + 0x9E3779B97F4A7C15ull * (2 * r + 2);
    y = (y ^ (y >> 30)) * 0xBF58476D1CE4E5B9ull;
    y = (y ^ (y >> 27)) * 0x94D049BB133111EBull;
    y ^= y >> 31;
    const double re = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    const double im = (double)(y >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    const float rh = __double2float_rn(re), ih = __double2float_rn(im);
    dst[r * ld] = make_float4(rh, __double2float_rn(re - rh), ih, __double2float_rn(im - ih));
  }
}

swi::StencilC64Params stencil_c64_params(const swi_ctx* c) {
  swi::StencilC64Params P;
  P.nx = c->nx;
  P.ny = c->ny;
  P.nz = c->nz;
  P.bc = c->bc;
  for (int m = 0; m < 7; ++m) P.cm[m] = (float)(-kFD[m] / (2.0 * c->h * c->h));
  P.V = c->V32.as<float>();
  P.G = c->G32.as<float>();
  P.VG = c->VG32.as<float2>();
  return P;
}

template <bool DS>
swi_status solve_sv(swi_ctx* c, const swi_solve_opts& opt, swi_solve_info* info) {
  using Tr = SV<DS>;
  using T = typename Tr::T;
  using Win = SvWin<DS>;
  const int nb = opt.block > 0 ? opt.block : 1;
  if (nb != 1 && nb != 2) return fail(c, SWI_EINVAL, "single-vector windows: blocks of 1 or 2 vectors");
  const double rel_tol = opt.rel_tol > 0 ? opt.rel_tol : 1e-10;
  const double eq_rtol = opt.eq_rtol > 0 ? opt.eq_rtol : (DS ? 1e-8 : 1e-5);
  const double drop_tol = opt.drop_tol > 0 ? opt.drop_tol : (DS ? 1e-6 : 1e-2);
  const long long budget = opt.max_matvecs > 0 ? opt.max_matvecs : 2000000LL;
  const unsigned long long seed = opt.seed ? opt.seed : 1ull;
  const double anorm = gershgorin(c);
  const int nwin = (int)c->sigma.size();
  if (nwin > swi::kMaxBatch) return fail(c, SWI_EINVAL, "at most 64 windows per solve");
  c->arith = SWI_ARITH_DS;
  if (!DS) swi::stencil_c64_tma_error(true);
  const double t0 = swi::now_seconds();
  const size_t N = c->N;
  const int max_basis = nb == 1 ? 1000 : 510;

  std::vector<std::unique_ptr<Win>> win(nwin);
  size_t total_out = 0;
  int max_m = 1;
  for (int j = 0; j < nwin; ++j) {
    win[j].reset(new Win());
    Win& w = *win[j];
    w.sigma = DS ? c->sigma[j] : (double)(float)c->sigma[j];
    w.sig_im = c->sigma_im.size() == c->sigma.size() ? c->sigma_im[j] : 0.0;
    w.nreq = c->nreq[j];
    w.col = j;
    int keep = opt.keep > 0 ? opt.keep : std::max(w.nreq + (w.nreq + 1) / 2, w.nreq + nb);
    // the default basis leaves room for 128 to 144 new vectors per restart
    // cycle (the stagger by window index keeps equal windows from restarting
    // together); it keeps the projected matrix near 230-250 for the usual
    // requests, where its Schur step stays short
    int m = opt.max_basis > 0 ? opt.max_basis : std::max(2 * w.nreq + 1, keep + 128 + 8 * (j % 3));
    if (keep > m - nb) keep = m - nb;
    if (keep < w.nreq) return fail(c, SWI_EINVAL, "max_basis too small for the window request");
    if (m > max_basis)
      return fail(c, SWI_EINVAL, nb == 1 ? "single-vector windows: basis of at most 1000 vectors"
                                         : "2-vector blocks: basis of at most 510 vectors");
    if (m + nb > c->N) return fail(c, SWI_EINVAL, "basis larger than the problem dimension");
    w.m = m;
    w.keep = keep;
    w.ldq = DS ? (m + nb + 1) / 2 * 2 : (m + nb + 3) / 4 * 4;  // >= m + nb columns, rows on 32-byte boundaries
    w.ldh = m + nb;
    max_m = std::max(max_m, m);
    total_out += w.nreq;
  }
  // row chunks of the Gram-Schmidt passes: sized each step for the windows
  // still expanding (at least 256 rows per chunk, so at most this many chunks)
  const int max_chunks = (c->N + 255) / 256;
  for (int j = 0; j < nwin; ++j) {
    Win& w = *win[j];
    const size_t hh = (size_t)w.ldh * w.ldh;
    w.Q.ensure(sizeof(T) * N * w.ldq);
    w.H.ensure(sizeof(double2) * hh);
    w.Z.ensure(sizeof(double2) * hh);
    w.S.ensure(sizeof(double2) * hh);
    w.Bz.ensure(sizeof(double2) * nb * w.ldh);
    w.theta.ensure(sizeof(double2) * w.ldh);
    w.resid.ensure(sizeof(double) * w.ldh);
    w.Hw.ensure(16 * hh);
    w.Zw.ensure(16 * hh);
    w.Hsave.ensure(sizeof(double2) * hh);
    w.Yw.ensure(sizeof(double2) * w.ldh * w.nreq);
    w.eps_w.ensure(sizeof(double2) * w.nreq);
    w.res_w.ensure(sizeof(double) * w.nreq);
    w.C1.ensure(sizeof(double2) * w.ldh * nb);
    w.C2.ensure(sizeof(double2) * w.ldh * nb);
    if (!DS) w.Z32.ensure(sizeof(float2) * hh);
    w.rinv.ensure(sizeof(double2) * 16);  // R^-1, R, breakdown flag
    w.part.ensure(sizeof(double2) * (size_t)max_chunks * w.ldh * nb);
    SWI_CUDA_TRY(cudaMemsetAsync(w.H.p, 0, sizeof(double2) * hh, c->stream));
    SWI_CUDA_TRY(cudaMemsetAsync(w.Q.p, 0, sizeof(T) * N * w.ldq, c->stream));
    SWI_CUDA_TRY(cudaMemsetAsync(w.rinv.p, 0, sizeof(double2) * 16, c->stream));
  }
  const int n_all = (int)total_out;
  c->Uall.ensure(sizeof(double2) * N * n_all);
  c->ordinfo.ensure(sizeof(int) * 4 * nwin);
  // newest block of every window (columns [j nb, j nb + nb)) and its image
  // under A - sigma_j (in the double-single form the image is kept split, four
  // floats per entry, while it is orthogonalised); a complex128 work block for
  // the restart rotations and the delivered Ritz vectors
  DevMem Vcur, Wblk, sigt, Tmp;
  const int ncv = nwin * nb;
  const int ldv = ncv + (ncv & 1);  // even: 16-byte rows for the tensor-map-staged stencil
  Vcur.ensure(sizeof(T) * N * ldv);
  Wblk.ensure(sizeof(T) * N * ldv);
  SWI_CUDA_TRY(cudaMemsetAsync(Vcur.p, 0, sizeof(T) * N * ldv, c->stream));
  sigt.ensure(sizeof(double) * std::max(ncv, 4));
  Tmp.ensure(sizeof(double2) * N * (max_m + nb));
  {
    std::vector<typename Tr::Sig> sg(ncv);
    for (int j = 0; j < nwin; ++j)
      for (int b = 0; b < nb; ++b) sg[j * nb + b] = (typename Tr::Sig)win[j]->sigma;
    SWI_CUDA_TRY(cudaMemcpyAsync(sigt.p, sg.data(), sizeof(typename Tr::Sig) * ncv, cudaMemcpyHostToDevice,
                                 c->stream));
    sync(c->stream);
  }
  const swi::StencilParams P64 = stencil_params(c);
  const swi::StencilC64Params P32 = stencil_c64_params(c);
  auto apply_all = [&]() {
    if constexpr (DS) {
      swi::StencilBatch sb;
      sb.n = 0;
      for (int c0 = 0; c0 < ncv; c0 += 32)
        sb.blk[sb.n++] = swi::StencilBlock{reinterpret_cast<const double2*>(Vcur.p) + c0,
                                           reinterpret_cast<double2*>(Wblk.p) + c0, ldv, ldv,
                                           std::min(32, ncv - c0), c0, 1};
      swi::launch_stencil_ds(P64, sb, sigt.as<double>(), c->stream, &c->launches);
    } else {
      swi::launch_stencil_c64(P32, Vcur.as<float2>(), ldv, Wblk.as<float2>(), ldv, ncv, sigt.as<float>(),
                              c->stream, &c->launches);
    }
  };
  // Orthonormalise the blocks W[:, j nb : j nb + nb] of the given windows:
  // w^H w, one Cholesky factor for nb = 1, Cholesky-QR twice for nb = 2; R
  // goes below the block's column of H (when hrow is set), the block into the
  // basis at column dst_col and into Vcur.
  auto orthonormalise = [&](const std::vector<Win*>& ws, const std::vector<int>& dst_col, bool hrow, int rpc) {
    const int na = (int)ws.size();
    const int nchunks = (c->N + rpc - 1) / rpc;
    swi::SvReduceBatch r1, r2;
    swi::SvNormBatch n1, n2;
    swi::SvBatch g;
    r1.n = r2.n = n1.n = n2.n = g.n = na;
    for (int q = 0; q < na; ++q) {
      Win& w = *ws[q];
      T* wc = Wblk.as<T>() + w.col * nb;
      T* Qd = w.Q.template as<T>() + dst_col[q];
      double2* Hr = hrow ? w.H.template as<double2>() + (long long)(w.p + nb) * w.ldh + w.p : nullptr;
      double2* pp = w.part.template as<double2>();
      double2* ri = w.rinv.template as<double2>();
      r1.job[q] = swi::SvReduceJob{pp, w.ldh * nb, nchunks, 0, nb, 1, nullptr, nb == 1 ? Hr : nullptr, w.ldh, ri};
      g.job[q] = swi::SvJob{w.Q.p, w.ldq, 0, wc, ldv, nullptr, pp, w.ldh * nb};
      r2.job[q] = swi::SvReduceJob{pp, w.ldh * nb, nchunks, 0, nb, 2, nullptr, Hr, w.ldh, ri};
      if (nb == 1) {
        n1.job[q] = swi::SvNormJob{wc, ldv, Qd, w.ldq, Vcur.as<T>() + w.col * nb, ldv, ri, 0};
      } else {
        n1.job[q] = swi::SvNormJob{wc, ldv, wc, ldv, nullptr, 0, ri, 1};
        n2.job[q] = swi::SvNormJob{wc, ldv, Qd, w.ldq, Vcur.as<T>() + w.col * nb, ldv, ri, 0};
      }
    }
    swi::launch_sv_pass(g, swi::SV_WGRAM, DS, nb, c->N, rpc, c->stream, &c->launches);
    swi::launch_sv_reduce(r1, c->stream, &c->launches);
    swi::launch_sv_normalize(n1, DS, nb, c->N, c->stream, &c->launches);
    if (nb == 1) return;
    swi::launch_sv_pass(g, swi::SV_WGRAM, DS, nb, c->N, rpc, c->stream, &c->launches);
    swi::launch_sv_reduce(r2, c->stream, &c->launches);
    swi::launch_sv_normalize(n2, DS, nb, c->N, c->stream, &c->launches);
  };

  // start blocks: random, orthonormalised, in columns [0, nb) of each basis and in Vcur
  {
    std::vector<Win*> all;
    std::vector<int> zero(nwin, 0);
    for (int j = 0; j < nwin; ++j) {
      Win& w = *win[j];
      all.push_back(&w);
      for (int b = 0; b < nb; ++b) {
        const unsigned long long sd = seed * 1000003ull + (unsigned long long)j * nb + b;
        if constexpr (DS)
          random_col_ds_kernel<<<std::min((c->N + 255) / 256, 1024), 256, 0, c->stream>>>(
              Wblk.as<float4>() + j * nb + b, ldv, c->N, sd);
        else
          swi::launch_random_col_c64(Wblk.as<float2>() + j * nb + b, ldv, c->N, sd, c->stream, &c->launches);
        SWI_CHECK_LAUNCH();
      }
    }
    orthonormalise(all, zero, false, swi::sv_rows_per_chunk(c->N, nwin));
  }

  const double tol_abs = rel_tol * anorm;
  std::vector<int> out_off(nwin);
  {
    int o2 = 0;
    for (int j = 0; j < nwin; ++j) {
      out_off[j] = o2;
      o2 += win[j]->nreq;
    }
  }

  struct SideRes {
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> ready, done;
    cudaEvent_t lag[2] = {nullptr, nullptr};
    int* oi = nullptr;
    ~SideRes() {
      for (auto x : lag)
        if (x) cudaEventDestroy(x);
      for (auto x : st)
        if (x) cudaStreamDestroy(x);
      for (auto x : ready)
        if (x) cudaEventDestroy(x);
      for (auto x : done)
        if (x) cudaEventDestroy(x);
      if (oi) cudaFreeHost(oi);
    }
  } side;
  side.st.assign(nwin, nullptr);
  side.ready.assign(nwin, nullptr);
  side.done.assign(nwin, nullptr);
  for (int j = 0; j < nwin; ++j) {
    SWI_CUDA_TRY(cudaStreamCreateWithFlags(&side.st[j], cudaStreamNonBlocking));
    SWI_CUDA_TRY(cudaEventCreateWithFlags(&side.ready[j], cudaEventDisableTiming));
    SWI_CUDA_TRY(cudaEventCreateWithFlags(&side.done[j], cudaEventDisableTiming));
  }
  SWI_CUDA_TRY(cudaMallocHost(&side.oi, sizeof(int) * 4 * nwin));
  for (auto& e : side.lag) SWI_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  std::vector<int> in_schur(nwin, 0);

  // the window's first ncol basis columns as complex128 [N][ld] (the complex64
  // form widens them into Tmp)
  auto basis64 = [&](Win& w, int ncol, int& ld) -> const double2* {
    if constexpr (DS) {
      ld = w.ldq;
      return w.Q.template as<double2>();
    } else {
      swi::launch_widen(w.Q.template as<float2>(), w.ldq, Tmp.as<double2>(), w.ldh, c->N, ncol, c->stream,
                        &c->launches);
      ld = w.ldh;
      return Tmp.as<double2>();
    }
  };

  // the projected eigenproblem of window j (order w.p) on its own stream; the
  // double-single kernel, or after it gave up the native FP64 one on the
  // saved matrix
  auto launch_schur = [&](Win& w, bool f64) {
    const int j = w.col;
    cudaStream_t sj = side.st[j];
    const size_t hh = (size_t)w.ldh * w.ldh;
    if (f64) SWI_CUDA_TRY(cudaMemcpyAsync(w.H.p, w.Hsave.p, sizeof(double2) * hh, cudaMemcpyDeviceToDevice, sj));
    else SWI_CUDA_TRY(cudaMemcpyAsync(w.Hsave.p, w.H.p, sizeof(double2) * hh, cudaMemcpyDeviceToDevice, sj));
    // as ARPACK does, keep more Ritz vectors once some wanted pairs have converged
    const int keep_eff = std::min(w.m - nb, w.keep + std::min(w.nconv, (w.m - w.keep) / 2));
    swi::SchurBatch sb;
    sb.n = 1;
    // B: the nb coupling rows of the Arnoldi relation, rows [p, p + nb) of H
    double2* H = w.H.template as<double2>();
    sb.job[0] = swi::SchurJob{H, w.Z.template as<double2>(), H + (long long)w.p * w.ldh, w.Bz.template as<double2>(),
                              w.theta.template as<double2>(), w.resid.template as<double>(), w.S.template as<double2>(),
                              c->ordinfo.as<int>() + 4 * j, w.p, w.ldh, nb, keep_eff, w.nreq, w.m - nb, tol_abs,
                              w.Hw.p, w.Zw.p, w.sig_im};
    {
      ProfScope ps(c, SWI_K_SCHUR, 0.0, 0.0, sj);
      if (f64) swi::launch_schur_batch(sb, sj, &c->launches);
      else swi::launch_schur_ds_batch(sb, sj, &c->launches);
    }
    SWI_CUDA_TRY(cudaMemcpyAsync(side.oi + 4 * j, c->ordinfo.as<int>() + 4 * j, sizeof(int) * 4,
                                 cudaMemcpyDeviceToHost, sj));
    SWI_CUDA_TRY(cudaEventRecord(side.done[j], sj));
    in_schur[j] = 1;
  };

  auto finish_restart = [&](int j) {
    Win& w = *win[j];
    const int* oi = side.oi + 4 * j;
    const int kk = oi[0], nconv = oi[1], st = oi[2];
    const int n = w.p;  // order of the projected matrix
    if (st != 0 && !w.retry) {  // the double-single QR gave up: the FP64 kernel on the same matrix
      w.retry = true;
      w.schur_retries++;
      launch_schur(w, true);
      return;
    }
    w.retry = false;
    SWI_CUDA_TRY(cudaStreamWaitEvent(c->stream, side.done[j], 0));
    w.restarts++;
    w.nconv = nconv;
    if (c->prof_on) c->schur_flops += 64.0 / 3.0 * (double)n * n * n + 20.0 * 1024.0 * (double)oi[3];
    if (st != 0) w.failed = true;
    if (st != 0 || nconv >= w.nreq || w.matvecs >= budget) {
      // Ritz vectors of the wanted pairs into Uall (complex128)
      int ldb = 0;
      const double2* Qb = basis64(w, n, ldb);
      swi::RitzBatch fin;
      fin.n = 1;
      fin.job[0] = swi::RitzJob{w.Z.template as<double2>(), w.S.template as<double2>(), w.theta.template as<double2>(),
                                w.resid.template as<double>(), c->ordinfo.as<int>() + 4 * j, w.Yw.template as<double2>(),
                                w.eps_w.template as<double2>(), w.res_w.template as<double>(), n, w.ldh, w.nreq,
                                w.nreq, w.sigma, w.sig_im};
      swi::RowGemmBatch rb;
      rb.n = 1;
      rb.job[0] = swi::RowGemmJob{Qb, w.Yw.template as<double2>(), nullptr, c->Uall.as<double2>() + out_off[j], ldb,
                                  w.nreq, 0, n_all, n, w.nreq, 1.0, 0.0};
      ProfScope ps(c, SWI_K_ROTATE, 8.0 * c->N * (double)n * w.nreq, 16.0 * c->N * (double)(n + w.nreq));
      swi::launch_ritz_batch(fin, c->stream, &c->launches);
      rowgemm_dispatch(SWI_ARITH_DS, rb, c->N, c->stream, &c->launches);
      w.done = true;
      return;
    }
    if (kk + nb > w.m || kk < w.nreq || kk > n) throw Error{SWI_ECUDA, "internal: restart size out of range"};
    {
      // thick restart: Q[:, 0:kk] = Q[:, 0:n] Z[:, 0:kk]; the residual block
      // (columns [n, n + nb), also held in Vcur) becomes columns [kk, kk + nb)
      ProfScope ps(c, SWI_K_ROTATE, 8.0 * c->N * (double)n * kk, sizeof(T) * c->N * (double)(n + kk));
      if constexpr (DS) {
        swi::RowGemmBatch rb;
        rb.n = 1;
        rb.job[0] = swi::RowGemmJob{w.Q.template as<double2>(), w.Z.template as<double2>(), nullptr,
                                    Tmp.as<double2>(), w.ldq, w.ldh, 0, w.ldh, n, kk, 1.0, 0.0};
        rowgemm_dispatch(SWI_ARITH_DS, rb, c->N, c->stream, &c->launches);
        swi::launch_copy_block(Tmp.as<double2>(), w.ldh, w.Q.template as<double2>(), w.ldq, c->N, kk, c->stream,
                               &c->launches);
        swi::launch_copy_block(Vcur.as<double2>() + w.col * nb, ldv, w.Q.template as<double2>() + kk, w.ldq, c->N,
                               nb, c->stream, &c->launches);
      } else {
        swi::launch_z_to_c64(w.Z.template as<double2>(), w.ldh, n, kk, w.Z32.template as<float2>(), kk, c->stream,
                             &c->launches);
        swi::launch_c64_rotate_inplace(w.Q.template as<float2>(), w.ldq, c->N, n, w.Z32.template as<float2>(), kk,
                                       kk, c->stream, &c->launches);
        for (int b = 0; b < nb; ++b)
          swi::launch_copy_col_c64(Vcur.as<float2>() + w.col * nb + b, ldv, w.Q.template as<float2>() + kk + b,
                                   w.ldq, c->N, c->stream, &c->launches);
      }
      launch_restart_h(w.H.template as<double2>(), w.ldh, w.ldh, kk, nb, w.Bz.template as<double2>(), c->stream,
                       &c->launches);
    }
    w.p = kk;  // the newest block (already in Vcur) is now columns [kk, kk + nb)
  };

  const long long max_steps = 100000000LL;
  for (long long step = 0; step < max_steps; ++step) {
    // keep the host at most two steps ahead of the device
    if (step >= 2) SWI_CUDA_TRY(cudaEventSynchronize(side.lag[step & 1]));
    for (int j = 0; j < nwin; ++j) {
      if (!in_schur[j]) continue;
      const cudaError_t q = cudaEventQuery(side.done[j]);
      if (q == cudaErrorNotReady) continue;
      SWI_CUDA_TRY(q);
      in_schur[j] = 0;
      finish_restart(j);  // may start the FP64 retry (in_schur set again)
    }
    std::vector<Win*> act;
    int pending = -1;
    for (int j = 0; j < nwin; ++j) {
      if (win[j]->done) continue;
      if (in_schur[j]) {
        if (pending < 0) pending = j;
        continue;
      }
      act.push_back(win[j].get());
    }
    if (act.empty()) {
      if (pending < 0) break;
      SWI_CUDA_TRY(cudaEventSynchronize(side.done[pending]));
      continue;
    }
    const int na = (int)act.size();
    const double Nn = (double)c->N;
    const int rpc = swi::sv_rows_per_chunk(c->N, na);
    const int nchunks = (c->N + rpc - 1) / rpc;
    // 1) W[:, j nb : j nb + nb] = (A - sigma_j) Q_j[:, p : p + nb] for every window
    //    (columns of waiting windows are computed and ignored)
    {
      ProfScope ps(c, SWI_K_STENCIL, kStencilFlops * Nn * ncv, (2.0 * sizeof(T) * ncv + 8.0) * Nn);
      apply_all();
    }
    // 2) classical Gram-Schmidt twice against Q[:, 0:p+nb]: Gram, update
    //    fused with the second Gram, update; then the block's Cholesky-QR
    double ncol = 0.0;
    swi::SvBatch g0, g1, g2;
    swi::SvReduceBatch r0, r1;
    g0.n = g1.n = g2.n = r0.n = r1.n = na;
    std::vector<int> dst(na);
    for (int q = 0; q < na; ++q) {
      Win& w = *act[q];
      if (w.p + 2 * nb > w.ldq || w.p + 2 * nb > w.ldh)
        throw Error{SWI_ECUDA, "internal: Krylov block beyond the basis buffer"};
      const int nc = w.p + nb;
      ncol += nc;
      const void* Qp = w.Q.p;
      T* wc = Wblk.as<T>() + w.col * nb;
      double2* pp = w.part.template as<double2>();
      double2* hcol = w.H.template as<double2>() + w.p;
      const int ldp = w.ldh * nb;
      g0.job[q] = swi::SvJob{Qp, w.ldq, nc, wc, ldv, nullptr, pp, ldp};
      g1.job[q] = swi::SvJob{Qp, w.ldq, nc, wc, ldv, w.C1.template as<double2>(), pp, ldp};
      g2.job[q] = swi::SvJob{Qp, w.ldq, nc, wc, ldv, w.C2.template as<double2>(), pp, ldp};
      r0.job[q] = swi::SvReduceJob{pp, ldp, nchunks, nc, nb, 0, w.C1.template as<double2>(), hcol, w.ldh, nullptr};
      r1.job[q] = swi::SvReduceJob{pp, ldp, nchunks, nc, nb, 0, w.C2.template as<double2>(), hcol, w.ldh, nullptr};
      dst[q] = w.p + nb;
    }
    // profile classes: the first Gram pass; the update fused with the second
    // Gram (the accurate pass); the second update with the block's Cholesky-QR.
    // Bytes: each basis read once per pass plus the new vectors; flops: 8 per
    // complex multiply-add and new vector
    const double wbytes = 16.0 * Nn * na * nb;
    {
      ProfScope ps(c, SWI_K_GRAM, 8.0 * Nn * ncol * nb, sizeof(T) * Nn * ncol + wbytes);
      swi::launch_sv_pass(g0, swi::SV_GRAM, DS, nb, c->N, rpc, c->stream, &c->launches);
      swi::launch_sv_reduce(r0, c->stream, &c->launches);
    }
    {
      ProfScope ps(c, SWI_K_UPDATE, 2.0 * 8.0 * Nn * ncol * nb, sizeof(T) * Nn * ncol + 2.0 * wbytes);
      swi::launch_sv_pass(g1, swi::SV_UPDATE_GRAM, DS, nb, c->N, rpc, c->stream, &c->launches);
      swi::launch_sv_reduce(r1, c->stream, &c->launches);
    }
    {
      ProfScope ps(c, SWI_K_CHOLQR, 8.0 * Nn * ncol * nb, sizeof(T) * Nn * ncol + 6.0 * wbytes);
      swi::launch_sv_pass(g2, swi::SV_UPDATE, DS, nb, c->N, rpc, c->stream, &c->launches);
      orthonormalise(act, dst, true, rpc);
    }
    // 3) windows whose next block would not fit: projected eigenproblem on their own stream
    for (int q = 0; q < na; ++q) {
      Win& w = *act[q];
      const int j = w.col;
      w.p += nb;
      w.matvecs += nb;
      if (w.p + nb <= w.m) continue;
      SWI_CUDA_TRY(cudaEventRecord(side.ready[j], c->stream));
      SWI_CUDA_TRY(cudaStreamWaitEvent(side.st[j], side.ready[j], 0));
      launch_schur(w, false);
    }
    SWI_CUDA_TRY(cudaEventRecord(side.lag[step & 1], c->stream));
  }

  // ---- eigenvalue estimates and window statistics, then the merge (as in the block form)
  std::vector<double2> eps_all(n_all);
  std::vector<int> win_of(n_all);
  c->winfo.assign(nwin, swi_window_info());
  bool any_fail = false, any_noconv = false, any_breakdown = false;
  for (int j = 0; j < nwin; ++j) {
    Win& w = *win[j];
    std::vector<double> rw(w.nreq);
    SWI_CUDA_TRY(cudaMemcpyAsync(eps_all.data() + out_off[j], w.eps_w.p, sizeof(double2) * w.nreq,
                                 cudaMemcpyDeviceToHost, c->stream));
    SWI_CUDA_TRY(cudaMemcpyAsync(rw.data(), w.res_w.p, sizeof(double) * w.nreq, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    for (int q = 0; q < w.nreq; ++q) win_of[out_off[j] + q] = j;
    swi_window_info& wi = c->winfo[j];
    wi.sigma = w.sigma;
    wi.n_req = w.nreq;
    wi.n_conv = w.nconv;
    wi.matvecs = w.matvecs;
    wi.restarts = w.restarts;
    wi.basis = w.m;
    double mr = 0.0;
    for (double r : rw) mr = std::max(mr, r / anorm);
    wi.max_res = mr;
    wi.schur_retries = w.schur_retries;
    double2 flag;
    SWI_CUDA_TRY(cudaMemcpy(&flag, w.rinv.template as<double2>() + 8, sizeof(double2), cudaMemcpyDeviceToHost));
    if (flag.x != 0.0) any_breakdown = true;
    any_fail |= w.failed;
    any_noconv |= (w.nconv < w.nreq);
  }
  win.clear();
  Tmp.release();
  Vcur.release();
  Wblk.release();
  const double t1 = swi::now_seconds();
  int minfo[4];
  merge_pairs(c, c->Uall.as<double2>(), n_all, eps_all, win_of, nwin, eq_rtol, drop_tol, opt.n_keep, minfo);
  record_windows(c, eps_all, win_of, nwin);
  const int nout = minfo[0];
  c->Uall.release();
  {
    ProfScope ps(c, SWI_K_MERGE, kStencilFlops * c->N * (double)nout, 48.0 * c->N * (double)nout);
    explicit_residuals(c, c->U.as<double2>(), nout, c->eps.as<double2>(), nout, c->resid);
  }
  const double t2 = swi::now_seconds();
  int nconv = 0;
  double maxr = 0.0;
  for (double r : c->resid) {
    if (r <= rel_tol) ++nconv;
    maxr = std::max(maxr, r);
  }
  long long mv = 0;
  for (auto& wi : c->winfo) mv += wi.matvecs;
  if (info) {
    info->n_windows = nwin;
    info->n_pairs = nout;
    info->n_converged = nconv;
    info->n_duplicates = minfo[1];
    info->n_holes = minfo[2];
    info->matvecs = mv;
    info->max_rel_res = maxr;
    info->anorm = anorm;
    info->t_krylov_s = t1 - t0;
    info->t_merge_s = t2 - t1;
  }
  if (!DS && swi::stencil_c64_tma_error(true))
    return fail(c, SWI_ETIMEOUT, "a stencil block gave up waiting for its tensor-map copy");
  if (any_fail) return fail(c, SWI_ENOCONV, "a window's projected eigenproblem did not converge");
  if (any_breakdown) return fail(c, SWI_ENOCONV, "a window's new Krylov vectors became linearly dependent");
  if (minfo[3] != 0) return fail(c, SWI_EINVAL, "merge: equal-eigenvalue component too large");
  if (any_noconv) return fail(c, SWI_ENOCONV, "some window did not converge within its matvec budget");
  if (nconv < nout) return fail(c, SWI_ENOCONV, "pairs above rel_tol in the explicit FP64 residual check");
  if (minfo[2] > 0) return fail(c, SWI_HOLES, std::to_string(minfo[2]) + " interface(s) without redundancy");
  return SWI_OK;
}

}  // namespace

swi_status do_solve_sv(swi_ctx* c, const swi_solve_opts* o, swi_solve_info* info) {
  if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set before solve");
  if (c->sigma.empty()) return fail(c, SWI_ESTATE, "windows must be set before solve");
  swi_solve_opts opt;
  std::memset(&opt, 0, sizeof(opt));
  if (o) opt = *o;
  if (c->precision == SWI_PREC_MIXED) return solve_sv<false>(c, opt, info);
  return solve_sv<true>(c, opt, info);
}

}  // namespace host
}  // namespace swi
