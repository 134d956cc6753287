// C ABI and host-side runtime of the partitioned shift-without-invert solver.
//
// The host plans and sequences; every O(N) step runs in this library's
// kernels on the context's stream.  One solve batches all windows (the
// paper's independent partitions, Section 2.1) into shared launches: the
// stencil applies (A - sigma_j) to the new block of every active window in one
// launch, the orthogonalisation and Cholesky-QR of all windows go out as
// batched launches, and windows that reach their maximum basis restart
// together.  The host reads back only a few status words per restart.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <mutex>
#include <atomic>
#include <thread>
#include <vector>

#include "merge.cuh"
#include "swi_internal.cuh"
#include "transport.cuh"
#include "host.cuh"

using swi::Error;
using namespace swi::host;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace swi {
namespace host {


cudaEvent_t take_event(swi_ctx* c) {
  if (!c->evpool.empty()) {
    cudaEvent_t e = c->evpool.back();
    c->evpool.pop_back();
    return e;
  }
  cudaEvent_t e;
  SWI_CUDA_TRY(cudaEventCreate(&e));
  return e;
}

ProfScope::ProfScope(swi_ctx* ctx, int k, double f, double by, cudaStream_t stream)
    : c(ctx), kind(k), flops(f), bytes(by), st(stream ? stream : ctx->stream) {
  if (c->prof_on) {
    a = take_event(c);
    SWI_CUDA_TRY(cudaEventRecord(a, st));
  }
}
ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b = nullptr;
  if (!c->evpool.empty()) {
    b = c->evpool.back();
    c->evpool.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    return;
  }
  if (cudaEventRecord(b, st) != cudaSuccess) return;
  c->prof.push_back({kind, a, b, flops, bytes});
}

// Tall-skinny products: double-single on the FP32 pipes (default) or native FP64.
void gram_dispatch(int arith, const swi::GramBatch& b, int N, const double* w, int bilinear, double2* work,
                   size_t work_elems, cudaStream_t s, long long* launches) {
  if (arith == SWI_ARITH_F64) swi::launch_gram(b, N, w, bilinear, work, work_elems, s, launches);
  else swi::launch_gram_df(b, N, w, bilinear, work, work_elems, s, launches);
}
void rowgemm_dispatch(int arith, const swi::RowGemmBatch& b, int N, cudaStream_t s, long long* launches) {
  if (arith == SWI_ARITH_F64) swi::launch_rowgemm(b, N, s, launches);
  else swi::launch_rowgemm_df(b, N, s, launches);
}

swi_status fail(swi_ctx* ctx, swi_status code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return code;
}

template <class F>
swi_status guarded(swi_ctx* ctx, F&& f) {
  if (!ctx) return fail(nullptr, SWI_EINVAL, "null context");
  try {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(ctx, SWI_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return f();
  } catch (const Error& e) {
    return fail(ctx, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(ctx, SWI_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(ctx, SWI_ECUDA, "unexpected exception");
  }
}

swi::StencilParams stencil_params(const swi_ctx* c) {
  swi::StencilParams P;
  P.nx = c->nx;
  P.ny = c->ny;
  P.nz = c->nz;
  P.bc = c->bc;
  for (int m = 0; m < 7; ++m) P.cm[m] = -kFD[m] / (2.0 * c->h * c->h);
  P.V = c->V.as<double>();
  P.G = c->G.as<double>();
  return P;
}

double gershgorin(const swi_ctx* c) {
  double s = std::fabs(kFD[0]);
  for (int m = 1; m < 7; ++m) s += 2.0 * std::fabs(kFD[m]);
  return 3.0 * 0.5 / (c->h * c->h) * s + c->maxabsV + c->maxG;
}

void copy_in(DevMem& dst, const void* src, size_t bytes, bool on_device, cudaStream_t s) {
  dst.ensure(bytes);
  SWI_CUDA_TRY(cudaMemcpyAsync(dst.p, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

void sync(cudaStream_t s) { SWI_CUDA_TRY(cudaStreamSynchronize(s)); }

// Y[:, c] = (A - sigma_c) X[:, c] in chunks of columns, sigma from the context's sigma table
void apply_block(swi_ctx* c, const double2* X, int ldx, double2* Y, int ldy, int ncols, bool ds) {
  const swi::StencilParams P = stencil_params(c);
  for (int c0 = 0; c0 < ncols; c0 += 32) {
    swi::StencilBatch bt;
    bt.n = 1;
    bt.blk[0] = swi::StencilBlock{X + c0, Y + c0, ldx, ldy, std::min(32, ncols - c0), c0};
    if (ds)
      swi::launch_stencil_ds(P, bt, c->sig_dev.as<double>(), c->stream, &c->launches);
    else
      swi::launch_stencil(P, bt, c->sig_dev.as<double>(), c->stream, &c->launches);
  }
}

// explicit relative residuals of (eps, U) -> host vector
void explicit_residuals(swi_ctx* c, const double2* Ud, int ldu, const double2* epsd, int n, std::vector<double>& out) {
  out.assign(n, 0.0);
  if (n == 0) return;
  c->sig_dev.ensure(sizeof(double) * std::max(n, 64));
  SWI_CUDA_TRY(cudaMemsetAsync(c->sig_dev.p, 0, sizeof(double) * n, c->stream));
  c->scratch.ensure(sizeof(double2) * (size_t)c->N * n);
  apply_block(c, Ud, ldu, c->scratch.as<double2>(), n, n);
  c->colwork.ensure(sizeof(double) * (size_t)n * 1024);
  c->dres.ensure(sizeof(double) * 2 * n);
  // ||u_k|| and ||A u_k - eps_k u_k||
  swi::launch_colnorm_resid(Ud, ldu, Ud, ldu, nullptr, n, c->N, c->dres.as<double>() + n, c->colwork.as<double>(),
                            c->colwork.bytes / sizeof(double), c->stream, &c->launches);
  swi::launch_colnorm_resid(Ud, ldu, c->scratch.as<double2>(), n, epsd, n, c->N, c->dres.as<double>(),
                            c->colwork.as<double>(), c->colwork.bytes / sizeof(double), c->stream, &c->launches);
  std::vector<double> both(2 * n);
  SWI_CUDA_TRY(cudaMemcpyAsync(both.data(), c->dres.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->stream));
  sync(c->stream);
  std::vector<double> unorm(both.begin() + n, both.end());
  std::copy(both.begin(), both.begin() + n, out.begin());
  const double an = gershgorin(c);
  for (int k = 0; k < n; ++k) out[k] = out[k] / (an * std::max(unorm[k], 1e-300));
}

void gram_work_ensure(swi_ctx* c, size_t elems) {
  c->gram_work.ensure(sizeof(double2) * std::max<size_t>(elems, 1 << 20));
}

// Cholesky-QR2 of the blocks W_j (N x b, ld b) into Q_j[:, col : col+b]; R1, R2 kept per window.
void cholqr2(swi_ctx* c, std::vector<Window*>& ws, const std::vector<int>& col, int b) {
  const int nb = (int)ws.size();
  if (nb == 0) return;
  // device pointer tables for the Cholesky kernel: [G..., R..., Rinv...]
  c->ptrs.ensure(sizeof(void*) * 3 * swi::kMaxBatch);
  c->cholstat.ensure(sizeof(int) * swi::kMaxBatch);
  auto gram_of = [&](bool second) {
    swi::GramBatch gb;
    gb.n = nb;
    for (int q = 0; q < nb; ++q) {
      Window& w = *ws[q];
      const double2* X = second ? w.Q[w.cur].as<double2>() + col[q] : w.W.as<double2>();
      const int ldx = second ? w.ld : b;
      gb.job[q] = swi::GramJob{X, X, w.G.as<double2>(), ldx, ldx, b, b, b, 0};
    }
    gram_dispatch(c->arith,gb, c->N, nullptr, 0, c->gram_work.as<double2>(), c->gram_work.bytes / sizeof(double2),
                     c->stream, &c->launches);
  };
  auto chol_of = [&](bool second) {
    swi::CholBatch cb;
    cb.n = nb;
    for (int q = 0; q < nb; ++q) {
      cb.G[q] = ws[q]->G.as<double2>();
      cb.R[q] = (second ? ws[q]->R2 : ws[q]->R1).as<double2>();
      cb.Rinv[q] = (second ? ws[q]->R2i : ws[q]->R1i).as<double2>();
    }
    swi::launch_chol_batch(cb, b, c->cholstat.as<int>(), c->stream, &c->launches);
  };
  gram_of(false);
  chol_of(false);
  {
    swi::RowGemmBatch rb;
    rb.n = nb;
    for (int q = 0; q < nb; ++q) {
      Window& w = *ws[q];
      rb.job[q] = swi::RowGemmJob{w.W.as<double2>(), w.R1i.as<double2>(), nullptr, w.Q[w.cur].as<double2>() + col[q],
                                  b, b, 0, w.ld, b, b, 1.0, 0.0};
    }
    rowgemm_dispatch(c->arith,rb, c->N, c->stream, &c->launches);
  }
  gram_of(true);
  chol_of(true);
  {
    swi::RowGemmBatch rb;
    rb.n = nb;
    for (int q = 0; q < nb; ++q) {
      Window& w = *ws[q];
      rb.job[q] = swi::RowGemmJob{w.Q[w.cur].as<double2>() + col[q], w.R2i.as<double2>(), nullptr, w.W.as<double2>(),
                                  w.ld, b, 0, b, b, b, 1.0, 0.0};
    }
    rowgemm_dispatch(c->arith,rb, c->N, c->stream, &c->launches);
  }
  for (int q = 0; q < nb; ++q) {
    Window& w = *ws[q];
    swi::launch_copy_block(w.W.as<double2>(), b, w.Q[w.cur].as<double2>() + col[q], w.ld, c->N, b, c->stream,
                           &c->launches);
  }
}

// Algorithm 2 over n_all pairs of nwin windows (U [N][ldu] on the device, not
// the context's own pair buffer; eps and window index on the host, windows in
// shift order), selection of the n_keep lowest (0: all), U^T U = I; the
// survivors become the context's pairs.  minfo: nout, n_dup, n_holes, status.
void merge_pairs(swi_ctx* c, const double2* Uin, int ldu, const std::vector<double2>& eps_all,
                 const std::vector<int>& win_of, int nwin, double eq_rtol, double drop_tol, int n_keep, int* minfo) {
  const int n_all = (int)eps_all.size();
  const int pair_cap = std::max(4 * n_all, 1024);
  c->m_eps_all.ensure(sizeof(double2) * n_all);
  c->m_win.ensure(sizeof(int) * n_all);
  SWI_CUDA_TRY(cudaMemcpyAsync(c->m_eps_all.p, eps_all.data(), sizeof(double2) * n_all, cudaMemcpyHostToDevice,
                               c->stream));
  SWI_CUDA_TRY(cudaMemcpyAsync(c->m_win.p, win_of.data(), sizeof(int) * n_all, cudaMemcpyHostToDevice, c->stream));
  c->m_comp.ensure(sizeof(int) * n_all);
  c->m_pairs.ensure(sizeof(int) * 2 * pair_cap);
  c->m_counts.ensure(sizeof(int) * 4);
  c->m_work.ensure(sizeof(double2) * (size_t)pair_cap * 2 * 304);
  c->m_gram.ensure(sizeof(double2) * 2 * pair_cap);
  c->m_kept.ensure(sizeof(int) * n_all);
  c->m_order.ensure(sizeof(int) * n_all);
  c->m_holes.ensure(sizeof(int) * (nwin + 1));
  c->m_src.ensure(sizeof(int) * swi::merge_src_elems(n_all));
  c->m_coef.ensure(sizeof(double2) * swi::merge_coef_elems(n_all));
  c->m_nterm.ensure(sizeof(int) * (n_all + 1));
  c->m_info.ensure(sizeof(int) * 4);
  c->m_eps_out.ensure(sizeof(double2) * n_all);
  swi::MergeArgs ma;
  ma.U = Uin;
  ma.ldu = ldu;
  ma.N = c->N;
  ma.n = n_all;
  ma.p = nwin;
  ma.eps = c->m_eps_all.as<double2>();
  ma.win = c->m_win.as<int>();
  ma.eq_rtol = eq_rtol;
  ma.drop_tol = drop_tol;
  ma.n_keep = n_keep;
  ma.comp = c->m_comp.as<int>();
  ma.pairs = c->m_pairs.as<int>();
  ma.pair_cap = pair_cap;
  ma.counts = c->m_counts.as<int>();
  ma.work = c->m_work.as<double2>();
  ma.work_elems = c->m_work.bytes / sizeof(double2);
  ma.gram = c->m_gram.as<double2>();
  ma.kept = c->m_kept.as<int>();
  ma.order = c->m_order.as<int>();
  ma.holes = c->m_holes.as<int>();
  ma.src = c->m_src.as<int>();
  ma.coef = c->m_coef.as<double2>();
  ma.nterm = c->m_nterm.as<int>();
  ma.out_eps = c->m_eps_out.as<double2>();
  ma.info = c->m_info.as<int>();
  {
    ProfScope ps(c, SWI_K_MERGE, 0.0, 16.0 * c->N * (double)n_all);
    swi::merge_run(ma, c->stream, &c->launches);
  }
  SWI_CUDA_TRY(cudaMemcpyAsync(minfo, c->m_info.p, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
  sync(c->stream);
  const int nout = minfo[0];
  c->U.ensure(sizeof(double2) * (size_t)c->N * std::max(nout, 1));
  c->eps.ensure(sizeof(double2) * std::max(nout, 1));
  ma.out_U = c->U.as<double2>();
  ma.ldo = nout;
  {
    ProfScope ps(c, SWI_K_MERGE, 0.0, 16.0 * c->N * (double)(n_all + nout));
    swi::merge_apply(ma, nout, c->stream, &c->launches);
  }
  SWI_CUDA_TRY(cudaMemcpyAsync(c->eps.p, c->m_eps_out.p, sizeof(double2) * nout, cudaMemcpyDeviceToDevice, c->stream));
  c->npairs = nout;
  c->have_RL = false;
}

}  // namespace host
}  // namespace swi

namespace {
using namespace swi::host;

}  // namespace

void swi::host::record_windows(swi_ctx* c, const std::vector<double2>& eps_all, const std::vector<int>& win_of,
                               int nwin) {
  c->last_sigma = c->sigma;
  c->last_complex = false;
  for (double v : c->sigma_im) c->last_complex = c->last_complex || v != 0.0;
  c->last_eps_win = eps_all;
  c->last_win_of = win_of;
  c->last_holes.assign(std::max(0, nwin - 1), 0);
  if (nwin > 1)
    SWI_CUDA_TRY(cudaMemcpy(c->last_holes.data(), c->m_holes.p, sizeof(int) * (nwin - 1), cudaMemcpyDeviceToHost));
}

namespace {

swi_status do_solve(swi_ctx* c, const swi_solve_opts* o, swi_solve_info* info) {
  if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set before solve");
  if (c->sigma.empty()) return fail(c, SWI_ESTATE, "windows must be set before solve");
  for (double v : c->sigma_im)
    if (v != 0.0) return fail(c, SWI_EINVAL, "complex shifts need windows of 1 or 2 vectors (double-single or mixed)");
  swi_solve_opts opt;
  std::memset(&opt, 0, sizeof(opt));
  if (o) opt = *o;
  const int b = opt.block > 0 ? opt.block : 16;
  if (b > 32) return fail(c, SWI_EINVAL, "block width must be <= 32");
  const double rel_tol = opt.rel_tol > 0 ? opt.rel_tol : 1e-10;
  const double eq_rtol = opt.eq_rtol > 0 ? opt.eq_rtol : 1e-8;
  const double drop_tol = opt.drop_tol > 0 ? opt.drop_tol : 1e-6;
  const long long budget = opt.max_matvecs > 0 ? opt.max_matvecs : 2000000LL;
  const unsigned long long seed = opt.seed ? opt.seed : 1ull;
  const double anorm = gershgorin(c);
  if (opt.arith != 0 && opt.arith != SWI_ARITH_DS && opt.arith != SWI_ARITH_F64)
    return fail(c, SWI_EINVAL, "unknown arithmetic");
  c->arith = opt.arith == SWI_ARITH_F64 ? SWI_ARITH_F64 : SWI_ARITH_DS;
  const int nwin = (int)c->sigma.size();
  if (nwin > swi::kMaxBatch) return fail(c, SWI_EINVAL, "at most 64 windows per solve");
  const double t0 = swi::now_seconds();

  // ---- per-window sizes and buffers
  std::vector<std::unique_ptr<Window>> win(nwin);
  size_t total_out = 0;
  for (int j = 0; j < nwin; ++j) {
    win[j].reset(new Window());
    Window& w = *win[j];
    w.sigma = c->sigma[j];
    w.nreq = c->nreq[j];
    int keep = opt.keep > 0 ? opt.keep : std::max(w.nreq + (w.nreq + 1) / 2, w.nreq + b);
    // Default basis: keep + 8 blocks, plus 0-2 extra blocks by window index so
    // equal windows restart at different steps and their Schur steps (one CTA
    // each) overlap the other windows' expansion instead of coinciding.
    int m = opt.max_basis > 0 ? opt.max_basis : std::max(2 * w.nreq + 1, keep + (8 + j % 3) * b);
    m = (m + b - 1) / b * b;
    if (keep > m - b) keep = m - b;
    if (keep < w.nreq) return fail(c, SWI_EINVAL, "max_basis too small for the window request");
    if (m > 1024) return fail(c, SWI_EINVAL, "basis larger than 1024 is not supported");
    if (m + b > c->N) return fail(c, SWI_EINVAL, "basis larger than the problem dimension");
    w.m = m;
    w.keep = keep;
    w.ld = m + b;
    const size_t N = c->N;
    w.Q[0].ensure(sizeof(double2) * N * w.ld);
    w.Q[1].ensure(sizeof(double2) * N * w.ld);
    w.W.ensure(sizeof(double2) * N * b);
    w.H.ensure(sizeof(double2) * w.ld * w.ld);
    w.Z.ensure(sizeof(double2) * w.ld * w.ld);
    w.S.ensure(sizeof(double2) * w.ld * w.ld);
    w.Bm.ensure(sizeof(double2) * b * w.ld);
    w.Bz.ensure(sizeof(double2) * b * w.ld);
    w.theta.ensure(sizeof(double2) * w.ld);
    w.resid.ensure(sizeof(double) * w.ld);
    w.C1.ensure(sizeof(double2) * w.ld * b);
    w.C2.ensure(sizeof(double2) * w.ld * b);
    w.G.ensure(sizeof(double2) * b * b);
    w.R1.ensure(sizeof(double2) * b * b);
    w.R1i.ensure(sizeof(double2) * b * b);
    w.R2.ensure(sizeof(double2) * b * b);
    w.R2i.ensure(sizeof(double2) * b * b);
    w.Zext.ensure(sizeof(double2) * w.ld * w.ld);
    if (c->arith != SWI_ARITH_F64) {
      w.Hw.ensure(16 * (size_t)w.ld * w.ld);
      w.Zw.ensure(16 * (size_t)w.ld * w.ld);
    }
    w.Yw.ensure(sizeof(double2) * w.ld * w.nreq);
    w.eps_w.ensure(sizeof(double2) * w.nreq);
    w.res_w.ensure(sizeof(double) * w.nreq);
    total_out += w.nreq;
  }
  const int n_all = (int)total_out;
  c->Uall.ensure(sizeof(double2) * (size_t)c->N * n_all);
  c->ordinfo.ensure(sizeof(int) * 4 * nwin);
  gram_work_ensure(c, (size_t)4 << 20);
  // per-column shift table for the batched stencil
  {
    std::vector<double> sg((size_t)nwin * b);
    for (int j = 0; j < nwin; ++j)
      for (int q = 0; q < b; ++q) sg[(size_t)j * b + q] = c->sigma[j];
    c->sig_dev.ensure(sizeof(double) * std::max<size_t>(sg.size(), 64));
    SWI_CUDA_TRY(cudaMemcpyAsync(c->sig_dev.p, sg.data(), sizeof(double) * sg.size(), cudaMemcpyHostToDevice,
                                 c->stream));
    sync(c->stream);
  }

  // ---- start blocks: random, orthonormalised
  {
    std::vector<Window*> ws;
    std::vector<int> col;
    for (int j = 0; j < nwin; ++j) {
      Window& w = *win[j];
      swi::launch_random_block(w.W.as<double2>(), b, 0, b, c->N, seed * 1000003ull + j, c->stream, &c->launches);
      ws.push_back(&w);
      col.push_back(0);
    }
    cholqr2(c, ws, col, b);
  }

  const swi::StencilParams P = stencil_params(c);
  const double tol_abs = rel_tol * anorm;
  std::vector<int> out_off(nwin);
  {
    int o2 = 0;
    for (int j = 0; j < nwin; ++j) {
      out_off[j] = o2;
      o2 += win[j]->nreq;
    }
  }

  // ---- the batched Krylov-Schur loop
  // Windows expand in lockstep: one launch per kernel serves every expanding
  // window.  A window whose next block would not fit runs its projected
  // eigenproblem (one CTA) on a stream of its own and sits out of the batch
  // until that finishes, so the Schur step overlaps the other windows' GEMMs.
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

  // Act on a finished Schur step of window j: finalise or thick-restart (context stream).
  auto finish_restart = [&](int j) {
    Window& w = *win[j];
    const int* oi = side.oi + 4 * j;
    const int k = oi[0], nconv = oi[1], st = oi[2];
    if (c->prof_on && c->arith != SWI_ARITH_F64) {
      // Hessenberg reduction with accumulation ~ 64/3 m^3 real flops, plus 20
      // flops per complex Givens pair update counted by the kernel
      const double mm = (double)w.p;
      c->schur_flops += 64.0 / 3.0 * mm * mm * mm + 20.0 * 1024.0 * (double)oi[3];
    }
    SWI_CUDA_TRY(cudaStreamWaitEvent(c->stream, side.done[j], 0));
    w.restarts++;
    w.nconv = nconv;
    if (st != 0) w.failed = true;
    if (st != 0 || nconv >= w.nreq || w.matvecs >= budget) {
      swi::RitzBatch fin;
      fin.n = 1;
      fin.job[0] = swi::RitzJob{w.Z.as<double2>(), w.S.as<double2>(), w.theta.as<double2>(), w.resid.as<double>(),
                                c->ordinfo.as<int>() + 4 * j, w.Yw.as<double2>(), w.eps_w.as<double2>(),
                                w.res_w.as<double>(), w.p, w.ld, w.nreq, w.nreq, w.sigma};
      swi::RowGemmBatch rb;
      rb.n = 1;
      rb.job[0] = swi::RowGemmJob{w.Q[w.cur].as<double2>(), w.Yw.as<double2>(), nullptr,
                                  c->Uall.as<double2>() + out_off[j], w.ld, w.nreq, 0, n_all, w.p, w.nreq, 1.0, 0.0};
      ProfScope ps(c, SWI_K_ROTATE, 8.0 * c->N * (double)w.p * w.nreq, 16.0 * c->N * (double)(w.p + w.nreq));
      swi::launch_ritz_batch(fin, c->stream, &c->launches);
      rowgemm_dispatch(c->arith,rb, c->N, c->stream, &c->launches);
      w.done = true;
      return;
    }
    if (k + b > w.m || k < w.nreq) throw Error{SWI_ECUDA, "internal: restart size out of range"};
    swi::ZextBatch zb;
    zb.n = 1;
    zb.job[0] = swi::ZextJob{w.Z.as<double2>(), w.Zext.as<double2>(), w.ld, k + b, w.p, k, b};
    swi::RowGemmBatch rb;
    rb.n = 1;
    rb.job[0] = swi::RowGemmJob{w.Q[w.cur].as<double2>(), w.Zext.as<double2>(), nullptr, w.Q[1 - w.cur].as<double2>(),
                                w.ld, k + b, 0, w.ld, w.p + b, k + b, 1.0, 0.0};
    {
      ProfScope ps(c, SWI_K_ROTATE, 8.0 * c->N * (double)(w.p + b) * (k + b),
                   16.0 * c->N * (double)(w.p + b + k + b));
      swi::launch_zext_batch(zb, c->stream, &c->launches);
      rowgemm_dispatch(c->arith,rb, c->N, c->stream, &c->launches);
    }
    w.cur = 1 - w.cur;
    swi::launch_copy_block(w.Bz.as<double2>(), w.ld, w.Bm.as<double2>(), w.ld, b, k, c->stream, &c->launches);
    w.p = k;
  };

  const long long max_steps = 100000000LL;
  for (long long step = 0; step < max_steps; ++step) {
    // Keep the host at most two steps ahead of the device.  Unbounded, the
    // launch queue holds ~1 s of steps, and a window whose Schur step has
    // finished would rejoin the batch only behind all of them, idle meanwhile.
    if (step >= 2) SWI_CUDA_TRY(cudaEventSynchronize(side.lag[step & 1]));
    // collect finished restarts
    for (int j = 0; j < nwin; ++j) {
      if (!in_schur[j]) continue;
      const cudaError_t q = cudaEventQuery(side.done[j]);
      if (q == cudaErrorNotReady) continue;
      SWI_CUDA_TRY(q);
      in_schur[j] = 0;
      finish_restart(j);
    }
    std::vector<Window*> act;
    std::vector<int> idx;
    int pending = -1;
    for (int j = 0; j < nwin; ++j) {
      if (win[j]->done) continue;
      if (in_schur[j]) {
        if (pending < 0) pending = j;
        continue;
      }
      act.push_back(win[j].get());
      idx.push_back(j);
    }
    if (act.empty()) {
      if (pending < 0) break;
      SWI_CUDA_TRY(cudaEventSynchronize(side.done[pending]));
      continue;
    }
    const int na = (int)act.size();
    // 1) W_j = (A - sigma_j) V_j for every active window, one launch
    {
      swi::StencilBatch sb;
      sb.n = na;
      for (int q = 0; q < na; ++q) {
        Window& w = *act[q];
        if (w.p + 2 * b > w.ld) throw Error{SWI_ECUDA, "internal: Krylov block beyond the basis buffer"};
        sb.blk[q] = swi::StencilBlock{w.Q[w.cur].as<double2>() + w.p, w.W.as<double2>(), w.ld, b, b, idx[q] * b};
      }
      const double Nn = (double)c->N;
      ProfScope ps(c, SWI_K_STENCIL, kStencilFlops * Nn * b * na, (32.0 * b + 16.0) * Nn * na);
      if (c->arith == SWI_ARITH_F64)
        swi::launch_stencil(P, sb, c->sig_dev.as<double>(), c->stream, &c->launches);
      else
        swi::launch_stencil_ds(P, sb, c->sig_dev.as<double>(), c->stream, &c->launches);
    }
    // 2) block classical Gram-Schmidt, twice, against [Q_j V_j]
    for (int pass = 0; pass < 2; ++pass) {
      swi::GramBatch gb;
      gb.n = na;
      swi::RowGemmBatch rb;
      rb.n = na;
      double ncol = 0.0;
      for (int q = 0; q < na; ++q) {
        Window& w = *act[q];
        double2* C = (pass == 0 ? w.C1 : w.C2).as<double2>();
        gb.job[q] = swi::GramJob{w.Q[w.cur].as<double2>(), w.W.as<double2>(), C, w.ld, b, b, w.p + b, b, 0};
        rb.job[q] = swi::RowGemmJob{w.Q[w.cur].as<double2>(), C, w.W.as<double2>(), w.W.as<double2>(),
                                    w.ld, b, b, b, w.p + b, b, -1.0, 1.0};
        ncol += w.p + b;
      }
      const double Nn = (double)c->N;
      {
        ProfScope ps(c, SWI_K_GRAM, 8.0 * Nn * ncol * b, 16.0 * Nn * (ncol + na * b));
        gram_dispatch(c->arith,gb, c->N, nullptr, 0, c->gram_work.as<double2>(), c->gram_work.bytes / sizeof(double2),
                         c->stream, &c->launches);
      }
      {
        ProfScope ps(c, SWI_K_UPDATE, 8.0 * Nn * ncol * b, 16.0 * Nn * (ncol + 2.0 * na * b));
        rowgemm_dispatch(c->arith,rb, c->N, c->stream, &c->launches);
      }
    }
    // 3) Cholesky-QR2 of the remainder into Q_j[:, p+b : p+2b]
    {
      std::vector<int> col(na);
      for (int q = 0; q < na; ++q) col[q] = act[q]->p + b;
      const double Nn = (double)c->N;
      ProfScope ps(c, SWI_K_CHOLQR, 4.0 * 8.0 * Nn * b * b * na, 5.0 * 16.0 * Nn * b * na);
      cholqr2(c, act, col, b);
    }
    // 4) projected matrix and coupling rows
    {
      swi::HUpdBatch hb;
      hb.n = na;
      for (int q = 0; q < na; ++q) {
        Window& w = *act[q];
        hb.job[q] = swi::HUpdJob{w.H.as<double2>(), w.Bm.as<double2>(), w.C1.as<double2>(), w.C2.as<double2>(),
                                 w.R1.as<double2>(), w.R2.as<double2>(), w.ld, w.p, b};
      }
      swi::launch_hupdate_batch(hb, c->stream, &c->launches);
    }
    // 5) windows whose next block would not fit: Schur step on their own stream
    for (int q = 0; q < na; ++q) {
      Window& w = *act[q];
      const int j = idx[q];
      w.p += b;
      w.matvecs += b;
      if (w.p + b <= w.m) continue;
      if (w.p > w.m || w.keep + b > w.m) throw Error{SWI_ECUDA, "internal: basis bookkeeping out of range"};
      // As ARPACK does, keep more Ritz vectors once some wanted pairs have
      // converged, so the rest keep room in the restarted basis.
      const int keep_eff = std::min(w.m - b, w.keep + std::min(w.nconv, (w.m - w.keep) / 2));
      swi::SchurBatch sb;
      sb.n = 1;
      sb.job[0] = swi::SchurJob{w.H.as<double2>(), w.Z.as<double2>(), w.Bm.as<double2>(), w.Bz.as<double2>(),
                                w.theta.as<double2>(), w.resid.as<double>(), w.S.as<double2>(),
                                c->ordinfo.as<int>() + 4 * j, w.p, w.ld, b, keep_eff, w.nreq, w.m - b, tol_abs,
                                w.Hw.p, w.Zw.p};
      SWI_CUDA_TRY(cudaEventRecord(side.ready[j], c->stream));
      SWI_CUDA_TRY(cudaStreamWaitEvent(side.st[j], side.ready[j], 0));
      {
        ProfScope ps(c, SWI_K_SCHUR, 0.0, 0.0, side.st[j]);
        if (c->arith == SWI_ARITH_F64) swi::launch_schur_batch(sb, side.st[j], &c->launches);
        else swi::launch_schur_ds_batch(sb, side.st[j], &c->launches);
      }
      SWI_CUDA_TRY(cudaMemcpyAsync(side.oi + 4 * j, c->ordinfo.as<int>() + 4 * j, sizeof(int) * 4,
                                   cudaMemcpyDeviceToHost, side.st[j]));
      SWI_CUDA_TRY(cudaEventRecord(side.done[j], side.st[j]));
      in_schur[j] = 1;
    }
    SWI_CUDA_TRY(cudaEventRecord(side.lag[step & 1], c->stream));
  }
  // ---- gather eigenvalue estimates and window statistics
  std::vector<double2> eps_all(n_all);
  std::vector<int> win_of(n_all);
  c->winfo.assign(nwin, swi_window_info());
  bool any_fail = false, any_noconv = false;
  for (int j = 0; j < nwin; ++j) {
    Window& w = *win[j];
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
    any_fail |= w.failed;
    any_noconv |= (w.nconv < w.nreq);
  }
  win.clear();  // free the Krylov bases before the merge
  const double t1 = swi::now_seconds();

  // ---- Algorithm 2 merge, selection, U^T U = I
  int minfo[4];
  merge_pairs(c, c->Uall.as<double2>(), n_all, eps_all, win_of, nwin, eq_rtol, drop_tol, opt.n_keep, minfo);
  record_windows(c, eps_all, win_of, nwin);
  const int nout = minfo[0];
  c->Uall.release();
  // explicit FP64 residuals of the delivered pairs
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
  if (any_fail) return fail(c, SWI_ENOCONV, "a window's projected eigenproblem did not converge");
  if (minfo[3] != 0) return fail(c, SWI_EINVAL, "merge: equal-eigenvalue component too large");
  if (any_noconv) return fail(c, SWI_ENOCONV, "some window did not converge within its matvec budget");
  if (minfo[2] > 0) return fail(c, SWI_HOLES, std::to_string(minfo[2]) + " interface(s) without redundancy");
  return SWI_OK;
}

// Residual-correction sweeps (Rayleigh-Ritz on span[U_g, R_u] per group of
// consecutive pairs, in the unconjugated form under which the eigenvectors of
// the complex-symmetric A are bi-orthogonal, then Algorithm 2 over all pairs as
// one window); see swi_refine in swi.h.
swi_status do_refine(swi_ctx* c, const swi_refine_opts* o, swi_refine_info* info) {
  if (c->npairs <= 0) return fail(c, SWI_ESTATE, "no eigenpairs");
  if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set");
  swi_refine_opts opt;
  std::memset(&opt, 0, sizeof(opt));
  if (o) opt = *o;
  const int max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : 3;
  const int g = opt.group > 0 ? opt.group : 16;
  if (g > 32) return fail(c, SWI_EINVAL, "group must be <= 32");
  if (opt.arith != 0 && opt.arith != SWI_ARITH_DS && opt.arith != SWI_ARITH_F64)
    return fail(c, SWI_EINVAL, "unknown arithmetic");
  if (opt.rel_tol < 0 || opt.eq_rtol < 0 || opt.drop_tol < 0) return fail(c, SWI_EINVAL, "negative tolerance");
  const double rel_tol = opt.rel_tol > 0 ? opt.rel_tol : 1e-10;
  const double near_tol = opt.near_tol > 0 ? opt.near_tol : 1e-3;
  const double eq_rtol = opt.eq_rtol > 0 ? opt.eq_rtol : 1e-8;
  const double drop_tol = opt.drop_tol > 0 ? opt.drop_tol : 1e-6;
  c->arith = opt.arith == SWI_ARITH_F64 ? SWI_ARITH_F64 : SWI_ARITH_DS;
  const double t0 = swi::now_seconds();
  const size_t N = c->N;
  if ((size_t)2 * g > N) return fail(c, SWI_EINVAL, "group larger than half the problem dimension");

  // one group's workspace, reused group after group on the context's stream
  Window w;
  const int ld = 2 * g;
  w.ld = ld;
  w.Q[0].ensure(sizeof(double2) * N * ld);
  w.W.ensure(sizeof(double2) * N * g);
  w.C1.ensure(sizeof(double2) * ld * g);
  w.C2.ensure(sizeof(double2) * ld * g);
  w.G.ensure(sizeof(double2) * g * g);
  w.R1.ensure(sizeof(double2) * g * g);
  w.R1i.ensure(sizeof(double2) * g * g);
  w.R2.ensure(sizeof(double2) * g * g);
  w.R2i.ensure(sizeof(double2) * g * g);
  w.H.ensure(sizeof(double2) * ld * ld);
  w.Z.ensure(sizeof(double2) * ld * ld);
  w.S.ensure(sizeof(double2) * ld * ld);
  w.Bm.ensure(sizeof(double2) * ld);
  w.Bz.ensure(sizeof(double2) * ld);
  w.theta.ensure(sizeof(double2) * ld);
  w.resid.ensure(sizeof(double) * ld);
  w.Yw.ensure(sizeof(double2) * ld * g);
  w.eps_w.ensure(sizeof(double2) * g);
  w.res_w.ensure(sizeof(double) * g);
  if (c->arith != SWI_ARITH_F64) {
    w.Hw.ensure(16 * (size_t)ld * ld);
    w.Zw.ensure(16 * (size_t)ld * ld);
  }
  SWI_CUDA_TRY(cudaMemsetAsync(w.Bm.p, 0, sizeof(double2) * ld, c->stream));  // no residual coupling
  DevMem Xu, AQ, Sb, Unew, epsnew, eu, idx_dev, oinfo, sstat;
  Sb.ensure(sizeof(double2) * ld * ld);
  Xu.ensure(sizeof(double2) * N * g);
  AQ.ensure(sizeof(double2) * N * ld);
  gram_work_ensure(c, (size_t)4 << 20);
  c->sig_dev.ensure(sizeof(double) * std::max(ld, 64));

  long long mv = 0;
  int n_dropped = 0, sweeps = 0;
  if (c->resid.size() != (size_t)c->npairs) {
    explicit_residuals(c, c->U.as<double2>(), c->npairs, c->eps.as<double2>(), c->npairs, c->resid);
    mv += c->npairs;
  }
  double max_in = 0.0;
  for (double r : c->resid) max_in = std::max(max_in, r);
  auto all_converged = [&]() {
    for (double r : c->resid)
      if (!(r <= rel_tol)) return false;
    return true;
  };
  while (sweeps < max_sweeps && !all_converged()) {
    const int n = c->npairs;
    const int ngroups = (n + g - 1) / g;
    std::vector<double2> eh(n);
    SWI_CUDA_TRY(cudaMemcpyAsync(eh.data(), c->eps.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    // unconverged pairs of every group, uploaded once
    std::vector<int> idx, ioff(ngroups + 1, 0);
    for (int gi = 0; gi < ngroups; ++gi) {
      double gmax = 0.0;
      for (int k = gi * g; k < std::min(n, gi * g + g); ++k) gmax = std::max(gmax, c->resid[k]);
      if (gmax <= near_tol)  // a group far from convergence is left as it is
        for (int k = gi * g; k < std::min(n, gi * g + g); ++k)
          if (!(c->resid[k] <= rel_tol)) idx.push_back(k);
      ioff[gi + 1] = (int)idx.size();
    }
    idx_dev.ensure(sizeof(int) * std::max<size_t>(idx.size(), 1));
    SWI_CUDA_TRY(cudaMemcpyAsync(idx_dev.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, c->stream));
    Unew.ensure(sizeof(double2) * N * n);
    epsnew.ensure(sizeof(double2) * n);
    eu.ensure(sizeof(double2) * g);
    oinfo.ensure(sizeof(int) * 4 * ngroups);
    SWI_CUDA_TRY(cudaMemsetAsync(oinfo.p, 0, sizeof(int) * 4 * ngroups, c->stream));
    sstat.ensure(sizeof(int) * ngroups);
    SWI_CUDA_TRY(cudaMemsetAsync(sstat.p, 0, sizeof(int) * ngroups, c->stream));
    std::vector<Window*> ws{&w};
    for (int gi = 0; gi < ngroups; ++gi) {
      const int lo = gi * g, ng = std::min(g, n - lo), nu = ioff[gi + 1] - ioff[gi];
      double2* Ug = c->U.as<double2>() + lo;
      if (nu == 0) {  // converged group: kept as it is
        swi::launch_copy_block(Ug, n, Unew.as<double2>() + lo, n, c->N, ng, c->stream, &c->launches);
        SWI_CUDA_TRY(cudaMemcpyAsync(epsnew.as<double2>() + lo, c->eps.as<double2>() + lo, sizeof(double2) * ng,
                                     cudaMemcpyDeviceToDevice, c->stream));
        continue;
      }
      const int m = ng + nu;
      const int* ig = idx_dev.as<int>() + ioff[gi];
      // Q[:, 0:ng] = orthonormal basis of U_g
      swi::launch_copy_block(Ug, n, w.W.as<double2>(), ng, c->N, ng, c->stream, &c->launches);
      cholqr2(c, ws, {0}, ng);
      // R_u = A U_u - U_u diag(eps_u)
      swi::launch_gather_cols(Ug - lo, n, ig, nu, Xu.as<double2>(), nu, c->N, c->stream, &c->launches);
      swi::launch_gather_cols(c->eps.as<double2>(), 0, ig, nu, eu.as<double2>(), 0, 1, c->stream, &c->launches);
      SWI_CUDA_TRY(cudaMemsetAsync(c->sig_dev.p, 0, sizeof(double) * nu, c->stream));
      apply_block(c, Xu.as<double2>(), nu, w.W.as<double2>(), nu, nu);
      swi::launch_sub_diag(w.W.as<double2>(), nu, Xu.as<double2>(), nu, eu.as<double2>(), nu, c->N, c->stream,
                           &c->launches);
      // block Gram-Schmidt twice against Q[:, 0:ng], then Cholesky-QR2 into Q[:, ng:m]
      for (int pass = 0; pass < 2; ++pass) {
        swi::GramBatch gb;
        gb.n = 1;
        gb.job[0] = swi::GramJob{w.Q[0].as<double2>(), w.W.as<double2>(), w.C1.as<double2>(), ld, nu, nu, ng, nu, 0};
        gram_dispatch(c->arith, gb, c->N, nullptr, 0, c->gram_work.as<double2>(),
                      c->gram_work.bytes / sizeof(double2), c->stream, &c->launches);
        swi::RowGemmBatch rb;
        rb.n = 1;
        rb.job[0] = swi::RowGemmJob{w.Q[0].as<double2>(), w.C1.as<double2>(), w.W.as<double2>(), w.W.as<double2>(),
                                    ld, nu, nu, nu, ng, nu, -1.0, 1.0};
        rowgemm_dispatch(c->arith, rb, c->N, c->stream, &c->launches);
      }
      cholqr2(c, ws, {ng}, nu);
      // (A - sigma_g) Q, sigma_g the middle of the group's real parts
      double rmin = eh[lo].x, rmax = eh[lo].x;
      for (int k = lo; k < lo + ng; ++k) {
        rmin = std::min(rmin, eh[k].x);
        rmax = std::max(rmax, eh[k].x);
      }
      const double sigma_g = 0.5 * (rmin + rmax);
      {
        std::vector<double> sg(m, sigma_g);
        SWI_CUDA_TRY(cudaMemcpyAsync(c->sig_dev.p, sg.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
        apply_block(c, w.Q[0].as<double2>(), ld, AQ.as<double2>(), ld, m);
        sync(c->stream);  // sg leaves scope
      }
      {
        // the pencil in the unconjugated form: K = Q^T (A - sigma_g) Q, S = Q^T Q, H = S^-1 K
        swi::GramBatch gb;
        gb.n = 1;
        gb.job[0] = swi::GramJob{w.Q[0].as<double2>(), AQ.as<double2>(), w.H.as<double2>(), ld, ld, ld, m, m, 0};
        gram_dispatch(c->arith, gb, c->N, nullptr, 1, c->gram_work.as<double2>(),
                      c->gram_work.bytes / sizeof(double2), c->stream, &c->launches);
        gb.job[0] = swi::GramJob{w.Q[0].as<double2>(), w.Q[0].as<double2>(), Sb.as<double2>(), ld, ld, ld, m, m, 0};
        gram_dispatch(c->arith, gb, c->N, nullptr, 1, c->gram_work.as<double2>(),
                      c->gram_work.bytes / sizeof(double2), c->stream, &c->launches);
        swi::launch_small_solve(Sb.as<double2>(), w.H.as<double2>(), m, ld, sstat.as<int>() + gi, c->stream,
                                &c->launches);
      }
      // Schur form, the ng Ritz values of smallest magnitude, their vectors
      swi::SchurBatch sb;
      sb.n = 1;
      sb.job[0] = swi::SchurJob{w.H.as<double2>(), w.Z.as<double2>(), w.Bm.as<double2>(), w.Bz.as<double2>(),
                                w.theta.as<double2>(), w.resid.as<double>(), w.S.as<double2>(),
                                oinfo.as<int>() + 4 * gi, m, ld, 1, ng, ng, ng, 1.0, w.Hw.p, w.Zw.p};
      // the group's projected problem is small (order <= 2 n_g): native FP64
      swi::launch_schur_batch(sb, c->stream, &c->launches);
      swi::RitzBatch fin;
      fin.n = 1;
      fin.job[0] = swi::RitzJob{w.Z.as<double2>(), w.S.as<double2>(), w.theta.as<double2>(), w.resid.as<double>(),
                                oinfo.as<int>() + 4 * gi, w.Yw.as<double2>(), w.eps_w.as<double2>(),
                                w.res_w.as<double>(), m, ld, ng, ng, sigma_g};
      swi::launch_ritz_batch(fin, c->stream, &c->launches);
      swi::RowGemmBatch rb;
      rb.n = 1;
      rb.job[0] = swi::RowGemmJob{w.Q[0].as<double2>(), w.Yw.as<double2>(), nullptr, Unew.as<double2>() + lo, ld, ng, 0,
                                  n, m, ng, 1.0, 0.0};
      rowgemm_dispatch(c->arith, rb, c->N, c->stream, &c->launches);
      SWI_CUDA_TRY(cudaMemcpyAsync(epsnew.as<double2>() + lo, w.eps_w.p, sizeof(double2) * ng,
                                   cudaMemcpyDeviceToDevice, c->stream));
      mv += nu + m;
    }
    std::vector<int> oi(4 * ngroups), si(ngroups);
    std::vector<double2> en(n);
    SWI_CUDA_TRY(cudaMemcpyAsync(oi.data(), oinfo.p, sizeof(int) * 4 * ngroups, cudaMemcpyDeviceToHost, c->stream));
    SWI_CUDA_TRY(cudaMemcpyAsync(si.data(), sstat.p, sizeof(int) * ngroups, cudaMemcpyDeviceToHost, c->stream));
    SWI_CUDA_TRY(cudaMemcpyAsync(en.data(), epsnew.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    for (int gi = 0; gi < ngroups; ++gi) {
      if (si[gi] != 0) return fail(c, SWI_ENOCONV, "refine: singular Q^T Q in a group");
      if (oi[4 * gi + 2] != 0) return fail(c, SWI_ENOCONV, "refine: a projected eigenproblem did not converge");
    }
    // a group's Rayleigh-Ritz pairs replace its previous ones unless they
    // lower the number of the group's pairs at rel_tol or raise its largest
    // explicit residual more than tenfold (a sweep sharpens eigenvalues, which
    // a residual need not show; far from convergence, though, it can move
    // pairs away from converged ones)
    {
      std::vector<double> rn;
      explicit_residuals(c, Unew.as<double2>(), n, epsnew.as<double2>(), n, rn);
      mv += n;
      for (int gi = 0; gi < ngroups; ++gi) {
        const int lo = gi * g, ng = std::min(g, n - lo);
        if (ioff[gi + 1] == ioff[gi]) continue;
        double before = 0.0, after = 0.0;
        int conv_before = 0, conv_after = 0;
        for (int k = lo; k < lo + ng; ++k) {
          before = std::max(before, c->resid[k]);
          after = std::max(after, rn[k]);
          conv_before += c->resid[k] <= rel_tol;
          conv_after += rn[k] <= rel_tol;
        }
        if (conv_after >= conv_before && after <= 10.0 * before) continue;
        swi::launch_copy_block(c->U.as<double2>() + lo, n, Unew.as<double2>() + lo, n, c->N, ng, c->stream,
                               &c->launches);
        SWI_CUDA_TRY(cudaMemcpyAsync(epsnew.as<double2>() + lo, c->eps.as<double2>() + lo, sizeof(double2) * ng,
                                     cudaMemcpyDeviceToDevice, c->stream));
        SWI_CUDA_TRY(cudaMemcpyAsync(en.data() + lo, c->eps.as<double2>() + lo, sizeof(double2) * ng,
                                     cudaMemcpyDeviceToHost, c->stream));
      }
      sync(c->stream);
    }
    // Algorithm 2 over the refined pairs as one window, U^T U = I
    int minfo[4];
    merge_pairs(c, Unew.as<double2>(), n, en, std::vector<int>(n, 0), 1, eq_rtol, drop_tol, 0, minfo);
    if (minfo[3] != 0) return fail(c, SWI_EINVAL, "merge: equal-eigenvalue component too large");
    n_dropped += minfo[1];
    explicit_residuals(c, c->U.as<double2>(), c->npairs, c->eps.as<double2>(), c->npairs, c->resid);
    mv += c->npairs;
    ++sweeps;
  }
  int nconv = 0;
  double maxr = 0.0;
  for (double r : c->resid) {
    if (r <= rel_tol) ++nconv;
    maxr = std::max(maxr, r);
  }
  if (info) {
    info->sweeps = sweeps;
    info->n_pairs = c->npairs;
    info->n_converged = nconv;
    info->n_dropped = n_dropped;
    info->matvecs = mv;
    info->max_rel_res_in = max_in;
    info->max_rel_res = maxr;
    info->t_s = swi::now_seconds() - t0;
  }
  if (nconv < c->npairs) return fail(c, SWI_ENOCONV, "pairs above rel_tol after the last sweep");
  return SWI_OK;
}

void ensure_RL(swi_ctx* c) {
  if (c->have_RL) return;
  const int n = c->npairs;
  const size_t nn = (size_t)n * n;
  c->MR.ensure(sizeof(double2) * nn);
  c->ML.ensure(sizeof(double2) * nn);
  c->Rm.ensure(sizeof(double2) * nn);
  c->Lm.ensure(sizeof(double2) * nn);
  c->Wm.ensure(sizeof(double2) * nn);
  if (c->contract == SWI_CONTRACT_F32) {
    const long long rR = c->gR_hi - c->gR_lo, rL = c->gL_hi - c->gL_lo;
    const int kR = swi::proj_f32_chunks(n, rR), kL = swi::proj_f32_chunks(n, rL);
    c->R32.ensure(sizeof(float2) * nn);
    c->L32.ensure(sizeof(float2) * nn);
    c->part32.ensure(sizeof(float2) * nn * (size_t)std::max(kR + kL, 1));
    const double2* U = c->U.as<double2>();
    ProfScope ps(c, SWI_K_PROJ, 8.0 * (double)(rR + rL) * n * n, 16.0 * (double)(rR + rL) * n + 8.0 * (rR + rL));
    swi::launch_proj_f32(U, n, n, c->gR.as<double>(), c->gR_lo, c->gR_hi, c->gL.as<double>(), c->gL_lo, c->gL_hi,
                         c->part32.as<float2>(), c->Rm.as<double2>(), c->Lm.as<double2>(), c->Wm.as<double2>(),
                         c->R32.as<float2>(), c->L32.as<float2>(), c->stream, &c->launches);
    c->have_RL = true;
    return;
  }
  gram_work_ensure(c, nn * 4);
  ProfScope ps(c, SWI_K_PROJ, 2.0 * 8.0 * c->N * (double)n * n, 2.0 * 16.0 * c->N * (double)n + 16.0 * c->N);
  swi::GramBatch gb;
  gb.n = 1;
  gb.job[0] = swi::GramJob{c->U.as<double2>(), c->U.as<double2>(), c->MR.as<double2>(), n, n, n, n, n, 0};
  gram_dispatch(c->arith,gb, c->N, c->gR.as<double>(), 0, c->gram_work.as<double2>(), c->gram_work.bytes / sizeof(double2),
                   c->stream, &c->launches);
  gb.job[0].C = c->ML.as<double2>();
  gram_dispatch(c->arith,gb, c->N, c->gL.as<double>(), 0, c->gram_work.as<double2>(), c->gram_work.bytes / sizeof(double2),
                   c->stream, &c->launches);
  swi::launch_wbuild(c->MR.as<double2>(), c->ML.as<double2>(), n, c->Rm.as<double2>(), c->Lm.as<double2>(),
                     c->Wm.as<double2>(), c->stream, &c->launches);
  c->have_RL = true;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// T(E) without any allocation, for callers that must not allocate device
// memory at call time (see swi_transmission_noalloc in swi.h).  All scratch
// lives in one file-scope device array, shared by every call on a device.
namespace {
constexpr int kNoAllocMaxPairs = 64;
constexpr int kNoAllocMaxEnergies = 1024;
constexpr size_t kNoAllocMat = (size_t)kNoAllocMaxPairs * kNoAllocMaxPairs;  // one n x n matrix
constexpr size_t kNoAllocWork = 64 * kNoAllocMat;                            // split-N partial sums
constexpr int kNoAllocSlab = 64 * 1024;  // grid rows per projection pass: 64 chunks of 1024 rows
// layout: MR, ML, R, L, W (n x n each), Gram partial sums, then E[1024], T[1024] as doubles
constexpr size_t kNoAllocElems = 5 * kNoAllocMat + kNoAllocWork + kNoAllocMaxEnergies;
}  // namespace

static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocElems];  // 4.6 MB per device

namespace {
std::mutex g_noalloc_mutex;
std::vector<void*> g_noalloc_addr;  // device address of g_noalloc_scratch, per device ordinal

// Once per device, with that device current: the array's device address.
double2* noalloc_scratch(int device) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if ((int)g_noalloc_addr.size() <= device) g_noalloc_addr.resize(device + 1, nullptr);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw Error{SWI_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    g_noalloc_addr[device] = p;
  }
  return static_cast<double2*>(g_noalloc_addr[device]);
}
}  // namespace

extern "C" {

swi_status swi_create(swi_ctx** out, int nx, int ny, int nz, double h, int bc, int precision, void* cuda_stream) {
  if (!out) return fail(nullptr, SWI_EINVAL, "out is NULL");
  *out = nullptr;
  if (nx < 6 || ny < 6 || nz < 6) return fail(nullptr, SWI_EINVAL, "each axis needs at least 6 points");
  if (!(h > 0.0) || !std::isfinite(h)) return fail(nullptr, SWI_EINVAL, "grid spacing must be positive");
  if (bc != SWI_BC_ODD && bc != SWI_BC_ZERO) return fail(nullptr, SWI_EINVAL, "unknown boundary rule");
  if (precision != SWI_PREC_F64 && precision != SWI_PREC_MIXED) return fail(nullptr, SWI_EINVAL, "unknown precision");
  const long long N = (long long)nx * ny * nz;
  if (N > (1LL << 31) - 1) return fail(nullptr, SWI_EINVAL, "grid too large");
  swi_ctx* c = nullptr;
  try {
    c = new swi_ctx();
  } catch (...) {
    return fail(nullptr, SWI_ENOMEM, "host allocation failed");
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(nullptr, SWI_ECUDA, "no CUDA device");
  }
  try {
    noalloc_scratch(c->device);  // device address of the no-allocation scratch, once per device
  } catch (const Error& e) {
    delete c;
    return fail(nullptr, e.code, e.msg);
  }
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->N = (int)N;
  c->h = h;
  c->bc = bc;
  c->precision = precision;
  *out = c;
  return SWI_OK;
}

// the packed (V, Gamma) planes of the TMA-staged complex64 stencil, once both are set
static void refresh_vg(swi_ctx* c) {
  if (!c->has_V || !c->has_G) return;
  const size_t nxp = (size_t)(c->nx + (c->nx & 1));
  c->VG32.ensure(sizeof(float2) * nxp * c->ny * c->nz);
  swi::launch_pack_vg(c->V32.as<float>(), c->G32.as<float>(), c->nx, c->ny, c->nz, c->VG32.as<float2>(), c->stream);
  sync(c->stream);
}

swi_status swi_set_potential(swi_ctx* c, const double* V, int on_device) {
  return guarded(c, [&]() -> swi_status {
    if (!V) return fail(c, SWI_EINVAL, "V is NULL");
    const size_t n = c->N;
    std::vector<double> h(n);
    if (on_device) {
      SWI_CUDA_TRY(cudaMemcpy(h.data(), V, sizeof(double) * n, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(h.data(), V, sizeof(double) * n);
    }
    if (!finite_all(h.data(), n)) return fail(c, SWI_EINVAL, "V has a non-finite value");
    double mx = 0.0;
    for (double v : h) mx = std::max(mx, std::fabs(v));
    copy_in(c->V, h.data(), sizeof(double) * n, false, c->stream);
    {
      std::vector<float> f(h.begin(), h.end());
      copy_in(c->V32, f.data(), sizeof(float) * n, false, c->stream);
      sync(c->stream);
    }
    sync(c->stream);
    c->maxabsV = mx;
    c->has_V = true;
    refresh_vg(c);
    return SWI_OK;
  });
}

swi_status swi_set_absorber(swi_ctx* c, const double* gL, const double* gR, int on_device) {
  return guarded(c, [&]() -> swi_status {
    if (!gL || !gR) return fail(c, SWI_EINVAL, "absorber is NULL");
    const size_t n = c->N;
    std::vector<double> l(n), r(n), g(n);
    if (on_device) {
      SWI_CUDA_TRY(cudaMemcpy(l.data(), gL, sizeof(double) * n, cudaMemcpyDeviceToHost));
      SWI_CUDA_TRY(cudaMemcpy(r.data(), gR, sizeof(double) * n, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(l.data(), gL, sizeof(double) * n);
      std::memcpy(r.data(), gR, sizeof(double) * n);
    }
    double mx = 0.0;
    long long lo[2] = {-1, -1}, hi[2] = {0, 0};
    for (size_t i = 0; i < n; ++i) {
      if (!std::isfinite(l[i]) || !std::isfinite(r[i]) || l[i] < 0.0 || r[i] < 0.0)
        return fail(c, SWI_EINVAL, "absorbers must be finite and non-negative");
      g[i] = l[i] + r[i];
      mx = std::max(mx, g[i]);
      // rows whose FP32 absorber is a normal number (those of the FP32 projections)
      const double v[2] = {l[i], r[i]};
      for (int k = 0; k < 2; ++k)
        if ((float)v[k] >= FLT_MIN) {
          if (lo[k] < 0) lo[k] = (long long)i;
          hi[k] = (long long)i + 1;
        }
    }
    copy_in(c->gL, l.data(), sizeof(double) * n, false, c->stream);
    copy_in(c->gR, r.data(), sizeof(double) * n, false, c->stream);
    copy_in(c->G, g.data(), sizeof(double) * n, false, c->stream);
    {
      std::vector<float> f(g.begin(), g.end());
      copy_in(c->G32, f.data(), sizeof(float) * n, false, c->stream);
      sync(c->stream);
    }
    sync(c->stream);
    c->maxG = mx;
    c->gL_lo = lo[0] < 0 ? 0 : lo[0];
    c->gL_hi = lo[0] < 0 ? 0 : hi[0];
    c->gR_lo = lo[1] < 0 ? 0 : lo[1];
    c->gR_hi = lo[1] < 0 ? 0 : hi[1];
    c->has_G = true;
    c->have_RL = false;
    refresh_vg(c);
    return SWI_OK;
  });
}

swi_status swi_set_windows(swi_ctx* c, int p, const double* sigma, const int* n_req) {
  return guarded(c, [&]() -> swi_status {
    if (p < 1 || !sigma || !n_req) return fail(c, SWI_EINVAL, "need p >= 1 windows");
    if (p > swi::kMaxBatch) return fail(c, SWI_EINVAL, "at most 64 windows");
    for (int j = 0; j < p; ++j) {
      if (!std::isfinite(sigma[j])) return fail(c, SWI_EINVAL, "non-finite shift");
      if (n_req[j] < 1) return fail(c, SWI_EINVAL, "each window needs n_req >= 1");
      if (j > 0 && !(sigma[j] > sigma[j - 1])) return fail(c, SWI_EINVAL, "shifts must be strictly increasing");
    }
    c->sigma.assign(sigma, sigma + p);
    c->sigma_im.clear();  // real shifts
    c->nreq.assign(n_req, n_req + p);
    return SWI_OK;
  });
}

swi_status swi_set_windows_complex(swi_ctx* c, int p, const double* sigma_re, const double* sigma_im,
                                   const int* n_req) {
  return guarded(c, [&]() -> swi_status {
    if (p < 1 || !sigma_re || !sigma_im || !n_req) return fail(c, SWI_EINVAL, "need p >= 1 windows");
    if (p > swi::kMaxBatch) return fail(c, SWI_EINVAL, "at most 64 windows");
    for (int j = 0; j < p; ++j) {
      if (!std::isfinite(sigma_re[j]) || !std::isfinite(sigma_im[j])) return fail(c, SWI_EINVAL, "non-finite shift");
      if (n_req[j] < 1) return fail(c, SWI_EINVAL, "each window needs n_req >= 1");
      if (j > 0 && !(sigma_re[j] > sigma_re[j - 1] || (sigma_re[j] == sigma_re[j - 1] && sigma_im[j] > sigma_im[j - 1])))
        return fail(c, SWI_EINVAL, "shifts must be strictly increasing by (Re, Im)");
    }
    c->sigma.assign(sigma_re, sigma_re + p);
    c->sigma_im.assign(sigma_im, sigma_im + p);
    c->nreq.assign(n_req, n_req + p);
    return SWI_OK;
  });
}

swi_status swi_plan_windows(swi_ctx* c, int n_r, int p, double e_min, double e_max, double inflate,
                            double* sigma_out, int* n_req_out) {
  return guarded(c, [&]() -> swi_status {
    if (n_r < 1 || p < 1 || p > swi::kMaxBatch) return fail(c, SWI_EINVAL, "need n_r >= 1 and 1 <= p <= 64");
    if (!(e_max > e_min)) return fail(c, SWI_EINVAL, "need e_max > e_min");
    if (!(inflate >= 1.0)) inflate = 1.0;
    // Algorithm 1: n_r,j (round / ceil heuristics), then E_S,j
    std::vector<long long> cnt(p + 1, 0);
    for (int j = 1; j <= p; ++j) {
      if (j <= p / 2.0) {
        const double x = 2.0 / (1.5 + (double)(j - 1) / p) * (double)n_r / p;
        cnt[j] = (long long)std::floor(x + 0.5);
      } else {
        cnt[j] = (long long)std::ceil(2.0 * n_r / p) - cnt[p - j + 1];
      }
    }
    std::vector<double> sg(p);
    std::vector<int> rq(p);
    const double step = (e_max - e_min) / c->N;
    double prev_s = e_min;
    long long prev_n = 0;
    for (int j = 1; j <= p; ++j) {
      const double s = prev_s + step * (double)(cnt[j] + prev_n) / 2.0;
      sg[j - 1] = s;
      rq[j - 1] = (int)std::max(1LL, (long long)std::ceil(cnt[j] * inflate));
      prev_s = s;
      prev_n = cnt[j];
    }
    for (int j = 1; j < p; ++j)
      if (!(sg[j] > sg[j - 1])) return fail(c, SWI_EINVAL, "plan produced non-increasing shifts");
    if (sigma_out) std::copy(sg.begin(), sg.end(), sigma_out);
    if (n_req_out) std::copy(rq.begin(), rq.end(), n_req_out);
    c->sigma = sg;
    c->sigma_im.clear();  // real shifts
    c->nreq = rq;
    return SWI_OK;
  });
}

swi_status apply_impl(swi_ctx* c, int nvec, const double* sigma, const void* X, void* Y, int on_device, bool ds) {
  return guarded(c, [&]() -> swi_status {
    if (nvec < 1 || !sigma || !X || !Y) return fail(c, SWI_EINVAL, "bad arguments");
    if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set");
    const size_t bytes = sizeof(double2) * (size_t)c->N * nvec;
    c->sig_dev.ensure(sizeof(double) * std::max(nvec, 64));
    SWI_CUDA_TRY(cudaMemcpyAsync(c->sig_dev.p, sigma, sizeof(double) * nvec, cudaMemcpyHostToDevice, c->stream));
    if (on_device) {
      apply_block(c, static_cast<const double2*>(X), nvec, static_cast<double2*>(Y), nvec, nvec, ds);
      sync(c->stream);
      return SWI_OK;
    }
    DevMem dx, dy;
    dx.ensure(bytes);
    dy.ensure(bytes);
    SWI_CUDA_TRY(cudaMemcpyAsync(dx.p, X, bytes, cudaMemcpyHostToDevice, c->stream));
    apply_block(c, dx.as<double2>(), nvec, dy.as<double2>(), nvec, nvec, ds);
    SWI_CUDA_TRY(cudaMemcpyAsync(Y, dy.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    return SWI_OK;
  });
}

swi_status swi_apply(swi_ctx* c, int nvec, const double* sigma, const void* X, void* Y, int on_device) {
  return apply_impl(c, nvec, sigma, X, Y, on_device, false);
}

swi_status swi_apply_ds(swi_ctx* c, int nvec, const double* sigma, const void* X, void* Y, int on_device) {
  return apply_impl(c, nvec, sigma, X, Y, on_device, true);
}

swi_status swi_apply_c64(swi_ctx* c, int nvec, const float* sigma, const void* X, void* Y, int on_device) {
  return guarded(c, [&]() -> swi_status {
    if (nvec < 1 || !sigma || !X || !Y) return fail(c, SWI_EINVAL, "bad arguments");
    if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set");
    const size_t bytes = sizeof(float2) * (size_t)c->N * nvec;
    c->sig_dev.ensure(sizeof(float) * std::max(nvec, 64));
    SWI_CUDA_TRY(cudaMemcpyAsync(c->sig_dev.p, sigma, sizeof(float) * nvec, cudaMemcpyHostToDevice, c->stream));
    swi::StencilC64Params P;
    P.nx = c->nx;
    P.ny = c->ny;
    P.nz = c->nz;
    P.bc = c->bc;
    for (int m = 0; m < 7; ++m) P.cm[m] = (float)(-kFD[m] / (2.0 * c->h * c->h));
    P.V = c->V32.as<float>();
    P.G = c->G32.as<float>();
    P.VG = c->VG32.as<float2>();
    const double Nn = (double)c->N;
    if (on_device) {
      ProfScope ps(c, SWI_K_STENCIL, kStencilFlops * Nn * nvec, (16.0 * nvec + 8.0) * Nn);
      swi::launch_stencil_c64(P, static_cast<const float2*>(X), nvec, static_cast<float2*>(Y), nvec, nvec,
                              c->sig_dev.as<float>(), c->stream, &c->launches);
      return SWI_OK;
    }
    swi::stencil_c64_tma_error(true);
    DevMem dx, dy;
    dx.ensure(bytes);
    dy.ensure(bytes);
    SWI_CUDA_TRY(cudaMemcpyAsync(dx.p, X, bytes, cudaMemcpyHostToDevice, c->stream));
    swi::launch_stencil_c64(P, dx.as<float2>(), nvec, dy.as<float2>(), nvec, nvec, c->sig_dev.as<float>(), c->stream,
                            &c->launches);
    SWI_CUDA_TRY(cudaMemcpyAsync(Y, dy.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    if (swi::stencil_c64_tma_error(true))
      return fail(c, SWI_ETIMEOUT, "a stencil block gave up waiting for its tensor-map copy");
    return SWI_OK;
  });
}

// the solver of the context's precision and the options' block width (block
// 0 selects the batched windows of 2-vector blocks; with native FP64, wide
// blocks of 16)
static swi_status solve_dispatch(swi_ctx* c, const swi_solve_opts* opts, swi_solve_info* info) {
  swi_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.block == 0) o.block = (o.arith == SWI_ARITH_F64 && c->precision != SWI_PREC_MIXED) ? 16 : 2;
  if (c->precision == SWI_PREC_MIXED) {
    if (o.block > 2) return fail(c, SWI_EINVAL, "SWI_PREC_MIXED runs windows of 1 or 2 vectors (block 0, 1 or 2)");
    if (o.arith == SWI_ARITH_F64) return fail(c, SWI_EINVAL, "SWI_PREC_MIXED has no native-FP64 form");
    return do_solve_sv(c, &o, info);
  }
  if (o.block <= 2 && o.arith != SWI_ARITH_F64) return do_solve_sv(c, &o, info);
  return do_solve(c, &o, info);
}

swi_status swi_solve(swi_ctx* c, const swi_solve_opts* opts, swi_solve_info* info) {
  return guarded(c, [&]() -> swi_status { return solve_dispatch(c, opts, info); });
}

swi_status swi_solve_batch(int n, swi_ctx* const* ctxs, const swi_solve_opts* opts, int workers,
                           swi_solve_info* infos, swi_status* status) {
  if (n < 1 || !ctxs) return fail(nullptr, SWI_EINVAL, "swi_solve_batch: need n >= 1 contexts");
  {
    std::vector<const swi_ctx*> seen;
    for (int i = 0; i < n; ++i) {
      if (!ctxs[i]) return fail(nullptr, SWI_EINVAL, "swi_solve_batch: null context");
      if (ctxs[i]->device != ctxs[0]->device)
        return fail(nullptr, SWI_EINVAL, "swi_solve_batch: contexts on different devices");
      seen.push_back(ctxs[i]);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(nullptr, SWI_EINVAL, "swi_solve_batch: a context appears twice");
  }
  // each system's solve on a host worker of its own (its own stream and side
  // streams): the device interleaves the systems' launches
  std::vector<swi_status> st(n, SWI_OK);
  // largest systems first (grid points x requested pairs), so that a worker
  // pool over uneven systems does not end on one large solve
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto work_of = [&](int i) {
    long long r = 0;
    for (int q : ctxs[i]->nreq) r += q;
    return (double)ctxs[i]->N * (double)std::max(r, 1LL);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work_of(a) > work_of(b); });
  std::atomic<int> next{0};
  int nw = workers > 0 ? workers : (int)std::thread::hardware_concurrency();
  nw = std::max(1, std::min(nw, n));
  auto work = [&]() {
    for (;;) {
      const int t = next.fetch_add(1);
      if (t >= n) return;
      const int i = order[t];
      swi_ctx* c = ctxs[i];
      swi_solve_info* inf = infos ? infos + i : nullptr;
      st[i] = guarded(c, [&]() -> swi_status {
        // a stream of the solve's own (contexts made on one caller stream would
        // otherwise serialise), ordered after and before the context's stream
        struct Own {
          cudaStream_t s = nullptr;
          cudaEvent_t e = nullptr;
          swi_ctx* c = nullptr;
          cudaStream_t orig = nullptr;
          ~Own() {
            if (c) c->stream = orig;
            if (e) cudaEventDestroy(e);
            if (s) cudaStreamDestroy(s);
          }
        } own;
        SWI_CUDA_TRY(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
        SWI_CUDA_TRY(cudaEventCreateWithFlags(&own.e, cudaEventDisableTiming));
        SWI_CUDA_TRY(cudaEventRecord(own.e, c->stream));
        SWI_CUDA_TRY(cudaStreamWaitEvent(own.s, own.e, 0));
        own.orig = c->stream;
        own.c = c;
        c->stream = own.s;
        const swi_status r = solve_dispatch(c, opts, inf);
        SWI_CUDA_TRY(cudaEventRecord(own.e, own.s));
        SWI_CUDA_TRY(cudaStreamWaitEvent(own.orig, own.e, 0));
        return r;
      });
    }
  };
  std::vector<std::thread> pool;
  try {
    for (int k = 1; k < nw; ++k) pool.emplace_back(work);
  } catch (...) {
    // fewer workers (thread creation failed): the ones running and this thread finish the batch
  }
  work();
  for (auto& t : pool) t.join();
  if (status) std::copy(st.begin(), st.end(), status);
  for (int i = 0; i < n; ++i)
    if (st[i] != SWI_OK) return st[i];
  return SWI_OK;
}

swi_status swi_solve_more(swi_ctx* c, int p, const double* sigma, const int* n_req, const swi_solve_opts* opts,
                          swi_solve_info* info) {
  return guarded(c, [&]() -> swi_status {
    if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set before solve");
    return do_solve_more(c, p, sigma, n_req, opts, info, solve_dispatch);
  });
}

swi_status swi_fill_holes(swi_ctx* c, double e_min, double e_max, int max_rounds, const swi_solve_opts* opts,
                          swi_solve_info* info, int* windows_added) {
  return guarded(c, [&]() -> swi_status {
    if (windows_added) *windows_added = 0;
    return do_fill_holes(c, e_min, e_max, max_rounds, opts, info, windows_added, solve_dispatch);
  });
}

swi_status swi_plan_windows_sampled(swi_ctx* c, int n_r, int p, const swi_plan_opts* opts, double* sigma_out,
                                    int* n_req_out, swi_plan_info* info) {
  return guarded(c, [&]() -> swi_status {
    return do_plan_sampled(c, n_r, p, opts, sigma_out, n_req_out, info, solve_dispatch);
  });
}

swi_status swi_get_windows(swi_ctx* c, int cap, double* sigma, int* holes, int* p) {
  return guarded(c, [&]() -> swi_status {
    const int pw = (int)c->last_sigma.size();
    if (p) *p = pw;
    for (int j = 0; j < cap && j < pw; ++j) {
      if (sigma) sigma[j] = c->last_sigma[j];
      if (holes) holes[j] = j + 1 < pw && j < (int)c->last_holes.size() ? c->last_holes[j] : 0;
    }
    return SWI_OK;
  });
}

swi_status swi_refine(swi_ctx* c, const swi_refine_opts* opts, swi_refine_info* info) {
  return guarded(c, [&]() -> swi_status { return do_refine(c, opts, info); });
}

swi_status swi_get_window_info(swi_ctx* c, int cap, swi_window_info* out, int* p) {
  return guarded(c, [&]() -> swi_status {
    if (p) *p = (int)c->winfo.size();
    if (out)
      for (int j = 0; j < cap && j < (int)c->winfo.size(); ++j) out[j] = c->winfo[j];
    return SWI_OK;
  });
}

swi_status swi_get_eigenpairs(swi_ctx* c, int* n, const void** eps_dev, const void** U_dev, int* ldU) {
  return guarded(c, [&]() -> swi_status {
    if (c->npairs <= 0) return fail(c, SWI_ESTATE, "no eigenpairs: call swi_solve first");
    if (n) *n = c->npairs;
    if (eps_dev) *eps_dev = c->eps.p;
    if (U_dev) *U_dev = c->U.p;
    if (ldU) *ldU = c->npairs;
    return SWI_OK;
  });
}

swi_status swi_copy_eigenpairs(swi_ctx* c, void* eps, void* U, int on_device) {
  return guarded(c, [&]() -> swi_status {
    if (c->npairs <= 0) return fail(c, SWI_ESTATE, "no eigenpairs: call swi_solve first");
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (eps) SWI_CUDA_TRY(cudaMemcpyAsync(eps, c->eps.p, sizeof(double2) * c->npairs, k, c->stream));
    if (U) SWI_CUDA_TRY(cudaMemcpyAsync(U, c->U.p, sizeof(double2) * (size_t)c->N * c->npairs, k, c->stream));
    sync(c->stream);
    return SWI_OK;
  });
}

swi_status swi_set_eigenpairs(swi_ctx* c, int n, const void* eps, const void* U, int on_device) {
  return guarded(c, [&]() -> swi_status {
    if (n < 1 || !eps || !U) return fail(c, SWI_EINVAL, "bad arguments");
    copy_in(c->eps, eps, sizeof(double2) * n, on_device != 0, c->stream);
    copy_in(c->U, U, sizeof(double2) * (size_t)c->N * n, on_device != 0, c->stream);
    sync(c->stream);
    c->npairs = n;
    c->have_RL = false;
    c->resid.clear();
    c->last_sigma.clear();  // restored pairs carry no window records
    c->last_complex = false;
    c->last_eps_win.clear();
    c->last_win_of.clear();
    c->last_holes.clear();
    return SWI_OK;
  });
}

swi_status swi_residuals(swi_ctx* c, double* res_out) {
  return guarded(c, [&]() -> swi_status {
    if (c->npairs <= 0) return fail(c, SWI_ESTATE, "no eigenpairs");
    if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set");
    if (!res_out) return fail(c, SWI_EINVAL, "res_out is NULL");
    std::vector<double> r;
    explicit_residuals(c, c->U.as<double2>(), c->npairs, c->eps.as<double2>(), c->npairs, r);
    std::copy(r.begin(), r.end(), res_out);
    return SWI_OK;
  });
}

swi_status swi_transmission(swi_ctx* c, int nE, const double* E, double* T_out) {
  return guarded(c, [&]() -> swi_status {
    if (c->npairs <= 0) return fail(c, SWI_ESTATE, "no eigenpairs");
    if (!c->has_G) return fail(c, SWI_ESTATE, "absorbers must be set");
    if (nE < 1 || !E || !T_out) return fail(c, SWI_EINVAL, "bad arguments");
    if (!finite_all(E, nE)) return fail(c, SWI_EINVAL, "non-finite energy");
    ensure_RL(c);
    copy_in(c->Ebuf, E, sizeof(double) * nE, false, c->stream);
    c->Tbuf.ensure(sizeof(double) * nE);
    {
      const double nn = (double)c->npairs * c->npairs;
      ProfScope ps(c, SWI_K_TRANS, 8.0 * nE * nn, 16.0 * nn);
      swi::launch_transmission(c->Wm.as<double2>(), c->eps.as<double2>(), c->npairs, c->Ebuf.as<double>(), nE,
                               c->Tbuf.as<double>(), nullptr, c->stream, &c->launches);
    }
    SWI_CUDA_TRY(cudaMemcpyAsync(T_out, c->Tbuf.p, sizeof(double) * nE, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    return SWI_OK;
  });
}

swi_status swi_set_contraction(swi_ctx* c, int contraction) {
  return guarded(c, [&]() -> swi_status {
    if (contraction != SWI_CONTRACT_F64 && contraction != SWI_CONTRACT_F32)
      return fail(c, SWI_EINVAL, "contraction must be SWI_CONTRACT_F64 or SWI_CONTRACT_F32");
    if (contraction != c->contract) c->have_RL = false;
    c->contract = contraction;
    return SWI_OK;
  });
}

swi_status swi_grad(swi_ctx* c, int nE, const double* E, const double* dLdT, double* dLdV, int dLdV_on_device,
                    double* dLdE) {
  return guarded(c, [&]() -> swi_status {
    if (c->npairs <= 0) return fail(c, SWI_ESTATE, "no eigenpairs");
    if (!c->has_G) return fail(c, SWI_ESTATE, "absorbers must be set");
    if (nE < 1 || !E) return fail(c, SWI_EINVAL, "bad arguments");
    if (dLdV && !dLdT) return fail(c, SWI_EINVAL, "dLdV needs dLdT");
    if (!finite_all(E, nE) || (dLdT && !finite_all(dLdT, nE))) return fail(c, SWI_EINVAL, "non-finite input");
    ensure_RL(c);
    const int n = c->npairs;
    copy_in(c->Ebuf, E, sizeof(double) * nE, false, c->stream);
    if (dLdE) {
      c->Tbuf.ensure(sizeof(double) * nE);
      c->dEbuf.ensure(sizeof(double) * nE);
      ProfScope ps(c, SWI_K_TRANS, 8.0 * nE * (double)n * n, 16.0 * (double)n * n);
      swi::launch_transmission(c->Wm.as<double2>(), c->eps.as<double2>(), n, c->Ebuf.as<double>(), nE,
                               c->Tbuf.as<double>(), c->dEbuf.as<double>(), c->stream, &c->launches);
      SWI_CUDA_TRY(cudaMemcpyAsync(dLdE, c->dEbuf.p, sizeof(double) * nE, cudaMemcpyDeviceToHost, c->stream));
    }
    if (dLdV && c->contract == SWI_CONTRACT_F32) {
      copy_in(c->wbuf, dLdT, sizeof(double) * nE, false, c->stream);
      c->gt32.ensure(sizeof(float2) * (size_t)nE * n);
      c->M32.ensure(sizeof(float2) * (size_t)n * n);
      DevMem tmp;
      double* dst = dLdV;
      if (!dLdV_on_device) {
        tmp.ensure(sizeof(double) * c->N);
        dst = tmp.as<double>();
      }
      {
        ProfScope ps(c, SWI_K_GRAD, 8.0 * (double)n * n * ((double)nE * n + c->N),
                     16.0 * c->N * (double)n + 8.0 * c->N);
        swi::launch_grad_f32(c->R32.as<float2>(), c->L32.as<float2>(), c->eps.as<double2>(), n, c->Ebuf.as<double>(),
                             c->wbuf.as<double>(), nE, c->gt32.as<float2>(), c->M32.as<float2>(), c->U.as<double2>(),
                             n, (long long)c->N, dst, c->stream, &c->launches);
      }
      if (!dLdV_on_device)
        SWI_CUDA_TRY(cudaMemcpyAsync(dLdV, dst, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
      sync(c->stream);
    } else if (dLdV) {
      copy_in(c->wbuf, dLdT, sizeof(double) * nE, false, c->stream);
      c->Mg.ensure(sizeof(double2) * (size_t)n * n);
      ProfScope ps(c, SWI_K_GRAD, 8.0 * (double)n * n * ((double)nE * n + c->N),
                   16.0 * c->N * (double)n * 2.0 + 8.0 * c->N);
      swi::launch_gradM(c->Rm.as<double2>(), c->Lm.as<double2>(), c->eps.as<double2>(), n, c->Ebuf.as<double>(),
                        c->wbuf.as<double>(), nE, c->Mg.as<double2>(), c->stream, &c->launches);
      c->scratch.ensure(sizeof(double2) * (size_t)c->N * n);
      swi::RowGemmBatch rb;
      rb.n = 1;
      rb.job[0] = swi::RowGemmJob{c->U.as<double2>(), c->Mg.as<double2>(), nullptr, c->scratch.as<double2>(), n, n, 0,
                                  n, n, n, 1.0, 0.0};
      rowgemm_dispatch(c->arith,rb, c->N, c->stream, &c->launches);
      DevMem tmp;
      double* dst = dLdV;
      if (!dLdV_on_device) {
        tmp.ensure(sizeof(double) * c->N);
        dst = tmp.as<double>();
      }
      swi::launch_rowdot(c->scratch.as<double2>(), n, c->U.as<double2>(), n, n, c->N, dst, c->stream, &c->launches);
      if (!dLdV_on_device)
        SWI_CUDA_TRY(cudaMemcpyAsync(dLdV, dst, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
      sync(c->stream);
    }
    sync(c->stream);
    if (dLdE && dLdT)  // chain rule: T_e depends on E_e alone
      for (int e = 0; e < nE; ++e) dLdE[e] *= dLdT[e];
    return SWI_OK;
  });
}

swi_status swi_profile(swi_ctx* c, int enable) {
  return guarded(c, [&]() -> swi_status {
    sync(c->stream);
    for (auto& r : c->prof) {
      c->evpool.push_back(r.a);
      c->evpool.push_back(r.b);
    }
    c->prof.clear();
    c->schur_flops = 0.0;
    c->prof_on = enable != 0;
    return SWI_OK;
  });
}

swi_status swi_profile_read(swi_ctx* c, swi_kernel_stats* out) {
  return guarded(c, [&]() -> swi_status {
    if (!out) return fail(c, SWI_EINVAL, "out is NULL");
    sync(c->stream);
    for (int k = 0; k < SWI_K_COUNT; ++k) out[k] = swi_kernel_stats{0, 0.0, 0.0, 0.0};
    for (auto& r : c->prof) {
      float ms = 0.f;
      SWI_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
      swi_kernel_stats& s = out[r.kind];
      s.launches += 1;
      s.ms += ms;
      s.flops += r.flops;
      s.bytes += r.bytes;
    }
    out[SWI_K_SCHUR].flops += c->schur_flops;
    return SWI_OK;
  });
}

}  // extern "C"

extern "C" {

swi_status swi_transmission_noalloc(swi_ctx* c, int nE, const double* E, double* T_out) {
  return guarded(c, [&]() -> swi_status {
    if (c->npairs <= 0) return fail(c, SWI_ESTATE, "no eigenpairs");
    if (!c->has_G) return fail(c, SWI_ESTATE, "absorbers must be set");
    if (nE < 1 || !E || !T_out) return fail(c, SWI_EINVAL, "bad arguments");
    if (c->npairs > kNoAllocMaxPairs)
      return fail(c, SWI_EINVAL, "swi_transmission_noalloc: at most 64 eigenpairs (context holds " +
                                     std::to_string(c->npairs) + "); use swi_transmission");
    if (nE > kNoAllocMaxEnergies)
      return fail(c, SWI_EINVAL, "swi_transmission_noalloc: at most 1024 energies per call");
    if (!finite_all(E, nE)) return fail(c, SWI_EINVAL, "non-finite energy");
    const int n = c->npairs;
    double2* base = noalloc_scratch(c->device);
    double2* MR = base;
    double2* ML = base + kNoAllocMat;
    double2* R = base + 2 * kNoAllocMat;
    double2* L = base + 3 * kNoAllocMat;
    double2* Wm = base + 4 * kNoAllocMat;
    double2* work = base + 5 * kNoAllocMat;
    double* Ed = reinterpret_cast<double*>(base + 5 * kNoAllocMat + kNoAllocWork);
    double* Td = Ed + kNoAllocMaxEnergies;
    // every scratch region below is fully overwritten before it is read, so
    // nothing needs clearing between calls
    SWI_CUDA_TRY(cudaMemcpyAsync(Ed, E, sizeof(double) * nE, cudaMemcpyHostToDevice, c->stream));
    // The projections run over slabs of kNoAllocSlab grid rows, each summed on
    // top of the previous ones: a slab fits the fixed partial-sum workspace
    // with the same at-most-1024-rows chunks that swi_transmission uses, at
    // any grid size.
    for (int r0 = 0; r0 < c->N; r0 += kNoAllocSlab) {
      const int rows = std::min(kNoAllocSlab, c->N - r0);
      const double2* Us = c->U.as<double2>() + (size_t)r0 * n;
      swi::GramBatch gb;
      gb.n = 1;
      gb.job[0] = swi::GramJob{Us, Us, MR, n, n, n, n, n, r0 > 0 ? 1 : 0};
      gram_dispatch(c->arith, gb, rows, c->gR.as<double>() + r0, 0, work, kNoAllocWork, c->stream, &c->launches);
      gb.job[0].C = ML;
      gram_dispatch(c->arith, gb, rows, c->gL.as<double>() + r0, 0, work, kNoAllocWork, c->stream, &c->launches);
    }
    swi::launch_wbuild(MR, ML, n, R, L, Wm, c->stream, &c->launches);
    swi::launch_transmission(Wm, c->eps.as<double2>(), n, Ed, nE, Td, nullptr, c->stream, &c->launches);
    SWI_CUDA_TRY(cudaMemcpyAsync(T_out, Td, sizeof(double) * nE, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    return SWI_OK;
  });
}

const char* swi_last_error(const swi_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

long long swi_launch_count(const swi_ctx* c) { return c ? c->launches : 0; }

swi_status swi_check_schur(swi_ctx* c, int m, int b, int keep, const double* H, const double* B, int arith,
                           double* T_out, double* Z_out, int* info_out) {
  return guarded(c, [&]() -> swi_status {
    if (m < 2 || m > 1024 || (b != 1 && b != 2) || keep < 1 || keep > m - b || !H || !T_out || !Z_out || !info_out)
      return fail(c, SWI_EINVAL, "check_schur: bad arguments");
    if (arith != SWI_ARITH_DS && arith != SWI_ARITH_F64) return fail(c, SWI_EINVAL, "unknown arithmetic");
    const size_t mm = (size_t)m * m;
    DevMem dH, dZ, dB, dBz, dth, dres, dS, dinfo, dHw, dZw;
    dH.ensure(sizeof(double2) * mm);
    dZ.ensure(sizeof(double2) * mm);
    dS.ensure(sizeof(double2) * mm);
    dB.ensure(sizeof(double2) * b * m);
    dBz.ensure(sizeof(double2) * b * m);
    dth.ensure(sizeof(double2) * m);
    dres.ensure(sizeof(double) * m);
    dinfo.ensure(sizeof(int) * 4);
    dHw.ensure(16 * mm);
    dZw.ensure(16 * mm);
    SWI_CUDA_TRY(cudaMemcpyAsync(dH.p, H, sizeof(double2) * mm, cudaMemcpyHostToDevice, c->stream));
    if (B) SWI_CUDA_TRY(cudaMemcpyAsync(dB.p, B, sizeof(double2) * b * m, cudaMemcpyHostToDevice, c->stream));
    else SWI_CUDA_TRY(cudaMemsetAsync(dB.p, 0, sizeof(double2) * b * m, c->stream));
    SWI_CUDA_TRY(cudaMemsetAsync(dinfo.p, 0, sizeof(int) * 4, c->stream));
    swi::SchurBatch sb;
    sb.n = 1;
    sb.job[0] = swi::SchurJob{dH.as<double2>(), dZ.as<double2>(), dB.as<double2>(), dBz.as<double2>(),
                              dth.as<double2>(), dres.as<double>(), dS.as<double2>(), dinfo.as<int>(),
                              m, m, b, keep, keep, m - b, 0.0, dHw.p, dZw.p};
    if (arith == SWI_ARITH_F64) swi::launch_schur_batch(sb, c->stream, &c->launches);
    else swi::launch_schur_ds_batch(sb, c->stream, &c->launches);
    SWI_CUDA_TRY(cudaMemcpyAsync(T_out, dH.p, sizeof(double2) * mm, cudaMemcpyDeviceToHost, c->stream));
    SWI_CUDA_TRY(cudaMemcpyAsync(Z_out, dZ.p, sizeof(double2) * mm, cudaMemcpyDeviceToHost, c->stream));
    SWI_CUDA_TRY(cudaMemcpyAsync(info_out, dinfo.p, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
    return SWI_OK;
  });
}

void swi_destroy(swi_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  delete c;
}

}  // extern "C"
