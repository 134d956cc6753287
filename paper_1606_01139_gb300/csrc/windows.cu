// Window management above the solver: continuation runs and automated hole
// filling.
//
//  - Continuation (Section 2, extending a computed set of n_r pairs to n_r' by
//    adding windows while the old pairs are kept; Conclusions): the new
//    windows are solved on their own, then their pairs and the stored pairs
//    pass Algorithm 2 together, every stored pair assigned to the stored
//    window whose shift is nearest its real part, all windows in shift order.
//  - Hole filling (Algorithm 1's loop over interfaces that showed no
//    redundancy): for each hole a window at the middle of the gap between the
//    highest real part delivered by the lower window and the lowest delivered
//    by the upper one, requesting 3/2 of the gap's eigenvalue count at the
//    mean spacing of the two windows' eigenvalues plus 4 (Algorithm 1's
//    uniform (E_max - E_min)/N where they give none), at most 300; solved as
//    a continuation, repeated until no hole remains or the round limit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "host.cuh"

namespace swi {
namespace host {

namespace {

swi_status check_windows(swi_ctx* c, int p, const double* sigma, const int* n_req) {
  if (p < 1 || !sigma || !n_req) return fail(c, SWI_EINVAL, "need p >= 1 windows");
  if (p > swi::kMaxBatch) return fail(c, SWI_EINVAL, "at most 64 windows");
  for (int j = 0; j < p; ++j) {
    if (!std::isfinite(sigma[j])) return fail(c, SWI_EINVAL, "non-finite shift");
    if (n_req[j] < 1) return fail(c, SWI_EINVAL, "each window needs n_req >= 1");
    if (j > 0 && !(sigma[j] > sigma[j - 1])) return fail(c, SWI_EINVAL, "shifts must be strictly increasing");
  }
  return SWI_OK;
}

}  // namespace

swi_status do_solve_more(swi_ctx* c, int p, const double* sigma, const int* n_req, const swi_solve_opts* o,
                         swi_solve_info* info, swi_status (*solve)(swi_ctx*, const swi_solve_opts*, swi_solve_info*)) {
  const swi_status chk = check_windows(c, p, sigma, n_req);
  if (chk != SWI_OK) return chk;
  swi_solve_opts opt;
  std::memset(&opt, 0, sizeof(opt));
  if (o) opt = *o;
  if (c->npairs <= 0) {  // nothing stored: a plain solve
    c->sigma.assign(sigma, sigma + p);
    c->sigma_im.clear();  // real shifts
    c->nreq.assign(n_req, n_req + p);
    return solve(c, &opt, info);
  }
  const size_t N = c->N;
  const double t0 = swi::now_seconds();
  // the stored pairs and their windows
  const int n_old = c->npairs;
  DevMem Uold;
  Uold.ensure(sizeof(double2) * N * n_old);
  SWI_CUDA_TRY(cudaMemcpyAsync(Uold.p, c->U.p, sizeof(double2) * N * n_old, cudaMemcpyDeviceToDevice, c->stream));
  std::vector<double2> eps_old(n_old);
  SWI_CUDA_TRY(cudaMemcpyAsync(eps_old.data(), c->eps.p, sizeof(double2) * n_old, cudaMemcpyDeviceToHost, c->stream));
  sync(c->stream);
  // stored pairs without window records (restored by swi_set_eigenpairs, a
  // checkpoint): one window at the middle of their real parts
  if (c->last_sigma.empty()) {
    double lo = INFINITY, hi = -INFINITY;
    for (const double2& e : eps_old) {
      lo = std::min(lo, e.x);
      hi = std::max(hi, e.x);
    }
    c->last_sigma.assign(1, 0.5 * (lo + hi));
    c->last_eps_win = eps_old;
    c->last_win_of.assign(n_old, 0);
  }
  const std::vector<double> sig_old = c->last_sigma;
  const std::vector<double2> epsw_old = c->last_eps_win;
  const std::vector<int> winw_old = c->last_win_of;
  const std::vector<int> holes_old = c->last_holes;  // interfaces between stored windows
  std::vector<int> win_old(n_old);
  for (int k = 0; k < n_old; ++k) {
    int best = 0;
    for (int j = 1; j < (int)sig_old.size(); ++j)
      if (std::fabs(eps_old[k].x - sig_old[j]) < std::fabs(eps_old[k].x - sig_old[best])) best = j;
    win_old[k] = best;
  }
  // the new windows on their own (all their merged pairs kept)
  c->sigma.assign(sigma, sigma + p);
  c->sigma_im.clear();  // real shifts
  c->nreq.assign(n_req, n_req + p);
  swi_solve_opts inner = opt;
  inner.n_keep = 0;
  swi_solve_info inf_new;
  std::memset(&inf_new, 0, sizeof(inf_new));
  const swi_status st_new = solve(c, &inner, &inf_new);
  if (st_new != SWI_OK && st_new != SWI_ENOCONV && st_new != SWI_HOLES) return st_new;
  const int n_new = c->npairs;
  std::vector<double2> eps_new(n_new);
  SWI_CUDA_TRY(cudaMemcpyAsync(eps_new.data(), c->eps.p, sizeof(double2) * n_new, cudaMemcpyDeviceToHost, c->stream));
  sync(c->stream);
  const std::vector<double2> epsw_new = c->last_eps_win;
  const std::vector<int> winw_new = c->last_win_of;
  std::vector<int> win_new(n_new);
  for (int k = 0; k < n_new; ++k) {
    int best = 0;
    for (int j = 1; j < p; ++j)
      if (std::fabs(eps_new[k].x - sigma[j]) < std::fabs(eps_new[k].x - sigma[best])) best = j;
    win_new[k] = best;
  }
  // all windows in shift order (stored ones first on equal shifts)
  const int p_old = (int)sig_old.size(), p_all = p_old + p;
  if (p_all > swi::kMaxBatch) return fail(c, SWI_EINVAL, "continuation: more than 64 windows in all");
  std::vector<double> sig_all(p_all);
  for (int j = 0; j < p_old; ++j) sig_all[j] = sig_old[j];
  for (int j = 0; j < p; ++j) sig_all[p_old + j] = sigma[j];
  std::vector<int> ord(p_all), rank(p_all);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sig_all[a] < sig_all[b]; });
  for (int r = 0; r < p_all; ++r) rank[ord[r]] = r;
  // pairs grouped by window, windows in shift order
  struct Src {
    int win, col;
    bool old;
  };
  std::vector<Src> src;
  for (int k = 0; k < n_old; ++k) src.push_back({rank[win_old[k]], k, true});
  for (int k = 0; k < n_new; ++k) src.push_back({rank[p_old + win_new[k]], k, false});
  std::stable_sort(src.begin(), src.end(), [](const Src& a, const Src& b) { return a.win < b.win; });
  const int n_all = (int)src.size();
  c->Uall.ensure(sizeof(double2) * N * n_all);
  std::vector<double2> eps_all(n_all);
  std::vector<int> win_of(n_all);
  for (int q = 0; q < n_all; ++q) {
    const Src& sq = src[q];
    const double2* from = sq.old ? Uold.as<double2>() + sq.col : c->U.as<double2>() + sq.col;
    swi::launch_copy_block(from, sq.old ? n_old : n_new, c->Uall.as<double2>() + q, n_all, c->N, 1, c->stream,
                           &c->launches);
    eps_all[q] = sq.old ? eps_old[sq.col] : eps_new[sq.col];
    win_of[q] = sq.win;
  }
  const double eq_rtol = opt.eq_rtol > 0 ? opt.eq_rtol : (c->precision == SWI_PREC_MIXED ? 1e-5 : 1e-8);
  const double drop_tol = opt.drop_tol > 0 ? opt.drop_tol : (c->precision == SWI_PREC_MIXED ? 1e-2 : 1e-6);
  int minfo[4];
  merge_pairs(c, c->Uall.as<double2>(), n_all, eps_all, win_of, p_all, eq_rtol, drop_tol, opt.n_keep, minfo);
  // the windows of the union and the eigenvalues each delivered
  c->sigma.resize(p_all);
  c->sigma_im.clear();  // real shifts
  for (int r = 0; r < p_all; ++r) c->sigma[r] = sig_all[ord[r]];
  std::vector<double2> epsw;
  std::vector<int> winw;
  for (size_t k = 0; k < epsw_old.size(); ++k) {
    epsw.push_back(epsw_old[k]);
    winw.push_back(rank[winw_old[k]]);
  }
  for (size_t k = 0; k < epsw_new.size(); ++k) {
    epsw.push_back(epsw_new[k]);
    winw.push_back(rank[p_old + winw_new[k]]);
  }
  record_windows(c, epsw, winw, p_all);
  // An interface between two stored windows keeps the flag of the run that
  // computed them: the stored pairs are already free of redundancy, so the
  // union's merge cannot see it again.
  int holes = 0;
  for (int r = 0; r + 1 < p_all; ++r) {
    const int a = ord[r], b = ord[r + 1];
    if (a < p_old && b < p_old && r < (int)c->last_holes.size())
      c->last_holes[r] = (b == a + 1 && a < (int)holes_old.size()) ? holes_old[a] : 0;
    if (r < (int)c->last_holes.size()) holes += c->last_holes[r] != 0;
  }
  minfo[2] = holes;
  c->Uall.release();
  const int nout = minfo[0];
  explicit_residuals(c, c->U.as<double2>(), nout, c->eps.as<double2>(), nout, c->resid);
  const double rel_tol = opt.rel_tol > 0 ? opt.rel_tol : 1e-10;
  int nconv = 0;
  double maxr = 0.0;
  for (double r : c->resid) {
    if (r <= rel_tol) ++nconv;
    maxr = std::max(maxr, r);
  }
  if (info) {
    *info = inf_new;
    info->n_windows = p_all;
    info->n_pairs = nout;
    info->n_converged = nconv;
    info->n_duplicates = minfo[1];
    info->n_holes = minfo[2];
    info->max_rel_res = maxr;
    info->t_merge_s = swi::now_seconds() - t0 - inf_new.t_krylov_s;
  }
  if (minfo[3] != 0) return fail(c, SWI_EINVAL, "merge: equal-eigenvalue component too large");
  if (st_new == SWI_ENOCONV || nconv < nout) return fail(c, SWI_ENOCONV, "pairs above rel_tol after the continuation");
  if (minfo[2] > 0) return fail(c, SWI_HOLES, std::to_string(minfo[2]) + " interface(s) without redundancy");
  return SWI_OK;
}

swi_status do_fill_holes(swi_ctx* c, double e_min, double e_max, int max_rounds, const swi_solve_opts* o,
                         swi_solve_info* info, int* windows_added,
                         swi_status (*solve)(swi_ctx*, const swi_solve_opts*, swi_solve_info*)) {
  if (!(e_max > e_min) || !std::isfinite(e_min) || !std::isfinite(e_max))
    return fail(c, SWI_EINVAL, "need finite e_max > e_min");
  if (c->npairs <= 0 || c->last_sigma.empty()) return fail(c, SWI_ESTATE, "no solve to fill holes in");
  if (c->last_complex) return fail(c, SWI_EINVAL, "hole filling places windows on the real axis: the last solve used complex shifts");
  const int rounds = max_rounds > 0 ? max_rounds : 4;
  const double spacing = (e_max - e_min) / c->N;  // uniform-density spacing of Algorithm 1
  int added = 0;
  swi_status st = SWI_OK;
  for (int round = 0; round < rounds; ++round) {
    std::vector<double> sg;
    std::vector<int> rq;
    const int pw = (int)c->last_sigma.size();
    for (int i = 0; i + 1 < pw && i < (int)c->last_holes.size(); ++i) {
      if (!c->last_holes[i]) continue;
      double top = -INFINITY, bot = INFINITY;
      for (size_t k = 0; k < c->last_eps_win.size(); ++k) {
        if (c->last_win_of[k] == i) top = std::max(top, c->last_eps_win[k].x);
        if (c->last_win_of[k] == i + 1) bot = std::min(bot, c->last_eps_win[k].x);
      }
      if (!std::isfinite(top) || !std::isfinite(bot)) continue;
      const double s = 0.5 * (top + bot);
      // Algorithm 1's request uses the uniform spacing (E_max - E_min)/N; where
      // the two windows delivered eigenvalues, their own mean spacing is the
      // better estimate (the density of states varies by orders of magnitude
      // over a wire's spectrum), and the request stays within a window's reach
      double lo = INFINITY, hi = -INFINITY;
      int cnt = 0;
      for (size_t k = 0; k < c->last_eps_win.size(); ++k)
        if (c->last_win_of[k] == i || c->last_win_of[k] == i + 1) {
          lo = std::min(lo, c->last_eps_win[k].x);
          hi = std::max(hi, c->last_eps_win[k].x);
          ++cnt;
        }
      // (with the local spacing, 4 more: the new window must reach past both
      // edges of the gap to overlap its neighbours)
      const bool local = cnt >= 4 && hi > lo;
      const double sp = local ? (hi - lo) / (cnt - 1) : spacing;
      const int n = (int)std::min(300.0, std::max(1.0, std::ceil(1.5 * (bot - top) / sp) + (local ? 4 : 0)));
      if (!sg.empty() && !(s > sg.back())) continue;
      sg.push_back(s);
      rq.push_back(n);
    }
    if (sg.empty()) break;
    st = do_solve_more(c, (int)sg.size(), sg.data(), rq.data(), o, info, solve);
    added += (int)sg.size();
    if (st != SWI_OK && st != SWI_HOLES && st != SWI_ENOCONV) break;
    if (st != SWI_HOLES) break;
  }
  if (windows_added) *windows_added = added;
  return st;
}

}  // namespace host
}  // namespace swi

// ---------------------------------------------------------------------------
// Window planning with extremal estimates and density sampling (Section 2.2.1:
// two exterior Krylov solves bound the spectrum, E_min and E_max; a few small
// solves at sample points measure the spectral density, which the uniform
// estimate of Algorithm 1 lacks).  The samples march up the spectrum from
// E_min: each is one window of `sample_req` pairs at a loose tolerance, the
// next one's shift three quarters of the way up the real parts just found, and
// the eigenvalues above the previous window's highest real part are added to
// the sampled spectrum, until it holds n_r values.  The p windows are then
// cut from the sampled spectrum: runs of n_r,j consecutive real parts (equal
// counts, or Algorithm 1's n_r,j), the shift at the middle of each run, the
// request n_r,j inflated (the paper's placement with foreknowledge, Section 3).
namespace swi {
namespace host {

namespace {

std::vector<long long> alg1_counts(int n_r, int p) {
  std::vector<long long> cnt(p + 1, 0);
  for (int j = 1; j <= p; ++j) {
    if (j <= p / 2.0) {
      const double x = 2.0 / (1.5 + (double)(j - 1) / p) * (double)n_r / p;
      cnt[j] = (long long)std::floor(x + 0.5);
    } else {
      cnt[j] = (long long)std::ceil(2.0 * n_r / p) - cnt[p - j + 1];
    }
  }
  return std::vector<long long>(cnt.begin() + 1, cnt.end());
}

// real parts of the context's current pairs, ascending
std::vector<double> current_re(swi_ctx* c) {
  std::vector<double2> e(c->npairs);
  if (c->npairs > 0) {
    SWI_CUDA_TRY(cudaMemcpyAsync(e.data(), c->eps.p, sizeof(double2) * c->npairs, cudaMemcpyDeviceToHost, c->stream));
    sync(c->stream);
  }
  std::vector<double> r;
  for (const double2& x : e) r.push_back(x.x);
  std::sort(r.begin(), r.end());
  return r;
}

}  // namespace

swi_status do_plan_sampled(swi_ctx* c, int n_r, int p, const swi_plan_opts* po, double* sigma_out, int* n_req_out,
                           swi_plan_info* pinfo, swi_status (*solve)(swi_ctx*, const swi_solve_opts*, swi_solve_info*)) {
  if (!c->has_V || !c->has_G) return fail(c, SWI_ESTATE, "potential and absorbers must be set before planning");
  if (n_r < 1 || p < 1 || p > swi::kMaxBatch || p > n_r) return fail(c, SWI_EINVAL, "need 1 <= p <= min(n_r, 64)");
  swi_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  if (po) o = *po;
  const int q = o.sample_req > 0 ? o.sample_req : std::max(8, (2 * n_r + p - 1) / p);
  const int max_samples = o.max_samples > 0 ? o.max_samples : 64;
  const double tol = o.sample_tol > 0 ? o.sample_tol : 1e-5;
  const double inflate = o.inflate >= 1.0 ? o.inflate : 1.25;
  const int extra = o.extra > 0 ? o.extra : (o.extra < 0 ? 0 : 4);
  const long long budget = o.max_matvecs > 0 ? o.max_matvecs : 200000;
  const double t0 = swi::now_seconds();
  swi_solve_opts so;
  std::memset(&so, 0, sizeof(so));
  so.block = 2;  // both vectors of a doubly degenerate eigenvalue count
  so.rel_tol = tol;
  so.max_matvecs = budget;
  so.eq_rtol = 1e-6;
  so.drop_tol = 1e-3;
  long long mv = 0;
  // A8: two exterior solves, below and above the spectrum (Re eps >= min V since
  // the kinetic term is positive; |eps| <= ||A||_G)
  double vmin = 0.0;
  {
    std::vector<double> hv(c->N);
    SWI_CUDA_TRY(cudaMemcpy(hv.data(), c->V.p, sizeof(double) * c->N, cudaMemcpyDeviceToHost));
    vmin = *std::min_element(hv.begin(), hv.end());
  }
  const double an = gershgorin(c);
  double e_min, e_max;
  {
    const double sg[2] = {vmin - 1.0, an + 1.0};
    const int rq[2] = {2, 2};
    c->sigma.assign(sg, sg + 2);
    c->sigma_im.clear();  // real shifts
    c->nreq.assign(rq, rq + 2);
    swi_solve_info inf;
    const swi_status st = solve(c, &so, &inf);
    if (st != SWI_OK && st != SWI_HOLES && st != SWI_ENOCONV) return st;
    mv += inf.matvecs;
    const std::vector<double> r = current_re(c);
    if (r.size() < 2) return fail(c, SWI_ENOCONV, "planner: the extremal solves found no pairs");
    e_min = r.front();
    e_max = r.back();
  }
  // A10: sample the density upward from E_min
  std::vector<double> spec;
  double sig = e_min, prev_top = -INFINITY;
  int samples = 0;
  while ((int)spec.size() < n_r && samples < max_samples) {
    c->sigma.assign(1, sig);
    c->sigma_im.clear();  // real shifts
    c->nreq.assign(1, q);
    swi_solve_info inf;
    const swi_status st = solve(c, &so, &inf);
    if (st != SWI_OK && st != SWI_HOLES && st != SWI_ENOCONV) return st;
    mv += inf.matvecs;
    ++samples;
    const std::vector<double> r = current_re(c);
    if (r.empty()) return fail(c, SWI_ENOCONV, "planner: a sampling solve found no pairs");
    // add the sample's eigenvalues not yet counted, with multiplicity: a real
    // part that repeats (a twofold eigenvalue) counts as often as the sample
    // holds it, values the earlier samples found are not counted twice
    {
      const double tau_rel = std::max(1e-7, 100.0 * tol);
      const std::vector<double> have = spec;
      for (size_t i = 0; i < r.size(); ++i) {
        const double x = r[i], tau = tau_rel * std::max(1.0, std::fabs(x));
        if (x < prev_top - tau) continue;
        int rank = 0, old = 0;
        for (size_t k = 0; k <= i; ++k) rank += std::fabs(r[k] - x) <= tau;
        for (double y : have) old += std::fabs(y - x) <= tau;
        if (rank > old) spec.push_back(x);
      }
    }
    const double lo = r.front(), hi = r.back();
    if (!(hi > prev_top)) return fail(c, SWI_ENOCONV, "planner: the sampling made no progress");
    prev_top = hi;
    sig = lo + 0.75 * (hi - lo);
  }
  if ((int)spec.size() < n_r) return fail(c, SWI_ENOCONV, "planner: fewer than n_r eigenvalues sampled");
  std::sort(spec.begin(), spec.end());
  // the windows: runs of counts[j] consecutive sampled real parts
  std::vector<long long> counts;
  if (o.counts_rule == 1) {
    counts = alg1_counts(n_r, p);
  } else {
    counts.assign(p, n_r / p);
    for (int j = 0; j < n_r % p; ++j) counts[j] += 1;
  }
  std::vector<double> sg;
  std::vector<int> rq;
  size_t start = 0;
  for (int j = 0; j < p && start < (size_t)n_r; ++j) {
    const size_t stop = std::min<size_t>(n_r, start + (size_t)std::max(1LL, counts[j]));
    sg.push_back(0.5 * (spec[start] + spec[stop - 1]));
    rq.push_back((int)std::ceil(counts[j] * inflate) + extra);
    start = stop;
  }
  for (size_t j = 1; j < sg.size(); ++j)
    if (!(sg[j] > sg[j - 1])) return fail(c, SWI_EINVAL, "planner: coincident shifts (a degenerate run)");
  c->sigma = sg;
  c->sigma_im.clear();  // real shifts
  c->nreq = rq;
  if (sigma_out) std::copy(sg.begin(), sg.end(), sigma_out);
  if (n_req_out) std::copy(rq.begin(), rq.end(), n_req_out);
  if (pinfo) {
    pinfo->e_min = e_min;
    pinfo->e_max = e_max;
    pinfo->samples = samples;
    pinfo->windows = (int)sg.size();
    pinfo->matvecs = mv;
    pinfo->t_s = swi::now_seconds() - t0;
    pinfo->e_top = spec[n_r - 1];
  }
  return SWI_OK;
}

}  // namespace host
}  // namespace swi
