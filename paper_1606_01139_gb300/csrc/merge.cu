// Algorithm 2 on the device: combine windows, remove redundant pairs, flag holes,
// keep the lowest-real-part pairs and scale them to U^T U = I.
//
// Walking all computed pairs in order (windows by shift, each window's pairs
// by real part), a pair whose eigenvalue equals (|l_m - l_k| <= eq_rtol
// max(1, |l_k|)) that of an earlier kept pair is projected against it with the
// unconjugated product v_k -= v_m (v_m^T v_k)/(v_m^T v_m) (modified Gram-Schmidt
// in the bilinear form under which the eigenvectors are bi-orthogonal,
// Section 1); if ||v_k||_2 / ||v_k^0||_2 < drop_tol the pair is redundant and
// removed, which also marks the interfaces it straddles as redundant (no
// hole).  Survivors are scaled by 1/sqrt(v^T v).
//
// The projections are carried out on coefficients: every vector that
// Gram-Schmidt touches lies in the span of the original vectors of its
// equal-eigenvalue component, so only the Gram entries within components are
// needed (one pass over the N rows), the Gram-Schmidt itself runs on tiny
// matrices in one CTA, and a final pass forms the surviving combinations.
#include "swi_internal.cuh"
#include "merge.cuh"

namespace swi {

namespace {

constexpr int kMaxComp = 64;  // largest equal-eigenvalue component handled

__device__ __forceinline__ bool eq_test(double2 a, double2 b, double rtol) {
  return cabs(csub(a, b)) <= rtol * fmax(1.0, cabs(b));
}

// Single CTA: union-find over the equality relation, then the list of Gram
// pairs (a <= c within each component, including a == c).
__global__ void merge_plan_kernel(const double2* __restrict__ eps, int n, double rtol, int* comp, int* pairs,
                                  int pair_cap, int* counts) {
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) comp[i] = i;
  __syncthreads();
  if (tid == 0) {
    int status = 0;
    for (int k = 0; k < n; ++k) {
      for (int m = 0; m < k; ++m) {
        if (!eq_test(eps[m], eps[k], rtol)) continue;
        // union(m, k)
        int a = m, b = k;
        while (comp[a] != a) a = comp[a];
        while (comp[b] != b) b = comp[b];
        if (a != b) {
          if (a < b) comp[b] = a;
          else comp[a] = b;
        }
      }
    }
    for (int k = 0; k < n; ++k) {
      int a = k;
      while (comp[a] != a) a = comp[a];
      comp[k] = a;
    }
    // pairs within components
    int np = 0;
    for (int c = 0; c < n; ++c) {
      for (int a = 0; a < n; ++a) {
        if (comp[a] != comp[c] || a > c) continue;
        if (np < pair_cap) {
          pairs[2 * np] = a;
          pairs[2 * np + 1] = c;
        } else {
          status = 1;
        }
        ++np;
      }
    }
    counts[0] = np < pair_cap ? np : pair_cap;
    counts[1] = status;
  }
}

// Partial bilinear (u_a^T u_c) and Hermitian (u_a^H u_c) products for each pair
// over a chunk of rows.
__global__ void pair_gram_partial_kernel(const double2* __restrict__ U, int ld, int N, const int* __restrict__ pairs,
                                         const int* __restrict__ counts, int rows_per_chunk,
                                         double2* __restrict__ work) {
  const int np = counts[0];
  const int r0 = blockIdx.x * rows_per_chunk;
  const int r1 = min(N, r0 + rows_per_chunk);
  for (int q = threadIdx.x + blockIdx.y * blockDim.x; q < np; q += blockDim.x * gridDim.y) {
    const int a = pairs[2 * q], c = pairs[2 * q + 1];
    double2 gb = make_double2(0.0, 0.0), gh = make_double2(0.0, 0.0);
    for (int r = r0; r < r1; ++r) {
      const double2 ua = U[(long long)r * ld + a];
      const double2 uc = U[(long long)r * ld + c];
      cfma(gb, ua, uc);
      cfmac(gh, ua, uc);
    }
    work[((long long)blockIdx.x * np + q) * 2] = gb;
    work[((long long)blockIdx.x * np + q) * 2 + 1] = gh;
  }
}

__global__ void pair_gram_reduce_kernel(const double2* __restrict__ work, int nchunks, const int* counts,
                                        double2* __restrict__ gram) {
  const int np = counts[0];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  double2 gb = make_double2(0.0, 0.0), gh = make_double2(0.0, 0.0);
  for (int c = 0; c < nchunks; ++c) {
    gb = cadd(gb, work[((long long)c * np + q) * 2]);
    gh = cadd(gh, work[((long long)c * np + q) * 2 + 1]);
  }
  gram[2 * q] = gb;
  gram[2 * q + 1] = gh;
}

// Single thread: Algorithm 2 on coefficients, then selection of the lowest
// real parts.  Output: for each kept output column q (Re-ordered), up to
// kMaxComp (source, coefficient) terms.
__global__ void merge_mgs_kernel(const double2* __restrict__ eps, const int* __restrict__ win, int n, int p,
                                 double eq_rtol, double drop_tol, const int* __restrict__ comp,
                                 const int* __restrict__ pairs, const int* __restrict__ counts,
                                 const double2* __restrict__ gram, int n_keep, int* __restrict__ out_src,
                                 double2* __restrict__ out_coef, int* __restrict__ out_nterm,
                                 double2* __restrict__ out_eps, int* __restrict__ out_info, int* __restrict__ holes,
                                 int* __restrict__ kept_flag, int* __restrict__ order_tmp) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int np = counts[0];
  int status = counts[1] ? 1 : 0;
  for (int i = 0; i + 1 < p; ++i) holes[i] = 1;
  // lookup of the pair index of (a, c), a <= c: linear scan of the component's pairs
  auto find_pair = [&](int a, int c) -> int {
    if (a > c) {
      const int t = a;
      a = c;
      c = t;
    }
    for (int q = 0; q < np; ++q)
      if (pairs[2 * q] == a && pairs[2 * q + 1] == c) return q;
    return -1;
  };
  auto gbil = [&](int a, int c) -> double2 {  // u_a^T u_c (symmetric)
    const int q = find_pair(a, c);
    return q >= 0 ? gram[2 * q] : make_double2(0.0, 0.0);
  };
  auto gher = [&](int a, int c) -> double2 {  // u_a^H u_c
    if (a <= c) {
      const int q = find_pair(a, c);
      return q >= 0 ? gram[2 * q + 1] : make_double2(0.0, 0.0);
    }
    const int q = find_pair(c, a);
    return q >= 0 ? cconj(gram[2 * q + 1]) : make_double2(0.0, 0.0);
  };
  int n_dup = 0;
  int n_kept = 0;
  // coefficient store: for vector k, members of its component (local list) with coefficients
  // kept in out arrays indexed by k (temporarily, before selection)
  for (int k = 0; k < n; ++k) {
    // members of k's component with index <= k
    int mem[kMaxComp];
    int nm = 0;
    for (int a = 0; a <= k && nm < kMaxComp; ++a)
      if (comp[a] == comp[k]) mem[nm++] = a;
    if (nm >= kMaxComp) status = 2;
    double2 coef[kMaxComp];
    for (int t = 0; t < nm; ++t) coef[t] = make_double2(0.0, 0.0);
    coef[nm - 1] = make_double2(1.0, 0.0);  // mem[nm-1] == k
    int partner = -1;
    for (int t = 0; t + 1 < nm; ++t) {
      const int m = mem[t];
      if (!kept_flag[m]) continue;
      if (!eq_test(eps[m], eps[k], eq_rtol)) continue;
      // v_m = sum_s cm_s u_{mem s}; bilinear products through the Gram entries
      const double2* cm = out_coef + (long long)m * kMaxComp;  // stored aligned to mem of m (prefix of ours)
      double2 mtk = make_double2(0.0, 0.0), mtm = make_double2(0.0, 0.0);
      for (int s = 0; s <= t; ++s) {
        if (cm[s].x == 0.0 && cm[s].y == 0.0) continue;
        for (int r = 0; r < nm; ++r) {
          if (coef[r].x == 0.0 && coef[r].y == 0.0) continue;
          cfma(mtk, cmul(cm[s], coef[r]), gbil(mem[s], mem[r]));
        }
        for (int r = 0; r <= t; ++r) {
          if (cm[r].x == 0.0 && cm[r].y == 0.0) continue;
          cfma(mtm, cmul(cm[s], cm[r]), gbil(mem[s], mem[r]));
        }
      }
      const double2 alpha = cdiv(mtk, mtm);
      for (int s = 0; s <= t; ++s) coef[s] = csub(coef[s], cmul(alpha, cm[s]));
      partner = m;
    }
    // ||v||_2^2 = sum conj(c_s) c_r u_s^H u_r
    double v2 = 0.0;
    double2 vtv = make_double2(0.0, 0.0);
    for (int s = 0; s < nm; ++s) {
      if (coef[s].x == 0.0 && coef[s].y == 0.0) continue;
      for (int r = 0; r < nm; ++r) {
        if (coef[r].x == 0.0 && coef[r].y == 0.0) continue;
        const double2 h = gher(mem[s], mem[r]);
        const double2 cc = cmul(cconj(coef[s]), coef[r]);
        v2 += cc.x * h.x - cc.y * h.y;
        cfma(vtv, cmul(coef[s], coef[r]), gbil(mem[s], mem[r]));
      }
    }
    const double u2 = gher(k, k).x;
    const double ratio = sqrt(fmax(v2, 0.0) / fmax(u2, 1e-300));
    double2* ck = out_coef + (long long)k * kMaxComp;
    if (partner >= 0 && ratio < drop_tol) {
      kept_flag[k] = 0;
      ++n_dup;
      if (win[partner] != win[k]) {
        const int lo = win[partner] < win[k] ? win[partner] : win[k];
        const int hi = win[partner] < win[k] ? win[k] : win[partner];
        for (int i = lo; i < hi; ++i) holes[i] = 0;
      }
      for (int s = 0; s < kMaxComp; ++s) ck[s] = make_double2(0.0, 0.0);
      continue;
    }
    const double2 sc = cdiv(make_double2(1.0, 0.0), csqrt_p(vtv));
    for (int s = 0; s < kMaxComp; ++s) ck[s] = s < nm ? cmul(coef[s], sc) : make_double2(0.0, 0.0);
    kept_flag[k] = 1;
    ++n_kept;
  }
  // selection: the n_keep lowest by (Re, Im) among kept
  int nsel = 0;
  for (int k = 0; k < n; ++k)
    if (kept_flag[k]) order_tmp[nsel++] = k;
  // insertion sort by (Re, Im, index)
  for (int i = 1; i < nsel; ++i) {
    const int v = order_tmp[i];
    int j = i - 1;
    while (j >= 0) {
      const double2 a = eps[order_tmp[j]], b = eps[v];
      const bool greater = a.x > b.x || (a.x == b.x && (a.y > b.y || (a.y == b.y && order_tmp[j] > v)));
      if (!greater) break;
      order_tmp[j + 1] = order_tmp[j];
      --j;
    }
    order_tmp[j + 1] = v;
  }
  const int nout = (n_keep > 0 && n_keep < nsel) ? n_keep : nsel;
  for (int q = 0; q < nout; ++q) {
    const int k = order_tmp[q];
    out_eps[q] = eps[k];
    int nm = 0;
    for (int a = 0; a <= k && nm < kMaxComp; ++a) {
      if (comp[a] != comp[k]) continue;
      const double2 c = out_coef[(long long)k * kMaxComp + nm];
      out_src[(long long)q * kMaxComp + nm] = a;
      out_coef[(long long)(n + q) * kMaxComp + nm] = c;  // output coefficients stored after the n work rows
      ++nm;
    }
    out_nterm[q] = nm;
  }
  int nh = 0;
  for (int i = 0; i + 1 < p; ++i) nh += holes[i];
  out_info[0] = nout;
  out_info[1] = n_dup;
  out_info[2] = nh;
  out_info[3] = status;
}

__global__ void merge_apply_kernel(const double2* __restrict__ U, int ldu, int N, int nout, const int* __restrict__ src,
                                   const double2* __restrict__ coef, const int* __restrict__ nterm,
                                   double2* __restrict__ out, int ldo) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * nout) return;
  const long long r = t / nout;
  const int q = (int)(t % nout);
  double2 acc = make_double2(0.0, 0.0);
  const int nt = nterm[q];
  for (int e = 0; e < nt; ++e) {
    const double2 c = coef[(long long)q * kMaxComp + e];
    if (c.x == 0.0 && c.y == 0.0) continue;
    cfma(acc, c, U[r * ldu + src[(long long)q * kMaxComp + e]]);
  }
  out[r * ldo + q] = acc;
}

}  // namespace

size_t merge_coef_elems(int n) { return (size_t)(2 * n + 1) * kMaxComp; }
size_t merge_src_elems(int n) { return (size_t)(n + 1) * kMaxComp; }
int merge_max_comp() { return kMaxComp; }

void merge_run(const MergeArgs& a, cudaStream_t s, long long* launches) {
  merge_plan_kernel<<<1, 256, 0, s>>>(a.eps, a.n, a.eq_rtol, a.comp, a.pairs, a.pair_cap, a.counts);
  SWI_CHECK_LAUNCH();
  int nchunks = 2 * 152;
  if (nchunks > a.N) nchunks = a.N;
  while (nchunks > 1 && (size_t)nchunks * a.pair_cap * 2 > a.work_elems) nchunks /= 2;
  const int rows_per_chunk = (a.N + nchunks - 1) / nchunks;
  nchunks = (a.N + rows_per_chunk - 1) / rows_per_chunk;
  const int gy = (a.pair_cap + 255) / 256 < 8 ? (a.pair_cap + 255) / 256 : 8;
  pair_gram_partial_kernel<<<dim3(nchunks, gy), 256, 0, s>>>(a.U, a.ldu, a.N, a.pairs, a.counts, rows_per_chunk,
                                                             a.work);
  SWI_CHECK_LAUNCH();
  pair_gram_reduce_kernel<<<(a.pair_cap + 255) / 256, 256, 0, s>>>(a.work, nchunks, a.counts, a.gram);
  SWI_CHECK_LAUNCH();
  merge_mgs_kernel<<<1, 32, 0, s>>>(a.eps, a.win, a.n, a.p, a.eq_rtol, a.drop_tol, a.comp, a.pairs, a.counts,
                                     a.gram, a.n_keep, a.src, a.coef, a.nterm, a.out_eps, a.info, a.holes, a.kept,
                                     a.order);
  SWI_CHECK_LAUNCH();
  if (launches) *launches += 4;
}

void merge_apply(const MergeArgs& a, int nout, cudaStream_t s, long long* launches) {
  if (nout <= 0) return;
  const long long n = (long long)a.N * nout;
  merge_apply_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.U, a.ldu, a.N, nout, a.src,
                                                                   a.coef + (size_t)a.n * kMaxComp, a.nterm,
                                                                   a.out_U, a.ldo);
  SWI_CHECK_LAUNCH();
  if (launches) ++*launches;
}

}  // namespace swi
