// Device-side Algorithm 2 (combine windows, drop redundant pairs, hole flags).
#pragma once

#include "swi_internal.cuh"

namespace swi {

struct MergeArgs {
  // inputs
  const double2* U;     // [N][ldu] all windows' pairs, windows in shift order
  int ldu, N, n, p;     // n pairs from p windows
  const double2* eps;   // [n]
  const int* win;       // [n] window of each pair
  double eq_rtol, drop_tol;
  int n_keep;           // 0 = keep all survivors
  // scratch
  int* comp;            // [n]
  int* pairs;           // [2 * pair_cap]
  int pair_cap;
  int* counts;          // [2]
  double2* work;        // partial Gram sums
  size_t work_elems;
  double2* gram;        // [2 * pair_cap]
  int* kept;            // [n]
  int* order;           // [n]
  int* holes;           // [p]
  // outputs
  int* src;             // [(n+1) * maxcomp]
  double2* coef;        // [(2n+1) * maxcomp]
  int* nterm;           // [n]
  double2* out_eps;     // [n]
  int* info;            // [4]: nout, n_dup, n_holes, status
  double2* out_U;       // [N][ldo]
  int ldo;
};

size_t merge_coef_elems(int n);
size_t merge_src_elems(int n);
int merge_max_comp();
void merge_run(const MergeArgs& a, cudaStream_t s, long long* launches);
void merge_apply(const MergeArgs& a, int nout, cudaStream_t s, long long* launches);

}  // namespace swi
