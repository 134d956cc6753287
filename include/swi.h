/*
 * swi.h -- C ABI of the GB300 partitioned shift-without-invert eigensolver.
 *
 * Method: Feldman & Zhou, "A partitioned shift-without-invert algorithm to
 * improve parallel eigensolution efficiency in real-space electronic
 * transport".  The library finds the n_r eigenpairs of smallest real part of
 * the complex-symmetric operator
 *
 *     A = H_KS - i Gamma,   H_KS = -1/2 nabla^2_FD + V(r),          (Eq. 1)
 *
 * on a 3D real-space grid, by splitting the real axis into windows j with real
 * shifts sigma_j, solving each shifted problem (A - sigma_j) U = (eps - sigma_j) U
 * for the n_r,j eigenvalues closest to sigma_j with a Krylov iteration on the
 * shifted, never-inverted operator ('SM' selection, Eq. 3), merging the windows
 * (Algorithm 2), normalising U^T U = I, and evaluating the transmission
 * T(E) = Tr{G Gamma_R G^dagger Gamma_L} with G(E) = sum_k U_k U_k^T / (E - eps_k)
 * (Section 1) and its gradients.
 *
 * Conventions for every entry point:
 *  - Grid: nx * ny * nz points, spacing h (bohr); flat index (k*ny + j)*nx + i
 *    (x fastest).  Hartree units.  The kinetic term is the 12th-order (radius-6)
 *    central finite difference; each axis needs at least 6 points.
 *  - Complex numbers are interleaved (re, im) doubles (C99 double _Complex /
 *    numpy complex128 layout).
 *  - A block of vectors is row-major [N][ld]: the vector index is innermost
 *    (element (r, c) at r*ld + c).
 *  - Pointers flagged `on_device` are CUDA device pointers on the context's
 *    device; otherwise host pointers.  The library never keeps a caller's
 *    pointer: inputs are copied before the call returns (device-to-device
 *    copies are ordered on the context's stream).
 *  - The library owns every device buffer it allocates.  Pointers returned by
 *    getters are borrowed and stay valid until the next swi_solve,
 *    swi_set_eigenpairs or swi_destroy on the same context.
 *  - Errors are returned as swi_status; no exception crosses the ABI.
 *    swi_last_error(ctx) gives a message for the last failing call on ctx
 *    (swi_last_error(NULL) for a failed swi_create).
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef SWI_H
#define SWI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swi_ctx swi_ctx;

typedef enum {
  SWI_OK = 0,
  SWI_EINVAL = 1,    /* invalid argument (size, sign, order, NaN ...) */
  SWI_ENOMEM = 2,    /* device or host allocation failed */
  SWI_ECUDA = 3,     /* a CUDA call or kernel failed */
  SWI_ENOCONV = 4,   /* some window did not converge within its matvec budget */
  SWI_HOLES = 5,     /* merged windows show an interface without redundancy */
  SWI_ETIMEOUT = 6,  /* a bounded device wait gave up */
  SWI_ENOTIMPL = 7,  /* option not implemented */
  SWI_ESTATE = 8     /* call out of order (e.g. transmission before solve) */
} swi_status;

enum { SWI_BC_ODD = 0, SWI_BC_ZERO = 1 };        /* boundary rule, see swi_create */
enum { SWI_PREC_F64 = 0, SWI_PREC_MIXED = 1 };   /* arithmetic of the Krylov loop */
enum { SWI_ARITH_DS = 2, SWI_ARITH_F64 = 1 };     /* see swi_solve_opts.arith */

/* Options of swi_solve.  Zero-initialise and set what you need; zero fields
 * take the defaults given here. */
typedef struct {
  int block;            /* b, Krylov block width (default 2; 1..32).  b = 1
                           selects single-vector windows, the form of the
                           paper's implicitly restarted Arnoldi: every window
                           adds one vector per step, all windows share each
                           stencil and Gram-Schmidt launch, and the products
                           stream complex128 bases in double-single arithmetic.
                           b = 2 runs the same batched loop with two new
                           vectors per window and step (Cholesky-QR twice
                           inside the pair): one starting vector spans only one
                           vector of each eigenspace, so eigenvalues of
                           multiplicity two (a symmetric cross-section) need
                           b = 2 for both partners.  b >= 3 runs wide blocks
                           (block Gram-Schmidt on tensor-core digit products;
                           SWI_ARITH_F64 always runs that form, b = 0 there
                           meaning 16).  SWI_PREC_MIXED contexts run the 1- and
                           2-vector forms only, on complex64 bases with FP32
                           arithmetic */
  int max_basis;        /* m_j, basis size before a restart (default
                           max(2 n_req + 1, keep + (8 + j mod 3) b) rounded
                           up to b, j the window index: the stagger keeps
                           equal windows from restarting in step; for
                           b = 1 or 2 max(2 n_req + 1,
                           keep + 128 + 8 (j mod 3)), at most 1000 for
                           b = 1 and 510 for b = 2) */
  int keep;             /* Ritz vectors kept at a restart (default
                           max(n_req + ceil(n_req/2), n_req + b), at most
                           m_j - b) */
  int arith;            /* arithmetic of the Krylov loop and T(E):
                           0 or SWI_ARITH_DS (default) -- stencil, Cholesky-QR,
                           projected Schur step and T(E) projections in
                           double-single on the FP32 pipes; for b <= 2 the
                           Gram-Schmidt passes as described with the kernels
                           (FP32 first Gram and second update, double-single
                           accurate pass), for b >= 3 Gram-Schmidt products and
                           the restart rotation on the tensor cores with an
                           exact digit split; ~1e-13 relative;
                           SWI_ARITH_F64 -- native FP64 throughout.  The final
                           explicit residual check is native FP64 in both. */
  long long max_matvecs;/* per-window budget of operator applications per
                           vector (default 2,000,000) */
  double rel_tol;       /* convergence: ||A u - eps u|| <= rel_tol ||A||_G ||u||,
                           ||A||_G the Gershgorin bound (default 1e-10) */
  double eq_rtol;       /* Algorithm 2 equal-eigenvalue test
                           |l_m - l_k| <= eq_rtol max(1,|l_k|) (default 1e-8) */
  double drop_tol;      /* Algorithm 2 redundancy test ||v_k||/||v_k^0|| < drop_tol
                           (default 1e-6) */
  unsigned long long seed; /* seed of the random start blocks (default 1) */
  int n_keep;           /* pairs kept after the merge, lowest real part first
                           (0 = all merged pairs) */
  int reserved1;
} swi_solve_opts;

/* Per-window outcome of swi_solve. */
typedef struct {
  double sigma;         /* shift E_S,j */
  int n_req;            /* requested pairs n_r,j */
  int n_conv;           /* converged pairs delivered by the window */
  long long matvecs;    /* operator applications (vectors) */
  int restarts;
  int basis;            /* m_j used */
  double max_res;       /* largest relative residual of the delivered pairs */
  int schur_retries;    /* restarts whose double-single Schur step gave up and
                           were recomputed in native FP64 */
  int reserved;
} swi_window_info;

typedef struct {
  int n_windows;
  int n_pairs;          /* pairs after merge and selection */
  int n_converged;      /* of those, pairs whose explicitly recomputed relative
                           residual is <= rel_tol */
  int n_duplicates;     /* pairs removed as redundant by Algorithm 2 */
  int n_holes;          /* interfaces between adjacent windows with no redundancy */
  int reserved;
  long long matvecs;    /* total over windows */
  double max_rel_res;   /* largest explicit relative residual of the kept pairs */
  double anorm;         /* ||A||_G used for the relative residuals */
  double t_krylov_s;    /* wall time of the windowed Krylov phase */
  double t_merge_s;     /* wall time of merge, selection and normalisation */
} swi_solve_info;

/* Create a context on the current CUDA device for the operator
 * A = H_KS - i Gamma of Eq. 1 on an nx x ny x nz grid of spacing h (Section 1:
 * the Hamiltonian is applied as a matrix-free finite-difference formula, never
 * stored).  *out receives the context, owned by the caller (swi_destroy).
 *  bc: SWI_BC_ODD -- psi = 0 on the planes just outside the grid, ghosts by
 *      odd reflection u[-1-k] = -u[-1+k] (keeps A = A^T exactly);
 *      SWI_BC_ZERO -- every ghost is zero.
 *  precision: SWI_PREC_F64 -- complex128 Krylov vectors with FP64-class
 *      arithmetic (native FP64 or double-single, swi_solve_opts.arith);
 *      SWI_PREC_MIXED -- the reduced-precision form: swi_solve runs
 *      1- or 2-vector windows on complex64 Krylov vectors with FP32 stencil
 *      and products (FP32 accumulation within chunks of at most 1024 grid
 *      rows, FP64 across them) and the projected eigenproblems in
 *      double-single; the delivered pairs are complex128 and their explicit
 *      FP64 residuals are reported, at the accuracy of FP32 arithmetic.
 *      Everything after the solve (merge, T(E), gradients) is FP64 in both.
 *  cuda_stream: cudaStream_t (or NULL for the legacy default stream) on which
 *      every kernel of this context runs.
 * Errors: SWI_EINVAL (an axis < 6, h <= 0, unknown bc/precision),
 *         SWI_ENOMEM, SWI_ECUDA. */
swi_status swi_create(swi_ctx** out, int nx, int ny, int nz, double h, int bc,
                      int precision, void* cuda_stream);

/* Local potential V(r) of H_KS (Eq. 1), N doubles in Ha.  Errors: SWI_EINVAL
 * (NULL, non-finite value). */
swi_status swi_set_potential(swi_ctx* ctx, const double* V, int on_device);

/* Absorbing potentials Gamma_L, Gamma_R (Section 1): N doubles each, >= 0.
 * A = H_KS - i (Gamma_L + Gamma_R).  Errors: SWI_EINVAL (NULL, negative or
 * non-finite value). */
swi_status swi_set_absorber(swi_ctx* ctx, const double* gamma_L, const double* gamma_R,
                            int on_device);

/* Windows (Eq. 3): p real shifts sigma_j (strictly increasing) and requests
 * n_req[j] >= 1 (host arrays).  Errors: SWI_EINVAL. */
swi_status swi_set_windows(swi_ctx* ctx, int p, const double* sigma, const int* n_req);

/* Windows with complex shifts sigma_j = sigma_re[j] + i sigma_im[j]: the
 * two-dimensional partition Section 2 names for strongly non-Hermitian
 * problems, whose eigenvalues lie further below the real axis.  Window j
 * delivers the n_req[j] eigenpairs whose eigenvalues are nearest sigma_j (the
 * SM rule on A - sigma_j).  The operator applied is A - sigma_re[j]: the Krylov
 * space does not depend on the shift, and the imaginary part enters only the
 * selection, which ranks the Ritz values theta of A - sigma_re[j] by
 * |theta - i sigma_im[j]|.  Shifts strictly increasing by (Re, Im); host
 * arrays.  Solved by windows of 1 or 2 vectors (swi_solve with block 0, 1 or
 * 2 and the double-single or mixed arithmetic; SWI_EINVAL otherwise).  The
 * merged pairs are all kept when swi_solve_opts.n_keep is 0; the merge's
 * interface flags refer to consecutive windows in the order given, and
 * swi_fill_holes refuses such a solve (SWI_EINVAL).  swi_set_windows and the
 * planners set real shifts again; swi_get_windows reports the real parts.
 * Errors: SWI_EINVAL. */
swi_status swi_set_windows_complex(swi_ctx* ctx, int p, const double* sigma_re, const double* sigma_im,
                                   const int* n_req);

/* Plan p windows for the lowest n_r pairs with Algorithm 1: counts
 * n_r,j (round/ceil formulas) and shifts E_S,j = E_S,j-1 + ((E_max-E_min)/N)
 * (n_r,j + n_r,j-1)/2 with E_S,0 = E_min, n_r,0 = 0.  e_min/e_max are the
 * extremal real parts.  Requests are inflated: n_req = ceil(n_r,j * inflate).
 * Writes the plan into sigma_out/n_req_out (host, p entries each, may be NULL)
 * and sets it as the context's windows.  Errors: SWI_EINVAL. */
swi_status swi_plan_windows(swi_ctx* ctx, int n_r, int p, double e_min, double e_max,
                            double inflate, double* sigma_out, int* n_req_out);

/* Options and outcome of swi_plan_windows_sampled (zero-initialise; zero
 * fields take the defaults given here). */
typedef struct {
  int sample_req;          /* pairs per sampling window (default max(8, 2 n_r / p)) */
  int max_samples;         /* sampling windows at most (default 64) */
  double sample_tol;       /* relative residual of the sampling solves (default 1e-5) */
  double inflate;          /* request = ceil(n_r,j * inflate) + extra (default 1.25) */
  int extra;               /* added to every request (default 4; a negative value adds none) */
  int counts_rule;         /* 0: equal counts n_r / p (default); 1: Algorithm 1's n_r,j */
  long long max_matvecs;   /* operator applications per sampling window (default 200,000) */
} swi_plan_opts;

typedef struct {
  double e_min, e_max;     /* extremal real parts from the two exterior solves (Algorithm 1's inputs) */
  double e_top;            /* the n_r-th lowest sampled real part */
  int samples;             /* sampling windows solved */
  int windows;             /* windows planned */
  long long matvecs;       /* operator applications of all planning solves */
  double t_s;              /* wall time */
} swi_plan_info;

/* Plan p windows for the lowest n_r pairs without foreknowledge of the
 * spectrum (Section 2.2.1): two exterior single-vector solves, below min V and
 * above ||A||_G, give E_min and E_max; sampling solves of sample_req pairs at
 * a loose tolerance march up from E_min (each shift three quarters of the way
 * up the real parts the previous one found; the eigenvalues above its highest
 * real part are added) until n_r real parts are sampled; the windows are runs
 * of n_r,j consecutive sampled real parts (equal counts or Algorithm 1's
 * n_r,j), shift at the middle of each run, request ceil(n_r,j inflate) +
 * extra.  The plan becomes the context's windows and is written to
 * sigma_out / n_req_out (host arrays of p, may be NULL); info may be NULL.
 * The sampling solves replace the context's current pairs.  Errors:
 * SWI_EINVAL, SWI_ESTATE (no potential/absorbers), SWI_ENOCONV (the sampling
 * found too few pairs), SWI_ENOMEM, SWI_ECUDA. */
swi_status swi_plan_windows_sampled(swi_ctx* ctx, int n_r, int p, const swi_plan_opts* opts,
                                    double* sigma_out, int* n_req_out, swi_plan_info* info);

/* Apply the shifted operator to a block: Y[:, c] = (A - sigma[c]) X[:, c] for
 * c < nvec; X and Y are complex128 [N][nvec] (Eq. 3's matrix-vector product,
 * the hot kernel of the Krylov loop).  sigma is a host array of nvec doubles.
 * Errors: SWI_EINVAL, SWI_ESTATE (potential/absorber unset), SWI_ECUDA. */
swi_status swi_apply(swi_ctx* ctx, int nvec, const double* sigma, const void* X, void* Y,
                     int on_device);

/* swi_apply in double-single arithmetic (the operator of the double-single
 * Krylov loop): same arguments, complex128 in and out; every input value is
 * split into two floats and each of the 37 terms is an exact FMA product
 * summed with TwoSum, ~2^-48 relative per term.  Errors as swi_apply. */
swi_status swi_apply_ds(swi_ctx* ctx, int nvec, const double* sigma, const void* X, void* Y,
                        int on_device);

/* The same shifted operator on complex64 vectors with FP32 arithmetic (the
 * operator of the reduced-precision form): Y[:, c] = (A - sigma[c]) X[:, c],
 * X and Y complex64 [N][nvec] (interleaved re, im floats), sigma a host array
 * of nvec floats; V and Gamma are used as FP32 copies.  Error relative to the
 * FP64 operator: FP32 rounding of ~40 terms.  With on_device != 0, X and Y are
 * device pointers and the call returns without synchronising the context's
 * stream (the kernel is ordered on it); otherwise they are host arrays and the
 * call returns when Y is written.  Errors: SWI_EINVAL, SWI_ESTATE, SWI_ECUDA. */
swi_status swi_apply_c64(swi_ctx* ctx, int nvec, const float* sigma, const void* X, void* Y,
                         int on_device);

/* Solve all windows (batched on the device), merge them with Algorithm 2,
 * keep the lowest-real-part pairs and scale them to U^T U = I.
 * opts may be NULL (defaults); info may be NULL.
 * Returns SWI_OK, or SWI_ENOCONV / SWI_HOLES with the merged pairs still
 * available (partial result); SWI_ESTATE if windows/potential are unset. */
swi_status swi_solve(swi_ctx* ctx, const swi_solve_opts* opts, swi_solve_info* info);

/* The batching form: several independent systems (contexts of uneven grids,
 * potentials, absorbers and windows, all on one device) solved at once.  The
 * partition's independence (Section 2.1: windows, and here whole systems,
 * need nothing from one another until the merge) lets every system run its
 * swi_solve on a host worker and a stream of its own, so the device
 * interleaves the systems' stencil, Gram-Schmidt and Schur launches.  Each
 * context ends with its own merged pairs, as after swi_solve.
 *   n       number of contexts (>= 1, distinct, same device);
 *   ctxs    the contexts, each used by one worker at a time (no other call on
 *           them may run meanwhile);
 *   opts    as swi_solve, for every context (may be NULL);
 *   workers host workers (<= 0: min(n, hardware threads)); they take the
 *           systems largest first (grid points x requested pairs);
 *   infos   n records, status n codes (either may be NULL).
 * Returns SWI_OK when every solve did, else the first other status by context
 * order (each context's message in swi_last_error(ctx)).  The complex64
 * stencil's bounded-wait flag is per device, so with concurrent
 * SWI_PREC_MIXED solves a wait that ran out is reported by whichever solve
 * reads the flag first.  Errors: SWI_EINVAL (n < 1, NULL or repeated
 * contexts, contexts on different devices; message in swi_last_error(NULL)). */
swi_status swi_solve_batch(int n, swi_ctx* const* ctxs, const swi_solve_opts* opts, int workers,
                           swi_solve_info* infos, swi_status* status);

/* Continuation run (Section 2: a computed set of pairs is extended by adding
 * windows while the old pairs are kept; the paper's Conclusions): solve the p
 * new windows (sigma strictly increasing, n_req >= 1, host arrays) with the
 * context's solver and opts, then pass their pairs and the context's current
 * pairs through Algorithm 2 together -- each current pair belongs to the
 * window of the last solve whose shift is nearest its real part (pairs set by
 * swi_set_eigenpairs, e.g. restored from a checkpoint, form one window at the
 * middle of their real parts) -- all windows in shift order, keeping
 * opts->n_keep pairs (0: all) with U^T U = I.  With no current pairs it is a
 * plain solve of the new windows.  Returns as swi_solve (SWI_HOLES when an
 * interface of the union shows no redundancy); swi_get_windows then lists the
 * union's windows.  Errors: SWI_EINVAL (windows, or more than 64 in all),
 * SWI_ESTATE, SWI_ENOMEM, SWI_ECUDA. */
swi_status swi_solve_more(swi_ctx* ctx, int p, const double* sigma, const int* n_req,
                          const swi_solve_opts* opts, swi_solve_info* info);

/* Automated hole filling (Algorithm 1's loop over holes): for every interface
 * of the current windows that showed no redundancy in the last merge, a new
 * window at the middle of the gap between the highest real part delivered by
 * the lower window and the lowest delivered by the upper one, requesting
 * n = max(1, ceil(3/2 gap / ((e_max - e_min)/N))) pairs (e_min, e_max: the
 * extremal real parts of the spectrum, Algorithm 1's uniform-density scale);
 * the new windows are solved as a continuation (swi_solve_more), repeated
 * until no hole remains or max_rounds (0: 4) rounds ran.  *windows_added
 * (may be NULL) counts the windows inserted.  Returns SWI_OK, SWI_HOLES
 * (holes remain), SWI_ENOCONV, or the errors of swi_solve_more; SWI_ESTATE
 * without a previous solve. */
swi_status swi_fill_holes(swi_ctx* ctx, double e_min, double e_max, int max_rounds,
                          const swi_solve_opts* opts, swi_solve_info* info, int* windows_added);

/* Windows of the current pairs (shift order) and the interface flags of their
 * last merge: sigma[j] (may be NULL), holes[j] = 1 when the interface between
 * windows j and j + 1 showed no redundancy (0 for the last window); up to cap
 * entries, the window count in *p. */
swi_status swi_get_windows(swi_ctx* ctx, int cap, double* sigma, int* holes, int* p);

/* Per-window outcome of the last solve: fills up to `cap` entries, returns the
 * window count in *p. */
swi_status swi_get_window_info(swi_ctx* ctx, int cap, swi_window_info* out, int* p);

/* Borrowed device pointers to the current pairs (the eigenpairs of Eq. 1 that
 * Algorithm 2 kept, normalised to U^T U = I as Section 1 requires for the
 * spectral G): eps complex128[n], U complex128 [N][ldU] (row-major).  Valid
 * until the next call that changes the pairs.  Errors: SWI_ESTATE (no pairs). */
swi_status swi_get_eigenpairs(swi_ctx* ctx, int* n, const void** eps_dev, const void** U_dev,
                              int* ldU);

/* Copy the current pairs out: eps (n complex128), U ([N][n] complex128,
 * ld = n).  Either pointer may be NULL.  on_device selects the destination. */
swi_status swi_copy_eigenpairs(swi_ctx* ctx, void* eps, void* U, int on_device);

/* Replace the current pairs with caller-supplied ones (e.g. a previous run's,
 * Section 2's continuation runs): eps complex128[n], U complex128 [N][n],
 * assumed to satisfy U^T U = I. */
swi_status swi_set_eigenpairs(swi_ctx* ctx, int n, const void* eps, const void* U,
                              int on_device);

/* Explicit relative residuals ||A u_k - eps_k u_k|| / (||A||_G ||u_k||) of the
 * current pairs, A of Eq. 1 applied in native FP64 (the convergence measure of
 * the windows of Eq. 3; the paper states no tolerance), ||A||_G the Gershgorin
 * bound of A.  res_out: host array of n doubles.  Errors: SWI_ESTATE (no pairs). */
swi_status swi_residuals(swi_ctx* ctx, double* res_out);

/* Options of swi_refine (zero-initialise; zero fields take the defaults). */
typedef struct {
  int max_sweeps;       /* sweeps at most (default 3) */
  int group;            /* consecutive pairs (by real part) per Rayleigh-Ritz
                           problem, n_g (default 16; 1..32) */
  int arith;            /* as swi_solve_opts.arith for the products and the
                           projected Schur step; the stencil and the residuals
                           of a sweep are native FP64 in both */
  int reserved;
  double rel_tol;       /* target relative residual, as in swi_solve (default 1e-10) */
  double eq_rtol;       /* Algorithm 2 tests applied to the refined pairs, as */
  double drop_tol;      /* in swi_solve_opts (defaults 1e-8, 1e-6) */
  double near_tol;      /* groups whose largest relative residual is above it
                           are far from convergence and left as they are
                           (default 1e-3) */
} swi_refine_opts;

typedef struct {
  int sweeps;           /* sweeps carried out */
  int n_pairs;          /* pairs after the last sweep */
  int n_converged;      /* of those, pairs with relative residual <= rel_tol */
  int n_dropped;        /* pairs removed as redundant by Algorithm 2 */
  long long matvecs;    /* operator applications (vectors) */
  double max_rel_res_in;   /* largest relative residual before the first sweep */
  double max_rel_res;      /* ... and after the last one */
  double t_s;           /* wall time */
} swi_refine_info;

/* FP64 residual-correction sweeps on the current pairs (from swi_solve or
 * swi_set_eigenpairs): the Rayleigh-Ritz refinement of Section 1 applied to
 * the pairs themselves.  Pairs, ordered by real part, are cut into groups of
 * n_g; a group holding a pair with relative residual above rel_tol is
 * replaced by the Rayleigh-Ritz pairs of span[U_g, R_u], R_u = A U_u -
 * U_u diag(eps_u) over its unconverged pairs u: with Q an orthonormal basis
 * of that span (block Gram-Schmidt twice, Cholesky-QR2) and sigma_g the
 * middle of the group's real parts, the n_g eigenvalues theta of the pencil
 * Q^T (A - sigma_g) Q y = theta Q^T Q y (the unconjugated form, under which
 * the eigenvectors of the complex-symmetric A are bi-orthogonal, Section 1)
 * of smallest magnitude (the windows' SM selection, Eq. 3) give
 * eps = sigma_g + theta and U = Q y; a group keeps its new pairs unless they
 * lower its count of pairs at rel_tol or raise its largest explicit FP64
 * residual more than tenfold (otherwise the previous pairs are put back), and
 * a group whose largest residual is above near_tol is not swept.  All pairs then pass Algorithm 2 as
 * one window (equal-eigenvalue projection, redundancy drop, U^T U = I), and
 * the explicit FP64 residuals are recomputed; sweeps stop when every pair is
 * at rel_tol.  The pairs stay in library-owned memory (swi_get_eigenpairs).
 * Errors: SWI_ESTATE (no pairs, or no potential/absorbers), SWI_EINVAL,
 * SWI_ENOCONV (pairs above rel_tol after max_sweeps, the refined pairs are
 * kept; or a singular Q^T Q / an unconverged projected problem, the pairs of
 * the previous sweep are kept), SWI_ENOMEM, SWI_ECUDA. */
swi_status swi_refine(swi_ctx* ctx, const swi_refine_opts* opts, swi_refine_info* info);

/* T(E_e) = Tr{G Gamma_R G^dagger Gamma_L} (Section 1) for nE energies through
 * the spectral G of the current pairs:  R = U^T Gamma_R conj(U),
 * L = U^T Gamma_L conj(U), W = R o L, T_e = sum_kl g_ek W_kl conj(g_el),
 * g_ek = 1/(E_e - eps_k).  E, T_out: host arrays of nE doubles.
 * Errors: SWI_ESTATE (no pairs), SWI_EINVAL. */
swi_status swi_transmission(swi_ctx* ctx, int nE, const double* E, double* T_out);

/* Arithmetic of the T(E) and adjoint contractions of swi_transmission and
 * swi_grad (Section 1's T = Tr{G Gamma_R G^dagger Gamma_L} through the
 * spectral G).  SWI_CONTRACT_F64 (the default): FP64-class products.
 * SWI_CONTRACT_F32: FP32 products with FP32 accumulation:
 *  - the projections U^H Gamma U take U rounded to complex64 and run over the
 *    rows where the absorber, rounded to FP32, is a normal number (the other
 *    rows contribute exact zeros in FP32, or less than 2^-126 |U_ra||U_rc|);
 *    each thread adds 256-row block sums, and the row chunks' partial sums are
 *    added in FP64;
 *  - W = R o L, T_e and dT_e/dE_e are then formed in FP64 (n_E n^2 work);
 *  - the adjoint M = sum_e w_e D_e R conj(D_e) L^T D_e and
 *    dL/dV(r) = 2 Re sum_ac U_ra M_ac U_rc run in FP32 (U M is never stored:
 *    no N x n scratch), with |E_e - eps_k| above ~1e-38 so that g fits FP32.
 * The results carry FP32 rounding: relative to the sums of the magnitudes of
 * their terms, errors of order (accumulation length) x 2^-24.
 * swi_transmission_noalloc always uses the FP64-class products.  Changing the
 * setting drops the cached projections.  Errors: SWI_EINVAL (another value). */
enum {
  SWI_CONTRACT_F64 = 0,
  SWI_CONTRACT_F32 = 1
};
swi_status swi_set_contraction(swi_ctx* ctx, int contraction);

/* Vector-Jacobian product of T (the adjoint of the spectral T(E) of Section 1,
 * with dG = G dV G): given dL/dT_e (nE host doubles), writes
 *   dL/dV(r) = sum_e dLdT_e 2 Re[(G Gamma_R G^dagger Gamma_L G)_rr]
 *            = 2 Re sum_{a,c} U_ra M_ac U_rc,  M = sum_e dLdT_e D_e R conj(D_e) L^T D_e,
 *            D_e = diag(g_e)   (N doubles, on_device selects where), and
 *   dL/dE_e  = dLdT_e dT_e/dE_e,  dT_e/dE_e = -2 Re sum_kl g_ek^2 W_kl conj(g_el)
 *            (nE host doubles; with dLdT == NULL the bare dT_e/dE_e).
 * Either output may be NULL; dLdV needs dLdT.  Errors: SWI_ESTATE (no pairs or
 * no absorbers), SWI_EINVAL (NULL E, non-finite input). */
swi_status swi_grad(swi_ctx* ctx, int nE, const double* E, const double* dLdT, double* dLdV,
                    int dLdV_on_device, double* dLdE);

/* Per-kernel-class timing (CUDA events on the context's stream), for
 * roofline accounting.  Classes: */
enum {
  SWI_K_STENCIL = 0,  /* shifted stencil (A - sigma) X */
  SWI_K_GRAM = 1,     /* orthogonalisation inner products C = Q^H W (windows of
                         1-2 vectors: the first, FP32 Gram pass) */
  SWI_K_UPDATE = 2,   /* orthogonalisation update W -= Q C (windows of 1-2
                         vectors: the update fused with the second Gram pass) */
  SWI_K_CHOLQR = 3,   /* Cholesky-QR of each new block (windows of 1-2 vectors:
                         with the second, FP32 update) */
  SWI_K_SCHUR = 4,    /* projected eigenproblem (Schur form, SM selection, reordering) */
  SWI_K_ROTATE = 5,   /* thick-restart rotation Q Z and Ritz vectors */
  SWI_K_MERGE = 6,    /* Algorithm 2 and normalisation, explicit residuals */
  SWI_K_PROJ = 7,     /* Gamma-weighted projections U^H Gamma U of T(E) */
  SWI_K_TRANS = 8,    /* T(E) and dT/dE contraction */
  SWI_K_GRAD = 9,     /* adjoint dL/dV */
  SWI_K_COUNT = 10
};
typedef struct {
  long long launches; /* timed launch groups */
  double ms;          /* summed device time */
  double flops;       /* algorithmic floating-point operations (FMA = 2) */
  double bytes;       /* algorithmic HBM bytes (each operand read once, output written once) */
} swi_kernel_stats;

/* enable != 0: start recording (and clear previous records); 0: stop. */
swi_status swi_profile(swi_ctx* ctx, int enable);

/* Synchronise the stream and sum the records per class into out[SWI_K_COUNT]. */
swi_status swi_profile_read(swi_ctx* ctx, swi_kernel_stats* out);

/* T(E) for the context's current pairs, like swi_transmission, but without
 * allocating anything on the device or through any allocator.  The paper has
 * no counterpart: this exists for callers that must not allocate device
 * memory at call time -- hosts whose framework owns the whole device memory
 * budget (a caching allocator that must not see foreign allocations, a hard
 * memory cap) or whose allocations must all happen up front.
 *  - The call copies E in and T out through pageable host memory and
 *    synchronises the context's stream before it returns.
 *  - Limits: at most 64 eigenpairs in the context and 1024 energies per call;
 *    larger sizes return SWI_EINVAL (use swi_transmission instead).  Any grid
 *    size is accepted: the projections run over slabs of 65,536 grid rows.
 *  - Scratch: one file-scope device array of 4.6 MB that every GPU which loads
 *    the library holds until the process exits.  Its device address is looked
 *    up once per device ordinal (cudaGetSymbolAddress, with that device
 *    current) by swi_create; the call itself only reads the cached address.
 *  - Every call on a device shares that array, which keeps the last call's
 *    contents; calls whose work overlaps on the GPU (other host threads, other
 *    contexts on other streams) race on it and must be serialised by the
 *    caller.  Nothing in it needs clearing: each call overwrites what it reads.
 * E, T_out: host arrays of nE doubles.  Errors: SWI_ESTATE (no pairs or no
 * absorbers), SWI_EINVAL (sizes, NULL, non-finite energy), SWI_ECUDA. */
swi_status swi_transmission_noalloc(swi_ctx* ctx, int nE, const double* E, double* T_out);

/* Self-check of the projected eigenproblem of a thick restart (Section 2.1:
 * the exact-shift restart of the implicitly restarted Arnoldi method, which
 * the solver computes on the device once per restart of every window): the
 * complex Schur form H Z = Z T of an m x m matrix H, the `keep` Ritz values
 * of smallest magnitude moved to the leading block, with b coupling rows B
 * (the rows below H of the Arnoldi relation).  For tests of that kernel
 * against a host eigensolver; it touches no state of ctx but its stream.
 * H: m*m complex128 (interleaved re, im), row-major, host.  B: b*m complex128
 * row-major, host (b = 1 or 2; NULL: zero rows).  arith: SWI_ARITH_DS (the
 * solver's double-single kernel) or SWI_ARITH_F64.  T_out, Z_out: m*m complex128
 * row-major host arrays (T upper triangular, Z unitary, column i = Schur
 * vector i).  info_out[4]: kept columns, -, QR status (0 converged, 1
 * iteration limit, 3 m too large), Givens updates / 1024.  Errors: SWI_EINVAL
 * (m outside 2..1024, b, keep outside 1..m-b, NULL), SWI_ECUDA. */
swi_status swi_check_schur(swi_ctx* ctx, int m, int b, int keep, const double* H, const double* B, int arith,
                           double* T_out, double* Z_out, int* info_out);

/* Message of the last failing call on ctx (thread-local for ctx == NULL). */
const char* swi_last_error(const swi_ctx* ctx);

/* Number of this library's kernel launches on ctx since creation. */
long long swi_launch_count(const swi_ctx* ctx);

/* Free every buffer of ctx; NULL is ignored. */
void swi_destroy(swi_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SWI_H */
