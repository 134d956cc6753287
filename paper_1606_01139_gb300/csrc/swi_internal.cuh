// Internal declarations shared by the translation units of the library.
// Complex values are double2 (x = re, y = im); blocks of vectors are row-major
// [N][ld] with the vector index innermost.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/swi.h"

namespace swi {

// ---------------------------------------------------------------- complex math
__host__ __device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs(double2 a) { return hypot(a.x, a.y); }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
// principal square root
__host__ __device__ __forceinline__ double2 csqrt_p(double2 z) {
  double r = hypot(z.x, z.y);
  if (r == 0.0) return make_double2(0.0, 0.0);
  double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
  return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

// ---------------------------------------------------------------- error plumbing
struct Error {
  swi_status code;
  std::string msg;
};

#define SWI_CUDA_TRY(call)                                                                \
  do {                                                                                    \
    cudaError_t e__ = (call);                                                             \
    if (e__ != cudaSuccess)                                                               \
      throw ::swi::Error{SWI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)}; \
  } while (0)

#define SWI_CHECK_LAUNCH() SWI_CUDA_TRY(cudaGetLastError())

// ---------------------------------------------------------------- operator data
struct StencilParams {
  int nx, ny, nz;
  int bc;             // SWI_BC_ODD or SWI_BC_ZERO
  double cm[7];       // -c_m / (2 h^2), m = 0..6 (centre weight counts once per axis)
  const double* V;    // N
  const double* G;    // Gamma_L + Gamma_R, N
};

// One block of columns for the batched stencil: Y[:, c] = (A - sigma[c]) X[:, c]
struct StencilBlock {
  const double2* X;
  double2* Y;
  int ldx, ldy, ncols;
  int sigma_off;      // index into the sigma table of column 0
  int out_ds;         // double-single kernel: Y holds (re hi, re lo, im hi, im lo) floats instead of complex128
};

// complex64 form (FP32 arithmetic), one block of columns
struct StencilC64Params {
  int nx, ny, nz;
  int bc;
  float cm[7];       // -c_m / (2 h^2)
  const float* V;    // N
  const float* G;    // Gamma_L + Gamma_R, N
  const float2* VG;  // (V, Gamma) pairs, [nz][ny][nx rounded up to even] (the TMA-staged kernel)
};
// VG[(z ny + y) nxp + x] = (V, G) at (x, y, z), nxp = nx rounded up to even (padding zero)
void launch_pack_vg(const float* V, const float* G, int nx, int ny, int nz, float2* VG, cudaStream_t s);
void launch_stencil_c64(const StencilC64Params& P, const float2* X, int ldx, float2* Y, int ldy, int ncols,
                        const float* sigma_dev, cudaStream_t s, long long* launches);
// TMA-staged form (stencil_c64_tma.cu): needs an even ldx and a 16-byte aligned X
bool stencil_c64_tma_ok(const float2* X, int ldx);
void launch_stencil_c64_tma(const StencilC64Params& P, const float2* X, int ldx, float2* Y, int ldy, int ncols,
                            const float* sigma_dev, cudaStream_t s, long long* launches);
// nonzero if a TMA stencil block gave up a bounded wait since the last clear
int stencil_c64_tma_error(bool clear);

constexpr int kMaxBatch = 64;

struct StencilBatch {
  int n;
  StencilBlock blk[kMaxBatch];
};

void launch_stencil(const StencilParams& P, const StencilBatch& batch, const double* sigma_dev,
                    cudaStream_t s, long long* launches);
// The same batched operator in double-single arithmetic (complex128 in and out).
void launch_stencil_ds(const StencilParams& P, const StencilBatch& batch, const double* sigma_dev, cudaStream_t s,
                       long long* launches);

// ---------------------------------------------------------------- tall-skinny products
// C_j = op(X_j)^H diag(w) Y_j over the N rows (op = conj for the Hermitian
// product, identity-conjugate for the bilinear one), reduced deterministically.
struct GramJob {
  const double2* X;  // [N][ldx], columns [0, nx)
  const double2* Y;  // [N][ldy], columns [0, ny)
  double2* C;        // [nx][ldc] result (row i = column i of X)
  int ldx, ldy, ldc, nx, ny;
  int accumulate;    // C += result instead of C = result
};
struct GramBatch {
  int n;
  GramJob job[kMaxBatch];
};
// bilinear != 0: C = X^T diag(w) Y; else C = X^H diag(w) Y.  w may be NULL.
void launch_gram(const GramBatch& b, int N, const double* w, int bilinear, double2* work,
                 size_t work_elems, cudaStream_t s, long long* launches);

// Out[n, 0:ncols] = beta * Yin[n, 0:ncols] + alpha * X[n, 0:k] * M[0:k, 0:ncols]  (M is [k][ldm])
struct RowGemmJob {
  const double2* X;    // [N][ldx]
  const double2* M;    // [k][ldm] (device)
  const double2* Yin;  // [N][ldy] or NULL (beta ignored)
  double2* Out;        // [N][ldo]
  int ldx, ldm, ldy, ldo, k, ncols;
  double alpha, beta;
};
struct RowGemmBatch {
  int n;
  RowGemmJob job[kMaxBatch];
};
void launch_rowgemm(const RowGemmBatch& b, int N, cudaStream_t s, long long* launches);

// The same two products in double-single arithmetic on the FP32 pipes
// (FP64 inputs and outputs, ~1e-13 relative accuracy); see blockops_df.cu.
void launch_gram_df(const GramBatch& b, int N, const double* w, int bilinear, double2* work,
                    size_t work_elems, cudaStream_t s, long long* launches);
void launch_rowgemm_df(const RowGemmBatch& b, int N, cudaStream_t s, long long* launches);

// Per-column 2-norms of a residual block R = Y - X diag(theta): out[c] = ||Y[:,c] - theta_c X[:,c]||.
void launch_colnorm_resid(const double2* X, int ldx, const double2* Y, int ldy, const double2* theta,
                          int ncols, int N, double* out, double* work, size_t work_elems,
                          cudaStream_t s, long long* launches);

// Fill [N][ld] columns [c0, c0+ncols) with counter-based pseudo-random complex numbers.
void launch_random_block(double2* X, int ld, int c0, int ncols, int N, unsigned long long seed,
                         cudaStream_t s, long long* launches);

// ---------------------------------------------------------------- small dense (per window)
// Cholesky of Hermitian G (b x b, ld b) -> upper R with G = R^H R, and Rinv = R^{-1}.
// status[j] set to 1 if G is not numerically positive definite.
struct CholBatch {
  int n;
  const double2* G[kMaxBatch];
  double2* R[kMaxBatch];
  double2* Rinv[kMaxBatch];
};
void launch_chol_batch(const CholBatch& cb, int b, int* status, cudaStream_t s, long long* launches);

struct SchurJob {
  double2* H;        // [m][ld] in/out: on exit, T (upper triangular Schur form)
  double2* Z;        // [m][ld] out: unitary Schur vectors (column i = vector i)
  const double2* B;  // [b][ld] coupling rows (residual relation)
  double2* Bz;       // [b][ld] out: B Z[:, 0:k]
  double2* theta;    // [m] out: diag(T) after reordering
  double* resid;     // [m] out: ||B Z s_i|| / ||s_i|| for the kept Ritz vectors
  double2* S;        // [m][ld] out: eigenvectors of T[0:k,0:k] (columns), unit 2-norm
  int* ordinfo;      // [4]: out k (kept), nwanted_conv, status
  int m, ld, b, keep, nwant;
  int kmax;         // the kept block is never extended beyond kmax columns
  double tol_abs;    // absolute residual threshold
  void* Hw;          // [ld][ld] 16-byte work entries (double-single kernel only)
  void* Zw;          // [ld][ld] 16-byte work entries (double-single kernel only)
  double sig_im;     // imaginary part of a complex shift: the selection ranks |theta - i sig_im|
                     // (theta: eigenvalues of the projection of A - Re sigma)
};
struct SchurBatch {
  int n;
  SchurJob job[kMaxBatch];
};
void launch_schur_batch(const SchurBatch& b, cudaStream_t s, long long* launches);
// The same step in double-single arithmetic (schur_ds.cu); needs Hw, Zw.
void launch_schur_ds_batch(const SchurBatch& b, cudaStream_t s, long long* launches);

// Ritz coefficient matrix of the wanted pairs after a Schur step:
// Yw[:, q] = Z[:, 0:k] s_{w_q} (m x nwant, [m][ld]) and eps_w[q] = theta_{w_q} + sigma,
// wanted = the nwant smallest |theta| of the leading k, ordered by (Re, Im).
struct RitzJob {
  const double2* Z;
  const double2* S;
  const double2* theta;
  const double* resid;
  const int* ordinfo;
  double2* Yw;       // [m][ldy]
  double2* eps;      // [nwant]
  double* res_out;   // [nwant]
  int m, ld, ldy, nwant;
  double sigma;
  double sig_im;     // as SchurJob::sig_im (eps = theta + sigma, sigma the real shift applied)
};
struct RitzBatch {
  int n;
  RitzJob job[kMaxBatch];
};
void launch_ritz_batch(const RitzBatch& b, cudaStream_t s, long long* launches);
// H = S^-1 K (m x m, row-major, leading dimension ld; H holds K on entry, S is
// overwritten) by Gauss-Jordan elimination with partial pivoting, one CTA.
// *status (device): 0, or 1 + the column without a nonzero pivot.
void launch_small_solve(double2* S, double2* H, int m, int ld, int* status, cudaStream_t s, long long* launches);

// Block-Arnoldi bookkeeping after one expansion (A [Q V] = [Q V] H' + V' B'):
// H[0:p+b, p:p+b] = C1 + C2, H[p:p+b, 0:p] = B_old[:, 0:p], B = [0, R2 R1].
struct HUpdJob {
  double2* H;          // [ld][ld]
  double2* Bm;         // [b][ld]
  const double2* C1;   // [p+b][b]
  const double2* C2;   // [p+b][b]
  const double2* R1;   // [b][b]
  const double2* R2;   // [b][b]
  int ld, p, b;
};
struct HUpdBatch {
  int n;
  HUpdJob job[kMaxBatch];
};
void launch_hupdate_batch(const HUpdBatch& b, cudaStream_t s, long long* launches);

// Zext = [[Z[:, 0:k], 0], [0, I_b]]  ((m+b) x (k+b), [m+b][ldo]) for the thick restart.
struct ZextJob {
  const double2* Z;
  double2* Zext;
  int ldz, ldo, m, k, b;
};
struct ZextBatch {
  int n;
  ZextJob job[kMaxBatch];
};
void launch_zext_batch(const ZextBatch& b, cudaStream_t s, long long* launches);

// small element-wise helpers
void launch_copy_block(const double2* src, int lds, double2* dst, int ldd, int rows, int cols,
                       cudaStream_t s, long long* launches);
// dst[:, q] = src[:, idx[q]] for q < n (idx on the device)
void launch_gather_cols(const double2* src, int lds, const int* idx, int n, double2* dst, int ldd, int rows,
                        cudaStream_t s, long long* launches);
// Y[:, q] -= eps[q] X[:, q] for q < n (eps on the device)
void launch_sub_diag(double2* Y, int ldy, const double2* X, int ldx, const double2* eps, int n, int rows,
                     cudaStream_t s, long long* launches);

// ---------------------------------------------------------------- single-vector Krylov loop
// (krylov_sv.cu), also with blocks of nb = 2 new vectors per window and step.
// Per job (window): Q [N][ldq] basis columns [0, ncols) (complex64 or
// complex128; ncols may be 0), w the nb adjacent columns of a [N][ldw] block
// (complex64 in the FP32 form; in the double-single form four floats per
// entry, the heads and tails of the real and imaginary parts), c the
// [ncols][nb] FP64 coefficients, part [nchunks][ldp] FP64 chunk partials.
enum { SV_GRAM = 0, SV_UPDATE_GRAM = 1, SV_UPDATE = 2, SV_WGRAM = 3 };
struct SvJob {
  const void* Q;
  int ldq, ncols;
  void* w;
  int ldw;
  const double2* c;
  double2* part;
  int ldp;
};
struct SvBatch {
  int n;
  SvJob job[kMaxBatch];
};
// SV_GRAM: part = Q^H w ([ncols][nb]); SV_UPDATE_GRAM: w -= Q c, then
// part = Q^H w; SV_UPDATE: w -= Q c; SV_WGRAM: part = w^H w ([nb][nb], Q
// unused).  ds: complex128 basis with double-single products (the Gram pass
// and the update without a fused Gram in FP32, for the first pass and for the
// second pass's small coefficients), else complex64 in FP32.
void launch_sv_pass(const SvBatch& b, int mode, bool ds, int nb, int N, int rpc, cudaStream_t s,
                    long long* launches);
// rows per chunk for njobs windows (256 to 1024, a multiple of 8)
int sv_rows_per_chunk(int N, int njobs);
// Chunk sums.  mode 0: C[e] = sum of entry e < ncols * nb, added into
// H[(e / nb) * ldh + e % nb] when H is set.  mode 1: the Gram matrix G = w^H w
// of the block: R1 = chol(G) (upper, G = R1^H R1), r[0..nb^2) = R1^-1 and
// r[4..4+nb^2) = R1 (nb = 1: H[0] = ||w||).  mode 2 (nb = 2, the second
// Cholesky-QR pass): R2 = chol(G), r[0..4) = R2^-1, H[a * ldh + b] = (R2 R1)[a][b].
// A block whose Cholesky factor has a relative pivot below 1e-14 sets r[8] = 1.
struct SvReduceJob {
  const double2* part;
  int ldp, nchunks, ncols, nb;
  int mode;
  double2* C;
  double2* H;
  int ldh;
  double2* r;
};
struct SvReduceBatch {
  int n;
  SvReduceJob job[kMaxBatch];
};
void launch_sv_reduce(const SvReduceBatch& b, cudaStream_t s, long long* launches);
// dst1[:, b] (and dst2[:, b]) = sum_a w[:, a] r[a * nb + b] for b < nb, in the
// basis element type (out_w = 0) or in w's own format (out_w = 1, dst2 unused;
// in place allowed)
struct SvNormJob {
  const void* w;
  int ldw;
  void* dst1;
  int ld1;
  void* dst2;  // may be NULL
  int ld2;
  const double2* r;
  int out_w;
};
struct SvNormBatch {
  int n;
  SvNormJob job[kMaxBatch];
};
void launch_sv_normalize(const SvNormBatch& b, bool ds, int nb, int N, cudaStream_t s, long long* launches);
// Q[:, 0:k] = Q[:, 0:m] Z32 in place (FP32), Z32 [m][ldz] complex64
void launch_c64_rotate_inplace(float2* Q, int ldq, int N, int m, const float2* Z32, int ldz, int k, cudaStream_t s,
                               long long* launches);
void launch_z_to_c64(const double2* Z, int ldz, int m, int k, float2* Z32, int ld32, cudaStream_t s,
                     long long* launches);
// complex64 <-> complex128 copies of a [rows][cols] block
void launch_widen(const float2* src, int lds, double2* dst, int ldd, int rows, int cols, cudaStream_t s,
                  long long* launches);
void launch_narrow(const double2* src, int lds, float2* dst, int ldd, int rows, int cols, cudaStream_t s,
                   long long* launches);
void launch_copy_col_c64(const float2* src, int lds, float2* dst, int ldd, int rows, cudaStream_t s,
                         long long* launches);
void launch_random_col_c64(float2* dst, int ld, int rows, unsigned long long seed, cudaStream_t s,
                           long long* launches);

// ---------------------------------------------------------------- timing helper
double now_seconds();

}  // namespace swi
