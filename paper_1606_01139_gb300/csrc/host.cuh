// Host-side state of a solver context, shared by the translation units that
// drive the solves (capi.cu: the C ABI and the double-single solver;
// solve_mixed.cu: the complex64 single-vector solver).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "swi_internal.cuh"

namespace swi {
namespace host {

// 12th-order central second-difference weights (radius 6), c_0..c_6.
// Algorithmic FP64 flops of the stencil per grid point and vector: 18 neighbour
// pairs x (2 adds + 2 FMA) + the local term (2 MUL + 2 FMA) + the shift (2 adds).
constexpr double kStencilFlops = 18.0 * 6.0 + 6.0 + 2.0;

const double kFD[7] = {-5369.0 / 1800.0, 12.0 / 7.0, -15.0 / 56.0, 10.0 / 189.0,
                       -1.0 / 112.0,     2.0 / 1925.0, -1.0 / 16632.0};

struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t nbytes) {
    if (nbytes <= bytes) return;
    release();
    if (nbytes == 0) return;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      throw Error{SWI_ENOMEM, "cudaMalloc of " + std::to_string(nbytes) + " bytes failed"};
    }
    bytes = nbytes;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct Window {
  double sigma = 0.0;
  int nreq = 0, m = 0, keep = 0, ld = 0;  // ld: columns of the Q buffers (m + b)
  DevMem Q[2], W, H, Bm, Z, S, Bz, theta, resid, C1, C2, G, R1, R1i, R2, R2i, Zext, Yw, eps_w, res_w, Hw, Zw;
  int cur = 0, p = 0;
  bool done = false, failed = false;
  long long matvecs = 0;
  int restarts = 0;
  int nconv = 0;
  double max_res = 0.0;
};
}  // namespace host
}  // namespace swi


struct swi_ctx {
  using DevMem = swi::host::DevMem;
  int device = 0;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 0, N = 0;
  double h = 0.0;
  int bc = SWI_BC_ODD, precision = SWI_PREC_F64;
  DevMem V, G, gL, gR;
  DevMem V32, G32;  // FP32 copies for the complex64 stencil
  DevMem VG32;      // (V, Gamma) pairs with even row length, for the TMA-staged stencil
  bool has_V = false, has_G = false;
  double maxabsV = 0.0, maxG = 0.0;
  std::vector<double> sigma;
  std::vector<double> sigma_im;  // imaginary parts of complex shifts (empty: all real)
  std::vector<int> nreq;
  // windows of the current pairs: shifts (shift order), the eigenvalues each
  // window delivered before the merge, and the merge's interface flags
  // (1 = no redundancy across the interface: a presumed hole)
  std::vector<double> last_sigma;
  std::vector<double2> last_eps_win;
  std::vector<int> last_win_of;
  std::vector<int> last_holes;
  bool last_complex = false;  // the current pairs came from windows with complex shifts
  // current pairs
  int npairs = 0;
  DevMem eps, U;  // [n], [N][n]
  std::vector<double> resid;
  std::vector<swi_window_info> winfo;
  // rows of each absorber whose FP32 value is a normal number ([lo, hi), empty
  // when there is none): the row range of the FP32 projections
  long long gL_lo = 0, gL_hi = 0, gR_lo = 0, gR_hi = 0;
  // transport cache
  int contract = SWI_CONTRACT_F64;
  bool have_RL = false;
  DevMem MR, ML, Rm, Lm, Wm, Mg, Ebuf, Tbuf, dEbuf, wbuf;
  DevMem R32, L32, part32, gt32, M32;  // FP32 contractions
  // workspaces
  DevMem gram_work, sig_dev, colwork, scratch, Uall, ordinfo, cholstat, ptrs, dres;
  // merge scratch
  DevMem m_comp, m_pairs, m_counts, m_work, m_gram, m_kept, m_order, m_holes, m_src, m_coef, m_nterm, m_info,
      m_win, m_eps_all, m_eps_out;
  long long launches = 0;
  int arith = SWI_ARITH_DS;  // arithmetic of the tall-skinny products (last solve's choice)
  std::string err;
  // per-kernel-class event timing
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  bool prof_on = false;
  double schur_flops = 0.0;  // work of the Schur steps, known only after they ran
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> evpool;
  ~swi_ctx() {
    for (auto& r : prof) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : evpool) cudaEventDestroy(e);
  }
};


namespace swi {
namespace host {

cudaEvent_t take_event(swi_ctx* c);

// Records CUDA events around the launches of its scope when profiling is on.
struct ProfScope {
  swi_ctx* c;
  int kind;
  double flops, bytes;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(swi_ctx* ctx, int k, double f, double by, cudaStream_t stream = nullptr);
  ~ProfScope();
};

void gram_dispatch(int arith, const swi::GramBatch& b, int N, const double* w, int bilinear, double2* work,
                   size_t work_elems, cudaStream_t s, long long* launches);
void rowgemm_dispatch(int arith, const swi::RowGemmBatch& b, int N, cudaStream_t s, long long* launches);
swi_status fail(swi_ctx* ctx, swi_status code, const std::string& msg);
swi::StencilParams stencil_params(const swi_ctx* c);
double gershgorin(const swi_ctx* c);
void copy_in(DevMem& dst, const void* src, size_t bytes, bool on_device, cudaStream_t s);
void sync(cudaStream_t s);
void apply_block(swi_ctx* c, const double2* X, int ldx, double2* Y, int ldy, int ncols, bool ds = false);
void explicit_residuals(swi_ctx* c, const double2* Ud, int ldu, const double2* epsd, int n, std::vector<double>& out);
void gram_work_ensure(swi_ctx* c, size_t elems);
// after a solve's merge: remember its windows, their delivered eigenvalues and
// the interface flags (read from the merge's device array)
void record_windows(swi_ctx* c, const std::vector<double2>& eps_all, const std::vector<int>& win_of, int nwin);
// continuation and hole filling (windows.cu); solve is the context's solver
swi_status do_solve_more(swi_ctx* c, int p, const double* sigma, const int* n_req, const swi_solve_opts* o,
                         swi_solve_info* info, swi_status (*solve)(swi_ctx*, const swi_solve_opts*, swi_solve_info*));
swi_status do_fill_holes(swi_ctx* c, double e_min, double e_max, int max_rounds, const swi_solve_opts* o,
                         swi_solve_info* info, int* windows_added,
                         swi_status (*solve)(swi_ctx*, const swi_solve_opts*, swi_solve_info*));
swi_status do_plan_sampled(swi_ctx* c, int n_r, int p, const swi_plan_opts* po, double* sigma_out, int* n_req_out,
                           swi_plan_info* pinfo, swi_status (*solve)(swi_ctx*, const swi_solve_opts*, swi_solve_info*));
// the windowed solve with single-vector windows (solve_sv.cu): block width 1
// in an FP64 context, and every solve of a SWI_PREC_MIXED context
swi_status do_solve_sv(swi_ctx* c, const swi_solve_opts* o, swi_solve_info* info);
void merge_pairs(swi_ctx* c, const double2* Uin, int ldu, const std::vector<double2>& eps_all,
                 const std::vector<int>& win_of, int nwin, double eq_rtol, double drop_tol, int n_keep, int* minfo);

}  // namespace host
}  // namespace swi
