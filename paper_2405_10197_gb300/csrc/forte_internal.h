// Internal declarations shared by the translation units of libforte_gpu.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/forte_gpu.h"

namespace forte {

// Thread-local error text behind forte_last_error().
void set_error(const char *fmt, ...);
void clear_error();

#define FORTE_CUDA_TRY(expr)                                                               \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      forte::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,   \
                       __LINE__);                                                          \
      return FORTE_ERR_CUDA;                                                               \
    }                                                                                      \
  } while (0)

#define FORTE_LAUNCH_CHECK()                                                               \
  do {                                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                   \
    if (e_ != cudaSuccess) {                                                               \
      forte::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),         \
                       __FILE__, __LINE__);                                                \
      return FORTE_ERR_CUDA;                                                               \
    }                                                                                      \
  } while (0)

// One entry of the compact single-replacement list of a string I:
// E_pq |I> = sgn |J>,  valid when q is in I and (p not in I or p == q).
struct Repl {
  int J;          // address of the resulting string
  int8_t sgn;     // +1 / -1
  uint8_t pq;     // p * n + q
  uint8_t pair;   // symmetric pair index of {p, q}: max*(max+1)/2 + min
  uint8_t pad;
};
static_assert(sizeof(Repl) == 8, "Repl must pack into 8 bytes");

// Host-side string data of one spin.
struct SpinHost {
  int nel = 0;
  long long N = 0;
  int nk = 0;                      // entries per string in the compact list
  std::vector<uint32_t> str;       // masks, ascending
  std::vector<Repl> list;          // [N][nk]
  std::vector<int> csr_ptr;        // same-spin Hamiltonian, CSR [N+1]
  std::vector<int> csr_col;
  std::vector<double> csr_val;
  std::vector<double> diag;        // H_ss[I][I]
};

// Device-side copies of one spin's tables.
struct SpinDev {
  Repl *list = nullptr;
  int *csr_ptr = nullptr;
  int *csr_col = nullptr;
  double *csr_val = nullptr;
  float *csr_val32 = nullptr;
  uint32_t *str = nullptr;
  double *diag = nullptr;
  int *dense = nullptr;   // [N][n*n]: (J << 1) | (sgn < 0), or -1 when E_pq|I> = 0
  uint32_t *list4 = nullptr;  // [N][nk]: J | pair << 16 | (sgn < 0) << 31
  // [N][128]: scatter target of symmetric pair rs applied to string J:
  // I | (sgn < 0) << 14 for E_rs J = sgn I (r != s: the one of E_rs, E_sr that
  // does not vanish), 0xFFFF when neither applies or rs >= n(n+1)/2
  uint16_t *tabJ = nullptr;
};

// Scratch buffer that grows on demand and is owned by the context.
struct Scratch {
  void *ptr = nullptr;
  size_t bytes = 0;
  int ensure(size_t want);
  void release();
};

// One traced launch: events recorded before and after it on the context stream.
struct ProfRecord {
  const char *name;
  cudaEvent_t a, b;
};

}  // namespace forte

struct forte_ctx {
  int n = 0, na = 0, nb = 0;
  int npair = 0;
  long long Na = 0, Nb = 0, Ndet = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = FORTE_FP64;
  bool same_strings = false;  // alpha and beta tables identical (na == nb)

  std::vector<double> h, eri, kmat;  // host copies; kmat = h - 1/2 sum_r (pr|rq)
  forte::SpinHost sh[2];
  forte::SpinDev sd[2];

  double *d_gpair = nullptr;    // [npair][npair] (pq|rs) over symmetric pairs
  double *d_hdiag = nullptr;    // [Na][Nb]
  float *d_gpair32 = nullptr;   // FP32 copy for the mixed path
  // tensor-core operands of the integrals, [128][npair] (rows >= npair zero):
  // gT[rs][pq] = (pq|rs) split into BF16 hi + lo, and rounded to TF32
  uint16_t *d_gT_hi = nullptr, *d_gT_lo = nullptr;
  float *d_gT_t32 = nullptr;
  int *d_err = nullptr;         // device status of bounded waits: [0] flag (0 = ok), [2..3] wait budget
  unsigned long long wait_budget = 0;  // clock cycles of one pipeline wait (0: the default)
  // beta-string positions of the tensor-core alpha-beta kernel: strings grouped by a
  // linear 5-bit hash of their masks, one string per hash value in each aligned group
  // of 32 positions, so that the scatter of one warp meets 32 distinct banks
  long long ab_NBpos = 0;       // positions (multiple of 32); padding has no string
  uint16_t *d_abPosOf = nullptr;  // [N_beta]: position of each beta string
  int *d_abStrOf = nullptr;       // [ab_NBpos]: string at each position, -1 for padding
  uint16_t *d_abTab = nullptr;    // [tiles * 128][128]: position of E_rs (string at pos) | sign << 14
  uint16_t *d_abTabL = nullptr;   // the same entries lane-contiguous: [tiles][4][16 chunks][32 lanes][8]
  uint16_t *d_gTT_hi = nullptr, *d_gTT_lo = nullptr;  // [npair][128]: gT transposed (pair-major)
  bool ab_split = false;          // scatter into separate positive / negative accumulator words
  int8_t *d_abDcnt = nullptr;     // [N_beta]: (+) minus (-) signs of the replacements reaching each string
  // dense same-spin string Hamiltonians for the tensor-core same-spin sigma,
  // [N][N padded to 16] per spin (aliases when alpha and beta strings coincide)
  uint16_t *d_hd_hi[2] = {nullptr, nullptr}, *d_hd_lo[2] = {nullptr, nullptr};
  float *d_hd_t32[2] = {nullptr, nullptr};
  void *d_gpair2 = nullptr;                      // (hi, lo) FP32 pairs of d_gpair
  void *d_csr_val2[2] = {nullptr, nullptr};      // (hi, lo) pairs of the CSR values
  uint16_t *d_ozT = nullptr;    // [n*n][Nb padded to 64]: E_sr |Ib> of the beta strings (RDM Gram)
  double *d_g1tmp = nullptr;    // 1-RDM workspace of the tensor-core 2-RDM when the caller passes none
  float gmax = 0.f;             // max |(pq|rs)| (bounds the alpha-beta fixed-point scale)
  // FP64-class tensor-core alpha-beta term: digits of the integrals
  // [6][npair][128] (BF16 bits) and their row exponents [128]
  uint16_t *d_ozG = nullptr;
  int *d_ozGa = nullptr;
  uint16_t *d_ozTabT = nullptr;  // [128][Nb padded to 64]: the beta scatter table, pair-major
  double oz_gmax = 0.0;

  // Davidson controls and results
  int dv_max_sub = 12, dv_collapse = 2, dv_max_iter = 200;
  double dv_guard = 1e-8;
  int nroots_done = 0;
  int dv_iters = 0;
  std::vector<double> roots_E, roots_rnorm;
  double *d_roots = nullptr;    // [nroots][Ndet]
  size_t d_roots_cap = 0;
  double *d_guess = nullptr;    // restart vectors
  int nguess = 0;

  forte::Scratch sc_t1, sc_t2;     // sigma: transposes for the beta-beta term
  forte::Scratch sc_dv;            // Davidson subspace and work vectors
  forte::Scratch sc_small;         // small device arrays (dots, norms)
  unsigned *d_vk_count = nullptr;  // arrival counter of the fused reductions (zero between launches)
  forte::Scratch sc_rdm;           // RDM intermediates
  forte::Scratch sc_mixed;         // reduced-precision copies of vectors
  forte::Scratch sc_grad;          // per-state RDMs of the state-averaged gradient
  forte::Scratch sc_rdm3;          // 3-RDM intermediates
  forte::Scratch sc_gas;           // projected copy of the input of forte_sigma under a restriction
  forte::Scratch sc_spin;          // guess diagonal of a spin-parity sector
  forte::Scratch sc_aci;           // adaptive CI: masks, estimates, pristine diagonal, histograms
  forte::Scratch sc_df;            // (hi, lo) copy of the input of the double-FP32 sigma
  forte::Scratch sc_oz;            // digit bytes and scales of the tensor-core FP64-class sigma

  // occupation restriction (GAS / RAS): string classes per spin, allowed class pairs
  bool gas_on = false;
  long long gas_ndet = 0;
  int *d_gas_cls[2] = {nullptr, nullptr};  // [N_alpha], [N_beta]
  int gas_nc[2] = {0, 0};
  uint8_t *d_gas_ok = nullptr;             // [gas_nc[0]][gas_nc[1]]
  // the restricted sigma over the kept determinants only: kept alpha rows, and per
  // alpha class the beta strings of its allowed classes (offsets [nc_alpha + 1])
  int *d_gas_rows = nullptr;               // [gas_nrows]
  long long gas_nrows = 0;
  int *d_gas_boff = nullptr, *d_gas_blist = nullptr;
  int gas_maxnnz = 0;                      // longest same-spin CSR row (alpha)
  int *d_gas_coff = nullptr, *d_gas_cstr = nullptr;  // beta strings by class: [ncB + 1], [N_beta]
  unsigned long long *d_gas_reach = nullptr;         // [ncB]: classes reached by one beta replacement
  int gas_route = -1;                      // restricted sigma: -1 timed choice, 0 full grid, 1 kept only
  long long gas_ndiag = 0;                 // kept determinants with I_alpha == I_beta (n_alpha == n_beta)
  // restricted sigma path per vector type [FP64, FP32]: -1 not yet timed, 0 full
  // grid + projection, 1 kept determinants only; timed for the mode in gas_pick_mode
  int gas_pick[2] = {-1, -1};
  int gas_pick_mode[2] = {-1, -1};
  float gas_pick_ms[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // [type][grid, sparse]
  // spin-parity sector (Ms = 0): 0 off, +1 even S, -1 odd S
  int spin_parity = 0;
  // arbitrary determinant mask [Ndet] (the P and M spaces of adaptive CI)
  bool detmask_on = false;
  long long detmask_n = 0;
  long long detmask_ndiag = 0;  // masked-in determinants |I>|I> (square grids)
  uint8_t *d_detmask = nullptr;

  long long n_sigma_fp64 = 0, n_sigma_mixed = 0;
  bool prof_on = false;
  std::vector<forte::ProfRecord> prof;
  std::vector<cudaEvent_t> prof_pool;
};

namespace forte {

// Brackets one kernel launch with CUDA events when tracing is enabled.
struct ProfScope {
  forte_ctx *ctx;
  cudaEvent_t b = nullptr;
  ProfScope(forte_ctx *c, const char *name);
  ~ProfScope();
};

}  // namespace forte

#define FORTE_PROF(ctx, name) forte::ProfScope forte_prof_scope_(ctx, name)

namespace forte {

// setup.cu
// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum.
// Always the same value, so concurrent callers (batched solves) cannot undercut
// one another's launches.
cudaError_t set_smem_optin_max(const void *func);
int build_spin_tables(forte_ctx *ctx);
int upload_tables(forte_ctx *ctx);

// sigma_fp64.cu
int sigma_fp64(forte_ctx *ctx, const double *C, double *S, int nvec);
// the same with caller-provided beta-beta scratch T1, T2 (nvec * Ndet doubles each)
int sigma_fp64_scratch(forte_ctx *ctx, const double *C, double *S, int nvec, double *T1, double *T2);
int hdiag_build(forte_ctx *ctx);
// FP64-class sigma in double-FP32 arithmetic (relative error ~2^-46 per term);
// with_ab = false leaves out the alpha-beta term (same-spin terms only)
int sigma_df(forte_ctx *ctx, const double *C, double *S, int nvec, bool with_ab = true);

// sigma_oz.cu: FP64-class sigma whose alpha-beta term is formed from exact digit
// products on the tensor cores (precision mode FORTE_OZ64)
bool oz_ab_supported(const forte_ctx *ctx);
int sigma_oz64(forte_ctx *ctx, const double *C, double *S, int nvec);

int same_spin_f32(forte_ctx *ctx, const float *C32, float *S32, float *T1, float *T2, int nvec);

// sigma_ss_mma.cu: same-spin sigma of the reduced-precision modes as one dense
// tensor-core GEMM per vector (S32 = same-spin part, FP32)
bool ss_mma_supported(const forte_ctx *ctx);
int same_spin_mma(forte_ctx *ctx, const double *C, const uint16_t *Chi, const uint16_t *Clo, const float *Ct32,
                  void *tw, float *S32, int nvec, int mode);
int same_spin_mma(forte_ctx *ctx, const float *C, const uint16_t *Chi, const uint16_t *Clo, const float *Ct32,
                  void *tw, float *S32, int nvec, int mode);

// sigma_mixed.cu
int sigma_mixed(forte_ctx *ctx, const double *C, double *S, int nvec, int mode);
int sigma_mixed(forte_ctx *ctx, const float *C, float *S, int nvec, int mode);  // FP32 vectors
int mixed_setup(forte_ctx *ctx);
int mixed_status(forte_ctx *ctx);
// Allocate the device status array of the bounded waits (once) and write the wait budget.
int err_word_setup(forte_ctx *ctx);

// vec_kernels.cu: Davidson building blocks on FP64 vectors and on the FP32 vectors
// of the reduced-precision phase (HBM-bound; FP32 ones accumulate per warp in
// FP32, beyond that in FP64).  Reductions use the context's sc_small buffer.
int vk_multidot(forte_ctx *ctx, const double *V, int nv, long long ld, const double *x, long long n, double *out);
int vk_multidot(forte_ctx *ctx, const float *V, int nv, long long ld, const float *x, long long n, double *out);
int vk_combine(forte_ctx *ctx, const double *V, int nv, long long ld, const double *coef, int ncomb, double *out,
               long long ldo, long long n);
int vk_combine(forte_ctx *ctx, const float *V, int nv, long long ld, const double *coef, int ncomb, float *out,
               long long ldo, long long n);
// t = (H x - theta x) / (theta - H_II) for x = B u, |r|^2 into rnorm2.  With dots
// (not null) the residual norm goes to dots[0] instead, and dots[1 + i] = B_i . t
// (i < k), dots[1 + k] = |t|^2 are formed in the same pass; returns -1 (nothing
// launched) when the vectors do not suit the packet kernel that does this.
int vk_residual_precond(forte_ctx *ctx, const double *B, const double *S, int k, long long ld, const double *u,
                        double theta, double guard, double *t, double *rnorm2, long long n,
                        double *dots = nullptr);
int vk_residual_precond(forte_ctx *ctx, const float *B, const float *S, int k, long long ld, const double *u,
                        double theta, double guard, float *t, double *rnorm2, long long n, double *dots = nullptr);
// t_out = scale (t_in - B c), dots_out = [B^T t_out (zeros unless dots), |t_out|^2]
int vk_orth_update(forte_ctx *ctx, const double *B, int k, long long ld, const double *c, const double *t_in,
                   double *t_out, double *dots_out, long long n, bool dots = true, double scale = 1.0);
int vk_orth_update(forte_ctx *ctx, const float *B, int k, long long ld, const double *c, const float *t_in,
                   float *t_out, double *dots_out, long long n, bool dots = true, double scale = 1.0);
int vk_scale(forte_ctx *ctx, double *x, const double *src, double alpha, long long n);
int vk_scale(forte_ctx *ctx, float *x, const float *src, double alpha, long long n);
int vk_convert(forte_ctx *ctx, const double *x, float *y, long long n);
int vk_convert(forte_ctx *ctx, const float *x, double *y, long long n);
int vk_axpby(forte_ctx *ctx, double a, const double *x, double b, double *y, long long n);
// rinv = 1 / max(|theta - H_II|, guard); z = r * rinv with dot_out = [r . z, r . r]
int vk_precond_inv(forte_ctx *ctx, double theta, double guard, double *rinv, long long n);
int vk_precond_dot(forte_ctx *ctx, const double *r, const double *rinv, double *z, double *dot_out, long long n);
int vk_argmin_k(forte_ctx *ctx, const double *x, long long n, int k, long long *idx_out);
int vk_any_nonfinite(forte_ctx *ctx, const double *x, long long n, int *flag_host);

// gas.cu: occupation-restricted CI (P H P on the kept determinants)
int gas_set(forte_ctx *ctx, int nspace, const int *size, const int *gmin, const int *gmax, long long *ndet_out);
void gas_free(forte_ctx *ctx);
int gas_mask(forte_ctx *ctx, double *x, int nvec);  // zero the excluded entries of nvec vectors
int gas_mask(forte_ctx *ctx, float *x, int nvec);
// sigma = P H P C over the kept determinants only (C zero outside them; S written
// everywhere), in the precision of the vectors; gas_sparse() tells whether the
// restriction is small enough for it
bool gas_sparse(const forte_ctx *ctx);
int gas_sigma(forte_ctx *ctx, const double *C, double *S, int nvec);
int gas_sigma(forte_ctx *ctx, const float *C, float *S, int nvec);
long long space_dim(const forte_ctx *ctx);           // dimension of the space Davidson works in
int det_mask_fill(forte_ctx *ctx, double *x, int nvec, double value);  // value at the masked-out entries
int sigma_grid(forte_ctx *ctx, const double *C, double *S, int nvec);  // api.cu: unrestricted FP64-class sigma

// aci.cu: adaptive CI on the determinant grid
int aci_run(forte_ctx *ctx, double sigma, double gamma, int max_cycles, double tol, int parity, double *E_out,
            double *C_out, long long *nM_out, long long *nP_out, int *cycles_out);

// spin.cu: spin-parity sectors C^T = parity C for Ms = 0
int spin_set(forte_ctx *ctx, int parity);
int spin_project(forte_ctx *ctx, double *x, int nvec);  // x <- (x + parity x^T) / 2 (no-op when off)
int spin_project(forte_ctx *ctx, float *x, int nvec);
int spin_guess_diag(forte_ctx *ctx, const double **hd);  // diagonal that names one guess per sector pair

// rdm.cu
int rdm12_fp64(forte_ctx *ctx, const double *bra, const double *ket, double *g1, double *g2,
               bool tensor_ok = true);
int rdm3_fp64(forte_ctx *ctx, const double *C, double *g3);
// rdm_oz.cu: 2-RDM from the 1-RDM g1 and the tensor-core Gram of the
// symmetric / antisymmetric one-body images (reduced-precision modes, bra == ket)
bool rdm2_oz_supported(const forte_ctx *ctx);
int rdm2_oz(forte_ctx *ctx, const double *C, const double *g1, double *g2);
int sa_gradient(forte_ctx *ctx, int nstates, const double *weights, const double *C, double scale, double *dh,
                double *deri);

// Host Jacobi eigensolver for the small symmetric subspace matrix (ascending).
void sym_eig(int k, const double *A, double *w, double *U);

}  // namespace forte
