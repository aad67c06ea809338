// C ABI entry points: context life cycle, sigma dispatch, the Davidson-Liu
// driver (step a7, with the mixed-precision refinement of step a8) and the
// RDM calls (a9).  Every long-vector operation runs in this library's
// kernels; the host only solves the small subspace eigenproblem and decides
// convergence.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "forte_internal.h"

namespace forte {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

static cudaEvent_t prof_event(forte_ctx *ctx) {
  if (!ctx->prof_pool.empty()) {
    cudaEvent_t e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(forte_ctx *c, const char *name) : ctx(c) {
  if (!ctx || !ctx->prof_on) return;
  cudaEvent_t a = prof_event(ctx), e = prof_event(ctx);
  if (!a || !e) return;
  cudaEventRecord(a, ctx->stream);
  ctx->prof.push_back(ProfRecord{name, a, e});
  b = e;
}

ProfScope::~ProfScope() {
  if (b) cudaEventRecord(b, ctx->stream);
}

// Cyclic Jacobi eigensolver for a small symmetric matrix (Golub & Van Loan,
// Sec. 8.5): A row-major k x k; w ascending; U[i*k + j] = component i of
// eigenvector j.
void sym_eig(int k, const double *A, double *w, double *U) {
  std::vector<double> a(A, A + (size_t)k * k), v((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) v[(size_t)i * k + i] = 1.0;
  double fro = 0.0;
  for (double x : a) fro += x * x;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) off += a[(size_t)p * k + q] * a[(size_t)p * k + q];
    if (off <= 1e-32 * fro || off == 0.0) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        double apq = a[(size_t)p * k + q];
        if (apq == 0.0) continue;
        double tau = (a[(size_t)q * k + q] - a[(size_t)p * k + p]) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int r = 0; r < k; ++r) {
          double arp = a[(size_t)r * k + p], arq = a[(size_t)r * k + q];
          a[(size_t)r * k + p] = c * arp - s * arq;
          a[(size_t)r * k + q] = s * arp + c * arq;
        }
        for (int r = 0; r < k; ++r) {
          double apr = a[(size_t)p * k + r], aqr = a[(size_t)q * k + r];
          a[(size_t)p * k + r] = c * apr - s * aqr;
          a[(size_t)q * k + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < k; ++r) {
          double vrp = v[(size_t)r * k + p], vrq = v[(size_t)r * k + q];
          v[(size_t)r * k + p] = c * vrp - s * vrq;
          v[(size_t)r * k + q] = s * vrp + c * vrq;
        }
      }
  }
  std::vector<int> ord(k);
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int x, int y) { return a[(size_t)x * k + x] < a[(size_t)y * k + y]; });
  for (int j = 0; j < k; ++j) {
    w[j] = a[(size_t)ord[j] * k + ord[j]];
    for (int i = 0; i < k; ++i) U[(size_t)i * k + j] = v[(size_t)i * k + ord[j]];
  }
}

int err_word_setup(forte_ctx *ctx) {
  if (!ctx->d_err) FORTE_CUDA_TRY(cudaMalloc(&ctx->d_err, 4 * sizeof(int)));
  const unsigned long long b = ctx->wait_budget ? ctx->wait_budget : 4000000000ull;
  const int w[4] = {0, 0, (int)(unsigned)(b & 0xFFFFFFFFull), (int)(unsigned)(b >> 32)};
  FORTE_CUDA_TRY(cudaMemcpyAsync(ctx->d_err, w, sizeof(w), cudaMemcpyHostToDevice, ctx->stream));
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return FORTE_OK;
}

// sigma over the whole determinant grid (no restriction applied), FP64-class mode
int sigma_grid(forte_ctx *ctx, const double *C, double *S, int nvec) {
  if (ctx->precision == FORTE_FP64) return sigma_fp64(ctx, C, S, nvec);
  return oz_ab_supported(ctx) ? sigma_oz64(ctx, C, S, nvec) : sigma_df(ctx, C, S, nvec);
}

// Under a small occupation restriction (gas_sparse) sigma has two exact routes:
// the kernel over the kept determinants, or the full-grid kernels of the mode
// followed by the projection.  Unless the caller fixed the route
// (forte_set_gas_route), the first call for each vector type and mode runs both,
// timed with events on the context stream, and later calls take the faster; the
// result always comes from the route kept.
template <typename T, typename Grid>
static int gas_timed_route(forte_ctx *ctx, const T *C, T *S, int nvec, int mode, Grid &&grid) {
  if (ctx->gas_route == 1) return gas_sigma(ctx, C, S, nvec);
  const int slot = sizeof(T) == 8 ? 0 : 1;
  if (ctx->gas_pick[slot] >= 0 && ctx->gas_pick_mode[slot] == mode)
    return ctx->gas_pick[slot] ? gas_sigma(ctx, C, S, nvec) : grid();
  struct Ev {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~Ev() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  for (auto &x : ev.e) FORTE_CUDA_TRY(cudaEventCreate(&x));
  FORTE_CUDA_TRY(cudaEventRecord(ev.e[0], ctx->stream));
  int rc = grid();
  if (rc) return rc;
  FORTE_CUDA_TRY(cudaEventRecord(ev.e[1], ctx->stream));
  rc = gas_sigma(ctx, C, S, nvec);
  if (rc) return rc;
  FORTE_CUDA_TRY(cudaEventRecord(ev.e[2], ctx->stream));
  FORTE_CUDA_TRY(cudaEventSynchronize(ev.e[2]));
  float tg = 0.f, ts = 0.f;
  FORTE_CUDA_TRY(cudaEventElapsedTime(&tg, ev.e[0], ev.e[1]));
  FORTE_CUDA_TRY(cudaEventElapsedTime(&ts, ev.e[1], ev.e[2]));
  ctx->gas_pick_ms[slot][0] = tg;
  ctx->gas_pick_ms[slot][1] = ts;
  ctx->gas_pick[slot] = ts <= tg ? 1 : 0;
  ctx->gas_pick_mode[slot] = mode;
  return ctx->gas_pick[slot] ? FORTE_OK : grid();
}

// Under an occupation restriction the input vectors lie in the kept space and
// the output is projected onto it (sigma = P H P C).
static int sigma_dispatch(forte_ctx *ctx, const double *C, double *S, int nvec, int mode) {
  if (nvec <= 0) return FORTE_OK;
  auto grid = [&]() -> int {
    int rc;
    if (mode == FORTE_FP64)
      rc = sigma_fp64(ctx, C, S, nvec);
    else if (mode == FORTE_DF32)
      rc = sigma_df(ctx, C, S, nvec);
    else if (mode == FORTE_OZ64)
      rc = sigma_oz64(ctx, C, S, nvec);
    else
      rc = sigma_mixed(ctx, C, S, nvec, mode);
    if (rc) return rc;
    return gas_mask(ctx, S, nvec);
  };
  // FP64-class modes (DF32 / OZ64) are counted with the FP64 ones
  if (mode == FORTE_FP64 || mode == FORTE_DF32 || mode == FORTE_OZ64)
    ctx->n_sigma_fp64 += nvec;
  else
    ctx->n_sigma_mixed += nvec;
  if (gas_sparse(ctx)) return gas_timed_route(ctx, C, S, nvec, mode, grid);
  return grid();
}

static int sigma_dispatch(forte_ctx *ctx, const float *C, float *S, int nvec, int mode) {
  if (nvec <= 0) return FORTE_OK;
  if (mode == FORTE_FP64 || mode == FORTE_DF32 || mode == FORTE_OZ64) {
    set_error("FP32 vectors need a reduced-precision sigma");
    return FORTE_ERR_ARG;
  }
  ctx->n_sigma_mixed += nvec;
  auto grid = [&]() -> int {
    int rc = sigma_mixed(ctx, C, S, nvec, mode);
    if (rc) return rc;
    return gas_mask(ctx, S, nvec);
  };
  if (gas_sparse(ctx)) return gas_timed_route(ctx, C, S, nvec, mode, grid);
  return grid();
}

// ----------------------------------------------------------------- Davidson

struct DvResult {
  std::vector<double> E, rn;
  int iters = 0;
  bool converged = false;
  bool stalled = false;  // Davidson-Liu stopped early: the residual stopped falling
};

// Davidson-Liu with the diagonal preconditioner stalls when the target state is
// not dominated by the determinants of lowest H_II (theta then sits among many
// diagonal values and the corrections are nearly unit vectors).  The iteration is
// declared stalled when its largest residual has not halved over DV_STALL
// iterations; the solve then continues with Jacobi-Davidson from the Ritz vectors.
constexpr int DV_STALL = 50;

// Index of the largest |x| (ties: lowest index) and the sign of that entry.
__global__ void k_absmax(const double *__restrict__ x, long long n, double *bval, long long *bidx) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double best = -1.0;
  long long bi = -1;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double v = fabs(x[j]);
    if (v > best) { best = v; bi = j; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double v2 = sv[threadIdx.x + s];
      long long i2 = si[threadIdx.x + s];
      if (i2 >= 0 && (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x]))) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { bval[blockIdx.x] = sv[0]; bidx[blockIdx.x] = si[0]; }
}

// splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Guess vector k: unit vector at idx plus a deterministic perturbation of norm
// ~amp, entries amp*sqrt(12/n)*(u-1/2) with u = splitmix64(i + (k+1)*gamma)
// in [0,1).  The perturbation couples the spin-flip symmetry sectors so that
// roots of every total spin are reachable from closed-shell guesses.
template <typename T>
__global__ void k_guess(T *__restrict__ x, long long n, long long idx, int k, double amp) {
  const double scale = amp * sqrt(12.0 / (double)n);
  const unsigned long long key = (unsigned long long)(k + 1) * 0x9E3779B97F4A7C15ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = splitmix64((unsigned long long)i + key);
    double u = (double)(z >> 11) * 0x1.0p-53;
    x[i] = (T)(scale * (u - 0.5) + (i == idx ? 1.0 : 0.0));
  }
}

static int fix_sign(forte_ctx *ctx, double *x, long long n) {
  const unsigned nb = (unsigned)std::min<long long>((n + 255) / 256, 512);
  int rc = ctx->sc_small.ensure(sizeof(double) * nb * 2 + 64);
  if (rc) return rc;
  double *bv = (double *)ctx->sc_small.ptr;
  long long *bi = (long long *)(bv + nb);
  {
    FORTE_PROF(ctx, "absmax");
    k_absmax<<<nb, 256, 0, ctx->stream>>>(x, n, bv, bi);
  FORTE_LAUNCH_CHECK();
  }
  std::vector<double> hv(nb);
  std::vector<long long> hi(nb);
  FORTE_CUDA_TRY(cudaMemcpyAsync(hv.data(), bv, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream));
  FORTE_CUDA_TRY(cudaMemcpyAsync(hi.data(), bi, sizeof(long long) * nb, cudaMemcpyDeviceToHost, ctx->stream));
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  double best = -1;
  long long b = -1;
  for (unsigned i = 0; i < nb; ++i)
    if (hi[i] >= 0 && (hv[i] > best || (hv[i] == best && hi[i] < b))) { best = hv[i]; b = hi[i]; }
  if (b < 0) return FORTE_OK;
  double val;
  FORTE_CUDA_TRY(cudaMemcpy(&val, x + b, sizeof(double), cudaMemcpyDeviceToHost));
  if (val < 0) return vk_scale(ctx, x, x, -1.0, n);
  return FORTE_OK;
}

// Ritz vectors X = B U (first nroots columns of the coefficients) into the FP64
// output; FP32 bases combine into the workspace W first.
static int ritz_out(forte_ctx *ctx, const double *B, int k, long long N, const double *coef, int nroots, double *,
                    double *out) {
  return vk_combine(ctx, B, k, N, coef, nroots, out, N, N);
}
static int ritz_out(forte_ctx *ctx, const float *B, int k, long long N, const double *coef, int nroots, float *W,
                    double *out) {
  int rc = vk_combine(ctx, B, k, N, coef, nroots, W, N, N);
  if (rc) return rc;
  return vk_convert(ctx, W, out, (long long)nroots * N);
}

// Davidson-Liu with the sigma of `mode` on vectors of type T: FP64, or FP32 for
// the reduced-precision phase that precedes the FP64 refinement (the subspace
// matrix and its eigenproblem are FP64 in both).
// guess: ng FP64 device vectors (may be 0 -> unit vectors at the lowest H_II).
// On return the Ritz vectors are in out_roots [nroots][N] (FP64).
template <typename T>
static int davidson_run(forte_ctx *ctx, int nroots, double tol, int mode, const double *guess, int ng,
                        int max_iter, double *out_roots, DvResult &res) {
  cudaStream_t st = ctx->stream;
  const long long N = ctx->Ndet;
  const long long Nsp = space_dim(ctx);  // dimension of the (possibly restricted) space
  int maxsub = std::max(ctx->dv_max_sub * nroots, nroots + 1);
  maxsub = (int)std::min<long long>(maxsub, Nsp);
  maxsub = std::min(maxsub, 63);
  if (maxsub < nroots) { set_error("subspace limit below nroots"); return FORTE_ERR_ARG; }
  int keep = std::max(nroots, std::min(ctx->dv_collapse * nroots, maxsub - 1));
  keep = std::min(keep, maxsub);
  // device layout: B[maxsub], S[maxsub], T[nroots], W[keep] vectors; then small arrays
  size_t nvecs = (size_t)maxsub * 2 + nroots + keep;
  size_t small_off = ((sizeof(T) * nvecs * N + 255) / 256) * 256;
  // coef, u, d0, d1, d2 (4416 doubles), then per root [|r|^2, B^T t, |t|^2] (66 each)
  size_t small_bytes = sizeof(double) * (64 * 64 + 4 * 64 + 64 + 64 * 66);
  int rc = ctx->sc_dv.ensure(small_off + small_bytes + 256);
  if (rc) return rc;
  T *B = (T *)ctx->sc_dv.ptr;
  T *S = B + (size_t)maxsub * N;
  T *Tv = S + (size_t)maxsub * N;
  T *W = Tv + (size_t)nroots * N;
  double *d_coef = (double *)((char *)ctx->sc_dv.ptr + small_off);  // [64*64]
  double *d_u = d_coef + 64 * 64;                                    // [64]
  double *d_d0 = d_u + 64;                                           // [65]
  double *d_d1 = d_d0 + 65;                                          // [65]
  double *d_d2 = d_d1 + 65;                                          // [65]
  double *d_rd = d_coef + 64 * 64 + 4 * 64 + 64;                     // [64][66]

  int k = 0;
  if (ng > 0) {
    // orthonormalise the supplied vectors into B
    std::vector<double> h_d(65);
    for (int i = 0; i < ng && k < maxsub; ++i) {
      const T *t;
      if (sizeof(T) == sizeof(double)) {
        t = (const T *)(const void *)(guess + (size_t)i * N);
      } else {  // the FP32 copy of the guess goes into the next basis slot first
        if ((rc = vk_convert(ctx, guess + (size_t)i * N, (float *)(void *)(B + (size_t)k * N), N))) return rc;
        t = B + (size_t)k * N;
      }
      if ((rc = vk_orth_update(ctx, B, k, N, nullptr, t, B + (size_t)k * N, d_d0, N))) return rc;
      FORTE_CUDA_TRY(cudaMemcpyAsync(h_d.data(), d_d0, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
      FORTE_CUDA_TRY(cudaStreamSynchronize(st));
      double n0 = h_d[k];
      if ((rc = vk_orth_update(ctx, B, k, N, d_d0, B + (size_t)k * N, B + (size_t)k * N, d_d1, N))) return rc;
      if ((rc = vk_orth_update(ctx, B, k, N, d_d1, B + (size_t)k * N, B + (size_t)k * N, d_d2, N))) return rc;
      FORTE_CUDA_TRY(cudaMemcpyAsync(h_d.data(), d_d2, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
      FORTE_CUDA_TRY(cudaStreamSynchronize(st));
      double n2 = h_d[k];
      if (!(n2 > 1e-20 * n0) || !(n2 > 0)) continue;
      if ((rc = vk_scale(ctx, B + (size_t)k * N, B + (size_t)k * N, 1.0 / sqrt(n2), N))) return rc;
      ++k;
    }
  }
  if (k < nroots) {
    // unit vectors at the lowest diagonal elements not already spanned
    int need = nroots - k;
    std::vector<long long> idx(nroots + ng + 1);
    const double *hd = ctx->d_hdiag;
    if (ctx->spin_parity && (rc = spin_guess_diag(ctx, &hd))) return rc;  // one candidate per mirror pair
    if ((rc = vk_argmin_k(ctx, hd, N, std::min<long long>(N, need + k), idx.data()))) return rc;
    int used = 0;
    for (size_t c = 0; c < idx.size() && used < need && c < (size_t)std::min<long long>(N, need + k); ++c) {
      T *b = B + (size_t)k * N;
      {
        unsigned nbk = (unsigned)std::min<long long>((N + 255) / 256, 152LL * 16);
        {
          FORTE_PROF(ctx, "guess");
          k_guess<T><<<nbk, 256, 0, st>>>(b, N, idx[c], k, 0.02);
        FORTE_LAUNCH_CHECK();
        }
        if ((rc = gas_mask(ctx, b, 1))) return rc;
        if ((rc = spin_project(ctx, b, 1))) return rc;
      }
      if (k > 0) {
        // orthogonalise against the supplied guesses
        std::vector<double> h_d(65);
        if ((rc = vk_multidot(ctx, B, k, N, b, N, d_d0))) return rc;
        if ((rc = vk_orth_update(ctx, B, k, N, d_d0, b, b, d_d1, N))) return rc;
        if ((rc = vk_orth_update(ctx, B, k, N, d_d1, b, b, d_d2, N))) return rc;
        FORTE_CUDA_TRY(cudaMemcpyAsync(h_d.data(), d_d2, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
        FORTE_CUDA_TRY(cudaStreamSynchronize(st));
        if (!(h_d[k] > 1e-12)) continue;
        if ((rc = vk_scale(ctx, b, b, 1.0 / sqrt(h_d[k]), N))) return rc;
      } else {
        std::vector<double> h_d(2);
        if ((rc = vk_multidot(ctx, b, 1, N, b, N, d_d0))) return rc;
        FORTE_CUDA_TRY(cudaMemcpyAsync(h_d.data(), d_d0, sizeof(double), cudaMemcpyDeviceToHost, st));
        FORTE_CUDA_TRY(cudaStreamSynchronize(st));
        if ((rc = vk_scale(ctx, b, b, 1.0 / sqrt(h_d[0]), N))) return rc;
      }
      ++k;
      ++used;
    }
    if (k < nroots) { set_error("could not build %d guess vectors", nroots); return FORTE_ERR_ARG; }
  }
  // sigma of the initial basis and the subspace matrix G = B^T H B
  std::vector<double> G((size_t)64 * 64, 0.0);
  auto Gat = [&](int i, int j) -> double & { return G[(size_t)i * 64 + j]; };
  if ((rc = sigma_dispatch(ctx, B, S, k, mode))) return rc;
  std::vector<double> h_dots(65);
  for (int j = 0; j < k; ++j) {
    if ((rc = vk_multidot(ctx, B, k, N, S + (size_t)j * N, N, d_d0))) return rc;
    FORTE_CUDA_TRY(cudaMemcpyAsync(h_dots.data(), d_d0, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < k; ++i) Gat(i, j) = h_dots[i];
  }
  std::vector<double> Gk, w, U, coef;
  res.E.assign(nroots, 0.0);
  res.rn.assign(nroots, INFINITY);
  res.converged = false;
  res.stalled = false;
  double best_rn = INFINITY;
  int best_it = 0;
  for (int it = 1;; ++it) {
    // Rayleigh-Ritz on the symmetrised subspace matrix
    Gk.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Gk[(size_t)i * k + j] = 0.5 * (Gat(i, j) + Gat(j, i));
    w.assign(k, 0.0);
    U.assign((size_t)k * k, 0.0);
    sym_eig(k, Gk.data(), w.data(), U.data());
    // residuals and preconditioned corrections; where the packet kernel applies, the
    // same pass forms B^T t and |t|^2 for the Gram-Schmidt step of the new direction
    // (not in a spin-parity sector, where t is projected before that step)
    std::vector<double> rn2(nroots), hrd((size_t)nroots * 66);
    std::vector<char> fused(nroots, 0);
    bool any_fused = false;
    for (int r = 0; r < nroots; ++r) {
      std::vector<double> u(k);
      for (int i = 0; i < k; ++i) u[i] = U[(size_t)i * k + r];
      FORTE_CUDA_TRY(cudaMemcpyAsync(d_u, u.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
      T *t = Tv + (size_t)r * N;
      int rr = -1;
      if (ctx->spin_parity == 0)
        rr = vk_residual_precond(ctx, B, S, k, N, d_u, w[r], ctx->dv_guard, t, nullptr, N, d_rd + (size_t)r * 66);
      if (rr == -1) {
        rr = vk_residual_precond(ctx, B, S, k, N, d_u, w[r], ctx->dv_guard, t, d_d0 + r, N);
      } else if (rr == FORTE_OK) {
        fused[r] = 1;
        any_fused = true;
      }
      if (rr) return rr;
    }
    FORTE_CUDA_TRY(cudaMemcpyAsync(rn2.data(), d_d0, sizeof(double) * nroots, cudaMemcpyDeviceToHost, st));
    if (any_fused)
      FORTE_CUDA_TRY(cudaMemcpyAsync(hrd.data(), d_rd, sizeof(double) * hrd.size(), cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaStreamSynchronize(st));
    for (int r = 0; r < nroots; ++r)
      if (fused[r]) rn2[r] = hrd[(size_t)r * 66];
    const int k_res = k;  // B[0..k_res) as the fused dots saw it
    bool all = true, bad = false;
    for (int r = 0; r < nroots; ++r) {
      res.E[r] = w[r];
      res.rn[r] = sqrt(std::max(0.0, rn2[r]));
      if (!isfinite(rn2[r]) || !isfinite(w[r])) bad = true;
      if (!(res.rn[r] < tol)) all = false;
    }
    res.iters = it;
    if (bad) { set_error("non-finite residual or eigenvalue in Davidson"); return FORTE_ERR_NUMERIC; }
    const double max_rn = *std::max_element(res.rn.begin(), res.rn.end());
    if (max_rn < 0.5 * best_rn) {
      best_rn = max_rn;
      best_it = it;
    }
    res.stalled = !all && it - best_it >= DV_STALL;
    bool stop = all || it >= max_iter || k >= Nsp || res.stalled;
    if (stop) {
      coef.assign((size_t)k * nroots, 0.0);
      for (int i = 0; i < k; ++i)
        for (int r = 0; r < nroots; ++r) coef[(size_t)i * nroots + r] = U[(size_t)i * k + r];
      FORTE_CUDA_TRY(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, st));
      if ((rc = ritz_out(ctx, B, k, N, d_coef, nroots, W, out_roots))) return rc;
      res.converged = all || (k >= Nsp);
      return FORTE_OK;
    }
    int nnew_want = 0;
    for (int r = 0; r < nroots; ++r) nnew_want += (res.rn[r] < tol) ? 0 : 1;
    bool collapsed = false;
    if (k + nnew_want > maxsub && k > keep) {
      collapsed = true;
      // collapse onto the lowest `keep` Ritz vectors
      coef.assign((size_t)k * keep, 0.0);
      for (int i = 0; i < k; ++i)
        for (int c = 0; c < keep; ++c) coef[(size_t)i * keep + c] = U[(size_t)i * k + c];
      FORTE_CUDA_TRY(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, st));
      if ((rc = vk_combine(ctx, B, k, N, d_coef, keep, W, N, N))) return rc;
      FORTE_CUDA_TRY(cudaMemcpyAsync(B, W, sizeof(T) * keep * N, cudaMemcpyDeviceToDevice, st));
      if ((rc = vk_combine(ctx, S, k, N, d_coef, keep, W, N, N))) return rc;
      FORTE_CUDA_TRY(cudaMemcpyAsync(S, W, sizeof(T) * keep * N, cudaMemcpyDeviceToDevice, st));
      std::fill(G.begin(), G.end(), 0.0);
      for (int c = 0; c < keep; ++c) Gat(c, c) = w[c];
      k = keep;
    }
    const int k_old = k;
    for (int r = 0; r < nroots; ++r) {
      if (res.rn[r] < tol) continue;
      if (k >= maxsub) break;
      T *t = Tv + (size_t)r * N;
      T *b = B + (size_t)k * N;
      if ((rc = spin_project(ctx, t, 1))) return rc;  // the sigma rounding leaves the sector slightly
      std::vector<double> h_d(65);
      std::vector<double> h0(65);
      const double *c0 = d_d0;  // device B^T t
      const T *src = b;         // vector pass 1 reads
      if (fused[r] && !collapsed && k == k_res) {
        // B^T t and |t|^2 from the residual pass: no copy pass, no host wait
        for (int i = 0; i <= k; ++i) h0[i] = hrd[(size_t)r * 66 + 1 + i];
        c0 = d_rd + (size_t)r * 66 + 1;
        src = t;
      } else {
        if ((rc = vk_orth_update(ctx, B, k, N, nullptr, t, b, d_d0, N))) return rc;  // copy + B^T t + |t|^2
        FORTE_CUDA_TRY(cudaMemcpyAsync(h0.data(), d_d0, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
        FORTE_CUDA_TRY(cudaStreamSynchronize(st));
      }
      if (!(h0[k] > 0.0) || !isfinite(h0[k])) continue;  // no new direction from this root
      // second pass only when the first removes more than half of |t|^2 (the
      // criterion of Daniel, Gragg, Kaufman and Stewart, Math. Comp. 30 (1976) 772:
      // ||t1|| >= ||t0|| / sqrt(2), with ||t1||^2 = ||t0||^2 - ||B^T t0||^2), which is
      // known before pass 1: pass 1 forms B^T t1 only when pass 2 will use it
      double proj = 0.0;
      for (int i = 0; i < k; ++i) proj += h0[i] * h0[i];
      const bool second = !(h0[k] - proj >= 0.5 * h0[k]);
      if (!second) {
        // one pass, normalised in the same pass: |t - B c|^2 = |t|^2 - |c|^2 for
        // orthonormal B (relative error ~ |B^T B - I| |c|^2 / |t|^2, with
        // |c|^2 <= |t|^2 / 2 here)
        const double nn = h0[k] - proj;
        if ((rc = vk_orth_update(ctx, B, k, N, c0, src, b, d_d1, N, false, 1.0 / sqrt(nn)))) return rc;
        ++k;
        continue;
      }
      if ((rc = vk_orth_update(ctx, B, k, N, c0, src, b, d_d1, N, second))) return rc;  // CGS pass 1
      const double *dfin = d_d1;
      if (second) {
        if ((rc = vk_orth_update(ctx, B, k, N, d_d1, b, b, d_d2, N, false))) return rc;  // CGS pass 2
        dfin = d_d2;
      }
      FORTE_CUDA_TRY(cudaMemcpyAsync(h_d.data(), dfin, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, st));
      FORTE_CUDA_TRY(cudaStreamSynchronize(st));
      double nn = h_d[k];
      if (!(nn > 1e-24 * h0[k]) || !(nn > 0.0)) continue;  // linearly dependent: drop
      if ((rc = vk_scale(ctx, b, b, 1.0 / sqrt(nn), N))) return rc;
      ++k;
    }
    if (k == k_old) {
      // no new direction: report the current Ritz vectors
      coef.assign((size_t)k * nroots, 0.0);
      for (int i = 0; i < k; ++i)
        for (int r = 0; r < nroots; ++r) coef[(size_t)i * nroots + r] = U[(size_t)i * k + r];
      FORTE_CUDA_TRY(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, st));
      if ((rc = ritz_out(ctx, B, k, N, d_coef, nroots, W, out_roots))) return rc;
      return FORTE_OK;
    }
    if ((rc = sigma_dispatch(ctx, B + (size_t)k_old * N, S + (size_t)k_old * N, k - k_old, mode))) return rc;
    for (int j = k_old; j < k; ++j) {
      if ((rc = vk_multidot(ctx, B, k, N, S + (size_t)j * N, N, d_d0))) return rc;
      FORTE_CUDA_TRY(cudaMemcpyAsync(h_dots.data(), d_d0, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
      FORTE_CUDA_TRY(cudaStreamSynchronize(st));
      for (int i = 0; i < k; ++i) { Gat(i, j) = h_dots[i]; Gat(j, i) = h_dots[i]; }
    }
  }
}

// FP64 refinement of Ritz vectors computed with a reduced-precision sigma
// (step a8).  Outer loop in FP64: Rayleigh-Ritz over V = [X, T] with exact
// sigma vectors, exact residuals R = H x - theta x.  Corrections T solve the
// projected equation  P (H~ - theta) P t = -R,  t orthogonal to X, by
// preconditioned conjugate gradients whose operator H~ is the reduced-precision
// sigma and whose preconditioner is |theta - H_II|^-1 (Jacobi-Davidson with an
// inexact inner solve).  Each outer step costs one FP64 sigma per root.
static int refine_jd(forte_ctx *ctx, int nroots, double tol, int inner_mode, int outer_mode, const double *X0,
                     double *out, int max_outer, DvResult &res) {
  cudaStream_t st = ctx->stream;
  const long long N = ctx->Ndet;
  // thick restart: after each Rayleigh-Ritz step the basis keeps nroots extra Ritz
  // vectors besides the targets, so that a state close above the last target (a
  // gap comparable to the start vectors' residual) stays resolved instead of being
  // mixed into the targets at every collapse
  const int nextra = (int)std::max(0LL, std::min<long long>({(long long)nroots, 63LL - 2 * nroots,
                                                               space_dim(ctx) - nroots}));
  const int nkeep = nroots + nextra;
  const int kmax = std::min(63, std::max(nroots * (max_outer + 1), nkeep + nroots));
  // vectors: V[kmax], HV[kmax], W[nkeep] (collapse target, then residuals), PCG: x r z p q
  // and the inverse preconditioner diagonal
  size_t nvec = (size_t)2 * kmax + nkeep + 6;
  size_t small_off = sizeof(double) * nvec * N;
  int rc = ctx->sc_dv.ensure(small_off + sizeof(double) * (64 * 64 + 4 * 66) + 256);
  if (rc) return rc;
  double *V = (double *)ctx->sc_dv.ptr;
  double *HV = V + (size_t)kmax * N;
  double *W = HV + (size_t)kmax * N;
  double *px = W + (size_t)nkeep * N, *pr = px + N, *pz = pr + N, *pp = pz + N, *pq = pp + N, *pinv = pq + N;
  double *d_coef = (double *)((char *)ctx->sc_dv.ptr + small_off);
  double *d_a = d_coef + 64 * 64, *d_b = d_a + 66, *d_s = d_b + 66;
  auto fetch = [&](const double *src, int cnt, double *dst) -> int {
    FORTE_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaStreamSynchronize(st));
    return FORTE_OK;
  };
  // project v onto the complement of V[0..nk): two classical Gram-Schmidt passes
  auto project = [&](double *v, int nk) -> int {
    int r2;
    if ((r2 = vk_multidot(ctx, V, nk, N, v, N, d_a))) return r2;
    if ((r2 = vk_orth_update(ctx, V, nk, N, d_a, v, v, d_b, N))) return r2;
    return vk_orth_update(ctx, V, nk, N, d_b, v, v, d_a, N, false);
  };
  FORTE_CUDA_TRY(cudaMemcpyAsync(V, X0, sizeof(double) * nroots * N, cudaMemcpyDeviceToDevice, st));
  // the start vectors come from a reduced-precision (FP32) phase: orthonormalise
  // them in FP64, since the Rayleigh-Ritz step below takes V as orthonormal
  {
    std::vector<double> hn(2);
    for (int r = 0; r < nroots; ++r) {
      double *v = V + (size_t)r * N;
      if (r > 0 && (rc = project(v, r))) return rc;
      if ((rc = vk_multidot(ctx, v, 1, N, v, N, d_s))) return rc;
      if ((rc = fetch(d_s, 1, hn.data()))) return rc;
      if (!(hn[0] > 0.0) || !isfinite(hn[0])) { set_error("degenerate start vector in refinement"); return FORTE_ERR_NUMERIC; }
      if ((rc = vk_scale(ctx, v, v, 1.0 / sqrt(hn[0]), N))) return rc;
    }
  }
  if ((rc = sigma_dispatch(ctx, V, HV, nroots, outer_mode))) return rc;
  double prev_rn = INFINITY;
  int k = nroots;
  std::vector<double> G, Gk, w, U, coef, h(66);
  res.E.assign(nroots, 0.0);
  res.rn.assign(nroots, INFINITY);
  res.converged = false;
  for (int outer = 0;; ++outer) {
    // Rayleigh-Ritz over V[0..k)
    G.assign((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j) {
      if ((rc = vk_multidot(ctx, V, k, N, HV + (size_t)j * N, N, d_a))) return rc;
      if ((rc = fetch(d_a, k, h.data()))) return rc;
      for (int i = 0; i < k; ++i) G[(size_t)i * k + j] = h[i];
    }
    Gk.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Gk[(size_t)i * k + j] = 0.5 * (G[(size_t)i * k + j] + G[(size_t)j * k + i]);
    w.assign(k, 0.0);
    U.assign((size_t)k * k, 0.0);
    sym_eig(k, Gk.data(), w.data(), U.data());
    const int nk = std::min(k, nkeep);  // Ritz vectors kept
    coef.assign((size_t)k * nk, 0.0);
    for (int i = 0; i < k; ++i)
      for (int r = 0; r < nk; ++r) coef[(size_t)i * nk + r] = U[(size_t)i * k + r];
    FORTE_CUDA_TRY(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, st));
    if ((rc = vk_combine(ctx, V, k, N, d_coef, nk, W, N, N))) return rc;
    FORTE_CUDA_TRY(cudaMemcpyAsync(V, W, sizeof(double) * nk * N, cudaMemcpyDeviceToDevice, st));
    if ((rc = vk_combine(ctx, HV, k, N, d_coef, nk, W, N, N))) return rc;
    FORTE_CUDA_TRY(cudaMemcpyAsync(HV, W, sizeof(double) * nk * N, cudaMemcpyDeviceToDevice, st));
    k = nk;
    // exact residuals R_r = HV_r - theta_r V_r (kept in W)
    bool all = true;
    for (int r = 0; r < nroots; ++r) {
      double *R = W + (size_t)r * N;
      FORTE_CUDA_TRY(cudaMemcpyAsync(R, HV + (size_t)r * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      if ((rc = vk_axpby(ctx, -w[r], V + (size_t)r * N, 1.0, R, N))) return rc;
      if ((rc = vk_multidot(ctx, R, 1, N, R, N, d_a))) return rc;
      if ((rc = fetch(d_a, 1, h.data()))) return rc;
      res.E[r] = w[r];
      res.rn[r] = sqrt(std::max(0.0, h[0]));
      if (!isfinite(h[0]) || !isfinite(w[r])) { set_error("non-finite residual in refinement"); return FORTE_ERR_NUMERIC; }
      if (!(res.rn[r] < tol)) all = false;
    }
    res.iters = outer;
    // an outer step that does not halve the residual means the reduced-precision
    // inner operator no longer resolves the correction: continue with FP64 ones
    const double max_rn = *std::max_element(res.rn.begin(), res.rn.end());
    if (outer > 0 && max_rn > 0.5 * prev_rn) inner_mode = outer_mode;
    prev_rn = max_rn;
    if (all || outer >= max_outer) {
      FORTE_CUDA_TRY(cudaMemcpyAsync(out, V, sizeof(double) * nroots * N, cudaMemcpyDeviceToDevice, st));
      res.converged = all;
      return FORTE_OK;
    }
    const int k0 = k;
    for (int r = 0; r < nroots; ++r) {
      if (res.rn[r] < tol || k >= kmax) continue;
      const double theta = w[r];
      const double bnorm = res.rn[r];
      // inner stopping rule: the correction equation's residual reduced 50-fold
      // (measured at CAS(14,14): a tighter inner solve, aimed at reaching tol in one
      // outer step, took more inner sigmas and the same number of outer ones)
      const double inner_rtol = 0.02;
      // PCG on P (H~ - theta) P x = -R_r, starting from x = 0
      FORTE_CUDA_TRY(cudaMemsetAsync(px, 0, sizeof(double) * N, st));
      if ((rc = vk_scale(ctx, pr, W + (size_t)r * N, -1.0, N))) return rc;
      if ((rc = vk_precond_inv(ctx, theta, ctx->dv_guard, pinv, N))) return rc;
      if ((rc = vk_precond_dot(ctx, pr, pinv, pz, d_s, N))) return rc;
      if ((rc = fetch(d_s, 1, h.data()))) return rc;
      double rz = h[0];
      if ((rc = project(pz, nroots))) return rc;
      FORTE_CUDA_TRY(cudaMemcpyAsync(pp, pz, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      const int max_inner = 25;
      for (int it = 0; it < max_inner; ++it) {
        if ((rc = sigma_dispatch(ctx, pp, pq, 1, inner_mode))) return rc;
        // in a spin-parity sector, drop the other sector's part of the reduced-precision
        // error: states there may lie below theta, where H - theta is not positive
        if ((rc = spin_project(ctx, pq, 1))) return rc;
        if ((rc = vk_axpby(ctx, -theta, pp, 1.0, pq, N))) return rc;
        if ((rc = project(pq, nroots))) return rc;
        if ((rc = vk_multidot(ctx, pp, 1, N, pq, N, d_s))) return rc;
        if ((rc = fetch(d_s, 1, h.data()))) return rc;
        const double pAp = h[0];
        if (!(pAp > 0.0) || !(rz > 0.0)) break;  // lost positive definiteness
        const double alpha = rz / pAp;
        if ((rc = vk_axpby(ctx, alpha, pp, 1.0, px, N))) return rc;
        if ((rc = vk_axpby(ctx, -alpha, pq, 1.0, pr, N))) return rc;
        // preconditioned residual, r . z and |r|^2 in one pass (z unused on exit)
        if ((rc = vk_precond_dot(ctx, pr, pinv, pz, d_s, N))) return rc;
        if ((rc = fetch(d_s, 2, h.data()))) return rc;
        if (sqrt(std::max(0.0, h[1])) < inner_rtol * bnorm) break;
        const double rz_new = h[0];
        if ((rc = project(pz, nroots))) return rc;
        const double beta = rz_new / rz;
        rz = rz_new;
        if ((rc = vk_axpby(ctx, 1.0, pz, beta, pp, N))) return rc;
      }
      // append the correction: orthonormalise against V[0..k)
      double *vk = V + (size_t)k * N;
      FORTE_CUDA_TRY(cudaMemcpyAsync(vk, px, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      if ((rc = spin_project(ctx, vk, 1))) return rc;
      if ((rc = vk_orth_update(ctx, V, k, N, nullptr, vk, vk, d_b, N))) return rc;
      if ((rc = fetch(d_b, k + 1, h.data()))) return rc;
      const double n0 = h[k];
      double proj = 0.0;
      for (int i = 0; i < k; ++i) proj += h[i] * h[i];
      if (!(n0 > 0.0) || !isfinite(n0)) continue;
      if (n0 - proj >= 0.5 * n0) {
        // one Gram-Schmidt pass suffices (as in davidson_run); normalised in the same
        // pass with |v - V c|^2 = |v|^2 - |c|^2
        if ((rc = vk_orth_update(ctx, V, k, N, d_b, vk, vk, d_a, N, false, 1.0 / sqrt(n0 - proj)))) return rc;
        ++k;
        continue;
      }
      if ((rc = vk_orth_update(ctx, V, k, N, d_b, vk, vk, d_a, N))) return rc;        // pass 1
      if ((rc = vk_orth_update(ctx, V, k, N, d_a, vk, vk, d_b, N, false))) return rc;  // pass 2
      if ((rc = fetch(d_b + k, 1, h.data()))) return rc;
      if (!(h[0] > 1e-24 * n0) || !(h[0] > 0.0)) continue;
      if ((rc = vk_scale(ctx, vk, vk, 1.0 / sqrt(h[0]), N))) return rc;
      ++k;
    }
    if (k == k0) {
      FORTE_CUDA_TRY(cudaMemcpyAsync(out, V, sizeof(double) * nroots * N, cudaMemcpyDeviceToDevice, st));
      return FORTE_OK;
    }
    if ((rc = sigma_dispatch(ctx, V + (size_t)k0 * N, HV + (size_t)k0 * N, k - k0, outer_mode))) return rc;
  }
}

}  // namespace forte

using namespace forte;

extern "C" {

const char *forte_last_error(void) { return g_err; }

static bool sym_ok(double a, double b) { return fabs(a - b) <= 1e-12 * std::max(1.0, fabs(a)); }

forte_ctx *forte_cas_create(int norb, int nalpha, int nbeta, const double *h, const double *eri) {
  clear_error();
  if (norb < 1 || norb > 16 || nalpha < 0 || nalpha > norb || nbeta < 0 || nbeta > norb) {
    set_error("invalid sizes: norb=%d nalpha=%d nbeta=%d (need 1<=norb<=16, 0<=n<=norb)", norb, nalpha, nbeta);
    return nullptr;
  }
  if (!h || !eri) {
    set_error("h and eri must be non-NULL host pointers");
    return nullptr;
  }
  const int n = norb;
  for (int i = 0; i < n * n; ++i)
    if (!isfinite(h[i])) { set_error("h contains NaN/Inf"); return nullptr; }
  for (long i = 0; i < (long)n * n * n * n; ++i)
    if (!isfinite(eri[i])) { set_error("eri contains NaN/Inf"); return nullptr; }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      if (!sym_ok(h[p * n + q], h[q * n + p])) { set_error("h is not symmetric at (%d,%d)", p, q); return nullptr; }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
          double v = eri[(((size_t)p * n + q) * n + r) * n + s];
          if (!sym_ok(v, eri[(((size_t)q * n + p) * n + r) * n + s]) ||
              !sym_ok(v, eri[(((size_t)p * n + q) * n + s) * n + r]) ||
              !sym_ok(v, eri[(((size_t)r * n + s) * n + p) * n + q])) {
            set_error("eri lacks 8-fold symmetry at (%d,%d|%d,%d)", p, q, r, s);
            return nullptr;
          }
        }
  forte_ctx *ctx = new (std::nothrow) forte_ctx();
  if (!ctx) { set_error("host allocation failed"); return nullptr; }
  ctx->n = n; ctx->na = nalpha; ctx->nb = nbeta;
  ctx->npair = n * (n + 1) / 2;
  ctx->same_strings = (nalpha == nbeta);
  ctx->h.assign(h, h + n * n);
  ctx->eri.assign(eri, eri + (size_t)n * n * n * n);
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    set_error("no CUDA device available");
    delete ctx;
    return nullptr;
  }
  int rc = build_spin_tables(ctx);
  if (!rc) {
    ctx->Na = ctx->sh[0].N;
    ctx->Nb = ctx->same_strings ? ctx->sh[0].N : ctx->sh[1].N;
    ctx->Ndet = ctx->Na * ctx->Nb;
    if (ctx->same_strings) ctx->sh[1] = ctx->sh[0];
    rc = upload_tables(ctx);
  }
  if (!rc) rc = hdiag_build(ctx);
  if (rc) {
    std::string msg = g_err;
    forte_destroy(ctx);
    set_error("%s", msg.c_str());
    return nullptr;
  }
  return ctx;
}

void forte_destroy(forte_ctx *ctx) {
  if (!ctx) return;
  int nsp = ctx->same_strings ? 1 : 2;
  for (int s = 0; s < nsp; ++s) {
    SpinDev &D = ctx->sd[s];
    cudaFree(D.list); cudaFree(D.csr_ptr); cudaFree(D.csr_col); cudaFree(D.csr_val);
    cudaFree(D.csr_val32); cudaFree(D.str); cudaFree(D.diag); cudaFree(D.dense); cudaFree(D.list4); cudaFree(D.tabJ);
  }
  cudaFree(ctx->d_gpair); cudaFree(ctx->d_gpair32); cudaFree(ctx->d_hdiag);
  cudaFree(ctx->d_roots); cudaFree(ctx->d_guess);
  cudaFree(ctx->d_gT_hi); cudaFree(ctx->d_gT_lo); cudaFree(ctx->d_gT_t32); cudaFree(ctx->d_err);
  cudaFree(ctx->d_ozT); cudaFree(ctx->d_g1tmp); cudaFree(ctx->d_gpair2);
  cudaFree(ctx->d_ozG); cudaFree(ctx->d_ozGa); cudaFree(ctx->d_ozTabT);
  cudaFree(ctx->d_abPosOf); cudaFree(ctx->d_abStrOf); cudaFree(ctx->d_abTab); cudaFree(ctx->d_abTabL);
  cudaFree(ctx->d_gTT_hi); cudaFree(ctx->d_gTT_lo); cudaFree(ctx->d_abDcnt); cudaFree(ctx->d_vk_count);
  cudaFree(ctx->d_csr_val2[0]);
  if (!ctx->same_strings) cudaFree(ctx->d_csr_val2[1]);
  for (int s = 0; s < (ctx->same_strings ? 1 : 2); ++s) {
    cudaFree(ctx->d_hd_hi[s]); cudaFree(ctx->d_hd_lo[s]); cudaFree(ctx->d_hd_t32[s]);
  }
  ctx->sc_t1.release(); ctx->sc_t2.release(); ctx->sc_dv.release();
  ctx->sc_small.release(); ctx->sc_rdm.release(); ctx->sc_mixed.release(); ctx->sc_grad.release(); ctx->sc_df.release();
  ctx->sc_rdm3.release(); ctx->sc_gas.release(); ctx->sc_spin.release(); ctx->sc_aci.release();
  gas_free(ctx);
  ctx->sc_oz.release();
  for (auto &r : ctx->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : ctx->prof_pool) cudaEventDestroy(e);
  delete ctx;
}

int forte_set_stream(forte_ctx *ctx, void *s) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  ctx->stream = (cudaStream_t)s;
  return FORTE_OK;
}

int forte_set_precision(forte_ctx *ctx, int mode) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (mode != FORTE_FP64 && mode != FORTE_TF32 && mode != FORTE_BF16X2 && mode != FORTE_DF32 &&
      mode != FORTE_OZ64) {
    set_error("unknown precision mode %d", mode);
    return FORTE_ERR_ARG;
  }
  ctx->precision = mode;
  return FORTE_OK;
}

int forte_get_sizes(const forte_ctx *ctx, long long *na, long long *nb) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (na) *na = ctx->Na;
  if (nb) *nb = ctx->Nb;
  return FORTE_OK;
}

int forte_get_string_tables(const forte_ctx *ctx, int spin, unsigned *strings, int *J, signed char *sgn) {
  if (!ctx || (spin != 0 && spin != 1)) { set_error("bad context or spin"); return FORTE_ERR_ARG; }
  const SpinHost &S = ctx->sh[spin];
  const int n = ctx->n, n2 = n * n;
  if (strings) for (long long i = 0; i < S.N; ++i) strings[i] = S.str[i];
  if (J) for (long long i = 0; i < S.N * n2; ++i) J[i] = -1;
  if (sgn) memset(sgn, 0, (size_t)S.N * n2);
  for (long long I = 0; I < S.N; ++I)
    for (int e = 0; e < S.nk; ++e) {
      const Repl &r = S.list[(size_t)I * S.nk + e];
      if (J) J[(size_t)I * n2 + r.pq] = r.J;
      if (sgn) sgn[(size_t)I * n2 + r.pq] = r.sgn;
    }
  return FORTE_OK;
}

int forte_get_hdiag(const forte_ctx *ctx, double *hd) {
  if (!ctx || !hd) { set_error("NULL argument"); return FORTE_ERR_ARG; }
  FORTE_CUDA_TRY(cudaMemcpyAsync(hd, ctx->d_hdiag, sizeof(double) * ctx->Ndet, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
  return FORTE_OK;
}

int forte_sigma(forte_ctx *ctx, const double *C, double *S, int nvec) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (nvec < 0) { set_error("nvec < 0"); return FORTE_ERR_ARG; }
  if (nvec == 0) return FORTE_OK;
  if (!C || !S) { set_error("C and S must be device pointers"); return FORTE_ERR_ARG; }
  const char *c0 = (const char *)C, *c1 = c0 + sizeof(double) * ctx->Ndet * nvec;
  const char *s0 = (const char *)S, *s1 = s0 + sizeof(double) * ctx->Ndet * nvec;
  if (c0 < s1 && s0 < c1) { set_error("S overlaps C"); return FORTE_ERR_ARG; }
  if (ctx->gas_on) {  // P H P C: the entries of C outside the kept space count as zero
    int rc = ctx->sc_gas.ensure(sizeof(double) * ctx->Ndet * nvec + 256);
    if (rc) return rc;
    double *Cp = (double *)ctx->sc_gas.ptr;
    FORTE_CUDA_TRY(cudaMemcpyAsync(Cp, C, sizeof(double) * ctx->Ndet * nvec, cudaMemcpyDeviceToDevice, ctx->stream));
    if ((rc = gas_mask(ctx, Cp, nvec))) return rc;
    return sigma_dispatch(ctx, Cp, S, nvec, ctx->precision);
  }
  return sigma_dispatch(ctx, C, S, nvec, ctx->precision);
}

int forte_set_davidson_params(forte_ctx *ctx, int max_sub, int collapse, int max_iter, double guard) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (max_sub < 2 || collapse < 1 || collapse >= max_sub || max_iter < 1 || !(guard > 0)) {
    set_error("invalid Davidson parameters");
    return FORTE_ERR_ARG;
  }
  ctx->dv_max_sub = max_sub;
  ctx->dv_collapse = collapse;
  ctx->dv_max_iter = max_iter;
  ctx->dv_guard = guard;
  return FORTE_OK;
}

int forte_set_guess(forte_ctx *ctx, const double *C, int nvec) {
  if (!ctx || nvec < 0 || (nvec > 0 && !C)) { set_error("bad guess arguments"); return FORTE_ERR_ARG; }
  cudaFree(ctx->d_guess);
  ctx->d_guess = nullptr;
  ctx->nguess = 0;
  if (nvec == 0) return FORTE_OK;
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_guess, sizeof(double) * ctx->Ndet * nvec));
  FORTE_CUDA_TRY(cudaMemcpyAsync(ctx->d_guess, C, sizeof(double) * ctx->Ndet * nvec, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
  ctx->nguess = nvec;
  int rc = gas_mask(ctx, ctx->d_guess, nvec);
  if (rc) return rc;
  return spin_project(ctx, ctx->d_guess, nvec);
}

static int ensure_roots(forte_ctx *ctx, int nroots) {
  size_t want = sizeof(double) * ctx->Ndet * nroots;
  if (want > ctx->d_roots_cap) {
    cudaFree(ctx->d_roots);
    ctx->d_roots = nullptr;
    ctx->d_roots_cap = 0;
    if (cudaMalloc(&ctx->d_roots, want) != cudaSuccess) {
      set_error("cudaMalloc roots failed");
      return FORTE_ERR_ALLOC;
    }
    ctx->d_roots_cap = want;
  }
  return FORTE_OK;
}

int forte_davidson(forte_ctx *ctx, int nroots, double tol) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (nroots < 1 || nroots > space_dim(ctx) || nroots > 31) { set_error("nroots out of range"); return FORTE_ERR_ARG; }
  if (!(tol > 0)) { set_error("tol must be > 0"); return FORTE_ERR_ARG; }
  clear_error();
  int rc = ensure_roots(ctx, nroots);
  if (rc) return rc;
  DvResult res;
  ctx->nroots_done = 0;
  if (ctx->precision == FORTE_FP64 || ctx->precision == FORTE_DF32 || ctx->precision == FORTE_OZ64) {
    rc = davidson_run<double>(ctx, nroots, tol, ctx->precision, ctx->d_guess, ctx->nguess, ctx->dv_max_iter,
                              ctx->d_roots, res);
    if (rc) return mixed_status(ctx) ? FORTE_ERR_TIMEOUT : rc;  // an expired wait explains the failure
    if ((rc = mixed_status(ctx))) return rc;
    ctx->dv_iters = res.iters;
    // A converged Davidson-Liu is verified: its residuals come from the stored basis
    // and sigma vectors, which a long run can leave inconsistent (lost
    // orthogonality).  The Jacobi-Davidson pass below starts by orthonormalising the
    // Ritz vectors, recomputing their sigma and forming the exact residuals; when
    // those meet tol it returns at once (one sigma per root), otherwise it iterates.
    // A stalled Davidson-Liu continues there the same way.
    if (res.converged || res.stalled) {
      // Jacobi-Davidson from the Ritz vectors, inner solves in the same arithmetic
      const int it_dl = res.iters;
      rc = refine_jd(ctx, nroots, tol, ctx->precision, ctx->precision, ctx->d_roots, ctx->d_roots,
                     std::max(1, std::min(60, ctx->dv_max_iter - it_dl)), res);
      if (rc) return mixed_status(ctx) ? FORTE_ERR_TIMEOUT : rc;
      if ((rc = mixed_status(ctx))) return rc;
      ctx->dv_iters = it_dl + res.iters;
    }
  } else {
    // Davidson with the reduced-precision sigma down to a residual the mixed
    // operator can still resolve, then FP64 Jacobi-Davidson refinement whose
    // inner solves use the mixed sigma
    // (measured: handing over at 1e-2 .. 3e-1 to a reduced-precision Jacobi-Davidson
    // stage first needs as many sigma applications and is no faster)
    double tol_in = std::max(tol, ctx->precision == FORTE_TF32 ? 1e-2 : 1e-3);
    rc = davidson_run<float>(ctx, nroots, tol_in, ctx->precision, ctx->d_guess, ctx->nguess, ctx->dv_max_iter,
                             ctx->d_roots, res);
    if (rc) return mixed_status(ctx) ? FORTE_ERR_TIMEOUT : rc;
    if ((rc = mixed_status(ctx))) return rc;
    int it_in = res.iters;
    // outer sigma: FP64-class, with the tensor-core alpha-beta term where it applies
    const int outer = oz_ab_supported(ctx) ? FORTE_OZ64 : FORTE_DF32;
    rc = refine_jd(ctx, nroots, tol, ctx->precision, outer, ctx->d_roots, ctx->d_roots, 30, res);
    if (rc) return mixed_status(ctx) ? FORTE_ERR_TIMEOUT : rc;
    if ((rc = mixed_status(ctx))) return rc;
    ctx->dv_iters = it_in + res.iters;
  }
  for (int r = 0; r < nroots; ++r)
    if ((rc = fix_sign(ctx, ctx->d_roots + (size_t)r * ctx->Ndet, ctx->Ndet))) return rc;
  ctx->roots_E = res.E;
  ctx->roots_rnorm = res.rn;
  ctx->nroots_done = nroots;
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (!res.converged) {
    set_error("Davidson did not converge in %d iterations (max residual %.3e)", ctx->dv_iters,
              *std::max_element(res.rn.begin(), res.rn.end()));
    return FORTE_ERR_NOT_CONVERGED;
  }
  return FORTE_OK;
}

int forte_get_roots(const forte_ctx *ctx, double *E, double *C, double *rnorm, int *iters) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (ctx->nroots_done == 0) { set_error("no Davidson results"); return FORTE_ERR_ARG; }
  if (E) for (int r = 0; r < ctx->nroots_done; ++r) E[r] = ctx->roots_E[r];
  if (rnorm) for (int r = 0; r < ctx->nroots_done; ++r) rnorm[r] = ctx->roots_rnorm[r];
  if (iters) *iters = ctx->dv_iters;
  if (C)
    FORTE_CUDA_TRY(cudaMemcpyAsync(C, ctx->d_roots, sizeof(double) * ctx->Ndet * ctx->nroots_done,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
  return FORTE_OK;
}

int forte_rdms(forte_ctx *ctx, const double *C, double *g1, double *g2) {
  if (!ctx || !C) { set_error("NULL argument"); return FORTE_ERR_ARG; }
  if (!g1 && !g2) return FORTE_OK;
  return rdm12_fp64(ctx, C, C, g1, g2);
}

int forte_tdm1(forte_ctx *ctx, const double *bra, const double *ket, double *t1) {
  if (!ctx || !bra || !ket || !t1) { set_error("NULL argument"); return FORTE_ERR_ARG; }
  return rdm12_fp64(ctx, bra, ket, t1, nullptr);
}

int forte_set_gas(forte_ctx *ctx, int nspace, const int *size, const int *gmin, const int *gmax,
                  long long *ndet_out) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  return gas_set(ctx, nspace, size, gmin, gmax, ndet_out);
}

int forte_set_gas_route(forte_ctx *ctx, int route) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (route < -1 || route > 1) { set_error("route must be -1, 0 or 1"); return FORTE_ERR_ARG; }
  ctx->gas_route = route;
  for (int t = 0; t < 2; ++t) ctx->gas_pick[t] = ctx->gas_pick_mode[t] = -1;
  return FORTE_OK;
}

int forte_get_gas_route(const forte_ctx *ctx, int *route_fp64, int *route_fp32, double *ms) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  const bool cand = ctx->gas_on && !ctx->detmask_on && ctx->d_gas_reach;
  for (int t = 0; t < 2; ++t) {
    int r = -1;
    if (!ctx->gas_on) r = -1;
    else if (!gas_sparse(ctx)) r = 0;
    else if (ctx->gas_route == 1) r = 1;
    else r = ctx->gas_pick[t];
    if (t == 0 && route_fp64) *route_fp64 = r;
    if (t == 1 && route_fp32) *route_fp32 = r;
    if (ms) {
      ms[2 * t] = cand ? ctx->gas_pick_ms[t][0] : 0.0;
      ms[2 * t + 1] = cand ? ctx->gas_pick_ms[t][1] : 0.0;
    }
  }
  return FORTE_OK;
}

int forte_aci(forte_ctx *ctx, double sigma, double gamma, int max_cycles, double tol, int parity, double *E_out,
              double *C_out, long long *nM_out, long long *nP_out, int *cycles_out) {
  if (!ctx || !E_out) { set_error("NULL argument"); return FORTE_ERR_ARG; }
  if (!(sigma >= 0) || !isfinite(sigma) || !(gamma >= 0) || !isfinite(gamma) || max_cycles < 1 || !(tol > 0)) {
    set_error("invalid adaptive CI parameters");
    return FORTE_ERR_ARG;
  }
  if (ctx->gas_on || ctx->spin_parity) {
    set_error("adaptive CI runs on the unrestricted determinant grid (no forte_set_gas / spin parity)");
    return FORTE_ERR_ARG;
  }
  if (parity != 0 && parity != 1 && parity != -1) { set_error("parity must be -1, 0 or +1"); return FORTE_ERR_ARG; }
  if (parity != 0 && ctx->na != ctx->nb) { set_error("a parity sector needs n_alpha == n_beta"); return FORTE_ERR_ARG; }
  return aci_run(ctx, sigma, gamma, max_cycles, tol, parity, E_out, C_out, nM_out, nP_out, cycles_out);
}

int forte_set_spin_parity(forte_ctx *ctx, int parity) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  return spin_set(ctx, parity);
}

int forte_rdm3(forte_ctx *ctx, const double *C, double *g3) {
  if (!ctx || !C || !g3) { set_error("NULL argument"); return FORTE_ERR_ARG; }
  return rdm3_fp64(ctx, C, g3);
}

int forte_sa_gradient(forte_ctx *ctx, int nstates, const double *weights, const double *C, double scale,
                      double *dh, double *deri) {
  if (!ctx || nstates < 1 || !weights || !C || !dh || !deri) { set_error("bad arguments"); return FORTE_ERR_ARG; }
  for (int k = 0; k < nstates; ++k)
    if (!isfinite(weights[k])) { set_error("non-finite weight"); return FORTE_ERR_ARG; }
  if (!isfinite(scale)) { set_error("non-finite scale"); return FORTE_ERR_ARG; }
  return sa_gradient(ctx, nstates, weights, C, scale, dh, deri);
}

int forte_sa_energy(const forte_ctx *ctx, int nstates, const double *weights, double *E_sa) {
  if (!ctx || !weights || !E_sa) { set_error("NULL argument"); return FORTE_ERR_ARG; }
  if (nstates < 1 || nstates > ctx->nroots_done) {
    set_error("nstates = %d but the last Davidson solve holds %d roots", nstates, ctx->nroots_done);
    return FORTE_ERR_ARG;
  }
  double e = 0.0;
  for (int k = 0; k < nstates; ++k) {
    if (!isfinite(weights[k])) { set_error("non-finite weight"); return FORTE_ERR_ARG; }
    e += weights[k] * ctx->roots_E[k];
  }
  *E_sa = e;
  return FORTE_OK;
}

int forte_set_wait_budget(forte_ctx *ctx, unsigned long long cycles) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  ctx->wait_budget = cycles;
  return err_word_setup(ctx);
}

int forte_get_status(forte_ctx *ctx) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  FORTE_CUDA_TRY(cudaGetLastError());
  return mixed_status(ctx);
}

int forte_get_counters(const forte_ctx *ctx, long long *fp64, long long *mixed) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (fp64) *fp64 = ctx->n_sigma_fp64;
  if (mixed) *mixed = ctx->n_sigma_mixed;
  return FORTE_OK;
}

int forte_profile_enable(forte_ctx *ctx, int on) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (on) {
    FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (auto &r : ctx->prof) {
      ctx->prof_pool.push_back(r.a);
      ctx->prof_pool.push_back(r.b);
    }
    ctx->prof.clear();
  }
  ctx->prof_on = (on != 0);
  return FORTE_OK;
}

int forte_profile_query(forte_ctx *ctx, const char *kernel, int *launches, double *total_ms) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  int cnt = 0;
  double tot = 0.0;
  for (auto &r : ctx->prof) {
    if (kernel && strcmp(kernel, r.name) != 0) continue;
    float ms = 0.f;
    FORTE_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
    ++cnt;
    tot += ms;
  }
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = tot;
  return FORTE_OK;
}

const char *forte_profile_kernel_name(forte_ctx *ctx, int i) {
  if (!ctx || i < 0) return nullptr;
  std::vector<const char *> seen;
  for (auto &r : ctx->prof) {
    bool dup = false;
    for (auto *s : seen) dup |= (strcmp(s, r.name) == 0);
    if (!dup) seen.push_back(r.name);
  }
  return i < (int)seen.size() ? seen[i] : nullptr;
}

}  // extern "C"
