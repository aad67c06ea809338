// Spin-parity sectors for Ms = 0 (Sec. II.A.1: projection of the CI expansion
// on states of well-defined total spin).  For n_alpha = n_beta, exchanging the
// alpha and beta strings, C[Ia][Ib] -> C[Ib][Ia], commutes with the spin-free
// Hamiltonian; with alpha creators ordered first, a state of total spin S has
// C[Ib][Ia] = (-1)^S C[Ia][Ib].  Davidson restricted to the sector
// C^T = parity C finds only even-S (parity +1) or only odd-S (parity -1) roots.
//
// The projection x <- (x + parity x^T) / 2 is applied to the guesses and to
// every new correction vector; linear combinations of exactly symmetric (or
// antisymmetric) vectors stay exactly so, since every element and its mirror
// go through the same operations.
#include "forte_internal.h"

namespace forte {

constexpr int SP_T = 32;

// One 32 x 32 tile pair (ti, tj), ti <= tj, of vector blockIdx.z: both tiles
// are read before either is written, so the diagonal tiles work in place.
template <typename T>
__global__ void __launch_bounds__(256) k_spin_proj(T *__restrict__ x, long long N, float parity) {
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  __shared__ T A[SP_T][SP_T + 1], B[SP_T][SP_T + 1];
  T *v = x + (long long)blockIdx.z * N * N;
  const long long r0 = (long long)ti * SP_T, c0 = (long long)tj * SP_T;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < SP_T; i += blockDim.y) {
    const long long r = r0 + i, c = c0 + tx;
    if (r < N && c < N) A[i][tx] = v[r * N + c];  // A[i][j] = x[r0+i][c0+j]
    const long long r2 = c0 + i, c2 = r0 + tx;
    if (r2 < N && c2 < N) B[i][tx] = v[r2 * N + c2];  // B[i][j] = x[c0+i][r0+j]
  }
  __syncthreads();
  const T p = (T)parity, h = (T)0.5;
  for (int i = ty; i < SP_T; i += blockDim.y) {
    const long long r = r0 + i, c = c0 + tx;
    if (r < N && c < N) v[r * N + c] = h * (A[i][tx] + p * B[tx][i]);
    if (ti != tj) {
      const long long r2 = c0 + i, c2 = r0 + tx;
      if (r2 < N && c2 < N) v[r2 * N + c2] = h * (B[i][tx] + p * A[tx][i]);
    }
  }
}

template <typename T>
static int spin_proj_t(forte_ctx *ctx, T *x, int nvec) {
  if (ctx->spin_parity == 0 || nvec <= 0) return FORTE_OK;
  const long long N = ctx->Na;
  const unsigned nt = (unsigned)((N + SP_T - 1) / SP_T);
  FORTE_PROF(ctx, "spin_proj");
  k_spin_proj<T><<<dim3(nt, nt, (unsigned)nvec), dim3(SP_T, 8), 0, ctx->stream>>>(x, N, (float)ctx->spin_parity);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

int spin_project(forte_ctx *ctx, double *x, int nvec) { return spin_proj_t<double>(ctx, x, nvec); }
int spin_project(forte_ctx *ctx, float *x, int nvec) { return spin_proj_t<float>(ctx, x, nvec); }

// hd_out[ia][ib] = hdiag, or +inf where (ia, ib) is not the representative of
// its mirror pair (ia > ib) or cannot carry weight in the sector (ia == ib for
// parity -1): the lowest entries then name distinct sector guesses.
__global__ void k_spin_guess_diag(const double *__restrict__ hd, long long N, int parity, double *__restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N * N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long ia = i / N, ib = i % N;
    out[i] = (ia > ib || (ia == ib && parity < 0)) ? (double)INFINITY : hd[i];
  }
}

int spin_guess_diag(forte_ctx *ctx, const double **hd) {
  const long long N = ctx->Na;
  int rc = ctx->sc_spin.ensure(sizeof(double) * N * N + 256);
  if (rc) return rc;
  double *out = (double *)ctx->sc_spin.ptr;
  const unsigned nb = (unsigned)std::min<long long>((N * N + 255) / 256, 152LL * 16);
  {
    FORTE_PROF(ctx, "spin_guess_diag");
    k_spin_guess_diag<<<nb, 256, 0, ctx->stream>>>(ctx->d_hdiag, N, ctx->spin_parity, out);
    FORTE_LAUNCH_CHECK();
  }
  *hd = out;
  return FORTE_OK;
}

int spin_set(forte_ctx *ctx, int parity) {
  if (parity != 0 && parity != 1 && parity != -1) { set_error("parity must be -1, 0 or +1"); return FORTE_ERR_ARG; }
  if (parity != 0 && ctx->na != ctx->nb) {
    set_error("spin-parity sectors need n_alpha == n_beta (Ms = 0)");
    return FORTE_ERR_ARG;
  }
  ctx->spin_parity = parity;
  ctx->nroots_done = 0;  // earlier roots belong to another space
  int rc = spin_project(ctx, ctx->d_guess, ctx->nguess);
  if (rc) return rc;
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return FORTE_OK;
}

}  // namespace forte
