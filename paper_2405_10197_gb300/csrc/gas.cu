// Occupation-restricted CI (GAS / RAS), Sec. II.A.1: the active orbitals are
// split into consecutive spaces A_1 .. A_G and a determinant |Ia>|Ib> is kept
// when gmin[g] <= n_alpha(A_g) + n_beta(A_g) <= gmax[g] for every g.  The
// restriction is applied, as in the paper, at the level of the strings (each
// string's per-space occupation is its class) and of the allowed combinations
// of string classes (a small table ok[class_a][class_b]).
//
// The restricted Hamiltonian is P H P.  Vectors keep the [N_alpha][N_beta]
// layout of the full space, zero outside the kept determinants: every sigma is
// followed by a pass that zeroes the excluded entries (write-only: it reads the
// class table and stores a zero where a determinant is excluded), and the
// diagonal is +inf there, so that guesses and preconditioned corrections stay
// inside the restricted space.  The sigma kernels still sweep the full product
// space.
#include <map>
#include <vector>

#include "forte_internal.h"

namespace forte {

// x[row][ib] = value wherever ok[clsA[ia]][clsB[ib]] == 0, rows = nvec * NA
// (ia = row % NA).  One block per row in a grid-stride loop, threads along ib.
template <typename T>
__global__ void k_gas_fill(T *__restrict__ x, long long rows, long long NA, long long NB,
                           const int *__restrict__ clsA, const int *__restrict__ clsB,
                           const uint8_t *__restrict__ ok, int ncB, T value) {
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const uint8_t *okr = ok + (long long)clsA[row % NA] * ncB;
    T *xr = x + row * NB;
    for (long long ib = threadIdx.x; ib < NB; ib += blockDim.x)
      if (!okr[clsB[ib]]) xr[ib] = value;
  }
}

// x[v][i] = value wherever mask[i] == 0 (an arbitrary determinant mask).
template <typename T>
__global__ void k_det_fill(T *__restrict__ x, long long total, long long nd, const uint8_t *__restrict__ mask,
                           T value) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    if (!mask[i % nd]) x[i] = value;
}

template <typename T>
static int gas_fill(forte_ctx *ctx, T *x, int nvec, T value) {
  if (nvec <= 0) return FORTE_OK;
  if (ctx->detmask_on) {
    const long long total = (long long)nvec * ctx->Ndet;
    const unsigned nb = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 16);
    FORTE_PROF(ctx, "det_mask");
    k_det_fill<T><<<nb, 256, 0, ctx->stream>>>(x, total, ctx->Ndet, ctx->d_detmask, value);
    FORTE_LAUNCH_CHECK();
  }
  if (!ctx->gas_on) return FORTE_OK;
  const long long rows = (long long)nvec * ctx->Na;
  const unsigned nb = (unsigned)std::min<long long>(rows, 152LL * 16);
  const int nt = ctx->Nb >= 256 ? 256 : (ctx->Nb >= 64 ? 64 : 32);
  FORTE_PROF(ctx, "gas_mask");
  k_gas_fill<T><<<nb, nt, 0, ctx->stream>>>(x, rows, ctx->Na, ctx->Nb, ctx->d_gas_cls[0], ctx->d_gas_cls[1],
                                            ctx->d_gas_ok, ctx->gas_nc[1], value);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

int gas_mask(forte_ctx *ctx, double *x, int nvec) { return gas_fill<double>(ctx, x, nvec, 0.0); }
int gas_mask(forte_ctx *ctx, float *x, int nvec) { return gas_fill<float>(ctx, x, nvec, 0.0f); }

int det_mask_fill(forte_ctx *ctx, double *x, int nvec, double value) { return gas_fill<double>(ctx, x, nvec, value); }

long long space_dim(const forte_ctx *ctx) {
  if (ctx->detmask_on) {  // (no occupation restriction besides it; the mask is mirror-closed with a sector)
    if (ctx->spin_parity == 0) return ctx->detmask_n;
    const long long D = ctx->detmask_ndiag;
    return (ctx->detmask_n - D) / 2 + (ctx->spin_parity > 0 ? D : 0);
  }
  const long long K = ctx->gas_on ? ctx->gas_ndet : ctx->Ndet;
  if (ctx->spin_parity == 0) return K;
  // the kept set is symmetric under I_alpha <-> I_beta: mirror pairs plus the diagonal
  const long long D = ctx->gas_on ? ctx->gas_ndiag : ctx->Na;
  return (K - D) / 2 + (ctx->spin_parity > 0 ? D : 0);
}

static void gas_release(forte_ctx *ctx) {
  for (int s = 0; s < 2; ++s) {
    cudaFree(ctx->d_gas_cls[s]);
    ctx->d_gas_cls[s] = nullptr;
    ctx->gas_nc[s] = 0;
  }
  cudaFree(ctx->d_gas_ok);
  ctx->d_gas_ok = nullptr;
  ctx->gas_on = false;
  ctx->gas_ndet = 0;
  ctx->gas_ndiag = 0;
}

void gas_free(forte_ctx *ctx) { gas_release(ctx); }

int gas_set(forte_ctx *ctx, int nspace, const int *size, const int *gmin, const int *gmax, long long *ndet_out) {
  const int n = ctx->n;
  if (nspace < 0 || nspace > n) { set_error("nspace must be in [0, norb]"); return FORTE_ERR_ARG; }
  if (nspace > 0 && (!size || !gmin || !gmax)) { set_error("NULL space arrays"); return FORTE_ERR_ARG; }
  int tot = 0;
  for (int g = 0; g < nspace; ++g) {
    if (size[g] < 1) { set_error("space %d is empty", g); return FORTE_ERR_ARG; }
    if (gmin[g] < 0 || gmax[g] < gmin[g]) { set_error("space %d: need 0 <= gmin <= gmax", g); return FORTE_ERR_ARG; }
    tot += size[g];
  }
  if (nspace > 0 && tot != n) { set_error("space sizes add up to %d, not norb = %d", tot, n); return FORTE_ERR_ARG; }

  // classes of the strings of each spin: their per-space occupation vectors
  std::vector<int> cls[2];
  std::vector<std::vector<int>> occ[2];
  std::vector<long long> cnt[2];
  for (int s = 0; s < 2 && nspace > 0; ++s) {
    const SpinHost &H = ctx->sh[s];
    std::map<std::vector<int>, int> id;
    cls[s].resize(H.N);
    for (long long i = 0; i < H.N; ++i) {
      std::vector<int> o(nspace, 0);
      int orb = 0;
      for (int g = 0; g < nspace; ++g)
        for (int k = 0; k < size[g]; ++k, ++orb) o[g] += (int)((H.str[i] >> orb) & 1u);
      auto it = id.find(o);
      if (it == id.end()) {
        it = id.emplace(o, (int)occ[s].size()).first;
        occ[s].push_back(o);
        cnt[s].push_back(0);
      }
      cls[s][i] = it->second;
      ++cnt[s][it->second];
    }
  }
  const int ncA = (int)occ[0].size(), ncB = (int)occ[1].size();
  std::vector<uint8_t> ok((size_t)ncA * ncB, 0);
  long long ndet = 0;
  for (int a = 0; a < ncA; ++a)
    for (int b = 0; b < ncB; ++b) {
      bool keep = true;
      for (int g = 0; g < nspace; ++g) {
        const int e = occ[0][a][g] + occ[1][b][g];
        keep = keep && e >= gmin[g] && e <= gmax[g];
      }
      ok[(size_t)a * ncB + b] = keep;
      if (keep) ndet += cnt[0][a] * cnt[1][b];
    }
  if (nspace > 0 && ndet == 0) { set_error("the occupation restriction keeps no determinant"); return FORTE_ERR_ARG; }
  long long ndiag = 0;  // determinants |I>|I> (same string sets only)
  if (nspace > 0 && ctx->same_strings)
    for (size_t i = 0; i < cls[0].size(); ++i) ndiag += ok[(size_t)cls[0][i] * ncB + cls[1][i]];

  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  gas_release(ctx);
  int rc = hdiag_build(ctx);  // the unrestricted diagonal; excluded entries are set below
  if (rc) return rc;
  if (nspace == 0) {
    if (ndet_out) *ndet_out = ctx->Ndet;
    return FORTE_OK;
  }
  for (int s = 0; s < 2; ++s) {
    if (cudaMalloc(&ctx->d_gas_cls[s], sizeof(int) * cls[s].size()) != cudaSuccess) {
      gas_release(ctx);
      set_error("cudaMalloc of the string classes failed");
      return FORTE_ERR_ALLOC;
    }
    FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_cls[s], cls[s].data(), sizeof(int) * cls[s].size(), cudaMemcpyHostToDevice));
  }
  if (cudaMalloc(&ctx->d_gas_ok, ok.size()) != cudaSuccess) {
    gas_release(ctx);
    set_error("cudaMalloc of the class table failed");
    return FORTE_ERR_ALLOC;
  }
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_ok, ok.data(), ok.size(), cudaMemcpyHostToDevice));
  ctx->gas_nc[0] = ncA;
  ctx->gas_nc[1] = ncB;
  ctx->gas_ndet = ndet;
  ctx->gas_ndiag = ndiag;
  ctx->gas_on = true;
  if ((rc = gas_fill<double>(ctx, ctx->d_hdiag, 1, (double)INFINITY))) return rc;
  if (ctx->nguess > 0 && (rc = gas_mask(ctx, ctx->d_guess, ctx->nguess))) return rc;
  ctx->nroots_done = 0;  // earlier roots belong to another space
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (ndet_out) *ndet_out = ndet;
  return FORTE_OK;
}

}  // namespace forte
