// Occupation-restricted CI (GAS / RAS), Sec. II.A.1: the active orbitals are
// split into consecutive spaces A_1 .. A_G and a determinant |Ia>|Ib> is kept
// when gmin[g] <= n_alpha(A_g) + n_beta(A_g) <= gmax[g] for every g.  The
// restriction is applied, as in the paper, at the level of the strings (each
// string's per-space occupation is its class) and of the allowed combinations
// of string classes (a small table ok[class_a][class_b]).
//
// The restricted Hamiltonian is P H P.  Vectors keep the [N_alpha][N_beta]
// layout of the full space, zero outside the kept determinants, and the diagonal
// is +inf there, so that guesses and preconditioned corrections stay inside the
// restricted space.  When at most a quarter of the determinants is kept, sigma is
// formed over the kept determinants only (k_gas_sigma: each output from its
// same-spin Hamiltonian rows and its alpha-beta replacement pairs, skipping the
// source determinants of excluded class pairs), so its cost follows the kept
// space; otherwise the full-grid kernels run and a pass zeroes the excluded
// entries (write-only: it reads the class table and stores a zero where a
// determinant is excluded).
#include <algorithm>
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

constexpr int GAS_THREADS = 256;

// P H P C for the kept determinants of the kept alpha row Ia = rows[blockIdx.x]
// (vector blockIdx.y), every other entry of S left as it is (zero).
//  (1) alpha-beta, driven by the source beta strings: for each beta class cb whose
//      strings carry weight (some J_k of the row, k in L(Ia), has an allowed
//      (class(J_k), cb) pair: elsewhere C is zero) and reach an allowed output
//      class, tiles of TJ strings Jb of that class are gathered as
//      D[k][j] = C[J_k][Jb_j] for the allowed k only, and every replacement
//      E_rs Jb = s I_b with an allowed output adds
//      s * sum_k s_k (pq_k|rs) D[k][j] to the row accumulator (shared memory);
//  (2) per kept output: the accumulator plus the same-spin CSR terms
//      sum_Ja H_aa[Ia][Ja] C[Ja][Ib] + sum_Jb H_bb[Ib][Jb] C[Ia][Jb].
// Each (output, replacement pair) of Eq. 1's two-body alpha-beta part is formed
// once, and only where both its source and its output are kept.  T: FP64, or FP32
// for the FP32 vectors of the reduced-precision phase.
template <typename T>
__global__ void __launch_bounds__(GAS_THREADS) k_gas_sigma(
    const T *__restrict__ C, T *__restrict__ S, long long NB, long long vstride,
    const Repl *__restrict__ listA, int nkA, const Repl *__restrict__ listB, int nkB,
    const int *__restrict__ ptrA, const int *__restrict__ colA, const T *__restrict__ valA,
    const int *__restrict__ ptrB, const int *__restrict__ colB, const T *__restrict__ valB,
    const T *__restrict__ gpair, int npair, const int *__restrict__ clsA, const int *__restrict__ clsB,
    const uint8_t *__restrict__ ok, int ncB, const unsigned long long *__restrict__ reachB,
    const int *__restrict__ rows, const int *__restrict__ boff, const int *__restrict__ blist,
    const int *__restrict__ coff, const int *__restrict__ cstr, int TJ) {
  extern __shared__ __align__(16) uint8_t gsm[];
  const int Ia = rows[blockIdx.x];
  const int rb = ptrA[Ia], nnz = ptrA[Ia + 1] - rb;
  T *Gs = (T *)gsm;                                         // [nkA][npair] signed integral rows
  T *srow = Gs + (size_t)nkA * npair;                       // [NB] alpha-beta accumulator
  T *D = srow + NB;                                         // [nkA][TJ] gathered C rows
  T *sval = D + (size_t)nkA * TJ;                           // [nnz] CSR row Ia of H_aa
  Repl *Lb = (Repl *)(((uintptr_t)(sval + nnz) + 7) & ~(uintptr_t)7);  // [TJ][nkB]
  int *scol = (int *)(Lb + (size_t)TJ * nkB);               // [nnz]
  int *sJ = scol + nnz;                                     // [nkA]
  int *kcnt = sJ + nkA;                                     // [ncB]
  uint16_t *klist = (uint16_t *)(kcnt + ncB);               // [ncB][nkA]: k * npair of the allowed k
  uint8_t *sclsB = (uint8_t *)(klist + (size_t)ncB * nkA);  // [NB] beta classes
  const Repl *la = listA + (long long)Ia * nkA;
  const int ca = clsA[Ia];
  const uint8_t *okA = ok + (size_t)ca * ncB;
  for (int i = threadIdx.x; i < nkA * npair; i += GAS_THREADS) {
    const int e = i / npair, rs = i % npair;
    const Repl r = la[e];
    const T g = gpair[(size_t)r.pair * npair + rs];
    Gs[i] = r.sgn < 0 ? -g : g;
  }
  for (long long i = threadIdx.x; i < NB; i += GAS_THREADS) {
    srow[i] = T(0);
    sclsB[i] = (uint8_t)clsB[i];
  }
  for (int i = threadIdx.x; i < nnz; i += GAS_THREADS) {
    sval[i] = valA[rb + i];
    scol[i] = colA[rb + i];
  }
  for (int e = threadIdx.x; e < nkA; e += GAS_THREADS) sJ[e] = la[e].J;
  // allowed k per source beta class (ascending k: deterministic sums)
  for (int cb = threadIdx.x; cb < ncB; cb += GAS_THREADS) {
    int m = 0;
    for (int e = 0; e < nkA; ++e)
      if (ok[(size_t)clsA[la[e].J] * ncB + cb]) klist[(size_t)cb * nkA + m++] = (uint16_t)(e * npair);
    kcnt[cb] = m;
  }
  unsigned long long okmask = 0ull;
  for (int b = 0; b < ncB; ++b)
    if (okA[b]) okmask |= 1ull << b;
  __syncthreads();
  const T *Cv = C + (long long)blockIdx.y * vstride;
  T *Sv = S + (long long)blockIdx.y * vstride;
  for (int cb = 0; cb < ncB; ++cb) {
    const int kc = kcnt[cb];
    if (kc == 0 || !(reachB[cb] & okmask)) continue;
    const uint16_t *kl = klist + (size_t)cb * nkA;
    for (int s0 = coff[cb]; s0 < coff[cb + 1]; s0 += TJ) {
      const int tj = min(TJ, coff[cb + 1] - s0);
      __syncthreads();
      for (int i = threadIdx.x; i < kc * tj; i += GAS_THREADS) {
        const int kk = i / tj, j = i % tj;
        D[kk * TJ + j] = Cv[(long long)sJ[kl[kk] / npair] * NB + cstr[s0 + j]];
      }
      for (int i = threadIdx.x; i < tj * nkB; i += GAS_THREADS)
        Lb[i] = listB[(long long)cstr[s0 + i / nkB] * nkB + i % nkB];
      __syncthreads();
      for (int w = threadIdx.x; w < tj * nkB; w += GAS_THREADS) {
        const Repl rf = Lb[w];
        if (!((okmask >> sclsB[rf.J]) & 1ull)) continue;
        const int j = w / nkB;
        const T *g = Gs + rf.pair;
        const T *d = D + j;
        T acc = T(0);
        for (int kk = 0; kk < kc; ++kk) acc += g[kl[kk]] * d[kk * TJ];
        atomicAdd(&srow[rf.J], rf.sgn < 0 ? -acc : acc);
      }
    }
  }
  __syncthreads();
  for (int b = boff[ca] + threadIdx.x; b < boff[ca + 1]; b += GAS_THREADS) {
    const long long Ib = blist[b];
    T acc = srow[Ib];
    for (int e = 0; e < nnz; ++e) acc += sval[e] * Cv[(long long)scol[e] * NB + Ib];
    for (int f = ptrB[Ib]; f < ptrB[Ib + 1]; ++f) acc += valB[f] * Cv[(long long)Ia * NB + colB[f]];
    Sv[(long long)Ia * NB + Ib] = acc;
  }
}

static size_t gas_smem_bytes(size_t tsz, int nkA, int nkB, int npair, long long NB, int maxnnz, int ncB, int TJ) {
  return tsz * ((size_t)nkA * npair + NB + (size_t)nkA * TJ + maxnnz) + 8 + sizeof(Repl) * (size_t)TJ * nkB +
         sizeof(int) * ((size_t)maxnnz + nkA + ncB) + sizeof(uint16_t) * (size_t)ncB * nkA + NB + 16;
}

bool gas_sparse(const forte_ctx *ctx) {
  if (!ctx->gas_on || ctx->detmask_on || !ctx->d_gas_rows || !ctx->d_gas_reach || ctx->gas_route == 0) return false;
  return ctx->gas_route == 1 || 4 * ctx->gas_ndet <= ctx->Ndet;
}

template <typename T>
static int gas_sigma_t(forte_ctx *ctx, const T *C, T *S, int nvec) {
  if (nvec <= 0) return FORTE_OK;
  cudaStream_t st = ctx->stream;
  FORTE_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(T) * ctx->Ndet * nvec, st));
  if (ctx->gas_nrows == 0) return FORTE_OK;
  const int nkA = ctx->sh[0].nk, nkB = ctx->sh[1].nk, np = ctx->npair, ncB = ctx->gas_nc[1];
  // the widest source tile that keeps two blocks per SM, else one
  int TJ = 64;
  size_t smem = gas_smem_bytes(sizeof(T), nkA, nkB, np, ctx->Nb, ctx->gas_maxnnz, ncB, TJ);
  while (TJ > 16 && smem > 113 * 1024) {
    TJ /= 2;
    smem = gas_smem_bytes(sizeof(T), nkA, nkB, np, ctx->Nb, ctx->gas_maxnnz, ncB, TJ);
  }
  while (TJ > 8 && smem > 220 * 1024) {
    TJ /= 2;
    smem = gas_smem_bytes(sizeof(T), nkA, nkB, np, ctx->Nb, ctx->gas_maxnnz, ncB, TJ);
  }
  if (smem > 220 * 1024) {
    set_error("restricted sigma needs %zu bytes of shared memory", smem);
    return FORTE_ERR_ARG;
  }
  FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_gas_sigma<T>));
  const bool f32 = sizeof(T) == 4;
  const T *valA = f32 ? (const T *)(const void *)ctx->sd[0].csr_val32 : (const T *)(const void *)ctx->sd[0].csr_val;
  const T *valB = f32 ? (const T *)(const void *)ctx->sd[1].csr_val32 : (const T *)(const void *)ctx->sd[1].csr_val;
  const T *gp = f32 ? (const T *)(const void *)ctx->d_gpair32 : (const T *)(const void *)ctx->d_gpair;
  dim3 grid((unsigned)ctx->gas_nrows, (unsigned)nvec);
  FORTE_PROF(ctx, f32 ? "gas_sigma_f32" : "gas_sigma");
  k_gas_sigma<T><<<grid, GAS_THREADS, smem, st>>>(
      C, S, ctx->Nb, ctx->Ndet, ctx->sd[0].list, nkA, ctx->sd[1].list, nkB, ctx->sd[0].csr_ptr, ctx->sd[0].csr_col,
      valA, ctx->sd[1].csr_ptr, ctx->sd[1].csr_col, valB, gp, np, ctx->d_gas_cls[0], ctx->d_gas_cls[1],
      ctx->d_gas_ok, ncB, ctx->d_gas_reach, ctx->d_gas_rows, ctx->d_gas_boff, ctx->d_gas_blist, ctx->d_gas_coff,
      ctx->d_gas_cstr, TJ);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}
int gas_sigma(forte_ctx *ctx, const double *C, double *S, int nvec) { return gas_sigma_t(ctx, C, S, nvec); }
int gas_sigma(forte_ctx *ctx, const float *C, float *S, int nvec) { return gas_sigma_t(ctx, C, S, nvec); }

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
  cudaFree(ctx->d_gas_rows);
  cudaFree(ctx->d_gas_boff);
  cudaFree(ctx->d_gas_blist);
  cudaFree(ctx->d_gas_coff);
  cudaFree(ctx->d_gas_cstr);
  cudaFree(ctx->d_gas_reach);
  ctx->d_gas_rows = ctx->d_gas_boff = ctx->d_gas_blist = ctx->d_gas_coff = ctx->d_gas_cstr = nullptr;
  ctx->d_gas_reach = nullptr;
  ctx->gas_nrows = 0;
  for (int t = 0; t < 2; ++t) ctx->gas_pick[t] = ctx->gas_pick_mode[t] = -1;
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
  // lists of the restricted sigma: kept alpha rows; per alpha class the beta strings
  // of its allowed classes (ascending)
  {
    std::vector<int> rowsv, boff(ncA + 1, 0), blist;
    for (int a = 0; a < ncA; ++a) {
      for (long long j = 0; j < ctx->sh[1].N; ++j)
        if (ok[(size_t)a * ncB + cls[1][j]]) blist.push_back((int)j);
      boff[a + 1] = (int)blist.size();
    }
    for (long long i = 0; i < ctx->sh[0].N; ++i)
      if (boff[cls[0][i] + 1] > boff[cls[0][i]]) rowsv.push_back((int)i);
    int maxnnz = 0;
    for (long long i = 0; i < ctx->sh[0].N; ++i)
      maxnnz = std::max(maxnnz, ctx->sh[0].csr_ptr[i + 1] - ctx->sh[0].csr_ptr[i]);
    if (blist.empty()) blist.push_back(0);
    if (cudaMalloc(&ctx->d_gas_rows, sizeof(int) * std::max<size_t>(1, rowsv.size())) != cudaSuccess ||
        cudaMalloc(&ctx->d_gas_boff, sizeof(int) * boff.size()) != cudaSuccess ||
        cudaMalloc(&ctx->d_gas_blist, sizeof(int) * blist.size()) != cudaSuccess) {
      gas_release(ctx);
      set_error("cudaMalloc of the restricted-sigma lists failed");
      return FORTE_ERR_ALLOC;
    }
    if (!rowsv.empty())
      FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_rows, rowsv.data(), sizeof(int) * rowsv.size(), cudaMemcpyHostToDevice));
    FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_boff, boff.data(), sizeof(int) * boff.size(), cudaMemcpyHostToDevice));
    FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_blist, blist.data(), sizeof(int) * blist.size(), cudaMemcpyHostToDevice));
    ctx->gas_nrows = (long long)rowsv.size();
    ctx->gas_maxnnz = maxnnz;
  }
  // per beta class its strings (ascending) and the classes its replacements reach
  // (bit masks: the kept-only sigma needs at most 64 beta classes)
  if (ncB <= 64) {
    const SpinHost &B = ctx->sh[1];
    std::vector<int> coff(ncB + 1, 0), cstr;
    for (int b = 0; b < ncB; ++b) {
      for (long long j = 0; j < B.N; ++j)
        if (cls[1][j] == b) cstr.push_back((int)j);
      coff[b + 1] = (int)cstr.size();
    }
    std::vector<unsigned long long> reach(ncB, 0ull);
    for (long long j = 0; j < B.N; ++j)
      for (int m = 0; m < B.nk; ++m) reach[cls[1][j]] |= 1ull << cls[1][B.list[(size_t)j * B.nk + m].J];
    if (cudaMalloc(&ctx->d_gas_coff, sizeof(int) * coff.size()) != cudaSuccess ||
        cudaMalloc(&ctx->d_gas_cstr, sizeof(int) * std::max<size_t>(1, cstr.size())) != cudaSuccess ||
        cudaMalloc(&ctx->d_gas_reach, sizeof(unsigned long long) * reach.size()) != cudaSuccess) {
      gas_release(ctx);
      set_error("cudaMalloc of the restricted-sigma class lists failed");
      return FORTE_ERR_ALLOC;
    }
    FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_coff, coff.data(), sizeof(int) * coff.size(), cudaMemcpyHostToDevice));
    FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_cstr, cstr.data(), sizeof(int) * cstr.size(), cudaMemcpyHostToDevice));
    FORTE_CUDA_TRY(cudaMemcpy(ctx->d_gas_reach, reach.data(), sizeof(unsigned long long) * reach.size(),
                              cudaMemcpyHostToDevice));
  }
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
