// Adaptive configuration interaction (Sec. II.A.2) on the determinant grid of
// the CAS.  One cycle:
//   1. Psi_P, E_P: Davidson in the reference space P (determinant mask);
//   2. V = H Psi_P over the whole grid: one FP64-class sigma gives
//      <Phi_mu|H|Psi_P> for every determinant of the first-order interacting
//      space at once;
//   3. eps_mu = D/2 - sqrt(D^2/4 + V_mu^2), D = H_mumu - E_P: the lowest root of
//      the 2 x 2 problem [[E_P, V], [V, H_mumu]] minus E_P;
//   4. exclusion: the determinants with the smallest |eps| leave while their
//      summed |eps| stays at most sigma (equal values leave together);
//   5. Psi_M, E_M: Davidson in M = all determinants not excluded;
//   6. next P: the largest-c^2 determinants of M whose weights reach
//      1 - gamma sigma (equal values stay together).
// Stops when P repeats.  With a parity sector (n_alpha = n_beta) the P and M
// solves keep C^T = parity C, which picks the target spin parity and makes Psi_P
// unique where the two sectors' lowest states are (nearly) degenerate.  For n_alpha = n_beta the alpha <-> beta exchange
// commutes with H: mirror determinants carry equal |eps| and c^2 in exact
// arithmetic, so both take the larger computed value (rounding must not split
// a mirror pair at a threshold), and the start P is the lowest determinant with
// its mirror.  Steps 4 and 6 are threshold searches over the 64-bit
// patterns of non-negative doubles (monotone as unsigned integers): eight
// 256-bin histogram passes (count and sum per bin) narrow the threshold one
// byte at a time, the host walking the bins between passes.
#include <algorithm>
#include <vector>

#include "forte_internal.h"

namespace forte {

__global__ void k_aci_eps(const double *__restrict__ V, const double *__restrict__ hd,
                          const uint8_t *__restrict__ inP, double EP, long long N, double *__restrict__ a,
                          double *__restrict__ eps) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    if (inP[i]) {
      a[i] = (double)INFINITY;
      eps[i] = 0.0;
    } else {
      const double D = 0.5 * (hd[i] - EP);
      const double e = D - sqrt(D * D + V[i] * V[i]);
      eps[i] = e;
      a[i] = fabs(e);
    }
  }
}

// Per-bin count and sum of the entries whose key agrees with `prefix` above bit
// shift + 8 (all entries for shift = 56); bin = byte of the key at `shift`.
__global__ void k_aci_hist(const double *__restrict__ a, long long N, int shift, unsigned long long prefix,
                           unsigned long long *__restrict__ cnt, double *__restrict__ sum) {
  __shared__ double ss[256];
  __shared__ unsigned int sc[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) { ss[i] = 0.0; sc[i] = 0u; }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double v = a[i];
    const unsigned long long k = (unsigned long long)__double_as_longlong(v);
    if (shift < 56 && (k >> (shift + 8)) != prefix) continue;
    const int b = (int)((k >> shift) & 255ull);
    atomicAdd(&ss[b], v);
    atomicAdd(&sc[b], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (sc[i]) {
      atomicAdd(&sum[i], ss[i]);
      atomicAdd(&cnt[i], (unsigned long long)sc[i]);
    }
}

// maskM[i] = key(a[i]) >= kM; counts the kept entries (and those with I_a == I_b
// when N1 > 0, the side of a square grid) and sums the excluded eps
__global__ void k_aci_mask_m(const double *__restrict__ a, const double *__restrict__ eps, long long N, long long N1,
                             unsigned long long kM, uint8_t *__restrict__ maskM, unsigned long long *__restrict__ nM,
                             double *__restrict__ eps_excl) {
  unsigned long long c = 0, cd = 0;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const bool keep = (unsigned long long)__double_as_longlong(a[i]) >= kM;
    maskM[i] = keep;
    if (keep) {
      ++c;
      if (N1 > 0 && i / N1 == i % N1) ++cd;
    } else {
      s += eps[i];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    cd += __shfl_xor_sync(0xffffffffu, cd, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(nM, c);
    atomicAdd(nM + 2, cd);
    atomicAdd(eps_excl, s);
  }
}

// x[i][i] = v on a square grid of side N1
__global__ void k_aci_diag_fill(double *__restrict__ x, long long N1, double v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N1; i += (long long)gridDim.x * blockDim.x)
    x[i * N1 + i] = v;
}

// y[ia][ib] = max(x[ia][ib], x[ib][ia]) on a square grid
__global__ void k_aci_mirror_max(const double *__restrict__ x, long long N1, double *__restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N1 * N1;
       i += (long long)gridDim.x * blockDim.x) {
    const long long ia = i / N1, ib = i % N1;
    y[i] = fmax(x[i], x[ib * N1 + ia]);
  }
}

__global__ void k_aci_c2(const double *__restrict__ C, const uint8_t *__restrict__ maskM, long long N,
                         double *__restrict__ c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    c2[i] = maskM[i] ? C[i] * C[i] : 0.0;
}

__device__ __forceinline__ unsigned long long aci_mix(unsigned long long x) {  // splitmix64 output function
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Second Davidson guess next to the previous state: entries u - 1/2, u uniform in
// [0, 1) from splitmix64 (i + cycle key).  A state of definite spin symmetry
// alone keeps the subspace inside its own symmetry sector, whose lowest root need
// not be the ground state; this vector has weight in every sector.
__global__ void k_aci_pert(double *__restrict__ x, long long N, unsigned long long key) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    x[i] = (double)(aci_mix((unsigned long long)i + key) >> 11) * 0x1.0p-53 - 0.5;
}

// maskP[i] = maskM[i] && (all || key(c2[i]) >= kP); count, an order-free hash of
// the set and (N1 > 0) the count of entries with I_a == I_b; nP[0..2] = count, hash, diagonal
__global__ void k_aci_mask_p(const double *__restrict__ c2, const uint8_t *__restrict__ maskM, long long N,
                             long long N1, unsigned long long kP, int all, uint8_t *__restrict__ maskP,
                             unsigned long long *__restrict__ nP) {
  unsigned long long c = 0, h = 0, cd = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const bool keep = maskM[i] && (all || (unsigned long long)__double_as_longlong(c2[i]) >= kP);
    maskP[i] = keep;
    if (keep) {
      ++c;
      h += aci_mix((unsigned long long)i);
      if (N1 > 0 && i / N1 == i % N1) ++cd;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    h += __shfl_xor_sync(0xffffffffu, h, o);
    cd += __shfl_xor_sync(0xffffffffu, cd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(nP, c);
    atomicAdd(nP + 1, h);
    atomicAdd(nP + 2, cd);
  }
}

namespace {

struct AciWork {
  double *hd, *V, *a, *eps, *psi;
  uint8_t *mP, *mM, *mPn;
  unsigned long long *cnt;  // [256] + 4 counters
  double *sum;              // [256] + 1
};

unsigned grid_for(long long N) { return (unsigned)std::min<long long>((N + 255) / 256, 152LL * 8); }

// Ascending (asc): key of the first value whose inclusion lifts the running sum
// of the sorted values above `limit`.  Descending: key of the first value (from
// the top) at which the running sum reaches `limit`.  found = false when no
// value does.
int radix_walk(forte_ctx *ctx, const double *a, long long N, double limit, bool asc, AciWork &w,
               unsigned long long *key, bool *found) {
  cudaStream_t st = ctx->stream;
  unsigned long long prefix = 0;
  double base = 0.0;
  std::vector<unsigned long long> hc(256);
  std::vector<double> hs(256);
  for (int shift = 56; shift >= 0; shift -= 8) {
    FORTE_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned long long) * 256, st));
    FORTE_CUDA_TRY(cudaMemsetAsync(w.sum, 0, sizeof(double) * 256, st));
    {
      FORTE_PROF(ctx, "aci_hist");
      k_aci_hist<<<grid_for(N), 256, 0, st>>>(a, N, shift, prefix, w.cnt, w.sum);
      FORTE_LAUNCH_CHECK();
    }
    FORTE_CUDA_TRY(cudaMemcpyAsync(hc.data(), w.cnt, sizeof(unsigned long long) * 256, cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaMemcpyAsync(hs.data(), w.sum, sizeof(double) * 256, cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaStreamSynchronize(st));
    int b1 = -1;
    double cum = base;
    for (int k = 0; k < 256; ++k) {
      const int b = asc ? k : 255 - k;
      if (!hc[b]) continue;
      if (asc ? (cum + hs[b] > limit) : (cum + hs[b] >= limit)) {
        b1 = b;
        break;
      }
      cum += hs[b];
    }
    if (b1 < 0) {
      *found = false;
      return FORTE_OK;
    }
    base = cum;
    prefix = (prefix << 8) | (unsigned long long)b1;
  }
  *key = prefix;
  *found = true;
  return FORTE_OK;
}

}  // namespace

static int aci_body(forte_ctx *ctx, double sigma, double gamma, int max_cycles, double tol, int parity,
                    double *E_out, double *C_out, long long *nM_out, long long *nP_out, int *cycles_out,
                    const double **hd_saved) {
  cudaStream_t st = ctx->stream;
  const long long N = ctx->Ndet;
  const size_t vd = ((sizeof(double) * N + 255) / 256) * 256, vb = ((size_t)N + 255) / 256 * 256;
  const size_t v2 = ((sizeof(double) * 2 * N + 255) / 256) * 256;  // psi and the perturbation, stride N
  int rc = ctx->sc_aci.ensure(4 * vd + v2 + 3 * vb + sizeof(unsigned long long) * 260 + sizeof(double) * 257 + 256);
  if (rc) return rc;
  char *p = (char *)ctx->sc_aci.ptr;
  AciWork w;
  w.hd = (double *)p; p += vd;
  w.V = (double *)p; p += vd;
  w.a = (double *)p; p += vd;
  w.eps = (double *)p; p += vd;
  w.psi = (double *)p; p += v2;
  w.mP = (uint8_t *)p; p += vb;
  w.mM = (uint8_t *)p; p += vb;
  w.mPn = (uint8_t *)p; p += vb;
  w.cnt = (unsigned long long *)p; p += sizeof(unsigned long long) * 260;
  w.sum = (double *)p;
  unsigned long long *d_n = w.cnt + 256;  // [0] count, [1] hash, [2] diagonal count
  double *d_es = w.sum + 256;

  // the unrestricted diagonal, kept while the masks change d_hdiag
  if ((rc = hdiag_build(ctx))) return rc;
  FORTE_CUDA_TRY(cudaMemcpyAsync(w.hd, ctx->d_hdiag, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  *hd_saved = w.hd;
  auto uninstall = [&]() {
    ctx->detmask_on = false;
    ctx->d_detmask = nullptr;
    ctx->detmask_n = 0;
    ctx->detmask_ndiag = 0;
    ctx->spin_parity = 0;
    cudaMemcpyAsync(ctx->d_hdiag, w.hd, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    forte_set_guess(ctx, nullptr, 0);
    ctx->nroots_done = 0;
  };
  auto install = [&](uint8_t *mask, long long cnt, long long ndiag) -> int {
    ctx->d_detmask = mask;
    ctx->detmask_n = cnt;
    ctx->detmask_ndiag = ndiag;
    ctx->detmask_on = true;
    FORTE_CUDA_TRY(cudaMemcpyAsync(ctx->d_hdiag, w.hd, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    return det_mask_fill(ctx, ctx->d_hdiag, 1, (double)INFINITY);
  };
  unsigned long long pert_key = 0x2545F4914F6CDD1Dull;
  auto solve = [&](uint8_t *mask, long long cnt, long long ndiag, bool guess, double *E) -> int {
    int r;
    if ((r = install(mask, cnt, ndiag))) return r;
    if (guess) {  // [previous state, perturbation]; both projected onto the space
      pert_key += 0x9E3779B97F4A7C15ull;
      k_aci_pert<<<grid_for(N), 256, 0, st>>>(w.psi + N, N, pert_key);
      FORTE_LAUNCH_CHECK();
    }
    if ((r = forte_set_guess(ctx, guess ? w.psi : nullptr, guess ? (cnt > 1 ? 2 : 1) : 0))) return r;
    if ((r = forte_davidson(ctx, 1, tol))) return r;
    *E = ctx->roots_E[0];
    return FORTE_OK;
  };
  auto fail = [&](int r) {
    uninstall();
    return r;
  };

  const bool mirror = ctx->same_strings;  // n_alpha == n_beta: square grid, mirror pairs
  auto mirror_max = [&](const double *x, double *y) -> int {
    FORTE_PROF(ctx, "aci_mirror");
    k_aci_mirror_max<<<grid_for(N), 256, 0, st>>>(x, ctx->Na, y);
    FORTE_LAUNCH_CHECK();
    return FORTE_OK;
  };
  // the start determinant: lowest diagonal (outside I_a == I_b for the odd sector)
  long long i0 = 0;
  const double *hstart = w.hd;
  if (parity < 0) {
    FORTE_CUDA_TRY(cudaMemcpyAsync(w.V, w.hd, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    k_aci_diag_fill<<<grid_for(ctx->Na), 256, 0, st>>>(w.V, ctx->Na, (double)INFINITY);
    FORTE_LAUNCH_CHECK();
    hstart = w.V;
  }
  if ((rc = vk_argmin_k(ctx, hstart, N, 1, &i0))) return rc;
  FORTE_CUDA_TRY(cudaMemsetAsync(w.mP, 0, (size_t)N, st));
  const uint8_t one = 1;
  FORTE_CUDA_TRY(cudaMemcpyAsync(w.mP + i0, &one, 1, cudaMemcpyHostToDevice, st));
  long long nP = 1, nM = 0, nPd = 0, nMd = 0;
  if (mirror) {
    const long long i1 = (i0 % ctx->Nb) * ctx->Nb + i0 / ctx->Nb;
    if (i1 != i0) {
      FORTE_CUDA_TRY(cudaMemcpyAsync(w.mP + i1, &one, 1, cudaMemcpyHostToDevice, st));
      nP = 2;
    } else {
      nPd = 1;
    }
  }
  const long long N1 = mirror ? ctx->Na : 0;
  ctx->spin_parity = parity;  // the P / M solves run in the sector; reset by uninstall()
  bool have_psi = false;
  std::vector<std::pair<long long, unsigned long long>> seen;
  double E_M = 0.0, eps_excl = 0.0;
  for (int cycle = 1;; ++cycle) {
    double E_P;
    if ((rc = solve(w.mP, nP, nPd, have_psi, &E_P))) return fail(rc);
    // V = H Psi_P over the grid, estimates, exclusion
    if ((rc = sigma_grid(ctx, ctx->d_roots, w.V, 1))) return fail(rc);
    {
      FORTE_PROF(ctx, "aci_eps");
      k_aci_eps<<<grid_for(N), 256, 0, st>>>(w.V, w.hd, w.mP, E_P, N, w.a, w.eps);
      FORTE_LAUNCH_CHECK();
    }
    double *aa = w.a;
    if (mirror) {
      if ((rc = mirror_max(w.a, w.V))) return fail(rc);
      aa = w.V;
    }
    unsigned long long kM = 0;
    bool fM = false;
    if ((rc = radix_walk(ctx, aa, N, sigma, true, w, &kM, &fM))) return fail(rc);
    if (!fM) kM = 0x7FF0000000000000ull;  // every finite estimate is excluded
    FORTE_CUDA_TRY(cudaMemsetAsync(d_n, 0, sizeof(unsigned long long) * 3, st));
    FORTE_CUDA_TRY(cudaMemsetAsync(d_es, 0, sizeof(double), st));
    {
      FORTE_PROF(ctx, "aci_mask");
      k_aci_mask_m<<<grid_for(N), 256, 0, st>>>(aa, w.eps, N, N1, kM, w.mM, d_n, d_es);
      FORTE_LAUNCH_CHECK();
    }
    unsigned long long hn[3];
    FORTE_CUDA_TRY(cudaMemcpyAsync(hn, d_n, sizeof(hn), cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaMemcpyAsync(&eps_excl, d_es, sizeof(double), cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaStreamSynchronize(st));
    nM = (long long)hn[0];
    nMd = (long long)hn[2];
    // Psi_M (started from Psi_P)
    FORTE_CUDA_TRY(cudaMemcpyAsync(w.psi, ctx->d_roots, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    if ((rc = solve(w.mM, nM, nMd, true, &E_M))) return fail(rc);
    FORTE_CUDA_TRY(cudaMemcpyAsync(w.psi, ctx->d_roots, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    // next reference space
    {
      FORTE_PROF(ctx, "aci_c2");
      k_aci_c2<<<grid_for(N), 256, 0, st>>>(w.psi, w.mM, N, w.a);
      FORTE_LAUNCH_CHECK();
    }
    double *c2 = w.a;
    if (mirror) {
      if ((rc = mirror_max(w.a, w.V))) return fail(rc);
      c2 = w.V;
    }
    unsigned long long kP = 0;
    bool fP = false;
    if ((rc = radix_walk(ctx, c2, N, 1.0 - gamma * sigma, false, w, &kP, &fP))) return fail(rc);
    FORTE_CUDA_TRY(cudaMemsetAsync(d_n, 0, sizeof(unsigned long long) * 3, st));
    {
      FORTE_PROF(ctx, "aci_mask");
      k_aci_mask_p<<<grid_for(N), 256, 0, st>>>(c2, w.mM, N, N1, kP, fP ? 0 : 1, w.mPn, d_n);
      FORTE_LAUNCH_CHECK();
    }
    unsigned long long hv[3];
    FORTE_CUDA_TRY(cudaMemcpyAsync(hv, d_n, sizeof(hv), cudaMemcpyDeviceToHost, st));
    FORTE_CUDA_TRY(cudaStreamSynchronize(st));
    const std::pair<long long, unsigned long long> key((long long)hv[0], hv[1]);
    nP = (long long)hv[0];
    nPd = (long long)hv[2];
    std::swap(w.mP, w.mPn);
    have_psi = true;
    if (std::find(seen.begin(), seen.end(), key) != seen.end() || cycle >= max_cycles) {
      E_out[0] = E_M;
      E_out[1] = E_M + eps_excl;
      if (C_out)
        FORTE_CUDA_TRY(cudaMemcpyAsync(C_out, w.psi, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      if (nM_out) *nM_out = nM;
      if (nP_out) *nP_out = nP;
      if (cycles_out) *cycles_out = cycle;
      uninstall();
      FORTE_CUDA_TRY(cudaStreamSynchronize(st));
      return FORTE_OK;
    }
    seen.push_back(key);
  }
}

int aci_run(forte_ctx *ctx, double sigma, double gamma, int max_cycles, double tol, int parity, double *E_out,
            double *C_out, long long *nM_out, long long *nP_out, int *cycles_out) {
  const double *hd = nullptr;
  const int rc = aci_body(ctx, sigma, gamma, max_cycles, tol, parity, E_out, C_out, nM_out, nP_out, cycles_out, &hd);
  // on every exit, also the early ones: the context is unrestricted again
  ctx->detmask_on = false;
  ctx->d_detmask = nullptr;
  ctx->detmask_n = 0;
  ctx->detmask_ndiag = 0;
  ctx->spin_parity = 0;
  ctx->nroots_done = 0;
  if (hd) cudaMemcpyAsync(ctx->d_hdiag, hd, sizeof(double) * ctx->Ndet, cudaMemcpyDeviceToDevice, ctx->stream);
  forte_set_guess(ctx, nullptr, 0);
  cudaStreamSynchronize(ctx->stream);
  return rc;
}

}  // namespace forte
