// Spin-free 1- and 2-RDMs (step a9), Sec. II.A.1 Eqs. (gamma_1), (gamma_2)
// summed over spin:
//   gamma_pq   = <bra| E_pq |ket>
//   Gamma_pqrs = <bra| E_pq E_rs |ket> - d_qr gamma_ps = <E_qp bra | E_rs ket> - d_qr gamma_ps
// The 2-RDM is a Gram matrix of the one-body images D^{rs} = E_rs |ket>
// (alpha and beta parts added), taken over all determinants.
#include <algorithm>

#include "forte_internal.h"

namespace forte {

__device__ __forceinline__ double warp_sum_r(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// part[row][pq] = sum_{e in L(row), pq_e = pq} s_e * <bra[J_e,:], ket[row,:]>
// (rows of one spin; the other spin's strings run along the columns).
__global__ void k_g1_part(const Repl *__restrict__ list, int nk, const double *__restrict__ bra,
                          const double *__restrict__ ket, long long ncol, int n2,
                          double *__restrict__ part) {
  __shared__ double acc[256];
  __shared__ double red[32];
  const long long row = blockIdx.x;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const double *kr = ket + row * ncol;
  for (int e = 0; e < nk; ++e) {
    Repl r = list[row * nk + e];
    const double *br = bra + (long long)r.J * ncol;
    double s = 0.0;
    for (long long c = threadIdx.x; c < ncol; c += blockDim.x) s += br[c] * kr[c];
    s = warp_sum_r(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      acc[r.pq] += r.sgn * t;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n2; i += blockDim.x) part[row * n2 + i] = acc[i];
}

// out[j] = sum_b part[b][j] + sum_b part2[b][j]   (grid.x = n2)
__global__ void k_sum_cols2(const double *__restrict__ part, long long nb1, const double *__restrict__ part2,
                            long long nb2, int m, double *__restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long b = threadIdx.x; b < nb1; b += blockDim.x) s += part[b * m + blockIdx.x];
  for (long long b = threadIdx.x; b < nb2; b += blockDim.x) s += part2[b * m + blockIdx.x];
  s = warp_sum_r(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

template <typename T>
__global__ void k_transpose_r(const T *__restrict__ X, T *__restrict__ Y, long long R, long long Cc) {
  __shared__ T tile[32][33];
  long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    long long r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Cc) tile[i][threadIdx.x] = X[r * Cc + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    long long c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < Cc) Y[c * R + r] = tile[threadIdx.x][i];
  }
}

// D[rs][Ia][Ib] = (E_rs ket)[Ia,Ib]
//   = sgn_a * ket[Ja, Ib]  (E_sr Ia = sgn_a Ja)  +  sgn_b * ket[Ia, Jb]  (E_sr Ib = sgn_b Jb)
__global__ void k_build_D(const int *__restrict__ denseA, const int *__restrict__ denseB, int n,
                          const double *__restrict__ ket, long long NA, long long NB,
                          double *__restrict__ D) {
  const long long nd = NA * NB;
  const int n2 = n * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nd;
       i += (long long)gridDim.x * blockDim.x) {
    const long long ia = i / NB, ib = i % NB;
    const int *ta = denseA + ia * n2;
    const int *tb = denseB + ib * n2;
    for (int r = 0; r < n; ++r)
      for (int s = 0; s < n; ++s) {
        double v = 0.0;
        int x = ta[s * n + r];
        if (x >= 0) v += ((x & 1) ? -1.0 : 1.0) * ket[(long long)(x >> 1) * NB + ib];
        int y = tb[s * n + r];
        if (y >= 0) v += ((y & 1) ? -1.0 : 1.0) * ket[ia * NB + (y >> 1)];
        D[(long long)(r * n + s) * nd + i] = v;
      }
  }
}

constexpr int GT = 64;   // Gram tile
constexpr int GK = 32;   // K slab

// part[split][a][b] = sum_{k in split's range} X[a][k] Y[b][k]; m x m output in GT tiles.
// With sym (X == Y) only the tiles ta <= tb are formed (grid.x = ntile(ntile+1)/2).
__global__ void __launch_bounds__(256) k_gram(const double *__restrict__ X, const double *__restrict__ Y,
                                              int m, long long K, long long kper, int sym,
                                              double *__restrict__ part) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int ntile = (m + GT - 1) / GT;
  int ta = blockIdx.x / ntile, tb = blockIdx.x % ntile;
  if (sym) {
    int rem = blockIdx.x;
    ta = 0;
    while (rem >= ntile - ta) {
      rem -= ntile - ta;
      ++ta;
    }
    tb = ta + rem;
  }
  const int a0 = ta * GT, b0 = tb * GT;
  const long long k0 = (long long)blockIdx.y * kper, k1 = min(K, k0 + kper);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (long long kk = k0; kk < k1; kk += GK) {
    __syncthreads();
    for (int i = threadIdx.x; i < GT * GK; i += 256) {
      int r = i / GK, c = i % GK;
      long long k = kk + c;
      As[c][r] = (a0 + r < m && k < k1) ? X[(long long)(a0 + r) * K + k] : 0.0;
      Bs[c][r] = (b0 + r < m && k < k1) ? Y[(long long)(b0 + r) * K + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < GK; ++c) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[c][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[c][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
  }
  double *P = part + (long long)blockIdx.y * m * m;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int a = a0 + ty * 4 + i, b = b0 + tx * 4 + j;
      if (a < m && b < m) P[(long long)a * m + b] = acc[i][j];
    }
}

// g2[p][q][r][s] = sum_split part[split][(q,p)][(r,s)] - d_qr g1[p][s]
__global__ void k_finish_g2(const double *__restrict__ part, int nsplit, int n, int sym,
                            const double *__restrict__ g1, double *__restrict__ g2) {
  const int m = n * n;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * m) return;
  int p = i / (n * n * n), q = (i / (n * n)) % n, r = (i / n) % n, s = i % n;
  int a = q * n + p, b = r * n + s;
  if (sym && a / GT > b / GT) {  // only tiles ta <= tb were formed; the Gram is symmetric
    const int t = a;
    a = b;
    b = t;
  }
  long long idx = (long long)a * m + b;
  double v = 0.0;
  for (int t = 0; t < nsplit; ++t) v += part[(long long)t * m * m + idx];
  if (q == r) v -= g1[p * n + s];
  g2[i] = v;
}

// Gamma3[p][q][r][s][t][u] for one (t,u):
//   sum_split part[split][(q,p)][(r,s)] - d_qt G2_purs - d_st G2_pqru - d_qr (G2_pstu + d_st g1_pu)
// where part holds <E_qp C | E_rs E_tu C> (normal ordering of E_pq E_rs E_tu, Sec. II.A.1).
__global__ void k_finish_g3(const double *__restrict__ part, int nsplit, int n, int t, int u,
                            const double *__restrict__ g1, const double *__restrict__ g2,
                            double *__restrict__ g3) {
  const int m = n * n;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * m) return;
  int p = i / (n * n * n), q = (i / (n * n)) % n, r = (i / n) % n, s = i % n;
  long long idx = (long long)(q * n + p) * m + (r * n + s);
  double v = 0.0;
  for (int k = 0; k < nsplit; ++k) v += part[(long long)k * m * m + idx];
  if (q == t) v -= g2[((p * n + u) * n + r) * n + s];
  if (s == t) v -= g2[((p * n + q) * n + r) * n + u];
  if (q == r) {
    v -= g2[((p * n + s) * n + t) * n + u];
    if (s == t) v -= g1[p * n + u];
  }
  g3[(long long)i * m + t * n + u] = v;
}

// Adjoint of the state-averaged energy E_SA = sum_k w_k E_k (Sec. II.B):
// dh += c1 gamma^k, deri += c2 Gamma^k for one state (c1 = scale w_k, c2 = scale w_k / 2).
__global__ void k_sa_accum(const double *__restrict__ g1, const double *__restrict__ g2, int n, double c1,
                           double c2, double *__restrict__ dh, double *__restrict__ deri) {
  const int n2 = n * n, n4 = n2 * n2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
    deri[i] += c2 * g2[i];
    if (i < n2) dh[i] += c1 * g1[i];
  }
}

int sa_gradient(forte_ctx *ctx, int nstates, const double *weights, const double *C, double scale, double *dh,
                double *deri) {
  const int n = ctx->n, n2 = n * n;
  int rc = ctx->sc_grad.ensure(sizeof(double) * ((size_t)n2 + (size_t)n2 * n2) + 256);
  if (rc) return rc;
  double *g1 = (double *)ctx->sc_grad.ptr, *g2 = g1 + n2;
  for (int k = 0; k < nstates; ++k) {
    const double *ck = C + (size_t)k * ctx->Ndet;
    if ((rc = rdm12_fp64(ctx, ck, ck, g1, g2))) return rc;
    const double c1 = scale * weights[k], c2 = 0.5 * scale * weights[k];
    {
      FORTE_PROF(ctx, "sa_accum");
      k_sa_accum<<<(unsigned)std::min(1024, (n2 * n2 + 255) / 256), 256, 0, ctx->stream>>>(g1, g2, n, c1, c2, dh,
                                                                                          deri);
      FORTE_LAUNCH_CHECK();
    }
  }
  return FORTE_OK;
}

int rdm12_fp64(forte_ctx *ctx, const double *bra, const double *ket, double *g1, double *g2, bool tensor_ok) {
  cudaStream_t st = ctx->stream;
  const int n = ctx->n, n2 = n * n;
  const long long NA = ctx->Na, NB = ctx->Nb, ND = ctx->Ndet;
  // workspace: transposes of bra/ket, g1 partials, g1 (when the caller passed none)
  size_t off_T = 0;
  size_t sz_T = sizeof(double) * ND * 2;
  size_t off_P = off_T + sz_T;
  size_t sz_P = sizeof(double) * (size_t)(NA + NB) * n2;
  size_t off_g1 = off_P + sz_P;
  size_t sz_g1 = sizeof(double) * n2;
  size_t base_bytes = off_g1 + sz_g1 + 256;
  // 2-RDM: D for ket (and bra when different), Gram partials; the reduced-precision
  // modes take the tensor-core Gram (rdm_oz.cu) for bra == ket
  const bool same = (bra == ket);
  const bool oz = tensor_ok && g2 && same && ctx->precision != FORTE_FP64 && rdm2_oz_supported(ctx);
  const int nsplit = 64;
  size_t off_D = (base_bytes + 255) & ~(size_t)255;
  size_t sz_D = (g2 && !oz) ? sizeof(double) * (size_t)n2 * ND * (same ? 1 : 2) : 0;
  size_t off_G = off_D + sz_D;
  size_t sz_G = (g2 && !oz) ? sizeof(double) * (size_t)nsplit * n2 * n2 : 0;
  int rc = ctx->sc_rdm.ensure(off_G + sz_G + 256);
  if (rc) return rc;
  char *w = (char *)ctx->sc_rdm.ptr;
  double *Tb = (double *)(w + off_T), *Tk = Tb + ND;
  double *P = (double *)(w + off_P);
  double *g1w = g1 ? g1 : (double *)(w + off_g1);
  if (oz && !g1) {  // the Gram step reallocates sc_rdm: keep the 1-RDM elsewhere
    if (!ctx->d_g1tmp) FORTE_CUDA_TRY(cudaMalloc(&ctx->d_g1tmp, sizeof(double) * n2));
    g1w = ctx->d_g1tmp;
  }

  // gamma: alpha rows, then beta rows on the transposed vectors
  {
    FORTE_PROF(ctx, "g1_part");
    k_g1_part<<<(unsigned)NA, 256, 0, st>>>(ctx->sd[0].list, ctx->sh[0].nk, bra, ket, NB, n2, P);
  FORTE_LAUNCH_CHECK();
  }
  dim3 tb(32, 8), tg((unsigned)((NB + 31) / 32), (unsigned)((NA + 31) / 32));
  {
    FORTE_PROF(ctx, "transpose_r");
    k_transpose_r<double><<<tg, tb, 0, st>>>(ket, Tk, NA, NB);
  FORTE_LAUNCH_CHECK();
  }
  const double *TbraP = Tk;
  if (!same) {
    {
      FORTE_PROF(ctx, "transpose_r");
      k_transpose_r<double><<<tg, tb, 0, st>>>(bra, Tb, NA, NB);
    FORTE_LAUNCH_CHECK();
    }
    TbraP = Tb;
  }
  const int nkB = ctx->sh[ctx->same_strings ? 0 : 1].nk;
  {
    FORTE_PROF(ctx, "g1_part");
    k_g1_part<<<(unsigned)NB, 256, 0, st>>>(ctx->sd[1].list, nkB, TbraP, Tk, NA, n2, P + NA * n2);
  FORTE_LAUNCH_CHECK();
  }
  {
    FORTE_PROF(ctx, "sum_cols2");
    k_sum_cols2<<<n2, 256, 0, st>>>(P, NA, P + NA * n2, NB, n2, g1w);
  FORTE_LAUNCH_CHECK();
  }
  if (!g2) return FORTE_OK;
  if (oz) {
    if ((rc = rdm2_oz(ctx, ket, g1w, g2))) return rc;
    return mixed_status(ctx);  // bounded waits of the tensor-core kernel (synchronises the stream)
  }

  double *Dk = (double *)(w + off_D);
  double *Db = same ? Dk : Dk + (size_t)n2 * ND;
  unsigned nbD = (unsigned)std::min<long long>((ND + 255) / 256, 152LL * 32);
  {
    FORTE_PROF(ctx, "build_D");
    k_build_D<<<nbD, 256, 0, st>>>(ctx->sd[0].dense, ctx->sd[1].dense, n, ket, NA, NB, Dk);
  FORTE_LAUNCH_CHECK();
  }
  if (!same) {
    {
      FORTE_PROF(ctx, "build_D");
      k_build_D<<<nbD, 256, 0, st>>>(ctx->sd[0].dense, ctx->sd[1].dense, n, bra, NA, NB, Db);
    FORTE_LAUNCH_CHECK();
    }
  }
  double *G = (double *)(w + off_G);
  const int ntile = (n2 + GT - 1) / GT;
  long long kper = (ND + nsplit - 1) / nsplit;
  const int sym = same ? 1 : 0;
  dim3 gg(sym ? ntile * (ntile + 1) / 2 : ntile * ntile, nsplit);
  // M[a][b] = <D_bra^a, D_ket^b>, where D_bra^{qp} = E_qp bra
  {
    FORTE_PROF(ctx, "gram");
    k_gram<<<gg, 256, 0, st>>>(Db, Dk, n2, ND, kper, sym, G);
  FORTE_LAUNCH_CHECK();
  }
  {
    FORTE_PROF(ctx, "finish_g2");
    k_finish_g2<<<(n2 * n2 + 255) / 256, 256, 0, st>>>(G, nsplit, n, sym, g1w, g2);
  FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

// Spin-free 3-RDM of one state (Sec. II.A.1, gamma_3 summed over spin), FP64:
//   <E_pq E_rs E_tu> = <E_qp C | E_rs F^{tu}>,  F^{tu} = E_tu C = D^{tu},
// so for each (t,u) the one-body images of F^{tu} are built and contracted with
// D by the Gram kernel; the lower-rank terms of the normal ordering are then
// taken off with the FP64 1- and 2-RDMs.  Cost n^2 (build_D + n^4 ND Gram).
int rdm3_fp64(forte_ctx *ctx, const double *C, double *g3) {
  cudaStream_t st = ctx->stream;
  const int n = ctx->n, n2 = n * n;
  const long long NA = ctx->Na, NB = ctx->Nb, ND = ctx->Ndet;
  const int nsplit = (int)std::min<long long>(64, std::max<long long>(1, ND / 256));
  const size_t sz_g1 = sizeof(double) * n2, sz_g2 = sizeof(double) * n2 * n2;
  const size_t sz_D = sizeof(double) * (size_t)n2 * ND;
  const size_t off_g2 = (sz_g1 + 255) & ~(size_t)255;
  const size_t off_D = (off_g2 + sz_g2 + 255) & ~(size_t)255;
  const size_t off_F = (off_D + sz_D + 255) & ~(size_t)255;
  const size_t off_P = (off_F + sz_D + 255) & ~(size_t)255;
  int rc = ctx->sc_rdm3.ensure(off_P + sizeof(double) * (size_t)nsplit * n2 * n2 + 256);
  if (rc) return rc;
  char *w = (char *)ctx->sc_rdm3.ptr;
  double *g1 = (double *)w, *g2 = (double *)(w + off_g2);
  double *D = (double *)(w + off_D), *F = (double *)(w + off_F), *P = (double *)(w + off_P);
  if ((rc = rdm12_fp64(ctx, C, C, g1, g2, false))) return rc;
  const unsigned nbD = (unsigned)std::min<long long>((ND + 255) / 256, 152LL * 32);
  {
    FORTE_PROF(ctx, "build_D");
    k_build_D<<<nbD, 256, 0, st>>>(ctx->sd[0].dense, ctx->sd[1].dense, n, C, NA, NB, D);
    FORTE_LAUNCH_CHECK();
  }
  const int ntile = (n2 + GT - 1) / GT;
  const long long kper = (ND + nsplit - 1) / nsplit;
  const dim3 gg(ntile * ntile, nsplit);
  for (int t = 0; t < n; ++t)
    for (int u = 0; u < n; ++u) {
      {
        FORTE_PROF(ctx, "build_D");
        k_build_D<<<nbD, 256, 0, st>>>(ctx->sd[0].dense, ctx->sd[1].dense, n, D + (size_t)(t * n + u) * ND, NA,
                                       NB, F);
        FORTE_LAUNCH_CHECK();
      }
      {
        FORTE_PROF(ctx, "gram");
        k_gram<<<gg, 256, 0, st>>>(D, F, n2, ND, kper, 0, P);
        FORTE_LAUNCH_CHECK();
      }
      {
        FORTE_PROF(ctx, "finish_g3");
        k_finish_g3<<<(n2 * n2 + 255) / 256, 256, 0, st>>>(P, nsplit, n, t, u, g1, g2, g3);
        FORTE_LAUNCH_CHECK();
      }
    }
  return FORTE_OK;
}

}  // namespace forte
