// FP64 sigma build  sigma = H C  in the alpha-string x beta-string basis
// (Sec. II.A.1; Hamiltonian Eq. 1 in the spin-free form
//  H = sum_pq k_pq E_pq + 1/2 sum_pqrs (pq|rs) E_pq E_rs,  k_pq = h_pq - 1/2 sum_r (pr|rq)).
//
// Split by spin:
//   sigma_aa[Ia,Ib] = sum_Ja  H_aa[Ia,Ja] C[Ja,Ib]      (same-spin string Hamiltonian, CSR)
//   sigma_bb[Ia,Ib] = sum_Jb  H_bb[Ib,Jb] C[Ia,Jb]      (same kernel on C transposed)
//   sigma_ab[Ia,Ib] = sum_{e in L(Ia)} sum_{f in L(Jb)} s_e s_f (pq_e|rs_f) C[J_e, Jb],
//                     scattered to Ib = J_f for every Jb
// where L(I) is the signed single-replacement list of string I.
#include <algorithm>

#include "forte_internal.h"

namespace forte {

constexpr int SS_THREADS = 256;
constexpr int SS_CPT = 2;              // output columns per thread
constexpr int SS_SEG = 512;            // CSR entries staged per pass

// Y[row, c] (+)= sum_nz val * X[col, c]; rows of X and Y are ncol long.
// grid.x = nrow * nchunk, grid.y = vector.
template <typename T>
__global__ void __launch_bounds__(SS_THREADS) k_ss_spmm(const int *__restrict__ ptr,
                                                        const int *__restrict__ col,
                                                        const T *__restrict__ val,
                                                        const T *__restrict__ X, T *__restrict__ Y,
                                                        long long nrow, long long ncol, int nchunk,
                                                        long long vstride, int accumulate) {
  __shared__ int s_col[SS_SEG];
  __shared__ T s_val[SS_SEG];
  const long long row = blockIdx.x / nchunk;
  const int chunk = blockIdx.x % nchunk;
  const T *Xv = X + (long long)blockIdx.y * vstride;
  T *Yv = Y + (long long)blockIdx.y * vstride;
  long long c0 = (long long)chunk * SS_THREADS * SS_CPT + threadIdx.x;
  T acc[SS_CPT];
#pragma unroll
  for (int k = 0; k < SS_CPT; ++k) acc[k] = T(0);
  const int b = ptr[row], e = ptr[row + 1];
  for (int s0 = b; s0 < e; s0 += SS_SEG) {
    int cnt = min(SS_SEG, e - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += SS_THREADS) {
      s_col[i] = col[s0 + i];
      s_val[i] = val[s0 + i];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
      const T v = s_val[i];
      const T *xr = Xv + (long long)s_col[i] * ncol;
#pragma unroll
      for (int k = 0; k < SS_CPT; ++k) {
        long long c = c0 + (long long)k * SS_THREADS;
        if (c < ncol) acc[k] += v * xr[c];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < SS_CPT; ++k) {
    long long c = c0 + (long long)k * SS_THREADS;
    if (c < ncol) {
      T *y = Yv + row * ncol + c;
      *y = accumulate ? *y + acc[k] : acc[k];
    }
  }
}

// Y[c][r] (+)= X[r][c] for an R x Cc matrix per vector.
template <typename T>
__global__ void k_transpose(const T *__restrict__ X, T *__restrict__ Y, long long R, long long Cc,
                            long long vstride, int accumulate) {
  __shared__ T tile[32][33];
  const T *Xv = X + (long long)blockIdx.z * vstride;
  T *Yv = Y + (long long)blockIdx.z * vstride;
  long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    long long r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Cc) tile[i][threadIdx.x] = Xv[r * Cc + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    long long c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < Cc) {
      T v = tile[threadIdx.x][i];
      T *y = Yv + c * R + r;
      *y = accumulate ? *y + v : v;
    }
  }
}

constexpr int AB_THREADS = 256;

// sigma_ab for one alpha string Ia (blockIdx.x) and one vector (blockIdx.y).
// Shared memory: Gs[nkA][npair] signed integral rows, srow[NB] output row,
// D[nkA][TJ] gathered C rows, Lb[TJ][nkB] beta replacement lists of the tile.
__global__ void __launch_bounds__(AB_THREADS) k_ab_fp64(const Repl *__restrict__ listA, int nkA,
                                                        const Repl *__restrict__ listB, int nkB,
                                                        long long NB, const double *__restrict__ gpair,
                                                        int npair, const double *__restrict__ C,
                                                        double *__restrict__ S, long long vstride,
                                                        int TJ) {
  extern __shared__ double smem[];
  double *Gs = smem;                                  // nkA * npair
  double *srow = Gs + (size_t)nkA * npair;            // NB
  double *D = srow + NB;                              // nkA * TJ
  Repl *Lb = reinterpret_cast<Repl *>(D + (size_t)nkA * TJ);  // TJ * nkB
  const long long Ia = blockIdx.x;
  const double *Cv = C + (long long)blockIdx.y * vstride;
  double *Sv = S + (long long)blockIdx.y * vstride;
  const Repl *la = listA + Ia * nkA;
  __shared__ int s_J[80];
  for (int e = threadIdx.x; e < nkA; e += AB_THREADS) s_J[e] = la[e].J;
  for (int i = threadIdx.x; i < nkA * npair; i += AB_THREADS) {
    int e = i / npair, rs = i % npair;
    Repl r = la[e];
    Gs[i] = r.sgn * gpair[(size_t)r.pair * npair + rs];
  }
  for (long long i = threadIdx.x; i < NB; i += AB_THREADS) srow[i] = 0.0;
  __syncthreads();
  for (long long j0 = 0; j0 < NB; j0 += TJ) {
    const int tj = (int)min((long long)TJ, NB - j0);
    for (int i = threadIdx.x; i < nkA * tj; i += AB_THREADS) {
      int e = i / tj, j = i % tj;
      D[e * TJ + j] = Cv[(long long)s_J[e] * NB + j0 + j];
    }
    for (int i = threadIdx.x; i < tj * nkB; i += AB_THREADS) Lb[i] = listB[j0 * nkB + i];
    __syncthreads();
    const int npairs_tile = tj * nkB;
    for (int w = threadIdx.x; w < npairs_tile; w += AB_THREADS) {
      const int j = w / nkB;
      const Repl rf = Lb[w];
      const double *g = Gs + rf.pair;
      const double *d = D + j;
      double acc = 0.0;
#pragma unroll 8
      for (int e = 0; e < nkA; ++e) acc += g[e * npair] * d[e * TJ];
      atomicAdd(&srow[rf.J], rf.sgn * acc);
    }
    __syncthreads();
  }
  for (long long i = threadIdx.x; i < NB; i += AB_THREADS) Sv[Ia * NB + i] += srow[i];
}

static size_t ab_smem_bytes(int nkA, int nkB, int npair, long long NB, int TJ) {
  return sizeof(double) * ((size_t)nkA * npair + NB + (size_t)nkA * TJ) + sizeof(Repl) * (size_t)TJ * nkB;
}

int sigma_fp64(forte_ctx *ctx, const double *C, double *S, int nvec) {
  // beta-beta scratch: T1 = C^T, T2 = H_bb T1 (grown on demand)
  const long long ND = ctx->Ndet;
  int rc = ctx->sc_t1.ensure(sizeof(double) * ND * nvec);
  if (rc) return rc;
  rc = ctx->sc_t2.ensure(sizeof(double) * ND * nvec);
  if (rc) return rc;
  return sigma_fp64_scratch(ctx, C, S, nvec, (double *)ctx->sc_t1.ptr, (double *)ctx->sc_t2.ptr);
}

// The FP64 sigma with caller-provided scratch T1, T2 (each >= nvec * Ndet
// doubles); allocates nothing.  Shared by forte_sigma (context scratch) and
// forte_sigma_fp64_noalloc (the library's fixed array).
int sigma_fp64_scratch(forte_ctx *ctx, const double *C, double *S, int nvec, double *T1, double *T2) {
  cudaStream_t st = ctx->stream;
  const long long NA = ctx->Na, NB = ctx->Nb, ND = ctx->Ndet;
  // alpha-alpha: S = H_aa C
  {
    int nchunk = (int)((NB + SS_THREADS * SS_CPT - 1) / (SS_THREADS * SS_CPT));
    dim3 grid((unsigned)(NA * nchunk), nvec);
    FORTE_PROF(ctx, "ss_spmm");
    k_ss_spmm<double><<<grid, SS_THREADS, 0, st>>>(ctx->sd[0].csr_ptr, ctx->sd[0].csr_col,
                                                   ctx->sd[0].csr_val, C, S, NA, NB, nchunk, ND, 0);
    FORTE_LAUNCH_CHECK();
  }
  // beta-beta: T1 = C^T, T2 = H_bb T1, S += T2^T
  {
    dim3 tb(32, 8);
    dim3 g1((unsigned)((NB + 31) / 32), (unsigned)((NA + 31) / 32), nvec);
    {
      FORTE_PROF(ctx, "transpose");
      k_transpose<double><<<g1, tb, 0, st>>>(C, T1, NA, NB, ND, 0);
      FORTE_LAUNCH_CHECK();
    }
    int nchunk = (int)((NA + SS_THREADS * SS_CPT - 1) / (SS_THREADS * SS_CPT));
    dim3 grid((unsigned)(NB * nchunk), nvec);
    {
      FORTE_PROF(ctx, "ss_spmm");
      k_ss_spmm<double><<<grid, SS_THREADS, 0, st>>>(ctx->sd[1].csr_ptr, ctx->sd[1].csr_col,
                                                     ctx->sd[1].csr_val, T1, T2, NB, NA, nchunk, ND, 0);
      FORTE_LAUNCH_CHECK();
    }
    dim3 g2((unsigned)((NA + 31) / 32), (unsigned)((NB + 31) / 32), nvec);
    {
      FORTE_PROF(ctx, "transpose");
      k_transpose<double><<<g2, tb, 0, st>>>(T2, S, NB, NA, ND, 1);
      FORTE_LAUNCH_CHECK();
    }
  }
  // alpha-beta
  const int nkA = ctx->sh[0].nk, nkB = ctx->sh[ctx->same_strings ? 0 : 1].nk;
  if (nkA > 0 && nkB > 0) {
    if (nkA > 80) {
      set_error("alpha replacement list too long (%d)", nkA);
      return FORTE_ERR_ARG;
    }
    int TJ = 64;
    size_t smem = ab_smem_bytes(nkA, nkB, ctx->npair, NB, TJ);
    while (smem > 220 * 1024 && TJ > 8) {
      TJ /= 2;
      smem = ab_smem_bytes(nkA, nkB, ctx->npair, NB, TJ);
    }
    if (smem > 220 * 1024) {
      set_error("alpha-beta FP64 kernel needs %zu bytes of shared memory", smem);
      return FORTE_ERR_ARG;
    }
    FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_ab_fp64));
    dim3 grid((unsigned)NA, nvec);
    FORTE_PROF(ctx, "ab_fp64");
    k_ab_fp64<<<grid, AB_THREADS, smem, st>>>(ctx->sd[0].list, nkA, ctx->sd[1].list, nkB, NB, ctx->d_gpair,
                                              ctx->npair, C, S, ND, TJ);
    FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

// FP32 same-spin term for the reduced-precision path:
//   S32 = H_aa C32  then  S32 += (H_bb C32^T)^T,  via the scratch buffers T1/T2.
int same_spin_f32(forte_ctx *ctx, const float *C32, float *S32, float *T1, float *T2, int nvec) {
  cudaStream_t st = ctx->stream;
  const long long NA = ctx->Na, NB = ctx->Nb, ND = ctx->Ndet;
  {
    int nchunk = (int)((NB + SS_THREADS * SS_CPT - 1) / (SS_THREADS * SS_CPT));
    dim3 grid((unsigned)(NA * nchunk), nvec);
    {
      FORTE_PROF(ctx, "ss_spmm_f32");
      k_ss_spmm<float><<<grid, SS_THREADS, 0, st>>>(ctx->sd[0].csr_ptr, ctx->sd[0].csr_col,
                                                    ctx->sd[0].csr_val32, C32, S32, NA, NB, nchunk, ND, 0);
      FORTE_LAUNCH_CHECK();
    }
  }
  dim3 tb(32, 8);
  dim3 g1((unsigned)((NB + 31) / 32), (unsigned)((NA + 31) / 32), nvec);
  {
    FORTE_PROF(ctx, "transpose_f32");
    k_transpose<float><<<g1, tb, 0, st>>>(C32, T1, NA, NB, ND, 0);
    FORTE_LAUNCH_CHECK();
  }
  {
    int nchunk = (int)((NA + SS_THREADS * SS_CPT - 1) / (SS_THREADS * SS_CPT));
    dim3 grid((unsigned)(NB * nchunk), nvec);
    FORTE_PROF(ctx, "ss_spmm_f32");
    k_ss_spmm<float><<<grid, SS_THREADS, 0, st>>>(ctx->sd[1].csr_ptr, ctx->sd[1].csr_col,
                                                  ctx->sd[1].csr_val32, T1, T2, NB, NA, nchunk, ND, 0);
    FORTE_LAUNCH_CHECK();
  }
  dim3 g2((unsigned)((NA + 31) / 32), (unsigned)((NB + 31) / 32), nvec);
  {
    FORTE_PROF(ctx, "transpose_f32");
    k_transpose<float><<<g2, tb, 0, st>>>(T2, S32, NB, NA, ND, 1);
    FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

// H_II = H_aa[Ia,Ia] + H_bb[Ib,Ib] + sum_{i in Ia, j in Ib} (ii|jj)
__global__ void k_hdiag(const double *__restrict__ dA, const double *__restrict__ dB,
                        const double *__restrict__ W, const uint32_t *__restrict__ strB, int n,
                        long long NA, long long NB, double *__restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NA * NB) return;
  long long ia = i / NB, ib = i % NB;
  uint32_t s = strB[ib];
  double v = dA[ia] + dB[ib];
  const double *w = W + ia * n;
  while (s) {
    int j = __ffs(s) - 1;
    v += w[j];
    s &= s - 1;
  }
  out[i] = v;
}

int hdiag_build(forte_ctx *ctx) {
  const int n = ctx->n;
  const SpinHost &A = ctx->sh[0];
  std::vector<double> W((size_t)A.N * n, 0.0);
  for (long long ia = 0; ia < A.N; ++ia)
    for (int j = 0; j < n; ++j) {
      double v = 0.0;
      for (int i = 0; i < n; ++i)
        if ((A.str[ia] >> i) & 1u) v += ctx->eri[(((size_t)i * n + i) * n + j) * n + j];
      W[(size_t)ia * n + j] = v;
    }
  double *dW = nullptr;
  FORTE_CUDA_TRY(cudaMalloc(&dW, sizeof(double) * W.size()));
  FORTE_CUDA_TRY(cudaMemcpy(dW, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice));
  if (!ctx->d_hdiag) {
    cudaError_t e = cudaMalloc(&ctx->d_hdiag, sizeof(double) * ctx->Ndet);
    if (e != cudaSuccess) {
      cudaFree(dW);
      set_error("cudaMalloc hdiag failed: %s", cudaGetErrorString(e));
      return FORTE_ERR_ALLOC;
    }
  }
  long long nt = ctx->Ndet;
  k_hdiag<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(
      ctx->sd[0].diag, ctx->sd[1].diag, dW, ctx->sd[1].str, n, ctx->Na, ctx->Nb, ctx->d_hdiag);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(dW);
  if (e != cudaSuccess) {
    set_error("hdiag kernel failed: %s", cudaGetErrorString(e));
    return FORTE_ERR_CUDA;
  }
  return FORTE_OK;
}

// ============================================================================
// FP64-class sigma in double-FP32 arithmetic (precision FORTE_DF32, and the
// refinement operator of the reduced-precision modes).
//
// Every FP64 operand x is held as an unevaluated pair x = hi + lo of FP32 values
// (hi = fl32(x), lo = fl32(x - hi); |x - hi - lo| <= 2^-48 |x|).  A product term
// a b adds hi_a hi_b exactly (the FMA residual of the FP32 product), the cross
// terms hi_a lo_b + lo_a hi_b in FP32, and drops lo_a lo_b (2^-48 relative); the
// running sum is a compensated pair (TwoSum of Knuth, TAOCP vol. 2, Sec. 4.2.2).
// Relative error per product about 2^-46.  The FP32 pipe of this GPU issues 64
// times the FP64 pipe's operations, so ~12 FP32 operations per term beat one DFMA.
// ============================================================================

__device__ __forceinline__ void df_fma(float &ah, float &al, float2 a, float2 b) {
  const float p = a.x * b.x;
  const float pe = fmaf(a.x, b.x, -p);
  const float c = fmaf(a.x, b.y, a.y * b.x);
  const float s = ah + p;
  const float bb = s - ah;
  const float e = (ah - (s - bb)) + (p - bb);
  ah = s;
  al += e + (pe + c);
}

// Y[c][r] = X[r][c] for an R x Cc matrix of (hi, lo) pairs per vector.
__global__ void k_transpose_df(const float2 *__restrict__ X, float2 *__restrict__ Y, long long R, long long Cc,
                               long long vstride) {
  __shared__ float2 tile[32][33];
  const float2 *Xv = X + (long long)blockIdx.z * vstride;
  float2 *Yv = Y + (long long)blockIdx.z * vstride;
  const long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long long r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < Cc) tile[i][threadIdx.x] = Xv[r * Cc + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long long c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < Cc) Yv[c * R + r] = tile[threadIdx.x][i];
  }
}

// x -> (hi, lo)
__global__ void k_df_split(const double *__restrict__ x, float2 *__restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    y[i] = make_float2(h, (float)(v - (double)h));
  }
}

// Same-spin CSR product in double-FP32: Y[row, c] (+)= sum_nz val * X[col, c],
// X and val as (hi, lo) pairs, Y FP64.  grid.x = nrow * nchunk, grid.y = vector.
__global__ void __launch_bounds__(SS_THREADS) k_ss_spmm_df(const int *__restrict__ ptr, const int *__restrict__ col,
                                                           const float2 *__restrict__ val, const float2 *__restrict__ X,
                                                           double *__restrict__ Y, long long nrow, long long ncol,
                                                           int nchunk, long long vstride, int accumulate) {
  __shared__ int s_col[SS_SEG];
  __shared__ float2 s_val[SS_SEG];
  const long long row = blockIdx.x / nchunk;
  const int chunk = blockIdx.x % nchunk;
  const float2 *Xv = X + (long long)blockIdx.y * vstride;
  double *Yv = Y + (long long)blockIdx.y * vstride;
  const long long c0 = (long long)chunk * SS_THREADS * SS_CPT + threadIdx.x;
  float ah[SS_CPT], al[SS_CPT];
#pragma unroll
  for (int k = 0; k < SS_CPT; ++k) ah[k] = al[k] = 0.f;
  const int b = ptr[row], e = ptr[row + 1];
  for (int s0 = b; s0 < e; s0 += SS_SEG) {
    const int cnt = min(SS_SEG, e - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += SS_THREADS) {
      s_col[i] = col[s0 + i];
      s_val[i] = val[s0 + i];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
      const float2 v = s_val[i];
      const float2 *xr = Xv + (long long)s_col[i] * ncol;
#pragma unroll
      for (int k = 0; k < SS_CPT; ++k) {
        const long long c = c0 + (long long)k * SS_THREADS;
        if (c < ncol) df_fma(ah[k], al[k], v, xr[c]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < SS_CPT; ++k) {
    const long long c = c0 + (long long)k * SS_THREADS;
    if (c < ncol) {
      double *y = Yv + row * ncol + c;
      const double r = (double)ah[k] + (double)al[k];
      *y = accumulate ? *y + r : r;
    }
  }
}

// sigma_ab in double-FP32 for one alpha string Ia (blockIdx.x) and one vector
// (blockIdx.y): k_ab_fp64 with (hi, lo) operands; the output row stays FP64.
// 16 warps and 32-string tiles: two CTAs fit on an SM, so the tile gathers of one
// overlap the shared-memory-bound inner products of the other.
constexpr int AB_DF_THREADS = 512;
constexpr int AB_DF_TJ = 32;
__global__ void __launch_bounds__(AB_DF_THREADS) k_ab_df(const Repl *__restrict__ listA, int nkA,
                                                      const Repl *__restrict__ listB, int nkB, long long NB,
                                                      const float2 *__restrict__ gpair2, int npair,
                                                      const float2 *__restrict__ C2, double *__restrict__ S,
                                                      long long vstride, int TJ) {
  extern __shared__ double smem[];
  float2 *Gs = reinterpret_cast<float2 *>(smem);                 // nkA * npair
  double *srow = smem + (size_t)nkA * npair;                     // NB
  float2 *D = reinterpret_cast<float2 *>(srow + NB);              // nkA * TJ
  Repl *Lb = reinterpret_cast<Repl *>(D + (size_t)nkA * TJ);      // TJ * nkB
  const long long Ia = blockIdx.x;
  const float2 *Cv = C2 + (long long)blockIdx.y * vstride;
  double *Sv = S + (long long)blockIdx.y * vstride;
  const Repl *la = listA + Ia * nkA;
  __shared__ int s_J[80];
  for (int e = threadIdx.x; e < nkA; e += AB_DF_THREADS) s_J[e] = la[e].J;
  for (int i = threadIdx.x; i < nkA * npair; i += AB_DF_THREADS) {
    const int e = i / npair, rs = i % npair;
    const Repl r = la[e];
    float2 g = gpair2[(size_t)r.pair * npair + rs];
    if (r.sgn < 0) g = make_float2(-g.x, -g.y);
    Gs[i] = g;
  }
  for (long long i = threadIdx.x; i < NB; i += AB_DF_THREADS) srow[i] = 0.0;
  __syncthreads();
  for (long long j0 = 0; j0 < NB; j0 += TJ) {
    const int tj = (int)min((long long)TJ, NB - j0);
    for (int i = threadIdx.x; i < nkA * tj; i += AB_DF_THREADS) {
      const int e = i / tj, j = i % tj;
      D[e * TJ + j] = Cv[(long long)s_J[e] * NB + j0 + j];
    }
    for (int i = threadIdx.x; i < tj * nkB; i += AB_DF_THREADS) Lb[i] = listB[j0 * nkB + i];
    __syncthreads();
    const int npairs_tile = tj * nkB;
    for (int w = threadIdx.x; w < npairs_tile; w += AB_DF_THREADS) {
      const int j = w / nkB;
      const Repl rf = Lb[w];
      const float2 *g = Gs + rf.pair;
      const float2 *d = D + j;
      float ah = 0.f, al = 0.f;
#pragma unroll 8
      for (int e = 0; e < nkA; ++e) df_fma(ah, al, g[e * npair], d[e * TJ]);
      atomicAdd(&srow[rf.J], rf.sgn * ((double)ah + (double)al));
    }
    __syncthreads();
  }
  for (long long i = threadIdx.x; i < NB; i += AB_DF_THREADS) Sv[Ia * NB + i] += srow[i];
}

static int df_setup(forte_ctx *ctx) {
  if (ctx->d_gpair2) return FORTE_OK;
  const int np = ctx->npair;
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_gpair2, sizeof(float2) * (size_t)np * np));
  k_df_split<<<(unsigned)std::min<long long>(((long long)np * np + 255) / 256, 1024), 256, 0, ctx->stream>>>(
      ctx->d_gpair, (float2 *)ctx->d_gpair2, (long long)np * np);
  FORTE_LAUNCH_CHECK();
  const int nsp = ctx->same_strings ? 1 : 2;
  for (int s = 0; s < nsp; ++s) {
    const long long nnz = (long long)ctx->sh[s].csr_col.size();
    FORTE_CUDA_TRY(cudaMalloc(&ctx->d_csr_val2[s], sizeof(float2) * (size_t)std::max(1LL, nnz)));
    if (nnz > 0) {
      k_df_split<<<(unsigned)std::min<long long>((nnz + 255) / 256, 152LL * 16), 256, 0, ctx->stream>>>(
          ctx->sd[s].csr_val, (float2 *)ctx->d_csr_val2[s], nnz);
      FORTE_LAUNCH_CHECK();
    }
  }
  if (ctx->same_strings) ctx->d_csr_val2[1] = ctx->d_csr_val2[0];
  return FORTE_OK;
}

int sigma_df(forte_ctx *ctx, const double *C, double *S, int nvec, bool with_ab) {
  int rc = df_setup(ctx);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const long long NA = ctx->Na, NB = ctx->Nb, ND = ctx->Ndet;
  const size_t nf = (size_t)nvec * ND;
  if ((rc = ctx->sc_df.ensure(sizeof(float2) * nf + 256))) return rc;
  if ((rc = ctx->sc_t1.ensure(sizeof(float2) * nf + 256))) return rc;
  if ((rc = ctx->sc_t2.ensure(sizeof(double) * nf + 256))) return rc;
  float2 *C2 = (float2 *)ctx->sc_df.ptr, *T1 = (float2 *)ctx->sc_t1.ptr;
  double *T2 = (double *)ctx->sc_t2.ptr;
  const float2 *v2a = (const float2 *)ctx->d_csr_val2[0], *v2b = (const float2 *)ctx->d_csr_val2[1];
  {
    FORTE_PROF(ctx, "df_split");
    k_df_split<<<(unsigned)std::min<size_t>((nf + 255) / 256, 152 * 16), 256, 0, st>>>(C, C2, (long long)nf);
    FORTE_LAUNCH_CHECK();
  }
  {
    const int nchunk = (int)((NB + SS_THREADS * SS_CPT - 1) / (SS_THREADS * SS_CPT));
    dim3 grid((unsigned)(NA * nchunk), nvec);
    FORTE_PROF(ctx, "ss_spmm_df");
    k_ss_spmm_df<<<grid, SS_THREADS, 0, st>>>(ctx->sd[0].csr_ptr, ctx->sd[0].csr_col, v2a, C2, S, NA, NB, nchunk, ND, 0);
    FORTE_LAUNCH_CHECK();
  }
  {
    dim3 tb(32, 8);
    dim3 g1((unsigned)((NB + 31) / 32), (unsigned)((NA + 31) / 32), nvec);
    {
      FORTE_PROF(ctx, "transpose");
      k_transpose_df<<<g1, tb, 0, st>>>(C2, T1, NA, NB, ND);
      FORTE_LAUNCH_CHECK();
    }
    const int nchunk = (int)((NA + SS_THREADS * SS_CPT - 1) / (SS_THREADS * SS_CPT));
    dim3 grid((unsigned)(NB * nchunk), nvec);
    {
      FORTE_PROF(ctx, "ss_spmm_df");
      k_ss_spmm_df<<<grid, SS_THREADS, 0, st>>>(ctx->sd[1].csr_ptr, ctx->sd[1].csr_col, v2b, T1, T2, NB, NA, nchunk, ND,
                                                0);
      FORTE_LAUNCH_CHECK();
    }
    dim3 g2((unsigned)((NA + 31) / 32), (unsigned)((NB + 31) / 32), nvec);
    {
      FORTE_PROF(ctx, "transpose");
      k_transpose<double><<<g2, tb, 0, st>>>(T2, S, NB, NA, ND, 1);
      FORTE_LAUNCH_CHECK();
    }
  }
  const int nkA = ctx->sh[0].nk, nkB = ctx->sh[ctx->same_strings ? 0 : 1].nk;
  if (with_ab && nkA > 0 && nkB > 0) {
    if (nkA > 80) {
      set_error("alpha replacement list too long (%d)", nkA);
      return FORTE_ERR_ARG;
    }
    int TJ = AB_DF_TJ;
    size_t smem = ab_smem_bytes(nkA, nkB, ctx->npair, NB, TJ);
    while (smem > 220 * 1024 && TJ > 8) {
      TJ /= 2;
      smem = ab_smem_bytes(nkA, nkB, ctx->npair, NB, TJ);
    }
    if (smem > 220 * 1024) {
      set_error("alpha-beta double-FP32 kernel needs %zu bytes of shared memory", smem);
      return FORTE_ERR_ARG;
    }
    FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_ab_df));
    dim3 grid((unsigned)NA, nvec);
    FORTE_PROF(ctx, "ab_df");
    k_ab_df<<<grid, AB_DF_THREADS, smem, st>>>(ctx->sd[0].list, nkA, ctx->sd[1].list, nkB, NB,
                                            (const float2 *)ctx->d_gpair2, ctx->npair, C2, S, ND, TJ);
    FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

}  // namespace forte
