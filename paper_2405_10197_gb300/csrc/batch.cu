// Batched solve of many independent active-space problems (step a11): each
// problem is an ActiveSpaceMethod instance in the paper's terms (Sec. III,
// ActiveSpaceSolver), and CASCI (Sec. II.A.1) is solved for each of them.
//
// Design: problems with the same (n, n_alpha, n_beta) form a size class that
// shares its string lists, replacement lists and the sparsity pattern of the
// same-spin string Hamiltonians; only integral-dependent data (CSR values,
// pair integrals, H_II pieces) are per problem.  Every class is ONE kernel
// launch with one CTA per problem; a CTA runs the whole Davidson-Liu solve of
// its problem on the device (sigma, subspace matrix, a warp-parallel Jacobi
// eigensolver, residuals, preconditioner, Gram-Schmidt, collapse) and writes
// the energies -- no host round trip, no per-problem launch, no per-problem
// allocation (one pooled cudaMalloc for the batch).  The class launches run
// concurrently, captured once into a CUDA graph.
//
// Arithmetic of the per-CTA sigma:
//   FORTE_FP64                  FP64 throughout;
//   FORTE_DF32 / FORTE_OZ64     double-FP32 (FP64-class, relative ~2^-46 per term);
//   FORTE_TF32 / FORTE_BF16X2   FP32 sigma for the Davidson phase down to a residual
//                               of max(tol, 3e-4), then the double-FP32 sigma from the
//                               Ritz vectors to tol (the tensor-core kernels are built
//                               for one problem spread over the GPU, not one CTA).
// Davidson vectors, the subspace matrix and its eigenproblem are FP64 in every mode.
//
// Autotuner: before the solve, for each class and each arithmetic the solve uses,
// the per-CTA sigma runs once on the first problems of the class for every
// candidate (threads per CTA x beta tile width of the alpha-beta term) that fits
// in shared memory; the fastest candidate (CUDA events) is used for the solve
// and reported by forte_batch_tuning.  It then times one Davidson iteration of
// the class's first problem on the single-problem path (forte_cas_create /
// forte_davidson, with the tensor-core sigma in the reduced-precision modes) and
// sends the class there when P iterations of that path cost less than one class
// sigma round (t_sigma x waves of resident CTAs).
//
// Problems with more than BT_MAX_DET determinants are large enough to occupy the
// whole GPU on their own and always take the single-problem path.  (One CTA per
// such problem would spend minutes per FP64 solve on one SM.)  The class launches
// are captured into one graph and launched without waiting; the single-problem
// path runs meanwhile on BT_WORKERS host threads with their own streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <chrono>
#include <thread>
#include <type_traits>
#include <vector>

#include "forte_internal.h"

namespace forte {

int build_spin_tables(forte_ctx *ctx);

namespace {

constexpr int BT_MAXK = 36;               // subspace vectors per problem (12 per root, 3 roots)
constexpr int BT_LD = 37;                 // leading dimension of the small matrices in shared memory
constexpr int BT_SEG = 512;               // CSR entries staged per pass
constexpr long long BT_MAX_DET = 100000;  // larger problems take the single-problem path
constexpr int BT_MAX_ROOTS = 3;
constexpr int BT_WORKERS = 8;             // host threads of the single-problem path

enum { AR_F64 = 0, AR_F32 = 1, AR_DF = 2 };

// Everything a CTA needs about its class and its problem (kernel parameter).
struct BClass {
  int n, nkA, nkB, npair, P;
  long long NA, NB, N;
  const Repl *listA, *listB;
  const int *ptrA, *colA, *ptrB, *colB;
  long long nnzA, nnzB;
  const double *valA, *valB;    // [P][nnz]
  const float *valA32, *valB32;
  const float2 *valA2, *valB2;
  const double *diagA, *diagB;  // [P][NA], [P][NB]: same-spin diagonals
  const double *Wd;             // [P][NA][n]: sum_{i in Ia} (ii|jj)
  const uint32_t *strB;
  const double *gp;             // [P][npair][npair]
  const float *gp32;
  const float2 *gp2;
  const int *nroots;            // [P]
  const int *eoff;              // [P]: offset of the problem's energies
  const int *gidx;              // [P]: index of the problem in the batch (status, iterations)
  const long long *woff;        // [P]: offset of the problem's workspace (doubles)
  double *work;
  double *E, *rn;               // [sum nroots]
  int *iters, *status;          // [nprob], by batch index (gidx)
  double tol, tol1;             // final tolerance; end of the FP32 phase (mixed)
  int max_iter, mode, TJ;       // mode: 0 FP64, 1 FP32 then double-FP32, 2 double-FP32
  int probe;                    // > 0: run `probe` sigma builds only (autotuner)
};

// --------------------------------------------------------------- arithmetic
__device__ __forceinline__ void df_fma2(float &ah, float &al, float2 a, float2 b) {
  const float p = a.x * b.x;
  const float pe = fmaf(a.x, b.x, -p);
  const float c = fmaf(a.x, b.y, a.y * b.x);
  const float s = ah + p;
  const float bb = s - ah;
  const float e = (ah - (s - bb)) + (p - bb);
  ah = s;
  al += e + (pe + c);
}

template <int AR>
struct Ar;
template <>
struct Ar<AR_F64> {
  using X = double;
  using R = double;  // alpha-beta row accumulator
  struct Acc {
    double a = 0.0;
    __device__ void add(double g, double x) { a = fma(g, x, a); }
    __device__ double val() const { return a; }
  };
  static __device__ X cvt(double v) { return v; }
  static __device__ X neg(X v) { return -v; }
};
template <>
struct Ar<AR_F32> {
  using X = float;
  using R = float;
  struct Acc {
    float a = 0.f;
    __device__ void add(float g, float x) { a = fmaf(g, x, a); }
    __device__ double val() const { return (double)a; }
  };
  static __device__ X cvt(double v) { return (float)v; }
  static __device__ X neg(X v) { return -v; }
};
template <>
struct Ar<AR_DF> {
  using X = float2;
  using R = double;
  struct Acc {
    float h = 0.f, l = 0.f;
    __device__ void add(float2 g, float2 x) { df_fma2(h, l, g, x); }
    __device__ double val() const { return (double)h + (double)l; }
  };
  static __device__ X cvt(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  }
  static __device__ X neg(X v) { return make_float2(-v.x, -v.y); }
};

template <int AR>
__device__ __forceinline__ const typename Ar<AR>::X *csr_vals(const BClass &c, int q, int spin) {
  if (AR == AR_F64) return (const typename Ar<AR>::X *)((spin ? c.valB : c.valA) + (long long)q * (spin ? c.nnzB : c.nnzA));
  if (AR == AR_F32)
    return (const typename Ar<AR>::X *)((spin ? c.valB32 : c.valA32) + (long long)q * (spin ? c.nnzB : c.nnzA));
  return (const typename Ar<AR>::X *)((spin ? c.valB2 : c.valA2) + (long long)q * (spin ? c.nnzB : c.nnzA));
}
template <int AR>
__device__ __forceinline__ const typename Ar<AR>::X *pair_ints(const BClass &c, int q) {
  const long long o = (long long)q * c.npair * c.npair;
  if (AR == AR_F64) return (const typename Ar<AR>::X *)(c.gp + o);
  if (AR == AR_F32) return (const typename Ar<AR>::X *)(c.gp32 + o);
  return (const typename Ar<AR>::X *)(c.gp2 + o);
}

// --------------------------------------------------------------- block reductions
// Sums m <= 4 per-thread values over the CTA; every thread receives the sums.
template <int NT>
__device__ __forceinline__ void cta_sum4(double (&v)[4], int m, double *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (c >= m) break;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
  }
  __syncthreads();
  if (lane == 0)
    for (int c = 0; c < m; ++c) red[w * 4 + c] = v[c];
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    double s = 0.0;
    for (int i = 0; i < NT / 32; ++i) s += red[i * 4 + c];
    v[c] = s;
  }
  __syncthreads();
}

// out[j] = V_j . x for j < m (V rows ld apart); out in shared memory.
template <int NT>
__device__ void cta_dots(const double *V, int m, long long ld, const double *x, long long N, double *out,
                         double *red) {
  for (int j0 = 0; j0 < m; j0 += 4) {
    const int mm = min(4, m - j0);
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = threadIdx.x; i < N; i += NT) {
      const double xi = x[i];
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < mm) p[c] = fma(V[(long long)(j0 + c) * ld + i], xi, p[c]);
    }
    cta_sum4<NT>(p, mm, red);
    if (threadIdx.x == 0)
      for (int c = 0; c < mm; ++c) out[j0 + c] = p[c];
  }
  __syncthreads();
}

// out_c = sum_j coef[j * ncol + c] V_j for c < ncol <= 6 (out may not alias V).
template <int NT>
__device__ void cta_combine(const double *V, int m, long long ld, const double *coef, int ncol, double *out,
                            long long ldo, long long N) {
  for (long long i = threadIdx.x; i < N; i += NT) {
    double a[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < m; ++j) {
      const double vj = V[(long long)j * ld + i];
#pragma unroll
      for (int c = 0; c < 6; ++c)
        if (c < ncol) a[c] = fma(coef[j * ncol + c], vj, a[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (c < ncol) out[(long long)c * ldo + i] = a[c];
  }
  __syncthreads();
}

// t -= sum_j d_j V_j ; returns |t|^2 (every thread).
template <int NT>
__device__ double cta_orth_update(const double *V, int m, long long ld, const double *d, double *t, long long N,
                                  double *red) {
  double p[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long i = threadIdx.x; i < N; i += NT) {
    double ti = t[i];
    for (int j = 0; j < m; ++j) ti = fma(-d[j], V[(long long)j * ld + i], ti);
    t[i] = ti;
    p[0] = fma(ti, ti, p[0]);
  }
  cta_sum4<NT>(p, 1, red);
  return p[0];
}

// --------------------------------------------------------------- warp Jacobi
// Cyclic Jacobi (Golub & Van Loan, Sec. 8.5) on the k x k symmetric matrix A
// (shared, ld BT_LD) by one warp: rotations in sequence, each rotation's row and
// column updates spread over the lanes.  On return A's diagonal holds the
// eigenvalues, V (shared, ld BT_LD) the eigenvectors as columns, and
// perm[0..k) the ascending order.
__device__ void warp_jacobi(double *A, double *V, int k, int *perm) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < k * k; i += 32) V[(i / k) * BT_LD + (i % k)] = (i / k == i % k) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = lane; i < k * k; i += 32) {
    const double a = A[(i / k) * BT_LD + (i % k)];
    fro += a * a;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  __syncwarp();
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = lane; i < k * k; i += 32) {
      const int r = i / k, cc = i % k;
      if (r < cc) off += A[r * BT_LD + cc] * A[r * BT_LD + cc];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if (off <= 1e-32 * fro || off == 0.0) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[p * BT_LD + q];
        if (apq == 0.0) continue;
        const double tau = (A[q * BT_LD + q] - A[p * BT_LD + p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        __syncwarp();
        // columns p, q
        for (int i = lane; i < k; i += 32) {
          const double aip = A[i * BT_LD + p], aiq = A[i * BT_LD + q];
          A[i * BT_LD + p] = cs * aip - sn * aiq;
          A[i * BT_LD + q] = sn * aip + cs * aiq;
          const double vip = V[i * BT_LD + p], viq = V[i * BT_LD + q];
          V[i * BT_LD + p] = cs * vip - sn * viq;
          V[i * BT_LD + q] = sn * vip + cs * viq;
        }
        __syncwarp();
        // rows p, q
        for (int i = lane; i < k; i += 32) {
          const double api = A[p * BT_LD + i], aqi = A[q * BT_LD + i];
          A[p * BT_LD + i] = cs * api - sn * aqi;
          A[q * BT_LD + i] = sn * api + cs * aqi;
        }
        __syncwarp();
      }
  }
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < k; ++i) perm[i] = i;
    for (int i = 0; i < k; ++i)  // selection sort, ties keep the lower index
      for (int j = i + 1; j < k; ++j)
        if (A[perm[j] * BT_LD + perm[j]] < A[perm[i] * BT_LD + perm[i]]) {
          const int tmp = perm[i];
          perm[i] = perm[j];
          perm[j] = tmp;
        }
  }
  __syncwarp();
}

// --------------------------------------------------------------- sigma of one CTA
struct SigmaWs {
  void *xs, *xt;   // x (or its converted copy) and its transpose, N elements of Ar<AR>::X
  double *yt;      // transposed beta-beta result, N doubles
};

// y[Ia][Ib] = sum_J H[Ia][J] x[J][Ib] (CSR rows of one spin), rows of length ncol.
template <int AR, int NT>
__device__ void cta_csr(const int *ptr, const int *col, const typename Ar<AR>::X *val, const typename Ar<AR>::X *x,
                        double *y, long long nrow, long long ncol, uint8_t *smem) {
  using X = typename Ar<AR>::X;
  int *scol = (int *)smem;
  X *sval = (X *)(smem + BT_SEG * sizeof(int));
  for (long long r = 0; r < nrow; ++r) {
    const int b = ptr[r], e = ptr[r + 1];
    for (long long c0 = 0; c0 < ncol; c0 += 4 * NT) {
      typename Ar<AR>::Acc acc[4];
      for (int s0 = b; s0 < e; s0 += BT_SEG) {
        const int cnt = min(BT_SEG, e - s0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += NT) {
          scol[i] = col[s0 + i];
          sval[i] = val[s0 + i];
        }
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
          const X v = sval[i];
          const X *xr = x + (long long)scol[i] * ncol;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const long long cc = c0 + threadIdx.x + (long long)u * NT;
            if (cc < ncol) acc[u].add(v, xr[cc]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long cc = c0 + threadIdx.x + (long long)u * NT;
        if (cc < ncol) y[r * ncol + cc] = acc[u].val();
      }
    }
  }
  __syncthreads();
}

// out[c][r] = in[r][c] (+ out when accumulate) for an R x Cc matrix, tiles of 32 x 32.
template <typename TI, typename TO, int NT>
__device__ void cta_transpose(const TI *in, TO *out, long long R, long long Cc, bool accumulate, uint8_t *smem) {
  TI *tile = (TI *)smem;  // [32][33]
  for (long long r0 = 0; r0 < R; r0 += 32)
    for (long long c0 = 0; c0 < Cc; c0 += 32) {
      __syncthreads();
      for (int i = threadIdx.x; i < 32 * 32; i += NT) {
        const long long r = r0 + i / 32, c = c0 + i % 32;
        if (r < R && c < Cc) tile[(i / 32) * 33 + i % 32] = in[r * Cc + c];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 32 * 32; i += NT) {
        const long long c = c0 + i / 32, r = r0 + i % 32;
        if (r < R && c < Cc) {
          const TI v = tile[(i % 32) * 33 + i / 32];
          TO *o = out + c * R + r;
          if constexpr (std::is_same<TI, double>::value) {
            if (accumulate)
              *o = *o + v;
            else
              *o = v;
          } else {
            *o = v;
          }
        }
      }
    }
  __syncthreads();
}

// sigma = H x for problem q (Eq. 1 in the string basis, the three terms of the
// FP64 kernels of the single-problem path) in arithmetic AR.
template <int AR, int NT>
__device__ void cta_sigma(const BClass &c, int q, const double *x, double *y, const SigmaWs &ws, uint8_t *smem) {
  using X = typename Ar<AR>::X;
  using R = typename Ar<AR>::R;
  const long long NA = c.NA, NB = c.NB, N = c.N;
  const X *xs;
  if (AR == AR_F64) {
    xs = (const X *)x;
  } else {
    X *w = (X *)ws.xs;
    for (long long i = threadIdx.x; i < N; i += NT) w[i] = Ar<AR>::cvt(x[i]);
    __syncthreads();
    xs = w;
  }
  // alpha-alpha
  cta_csr<AR, NT>(c.ptrA, c.colA, csr_vals<AR>(c, q, 0), xs, y, NA, NB, smem);
  // beta-beta on the transpose
  X *xt = (X *)ws.xt;
  cta_transpose<X, X, NT>(xs, xt, NA, NB, false, smem);
  cta_csr<AR, NT>(c.ptrB, c.colB, csr_vals<AR>(c, q, 1), xt, ws.yt, NB, NA, smem);
  cta_transpose<double, double, NT>(ws.yt, y, NB, NA, true, smem);
  // alpha-beta, per alpha string: gathered rows x signed integral block, scattered
  const int nkA = c.nkA, nkB = c.nkB, np = c.npair, TJ = c.TJ;
  if (nkA == 0 || nkB == 0) return;
  const X *g = pair_ints<AR>(c, q);
  uint8_t *p = smem;
  X *Gs = (X *)p;
  p += sizeof(X) * ((nkA * np + 1) & ~1);
  R *srow = (R *)p;
  p += sizeof(R) * ((NB + 1) & ~1LL);
  X *D = (X *)p;
  p += sizeof(X) * nkA * TJ;
  Repl *Lb = (Repl *)p;
  p += sizeof(Repl) * TJ * nkB;
  int *sJ = (int *)p;
  for (long long Ia = 0; Ia < NA; ++Ia) {
    const Repl *la = c.listA + Ia * nkA;
    __syncthreads();
    for (int e = threadIdx.x; e < nkA; e += NT) sJ[e] = la[e].J;
    for (int i = threadIdx.x; i < nkA * np; i += NT) {
      const int e = i / np, rs = i % np;
      const Repl r = la[e];
      const X v = g[(long long)r.pair * np + rs];
      Gs[i] = r.sgn < 0 ? Ar<AR>::neg(v) : v;
    }
    for (long long i = threadIdx.x; i < NB; i += NT) srow[i] = R(0);
    for (long long j0 = 0; j0 < NB; j0 += TJ) {
      const int tj = (int)min((long long)TJ, NB - j0);
      __syncthreads();
      for (int i = threadIdx.x; i < nkA * tj; i += NT) {
        const int e = i / tj, j = i % tj;
        D[e * TJ + j] = xs[(long long)sJ[e] * NB + j0 + j];
      }
      for (int i = threadIdx.x; i < tj * nkB; i += NT) Lb[i] = c.listB[j0 * nkB + i];
      __syncthreads();
      for (int w = threadIdx.x; w < tj * nkB; w += NT) {
        const int j = w / nkB;
        const Repl rf = Lb[w];
        typename Ar<AR>::Acc acc;
        for (int e = 0; e < nkA; ++e) acc.add(Gs[e * np + rf.pair], D[e * TJ + j]);
        const double v = acc.val();
        atomicAdd(&srow[rf.J], (R)(rf.sgn < 0 ? -v : v));
      }
    }
    __syncthreads();
    for (long long i = threadIdx.x; i < NB; i += NT) y[Ia * NB + i] += (double)srow[i];
  }
  __syncthreads();
}

// Shared memory of the alpha-beta term (the largest sigma area).
__host__ __device__ inline size_t ab_bytes(int ar, int nkA, int nkB, int np, long long NB, int TJ) {
  const size_t xs = ar == AR_F32 ? 4 : 8, rs = ar == AR_F32 ? 4 : 8;
  return xs * ((nkA * np + 1) & ~1) + rs * ((NB + 1) & ~1LL) + xs * nkA * TJ + sizeof(Repl) * TJ * nkB +
         sizeof(int) * ((nkA + 1) & ~1) + 64;
}
__host__ __device__ inline size_t sigma_bytes(int ar, int nkA, int nkB, int np, long long NB, int TJ) {
  size_t b = ab_bytes(ar, nkA, nkB, np, NB, TJ);
  b = b > (size_t)BT_SEG * 12 + 64 ? b : (size_t)BT_SEG * 12 + 64;  // CSR staging
  b = b > 32 * 33 * 8 + 64 ? b : 32 * 33 * 8 + 64;                   // transpose tile
  return (b + 255) & ~(size_t)255;
}
constexpr size_t DV_BYTES = (3 * BT_MAXK * BT_LD + 64 + 64 + 256 + 64 + 4 * 32) * 8 + 64 * 4;

// --------------------------------------------------------------- the solve kernel
template <int NT>
__global__ void __launch_bounds__(NT) k_batch_davidson(const BClass c) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int q = blockIdx.x;
  if (q >= c.P) return;
  const long long N = c.N;
  const int nr = c.nroots[q];
  // shared: Davidson small arrays, then the sigma area
  double *G = (double *)smem_raw;          // [BT_MAXK][BT_LD] subspace matrix B^T H B
  double *Aj = G + BT_MAXK * BT_LD;        // Jacobi work matrix
  double *U = Aj + BT_MAXK * BT_LD;        // eigenvectors
  double *dots = U + BT_MAXK * BT_LD;      // [64]
  double *d2 = dots + 64;                  // [64]
  double *coef = d2 + 64;                  // [256]: up to 36 x 6 combination coefficients
  double *wv = coef + 256;                 // [64]
  double *red = wv + 64;                   // [4 * 32]
  int *perm = (int *)(red + 4 * 32);       // [64]
  uint8_t *sig = smem_raw + DV_BYTES;
  // workspace of this problem
  const int maxsub = min(12 * nr, (int)min((long long)BT_MAXK, N));
  const int keep = min(2 * nr, maxsub - 1) > nr ? min(2 * nr, maxsub - 1) : nr;
  double *B = c.work + c.woff[q];
  double *S = B + (long long)maxsub * N;
  double *T = S + (long long)maxsub * N;     // [nr][N] corrections
  double *W = T + (long long)nr * N;         // [keep][N] collapse / Ritz vectors
  double *hd = W + (long long)max(keep, nr) * N;
  SigmaWs ws;
  ws.xs = hd + N;
  ws.xt = hd + 2 * N;
  ws.yt = hd + 3 * N;

  // H_II = H_aa[Ia,Ia] + H_bb[Ib,Ib] + sum_{i in Ia, j in Ib} (ii|jj)
  {
    const double *dA = c.diagA + (long long)q * c.NA, *dB = c.diagB + (long long)q * c.NB;
    const double *Wd = c.Wd + (long long)q * c.NA * c.n;
    for (long long i = threadIdx.x; i < N; i += NT) {
      const long long ia = i / c.NB, ib = i % c.NB;
      double v = dA[ia] + dB[ib];
      for (uint32_t s = c.strB[ib]; s; s &= s - 1) v += Wd[ia * c.n + __ffs(s) - 1];
      hd[i] = v;
    }
  }
  __syncthreads();

  if (c.probe > 0) {  // autotuner: sigma builds only
    for (long long i = threadIdx.x; i < N; i += NT) B[i] = 1.0 / (1.0 + (double)(i % 7));
    __syncthreads();
    for (int r = 0; r < c.probe; ++r) {
      if (c.mode == 1)
        cta_sigma<AR_F32, NT>(c, q, B, S, ws, sig);
      else if (c.mode == 2)
        cta_sigma<AR_DF, NT>(c, q, B, S, ws, sig);
      else
        cta_sigma<AR_F64, NT>(c, q, B, S, ws, sig);
    }
    return;
  }

  // arithmetic phase: 0 FP64, 1 FP32, 2 double-FP32
  int phase = c.mode == 0 ? AR_F64 : (c.mode == 1 ? AR_F32 : AR_DF);
  auto sigma = [&](const double *x, double *y) {
    if (phase == AR_F32)
      cta_sigma<AR_F32, NT>(c, q, x, y, ws, sig);
    else if (phase == AR_DF)
      cta_sigma<AR_DF, NT>(c, q, x, y, ws, sig);
    else
      cta_sigma<AR_F64, NT>(c, q, x, y, ws, sig);
  };

  // guess: unit vectors at the lowest H_II (ties: lowest index) plus the splitmix64
  // perturbation of norm ~0.02 of the single-problem path, orthonormalised
  int k = 0;
  {
    long long *pick = (long long *)coef;  // [nr]
    for (int r = 0; r < nr; ++r) {
      double bv = INFINITY;
      long long bi = N;
      for (long long i = threadIdx.x; i < N; i += NT) {
        bool used = false;
        for (int u = 0; u < r; ++u) used |= (pick[u] == i);
        if (!used && (hd[i] < bv || (hd[i] == bv && i < bi))) {
          bv = hd[i];
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov < bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      __syncthreads();
      if ((threadIdx.x & 31) == 0) {
        red[(threadIdx.x >> 5) * 2] = bv;
        ((long long *)red)[(threadIdx.x >> 5) * 2 + 1] = bi;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double v = INFINITY;
        long long ii = N;
        for (int w = 0; w < NT / 32; ++w) {
          const double ov = red[w * 2];
          const long long oi = ((long long *)red)[w * 2 + 1];
          if (ov < v || (ov == v && oi < ii)) {
            v = ov;
            ii = oi;
          }
        }
        pick[r] = ii;
      }
      __syncthreads();
    }
    const double scale = 0.02 * sqrt(12.0 / (double)N);
    for (int r = 0; r < nr; ++r) {
      double *b = B + (long long)k * N;
      const unsigned long long key = (unsigned long long)(r + 1) * 0x9E3779B97F4A7C15ull;
      const long long idx = pick[r];
      for (long long i = threadIdx.x; i < N; i += NT) {
        unsigned long long z = (unsigned long long)i + key;
        z += 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * 0x1.0p-53;
        b[i] = scale * (u - 0.5) + (i == idx ? 1.0 : 0.0);
      }
      __syncthreads();
      double nn = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        if (k > 0) cta_dots<NT>(B, k, N, b, N, dots, red);
        nn = cta_orth_update<NT>(B, k, N, dots, b, N, red);
      }
      if (nn > 1e-24) {
        const double s = 1.0 / sqrt(nn);
        for (long long i = threadIdx.x; i < N; i += NT) b[i] *= s;
        __syncthreads();
        ++k;
      }
    }
  }
  auto build_G = [&](int j0, int j1) {  // columns j0..j1-1 of G (and the mirrored rows)
    for (int j = j0; j < j1; ++j) {
      cta_dots<NT>(B, k, N, S + (long long)j * N, N, dots, red);
      if (threadIdx.x < k) {
        G[threadIdx.x * BT_LD + j] = dots[threadIdx.x];
        G[j * BT_LD + threadIdx.x] = dots[threadIdx.x];
      }
      __syncthreads();
    }
  };
  for (int j = 0; j < k; ++j) sigma(B + (long long)j * N, S + (long long)j * N);
  build_G(0, k);

  int it = 0, st = FORTE_ERR_NOT_CONVERGED;
  const int p1_cap = c.max_iter / 2;
  for (it = 1; it <= c.max_iter; ++it) {
    // Rayleigh-Ritz on the symmetrised subspace matrix
    for (int i = threadIdx.x; i < k * k; i += NT) {
      const int r = i / k, cc = i % k;
      Aj[r * BT_LD + cc] = 0.5 * (G[r * BT_LD + cc] + G[cc * BT_LD + r]);
    }
    __syncthreads();
    if (threadIdx.x < 32) warp_jacobi(Aj, U, k, perm);
    __syncthreads();
    if (threadIdx.x < k) wv[threadIdx.x] = Aj[perm[threadIdx.x] * BT_LD + perm[threadIdx.x]];
    __syncthreads();
    // residuals r = S u - theta B u, preconditioned t = r / (theta - H_II)
    bool all = true;
    double rmax = 0.0;
    for (int r = 0; r < nr; ++r) {
      const double th = wv[r];
      const int pc = perm[r];
      double *t = T + (long long)r * N;
      double p[4] = {0.0, 0.0, 0.0, 0.0};
      for (long long i = threadIdx.x; i < N; i += NT) {
        double v = 0.0;
        for (int j = 0; j < k; ++j) {
          const double u = U[j * BT_LD + pc];
          v = fma(u, S[(long long)j * N + i] - th * B[(long long)j * N + i], v);
        }
        p[0] = fma(v, v, p[0]);
        double den = th - hd[i];
        if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
        t[i] = v / den;
      }
      cta_sum4<NT>(p, 1, red);
      const double rn = sqrt(fmax(0.0, p[0]));
      if (threadIdx.x == 0) d2[r] = rn;
      if (!(rn < c.tol)) all = false;
      rmax = fmax(rmax, rn);
      if (!isfinite(rn) || !isfinite(th)) {
        st = FORTE_ERR_NUMERIC;
        all = true;
      }
    }
    __syncthreads();
    if (st == FORTE_ERR_NUMERIC) break;
    // end of the FP32 phase (a residual below tol there certifies nothing): restart
    // from the Ritz vectors with the FP64-class sigma
    // the Ritz vectors x_r = B u_r into W
    auto ritz_to_W = [&]() {
      for (int i = threadIdx.x; i < k * nr; i += NT) coef[i] = U[(i / nr) * BT_LD + perm[i % nr]];
      __syncthreads();
      cta_combine<NT>(B, k, N, coef, nr, W, N, N);
    };
    // restart the subspace from the vectors in W: orthonormalised (two Gram-Schmidt
    // passes), sigma recomputed in the current arithmetic
    auto restart_from_W = [&]() {
      for (long long i = threadIdx.x; i < (long long)nr * N; i += NT) B[i] = W[i];
      __syncthreads();
      k = nr;
      for (int r = 0; r < nr; ++r) {
        double *b = B + (long long)r * N;
        double nn = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
          if (r > 0) cta_dots<NT>(B, r, N, b, N, dots, red);
          nn = cta_orth_update<NT>(B, r, N, dots, b, N, red);
        }
        const double s = 1.0 / sqrt(fmax(nn, 1e-300));
        for (long long i = threadIdx.x; i < N; i += NT) b[i] *= s;
        __syncthreads();
      }
      for (int j = 0; j < k; ++j) sigma(B + (long long)j * N, S + (long long)j * N);
      build_G(0, k);
    };
    if (phase == AR_F32 && (all || rmax < c.tol1 || it >= p1_cap)) {
      ritz_to_W();
      phase = AR_DF;
      restart_from_W();
      continue;
    }
    if (all) {
      // Verified convergence: the residual above is formed from the stored basis and
      // its sigma, and a basis that has lost orthogonality over a long run can show
      // a small residual for a vector that is not an eigenvector (a combination of
      // nearly parallel basis vectors).  Each Ritz vector is therefore formed, its
      // sigma recomputed, and the residual of the normalised vector at its Rayleigh
      // quotient must meet tol; otherwise the subspace restarts from these vectors.
      ritz_to_W();
      bool verified = true;
      for (int r = 0; r < nr; ++r) {
        const double *x = W + (long long)r * N;
        double *sx = T + (long long)r * N;
        sigma(x, sx);
        double p[4] = {0.0, 0.0, 0.0, 0.0};
        for (long long i = threadIdx.x; i < N; i += NT) {
          p[0] = fma(x[i], x[i], p[0]);
          p[1] = fma(x[i], sx[i], p[1]);
        }
        cta_sum4<NT>(p, 2, red);
        const double xx = p[0], th = p[1] / fmax(xx, 1e-300);
        double q[4] = {0.0, 0.0, 0.0, 0.0};
        for (long long i = threadIdx.x; i < N; i += NT) {
          const double v = fma(-th, x[i], sx[i]);
          q[0] = fma(v, v, q[0]);
        }
        cta_sum4<NT>(q, 1, red);
        const double rn = sqrt(fmax(0.0, q[0]) / fmax(xx, 1e-300));
        if (threadIdx.x == 0) {
          wv[r] = th;
          d2[r] = rn;
        }
        if (!(rn < c.tol) || !isfinite(th)) verified = false;
      }
      __syncthreads();
      if (verified) {
        st = FORTE_OK;
        break;
      }
      restart_from_W();
      continue;
    }
    int nnew = 0;
    for (int r = 0; r < nr; ++r) nnew += (d2[r] < c.tol) ? 0 : 1;
    if (k + nnew > maxsub && k > keep) {
      // collapse onto the lowest `keep` Ritz vectors
      for (int i = threadIdx.x; i < k * keep; i += NT) coef[i] = U[(i / keep) * BT_LD + perm[i % keep]];
      __syncthreads();
      cta_combine<NT>(B, k, N, coef, keep, W, N, N);
      for (long long i = threadIdx.x; i < (long long)keep * N; i += NT) B[i] = W[i];
      __syncthreads();
      cta_combine<NT>(S, k, N, coef, keep, W, N, N);
      for (long long i = threadIdx.x; i < (long long)keep * N; i += NT) S[i] = W[i];
      for (int i = threadIdx.x; i < BT_MAXK * BT_LD; i += NT) G[i] = 0.0;
      __syncthreads();
      if (threadIdx.x < keep) G[threadIdx.x * BT_LD + threadIdx.x] = wv[threadIdx.x];
      __syncthreads();
      k = keep;
    }
    const int k_old = k;
    for (int r = 0; r < nr; ++r) {
      if (d2[r] < c.tol || k >= maxsub) continue;
      double *t = T + (long long)r * N;
      double *b = B + (long long)k * N;
      double p[4] = {0.0, 0.0, 0.0, 0.0};
      for (long long i = threadIdx.x; i < N; i += NT) {
        b[i] = t[i];
        p[0] = fma(t[i], t[i], p[0]);
      }
      cta_sum4<NT>(p, 1, red);
      const double n0 = p[0];
      cta_dots<NT>(B, k, N, b, N, dots, red);
      double proj = 0.0;
      for (int i = 0; i < k; ++i) proj += dots[i] * dots[i];
      double nn = cta_orth_update<NT>(B, k, N, dots, b, N, red);
      if (!(n0 - proj >= 0.5 * n0)) {  // second pass (Daniel-Gragg-Kaufman-Stewart)
        cta_dots<NT>(B, k, N, b, N, dots, red);
        nn = cta_orth_update<NT>(B, k, N, dots, b, N, red);
      }
      if (!(nn > 1e-24 * n0) || !(nn > 0.0)) continue;
      const double s = 1.0 / sqrt(nn);
      for (long long i = threadIdx.x; i < N; i += NT) b[i] *= s;
      __syncthreads();
      ++k;
    }
    if (k == k_old) break;  // no new direction: keep the current Ritz values
    for (int j = k_old; j < k; ++j) sigma(B + (long long)j * N, S + (long long)j * N);
    build_G(k_old, k);
  }
  if (threadIdx.x < nr) {
    c.E[c.eoff[q] + threadIdx.x] = wv[threadIdx.x];
    c.rn[c.eoff[q] + threadIdx.x] = d2[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    c.iters[c.gidx[q]] = min(it, c.max_iter);
    c.status[c.gidx[q]] = st;
  }
}

// --------------------------------------------------------------- host side
struct ClassHost {
  int n, na, nb;
  std::vector<int> probs;  // indices into the batch
  BClass dev{};
  int NT = 256, TJ = 32;
  double probe_ms = 0.0, single_ms = 0.0;
  int path = 0;  // 0: class launch, 1: single-problem path
  long long work_doubles = 0;
};

struct TuneRecord {
  int n, na, nb, threads, tile;
  double sigma_ms;        // one per-CTA sigma of the class's first problems (one CTA each)
  int path;               // 0: class launch, 1: single-problem path
  double single_iter_ms;  // one Davidson iteration of one problem on the single-problem path
  int problems, ctas_per_sm;
};
std::mutex g_tune_mu;
std::vector<TuneRecord> g_tune;
int g_stats[3] = {0, 0, 0};  // last batch: problems in class launches, on the single-problem path, retried

template <int NT>
cudaError_t launch_class(const BClass &c, size_t smem, cudaStream_t st) {
  k_batch_davidson<NT><<<c.P, NT, smem, st>>>(c);
  return cudaGetLastError();
}
// Dynamic shared memory up to the device maximum for every block size (set once,
// before any launch or capture).
cudaError_t allow_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_davidson<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_davidson<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_davidson<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}
cudaError_t launch_any(int NT, const BClass &c, size_t smem, cudaStream_t st) {
  if (NT == 128) return launch_class<128>(c, smem, st);
  if (NT == 512) return launch_class<512>(c, smem, st);
  return launch_class<256>(c, smem, st);
}

size_t class_smem(const BClass &c, int ar, int TJ) {
  size_t s = sigma_bytes(ar, c.nkA, c.nkB, c.npair, c.NB, TJ);
  if (ar == AR_F32) s = std::max(s, sigma_bytes(AR_DF, c.nkA, c.nkB, c.npair, c.NB, TJ));
  return DV_BYTES + s;
}

}  // namespace
}  // namespace forte

using namespace forte;

extern "C" int forte_batch_solve(int nprob, const int *norb, const int *nalpha, const int *nbeta,
                                 const int *nroots, const double *const *h, const double *const *eri,
                                 int precision, double tol, int max_iter, double *E_out, int *status_out) {
  clear_error();
  if (nprob < 0 || (nprob > 0 && (!norb || !nalpha || !nbeta || !nroots || !h || !eri || !E_out))) {
    set_error("forte_batch_solve: bad arguments");
    return FORTE_ERR_ARG;
  }
  if (precision != FORTE_FP64 && precision != FORTE_TF32 && precision != FORTE_BF16X2 && precision != FORTE_DF32 &&
      precision != FORTE_OZ64) {
    set_error("forte_batch_solve: unknown precision %d", precision);
    return FORTE_ERR_ARG;
  }
  if (!(tol > 0)) {
    set_error("forte_batch_solve: tol must be > 0");
    return FORTE_ERR_ARG;
  }
  if (max_iter <= 0) max_iter = 400;
  if (nprob == 0) return FORTE_OK;
  std::vector<long long> eoff(nprob + 1, 0), ndet(nprob, 0);
  for (int i = 0; i < nprob; ++i) {
    if (norb[i] < 1 || norb[i] > 16 || nroots[i] < 1 || nalpha[i] < 0 || nbeta[i] < 0 || nalpha[i] > norb[i] ||
        nbeta[i] > norb[i] || !h[i] || !eri[i]) {
      set_error("forte_batch_solve: bad sizes or NULL integrals for problem %d", i);
      return FORTE_ERR_ARG;
    }
    eoff[i + 1] = eoff[i] + nroots[i];
    long long a = 1, b = 1;
    for (int k = 1; k <= nalpha[i]; ++k) a = a * (norb[i] - nalpha[i] + k) / k;
    for (int k = 1; k <= nbeta[i]; ++k) b = b * (norb[i] - nbeta[i] + k) / k;
    ndet[i] = a * b;
    if (nroots[i] > ndet[i]) {
      set_error("forte_batch_solve: problem %d asks for %d roots of a %lld-determinant space", i, nroots[i], ndet[i]);
      return FORTE_ERR_ARG;
    }
  }
  const int mode = precision == FORTE_FP64 ? 0 : ((precision == FORTE_TF32 || precision == FORTE_BF16X2) ? 1 : 2);
  int dev = 0;
  FORTE_CUDA_TRY(cudaGetDevice(&dev));
  int smem_optin = 0, nsm = 0;
  FORTE_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  FORTE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int worst = FORTE_OK;
  std::string first_msg;
  auto note = [&](int i, int rc, const char *msg) {
    if (status_out) status_out[i] = rc;
    if (rc > worst) worst = rc;
    if (rc && first_msg.empty()) first_msg = "problem " + std::to_string(i) + ": " + msg;
  };

  // ---- classes; problems beyond the in-CTA limits go to the single-problem path
  std::vector<ClassHost> classes;
  std::vector<int> singles;
  for (int i = 0; i < nprob; ++i) {
    if (ndet[i] > BT_MAX_DET || nroots[i] > BT_MAX_ROOTS) {
      singles.push_back(i);
      continue;
    }
    size_t c = 0;
    for (; c < classes.size(); ++c)
      if (classes[c].n == norb[i] && classes[c].na == nalpha[i] && classes[c].nb == nbeta[i]) break;
    if (c == classes.size()) {
      ClassHost ch;
      ch.n = norb[i];
      ch.na = nalpha[i];
      ch.nb = nbeta[i];
      classes.push_back(ch);
    }
    classes[c].probs.push_back(i);
  }

  // ---- host tables per problem (strings, lists, CSR of the same-spin Hamiltonians)
  struct Pool {
    std::vector<char> host;
    size_t used = 0;
    size_t add(const void *src, size_t bytes) {
      const size_t at = (used + 255) & ~(size_t)255;
      if (host.size() < at + bytes) host.resize(std::max(host.size() * 2, at + bytes));
      if (src && bytes) memcpy(host.data() + at, src, bytes);
      used = at + bytes;
      return at;
    }
  } pool;
  struct Off {
    size_t listA, listB, ptrA, colA, ptrB, colB, valA, valB, valA32, valB32, valA2, valB2, diagA, diagB, Wd, strB,
        gp, gp32, gp2, nroots, eoff, gidx, woff;
  };
  std::vector<Off> offs(classes.size());
  long long work_total = 0;
  std::vector<std::vector<long long>> woffs(classes.size());
  for (size_t ci = 0; ci < classes.size(); ++ci) {
    ClassHost &ch = classes[ci];
    const int P = (int)ch.probs.size();
    std::vector<double> vA, vB, dA, dB, Wd, gp;
    std::vector<float> vA32, vB32, gp32;
    std::vector<float> vA2, vB2, gp2;
    forte_ctx tmpl;
    int n = ch.n, np = n * (n + 1) / 2;
    long long nnzA = -1, nnzB = -1;
    for (int pi = 0; pi < P; ++pi) {
      const int i = ch.probs[pi];
      forte_ctx t;
      t.n = n;
      t.na = ch.na;
      t.nb = ch.nb;
      t.npair = np;
      t.same_strings = (ch.na == ch.nb);
      t.h.assign(h[i], h[i] + n * n);
      t.eri.assign(eri[i], eri[i] + (size_t)n * n * n * n);
      for (double x : t.h)
        if (!std::isfinite(x)) { set_error("forte_batch_solve: problem %d: h contains NaN/Inf", i); return FORTE_ERR_ARG; }
      for (double x : t.eri)
        if (!std::isfinite(x)) { set_error("forte_batch_solve: problem %d: eri contains NaN/Inf", i); return FORTE_ERR_ARG; }
      int rc = build_spin_tables(&t);
      if (rc) return rc;
      if (t.same_strings) t.sh[1] = t.sh[0];
      const SpinHost &A = t.sh[0], &Bs = t.sh[1];
      if (pi == 0) {
        tmpl.sh[0] = A;
        tmpl.sh[1] = Bs;
        nnzA = (long long)A.csr_col.size();
        nnzB = (long long)Bs.csr_col.size();
      } else if ((long long)A.csr_col.size() != nnzA || (long long)Bs.csr_col.size() != nnzB ||
                 A.csr_col != tmpl.sh[0].csr_col || Bs.csr_col != tmpl.sh[1].csr_col) {
        set_error("forte_batch_solve: internal: same-spin sparsity differs inside a class");
        return FORTE_ERR_ARG;
      }
      vA.insert(vA.end(), A.csr_val.begin(), A.csr_val.end());
      vB.insert(vB.end(), Bs.csr_val.begin(), Bs.csr_val.end());
      dA.insert(dA.end(), A.diag.begin(), A.diag.end());
      dB.insert(dB.end(), Bs.diag.begin(), Bs.diag.end());
      for (long long ia = 0; ia < A.N; ++ia)
        for (int j = 0; j < n; ++j) {
          double v = 0.0;
          for (int ii = 0; ii < n; ++ii)
            if ((A.str[ia] >> ii) & 1u) v += t.eri[(((size_t)ii * n + ii) * n + j) * n + j];
          Wd.push_back(v);
        }
      std::vector<double> g((size_t)np * np);
      for (int p = 0; p < n; ++p)
        for (int qq = 0; qq <= p; ++qq)
          for (int r = 0; r < n; ++r)
            for (int s = 0; s <= r; ++s)
              g[(size_t)(p * (p + 1) / 2 + qq) * np + (r * (r + 1) / 2 + s)] =
                  t.eri[(((size_t)p * n + qq) * n + r) * n + s];
      gp.insert(gp.end(), g.begin(), g.end());
    }
    auto split = [](const std::vector<double> &x, std::vector<float> &f32, std::vector<float> &f2) {
      f32.resize(x.size());
      f2.resize(2 * x.size());
      for (size_t k = 0; k < x.size(); ++k) {
        f32[k] = (float)x[k];
        const float hh = (float)x[k];
        f2[2 * k] = hh;
        f2[2 * k + 1] = (float)(x[k] - (double)hh);
      }
    };
    split(vA, vA32, vA2);
    split(vB, vB32, vB2);
    split(gp, gp32, gp2);
    const SpinHost &A = tmpl.sh[0], &Bs = tmpl.sh[1];
    Off &o = offs[ci];
    o.listA = pool.add(A.list.data(), sizeof(Repl) * A.list.size());
    o.listB = pool.add(Bs.list.data(), sizeof(Repl) * Bs.list.size());
    o.ptrA = pool.add(A.csr_ptr.data(), sizeof(int) * A.csr_ptr.size());
    o.colA = pool.add(A.csr_col.data(), sizeof(int) * A.csr_col.size());
    o.ptrB = pool.add(Bs.csr_ptr.data(), sizeof(int) * Bs.csr_ptr.size());
    o.colB = pool.add(Bs.csr_col.data(), sizeof(int) * Bs.csr_col.size());
    o.valA = pool.add(vA.data(), sizeof(double) * vA.size());
    o.valB = pool.add(vB.data(), sizeof(double) * vB.size());
    o.valA32 = pool.add(vA32.data(), sizeof(float) * vA32.size());
    o.valB32 = pool.add(vB32.data(), sizeof(float) * vB32.size());
    o.valA2 = pool.add(vA2.data(), sizeof(float) * vA2.size());
    o.valB2 = pool.add(vB2.data(), sizeof(float) * vB2.size());
    o.diagA = pool.add(dA.data(), sizeof(double) * dA.size());
    o.diagB = pool.add(dB.data(), sizeof(double) * dB.size());
    o.Wd = pool.add(Wd.data(), sizeof(double) * Wd.size());
    o.strB = pool.add(Bs.str.data(), sizeof(uint32_t) * Bs.str.size());
    o.gp = pool.add(gp.data(), sizeof(double) * gp.size());
    o.gp32 = pool.add(gp32.data(), sizeof(float) * gp32.size());
    o.gp2 = pool.add(gp2.data(), sizeof(float) * gp2.size());
    std::vector<int> nr(P), eo(P);
    std::vector<long long> wo(P);
    std::vector<int> gi(P);
    const long long N = A.N * Bs.N;
    for (int pi = 0; pi < P; ++pi) {
      const int i = ch.probs[pi];
      nr[pi] = nroots[i];
      eo[pi] = (int)eoff[i];
      gi[pi] = i;
      const int maxsub = (int)std::min<long long>(std::min(12 * nroots[i], BT_MAXK), N);
      const int keep = std::max(nroots[i], std::min(2 * nroots[i], maxsub - 1));
      wo[pi] = work_total;
      work_total += (long long)(2 * maxsub + nroots[i] + std::max(keep, nroots[i]) + 4) * N;
      work_total = (work_total + 31) & ~31LL;
    }
    o.nroots = pool.add(nr.data(), sizeof(int) * P);
    o.eoff = pool.add(eo.data(), sizeof(int) * P);
    o.gidx = pool.add(gi.data(), sizeof(int) * P);
    o.woff = pool.add(wo.data(), sizeof(long long) * P);
    BClass &c = ch.dev;
    c.n = n;
    c.nkA = A.nk;
    c.nkB = Bs.nk;
    c.npair = np;
    c.P = P;
    c.NA = A.N;
    c.NB = Bs.N;
    c.N = N;
    c.nnzA = nnzA;
    c.nnzB = nnzB;
    c.tol = tol;
    c.tol1 = std::max(tol, 3e-4);
    c.max_iter = max_iter;
    c.mode = mode;
  }
  const long long nE = eoff[nprob];
  const size_t off_E = pool.add(nullptr, sizeof(double) * nE);
  const size_t off_rn = pool.add(nullptr, sizeof(double) * nE);
  const size_t off_it = pool.add(nullptr, sizeof(int) * nprob);
  const size_t off_st = pool.add(nullptr, sizeof(int) * nprob);
  const size_t table_bytes = pool.used;
  const size_t total_bytes = ((table_bytes + 255) & ~(size_t)255) + sizeof(double) * (size_t)work_total;

  // ---- the single-problem path (problems beyond the in-CTA limits and classes the
  // autotuner sends there), on worker threads with their own streams
  std::mutex mu;
  std::atomic<int> next_single(0);
  auto single_worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t sx = nullptr;
    if (cudaStreamCreateWithFlags(&sx, cudaStreamNonBlocking) != cudaSuccess) sx = nullptr;
    for (;;) {
      const int kk = next_single.fetch_add(1);
      if (kk >= (int)singles.size()) break;
      const int i = singles[kk];
      int rc = FORTE_OK;
      std::string msg;
      forte_ctx *ctx = forte_cas_create(norb[i], nalpha[i], nbeta[i], h[i], eri[i]);
      if (!ctx) rc = FORTE_ERR_ARG;
      if (!rc && sx) rc = forte_set_stream(ctx, sx);
      if (!rc) rc = forte_set_precision(ctx, precision);
      if (!rc) rc = forte_set_davidson_params(ctx, 12, 2, max_iter, 1e-8);
      if (!rc) rc = forte_davidson(ctx, nroots[i], tol);
      if (rc == FORTE_OK || rc == FORTE_ERR_NOT_CONVERGED) {
        const int rc2 = forte_get_roots(ctx, E_out + eoff[i], nullptr, nullptr, nullptr);
        if (rc2) rc = rc2;
      }
      if (rc) msg = forte_last_error();
      forte_destroy(ctx);
      std::lock_guard<std::mutex> lock(mu);
      note(i, rc, msg.c_str());
    }
    if (sx) {
      cudaStreamSynchronize(sx);
      cudaStreamDestroy(sx);
    }
  };
  // Host wall time (ms) of one Davidson iteration of problem i on the single-problem
  // path: forte_davidson capped at 2 and at 6 iterations after a 1-iteration run
  // that builds the lazy tables; (t6 - t2) / 4 leaves out the set-up and the first
  // sigma builds and keeps the per-iteration launch and host costs.
  auto single_iter_ms = [&](int i) -> double {
    forte_ctx *ctx = forte_cas_create(norb[i], nalpha[i], nbeta[i], h[i], eri[i]);
    if (!ctx) return INFINITY;
    const int cap[3] = {1, 2, 6};
    double t[3] = {0.0, 0.0, 0.0};
    bool ok = forte_set_precision(ctx, precision) == FORTE_OK;
    for (int r = 0; r < 3 && ok; ++r) {
      ok = forte_set_davidson_params(ctx, 12, 2, cap[r], 1e-8) == FORTE_OK;
      const auto t0 = std::chrono::steady_clock::now();
      const int rc = ok ? forte_davidson(ctx, nroots[i], 1e-14) : FORTE_ERR_ARG;
      t[r] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      ok = (rc == FORTE_OK || rc == FORTE_ERR_NOT_CONVERGED);
    }
    forte_destroy(ctx);
    clear_error();
    return ok ? std::max(1e-3, (t[2] - t[1]) / 4.0) : INFINITY;
  };

  // ---- one pooled device allocation for the batch
  char *dbuf = nullptr;
  if (!classes.empty()) {
    cudaError_t e = cudaMalloc(&dbuf, total_bytes);
    if (e != cudaSuccess) {
      set_error("forte_batch_solve: cudaMalloc(%zu) failed: %s", total_bytes, cudaGetErrorString(e));
      return FORTE_ERR_ALLOC;
    }
  }
  struct Guard {
    char *p;
    std::vector<cudaStream_t> s;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    ~Guard() {
      if (ge) cudaGraphExecDestroy(ge);
      if (g) cudaGraphDestroy(g);
      for (auto x : s) cudaStreamDestroy(x);
      if (p) cudaFree(p);
    }
  } guard{dbuf, {}};
  double *dwork = (double *)(dbuf + ((table_bytes + 255) & ~(size_t)255));
  if (!classes.empty()) {
    FORTE_CUDA_TRY(cudaMemcpy(dbuf, pool.host.data(), table_bytes, cudaMemcpyHostToDevice));
    for (int s = 0; s < (int)classes.size(); ++s) {
      cudaStream_t x = nullptr;
      FORTE_CUDA_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
      guard.s.push_back(x);
    }
  }
  for (size_t ci = 0; ci < classes.size(); ++ci) {
    BClass &c = classes[ci].dev;
    const Off &o = offs[ci];
    c.listA = (const Repl *)(dbuf + o.listA);
    c.listB = (const Repl *)(dbuf + o.listB);
    c.ptrA = (const int *)(dbuf + o.ptrA);
    c.colA = (const int *)(dbuf + o.colA);
    c.ptrB = (const int *)(dbuf + o.ptrB);
    c.colB = (const int *)(dbuf + o.colB);
    c.valA = (const double *)(dbuf + o.valA);
    c.valB = (const double *)(dbuf + o.valB);
    c.valA32 = (const float *)(dbuf + o.valA32);
    c.valB32 = (const float *)(dbuf + o.valB32);
    c.valA2 = (const float2 *)(dbuf + o.valA2);
    c.valB2 = (const float2 *)(dbuf + o.valB2);
    c.diagA = (const double *)(dbuf + o.diagA);
    c.diagB = (const double *)(dbuf + o.diagB);
    c.Wd = (const double *)(dbuf + o.Wd);
    c.strB = (const uint32_t *)(dbuf + o.strB);
    c.gp = (const double *)(dbuf + o.gp);
    c.gp32 = (const float *)(dbuf + o.gp32);
    c.gp2 = (const float2 *)(dbuf + o.gp2);
    c.nroots = (const int *)(dbuf + o.nroots);
    c.eoff = (const int *)(dbuf + o.eoff);
    c.gidx = (const int *)(dbuf + o.gidx);
    c.woff = (const long long *)(dbuf + o.woff);
    c.work = dwork;
    c.E = (double *)(dbuf + off_E);
    c.rn = (double *)(dbuf + off_rn);
    c.iters = (int *)(dbuf + off_it);
    c.status = (int *)(dbuf + off_st);
  }

  if (!classes.empty()) FORTE_CUDA_TRY(allow_smem(smem_optin));
  // ---- autotuner: threads per CTA x beta tile width, per class, on the arithmetic
  // that carries most sigma builds (FP32 in the mixed modes)
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
  }
  for (size_t ci = 0; ci < classes.size(); ++ci) {
    ClassHost &ch = classes[ci];
    BClass probe = ch.dev;
    const int ar = mode == 0 ? AR_F64 : (mode == 1 ? AR_F32 : AR_DF);
    probe.P = std::min(ch.dev.P, nsm);
    probe.probe = 1;
    probe.mode = mode == 0 ? 0 : (mode == 1 ? 1 : 2);
    const int nts[3] = {128, 256, 512};
    const int tjs[3] = {16, 32, 64};
    double best = INFINITY;
    bool any = false;
    cudaEvent_t a, b;
    FORTE_CUDA_TRY(cudaEventCreate(&a));
    FORTE_CUDA_TRY(cudaEventCreate(&b));
    for (int tj : tjs)
      for (int nt : nts) {
        const size_t smem = class_smem(ch.dev, ar, tj);
        if (smem > (size_t)smem_optin) continue;
        probe.TJ = tj;
        FORTE_CUDA_TRY(cudaEventRecord(a, guard.s[ci]));
        cudaError_t e = launch_any(nt, probe, smem, guard.s[ci]);
        if (e != cudaSuccess) continue;
        FORTE_CUDA_TRY(cudaEventRecord(b, guard.s[ci]));
        FORTE_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        FORTE_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        any = true;
        if (ms < best) {
          best = ms;
          ch.NT = nt;
          ch.TJ = tj;
        }
      }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!any) {
      set_error("forte_batch_solve: no kernel configuration fits class (%d, %d, %d)", ch.n, ch.na, ch.nb);
      return FORTE_ERR_ARG;
    }
    ch.probe_ms = best;
    ch.dev.TJ = ch.TJ;
    ch.dev.probe = 0;
    // path: one class launch costs about probe_ms per sigma round for every wave of
    // resident CTAs; the single-problem path costs single_iter_ms per problem and
    // iteration (no credit for overlap between workers)
    int per_sm = 0;
    cudaError_t oe = cudaSuccess;
    const size_t smem = class_smem(ch.dev, ar, ch.TJ);
    if (ch.NT == 128) oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_davidson<128>, 128, smem);
    else if (ch.NT == 512) oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_davidson<512>, 512, smem);
    else oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_davidson<256>, 256, smem);
    if (oe != cudaSuccess || per_sm < 1) per_sm = 1;
    const int P = ch.dev.P;
    const double waves = std::ceil((double)P / (double)(per_sm * nsm));
    ch.single_ms = single_iter_ms(ch.probs[0]);
    ch.path = (best * waves <= (double)P * ch.single_ms) ? 0 : 1;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.push_back(TuneRecord{ch.n, ch.na, ch.nb, ch.NT, ch.TJ, best, ch.path, ch.single_ms, P, per_sm});
  }
  for (const ClassHost &ch : classes)
    if (ch.path == 1) singles.insert(singles.end(), ch.probs.begin(), ch.probs.end());

  // ---- the solve: one launch per class-launch class on its own stream, captured
  // as one graph and launched without waiting; the single-problem path runs on
  // the worker threads meanwhile (their kernels take the SMs the classes leave)
  std::vector<size_t> launched;
  int n_launched = 0, n_retried = 0;
  const int n_single = (int)singles.size();
  for (size_t ci = 0; ci < classes.size(); ++ci)
    if (classes[ci].path == 0) {
      launched.push_back(ci);
      n_launched += (int)classes[ci].probs.size();
    }
  cudaError_t ce = cudaSuccess;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  if (!launched.empty()) {
    cudaStream_t s0 = guard.s[launched[0]];
    FORTE_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    FORTE_CUDA_TRY(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    ce = cudaEventRecord(fork, s0);
    // the largest class first: its CTAs run longest
    std::vector<size_t> order = launched;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return classes[x].dev.N > classes[y].dev.N; });
    for (size_t oi = 0; oi < order.size() && ce == cudaSuccess; ++oi) {
      const size_t ci = order[oi];
      cudaStream_t sx = guard.s[ci];
      if (sx != s0) ce = cudaStreamWaitEvent(sx, fork, 0);
      const int ar = mode == 0 ? AR_F64 : (mode == 1 ? AR_F32 : AR_DF);
      if (ce == cudaSuccess) ce = launch_any(classes[ci].NT, classes[ci].dev, class_smem(classes[ci].dev, ar, classes[ci].TJ), sx);
      if (ce == cudaSuccess && sx != s0) {
        cudaEvent_t ev;
        ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (ce == cudaSuccess) {
          joins.push_back(ev);
          ce = cudaEventRecord(ev, sx);
          if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s0, ev, 0);
        }
      }
    }
    cudaError_t ce2 = cudaStreamEndCapture(s0, &guard.g);
    if (ce == cudaSuccess) ce = ce2;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&guard.ge, guard.g, 0);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(guard.ge, s0);
  }
  {
    std::vector<std::thread> workers;
    for (int w = 0; w < std::min<int>(BT_WORKERS, (int)singles.size()); ++w) workers.emplace_back(single_worker);
    for (auto &x : workers) x.join();
  }
  if (!launched.empty()) {
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(guard.s[launched[0]]);
    for (auto ev : joins) cudaEventDestroy(ev);
    cudaEventDestroy(fork);
    if (ce != cudaSuccess) {
      set_error("forte_batch_solve: batched launch failed: %s", cudaGetErrorString(ce));
      return FORTE_ERR_CUDA;
    }
    std::vector<double> Eh(nE);
    std::vector<int> sth(nprob, FORTE_OK);
    FORTE_CUDA_TRY(cudaMemcpy(Eh.data(), dbuf + off_E, sizeof(double) * nE, cudaMemcpyDeviceToHost));
    FORTE_CUDA_TRY(cudaMemcpy(sth.data(), dbuf + off_st, sizeof(int) * nprob, cudaMemcpyDeviceToHost));
    // a problem whose in-CTA Davidson-Liu did not converge is solved again on the
    // single-problem path, whose solver continues a stalled Davidson-Liu with
    // Jacobi-Davidson
    std::vector<int> retry;
    {
      std::lock_guard<std::mutex> lock(mu);
      for (size_t ci : launched)
        for (int i : classes[ci].probs) {
          for (int r = 0; r < nroots[i]; ++r) E_out[eoff[i] + r] = Eh[eoff[i] + r];
          if (sth[i] == FORTE_ERR_NOT_CONVERGED) {
            retry.push_back(i);
            continue;
          }
          note(i, sth[i], sth[i] ? "non-finite residual" : "");
        }
    }
    if (!retry.empty()) {
      singles = retry;
      next_single = 0;
      std::vector<std::thread> workers;
      for (int w = 0; w < std::min<int>(BT_WORKERS, (int)singles.size()); ++w) workers.emplace_back(single_worker);
      for (auto &x : workers) x.join();
    }
    n_retried = (int)retry.size();
  }

  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_stats[0] = n_launched;
    g_stats[1] = n_single;
    g_stats[2] = n_retried;
  }
  if (worst) set_error("%s", first_msg.c_str());
  return worst;
}

extern "C" int forte_batch_stats(int *class_launch, int *single_path, int *retried) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (class_launch) *class_launch = g_stats[0];
  if (single_path) *single_path = g_stats[1];
  if (retried) *retried = g_stats[2];
  return FORTE_OK;
}

extern "C" int forte_batch_tuning(int max_classes, int *nclass, int *norb, int *nalpha, int *nbeta, int *threads,
                                  int *tile, double *sigma_ms, int *path, double *single_iter_ms, int *problems,
                                  int *ctas_per_sm) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (nclass) *nclass = (int)g_tune.size();
  for (int i = 0; i < (int)g_tune.size() && i < max_classes; ++i) {
    if (norb) norb[i] = g_tune[i].n;
    if (nalpha) nalpha[i] = g_tune[i].na;
    if (nbeta) nbeta[i] = g_tune[i].nb;
    if (threads) threads[i] = g_tune[i].threads;
    if (tile) tile[i] = g_tune[i].tile;
    if (sigma_ms) sigma_ms[i] = g_tune[i].sigma_ms;
    if (path) path[i] = g_tune[i].path;
    if (single_iter_ms) single_iter_ms[i] = g_tune[i].single_iter_ms;
    if (problems) problems[i] = g_tune[i].problems;
    if (ctas_per_sm) ctas_per_sm[i] = g_tune[i].ctas_per_sm;
  }
  return FORTE_OK;
}
