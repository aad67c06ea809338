// Davidson-Liu building blocks on long vectors (step a7), for FP64 vectors and
// for the FP32 vectors of the reduced-precision phase.  Each kernel streams its
// operands once; reductions go through per-block partial sums (FP64) and a second
// pass, so results do not depend on atomic ordering.  FP32 kernels accumulate in
// FP32 within a warp and in FP64 across warps and blocks.
#include "forte_internal.h"

namespace forte {

constexpr int VK_THREADS = 256;
constexpr int VK_EPT = 16;  // elements per thread per block
constexpr long long VK_CHUNK = (long long)VK_THREADS * VK_EPT;
constexpr int VK_MAXV = 64;  // vectors handled by one multidot / update launch

static inline unsigned vk_blocks(long long n) { return (unsigned)((n + VK_CHUNK - 1) / VK_CHUNK); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread returns the total.  red must hold 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  return red[0];
}

// Block-wide sum of per-thread values of type T: warp sums in T, the sum over
// warps in FP64 (one warp); every thread returns the total.  red holds 32 doubles.
template <typename T>
__device__ __forceinline__ double block_sum_t(T v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = (double)v;
  __syncthreads();
  double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  return red[0];
}

// Second pass of a reduction, fused into the kernel that writes the partials: every
// block publishes its partials part[block][0..m) and counts itself in; the last block
// to arrive sums part[b][c] over b (strided by thread, then block_sum: the order of
// a separate 256-thread pass) into out[c] and resets the counter for the next
// launch on the stream.  No block waits for another.
__device__ __forceinline__ void last_block_sums(const double *part, int m, double *__restrict__ out,
                                                unsigned *counter, double *red) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nblk = (int)gridDim.x;
  for (int c = 0; c < m; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(part + (long long)b * m + c);
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[c] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// part[block][i] = sum over the block's chunk of V_i . x   (i < nv)
template <typename T>
__global__ void __launch_bounds__(VK_THREADS) k_multidot(const T *__restrict__ V, int nv, long long ld,
                                                         const T *__restrict__ x, long long n,
                                                         double *__restrict__ part, double *__restrict__ out,
                                                         unsigned *counter) {
  __shared__ double red[32];
  const long long base = (long long)blockIdx.x * VK_CHUNK + threadIdx.x;
  T xr[VK_EPT];
#pragma unroll
  for (int k = 0; k < VK_EPT; ++k) {
    long long j = base + (long long)k * VK_THREADS;
    xr[k] = (j < n) ? x[j] : T(0);
  }
  for (int i = 0; i < nv; ++i) {
    const T *v = V + (long long)i * ld;
    T a = 0;
#pragma unroll
    for (int k = 0; k < VK_EPT; ++k) {
      long long j = base + (long long)k * VK_THREADS;
      if (j < n) a += v[j] * xr[k];
    }
    const double at = block_sum_t<T>(a, red);
    if (threadIdx.x == 0) part[(long long)blockIdx.x * nv + i] = at;
  }
  last_block_sums(part, nv, out, counter, red);
}

// out_{c0+c} = sum_i coef[i*ncomb + c0 + c] V_i  for c < NC.  NC is a template
// parameter: the FP64 pipe of this GPU is narrow enough that issuing
// predicated-off multiply-adds for unused outputs would dominate the kernel.
template <int NC, typename T>
__global__ void __launch_bounds__(VK_THREADS) k_combine(const T *__restrict__ V, int nv, long long ld,
                                                        const double *__restrict__ coef, int ncomb, int c0,
                                                        T *__restrict__ out, long long ldo, long long n) {
  __shared__ T sc[VK_MAXV * NC];
  for (int i = threadIdx.x; i < nv * NC; i += blockDim.x) sc[i] = (T)coef[(i / NC) * ncomb + c0 + i % NC];
  __syncthreads();
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0;
#pragma unroll 4
    for (int i = 0; i < nv; ++i) {
      const T v = V[(long long)i * ld + j];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += sc[i * NC + c] * v;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) out[(long long)(c0 + c) * ldo + j] = acc[c];
  }
}

// r = sum_i u_i S_i - theta sum_i u_i B_i ;  t = r / (theta - hdiag) (guarded);
// part[block] = sum r^2 over the block's chunk.
template <typename T>
__global__ void __launch_bounds__(VK_THREADS) k_residual_precond(
    const T *__restrict__ B, const T *__restrict__ S, int k, long long ld,
    const double *__restrict__ u, double theta, const double *__restrict__ hd, double guard,
    T *__restrict__ t, long long n, double *__restrict__ part, double *__restrict__ out, unsigned *counter) {
  __shared__ double red[32];
  __shared__ T su[VK_MAXV];
  for (int i = threadIdx.x; i < k; i += blockDim.x) su[i] = (T)u[i];
  __syncthreads();
  const long long base = (long long)blockIdx.x * VK_CHUNK + threadIdx.x;
  const T th = (T)theta;
  T rr = 0;
#pragma unroll 4
  for (int e = 0; e < VK_EPT; ++e) {
    long long j = base + (long long)e * VK_THREADS;
    if (j >= n) break;
    T hx = 0, x = 0;
    for (int i = 0; i < k; ++i) {
      hx += su[i] * S[(long long)i * ld + j];
      x += su[i] * B[(long long)i * ld + j];
    }
    const T r = hx - th * x;
    rr += r * r;
    double den = theta - hd[j];
    if (fabs(den) < guard) den = (den >= 0.0) ? guard : -guard;
    t[j] = r / (T)den;
  }
  const double rt = block_sum_t<T>(rr, red);
  if (threadIdx.x == 0) part[blockIdx.x] = rt;
  last_block_sums(part, 1, out, counter, red);
}

// t_out = t_in - sum_i c_i B_i ; part[block][i] = B_i . t_out (i < k), part[block][k] = |t_out|^2.
// Without DOTS the B_i . t_out are not formed (a second read of every B_i) and part
// holds zeros there.  c == nullptr: no update (t_out = t_in; the B_i are read once,
// for the dots).
template <typename T, bool DOTS>
__global__ void __launch_bounds__(VK_THREADS) k_orth_update(const T *__restrict__ Bm, int k,
                                                            long long ld, const double *__restrict__ c,
                                                            const T *t_in, T *t_out, long long n,
                                                            double *__restrict__ part, double *__restrict__ out,
                                                            unsigned *counter) {
  __shared__ double red[32];
  __shared__ T sc[VK_MAXV];
  const int ku = c ? k : 0;  // vectors to subtract
  for (int i = threadIdx.x; i < ku; i += blockDim.x) sc[i] = (T)c[i];
  __syncthreads();
  const long long base = (long long)blockIdx.x * VK_CHUNK + threadIdx.x;
  T tr[VK_EPT];
#pragma unroll
  for (int e = 0; e < VK_EPT; ++e) {
    long long j = base + (long long)e * VK_THREADS;
    tr[e] = (j < n) ? t_in[j] : T(0);
  }
  for (int i = 0; i < ku; ++i) {
    const T *b = Bm + (long long)i * ld;
#pragma unroll
    for (int e = 0; e < VK_EPT; ++e) {
      long long j = base + (long long)e * VK_THREADS;
      if (j < n) tr[e] -= sc[i] * b[j];
    }
  }
  T nn = 0;
#pragma unroll
  for (int e = 0; e < VK_EPT; ++e) {
    long long j = base + (long long)e * VK_THREADS;
    if (j < n) {
      t_out[j] = tr[e];
      nn += tr[e] * tr[e];
    }
  }
  if (DOTS) {
    for (int i = 0; i < k; ++i) {
      const T *b = Bm + (long long)i * ld;
      T a = 0;
#pragma unroll
      for (int e = 0; e < VK_EPT; ++e) {
        long long j = base + (long long)e * VK_THREADS;
        if (j < n) a += b[j] * tr[e];
      }
      const double at = block_sum_t<T>(a, red);
      if (threadIdx.x == 0) part[(long long)blockIdx.x * (k + 1) + i] = at;
    }
  } else {
    for (int i = threadIdx.x; i < k; i += blockDim.x) part[(long long)blockIdx.x * (k + 1) + i] = 0.0;
  }
  const double nt = block_sum_t<T>(nn, red);
  if (threadIdx.x == 0) part[(long long)blockIdx.x * (k + 1) + k] = nt;
  last_block_sums(part, k + 1, out, counter, red);
}

// y = a x + b y
__global__ void k_axpby(double a, const double *__restrict__ x, double b, double *__restrict__ y, long long n) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x)
    y[j] = a * x[j] + b * y[j];
}

// z = r / |theta - hdiag| with the magnitude clamped below at guard; part[block] = r . z
__global__ void __launch_bounds__(VK_THREADS) k_precond_dot(const double *__restrict__ r, double theta,
                                                            const double *__restrict__ hd, double guard,
                                                            double *__restrict__ z, long long n,
                                                            double *__restrict__ part, double *__restrict__ out,
                                                            unsigned *counter) {
  __shared__ double red[32];
  const long long base = (long long)blockIdx.x * VK_CHUNK + threadIdx.x;
  double acc = 0.0;
#pragma unroll 4
  for (int e = 0; e < VK_EPT; ++e) {
    long long j = base + (long long)e * VK_THREADS;
    if (j >= n) break;
    double den = fabs(theta - hd[j]);
    if (den < guard) den = guard;
    const double rv = r[j];
    const double zv = rv / den;
    z[j] = zv;
    acc += rv * zv;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  last_block_sums(part, 1, out, counter, red);
}

template <typename T>
__global__ void k_scale(T *__restrict__ x, const T *__restrict__ src, double alpha, long long n) {
  const T al = (T)alpha;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x)
    x[j] = al * src[j];
}

template <typename TI, typename TO>
__global__ void k_convert(const TI *__restrict__ x, TO *__restrict__ y, long long n) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x)
    y[j] = (TO)x[j];
}

// Block minimum of (value, index) over entries not in excl[0..nex); lexicographic.
__global__ void k_argmin(const double *__restrict__ x, long long n, const long long *__restrict__ excl,
                         int nex, double *__restrict__ bval, long long *__restrict__ bidx) {
  __shared__ double sv[VK_THREADS];
  __shared__ long long si[VK_THREADS];
  double best = INFINITY;
  long long bi = -1;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double v = x[j];
    bool skip = false;
    for (int e = 0; e < nex; ++e) skip |= (excl[e] == j);
    if (skip) continue;
    if (bi < 0 || v < best || (v == best && j < bi)) { best = v; bi = j; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double v2 = sv[threadIdx.x + s];
      long long i2 = si[threadIdx.x + s];
      double v1 = sv[threadIdx.x];
      long long i1 = si[threadIdx.x];
      bool take = (i2 >= 0) && (i1 < 0 || v2 < v1 || (v2 == v1 && i2 < i1));
      if (take) { sv[threadIdx.x] = v2; si[threadIdx.x] = i2; }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { bval[blockIdx.x] = sv[0]; bidx[blockIdx.x] = si[0]; }
}

__global__ void k_nonfinite(const double *__restrict__ x, long long n, int *flag) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[j])) *flag = 1;
}

// ------------------------------------------------------------------ host wrappers

// Partials of the reductions in the context's small scratch, and the arrival counter
// of the fused second pass (zeroed once; every reduction leaves it at zero).
static int part_buffer(forte_ctx *ctx, size_t doubles, double **p, unsigned **counter) {
  int rc = ctx->sc_small.ensure(sizeof(double) * (doubles + 64));
  if (rc) return rc;
  *p = (double *)ctx->sc_small.ptr;
  if (!ctx->d_vk_count) {
    FORTE_CUDA_TRY(cudaMalloc(&ctx->d_vk_count, sizeof(unsigned)));
    FORTE_CUDA_TRY(cudaMemsetAsync(ctx->d_vk_count, 0, sizeof(unsigned), ctx->stream));
  }
  *counter = ctx->d_vk_count;
  return FORTE_OK;
}

template <typename T>
static int vk_multidot_t(forte_ctx *ctx, const T *V, int nv, long long ld, const T *x, long long n, double *out) {
  if (nv <= 0) return FORTE_OK;
  if (nv > VK_MAXV) { set_error("multidot: too many vectors (%d)", nv); return FORTE_ERR_ARG; }
  unsigned nb = vk_blocks(n);
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, (size_t)nb * nv, &part, &cnt);
  if (rc) return rc;
  FORTE_PROF(ctx, "multidot");
  k_multidot<T><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, x, n, part, out, cnt);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

template <typename T>
static int vk_combine_t(forte_ctx *ctx, const T *V, int nv, long long ld, const double *coef, int ncomb, T *out,
                        long long ldo, long long n) {
  if (nv > VK_MAXV || ncomb > 64) { set_error("combine: too many vectors"); return FORTE_ERR_ARG; }
  unsigned nb = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
  // outputs in groups of 8, 4, 2, 1 (each group streams V once)
  for (int c0 = 0; c0 < ncomb;) {
    const int left = ncomb - c0, g = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    FORTE_PROF(ctx, "combine");
    if (g == 8)
      k_combine<8, T><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, coef, ncomb, c0, out, ldo, n);
    else if (g == 4)
      k_combine<4, T><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, coef, ncomb, c0, out, ldo, n);
    else if (g == 2)
      k_combine<2, T><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, coef, ncomb, c0, out, ldo, n);
    else
      k_combine<1, T><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, coef, ncomb, c0, out, ldo, n);
    FORTE_LAUNCH_CHECK();
    c0 += g;
  }
  return FORTE_OK;
}

template <typename T>
static int vk_residual_precond_t(forte_ctx *ctx, const T *B, const T *S, int k, long long ld, const double *u,
                                 double theta, double guard, T *t, double *rnorm2, long long n) {
  if (k > VK_MAXV) { set_error("residual: subspace too large (%d)", k); return FORTE_ERR_ARG; }
  unsigned nb = vk_blocks(n);
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, nb, &part, &cnt);
  if (rc) return rc;
  FORTE_PROF(ctx, "residual_precond");
  k_residual_precond<T><<<nb, VK_THREADS, 0, ctx->stream>>>(B, S, k, ld, u, theta, ctx->d_hdiag, guard, t, n,
                                                            part, rnorm2, cnt);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

template <typename T>
static int vk_orth_update_t(forte_ctx *ctx, const T *B, int k, long long ld, const double *c, const T *t_in,
                            T *t_out, double *dots_out, long long n, bool dots) {
  if (k + 1 > VK_MAXV) { set_error("orth: subspace too large (%d)", k); return FORTE_ERR_ARG; }
  unsigned nb = vk_blocks(n);
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, (size_t)nb * (k + 1), &part, &cnt);
  if (rc) return rc;
  FORTE_PROF(ctx, "orth_update");
  if (dots)
    k_orth_update<T, true><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, n, part, dots_out, cnt);
  else
    k_orth_update<T, false><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, n, part, dots_out, cnt);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

template <typename T>
static int vk_scale_t(forte_ctx *ctx, T *x, const T *src, double alpha, long long n) {
  unsigned nb = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
  {
    FORTE_PROF(ctx, "scale");
    k_scale<T><<<nb, 256, 0, ctx->stream>>>(x, src, alpha, n);
  FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

int vk_multidot(forte_ctx *ctx, const double *V, int nv, long long ld, const double *x, long long n, double *out) {
  return vk_multidot_t(ctx, V, nv, ld, x, n, out);
}
int vk_multidot(forte_ctx *ctx, const float *V, int nv, long long ld, const float *x, long long n, double *out) {
  return vk_multidot_t(ctx, V, nv, ld, x, n, out);
}
int vk_combine(forte_ctx *ctx, const double *V, int nv, long long ld, const double *coef, int ncomb, double *out,
               long long ldo, long long n) {
  return vk_combine_t(ctx, V, nv, ld, coef, ncomb, out, ldo, n);
}
int vk_combine(forte_ctx *ctx, const float *V, int nv, long long ld, const double *coef, int ncomb, float *out,
               long long ldo, long long n) {
  return vk_combine_t(ctx, V, nv, ld, coef, ncomb, out, ldo, n);
}
int vk_residual_precond(forte_ctx *ctx, const double *B, const double *S, int k, long long ld, const double *u,
                        double theta, double guard, double *t, double *rnorm2, long long n) {
  return vk_residual_precond_t(ctx, B, S, k, ld, u, theta, guard, t, rnorm2, n);
}
int vk_residual_precond(forte_ctx *ctx, const float *B, const float *S, int k, long long ld, const double *u,
                        double theta, double guard, float *t, double *rnorm2, long long n) {
  return vk_residual_precond_t(ctx, B, S, k, ld, u, theta, guard, t, rnorm2, n);
}
int vk_orth_update(forte_ctx *ctx, const double *B, int k, long long ld, const double *c, const double *t_in,
                   double *t_out, double *dots_out, long long n, bool dots) {
  return vk_orth_update_t(ctx, B, k, ld, c, t_in, t_out, dots_out, n, dots);
}
int vk_orth_update(forte_ctx *ctx, const float *B, int k, long long ld, const double *c, const float *t_in,
                   float *t_out, double *dots_out, long long n, bool dots) {
  return vk_orth_update_t(ctx, B, k, ld, c, t_in, t_out, dots_out, n, dots);
}
int vk_scale(forte_ctx *ctx, double *x, const double *src, double alpha, long long n) {
  return vk_scale_t(ctx, x, src, alpha, n);
}
int vk_scale(forte_ctx *ctx, float *x, const float *src, double alpha, long long n) {
  return vk_scale_t(ctx, x, src, alpha, n);
}
template <typename TI, typename TO>
static int vk_convert_t(forte_ctx *ctx, const TI *x, TO *y, long long n) {
  unsigned nb = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
  FORTE_PROF(ctx, "convert");
  k_convert<TI, TO><<<nb, 256, 0, ctx->stream>>>(x, y, n);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}
int vk_convert(forte_ctx *ctx, const double *x, float *y, long long n) { return vk_convert_t(ctx, x, y, n); }
int vk_convert(forte_ctx *ctx, const float *x, double *y, long long n) { return vk_convert_t(ctx, x, y, n); }

int vk_axpby(forte_ctx *ctx, double a, const double *x, double b, double *y, long long n) {
  unsigned nb = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
  {
    FORTE_PROF(ctx, "axpby");
    k_axpby<<<nb, 256, 0, ctx->stream>>>(a, x, b, y, n);
    FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

int vk_precond_dot(forte_ctx *ctx, const double *r, double theta, double guard, double *z, double *dot_out,
                   long long n) {
  unsigned nb = vk_blocks(n);
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, nb, &part, &cnt);
  if (rc) return rc;
  FORTE_PROF(ctx, "precond_dot");
  k_precond_dot<<<nb, VK_THREADS, 0, ctx->stream>>>(r, theta, ctx->d_hdiag, guard, z, n, part, dot_out, cnt);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

// k smallest entries (ties: lowest index), host output idx_out[k].
int vk_argmin_k(forte_ctx *ctx, const double *x, long long n, int k, long long *idx_out) {
  const unsigned nb = (unsigned)std::min<long long>((n + VK_THREADS - 1) / VK_THREADS, 1024);
  size_t need = sizeof(double) * nb + sizeof(long long) * nb + sizeof(long long) * (k + 1);
  int rc = ctx->sc_small.ensure(need + 256);
  if (rc) return rc;
  double *bval = (double *)ctx->sc_small.ptr;
  long long *bidx = (long long *)(bval + nb);
  long long *excl = bidx + nb;
  std::vector<double> hv(nb);
  std::vector<long long> hi(nb);
  for (int r = 0; r < k; ++r) {
    if (r > 0)
      FORTE_CUDA_TRY(cudaMemcpyAsync(excl, idx_out, sizeof(long long) * r, cudaMemcpyHostToDevice, ctx->stream));
    {
      FORTE_PROF(ctx, "argmin");
      k_argmin<<<nb, VK_THREADS, 0, ctx->stream>>>(x, n, excl, r, bval, bidx);
    FORTE_LAUNCH_CHECK();
    }
    FORTE_CUDA_TRY(cudaMemcpyAsync(hv.data(), bval, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    FORTE_CUDA_TRY(cudaMemcpyAsync(hi.data(), bidx, sizeof(long long) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    double best = INFINITY;
    long long bi = -1;
    for (unsigned b = 0; b < nb; ++b) {
      if (hi[b] < 0) continue;
      if (bi < 0 || hv[b] < best || (hv[b] == best && hi[b] < bi)) { best = hv[b]; bi = hi[b]; }
    }
    if (bi < 0) { set_error("argmin: fewer than %d entries", k); return FORTE_ERR_ARG; }
    idx_out[r] = bi;
  }
  return FORTE_OK;
}

int vk_any_nonfinite(forte_ctx *ctx, const double *x, long long n, int *flag_host) {
  int rc = ctx->sc_small.ensure(256);
  if (rc) return rc;
  int *flag = (int *)ctx->sc_small.ptr;
  FORTE_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  unsigned nb = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 8);
  {
    FORTE_PROF(ctx, "nonfinite");
    k_nonfinite<<<nb, 256, 0, ctx->stream>>>(x, n, flag);
  FORTE_LAUNCH_CHECK();
  }
  FORTE_CUDA_TRY(cudaMemcpyAsync(flag_host, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return FORTE_OK;
}

}  // namespace forte
