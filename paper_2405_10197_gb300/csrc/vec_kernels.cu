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

// z = r * rinv (the inverse of the preconditioner's diagonal); out = [r . z, r . r]
__global__ void __launch_bounds__(VK_THREADS) k_precond_dot(const double *__restrict__ r, const double *__restrict__ rinv,
                                                            double *__restrict__ z, long long n,
                                                            double *__restrict__ part, double *__restrict__ out,
                                                            unsigned *counter) {
  __shared__ double red[32];
  const long long base = (long long)blockIdx.x * VK_CHUNK + threadIdx.x;
  double acc = 0.0, rr = 0.0;
#pragma unroll 4
  for (int e = 0; e < VK_EPT; ++e) {
    long long j = base + (long long)e * VK_THREADS;
    if (j >= n) break;
    const double rv = r[j];
    const double zv = rv * rinv[j];
    z[j] = zv;
    acc += rv * zv;
    rr += rv * rv;
  }
  acc = block_sum(acc, red);
  rr = block_sum(rr, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc;
    part[2 * blockIdx.x + 1] = rr;
  }
  last_block_sums(part, 2, out, counter, red);
}

// rinv = 1 / |theta - hdiag| with the magnitude clamped below at guard: the FP64
// divisions of the diagonal preconditioner, done once per correction solve (the FP64
// pipe of this GPU makes a division per element and application the bound otherwise)
__global__ void k_precond_inv(const double *__restrict__ hd, double theta, double guard, double *__restrict__ rinv,
                              long long n) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    double den = fabs(theta - hd[j]);
    if (den < guard) den = guard;
    rinv[j] = 1.0 / den;
  }
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

// ------------------------------------------------------------------ packet kernels
// The kernels below move every operand in 16-byte packets (float4 / double2), run a
// persistent grid (4 resident blocks of 256 threads per SM) over chunks of
// VK_THREADS x VP_PER packets, keep per-warp partial sums in shared memory across the
// chunks of a block (no block barrier per chunk, one reduction per block instead of
// one per 4096 elements), and finish with the fused last-block pass.  They need the
// element count and the leading dimension to be multiples of the packet and 16-byte
// aligned bases; the element kernels above serve every other case.  Per element they
// do the arithmetic of the element kernels in the same order; only the order of the
// partial sums differs (fixed for a given grid, so results are reproducible).
template <typename T>
struct Pk;
template <>
struct Pk<float> {
  using V = float4;
  static constexpr int P = 4;
};
template <>
struct Pk<double> {
  using V = double2;
  static constexpr int P = 2;
};

constexpr int VP_PER = 4;                   // packets per thread per chunk
constexpr int VP_CH = VK_THREADS * VP_PER;  // packets per chunk
constexpr int VP_WARPS = VK_THREADS / 32;
constexpr int VP_BPS = 4;                   // resident blocks per SM (64 registers a thread)

template <typename T>
__device__ __forceinline__ void pk_ld(const T *p, long long q, T (&x)[Pk<T>::P]) {
  const typename Pk<T>::V v = reinterpret_cast<const typename Pk<T>::V *>(p)[q];
  if constexpr (Pk<T>::P == 4) {
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else {
    x[0] = v.x; x[1] = v.y;
  }
}
template <typename T>
__device__ __forceinline__ void pk_st(T *p, long long q, const T (&x)[Pk<T>::P]) {
  typename Pk<T>::V v;
  if constexpr (Pk<T>::P == 4) {
    v.x = x[0]; v.y = x[1]; v.z = x[2]; v.w = x[3];
  } else {
    v.x = x[0]; v.y = x[1];
  }
  reinterpret_cast<typename Pk<T>::V *>(p)[q] = v;
}
// the P FP64 diagonal entries of packet q (hd is FP64 for either vector type)
template <int P>
__device__ __forceinline__ void hd_ld(const double *hd, long long q, double (&h)[P]) {
  const double2 a = reinterpret_cast<const double2 *>(hd)[q * (P / 2)];
  h[0] = a.x;
  h[1] = a.y;
  if constexpr (P == 4) {
    const double2 b = reinterpret_cast<const double2 *>(hd)[q * 2 + 1];
    h[2] = b.x;
    h[3] = b.y;
  }
}

// Lane 0 adds the warp's sum of v (summed in T across the warp) to acc[warp].
template <typename T>
__device__ __forceinline__ void warp_add(T v, double *acc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) acc[threadIdx.x >> 5] += (double)v;
}

// part[block][i] = sum over warps of sw[i][warp], i < m (warps in a fixed order).
__device__ __forceinline__ void block_partials(const double *sw, int m, double *part) {
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < VP_WARPS; ++w) s += sw[i * VP_WARPS + w];
    part[(long long)blockIdx.x * m + i] = s;
  }
}

// out[i] = V_i . x (i < nv); np = packets per vector.
template <typename T>
__global__ void __launch_bounds__(VK_THREADS, VP_BPS) k_multidot_p(const T *__restrict__ V, int nv, long long ld,
                                                           const T *__restrict__ x, long long np,
                                                           double *__restrict__ part, double *__restrict__ out,
                                                           unsigned *counter) {
  constexpr int P = Pk<T>::P;
  __shared__ double red[32];
  __shared__ double sw[VK_MAXV * VP_WARPS];
  for (int i = threadIdx.x; i < nv * VP_WARPS; i += blockDim.x) sw[i] = 0.0;
  __syncthreads();
  const long long nch = (np + VP_CH - 1) / VP_CH;
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long q0 = ch * VP_CH + threadIdx.x;
    T xr[VP_PER][P];
#pragma unroll
    for (int e = 0; e < VP_PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
        pk_ld(x, q, xr[e]);
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) xr[e][p] = T(0);
      }
    }
    for (int i = 0; i < nv; ++i) {
      const T *v = V + (long long)i * ld;
      T a = 0;
#pragma unroll
      for (int e = 0; e < VP_PER; ++e) {
        const long long q = q0 + (long long)e * VK_THREADS;
        if (q < np) {
          T vv[P];
          pk_ld(v, q, vv);
#pragma unroll
          for (int p = 0; p < P; ++p) a += vv[p] * xr[e][p];
        }
      }
      warp_add(a, sw + i * VP_WARPS);
    }
  }
  block_partials(sw, nv, part);
  last_block_sums(part, nv, out, counter, red);
}

// The same for nv <= KMAX: loop over the vectors unrolled, partial sums of the
// block's chunks in registers, one warp reduction per vector and block.
template <typename T, int KMAX>
__global__ void __launch_bounds__(VK_THREADS, VP_BPS) k_multidot_u(const T *__restrict__ V, int nv, long long ld,
                                                                   const T *__restrict__ x, long long np,
                                                                   double *__restrict__ part,
                                                                   double *__restrict__ out, unsigned *counter) {
  constexpr int P = Pk<T>::P;
  __shared__ double red[32];
  __shared__ double sw[KMAX * VP_WARPS];
  for (int i = threadIdx.x; i < nv * VP_WARPS; i += blockDim.x) sw[i] = 0.0;
  __syncthreads();
  T acc[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) acc[i] = T(0);
  const long long nch = (np + VP_CH - 1) / VP_CH;
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long q0 = ch * VP_CH + threadIdx.x;
    T xr[VP_PER][P];
#pragma unroll
    for (int e = 0; e < VP_PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
        pk_ld(x, q, xr[e]);
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) xr[e][p] = T(0);
      }
    }
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      if (i < nv) {
        const T *v = V + (long long)i * ld;
#pragma unroll
        for (int e = 0; e < VP_PER; ++e) {
          const long long q = q0 + (long long)e * VK_THREADS;
          if (q < np) {
            T vv[P];
            pk_ld(v, q, vv);
#pragma unroll
            for (int p = 0; p < P; ++p) acc[i] += vv[p] * xr[e][p];
          }
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < KMAX; ++i)
    if (i < nv) warp_add(acc[i], sw + i * VP_WARPS);
  block_partials(sw, nv, part);
  last_block_sums(part, nv, out, counter, red);
}

// t_out = scale (t_in - sum_i c_i B_i); out = [B_i . t_out (i < k, zeros unless DOTS),
// |t_out|^2].  c == nullptr: no update.  t_in may alias t_out.
template <typename T, bool DOTS>
__global__ void __launch_bounds__(VK_THREADS, VP_BPS) k_orth_update_p(const T *__restrict__ Bm, int k, long long ld,
                                                              const double *__restrict__ c, const T *t_in,
                                                              T *t_out, long long np, double scale,
                                                              double *__restrict__ part, double *__restrict__ out,
                                                              unsigned *counter) {
  constexpr int P = Pk<T>::P;
  __shared__ double red[32];
  __shared__ double sw[(VK_MAXV + 1) * VP_WARPS];
  __shared__ T sc[VK_MAXV];
  const int ku = c ? k : 0;
  for (int i = threadIdx.x; i < ku; i += blockDim.x) sc[i] = (T)c[i];
  for (int i = threadIdx.x; i < (k + 1) * VP_WARPS; i += blockDim.x) sw[i] = 0.0;
  __syncthreads();
  const T s = (T)scale;
  const bool scaled = scale != 1.0;  // FP64 multiplies cost FP64-pipe slots: skip the identity
  const long long nch = (np + VP_CH - 1) / VP_CH;
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long q0 = ch * VP_CH + threadIdx.x;
    T tr[VP_PER][P];
#pragma unroll
    for (int e = 0; e < VP_PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
        pk_ld(t_in, q, tr[e]);
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) tr[e][p] = T(0);
      }
    }
    for (int i = 0; i < ku; ++i) {
      const T *b = Bm + (long long)i * ld;
      const T ci = sc[i];
#pragma unroll
      for (int e = 0; e < VP_PER; ++e) {
        const long long q = q0 + (long long)e * VK_THREADS;
        if (q < np) {
          T bv[P];
          pk_ld(b, q, bv);
#pragma unroll
          for (int p = 0; p < P; ++p) tr[e][p] -= ci * bv[p];
        }
      }
    }
    T nn = 0;
#pragma unroll
    for (int e = 0; e < VP_PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (scaled) tr[e][p] *= s;
          nn += tr[e][p] * tr[e][p];
        }
        pk_st(t_out, q, tr[e]);
      }
    }
    warp_add(nn, sw + k * VP_WARPS);
    if (DOTS) {
      for (int i = 0; i < k; ++i) {
        const T *b = Bm + (long long)i * ld;
        T a = 0;
#pragma unroll
        for (int e = 0; e < VP_PER; ++e) {
          const long long q = q0 + (long long)e * VK_THREADS;
          if (q < np) {
            T bv[P];
            pk_ld(b, q, bv);
#pragma unroll
            for (int p = 0; p < P; ++p) a += bv[p] * tr[e][p];
          }
        }
        warp_add(a, sw + i * VP_WARPS);
      }
    }
  }
  block_partials(sw, k + 1, part);
  last_block_sums(part, k + 1, out, counter, red);
}

// The same for k <= KMAX: loops over the basis unrolled, partial sums in registers.
template <typename T, bool DOTS, int KMAX>
__global__ void __launch_bounds__(VK_THREADS, VP_BPS) k_orth_update_u(const T *__restrict__ Bm, int k, long long ld,
                                                                      const double *__restrict__ c, const T *t_in,
                                                                      T *t_out, long long np, double scale,
                                                                      double *__restrict__ part,
                                                                      double *__restrict__ out, unsigned *counter) {
  constexpr int P = Pk<T>::P;
  __shared__ double red[32];
  __shared__ double sw[(KMAX + 1) * VP_WARPS];
  __shared__ T sc[KMAX];
  const int ku = c ? k : 0;
  for (int i = threadIdx.x; i < ku; i += blockDim.x) sc[i] = (T)c[i];
  for (int i = threadIdx.x; i < (k + 1) * VP_WARPS; i += blockDim.x) sw[i] = 0.0;
  __syncthreads();
  const T s = (T)scale;
  const bool scaled = scale != 1.0;
  T nn = 0, acc[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) acc[i] = T(0);
  const long long nch = (np + VP_CH - 1) / VP_CH;
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long q0 = ch * VP_CH + threadIdx.x;
    T tr[VP_PER][P];
#pragma unroll
    for (int e = 0; e < VP_PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
        pk_ld(t_in, q, tr[e]);
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) tr[e][p] = T(0);
      }
    }
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      if (i < ku) {
        const T *b = Bm + (long long)i * ld;
        const T ci = sc[i];
#pragma unroll
        for (int e = 0; e < VP_PER; ++e) {
          const long long q = q0 + (long long)e * VK_THREADS;
          if (q < np) {
            T bv[P];
            pk_ld(b, q, bv);
#pragma unroll
            for (int p = 0; p < P; ++p) tr[e][p] -= ci * bv[p];
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < VP_PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (scaled) tr[e][p] *= s;
          nn += tr[e][p] * tr[e][p];
        }
        pk_st(t_out, q, tr[e]);
      }
    }
    if (DOTS) {
#pragma unroll
      for (int i = 0; i < KMAX; ++i) {
        if (i < k) {
          const T *b = Bm + (long long)i * ld;
#pragma unroll
          for (int e = 0; e < VP_PER; ++e) {
            const long long q = q0 + (long long)e * VK_THREADS;
            if (q < np) {
              T bv[P];
              pk_ld(b, q, bv);
#pragma unroll
              for (int p = 0; p < P; ++p) acc[i] += bv[p] * tr[e][p];
            }
          }
        }
      }
    }
  }
  warp_add(nn, sw + k * VP_WARPS);
  if (DOTS) {
#pragma unroll
    for (int i = 0; i < KMAX; ++i)
      if (i < k) warp_add(acc[i], sw + i * VP_WARPS);
  }
  block_partials(sw, k + 1, part);
  last_block_sums(part, k + 1, out, counter, red);
}

// r = sum_i u_i S_i - theta sum_i u_i B_i ;  t = r / (theta - hdiag) (guarded).
// out[0] = |r|^2; with DOTS also out[1 + i] = B_i . t (i < k) and out[1 + k] = |t|^2,
// which the Gram-Schmidt step of the new direction needs (B is read here anyway).
// PER packets per thread per chunk: the dots re-read the chunk's B_i right after
// forming t, and a small chunk keeps the 2k vectors of all resident chunks (~70 MB
// at PER = 2) within L2, so the re-read does not reach DRAM.
template <typename T, bool DOTS, int PER>
__global__ void __launch_bounds__(VK_THREADS, VP_BPS) k_residual_precond_p(
    const T *__restrict__ B, const T *__restrict__ S, int k, long long ld, const double *__restrict__ u,
    double theta, const double *__restrict__ hd, double guard, T *__restrict__ t, long long np,
    double *__restrict__ part, double *__restrict__ out, unsigned *counter) {
  constexpr int P = Pk<T>::P;
  __shared__ double red[32];
  __shared__ double sw[(VK_MAXV + 2) * VP_WARPS];
  __shared__ T su[VK_MAXV];
  const int m = DOTS ? k + 2 : 1;
  for (int i = threadIdx.x; i < k; i += blockDim.x) su[i] = (T)u[i];
  for (int i = threadIdx.x; i < m * VP_WARPS; i += blockDim.x) sw[i] = 0.0;
  __syncthreads();
  const T th = (T)theta;
  const long long nch = (np + (VK_THREADS * PER) - 1) / (VK_THREADS * PER);
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long q0 = ch * (VK_THREADS * PER) + threadIdx.x;
    T hx[PER][P], xv[PER][P];
#pragma unroll
    for (int e = 0; e < PER; ++e)
#pragma unroll
      for (int p = 0; p < P; ++p) hx[e][p] = xv[e][p] = T(0);
    for (int i = 0; i < k; ++i) {
      const T ui = su[i];
      const T *sp = S + (long long)i * ld, *bp = B + (long long)i * ld;
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const long long q = q0 + (long long)e * VK_THREADS;
        if (q < np) {
          T sv[P], bv[P];
          pk_ld(sp, q, sv);
          pk_ld(bp, q, bv);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            hx[e][p] += ui * sv[p];
            xv[e][p] += ui * bv[p];
          }
        }
      }
    }
    T rr = 0, tt = 0;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
        double h[P];
        hd_ld<P>(hd, q, h);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const T r = hx[e][p] - th * xv[e][p];
          rr += r * r;
          double den = theta - h[p];
          if (fabs(den) < guard) den = (den >= 0.0) ? guard : -guard;
          hx[e][p] = r / (T)den;  // hx now holds t
          tt += hx[e][p] * hx[e][p];
        }
        pk_st(t, q, hx[e]);
      }
    }
    warp_add(rr, sw);
    if (DOTS) {
      warp_add(tt, sw + (k + 1) * VP_WARPS);
      for (int i = 0; i < k; ++i) {
        const T *bp = B + (long long)i * ld;
        T a = 0;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
          const long long q = q0 + (long long)e * VK_THREADS;
          if (q < np) {
            T bv[P];
            pk_ld(bp, q, bv);
#pragma unroll
            for (int p = 0; p < P; ++p) a += bv[p] * hx[e][p];
          }
        }
        warp_add(a, sw + (1 + i) * VP_WARPS);
      }
    }
  }
  block_partials(sw, m, part);
  last_block_sums(part, m, out, counter, red);
}

// The same for k <= KMAX with the loops over the basis unrolled (the loads of all k
// vectors of a chunk can be in flight together) and the partial sums of the block's
// chunks kept in registers, reduced over the warp once per block.
template <typename T, bool DOTS, int PER, int KMAX>
__global__ void __launch_bounds__(VK_THREADS, VP_BPS) k_residual_precond_u(
    const T *__restrict__ B, const T *__restrict__ S, int k, long long ld, const double *__restrict__ u,
    double theta, const double *__restrict__ hd, double guard, T *__restrict__ t, long long np,
    double *__restrict__ part, double *__restrict__ out, unsigned *counter) {
  constexpr int P = Pk<T>::P;
  __shared__ double red[32];
  __shared__ double sw[(KMAX + 2) * VP_WARPS];
  __shared__ T su[KMAX];
  const int m = DOTS ? k + 2 : 1;
  for (int i = threadIdx.x; i < k; i += blockDim.x) su[i] = (T)u[i];
  for (int i = threadIdx.x; i < m * VP_WARPS; i += blockDim.x) sw[i] = 0.0;
  __syncthreads();
  const T th = (T)theta;
  T rr = 0, tt = 0, acc[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) acc[i] = T(0);
  const long long nch = (np + (VK_THREADS * PER) - 1) / (VK_THREADS * PER);
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long q0 = ch * (VK_THREADS * PER) + threadIdx.x;
    T hx[PER][P], xv[PER][P];
#pragma unroll
    for (int e = 0; e < PER; ++e)
#pragma unroll
      for (int p = 0; p < P; ++p) hx[e][p] = xv[e][p] = T(0);
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      if (i < k) {
        const T ui = su[i];
        const T *sp = S + (long long)i * ld, *bp = B + (long long)i * ld;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
          const long long q = q0 + (long long)e * VK_THREADS;
          if (q < np) {
            T sv[P], bv[P];
            pk_ld(sp, q, sv);
            pk_ld(bp, q, bv);
#pragma unroll
            for (int p = 0; p < P; ++p) {
              hx[e][p] += ui * sv[p];
              xv[e][p] += ui * bv[p];
            }
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
        double h[P];
        hd_ld<P>(hd, q, h);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const T r = hx[e][p] - th * xv[e][p];
          rr += r * r;
          double den = theta - h[p];
          if (fabs(den) < guard) den = (den >= 0.0) ? guard : -guard;
          hx[e][p] = r / (T)den;  // hx now holds t
          tt += hx[e][p] * hx[e][p];
        }
        pk_st(t, q, hx[e]);
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) hx[e][p] = T(0);
      }
    }
    if (DOTS) {
#pragma unroll
      for (int i = 0; i < KMAX; ++i) {
        if (i < k) {
          const T *bp = B + (long long)i * ld;
#pragma unroll
          for (int e = 0; e < PER; ++e) {
            const long long q = q0 + (long long)e * VK_THREADS;
            if (q < np) {
              T bv[P];
              pk_ld(bp, q, bv);
#pragma unroll
              for (int p = 0; p < P; ++p) acc[i] += bv[p] * hx[e][p];
            }
          }
        }
      }
    }
  }
  warp_add(rr, sw);
  if (DOTS) {
    warp_add(tt, sw + (k + 1) * VP_WARPS);
#pragma unroll
    for (int i = 0; i < KMAX; ++i)
      if (i < k) warp_add(acc[i], sw + (1 + i) * VP_WARPS);
  }
  block_partials(sw, m, part);
  last_block_sums(part, m, out, counter, red);
}

// z = r * rinv; out[0] = r . z, out[1] = r . r
__global__ void __launch_bounds__(VK_THREADS, VP_BPS) k_precond_dot_p(const double *__restrict__ r,
                                                                      const double *__restrict__ rinv,
                                                                      double *__restrict__ z, long long np,
                                                                      double *__restrict__ part, double *__restrict__ out,
                                                                      unsigned *counter) {
  __shared__ double red[32];
  __shared__ double sw[2 * VP_WARPS];
  if (threadIdx.x < 2 * VP_WARPS) sw[threadIdx.x] = 0.0;
  __syncthreads();
  const long long nch = (np + VP_CH - 1) / VP_CH;
  for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long long q0 = ch * VP_CH + threadIdx.x;
    double acc = 0.0, rr = 0.0;
#pragma unroll
    for (int e = 0; e < VP_PER; ++e) {
      const long long q = q0 + (long long)e * VK_THREADS;
      if (q < np) {
        double rv[2], iv[2], zv[2];
        pk_ld(r, q, rv);
        pk_ld(rinv, q, iv);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          zv[p] = rv[p] * iv[p];
          acc += rv[p] * zv[p];
          rr += rv[p] * rv[p];
        }
        pk_st(z, q, zv);
      }
    }
    warp_add(acc, sw);
    warp_add(rr, sw + VP_WARPS);
  }
  block_partials(sw, 2, part);
  last_block_sums(part, 2, out, counter, red);
}

// y = a x + b y and x = alpha src over packets (grid-stride).  With a or b equal to 1
// the update is one fused multiply-add per element (the FP64 pipe is the bound of
// these kernels on this GPU, not HBM).
__global__ void k_axpby_p(double a, const double *__restrict__ x, double b, double *__restrict__ y, long long np) {
  const int form = b == 1.0 ? 1 : (a == 1.0 ? 2 : 0);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (long long)gridDim.x * blockDim.x) {
    double xv[2], yv[2];
    pk_ld(x, q, xv);
    pk_ld((const double *)y, q, yv);
#pragma unroll
    for (int p = 0; p < 2; ++p)
      yv[p] = form == 1 ? fma(a, xv[p], yv[p]) : form == 2 ? fma(b, yv[p], xv[p]) : a * xv[p] + b * yv[p];
    pk_st(y, q, yv);
  }
}
template <typename T>
__global__ void k_scale_p(T *x, const T *src, double alpha, long long np) {
  constexpr int P = Pk<T>::P;
  const T al = (T)alpha;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (long long)gridDim.x * blockDim.x) {
    T v[P];
    pk_ld(src, q, v);
#pragma unroll
    for (int p = 0; p < P; ++p) v[p] = al * v[p];
    pk_st(x, q, v);
  }
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

// Packet kernels apply when the count and the leading dimension are multiples of the
// packet (16 bytes) and every vector base is 16-byte aligned.
template <typename T>
static bool vp_ok(long long n, long long ld, std::initializer_list<const void *> ptrs) {
  constexpr long long P = Pk<T>::P;
  if (n % P != 0 || ld % P != 0) return false;
  for (const void *q : ptrs)
    if (q && ((uintptr_t)q & 15u) != 0) return false;
  return true;
}
// persistent grid: VP_BPS resident blocks of VK_THREADS per SM, at least one block
static unsigned vp_grid(const forte_ctx *ctx, long long np) {
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || nsm <= 0) {
    cudaGetLastError();
    nsm = 152;
  }
  const long long nch = (np + VP_CH - 1) / VP_CH;
  return (unsigned)std::max<long long>(1, std::min<long long>(nch, (long long)VP_BPS * nsm));
}

template <typename T>
static int vk_multidot_t(forte_ctx *ctx, const T *V, int nv, long long ld, const T *x, long long n, double *out) {
  if (nv <= 0) return FORTE_OK;
  if (nv > VK_MAXV) { set_error("multidot: too many vectors (%d)", nv); return FORTE_ERR_ARG; }
  const bool pk = vp_ok<T>(n, ld, {V, x});
  const unsigned nb = pk ? vp_grid(ctx, n / Pk<T>::P) : vk_blocks(n);
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, (size_t)nb * nv, &part, &cnt);
  if (rc) return rc;
  FORTE_PROF(ctx, "multidot");
  if (pk && nv <= 4)
    k_multidot_u<T, 4><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, x, n / Pk<T>::P, part, out, cnt);
  else if (pk && nv <= 8)
    k_multidot_u<T, 8><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, x, n / Pk<T>::P, part, out, cnt);
  else if (pk && nv <= 16)
    k_multidot_u<T, 16><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, x, n / Pk<T>::P, part, out, cnt);
  else if (pk)
    k_multidot_p<T><<<nb, VK_THREADS, 0, ctx->stream>>>(V, nv, ld, x, n / Pk<T>::P, part, out, cnt);
  else
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
                                 double theta, double guard, T *t, double *rnorm2, long long n, double *dots) {
  if (k > VK_MAXV) { set_error("residual: subspace too large (%d)", k); return FORTE_ERR_ARG; }
  const bool pk = vp_ok<T>(n, ld, {B, S, t, ctx->d_hdiag});
  if (dots && !pk) return -1;  // no fused dots: the caller forms them with vk_orth_update
  const unsigned nb = pk ? vp_grid(ctx, 2 * (n / Pk<T>::P)) : vk_blocks(n);  // chunks of half the packets
  const int m = dots ? k + 2 : 1;
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, (size_t)nb * m, &part, &cnt);
  if (rc) return rc;
  FORTE_PROF(ctx, "residual_precond");
  const long long npk = n / Pk<T>::P;
  const double *hd = ctx->d_hdiag;
#define FORTE_RESID_U(KM)                                                                                            \
  do {                                                                                                               \
    if (dots)                                                                                                        \
      k_residual_precond_u<T, true, 2, KM><<<nb, VK_THREADS, 0, ctx->stream>>>(B, S, k, ld, u, theta, hd, guard, t,  \
                                                                               npk, part, dots, cnt);                \
    else                                                                                                             \
      k_residual_precond_u<T, false, 2, KM><<<nb, VK_THREADS, 0, ctx->stream>>>(B, S, k, ld, u, theta, hd, guard, t, \
                                                                                npk, part, rnorm2, cnt);             \
  } while (0)
  if (pk && k <= 4)
    FORTE_RESID_U(4);
  else if (pk && k <= 8)
    FORTE_RESID_U(8);
  else if (pk && k <= 16 && sizeof(T) == 4)  // FP64 accumulators for 16 vectors would spill
    FORTE_RESID_U(16);
#undef FORTE_RESID_U
  else if (pk && dots)
    k_residual_precond_p<T, true, 2><<<nb, VK_THREADS, 0, ctx->stream>>>(B, S, k, ld, u, theta, hd, guard, t, npk,
                                                                         part, dots, cnt);
  else if (pk)
    k_residual_precond_p<T, false, 2><<<nb, VK_THREADS, 0, ctx->stream>>>(B, S, k, ld, u, theta, hd, guard, t, npk,
                                                                          part, rnorm2, cnt);
  else
    k_residual_precond<T><<<nb, VK_THREADS, 0, ctx->stream>>>(B, S, k, ld, u, theta, ctx->d_hdiag, guard, t, n,
                                                              part, rnorm2, cnt);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

// d[i] *= s (i < k), d[k] *= s^2: dots and squared norm of a vector scaled by s
__global__ void k_rescale_dots(double *d, int k, double s) {
  for (int i = threadIdx.x; i <= k; i += blockDim.x) d[i] *= (i < k) ? s : s * s;
}
static int vk_rescale_dots(forte_ctx *ctx, double *d, int k, double s) {
  FORTE_PROF(ctx, "rescale_dots");
  k_rescale_dots<<<1, 64, 0, ctx->stream>>>(d, k, s);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

template <typename T>
static int vk_orth_update_t(forte_ctx *ctx, const T *B, int k, long long ld, const double *c, const T *t_in,
                            T *t_out, double *dots_out, long long n, bool dots, double scale) {
  if (k + 1 > VK_MAXV) { set_error("orth: subspace too large (%d)", k); return FORTE_ERR_ARG; }
  const bool pk = vp_ok<T>(n, ld, {B, t_in, t_out});
  const unsigned nb = pk ? vp_grid(ctx, n / Pk<T>::P) : vk_blocks(n);
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, (size_t)nb * (k + 1), &part, &cnt);
  if (rc) return rc;
  if (!pk && scale != 1.0) {  // element path: the scale is a separate pass
    if ((rc = vk_orth_update_t(ctx, B, k, ld, c, t_in, t_out, dots_out, n, dots, 1.0))) return rc;
    if ((rc = vk_scale(ctx, t_out, t_out, scale, n))) return rc;
    // |t_out|^2 and the dots scale with scale^2 and scale
    return vk_rescale_dots(ctx, dots_out, k, scale);
  }
  FORTE_PROF(ctx, "orth_update");
  const long long npk = n / Pk<T>::P;
#define FORTE_ORTH_U(KM)                                                                                    \
  do {                                                                                                      \
    if (dots)                                                                                               \
      k_orth_update_u<T, true, KM><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, npk, scale, \
                                                                       part, dots_out, cnt);                \
    else                                                                                                    \
      k_orth_update_u<T, false, KM><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, npk,      \
                                                                        scale, part, dots_out, cnt);        \
  } while (0)
  if (pk && k <= 4)
    FORTE_ORTH_U(4);
  else if (pk && k <= 8)
    FORTE_ORTH_U(8);
  else if (pk && k <= 16 && sizeof(T) == 4)
    FORTE_ORTH_U(16);
#undef FORTE_ORTH_U
  else if (pk && dots)
    k_orth_update_p<T, true><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, n / Pk<T>::P, scale,
                                                                 part, dots_out, cnt);
  else if (pk)
    k_orth_update_p<T, false><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, n / Pk<T>::P, scale,
                                                                  part, dots_out, cnt);
  else if (dots)
    k_orth_update<T, true><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, n, part, dots_out, cnt);
  else
    k_orth_update<T, false><<<nb, VK_THREADS, 0, ctx->stream>>>(B, k, ld, c, t_in, t_out, n, part, dots_out, cnt);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

template <typename T>
static int vk_scale_t(forte_ctx *ctx, T *x, const T *src, double alpha, long long n) {
  FORTE_PROF(ctx, "scale");
  if (vp_ok<T>(n, n, {x, src})) {
    const long long np = n / Pk<T>::P;
    k_scale_p<T><<<(unsigned)std::min<long long>((np + 255) / 256, 152LL * 16), 256, 0, ctx->stream>>>(x, src, alpha,
                                                                                                       np);
  } else {
    k_scale<T><<<(unsigned)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, ctx->stream>>>(x, src, alpha, n);
  }
  FORTE_LAUNCH_CHECK();
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
                        double theta, double guard, double *t, double *rnorm2, long long n, double *dots) {
  return vk_residual_precond_t(ctx, B, S, k, ld, u, theta, guard, t, rnorm2, n, dots);
}
int vk_residual_precond(forte_ctx *ctx, const float *B, const float *S, int k, long long ld, const double *u,
                        double theta, double guard, float *t, double *rnorm2, long long n, double *dots) {
  return vk_residual_precond_t(ctx, B, S, k, ld, u, theta, guard, t, rnorm2, n, dots);
}
int vk_orth_update(forte_ctx *ctx, const double *B, int k, long long ld, const double *c, const double *t_in,
                   double *t_out, double *dots_out, long long n, bool dots, double scale) {
  return vk_orth_update_t(ctx, B, k, ld, c, t_in, t_out, dots_out, n, dots, scale);
}
int vk_orth_update(forte_ctx *ctx, const float *B, int k, long long ld, const double *c, const float *t_in,
                   float *t_out, double *dots_out, long long n, bool dots, double scale) {
  return vk_orth_update_t(ctx, B, k, ld, c, t_in, t_out, dots_out, n, dots, scale);
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
  FORTE_PROF(ctx, "axpby");
  if (vp_ok<double>(n, n, {x, y})) {
    const long long np = n / 2;
    k_axpby_p<<<(unsigned)std::min<long long>((np + 255) / 256, 152LL * 16), 256, 0, ctx->stream>>>(a, x, b, y, np);
  } else {
    k_axpby<<<(unsigned)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, ctx->stream>>>(a, x, b, y, n);
  }
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

int vk_precond_inv(forte_ctx *ctx, double theta, double guard, double *rinv, long long n) {
  FORTE_PROF(ctx, "precond_inv");
  k_precond_inv<<<(unsigned)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, ctx->stream>>>(
      ctx->d_hdiag, theta, guard, rinv, n);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

int vk_precond_dot(forte_ctx *ctx, const double *r, const double *rinv, double *z, double *dot_out, long long n) {
  const bool pk = vp_ok<double>(n, n, {r, z, rinv});
  const unsigned nb = pk ? vp_grid(ctx, n / 2) : vk_blocks(n);
  double *part;
  unsigned *cnt;
  int rc = part_buffer(ctx, (size_t)2 * nb, &part, &cnt);
  if (rc) return rc;
  FORTE_PROF(ctx, "precond_dot");
  if (pk)
    k_precond_dot_p<<<nb, VK_THREADS, 0, ctx->stream>>>(r, rinv, z, n / 2, part, dot_out, cnt);
  else
    k_precond_dot<<<nb, VK_THREADS, 0, ctx->stream>>>(r, rinv, z, n, part, dot_out, cnt);
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
