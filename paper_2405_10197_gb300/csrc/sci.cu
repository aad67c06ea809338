// Sigma over an arbitrary list of determinants (the selected-CI data path of
// Sec. II.A.2, adaptive CI): S[v][i] = sum_j <D_i|H|D_j> C[v][j], H of Eq. 1.
//
// Determinants are 64-bit words over 2n spin orbitals (n <= 32): alpha orbital p
// at bit p, beta orbital p at bit n + p, creation operators ordered by spin
// orbital index (alpha before beta).  The list is arbitrary (any order, any mix of
// (n_alpha, n_beta) sectors); the matrix elements follow the Slater-Condon rules,
// evaluated on the device from the spin-free integrals.
//
// Design (one GPU, lists of ~1e3 .. 1e6 determinants): every pair (i, j) is
// screened by popcount(D_i ^ D_j) <= 4, as in an N-body kernel: a thread owns one
// determinant i, the block stages tiles of the j list (words and coefficients) in
// shared memory, and the j range is split over blockIdx.y so that short lists
// still fill the SMs.  Pairs that pass the screen evaluate <D_i|H|D_j> and
// accumulate; the per-split partial sums are added in a fixed order by a second
// kernel (deterministic).  The diagonal <D_i|H|D_i> is formed once per i in the
// pass, like any other pair.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "forte_internal.h"

struct forte_sci {
  int n = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  double *d_h = nullptr;    // [n][n]
  double *d_eri = nullptr;  // [n][n][n][n], chemist order
  forte::Scratch part;      // partial sums [split][nvec][ndet]
};

namespace forte {
namespace {

constexpr int SCI_THREADS = 128;
constexpr int SCI_TILE = 256;  // j determinants staged per pass
constexpr int SCI_NV = 4;      // vectors per launch

__device__ __forceinline__ int below(uint64_t d, int P) {  // occupied spin orbitals below P
  return __popcll(d & ((1ull << P) - 1ull));
}

// <D_I|H|D_J> for words that differ in at most 4 bits and lie in the same
// (n_alpha, n_beta) sector.  Spin orbital P: spatial P % n, spin P / n; the
// antisymmetrised integral <PQ||RS> = <PQ|RS> - <PQ|SR>, <PQ|RS> = (pr|qs) when
// spin(P) = spin(R) and spin(Q) = spin(S), else 0.
__device__ double sc_element(int n, const double *__restrict__ h, const double *__restrict__ eri, uint64_t I,
                             uint64_t J) {
  const uint64_t x = I ^ J;
  const int nd = __popcll(x);
  const long long n2 = (long long)n * n, n3 = n2 * n;
  auto g = [&](int p, int q, int r, int s) -> double { return __ldg(eri + p * n3 + q * n2 + r * n + s); };
  if (nd == 0) {
    // sum_P h_PP + sum_{P<Q} <PQ||PQ>
    double e = 0.0;
    for (uint64_t a = I; a; a &= a - 1) {
      const int P = __ffsll((long long)a) - 1, p = P % n;
      e += __ldg(h + p * n + p);
      for (uint64_t b = a & (a - 1); b; b &= b - 1) {
        const int Q = __ffsll((long long)b) - 1, q = Q % n;
        e += g(p, p, q, q);
        if (P / n == Q / n) e -= g(p, q, q, p);
      }
    }
    return e;
  }
  if (nd == 2) {
    // D_I = a+_M a_R D_J: M in I only, R in J only, same spin
    const uint64_t mi = x & I, rj = x & J;
    const int M = __ffsll((long long)mi) - 1, R = __ffsll((long long)rj) - 1;
    if (M / n != R / n) return 0.0;
    const int m = M % n, r = R % n;
    // phase of a+_M a_R on D_J
    const uint64_t t = J & ~(1ull << R);
    const int ph = ((below(J, R) + below(t, M)) & 1) ? -1 : 1;
    double v = __ldg(h + m * n + r);
    for (uint64_t a = t; a; a &= a - 1) {  // K in J, K != R
      const int K = __ffsll((long long)a) - 1, k = K % n;
      v += g(m, r, k, k);
      if (K / n == M / n) v -= g(m, k, k, r);
    }
    return ph * v;
  }
  if (nd == 4) {
    // D_I = a+_M a+_O a_S a_R D_J with M < O in I only, R < S in J only:
    // <MO||RS> times the phase of the operator string applied to D_J
    uint64_t mi = x & I, rj = x & J;
    const int M = __ffsll((long long)mi) - 1;
    mi &= mi - 1;
    const int O = __ffsll((long long)mi) - 1;
    const int R = __ffsll((long long)rj) - 1;
    rj &= rj - 1;
    const int S = __ffsll((long long)rj) - 1;
    uint64_t t = J;
    int c = below(t, R);
    t &= ~(1ull << R);
    c += below(t, S);
    t &= ~(1ull << S);
    c += below(t, O);
    t |= 1ull << O;
    c += below(t, M);
    const int sM = M / n, sO = O / n, sR = R / n, sS = S / n;
    double v = 0.0;
    if (sM == sR && sO == sS) v += g(M % n, R % n, O % n, S % n);  // <MO|RS> = (mr|os)
    if (sM == sS && sO == sR) v -= g(M % n, S % n, O % n, R % n);  // <MO|SR> = (ms|or)
    return (c & 1) ? -v : v;
  }
  return 0.0;
}

// part[y][v][i] = sum over the j of split y of <D_i|H|D_j> C[v0 + v][j], v < nv.
__global__ void __launch_bounds__(SCI_THREADS) k_sci_sigma(int n, const double *__restrict__ h,
                                                            const double *__restrict__ eri, long long nd,
                                                            const uint64_t *__restrict__ dets,
                                                            const double *__restrict__ C, int v0, int nv,
                                                            long long jchunk, double *__restrict__ part) {
  __shared__ uint64_t sd[SCI_TILE];
  __shared__ double sc[SCI_NV][SCI_TILE];
  const long long i = (long long)blockIdx.x * SCI_THREADS + threadIdx.x;
  const uint64_t amask = (n >= 32) ? 0xFFFFFFFFull : ((1ull << n) - 1ull);
  const uint64_t I = i < nd ? dets[i] : 0ull;
  const int na = __popcll(I & amask), nb = __popcll(I & ~amask);
  double acc[SCI_NV] = {0.0, 0.0, 0.0, 0.0};
  const long long j0 = (long long)blockIdx.y * jchunk, j1 = min(nd, j0 + jchunk);
  for (long long t0 = j0; t0 < j1; t0 += SCI_TILE) {
    const int tj = (int)min((long long)SCI_TILE, j1 - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < tj; k += SCI_THREADS) {
      sd[k] = dets[t0 + k];
      for (int v = 0; v < nv; ++v) sc[v][k] = C[(long long)(v0 + v) * nd + t0 + k];
    }
    __syncthreads();
    if (i < nd) {
      for (int k = 0; k < tj; ++k) {
        const uint64_t J = sd[k];
        if (__popcll(I ^ J) > 4) continue;
        if (__popcll(J & amask) != na || __popcll(J & ~amask) != nb) continue;
        const double hij = sc_element(n, h, eri, I, J);
        for (int v = 0; v < nv; ++v) acc[v] = fma(hij, sc[v][k], acc[v]);
      }
    }
  }
  if (i < nd)
    for (int v = 0; v < nv; ++v) part[((long long)blockIdx.y * nv + v) * nd + i] = acc[v];
}

// S[v0 + v][i] = sum over y of part[y][v][i], in split order.
__global__ void k_sci_reduce(const double *__restrict__ part, int ns, int nv, long long nd, int v0,
                             double *__restrict__ S) {
  const long long tot = (long long)nv * nd;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int y = 0; y < ns; ++y) s += part[(long long)y * tot + e];
    S[(long long)v0 * nd + e] = s;
  }
}

}  // namespace
}  // namespace forte

using namespace forte;

extern "C" {

forte_sci *forte_sci_create(int norb, const double *h, const double *eri) {
  clear_error();
  if (norb < 1 || norb > 32) {
    set_error("forte_sci_create: norb must be in 1..32 (2 norb spin orbitals in a 64-bit word)");
    return nullptr;
  }
  if (!h || !eri) {
    set_error("forte_sci_create: NULL integrals");
    return nullptr;
  }
  const size_t n = (size_t)norb, n4 = n * n * n * n;
  for (size_t k = 0; k < n * n; ++k)
    if (!std::isfinite(h[k])) { set_error("forte_sci_create: h contains NaN/Inf"); return nullptr; }
  for (size_t k = 0; k < n4; ++k)
    if (!std::isfinite(eri[k])) { set_error("forte_sci_create: eri contains NaN/Inf"); return nullptr; }
  forte_sci *s = new forte_sci();
  s->n = norb;
  if (cudaGetDevice(&s->device) != cudaSuccess || cudaMalloc(&s->d_h, sizeof(double) * n * n) != cudaSuccess ||
      cudaMalloc(&s->d_eri, sizeof(double) * n4) != cudaSuccess ||
      cudaMemcpy(s->d_h, h, sizeof(double) * n * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_eri, eri, sizeof(double) * n4, cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("forte_sci_create: device allocation or copy failed");
    cudaFree(s->d_h);
    cudaFree(s->d_eri);
    delete s;
    return nullptr;
  }
  return s;
}

void forte_sci_destroy(forte_sci *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaFree(s->d_h);
  cudaFree(s->d_eri);
  s->part.release();
  delete s;
}

int forte_sci_set_stream(forte_sci *s, void *cuda_stream) {
  if (!s) { set_error("NULL handle"); return FORTE_ERR_ARG; }
  s->stream = (cudaStream_t)cuda_stream;
  return FORTE_OK;
}

int forte_sci_sigma(forte_sci *s, long long ndet, const uint64_t *dets, const double *C, double *S, int nvec) {
  if (!s) { set_error("NULL handle"); return FORTE_ERR_ARG; }
  if (ndet < 0 || nvec < 0) { set_error("forte_sci_sigma: ndet and nvec must be >= 0"); return FORTE_ERR_ARG; }
  if (ndet == 0 || nvec == 0) return FORTE_OK;
  if (!dets || !C || !S) { set_error("forte_sci_sigma: NULL argument"); return FORTE_ERR_ARG; }
  if (ndet > (1LL << 31)) { set_error("forte_sci_sigma: at most 2^31 determinants"); return FORTE_ERR_ARG; }
  int nsm = 0;
  FORTE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device));
  const long long nbx = (ndet + SCI_THREADS - 1) / SCI_THREADS;
  // split the j range so that about 8 blocks per SM are in flight, each split at
  // least one tile long
  long long ns = std::max(1LL, std::min((8LL * nsm + nbx - 1) / nbx, (ndet + SCI_TILE - 1) / SCI_TILE));
  ns = std::min(ns, 65535LL);
  const long long jchunk = ((ndet + ns - 1) / ns + SCI_TILE - 1) / SCI_TILE * SCI_TILE;
  ns = (ndet + jchunk - 1) / jchunk;
  const int nvl = std::min(nvec, SCI_NV);
  int rc = s->part.ensure(sizeof(double) * (size_t)ns * nvl * ndet);
  if (rc) return rc;
  double *part = (double *)s->part.ptr;
  for (int v0 = 0; v0 < nvec; v0 += SCI_NV) {
    const int nv = std::min(SCI_NV, nvec - v0);
    dim3 grid((unsigned)nbx, (unsigned)ns);
    k_sci_sigma<<<grid, SCI_THREADS, 0, s->stream>>>(s->n, s->d_h, s->d_eri, ndet, dets, C, v0, nv, jchunk, part);
    FORTE_LAUNCH_CHECK();
    const long long tot = (long long)nv * ndet;
    k_sci_reduce<<<(unsigned)std::min<long long>((tot + 255) / 256, 152LL * 16), 256, 0, s->stream>>>(
        part, (int)ns, nv, ndet, v0, S);
    FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

}  // extern "C"
