// Host set-up of a CAS problem: string enumeration and addressing (a1), the
// signed single-replacement lists (a2) and the same-spin string Hamiltonian
// in CSR form (a3).
//
// Strings of one spin are the n-bit masks with n_sigma bits set (Sec. II.A.1,
// string-based CI).  They are generated in ascending order with the
// next-combination bit trick, and the address of a string is its
// colexicographic rank  r(S) = sum_k C(p_k, k+1)  over its occupied orbitals
// p_0 < p_1 < ...; the paper's hash-table addressing is replaced by this
// closed form, which needs no lookup.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>

#include "forte_internal.h"

namespace forte {

static long long binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

static long long colex_rank(uint32_t s) {
  long long r = 0;
  int k = 0;
  while (s) {
    int p = __builtin_ctz(s);
    r += binom(p, k + 1);
    ++k;
    s &= s - 1;
  }
  return r;
}

// Phase of a+_p a_q on string s (q occupied; p empty or p == q):
// (-1)^(number of occupied orbitals strictly between p and q).
static int repl_sign(uint32_t s, int p, int q) {
  if (p == q) return 1;
  int lo = p < q ? p : q, hi = p < q ? q : p;
  uint32_t between = ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
  return (__builtin_popcount(s & between) & 1) ? -1 : 1;
}

static int pair_index(int p, int q) {
  int a = p > q ? p : q, b = p > q ? q : p;
  return a * (a + 1) / 2 + b;
}

static int build_one_spin(forte_ctx *ctx, SpinHost &S, int nel) {
  const int n = ctx->n;
  S.nel = nel;
  S.N = binom(n, nel);
  S.nk = nel * (n - nel) + nel;
  S.str.resize(S.N);
  // ascending masks with nel bits
  if (nel == 0) {
    S.str[0] = 0u;
  } else {
    uint32_t v = (nel >= 32) ? 0xffffffffu : ((1u << nel) - 1u);
    for (long long i = 0; i < S.N; ++i) {
      S.str[i] = v;
      uint32_t t = v | (v - 1u);
      v = (t + 1u) | (((~t & -~t) - 1u) >> (__builtin_ctz(v) + 1));
    }
  }
  for (long long i = 0; i < S.N; ++i) {
    if (colex_rank(S.str[i]) != i) {
      set_error("internal: colex rank mismatch at string %lld", i);
      return FORTE_ERR_ARG;
    }
  }
  // compact replacement lists, entries sorted by p*n+q
  S.list.assign((size_t)S.N * S.nk, Repl{});
  for (long long I = 0; I < S.N; ++I) {
    uint32_t s = S.str[I];
    int c = 0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        if (!((s >> q) & 1u)) continue;
        if (p != q && ((s >> p) & 1u)) continue;
        uint32_t t = (s & ~(1u << q)) | (1u << p);
        Repl r;
        r.J = (int)colex_rank(t);
        r.sgn = (int8_t)repl_sign(s, p, q);
        r.pq = (uint8_t)(p * n + q);
        r.pair = (uint8_t)pair_index(p, q);
        r.pad = 0;
        S.list[(size_t)I * S.nk + c++] = r;
      }
    if (c != S.nk) {
      set_error("internal: replacement count %d != %d", c, S.nk);
      return FORTE_ERR_ARG;
    }
  }
  // Same-spin string Hamiltonian  H_ss = sum_pq k_pq E_pq + 1/2 sum (pq|rs) E_pq E_rs,
  // column J built by applying it to |J>; H_ss is symmetric, so column J is row J.
  const long long N = S.N;
  const int nk = S.nk;
  const double *g = ctx->eri.data();
  const double *km = ctx->kmat.data();
  std::vector<std::vector<int>> rc(N);
  std::vector<std::vector<double>> rv(N);
  auto worker = [&](long long j0, long long j1) {
    std::vector<double> acc(N, 0.0);
    std::vector<char> mark(N, 0);
    std::vector<long long> touched;
    touched.reserve(1 + nk * nk);
    for (long long J = j0; J < j1; ++J) {
      touched.clear();
      for (int e = 0; e < nk; ++e) {
        const Repl &re = S.list[(size_t)J * nk + e];
        int pe = re.pq / n, qe = re.pq % n;
        long long K = re.J;
        if (!mark[K]) { mark[K] = 1; touched.push_back(K); }
        acc[K] += km[pe * n + qe] * re.sgn;
        for (int f = 0; f < nk; ++f) {
          const Repl &rf = S.list[(size_t)K * nk + f];
          int pf = rf.pq / n, qf = rf.pq % n;
          long long I = rf.J;
          double gv = g[(((size_t)pf * n + qf) * n + pe) * n + qe];
          if (!mark[I]) { mark[I] = 1; touched.push_back(I); }
          acc[I] += 0.5 * gv * re.sgn * rf.sgn;
        }
      }
      std::sort(touched.begin(), touched.end());
      rc[J].resize(touched.size());
      rv[J].resize(touched.size());
      for (size_t t = 0; t < touched.size(); ++t) {
        rc[J][t] = (int)touched[t];
        rv[J][t] = acc[touched[t]];
        acc[touched[t]] = 0.0;
        mark[touched[t]] = 0;
      }
    }
  };
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (N < 256) nth = 1;
  std::vector<std::thread> th;
  long long chunk = (N + nth - 1) / nth;
  for (unsigned t = 0; t < nth; ++t) {
    long long a = t * chunk, b = std::min(N, a + chunk);
    if (a < b) th.emplace_back(worker, a, b);
  }
  for (auto &x : th) x.join();
  S.csr_ptr.assign(N + 1, 0);
  for (long long I = 0; I < N; ++I) S.csr_ptr[I + 1] = S.csr_ptr[I] + (int)rc[I].size();
  S.csr_col.resize(S.csr_ptr[N]);
  S.csr_val.resize(S.csr_ptr[N]);
  S.diag.assign(N, 0.0);
  for (long long I = 0; I < N; ++I) {
    std::copy(rc[I].begin(), rc[I].end(), S.csr_col.begin() + S.csr_ptr[I]);
    std::copy(rv[I].begin(), rv[I].end(), S.csr_val.begin() + S.csr_ptr[I]);
    for (size_t t = 0; t < rc[I].size(); ++t)
      if (rc[I][t] == I) S.diag[I] = rv[I][t];
  }
  return FORTE_OK;
}

cudaError_t set_smem_optin_max(const void *func) {
  int dev = 0, mx = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  // the limit covers static + dynamic shared memory
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
}

int build_spin_tables(forte_ctx *ctx) {
  const int n = ctx->n;
  ctx->kmat.assign((size_t)n * n, 0.0);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double v = ctx->h[p * n + q];
      for (int r = 0; r < n; ++r) v -= 0.5 * ctx->eri[(((size_t)p * n + r) * n + r) * n + q];
      ctx->kmat[p * n + q] = v;
    }
  int st = build_one_spin(ctx, ctx->sh[0], ctx->na);
  if (st) return st;
  if (ctx->same_strings) return FORTE_OK;
  return build_one_spin(ctx, ctx->sh[1], ctx->nb);
}

template <typename T>
static int upload(T **dst, const T *src, size_t count) {
  size_t bytes = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc((void **)dst, bytes);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return FORTE_ERR_ALLOC;
  }
  if (count) FORTE_CUDA_TRY(cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
  return FORTE_OK;
}

int upload_tables(forte_ctx *ctx) {
  int nsp = ctx->same_strings ? 1 : 2;
  for (int s = 0; s < nsp; ++s) {
    SpinHost &H = ctx->sh[s];
    SpinDev &D = ctx->sd[s];
    int st;
    if ((st = upload(&D.list, H.list.data(), H.list.size()))) return st;
    if ((st = upload(&D.csr_ptr, H.csr_ptr.data(), H.csr_ptr.size()))) return st;
    if ((st = upload(&D.csr_col, H.csr_col.data(), H.csr_col.size()))) return st;
    if ((st = upload(&D.csr_val, H.csr_val.data(), H.csr_val.size()))) return st;
    std::vector<float> v32(H.csr_val.begin(), H.csr_val.end());
    if ((st = upload(&D.csr_val32, v32.data(), v32.size()))) return st;
    if ((st = upload(&D.str, H.str.data(), H.str.size()))) return st;
    if ((st = upload(&D.diag, H.diag.data(), H.diag.size()))) return st;
    const int n = ctx->n, n2 = n * n;
    std::vector<int> dense((size_t)H.N * n2, -1);
    for (long long I = 0; I < H.N; ++I)
      for (int e = 0; e < H.nk; ++e) {
        const Repl &r = H.list[(size_t)I * H.nk + e];
        dense[(size_t)I * n2 + r.pq] = (r.J << 1) | (r.sgn < 0 ? 1 : 0);
      }
    if ((st = upload(&D.dense, dense.data(), dense.size()))) return st;
    if (H.N <= 65536) {
      std::vector<uint32_t> l4(H.list.size());
      for (size_t i = 0; i < l4.size(); ++i) {
        const Repl &r = H.list[i];
        l4[i] = (uint32_t)r.J | ((uint32_t)r.pair << 16) | (r.sgn < 0 ? 0x80000000u : 0u);
      }
      if ((st = upload(&D.list4, l4.data(), l4.size()))) return st;
    }
    if (H.N < 16384 && ctx->npair <= 128) {
      std::vector<uint16_t> tab((size_t)H.N * 128, 0xFFFFu);
      for (long long J = 0; J < H.N; ++J)
        for (int e = 0; e < H.nk; ++e) {
          const Repl &r = H.list[(size_t)J * H.nk + e];
          tab[(size_t)J * 128 + r.pair] = (uint16_t)(r.J | (r.sgn < 0 ? 0x4000 : 0));
        }
      if ((st = upload(&D.tabJ, tab.data(), tab.size()))) return st;
    }
  }
  if (ctx->same_strings) ctx->sd[1] = ctx->sd[0];
  // (pq|rs) over symmetric pairs
  const int n = ctx->n, np = ctx->npair;
  std::vector<double> gp((size_t)np * np, 0.0);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q <= p; ++q)
      for (int r = 0; r < n; ++r)
        for (int s = 0; s <= r; ++s)
          gp[(size_t)pair_index(p, q) * np + pair_index(r, s)] =
              ctx->eri[(((size_t)p * n + q) * n + r) * n + s];
  int st;
  if ((st = upload(&ctx->d_gpair, gp.data(), gp.size()))) return st;
  std::vector<float> gp32(gp.begin(), gp.end());
  if ((st = upload(&ctx->d_gpair32, gp32.data(), gp32.size()))) return st;
  return FORTE_OK;
}

int Scratch::ensure(size_t want) {
  if (want <= bytes) return FORTE_OK;
  if (ptr) {
    // queued kernels may still read the old buffer
    cudaDeviceSynchronize();
    cudaFree(ptr);
  }
  ptr = nullptr;
  bytes = 0;
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    ptr = nullptr;
    set_error("cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    return FORTE_ERR_ALLOC;
  }
  bytes = want;
  return FORTE_OK;
}

void Scratch::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

}  // namespace forte
