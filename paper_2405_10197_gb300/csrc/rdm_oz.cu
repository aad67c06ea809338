// Spin-free 2-RDM Gram matrix on the 5th-generation tensor cores (step a9,
// Sec. II.A.1, Eq. (gamma_2)), used by the reduced-precision modes.
//
// The 2-RDM is the Gram matrix M[a][b] = <D^a, D^b> of the one-body images
// D^{rs} = E_rs |C> (Gamma_pqrs = M[(q,p),(r,s)] - d_qr gamma_ps).  Two facts cut
// its cost:
//
// 1. Symmetric / antisymmetric split.  With u_{rs} = D^{rs} + D^{sr} (r > s),
//    u_{rr} = D^{rr} and v_{rs} = D^{rs} - D^{sr} (r > s), the cross products are
//    fixed by the 1-RDM: for real C and the commutator [E_pq, E_rs] =
//    d_qr E_ps - d_ps E_rq,
//      <D^{rs} + D^{sr}, D^{pq} - D^{qp}> = d_rp g_sq - d_sq g_pr - d_rq g_sp + d_sp g_qr.
//    Only the two Gram matrices G+ = <u,u> (n(n+1)/2 rows) and G- = <v,v>
//    (n(n-1)/2 rows) are formed over the determinants: half of the n^2 x n^2 work.
//
// 2. Exact integer products on the BF16 tensor cores (the splitting scheme of
//    Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012) 95, with the
//    integer slices of its later tensor-core variants).  C is turned into 52-bit
//    fixed point, each row of u (or v) is shifted so that |X| <= 2^45, and X is
//    written as six balanced base-256 digits X = sum_i d_i 256^(6-i), |d_1| <= 32,
//    d_2..d_6 in [-128, 127]; every digit is exact in BF16.  For a chunk of 64
//    determinants the level sums  L_t = sum_{i+j=t} sum_k d_i(a,k) d_j(b,k),
//    t = 2..8, are integers below 2^23 and are summed exactly by the MMA in FP32
//    (one TMEM accumulator per level).  Pairs with i + j > 8 are dropped: their
//    weight is at most 2^-49.99 of 64 times the product of the two row maxima.  The epilogue
//    folds the levels into one 64-bit integer per Gram element (units of 2^6 L_8,
//    the only rounding being L_7 and L_8 to even integers and L_8 to units of
//    2^5) and flushes it to an FP64 partial sum every 16 chunks.
//
// Kernel structure (one CTA per SM, persistent over alpha strings Ia; 20 warps):
//   * warps 0-2 (producers) form u or v for the 64 determinants (Ia, Ib0..Ib0+63)
//     of a chunk from the fixed-point C (alpha part: rows C[E_sr Ia, :], beta
//     part: the row C[Ia, :] staged in shared memory), digit them and write the
//     six K-major, 128-byte-swizzled digit slices of a 2-deep stage ring;
//   * one thread of warp 3 issues, per level, the tcgen05.mma chain into one of
//     four TMEM accumulators (M = 128 rows, N = padded row count);
//   * warps 4-19 (epilogue) read each level with tcgen05.ld and accumulate.
// Every mbarrier wait is bounded (the context status word is raised on expiry,
// the other roles stop, TMEM is released).
#include <algorithm>
#include <type_traits>

#include "forte_internal.h"
#include "oz_digits.cuh"
#include "tc_ptx.cuh"

namespace forte {

constexpr int OZ_KC = 64;
constexpr int OZ_SLOTS = 4;
constexpr int OZ_PROD_WARPS = 3;
constexpr int OZ_MMA_WARP = OZ_PROD_WARPS;  // lane 0 issues the MMAs, the warp owns TMEM
constexpr int OZ_RB = 4;                    // rows per producer load batch
constexpr int OZ_EPI_WARPS = 16;
constexpr int OZ_THREADS = 32 * (OZ_PROD_WARPS + 1 + OZ_EPI_WARPS);  // 20 warps: 96 registers
constexpr int OZ_FLUSH = 16;
constexpr int OZ_CBITS = 52;        // |C_fix| <= 2^52

template <int N>
struct OzLayout {
  static constexpr int SLICE = N * 128;                              // N rows of 128 bytes
  static constexpr int STAGE = OZ_DIGITS * SLICE + (128 - N) * 128;  // A reads 128 rows of the last slice
  static constexpr int OFF_CROW = 2 * STAGE;
};

// ------------------------------------------------------------ small kernels

// amax = bits of max |x| (non-negative doubles order as their bit patterns)
__global__ void k_oz_absmax(const double *__restrict__ x, long long n, unsigned long long *amax) {
  __shared__ unsigned long long red[32];
  unsigned long long m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(fabs(x[i])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    atomicMax(amax, m);
  }
}

__device__ __forceinline__ int oz_cexp(const unsigned long long *amax) {
  const double cm = __longlong_as_double((long long)*amax);
  int e = 0;
  if (cm > 0.0) frexp(cm, &e);  // |C| <= cm < 2^e
  return e;
}

// Cfix[Ia][i] = rint(C[Ia][i] 2^(52 - e)), zero for the padding columns i >= NB.
__global__ void k_oz_cfix(const double *__restrict__ C, long long NA, long long NB, long long NbP,
                          const unsigned long long *__restrict__ amax, long long *__restrict__ Cfix) {
  const int e = oz_cexp(amax);
  const long long tot = NA * NbP;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / NbP, col = i % NbP;
    Cfix[i] = col < NB ? llrint(ldexp(C[row * NB + col], OZ_CBITS - e)) : 0LL;
  }
}

// T[ps][Ib] = E_sr |Ib> of the beta strings (ps = s n + r), as J | (sgn < 0) << 15,
// 0xFFFF where it vanishes or Ib >= NB.
__global__ void k_oz_denseT(const int *__restrict__ dense, int n2, long long NB, long long NbP,
                            uint16_t *__restrict__ T) {
  const long long tot = (long long)n2 * NbP;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long ps = i / NbP, ib = i % NbP;
    uint16_t w = 0xFFFFu;
    if (ib < NB) {
      const int x = dense[ib * n2 + ps];
      if (x >= 0) w = (uint16_t)((x >> 1) | ((x & 1) << 15));
    }
    T[i] = w;
  }
}

// Row (r, s) of the u rows (gram 0) or v rows (gram 1): pairs r > s first, in
// the order r(r-1)/2 + s, then (for u) the diagonal (r, r).
__device__ __forceinline__ void oz_row(int a, int n, int &r, int &s) {
  const int T = n * (n - 1) / 2;
  if (a >= T) {
    r = s = a - T;
    return;
  }
  int x = 1;
  while (x * (x + 1) / 2 <= a) ++x;
  r = x;
  s = a - x * (x - 1) / 2;
}

// x = (E_rs C)[Ia, Ib] for a pair of columns Ib, Ib+1 in fixed point:
// alpha part sgn C[E_sr Ia, Ib] (ea = (J << 1) | neg, or -1), beta part
// sgn C[Ia, E_sr Ib] from the staged row (tb = the two 16-bit table entries).
__device__ __forceinline__ void oz_pair(int ea, uint32_t tb, const long long *__restrict__ Cfix, long long NbP,
                                        long long Ib, const long long *crow, long long &x0, long long &x1) {
  x0 = 0;
  x1 = 0;
  if (ea >= 0) {
    const longlong2 c = __ldg((const longlong2 *)(Cfix + (long long)(ea >> 1) * NbP + Ib));
    x0 = (ea & 1) ? -c.x : c.x;
    x1 = (ea & 1) ? -c.y : c.y;
  }
  const uint32_t w0 = tb & 0xFFFFu, w1 = tb >> 16;
  if (w0 != 0xFFFFu) {
    const long long c = crow[w0 & 0x7FFFu];
    x0 += (w0 & 0x8000u) ? -c : c;
  }
  if (w1 != 0xFFFFu) {
    const long long c = crow[w1 & 0x7FFFu];
    x1 += (w1 & 0x8000u) ? -c : c;
  }
}

__device__ __forceinline__ long long oz_value(int gram, int r, int s, long long xrs, long long xsr) {
  return gram ? xrs - xsr : (r == s ? xrs : xrs + xsr);
}

// rowmax[g][a] = max over determinants of |u_a| (g = 0) and |v_a| (g = 1).
// One block per alpha string; warp w takes the pairs r >= s with index w, w + 8, ...
// and forms D^{rs} and D^{sr} once for both u_rs = D^{rs} + D^{sr} and
// v_rs = D^{rs} - D^{sr} (u_rr = D^{rr}).
__global__ void __launch_bounds__(256) k_oz_rowmax(const long long *__restrict__ Cfix, const int *__restrict__ denseA,
                                                   const uint16_t *__restrict__ T, int n, long long NA, long long NB,
                                                   long long NbP, unsigned long long *__restrict__ rowmax) {
  extern __shared__ long long crow[];
  __shared__ int atab[256];
  const int n2 = n * n, nU = n * (n + 1) / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long Ia = blockIdx.x; Ia < NA; Ia += gridDim.x) {
    __syncthreads();
    for (long long i = threadIdx.x; i < NbP; i += blockDim.x) crow[i] = Cfix[Ia * NbP + i];
    for (int i = threadIdx.x; i < n2; i += blockDim.x) atab[i] = denseA[Ia * n2 + i];
    __syncthreads();
    for (int a = warp; a < nU; a += 8) {  // u row index a: pairs r > s first, then the diagonal
      int r, s;
      oz_row(a, n, r, s);
      const int e1 = atab[s * n + r], e2 = atab[r * n + s];
      const uint16_t *t1 = T + (size_t)(s * n + r) * NbP, *t2 = T + (size_t)(r * n + s) * NbP;
      unsigned long long mu = 0, mv = 0;
      for (long long Ib = 2 * lane; Ib < NB; Ib += 64) {
        long long a0, a1, b0 = 0, b1 = 0;
        oz_pair(e1, *(const uint32_t *)(t1 + Ib), Cfix, NbP, Ib, crow, a0, a1);
        if (r != s) oz_pair(e2, *(const uint32_t *)(t2 + Ib), Cfix, NbP, Ib, crow, b0, b1);
        const long long u0 = oz_value(0, r, s, a0, b0), u1 = oz_value(0, r, s, a1, b1);
        const long long v0 = a0 - b0, v1 = a1 - b1;
        mu = max(mu, (unsigned long long)(u0 < 0 ? -u0 : u0));
        mu = max(mu, (unsigned long long)(u1 < 0 ? -u1 : u1));
        mv = max(mv, (unsigned long long)(v0 < 0 ? -v0 : v0));
        mv = max(mv, (unsigned long long)(v1 < 0 ? -v1 : v1));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mu = max(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        mv = max(mv, __shfl_xor_sync(0xffffffffu, mv, o));
      }
      if (lane == 0 && mu) atomicMax(rowmax + a, mu);
      // the v rows are the pairs r > s in the same order (index a < n(n-1)/2)
      if (lane == 0 && mv && r != s) atomicMax(rowmax + 128 + a, mv);
    }
  }
}

// sh[g][a]: X = u >> sh (rounded) or u << -sh, so that |X| <= 2^45.
__global__ void k_oz_shift(const unsigned long long *__restrict__ rowmax, int *__restrict__ sh) {
  const int i = threadIdx.x;  // 256 = 2 x 128
  const unsigned long long m = rowmax[i];
  sh[i] = m ? (64 - __clzll((long long)m)) - OZ_XBITS : 0;
}

// ------------------------------------------------------------ digit slices

__device__ __forceinline__ long long oz_scale(long long u, int sh) {
  return sh > 0 ? ((u + (1LL << (sh - 1))) >> sh) : (u << (-sh));
}

// Six BF16 digit slices of X0 (column Ib) and X1 (column Ib+1), packed in pairs:
// out[i] holds digit d_(i+1) of both columns.
__device__ __forceinline__ void oz_digits2(long long X0, long long X1, uint32_t (&out)[OZ_DIGITS]) {
  const unsigned long long Y0 = (unsigned long long)X0 + 0x8080808080ull;
  const unsigned long long Y1 = (unsigned long long)X1 + 0x8080808080ull;
  const uint32_t l0 = (uint32_t)Y0, h0 = (uint32_t)(Y0 >> 32), l1 = (uint32_t)Y1, h1 = (uint32_t)(Y1 >> 32);
  const uint32_t f10 = __float_as_uint(__int_as_float(0x4B400000 + ((int)h0 >> 8)) - 12582912.0f);
  const uint32_t f11 = __float_as_uint(__int_as_float(0x4B400000 + ((int)h1 >> 8)) - 12582912.0f);
  out[0] = __byte_perm(f10, f11, 0x7632u);
  out[1] = __byte_perm(oz_dig(h0, 0), oz_dig(h1, 0), 0x7632u);
  out[2] = __byte_perm(oz_dig(l0, 3), oz_dig(l1, 3), 0x7632u);
  out[3] = __byte_perm(oz_dig(l0, 2), oz_dig(l1, 2), 0x7632u);
  out[4] = __byte_perm(oz_dig(l0, 1), oz_dig(l1, 1), 0x7632u);
  out[5] = __byte_perm(oz_dig(l0, 0), oz_dig(l1, 0), 0x7632u);
}

// Load W (<= 16, a multiple of 4) consecutive accumulator columns.
template <int W>
__device__ __forceinline__ void tmem_ldw(uint32_t taddr, uint32_t *r) {
  static_assert(W % 4 == 0 && W <= 16, "column block");
  if constexpr (W == 16) {
    tmem_ld16(taddr, r);
  } else {
    int o = 0;
    if constexpr ((W & 8) != 0) {
      tmem_ld8(taddr, r);
      o = 8;
    }
    if constexpr ((W & 4) != 0) tmem_ld4(taddr + o, r + o);
  }
  tmem_wait_ld();
}

// One level of one chunk in the epilogue: wait for the accumulator, read this
// warp's NC columns in blocks of 8 (4 for the tail), release the accumulator
// after the last read, fold the level into acc.
template <int T, int N>
__device__ __forceinline__ bool oz_epi_level(uint32_t tbase, int lane, long long &q, uint64_t *tfull,
                                             uint64_t *tempty, volatile int *sAbort,
                                             unsigned long long (&acc)[N / 4]) {
  constexpr int NC = N / 4;
  const int slot = (int)(q % OZ_SLOTS);
  if (!__all_sync(0xffffffffu, mbar_wait_ab(&tfull[slot], (uint32_t)((q / OZ_SLOTS) & 1), sAbort))) return false;
  tc_fence_after();
  const uint32_t taddr = tbase + (uint32_t)(slot * N);
#pragma unroll
  for (int h = 0; h < NC; h += 8) {
    uint32_t v[8];
    if (h + 8 <= NC) {
      tmem_ldw<8>(taddr + h, v);
    } else {
      tmem_ldw<4>(taddr + h, v);
    }
    if (h + 8 >= NC) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[slot]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (h + k < NC) oz_acc_level<T>(acc[h + k], v[k]);
  }
  ++q;
  return true;
}

// ------------------------------------------------------------ the Gram kernel

template <int N>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_gram_oz(int gram, int n, int nrows, const int *__restrict__ shv, const long long *__restrict__ Cfix,
              const int *__restrict__ denseA, const uint16_t *__restrict__ T, long long NA, long long NbP,
              double *__restrict__ part, int *__restrict__ err) {
  using L = OzLayout<N>;
  constexpr int NC = N / 4;  // accumulator columns per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  long long *crow = (long long *)(sm + L::OFF_CROW);
  int *atab = (int *)(crow + NbP);
  uint8_t *sR = (uint8_t *)(atab + 256);
  uint8_t *sS = sR + 128;
  int *sSh = (int *)(sS + 128);
  uint64_t *bar = (uint64_t *)(sSh + 128);
  uint64_t *full = bar, *empty = bar + 2, *tfull = bar + 4, *tempty = bar + 4 + OZ_SLOTS;
  uint64_t *rowbar = tempty + OZ_SLOTS;  // producer warps: staged row in use / ready
  uint32_t *sTmem = (uint32_t *)(rowbar + 1);
  volatile int *sAbort = (volatile int *)(sTmem + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n2 = n * n;
  const long long nunit = NA > blockIdx.x ? (NA - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nchunk = (int)(NbP / OZ_KC);
  const long long total = nunit * nchunk;

  if (warp == OZ_MMA_WARP) tmem_alloc(sTmem, 512);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], OZ_PROD_WARPS);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < OZ_SLOTS; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], OZ_EPI_WARPS);
    }
    mbar_init(rowbar, OZ_PROD_WARPS);
    abort_word_init(sAbort, err);
    fence_mbar_init();
  }
  if (tid < 128) {
    int r = 0, s = 0;
    if (tid < nrows) oz_row(tid, n, r, s);
    sR[tid] = (uint8_t)r;
    sS[tid] = (uint8_t)s;
    sSh[tid] = tid < nrows ? shv[gram * 128 + tid] : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  long long issued = 0;  // chunks whose MMAs were committed

  if (warp < OZ_PROD_WARPS) {
    // ================= producers
    long long it = 0;
    uint32_t rph = 0;
    bool ok = true;
    // all producer warps meet on rowbar (bounded): returns false on abort / expiry
    auto meet = [&]() {
      __syncwarp();
      if (lane == 0) mbar_arrive(rowbar);
      const bool w = __all_sync(0xffffffffu, mbar_wait_ab(rowbar, rph & 1u, sAbort));
      ++rph;
      return w;
    };
    for (long long Ia = blockIdx.x; Ia < NA && ok; Ia += gridDim.x) {
      if (!meet()) {  // the previous unit's row is no longer read
        ok = false;
        break;
      }
      for (long long i = tid; i < NbP / 2; i += 32 * OZ_PROD_WARPS)
        ((longlong2 *)crow)[i] = __ldg((const longlong2 *)(Cfix + Ia * NbP) + i);
      for (int i = tid; i < n2; i += 32 * OZ_PROD_WARPS) atab[i] = denseA[Ia * n2 + i];
      if (!meet()) {
        ok = false;
        break;
      }
      for (int kc = 0; kc < nchunk; ++kc, ++it) {
        const int st = (int)(it & 1);
        if (it >= 2 && !__all_sync(0xffffffffu, mbar_wait_ab(&empty[st], (uint32_t)(((it >> 1) - 1) & 1), sAbort))) {
          *sAbort = 1;
          atomicOr(err, 8);
          ok = false;
          break;
        }
        uint8_t *stage = sm + st * L::STAGE;
        const long long Ib = (long long)kc * OZ_KC + 2 * lane;
        // rows a = warp + PW (b + RB c): the global loads of RB rows are issued
        // together, then the rows are formed, digited and stored
        for (int a0 = warp; a0 < nrows; a0 += OZ_PROD_WARPS * OZ_RB) {
          int ea[OZ_RB][2];
          uint32_t tb[OZ_RB][2];
          longlong2 ca[OZ_RB][2];
#pragma unroll
          for (int b = 0; b < OZ_RB; ++b) {
            const int a = a0 + OZ_PROD_WARPS * b;
#pragma unroll
            for (int o = 0; o < 2; ++o) {
              ea[b][o] = -1;
              tb[b][o] = 0xFFFFFFFFu;
              ca[b][o] = make_longlong2(0, 0);
            }
            if (a < nrows) {
              const int r = sR[a], s = sS[a];
#pragma unroll
              for (int o = 0; o < 2; ++o) {
                if (o == 1 && r == s) break;
                const int ps = o ? r * n + s : s * n + r;
                ea[b][o] = atab[ps];
                tb[b][o] = __ldg((const uint32_t *)(T + (size_t)ps * NbP + Ib));
                if (ea[b][o] >= 0) ca[b][o] = __ldg((const longlong2 *)(Cfix + (long long)(ea[b][o] >> 1) * NbP + Ib));
              }
            }
          }
#pragma unroll
          for (int b = 0; b < OZ_RB; ++b) {
            const int a = a0 + OZ_PROD_WARPS * b;
            if (a >= nrows) break;
            const int r = sR[a], s = sS[a];
            long long x[2][2];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
              const bool neg = ea[b][o] & 1;
              x[o][0] = neg ? -ca[b][o].x : ca[b][o].x;
              x[o][1] = neg ? -ca[b][o].y : ca[b][o].y;
              const uint32_t w0 = tb[b][o] & 0xFFFFu, w1 = tb[b][o] >> 16;
              if (w0 != 0xFFFFu) {
                const long long c = crow[w0 & 0x7FFFu];
                x[o][0] += (w0 & 0x8000u) ? -c : c;
              }
              if (w1 != 0xFFFFu) {
                const long long c = crow[w1 & 0x7FFFu];
                x[o][1] += (w1 & 0x8000u) ? -c : c;
              }
            }
            const int sh = sSh[a];
            const long long X0 = oz_scale(oz_value(gram, r, s, x[0][0], x[1][0]), sh);
            const long long X1 = oz_scale(oz_value(gram, r, s, x[0][1], x[1][1]), sh);
            uint32_t w[OZ_DIGITS];
            oz_digits2(X0, X1, w);
            uint8_t *dst = stage + swz((uint32_t)a, 4u * lane);
#pragma unroll
            for (int d = 0; d < OZ_DIGITS; ++d) *(uint32_t *)(dst + d * L::SLICE) = w[d];
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[st]);
      }
    }
  } else if (warp == OZ_MMA_WARP) {
    // ================= MMA issuer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
      long long q = 0;
      for (long long it = 0; it < total; ++it) {
        const int st = (int)(it & 1);
        if (!mbar_wait_ab(&full[st], (uint32_t)((it >> 1) & 1), sAbort)) {
          *sAbort = 1;
          atomicOr(err, 8);
          break;
        }
        tc_fence_after();
        const uint64_t base = desc_kmajor_sw128(smem_u32(sm + st * L::STAGE));
        // one level: wait for its accumulator slot, issue its chain, commit
        auto level = [&](auto tc) -> bool {
          constexpr int T = decltype(tc)::value;
          const int slot = (int)(q % OZ_SLOTS);
          if (q >= OZ_SLOTS && !mbar_wait_ab(&tempty[slot], (uint32_t)(((q / OZ_SLOTS) - 1) & 1), sAbort)) return false;
          tc_fence_after();
          oz_issue_level<T, L::SLICE / 16, L::SLICE / 16, OZ_KC / 16>(tmem + (uint32_t)(slot * N), base, base, idesc);
          mma_commit(&tfull[slot]);
          ++q;
          return true;
        };
        const bool ok = level(std::integral_constant<int, 2>{}) && level(std::integral_constant<int, 3>{}) &&
                        level(std::integral_constant<int, 4>{}) && level(std::integral_constant<int, 5>{}) &&
                        level(std::integral_constant<int, 6>{}) && level(std::integral_constant<int, 7>{}) &&
                        level(std::integral_constant<int, 8>{});
        mma_commit(&empty[st]);  // also covers a chunk cut short by an abort
        issued = it + 1;
        if (!ok) {
          *sAbort = 1;
          atomicOr(err, 8);
          break;
        }
      }
    }
    __syncwarp();
  } else {
    // ================= epilogue: lane = Gram row, NC columns per warp
    const int quarter = warp & 3, cg = (warp - OZ_MMA_WARP - 1) >> 2;
    const int row = quarter * 32 + lane, col0 = cg * NC;
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
    unsigned long long acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0ull;
    long long q = 0;
    int nch = 0;
    bool first = true, ok = true;
    double *P = part + ((size_t)blockIdx.x * N + row) * N + col0;
    for (long long it = 0; it < total; ++it) {
      ok = oz_epi_level<2, N>(tbase, lane, q, tfull, tempty, sAbort, acc) &&
           oz_epi_level<3, N>(tbase, lane, q, tfull, tempty, sAbort, acc) &&
           oz_epi_level<4, N>(tbase, lane, q, tfull, tempty, sAbort, acc) &&
           oz_epi_level<5, N>(tbase, lane, q, tfull, tempty, sAbort, acc) &&
           oz_epi_level<6, N>(tbase, lane, q, tfull, tempty, sAbort, acc) &&
           oz_epi_level<7, N>(tbase, lane, q, tfull, tempty, sAbort, acc) &&
           oz_epi_level<8, N>(tbase, lane, q, tfull, tempty, sAbort, acc);
      if (!ok) {
        *sAbort = 1;
        atomicOr(err, 8);
        break;
      }
      if (++nch == OZ_FLUSH || it + 1 == total) {
        const unsigned long long bias = (unsigned long long)nch * oz_bias();
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          if (row < N) {  // TMEM lanes N..127 hold padding rows: the partials are [N][N]
            const double x = (double)(long long)(acc[k] - bias);
            P[k] = first ? x : P[k] + x;
          }
          acc[k] = 0ull;
        }
        first = false;
        nch = 0;
      }
    }
    if (first && ok && row < N) {
#pragma unroll
      for (int k = 0; k < NC; ++k) P[k] = 0.0;  // no work for this CTA
    }
  }
  __syncthreads();
  if (*sAbort) {
    if (warp == OZ_MMA_WARP && lane == 0) {
      // wait (bounded) for the last committed chunk's MMAs before TMEM is released
      if (issued > 0) mbar_wait(&empty[(int)((issued - 1) & 1)], (uint32_t)(((issued - 1) >> 1) & 1));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == OZ_MMA_WARP) tmem_dealloc(tmem, 512);
}

// G[a][b] = 2^(38 + sh_a + sh_b + 2(e - 52)) sum_cta part[cta][a][b]   (a, b < nrows)
__global__ void k_oz_reduce(const double *__restrict__ part, int ncta, int N, int nrows, const int *__restrict__ sh,
                            const unsigned long long *__restrict__ amax, double *__restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * nrows) return;
  const int a = i / nrows, b = i % nrows;
  double s = 0.0;
  for (int c = 0; c < ncta; ++c) s += part[((size_t)c * N + a) * N + b];
  const int e = oz_cexp(amax);
  G[i] = ldexp(s, 38 + sh[a] + sh[b] + 2 * (e - OZ_CBITS));
}

// Gamma_pqrs = M[(q,p),(r,s)] - d_qr g_ps, M assembled from G+ (rows u), G- (rows v)
// and the cross products given by the 1-RDM g.
__device__ __forceinline__ void oz_coef(int x, int y, int n, double &cu, double &cv, int &iu, int &iv) {
  const int T = n * (n - 1) / 2;
  if (x > y) {
    cu = 0.5; cv = 0.5; iu = iv = x * (x - 1) / 2 + y;
  } else if (x < y) {
    cu = 0.5; cv = -0.5; iu = iv = y * (y - 1) / 2 + x;
  } else {
    cu = 1.0; cv = 0.0; iu = T + x; iv = -1;
  }
}
__device__ __forceinline__ double oz_cross(int iu, int iv, int n, const double *__restrict__ g) {
  int r, s, p, q;
  oz_row(iu, n, r, s);
  oz_row(iv, n, p, q);
  double c = 0.0;
  if (r == p) c += g[s * n + q];
  if (s == q) c -= g[p * n + r];
  if (r == q) c -= g[s * n + p];
  if (s == p) c += g[q * n + r];
  return r == s ? 0.5 * c : c;
}
__global__ void k_oz_assemble(const double *__restrict__ Gu, const double *__restrict__ Gv, const double *__restrict__ g,
                              int n, double *__restrict__ g2) {
  const int n2 = n * n, nU = n * (n + 1) / 2, nV = n * (n - 1) / 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2 * n2) return;
  const int p = i / (n * n2), q = (i / n2) % n, r = (i / n) % n, s = i % n;
  double cu, cv, du, dv;
  int iu, iv, ju, jv;
  oz_coef(q, p, n, cu, cv, iu, iv);
  oz_coef(r, s, n, du, dv, ju, jv);
  double m = cu * du * Gu[iu * nU + ju];
  if (iv >= 0 && jv >= 0) m += cv * dv * Gv[iv * nV + jv];
  if (jv >= 0) m += cu * dv * oz_cross(iu, jv, n, g);
  if (iv >= 0) m += cv * du * oz_cross(ju, iv, n, g);
  if (q == r) m -= g[p * n + s];
  g2[i] = m;
}

// ------------------------------------------------------------ host side

static int oz_pad16(int x) { return ((x + 15) / 16) * 16; }

template <int N>
static size_t oz_smem(long long NbP) {
  return 1024 + (size_t)OzLayout<N>::OFF_CROW + 8 * (size_t)NbP + 4 * 256 + 128 + 128 + 4 * 128 +
         8 * (5 + 2 * OZ_SLOTS) + 32;
}

static size_t oz_smem_n(int N, long long NbP) {
  switch (N) {
    case 16: return oz_smem<16>(NbP);
    case 32: return oz_smem<32>(NbP);
    case 48: return oz_smem<48>(NbP);
    case 64: return oz_smem<64>(NbP);
    case 80: return oz_smem<80>(NbP);
    case 96: return oz_smem<96>(NbP);
    case 112: return oz_smem<112>(NbP);
    default: return oz_smem<128>(NbP);
  }
}

bool rdm2_oz_supported(const forte_ctx *ctx) {
  const int n = ctx->n;
  if (n < 2 || n > 15 || ctx->Nb >= 32768 || ctx->Na < 1) return false;
  const long long NbP = (ctx->Nb + OZ_KC - 1) / OZ_KC * OZ_KC;
  const size_t lim = 232448;
  return oz_smem_n(oz_pad16(n * (n + 1) / 2), NbP) <= lim && oz_smem_n(oz_pad16(std::max(1, n * (n - 1) / 2)), NbP) <= lim;
}

template <int N>
static int oz_launch(forte_ctx *ctx, int gram, int nrows, int ncta, const int *sh, const long long *Cfix,
                     const uint16_t *T, long long NbP, double *part) {
  const size_t smem = oz_smem<N>(NbP);
  FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_gram_oz<N>));
  FORTE_PROF(ctx, gram ? "gram_oz_v" : "gram_oz_u");
  k_gram_oz<N><<<ncta, OZ_THREADS, smem, ctx->stream>>>(gram, ctx->n, nrows, sh, Cfix, ctx->sd[0].dense, T, ctx->Na,
                                                       NbP, part, ctx->d_err);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

static int oz_dispatch(forte_ctx *ctx, int N, int gram, int nrows, int ncta, const int *sh, const long long *Cfix,
                       const uint16_t *T, long long NbP, double *part) {
  switch (N) {
    case 16: return oz_launch<16>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
    case 32: return oz_launch<32>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
    case 48: return oz_launch<48>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
    case 64: return oz_launch<64>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
    case 80: return oz_launch<80>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
    case 96: return oz_launch<96>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
    case 112: return oz_launch<112>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
    default: return oz_launch<128>(ctx, gram, nrows, ncta, sh, Cfix, T, NbP, part);
  }
}

int rdm2_oz(forte_ctx *ctx, const double *C, const double *g1, double *g2) {
  cudaStream_t st = ctx->stream;
  const int n = ctx->n, n2 = n * n;
  const int nU = n * (n + 1) / 2, nV = n * (n - 1) / 2;
  const int NU = oz_pad16(nU), NV = oz_pad16(std::max(1, nV));
  const long long NA = ctx->Na, NB = ctx->Nb, NbP = (NB + OZ_KC - 1) / OZ_KC * OZ_KC;
  int nsm = 0;
  FORTE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  const int ncta = (int)std::min<long long>(nsm, NA);
  if (!ctx->d_err) {
    const int rc_err = err_word_setup(ctx);
    if (rc_err) return rc_err;
  }
  if (!ctx->d_ozT) {
    FORTE_CUDA_TRY(cudaMalloc(&ctx->d_ozT, sizeof(uint16_t) * (size_t)n2 * NbP));
    FORTE_PROF(ctx, "oz_denseT");
    k_oz_denseT<<<(unsigned)std::min<long long>(((long long)n2 * NbP + 255) / 256, 152LL * 32), 256, 0, st>>>(
        ctx->sd[1].dense, n2, NB, NbP, ctx->d_ozT);
    FORTE_LAUNCH_CHECK();
  }
  // workspace: Cfix, max |C|, row maxima, shifts, partial Grams, G+, G-
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_cfix = take(sizeof(long long) * (size_t)NA * NbP);
  const size_t o_amax = take(sizeof(unsigned long long));
  const size_t o_rmax = take(sizeof(unsigned long long) * 256);
  const size_t o_sh = take(sizeof(int) * 256);
  const size_t o_pu = take(sizeof(double) * (size_t)ncta * NU * NU);
  const size_t o_pv = take(sizeof(double) * (size_t)ncta * NV * NV);
  const size_t o_gu = take(sizeof(double) * (size_t)nU * nU);
  const size_t o_gv = take(sizeof(double) * (size_t)std::max(1, nV * nV));
  int rc = ctx->sc_rdm.ensure(off + 256);
  if (rc) return rc;
  char *w = (char *)ctx->sc_rdm.ptr;
  long long *Cfix = (long long *)(w + o_cfix);
  unsigned long long *amax = (unsigned long long *)(w + o_amax), *rmax = (unsigned long long *)(w + o_rmax);
  int *sh = (int *)(w + o_sh);
  double *PU = (double *)(w + o_pu), *PV = (double *)(w + o_pv), *GU = (double *)(w + o_gu),
         *GV = (double *)(w + o_gv);

  FORTE_CUDA_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned long long), st));
  FORTE_CUDA_TRY(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long) * 256, st));
  {
    FORTE_PROF(ctx, "oz_absmax");
    k_oz_absmax<<<(unsigned)std::min<long long>((NA * NB + 255) / 256, 152LL * 8), 256, 0, st>>>(C, NA * NB, amax);
    FORTE_LAUNCH_CHECK();
  }
  {
    FORTE_PROF(ctx, "oz_cfix");
    k_oz_cfix<<<(unsigned)std::min<long long>((NA * NbP + 255) / 256, 152LL * 32), 256, 0, st>>>(C, NA, NB, NbP,
                                                                                                 amax, Cfix);
    FORTE_LAUNCH_CHECK();
  }
  {
    const size_t sm = sizeof(long long) * (size_t)NbP;
    if (sm > 48 * 1024) FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_oz_rowmax));
    FORTE_PROF(ctx, "oz_rowmax");
    k_oz_rowmax<<<(unsigned)std::min<long long>(NA, (long long)nsm * 8), 256, sm, st>>>(Cfix, ctx->sd[0].dense,
                                                                                      ctx->d_ozT, n, NA, NB, NbP, rmax);
    FORTE_LAUNCH_CHECK();
  }
  {
    FORTE_PROF(ctx, "oz_shift");
    k_oz_shift<<<1, 256, 0, st>>>(rmax, sh);
    FORTE_LAUNCH_CHECK();
  }
  if ((rc = oz_dispatch(ctx, NU, 0, nU, ncta, sh, Cfix, ctx->d_ozT, NbP, PU))) return rc;
  if (nV > 0 && (rc = oz_dispatch(ctx, NV, 1, nV, ncta, sh, Cfix, ctx->d_ozT, NbP, PV))) return rc;
  {
    FORTE_PROF(ctx, "oz_reduce");
    k_oz_reduce<<<(nU * nU + 127) / 128, 128, 0, st>>>(PU, ncta, NU, nU, sh, amax, GU);
    FORTE_LAUNCH_CHECK();
    if (nV > 0) {
      k_oz_reduce<<<(nV * nV + 127) / 128, 128, 0, st>>>(PV, ncta, NV, nV, sh + 128, amax, GV);
      FORTE_LAUNCH_CHECK();
    }
  }
  {
    FORTE_PROF(ctx, "oz_assemble");
    k_oz_assemble<<<(n2 * n2 + 255) / 256, 256, 0, st>>>(GU, GV, g1, n, g2);
    FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

}  // namespace forte
