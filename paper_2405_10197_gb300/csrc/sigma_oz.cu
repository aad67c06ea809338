// FP64-class alpha-beta sigma on the BF16 tensor cores (precision mode
// FORTE_OZ64; the alpha-beta part of steps a5/a6, Sec. II.A.1, Eq. 1 applied in
// the determinant basis):
//
//   sigma[Ia][E_rs Jb] += s F[rs][Jb],   F[rs][Jb] = sum_k A[rs][k] B[Jb][k],
//   A[rs][k] = s_k (pq_k|rs)   (k over L(Ia), the single replacements of Ia)
//   B[Jb][k] = C[J_k][Jb]
//
// the contraction of the reduced-precision alpha-beta kernel, here with exact
// integer digit products (oz_digits.cuh).  Row rs of the integrals is held in
// fixed point relative to its own maximum, the columns Jb of a 64-string tile of C
// relative to the maximum of |C| over that tile, both with |X| <= 2^45, six BF16
// digits each; the levels t = 2..8 (26 digit-pair MMAs per 16-deep K step) are
// exact.  Each F element is an exact 64-bit integer up to the dropped levels (at
// most 2^-49.99 of K times the product of the two scales); it is rounded once onto
// the 64-bit fixed-point grid of the output row (2^-62 of the bound
// n_kl(alpha) n_kl(beta) max|g| max|C|) and added with integer shared-memory
// reductions, so the sum does not depend on the order of the atomics.  The
// quantisation of the operands to 45 bits (2^-46 of the row / tile maximum) is the
// leading error.
//
// Kernel structure (one CTA per SM, persistent over the items (vector, Ia);
// 24 warps, warp-specialised).  Each 64-column MMA reads its B operand (2 KB) from
// shared memory and its A operand from tensor memory, so that the shared-memory
// port is not taken by re-reading A for each of the 104 MMAs of a tile:
//   * warps 0-3 (producers): per item, once the MMAs of the previous item are
//     done, write the A digits (signed integral rows, six slices of 32 columns)
//     into their 32-lane quarter of tensor memory; per tile of 64 beta strings,
//     gather the n_kl digit rows of C (one byte per digit), convert the digits to
//     BF16 and write the six K-major, 128-byte-swizzled slices of a 3-deep ring;
//   * one thread of warp 4 (MMA issuer, TMEM owner): per tile and level the MMA
//     chain (M = 128 pair rows, N = 64 strings) into one of five 64-column TMEM
//     accumulators;
//   * warps 8-23 (epilogue): lane = pair rs, 16 beta strings per warp; fold the
//     seven levels of a tile into 64-bit integers and add them to the output row
//     with three 32-bit shared-memory reductions each;
//   * warps 5-7: write the finished row of the previous item out and clear it.
// Every mbarrier wait is bounded; on expiry the context's status word is raised,
// the other roles stop, the MMA thread drains its own MMAs (bounded), TMEM is
// released and the CTA exits.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "forte_internal.h"
#include "oz_digits.cuh"
#include "tc_ptx.cuh"

namespace forte {

constexpr int ZB_THREADS = 768;                              // 24 warps: 80 registers
constexpr int ZB_TN = 64;                                    // beta strings per tile (MMA N)
constexpr int ZB_SLICE_B = ZB_TN * 128;                      // one digit slice of a stage: 8 KB
constexpr int ZB_STAGE = OZ_DIGITS * ZB_SLICE_B;             // 48 KB
constexpr int ZB_NSTAGE = 3;
constexpr int ZB_OFF_ROW = ZB_NSTAGE * ZB_STAGE;
constexpr int ZB_SLOTS = 5;                                  // TMEM accumulators of 64 columns
constexpr int ZB_ACOL = ZB_SLOTS * ZB_TN;                    // then A: 6 digit slices x 32 columns
constexpr int ZB_MAXNB = 16383;                              // scatter targets are 14-bit
static_assert(ZB_ACOL + OZ_DIGITS * 32 <= 512, "tensor memory budget");

static size_t zb_smem_bytes(long long NB) {
  return 1024 + (size_t)ZB_OFF_ROW + 3 * sizeof(uint32_t) * (size_t)NB + 16 + 8 * (2 * ZB_NSTAGE + 2 * ZB_SLOTS + 5) +
         32;
}

// ------------------------------------------------------------ C digits

// tmax[v][t] = bits of max |C[v][:, 64t .. 64t+63]|, cmax[v] = bits of max |C[v]|
// (non-negative doubles order as their bit patterns).  grid = (column blocks,
// row blocks, vector); thread = column, a warp = half a tile.
__global__ void k_zb_tilemax(const double *__restrict__ C, long long NA, long long NB, long long NBp, int rows_per,
                             unsigned long long *__restrict__ tmax, unsigned long long *__restrict__ cmax) {
  const long long v = blockIdx.z;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long r0 = (long long)blockIdx.y * rows_per, r1 = min(NA, r0 + rows_per);
  unsigned long long m = 0;
  if (j < NB)
    for (long long r = r0; r < r1; ++r)
      m = max(m, (unsigned long long)__double_as_longlong(fabs(C[(v * NA + r) * NB + j])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) {
    atomicMax(tmax + v * (NBp / ZB_TN) + j / ZB_TN, m);
    atomicMax(cmax + v, m);
  }
}

// Tile exponent cb[v][t]: |rint(C 2^cb)| <= 2^45 over tile t (0 for an all-zero
// tile), and the output-grid exponent eS[v] = e(bound) - 62 with
// bound = n_kl(alpha) n_kl(beta) max|g| max|C| < 2^e(bound).
__global__ void k_zb_scales(const unsigned long long *__restrict__ tmax, const unsigned long long *__restrict__ cmax,
                            long long ntile, double gbound, int *__restrict__ cb, int *__restrict__ eS) {
  const long long v = blockIdx.y;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ntile; t += (long long)gridDim.x * blockDim.x) {
    const double m = __longlong_as_double((long long)tmax[v * ntile + t]);
    int e = 0;
    if (m > 0.0) frexp(m, &e);  // m < 2^e
    cb[v * ntile + t] = m > 0.0 ? OZ_XBITS - e : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double b = gbound * __longlong_as_double((long long)cmax[v]);
    int e = 0;
    if (b > 0.0) frexp(b, &e);
    eS[v] = b > 0.0 ? e - 62 : 0;
  }
}

// Cd[v][d][Ja][j] = digit d_(d+1) of rint(C[v][Ja][j] 2^cb[v][j / 64]) + 128 (bytes;
// 0x80 = digit 0 for the padding columns j >= NB).  Thread = 4 consecutive columns.
__global__ void k_zb_cdig(const double *__restrict__ C, long long NA, long long NB, long long NBp,
                          const int *__restrict__ cb, uint8_t *__restrict__ Cd) {
  const long long v = blockIdx.y;
  const long long nq = NA * (NBp / 4);
  const size_t plane = (size_t)NA * NBp;
  uint8_t *Cv = Cd + (size_t)v * OZ_DIGITS * plane;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (long long)gridDim.x * blockDim.x) {
    const long long Ja = i / (NBp / 4), j0 = (i % (NBp / 4)) * 4;
    uint32_t w[OZ_DIGITS] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const long long j = j0 + c;
      long long X = 0;
      if (j < NB) X = llrint(ldexp(C[(v * NA + Ja) * NB + j], cb[v * (NBp / ZB_TN) + j / ZB_TN]));
      const long long Y = X + 0x8080808080LL;
      w[0] |= (uint32_t)((Y >> 40) + 128) << (8 * c);
#pragma unroll
      for (int d = 1; d < OZ_DIGITS; ++d) w[d] |= (uint32_t)((Y >> (8 * (5 - d))) & 0xFF) << (8 * c);
    }
#pragma unroll
    for (int d = 0; d < OZ_DIGITS; ++d) *(uint32_t *)(Cv + d * plane + Ja * NBp + j0) = w[d];
  }
}

// tabT[rs][j] = tabJ[j][rs] (scatter target of pair rs on beta string j),
// 0xFFFF for the padding strings j >= NB.
__global__ void k_zb_tabT(const uint16_t *__restrict__ tabJ, long long NB, long long NBp, uint16_t *__restrict__ tabT) {
  const long long tot = 128 * NBp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long rs = i / NBp, j = i % NBp;
    tabT[i] = j < NB ? tabJ[j * 128 + rs] : (uint16_t)0xFFFFu;
  }
}

// ------------------------------------------------------------ the kernel

// Ring position of the accumulator slots: slot = q mod ZB_SLOTS, round = q / ZB_SLOTS.
struct ZbRing {
  int slot = 0;
  uint32_t round = 0;
  __device__ __forceinline__ void next() {
    if (++slot == ZB_SLOTS) {
      slot = 0;
      ++round;
    }
  }
};

// Fold level LV of the 16 accumulator columns of this warp (one TMEM slot).
template <int LV>
__device__ __forceinline__ bool zb_level(uint32_t taddr_base, int lane, ZbRing &q, uint64_t *tfull, uint64_t *tempty,
                                         volatile int *sAbort, unsigned long long (&acc)[16]) {
  if (!__all_sync(0xffffffffu, mbar_wait_ab(&tfull[q.slot], q.round & 1u, sAbort))) return false;
  tc_fence_after();
  // two 8-column halves: the register peak stays at acc + 8
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t r[8];
    tmem_ld8(taddr_base + (uint32_t)(q.slot * ZB_TN + 8 * h), r);
    tmem_wait_ld();
    if (h == 1) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[q.slot]);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) oz_acc_level<LV>(acc[8 * h + c], r[c]);
  }
  q.next();
  return true;
}

// The MMA chain of level LV with A (the integral digits) in tensor memory: digit
// slice i occupies 32 columns from a_t + 32 (i - 1), a K step is 8 columns.
template <int LV>
__device__ __forceinline__ void zb_issue_level(uint32_t d, uint32_t a_t, uint64_t b0, uint32_t idesc) {
  constexpr int lo = LV - OZ_DIGITS > 1 ? LV - OZ_DIGITS : 1;
  constexpr int hi = LV - 1 < OZ_DIGITS ? LV - 1 : OZ_DIGITS;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int ia = lo; ia <= hi; ++ia)
      mma_issue_ta(d, a_t + (uint32_t)(32 * (ia - 1) + 8 * ks),
                   b0 + (uint64_t)((LV - ia - 1) * (ZB_SLICE_B / 16) + 2 * ks), idesc,
                   (ks == 0 && ia == lo) ? 0u : 1u);
}

__global__ void __launch_bounds__(ZB_THREADS, 1)
    k_ab_oz(const Repl *__restrict__ listA, int nkA, const uint16_t *__restrict__ tabT, long long NA, long long NB,
            long long NBp, const uint16_t *__restrict__ Gd, int npair, const int *__restrict__ ga,
            const uint8_t *__restrict__ Cd, const int *__restrict__ cb, const int *__restrict__ eS,
            double *__restrict__ S, long long nitems, int *__restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  // the swizzle pattern is a function of the shared-space address: align there
  uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *sB = sm;
  // fixed-point output row as three 32-bit words per string (bits 0-20, 21-41, 42-63)
  uint32_t *row0 = (uint32_t *)(sm + ZB_OFF_ROW), *row1 = row0 + NB, *row2 = row1 + NB;
  uint64_t *bar = (uint64_t *)(((uintptr_t)(row2 + NB) + 15) & ~(uintptr_t)15);
  uint64_t *full = bar, *empty = bar + ZB_NSTAGE, *tfull = bar + 2 * ZB_NSTAGE, *tempty = tfull + ZB_SLOTS;
  uint64_t *aFull = tempty + ZB_SLOTS, *aEmpty = aFull + 1, *accReady = aEmpty + 1, *accDone = accReady + 1;
  uint64_t *drain = accDone + 1;
  uint32_t *sTmem = (uint32_t *)(drain + 1);
  volatile int *sAbort = (volatile int *)(sTmem + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long nloc = nitems > blockIdx.x ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int ntiles = (int)(NBp / ZB_TN);
  const size_t plane = (size_t)NA * NBp;

  if (warp == 4) tmem_alloc(sTmem, 512);
  if (tid == 0) {
    for (int i = 0; i < ZB_NSTAGE; ++i) {
      mbar_init(&full[i], 4);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < ZB_SLOTS; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 16);
    }
    mbar_init(aFull, 4);
    mbar_init(aEmpty, 1);
    mbar_init(accReady, 3);
    mbar_init(accDone, 16);
    mbar_init(drain, 1);
    abort_word_init(sAbort, err);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t a_t = tmem + ZB_ACOL;  // A (integral digits) columns
  auto fail = [&]() {
    *sAbort = 1;
    atomicOr(err, 4);
  };

  if (warp >= 5 && warp < 8) {
    // ================= write-out (96 threads): S[v][Ia][:] += row 2^eS, then clear
    const int st = tid - 160;
    for (long long i = 0; i <= nloc; ++i) {
      if (i >= 1) {
        if (!__all_sync(0xffffffffu, mbar_wait_ab(accDone, (uint32_t)((i - 1) & 1), sAbort))) {
          fail();
          break;
        }
        const long long w = blockIdx.x + (i - 1) * gridDim.x, v = w / NA, Ia = w % NA;
        const int e = eS[v];
        double *out = S + (v * NA + Ia) * NB;
        for (long long x = st; x < NB; x += 96) {
          const long long tot = ((long long)(int)row2[x] << 42) + ((long long)row1[x] << 21) + (long long)row0[x];
          out[x] += ldexp((double)tot, e);
          row0[x] = 0u;
          row1[x] = 0u;
          row2[x] = 0u;
        }
      } else {
        for (long long x = st; x < NB; x += 96) row0[x] = row1[x] = row2[x] = 0u;
      }
      if (i < nloc) {
        __syncwarp();
        if (lane == 0) mbar_arrive(accReady);
      }
    }
  } else if (warp < 4) {
    // ================= producers: per item, the A digits of their TMEM lane quarter;
    // per tile, B[j][k] digits: warp p owns strings 16p..16p+15, lane the
    // replacement pair k = 2 lane, 2 lane + 1
    bool ok = true;
    for (long long i = 0; i < nloc && ok; ++i) {
      const long long w = blockIdx.x + i * gridDim.x, v = w / NA, Ia = w % NA;
      const Repl *la = listA + Ia * nkA;
      // A[rs][k] = s_k G[pair_k][rs] into lanes rs = 32 warp + lane, once the MMAs of
      // the previous item no longer read A
      if (i >= 1 && !__all_sync(0xffffffffu, mbar_wait_ab(aEmpty, (uint32_t)((i - 1) & 1), sAbort))) {
        fail();
        break;
      }
      tc_fence_after();
      {
        const int rs = 32 * warp + lane;
        const bool rv = rs < npair;
#pragma unroll 1
        for (int d = 0; d < OZ_DIGITS; ++d) {
          uint32_t wv[32];
          const uint16_t *gd = Gd + (size_t)d * npair * 128 + (rv ? rs : 0);
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int k0 = 2 * c, k1 = k0 + 1;
            uint32_t x = 0;
            if (rv && k0 < nkA) {
              const Repl r = la[k0];
              x = (uint32_t)(gd[(size_t)r.pair * 128] ^ (r.sgn < 0 ? 0x8000u : 0u));
            }
            if (rv && k1 < nkA) {
              const Repl r = la[k1];
              x |= (uint32_t)(gd[(size_t)r.pair * 128] ^ (r.sgn < 0 ? 0x8000u : 0u)) << 16;
            }
            wv[c] = x;
          }
          tmem_st32(a_t + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * d), wv);
        }
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(aFull);

      const uint8_t *Cv = Cd + (size_t)v * OZ_DIGITS * plane;
      const int k0 = 2 * lane, k1 = k0 + 1;
      const bool v0 = k0 < nkA, v1 = k1 < nkA;
      const uint8_t *r0 = Cv + (size_t)(v0 ? la[k0].J : 0) * NBp, *r1 = Cv + (size_t)(v1 ? la[k1].J : 0) * NBp;
      // digit planes of a tile in a 2-deep register ring: plane d + 2 (or the
      // first planes of the next tile) is loaded while plane d is converted
      uint4 ga[2], gb[2];
      auto load = [&](int d, int t, int slot) {
        const long long col = (long long)t * ZB_TN + 16 * warp;
        ga[slot] = make_uint4(0x80808080u, 0x80808080u, 0x80808080u, 0x80808080u);
        gb[slot] = ga[slot];
        if (v0) ga[slot] = __ldg((const uint4 *)(r0 + d * plane + col));
        if (v1) gb[slot] = __ldg((const uint4 *)(r1 + d * plane + col));
      };
      load(0, 0, 0);
      load(1, 0, 1);
      for (int t = 0; t < ntiles; ++t) {
        const long long gt = i * ntiles + t;
        const int s = (int)(gt % ZB_NSTAGE);
        const long long u = gt / ZB_NSTAGE;
        if (gt >= ZB_NSTAGE && !__all_sync(0xffffffffu, mbar_wait_ab(&empty[s], (uint32_t)((u - 1) & 1), sAbort))) {
          fail();
          ok = false;
          break;
        }
        uint8_t *stg = sB + s * ZB_STAGE;
#pragma unroll
        for (int d = 0; d < OZ_DIGITS; ++d) {
          const int sl = d & 1;
          const uint32_t a[4] = {ga[sl].x, ga[sl].y, ga[sl].z, ga[sl].w};
          const uint32_t b[4] = {gb[sl].x, gb[sl].y, gb[sl].z, gb[sl].w};
          if (d + 2 < OZ_DIGITS)
            load(d + 2, t, sl);
          else if (t + 1 < ntiles)
            load(d + 2 - OZ_DIGITS, t + 1, sl);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const uint32_t f0 = oz_dig(a[jj >> 2], (uint32_t)(jj & 3)), f1 = oz_dig(b[jj >> 2], (uint32_t)(jj & 3));
            *(uint32_t *)(stg + d * ZB_SLICE_B + swz((uint32_t)(16 * warp + jj), 4u * lane)) =
                __byte_perm(f0, f1, 0x7632u);
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);
      }
    }
  } else if (warp == 4) {
    // ================= MMA issuer: D[rs][j] (+)= sum_k A_i[rs][k] B_j[j][k] over
    // the digit pairs (i, j) of one level
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ZB_TN >> 3) << 17) | ((128u >> 4) << 24);
      bool ok = true;
      ZbRing q;
      long long nq = 0;  // levels issued
      for (long long i = 0; i < nloc && ok; ++i) {
        if (!mbar_wait_ab(aFull, (uint32_t)(i & 1), sAbort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int t = 0; t < ntiles && ok; ++t) {
          const long long gt = i * ntiles + t;
          const int s = (int)(gt % ZB_NSTAGE);
          if (!mbar_wait_ab(&full[s], (uint32_t)((gt / ZB_NSTAGE) & 1), sAbort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t b0 = desc_kmajor_sw128(smem_u32(sB + s * ZB_STAGE));
          // one level: wait for its accumulator slot, issue its chain, commit
          auto level = [&](auto lvc) -> bool {
            constexpr int LV = decltype(lvc)::value;
            if (nq >= ZB_SLOTS && !mbar_wait_ab(&tempty[q.slot], (q.round - 1u) & 1u, sAbort)) return false;
            tc_fence_after();
            zb_issue_level<LV>(tmem + (uint32_t)(q.slot * ZB_TN), a_t, b0, idesc);
            mma_commit(&tfull[q.slot]);
            q.next();
            ++nq;
            return true;
          };
          ok = level(std::integral_constant<int, 2>{}) && level(std::integral_constant<int, 3>{}) &&
               level(std::integral_constant<int, 4>{}) && level(std::integral_constant<int, 5>{}) &&
               level(std::integral_constant<int, 6>{}) && level(std::integral_constant<int, 7>{}) &&
               level(std::integral_constant<int, 8>{});
          if (!ok) break;
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(aEmpty);  // A free once this item's MMAs are done
      }
      if (!ok) fail();
    }
    __syncwarp();
  } else {
    // ================= epilogue: lane = pair rs, 16 strings of each tile per warp
    const int qd = warp & 3, cg = (warp - 8) >> 2;
    const int rs = 32 * qd + lane, col0 = 16 * cg;
    const int gar = rs < npair ? ga[rs] : 0;
    const uint32_t tb = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)col0;
    const int ntl = (int)(NBp / ZB_TN);
    const uint16_t *trow = tabT + (size_t)rs * NBp + col0;  // this lane's scatter targets
    bool ok = true;
    ZbRing q;
    for (long long i = 0; i < nloc && ok; ++i) {
      const long long w = blockIdx.x + i * gridDim.x, v = w / NA;
      const int ev = eS[v];
      const int *cbv = cb + v * ntl;
      if (!__all_sync(0xffffffffu, mbar_wait_ab(accReady, (uint32_t)(i & 1), sAbort))) {
        fail();
        break;
      }
      for (int t = 0; t < ntiles; ++t) {
        // the tile's scatter targets and scale, loaded while the levels are folded
        uint4 tg0 = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu), tg1 = tg0;
        if (rs < npair) {
          tg0 = __ldg((const uint4 *)(trow + (size_t)t * ZB_TN));
          tg1 = __ldg((const uint4 *)(trow + (size_t)t * ZB_TN + 8));
        }
        const int r = gar + cbv[t] + ev - 38;  // value = F 2^-r on the row grid
        unsigned long long acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0ull;
        ok = zb_level<2>(tb, lane, q, tfull, tempty, sAbort, acc) && zb_level<3>(tb, lane, q, tfull, tempty, sAbort, acc) &&
             zb_level<4>(tb, lane, q, tfull, tempty, sAbort, acc) && zb_level<5>(tb, lane, q, tfull, tempty, sAbort, acc) &&
             zb_level<6>(tb, lane, q, tfull, tempty, sAbort, acc) && zb_level<7>(tb, lane, q, tfull, tempty, sAbort, acc) &&
             zb_level<8>(tb, lane, q, tfull, tempty, sAbort, acc);
        if (!ok) {
          fail();
          break;
        }
        const uint32_t tw[8] = {tg0.x, tg0.y, tg0.z, tg0.w, tg1.x, tg1.y, tg1.z, tg1.w};
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const uint32_t en = (c & 1) ? (tw[c >> 1] >> 16) : (tw[c >> 1] & 0xFFFFu);
          if (en == 0xFFFFu) continue;
          const long long F = (long long)(acc[c] - oz_bias());
          long long val;
          if (r <= 0)
            val = F << min(-r, 62);
          else if (r > 62)
            val = 0;
          else
            val = (F + (1LL << (r - 1))) >> r;
          if (en & 0x4000u) val = -val;
          // three 32-bit integer reductions (native in shared memory; 64-bit ones are not):
          // bits 0-20 and 21-41 as unsigned parts, the rest signed; at most 64
          // contributions per string and item keep every word inside 32 bits
          const uint32_t x = en & 0x3FFFu;
          atomicAdd(&row0[x], (uint32_t)(val & 0x1FFFFF));
          atomicAdd(&row1[x], (uint32_t)((val >> 21) & 0x1FFFFF));
          atomicAdd(&row2[x], (uint32_t)(int)(val >> 42));
        }
      }
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(accDone);
    }
  }
  __syncthreads();
  if (*sAbort && warp == 4 && lane == 0) {
    mma_commit(drain);  // tracks every MMA this thread issued
    mbar_wait(drain, 0u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 4) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------ host side

bool oz_ab_supported(const forte_ctx *ctx) {
  const int nkA = ctx->sh[0].nk;
  return ctx->npair <= 128 && nkA <= 64 && ctx->Nb <= ZB_MAXNB && zb_smem_bytes(ctx->Nb) <= 232448;
}

// Digits of the integrals: Gd[d][pq][rs] = digit d_(d+1) of rint((pq|rs) 2^ga[rs])
// (BF16 bits, rs < 128, zero for rs >= npair), ga[rs] = 45 - e(max_pq |(pq|rs)|).
static int oz_ab_setup(forte_ctx *ctx) {
  if (ctx->d_ozG) return FORTE_OK;
  const int np = ctx->npair;
  std::vector<double> g((size_t)np * np);
  FORTE_CUDA_TRY(cudaMemcpy(g.data(), ctx->d_gpair, sizeof(double) * g.size(), cudaMemcpyDeviceToHost));
  std::vector<int> ga(128, 0);
  std::vector<uint16_t> gd((size_t)OZ_DIGITS * np * 128, 0);
  double gmax = 0.0;
  for (int rs = 0; rs < np; ++rs) {
    double m = 0.0;
    for (int pq = 0; pq < np; ++pq) m = std::max(m, std::fabs(g[(size_t)pq * np + rs]));
    gmax = std::max(gmax, m);
    int e = 0;
    if (m > 0.0) std::frexp(m, &e);
    ga[rs] = m > 0.0 ? OZ_XBITS - e : 0;
    for (int pq = 0; pq < np; ++pq) {
      const long long X = std::llrint(std::ldexp(g[(size_t)pq * np + rs], ga[rs]));
      const long long Y = X + 0x8080808080LL;
      for (int d = 0; d < OZ_DIGITS; ++d) {
        const long long dig = d == 0 ? (Y >> 40) : ((Y >> (8 * (5 - d))) & 0xFF) - 128;
        const float f = (float)dig;  // |dig| <= 128: exact in BF16
        uint32_t b;
        std::memcpy(&b, &f, 4);
        gd[((size_t)d * np + pq) * 128 + rs] = (uint16_t)(b >> 16);
      }
    }
  }
  ctx->oz_gmax = gmax;
  const long long NBp = (ctx->Nb + ZB_TN - 1) / ZB_TN * ZB_TN;
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_ozTabT, sizeof(uint16_t) * 128 * NBp));
  k_zb_tabT<<<(unsigned)std::min<long long>((128 * NBp + 255) / 256, 152LL * 16), 256, 0, ctx->stream>>>(
      ctx->sd[1].tabJ, ctx->Nb, NBp, ctx->d_ozTabT);
  FORTE_LAUNCH_CHECK();
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_ozG, sizeof(uint16_t) * gd.size()));
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_ozGa, sizeof(int) * 128));
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_ozG, gd.data(), sizeof(uint16_t) * gd.size(), cudaMemcpyHostToDevice));
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_ozGa, ga.data(), sizeof(int) * 128, cudaMemcpyHostToDevice));
  if (!ctx->d_err) {
    const int rc_err = err_word_setup(ctx);
    if (rc_err) return rc_err;
  }
  return FORTE_OK;
}

// S += sigma_ab(C) (FP64 vectors [nvec][NA][NB]).
static int sigma_ab_oz(forte_ctx *ctx, const double *C, double *S, int nvec) {
  const int nkA = ctx->sh[0].nk, nkB = ctx->sh[ctx->same_strings ? 0 : 1].nk;
  if (nkA <= 0 || nkB <= 0) return FORTE_OK;
  int rc = oz_ab_setup(ctx);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const long long NA = ctx->Na, NB = ctx->Nb;
  const long long NBp = (NB + ZB_TN - 1) / ZB_TN * ZB_TN;
  const size_t ndig = (size_t)nvec * OZ_DIGITS * NA * NBp;
  const long long ntl = NBp / ZB_TN;
  const size_t ncol = (size_t)nvec * ntl;
  const size_t bytes = ndig + 256 + ncol * 8 + 256 + (size_t)nvec * 8 + 256 + ncol * 4 + 256 + (size_t)nvec * 4 + 256;
  if ((rc = ctx->sc_oz.ensure(bytes))) return rc;
  auto align = [](uint8_t *p) { return (uint8_t *)(((uintptr_t)p + 255) & ~(uintptr_t)255); };
  uint8_t *Cd = (uint8_t *)ctx->sc_oz.ptr;
  unsigned long long *tmax = (unsigned long long *)align(Cd + ndig);
  unsigned long long *cmax = (unsigned long long *)align((uint8_t *)(tmax + ncol));
  int *cb = (int *)align((uint8_t *)(cmax + nvec));
  int *eS = (int *)align((uint8_t *)(cb + ncol));
  FORTE_CUDA_TRY(cudaMemsetAsync(tmax, 0, ncol * 8, st));
  FORTE_CUDA_TRY(cudaMemsetAsync(cmax, 0, (size_t)nvec * 8, st));
  {
    const int rows_per = 64;
    dim3 grid((unsigned)((NB + 255) / 256), (unsigned)((NA + rows_per - 1) / rows_per), (unsigned)nvec);
    FORTE_PROF(ctx, "zb_tilemax");
    k_zb_tilemax<<<grid, 256, 0, st>>>(C, NA, NB, NBp, rows_per, tmax, cmax);
    FORTE_LAUNCH_CHECK();
  }
  {
    const double gbound = (double)nkA * (double)nkB * ctx->oz_gmax;
    dim3 grid((unsigned)((ntl + 255) / 256), (unsigned)nvec);
    FORTE_PROF(ctx, "zb_scales");
    k_zb_scales<<<grid, 256, 0, st>>>(tmax, cmax, ntl, gbound, cb, eS);
    FORTE_LAUNCH_CHECK();
  }
  {
    const long long nq = NA * (NBp / 4);
    dim3 grid((unsigned)std::min<long long>((nq + 255) / 256, 152LL * 16), (unsigned)nvec);
    FORTE_PROF(ctx, "zb_cdig");
    k_zb_cdig<<<grid, 256, 0, st>>>(C, NA, NB, NBp, cb, Cd);
    FORTE_LAUNCH_CHECK();
  }
  const size_t smem = zb_smem_bytes(NB);
  int nsm = 0;
  FORTE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  const long long nitems = NA * nvec;
  dim3 grid((unsigned)std::min<long long>(nitems, nsm));
  FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_ab_oz));
  FORTE_PROF(ctx, "ab_oz");
  k_ab_oz<<<grid, ZB_THREADS, smem, st>>>(ctx->sd[0].list, nkA, ctx->d_ozTabT, NA, NB, NBp, ctx->d_ozG, ctx->npair,
                                          ctx->d_ozGa, Cd, cb, eS, S, nitems, ctx->d_err);
  FORTE_LAUNCH_CHECK();
  return FORTE_OK;
}

// FORTE_OZ64 sigma: same-spin terms in double-FP32, alpha-beta term as exact digit
// products on the tensor cores; the double-FP32 alpha-beta kernel where the
// tensor-core one does not apply (more than 15 orbitals, n_kl > 64).
int sigma_oz64(forte_ctx *ctx, const double *C, double *S, int nvec) {
  if (!oz_ab_supported(ctx)) return sigma_df(ctx, C, S, nvec, true);
  int rc = sigma_df(ctx, C, S, nvec, false);
  if (rc) return rc;
  return sigma_ab_oz(ctx, C, S, nvec);
}

}  // namespace forte
