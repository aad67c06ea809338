// Reduced-precision sigma build (steps a5, a6, a8 of the hot path).
//
//   same-spin terms: one dense tensor-core GEMM (sigma_ss_mma.cu); FP32 CSR gathers
//       only when the dense string Hamiltonians would exceed 4 GB;
//   alpha-beta term: per alpha string Ia, on the 5th-generation tensor cores
//       F[rs][Jb] = sum_k  A[rs][k] * B[Jb][k]
//       A[rs][k]  = s_k (pq_k|rs)            k over L(Ia), the replacements of Ia
//       B[Jb][k]  = C[J_k][Jb]               gathered rows of C
//     followed by the signed scatter  sigma[Ia][E_rs Jb] += s F[rs][Jb]  over the
//     replacement list L(Jb).  In the MMA the gathered C tile is M=128 (128 beta
//     strings), the integral block N=112/128 (symmetric pairs rs, zero padded),
//     K=64 (n_kl <= 64, zero padded).
//
// Bank-conflict-free scatter.  The beta strings are placed at "positions": a
// linear 5-bit hash h(J) = XOR of per-orbital codes over the occupied orbitals
// sorts them into 32 classes, and position 32 g + c holds the g-th string of
// class c (positions without a string are padding).  Tiles, the fixed-point
// accumulator row and the scatter table all use positions.  A replacement flips
// two occupations, E_rs J = J xor {r, s}, so h(E_rs J) = h(J) xor h({r, s}): for a
// fixed pair rs the 32 lanes of a warp (32 strings of distinct classes) reach 32
// distinct classes, i.e. 32 distinct shared-memory banks, and every integer
// reduction of the scatter is a single wavefront.
//
// Operands: FORTE_BF16X2 splits x = hi + lo (hi = RNE_bf16(x), lo = RNE_bf16(x - hi))
// and forms hi*hi + hi*lo + lo*hi (kind::f16, FP32 accumulate); FORTE_TF32 rounds to
// TF32 with round-to-nearest-even before the MMA (kind::tf32, FP32 accumulate).
//
// Kernel structure (persistent: one CTA per SM loops over the items (vector, Ia);
// 8 + MX_EPI = 24 warps, warp-specialised):
//   * warps 5-7 (set-up) build A for the next item in the other half of a double
//     buffer (K-major, 128-byte swizzle) and write out the sigma row of the item
//     before last from the other half of a double-buffered accumulator row;
//   * warps 0-3 (producers) gather the n_kl C rows of each 128-column beta tile,
//     transpose them into a K-major swizzled stage of a 3-deep ring and arrive on
//     its `full` mbarrier;
//   * one thread of warp 4 issues the tcgen05.mma chain of the tile into one of
//     four 128-column TMEM accumulators and commits to the stage's `empty` and the
//     accumulator's `tfull` mbarriers;
//   * warps 8-23 (epilogue, four per TMEM lane quarter) read the accumulator with
//     tcgen05.ld, convert each valid element to fixed point and add it to the sigma
//     row in shared memory with integer reductions (positive and negative parts in
//     separate words), then arrive on the accumulator's `tempty` mbarrier.
// The rings run across item boundaries, so one item's set-up and drain overlap
// its neighbours' tiles.
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel raises the
// context's device status word, the other roles stop, the MMA thread drains its
// own MMAs (bounded), TMEM is freed and the CTA exits.
#include <cuda_bf16.h>

#include <algorithm>
#include <string>

#include "bf16_split.h"
#include "forte_internal.h"
#include "tc_ptx.cuh"

namespace forte {

// epilogue warps (a multiple of 4: the same number per TMEM lane quarter)
#ifndef FORTE_AB_EPI_WARPS
#define FORTE_AB_EPI_WARPS 16
#endif
constexpr int MX_EPI = FORTE_AB_EPI_WARPS;
constexpr int MX_THREADS = (8 + MX_EPI) * 32;  // producers, MMA, set-up, epilogue
constexpr int MX_TILE_N = 128;
constexpr int MX_STAGE = 32768;               // one B stage: 32 KB

// ------------------------------------------------------------ conversion kernels

// C (FP64 [v][NA][NB]) -> C32 (FP32, same layout) and the tensor-core copy in a
// row-padded layout [v][NA][NBp] (NBp multiple of 16, zero padding); also the
// per-vector bound cmax_bits[v] = bits of max |C| (non-negative floats order as
// their bit patterns).  grid.y = vector.
template <int MODE, typename TI>
__global__ void k_split(const TI *__restrict__ C, float *__restrict__ C32, uint16_t *__restrict__ hi,
                        uint16_t *__restrict__ lo, float *__restrict__ t32, long long NA, long long NB,
                        long long NBp, unsigned *__restrict__ cmax_bits) {
  __shared__ unsigned red[32];
  const long long v = blockIdx.y;
  const long long per = NA * NBp;
  const TI *Cv = C + v * NA * NB;
  float *C32v = C32 ? C32 + v * NA * NB : nullptr;
  unsigned mx = 0u;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i % NBp, row = i / NBp;
    double x = 0.0;
    if (b < NB) {
      x = (double)Cv[row * NB + b];
      if (C32v) C32v[row * NB + b] = (float)x;
    }
    mx = max(mx, __float_as_uint(fabsf((float)x)));
    if (MODE == FORTE_BF16X2) {
      const double h = rne_drop(x, 45);
      const double l = rne_drop(x - h, 45);
      hi[v * per + i] = bf16_bits(h);
      lo[v * per + i] = bf16_bits(l);
    } else {
      t32[v * per + i] = (float)rne_drop(x, 42);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0u;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    atomicMax(cmax_bits + v, m);
  }
}

// The same split without 64-bit index arithmetic: one thread per padded element of
// one (vector, alpha string) row.  The BF16 hi part is x rounded to nearest even,
// x - hi is exact in the input precision, the TF32 copy keeps 10 mantissa bits
// (nearest even): bit-identical to k_split.  grid = (column blocks, NA, vector).
__device__ __forceinline__ void split_bf16(float x, uint16_t &h, uint16_t &l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(x);
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hb)));
}
__device__ __forceinline__ void split_bf16(double x, uint16_t &h, uint16_t &l) {
  if (bf16_split_bits(x, h, l)) return;  // integer path; conversions for the rest
  const __nv_bfloat16 hb = __double2bfloat16(x);
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(__double2bfloat16(x - (double)__bfloat162float(hb)));
}
// bits of (float)|x| (non-negative floats order as their bit patterns)
__device__ __forceinline__ unsigned abs_bits(float x) { return __float_as_uint(fabsf(x)); }
__device__ __forceinline__ unsigned abs_bits(double x) {
  uint32_t b;
  return f32_abs_bits(x, b) ? b : __float_as_uint(fabsf((float)x));
}
__device__ __forceinline__ float tf32_rne(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0xFFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & ~0x1FFFu);
}
__device__ __forceinline__ float tf32_rne(double x) { return (float)rne_drop(x, 42); }

// Besides the row-padded copy it writes the copy in beta positions (row length
// NBpos, strOf[b] = string at position b, -1 for padding) that the alpha-beta
// kernel gathers; its rounding is the same.
template <int MODE, typename TI>
__global__ void __launch_bounds__(256) k_split_rows(const TI *__restrict__ C, uint16_t *__restrict__ hi,
                                                    uint16_t *__restrict__ lo, float *__restrict__ t32, long long NA,
                                                    long long NB, long long NBp, unsigned *__restrict__ cmax_bits,
                                                    const int *__restrict__ strOf, long long NBpos,
                                                    uint16_t *__restrict__ phi, uint16_t *__restrict__ plo,
                                                    float *__restrict__ pt32) {
  __shared__ unsigned red[8];
  // grid-stride over (row, 256-column block) pairs; one atomic per block at the end
  const long long v = blockIdx.z;
  const long long nbx = (std::max(NBp, strOf ? NBpos : 0LL) + 255) / 256;
  unsigned mx = 0u;
  for (long long w = blockIdx.x; w < NA * nbx; w += gridDim.x) {
    const long long row = w / nbx, b = (w % nbx) * 256 + threadIdx.x;
    if (b < NBp && (hi || t32)) {
      const TI x = b < NB ? C[(v * NA + row) * NB + b] : TI(0);
      mx = max(mx, abs_bits(x));
      const long long o = (v * NA + row) * NBp + b;
      if (MODE == FORTE_BF16X2)
        split_bf16(x, hi[o], lo[o]);
      else
        t32[o] = tf32_rne(x);
    }
    if (strOf && b < NBpos) {
      const int J = strOf[b];
      const TI x = J >= 0 ? C[(v * NA + row) * NB + J] : TI(0);
      const long long o = (v * NA + row) * NBpos + b;
      if (MODE == FORTE_BF16X2)
        split_bf16(x, phi[o], plo[o]);
      else
        pt32[o] = tf32_rne(x);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0u;
    for (int w = 0; w < 8; ++w) m = max(m, red[w]);
    if (m) atomicMax(cmax_bits + v, m);
  }
}

// gT[rs][pq] = (pq|rs) for rs < 128 (zero rows beyond npair), split/rounded.
__global__ void k_split_g(const double *__restrict__ gpair, int npair, uint16_t *__restrict__ hi,
                          uint16_t *__restrict__ lo, float *__restrict__ t32) {
  const int total = 128 * npair;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int rs = i / npair, pq = i % npair;
    const double x = (rs < npair) ? gpair[(size_t)pq * npair + rs] : 0.0;
    const double h = rne_drop(x, 45);
    hi[i] = bf16_bits(h);
    lo[i] = bf16_bits(rne_drop(x - h, 45));
    t32[i] = (float)rne_drop(x, 42);
  }
}

// gTT[pair][rs] = gT[rs][pair] (pair-major copy: the rs values of one pair are contiguous)
__global__ void k_pair_major(const uint16_t *__restrict__ hi, const uint16_t *__restrict__ lo, int npair,
                             uint16_t *__restrict__ thi, uint16_t *__restrict__ tlo) {
  const int total = 128 * npair;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int pr = i / 128, rs = i % 128;
    thi[i] = hi[rs * npair + pr];
    tlo[i] = lo[rs * npair + pr];
  }
}

__global__ void k_f32_to_f64(const float *__restrict__ a, double *__restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// ------------------------------------------------------------ the alpha-beta MMA kernel
//
// Scatter accumulation.  Every contribution f is turned into the fixed-point
// value V = rint(f 2^S) with |V| <= 2^22 (S per vector from the bound
// |f| <= n_kl * max|g| * max|C|, with 2% slack for the operand splits) and added
// with one 32-bit integer reduction into shared memory.  At most n_kl <= 64
// contributions reach one output, so the word cannot overflow, and the rounding
// adds at most 64 * 2^-23 = 7.6e-6 of the bound to an output: below the 2^-16
// relative error the BF16 hi/lo operands already carry.  Integer shared-memory
// reductions are native on the SM, FP32 ones are not; the sum is exact and
// independent of the order of the atomics.

// C-tile stages of the producer ring, per mode.  Each stage is 32 KB of shared
// memory, and what the kernel leaves of the SM's 256 KB is the L1 cache that holds
// the scatter table of the current and the next tile (28 KB each).  Measured at
// CAS(14,14): BF16x2 0.82 ms with 3 stages, 1.09 ms with 2; TF32 (whose producers
// transpose through registers) 1.72 ms with 3, 1.50 ms with 2.
#ifndef FORTE_AB_STAGES_BF16
#define FORTE_AB_STAGES_BF16 3
#endif
#ifndef FORTE_AB_STAGES_TF32
#define FORTE_AB_STAGES_TF32 2
#endif
__host__ __device__ constexpr int ws_stages(int mode) {
  return mode == FORTE_BF16X2 ? FORTE_AB_STAGES_BF16 : FORTE_AB_STAGES_TF32;
}
constexpr int WS_ACC = 4;                                 // TMEM accumulators of 128 columns
constexpr int MX_A_BYTES = 32768;                         // A operand: 2 x 16 KB
constexpr int WS_OFF_B = 2 * MX_A_BYTES;                  // A double-buffered across items
__host__ __device__ constexpr int ws_off_acc(int mode) { return WS_OFF_B + ws_stages(mode) * MX_STAGE; }
// warp roles: 0-3 producers, 4 MMA issuer (and TMEM owner), 5-7 item set-up and
// write-out, 8-15 epilogue

// One CTA per SM, persistent over the items w = (vector, Ia).  For item i the
// set-up warps write out item i-2's sigma row from acc[i&1] and clear it
// (`accReady`), then, once the MMAs of item i-2 are done with A[i&1] (`aEmpty`),
// build A[i&1] and the gather rows of item i (`aFull`).  The producers, the MMA
// thread and the epilogue run their tile rings across item boundaries, so the
// set-up and the drain of one item overlap the tiles of its neighbours.
// Shared-memory integer reduction at byte address addr.
__device__ __forceinline__ void red_add(uint32_t addr, int v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// Shared-memory integer reduction at byte address addr unless bit 1 of en is set (the
// "no target" marker 0xFFFF of the scatter table), without a branch.
__device__ __forceinline__ void red_add_if(uint32_t addr, int v, uint32_t en) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b32 t;\n and.b32 t, %2, 2;\n setp.eq.u32 p, t, 0;\n"
      " @p red.shared.add.u32 [%0], %1;\n}\n" ::"r"(addr), "r"(v), "r"(en)
      : "memory");
}

// Beta strings enter in positions (see the top of the file).  tabL holds the
// scatter targets lane-contiguously: entry e of chunk c (8 pairs) of the string at
// position pos = 128 t + 32 g + lane sits at tabL[(((t * 4 + g) * 16 + c) * 32 + lane) * 8 + e]
// as 4 x (target position) | (sign < 0), 0xFFFF when E_rs does not act; posOf[Jb] is
// the position of string Jb.
//
// FORTE_BF16X2: the gathered C tile is staged MN-major (positions contiguous):
//   stage = [part hi/lo: 16 KB][position half: 8 KB][K row k: 128 B of 64 positions],
// 128-byte swizzled, so each gathered C row is copied as it is (coalesced loads,
// conflict-free stores) and the tile is the MMA's A operand in MN-major form.  The
// integral block is built from the pair-major copy gTT[pair][rs] with coalesced
// loads.  FORTE_TF32 gathers and transposes the FP32 copy Ct32 into a K-major stage.
// Chi / Clo / Ct32: the C copies in positions, rows of NBpos.
// Warp roles: 0-3 producers, 4 MMA issuer (and TMEM owner), 5-7 item set-up and
// write-out, 8 .. 8 + MX_EPI - 1 epilogue (MX_EPI / 4 warps per TMEM lane quarter).
template <int MODE, typename TO, bool SPLIT>
__global__ void __launch_bounds__(MX_THREADS, 1)
    k_ab_mma(const Repl *__restrict__ listA, int nkA, int nkB,
             const uint16_t *__restrict__ tabL, const uint16_t *__restrict__ posOf, const int8_t *__restrict__ dcnt,
             int nN, long long NA,
             long long NB, long long NBpos, const uint16_t *__restrict__ gTT_hi, const uint16_t *__restrict__ gTT_lo,
             const float *__restrict__ gT_t32, int npair, float gmax, const unsigned *__restrict__ cmax_bits,
             const uint16_t *__restrict__ Chi, const uint16_t *__restrict__ Clo, const float *__restrict__ Ct32,
             const float *__restrict__ Sss, TO *__restrict__ S, long long nitems, int *__restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int WS_STAGES = ws_stages(MODE);
  constexpr int WS_OFF_ACC = ws_off_acc(MODE);
  // the swizzle pattern is a function of the shared-space address: align there
  uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *sB = sm + WS_OFF_B;
  const long long NB4 = NBpos;                   // a multiple of 32
  // accumulator row per buffer: [NBpos] by position, or with SPLIT [NBpos] for the
  // positive contributions, [NBpos] for the negative ones and 32 spare words
  const long long ACCW = SPLIT ? 2 * NB4 + 32 : NB4;
  int *accb = (int *)(sm + WS_OFF_ACC);          // acc[2][ACCW]
  int *sJb = accb + 2 * ACCW;                    // gathered strings J_k [2][64]
  uint64_t *bar = (uint64_t *)(((uintptr_t)(sJb + 128) + 15) & ~(uintptr_t)15);
  uint64_t *full = bar, *empty = bar + WS_STAGES, *tfull = bar + 2 * WS_STAGES, *tempty = tfull + WS_ACC;
  uint64_t *aFull = tempty + WS_ACC, *aEmpty = aFull + 2, *accReady = aEmpty + 2, *accDone = accReady + 2;
  uint64_t *drain = accDone + 2;
  uint32_t *sTmem = (uint32_t *)(drain + 1);
  volatile int *sAbort = (volatile int *)(sTmem + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long nloc = nitems > blockIdx.x ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long vpad = NA * NBpos, v64 = NA * NB;
  const int ntiles = (int)((NBpos + MX_TILE_N - 1) / MX_TILE_N);
  // fixed-point exponent of vector v (bound |f| <= 1.02 n_kl max|g| max|C|)
  auto sx_of = [&](long long v) -> int {
    const float bound = 1.02f * (float)nkA * gmax * __uint_as_float(cmax_bits[v]);
    int eb = 0;
    if (bound > 0.f) frexpf(bound, &eb);
    return (bound > 0.f) ? min(100, 22 - eb) : 0;
  };

  // K rows k >= n_kl are never written and must read as zero
  for (int i = tid; i < WS_STAGES * MX_STAGE / 16; i += MX_THREADS) ((uint4 *)sB)[i] = make_uint4(0, 0, 0, 0);
  fence_proxy_async();
  if (warp == 4) tmem_alloc(sTmem, WS_ACC * MX_TILE_N);
  if (tid == 0) {
    for (int i = 0; i < WS_STAGES; ++i) {
      mbar_init(&full[i], 4);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < WS_ACC; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], MX_EPI);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&aFull[i], 3);
      mbar_init(&aEmpty[i], 1);
      mbar_init(&accReady[i], 3);
      mbar_init(&accDone[i], MX_EPI);
    }
    mbar_init(drain, 1);
    abort_word_init(sAbort, err);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  auto fail = [&]() {
    *sAbort = 1;
    atomicOr(err, 1);
  };

  if (warp >= 5 && warp < 8) {
    // ================= set-up / write-out (96 threads)
    const int st = tid - 160;
    for (long long i = 0; i < nloc + 2; ++i) {
      const int buf = (int)(i & 1);
      int *acc = accb + buf * ACCW;
      if (i >= 2) {
        // write out item i-2 and clear its accumulator row
        if (!__all_sync(0xffffffffu, mbar_wait_ab(&accDone[buf], (uint32_t)(((i - 2) >> 1) & 1), sAbort))) {
          fail();
          break;
        }
        const long long w = blockIdx.x + (i - 2) * gridDim.x, v = w / NA, Ia = w % NA;
        const int Sx = sx_of(v);
        const float *ss = Sss + v * v64 + Ia * NB;
        TO *out = S + v * v64 + Ia * NB;
        // every output received n_kl(beta) contributions carrying bits(1.5 2^23) each
        // (SPLIT: npos(x) of them in the positive word, nneg(x) in the negative one,
        // dcnt[x] = npos(x) - nneg(x))
        const uint32_t bias = (uint32_t)nkB * 0x4B400000u;
        // padding positions never receive a contribution and stay zero
        for (long long x = st; x < NB; x += 96) {
          const int ps = __ldg(posOf + x);
          uint32_t vfix;
          if (SPLIT) {
            vfix = (uint32_t)acc[ps] - (uint32_t)acc[NB4 + ps] - (uint32_t)(int)__ldg(dcnt + x) * 0x4B400000u;
            acc[NB4 + ps] = 0;
          } else {
            vfix = (uint32_t)acc[ps] - bias;
          }
          out[x] = (TO)((double)ss[x] + ldexp((double)(int)vfix, -Sx));
          acc[ps] = 0;
        }
      } else {
        for (long long x = st; x < (SPLIT ? 2 * NB4 : NB4); x += 96) acc[x] = 0;
      }
      if (i >= nloc) continue;
      __syncwarp();
      if (lane == 0) mbar_arrive(&accReady[buf]);
      // integral operand and gather rows of item i, once the MMAs of item i-2 are done
      if (i >= 2 && !__all_sync(0xffffffffu, mbar_wait_ab(&aEmpty[buf], (uint32_t)(((i - 2) >> 1) & 1), sAbort))) {
        fail();
        break;
      }
      const long long Ia = (blockIdx.x + i * gridDim.x) % NA;
      const Repl *la = listA + Ia * nkA;
      uint8_t *sA = sm + buf * MX_A_BYTES;
      if (warp == 5) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = lane + 32 * h;
          sJb[buf * 64 + k] = k < nkA ? la[k].J : 0;
        }
      }
      // A[rs][k] = s_k (pq_k|rs), K-major swizzled
      if (MODE == FORTE_BF16X2) {
        // lanes over rs (coalesced rows of the pair-major copy), warps over k
        for (int k = warp - 5; k < 64; k += 3) {
          int pr = 0;
          bool neg = false;
          if (k < nkA) {
            const Repl r = la[k];
            pr = r.pair;
            neg = r.sgn < 0;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int rs = lane + 32 * q;
            uint16_t h = 0, l = 0;
            if (k < nkA && rs < npair) {
              h = gTT_hi[pr * 128 + rs];
              l = gTT_lo[pr * 128 + rs];
              if (neg) { h ^= 0x8000u; l ^= 0x8000u; }
            }
            *(uint16_t *)(sA + swz(rs, 2 * k)) = h;
            *(uint16_t *)(sA + 16384 + swz(rs, 2 * k)) = l;
          }
        }
      } else {
        for (int idx = st; idx < 128 * 64; idx += 96) {
          const int k = idx & 63, rs = idx >> 6;
          float val = 0.f;
          if (rs < npair && k < nkA) {
            const Repl r = la[k];
            val = gT_t32[rs * npair + r.pair];
            if (r.sgn < 0) val = -val;
          }
          *(float *)(sA + (k >> 5) * 16384 + swz(rs, (k & 31) * 4)) = val;
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aFull[buf]);
    }
  } else if (warp < 4) {
    if (MODE == FORTE_BF16X2) {
      // ================= producers: C rows J_k of each tile, copied as they are into the
      // MN-major stage (K row k = 128 bytes of 64 positions per half) with asynchronous
      // 16-byte copies: warp w copies rows k = w, w + 4, ...; lanes 0-15 one row and
      // lanes 16-31 the next, lane c moving positions 8c..8c+7 (chunk c & 7 of half c >> 3),
      // so the reads are whole row segments and every 128-byte stage row is written in
      // one go.  Two tiles are in flight per warp: the stage of a tile is announced
      // (copies complete, proxy fence, arrive) after the next tile's copies are issued.
      bool ok = true;
      const int cpos = 8 * (lane & 15);
      const uint32_t hoff = (uint32_t)(cpos >> 6) * 8192u, cbyte = (uint32_t)(cpos & 63) * 2u;
      int pending = -1;  // stage whose copies are issued but not yet announced
      auto announce = [&](int n_in_flight) {
        if (n_in_flight)
          asm volatile("cp.async.wait_group 1;" ::: "memory");
        else
          asm volatile("cp.async.wait_group 0;" ::: "memory");
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[pending]);
      };
      for (long long i = 0; i < nloc && ok; ++i) {
        const int buf = (int)(i & 1);
        if (!__all_sync(0xffffffffu, mbar_wait_ab(&aFull[buf], (uint32_t)((i >> 1) & 1), sAbort))) {
          fail();
          break;
        }
        const long long v = (blockIdx.x + i * gridDim.x) / NA;
        const int *sJ = sJb + buf * 64;
        for (int t = 0; t < ntiles; ++t) {
          const long long gt = i * ntiles + t;
          const int s = (int)(gt % WS_STAGES);
          const long long u = gt / WS_STAGES;
          if (gt >= WS_STAGES && !__all_sync(0xffffffffu, mbar_wait_ab(&empty[s], (uint32_t)((u - 1) & 1), sAbort))) {
            fail();
            ok = false;
            break;
          }
          const long long col = (long long)t * MX_TILE_N + cpos;
          const uint32_t nbytes = col < NBpos ? 16u : 0u;  // zero fill beyond the last position
          const uint32_t stg = smem_u32(sB + s * MX_STAGE);
          for (int k = warp + 4 * (lane >> 4); k < nkA; k += 8) {
            const long long o = (v * NA + sJ[k]) * NBpos + (nbytes ? col : 0);
            const uint32_t d = stg + hoff + swz((uint32_t)k, cbyte);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(Chi + o), "r"(nbytes)
                         : "memory");
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d + 16384u), "l"(Clo + o), "r"(nbytes)
                         : "memory");
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
          if (pending >= 0) announce(1);
          pending = s;
        }
        // the item's last stage before the next item's rows are awaited
        if (pending >= 0) {
          announce(0);
          pending = -1;
        }
      }
      if (pending >= 0) announce(0);  // (an abort between issue and announce)
    } else {
      // ================= producers: B[j][k] = C[J_k][j0 + j], warp p owns columns 32p..32p+31
      bool ok = true;
      for (long long i = 0; i < nloc && ok; ++i) {
        const int buf = (int)(i & 1);
        if (!__all_sync(0xffffffffu, mbar_wait_ab(&aFull[buf], (uint32_t)((i >> 1) & 1), sAbort))) {
          fail();
          break;
        }
        const long long v = (blockIdx.x + i * gridDim.x) / NA;
        const int *sJ = sJb + buf * 64;
        for (int t = 0; t < ntiles; ++t) {
          const long long gt = i * ntiles + t;
          const int s = (int)(gt % WS_STAGES);
          const long long u = gt / WS_STAGES;
          const long long col0 = (long long)t * MX_TILE_N + 32 * warp;
          uint4 g[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) g[q] = make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int atom = 0; atom < 2; ++atom) {
            const int k = 32 * atom + lane;
            if (k < nkA) {
              const float *src = Ct32 + v * vpad + (long long)sJ[k] * NBpos;
#pragma unroll
              for (int c = 0; c < 8; c += 2)
                if (col0 + 4 * c < NBpos) ldg256(src + col0 + 4 * c, g[atom * 8 + c], g[atom * 8 + c + 1]);
            }
          }
          if (gt >= WS_STAGES && !__all_sync(0xffffffffu, mbar_wait_ab(&empty[s], (uint32_t)((u - 1) & 1), sAbort))) {
            fail();
            ok = false;
            break;
          }
          uint8_t *stg = sB + s * MX_STAGE;
#pragma unroll
          for (int atom = 0; atom < 2; ++atom) {
            uint8_t *dst = stg + atom * 16384;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const uint4 q = g[atom * 8 + c];
              *(uint32_t *)(dst + swz(32 * warp + 4 * c + 0, 4 * lane)) = q.x;
              *(uint32_t *)(dst + swz(32 * warp + 4 * c + 1, 4 * lane)) = q.y;
              *(uint32_t *)(dst + swz(32 * warp + 4 * c + 2, 4 * lane)) = q.z;
              *(uint32_t *)(dst + swz(32 * warp + 4 * c + 3, 4 * lane)) = q.w;
            }
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[s]);
        }
      }
    }
  } else if (warp == 4) {
    // ================= MMA issuer
    if (lane == 0) {
      // D[j][rs] = sum_k B[j][k] A[rs][k]: the gathered C tile is the M=128 operand,
      // the integral block the N=nN operand, so TMEM lanes are beta positions.
      // BF16X2: the C tile is MN-major (transpose bit 15 of the instruction descriptor)
      const uint32_t idesc = (MODE == FORTE_BF16X2)
                                 ? ((1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (((uint32_t)nN >> 3) << 17) |
                                    ((128u >> 4) << 24))
                                 : ((1u << 4) | (2u << 7) | (2u << 10) | (((uint32_t)nN >> 3) << 17) | ((128u >> 4) << 24));
      bool ok = true;
      for (long long i = 0; i < nloc && ok; ++i) {
        const int buf = (int)(i & 1);
        if (!mbar_wait_ab(&aFull[buf], (uint32_t)((i >> 1) & 1), sAbort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sm + buf * MX_A_BYTES);
        for (int t = 0; t < ntiles; ++t) {
          const long long gt = i * ntiles + t;
          const int s = (int)(gt % WS_STAGES), b = (int)(gt % WS_ACC);
          const long long u = gt / WS_STAGES, ub = gt / WS_ACC;
          if (!mbar_wait_ab(&full[s], (uint32_t)(u & 1), sAbort) ||
              (gt >= WS_ACC && !mbar_wait_ab(&tempty[b], (uint32_t)((ub - 1) & 1), sAbort))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(b * MX_TILE_N);
          const uint64_t ad = desc_kmajor_sw128(a0);
          if (MODE == FORTE_BF16X2) {
            // hi*hi + lo*hi + hi*lo  (C part first, integral part second); offsets in
            // 16-byte units: C part 16 KB, integral part 16 KB; a K step of 16 is
            // 16 C rows (2048 bytes) and 32 bytes of each integral row
            const uint64_t cd = desc_mnmajor_sw128(smem_u32(sB + s * MX_STAGE), 8192u);
            constexpr uint32_t coff[3] = {0u, 1024u, 0u}, goff[3] = {0u, 0u, 1024u};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                mma_issue<MODE>(d, cd + (coff[p] + 128u * ks), ad + (goff[p] + 2u * ks), idesc, (p | ks) != 0);
          } else {
            const uint64_t bd = desc_kmajor_sw128(smem_u32(sB + s * MX_STAGE));
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
              const uint32_t off = (uint32_t)(ks >> 2) * 1024u + 2u * (ks & 3);
              mma_issue<MODE>(d, bd + off, ad + off, idesc, ks != 0);
            }
          }
          mma_commit(&empty[s]);
          mma_commit(&tfull[b]);
        }
        if (ok) mma_commit(&aEmpty[buf]);  // A[buf] free once this item's MMAs are done
      }
      if (!ok) fail();
    }
    __syncwarp();
  } else {
    // ================= epilogue: thread = beta position 128 t + 32 lg + lane (accumulator
    //                   lane); the MX_EPI / 4 warps of a lane quarter split the chunks of 8
    //                   pairs rs (accumulator columns) c0 .. c1-1
    constexpr int PER_Q = MX_EPI / 4;                       // warps per lane quarter
    constexpr int MAXQ = (16 + PER_Q - 1) / PER_Q;          // chunks per warp, at most
    const int e = warp - 8, lg = warp & 3, part = e >> 2;
    const int nch = nN >> 3, c0 = part * nch / PER_Q, c1 = (part + 1) * nch / PER_Q, nq = c1 - c0;
    bool ok = true;
    for (long long i = 0; i < nloc && ok; ++i) {
      const int buf = (int)(i & 1);
      int *acc = accb + buf * ACCW;
      const float fscale = ldexpf(1.f, sx_of((blockIdx.x + i * gridDim.x) / NA));
      const uint32_t acc_s = smem_u32(acc);
      if (!__all_sync(0xffffffffu, mbar_wait_ab(&accReady[buf], (uint32_t)((i >> 1) & 1), sAbort))) {
        fail();
        break;
      }
      for (int t = 0; t < ntiles; ++t) {
        const long long gt = i * ntiles + t;
        const int b = (int)(gt % WS_ACC);
        const long long ub = gt / WS_ACC;
        uint4 tg[MAXQ];
        {
          // this warp's chunks of 8 pairs: 32 lanes read 512 contiguous bytes each
          const uint4 *rowq = (const uint4 *)tabL + ((long long)(t * 4 + lg) * 16 + c0) * 32 + lane;
#pragma unroll
          for (int q = 0; q < MAXQ; ++q)
            tg[q] = (q < nq) ? __ldg(rowq + q * 32) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
          // the next tile's entries into L1 now: they are L2 hits (the table depends
          // on the tile only), and an L2 round trip per tile stalled the scatter
          const int tn = (t + 1 < ntiles) ? t + 1 : 0;
          const uint4 *nxt = (const uint4 *)tabL + ((long long)(tn * 4 + lg) * 16 + c0) * 32 + lane;
#pragma unroll
          for (int q = 0; q < MAXQ; ++q)
            if (q < nq) asm volatile("prefetch.global.L1 [%0];" ::"l"(nxt + q * 32));
        }
        if (!__all_sync(0xffffffffu, mbar_wait_ab(&tfull[b], (uint32_t)(ub & 1), sAbort))) {
          fail();
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * MX_TILE_N + 8 * c0);
        // all of this warp's columns in one round trip, then the accumulator is released
        // before the scatter (a load / wait per 8-column block left the warps waiting on
        // tensor-memory latency and the MMA thread waiting on them)
        uint32_t ra[8 * MAXQ];
#pragma unroll
        for (int q = 0; q < MAXQ; ++q)
          if (q < nq) tmem_ld8(taddr + 8 * q, ra + 8 * q);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) {
          if (q >= nq) break;
          const uint4 tq = tg[q];
          const uint32_t wv[4] = {tq.x, tq.y, tq.z, tq.w};
          if (SPLIT) {
            // entry = byte offset of the word that takes the contribution: the target's
            // positive or negative word (the sign of the replacement), or for a slot
            // without target one of the 32 spare words, in the bank its target would
            // have had, so every reduction of the warp still meets 32 distinct banks
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const uint32_t off = (c & 1) ? (wv[c >> 1] >> 16) : (wv[c >> 1] & 0xFFFFu);
              const float tv = fmaf(__uint_as_float(ra[8 * q + c]), fscale, 12582912.0f);
              red_add(acc_s + off, __float_as_int(tv));
            }
            continue;
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            // entry in the low half of en (the high half is ignored by the masks below)
            const uint32_t en = (c & 1) ? (wv[c >> 1] >> 16) : wv[c >> 1];
            // the sign (bit 0) onto the float's sign bit
            const uint32_t rv = ra[8 * q + c] ^ (en << 31);
            // bits(f 2^S + 1.5 2^23) = bits(1.5 2^23) + rint(f 2^S) for |f 2^S| <= 2^22: one
            // FMA, no conversion instruction (those run on the narrow FP64 / conversion
            // pipe).  The constant bits(1.5 2^23) is added n_kl(beta) times to every output
            // per item (each output has exactly that many replacements) and is removed
            // once, modulo 2^32, at write-out.  The reduction is predicated, not branched.
            const float tv = fmaf(__uint_as_float(rv), fscale, 12582912.0f);
            red_add_if(acc_s + (en & 0xFFFCu), __float_as_int(tv), en);
          }
        }
      }
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&accDone[buf]);
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
  if (warp == 4) tmem_dealloc(tmem, WS_ACC * MX_TILE_N);
}

// ------------------------------------------------------------ host side

static size_t mx_smem_bytes(long long NBpos, bool split, int mode) {
  return 1024 + (size_t)ws_off_acc(mode) + 2 * sizeof(int) * (size_t)(split ? 2 * NBpos + 32 : NBpos) + 2 * 64 * 4 +
         16 + 8 * (2 * ws_stages(mode) + 2 * WS_ACC + 9) + 16 + 64;
}

static uint64_t splitmix64_next(uint64_t &state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Beta-string positions of the alpha-beta kernel (see the top of the file).  The
// per-orbital 5-bit codes are drawn from a fixed-seed generator; of 1024 draws the
// one whose largest hash class is smallest is kept (fewest padding positions; at
// CAS(14,14) 3584 positions for 3432 strings).
static int ab_positions(forte_ctx *ctx) {
  if (ctx->d_abTab) return FORTE_OK;
  const SpinHost &B = ctx->sh[ctx->same_strings ? 0 : 1];
  const int n = ctx->n;
  const long long NB = B.N;
  std::vector<unsigned> hs((size_t)NB);
  unsigned best[32] = {0};
  long long bestG = -1;
  uint64_t state = 0x2405101970000000ull;
  for (int trial = 0; trial < 1024; ++trial) {
    unsigned code[32];
    for (int p = 0; p < n; ++p) code[p] = (unsigned)(splitmix64_next(state) >> 59);
    long long cnt[32] = {0}, G = 0;
    for (long long J = 0; J < NB; ++J) {
      unsigned h = 0;
      for (uint32_t m = B.str[J]; m; m &= m - 1) h ^= code[__builtin_ctz(m)];
      G = std::max(G, ++cnt[h]);
    }
    if (bestG < 0 || G < bestG) {
      bestG = G;
      std::copy(code, code + 32, best);
    }
  }
  const long long NBpos = 32 * bestG;
  if (NBpos > 0x3FFF) {
    set_error("alpha-beta MMA kernel: %lld beta positions exceed the 14-bit scatter table", NBpos);
    return FORTE_ERR_ARG;
  }
  std::vector<uint16_t> posOf((size_t)NB);
  std::vector<int> strOf((size_t)NBpos, -1);
  long long next[32] = {0};
  for (long long J = 0; J < NB; ++J) {
    unsigned h = 0;
    for (uint32_t m = B.str[J]; m; m &= m - 1) h ^= best[__builtin_ctz(m)];
    const long long pos = 32 * next[h]++ + h;
    posOf[J] = (uint16_t)pos;
    strOf[pos] = (int)J;
  }
  const long long rows = (NBpos + MX_TILE_N - 1) / MX_TILE_N * MX_TILE_N;
  std::vector<uint16_t> tab((size_t)rows * 128, 0xFFFFu);
  for (long long pos = 0; pos < NBpos; ++pos) {
    const int J = strOf[pos];
    if (J < 0) continue;
    for (int e = 0; e < B.nk; ++e) {
      const Repl &r = B.list[(size_t)J * B.nk + e];
      tab[(size_t)pos * 128 + r.pair] = (uint16_t)(posOf[r.J] | (r.sgn < 0 ? 0x4000 : 0));
    }
  }
  // The same entries lane-contiguous for the epilogue's coalesced loads.  When the
  // split accumulator row fits in shared memory, an entry is the byte offset of the
  // word that takes the contribution: 4 pos(target) for a positive sign,
  // 4 (NBpos + pos(target)) for a negative one, and for a slot without target
  // 4 (2 NBpos + (lane ^ h_rs)), the spare word in the bank the target would have had
  // (pos = 32 j + h(string) and h(E_rs J) = h(J) ^ code[r] ^ code[s]).  Otherwise it is
  // the byte offset of the target with the sign in bit 0 (positions < 16384, so
  // offsets fit 16 bits with bits 0-1 free; 0xFFFF, bit 1 set, marks "no target").
  // (one table for both modes: decided with the larger stage ring)
  const bool split = std::max(mx_smem_bytes(NBpos, true, FORTE_BF16X2), mx_smem_bytes(NBpos, true, FORTE_TF32)) <= 232448;
  std::vector<unsigned> hpair(128, 0u);
  for (int r = 0; r < n; ++r)
    for (int s2 = 0; s2 <= r; ++s2) hpair[r * (r + 1) / 2 + s2] = (r == s2) ? 0u : (best[r] ^ best[s2]);
  std::vector<uint16_t> tabL(tab.size(), 0xFFFFu);
  for (long long pos = 0; pos < rows; ++pos) {
    const long long t = pos / 128, g = (pos % 128) / 32, ln = pos % 32;
    for (int c = 0; c < 16; ++c)
      for (int e = 0; e < 8; ++e) {
        const int rs = c * 8 + e;
        const uint16_t en = tab[(size_t)pos * 128 + rs];
        uint16_t v;
        if (split)
          v = en == 0xFFFFu ? (uint16_t)(4 * (2 * NBpos + (long long)((unsigned)ln ^ hpair[rs])))
                            : (uint16_t)(4 * ((en & 0x3FFFu) + ((en >> 14) & 1u ? NBpos : 0)));
        else
          v = en == 0xFFFFu ? (uint16_t)0xFFFFu : (uint16_t)(((en & 0x3FFFu) << 2) | ((en >> 14) & 1u));
        tabL[(size_t)((((t * 4 + g) * 16 + c) * 32 + ln) * 8 + e)] = v;
      }
  }
  // npos(x) - nneg(x): signs of the replacements that reach each beta string
  std::vector<int8_t> dcnt((size_t)NB, 0);
  for (long long J = 0; J < NB; ++J)
    for (int e = 0; e < B.nk; ++e) {
      const Repl &r = B.list[(size_t)J * B.nk + e];
      dcnt[r.J] = (int8_t)(dcnt[r.J] + (r.sgn < 0 ? -1 : 1));
    }
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_abDcnt, dcnt.size()));
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_abDcnt, dcnt.data(), dcnt.size(), cudaMemcpyHostToDevice));
  ctx->ab_split = split;
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_abTabL, sizeof(uint16_t) * tabL.size()));
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_abTabL, tabL.data(), sizeof(uint16_t) * tabL.size(), cudaMemcpyHostToDevice));
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_abPosOf, sizeof(uint16_t) * posOf.size()));
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_abStrOf, sizeof(int) * strOf.size()));
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_abTab, sizeof(uint16_t) * tab.size()));
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_abPosOf, posOf.data(), sizeof(uint16_t) * posOf.size(), cudaMemcpyHostToDevice));
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_abStrOf, strOf.data(), sizeof(int) * strOf.size(), cudaMemcpyHostToDevice));
  FORTE_CUDA_TRY(cudaMemcpy(ctx->d_abTab, tab.data(), sizeof(uint16_t) * tab.size(), cudaMemcpyHostToDevice));
  ctx->ab_NBpos = NBpos;
  return FORTE_OK;
}

int mixed_setup(forte_ctx *ctx) {
  const int np = ctx->npair;
  if (ctx->d_gT_hi) return FORTE_OK;
  double gm = 0.0;
  for (double x : ctx->eri) gm = std::max(gm, fabs(x));
  ctx->gmax = (float)(gm * (1.0 + 1e-6));
  size_t cnt = (size_t)128 * np;
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_gT_hi, cnt * sizeof(uint16_t)));
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_gT_lo, cnt * sizeof(uint16_t)));
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_gT_t32, cnt * sizeof(float)));
  if (!ctx->d_err) {
    const int rc_err = err_word_setup(ctx);
    if (rc_err) return rc_err;
  }
  k_split_g<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(ctx->d_gpair, np, ctx->d_gT_hi, ctx->d_gT_lo,
                                                                    ctx->d_gT_t32);
  FORTE_LAUNCH_CHECK();
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_gTT_hi, cnt * sizeof(uint16_t)));
  FORTE_CUDA_TRY(cudaMalloc(&ctx->d_gTT_lo, cnt * sizeof(uint16_t)));
  k_pair_major<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(ctx->d_gT_hi, ctx->d_gT_lo, np, ctx->d_gTT_hi,
                                                                       ctx->d_gTT_lo);
  FORTE_LAUNCH_CHECK();
  if (ctx->sh[0].nk > 0 && ctx->sh[ctx->same_strings ? 0 : 1].nk > 0) return ab_positions(ctx);
  return FORTE_OK;
}

// C, S: FP64 vectors, or the FP32 vectors of the reduced-precision Davidson phase.
template <typename T>
static int sigma_mixed_t(forte_ctx *ctx, const T *C, T *S, int nvec, int mode) {
  if (mode != FORTE_BF16X2 && mode != FORTE_TF32) {
    set_error("unknown precision mode %d", mode);
    return FORTE_ERR_ARG;
  }
  const int nkA = ctx->sh[0].nk, nkB = ctx->sh[1].nk;
  if (nkA > 64 || ctx->npair > 128) {
    set_error("reduced-precision sigma supports n_kl <= 64 and n(n+1)/2 <= 128 (norb <= 15); use FORTE_FP64");
    return FORTE_ERR_ARG;
  }
  int rc = mixed_setup(ctx);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const long long NA = ctx->Na, NB = ctx->Nb, ND = ctx->Ndet;
  const long long NBp = (NB + 15) & ~15LL;
  const size_t nf = (size_t)nvec * ND, np = (size_t)nvec * NA * NBp;
  // scratch: C32, T1, T2, S32 (FP32, ND each) + tensor-core copy (2 x u16 or 1 x f32 per
  // padded element) + per-vector max |C|
  // + the transposed copies of the tensor-core same-spin GEMM (4 bytes per element)
  const bool ssm = ss_mma_supported(ctx);
  const size_t ntw = ssm ? (size_t)nvec * NB * ((NA + 15) & ~15LL) * 4 : 0;
  // the C copy in beta positions for the alpha-beta kernel (4 bytes per element)
  const long long NBpos = ctx->ab_NBpos;
  const bool ab = nkA > 0 && nkB > 0;
  const size_t npos = ab ? (size_t)nvec * NA * NBpos : 0;
  const size_t bytes = 4 * nf * sizeof(float) + np * 4 + ntw + npos * 4 + 1536 + 512 + sizeof(unsigned) * nvec;
  if ((rc = ctx->sc_mixed.ensure(bytes))) return rc;
  float *C32 = (float *)ctx->sc_mixed.ptr;
  // the FP32 copy of C feeds only the CSR fallback of the same-spin term
  float *C32w = (!ssm && sizeof(T) == 8) ? C32 : nullptr;
  const float *C32r = sizeof(T) == 8 ? C32 : (const float *)(const void *)C;
  float *T1 = C32 + nf, *T2 = T1 + nf, *S32 = T2 + nf;
  uint8_t *tc = (uint8_t *)(((uintptr_t)(S32 + nf) + 255) & ~(uintptr_t)255);
  uint16_t *Chi = (uint16_t *)tc, *Clo = Chi + np;
  float *Ct32 = (float *)tc;
  uint8_t *tw = (uint8_t *)(((uintptr_t)(tc + np * 4) + 255) & ~(uintptr_t)255);
  uint8_t *tp = (uint8_t *)(((uintptr_t)(tw + ntw) + 255) & ~(uintptr_t)255);
  uint16_t *Phi = ab ? (uint16_t *)tp : nullptr, *Plo = ab ? Phi + npos : nullptr;
  float *Pt32 = ab ? (float *)tp : nullptr;
  const int *strOf = ab ? ctx->d_abStrOf : nullptr;
  unsigned *cmax = (unsigned *)(((uintptr_t)(tp + npos * 4) + 255) & ~(uintptr_t)255);
  FORTE_CUDA_TRY(cudaMemsetAsync(cmax, 0, sizeof(unsigned) * nvec, st));
  {
    const long long per = NA * NBp;
    dim3 grid((unsigned)std::min<long long>((per + 255) / 256, 152LL * 16), (unsigned)nvec);
    FORTE_PROF(ctx, "split");
    const long long wcols = std::max(NBp, ab ? NBpos : 0LL);
    dim3 g2((unsigned)std::min<long long>(NA * ((wcols + 255) / 256), 152LL * 8), 1u, (unsigned)nvec);
    if (!C32w) {  // no FP32 copy wanted: the row kernel writes both copies
      if (mode == FORTE_BF16X2)
        k_split_rows<FORTE_BF16X2, T><<<g2, 256, 0, st>>>(C, Chi, Clo, nullptr, NA, NB, NBp, cmax, strOf, NBpos, Phi,
                                                          Plo, nullptr);
      else
        k_split_rows<FORTE_TF32, T><<<g2, 256, 0, st>>>(C, nullptr, nullptr, Ct32, NA, NB, NBp, cmax, strOf, NBpos,
                                                        nullptr, nullptr, Pt32);
    } else {
      if (mode == FORTE_BF16X2)
        k_split<FORTE_BF16X2, T><<<grid, 256, 0, st>>>(C, C32w, Chi, Clo, nullptr, NA, NB, NBp, cmax);
      else
        k_split<FORTE_TF32, T><<<grid, 256, 0, st>>>(C, C32w, nullptr, nullptr, Ct32, NA, NB, NBp, cmax);
      FORTE_LAUNCH_CHECK();
      if (ab) {  // positional copy only (the row copy is written above)
        if (mode == FORTE_BF16X2)
          k_split_rows<FORTE_BF16X2, T><<<g2, 256, 0, st>>>(C, nullptr, nullptr, nullptr, NA, NB, NBp, cmax, strOf,
                                                            NBpos, Phi, Plo, nullptr);
        else
          k_split_rows<FORTE_TF32, T><<<g2, 256, 0, st>>>(C, nullptr, nullptr, nullptr, NA, NB, NBp, cmax, strOf,
                                                          NBpos, nullptr, nullptr, Pt32);
      }
    }
    FORTE_LAUNCH_CHECK();
  }
  if (ssm)
    rc = same_spin_mma(ctx, C, Chi, Clo, Ct32, tw, S32, nvec, mode);
  else
    rc = same_spin_f32(ctx, C32r, S32, T1, T2, nvec);
  if (rc) return rc;
  if (ab) {
    const int nN = ctx->npair <= 112 ? 112 : 128;
    const bool split = ctx->ab_split;
    const size_t smem = mx_smem_bytes(NBpos, split, mode);
    if (smem > 232448) {
      set_error("alpha-beta MMA kernel needs %zu bytes of shared memory", smem);
      return FORTE_ERR_ARG;
    }
    int nsm = 0;
    FORTE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const long long nitems = NA * nvec;
    dim3 grid((unsigned)std::min<long long>(nitems, nsm));
    auto launch = [&](auto kern, const char *name, const uint16_t *ph, const uint16_t *pl, const float *pt) -> int {
      FORTE_CUDA_TRY(set_smem_optin_max((const void *)kern));
      FORTE_PROF(ctx, name);
      kern<<<grid, MX_THREADS, smem, st>>>(ctx->sd[0].list, nkA, nkB, ctx->d_abTabL, ctx->d_abPosOf, ctx->d_abDcnt, nN,
                                           NA, NB, NBpos, ctx->d_gTT_hi, ctx->d_gTT_lo, ctx->d_gT_t32, ctx->npair,
                                           ctx->gmax, cmax, ph, pl, pt, S32, S, nitems, ctx->d_err);
      FORTE_LAUNCH_CHECK();
      return FORTE_OK;
    };
    if (mode == FORTE_BF16X2)
      rc = split ? launch(k_ab_mma<FORTE_BF16X2, T, true>, "ab_mma_bf16x2", Phi, Plo, nullptr)
                 : launch(k_ab_mma<FORTE_BF16X2, T, false>, "ab_mma_bf16x2", Phi, Plo, nullptr);
    else
      rc = split ? launch(k_ab_mma<FORTE_TF32, T, true>, "ab_mma_tf32", nullptr, nullptr, Pt32)
                 : launch(k_ab_mma<FORTE_TF32, T, false>, "ab_mma_tf32", nullptr, nullptr, Pt32);
    if (rc) return rc;
  } else if (sizeof(T) == 8) {
    FORTE_PROF(ctx, "f32_to_f64");
    k_f32_to_f64<<<(unsigned)std::min<size_t>((nf + 255) / 256, 152 * 32), 256, 0, st>>>(S32, (double *)(void *)S,
                                                                                     (long long)nf);
    FORTE_LAUNCH_CHECK();
  } else {
    FORTE_CUDA_TRY(cudaMemcpyAsync((void *)S, S32, sizeof(float) * nf, cudaMemcpyDeviceToDevice, st));
  }
  return FORTE_OK;
}

int sigma_mixed(forte_ctx *ctx, const double *C, double *S, int nvec, int mode) {
  return sigma_mixed_t(ctx, C, S, nvec, mode);
}
int sigma_mixed(forte_ctx *ctx, const float *C, float *S, int nvec, int mode) {
  return sigma_mixed_t(ctx, C, S, nvec, mode);
}

// Device status of bounded waits: FORTE_OK, or FORTE_ERR_TIMEOUT (and reset).
int mixed_status(forte_ctx *ctx) {
  if (!ctx->d_err) return FORTE_OK;
  int h = 0;
  FORTE_CUDA_TRY(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  FORTE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (h) {
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    // one bit per kernel (the value each kernel ORs into the flag)
    std::string who;
    const char *names[4] = {"alpha-beta MMA", "same-spin MMA", "digit-slice alpha-beta", "digit-slice 2-RDM Gram"};
    for (int b = 0; b < 4; ++b)
      if (h & (1 << b)) who += (who.empty() ? "" : ", ") + std::string(names[b]);
    set_error("a bounded device wait expired in: %s", who.c_str());
    return FORTE_ERR_TIMEOUT;
  }
  return FORTE_OK;
}

}  // namespace forte
