// Same-spin part of the reduced-precision sigma (steps a5, a6: Sec. II.A, the
// alpha-alpha and beta-beta terms of Eq. (sigma)) as one dense GEMM per vector on
// the 5th-generation tensor cores.
//
//   S_ss[Ia][Ib] = sum_Ja H_a[Ia][Ja] C[Ja][Ib] + sum_Jb C[Ia][Jb] H_b[Ib][Jb]
//
// H_a, H_b are the same-spin string Hamiltonians (one-body k plus the same-spin
// two-body term, diagonal included), held dense.  Concatenating the contraction
// index K = [Ja | Jb] makes this one product S_ss = A B^T with
//   A = [H_a | C]    (M = Na rows, alpha strings),
//   B = [C^T | H_b]  (N = Nb rows, beta strings; H_b is symmetric),
// both K-major.  The string Hamiltonians are sparse (491 of 3432 entries per row
// at CAS(14,14)), so the dense product does ~7x the multiply-adds of the CSR
// product, on the tensor pipe instead of the FP32 pipe.
//
// Operands: FORTE_BF16X2 splits x = hi + lo and forms hi*hi + hi*lo + lo*hi with
// FP32 accumulation; FORTE_TF32 rounds to TF32.  Tiles of 128 x 256 outputs; the
// K tiles (128 bytes per row: 64 BF16 or 32 TF32 elements) arrive by TMA in the
// 128-byte swizzle that the MMA descriptors read.
//
// Kernel structure (persistent, one CTA per SM, 8 warps):
//   * warp 0, one thread: TMA loads of the A and B tiles into a stage ring,
//     completing on the stage's `full` mbarrier;
//   * warp 1, one thread: tcgen05.mma chain of a tile into one of two 256-column
//     TMEM accumulators, commits to the stage's `empty` and the accumulator's
//     `tfull` mbarriers (warp 1 owns the TMEM allocation);
//   * warps 4-7: tcgen05.ld of the accumulator (lane = alpha string), FP32 rows
//     of S_ss to global memory, `tempty` arrive.
// Every mbarrier wait is bounded; on expiry the context status word is raised,
// the roles stop, the MMA thread drains its MMAs (bounded) and TMEM is freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "bf16_split.h"
#include "forte_internal.h"
#include "tc_ptx.cuh"

namespace forte {

constexpr int SSM_BM = 128, SSM_BN = 256;
constexpr int SSM_THREADS = 256;

struct SsmMaps {
  CUtensorMap a_h[2];   // H_a  hi / lo (or TF32 in [0]): [Na][NaP], box K x 128
  CUtensorMap a_c[2];   // C    hi / lo: [nvec][Na][NbP], box K x 128
  CUtensorMap b_ct[2];  // C^T  hi / lo: [nvec][Nb][NaP], box K x 256
  CUtensorMap b_h[2];   // H_b  hi / lo: [Nb][NbP], box K x 256
};

template <int MODE>
struct SsmCfg {
  static constexpr int KT = MODE == FORTE_BF16X2 ? 64 : 32;  // K elements per 128-byte row
  static constexpr int NPART = MODE == FORTE_BF16X2 ? 2 : 1;
  static constexpr int A_BYTES = SSM_BM * 128;
  static constexpr int B_BYTES = SSM_BN * 128;
  static constexpr int STAGE = NPART * (A_BYTES + B_BYTES);
  static constexpr int NSTAGE = MODE == FORTE_BF16X2 ? 2 : 4;
};

template <int MODE>
__global__ void __launch_bounds__(SSM_THREADS, 1)
    k_ss_mma(const __grid_constant__ SsmMaps maps, long long NA, long long NB, int nKa, int nKb, int mt, int nt,
             int ntiles, float *__restrict__ S, int *__restrict__ err) {
  using Cf = SsmCfg<MODE>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t *bar = (uint64_t *)(sm + Cf::NSTAGE * Cf::STAGE);
  uint64_t *full = bar, *empty = bar + Cf::NSTAGE, *tfull = bar + 2 * Cf::NSTAGE, *tempty = tfull + 2;
  uint64_t *drain = tempty + 2;
  uint32_t *sTmem = (uint32_t *)(drain + 1);
  volatile int *sAbort = (volatile int *)(sTmem + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nK = nKa + nKb;
  if (warp == 1) tmem_alloc(sTmem, 512);
  if (tid == 0) {
    for (int i = 0; i < Cf::NSTAGE; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(drain, 1);
    abort_word_init(sAbort, err);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;

  if (warp == 0) {
    // ================= TMA producer
    if (lane == 0) {
      for (int p = 0; p < Cf::NPART; ++p) {
        tma_prefetch_map(&maps.a_h[p]);
        tma_prefetch_map(&maps.a_c[p]);
        tma_prefetch_map(&maps.b_ct[p]);
        tma_prefetch_map(&maps.b_h[p]);
      }
      long long it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int v = tile / (mt * nt), rem = tile % (mt * nt), mi = rem / nt, ni = rem % nt;
        for (int kt = 0; kt < nK; ++kt, ++it) {
          const int s = (int)(it % Cf::NSTAGE);
          const long long u = it / Cf::NSTAGE;
          if (it >= Cf::NSTAGE && !mbar_wait_ab(&empty[s], (uint32_t)((u - 1) & 1), sAbort)) {
            *sAbort = 1;
            atomicOr(err, 2);
            ok = false;
            break;
          }
          uint8_t *st = sm + s * Cf::STAGE;
          mbar_expect_tx(&full[s], (uint32_t)Cf::STAGE);
#pragma unroll
          for (int p = 0; p < Cf::NPART; ++p) {
            uint8_t *a = st + p * Cf::A_BYTES;
            uint8_t *b = st + Cf::NPART * Cf::A_BYTES + p * Cf::B_BYTES;
            if (kt < nKa) {
              tma_load_3d(a, &maps.a_h[p], kt * Cf::KT, mi * SSM_BM, 0, &full[s]);
              tma_load_3d(b, &maps.b_ct[p], kt * Cf::KT, ni * SSM_BN, v, &full[s]);
            } else {
              const int x = (kt - nKa) * Cf::KT;
              tma_load_3d(a, &maps.a_c[p], x, mi * SSM_BM, v, &full[s]);
              tma_load_3d(b, &maps.b_h[p], x, ni * SSM_BN, 0, &full[s]);
            }
          }
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA can exit (stages not
        // yet reused, so the parity of their last phase is still current)
        for (long long g = it > Cf::NSTAGE ? it - Cf::NSTAGE : 0; g < it; ++g)
          mbar_wait(&full[g % Cf::NSTAGE], (uint32_t)((g / Cf::NSTAGE) & 1));
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ================= MMA issuer
    if (lane == 0) {
      const uint32_t fmt = MODE == FORTE_BF16X2 ? 1u : 2u;
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(SSM_BN >> 3) << 17) |
                             ((uint32_t)(SSM_BM >> 4) << 24);
      long long it = 0;
      int lt = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        const int b = lt & 1, ub = lt >> 1;
        if (lt >= 2 && !mbar_wait_ab(&tempty[b], (uint32_t)((ub - 1) & 1), sAbort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * SSM_BN);
        for (int kt = 0; kt < nK; ++kt, ++it) {
          const int s = (int)(it % Cf::NSTAGE);
          if (!mbar_wait_ab(&full[s], (uint32_t)((it / Cf::NSTAGE) & 1), sAbort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sm + s * Cf::STAGE);
          const uint32_t b0 = a0 + (uint32_t)(Cf::NPART * Cf::A_BYTES);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            if (MODE == FORTE_BF16X2) {
              // hi*hi + hi*lo + lo*hi
              const uint32_t ao[3] = {0u, 0u, (uint32_t)Cf::A_BYTES}, bo[3] = {0u, (uint32_t)Cf::B_BYTES, 0u};
#pragma unroll
              for (int p = 0; p < 3; ++p)
                mma_issue<MODE>(d, desc_kmajor_sw128(a0 + ao[p] + 32u * ks), desc_kmajor_sw128(b0 + bo[p] + 32u * ks),
                                idesc, (kt | ks | p) != 0);
            } else {
              mma_issue<MODE>(d, desc_kmajor_sw128(a0 + 32u * ks), desc_kmajor_sw128(b0 + 32u * ks), idesc,
                              (kt | ks) != 0);
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[b]);
      }
      if (!ok) {
        *sAbort = 1;
        atomicOr(err, 2);
      }
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ================= epilogue: lane = alpha string of the tile
    const int quarter = warp & 3;
    const bool vec4 = (NB & 3) == 0;
    int lt = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      const int v = tile / (mt * nt), rem = tile % (mt * nt), mi = rem / nt, ni = rem % nt;
      const int b = lt & 1, ub = lt >> 1;
      if (!__all_sync(0xffffffffu, mbar_wait_ab(&tfull[b], (uint32_t)(ub & 1), sAbort))) {
        *sAbort = 1;
        atomicOr(err, 2);
        break;
      }
      tc_fence_after();
      const long long row = (long long)mi * SSM_BM + quarter * 32 + lane;
      float *out = S + ((long long)v * NA + row) * NB;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * SSM_BN);
#pragma unroll 1
      for (int c0 = 0; c0 < SSM_BN; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const long long col = (long long)ni * SSM_BN + c0;
        if (row < NA) {
          if (vec4 && col + 16 <= NB) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              *(float4 *)(out + col + 4 * q) = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                                           __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col + j < NB) out[col + j] = __uint_as_float(r[j]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  __syncthreads();
  if (*sAbort && warp == 1 && lane == 0) {
    mma_commit(drain);  // tracks every MMA this thread issued
    mbar_wait(drain, 0u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------ operand preparation

// Dense same-spin Hamiltonian from the CSR rows: hi / lo BF16 (and TF32) copies,
// row pitch Np (the padding columns stay zero).  One block per row.
__global__ void k_dense_h(const int *__restrict__ ptr, const int *__restrict__ col, const double *__restrict__ val,
                          long long N, long long Np, uint16_t *__restrict__ hi, uint16_t *__restrict__ lo,
                          float *__restrict__ t32) {
  const long long r = blockIdx.x;
  for (int e = ptr[r] + threadIdx.x; e < ptr[r + 1]; e += blockDim.x) {
    const double x = val[e];
    const long long i = r * Np + col[e];
    const double h = rne_drop(x, 45);
    hi[i] = bf16_bits(h);
    lo[i] = bf16_bits(rne_drop(x - h, 45));
    t32[i] = (float)rne_drop(x, 42);
  }
}

// Transposed split copies of C for the same-spin GEMM: T[v][b][a] = split(C[v][a][b]),
// a padded to NAp with zeros.  64 x 64 tiles, each thread writes two consecutive
// transposed elements as one 32-bit (BF16 pair) or 64-bit (TF32 pair) store.  BF16:
// hi = x rounded to nearest even, lo = the remainder rounded likewise; TF32: 10
// mantissa bits, nearest even.  grid = (NAp / 64, NB / 64,
// vector), block (32, 8).
__device__ __forceinline__ uint32_t ssm_bf16_hi(float x, uint16_t &lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  return __bfloat16_as_ushort(h);
}
__device__ __forceinline__ uint32_t ssm_bf16_hi(double x, uint16_t &lo) {
  uint16_t hb;
  if (bf16_split_bits(x, hb, lo)) return hb;  // integer path; conversions for the rest
  const __nv_bfloat16 h = __double2bfloat16(x);
  lo = __bfloat16_as_ushort(__double2bfloat16(x - (double)__bfloat162float(h)));
  return __bfloat16_as_ushort(h);
}
__device__ __forceinline__ float ssm_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0xFFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & ~0x1FFFu);
}
__device__ __forceinline__ float ssm_tf32(double x) { return (float)rne_drop(x, 42); }

template <int MODE, typename TI>
__global__ void __launch_bounds__(256) k_split_t64(const TI *__restrict__ C, long long NA, long long NB,
                                                   long long NAp, uint16_t *__restrict__ hi, uint16_t *__restrict__ lo,
                                                   float *__restrict__ t32) {
  __shared__ TI tile[64][65];
  const long long v = blockIdx.z;
  const long long a0 = (long long)blockIdx.x * 64, b0 = (long long)blockIdx.y * 64;
  const TI *Cv = C + v * NA * NB;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 64; i += 8)
    for (int j = tx; j < 64; j += 32) {
      const long long a = a0 + i, b = b0 + j;
      tile[i][j] = (a < NA && b < NB) ? Cv[a * NB + b] : TI(0);
    }
  __syncthreads();
  const long long a = a0 + 2 * tx;
  for (int i = ty; i < 64; i += 8) {
    const long long b = b0 + i;
    if (b >= NB || a >= NAp) continue;
    const TI x0 = tile[2 * tx][i], x1 = tile[2 * tx + 1][i];
    const long long o = (v * NB + b) * NAp + a;  // even: NAp and a are even
    if (MODE == FORTE_BF16X2) {
      uint16_t l0, l1;
      const uint32_t h0 = ssm_bf16_hi(x0, l0), h1 = ssm_bf16_hi(x1, l1);
      *(uint32_t *)(hi + o) = h0 | (h1 << 16);
      *(uint32_t *)(lo + o) = (uint32_t)l0 | ((uint32_t)l1 << 16);
    } else {
      *(float2 *)(t32 + o) = make_float2(ssm_tf32(x0), ssm_tf32(x1));
    }
  }
}

// ------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 3-D map over [nmat][rows][pitch] elements with the logical extent K x rows
// (reads beyond K or rows fill zeros); box = 128 bytes x box_rows, 128-byte swizzle.
static int make_map(CUtensorMap *m, bool f32, const void *base, long long K, long long rows, long long nmat,
                    long long pitch, int box_rows) {
  auto enc = tma_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return FORTE_ERR_CUDA;
  }
  const int es = f32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nmat};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * es), (cuuint64_t)(pitch * es * rows)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                   const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FORTE_ERR_CUDA;
  }
  return FORTE_OK;
}

static long long pad16(long long x) { return (x + 15) & ~15LL; }

bool ss_mma_supported(const forte_ctx *ctx) {
  // dense string Hamiltonians of both spins: 8 bytes per element (hi, lo, TF32)
  const long long NA = ctx->Na, NB = ctx->Nb;
  const double bytes = 8.0 * ((double)NA * pad16(NA) + (ctx->same_strings ? 0.0 : (double)NB * pad16(NB)));
  return NA >= 1 && NB >= 1 && bytes <= 4.0e9 && tma_encoder() != nullptr;
}

static int ss_dense_setup(forte_ctx *ctx) {
  if (ctx->d_hd_hi[0]) return FORTE_OK;
  const int nsp = ctx->same_strings ? 1 : 2;
  for (int s = 0; s < nsp; ++s) {
    const long long N = s == 0 ? ctx->Na : ctx->Nb, Np = pad16(N);
    const size_t cnt = (size_t)N * Np;
    FORTE_CUDA_TRY(cudaMalloc(&ctx->d_hd_hi[s], cnt * sizeof(uint16_t)));
    FORTE_CUDA_TRY(cudaMalloc(&ctx->d_hd_lo[s], cnt * sizeof(uint16_t)));
    FORTE_CUDA_TRY(cudaMalloc(&ctx->d_hd_t32[s], cnt * sizeof(float)));
    FORTE_CUDA_TRY(cudaMemsetAsync(ctx->d_hd_hi[s], 0, cnt * sizeof(uint16_t), ctx->stream));
    FORTE_CUDA_TRY(cudaMemsetAsync(ctx->d_hd_lo[s], 0, cnt * sizeof(uint16_t), ctx->stream));
    FORTE_CUDA_TRY(cudaMemsetAsync(ctx->d_hd_t32[s], 0, cnt * sizeof(float), ctx->stream));
    k_dense_h<<<(unsigned)N, 128, 0, ctx->stream>>>(ctx->sd[s].csr_ptr, ctx->sd[s].csr_col, ctx->sd[s].csr_val, N, Np,
                                                    ctx->d_hd_hi[s], ctx->d_hd_lo[s], ctx->d_hd_t32[s]);
    FORTE_LAUNCH_CHECK();
  }
  if (ctx->same_strings) {
    ctx->d_hd_hi[1] = ctx->d_hd_hi[0];
    ctx->d_hd_lo[1] = ctx->d_hd_lo[0];
    ctx->d_hd_t32[1] = ctx->d_hd_t32[0];
  }
  return FORTE_OK;
}

// S32[v] = same-spin sigma of C[v] (FP64 input; Chi/Clo or Ct32 are the row-split
// copies [nvec][NA][NBp] made by the caller).  `tw` is workspace for the
// transposed copies: nvec * NB * NAp * 4 bytes.
template <typename TI>
static int same_spin_mma_t(forte_ctx *ctx, const TI *C, const uint16_t *Chi, const uint16_t *Clo, const float *Ct32,
                           void *tw, float *S32, int nvec, int mode) {
  int rc = ss_dense_setup(ctx);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const long long NA = ctx->Na, NB = ctx->Nb, NAp = pad16(NA), NBp = pad16(NB);
  const bool bf = mode == FORTE_BF16X2;
  uint16_t *Thi = (uint16_t *)tw, *Tlo = Thi + (size_t)nvec * NB * NAp;
  float *Tt = (float *)tw;
  {
    dim3 tb(32, 8);
    FORTE_PROF(ctx, "split_t");
    dim3 g64((unsigned)((NAp + 63) / 64), (unsigned)((NB + 63) / 64), (unsigned)nvec);
    if (bf)
      k_split_t64<FORTE_BF16X2, TI><<<g64, tb, 0, st>>>(C, NA, NB, NAp, Thi, Tlo, nullptr);
    else
      k_split_t64<FORTE_TF32, TI><<<g64, tb, 0, st>>>(C, NA, NB, NAp, nullptr, nullptr, Tt);
    FORTE_LAUNCH_CHECK();
  }
  SsmMaps maps;
  memset(&maps, 0, sizeof(maps));
  const int np = bf ? 2 : 1;
  for (int p = 0; p < np; ++p) {
    const void *ha = bf ? (const void *)(p ? ctx->d_hd_lo[0] : ctx->d_hd_hi[0]) : (const void *)ctx->d_hd_t32[0];
    const void *hb = bf ? (const void *)(p ? ctx->d_hd_lo[1] : ctx->d_hd_hi[1]) : (const void *)ctx->d_hd_t32[1];
    const void *cc = bf ? (const void *)(p ? Clo : Chi) : (const void *)Ct32;
    const void *ct = bf ? (const void *)(p ? Tlo : Thi) : (const void *)Tt;
    if ((rc = make_map(&maps.a_h[p], !bf, ha, NA, NA, 1, NAp, SSM_BM))) return rc;
    if ((rc = make_map(&maps.a_c[p], !bf, cc, NB, NA, nvec, NBp, SSM_BM))) return rc;
    if ((rc = make_map(&maps.b_ct[p], !bf, ct, NA, NB, nvec, NAp, SSM_BN))) return rc;
    if ((rc = make_map(&maps.b_h[p], !bf, hb, NB, NB, 1, NBp, SSM_BN))) return rc;
  }
  const int kt = bf ? 64 : 32;
  const int nKa = (int)((NA + kt - 1) / kt), nKb = (int)((NB + kt - 1) / kt);
  const int mt = (int)((NA + SSM_BM - 1) / SSM_BM), nt = (int)((NB + SSM_BN - 1) / SSM_BN);
  const long long ntiles = (long long)mt * nt * nvec;
  if (ntiles > 0x7FFFFFFF) {
    set_error("same-spin GEMM: too many tiles");
    return FORTE_ERR_ARG;
  }
  int nsm = 0;
  FORTE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  const unsigned grid = (unsigned)std::min<long long>(ntiles, nsm);
  if (bf) {
    const size_t smem = 1024 + SsmCfg<FORTE_BF16X2>::NSTAGE * SsmCfg<FORTE_BF16X2>::STAGE + 256;
    FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_ss_mma<FORTE_BF16X2>));
    FORTE_PROF(ctx, "ss_mma_bf16x2");
    k_ss_mma<FORTE_BF16X2><<<grid, SSM_THREADS, smem, st>>>(maps, NA, NB, nKa, nKb, mt, nt, (int)ntiles, S32,
                                                           ctx->d_err);
    FORTE_LAUNCH_CHECK();
  } else {
    const size_t smem = 1024 + SsmCfg<FORTE_TF32>::NSTAGE * SsmCfg<FORTE_TF32>::STAGE + 256;
    FORTE_CUDA_TRY(set_smem_optin_max((const void *)k_ss_mma<FORTE_TF32>));
    FORTE_PROF(ctx, "ss_mma_tf32");
    k_ss_mma<FORTE_TF32><<<grid, SSM_THREADS, smem, st>>>(maps, NA, NB, nKa, nKb, mt, nt, (int)ntiles, S32,
                                                         ctx->d_err);
    FORTE_LAUNCH_CHECK();
  }
  return FORTE_OK;
}

int same_spin_mma(forte_ctx *ctx, const double *C, const uint16_t *Chi, const uint16_t *Clo, const float *Ct32,
                  void *tw, float *S32, int nvec, int mode) {
  return same_spin_mma_t(ctx, C, Chi, Clo, Ct32, tw, S32, nvec, mode);
}
int same_spin_mma(forte_ctx *ctx, const float *C, const uint16_t *Chi, const uint16_t *Clo, const float *Ct32,
                  void *tw, float *S32, int nvec, int mode) {
  return same_spin_mma_t(ctx, C, Chi, Clo, Ct32, tw, S32, nvec, mode);
}

}  // namespace forte
