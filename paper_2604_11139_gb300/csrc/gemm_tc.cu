// BF16-split tensor-core GEMM (tcgen05 + TMA) for the projector contractions of the
// mixed-precision filter (Sec. 4.2: C_proj = <p|Psi>, Psi += P (D C_proj)).
//
// Complex GEMMs are run as real GEMMs on interleaved (re, im) data:
//   C = P^dagger Y  ->  C_r (2Np x M) = A1 (2Np x 2N) . Y_r (2N x M),
//                       A1 rows 2i / 2i+1 = column i of P / of iP as 2N reals;
//   Y += P Z        ->  Y_r (2N x M) = A2 (2N x 2Np) . Z_r (2Np x M),
//                       A2 rows 2g / 2g+1 = row g of conj(P) / of i conj(P) as 2Np reals.
// Every operand is split into bf16 pieces x = x_0 + x_1 (+ x_2), x_{p} = bf16(x - sum_{q<p} x_q),
// and the product sums the piece pairs (p, q) with p + q < pieces into one FP32
// accumulator in tensor memory (2 pieces: 3 products, ~2^-16 relative; 3 pieces:
// 6 products, ~2^-24).
//
// Kernel: one 128 x 128 output tile per CTA, K in 64-wide slices; warp 0 lane 0
// issues TMA loads (128B-swizzled, K-major) into a multi-stage ring, warp 1 lane 0
// issues tcgen05.mma from shared memory into 128-column TMEM accumulators, four warps
// promote them into a running sum and four more write the output (tcgen05.ld, one TMEM lane
// = one output row per thread).
// Every mbarrier wait is bounded; on expiry the kernel records the stage in *err, waits
// (bounded) for the copies and MMAs it has issued, releases TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "pw_internal.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

namespace pw {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int TILE_BYTES = BM * BK * 2;  // 16 KB; BN == BM
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr uint32_t kSpinTest = 1u << 12;  // wait limit of the failure-path test (no copies issued)

template <int P> struct Cfg {
  static constexpr int STAGE_BYTES = 2 * P * TILE_BYTES;
  static constexpr int STAGES = (P == 2) ? 3 : 2;
  static constexpr int NPROD = (P == 2) ? 3 : 6;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// bounded wait for the phase of parity `par` to complete; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par, uint32_t limit) {
  const uint32_t a = smem_u32(b);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(par)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}
// instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
      "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Asynchronous variants: the load's registers are valid only after tmem_wait_ld(r), whose
// in-out operands keep the compiler from using them earlier; the store is complete only
// after tmem_wait_st().
#define PW_R32(r) "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), \
  "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),     \
  "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]),   \
  "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
#define PW_W32(r) "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),          \
  "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),       \
  "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
#define PW_RW32(r) "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), \
  "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),           \
  "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),        \
  "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])

__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
      "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : PW_W32(r)
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : PW_RW32(r)::"memory");
}
__device__ __forceinline__ void tmem_st32_async(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      PW_R32(r)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void split_store(const TcEpi& e, int r, int j, float y) {
  float rem = y;
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    if (p < e.out_pieces) {
      const __nv_bfloat16 h = __float2bfloat16_rn(rem);
      e.split[(int64_t)p * e.split_piece_stride + (int64_t)j * e.split_ld + r] = h;
      rem -= __bfloat162float(h);
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Persistent, warp-specialised kernel.  Work unit = (split z, M tile, N tile), N fastest.
//   warp 0 lane 0: TMA producer over the units' K slices (ring of STAGES slots);
//   warp 1 lane 0: MMA issuer; each group of kprom 64-wide K slices accumulates into one
//                  of two TMEM buffers (128 columns each), starting from zero;
//   warps 2-5:     drain each finished buffer into a TMEM buffer holding the unit's
//                  running sum (round-to-nearest FP32 adds in registers, one output
//                  row per thread, 32 columns at a time); two running-sum buffers
//                  alternate between units;
//   warps 6-9:     run the output epilogue of a finished unit from its running-sum buffer
//                  while warps 2-5 accumulate the next unit in the other one.
// The tensor core adds its products into the TMEM accumulator with truncation; summing
// few K slices there (one with 3 pieces) and the groups in registers keeps the
// accumulated rounding bias below the error of the bf16 pieces themselves.
template <int P>
__global__ void __launch_bounds__(320, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                    int kchunk, int nsplit, int kprom, TcEpi epi, int* err,
                                                    uint32_t spin, int no_copies) {
  using CF = Cfg<P>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(base + CF::STAGES * CF::STAGE_BYTES);
  uint64_t* empty = full + CF::STAGES;
  uint64_t* tfull = empty + CF::STAGES;  // [2]
  uint64_t* tempty = tfull + 2;          // [2]
  uint64_t* sready = tempty + 2;         // [2] running sum of a unit complete (promotion -> output)
  uint64_t* sfree = sready + 2;          // [2] running-sum buffer written out (output -> promotion)
  uint64_t* mdone = sfree + 2;           // completion of every MMA issued (exit path)
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntn = (N + BN - 1) / BN, ntm = (M + BM - 1) / BM;
  const int nunits = ntn * ntm * nsplit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < CF::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
      mbar_init(&sready[b], 4);
      mbar_init(&sfree[b], 4);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(4 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int g = 0;
      int last_it[CF::STAGES];
      for (int s = 0; s < CF::STAGES; ++s) last_it[s] = -1;
      for (int u = blockIdx.x; u < nunits && !*abort_flag; u += gridDim.x) {
        const int n0 = (u % ntn) * BN, m0 = ((u / ntn) % ntm) * BM, z = u / (ntn * ntm);
        const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
        const int nkb = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % CF::STAGES, it = g / CF::STAGES;
          if (it > 0 && !mbar_wait(&empty[s], (it - 1) & 1, spin)) {
            atomicExch(err, 1);
            *abort_flag = 1;
            break;
          }
          if (no_copies) continue;
          last_it[s] = it;
          mbar_expect_tx(&full[s], CF::STAGE_BYTES);
          const uint32_t sb = smem_u32(base + s * CF::STAGE_BYTES);
          const int k = kbeg + kb * BK;
#pragma unroll
          for (int p = 0; p < P; ++p) tma_load_3d(sb + p * TILE_BYTES, &tmA, k, m0, p, &full[s]);
#pragma unroll
          for (int p = 0; p < P; ++p) tma_load_3d(sb + (P + p) * TILE_BYTES, &tmB, k, n0, p, &full[s]);
        }
      }
      // every copy issued has landed before the CTA may release its shared memory
      for (int s = 0; s < CF::STAGES; ++s)
        if (last_it[s] >= 0 && !mbar_wait(&full[s], last_it[s] & 1, spin)) atomicExch(err, 4);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      int g = 0;   // K slices issued (shared-memory ring)
      int G = 0;   // promotion groups issued (TMEM partial buffers)
      for (int u = blockIdx.x; u < nunits && !*abort_flag; u += gridDim.x) {
        const int z = u / (ntn * ntm);
        const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
        const int nkb = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % CF::STAGES, it = g / CF::STAGES;
          const bool gfirst = (kb % kprom) == 0;
          const bool glast = ((kb + 1) % kprom) == 0 || kb + 1 == nkb;
          const int tb = G & 1, tu = G >> 1;
          if (!mbar_wait(&full[s], it & 1, spin) || (gfirst && tu > 0 && !mbar_wait(&tempty[tb], (tu - 1) & 1, spin))) {
            atomicExch(err, 2);
            *abort_flag = 1;
            break;
          }
          fence_after();
          const uint32_t sb = smem_u32(base + s * CF::STAGE_BYTES);
          const uint32_t dt = tmem + (uint32_t)(tb * BN);
          // Correction products first, into a small accumulator, then the four hi x hi
          // products: only those four additions round at the full magnitude.
#pragma unroll
          for (int pr = CF::NPROD - 1; pr >= 0; --pr) {
            // piece pairs (a, b) with a + b < P: (0,0) (0,1) (1,0) [(0,2) (2,0) (1,1)]
            const int pa = (pr == 2 || pr == 5) ? 1 : (pr == 4 ? 2 : 0);
            const int pb = (pr == 1 || pr == 5) ? 1 : (pr == 3 ? 2 : 0);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t ad = sdesc(sb + pa * TILE_BYTES + kk * 32);
              const uint64_t bd = sdesc(sb + (P + pb) * TILE_BYTES + kk * 32);
              mma_bf16(dt, ad, bd, (!gfirst || pr < CF::NPROD - 1 || kk > 0) ? 1u : 0u);
            }
          }
          mma_commit(&empty[s]);
          if (glast) {
            mma_commit(&tfull[tb]);
            ++G;
          }
        }
      }
      // every MMA issued has completed before TMEM and shared memory are released
      mma_commit(mdone);
      if (!mbar_wait(mdone, 0, spin)) atomicExch(err, 5);
    }
  } else if (warp < 6) {
    // ---- promotion warps 2..5: TMEM lane quarter (warp % 4)
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    int G = 0;  // promotion groups drained
    int lu = 0;  // units of this CTA so far
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++lu) {
      const int z = u / (ntn * ntm);
      const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
      const int nkb = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;
      const int ngrp = (nkb + kprom - 1) / kprom;
      const int sb = lu & 1;
      const uint32_t sum_base = tmem + lane_off + (uint32_t)((2 + sb) * BN);  // running sum of this unit
      // the writers have finished the unit that used this running-sum buffer before
      if (lu >= 2 && !mbar_wait(&sfree[sb], ((lu >> 1) + 1) & 1, spin)) {
        atomicExch(err, 6);
        *abort_flag = 1;
        break;
      }
      bool ok = true;
      for (int kb = 0; kb < ngrp; ++kb, ++G) {
        const int tb = G & 1, tu = G >> 1;
        if (!mbar_wait(&tfull[tb], tu & 1, spin)) {
          ok = false;
          atomicExch(err, 3);
          *abort_flag = 1;
          break;
        }
        fence_after();
        // one load round trip per 32 columns: the slice's partial and the running sum are
        // loaded together, added in registers and stored back without waiting; the stores
        // are waited for once per slice
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
          uint32_t v[32], sm[32];
          tmem_ld32_async(tmem + lane_off + (uint32_t)(tb * BN + c * 32), v);
          if (kb > 0) {
            tmem_ld32_async(sum_base + (uint32_t)(c * 32), sm);
            tmem_wait_ld(v);
            tmem_wait_ld(sm);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = __float_as_uint(__uint_as_float(v[i]) + __uint_as_float(sm[i]));
          } else {
            tmem_wait_ld(v);
          }
          tmem_st32_async(sum_base + (uint32_t)(c * 32), v);
        }
        tmem_wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[tb]);
      }
      if (!ok) break;
      // the unit's running sum is complete: hand it to the writers
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sready[sb]);
    }
  } else {
    // ---- output warps 6..9: TMEM lane quarter (warp % 4); they write unit u's result while
    // the promotion warps already accumulate unit u + 1 in the other running-sum buffer
    const int q = warp & 3;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    int lu = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++lu) {
      const int n0 = (u % ntn) * BN, m0 = ((u / ntn) % ntm) * BM, z = u / (ntn * ntm);
      const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
      const int nkb = (kend > kbeg) ? (kend - kbeg + BK - 1) / BK : 0;
      const int sb = lu & 1;
      if (!mbar_wait(&sready[sb], (lu >> 1) & 1, spin)) {
        atomicExch(err, 7);
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t sum_base = tmem + lane_off + (uint32_t)((2 + sb) * BN);
      const int r = m0 + q * 32 + lane;
      float alpha = epi.alpha, shift = epi.shift;
      if (epi.mode == TC_EPI_CHEB && epi.dev_ce) {
        shift = (float)epi.dev_ce[0];
        alpha = (float)((epi.first ? 1.0 : 2.0) / epi.dev_ce[1]);
      }
#pragma unroll 1
      for (int c = 0; c < BN / 16; ++c) {
        uint32_t ar[16];
        float acc[16];
        if (nkb > 0) {
          tcp::tmem_ld16_async(sum_base + (uint32_t)(c * 16), ar);
          tcp::tmem_wait_ld16(ar);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[i] = __uint_as_float(ar[i]);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[i] = 0.f;
        }
        if (r >= M) continue;
        const int jc = n0 + c * 16;
        if (epi.mode == TC_EPI_PARTIAL) {
          float* __restrict__ o = epi.part + (int64_t)z * epi.part_split_stride + (int64_t)jc * epi.part_ld + r;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (jc + i < N) o[(int64_t)i * epi.part_ld] = acc[i];
        } else if (epi.mode == TC_EPI_STORE) {
          float* __restrict__ o = epi.out + (int64_t)jc * epi.ldo + r;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (jc + i < N) o[(int64_t)i * epi.ldo] = alpha * acc[i];
        } else if (epi.mode == TC_EPI_ACCUM) {
          float* __restrict__ o = epi.out + (int64_t)jc * epi.ldo + r;
          float wv[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) wv[i] = (jc + i < N) ? o[(int64_t)i * epi.ldo] : 0.f;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (jc + i < N) o[(int64_t)i * epi.ldo] = wv[i] + alpha * acc[i];
        } else {
          float* __restrict__ o = epi.out + (int64_t)jc * epi.ldo + r;
          const float* __restrict__ yk = epi.yk + (int64_t)jc * epi.ldyk + r;
          const float* __restrict__ ym = epi.ykm1 ? epi.ykm1 + (int64_t)jc * epi.ldykm1 + r : nullptr;
          // issue all loads of the 16 columns before using any of them
          float wv[16], y1[16], y2[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const bool v = (jc + i) < N;
            wv[i] = v ? o[(int64_t)i * epi.ldo] : 0.f;
            y1[i] = v ? yk[(int64_t)i * epi.ldyk] : 0.f;
            y2[i] = (v && ym) ? ym[(int64_t)i * epi.ldykm1] : 0.f;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (jc + i < N) {
              const float y = alpha * (wv[i] + acc[i] - shift * y1[i]) - epi.beta * y2[i];
              o[(int64_t)i * epi.ldo] = y;
              if (epi.out_pieces > 0) split_store(epi, r, jc + i, y);
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sfree[sb]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * BN));
  }
}

// sum of split-K partials into a complex64 column-major block (real view) with ld
__global__ void k_reduce_partials(const float* __restrict__ part, int nsplit, int64_t split_stride, int64_t part_ld,
                                  int M, int N, float* __restrict__ out, int64_t ldo) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  const int r = (int)(idx % M), j = (int)(idx / M);
  float s = 0.f;
  for (int z = 0; z < nsplit; ++z) s += part[z * split_stride + (int64_t)j * part_ld + r];
  out[(int64_t)j * ldo + r] = s;
}

// float real view (rows x cols, ld) -> bf16 pieces [pieces][cols][pitch], zero-padded to pitch
__global__ void k_split_f32(const float* __restrict__ x, int64_t ldx, int rows, int cols, int pieces,
                            __nv_bfloat16* __restrict__ out, int64_t pitch, int64_t piece_stride) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)pitch * cols) return;
  const int r = (int)(idx % pitch), j = (int)(idx / pitch);
  float rem = (r < rows) ? x[(int64_t)j * ldx + r] : 0.f;
  for (int p = 0; p < pieces; ++p) {
    const __nv_bfloat16 h = __float2bfloat16_rn(rem);
    out[(int64_t)p * piece_stride + (int64_t)j * pitch + r] = h;
    rem -= __bfloat162float(h);
  }
}

// FP64 complex P (npw x np, ld npw) -> bf16 pieces of A1 [pieces][2np][pitch1] and A2 [pieces][2npw][pitch2]
__global__ void k_build_a1(const double2* __restrict__ P, int npw, int np, int pieces, __nv_bfloat16* __restrict__ A1,
                           int64_t pitch, int64_t piece_stride) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)2 * np * pitch) return;
  const int64_t k = idx % pitch;
  const int row = (int)(idx / pitch);
  const int i = row >> 1, odd = row & 1;
  double v = 0.0;
  if (k < 2 * (int64_t)npw) {
    const double2 p = P[(int64_t)i * npw + (k >> 1)];
    // row 2i: (Pr, Pi) ; row 2i+1: (-Pi, Pr)
    v = odd ? ((k & 1) ? p.x : -p.y) : ((k & 1) ? p.y : p.x);
  }
  double rem = v;
  for (int q = 0; q < pieces; ++q) {
    const __nv_bfloat16 h = __double2bfloat16(rem);
    A1[(int64_t)q * piece_stride + (int64_t)row * pitch + k] = h;
    rem -= (double)__bfloat162float(h);
  }
}
__global__ void k_build_a2(const double2* __restrict__ P, int npw, int np, int pieces, __nv_bfloat16* __restrict__ A2,
                           int64_t pitch, int64_t piece_stride) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)2 * npw * pitch) return;
  const int64_t k = idx % pitch;
  const int64_t row = idx / pitch;
  const int64_t g = row >> 1;
  const int odd = (int)(row & 1);
  double v = 0.0;
  if (k < 2 * (int64_t)np) {
    const double2 p = P[(k >> 1) * npw + g];
    // row 2g: (Pr, -Pi) ; row 2g+1: (Pi, Pr)
    v = odd ? ((k & 1) ? p.x : p.y) : ((k & 1) ? -p.y : p.x);
  }
  double rem = v;
  for (int q = 0; q < pieces; ++q) {
    const __nv_bfloat16 h = __double2bfloat16(rem);
    A2[(int64_t)q * piece_stride + row * pitch + k] = h;
    rem -= (double)__bfloat162float(h);
  }
}

// ---- host side -----------------------------------------------------------------
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}

// 3-D map over [pieces][rows][pitch] bf16, box 64 x 128 x 1, 128B swizzle, zero fill out of range
static bool make_map(CUtensorMap* m, const __nv_bfloat16* ptr, int64_t kext, int64_t rows, int64_t pitch,
                     int pieces, int64_t piece_stride) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kext, (cuuint64_t)rows, (cuuint64_t)pieces};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * 2), (cuuint64_t)(piece_stride * 2)};
  cuuint32_t box[3] = {BK, 128, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)ptr, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool available() { return encode_fn() != nullptr; }

cudaError_t gemm(const Operand& A, const Operand& B, int M, int N, int K, int pieces, int nsplit, const TcEpi& epi,
                 int* err, cudaStream_t st, int test_no_copies) {
  const uint32_t spin = test_no_copies ? kSpinTest : kSpinLimit;
  // K slices summed in TMEM between promotions to the FP32 running sum.  One: with four
  // slices per promotion in the back-projection (2 pieces) the filter's eigenvalue error
  // against FP64 grew from 2.7e-7 to 6.8e-7 Ha on the 96^3 workload for 2.5% of speed.
  const int kprom = 1;
  if (M <= 0 || N <= 0) return cudaSuccess;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A.ptr, K, A.rows, A.pitch, pieces, A.piece_stride)) return cudaErrorInvalidValue;
  if (!make_map(&mb, B.ptr, K, B.rows, B.pitch, pieces, B.piece_stride)) return cudaErrorInvalidValue;
  if (nsplit < 1) nsplit = 1;
  int kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  if (kchunk < BK) kchunk = BK;
  nsplit = (K + kchunk - 1) / kchunk;
  if (nsplit < 1) nsplit = 1;
  const int units = ((N + BN - 1) / BN) * ((M + BM - 1) / BM) * nsplit;
  int nsm = 148;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  const int grid = std::min(units, nsm);
  cudaError_t e;
  if (pieces == 2) {
    if ((e = cudaFuncSetAttribute(k_tc_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<2>::SMEM))) return e;
    k_tc_gemm<2><<<grid, 320, Cfg<2>::SMEM, st>>>(ma, mb, M, N, K, kchunk, nsplit, kprom, epi, err, spin,
                                                   test_no_copies); count_launch();
  } else {
    if ((e = cudaFuncSetAttribute(k_tc_gemm<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<3>::SMEM))) return e;
    k_tc_gemm<3><<<grid, 320, Cfg<3>::SMEM, st>>>(ma, mb, M, N, K, kchunk, nsplit, kprom, epi, err, spin,
                                                   test_no_copies); count_launch();
  }
  return cudaGetLastError();
}

int split_count(int K, int nsplit) {
  int kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  if (kchunk < BK) kchunk = BK;
  const int n = (K + kchunk - 1) / kchunk;
  return n < 1 ? 1 : n;
}

cudaError_t reduce_partials(const float* part, int nsplit, int64_t split_stride, int64_t part_ld, int M, int N,
                            float* out, int64_t ldo, cudaStream_t st) {
  const int64_t t = (int64_t)M * N;
  if (t <= 0) return cudaSuccess;
  k_reduce_partials<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(part, nsplit, split_stride, part_ld, M, N, out, ldo); count_launch();
  return cudaGetLastError();
}

cudaError_t split_f32(const float* x, int64_t ldx, int rows, int cols, int pieces, __nv_bfloat16* out, int64_t pitch,
                      int64_t piece_stride, cudaStream_t st) {
  const int64_t t = pitch * cols;
  if (t <= 0) return cudaSuccess;
  k_split_f32<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(x, ldx, rows, cols, pieces, out, pitch, piece_stride); count_launch();
  return cudaGetLastError();
}

cudaError_t build_a(const double2* P, int npw, int np, int pieces, __nv_bfloat16* A1, int64_t pitch1, int64_t ps1,
                    __nv_bfloat16* A2, int64_t pitch2, int64_t ps2, cudaStream_t st) {
  int64_t t = (int64_t)2 * np * pitch1;
  k_build_a1<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(P, npw, np, pieces, A1, pitch1, ps1); count_launch();
  t = (int64_t)2 * npw * pitch2;
  k_build_a2<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(P, npw, np, pieces, A2, pitch2, ps2); count_launch();
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace pw
