// FP64-accurate complex GEMM on the bf16 tensor cores (tcgen05 + TMA) by exact digit slicing.
//
// GB300's FP64 pipe is ~1.2 TFLOP/s, so the FP64 contractions of the method (the projector
// products of the FP64 H-apply and filter, Sec. 4.2; the Rayleigh-Ritz Grams and rotations,
// Alg. 5) would be DFMA-bound.  Here each row of op(A) and each column of op(B) is scaled by a
// power of two so that its largest entry lies in [1/4, 1/2), and every scaled entry is cut into
// seven balanced 7-bit integer digits, a = sum_s d_s 2^(-7 (s + 1)), |d_s| <= 64 (exact: 49
// bits, the remainder below 2^-50 of the row maximum).  A digit is an integer of magnitude
// <= 64 and so exactly a bf16; a product of two digits is an integer <= 2^12 and exact in the
// tensor core's FP32 accumulation.  The 28 digit products with s + t <= 6 are accumulated per
// anti-diagonal d = s + t in seven TMEM accumulators: a diagonal holds at most 7 products per
// K element, so over a K chunk of 256 its sum stays below 7 * 256 * 2^12 < 2^23 and every
// partial sum is an exact integer.  After each chunk the seven integers are combined exactly in
// 64-bit integer arithmetic, v = sum_d acc_d 2^(7 (6 - d)) < 2^62.1, and v is added to an FP64
// running sum; the result is 2^(e_row + e_col - 56) times that sum.  The dropped products
// (s + t >= 7) are below 2^-44 of |a_max| |b_max| per K element, the FP64 rounding of v and of
// the running sum are ordinary FP64 roundings.
//
// Complex operands are realified: op(A) (M x K) becomes the 2M x 2K real matrix whose rows 2i
// and 2i+1 are (Re a, -Im a) and (Im a, Re a) per entry, op(B) (K x N) the N x 2K matrix of
// interleaved (Re b, Im b) along K, so that row 2i (2i+1) of the product is Re (Im) of row i of
// the complex product: the output is the column-major complex block viewed as doubles.
//
// Kernel: persistent, one 128 (realified rows) x 64 (columns) output tile per work unit.
// Warp 0 lane 0 issues TMA loads of all seven digit planes of a 32-wide K slice of both
// operands (64-byte swizzle) into a two-stage ring; warp 1 lane 0 issues the 56 tcgen05.mma
// (28 digit pairs x 2 K steps of 16) per slice; warps 2-17 drain the seven accumulators once
// per 256-wide K chunk (one TMEM lane = one output row per thread, 16 columns per warp).
// Every mbarrier wait is bounded; on expiry the kernel records the stage, waits (bounded) for
// the copies and MMAs it has issued, releases TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "pw_internal.cuh"
#include "tc_ptx.cuh"
#include "zgemm.cuh"

namespace pw {
namespace oz {
using namespace tcp;

constexpr int S = kDigits;
constexpr int BM = 128, BN = 64, BK = 32;
constexpr int KC = 256;                      // K elements per exact chunk
constexpr int SLICES_PER_CHUNK = KC / BK;    // 8
constexpr int STAGES = 2;
constexpr int A_TILE = BM * BK * 2;          // 8 KB per digit plane
constexpr int B_TILE = BN * BK * 2;          // 4 KB per digit plane
constexpr int STAGE_BYTES = S * (A_TILE + B_TILE);
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int EPI_WARPS = 16;                // 4 per TMEM lane quarter, 16 columns each
constexpr int THREADS = 32 * (2 + EPI_WARPS);
constexpr uint32_t kTmemCols = 512;          // 7 accumulators x 64 columns = 448 used
constexpr uint32_t kIdesc = idesc_bf16(BM, BN);
constexpr uint32_t kSpin = 1u << 24;
constexpr uint32_t kSpinTest = 1u << 12;

int64_t digit_pitch(int k2) { return ((int64_t)k2 + 7) / 8 * 8; }
size_t digit_bytes(int rows, int k2) { return sizeof(__nv_bfloat16) * (size_t)S * rows * digit_pitch(k2); }

// ---------------------------------------------------------------------------------------------
// slicing
// ---------------------------------------------------------------------------------------------
// 32 x 32 complex tile of op(X) staged through shared memory so that global reads are coalesced
// along whichever index of X is contiguous, and digits are written along K.
__device__ __forceinline__ void load_tile(const double2* __restrict__ X, int64_t sr, int64_t sl, int cj, int R,
                                          int K, int r0, int l0, double2 (*sm)[33]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool kc = (sl == 1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = ty + 8 * i;
    const int rr = kc ? a : tx, ll = kc ? tx : a;
    const int r = r0 + rr, l = l0 + ll;
    double2 v = make_double2(0.0, 0.0);
    if (r < R && l < K) {
      v = X[(int64_t)r * sr + (int64_t)l * sl];
      if (cj) v.y = -v.y;
    }
    sm[rr][ll] = v;
  }
}

__global__ void __launch_bounds__(256) k_oz_rowmax(const double2* __restrict__ X, int64_t sr, int64_t sl, int cj,
                                                   int R, int K, unsigned long long* __restrict__ amax) {
  __shared__ double2 sm[32][33];
  const int r0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  load_tile(X, sr, sl, cj, R, K, r0, l0, sm);
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = ty + 8 * i;
    const double2 v = sm[rr][tx];
    double m = fmax(fabs(v.x), fabs(v.y));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tx == 0 && r0 + rr < R && m > 0.0) atomicMax(&amax[r0 + rr], (unsigned long long)__double_as_longlong(m));
  }
}

// exponent e with max |entry| 2^-e in [1/4, 1/2): e = ilogb(max) + 2 (0 for a zero row)
__device__ __forceinline__ int row_exp(unsigned long long bits) {
  if (bits == 0ull) return 0;
  return ilogb(__longlong_as_double((long long)bits)) + 2;
}

// N = round(x 2^(49 - e)) as an integer (|N| <= 2^48 since |x| < 2^(e - 1)), by integer
// arithmetic on the FP64 representation (round half away from zero)
__device__ __forceinline__ long long scaled_int(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int bexp = (int)((bits >> 52) & 0x7ff);
  long long m = bits & 0xFFFFFFFFFFFFFll;
  int E;
  if (bexp == 0) {
    E = -1074;
  } else {
    m |= 0x10000000000000ll;
    E = bexp - 1075;
  }
  const int sh = E + 49 - e;
  long long n;
  if (m == 0) n = 0;
  else if (sh >= 0) n = m << sh;
  else if (sh < -62) n = 0;
  else n = (m + (1ll << (-sh - 1))) >> (-sh);
  return bits < 0 ? -n : n;
}

// balanced base-128 digits of n (|n| <= 2^48): n = sum_s d_s 128^(6 - s); the six lower digits
// are taken in [-64, 63] and the leading digit is what remains, which is within [-64, 64]
__device__ __forceinline__ void digits7(long long n, float (&d)[S]) {
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const long long q = (n + 64) >> 7;  // floor((n + 64) / 128)
    d[s] = (float)(n - q * 128);
    n = q;
  }
  d[0] = (float)n;
}

__global__ void __launch_bounds__(256) k_oz_slice(const double2* __restrict__ X, int64_t sr, int64_t sl, int cj,
                                                  int R, int K, int aform, __nv_bfloat16* __restrict__ dig,
                                                  int64_t pitch, int64_t plane,
                                                  const unsigned long long* __restrict__ amax, int* __restrict__ ex) {
  __shared__ double2 sm[32][33];
  const int r0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  load_tile(X, sr, sl, cj, R, K, r0, l0, sm);
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll 1
  for (int i = 0; i < 4; ++i) {
    const int rr = ty + 8 * i, r = r0 + rr, l = l0 + tx;
    if (r >= R || l >= K) continue;
    const int e = row_exp(amax[r]);
    if (blockIdx.y == 0 && tx == 0) ex[r] = e;
    const double2 v = sm[rr][tx];
    float dr[S], di[S];
    digits7(scaled_int(v.x, e), dr);
    digits7(scaled_int(v.y, e), di);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      __nv_bfloat16* p = dig + (int64_t)s * plane + 2 * (int64_t)l;
      if (aform) {
        *reinterpret_cast<__nv_bfloat162*>(p + (int64_t)(2 * r) * pitch) = __floats2bfloat162_rn(dr[s], -di[s]);
        *reinterpret_cast<__nv_bfloat162*>(p + (int64_t)(2 * r + 1) * pitch) = __floats2bfloat162_rn(di[s], dr[s]);
      } else {
        *reinterpret_cast<__nv_bfloat162*>(p + (int64_t)r * pitch) = __floats2bfloat162_rn(dr[s], di[s]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// GEMM
// ---------------------------------------------------------------------------------------------
struct Args {
  int M2, N, k2, kchunk, nsplit, ntm, ntn, nunits, lower, nlow;
  const int* ea;  // per complex row of op(A)
  const int* eb;  // per column of op(B)
  Epi<double> epi;
  double* part;   // [z][N][M2]
  int* err;
  uint32_t spin;
  int no_copies;
};

__device__ __forceinline__ void unit_of(const Args& a, int u, int& z, int& tm, int& tn) {
  if (a.lower) {
    z = u / a.nlow;
    const int l = u % a.nlow;
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= l) ++r;
    tm = r;
    tn = l - r * (r + 1) / 2;
  } else {
    tn = u % a.ntn;
    tm = (u / a.ntn) % a.ntm;
    z = u / (a.ntn * a.ntm);
  }
}

// epilogue on the realified view: element (R, j) of the output is double R of complex column j
__device__ __forceinline__ void oz_epi(const Epi<double>& e, int R, int j, double v) {
  double* o = reinterpret_cast<double*>(e.out) + (int64_t)j * 2 * e.ldo + R;
  switch (e.mode) {
    case EPI_STORE: *o = e.alpha * v; break;
    case EPI_ACCUM: *o = *o + e.alpha * v; break;
    case EPI_CHEB: {
      double alpha = e.alpha, shift = e.shift;
      if (e.dev_ce) {
        shift = e.dev_ce[0];
        alpha = (e.first ? 1.0 : 2.0) / e.dev_ce[1];
      }
      const double yk = reinterpret_cast<const double*>(e.yk)[(int64_t)j * 2 * e.ldy + R];
      double r = alpha * (*o + v - shift * yk);
      if (e.ykm1) r -= e.beta * reinterpret_cast<const double*>(e.ykm1)[(int64_t)j * 2 * e.ldy2 + R];
      *o = r;
    } break;
    default: break;
  }
}

__global__ void __launch_bounds__(THREADS, 1) k_oz_gemm(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmB, Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(base + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 1;
  uint64_t* mdone = tempty + 1;
  uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(tfull, 1);
    mbar_init(tempty, EPI_WARPS);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int g = 0;
      int last_it[STAGES];
      for (int s = 0; s < STAGES; ++s) last_it[s] = -1;
      for (int u = blockIdx.x; u < a.nunits && !*abort_flag; u += gridDim.x) {
        int z, tm, tn;
        unit_of(a, u, z, tm, tn);
        const int kb0 = z * a.kchunk, kb1 = min(a.k2, kb0 + a.kchunk);
        const int nsl = (kb1 - kb0 + BK - 1) / BK;
        for (int kb = 0; kb < nsl; ++kb, ++g) {
          const int s = g % STAGES, it = g / STAGES;
          if (it > 0 && !mbar_wait(&empty[s], (it - 1) & 1, a.spin)) {
            atomicExch(a.err, 1);
            *abort_flag = 1;
            break;
          }
          if (!a.no_copies) {
            mbar_expect_tx(&full[s], STAGE_BYTES);
            const uint32_t sb = smem_u32(base + s * STAGE_BYTES);
            const int k = kb0 + kb * BK;
            tma_load_3d(sb, &tmA, k, tm * BM, 0, &full[s]);
            tma_load_3d(sb + S * A_TILE, &tmB, k, tn * BN, 0, &full[s]);
            last_it[s] = it;
          }
        }
      }
      // every copy this thread issued has landed before the CTA may exit
      for (int s = 0; s < STAGES; ++s)
        if (last_it[s] >= 0 && !mbar_wait(&full[s], last_it[s] & 1, a.spin)) atomicExch(a.err, 4);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      int g = 0, c = 0;
      for (int u = blockIdx.x; u < a.nunits && !*abort_flag; u += gridDim.x) {
        int z, tm, tn;
        unit_of(a, u, z, tm, tn);
        const int kb0 = z * a.kchunk, kb1 = min(a.k2, kb0 + a.kchunk);
        const int nsl = (kb1 - kb0 + BK - 1) / BK;
        bool stop = false;
        for (int kb = 0; kb < nsl; ++kb, ++g) {
          const int s = g % STAGES, it = g / STAGES;
          const bool cfirst = (kb % SLICES_PER_CHUNK) == 0;
          const bool clast = (kb % SLICES_PER_CHUNK) == SLICES_PER_CHUNK - 1 || kb + 1 == nsl;
          if ((cfirst && c > 0 && !mbar_wait(tempty, (c - 1) & 1, a.spin)) || !mbar_wait(&full[s], it & 1, a.spin)) {
            atomicExch(a.err, 2);
            *abort_flag = 1;
            stop = true;
            break;
          }
          fence_after();
          // descriptors advance by (byte offset >> 4) in their start-address field
          const uint64_t ad0 = sdesc_k(smem_u32(base + s * STAGE_BYTES), 512, 4);
          const uint64_t bd0 = ad0 + (uint64_t)((S * A_TILE) >> 4);
#pragma unroll 1
          for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
            for (int d = 0; d < S; ++d) {
#pragma unroll
              for (int p = 0; p <= d; ++p) {
                const uint64_t ad = ad0 + (uint64_t)((p * A_TILE + kk * 32) >> 4);
                const uint64_t bd = bd0 + (uint64_t)(((d - p) * B_TILE + kk * 32) >> 4);
                mma_bf16_id(tmem + (uint32_t)(d * BN), ad, bd, kIdesc, (cfirst && kk == 0 && p == 0) ? 0u : 1u);
              }
            }
          }
          mma_commit(&empty[s]);
          if (clast) {
            mma_commit(tfull);
            ++c;
          }
        }
        if (stop) break;
      }
      // every MMA this thread issued has completed before TMEM is released
      mma_commit(mdone);
      if (!mbar_wait(mdone, 0, a.spin)) atomicExch(a.err, 5);
    }
  } else {
    // ---- epilogue warps 2..17: TMEM lane quarter warp % 4, 16-column group (warp - 2) / 4
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 16);
    int c = 0;
    for (int u = blockIdx.x; u < a.nunits && !*abort_flag; u += gridDim.x) {
      int z, tm, tn;
      unit_of(a, u, z, tm, tn);
      const int kb0 = z * a.kchunk, kb1 = min(a.k2, kb0 + a.kchunk);
      const int nsl = (kb1 - kb0 + BK - 1) / BK;
      const int nch = (nsl + SLICES_PER_CHUNK - 1) / SLICES_PER_CHUNK;
      double sum[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) sum[i] = 0.0;
      bool ok = true;
      for (int ch = 0; ch < nch; ++ch, ++c) {
        if (!mbar_wait(tfull, c & 1, a.spin)) {
          atomicExch(a.err, 3);
          *abort_flag = 1;
          ok = false;
          break;
        }
        fence_after();
        long long v[16];
#pragma unroll
        for (int d = 0; d < S; ++d) {
          uint32_t r[16];
          tmem_ld16_async(tl + (uint32_t)(d * BN), r);
          tmem_wait_ld16(r);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const long long x = (long long)__float2int_rn(__uint_as_float(r[i]));
            v[i] = d ? v[i] * 128 + x : x;
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty);
#pragma unroll
        for (int i = 0; i < 16; ++i) sum[i] += __ll2double_rn(v[i]);
      }
      if (!ok) break;
      const int R = tm * BM + q * 32 + lane;
      if (R < a.M2) {
        const int er = a.ea[R >> 1] - 56;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = tn * BN + h * 16 + i;
          if (j < a.N) {
            const double val = ldexp(sum[i], er + a.eb[j]);
            if (a.nsplit > 1) a.part[((int64_t)z * a.N + j) * a.M2 + R] = val;
            else oz_epi(a.epi, R, j, val);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

__global__ void k_oz_reduce(int M2, int N, int nsplit, const double* __restrict__ part, Epi<double> epi, int lower) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M2 * N) return;
  const int R = (int)(idx % M2), j = (int)(idx / M2);
  if (lower && (R >> 1) / BN < j / BN) return;  // tile above the diagonal: not computed
  double s = 0.0;
  for (int z = 0; z < nsplit; ++z) s += part[((int64_t)z * N + j) * M2 + R];
  oz_epi(epi, R, j, s);
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
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

bool available() { return encode_fn() != nullptr; }

// 3-D map over the digit planes [S][rows][pitch], box 32 (K) x box_rows x S, 64-byte swizzle,
// zero fill beyond k2 and beyond the rows
static bool make_map(CUtensorMap* m, const Digits& d, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)d.k2, (cuuint64_t)d.rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)(d.pitch * 2), (cuuint64_t)(d.plane * 2)};
  cuuint32_t box[3] = {BK, (cuuint32_t)box_rows, S};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)d.dig, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t slice(const double2* X, int64_t sr, int64_t sl, int cj, int R, int K, int aform, __nv_bfloat16* dig,
                  int64_t pitch, int64_t plane, unsigned long long* amax, int* exp, cudaStream_t st) {
  if (R <= 0 || K <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned long long) * (size_t)R, st);
  if (e != cudaSuccess) return e;
  const dim3 grid((R + 31) / 32, (K + 31) / 32);
  k_oz_rowmax<<<grid, 256, 0, st>>>(X, sr, sl, cj, R, K, amax); count_launch();
  k_oz_slice<<<grid, 256, 0, st>>>(X, sr, sl, cj, R, K, aform, dig, pitch, plane, amax, exp); count_launch();
  return cudaGetLastError();
}

int split_count(int M2, int N, int k2, int lower) {
  int nsm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int ntm = (M2 + BM - 1) / BM, ntn = (N + BN - 1) / BN;
  const int tiles = lower ? ntm * (ntm + 1) / 2 : ntm * ntn;
  const int maxs = std::max(1, std::min(64, (k2 + 4 * KC - 1) / (4 * KC)));  // at least 4 chunks per split
  int best = 1;
  double beff = -1;
  for (int c = 1; c <= maxs; ++c) {
    const int u = tiles * c;
    const double eff = (double)u / ((double)((u + nsm - 1) / nsm) * nsm);
    if (eff > beff + 0.02) { beff = eff; best = c; }
  }
  return best;
}

cudaError_t gemm(const Digits& A, const Digits& B, int M, int N, int K, const Epi<double>& epi, int lower,
                 int nsplit, double* part, int* err, int test_no_copies, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (lower && M != N) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, BM) || !make_map(&mb, B, BN)) return cudaErrorInvalidValue;
  Args a;
  a.M2 = 2 * M;
  a.N = N;
  a.k2 = 2 * K;
  if (nsplit < 1) nsplit = 1;
  int kchunk = (a.k2 + nsplit - 1) / nsplit;
  kchunk = std::max(KC, (kchunk + KC - 1) / KC * KC);
  nsplit = (a.k2 + kchunk - 1) / kchunk;
  if (nsplit > 1 && !part) return cudaErrorInvalidValue;
  a.kchunk = kchunk;
  a.nsplit = nsplit;
  a.ntm = (a.M2 + BM - 1) / BM;
  a.ntn = (N + BN - 1) / BN;
  a.lower = lower;
  a.nlow = a.ntm * (a.ntm + 1) / 2;
  a.nunits = (lower ? a.nlow : a.ntm * a.ntn) * nsplit;
  a.ea = A.exp;
  a.eb = B.exp;
  a.epi = epi;
  a.part = part;
  a.err = err;
  a.spin = test_no_copies ? kSpinTest : kSpin;
  a.no_copies = test_no_copies;
  int nsm = 148, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(a.nunits, nsm);
  cudaError_t e = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e != cudaSuccess) return e;
  k_oz_gemm<<<grid, THREADS, SMEM, st>>>(ma, mb, a); count_launch();
  if (nsplit > 1) {
    const int64_t t = (int64_t)a.M2 * N;
    k_oz_reduce<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(a.M2, N, nsplit, part, epi, lower); count_launch();
  }
  return cudaGetLastError();
}

}  // namespace oz
}  // namespace pw
