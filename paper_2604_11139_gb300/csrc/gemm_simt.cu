// Complex GEMMs on the CUDA cores (FP64 DFMA / FP32 FFMA) for the projector
// contractions C_proj = P^dagger Psi and Psi += P (D C_proj) (Sec. 4.2), the
// Rayleigh-Ritz Grams and rotations (Alg. 5) and the small projector-space
// products.  On GB300 FP64 has no fast tensor path, so the FP64 forms are
// DFMA-bound; the kernel keeps a 64x64 complex tile per CTA with a 4x4 register
// tile per thread and stages 16-deep K slices through shared memory.
#include "pw_internal.cuh"

namespace pw {

template <typename T>
__device__ __forceinline__ void epi_apply(const Epi<T>& e, int m, int n, cplx<T> v) {
  using C = cplx<T>;
  C* o = e.out + m + (int64_t)n * e.ldo;
  switch (e.mode) {
    case EPI_STORE: *o = cscale(v, e.alpha); break;
    case EPI_ACCUM: *o = cadd(*o, cscale(v, e.alpha)); break;
    case EPI_CHEB: {
      const C w = *o;
      const C yk = e.yk[m + (int64_t)n * e.ldy];
      T alpha = e.alpha, shift = e.shift;
      if (e.dev_ce) { shift = (T)e.dev_ce[0]; alpha = (T)((e.first ? 1.0 : 2.0) / e.dev_ce[1]); }
      C r = cscale(csub(cadd(w, v), cscale(yk, shift)), alpha);
      if (e.ykm1) r = csub(r, cscale(e.ykm1[m + (int64_t)n * e.ldy2], e.beta));
      *o = r;
    } break;
    default: break;
  }
}

constexpr int BM = 64, BN = 64, BK = 16;

// row and column of the lth tile on or below the diagonal (row-major order of the lower triangle)
__device__ __forceinline__ void lower_tile(int l, int& bi, int& bj) {
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= l) ++r;
  bi = r;
  bj = l - r * (r + 1) / 2;
}

template <typename T, int TA, int TB>
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int K, const cplx<T>* __restrict__ A, int64_t lda,
                                               const cplx<T>* __restrict__ B, int64_t ldb, Epi<T> epi,
                                               int kchunk, cplx<T>* __restrict__ ws, int tri) {
  using C = cplx<T>;
  __shared__ C As[BK][BM + 1];
  __shared__ C Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int bi = blockIdx.x, bj = blockIdx.y;
  if (tri == GEMM_LOWER_OUT) lower_tile(blockIdx.x, bi, bj);
  const int m0 = bi * BM, n0 = bj * BN;
  const int kb = blockIdx.z * kchunk;
  int ke = min(K, kb + kchunk);
  if (tri == GEMM_B_UPPER) ke = min(ke, n0 + BN);  // op(B)[k][n] = 0 for k > n
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
  for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int lin = tid + 256 * e;
      int mm, kk;
      if (TA == 0) { mm = lin % BM; kk = lin / BM; } else { kk = lin % BK; mm = lin / BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      C v = czero<C>();
      if (gm < M && gk < ke) v = (TA == 0) ? A[gm + gk * lda] : cconj(A[gk + gm * lda]);
      As[kk][mm] = v;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int lin = tid + 256 * e;
      int nn, kk;
      if (TB == 0) { kk = lin % BK; nn = lin / BK; } else { nn = lin % BN; kk = lin / BN; }
      const int gn = n0 + nn, gk = k0 + kk;
      C v = czero<C>();
      if (gn < N && gk < ke) v = (TB == 0) ? B[gk + gn * ldb] : cconj(B[gn + gk * ldb]);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  if (gridDim.z > 1) {
    C* w = ws + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < M && n < N) w[m + (int64_t)n * M] = acc[i][j];
      }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < M && n < N) epi_apply<T>(epi, m, n, acc[i][j]);
      }
  }
}

template <typename T>
__global__ void k_splitk_reduce(int M, int N, int nsplit, const cplx<T>* __restrict__ ws, Epi<T> epi, int tri) {
  using C = cplx<T>;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  const int m = (int)(idx % M), n = (int)(idx / M);
  if (tri == GEMM_LOWER_OUT && m / BM < n / BN) return;  // tile above the diagonal: never computed
  C s = czero<C>();
  for (int z = 0; z < nsplit; ++z) s = cadd(s, ws[z * (int64_t)M * N + idx]);
  epi_apply<T>(epi, m, n, s);
}

// Matrix-vector forms (N <= GEMV_MAXN columns of op(B), B as stored): a 64-wide output tile would
// spend 64 / N times the arithmetic, so these read A once at memory speed instead.
constexpr int GEMV_MAXN = 4;

// out[m][j] = sum_k conj(A[k][m]) B[k][j]: one CTA per m, the K loop strided over its threads
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_cgemv_t(int M, int K, const cplx<T>* __restrict__ A, int64_t lda,
                                                 const cplx<T>* __restrict__ B, int64_t ldb, Epi<T> epi) {
  using C = cplx<T>;
  __shared__ C red[8][NB];
  const int m = blockIdx.x;
  C acc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] = czero<C>();
  const C* a = A + (int64_t)m * lda;
#pragma unroll 4
  for (int k = threadIdx.x; k < K; k += 256) {
    const C x = a[k];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const C b = B[k + (int64_t)j * ldb];
      acc[j].x = fma(x.x, b.x, acc[j].x);
      acc[j].x = fma(x.y, b.y, acc[j].x);
      acc[j].y = fma(x.x, b.y, acc[j].y);
      acc[j].y = fma(-x.y, b.x, acc[j].y);
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, o);
      acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, o);
    }
    if (lane == 0) red[w][j] = acc[j];
  }
  __syncthreads();
  if (threadIdx.x < NB) {
    const int j = threadIdx.x;
    C s = czero<C>();
    for (int q = 0; q < 8; ++q) s = cadd(s, red[q][j]);
    epi_apply<T>(epi, m, j, s);
  }
}

// out[i][j] = sum_k A[i][k] B[k][j]: one thread per row i, B's few columns broadcast; the K
// loop is unrolled so that several rows of A are in flight per thread
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_cgemv_n(int M, int K, const cplx<T>* __restrict__ A, int64_t lda,
                                                 const cplx<T>* __restrict__ B, int64_t ldb, Epi<T> epi) {
  using C = cplx<T>;
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i >= M) return;
  C acc[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j] = czero<C>();
#pragma unroll 8
  for (int k = 0; k < K; ++k) {
    const C x = A[i + (int64_t)k * lda];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const C b = B[k + (int64_t)j * ldb];
      acc[j].x = fma(x.x, b.x, acc[j].x);
      acc[j].x = fma(-x.y, b.y, acc[j].x);
      acc[j].y = fma(x.x, b.y, acc[j].y);
      acc[j].y = fma(x.y, b.x, acc[j].y);
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) epi_apply<T>(epi, i, j, acc[j]);
}

template <typename T, int NB>
static void launch_gemv(int ta, int M, int K, const cplx<T>* A, int64_t lda, const cplx<T>* B, int64_t ldb,
                        const Epi<T>& epi, cudaStream_t st) {
  if (ta == 1) k_cgemv_t<T, NB><<<M, 256, 0, st>>>(M, K, A, lda, B, ldb, epi);
  else k_cgemv_n<T, NB><<<(M + 255) / 256, 256, 0, st>>>(M, K, A, lda, B, ldb, epi);
  count_launch();
}

template <typename T>
cudaError_t launch_cgemm(int ta, int tb, int M, int N, int K, const cplx<T>* A, int64_t lda,
                         const cplx<T>* B, int64_t ldb, const Epi<T>& epi, int nsplit, cplx<T>* ws,
                         cudaStream_t st, int tri) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (tri == GEMM_LOWER_OUT && M != N) return cudaErrorInvalidValue;
  if (tri == GEMM_B_UPPER && N > K) return cudaErrorInvalidValue;
  if (N <= GEMV_MAXN && tb == 0 && tri == GEMM_FULL && K > 0) {
    switch (N) {
      case 1: launch_gemv<T, 1>(ta, M, K, A, lda, B, ldb, epi, st); break;
      case 2: launch_gemv<T, 2>(ta, M, K, A, lda, B, ldb, epi, st); break;
      case 3: launch_gemv<T, 3>(ta, M, K, A, lda, B, ldb, epi, st); break;
      default: launch_gemv<T, 4>(ta, M, K, A, lda, B, ldb, epi, st); break;
    }
    return cudaGetLastError();
  }
  if (K <= 0) nsplit = 1;
  if (nsplit < 1) nsplit = 1;
  int kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  if (kchunk <= 0) kchunk = BK;
  nsplit = (K + kchunk - 1) / kchunk;
  if (nsplit < 1) nsplit = 1;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  dim3 grid(tm, tn, nsplit);
  if (tri == GEMM_LOWER_OUT) grid = dim3(tm * (tm + 1) / 2, 1, nsplit);
  if (ta == 0 && tb == 0) k_cgemm<T, 0, 0><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, epi, kchunk, ws, tri);
  else if (ta == 1 && tb == 0) k_cgemm<T, 1, 0><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, epi, kchunk, ws, tri);
  else if (ta == 0 && tb == 1) k_cgemm<T, 0, 1><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, epi, kchunk, ws, tri);
  else k_cgemm<T, 1, 1><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, epi, kchunk, ws, tri);
  count_launch();
  if (nsplit > 1) {
    const int64_t tot = (int64_t)M * N;
    k_splitk_reduce<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, nsplit, ws, epi, tri); count_launch();
  }
  return cudaGetLastError();
}

// Z = D C with D real (nproj x nproj, column-major) applied block by block
template <typename T>
__global__ void k_dblock(int nproj, int nband, const T* __restrict__ D, const int* __restrict__ blk0,
                         const int* __restrict__ blklen, const cplx<T>* __restrict__ Cm, int64_t ldc,
                         cplx<T>* __restrict__ Z, int64_t ldz) {
  using C = cplx<T>;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nproj * nband) return;
  const int p = (int)(idx % nproj), j = (int)(idx / nproj);
  const int q0 = blk0[p], nq = blklen[p];
  C s = czero<C>();
  for (int q = q0; q < q0 + nq; ++q) {
    const T d = D[p + (int64_t)q * nproj];
    const C c = Cm[q + (int64_t)j * ldc];
    s.x = fma(d, c.x, s.x);
    s.y = fma(d, c.y, s.y);
  }
  Z[p + (int64_t)j * ldz] = s;
}

template <typename T>
cudaError_t launch_dblock(int nproj, int nband, const T* D, const int* blk0, const int* blklen,
                          const cplx<T>* Cm, int64_t ldc, cplx<T>* Z, int64_t ldz, cudaStream_t st) {
  const int64_t tot = (int64_t)nproj * nband;
  if (tot <= 0) return cudaSuccess;
  k_dblock<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nproj, nband, D, blk0, blklen, Cm, ldc, Z, ldz); count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_cgemm<double>(int, int, int, int, int, const double2*, int64_t, const double2*,
                                          int64_t, const Epi<double>&, int, double2*, cudaStream_t, int);
template cudaError_t launch_cgemm<float>(int, int, int, int, int, const float2*, int64_t, const float2*,
                                         int64_t, const Epi<float>&, int, float2*, cudaStream_t, int);
template cudaError_t launch_dblock<double>(int, int, const double*, const int*, const int*, const double2*,
                                           int64_t, double2*, int64_t, cudaStream_t);
template cudaError_t launch_dblock<float>(int, int, const float*, const int*, const int*, const float2*,
                                          int64_t, float2*, int64_t, cudaStream_t);

}  // namespace pw
