// FP64 dense linear algebra of the subspace step, all on the GPU (Alg. 5, Alg. 9):
// Hermitian symmetrisation, blocked Cholesky (potrf), triangular inverse
// (the trsm of S-Ortho done as an explicit inverse and a GEMM), a parallel
// cyclic Jacobi eigensolver for the reduced Hermitian matrix (the hegvd step,
// after Cholesky reduction), eigenpair sorting, column reductions (Rayleigh
// quotients, residual norms) and the Lanczos helpers of the spectrum bound.
#include <math.h>

#include <algorithm>

#include "pw_internal.cuh"
#include "la.cuh"

namespace pw {

// ---- symmetrisation ---------------------------------------------------------------
__global__ void k_herm_sym(double2* A, int64_t lda, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n || i < j) return;
  if (i == j) { A[i + i * lda].y = 0.0; return; }
  const double2 a = A[i + j * lda], b = A[j + i * lda];
  const double2 m = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  A[i + j * lda] = m;
  A[j + i * lda] = cconj(m);
}

cudaError_t la_herm_sym(double2* A, int64_t lda, int n, cudaStream_t st) {
  dim3 b(16, 16), g((n + 15) / 16, (n + 15) / 16);
  k_herm_sym<<<g, b, 0, st>>>(A, lda, n); count_launch();
  return cudaGetLastError();
}

// upper triangle from the lower one (a Gram matrix of which only the lower tiles were computed)
__global__ void k_herm_from_lower(double2* A, int64_t lda, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n || i < j) return;
  if (i == j) { A[i + i * lda].y = 0.0; return; }
  A[j + i * lda] = cconj(A[i + j * lda]);
}

cudaError_t la_herm_from_lower(double2* A, int64_t lda, int n, cudaStream_t st) {
  dim3 b(16, 16), g((n + 15) / 16, (n + 15) / 16);
  k_herm_from_lower<<<g, b, 0, st>>>(A, lda, n); count_launch();
  return cudaGetLastError();
}

// ---- blocked Cholesky A = L L^dagger (lower, in place; strict upper part zeroed) ---
constexpr int NB = 32;

__global__ void k_chol_diag(double2* A, int64_t lda, int k0, int kb, int* flag) {
  __shared__ double2 S[NB][NB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 32
  if (tx < kb && ty < kb) S[ty][tx] = A[(k0 + ty) + (int64_t)(k0 + tx) * lda];  // S[row][col]
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tx == 0 && ty == 0) {
      double d = S[j][j].x;
      if (!(d > 0.0) || !isfinite(d)) { atomicExch(flag, 1); d = 1.0; }
      S[j][j] = make_double2(sqrt(d), 0.0);
    }
    __syncthreads();
    const double dj = S[j][j].x;
    if (tx == 0 && ty > j && ty < kb) S[ty][j] = cscale(S[ty][j], 1.0 / dj);
    __syncthreads();
    // trailing: S[i][k] -= S[i][j] conj(S[k][j]) for j < k <= i
    if (ty > j && ty < kb && tx > j && tx <= ty) S[ty][tx] = csub(S[ty][tx], cmul(S[ty][j], cconj(S[tx][j])));
    __syncthreads();
  }
  if (tx < kb && ty < kb) {
    const double2 v = (tx <= ty) ? S[ty][tx] : make_double2(0.0, 0.0);
    A[(k0 + ty) + (int64_t)(k0 + tx) * lda] = v;
  }
}

// rows i >= k0+kb: L21[i,:] = A21[i,:] L11^{-dagger}
__global__ void k_chol_panel(double2* A, int64_t lda, int n, int k0, int kb) {
  __shared__ double2 Ls[NB][NB + 1];
  const int t = threadIdx.x;
  for (int e = t; e < kb * kb; e += blockDim.x) {
    const int r = e % kb, c = e / kb;
    Ls[r][c] = A[(k0 + r) + (int64_t)(k0 + c) * lda];
  }
  __syncthreads();
  const int i = k0 + kb + blockIdx.x * blockDim.x + t;
  if (i >= n) return;
  double2 x[NB];
  for (int j = 0; j < kb; ++j) {
    double2 s = A[i + (int64_t)(k0 + j) * lda];
    for (int tt = 0; tt < j; ++tt) s = csub(s, cmul(x[tt], cconj(Ls[j][tt])));
    x[j] = cscale(s, 1.0 / Ls[j][j].x);
  }
  for (int j = 0; j < kb; ++j) A[i + (int64_t)(k0 + j) * lda] = x[j];
}

// trailing update of the lower triangle: A[i][j] -= sum_t L[i][t] conj(L[j][t])
__global__ void k_chol_update(double2* A, int64_t lda, int n, int k0, int kb) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bj > bi) return;
  __shared__ double2 Li[32][NB + 1], Lj[32][NB + 1];
  const int s0 = k0 + kb;
  const int i0 = s0 + bi * 32, j0 = s0 + bj * 32;
  const int t = threadIdx.x;  // 256
  for (int e = t; e < 32 * kb; e += 256) {
    const int r = e % 32, c = e / 32;
    Li[r][c] = (i0 + r < n) ? A[(i0 + r) + (int64_t)(k0 + c) * lda] : make_double2(0, 0);
    Lj[r][c] = (j0 + r < n) ? A[(j0 + r) + (int64_t)(k0 + c) * lda] : make_double2(0, 0);
  }
  __syncthreads();
  for (int e = t; e < 32 * 32; e += 256) {
    const int r = e % 32, c = e / 32;
    const int i = i0 + r, j = j0 + c;
    if (i >= n || j >= n || j > i) continue;
    double2 s = make_double2(0, 0);
    for (int tt = 0; tt < kb; ++tt) {
      const double2 a = Li[r][tt], b = Lj[c][tt];
      s.x += a.x * b.x + a.y * b.y;
      s.y += a.y * b.x - a.x * b.y;
    }
    A[i + (int64_t)j * lda] = csub(A[i + (int64_t)j * lda], s);
  }
}

__global__ void k_zero_upper(double2* A, int64_t lda, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < n && j < n && j > i) A[i + (int64_t)j * lda] = make_double2(0, 0);
}

cudaError_t la_zero_upper(double2* A, int64_t lda, int n, cudaStream_t st) {
  dim3 b(16, 16), g((n + 15) / 16, (n + 15) / 16);
  k_zero_upper<<<g, b, 0, st>>>(A, lda, n); count_launch();
  return cudaGetLastError();
}

cudaError_t la_cholesky(double2* A, int64_t lda, int n, int* flag, cudaStream_t st) {
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    k_chol_diag<<<1, dim3(32, 32), 0, st>>>(A, lda, k0, kb, flag); count_launch();
    const int rest = n - k0 - kb;
    if (rest > 0) {
      k_chol_panel<<<(rest + 127) / 128, 128, 0, st>>>(A, lda, n, k0, kb); count_launch();
      const int nt = (rest + 31) / 32;
      k_chol_update<<<dim3(nt, nt), 256, 0, st>>>(A, lda, n, k0, kb); count_launch();
    }
  }
  // zero the strict upper triangle
  dim3 zb(16, 16), zg((n + 15) / 16, (n + 15) / 16);
  k_zero_upper<<<zg, zb, 0, st>>>(A, lda, n); count_launch();
  return cudaGetLastError();
}

// ---- triangular inverse X = L^{-1} (lower) -------------------------------------------
__global__ void k_transpose(const double2* A, int64_t lda, int n, double2* At) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < n && j < n) At[j + (int64_t)i * n] = A[i + (int64_t)j * lda];
}

// one warp per column j of X; Lt holds L row-major (Lt[t + i n] = L[i][t])
__global__ void k_trinv(const double2* __restrict__ Lt, int n, double2* __restrict__ X, int64_t ldx) {
  extern __shared__ double2 xs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= n) return;
  double2* x = xs + (int64_t)warp * n;
  for (int i = lane; i < j; i += 32) X[i + (int64_t)j * ldx] = make_double2(0, 0);
  if (lane == 0) {
    const double d = Lt[j + (int64_t)j * n].x;
    x[j] = make_double2(1.0 / d, 0.0);
    X[j + (int64_t)j * ldx] = x[j];
  }
  __syncwarp();
  for (int i = j + 1; i < n; ++i) {
    const double2* row = Lt + (int64_t)i * n;
    double sr = 0, si = 0;
    for (int t = j + lane; t < i; t += 32) {
      const double2 a = row[t], b = x[t];
      sr += a.x * b.x - a.y * b.y;
      si += a.x * b.y + a.y * b.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      const double d = row[i].x;
      x[i] = make_double2(-sr / d, -si / d);
      X[i + (int64_t)j * ldx] = x[i];
    }
    __syncwarp();
  }
}

cudaError_t la_trinv_lower(const double2* L, int64_t lda, int n, double2* X, int64_t ldx, double2* tmp,
                           cudaStream_t st) {
  dim3 b(16, 16), g((n + 15) / 16, (n + 15) / 16);
  k_transpose<<<g, b, 0, st>>>(L, lda, n, tmp); count_launch();
  const int wpb = 4;
  const size_t sm = sizeof(double2) * (size_t)n * wpb;
  cudaError_t e = cudaFuncSetAttribute(k_trinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  k_trinv<<<(n + wpb - 1) / wpb, 32 * wpb, sm, st>>>(tmp, n, X, ldx); count_launch();
  return cudaGetLastError();
}

// ---- parallel cyclic Jacobi for Hermitian A (n x n, lda = n) ---------------------------
// Templated on the complex type: FP64 for the eigensolve itself, FP32 for the pre-rotation of
// the mixed solver (la_jacobi_eigh32 below).
template <typename C> struct RotT {
  using R = decltype(C{}.x);
  R c, s;
  C ph;
};  // J = [[c, s], [-s ph, c ph]]

__device__ __forceinline__ void rr_pair(int t, int i, int np, int& p, int& q) {
  auto pos = [&](int s) { return s == 0 ? 0 : ((s - 1 + t) % (np - 1)) + 1; };
  p = pos(i);
  q = pos(np - 1 - i);
}

template <typename C>
__device__ __forceinline__ RotT<C> jac_rot(const C* A, int n, int p, int q) {
  using R = typename RotT<C>::R;
  RotT<C> r;
  r.c = (R)1;
  r.s = (R)0;
  r.ph.x = (R)1;
  r.ph.y = (R)0;
  if (p >= n || q >= n) return r;
  const R a = A[p + (int64_t)p * n].x, d = A[q + (int64_t)q * n].x;
  const C b = A[p + (int64_t)q * n];
  const R ab = hypot(b.x, b.y);
  if (!(ab > (R)(sizeof(R) == 8 ? 1e-300 : 1e-37))) return r;
  const R tau = (d - a) / ((R)2 * ab);
  const R t = (tau >= 0 ? (R)1 : (R)-1) / (fabs(tau) + sqrt((R)1 + tau * tau));
  r.c = (R)1 / sqrt((R)1 + t * t);
  r.s = t * r.c;
  r.ph.x = b.x / ab;
  r.ph.y = -b.y / ab;
  return r;
}

// the rotation of every pair of round t, computed once (FP64 square roots and divisions
// are the expensive part of a round).  One pair per CTA of one warp: FP64 issues at a small
// fraction of the FP32 rate, so the pairs are spread over the SMs rather than queued on one.
template <typename C>
__global__ void k_jacobi_rot(const C* __restrict__ A, int n, int np, int t, RotT<C>* __restrict__ rot) {
  const int i = blockIdx.x;
  if (i >= np / 2 || threadIdx.x != 0) return;
  int p, q;
  rr_pair(t, i, np, p, q);
  rot[i] = jac_rot(A, n, p, q);
}

template <typename C>
__global__ void k_jacobi_round(const C* __restrict__ Ao, C* __restrict__ An, const C* __restrict__ Vo,
                               C* __restrict__ Vn, int n, int np, int t, const RotT<C>* __restrict__ rot) {
  const int npair = np / 2;
  const int64_t nblk = (int64_t)npair * npair;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  C z;
  z.x = 0;
  z.y = 0;
  if (idx < nblk) {
    const int I = (int)(idx % npair), Jx = (int)(idx / npair);
    int pI, qI, pJ, qJ;
    rr_pair(t, I, np, pI, qI);
    rr_pair(t, Jx, np, pJ, qJ);
    const RotT<C> ri = rot[I], rj = rot[Jx];
    const bool vpI = pI < n, vqI = qI < n, vpJ = pJ < n, vqJ = qJ < n;
    const C b00 = (vpI && vpJ) ? Ao[pI + (int64_t)pJ * n] : z;
    const C b01 = (vpI && vqJ) ? Ao[pI + (int64_t)qJ * n] : z;
    const C b10 = (vqI && vpJ) ? Ao[qI + (int64_t)pJ * n] : z;
    const C b11 = (vqI && vqJ) ? Ao[qI + (int64_t)qJ * n] : z;
    // T = blk * J_J ;  J_J = [[c, s], [-s ph, c ph]]
    const C mJ10 = cscale(rj.ph, -rj.s), mJ11 = cscale(rj.ph, rj.c);
    const C t00 = cadd(cscale(b00, rj.c), cmul(b01, mJ10));
    const C t01 = cadd(cscale(b00, rj.s), cmul(b01, mJ11));
    const C t10 = cadd(cscale(b10, rj.c), cmul(b11, mJ10));
    const C t11 = cadd(cscale(b10, rj.s), cmul(b11, mJ11));
    // N = J_I^H T ; J_I^H = [[c, -s conj(ph)], [s, c conj(ph)]]
    const C h01 = cscale(cconj(ri.ph), -ri.s), h11 = cscale(cconj(ri.ph), ri.c);
    const C n00 = cadd(cscale(t00, ri.c), cmul(h01, t10));
    const C n01 = cadd(cscale(t01, ri.c), cmul(h01, t11));
    const C n10 = cadd(cscale(t00, ri.s), cmul(h11, t10));
    const C n11 = cadd(cscale(t01, ri.s), cmul(h11, t11));
    if (vpI && vpJ) An[pI + (int64_t)pJ * n] = n00;
    if (vpI && vqJ) An[pI + (int64_t)qJ * n] = n01;
    if (vqI && vpJ) An[qI + (int64_t)pJ * n] = n10;
    if (vqI && vqJ) An[qI + (int64_t)qJ * n] = n11;
  } else if (idx < nblk + (int64_t)n * npair) {
    const int64_t k = idx - nblk;
    const int r = (int)(k % n), Jx = (int)(k / n);
    int pJ, qJ;
    rr_pair(t, Jx, np, pJ, qJ);
    const RotT<C> rj = rot[Jx];
    const bool vp = pJ < n, vq = qJ < n;
    const C vpv = vp ? Vo[r + (int64_t)pJ * n] : z;
    const C vqv = vq ? Vo[r + (int64_t)qJ * n] : z;
    const C mJ10 = cscale(rj.ph, -rj.s), mJ11 = cscale(rj.ph, rj.c);
    if (vp) Vn[r + (int64_t)pJ * n] = cadd(cscale(vpv, rj.c), cmul(vqv, mJ10));
    if (vq) Vn[r + (int64_t)qJ * n] = cadd(cscale(vpv, rj.s), cmul(vqv, mJ11));
  }
}

// One pairing round with the rotations computed inside the kernel (used in FP32, where a
// rotation costs a few instructions against a launch): a CTA updates a 16 x 16 tile of 2 x 2
// blocks of A (pairs I, J) or a 16-row x 16-pair tile of V after its first threads have
// computed the rotations the tile needs from the round's input matrix.
constexpr int kJT = 16;
template <typename C>
__global__ void __launch_bounds__(256) k_jacobi_round_fused(const C* __restrict__ Ao, C* __restrict__ An,
                                                           const C* __restrict__ Vo, C* __restrict__ Vn, int n,
                                                           int np, int t, int ta) {
  __shared__ RotT<C> ri_s[kJT], rj_s[kJT];
  const int npair = np / 2;
  const int tx = threadIdx.x % kJT, ty = threadIdx.x / kJT;
  const bool is_a = (int)blockIdx.x < ta;
  int I0 = 0, J0, r0 = 0;
  if (is_a) {
    const int tpr = (npair + kJT - 1) / kJT;
    I0 = (blockIdx.x % tpr) * kJT;
    J0 = (blockIdx.x / tpr) * kJT;
  } else {
    const int b = blockIdx.x - ta;
    const int tpr = (n + kJT - 1) / kJT;
    r0 = (b % tpr) * kJT;
    J0 = (b / tpr) * kJT;
  }
  if (threadIdx.x < kJT) {
    const int J = J0 + threadIdx.x;
    if (J < npair) {
      int p, q;
      rr_pair(t, J, np, p, q);
      rj_s[threadIdx.x] = jac_rot(Ao, n, p, q);
    }
  } else if (is_a && threadIdx.x < 2 * kJT) {
    const int I = I0 + threadIdx.x - kJT;
    if (I < npair) {
      int p, q;
      rr_pair(t, I, np, p, q);
      ri_s[threadIdx.x - kJT] = jac_rot(Ao, n, p, q);
    }
  }
  __syncthreads();
  C z;
  z.x = 0;
  z.y = 0;
  if (is_a) {
    const int I = I0 + tx, Jx = J0 + ty;
    if (I >= npair || Jx >= npair) return;
    int pI, qI, pJ, qJ;
    rr_pair(t, I, np, pI, qI);
    rr_pair(t, Jx, np, pJ, qJ);
    const RotT<C> ri = ri_s[tx], rj = rj_s[ty];
    const bool vpI = pI < n, vqI = qI < n, vpJ = pJ < n, vqJ = qJ < n;
    const C b00 = (vpI && vpJ) ? Ao[pI + (int64_t)pJ * n] : z;
    const C b01 = (vpI && vqJ) ? Ao[pI + (int64_t)qJ * n] : z;
    const C b10 = (vqI && vpJ) ? Ao[qI + (int64_t)pJ * n] : z;
    const C b11 = (vqI && vqJ) ? Ao[qI + (int64_t)qJ * n] : z;
    const C mJ10 = cscale(rj.ph, -rj.s), mJ11 = cscale(rj.ph, rj.c);
    const C t00 = cadd(cscale(b00, rj.c), cmul(b01, mJ10));
    const C t01 = cadd(cscale(b00, rj.s), cmul(b01, mJ11));
    const C t10 = cadd(cscale(b10, rj.c), cmul(b11, mJ10));
    const C t11 = cadd(cscale(b10, rj.s), cmul(b11, mJ11));
    const C h01 = cscale(cconj(ri.ph), -ri.s), h11 = cscale(cconj(ri.ph), ri.c);
    if (vpI && vpJ) An[pI + (int64_t)pJ * n] = cadd(cscale(t00, ri.c), cmul(h01, t10));
    if (vpI && vqJ) An[pI + (int64_t)qJ * n] = cadd(cscale(t01, ri.c), cmul(h01, t11));
    if (vqI && vpJ) An[qI + (int64_t)pJ * n] = cadd(cscale(t00, ri.s), cmul(h11, t10));
    if (vqI && vqJ) An[qI + (int64_t)qJ * n] = cadd(cscale(t01, ri.s), cmul(h11, t11));
  } else {
    const int r = r0 + tx, Jx = J0 + ty;
    if (r >= n || Jx >= npair) return;
    int pJ, qJ;
    rr_pair(t, Jx, np, pJ, qJ);
    const RotT<C> rj = rj_s[ty];
    const bool vp = pJ < n, vq = qJ < n;
    const C vpv = vp ? Vo[r + (int64_t)pJ * n] : z;
    const C vqv = vq ? Vo[r + (int64_t)qJ * n] : z;
    const C mJ10 = cscale(rj.ph, -rj.s), mJ11 = cscale(rj.ph, rj.c);
    if (vp) Vn[r + (int64_t)pJ * n] = cadd(cscale(vpv, rj.c), cmul(vqv, mJ10));
    if (vq) Vn[r + (int64_t)qJ * n] = cadd(cscale(vpv, rj.s), cmul(vqv, mJ11));
  }
}

template <typename C>
__global__ void k_eye(C* V, int n) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  V[idx].x = (i == j) ? 1 : 0;
  V[idx].y = 0;
}

// out[0] = sum_{i != j} |A_ij|^2, out[1] = sum_i A_ii^2 (accumulated in FP64)
template <typename C>
__global__ void k_offnorm(const C* A, int n, double* out) {
  __shared__ double so[256], sd[256];
  double o = 0, d = 0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    const double ax = A[idx].x, ay = A[idx].y;
    if (i == j) d += ax * ax; else o += ax * ax + ay * ay;
  }
  so[threadIdx.x] = o; sd[threadIdx.x] = d;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { so[threadIdx.x] += so[threadIdx.x + s]; sd[threadIdx.x] += sd[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { atomicAdd(out, so[0]); atomicAdd(out + 1, sd[0]); }
}

// cyclic Jacobi sweeps on A (n x n, lda n, destroyed; the rotated matrix ends in A) with the
// accumulated rotations in V; ws: 2 n*n + n + 2 complex of type C.  Returns the sweeps done.
template <typename C>
int jacobi_sweeps(C* A, int n, C* V, C* ws, double* norms_dev, cudaStream_t st, int max_sweeps, double tol,
                  bool* converged, C** A_out, C** V_out) {
  C* A2 = ws;
  C* V2 = ws + (int64_t)n * n;
  RotT<C>* rot = reinterpret_cast<RotT<C>*>(ws + 2 * (int64_t)n * n);
  const int64_t nn = (int64_t)n * n;
  k_eye<C><<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(V, n); count_launch();
  const int np = (n % 2) ? n + 1 : n;
  const int npair = np / 2;
  const int64_t work = (int64_t)npair * npair + (int64_t)n * npair;
  const unsigned nblk = (unsigned)((work + 255) / 256);
  C *Acur = A, *Anext = A2, *Vcur = V, *Vnext = V2;
  int sweep = 0;
  bool conv = (n <= 1);
  double h[2];
  double prev_off = INFINITY;
  // FP32: one launch per round, the rotations recomputed per CTA; FP64: the rotations once per
  // round in their own launch (recomputing them per CTA costs more FP64 time than the launch)
  constexpr bool kFused = sizeof(C) == 8;
  const int tpa = (npair + kJT - 1) / kJT, ta = tpa * tpa, tv = ((n + kJT - 1) / kJT) * tpa;
  while (!conv && sweep < max_sweeps) {
    for (int t = 0; t < np - 1; ++t) {
      if (kFused) {
        k_jacobi_round_fused<C><<<ta + tv, 256, 0, st>>>(Acur, Anext, Vcur, Vnext, n, np, t, ta); count_launch();
      } else {
        k_jacobi_rot<C><<<npair, 32, 0, st>>>(Acur, n, np, t, rot); count_launch();
        k_jacobi_round<C><<<nblk, 256, 0, st>>>(Acur, Anext, Vcur, Vnext, n, np, t, rot); count_launch();
      }
      C* x = Acur; Acur = Anext; Anext = x;
      x = Vcur; Vcur = Vnext; Vnext = x;
    }
    ++sweep;
    cudaMemsetAsync(norms_dev, 0, 2 * sizeof(double), st);
    k_offnorm<C><<<64, 256, 0, st>>>(Acur, n, norms_dev); count_launch();
    cudaError_t e = cudaMemcpyAsync(h, norms_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return -1;
    // converged below tol * ||A||_F, or stalled at the rounding floor (no halving in a sweep)
    const double off = sqrt(h[0]), nrm = sqrt(h[0] + h[1]);
    const double floor_rel = sizeof(C) == 16 ? 1e-10 : 1e-4;
    if (off <= tol * nrm) conv = true;
    else if (off <= floor_rel * nrm && off > 0.5 * prev_off) conv = true;
    prev_off = off;
  }
  *converged = conv;
  *A_out = Acur;
  *V_out = Vcur;
  return sweep;
}

// ascending sort of the diagonal with its eigenvectors (rank by counting; ties by index)
__global__ void k_sort_eig(const double2* A, const double2* V, int n, double* eig, double2* U) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const double li = A[i + (int64_t)i * n].x;
  __shared__ int rank;
  if (threadIdx.x == 0) rank = 0;
  __syncthreads();
  int r = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double lj = A[j + (int64_t)j * n].x;
    if (lj < li || (lj == li && j < i)) ++r;
  }
  atomicAdd(&rank, r);
  __syncthreads();
  const int rk = rank;
  if (threadIdx.x == 0) eig[rk] = li;
  for (int k = threadIdx.x; k < n; k += blockDim.x) U[k + (int64_t)rk * n] = V[k + (int64_t)i * n];
}

int la_jacobi_eigh(double2* A, int n, double2* U, double* eig, double2* ws, double* norms_dev,
                   cudaStream_t st, int max_sweeps, double tol, int* sweeps_out) {
  // ws: 3 n*n + n + 2 complex (V, then the A copy, V copy and rotations of a round)
  double2* V = ws;
  bool conv = false;
  double2 *Af = nullptr, *Vf = nullptr;
  const int sweep = jacobi_sweeps<double2>(A, n, V, ws + (int64_t)n * n, norms_dev, st, max_sweeps, tol, &conv, &Af,
                                           &Vf);
  if (sweep < 0) return cuda_status(cudaGetLastError(), "jacobi");
  if (sweeps_out) *sweeps_out = sweep;
  k_sort_eig<<<n, 128, 0, st>>>(Af, Vf, n, eig, U); count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "jacobi sort");
  return conv ? PW_OK : set_error(PW_ENOTCONV, "Jacobi eigensolver: %d sweeps without convergence", sweep);
}

// FP32 Jacobi pre-rotation of the mixed solver: A (complex64 n x n, destroyed) is rotated
// until its off-diagonal part is below tol (relative) or stops decreasing; V (complex64 n x n)
// receives the accumulated rotation.  ws: 2 n*n + n + 2 complex64.
int la_jacobi_rotate32(float2* A, int n, float2* V, float2* ws, double* norms_dev, cudaStream_t st, int max_sweeps,
                       double tol, int* sweeps_out) {
  bool conv = false;
  float2 *Af = nullptr, *Vf = nullptr;
  const int sweep = jacobi_sweeps<float2>(A, n, V, ws, norms_dev, st, max_sweeps, tol, &conv, &Af, &Vf);
  if (sweep < 0) return cuda_status(cudaGetLastError(), "jacobi (FP32)");
  if (Vf != V) {
    cudaError_t e = cudaMemcpyAsync(V, Vf, sizeof(float2) * (size_t)n * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "jacobi (FP32) copy");
  }
  if (sweeps_out) *sweeps_out = sweep;
  return PW_OK;
}

// ---- column reductions ------------------------------------------------------------
// out[j] = sum_g conj(A[g, j]) B[g, j]
template <typename T>
__global__ void k_coldot(const cplx<T>* A, int64_t lda, const cplx<T>* B, int64_t ldb, int npw, double2* out) {
  const int j = blockIdx.x;
  const cplx<T>* a = A + (int64_t)j * lda;
  const cplx<T>* b = B + (int64_t)j * ldb;
  double sr = 0, si = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double ax = a[g].x, ay = a[g].y, bx = b[g].x, by = b[g].y;
    sr += ax * bx + ay * by;
    si += ax * by - ay * bx;
  }
  __shared__ double s1[256], s2[256];
  s1[threadIdx.x] = sr; s2[threadIdx.x] = si;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { s1[threadIdx.x] += s1[threadIdx.x + s]; s2[threadIdx.x] += s2[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = make_double2(s1[0], s2[0]);
}

cudaError_t la_coldot(const double2* A, int64_t lda, const double2* B, int64_t ldb, int npw, int m,
                      double2* out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_coldot<double><<<m, 256, 0, st>>>(A, lda, B, ldb, npw, out); count_launch();
  return cudaGetLastError();
}

// r_j = || HY_j - eig_j SY_j ||
__global__ void k_resid(const double2* HY, int64_t ldh, const double2* SY, int64_t lds, int npw, const double* eig,
                        double* r) {
  const int j = blockIdx.x;
  const double l = eig[j];
  double s = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 h = HY[g + (int64_t)j * ldh], sv = SY[g + (int64_t)j * lds];
    const double x = h.x - l * sv.x, y = h.y - l * sv.y;
    s += x * x + y * y;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) r[j] = sqrt(sh[0]);
}

cudaError_t la_resid(const double2* HY, int64_t ldh, const double2* SY, int64_t lds, int npw, int m,
                     const double* eig, double* r, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_resid<<<m, 256, 0, st>>>(HY, ldh, SY, lds, npw, eig, r); count_launch();
  return cudaGetLastError();
}

// rq[j] = Re(num_j) / Re(den_j); mm[0] = min, mm[1] = max
__global__ void k_rq_minmax(const double2* num, const double2* den, int m, double* rq, double* mm) {
  __shared__ double smin[256], smax[256];
  double lo = INFINITY, hi = -INFINITY;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double v = num[j].x / den[j].x;
    rq[j] = v;
    lo = fmin(lo, v); hi = fmax(hi, v);
  }
  smin[threadIdx.x] = lo; smax[threadIdx.x] = hi;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { mm[0] = smin[0]; mm[1] = smax[0]; }
}

cudaError_t la_rq_minmax(const double2* num, const double2* den, int m, double* rq, double* mm, cudaStream_t st) {
  k_rq_minmax<<<1, 256, 0, st>>>(num, den, m, rq, mm); count_launch();
  return cudaGetLastError();
}

// ---- Lanczos helpers (one vector) ---------------------------------------------------
// ab: device array, alpha at ab[2k], beta at ab[2k+1]
__global__ void k_lz_dot(const double2* v, const double2* w, int n, double* alpha_out) {
  __shared__ double sh[1024];
  double s = 0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) s += v[g].x * w[g].x + v[g].y * w[g].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *alpha_out = sh[0];
}

// w <- w - alpha v - beta vprev ; beta_out = ||w|| ; vprev <- v ; v <- w / beta_out
__global__ void k_lz_update(double2* w, double2* v, double2* vprev, int n, const double* alpha,
                            const double* beta_prev, double* beta_out) {
  __shared__ double sh[1024];
  const double a = *alpha, b = beta_prev ? *beta_prev : 0.0;
  double s = 0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    double2 x = w[g];
    const double2 vv = v[g], vp = vprev[g];
    x.x -= a * vv.x + b * vp.x;
    x.y -= a * vv.y + b * vp.y;
    w[g] = x;
    s += x.x * x.x + x.y * x.y;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  const double nb = sqrt(sh[0]);
  const double inv = nb > 0 ? 1.0 / nb : 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    vprev[g] = v[g];
    v[g] = cscale(w[g], inv);
  }
  if (threadIdx.x == 0) *beta_out = nb;
}

__global__ void k_lz_normalize(const double2* v0, double2* v, double2* vprev, int n) {
  __shared__ double sh[1024];
  double s = 0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) s += v0[g].x * v0[g].x + v0[g].y * v0[g].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  const double inv = 1.0 / sqrt(sh[0]);
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    v[g] = cscale(v0[g], inv);
    vprev[g] = make_double2(0, 0);
  }
}

// largest eigenvalue of the k x k symmetric tridiagonal (alpha, beta) by Sturm bisection;
// out[0] = theta_max + |beta_k|, out[1] = theta_max
__global__ void k_lz_bound(const double* ab, int k, double* out) {
  if (threadIdx.x != 0) return;
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < k; ++i) {
    const double a = ab[2 * i];
    const double r = (i > 0 ? fabs(ab[2 * i - 1]) : 0.0) + (i < k - 1 ? fabs(ab[2 * i + 1]) : 0.0);
    lo = fmin(lo, a - r);
    hi = fmax(hi, a + r);
  }
  // count of eigenvalues < x
  for (int it = 0; it < 200; ++it) {
    const double x = 0.5 * (lo + hi);
    if (x == lo || x == hi) break;
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      const double b2 = (i > 0) ? ab[2 * i - 1] * ab[2 * i - 1] : 0.0;
      d = (ab[2 * i] - x) - (i > 0 ? b2 / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++cnt;
    }
    if (cnt == k) hi = x; else lo = x;
  }
  out[1] = hi;
  out[0] = hi + fabs(ab[2 * k - 1]);
}

cudaError_t la_lanczos(const double2* v0, int n, int steps, double2* v, double2* vprev, double2* w, double* ab,
                       double* bound, ApplyFn apply, void* ctx, cudaStream_t st) {
  k_lz_normalize<<<1, 1024, 0, st>>>(v0, v, vprev, n); count_launch();
  for (int k = 0; k < steps; ++k) {
    int s = apply(ctx, v, w);
    if (s != PW_OK) return cudaErrorUnknown;
    k_lz_dot<<<1, 1024, 0, st>>>(v, w, n, ab + 2 * k); count_launch();
    k_lz_update<<<1, 1024, 0, st>>>(w, v, vprev, n, ab + 2 * k, k > 0 ? ab + 2 * k - 1 : nullptr, ab + 2 * k + 1); count_launch();
  }
  k_lz_bound<<<1, 32, 0, st>>>(ab, steps, bound); count_launch();
  return cudaGetLastError();
}

// ---- conversions ----------------------------------------------------------------
__global__ void k_c128_to_c64(const double2* a, int64_t lda, float2* b, int64_t ldb, int n, int m) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * m) return;
  const int g = (int)(idx % n), j = (int)(idx / n);
  const double2 v = a[g + j * lda];
  b[g + j * ldb] = make_float2((float)v.x, (float)v.y);
}
__global__ void k_c64_to_c128(const float2* a, int64_t lda, double2* b, int64_t ldb, int n, int m) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * m) return;
  const int g = (int)(idx % n), j = (int)(idx / n);
  const float2 v = a[g + j * lda];
  b[g + j * ldb] = make_double2(v.x, v.y);
}
cudaError_t la_to_c64(const double2* a, int64_t lda, float2* b, int64_t ldb, int n, int m, cudaStream_t st) {
  const int64_t t = (int64_t)n * m;
  if (t <= 0) return cudaSuccess;
  k_c128_to_c64<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(a, lda, b, ldb, n, m); count_launch();
  return cudaGetLastError();
}
cudaError_t la_to_c128(const float2* a, int64_t lda, double2* b, int64_t ldb, int n, int m, cudaStream_t st) {
  const int64_t t = (int64_t)n * m;
  if (t <= 0) return cudaSuccess;
  k_c64_to_c128<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(a, lda, b, ldb, n, m); count_launch();
  return cudaGetLastError();
}


// ---- LOBPCG helpers (Alg. 11) ----------------------------------------------------------
// W_j = K_j (HX_j - lam_j SX_j), K_j the Teter-Payne-Allan preconditioner of band j,
// K = p / (p + 16 x^4), p = 27 + 18 x + 12 x^2 + 8 x^3, x = t_G / E_kin(X_j),
// E_kin = sum t_G |x_G|^2 / sum |x_G|^2; rn[j] = || HX_j - lam_j SX_j || before K
__global__ void __launch_bounds__(256) k_lob_resid(const double2* __restrict__ HX, const double2* __restrict__ SX,
                                                   const double2* __restrict__ X, int64_t ld, int npw,
                                                   const double* __restrict__ lam, const double* __restrict__ kin,
                                                   double2* __restrict__ W, int64_t ldw, double* __restrict__ rn) {
  const int j = blockIdx.x;
  const double l = lam[j];
  const double2* h = HX + (int64_t)j * ld;
  const double2* s = SX + (int64_t)j * ld;
  const double2* x = X + (int64_t)j * ld;
  double sk = 0, sn = 0, sr = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 xv = x[g];
    const double a = xv.x * xv.x + xv.y * xv.y;
    sk += kin[g] * a;
    sn += a;
    const double rx = h[g].x - l * s[g].x, ry = h[g].y - l * s[g].y;
    sr += rx * rx + ry * ry;
  }
  __shared__ double s1[256], s2[256], s3[256];
  s1[threadIdx.x] = sk; s2[threadIdx.x] = sn; s3[threadIdx.x] = sr;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
      s3[threadIdx.x] += s3[threadIdx.x + o];
    }
    __syncthreads();
  }
  const double ekin = s1[0] / s2[0];
  if (threadIdx.x == 0) rn[j] = sqrt(s3[0]);
  double2* w = W + (int64_t)j * ldw;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double xx = kin[g] / ekin;
    const double p = 27.0 + xx * (18.0 + xx * (12.0 + 8.0 * xx));
    const double x2 = xx * xx;
    const double k = p / (p + 16.0 * x2 * x2);
    w[g] = make_double2(k * (h[g].x - l * s[g].x), k * (h[g].y - l * s[g].y));
  }
}

cudaError_t la_lob_resid(const double2* HX, const double2* SX, const double2* X, int64_t ld, int npw, int m,
                         const double* lam, const double* kin, double2* W, int64_t ldw, double* rn, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_lob_resid<<<m, 256, 0, st>>>(HX, SX, X, ld, npw, lam, kin, W, ldw, rn); count_launch();
  return cudaGetLastError();
}

// B (k x 2 keep, ld k) = [C with its first `keep` rows zeroed | C], C (k x keep, ld k): Z B gives
// [P_new | Psi_new] in one product
__global__ void k_lob_coef(const double2* __restrict__ C, int k, int keep, double2* __restrict__ B) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * 2 * keep) return;
  const int r = (int)(idx % k), c = (int)(idx / k);
  const double2 v = C[(int64_t)(c % keep) * k + r];
  B[idx] = (c < keep && r < keep) ? make_double2(0.0, 0.0) : v;
}

cudaError_t la_lob_coef(const double2* C, int k, int keep, double2* B, cudaStream_t st) {
  const int64_t n = (int64_t)k * 2 * keep;
  if (n <= 0) return cudaSuccess;
  k_lob_coef<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(C, k, keep, B); count_launch();
  return cudaGetLastError();
}


// ---- spectrum slicing: per-column Chebyshev sums over the filter's steps ----------------
// out[:, j] (=, or +=) coef[j] y[:, j]
template <typename T>
__global__ void k_cheb_acc(const cplx<T>* __restrict__ y, int64_t ldy, int npw, int nband,
                           const double* __restrict__ coef, cplx<T>* __restrict__ out, int64_t ldo, int first) {
  const int64_t total = (int64_t)npw * nband;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(idx % npw), j = (int)(idx / npw);
    const T c = (T)coef[j];
    const cplx<T> v = y[(int64_t)j * ldy + g];
    cplx<T>* o = out + (int64_t)j * ldo + g;
    if (first) {
      o->x = c * v.x;
      o->y = c * v.y;
    } else {
      o->x += c * v.x;
      o->y += c * v.y;
    }
  }
}

template <typename T>
cudaError_t la_cheb_acc(const cplx<T>* y, int64_t ldy, int npw, int nband, const double* coef, cplx<T>* out,
                        int64_t ldo, int first, cudaStream_t st) {
  const int64_t total = (int64_t)npw * nband;
  if (total <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_cheb_acc<T><<<grid, 256, 0, st>>>(y, ldy, npw, nband, coef, out, ldo, first); count_launch();
  return cudaGetLastError();
}
template cudaError_t la_cheb_acc<float>(const cplx<float>*, int64_t, int, int, const double*, cplx<float>*, int64_t,
                                        int, cudaStream_t);
template cudaError_t la_cheb_acc<double>(const cplx<double>*, int64_t, int, int, const double*, cplx<double>*,
                                         int64_t, int, cudaStream_t);

}  // namespace pw
