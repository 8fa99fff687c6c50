// FP64 dense linear algebra launchers (la_fp64.cu).
#pragma once
#include "pw_internal.cuh"

namespace pw {
typedef int (*ApplyFn)(void* ctx, const double2* v, double2* w);

cudaError_t la_herm_sym(double2* A, int64_t lda, int n, cudaStream_t st);
// A[j][i] = conj(A[i][j]) for i > j, real diagonal (the lower triangle is kept)
cudaError_t la_herm_from_lower(double2* A, int64_t lda, int n, cudaStream_t st);
// lower Cholesky in place; *flag set to 1 (device) if a pivot is not positive
cudaError_t la_cholesky(double2* A, int64_t lda, int n, int* flag, cudaStream_t st);
cudaError_t la_zero_upper(double2* A, int64_t lda, int n, cudaStream_t st);
// X = L^{-1}; tmp: n*n complex scratch
cudaError_t la_trinv_lower(const double2* L, int64_t lda, int n, double2* X, int64_t ldx, double2* tmp,
                           cudaStream_t st);
// eigenpairs of Hermitian A (n x n, lda n; destroyed): eig ascending (device), U (n x n);
// ws: 3 n*n + n + 2 complex; norms_dev: 2 doubles.  Synchronises the stream once per sweep.
int la_jacobi_eigh(double2* A, int n, double2* U, double* eig, double2* ws, double* norms_dev,
                   cudaStream_t st, int max_sweeps, double tol, int* sweeps_out);
// FP32 Jacobi pre-rotation: V (n x n) <- the rotation that brings A (complex64, destroyed) to
// off-diagonal norm below tol relative (or to the FP32 floor); ws: 2 n*n + n + 2 complex64
int la_jacobi_rotate32(float2* A, int n, float2* V, float2* ws, double* norms_dev, cudaStream_t st, int max_sweeps,
                       double tol, int* sweeps_out);
cudaError_t la_coldot(const double2* A, int64_t lda, const double2* B, int64_t ldb, int npw, int m,
                      double2* out, cudaStream_t st);
cudaError_t la_resid(const double2* HY, int64_t ldh, const double2* SY, int64_t lds, int npw, int m,
                     const double* eig, double* r, cudaStream_t st);
cudaError_t la_rq_minmax(const double2* num, const double2* den, int m, double* rq, double* mm, cudaStream_t st);
// steps-step Lanczos from v0; ab: 2*steps doubles; bound: 2 doubles {theta+|beta|, theta}
cudaError_t la_lanczos(const double2* v0, int n, int steps, double2* v, double2* vprev, double2* w, double* ab,
                       double* bound, ApplyFn apply, void* ctx, cudaStream_t st);
cudaError_t la_to_c64(const double2* a, int64_t lda, float2* b, int64_t ldb, int n, int m, cudaStream_t st);
cudaError_t la_to_c128(const float2* a, int64_t lda, double2* b, int64_t ldb, int n, int m, cudaStream_t st);
// LOBPCG: W = K (HX - lam SX) with the Teter-Payne-Allan preconditioner, rn = residual norms
cudaError_t la_lob_resid(const double2* HX, const double2* SX, const double2* X, int64_t ld, int npw, int m,
                         const double* lam, const double* kin, double2* W, int64_t ldw, double* rn, cudaStream_t st);
// B (k x 2 keep) = [C without its first keep rows | C]
cudaError_t la_lob_coef(const double2* C, int k, int keep, double2* B, cudaStream_t st);
// spectrum slicing: out[:, j] = (first ? 0 : out[:, j]) + coef[j] y[:, j] (coef: device, nband)
template <typename T>
cudaError_t la_cheb_acc(const cplx<T>* y, int64_t ldy, int npw, int nband, const double* coef, cplx<T>* out,
                        int64_t ldo, int first, cudaStream_t st);
}  // namespace pw
