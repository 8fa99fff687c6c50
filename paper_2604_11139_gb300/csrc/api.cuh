// Internal entry points of pw_api.cu used by the other host translation units.
#pragma once
#include "pw_internal.cuh"

namespace pw {
namespace api {
int check(pw_ctx* ctx);
int check_blk(pw_ctx* ctx, const void* p, int64_t ld, int nband);
// hpsi = H psi in FP64 (S not formed)
int apply64(pw_ctx* ctx, const double2* psi, int64_t ld, int nband, double2* hpsi, int64_t ldo);
// dst = alpha ((H - shift) cur) - beta prev (prev may be NULL), S = I; C_out (nproj x nband, may be NULL) = P^dagger cur
template <typename T>
int recur(pw_ctx* ctx, const cplx<T>* cur, int64_t ldc, const cplx<T>* prev, int64_t ldp, cplx<T>* dst, int64_t ldd,
          int nband, double alpha, double beta, double shift, cplx<T>* C_out);
// two S-Ortho passes + Rayleigh-Ritz on Y (in place); Q (ld npw), X (m x m) and device Ritz values optional
int rr(pw_ctx* ctx, double2* Y, int64_t ldy, int m, double* eig_h, double2* q_out, double2* x_out,
       double* eig_dev_out);
// largest Rayleigh quotient of psi (nband > 0) and the Lanczos upper bound (steps > 0)
int bounds(pw_ctx* ctx, const double2* psi, int64_t ld, int nband, int steps, const double2* v0, double* rq_max,
           double* upper);
int fft_band_batch(const pw_ctx* ctx, int nband, size_t elem);
int gemm_nsplit(int m, int n, int k);
}  // namespace api
}  // namespace pw
