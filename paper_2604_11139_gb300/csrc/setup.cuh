// Setup-kernel launchers (setup_kernels.cu).
#pragma once
#include "pw_internal.cuh"

namespace pw {
constexpr int kMaxChan = 8;
struct ProjParams {
  double B[9];      // reciprocal vectors, rows b1, b2, b3 (a_i . b_j = 2 pi delta_ij)
  double kred[3];   // k-point, reduced coordinates
  const double* tau;  // device, natom*3 cartesian
  int nchan;
  double sigma[kMaxChan];
};
cudaError_t setup_projectors(int npw, const int* miller_dev, const ProjParams& pp, int natom, double2* P,
                             cudaStream_t st);
cudaError_t setup_vperm(const double* V, const int* n, int* const* rho, double scale, double* out64, float* out32,
                        cudaStream_t st);
// complex64 copy only (the x-line forms with the radix order of the x plan swapped)
cudaError_t setup_vperm32(const double* V, const int* n, int* const* rho, double scale, float* out32,
                          cudaStream_t st);
cudaError_t setup_unperm(const double* in, const int* n, int* const* rho, double* out, int accumulate,
                         cudaStream_t st);
cudaError_t cast_d2f(const double* a, float* b, int64_t n, cudaStream_t st);
cudaError_t cast_z2c(const double2* a, float2* b, int64_t n, cudaStream_t st);
cudaError_t cast_r2z(const double* a, double2* b, int64_t n, cudaStream_t st);
cudaError_t add_diag(double2* A, int n, double shift, cudaStream_t st);
}  // namespace pw
