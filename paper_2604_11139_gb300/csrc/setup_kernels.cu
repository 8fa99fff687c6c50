// Setup kernels run once per context: projector matrix generation (Sec. 4.2,
// P = <G|p_i^R>), the permuted local-potential grid, the un-permutation of a
// grid accumulated in the FFT's digit-reversed order, and precision casts.
#include <math.h>

#include "pw_internal.cuh"
#include "setup.cuh"

namespace pw {

// P[g + col*npw]: col = (atom*nchan + chan)*4 + m, m in {s, px, py, pz}
//   s:   exp(-q^2 s^2/2) e^{-i q.R};  p_a: (-i) q_a s exp(-q^2 s^2/2) e^{-i q.R}
__global__ void k_projectors(int npw, const int* __restrict__ miller, ProjParams pp, double2* __restrict__ P) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int atom = blockIdx.y;
  if (g >= npw) return;
  const double h = miller[3 * g], k = miller[3 * g + 1], l = miller[3 * g + 2];
  double q[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    q[c] = (h + pp.kred[0]) * pp.B[0 * 3 + c] + (k + pp.kred[1]) * pp.B[1 * 3 + c] + (l + pp.kred[2]) * pp.B[2 * 3 + c];
  const double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
  const double* R = pp.tau + 3 * atom;
  const double arg = -(q[0] * R[0] + q[1] * R[1] + q[2] * R[2]);
  double sn, cs;
  sincos(arg, &sn, &cs);
  for (int ch = 0; ch < pp.nchan; ++ch) {
    const double s = pp.sigma[ch];
    const double f = exp(-0.5 * q2 * s * s);
    const int col0 = (atom * pp.nchan + ch) * 4;
    P[g + (int64_t)col0 * npw] = make_double2(f * cs, f * sn);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double amp = q[a] * s * f;  // times (-i) e^{i arg}: (-i)(cs + i sn) = sn - i cs
      P[g + (int64_t)(col0 + 1 + a) * npw] = make_double2(amp * sn, -amp * cs);
    }
  }
}

__global__ void k_colnorm_scale(double2* P, int npw, int ncol) {
  const int c = blockIdx.x;
  double2* col = P + (int64_t)c * npw;
  double s = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s += col[g].x * col[g].x + col[g].y * col[g].y;
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  const double inv = sh[0] > 0 ? 1.0 / sqrt(sh[0]) : 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) col[g] = cscale(col[g], inv);
}

cudaError_t setup_projectors(int npw, const int* miller_dev, const ProjParams& pp, int natom, double2* P,
                             cudaStream_t st) {
  if (npw <= 0 || natom <= 0) return cudaSuccess;
  k_projectors<<<dim3((npw + 127) / 128, natom), 128, 0, st>>>(npw, miller_dev, pp, P); count_launch();
  k_colnorm_scale<<<natom * pp.nchan * 4, 256, 0, st>>>(P, npw, natom * pp.nchan * 4); count_launch();
  return cudaGetLastError();
}

// vperm[jx][jy][jz] = V[rho_x(jx)][rho_y(jy)][rho_z(jz)] * scale
template <typename T>
__global__ void k_vperm(const double* __restrict__ V, int n1, int n2, int n3, const int* __restrict__ r1,
                        const int* __restrict__ r2, const int* __restrict__ r3, double scale, T* __restrict__ out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)n1 * n2 * n3;
  if (idx >= tot) return;
  const int jz = (int)(idx % n3);
  const int jy = (int)((idx / n3) % n2);
  const int jx = (int)(idx / ((int64_t)n2 * n3));
  const int64_t src = ((int64_t)r1[jx] * n2 + r2[jy]) * n3 + r3[jz];
  out[idx] = (T)(V[src] * scale);
}

cudaError_t setup_vperm(const double* V, const int* n, int* const* rho, double scale, double* out64, float* out32,
                        cudaStream_t st) {
  const int64_t tot = (int64_t)n[0] * n[1] * n[2];
  const unsigned nb = (unsigned)((tot + 255) / 256);
  k_vperm<double><<<nb, 256, 0, st>>>(V, n[0], n[1], n[2], rho[0], rho[1], rho[2], scale, out64); count_launch();
  k_vperm<float><<<nb, 256, 0, st>>>(V, n[0], n[1], n[2], rho[0], rho[1], rho[2], scale, out32); count_launch();
  return cudaGetLastError();
}

cudaError_t setup_vperm32(const double* V, const int* n, int* const* rho, double scale, float* out32,
                          cudaStream_t st) {
  const int64_t tot = (int64_t)n[0] * n[1] * n[2];
  const unsigned nb = (unsigned)((tot + 255) / 256);
  k_vperm<float><<<nb, 256, 0, st>>>(V, n[0], n[1], n[2], rho[0], rho[1], rho[2], scale, out32); count_launch();
  return cudaGetLastError();
}

// out[rho_x(jx)][rho_y(jy)][rho_z(jz)] (+)= in[jx][jy][jz]
__global__ void k_unperm(const double* __restrict__ in, int n1, int n2, int n3, const int* __restrict__ r1,
                         const int* __restrict__ r2, const int* __restrict__ r3, double* __restrict__ out,
                         int accumulate) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)n1 * n2 * n3;
  if (idx >= tot) return;
  const int jz = (int)(idx % n3);
  const int jy = (int)((idx / n3) % n2);
  const int jx = (int)(idx / ((int64_t)n2 * n3));
  const int64_t dst = ((int64_t)r1[jx] * n2 + r2[jy]) * n3 + r3[jz];
  out[dst] = accumulate ? out[dst] + in[idx] : in[idx];
}

cudaError_t setup_unperm(const double* in, const int* n, int* const* rho, double* out, int accumulate,
                         cudaStream_t st) {
  const int64_t tot = (int64_t)n[0] * n[1] * n[2];
  k_unperm<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, n[0], n[1], n[2], rho[0], rho[1], rho[2], out,
                                                          accumulate); count_launch();
  return cudaGetLastError();
}

__global__ void k_d2f(const double* a, float* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_z2c(const double2* a, float2* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
cudaError_t cast_d2f(const double* a, float* b, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_d2f<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n); count_launch();
  return cudaGetLastError();
}
cudaError_t cast_z2c(const double2* a, float2* b, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_z2c<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n); count_launch();
  return cudaGetLastError();
}

// real (column-major) -> complex
__global__ void k_r2z(const double* a, double2* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2(a[i], 0.0);
}
cudaError_t cast_r2z(const double* a, double2* b, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_r2z<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n); count_launch();
  return cudaGetLastError();
}

// A = B + I*shift (complex n x n, B may alias A)
__global__ void k_add_diag(double2* A, int n, double shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + (int64_t)i * n].x += shift;
}
cudaError_t add_diag(double2* A, int n, double shift, cudaStream_t st) {
  k_add_diag<<<(n + 255) / 256, 256, 0, st>>>(A, n, shift); count_launch();
  return cudaGetLastError();
}

}  // namespace pw
