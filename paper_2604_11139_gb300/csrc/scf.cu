// Self-consistent field loop around the filter (Alg. 3): occupations, density, the
// Hartree + exchange potential of the density, linear mixing.
//
// Alg. 3 repeats [solve H Psi = Lambda S Psi -> occupations from Lambda -> density from the
// occupations and Psi] until self-consistent, without saying how the density sets the next
// Hamiltonian.  The loop here closes it with the smallest published model that feeds the
// density back: insulating filling (the lowest nocc states doubly occupied), the Hartree
// potential of Poisson's equation in reciprocal space, V_H(G) = 4 pi rho(G) / |G|^2 (G != 0;
// a neutralising background at G = 0), and the local-density exchange of Dirac (1930),
// v_x = -(3 rho / pi)^(1/3), energy density rho e_x with e_x = -(3/4) (3/pi)^(1/3) rho^(1/3)
// (correlation left out); the next input potential is V + beta (V_ion + V_H + v_x - V).
//
// The reciprocal-space steps use a second context whose plane-wave sphere is the density
// sphere |G|^2/2 <= 4 E_cut on the same cell and box (Gamma point, no projectors): rho(G) is
// its local-potential apply of rho to the constant function (the G = 0 basis vector), and
// V_H(r) is its density contraction of V_H(G) against the same constant function.
#include <math.h>

#include <algorithm>
#include <vector>

#include "pw_internal.cuh"

namespace pw {
namespace {

constexpr double kPiS = 3.14159265358979323846264338327950288;

// V_H(G) = 4 pi rho(G) / |G|^2, |G|^2 = 2 x the sphere's kinetic energy; 0 at G = 0
__global__ void k_hartree_g(int n, const double* __restrict__ kin, double2* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double g2 = 2.0 * kin[i];
  const double f = g2 > 0.0 ? 4.0 * kPiS / g2 : 0.0;
  g[i] = make_double2(g[i].x * f, g[i].y * f);
}

// per grid point: v_x, V_out = V_ion + V_H + v_x, V_new = V_in + beta (V_out - V_in); sums
// s[0] += (V_in - V_ion) rho, s[1] += V_H rho, s[2] += rho e_x, s[4] += rho; s[3] = max |V_out - V_in|
__global__ void __launch_bounds__(256) k_scf_mix(int64_t n, const double* __restrict__ rho,
                                                 const double* __restrict__ vion, const double* __restrict__ vin,
                                                 const double* __restrict__ vh, double beta, double* __restrict__ vnew,
                                                 double* __restrict__ sums) {
  __shared__ double red[5][8];
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double r = fmax(rho[i], 0.0);
    const double c = cbrt(3.0 * r / kPiS);     // (3 rho / pi)^(1/3)
    const double vx = -c;
    const double ex = -0.75 * c * r;            // rho e_x = -(3/4) (3/pi)^(1/3) rho^(4/3)
    const double vout = vion[i] + vh[i] + vx;
    const double d = vout - vin[i];
    vnew[i] = vin[i] + beta * d;
    a0 += (vin[i] - vion[i]) * rho[i];
    a1 += vh[i] * rho[i];
    a2 += ex;
    a3 = fmax(a3, fabs(d));
    a4 += rho[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    a3 = fmax(a3, __shfl_xor_sync(0xffffffffu, a3, o));
    a4 += __shfl_xor_sync(0xffffffffu, a4, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[0][w] = a0; red[1][w] = a1; red[2][w] = a2; red[3][w] = a3; red[4][w] = a4; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = 0, b1 = 0, b2 = 0, b3 = 0, b4 = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      b0 += red[0][q]; b1 += red[1][q]; b2 += red[2][q]; b3 = fmax(b3, red[3][q]); b4 += red[4][q];
    }
    atomicAdd(&sums[0], b0);
    atomicAdd(&sums[1], b1);
    atomicAdd(&sums[2], b2);
    atomicMax((unsigned long long*)&sums[3], (unsigned long long)__double_as_longlong(b3));  // b3 >= 0
    atomicAdd(&sums[4], b4);
  }
}

int g0_index(const pw_ctx* d) {
  for (int i = 0; i < d->npw; ++i)
    if (d->miller[3 * i] == 0 && d->miller[3 * i + 1] == 0 && d->miller[3 * i + 2] == 0) return i;
  return -1;
}

double cell_volume(const double* a) {
  return fabs(a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
              a[2] * (a[3] * a[7] - a[4] * a[6]));
}

}  // namespace
}  // namespace pw

using namespace pw;

#define SCF_TRY(expr)              \
  do {                             \
    const int _s = (expr);         \
    if (_s != PW_OK) return _s;    \
  } while (0)
#define SCF_CU(expr, where)                                                           \
  do {                                                                                \
    const cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) { dctx->poisoned = true; return cuda_status(_e, where); }  \
  } while (0)

extern "C" PW_API int pw_scf_potential(pw_ctx* dctx, const double* rho, const double* vion, const double* vin,
                                       double beta, double* vnew, double* out) {
  if (!dctx || !rho || !vion || !vin || !vnew || !out) return set_error(PW_EINVAL, "NULL argument");
  if (dctx->poisoned) return set_error(PW_ECUDA, "context poisoned by an earlier CUDA error");
  if (dctx->nproj != 0 || dctx->kpt[0] != 0.0 || dctx->kpt[1] != 0.0 || dctx->kpt[2] != 0.0)
    return set_error(PW_EINVAL, "the density context must be a Gamma-point context without projectors");
  const int g0 = g0_index(dctx);
  if (g0 < 0) return set_error(PW_EINVAL, "the density context's sphere has no G = 0");
  const cudaStream_t st = dctx->stream;
  const int npw = dctx->npw;
  const int64_t ntot = (int64_t)dctx->n[0] * dctx->n[1] * dctx->n[2];
  int status = PW_OK;
  // [e_0 | rho(G) / V_H(G) | V_H(r) | sums]
  unsigned char* w = (unsigned char*)ws_get(dctx, WS_SCF, sizeof(double2) * 2 * (size_t)npw + sizeof(double) * ntot +
                                                             64, &status);
  if (!w) return status;
  double2* e0 = (double2*)w;
  double2* rg = e0 + npw;
  double* vh = (double*)(rg + npw);
  double* sums = vh + ntot;
  const double one[2] = {1.0, 0.0};
  SCF_CU(cudaMemsetAsync(e0, 0, sizeof(double2) * npw, st), "scf e0");
  SCF_CU(cudaMemcpyAsync(e0 + g0, one, sizeof(double2), cudaMemcpyHostToDevice, st), "scf e0");
  // rho(G) = (1/n) sum_j rho(r_j) e^{-iG.r_j} on the density sphere
  SCF_TRY(pw_local_apply(dctx, rho, 1.0, e0, npw, 1, rg, npw, PW_FP64));
  k_hartree_g<<<(npw + 255) / 256, 256, 0, st>>>(npw, dctx->kin64, rg); count_launch();
  SCF_CU(cudaGetLastError(), "hartree");
  // V_H(r) = Re sum_G V_H(G) e^{iG.r}
  const double wone = 1.0;
  SCF_TRY(pw_density_grad(dctx, rg, e0, npw, 1, &wone, vh, 0));
  SCF_CU(cudaMemsetAsync(sums, 0, 5 * sizeof(double), st), "scf sums");
  k_scf_mix<<<304, 256, 0, st>>>(ntot, rho, vion, vin, vh, beta, vnew, sums); count_launch();
  SCF_CU(cudaGetLastError(), "scf mix");
  double h[5];
  SCF_CU(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st), "scf sums copy");
  SCF_CU(cudaStreamSynchronize(st), "scf sync");
  const double dv = cell_volume(dctx->lattice) / (double)ntot;
  out[0] = dv * h[0];          // (Omega/n) sum (V_in - V_ion) rho
  out[1] = 0.5 * dv * h[1];    // E_H
  out[2] = dv * h[2];          // E_x
  out[3] = h[3];               // max |V_out - V_in|
  out[4] = dv * h[4];          // electrons
  return PW_OK;
}

extern "C" PW_API int pw_scf_run(pw_ctx* ctx, pw_ctx* dctx, void* psi, int64_t ld, int nband, int nocc, int degree,
                                 int cycles, int max_iter, double beta, double tol, const void* v0,
                                 const double* vion, int precision, double* eig, double* history, int* iterations) {
  if (!ctx || !dctx || !psi || !v0 || !vion || !eig) return set_error(PW_EINVAL, "NULL argument");
  if (ctx->poisoned) return set_error(PW_ECUDA, "context poisoned by an earlier CUDA error");
  if (nocc < 1 || nocc > nband || max_iter < 1 || !(beta > 0.0) || degree < 1 || cycles < 1)
    return set_error(PW_EINVAL, "bad SCF parameters");
  for (int i = 0; i < 3; ++i)
    if (ctx->n[i] != dctx->n[i]) return set_error(PW_EINVAL, "the density context must share the FFT box");
  const cudaStream_t st = ctx->stream;
  const int64_t ntot = (int64_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  const double omega = cell_volume(ctx->lattice);
  double* buf = nullptr;  // [V_ion | V_in | V_new | rho]
  cudaError_t e = cudaMalloc(&buf, sizeof(double) * 4 * (size_t)ntot);
  if (e != cudaSuccess) return cuda_status(e, "scf buffers");
  struct Free { double* p; ~Free() { if (p) cudaFree(p); } } guard{buf};
  double* vi = buf;
  double* vin = buf + ntot;
  double* vnew = buf + 2 * ntot;
  double* rho = buf + 3 * ntot;
  e = cudaMemcpyAsync(vi, vion, sizeof(double) * ntot, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vin, vi, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "scf start");
  SCF_TRY(pw_ctx_set_vloc(ctx, vin));
  std::vector<double> w(nocc, 2.0 / omega);
  int it = 0;
  bool conv = false;
  for (; it < max_iter; ++it) {
    SCF_TRY(pw_chebfi_solve(ctx, psi, ld, nband, degree, cycles, 10, v0, precision, eig, nullptr, nullptr));
    SCF_TRY(pw_density_grad(ctx, psi, nullptr, ld, nocc, w.data(), rho, 0));
    double s[5];
    SCF_TRY(pw_scf_potential(dctx, rho, vi, vin, beta, vnew, s));
    double eb = 0.0;
    for (int i = 0; i < nocc; ++i) eb += 2.0 * eig[i];
    if (history) {
      history[2 * it] = eb - s[0] + s[1] + s[2];
      history[2 * it + 1] = s[3];
    }
    if (s[3] < tol) {
      conv = true;
      ++it;
      break;
    }
    std::swap(vin, vnew);
    SCF_TRY(pw_ctx_set_vloc(ctx, vin));
  }
  if (iterations) *iterations = it;
  if (!conv) return set_error(PW_ENOTCONV, "SCF not converged in %d iterations", max_iter);
  return PW_OK;
}
