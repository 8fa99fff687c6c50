// Gamma-point pairing of bands that are real in r-space: two such bands travel as one
// complex band, so the filter's FFTs and projector GEMMs run on half as many bands.
//
// At k = 0 the plane-wave sphere is symmetric under G -> -G and, in the canonical order
// (Miller indices ascending lexicographically), negation reverses the order: the partner of
// index i is npw - 1 - i.  A function real in r-space has c(-G) = conj c(G).  H maps such
// functions to such functions when V_loc, D and Q are real and the projectors satisfy
// P(-G) = conj P(G) (true for the generated s/p projectors: real radial form factors times
// (-i) q_a for p and the phase e^{-i G.R}).  H is linear, so for c = a + i b,
// H c = H a + i H b, and any polynomial p(A) of A = S^-1 H gives p(A) c = p(A) a + i p(A) b:
// the Chebyshev filter of 2 m such bands is the filter of m packed bands.  Unpacking uses
// a(G) = (c(G) + conj c(-G)) / 2 and b(G) = (c(G) - conj c(-G)) / (2 i).
#include "pw_internal.cuh"

namespace pw {
namespace {

// psi <- (psi(G) + conj psi(-G)) / 2, pairs (i, npw - 1 - i) handled by one thread
template <typename C>
__global__ void k_gamma_sym(C* __restrict__ psi, int64_t ld, int npw, int nband) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int half = (npw + 1) / 2;
  if (idx >= (int64_t)half * nband) return;
  const int i = (int)(idx % half), j = (int)(idx / half);
  C* p = psi + (int64_t)j * ld;
  const int m = npw - 1 - i;
  const C v = p[i], w = p[m];
  C r;
  r.x = 0.5f * (v.x + w.x);
  r.y = 0.5f * (v.y - w.y);
  p[i] = r;
  r.y = -r.y;
  p[m] = r;  // conj of the partner's value (equal to r itself when i == m, where r.y = 0)
}

// c_j = a_{2j} + i a_{2j+1}
template <typename C>
__global__ void k_gamma_pack(const C* __restrict__ a, int64_t lda, int npw, int npair, C* __restrict__ c,
                             int64_t ldc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)npw * npair) return;
  const int i = (int)(idx % npw), j = (int)(idx / npw);
  const C x = a[(int64_t)(2 * j) * lda + i], y = a[(int64_t)(2 * j + 1) * lda + i];
  C r;
  r.x = x.x - y.y;
  r.y = x.y + y.x;
  c[(int64_t)j * ldc + i] = r;
}

// a_{2j}(G) = (c(G) + conj c(-G)) / 2, a_{2j+1}(G) = (c(G) - conj c(-G)) / (2 i)
template <typename C>
__global__ void k_gamma_unpack(const C* __restrict__ c, int64_t ldc, int npw, int npair, C* __restrict__ a,
                               int64_t lda) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)npw * npair) return;
  const int i = (int)(idx % npw), j = (int)(idx / npw);
  const C u = c[(int64_t)j * ldc + i], w = c[(int64_t)j * ldc + (npw - 1 - i)];
  C x, y;
  x.x = 0.5f * (u.x + w.x);
  x.y = 0.5f * (u.y - w.y);
  // d = u - conj w; d / (2 i) = (d.y, -d.x) / 2
  y.x = 0.5f * (u.y + w.y);
  y.y = -0.5f * (u.x - w.x);
  a[(int64_t)(2 * j) * lda + i] = x;
  a[(int64_t)(2 * j + 1) * lda + i] = y;
}

int gamma_check(pw_ctx* ctx, int precision) {
  if (!ctx) return set_error(PW_EINVAL, "NULL context");
  if (ctx->poisoned) return set_error(PW_ECUDA, "context poisoned by an earlier CUDA error");
  if (ctx->kpt[0] != 0.0 || ctx->kpt[1] != 0.0 || ctx->kpt[2] != 0.0)
    return set_error(PW_EINVAL, "Gamma-point pairing needs k = 0");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  return PW_OK;
}

template <typename C>
cudaError_t launch(int op, pw_ctx* ctx, const void* x, int64_t ldx, int n, void* y, int64_t ldy) {
  const int npw = ctx->npw;
  const cudaStream_t st = ctx->stream;
  if (op == 0) {
    const int64_t t = (int64_t)((npw + 1) / 2) * n;
    if (t > 0) { k_gamma_sym<C><<<(unsigned)((t + 255) / 256), 256, 0, st>>>((C*)y, ldy, npw, n); count_launch(); }
  } else {
    const int64_t t = (int64_t)npw * (n / 2);
    if (t <= 0) return cudaSuccess;
    if (op == 1) k_gamma_pack<C><<<(unsigned)((t + 255) / 256), 256, 0, st>>>((const C*)x, ldx, npw, n / 2, (C*)y, ldy);
    else k_gamma_unpack<C><<<(unsigned)((t + 255) / 256), 256, 0, st>>>((const C*)x, ldx, npw, n / 2, (C*)y, ldy);
    count_launch();
  }
  return cudaGetLastError();
}

int run(int op, pw_ctx* ctx, const void* x, int64_t ldx, int nband, void* y, int64_t ldy, int precision) {
  int s = gamma_check(ctx, precision);
  if (s != PW_OK) return s;
  if (nband < 0 || (op != 0 && nband % 2)) return set_error(PW_EINVAL, "pairing needs an even, non-negative nband");
  if ((op != 0 && !x) || !y) return set_error(PW_EINVAL, "NULL block");
  if ((op != 0 && ldx < ctx->npw) || ldy < ctx->npw) return set_error(PW_EINVAL, "ld < npw (%d)", ctx->npw);
  if (op != 0 && x == y) return set_error(PW_EINVAL, "input and output must not alias");
  const cudaError_t e = precision == PW_FP64 ? launch<double2>(op, ctx, x, ldx, nband, y, ldy)
                                             : launch<float2>(op, ctx, x, ldx, nband, y, ldy);
  if (e != cudaSuccess) {
    ctx->poisoned = true;
    return cuda_status(e, "Gamma pairing");
  }
  return PW_OK;
}

}  // namespace
}  // namespace pw

using namespace pw;

extern "C" PW_API int pw_gamma_symmetrize(pw_ctx* ctx, void* psi, int64_t ld, int nband, int precision) {
  return run(0, ctx, nullptr, 0, nband, psi, ld, precision);
}

extern "C" PW_API int pw_gamma_pack(pw_ctx* ctx, const void* a, int64_t lda, int nband, void* c, int64_t ldc,
                                    int precision) {
  return run(1, ctx, a, lda, nband, c, ldc, precision);
}

extern "C" PW_API int pw_gamma_unpack(pw_ctx* ctx, const void* c, int64_t ldc, int nband, void* a, int64_t lda,
                                      int precision) {
  return run(2, ctx, c, ldc, nband, a, lda, precision);
}
