// Differentiation form of the ChebFi cycle: a taped forward (Chebyshev filter of
// Sec. 3.3 / Alg. 12, two S-Ortho passes of Alg. 9, Rayleigh-Ritz of Alg. 5, for
// S = I) and its hand-written reverse-mode adjoint, giving dL/dV_loc(r_j) and
// dL/dD_ab from the adjoints of the Ritz values and Ritz vectors.
//
// Gradient convention (PyTorch's, complex): the adjoint of a complex block Z is
// Zb = dL/dRe Z + i dL/dIm Z, so dL = Re tr(Zb^H dZ).  Per cycle, going backwards:
//   K = Psi^H Psib,  G_ij = K_ij / (lam_j - lam_i) on kept pairs, G_ii = lamb_i,
//   Ab = Herm(X G X^H)                                      (Hermitian eigen-adjoint)
//   Qb = Psib X^H + 2 H Q Ab;  dV += (1/n) Re[conj(Q Ab)(r) Q(r)];  dD += Re[(P^H Q Ab)(P^H Q)^H]
//   Ym_b = (I - Q Q^H) Qb R^-H,  R = Q^H Y_m                (the cycle sees Y_m only through its span)
//   Z_m = Ym_b,  Z_k = alpha_k (H - c) Z_{k+1} - Z_{k+2},   alpha_0 = 1/e, alpha_k = 2/e
//   dV += (alpha_k/n) Re[conj(Z_{k+1})(r) Y_k(r)],  dD += alpha_k Re[(P^H Z_{k+1})(P^H Y_k)^H]
//   Psib of the previous cycle = Z_0.
// The filter cut a and the Lanczos bound b are held fixed (not differentiated).
// Earlier cycles keep no eigenvector-coupling pair: the next cycle depends on their
// Ritz vectors only through the span, so those terms vanish identically.
//
// Recurrence checkpointing: the forward keeps the pairs (Y_{js}, Y_{js+1}) of every
// segment of s = ckpt steps (and P^dagger Y_k for every k, which is small); the backward
// recomputes the other iterates of a segment from its pair when it reaches it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "api.cuh"
#include "la.cuh"
#include "pw_internal.cuh"
#include "setup.cuh"

namespace pw {
namespace {

// G (m x m, column-major) from K = Psi^H Psib: G_ij = K_ij / (lam_j - lam_i) for kept
// pairs i != j (zero when the two values coincide exactly), G_ii = lamb_i (0 if lamb NULL).
// keep: split < 0 -> every pair; else pairs with exactly one index below split.
__global__ void k_eig_adjoint(const double2* __restrict__ K, const double* __restrict__ lam,
                              const double* __restrict__ lamb, int m, int split, double2* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= m || j >= m) return;
  double2 g = make_double2(0.0, 0.0);
  if (i == j) {
    g.x = lamb ? lamb[i] : 0.0;
  } else {
    const bool keep = split < 0 || ((i < split) != (j < split));
    const double gap = lam[j] - lam[i];
    if (keep && gap != 0.0) {
      const double2 k = K[i + (int64_t)j * m];
      g = make_double2(k.x / gap, k.y / gap);
    }
  }
  G[i + (int64_t)j * m] = g;
}

template <typename T>
__global__ void k_fill(T* __restrict__ w, int n, T v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = v;
}

// out (+)= Re(acc), n entries
__global__ void k_real_part(const double2* __restrict__ acc, int64_t n, double* __restrict__ out, int accumulate) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = accumulate ? out[i] + acc[i].x : acc[i].x;
}

}  // namespace
}  // namespace pw

using namespace pw;

struct pw_diff {
  pw_ctx* ctx = nullptr;
  int M = 0, m = 0, cycles = 0, ckpt = 1, precision = 0;
  size_t esz = 16;  // bytes per complex element of the filter blocks (16: complex128, 8: complex64)
  uint64_t param_gen = 0;
  bool taped = false;
  double upper = 0;
  std::vector<double> cuts, cc, ee;
  std::vector<void*> owned;
  int64_t bytes = 0;
  // tape: per cycle and step k < m, the stored iterate Y_k (or NULL) and P^dagger Y_k
  std::vector<void*> ytape, ctape;
  std::vector<double2*> Qt, Xt, Lt;  // Q (N x M), X (M x M), (R^H)^-1 (M x M) per cycle
  std::vector<double*> lamt;         // Ritz values per cycle (device)
  // work blocks (element type of the precision) and FP64 buffers
  void* work[3] = {nullptr, nullptr, nullptr};
  void* ym = nullptr;
  std::vector<void*> seg;  // recomputed iterates of one segment (ckpt - 2 blocks)
  void* zb[3] = {nullptr, nullptr, nullptr};
  double2 *HQ = nullptr, *PB = nullptr, *QB = nullptr, *QA = nullptr, *Y64 = nullptr;
  double2 *mK = nullptr, *mT = nullptr, *mG = nullptr, *mA = nullptr;
  double2 *CQ = nullptr, *CA = nullptr, *cz64 = nullptr, *ck64 = nullptr, *dDacc = nullptr, *gsplit = nullptr;
  void* cz = nullptr;
  double* den = nullptr;
  double* lamb = nullptr;
  void* wdev = nullptr;
  std::vector<double> eig_h;
};

namespace {

#define PW_TRY(expr)            \
  do {                          \
    int _s = (expr);            \
    if (_s != PW_OK) return _s; \
  } while (0)
#define CU_TRY(expr, where)                                                          \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) {                                                         \
      ctx->poisoned = true;                                                          \
      return cuda_status(_e, where);                                                 \
    }                                                                                \
  } while (0)

template <typename X>
int dalloc(pw_diff* df, X** p, size_t n) {
  void* q = nullptr;
  const size_t b = sizeof(X) * std::max<size_t>(n, 1);
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_status(e, "differentiation tape allocation");
  }
  df->owned.push_back(q);
  df->bytes += (int64_t)b;
  *p = (X*)q;
  return PW_OK;
}

bool stored(const pw_diff* df, int k) { return df->ckpt <= 1 || (k % df->ckpt) < 2; }

int create_impl(pw_ctx* ctx, int M, int m, int cycles, int ckpt, int precision, pw_diff** out) {
  pw_diff* df = new (std::nothrow) pw_diff();
  if (!df) return set_error(PW_ENOMEM, "host allocation");
  *out = df;
  df->ctx = ctx;
  df->M = M;
  df->m = m;
  df->cycles = cycles;
  df->ckpt = std::max(1, ckpt);
  df->precision = precision;
  df->esz = precision == PW_MIXED ? 8 : 16;
  const size_t N = (size_t)ctx->npw, np = (size_t)std::max(ctx->nproj, 1);
  const size_t blk = N * M * df->esz;
  df->ytape.assign((size_t)cycles * m, nullptr);
  df->ctape.assign((size_t)cycles * m, nullptr);
  for (int t = 0; t < cycles; ++t) {
    for (int k = 0; k < m; ++k) {
      unsigned char* p;
      if (stored(df, k)) {
        PW_TRY(dalloc(df, &p, blk));
        df->ytape[(size_t)t * m + k] = p;
      }
      PW_TRY(dalloc(df, &p, np * M * df->esz));
      df->ctape[(size_t)t * m + k] = p;
    }
    double2 *q, *x, *l;
    double* lam;
    PW_TRY(dalloc(df, &q, N * M));
    PW_TRY(dalloc(df, &x, (size_t)M * M));
    PW_TRY(dalloc(df, &l, (size_t)M * M));
    PW_TRY(dalloc(df, &lam, (size_t)M));
    df->Qt.push_back(q);
    df->Xt.push_back(x);
    df->Lt.push_back(l);
    df->lamt.push_back(lam);
  }
  unsigned char* p;
  for (int i = 0; i < 3; ++i) {
    PW_TRY(dalloc(df, &p, blk));
    df->work[i] = p;
    PW_TRY(dalloc(df, &p, blk));
    df->zb[i] = p;
  }
  PW_TRY(dalloc(df, &p, blk));
  df->ym = p;
  for (int i = 0; i + 2 < df->ckpt; ++i) {
    PW_TRY(dalloc(df, &p, blk));
    df->seg.push_back(p);
  }
  PW_TRY(dalloc(df, &df->HQ, N * M));
  PW_TRY(dalloc(df, &df->PB, N * M));
  PW_TRY(dalloc(df, &df->QB, N * M));
  PW_TRY(dalloc(df, &df->QA, N * M));
  PW_TRY(dalloc(df, &df->Y64, N * M));
  PW_TRY(dalloc(df, &df->mK, (size_t)M * M));
  PW_TRY(dalloc(df, &df->mT, (size_t)M * M));
  PW_TRY(dalloc(df, &df->mG, (size_t)M * M));
  PW_TRY(dalloc(df, &df->mA, (size_t)M * M));
  PW_TRY(dalloc(df, &df->CQ, np * M));
  PW_TRY(dalloc(df, &df->CA, np * M));
  PW_TRY(dalloc(df, &df->cz64, np * M));
  PW_TRY(dalloc(df, &df->ck64, np * M));
  PW_TRY(dalloc(df, &df->dDacc, np * np));
  const int ns = api::gemm_nsplit(M, M, ctx->npw);
  PW_TRY(dalloc(df, &df->gsplit, (size_t)std::max(ns, api::gemm_nsplit((int)np, M, ctx->npw)) *
                                     std::max((size_t)M * M, np * M)));
  PW_TRY(dalloc(df, &p, np * M * df->esz));
  df->cz = p;
  PW_TRY(dalloc(df, &df->den, (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2]));
  PW_TRY(dalloc(df, &df->lamb, (size_t)M));
  PW_TRY(dalloc(df, &p, (size_t)M * 8));
  df->wdev = p;
  df->eig_h.assign(M, 0.0);
  return PW_OK;
}

// The context may already be gone (the handle only borrows it); cudaFree waits for the
// device, so nothing of the context is touched here.
void destroy(pw_diff* df) {
  if (!df) return;
  for (void* p : df->owned) cudaFree(p);
  delete df;
}

// complex128 <-> filter element type copies of N x M blocks
template <typename T>
cudaError_t to_t(const double2* a, int64_t lda, cplx<T>* b, int64_t ldb, int n, int m, cudaStream_t st) {
  if constexpr (std::is_same<T, double>::value)
    return cudaMemcpy2DAsync(b, sizeof(double2) * ldb, a, sizeof(double2) * lda, sizeof(double2) * n, m,
                             cudaMemcpyDeviceToDevice, st);
  else
    return la_to_c64(a, lda, b, ldb, n, m, st);
}
template <typename T>
cudaError_t from_t(const cplx<T>* a, int64_t lda, double2* b, int64_t ldb, int n, int m, cudaStream_t st) {
  if constexpr (std::is_same<T, double>::value)
    return cudaMemcpy2DAsync(b, sizeof(double2) * ldb, a, sizeof(double2) * lda, sizeof(double2) * n, m,
                             cudaMemcpyDeviceToDevice, st);
  else
    return la_to_c128(a, lda, b, ldb, n, m, st);
}

Epi<double> epi64(int mode, double2* out, int64_t ldo, double alpha = 1.0) {
  Epi<double> e;
  e.mode = mode; e.out = out; e.ldo = ldo; e.alpha = alpha; e.beta = 0; e.shift = 0;
  e.yk = nullptr; e.ykm1 = nullptr; e.ldy = 0; e.ldy2 = 0; e.dev_ce = nullptr; e.first = 0;
  return e;
}

// location of Y_k during the forward: its tape slot when stored, else a rotating work block
template <typename T>
cplx<T>* fwd_loc(pw_diff* df, int t, int k) {
  if (k == df->m) return (cplx<T>*)df->ym;
  void* p = df->ytape[(size_t)t * df->m + k];
  return (cplx<T>*)(p ? p : df->work[k % 3]);
}

template <typename T>
int forward_t(pw_diff* df, double2* psi, int64_t ld, int steps, const double2* v0, const double* bounds_in,
              double* eig, double* bounds_out) {
  pw_ctx* ctx = df->ctx;
  const int M = df->M, m = df->m, N = ctx->npw;
  const cudaStream_t st = ctx->stream;
  double a = 0;
  if (bounds_in) {
    df->upper = bounds_in[0];
  } else {
    PW_TRY(api::bounds(ctx, psi, ld, M, steps, v0, &a, &df->upper));
  }
  df->cuts.assign(df->cycles, 0.0);
  df->cc.assign(df->cycles, 0.0);
  df->ee.assign(df->cycles, 0.0);
  for (int t = 0; t < df->cycles; ++t) {
    if (bounds_in) a = bounds_in[1 + t];
    if (!(df->upper > a)) return set_error(PW_EINVAL, "filter interval needs upper > cut (cycle %d: a=%g, b=%g)", t, a,
                                           df->upper);
    df->cuts[t] = a;
    const double c = 0.5 * (df->upper + a), e = 0.5 * (df->upper - a);
    df->cc[t] = c;
    df->ee[t] = e;
    CU_TRY(to_t<T>(psi, ld, fwd_loc<T>(df, t, 0), N, N, M, st), "filter input");
    for (int k = 0; k < m; ++k) {
      const double alpha = (k == 0 ? 1.0 : 2.0) / e;
      PW_TRY(api::recur<T>(ctx, fwd_loc<T>(df, t, k), N, k > 0 ? fwd_loc<T>(df, t, k - 1) : nullptr, N,
                           fwd_loc<T>(df, t, k + 1), N, M, alpha, 1.0, c,
                           (cplx<T>*)df->ctape[(size_t)t * m + k]));
    }
    CU_TRY(from_t<T>((const cplx<T>*)df->ym, N, psi, ld, N, M, st), "filter output");
    CU_TRY(cudaMemcpy2DAsync(df->Y64, sizeof(double2) * N, psi, sizeof(double2) * ld, sizeof(double2) * N, M,
                             cudaMemcpyDeviceToDevice, st), "keep Y_m");
    PW_TRY(api::rr(ctx, psi, ld, M, df->eig_h.data(), df->Qt[t], df->Xt[t], df->lamt[t]));
    // R^H = Y_m^H Q (lower triangular), kept as its inverse
    const int ns = api::gemm_nsplit(M, M, N);
    CU_TRY(launch_cgemm<double>(1, 0, M, M, N, df->Y64, N, df->Qt[t], N, epi64(EPI_STORE, df->mT, M), ns, df->gsplit,
                                st), "R^H");
    CU_TRY(la_zero_upper(df->mT, M, M, st), "R^H lower");
    CU_TRY(la_trinv_lower(df->mT, M, M, df->Lt[t], M, df->mG, st), "R^H inverse");
    a = df->eig_h[M - 1];
  }
  if (eig) memcpy(eig, df->eig_h.data(), sizeof(double) * M);
  if (bounds_out) {
    bounds_out[0] = df->upper;
    for (int t = 0; t < df->cycles; ++t) bounds_out[1 + t] = df->cuts[t];
  }
  CU_TRY(cudaStreamSynchronize(st), "forward sync");
  df->taped = true;
  df->param_gen = ctx->param_gen;
  return PW_OK;
}

// accumulates weight * Re[conj(a)(r) b(r)] into the permuted grid and weight * (P^H a)(P^H b)^H into dDacc
template <typename T>
int contract(pw_diff* df, const cplx<T>* a, const cplx<T>* b, const cplx<T>* Ca, const cplx<T>* Cb, double weight) {
  pw_ctx* ctx = df->ctx;
  const int M = df->M, np = ctx->nproj;
  const cudaStream_t st = ctx->stream;
  const double n = (double)ctx->n[0] * ctx->n[1] * ctx->n[2];
  k_fill<T><<<(M + 127) / 128, 128, 0, st>>>((T*)df->wdev, M, (T)(weight / n));
  count_launch();
  const int bb = std::max(1, api::fft_band_batch(ctx, M, sizeof(cplx<T>)) / 2);
  const int64_t hb_bs = (int64_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2];
  int status = PW_OK;
  cplx<T>* hb = (cplx<T>*)ws_get(ctx, WS_HB, sizeof(cplx<T>) * (size_t)hb_bs * bb * 2, &status);
  if (!hb) return status;
  const cplx<T>* tw;
  if constexpr (std::is_same<T, double>::value) tw = ctx->tw64; else tw = ctx->tw32;
  CU_TRY(launch_density<T>(ctx->plan, tw, ctx->sp, a, b, ctx->npw, M, (const T*)df->wdev, df->den, hb, bb, st),
         "adjoint density contraction");
  if (np > 0) {
    const double2 *ca64, *cb64;
    if constexpr (std::is_same<T, double>::value) {
      ca64 = Ca;
      cb64 = Cb;
    } else {
      CU_TRY(la_to_c128(Ca, np, df->cz64, np, np, M, st), "projection cast");
      CU_TRY(la_to_c128(Cb, np, df->ck64, np, np, M, st), "projection cast");
      ca64 = df->cz64;
      cb64 = df->ck64;
    }
    CU_TRY(launch_cgemm<double>(0, 1, np, np, M, ca64, np, cb64, np, epi64(EPI_ACCUM, df->dDacc, np, weight), 1,
                                nullptr, st), "adjoint D contraction");
  }
  return PW_OK;
}

template <typename T>
int backward_t(pw_diff* df, const double* eigbar, const double2* psibar, int64_t ldb, int split, double* dV,
               double* dD, int accumulate) {
  pw_ctx* ctx = df->ctx;
  using C = cplx<T>;
  const int M = df->M, m = df->m, N = ctx->npw, np = ctx->nproj;
  const cudaStream_t st = ctx->stream;
  const size_t ntot = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  CU_TRY(cudaMemsetAsync(df->den, 0, sizeof(double) * ntot, st), "adjoint grid reset");
  CU_TRY(cudaMemsetAsync(df->dDacc, 0, sizeof(double2) * (size_t)std::max(np, 1) * std::max(np, 1), st),
         "adjoint D reset");
  if (psibar)
    CU_TRY(cudaMemcpy2DAsync(df->PB, sizeof(double2) * N, psibar, sizeof(double2) * ldb, sizeof(double2) * N, M,
                             cudaMemcpyDeviceToDevice, st), "Psi adjoint");
  else
    CU_TRY(cudaMemsetAsync(df->PB, 0, sizeof(double2) * (size_t)N * M, st), "Psi adjoint reset");
  const bool have_lb = eigbar != nullptr;
  if (have_lb) CU_TRY(cudaMemcpyAsync(df->lamb, eigbar, sizeof(double) * M, cudaMemcpyHostToDevice, st), "eig adjoint");
  const int ns = api::gemm_nsplit(M, M, N);
  const dim3 b2(16, 16), g2((M + 15) / 16, (M + 15) / 16);
  for (int t = df->cycles - 1; t >= 0; --t) {
    const bool last = (t == df->cycles - 1);
    const double2 *Q = df->Qt[t], *X = df->Xt[t];
    // Qb = Psib X^H
    CU_TRY(launch_cgemm<double>(0, 1, N, M, M, df->PB, N, X, M, epi64(EPI_STORE, df->QB, N), 1, nullptr, st),
           "Qb = Psib X^H");
    const bool keep_any = split < 0 || (split > 0 && split < M);
    if (last && (have_lb || keep_any)) {
      // K = X^H (Q^H Psib); G; Ab = Herm(X G X^H)
      CU_TRY(launch_cgemm<double>(1, 0, M, M, N, Q, N, df->PB, N, epi64(EPI_STORE, df->mT, M), ns, df->gsplit, st),
             "Q^H Psib");
      CU_TRY(launch_cgemm<double>(1, 0, M, M, M, X, M, df->mT, M, epi64(EPI_STORE, df->mK, M), 1, nullptr, st),
             "K");
      k_eig_adjoint<<<g2, b2, 0, st>>>(df->mK, df->lamt[t], have_lb ? df->lamb : nullptr, M, split, df->mG);
      count_launch();
      CU_TRY(launch_cgemm<double>(0, 1, M, M, M, df->mG, M, X, M, epi64(EPI_STORE, df->mT, M), 1, nullptr, st),
             "G X^H");
      CU_TRY(launch_cgemm<double>(0, 0, M, M, M, X, M, df->mT, M, epi64(EPI_STORE, df->mA, M), 1, nullptr, st),
             "X G X^H");
      CU_TRY(la_herm_sym(df->mA, M, M, st), "Ab Hermitian part");
      // Qb += 2 H Q Ab ; direct parameter terms of A = Q^H H Q
      PW_TRY(api::apply64(ctx, Q, N, M, df->HQ, N));
      CU_TRY(launch_cgemm<double>(0, 0, N, M, M, df->HQ, N, df->mA, M, epi64(EPI_ACCUM, df->QB, N, 2.0), 1, nullptr,
                                  st), "Qb += 2 HQ Ab");
      CU_TRY(launch_cgemm<double>(0, 0, N, M, M, Q, N, df->mA, M, epi64(EPI_STORE, df->QA, N), 1, nullptr, st),
             "Q Ab");
      if (np > 0) {
        const int nsp = api::gemm_nsplit(np, M, N);
        CU_TRY(launch_cgemm<double>(1, 0, np, M, N, ctx->P64, N, df->QA, N, epi64(EPI_STORE, df->CA, np), nsp,
                                    df->gsplit, st), "P^H Q Ab");
        CU_TRY(launch_cgemm<double>(1, 0, np, M, N, ctx->P64, N, Q, N, epi64(EPI_STORE, df->CQ, np), nsp,
                                    df->gsplit, st), "P^H Q");
      }
      PW_TRY(contract<double>(df, df->QA, Q, df->CA, df->CQ, 1.0));
    }
    // span projection and R^-H:  Ym_b = (Qb - Q (Q^H Qb)) (R^H)^-1
    CU_TRY(launch_cgemm<double>(1, 0, M, M, N, Q, N, df->QB, N, epi64(EPI_STORE, df->mT, M), ns, df->gsplit, st),
           "Q^H Qb");
    CU_TRY(launch_cgemm<double>(0, 0, N, M, M, Q, N, df->mT, M, epi64(EPI_ACCUM, df->QB, N, -1.0), 1, nullptr, st),
           "project out span");
    CU_TRY(launch_cgemm<double>(0, 0, N, M, M, df->QB, N, df->Lt[t], M, epi64(EPI_STORE, df->HQ, N), 1, nullptr, st),
           "Ym_b");
    // adjoint recurrence, from Z_m down to Z_0
    C* zbuf[3] = {(C*)df->zb[0], (C*)df->zb[1], (C*)df->zb[2]};
    auto zl = [&](int k) { return zbuf[k % 3]; };
    CU_TRY(to_t<T>(df->HQ, N, zl(m), N, N, M, st), "Z_m");
    const double c = df->cc[t], e = df->ee[t];
    int seg_lo = -1;  // first step of the segment whose iterates are in df->seg
    for (int k = m - 1; k >= 0; --k) {
      const C* yk;
      if (df->ytape[(size_t)t * m + k]) {
        yk = (const C*)df->ytape[(size_t)t * m + k];
      } else {
        const int s = df->ckpt, j0 = (k / s) * s;
        if (seg_lo != j0) {
          // recompute Y_{j0+2} .. Y_{min(j0+s, m)-1} from the stored pair (Y_{j0}, Y_{j0+1})
          const int hi = std::min(j0 + s, m) - 1;
          for (int q = j0 + 2; q <= hi; ++q) {
            auto loc = [&](int i) -> C* {
              return i < j0 + 2 ? (C*)df->ytape[(size_t)t * m + i] : (C*)df->seg[i - j0 - 2];
            };
            PW_TRY(api::recur<T>(ctx, loc(q - 1), N, loc(q - 2), N, loc(q), N, M, 2.0 / e, 1.0, c, nullptr));
          }
          seg_lo = j0;
        }
        yk = (const C*)df->seg[k - j0 - 2];
      }
      const double alpha = (k == 0 ? 1.0 : 2.0) / e;
      // Z_k = alpha (H - c) Z_{k+1} - Z_{k+2};  cz = P^H Z_{k+1}
      PW_TRY(api::recur<T>(ctx, zl(k + 1), N, (k + 2 <= m) ? zl(k + 2) : nullptr, N, zl(k), N, M, alpha, 1.0, c,
                           (C*)df->cz));
      PW_TRY(contract<T>(df, zl(k + 1), yk, (const C*)df->cz, (const C*)df->ctape[(size_t)t * m + k], alpha));
    }
    CU_TRY(from_t<T>(zl(0), N, df->PB, N, N, M, st), "Psi adjoint of the previous cycle");
  }
  if (dV) CU_TRY(setup_unperm(df->den, ctx->n, ctx->rho_perm, dV, accumulate, st), "dV unpermute");
  if (dD && np > 0) {
    const int64_t nn = (int64_t)np * np;
    k_real_part<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(df->dDacc, nn, dD, accumulate);
    count_launch();
    CU_TRY(cudaGetLastError(), "dD");
  }
  CU_TRY(cudaStreamSynchronize(st), "backward sync");
  return PW_OK;
}

}  // namespace

extern "C" {

PW_API int pw_ctx_set_vloc(pw_ctx* ctx, const double* vloc) {
  PW_TRY(api::check(ctx));
  if (!vloc) return set_error(PW_EINVAL, "vloc is NULL");
  const cudaStream_t st = ctx->stream;
  const size_t ntot = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  int status = PW_OK;
  double* raw = (double*)ws_get(ctx, WS_VPOT, sizeof(double) * ntot, &status);
  if (!raw) return status;
  CU_TRY(cudaMemcpyAsync(raw, vloc, sizeof(double) * ntot, cudaMemcpyDefault, st), "vloc copy");
  CU_TRY(setup_vperm(raw, ctx->n, ctx->rho_perm, 1.0 / (double)ntot, ctx->vperm64, ctx->vperm32, st), "vperm");
  if (ctx->vperm32_sw) {
    int* rho_sw[3] = {ctx->rho_x_sw, ctx->rho_perm[1], ctx->rho_perm[2]};
    CU_TRY(setup_vperm32(raw, ctx->n, rho_sw, 1.0 / (double)ntot, ctx->vperm32_sw, st), "vperm (swapped x plan)");
  }
  CU_TRY(cudaStreamSynchronize(st), "vloc sync");
  ctx->param_gen++;
  return PW_OK;
}

PW_API int pw_ctx_set_D(pw_ctx* ctx, const double* D) {
  PW_TRY(api::check(ctx));
  if (!D) return set_error(PW_EINVAL, "D is NULL");
  if (ctx->has_q) return set_error(PW_EUNSUPPORTED, "replacing D needs S = I (the Woodbury E depends on D)");
  const int np = ctx->nproj;
  if (np == 0) return PW_OK;
  std::vector<double> h((size_t)np * np);
  CU_TRY(cudaMemcpy(h.data(), D, sizeof(double) * h.size(), cudaMemcpyDefault), "D copy");
  for (int j = 0; j < np; ++j)
    for (int i = 0; i < np; ++i) {
      const bool inside = ctx->blk0_h[i] == ctx->blk0_h[j];
      if (!inside && h[i + (size_t)j * np] != 0.0)
        return set_error(PW_EINVAL, "D(%d,%d) lies outside the context's D blocks", i, j);
    }
  const cudaStream_t st = ctx->stream;
  CU_TRY(cudaMemcpyAsync(ctx->D64, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st), "D upload");
  CU_TRY(cast_d2f(ctx->D64, ctx->D32, (int64_t)h.size(), st), "D cast");
  CU_TRY(cudaStreamSynchronize(st), "D sync");
  ctx->param_gen++;
  return PW_OK;
}

PW_API int pw_local_apply(pw_ctx* ctx, const double* v, double alpha, const void* psi, int64_t ld, int nband,
                          void* out, int64_t ldo, int precision) {
  PW_TRY(api::check(ctx));
  PW_TRY(api::check_blk(ctx, psi, ld, nband));
  if (!v || (nband > 0 && !out)) return set_error(PW_EINVAL, "NULL potential or output");
  if (ldo < ctx->npw) return set_error(PW_EINVAL, "ldo < npw");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  if (nband == 0) return PW_OK;
  const cudaStream_t st = ctx->stream;
  const size_t ntot = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  const size_t npw = (size_t)ctx->npw;
  int status = PW_OK;
  // [permuted V/n in FP64 | in FP32 | zero kinetic FP64 | FP32]
  unsigned char* w = (unsigned char*)ws_get(ctx, WS_VPOT, 12 * ntot + 12 * npw + 64, &status);
  if (!w) return status;
  double* vp64 = (double*)w;
  float* vp32 = (float*)(w + 8 * ntot);
  double* k64 = (double*)(w + ((12 * ntot + 15) / 16) * 16);
  float* k32 = (float*)(k64 + npw);
  CU_TRY(setup_vperm(v, ctx->n, ctx->rho_perm, alpha / (double)ntot, vp64, vp32, st), "potential permute");
  CU_TRY(cudaMemsetAsync(k64, 0, 12 * npw, st), "zero kinetic");
  if (precision == PW_FP64) {
    const int bb = api::fft_band_batch(ctx, nband, 16);
    const int64_t hb_bs = (int64_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2];
    double2* hb = (double2*)ws_get(ctx, WS_HB, sizeof(double2) * (size_t)hb_bs * bb, &status);
    if (!hb) return status;
    CU_TRY(launch_local_apply<double>(ctx->plan, ctx->tw64, ctx->sp, vp64, k64, (const double2*)psi, ld, nband,
                                      (double2*)out, ldo, hb, bb, st, ctx), "local apply");
  } else {
    const int bb = api::fft_band_batch(ctx, nband, 8);
    const int64_t hb_bs = (int64_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2];
    float2* hb = (float2*)ws_get(ctx, WS_HB, sizeof(float2) * (size_t)hb_bs * bb, &status);
    if (!hb) return status;
    CU_TRY(launch_local_apply<float>(ctx->plan, ctx->tw32, ctx->sp, vp32, k32, (const float2*)psi, ld, nband,
                                     (float2*)out, ldo, hb, bb, st, ctx), "local apply");
  }
  return PW_OK;
}

PW_API int pw_diff_create(pw_ctx* ctx, int nband, int degree, int cycles, int ckpt, int precision, pw_diff** out) {
  PW_TRY(api::check(ctx));
  if (!out) return set_error(PW_EINVAL, "NULL output");
  *out = nullptr;
  if (nband <= 0 || degree <= 0 || cycles <= 0) return set_error(PW_EINVAL, "nband, degree and cycles must be positive");
  if (ckpt < 0) return set_error(PW_EINVAL, "checkpoint interval must be >= 0");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  if (ctx->has_q) return set_error(PW_EUNSUPPORTED, "the differentiation form needs S = I (Q == NULL)");
  if (nband > ctx->npw) return set_error(PW_EINVAL, "nband > npw");
  pw_diff* df = nullptr;
  const int s = create_impl(ctx, nband, degree, cycles, ckpt, precision, &df);
  if (s != PW_OK) {
    destroy(df);
    return s;
  }
  *out = df;
  return PW_OK;
}

PW_API int pw_diff_destroy(pw_diff* df) {
  destroy(df);
  return PW_OK;
}

PW_API int pw_diff_tape_bytes(const pw_diff* df, int64_t* bytes) {
  if (!df || !bytes) return set_error(PW_EINVAL, "NULL argument");
  *bytes = df->bytes;
  return PW_OK;
}

PW_API int pw_diff_forward(pw_diff* df, void* psi, int64_t ld, int lanczos_steps, const void* v0,
                           const double* bounds_in, double* eig, double* bounds_out) {
  if (!df) return set_error(PW_EINVAL, "NULL differentiation handle");
  pw_ctx* ctx = df->ctx;
  PW_TRY(api::check(ctx));
  PW_TRY(api::check_blk(ctx, psi, ld, df->M));
  if (!bounds_in && (lanczos_steps <= 0 || !v0)) return set_error(PW_EINVAL, "no bounds and no Lanczos start vector");
  df->taped = false;
  if (df->precision == PW_MIXED)
    return forward_t<float>(df, (double2*)psi, ld, lanczos_steps, (const double2*)v0, bounds_in, eig, bounds_out);
  return forward_t<double>(df, (double2*)psi, ld, lanczos_steps, (const double2*)v0, bounds_in, eig, bounds_out);
}

PW_API int pw_diff_backward(pw_diff* df, const double* eig_bar, const void* psi_bar, int64_t ld, int split, double* dV,
                            double* dD, int accumulate) {
  if (!df) return set_error(PW_EINVAL, "NULL differentiation handle");
  pw_ctx* ctx = df->ctx;
  PW_TRY(api::check(ctx));
  if (!df->taped) return set_error(PW_EINVAL, "no forward tape (pw_diff_forward first)");
  if (ctx->param_gen != df->param_gen) return set_error(PW_EINVAL, "V_loc or D changed since the forward");
  if (psi_bar) PW_TRY(api::check_blk(ctx, psi_bar, ld, df->M));
  if (split > df->M) return set_error(PW_EINVAL, "split > nband");
  if (df->precision == PW_MIXED)
    return backward_t<float>(df, eig_bar, (const double2*)psi_bar, ld, split, dV, dD, accumulate);
  return backward_t<double>(df, eig_bar, (const double2*)psi_bar, ld, split, dV, dD, accumulate);
}

}  // extern "C"
