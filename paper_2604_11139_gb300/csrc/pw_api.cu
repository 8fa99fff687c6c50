// C ABI of the Chebyshev-filtered plane-wave H-apply: context set-up (plane-wave
// sphere, FFT plans, projectors, Woodbury matrices) and the entry points of pw.h.
// Host code here only builds index and coefficient tables, sizes workspaces and
// sequences kernel launches; every arithmetic step of the path runs in the kernels
// of fft_local.cu, gemm_simt.cu, gemm_tc.cu, zgemm_tc.cu, la_fp64.cu and
// setup_kernels.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "la.cuh"
#include "pw_internal.cuh"
#include "setup.cuh"
#include "tc.cuh"
#include "zgemm.cuh"

namespace pw {

static thread_local char g_err[512] = "";

int set_error(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return PW_OK;
  const int s = (e == cudaErrorMemoryAllocation) ? PW_ENOMEM : PW_ECUDA;
  return set_error(s, "%s: %s", where, cudaGetErrorString(e));
}

void* ws_get(pw_ctx* c, int slot, size_t bytes, int* status) {
  if (slot < 0 || slot >= WS_NUM) {
    *status = set_error(PW_EINVAL, "workspace slot %d out of range", slot);
    return nullptr;
  }
  if (bytes == 0) bytes = 16;
  pw_ctx::Buf& b = c->ws[slot];
  if (b.bytes >= bytes) return b.p;
  if (b.p) {
    cudaStreamSynchronize(c->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    *status = cuda_status(e, "workspace allocation");
    return nullptr;
  }
  b.bytes = bytes;
  c->ws_gen++;
  return b.p;
}

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static cudaEvent_t prof_event(pw_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

void prof_begin(pw_ctx* c, int cls) {
  if (!c || !c->prof_on || (c->prof_suspend > 0 && cls != PW_PROF_RR)) return;
  cudaEvent_t e = prof_event(c);
  if (e) cudaEventRecord(e, c->stream);
  c->prof_open[cls] = e;
}

void prof_end(pw_ctx* c, int cls) {
  if (!c || !c->prof_on || !c->prof_open[cls] || (c->prof_suspend > 0 && cls != PW_PROF_RR)) return;
  cudaEvent_t e = prof_event(c);
  if (!e) return;
  cudaEventRecord(e, c->stream);
  c->prof_recs.push_back({cls, c->prof_open[cls], e});
  c->prof_open[cls] = nullptr;
}

struct ProfScope {
  pw_ctx* c;
  int cls;
  ProfScope(pw_ctx* c_, int cls_) : c(c_), cls(cls_) {
    prof_begin(c, cls);
    if (cls == PW_PROF_RR && c) c->prof_suspend++;
  }
  ~ProfScope() {
    if (cls == PW_PROF_RR && c) c->prof_suspend--;
    prof_end(c, cls);
  }
};

}  // namespace pw

using namespace pw;

#define PW_TRY(expr)                    \
  do {                                  \
    int _s = (expr);                    \
    if (_s != PW_OK) return _s;         \
  } while (0)
#define CU_TRY(expr, where)                                          \
  do {                                                               \
    cudaError_t _e = (expr);                                         \
    if (_e != cudaSuccess) { ctx->poisoned = true; return cuda_status(_e, where); } \
  } while (0)
#define WS(ptr, T, slot, count)                                               \
  T* ptr;                                                                     \
  do {                                                                        \
    int _st = PW_OK;                                                          \
    ptr = (T*)ws_get(ctx, slot, sizeof(T) * (size_t)(count), &_st);           \
    if (!ptr) return _st;                                                     \
  } while (0)

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// host-side planning
// ---------------------------------------------------------------------------
bool factorize(int n, FftDim& d) {
  const CPlan p = make_cplan(n);
  if (n < 1 || p.nst < 0 || (n > 1 && p.nst == 0)) return false;
  d.n = n;
  d.nst = p.nst;
  for (int s = 0; s < p.nst; ++s) {
    d.radix[s] = p.radix[s];
    d.L[s] = p.L[s];
  }
  return true;
}

// position j of a DIF output holds frequency rho(j)
std::vector<int> digit_reversal(const FftDim& d) {
  std::vector<int> r(d.n);
  for (int j = 0; j < d.n; ++j) {
    int t = j, f = 0, mult = 1, q = d.n;
    for (int s = 0; s < d.nst; ++s) {
      q /= d.radix[s];
      const int m = t / q;
      t %= q;
      f += m * mult;
      mult *= d.radix[s];
    }
    r[j] = f;
  }
  return r;
}

void block_structure(const double* A, int n, std::vector<int>& b0, std::vector<int>& bl) {
  b0.assign(n, 0);
  bl.assign(n, 0);
  int s = 0;
  while (s < n) {
    int e = s + 1, reach = s;
    for (int i = s; i < e; ++i) {
      for (int j = 0; j < n; ++j)
        if (A[i + (size_t)j * n] != 0.0 || A[j + (size_t)i * n] != 0.0) reach = std::max(reach, j);
      if (reach + 1 > e) e = reach + 1;
    }
    for (int i = s; i < e; ++i) { b0[i] = s; bl[i] = e - s; }
    s = e;
  }
}

void inv3(const double* a, double* out) {  // out = inverse of row-major 3x3
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  out[0] = (a[4] * a[8] - a[5] * a[7]) / det;
  out[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  out[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  out[3] = (a[5] * a[6] - a[3] * a[8]) / det;
  out[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  out[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  out[6] = (a[3] * a[7] - a[4] * a[6]) / det;
  out[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  out[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

template <typename X>
int upload(pw_ctx* ctx, X** dst, const X* src, size_t n) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(X) * std::max<size_t>(n, 1));
  if (e != cudaSuccess) return cuda_status(e, "context allocation");
  ctx->owned.push_back(p);
  *dst = (X*)p;
  if (src && n) {
    e = cudaMemcpy(p, src, sizeof(X) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e, "context upload");
  }
  return PW_OK;
}

// K splits for `tiles` output tiles: the SIMT GEMM holds 2 CTAs per SM (128 registers x 256
// threads), so tiles x splits stays within one wave of 2 x 152 CTAs
int nsplit_tiles(int tiles, int k) {
  int s = (2 * 152) / tiles;
  s = std::min(s, std::max(1, k / 512));
  return std::max(1, std::min(s, 64));
}
int nsplit_for(int m, int n, int k) { return nsplit_tiles(((m + 63) / 64) * ((n + 63) / 64), k); }

template <typename T> struct Prec;
template <> struct Prec<double> {
  static const double2* P(const pw_ctx* c) { return c->P64; }
  static const double* D(const pw_ctx* c) { return c->D64; }
  static const double* kin(const pw_ctx* c) { return c->kin64; }
  static const double* vp(const pw_ctx* c) { return c->vperm64; }
  static const double2* tw(const pw_ctx* c) { return c->tw64; }
  static const double2* K(const pw_ctx* c) { return c->K64; }
  static const double2* E(const pw_ctx* c) { return c->E64; }
  static const double2* B(const pw_ctx* c) { return c->B64; }
};
template <> struct Prec<float> {
  static const float2* P(const pw_ctx* c) { return c->P32; }
  static const float* D(const pw_ctx* c) { return c->D32; }
  static const float* kin(const pw_ctx* c) { return c->kin32; }
  static const float* vp(const pw_ctx* c) { return c->vperm32; }
  static const float2* tw(const pw_ctx* c) { return c->tw32; }
  static const float2* K(const pw_ctx* c) { return c->K32; }
  static const float2* E(const pw_ctx* c) { return c->E32; }
  static const float2* B(const pw_ctx* c) { return c->B32; }
};

template <typename T>
Epi<T> epi(int mode, cplx<T>* out, int64_t ldo, T alpha = 1) {
  Epi<T> e;
  e.mode = mode; e.out = out; e.ldo = ldo; e.alpha = alpha; e.beta = 0; e.shift = 0;
  e.yk = nullptr; e.ykm1 = nullptr; e.ldy = 0; e.ldy2 = 0;
  e.dev_ce = nullptr; e.first = 0;
  return e;
}

// Bands per FFT batch.  complex64: keep a batch's half-box planes near 48 MB so that
// pass 1 -> pass 2 -> pass 3 hand the planes over through the 129 MB L2 instead of
// HBM; complex128 (DFMA-bound) batches near 256 MB for fewer, larger launches.
int band_batch(const pw_ctx* ctx, int nband, size_t elem = 16) {
  const size_t per = (size_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2] * elem;
  const size_t target = ctx->fft_batch_bytes[elem == 8 ? 0 : 1];
  int bb = (int)std::max<size_t>(1, target / std::max<size_t>(per, 1));
  return std::max(1, std::min(bb, nband));
}

// ---------------------------------------------------------------------------
// tensor-core operands and helpers of the mixed path
// ---------------------------------------------------------------------------
int64_t round64(int64_t x) { return (x + 63) / 64 * 64; }

int ensure_tc(pw_ctx* ctx) {
  if (ctx->tc_built_pieces == ctx->tc_pieces && ctx->tcA1) return PW_OK;
  if (!tc::available()) return set_error(PW_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  const cudaStream_t st = ctx->stream;
  CU_TRY(cudaStreamSynchronize(st), "tc sync");
  if (ctx->tcA1) { cudaFree(ctx->tcA1); ctx->tcA1 = nullptr; }
  if (ctx->tcA2) { cudaFree(ctx->tcA2); ctx->tcA2 = nullptr; }
  const int np = ctx->nproj, npw = ctx->npw, pc = ctx->tc_pieces;
  ctx->kp1 = round64(2 * (int64_t)npw);
  ctx->kp2 = round64(2 * (int64_t)np);
  CU_TRY(cudaMalloc(&ctx->tcA1, sizeof(__nv_bfloat16) * (size_t)pc * 2 * np * ctx->kp1), "tc A1 allocation");
  CU_TRY(cudaMalloc(&ctx->tcA2, sizeof(__nv_bfloat16) * (size_t)pc * 2 * npw * ctx->kp2), "tc A2 allocation");
  if (!ctx->tc_err) {
    CU_TRY(cudaMalloc(&ctx->tc_err, sizeof(int)), "tc flag allocation");
    CU_TRY(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), st), "tc flag reset");
  }
  CU_TRY(tc::build_a(ctx->P64, npw, np, pc, (__nv_bfloat16*)ctx->tcA1, ctx->kp1, 2 * (int64_t)np * ctx->kp1,
                     (__nv_bfloat16*)ctx->tcA2, ctx->kp2, 2 * (int64_t)npw * ctx->kp2, st), "tc operands");
  ctx->tc_built_pieces = pc;
  return PW_OK;
}

int check_tc_flag(pw_ctx* ctx) {
  if (!ctx->tc_err) return PW_OK;
  int h = 0;
  CU_TRY(cudaMemcpyAsync(&h, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "tc flag copy");
  CU_TRY(cudaStreamSynchronize(ctx->stream), "tc flag sync");
  if (h) {
    ctx->poisoned = true;
    return set_error(PW_ETIMEDOUT, "a tensor-core GEMM wait expired (stage %d)", h);
  }
  return PW_OK;
}

// bf16 pieces [pieces][nb][pitch] of a complex64 block (rows = 2 * nrow reals)
int tc_split(pw_ctx* ctx, const float2* x, int64_t ld, int nrow, int nb, int64_t pitch, int slot,
             __nv_bfloat16** out) {
  const int pc = ctx->tc_pieces;
  WS(buf, __nv_bfloat16, slot, (size_t)pc * nb * pitch);
  CU_TRY(tc::split_f32((const float*)x, 2 * ld, 2 * nrow, nb, pc, buf, pitch, (int64_t)nb * pitch, ctx->stream),
         "bf16 split");
  *out = buf;
  return PW_OK;
}

// bf16 pieces of a complex64 block into rows of an existing buffer with piece stride `ps`
int tc_split_into(pw_ctx* ctx, const float2* x, int64_t ld, int nrow, int nb, int64_t pitch, int64_t ps,
                  __nv_bfloat16* buf) {
  CU_TRY(tc::split_f32((const float*)x, 2 * ld, 2 * nrow, nb, ctx->tc_pieces, buf, pitch, ps, ctx->stream),
         "bf16 split");
  return PW_OK;
}

// K splits of the projection GEMM for nb columns: whole waves of the persistent grid (every
// SM gets the same number of work units), unless pw_autotune timed the choices for nb
int tc_proj_split(const pw_ctx* ctx, int nb, int rule_only = 0) {
  if (!rule_only)
    for (const auto& e : ctx->tc_proj_splits)
      if (e.first == nb) return e.second;
  const int M = 2 * ctx->nproj, K = 2 * ctx->npw;
  const int tiles = ((M + 127) / 128) * ((nb + 127) / 128);
  int nsm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int ns = 1;
  double best = -1;
  for (int c = 1; c <= std::max(1, std::min(64, K / 256)); ++c) {
    const int cc = tc::split_count(K, c);
    const int u = cc * tiles;
    const double eff = (double)u / ((double)((u + nsm - 1) / nsm) * nsm);
    if (eff > best + 1e-9) { best = eff; ns = cc; }
  }
  return ns;
}

// C (np x nb complex64, ld np) = P^dagger Y from the bf16 pieces of Y
int tc_project(pw_ctx* ctx, const __nv_bfloat16* ysplit, int nb, float2* Cout, int force_split = 0) {
  const int np = ctx->nproj, npw = ctx->npw, pc = ctx->tc_pieces;
  const int M = 2 * np, N = nb, K = 2 * npw;
  const int ns = force_split > 0 ? tc::split_count(K, force_split) : tc_proj_split(ctx, nb);
  WS(part, float, WS_TCPART, (size_t)ns * M * N);
  tc::Operand A{(const __nv_bfloat16*)ctx->tcA1, M, ctx->kp1, (int64_t)M * ctx->kp1};
  tc::Operand B{ysplit, N, ctx->kp1, (int64_t)N * ctx->kp1};
  tc::TcEpi e{};
  e.mode = tc::TC_EPI_PARTIAL;
  e.part = part;
  e.part_ld = M;
  e.part_split_stride = (int64_t)M * N;
  const int test = ctx->test_wait_expiry;
  ctx->test_wait_expiry = 0;
  CU_TRY(tc::gemm(A, B, M, N, K, pc, ns, e, ctx->tc_err, ctx->stream, test), "tc projection");
  CU_TRY(tc::reduce_partials(part, ns, (int64_t)M * N, M, M, N, (float*)Cout, 2 * (int64_t)np, ctx->stream),
         "tc reduce");
  return PW_OK;
}

// back-projection Y (2 npw real rows x nb) (+)= P Z with the given epilogue (out / yk / split fields set by caller)
int tc_backproject(pw_ctx* ctx, const __nv_bfloat16* zsplit, int nb, tc::TcEpi e) {
  const int np = ctx->nproj, npw = ctx->npw, pc = ctx->tc_pieces;
  const int M = 2 * npw, N = nb, K = 2 * np;
  tc::Operand A{(const __nv_bfloat16*)ctx->tcA2, M, ctx->kp2, (int64_t)M * ctx->kp2};
  tc::Operand B{zsplit, N, ctx->kp2, (int64_t)N * ctx->kp2};
  const int test = ctx->test_wait_expiry;
  ctx->test_wait_expiry = 0;
  CU_TRY(tc::gemm(A, B, M, N, K, pc, 1, e, ctx->tc_err, ctx->stream, test), "tc back-projection");
  return PW_OK;
}

// ---------------------------------------------------------------------------
// FP64 GEMMs: FP64-accurate digit-sliced tensor-core GEMMs (zgemm_tc.cu), or DFMA
// ---------------------------------------------------------------------------
int ensure_err_flag(pw_ctx* ctx) {
  if (ctx->tc_err) return PW_OK;
  CU_TRY(cudaMalloc(&ctx->tc_err, sizeof(int)), "error flag allocation");
  CU_TRY(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->stream), "error flag reset");
  return PW_OK;
}

// digit planes of P^dagger and of P (the FP64 projector products), built once per context
int ensure_ozp(pw_ctx* ctx) {
  if (ctx->ozPH) return PW_OK;
  const int np = ctx->nproj, npw = ctx->npw;
  const cudaStream_t st = ctx->stream;
  const int64_t p1 = oz::digit_pitch(2 * npw), p2 = oz::digit_pitch(2 * np);
  WS(amax, unsigned long long, WS_OZAMAX, std::max(np, npw));
  CU_TRY(cudaMalloc(&ctx->ozPH, oz::digit_bytes(2 * np, 2 * npw)), "P^dagger digit planes");
  CU_TRY(cudaMalloc(&ctx->ozP, oz::digit_bytes(2 * npw, 2 * np)), "P digit planes");
  CU_TRY(cudaMalloc(&ctx->ozPH_exp, sizeof(int) * (size_t)np), "P^dagger exponents");
  CU_TRY(cudaMalloc(&ctx->ozP_exp, sizeof(int) * (size_t)npw), "P exponents");
  CU_TRY(oz::slice(ctx->P64, npw, 1, 1, np, npw, 1, (__nv_bfloat16*)ctx->ozPH, p1, 2 * (int64_t)np * p1, amax,
                   ctx->ozPH_exp, st), "P^dagger digits");
  CU_TRY(oz::slice(ctx->P64, 1, npw, 0, npw, np, 1, (__nv_bfloat16*)ctx->ozP, p2, 2 * (int64_t)npw * p2, amax,
                   ctx->ozP_exp, st), "P digits");
  return PW_OK;
}

// C (M x N) = op(A) op(B) in FP64 with the epilogue e (conventions of launch_cgemm).  The
// digit-sliced tensor-core GEMM runs unless the context asks for DFMA or op(B) has at most 4
// columns (matrix-vector forms, memory-bound); op(A) = P^dagger or P uses the context's cached
// digit planes.  dfma_ns / dfma_ws: split-K of the DFMA form.
int zgemm(pw_ctx* ctx, int ta, int tb, int M, int N, int K, const double2* A, int64_t lda, const double2* B,
          int64_t ldb, const Epi<double>& e, int dfma_ns, double2* dfma_ws, int tri, const char* where) {
  if (M <= 0 || N <= 0) return PW_OK;
  const cudaStream_t st = ctx->stream;
  if (!ctx->fp64_tc || N <= 4 || K <= 0 || !oz::available()) {
    CU_TRY(launch_cgemm<double>(ta, tb, M, N, K, A, lda, B, ldb, e, dfma_ns, dfma_ws, st, tri), where);
    return PW_OK;
  }
  PW_TRY(ensure_err_flag(ctx));
  const int lower = (tri == GEMM_LOWER_OUT);
  oz::Digits Ad{nullptr, 2 * M, 2 * K, oz::digit_pitch(2 * K), 0, nullptr};
  Ad.plane = (int64_t)Ad.rows * Ad.pitch;
  const bool is_p = (A == ctx->P64 && ctx->nproj > 0 && lda == ctx->npw);
  if (is_p && ta == 1 && M == ctx->nproj && K == ctx->npw) {
    PW_TRY(ensure_ozp(ctx));
    Ad.dig = (const __nv_bfloat16*)ctx->ozPH;
    Ad.exp = ctx->ozPH_exp;
  } else if (is_p && ta == 0 && M == ctx->npw && K == ctx->nproj) {
    PW_TRY(ensure_ozp(ctx));
    Ad.dig = (const __nv_bfloat16*)ctx->ozP;
    Ad.exp = ctx->ozP_exp;
  }
  oz::Digits Bd{nullptr, N, 2 * K, oz::digit_pitch(2 * K), 0, nullptr};
  Bd.plane = (int64_t)Bd.rows * Bd.pitch;
  WS(amax, unsigned long long, WS_OZAMAX, std::max(M, N));
  WS(ex, int, WS_OZEXP, (size_t)M + N);
  if (!Ad.dig) {
    WS(ad, __nv_bfloat16, WS_OZA, (size_t)oz::kDigits * Ad.plane);
    CU_TRY(oz::slice(A, ta ? lda : 1, ta ? 1 : lda, ta, M, K, 1, ad, Ad.pitch, Ad.plane, amax, ex, st), where);
    Ad.dig = ad;
    Ad.exp = ex;
  }
  WS(bd, __nv_bfloat16, WS_OZB, (size_t)oz::kDigits * Bd.plane);
  CU_TRY(oz::slice(B, tb ? 1 : ldb, tb ? ldb : 1, tb, N, K, 0, bd, Bd.pitch, Bd.plane, amax, ex + M, st), where);
  Bd.dig = bd;
  Bd.exp = ex + M;
  const int ns = oz::split_count(2 * M, N, 2 * K, lower);
  double* part = nullptr;
  if (ns > 1) {
    WS(pp, double, WS_OZPART, (size_t)ns * N * 2 * M);
    part = pp;
  }
  const int test = ctx->test_wait_expiry;
  ctx->test_wait_expiry = 0;
  CU_TRY(oz::gemm(Ad, Bd, M, N, K, e, lower, ns, part, ctx->tc_err, test, st), where);
  return PW_OK;
}

// complex GEMM of the filter / H-apply precision: FP64 through zgemm, complex64 on FFMA
template <typename T>
int cg(pw_ctx* ctx, int ta, int tb, int M, int N, int K, const cplx<T>* A, int64_t lda, const cplx<T>* B,
       int64_t ldb, const Epi<T>& e, int ns, cplx<T>* ws, cudaStream_t st, int tri, const char* where) {
  if constexpr (std::is_same<T, double>::value) {
    return zgemm(ctx, ta, tb, M, N, K, A, lda, B, ldb, e, ns, ws, tri, where);
  } else {
    CU_TRY(launch_cgemm<T>(ta, tb, M, N, K, A, lda, B, ldb, e, ns, ws, st, tri), where);
    return PW_OK;
  }
}

// ---------------------------------------------------------------------------
// H-apply (HX / HX_SX of Sec. 3.3)
// ---------------------------------------------------------------------------
template <typename T>
int apply_impl(pw_ctx* ctx, const cplx<T>* psi, int64_t ldpsi, int nband, cplx<T>* hpsi, cplx<T>* spsi,
               int64_t ldout) {
  using C = cplx<T>;
  const int npw = ctx->npw, np = ctx->nproj;
  const cudaStream_t st = ctx->stream;
  const int bb = band_batch(ctx, nband, sizeof(C));
  const int64_t hb_bs = (int64_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2];
  WS(hb, C, WS_HB, hb_bs * bb);
  WS(Cm, C, WS_C, (size_t)np * nband);
  WS(Z, C, WS_Z, (size_t)np * nband);
  const int ns = nsplit_for(np, nband, npw);
  WS(sp, C, WS_SPLIT, (size_t)ns * np * nband);
  CU_TRY(launch_local_apply<T>(ctx->plan, Prec<T>::tw(ctx), ctx->sp, Prec<T>::vp(ctx), Prec<T>::kin(ctx), psi,
                               ldpsi, nband, hpsi, ldout, hb, bb, st, ctx), "local apply");
  if (np > 0 && std::is_same<T, float>::value) {
    // mixed precision: BF16-split tensor-core projector GEMMs
    PW_TRY(ensure_tc(ctx));
    __nv_bfloat16 *ys, *zs;
    {
      ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
      PW_TRY(tc_split(ctx, (const float2*)psi, ldpsi, npw, nband, ctx->kp1, WS_YSPLIT, &ys));
      PW_TRY(tc_project(ctx, ys, nband, (float2*)Cm));
    }
    {
      ProfScope ps(ctx, PW_PROF_SMALL);
      CU_TRY(launch_dblock<T>(np, nband, Prec<T>::D(ctx), ctx->blk0, ctx->blklen, Cm, np, Z, np, st), "D block");
      PW_TRY(tc_split(ctx, (const float2*)Z, np, np, nband, ctx->kp2, WS_ZSPLIT, &zs));
    }
    ProfScope ps(ctx, PW_PROF_GEMM_BACK);
    tc::TcEpi e{};
    e.mode = tc::TC_EPI_ACCUM;
    e.out = (float*)hpsi;
    e.ldo = 2 * ldout;
    e.alpha = 1.f;
    PW_TRY(tc_backproject(ctx, zs, nband, e));
  } else if (np > 0) {
    {
      ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
      PW_TRY(cg<T>(ctx, 1, 0, np, nband, npw, Prec<T>::P(ctx), npw, psi, ldpsi, epi<T>(EPI_STORE, Cm, np), ns, sp, st, GEMM_FULL, "projection gemm"));
    }
    {
      ProfScope ps(ctx, PW_PROF_SMALL);
      CU_TRY(launch_dblock<T>(np, nband, Prec<T>::D(ctx), ctx->blk0, ctx->blklen, Cm, np, Z, np, st), "D block");
    }
    ProfScope ps(ctx, PW_PROF_GEMM_BACK);
    PW_TRY(cg<T>(ctx, 0, 0, npw, nband, np, Prec<T>::P(ctx), npw, Z, np, epi<T>(EPI_ACCUM, hpsi, ldout), 1, sp, st, GEMM_FULL, "back-projection gemm"));
  }
  if (spsi) {
    CU_TRY(cudaMemcpy2DAsync(spsi, sizeof(C) * ldout, psi, sizeof(C) * ldpsi, sizeof(C) * npw, nband,
                             cudaMemcpyDeviceToDevice, st), "copy S psi");
    if constexpr (std::is_same<T, double>::value) {
      if (ctx->has_q && np > 0) {
        CU_TRY(launch_dblock<double>(np, nband, ctx->Q64, ctx->qblk0, ctx->qblklen, Cm, np, Z, np, st), "Q block");
        PW_TRY(cg<T>(ctx, 0, 0, npw, nband, np, Prec<T>::P(ctx), npw, Z, np, epi<T>(EPI_ACCUM, spsi, ldout), 1, sp, st, GEMM_FULL, "overlap gemm"));
      }
    } else {
      if (ctx->has_q && np > 0) return set_error(PW_EUNSUPPORTED, "S apply is FP64 only");
    }
  }
  return PW_OK;
}

// S psi = psi + P Q P^dagger psi alone (FP64; the S-Ortho pass needs no H psi)
int apply_s64(pw_ctx* ctx, const double2* psi, int64_t ldpsi, int nband, double2* spsi, int64_t ldout) {
  const int npw = ctx->npw, np = ctx->nproj;
  const cudaStream_t st = ctx->stream;
  CU_TRY(cudaMemcpy2DAsync(spsi, sizeof(double2) * ldout, psi, sizeof(double2) * ldpsi, sizeof(double2) * npw, nband,
                           cudaMemcpyDeviceToDevice, st), "copy S psi");
  if (!ctx->has_q || np == 0) return PW_OK;
  WS(Cm, double2, WS_C, (size_t)np * nband);
  WS(Z, double2, WS_Z, (size_t)np * nband);
  const int ns = nsplit_for(np, nband, npw);
  WS(sp, double2, WS_SPLIT, (size_t)ns * np * nband);
  PW_TRY(cg<double>(ctx, 1, 0, np, nband, npw, ctx->P64, npw, psi, ldpsi, epi<double>(EPI_STORE, Cm, np), ns, sp, st,
                    GEMM_FULL, "S projection"));
  CU_TRY(launch_dblock<double>(np, nband, ctx->Q64, ctx->qblk0, ctx->qblklen, Cm, np, Z, np, st), "Q block");
  PW_TRY(cg<double>(ctx, 0, 0, npw, nband, np, ctx->P64, npw, Z, np, epi<double>(EPI_ACCUM, spsi, ldout), 1, sp, st,
                    GEMM_FULL, "S back-projection"));
  return PW_OK;
}

// ---------------------------------------------------------------------------
// Chebyshev filter (Alg. 7 / Alg. 12)
// ---------------------------------------------------------------------------
// Per-column Chebyshev sum carried along the filter's steps (spectrum slicing):
// out[:, j] = sum_k coef[k nband + j] T_k(A~) psi_j, coef on the device ((degree + 1) x nband)
template <typename T> struct ChebSum {
  cplx<T>* out;
  int64_t ldo;
  const double* coef;
};

template <typename T>
int filter_impl(pw_ctx* ctx, cplx<T>* psi, int64_t ldpsi, int nband, int degree, double a, double b,
                const double* dev_ce = nullptr, const ChebSum<T>* sum = nullptr) {
  using C = cplx<T>;
  if (degree <= 0 || nband <= 0) return PW_OK;
  // Y_k = T_k(A~) psi after step k (the unscaled recurrence); the sum takes coef_k Y_k
  auto add_term = [&](const C* y, int64_t ldy, int k) -> int {
    if (!sum) return PW_OK;
    ProfScope ps(ctx, PW_PROF_SMALL);
    CU_TRY(la_cheb_acc<T>(y, ldy, ctx->npw, nband, sum->coef + (size_t)k * nband, sum->out, sum->ldo, k == 0,
                          ctx->stream), "Chebyshev sum");
    return PW_OK;
  };
  PW_TRY(add_term(psi, ldpsi, 0));
  if (!dev_ce && !(b > a)) return set_error(PW_EINVAL, "filter interval needs upper > lower (a=%g, b=%g)", a, b);
  const int npw = ctx->npw, np = ctx->nproj;
  const cudaStream_t st = ctx->stream;
  const int bb = band_batch(ctx, nband, sizeof(C));
  const int64_t hb_bs = (int64_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2];
  WS(hb, C, WS_HB, hb_bs * bb);
  // With Q the step needs C_k = P^dagger Y_k and C_w = P^dagger W, W = (T + V) Y_k.  Only C_w
  // is a projection of the block: C_k follows the filter's recurrence in projector space,
  // P^dagger Y_{k+1} = alpha (C_w + (P^dagger P) Z - c C_k) - beta C_{k-1} (Z the step's
  // projector-space coefficients, Y_{k+1} = alpha (W + P Z - c Y_k) - beta Y_{k-1}), from the
  // stored P^dagger P: one N x N_p projection per step instead of two, the other an N_p x N_p
  // product.  C_0 is projected once.  Without Q, C_k itself is the one projection per step.
  const bool shadow = ctx->has_q && np > 0;
  const size_t pcol = (size_t)np * nband;
  WS(Cm, C, WS_C, pcol * (shadow ? 4 : 1));  // with Q: C_{k-1}, C_k, C_{k+1} rotating, then C_w
  WS(Z, C, WS_Z, pcol);
  C* Cw = shadow ? Cm + 3 * pcol : nullptr;
  auto Crot = [&](int j) { return Cm + (size_t)(((j % 3) + 3) % 3) * pcol; };
  const int ns = nsplit_for(np, nband, npw);
  WS(spl, C, WS_SPLIT, (size_t)ns * np * nband);
  WS(Y1, C, WS_Y1, (size_t)npw * nband);
  WS(Y2, C, WS_Y2, (size_t)npw * nband);
  C* buf[3] = {psi, Y1, Y2};
  const int64_t ld[3] = {ldpsi, npw, npw};
  const double cc = 0.5 * (b + a), e = 0.5 * (b - a);
  constexpr bool kMixed = std::is_same<T, float>::value;
  __nv_bfloat16* ys = nullptr;
  int64_t ys_ps = 0;  // piece stride of the bf16 pieces; kp1 is known once the operands of P exist
  if (kMixed && np > 0) {
    PW_TRY(ensure_tc(ctx));
    ys_ps = (int64_t)nband * ctx->kp1;
    ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
    WS(ysb, __nv_bfloat16, WS_YSPLIT, (size_t)ctx->tc_pieces * ys_ps);
    ys = ysb;
    PW_TRY(tc_split_into(ctx, (const float2*)psi, ldpsi, npw, nband, ctx->kp1, ys_ps, ys));
    if (shadow) PW_TRY(tc_project(ctx, ys, nband, (float2*)Crot(0)));  // C_0 = P^dagger Y_0
  } else if (shadow) {
    ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
    PW_TRY(cg<T>(ctx, 1, 0, np, nband, npw, Prec<T>::P(ctx), npw, psi, ldpsi, epi<T>(EPI_STORE, Crot(0), np), ns, spl,
                 st, GEMM_FULL, "filter projection of Y_0"));
  }
  // C_{k+1} = alpha (C_w + (P^dagger P) Z - c C_k) - beta C_{k-1}, the recurrence of the step
  // in projector space (with Q; not needed after the last step)
  auto shadow_step = [&](int k) -> int {
    if (!shadow || k + 1 >= degree) return PW_OK;
    ProfScope ps(ctx, PW_PROF_SMALL);
    C* next = Crot(k + 1);
    CU_TRY(cudaMemcpyAsync(next, Cw, sizeof(C) * pcol, cudaMemcpyDeviceToDevice, st), "C_w copy");
    Epi<T> ce = epi<T>(EPI_CHEB, next, np, (T)(k == 0 ? 1.0 / e : 2.0 / e));
    ce.beta = (T)1;
    ce.shift = (T)cc;
    ce.yk = Crot(k);
    ce.ldy = np;
    ce.ykm1 = (k == 0) ? nullptr : Crot(k - 1);
    ce.ldy2 = np;
    ce.dev_ce = dev_ce;
    ce.first = (k == 0);
    PW_TRY(cg<T>(ctx, 0, 0, np, nband, np, Prec<T>::B(ctx), np, Z, np, ce, 1, spl, st, GEMM_FULL,
                 "projector-space recurrence"));
    return PW_OK;
  };
  // complex64 with S = I and the warp-group plane kernels: the nonlocal term first
  // (projection, D, back-projection into PZ), then the FFT passes with the recurrence and
  // the bf16 split of Y_{k+1} fused into pass 3 (fewer block reads than the recurrence in
  // the back-projection epilogue)
  if constexpr (kMixed) {
    if (np > 0 && !ctx->has_q && local_apply_rec_supported(ctx->plan, ctx)) {
      WS(PZ, C, WS_PZ, (size_t)npw * nband);
      for (int k = 0; k < degree; ++k) {
        C* cur = buf[k % 3];
        C* prev = buf[(k + 2) % 3];
        C* dst = buf[(k + 1) % 3];
        const int64_t ldc = ld[k % 3], ldp = ld[(k + 2) % 3], ldd = ld[(k + 1) % 3];
        {
          ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
          PW_TRY(tc_project(ctx, ys, nband, (float2*)Cm));
        }
        __nv_bfloat16* zs;
        {
          ProfScope ps(ctx, PW_PROF_SMALL);
          CU_TRY(launch_dblock<T>(np, nband, Prec<T>::D(ctx), ctx->blk0, ctx->blklen, Cm, np, Z, np, st), "filter D");
          PW_TRY(tc_split(ctx, (const float2*)Z, np, np, nband, ctx->kp2, WS_ZSPLIT, &zs));
        }
        {
          ProfScope ps(ctx, PW_PROF_GEMM_BACK);
          tc::TcEpi te{};
          te.mode = tc::TC_EPI_STORE;
          te.out = (float*)PZ;
          te.ldo = 2 * (int64_t)npw;
          te.alpha = 1.f;
          PW_TRY(tc_backproject(ctx, zs, nband, te));
        }
        Pass3Rec rec{};
        rec.pz = (const float2*)PZ;
        rec.ldpz = npw;
        rec.ykm1 = (k == 0) ? nullptr : (const float2*)prev;
        rec.ldykm1 = ldp;
        rec.alpha = (float)(k == 0 ? 1.0 / e : 2.0 / e);
        rec.beta = 1.f;
        rec.shift = (float)cc;
        rec.dev_ce = dev_ce;
        rec.first = (k == 0);
        rec.split = (k + 1 < degree) ? (void*)ys : nullptr;
        rec.split_ld = ctx->kp1;
        rec.split_piece_stride = (int64_t)nband * ctx->kp1;
        rec.pieces = ctx->tc_pieces;
        CU_TRY(launch_local_apply_rec(ctx->plan, ctx->tw32, ctx->sp, ctx->vperm32, ctx->kin32, (const float2*)cur, ldc,
                                      nband, (float2*)dst, ldd, (float2*)hb, bb, st, ctx, rec), "filter local + recurrence");
        PW_TRY(add_term(dst, ldd, k + 1));
      }
      if (degree % 3 != 0) {
        CU_TRY(cudaMemcpy2DAsync(psi, sizeof(C) * ldpsi, buf[degree % 3], sizeof(C) * npw, sizeof(C) * npw, nband,
                                 cudaMemcpyDeviceToDevice, st), "filter copy-out");
      }
      return PW_OK;
    }
  }
  for (int k = 0; k < degree; ++k) {
    C* cur = buf[k % 3];
    C* prev = buf[(k + 2) % 3];
    C* dst = buf[(k + 1) % 3];
    const int64_t ldc = ld[k % 3], ldp = ld[(k + 2) % 3], ldd = ld[(k + 1) % 3];
    const T alpha = (T)(k == 0 ? 1.0 / e : 2.0 / e);
    // W = (T + V) Y_k
    CU_TRY(launch_local_apply<T>(ctx->plan, Prec<T>::tw(ctx), ctx->sp, Prec<T>::vp(ctx), Prec<T>::kin(ctx), cur,
                                 ldc, nband, dst, ldd, hb, bb, st, ctx), "filter local");
    if (kMixed && np > 0) {
      {
        ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
        if (shadow) {
          PW_TRY(tc_split_into(ctx, (const float2*)dst, ldd, npw, nband, ctx->kp1, ys_ps, ys));
          PW_TRY(tc_project(ctx, ys, nband, (float2*)Cw));  // P^dagger W; C_k from the recurrence
        } else {
          PW_TRY(tc_project(ctx, ys, nband, (float2*)Cm));
        }
      }
      __nv_bfloat16* zs;
      {
        ProfScope ps(ctx, PW_PROF_SMALL);
        if (!ctx->has_q) {
          CU_TRY(launch_dblock<T>(np, nband, Prec<T>::D(ctx), ctx->blk0, ctx->blklen, Cm, np, Z, np, st), "filter D");
        } else {
          PW_TRY(cg<T>(ctx, 0, 0, np, nband, np, Prec<T>::E(ctx), np, Crot(k), np, epi<T>(EPI_STORE, Z, np), 1, spl, st, GEMM_FULL, "filter E C"));
          PW_TRY(cg<T>(ctx, 0, 0, np, nband, np, Prec<T>::K(ctx), np, Cw, np, epi<T>(EPI_ACCUM, Z, np, (T)-1), 1, spl, st, GEMM_FULL, "filter K Cw"));
        }
        PW_TRY(tc_split(ctx, (const float2*)Z, np, np, nband, ctx->kp2, WS_ZSPLIT, &zs));
      }
      PW_TRY(shadow_step(k));
      ProfScope ps(ctx, PW_PROF_GEMM_BACK);
      tc::TcEpi te{};
      te.mode = tc::TC_EPI_CHEB;
      te.out = (float*)dst;
      te.ldo = 2 * ldd;
      te.yk = (const float*)cur;
      te.ldyk = 2 * ldc;
      te.ykm1 = (k == 0) ? nullptr : (const float*)prev;
      te.ldykm1 = 2 * ldp;
      te.alpha = (float)alpha;
      te.beta = 1.f;
      te.shift = (float)cc;
      te.dev_ce = dev_ce;
      te.first = (k == 0);
      te.split = ys;
      te.split_ld = ctx->kp1;
      te.split_piece_stride = ys_ps;
      // the next projection needs the pieces of Y_{k+1} only without Q (with Q it projects W)
      te.out_pieces = (!shadow && k + 1 < degree) ? ctx->tc_pieces : 0;
      PW_TRY(tc_backproject(ctx, zs, nband, te));
      PW_TRY(add_term(dst, ldd, k + 1));
      continue;
    }
    Epi<T> ce = epi<T>(EPI_CHEB, dst, ldd, alpha);
    ce.beta = (T)1;
    ce.shift = (T)cc;
    ce.yk = cur;
    ce.ldy = ldc;
    ce.ykm1 = (k == 0) ? nullptr : prev;
    ce.ldy2 = ldp;
    ce.dev_ce = dev_ce;
    ce.first = (k == 0);
    if (np > 0) {
      {
        ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
        // C = P^dagger Y_k (without Q), C_w = P^dagger W (with Q; C_k from the recurrence)
        if (!shadow)
          PW_TRY(cg<T>(ctx, 1, 0, np, nband, npw, Prec<T>::P(ctx), npw, cur, ldc, epi<T>(EPI_STORE, Cm, np), ns, spl, st, GEMM_FULL, "filter projection"));
        else
          PW_TRY(cg<T>(ctx, 1, 0, np, nband, npw, Prec<T>::P(ctx), npw, dst, ldd, epi<T>(EPI_STORE, Cw, np), ns, spl, st, GEMM_FULL, "filter projection of W"));
      }
      {
        ProfScope ps(ctx, PW_PROF_SMALL);
        if (!ctx->has_q) {
          CU_TRY(launch_dblock<T>(np, nband, Prec<T>::D(ctx), ctx->blk0, ctx->blklen, Cm, np, Z, np, st), "filter D");
        } else {
          // S^-1 H Y = W + P [E C - K P^dagger W],  E = (I - K P^dagger P) D  (Woodbury, Sec. 3.3)
          PW_TRY(cg<T>(ctx, 0, 0, np, nband, np, Prec<T>::E(ctx), np, Crot(k), np, epi<T>(EPI_STORE, Z, np), 1, spl, st, GEMM_FULL, "filter E C"));
          PW_TRY(cg<T>(ctx, 0, 0, np, nband, np, Prec<T>::K(ctx), np, Cw, np, epi<T>(EPI_ACCUM, Z, np, (T)-1), 1, spl, st, GEMM_FULL, "filter K Cw"));
        }
      }
      PW_TRY(shadow_step(k));
      ProfScope ps(ctx, PW_PROF_GEMM_BACK);
      PW_TRY(cg<T>(ctx, 0, 0, npw, nband, np, Prec<T>::P(ctx), npw, Z, np, ce, 1, spl, st, GEMM_FULL, "filter recurrence"));
    } else {
      ProfScope ps(ctx, PW_PROF_GEMM_BACK);
      PW_TRY(cg<T>(ctx, 0, 0, npw, nband, 0, Prec<T>::P(ctx), npw, Z, 1, ce, 1, spl, st, GEMM_FULL, "filter recurrence"));
    }
    PW_TRY(add_term(dst, ldd, k + 1));
  }
  if (degree % 3 != 0) {
    CU_TRY(cudaMemcpy2DAsync(psi, sizeof(C) * ldpsi, buf[degree % 3], sizeof(C) * npw, sizeof(C) * npw, nband,
                             cudaMemcpyDeviceToDevice, st), "filter copy-out");
  }
  return PW_OK;
}

// One step of the three-term recurrence with explicit coefficients, S = I:
//   dst = alpha ((H - shift) cur) - beta prev     (prev may be NULL)
// The forward filter steps and the steps of its adjoint (H is Hermitian, so the
// adjoint recurrence applies H itself) both have this form.  C_out (nproj x nband,
// ld nproj, may be NULL) receives P^dagger cur.
template <typename T>
int recur_step(pw_ctx* ctx, const cplx<T>* cur, int64_t ldc, const cplx<T>* prev, int64_t ldp, cplx<T>* dst,
               int64_t ldd, int nband, double alpha, double beta, double shift, cplx<T>* C_out) {
  using C = cplx<T>;
  if (ctx->has_q) return set_error(PW_EUNSUPPORTED, "the explicit recurrence step needs S = I (Q == NULL)");
  if (nband <= 0) return PW_OK;
  const int npw = ctx->npw, np = ctx->nproj;
  const cudaStream_t st = ctx->stream;
  const int bb = band_batch(ctx, nband, sizeof(C));
  const int64_t hb_bs = (int64_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2];
  WS(hb, C, WS_HB, hb_bs * bb);
  WS(Cm, C, WS_C, (size_t)np * nband);
  WS(Z, C, WS_Z, (size_t)np * nband);
  const int ns = nsplit_for(np, nband, npw);
  WS(spl, C, WS_SPLIT, (size_t)ns * np * nband);
  C* Cp = C_out ? C_out : Cm;
  CU_TRY(launch_local_apply<T>(ctx->plan, Prec<T>::tw(ctx), ctx->sp, Prec<T>::vp(ctx), Prec<T>::kin(ctx), cur, ldc,
                               nband, dst, ldd, hb, bb, st, ctx), "recurrence local");
  if constexpr (std::is_same<T, float>::value) {
    if (np > 0) {
      PW_TRY(ensure_tc(ctx));
      __nv_bfloat16 *ys, *zs;
      {
        ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
        PW_TRY(tc_split(ctx, (const float2*)cur, ldc, npw, nband, ctx->kp1, WS_YSPLIT, &ys));
        PW_TRY(tc_project(ctx, ys, nband, (float2*)Cp));
      }
      {
        ProfScope ps(ctx, PW_PROF_SMALL);
        CU_TRY(launch_dblock<T>(np, nband, Prec<T>::D(ctx), ctx->blk0, ctx->blklen, Cp, np, Z, np, st),
               "recurrence D");
        PW_TRY(tc_split(ctx, (const float2*)Z, np, np, nband, ctx->kp2, WS_ZSPLIT, &zs));
      }
      ProfScope ps(ctx, PW_PROF_GEMM_BACK);
      tc::TcEpi te{};
      te.mode = tc::TC_EPI_CHEB;
      te.out = (float*)dst;
      te.ldo = 2 * ldd;
      te.yk = (const float*)cur;
      te.ldyk = 2 * ldc;
      te.ykm1 = prev ? (const float*)prev : nullptr;
      te.ldykm1 = 2 * ldp;
      te.alpha = (float)alpha;
      te.beta = (float)beta;
      te.shift = (float)shift;
      PW_TRY(tc_backproject(ctx, zs, nband, te));
      return PW_OK;
    }
  }
  Epi<T> ce = epi<T>(EPI_CHEB, dst, ldd, (T)alpha);
  ce.beta = (T)beta;
  ce.shift = (T)shift;
  ce.yk = cur;
  ce.ldy = ldc;
  ce.ykm1 = prev;
  ce.ldy2 = ldp;
  if (np > 0) {
    {
      ProfScope ps(ctx, PW_PROF_GEMM_PROJ);
      PW_TRY(cg<T>(ctx, 1, 0, np, nband, npw, Prec<T>::P(ctx), npw, cur, ldc, epi<T>(EPI_STORE, Cp, np), ns, spl, st, GEMM_FULL, "recurrence projection"));
    }
    {
      ProfScope ps(ctx, PW_PROF_SMALL);
      CU_TRY(launch_dblock<T>(np, nband, Prec<T>::D(ctx), ctx->blk0, ctx->blklen, Cp, np, Z, np, st),
             "recurrence D");
    }
    ProfScope ps(ctx, PW_PROF_GEMM_BACK);
    PW_TRY(cg<T>(ctx, 0, 0, npw, nband, np, Prec<T>::P(ctx), npw, Z, np, ce, 1, spl, st, GEMM_FULL, "recurrence"));
  } else {
    ProfScope ps(ctx, PW_PROF_GEMM_BACK);
    PW_TRY(cg<T>(ctx, 0, 0, npw, nband, 0, Prec<T>::P(ctx), npw, Z, 1, ce, 1, spl, st, GEMM_FULL, "recurrence"));
  }
  return PW_OK;
}

// ---------------------------------------------------------------------------
// S-Ortho (Alg. 9) and Rayleigh-Ritz (Alg. 5), FP64
// ---------------------------------------------------------------------------
// G = Y^H B for a Hermitian result (B = S Y or H Y): only the tiles on and below the diagonal are
// computed; the upper triangle is the conjugate of the lower one
int gram_herm(pw_ctx* ctx, const double2* Y, int64_t ldy, const double2* B, int64_t ldb, int m, double2* G) {
  const cudaStream_t st = ctx->stream;
  const int tl = (m + 63) / 64;
  const int ns = nsplit_tiles(tl * (tl + 1) / 2, ctx->npw);
  WS(spl, double2, WS_SPLIT, (size_t)ns * m * m);
  PW_TRY(cg<double>(ctx, 1, 0, m, m, ctx->npw, Y, ldy, B, ldb, epi<double>(EPI_STORE, G, m), ns, spl, st, GEMM_LOWER_OUT, "gram"));
  CU_TRY(la_herm_from_lower(G, m, m, st), "gram Hermitian");
  return PW_OK;
}

// G = Y^H SY (herm.), L = chol(G), Linv = L^-1.  flag set on failure.
int gram_chol(pw_ctx* ctx, const double2* Y, int64_t ldy, const double2* SY, int64_t lds, int m, double2* G,
              double2* Linv, double2* tmp, int* flag) {
  const cudaStream_t st = ctx->stream;
  PW_TRY(gram_herm(ctx, Y, ldy, SY, lds, m, G));
  CU_TRY(la_cholesky(G, m, m, flag, st), "cholesky");
  CU_TRY(la_trinv_lower(G, m, m, Linv, m, tmp, st), "triangular inverse");
  return PW_OK;
}

int check_flag(pw_ctx* ctx, int* flag_dev, const char* what) {
  int h = 0;
  CU_TRY(cudaMemcpyAsync(&h, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "flag copy");
  CU_TRY(cudaStreamSynchronize(ctx->stream), "flag sync");
  if (h) return set_error(PW_ENOTSPD, "%s: matrix is not positive definite", what);
  return PW_OK;
}

// Hermitian eigensolve of a reduced matrix A (n x n, lda n, destroyed): U (n x n) and eig
// (device, ascending); jac: 3 n*n + n + 2 complex128, norms: 2 doubles (device).  From n = 128 an
// FP32 Jacobi pre-rotation first: V32 brings A near diagonal at the FP32 rate; V = V32 made
// unitary in FP64 (Cholesky-QR), A' = V^dagger A V by FP64-accurate GEMMs is then a similarity
// transform of A to rounding and nearly diagonal, so the FP64 Jacobi on A' needs only a few
// sweeps; U = V U'.
constexpr int kMixedEigMin = 128;
int eigh_impl(pw_ctx* ctx, double2* A, int n, double2* U, double* eig, double2* jac, double* norms, int* sweeps) {
  const cudaStream_t st = ctx->stream;
  if (n < kMixedEigMin) return la_jacobi_eigh(A, n, U, eig, jac, norms, st, 40, 1e-13, sweeps);
  const size_t nn = (size_t)n * n;
  const size_t bytes = sizeof(double2) * 5 * nn + sizeof(float2) * (4 * nn + n + 2) + 64;
  WS(mixb, unsigned char, WS_EIGMIX, bytes);
  double2* V = (double2*)mixb;
  double2* Vo = V + nn;
  double2* T = Vo + nn;
  double2* Gv = T + nn;
  double2* Lv = Gv + nn;
  float2* A32 = (float2*)(Lv + nn);
  float2* V32 = A32 + nn;
  float2* w32 = V32 + nn;
  int* flag = (int*)(w32 + 2 * nn + n + 2);
  CU_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st), "flag reset");
  CU_TRY(la_to_c64(A, n, A32, n, n, n, st), "eig: to c64");
  int sw32 = 0, sw64 = 0;
  PW_TRY(la_jacobi_rotate32(A32, n, V32, w32, norms, st, 30, 1e-6, &sw32));
  CU_TRY(la_to_c128(V32, n, V, n, n, n, st), "eig: to c128");
  // Vo = V L^{-dagger}, L L^dagger = V^dagger V
  PW_TRY(cg<double>(ctx, 1, 0, n, n, n, V, n, V, n, epi<double>(EPI_STORE, Gv, n), 1, nullptr, st, GEMM_FULL,
                    "eig basis Gram"));
  CU_TRY(la_herm_sym(Gv, n, n, st), "eig basis Gram sym");
  CU_TRY(la_cholesky(Gv, n, n, flag, st), "eig basis Cholesky");
  CU_TRY(la_trinv_lower(Gv, n, n, Lv, n, T, st), "eig basis triangular inverse");
  PW_TRY(cg<double>(ctx, 0, 1, n, n, n, V, n, Lv, n, epi<double>(EPI_STORE, Vo, n), 1, nullptr, st, GEMM_B_UPPER,
                    "eig basis orthonormalisation"));
  PW_TRY(check_flag(ctx, flag, "eigensolver basis Cholesky"));
  // A' = Vo^dagger A Vo (into A), FP64 Jacobi on it, U = Vo U'
  PW_TRY(cg<double>(ctx, 0, 0, n, n, n, A, n, Vo, n, epi<double>(EPI_STORE, T, n), 1, nullptr, st, GEMM_FULL,
                    "eig rotate 1"));
  PW_TRY(cg<double>(ctx, 1, 0, n, n, n, Vo, n, T, n, epi<double>(EPI_STORE, A, n), 1, nullptr, st, GEMM_FULL,
                    "eig rotate 2"));
  CU_TRY(la_herm_sym(A, n, n, st), "eig rotated sym");
  PW_TRY(la_jacobi_eigh(A, n, T, eig, jac, norms, st, 40, 1e-13, &sw64));
  PW_TRY(cg<double>(ctx, 0, 0, n, n, n, Vo, n, T, n, epi<double>(EPI_STORE, U, n), 1, nullptr, st, GEMM_FULL,
                    "eig back-rotation"));
  if (sweeps) *sweeps = sw64;
  return PW_OK;
}

// q_out (ld npw): the S-orthonormal block Q before the rotation; x_out (m x m): the rotation X
// (Psi = Q X); eig_dev_out (device, m): the Ritz values.  Each may be NULL.
//
// S-Ortho (Alg. 9) is Cholesky-QR in the S metric.  One pass leaves the block S-orthonormal to
// within about cond(Y)^2 * eps; the second pass is the Cholesky factor of the Rayleigh-Ritz overlap
// S_Psi itself (Alg. 5 reduces H_Psi with it), so the block is not rotated twice before H is applied:
// Psi = Y1 X with X = L^{-dagger} U, and Q = Y1 L^{-dagger} is formed only when it is asked for.
int rr_impl(pw_ctx* ctx, double2* Y, int64_t ldy, int m, double2* hpsi_out, double* eig_h, double* resid_h,
            double2* q_out = nullptr, double2* x_out = nullptr, double* eig_dev_out = nullptr) {
  PW_TRY(check_tc_flag(ctx));
  ProfScope rr_scope(ctx, PW_PROF_RR);
  const int npw = ctx->npw;
  const cudaStream_t st = ctx->stream;
  WS(HY, double2, WS_HY, (size_t)npw * m);
  WS(SYb, double2, WS_SY, (size_t)npw * m);
  WS(ROT, double2, WS_ROT, (size_t)npw * m);
  WS(G, double2, WS_GRAM, (size_t)m * m);
  WS(G2, double2, WS_GRAM2, (size_t)m * m);
  WS(Linv, double2, WS_LINV, (size_t)m * m);
  WS(tmp, double2, WS_TMP, (size_t)m * m);
  WS(U, double2, WS_U, (size_t)m * m);
  WS(jac, double2, WS_JAC, (size_t)3 * m * m + m + 2);
  WS(eig, double, WS_EIG, (size_t)2 * m + 4);
  WS(scal, int, WS_SCAL, 16);
  double* norms = eig + 2 * m;
  double* resid = eig + m;
  CU_TRY(cudaMemsetAsync(scal, 0, 16 * sizeof(int), st), "flag reset");
  // first Cholesky-QR pass in the S metric: Y <- Y L^{-dagger}
  {
    const double2* SY = Y;
    int64_t lds = ldy;
    if (ctx->has_q) {
      PW_TRY(apply_s64(ctx, Y, ldy, m, SYb, npw));
      SY = SYb;
      lds = npw;
    }
    PW_TRY(gram_chol(ctx, Y, ldy, SY, lds, m, G, Linv, tmp, scal));
    PW_TRY(cg<double>(ctx, 0, 1, npw, m, m, Y, ldy, Linv, m, epi<double>(EPI_STORE, ROT, npw), 1, nullptr, st, GEMM_B_UPPER, "s-ortho rotate"));
    CU_TRY(cudaMemcpy2DAsync(Y, sizeof(double2) * ldy, ROT, sizeof(double2) * npw, sizeof(double2) * npw, m,
                             cudaMemcpyDeviceToDevice, st), "s-ortho copy");
  }
  PW_TRY(check_flag(ctx, scal, "S-Ortho Cholesky"));
  // H Psi, S Psi
  PW_TRY(apply_impl<double>(ctx, Y, ldy, m, HY, ctx->has_q ? SYb : nullptr, npw));
  const double2* SY = ctx->has_q ? SYb : Y;
  const int64_t lds = ctx->has_q ? npw : ldy;
  // H_Psi = Psi^dagger (H Psi) -> G2
  PW_TRY(gram_herm(ctx, Y, ldy, HY, npw, m, G2));
  // S_Psi -> G, Cholesky (the second S-Ortho pass), Linv
  PW_TRY(gram_chol(ctx, Y, ldy, SY, lds, m, G, Linv, tmp, scal));
  // Cm = Linv H_Psi Linv^dagger
  CU_TRY(launch_cgemm<double>(0, 1, m, m, m, G2, m, Linv, m, epi<double>(EPI_STORE, tmp, m), 1, nullptr, st), "reduce 1");
  CU_TRY(launch_cgemm<double>(0, 0, m, m, m, Linv, m, tmp, m, epi<double>(EPI_STORE, G, m), 1, nullptr, st), "reduce 2");
  CU_TRY(la_herm_sym(G, m, m, st), "reduced sym");
  PW_TRY(check_flag(ctx, scal, "Rayleigh-Ritz Cholesky"));
  int sweeps = 0;
  PW_TRY(eigh_impl(ctx, G, m, U, eig, jac, norms, &sweeps));
  ctx->last_sweeps = sweeps;
  // X = Linv^dagger U  -> tmp
  CU_TRY(launch_cgemm<double>(1, 0, m, m, m, Linv, m, U, m, epi<double>(EPI_STORE, tmp, m), 1, nullptr, st), "back-transform");
  if (q_out)
    PW_TRY(cg<double>(ctx, 0, 1, npw, m, m, Y, ldy, Linv, m, epi<double>(EPI_STORE, q_out, npw), 1, nullptr, st, GEMM_B_UPPER, "Q"));
  if (x_out) CU_TRY(cudaMemcpyAsync(x_out, U, sizeof(double2) * m * m, cudaMemcpyDeviceToDevice, st), "copy X");
  if (eig_dev_out)
    CU_TRY(cudaMemcpyAsync(eig_dev_out, eig, sizeof(double) * m, cudaMemcpyDeviceToDevice, st), "copy eig");
  // rotate Y, HY, SY
  PW_TRY(cg<double>(ctx, 0, 0, npw, m, m, Y, ldy, tmp, m, epi<double>(EPI_STORE, ROT, npw), 1, nullptr, st, GEMM_FULL, "rotate Y"));
  CU_TRY(cudaMemcpy2DAsync(Y, sizeof(double2) * ldy, ROT, sizeof(double2) * npw, sizeof(double2) * npw, m,
                           cudaMemcpyDeviceToDevice, st), "rotate copy");
  PW_TRY(cg<double>(ctx, 0, 0, npw, m, m, HY, npw, tmp, m, epi<double>(EPI_STORE, ROT, npw), 1, nullptr, st, GEMM_FULL, "rotate HY"));
  double2* HYr = ROT;
  const double2* SYr = Y;
  int64_t ldsr = ldy;
  if (ctx->has_q) {
    PW_TRY(cg<double>(ctx, 0, 0, npw, m, m, SYb, npw, tmp, m, epi<double>(EPI_STORE, HY, npw), 1, nullptr, st, GEMM_FULL, "rotate SY"));
    SYr = HY;
    ldsr = npw;
  }
  CU_TRY(la_resid(HYr, npw, SYr, ldsr, npw, m, eig, resid, st), "residuals");
  if (hpsi_out)
    CU_TRY(cudaMemcpy2DAsync(hpsi_out, sizeof(double2) * ldy, HYr, sizeof(double2) * npw, sizeof(double2) * npw, m,
                             cudaMemcpyDeviceToDevice, st), "copy H psi");
  if (eig_h) CU_TRY(cudaMemcpyAsync(eig_h, eig, sizeof(double) * m, cudaMemcpyDeviceToHost, st), "eig copy");
  if (resid_h) CU_TRY(cudaMemcpyAsync(resid_h, resid, sizeof(double) * m, cudaMemcpyDeviceToHost, st), "resid copy");
  CU_TRY(cudaStreamSynchronize(st), "rr sync");
  return PW_OK;
}

// ---------------------------------------------------------------------------
// LOBPCG with b blocks and k line minimisations (Alg. 11), FP64, with S-Deflate (Alg. 8),
// S-Ortho (Alg. 9) and RR (Alg. 10) as its steps
// ---------------------------------------------------------------------------
// S-Ortho of the k columns of X with H X and S X: S_X = X^dagger S X = L L^dagger (Cholesky),
// each block <- (.) L^{-dagger}.  tmp: npw x k scratch (ld npw).
int sortho3(pw_ctx* ctx, double2* X, int64_t ldx, double2* HX, int64_t ldh, double2* SX, int64_t lds, int k,
            double2* tmp, int* flag, const char* what) {
  const int npw = ctx->npw;
  const cudaStream_t st = ctx->stream;
  WS(G, double2, WS_GRAM, (size_t)k * k);
  WS(Linv, double2, WS_LINV, (size_t)k * k);
  WS(t, double2, WS_TMP, (size_t)k * k);
  CU_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st), "flag reset");
  PW_TRY(gram_chol(ctx, X, ldx, SX, lds, k, G, Linv, t, flag));
  PW_TRY(check_flag(ctx, flag, what));
  double2* blocks[3] = {X, HX, SX};
  const int64_t lds3[3] = {ldx, ldh, lds};
  for (int b = 0; b < 3; ++b) {
    PW_TRY(cg<double>(ctx, 0, 1, npw, k, k, blocks[b], lds3[b], Linv, k, epi<double>(EPI_STORE, tmp, npw), 1, nullptr,
                      st, GEMM_B_UPPER, "s-ortho rotate"));
    CU_TRY(cudaMemcpy2DAsync(blocks[b], sizeof(double2) * lds3[b], tmp, sizeof(double2) * npw, sizeof(double2) * npw,
                             k, cudaMemcpyDeviceToDevice, st), "s-ortho copy");
  }
  return PW_OK;
}

// RR on the basis Z (k columns) with H Z, S Z: H_Z x = lambda S_Z x by Cholesky reduction and the
// Hermitian eigensolver; C (k x k, ld k) <- the eigenvector coefficients (ascending Ritz values,
// so the first `keep` columns are the kept pairs), *eig_dev <- the Ritz values (device, k)
int rr_coeffs(pw_ctx* ctx, const double2* Z, int64_t ldz, const double2* HZ, int64_t ldh, const double2* SZ,
              int64_t lds, int k, double2* C, double** eig_dev, int* flag) {
  const cudaStream_t st = ctx->stream;
  WS(G, double2, WS_GRAM, (size_t)k * k);
  WS(G2, double2, WS_GRAM2, (size_t)k * k);
  WS(Linv, double2, WS_LINV, (size_t)k * k);
  WS(tmp, double2, WS_TMP, (size_t)k * k);
  WS(U, double2, WS_U, (size_t)k * k);
  WS(jac, double2, WS_JAC, (size_t)3 * k * k + k + 2);
  WS(ev, double, WS_EIG, (size_t)2 * k + 4);
  CU_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st), "flag reset");
  PW_TRY(gram_herm(ctx, Z, ldz, HZ, ldh, k, G2));
  PW_TRY(gram_chol(ctx, Z, ldz, SZ, lds, k, G, Linv, tmp, flag));
  CU_TRY(launch_cgemm<double>(0, 1, k, k, k, G2, k, Linv, k, epi<double>(EPI_STORE, tmp, k), 1, nullptr, st), "reduce 1");
  CU_TRY(launch_cgemm<double>(0, 0, k, k, k, Linv, k, tmp, k, epi<double>(EPI_STORE, G, k), 1, nullptr, st), "reduce 2");
  CU_TRY(la_herm_sym(G, k, k, st), "reduced sym");
  PW_TRY(check_flag(ctx, flag, "LOBPCG Rayleigh-Ritz Cholesky"));
  int sweeps = 0;
  PW_TRY(eigh_impl(ctx, G, k, U, ev, jac, ev + 2 * k, &sweeps));
  CU_TRY(launch_cgemm<double>(1, 0, k, k, k, Linv, k, U, k, epi<double>(EPI_STORE, C, k), 1, nullptr, st), "back-transform");
  *eig_dev = ev;
  return PW_OK;
}

int lobpcg_impl(pw_ctx* ctx, double2* psi, int64_t ld, int M, int nblk, int nline, double tol, double* eig_h,
                double* resid_h, int* its_h) {
  PW_TRY(check_tc_flag(ctx));
  const int npw = ctx->npw, bs = M / nblk;
  const cudaStream_t st = ctx->stream;
  const size_t zs = (size_t)npw * 3 * bs;  // one of Z = [Psi_i W_i P_i], H Z, S Z
  WS(Zb, double2, WS_LOBZ, 3 * zs);
  WS(T, double2, WS_LOBT, (size_t)npw * std::max(3 * bs, M));
  WS(HY, double2, WS_HY, (size_t)npw * M);
  WS(SY, double2, WS_SY, (size_t)npw * M);
  const size_t kc = std::max((size_t)9 * bs * bs, (size_t)M * M);
  WS(Bb, double2, WS_LOBB, (size_t)6 * bs * bs + kc);
  double2* B = Bb;            // [C without the Psi rows | C], 3bs x 2bs
  double2* Cf = Bb + (size_t)6 * bs * bs;
  WS(R, double, WS_LOBR, (size_t)3 * M + 16);
  double* lam_all = R;         // device Ritz values, block by block
  double* rn = R + M;          // residual norms of the current block
  double* res_all = R + 2 * M;
  WS(dfl, double2, WS_LOBD, (size_t)M * bs);
  WS(scal, int, WS_SCAL, 16);
  double2 *Z = Zb, *HZ = Zb + zs, *SZ = Zb + 2 * zs;
  const size_t cb = (size_t)npw * bs;  // one column block
  std::vector<double> rn_h(bs);
  for (int i = 0; i < nblk; ++i) {
    double* lam = lam_all + (size_t)i * bs;
    const int mp = i * bs;
    // S-Deflate of A (bs columns, ld npw) against the finished blocks psi[:, 0:mp] (S psi in SY)
    auto deflate = [&](double2* A) -> int {
      PW_TRY(cg<double>(ctx, 1, 0, mp, bs, npw, SY, npw, A, npw, epi<double>(EPI_STORE, dfl, mp), 1, nullptr, st,
                        GEMM_FULL, "s-deflate overlap"));
      PW_TRY(cg<double>(ctx, 0, 0, npw, bs, mp, psi, ld, dfl, mp, epi<double>(EPI_ACCUM, A, npw, -1.0), 1, nullptr, st,
                        GEMM_FULL, "s-deflate update"));
      return PW_OK;
    };
    CU_TRY(cudaMemcpy2DAsync(Z, sizeof(double2) * npw, psi + (size_t)i * bs * ld, sizeof(double2) * ld,
                             sizeof(double2) * npw, bs, cudaMemcpyDeviceToDevice, st), "block copy");
    if (i > 0) PW_TRY(deflate(Z));
    PW_TRY(apply_impl<double>(ctx, Z, npw, bs, HZ, SZ, npw));
    PW_TRY(sortho3(ctx, Z, npw, HZ, npw, SZ, npw, bs, T, scal, "LOBPCG S-Ortho"));
    double* ev = nullptr;
    PW_TRY(rr_coeffs(ctx, Z, npw, HZ, npw, SZ, npw, bs, Cf, &ev, scal));
    for (double2* A : {Z, HZ, SZ}) {
      PW_TRY(cg<double>(ctx, 0, 0, npw, bs, bs, A, npw, Cf, bs, epi<double>(EPI_STORE, T, npw), 1, nullptr, st,
                        GEMM_FULL, "LOBPCG rotation"));
      CU_TRY(cudaMemcpyAsync(A, T, sizeof(double2) * cb, cudaMemcpyDeviceToDevice, st), "rotation copy");
    }
    CU_TRY(cudaMemcpyAsync(lam, ev, sizeof(double) * bs, cudaMemcpyDeviceToDevice, st), "Ritz values");
    int done = 0;
    for (int n = 0; n < nline; ++n) {
      // W = K (H - Lambda S) Psi_i; the block's line loop ends once every residual is below tol
      CU_TRY(la_lob_resid(HZ, SZ, Z, npw, npw, bs, lam, ctx->kin64, Z + cb, npw, rn, st), "LOBPCG residual");
      CU_TRY(cudaMemcpyAsync(rn_h.data(), rn, sizeof(double) * bs, cudaMemcpyDeviceToHost, st), "residual copy");
      CU_TRY(cudaStreamSynchronize(st), "residual sync");
      if (*std::max_element(rn_h.begin(), rn_h.end()) < tol) break;
      if (i > 0) PW_TRY(deflate(Z + cb));
      PW_TRY(apply_impl<double>(ctx, Z + cb, npw, bs, HZ + cb, SZ + cb, npw));
      const int kz = n == 0 ? 2 * bs : 3 * bs;
      PW_TRY(sortho3(ctx, Z, npw, HZ, npw, SZ, npw, kz, T, scal, "LOBPCG S-Ortho"));
      PW_TRY(rr_coeffs(ctx, Z, npw, HZ, npw, SZ, npw, kz, Cf, &ev, scal));
      CU_TRY(la_lob_coef(Cf, kz, bs, B, st), "LOBPCG coefficients");
      // [P_new | Psi_new] = Z B for Z, H Z, S Z; Psi_new = Psi part + P_new
      for (double2* A : {Z, HZ, SZ}) {
        PW_TRY(cg<double>(ctx, 0, 0, npw, 2 * bs, kz, A, npw, B, kz, epi<double>(EPI_STORE, T, npw), 1, nullptr, st,
                          GEMM_FULL, "LOBPCG update"));
        CU_TRY(cudaMemcpyAsync(A, T + cb, sizeof(double2) * cb, cudaMemcpyDeviceToDevice, st), "Psi update");
        CU_TRY(cudaMemcpyAsync(A + 2 * cb, T, sizeof(double2) * cb, cudaMemcpyDeviceToDevice, st), "P update");
      }
      CU_TRY(cudaMemcpyAsync(lam, ev, sizeof(double) * bs, cudaMemcpyDeviceToDevice, st), "Ritz values");
      done = n + 1;
    }
    if (its_h) its_h[i] = done;
    CU_TRY(cudaMemcpy2DAsync(psi + (size_t)i * bs * ld, sizeof(double2) * ld, Z, sizeof(double2) * npw,
                             sizeof(double2) * npw, bs, cudaMemcpyDeviceToDevice, st), "block store");
    CU_TRY(cudaMemcpyAsync(HY + (size_t)i * cb, HZ, sizeof(double2) * cb, cudaMemcpyDeviceToDevice, st), "H block");
    CU_TRY(cudaMemcpyAsync(SY + (size_t)i * cb, SZ, sizeof(double2) * cb, cudaMemcpyDeviceToDevice, st), "S block");
  }
  if (nblk > 1) {  // global S-Ortho + RR over all the bands
    PW_TRY(sortho3(ctx, psi, ld, HY, npw, SY, npw, M, T, scal, "LOBPCG final S-Ortho"));
    double* ev = nullptr;
    PW_TRY(rr_coeffs(ctx, psi, ld, HY, npw, SY, npw, M, Cf, &ev, scal));
    double2* blocks[3] = {psi, HY, SY};
    const int64_t lds3[3] = {ld, npw, npw};
    for (int b = 0; b < 3; ++b) {
      PW_TRY(cg<double>(ctx, 0, 0, npw, M, M, blocks[b], lds3[b], Cf, M, epi<double>(EPI_STORE, T, npw), 1, nullptr,
                        st, GEMM_FULL, "LOBPCG final rotation"));
      CU_TRY(cudaMemcpy2DAsync(blocks[b], sizeof(double2) * lds3[b], T, sizeof(double2) * npw, sizeof(double2) * npw,
                               M, cudaMemcpyDeviceToDevice, st), "final rotation copy");
    }
    CU_TRY(cudaMemcpyAsync(lam_all, ev, sizeof(double) * M, cudaMemcpyDeviceToDevice, st), "Ritz values");
  }
  CU_TRY(la_resid(HY, npw, SY, npw, npw, M, lam_all, res_all, st), "residuals");
  CU_TRY(cudaMemcpyAsync(eig_h, lam_all, sizeof(double) * M, cudaMemcpyDeviceToHost, st), "eig copy");
  if (resid_h) CU_TRY(cudaMemcpyAsync(resid_h, res_all, sizeof(double) * M, cudaMemcpyDeviceToHost, st), "resid copy");
  CU_TRY(cudaStreamSynchronize(st), "LOBPCG sync");
  return PW_OK;
}

// ---------------------------------------------------------------------------
// Spectrum slicing (the slice-wise solve the paper's closing section proposes)
// ---------------------------------------------------------------------------
// Jackson-damped Chebyshev coefficients of the indicator of [a, b] for a spectrum inside
// [lo, hi] (mapped to [-1, 1]; the slice clipped to it): out[j] = g_j mu_j, j = 0..degree
void window_coefficients(int degree, double a, double b, double lo, double hi, double* out) {
  const double pi = 3.14159265358979323846264338327950288;
  const double c = 0.5 * (hi + lo), e = 0.5 * (hi - lo);
  const double ta = std::min(std::max((a - c) / e, -1.0), 1.0), tb = std::min(std::max((b - c) / e, -1.0), 1.0);
  const double tha = std::acos(ta), thb = std::acos(tb);
  const double al = pi / (degree + 2);
  for (int j = 0; j <= degree; ++j) {
    const double g = ((1.0 - (double)j / (degree + 2)) * std::sin(al) * std::cos(j * al) +
                      std::cos(al) * std::sin(j * al) / (degree + 2)) / std::sin(al);
    const double mu = j == 0 ? (tha - thb) / pi : 2.0 * (std::sin(j * tha) - std::sin(j * thb)) / (j * pi);
    out[j] = g * mu;
  }
}

int check_slices(int nslice, int nper, int degree, double lo, double hi, const double* cuts) {
  if (nslice < 1 || nper < 1) return set_error(PW_EINVAL, "nslice and nper must be positive");
  if (degree < 1) return set_error(PW_EINVAL, "degree must be positive");
  if (!(hi > lo)) return set_error(PW_EINVAL, "spectrum bounds need hi > lo");
  if (!cuts) return set_error(PW_EINVAL, "NULL cuts");
  for (int s = 0; s < nslice; ++s)
    if (!(cuts[s + 1] > cuts[s])) return set_error(PW_EINVAL, "cuts must be strictly ascending");
  return PW_OK;
}

// every slice block of psi (nslice x nper bands) <- its window applied to it, one recurrence
template <typename T>
int slice_filter_impl(pw_ctx* ctx, cplx<T>* psi, int64_t ld, int nslice, int nper, int degree, double lo, double hi,
                      const double* cuts) {
  const int npw = ctx->npw, nband = nslice * nper;
  const cudaStream_t st = ctx->stream;
  std::vector<double> w(degree + 1), coef((size_t)(degree + 1) * nband);
  for (int s = 0; s < nslice; ++s) {
    window_coefficients(degree, cuts[s], cuts[s + 1], lo, hi, w.data());
    for (int k = 0; k <= degree; ++k)
      for (int j = 0; j < nper; ++j) coef[(size_t)k * nband + s * nper + j] = w[k];
  }
  WS(cd, double, WS_SLICEC, coef.size());
  WS(acc, cplx<T>, WS_SLICEA, (size_t)npw * nband);
  CU_TRY(cudaMemcpyAsync(cd, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, st), "coefficients");
  ChebSum<T> cs{acc, npw, cd};
  PW_TRY(filter_impl<T>(ctx, psi, ld, nband, degree, lo, hi, nullptr, &cs));
  CU_TRY(cudaMemcpy2DAsync(psi, sizeof(cplx<T>) * ld, acc, sizeof(cplx<T>) * npw, sizeof(cplx<T>) * npw, nband,
                           cudaMemcpyDeviceToDevice, st), "slice copy-out");
  CU_TRY(cudaStreamSynchronize(st), "slice sync");  // the host coefficients go out of scope
  return PW_OK;
}

struct LzCtx { pw_ctx* ctx; };
int lz_apply(void* p, const double2* v, double2* w) {
  pw_ctx* ctx = ((LzCtx*)p)->ctx;
  return apply_impl<double>(ctx, v, ctx->npw, 1, w, nullptr, ctx->npw);
}

int bounds_impl(pw_ctx* ctx, const double2* psi, int64_t ld, int nband, int steps, const double2* v0,
                double* rq_min, double* rq_max, double* upper) {
  const int npw = ctx->npw;
  const cudaStream_t st = ctx->stream;
  WS(rq, double2, WS_RQ, (size_t)3 * nband + 8);
  if (nband > 0) {
    WS(HY, double2, WS_HY, (size_t)npw * nband);
    WS(SYb, double2, WS_SY, (size_t)npw * nband);
    PW_TRY(apply_impl<double>(ctx, psi, ld, nband, HY, ctx->has_q ? SYb : nullptr, npw));
    const double2* SY = ctx->has_q ? SYb : psi;
    const int64_t lds = ctx->has_q ? npw : ld;
    CU_TRY(la_coldot(psi, ld, HY, npw, npw, nband, rq, st), "rq num");
    CU_TRY(la_coldot(psi, ld, SY, lds, npw, nband, rq + nband, st), "rq den");
    double* mm = (double*)(rq + 2 * nband);
    double* rqv = (double*)(rq + 2 * nband + 1);
    CU_TRY(la_rq_minmax(rq, rq + nband, nband, rqv, mm, st), "rq minmax");
    double h[2];
    CU_TRY(cudaMemcpyAsync(h, mm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "rq copy");
    CU_TRY(cudaStreamSynchronize(st), "rq sync");
    if (rq_min) *rq_min = h[0];
    if (rq_max) *rq_max = h[1];
  }
  if (steps > 0) {
    if (!v0) return set_error(PW_EINVAL, "Lanczos start vector is NULL");
    WS(lz, double2, WS_LZ, (size_t)3 * npw + 2 * steps + 8);
    double* ab = (double*)(lz + 3 * npw);
    double* bound = ab + 2 * steps;
    LzCtx lc{ctx};
    CU_TRY(la_lanczos(v0, npw, steps, lz, lz + npw, lz + 2 * npw, ab, bound, lz_apply, &lc, st), "lanczos");
    double h[2];
    CU_TRY(cudaMemcpyAsync(h, bound, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "bound copy");
    CU_TRY(cudaStreamSynchronize(st), "bound sync");
    if (upper) *upper = h[0];
  }
  return PW_OK;
}

int check_ctx(pw_ctx* ctx) {
  if (!ctx) return set_error(PW_EINVAL, "NULL context");
  if (ctx->poisoned) return set_error(PW_ECUDA, "context poisoned by an earlier CUDA error");
  return PW_OK;
}

int check_block(pw_ctx* ctx, const void* p, int64_t ld, int nband) {
  if (nband < 0) return set_error(PW_EINVAL, "nband < 0");
  if (nband > 0 && !p) return set_error(PW_EINVAL, "NULL block");
  if (ld < ctx->npw) return set_error(PW_EINVAL, "ld (%lld) < npw (%d)", (long long)ld, ctx->npw);
  return PW_OK;
}

// ---------------------------------------------------------------------------
// context creation
// ---------------------------------------------------------------------------
int create_impl(const pw_problem_desc* d, void* stream, pw_ctx** out) {
  if (!d || !out) return set_error(PW_EINVAL, "NULL argument");
  *out = nullptr;
  if (!d->vloc) return set_error(PW_EINVAL, "vloc is NULL");
  const bool given_p = d->proj != nullptr;
  if (given_p) {
    if (d->nproj < 1) return set_error(PW_EINVAL, "explicit projectors need nproj >= 1 (got %d)", d->nproj);
    if (!d->D) return set_error(PW_EINVAL, "explicit projectors need D");
  } else {
    if (d->natom < 0 || d->nchan < 0 || d->nchan > kMaxChan) return set_error(PW_EINVAL, "bad natom/nchan");
    if (d->natom > 0 && (!d->tau || !d->sigma || !d->D)) return set_error(PW_EINVAL, "tau/sigma/D missing");
  }
  if (!(d->ecut > 0)) return set_error(PW_EINVAL, "ecut must be positive");
  pw_ctx* ctx = new (std::nothrow) pw_ctx();
  if (!ctx) return set_error(PW_ENOMEM, "host allocation");
  *out = ctx;  // destroyed by the caller-facing wrapper on failure
  ctx->stream = (cudaStream_t)stream;
  memcpy(ctx->lattice, d->lattice, sizeof(ctx->lattice));
  memcpy(ctx->kpt, d->kpt, sizeof(ctx->kpt));
  ctx->ecut = d->ecut;
  for (int i = 0; i < 3; ++i) {
    ctx->n[i] = d->box[i];
    if (!factorize(d->box[i], ctx->plan.d[i]))
      return set_error(PW_EUNSUPPORTED, "box length %d does not factor into 2, 3, 5", d->box[i]);
    ctx->plan.n[i] = d->box[i];
  }
  // reciprocal vectors, rows b_i
  double Ainv[9], B[9];
  inv3(d->lattice, Ainv);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[i * 3 + j] = 2.0 * kPi * Ainv[j * 3 + i];
  double kc[3];
  for (int c = 0; c < 3; ++c) kc[c] = d->kpt[0] * B[c] + d->kpt[1] * B[3 + c] + d->kpt[2] * B[6 + c];
  const double gmax = sqrt(2.0 * d->ecut);
  const double kn = sqrt(kc[0] * kc[0] + kc[1] * kc[1] + kc[2] * kc[2]);
  int lim[3];
  for (int i = 0; i < 3; ++i) {
    const double an = sqrt(d->lattice[3 * i] * d->lattice[3 * i] + d->lattice[3 * i + 1] * d->lattice[3 * i + 1] +
                           d->lattice[3 * i + 2] * d->lattice[3 * i + 2]);
    lim[i] = (int)ceil((gmax + kn) * an / (2.0 * kPi)) + 1;
  }
  // sphere, already in ascending (h, k, l) order by construction of the loops
  std::vector<int> pl_h, pl_row0, rk, rl0, rcnt, rg0;
  int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int h = -lim[0]; h <= lim[0]; ++h) {
    bool plane_open = false;
    for (int k = -lim[1]; k <= lim[1]; ++k) {
      bool in_run = false;
      int last_l = 0;
      for (int l = -lim[2]; l <= lim[2]; ++l) {
        double q[3];
        for (int c = 0; c < 3; ++c) q[c] = h * B[c] + k * B[3 + c] + l * B[6 + c] + kc[c];
        const double t = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (t <= d->ecut) {
          if (!plane_open) {
            pl_h.push_back(h);
            pl_row0.push_back((int)rk.size());
            plane_open = true;
          }
          if (!in_run) {
            in_run = true;
            rk.push_back(k);
            rl0.push_back(l);
            rcnt.push_back(0);
            rg0.push_back(ctx->npw);
          } else if (l != last_l + 1) {
            return set_error(PW_EINVAL, "sphere row is not a contiguous run");
          }
          last_l = l;
          rcnt.back()++;
          ctx->miller.push_back(h);
          ctx->miller.push_back(k);
          ctx->miller.push_back(l);
          ctx->kin_h.push_back(t);
          const int m3[3] = {h, k, l};
          for (int c = 0; c < 3; ++c) { mn[c] = std::min(mn[c], m3[c]); mx[c] = std::max(mx[c], m3[c]); }
          ctx->npw++;
        }
      }
    }
  }
  pl_row0.push_back((int)rk.size());
  if (ctx->npw == 0) return set_error(PW_EINVAL, "empty plane-wave sphere");
  for (size_t p = 0; p < pl_h.size(); ++p)
    if (pl_h[p] != pl_h[0] + (int)p) return set_error(PW_EINVAL, "sphere x-planes are not a contiguous range");
  for (int c = 0; c < 3; ++c)
    if (mx[c] - mn[c] >= d->box[c]) return set_error(PW_EINVAL, "plane-wave sphere does not fit in the FFT box");
  ctx->sp.npw = ctx->npw;
  ctx->sp.nplane = (int)pl_h.size();
  ctx->sp.nrow = (int)rk.size();
  ctx->sp.max_rows = 0;
  for (int p = 0; p < ctx->sp.nplane; ++p) ctx->sp.max_rows = std::max(ctx->sp.max_rows, pl_row0[p + 1] - pl_row0[p]);
  ctx->sp.max_plane_g = 0;
  for (int p = 0; p < ctx->sp.nplane; ++p)  // a plane's coefficients are one contiguous block of the sphere
    ctx->sp.max_plane_g = std::max(ctx->sp.max_plane_g,
                                   (pl_row0[p + 1] < (int)rg0.size() ? rg0[pl_row0[p + 1]] : ctx->npw) -
                                       rg0[pl_row0[p]]);
  int* dv;
  PW_TRY(upload(ctx, &dv, pl_h.data(), pl_h.size())); ctx->sp.plane_h = dv;
  PW_TRY(upload(ctx, &dv, pl_row0.data(), pl_row0.size())); ctx->sp.plane_row0 = dv;
  PW_TRY(upload(ctx, &dv, rk.data(), rk.size())); ctx->sp.row_k = dv;
  PW_TRY(upload(ctx, &dv, rl0.data(), rl0.size())); ctx->sp.row_l0 = dv;
  PW_TRY(upload(ctx, &dv, rcnt.data(), rcnt.size())); ctx->sp.row_cnt = dv;
  PW_TRY(upload(ctx, &dv, rg0.data(), rg0.size())); ctx->sp.row_g0 = dv;
  int* miller_dev;
  PW_TRY(upload(ctx, &miller_dev, ctx->miller.data(), ctx->miller.size()));
  PW_TRY(upload(ctx, &ctx->kin64, ctx->kin_h.data(), ctx->kin_h.size()));
  std::vector<float> kin32(ctx->kin_h.begin(), ctx->kin_h.end());
  PW_TRY(upload(ctx, &ctx->kin32, kin32.data(), kin32.size()));
  // twiddles e^{-2 pi i j m / L}
  std::vector<double2> tw;
  for (int dd = 0; dd < 3; ++dd) {
    FftDim& f = ctx->plan.d[dd];
    f.tw_base = (int)tw.size();
    for (int s = 0; s < f.nst; ++s) {
      f.tw_off[s] = (int)tw.size();
      const int L = f.L[s], r = f.radix[s], q = L / r;
      for (int j = 0; j < q; ++j)
        for (int m = 1; m < r; ++m) {
          const long jm = ((long)j * m) % L;
          const double ang = -2.0 * kPi * (double)jm / (double)L;
          tw.push_back(make_double2(cos(ang), sin(ang)));
        }
    }
    f.tw_count = (int)tw.size() - f.tw_base;
  }
  std::vector<float2> tw32(tw.size());
  for (size_t i = 0; i < tw.size(); ++i) tw32[i] = make_float2((float)tw[i].x, (float)tw[i].y);
  PW_TRY(upload(ctx, &ctx->tw64, tw.data(), tw.size()));
  PW_TRY(upload(ctx, &ctx->tw32, tw32.data(), tw32.size()));
  for (int dd = 0; dd < 3; ++dd) {
    std::vector<int> r = digit_reversal(ctx->plan.d[dd]);
    PW_TRY(upload(ctx, &ctx->rho_perm[dd], r.data(), r.size()));
  }
  const cudaStream_t st = ctx->stream;
  CU_TRY(fft_set_constants(), "FFT constants");
  // permuted potential, scaled by 1 / n1n2n3 (the forward DFT normalisation)
  const size_t ntot = (size_t)d->box[0] * d->box[1] * d->box[2];
  double* vraw;
  PW_TRY(upload(ctx, &vraw, d->vloc, ntot));
  PW_TRY(upload(ctx, &ctx->vperm64, (const double*)nullptr, ntot));
  PW_TRY(upload(ctx, &ctx->vperm32, (const float*)nullptr, ntot));
  CU_TRY(setup_vperm(vraw, ctx->n, ctx->rho_perm, 1.0 / (double)ntot, ctx->vperm64, ctx->vperm32, st), "vperm");
  {
    const FftDim& dx = ctx->plan.d[0];
    if (dx.nst == 2 && dx.radix[0] != dx.radix[1]) {
      FftDim sw = dx;
      sw.radix[0] = dx.radix[1];
      sw.radix[1] = dx.radix[0];
      sw.L[1] = dx.n / sw.radix[0];
      std::vector<int> r = digit_reversal(sw);
      PW_TRY(upload(ctx, &ctx->rho_x_sw, r.data(), r.size()));
      PW_TRY(upload(ctx, &ctx->vperm32_sw, (const float*)nullptr, ntot));
      int* rho_sw[3] = {ctx->rho_x_sw, ctx->rho_perm[1], ctx->rho_perm[2]};
      CU_TRY(setup_vperm32(vraw, ctx->n, rho_sw, 1.0 / (double)ntot, ctx->vperm32_sw, st), "vperm (swapped x plan)");
    }
  }
  // projectors
  ctx->natom = given_p ? 0 : d->natom;
  ctx->nchan = given_p ? 0 : d->nchan;
  ctx->nproj = given_p ? d->nproj : d->natom * d->nchan * 4;
  const int np = ctx->nproj;
  PW_TRY(upload(ctx, &ctx->P64, given_p ? (const double2*)d->proj : (const double2*)nullptr,
                (size_t)ctx->npw * std::max(np, 1)));
  PW_TRY(upload(ctx, &ctx->P32, (const float2*)nullptr, (size_t)ctx->npw * std::max(np, 1)));
  if (given_p) {
    CU_TRY(cast_z2c(ctx->P64, ctx->P32, (int64_t)ctx->npw * np, st), "P cast");
  } else if (np > 0) {
    ProjParams pp;
    memcpy(pp.B, B, sizeof(B));
    memcpy(pp.kred, d->kpt, sizeof(pp.kred));
    double* tau_dev;
    PW_TRY(upload(ctx, &tau_dev, d->tau, (size_t)3 * d->natom));
    pp.tau = tau_dev;
    pp.nchan = d->nchan;
    for (int c = 0; c < d->nchan; ++c) pp.sigma[c] = d->sigma[c];
    CU_TRY(setup_projectors(ctx->npw, miller_dev, pp, d->natom, ctx->P64, st), "projectors");
    CU_TRY(cast_z2c(ctx->P64, ctx->P32, (int64_t)ctx->npw * np, st), "P cast");
  }
  // D and its block structure
  std::vector<double> Dh(std::max(np * np, 1), 0.0);
  if (np > 0) memcpy(Dh.data(), d->D, sizeof(double) * np * np);
  std::vector<int> b0, bl;
  block_structure(Dh.data(), np, b0, bl);
  PW_TRY(upload(ctx, &ctx->D64, Dh.data(), Dh.size()));
  PW_TRY(upload(ctx, &ctx->D32, (const float*)nullptr, Dh.size()));
  CU_TRY(cast_d2f(ctx->D64, ctx->D32, (int64_t)Dh.size(), st), "D cast");
  ctx->blk0_h = b0;
  ctx->blklen_h = bl;
  PW_TRY(upload(ctx, &ctx->blk0, b0.data(), std::max<size_t>(b0.size(), 1)));
  PW_TRY(upload(ctx, &ctx->blklen, bl.data(), std::max<size_t>(bl.size(), 1)));
  // Woodbury matrices for S^-1 (Sec. 3.3): K = (Q^-1 + P^dagger P)^-1, E = (I - K P^dagger P) D
  ctx->has_q = (d->Q != nullptr) && np > 0;
  if (ctx->has_q) {
    std::vector<int> qb0, qbl;
    block_structure(d->Q, np, qb0, qbl);
    PW_TRY(upload(ctx, &ctx->Q64, d->Q, (size_t)np * np));
    PW_TRY(upload(ctx, &ctx->qblk0, qb0.data(), qb0.size()));
    PW_TRY(upload(ctx, &ctx->qblklen, qbl.data(), qbl.size()));
    const size_t nn = (size_t)np * np;
    double2 *Bm, *Qz, *Li, *tmp, *Dz;
    PW_TRY(upload(ctx, &ctx->K64, (const double2*)nullptr, nn));
    PW_TRY(upload(ctx, &ctx->E64, (const double2*)nullptr, nn));
    PW_TRY(upload(ctx, &ctx->K32, (const float2*)nullptr, nn));
    PW_TRY(upload(ctx, &ctx->E32, (const float2*)nullptr, nn));
    PW_TRY(upload(ctx, &Bm, (const double2*)nullptr, nn));
    PW_TRY(upload(ctx, &Qz, (const double2*)nullptr, nn));
    PW_TRY(upload(ctx, &Li, (const double2*)nullptr, nn));
    PW_TRY(upload(ctx, &tmp, (const double2*)nullptr, nn));
    PW_TRY(upload(ctx, &Dz, (const double2*)nullptr, nn));
    int* flag;
    PW_TRY(upload(ctx, &flag, (const int*)nullptr, 1));
    CU_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st), "flag");
    const int ns = nsplit_for(np, np, ctx->npw);
    double2* spl;
    PW_TRY(upload(ctx, &spl, (const double2*)nullptr, (size_t)ns * nn));
    // B = P^dagger P
    CU_TRY(launch_cgemm<double>(1, 0, np, np, ctx->npw, ctx->P64, ctx->npw, ctx->P64, ctx->npw,
                                epi<double>(EPI_STORE, Bm, np), ns, spl, st), "P^dagger P");
    CU_TRY(la_herm_sym(Bm, np, np, st), "B sym");
    // Q^-1 = L^-dagger L^-1
    CU_TRY(cast_r2z(ctx->Q64, Qz, (int64_t)nn, st), "Q cast");
    CU_TRY(la_cholesky(Qz, np, np, flag, st), "Q cholesky");
    CU_TRY(la_trinv_lower(Qz, np, np, Li, np, tmp, st), "Q trinv");
    // Mm = Bm + Li^dagger Li  (accumulated into Bm copy `tmp`)
    CU_TRY(cudaMemcpyAsync(tmp, Bm, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st), "copy B");
    CU_TRY(launch_cgemm<double>(1, 0, np, np, np, Li, np, Li, np, epi<double>(EPI_ACCUM, tmp, np), 1, nullptr, st),
           "Q inverse");
    CU_TRY(la_herm_sym(tmp, np, np, st), "M sym");
    CU_TRY(la_cholesky(tmp, np, np, flag, st), "M cholesky");
    CU_TRY(la_trinv_lower(tmp, np, np, Li, np, Qz, st), "M trinv");
    CU_TRY(launch_cgemm<double>(1, 0, np, np, np, Li, np, Li, np, epi<double>(EPI_STORE, ctx->K64, np), 1, nullptr,
                                st), "K");
    // E = D - K (B D)
    CU_TRY(cast_r2z(ctx->D64, Dz, (int64_t)nn, st), "D cast");
    CU_TRY(launch_cgemm<double>(0, 0, np, np, np, Bm, np, Dz, np, epi<double>(EPI_STORE, tmp, np), 1, nullptr, st),
           "B D");
    CU_TRY(cudaMemcpyAsync(ctx->E64, Dz, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st), "copy D");
    CU_TRY(launch_cgemm<double>(0, 0, np, np, np, ctx->K64, np, tmp, np, epi<double>(EPI_ACCUM, ctx->E64, np, -1.0),
                                1, nullptr, st), "E");
    CU_TRY(cast_z2c(ctx->K64, ctx->K32, (int64_t)nn, st), "K cast");
    CU_TRY(cast_z2c(ctx->E64, ctx->E32, (int64_t)nn, st), "E cast");
    // P^dagger P stays: the filter's projector-space recurrence uses it
    ctx->B64 = Bm;
    PW_TRY(upload(ctx, &ctx->B32, (const float2*)nullptr, nn));
    CU_TRY(cast_z2c(ctx->B64, ctx->B32, (int64_t)nn, st), "P^dagger P cast");
    PW_TRY(check_flag(ctx, flag, "Woodbury set-up (Q or Q^-1 + P^dagger P)"));
  }
  CU_TRY(cudaStreamSynchronize(st), "context set-up");
  return PW_OK;
}

void destroy_impl(pw_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->tcA1) cudaFree(ctx->tcA1);
  if (ctx->tcA2) cudaFree(ctx->tcA2);
  if (ctx->tc_err) cudaFree(ctx->tc_err);
  if (ctx->ozPH) cudaFree(ctx->ozPH);
  if (ctx->ozP) cudaFree(ctx->ozP);
  if (ctx->ozPH_exp) cudaFree(ctx->ozPH_exp);
  if (ctx->ozP_exp) cudaFree(ctx->ozP_exp);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (void* p : ctx->owned) cudaFree(p);
  for (auto& b : ctx->ws)
    if (b.p) cudaFree(b.p);
  delete ctx;
}

}  // namespace

// ---------------------------------------------------------------------------
// internal entry points used by the adjoint translation unit (api.cuh)
// ---------------------------------------------------------------------------
namespace pw {
namespace api {
int check(pw_ctx* ctx) { return check_ctx(ctx); }
int check_blk(pw_ctx* ctx, const void* p, int64_t ld, int nband) { return check_block(ctx, p, ld, nband); }
int apply64(pw_ctx* ctx, const double2* psi, int64_t ld, int nband, double2* hpsi, int64_t ldo) {
  return apply_impl<double>(ctx, psi, ld, nband, hpsi, nullptr, ldo);
}
template <typename T>
int recur(pw_ctx* ctx, const cplx<T>* cur, int64_t ldc, const cplx<T>* prev, int64_t ldp, cplx<T>* dst, int64_t ldd,
          int nband, double alpha, double beta, double shift, cplx<T>* C_out) {
  return recur_step<T>(ctx, cur, ldc, prev, ldp, dst, ldd, nband, alpha, beta, shift, C_out);
}
template int recur<double>(pw_ctx*, const double2*, int64_t, const double2*, int64_t, double2*, int64_t, int, double,
                           double, double, double2*);
template int recur<float>(pw_ctx*, const float2*, int64_t, const float2*, int64_t, float2*, int64_t, int, double,
                          double, double, float2*);
int rr(pw_ctx* ctx, double2* Y, int64_t ldy, int m, double* eig_h, double2* q_out, double2* x_out,
       double* eig_dev_out) {
  return rr_impl(ctx, Y, ldy, m, nullptr, eig_h, nullptr, q_out, x_out, eig_dev_out);
}
int bounds(pw_ctx* ctx, const double2* psi, int64_t ld, int nband, int steps, const double2* v0, double* rq_max,
           double* upper) {
  return bounds_impl(ctx, psi, ld, nband, steps, v0, nullptr, rq_max, upper);
}
int fft_band_batch(const pw_ctx* ctx, int nband, size_t elem) { return band_batch(ctx, nband, elem); }
int gemm_nsplit(int m, int n, int k) { return nsplit_for(m, n, k); }
}  // namespace api
}  // namespace pw

// ---------------------------------------------------------------------------
// k-point batches: every k-point's filter captured into one CUDA graph
// ---------------------------------------------------------------------------
struct pw_batch {
  std::vector<pw_ctx*> ctx;
  cudaStream_t stream = nullptr;  // the caller's stream
  cudaStream_t cap = nullptr;     // the batch's own stream (captured, replayed)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  double* dev_ce = nullptr;  // {c, e} per k-point
  std::vector<double> host_ce;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> key_psi;
  std::vector<int64_t> key_ld;
  std::vector<uint64_t> key_gen;
  int key_nband = -1, key_degree = -1, key_prec = -1;
  std::vector<void*> y32;  // complex64 copies for the mixed solve
  std::vector<size_t> y32_bytes;
  bool poisoned = false;
};

namespace {

constexpr int kBatchStreams = 4;

void batch_free_graph(pw_batch* bt) {
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  bt->exec = nullptr;
  bt->graph = nullptr;
}

int batch_run_one(pw_batch* bt, int k, void* psi, int64_t ld, int nband, int degree, int precision) {
  pw_ctx* ctx = bt->ctx[k];
  if (precision == PW_FP64)
    return filter_impl<double>(ctx, (double2*)psi, ld, nband, degree, 0.0, 1.0, bt->dev_ce + 2 * k);
  return filter_impl<float>(ctx, (float2*)psi, ld, nband, degree, 0.0, 1.0, bt->dev_ce + 2 * k);
}

int batch_filter_body(pw_batch* bt, void* const* psi, const int64_t* ld, int nband, int degree, int precision) {
  const int nk = (int)bt->ctx.size();
  cudaError_t e;
  bool same = bt->exec && bt->key_nband == nband && bt->key_degree == degree && bt->key_prec == precision;
  for (int k = 0; same && k < nk; ++k)
    same = bt->key_psi[k] == psi[k] && bt->key_ld[k] == ld[k] && bt->key_gen[k] == bt->ctx[k]->ws_gen;
  if (same) {
    e = cudaGraphLaunch(bt->exec, bt->cap);
    if (e != cudaSuccess) { bt->poisoned = true; return cuda_status(e, "batch graph launch"); }
    return PW_OK;
  }
  // first call for this shape: run eagerly (allocates every workspace), then capture the
  // same launches, fanned out over kBatchStreams streams, for the following calls
  batch_free_graph(bt);
  std::vector<cudaStream_t> saved(nk);
  for (int k = 0; k < nk; ++k) {
    if (bt->ctx[k]->prof_on) return set_error(PW_EINVAL, "disable profiling on batched contexts");
    saved[k] = bt->ctx[k]->stream;
    bt->ctx[k]->stream = bt->cap;
  }
  int st = PW_OK;
  for (int k = 0; k < nk && st == PW_OK; ++k) st = batch_run_one(bt, k, psi[k], ld[k], nband, degree, precision);
  if (st != PW_OK) {
    for (int k = 0; k < nk; ++k) bt->ctx[k]->stream = saved[k];
    return st;
  }
  e = cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const int ns = (int)bt->side.size();
    cudaEventRecord(bt->ev[0], bt->cap);
    for (int i = 0; i < ns; ++i) cudaStreamWaitEvent(bt->side[i], bt->ev[0], 0);
    for (int k = 0; k < nk && st == PW_OK; ++k) {
      bt->ctx[k]->stream = bt->side[k % ns];
      st = batch_run_one(bt, k, psi[k], ld[k], nband, degree, precision);
    }
    for (int i = 0; i < ns; ++i) {
      cudaEventRecord(bt->ev[1 + i], bt->side[i]);
      cudaStreamWaitEvent(bt->cap, bt->ev[1 + i], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(bt->cap, &g);
    if (st == PW_OK && e2 == cudaSuccess && g) {
      bt->graph = g;
      e = cudaGraphInstantiate(&bt->exec, g, 0);
      if (e != cudaSuccess) { batch_free_graph(bt); st = cuda_status(e, "batch graph instantiate"); }
    } else {
      if (g) cudaGraphDestroy(g);
      if (st == PW_OK) st = cuda_status(e2 == cudaSuccess ? cudaErrorStreamCaptureInvalidated : e2, "batch capture");
    }
  } else {
    st = cuda_status(e, "batch capture begin");
  }
  for (int k = 0; k < nk; ++k) bt->ctx[k]->stream = saved[k];
  if (st != PW_OK) return st;
  bt->key_psi.assign(psi, psi + nk);
  bt->key_ld.assign(ld, ld + nk);
  bt->key_gen.resize(nk);
  for (int k = 0; k < nk; ++k) bt->key_gen[k] = bt->ctx[k]->ws_gen;
  bt->key_nband = nband;
  bt->key_degree = degree;
  bt->key_prec = precision;
  return PW_OK;
}

// the caller's stream -> batch stream (interval upload, graph or first run) -> the caller's stream
int batch_filter_impl(pw_batch* bt, void* const* psi, const int64_t* ld, int nband, int degree, const double* a,
                      const double* b, int precision) {
  const int nk = (int)bt->ctx.size();
  for (int k = 0; k < nk; ++k) {
    if (!(b[k] > a[k])) return set_error(PW_EINVAL, "k-point %d: filter interval needs upper > lower", k);
    bt->host_ce[2 * k] = 0.5 * (b[k] + a[k]);
    bt->host_ce[2 * k + 1] = 0.5 * (b[k] - a[k]);
  }
  cudaError_t e = cudaEventRecord(bt->ev_in, bt->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->cap, bt->ev_in, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->dev_ce, bt->host_ce.data(), sizeof(double) * 2 * nk, cudaMemcpyHostToDevice, bt->cap);
  if (e != cudaSuccess) { bt->poisoned = true; return cuda_status(e, "batch interval upload"); }
  const int st = batch_filter_body(bt, psi, ld, nband, degree, precision);
  e = cudaEventRecord(bt->ev_out, bt->cap);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->stream, bt->ev_out, 0);
  if (e != cudaSuccess) { bt->poisoned = true; return cuda_status(e, "batch join"); }
  return st;
}

}  // namespace

// ===========================================================================
// exported C ABI
// ===========================================================================
extern "C" {

PW_API int pw_ctx_create(const pw_problem_desc* desc, void* stream, pw_ctx** out) {
  pw_ctx* ctx = nullptr;
  int s = create_impl(desc, stream, &ctx);
  if (s != PW_OK) {
    destroy_impl(ctx);
    if (out) *out = nullptr;
    return s;
  }
  *out = ctx;
  return PW_OK;
}

PW_API int pw_ctx_destroy(pw_ctx* ctx) {
  destroy_impl(ctx);
  return PW_OK;
}

PW_API int pw_ctx_set_stream(pw_ctx* ctx, void* stream) {
  PW_TRY(check_ctx(ctx));
  ctx->stream = (cudaStream_t)stream;
  return PW_OK;
}

PW_API int pw_ctx_info(const pw_ctx* ctx, int* npw, int* nproj) {
  if (!ctx) return set_error(PW_EINVAL, "NULL context");
  if (npw) *npw = ctx->npw;
  if (nproj) *nproj = ctx->nproj;
  return PW_OK;
}

PW_API int pw_ctx_gvectors(const pw_ctx* ctx, int32_t* miller, double* kinetic) {
  if (!ctx) return set_error(PW_EINVAL, "NULL context");
  if (miller) memcpy(miller, ctx->miller.data(), sizeof(int32_t) * ctx->miller.size());
  if (kinetic) memcpy(kinetic, ctx->kin_h.data(), sizeof(double) * ctx->kin_h.size());
  return PW_OK;
}

PW_API int pw_ctx_projectors(const pw_ctx* ctx_c, void* P_out) {
  pw_ctx* ctx = const_cast<pw_ctx*>(ctx_c);
  PW_TRY(check_ctx(ctx));
  if (!P_out) return set_error(PW_EINVAL, "NULL output");
  CU_TRY(cudaMemcpyAsync(P_out, ctx->P64, sizeof(double2) * (size_t)ctx->npw * ctx->nproj, cudaMemcpyDeviceToDevice,
                         ctx->stream), "projector copy");
  return PW_OK;
}

PW_API int pw_hamiltonian_apply(pw_ctx* ctx, const void* psi, int64_t ldpsi, int nband, void* hpsi, void* spsi,
                                int64_t ldout, int precision) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_block(ctx, psi, ldpsi, nband));
  PW_TRY(check_block(ctx, hpsi, ldout, nband));
  if (nband == 0) return PW_OK;
  if (psi == hpsi || (spsi && psi == spsi)) return set_error(PW_EINVAL, "psi aliases an output");
  if (precision == PW_FP64)
    return apply_impl<double>(ctx, (const double2*)psi, ldpsi, nband, (double2*)hpsi, (double2*)spsi, ldout);
  if (precision == PW_MIXED) {
    if (spsi && ctx->has_q) return set_error(PW_EUNSUPPORTED, "S psi in mixed precision");
    return apply_impl<float>(ctx, (const float2*)psi, ldpsi, nband, (float2*)hpsi, (float2*)spsi, ldout);
  }
  return set_error(PW_EINVAL, "unknown precision %d", precision);
}

PW_API int pw_spectrum_bounds(pw_ctx* ctx, const void* psi, int64_t ld, int nband, int lanczos_steps, const void* v0,
                              double* rq_min, double* rq_max, double* upper) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_block(ctx, psi, ld, nband));
  if (lanczos_steps < 0) return set_error(PW_EINVAL, "lanczos_steps < 0");
  return bounds_impl(ctx, (const double2*)psi, ld, nband, lanczos_steps, (const double2*)v0, rq_min, rq_max, upper);
}

PW_API int pw_chebyshev_filter(pw_ctx* ctx, void* psi, int64_t ldpsi, int nband, int degree, double a, double b,
                               int precision) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_block(ctx, psi, ldpsi, nband));
  if (degree < 0) return set_error(PW_EINVAL, "degree < 0");
  if (precision == PW_FP64) return filter_impl<double>(ctx, (double2*)psi, ldpsi, nband, degree, a, b);
  if (precision == PW_MIXED) return filter_impl<float>(ctx, (float2*)psi, ldpsi, nband, degree, a, b);
  return set_error(PW_EINVAL, "unknown precision %d", precision);
}

PW_API int pw_rayleigh_ritz(pw_ctx* ctx, void* psi, int64_t ldpsi, int nband, void* hpsi, double* eig,
                            double* resid) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_block(ctx, psi, ldpsi, nband));
  if (nband == 0) return PW_OK;
  if (nband > ctx->npw) return set_error(PW_EINVAL, "more bands than plane waves");
  return rr_impl(ctx, (double2*)psi, ldpsi, nband, (double2*)hpsi, eig, resid);
}

PW_API int pw_slice_filter(pw_ctx* ctx, void* psi, int64_t ldpsi, int nslice, int nper, int degree, double lo,
                           double hi, const double* cuts, int precision) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_slices(nslice, nper, degree, lo, hi, cuts));
  PW_TRY(check_block(ctx, psi, ldpsi, nslice * nper));
  if (precision == PW_FP64)
    return slice_filter_impl<double>(ctx, (double2*)psi, ldpsi, nslice, nper, degree, lo, hi, cuts);
  if (precision == PW_MIXED)
    return slice_filter_impl<float>(ctx, (float2*)psi, ldpsi, nslice, nper, degree, lo, hi, cuts);
  return set_error(PW_EINVAL, "unknown precision");
}

PW_API int pw_spectrum_slice(pw_ctx* ctx, void* psi_v, int64_t ldpsi, int nslice, int nper, int degree, double lo,
                             double hi, const double* cuts, int precision, double* eig, double* resid) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_slices(nslice, nper, degree, lo, hi, cuts));
  PW_TRY(check_block(ctx, psi_v, ldpsi, nslice * nper));
  if (!eig) return set_error(PW_EINVAL, "eig is NULL");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  double2* psi = (double2*)psi_v;
  const int npw = ctx->npw, nband = nslice * nper;
  if (precision == PW_FP64) {
    PW_TRY(slice_filter_impl<double>(ctx, psi, ldpsi, nslice, nper, degree, lo, hi, cuts));
  } else {
    WS(y32, float2, WS_Y32, (size_t)npw * nband);
    CU_TRY(la_to_c64(psi, ldpsi, y32, npw, npw, nband, ctx->stream), "to c64");
    PW_TRY(slice_filter_impl<float>(ctx, y32, npw, nslice, nper, degree, lo, hi, cuts));
    CU_TRY(la_to_c128(y32, npw, psi, ldpsi, npw, nband, ctx->stream), "to c128");
  }
  // independent small Rayleigh-Ritz steps, one per slice
  for (int s = 0; s < nslice; ++s)
    PW_TRY(rr_impl(ctx, psi + (size_t)s * nper * ldpsi, ldpsi, nper, nullptr, eig + (size_t)s * nper,
                   resid ? resid + (size_t)s * nper : nullptr));
  return PW_OK;
}

PW_API int pw_lobpcg_solve(pw_ctx* ctx, void* psi, int64_t ldpsi, int nband, int nblocks, int nline, double tol,
                           double* eig, double* resid, int* iters) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_block(ctx, psi, ldpsi, nband));
  if (nband == 0) return PW_OK;
  if (!eig) return set_error(PW_EINVAL, "eig is NULL");
  if (nblocks < 1 || nband % nblocks) return set_error(PW_EINVAL, "nband (%d) must be a multiple of nblocks (%d)", nband, nblocks);
  if (nline < 0) return set_error(PW_EINVAL, "nline must be non-negative");
  return lobpcg_impl(ctx, (double2*)psi, ldpsi, nband, nblocks, nline, tol, eig, resid, iters);
}

PW_API int pw_chebfi_solve(pw_ctx* ctx, void* psi_v, int64_t ldpsi, int nband, int degree, int cycles,
                           int lanczos_steps, const void* v0, int precision, double* eig, double* resid,
                           double* bounds) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_block(ctx, psi_v, ldpsi, nband));
  if (nband == 0) return PW_OK;
  if (!eig) return set_error(PW_EINVAL, "eig is NULL");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  double2* psi = (double2*)psi_v;
  double rqmin = 0, a = 0, upper = 0;
  if (precision == PW_MIXED) {
    // the cut a is a filter parameter, not a result: the numerators of the Rayleigh
    // quotients of the starting block come from the complex64 H-apply (the FP64 apply of a
    // block costs as much as a filter's worth of mixed steps), the denominators from the FP64
    // S-apply (projector GEMMs only); the Lanczos bound stays FP64
    PW_TRY(bounds_impl(ctx, psi, ldpsi, 0, lanczos_steps, (const double2*)v0, nullptr, nullptr, &upper));
    const int npw = ctx->npw;
    const cudaStream_t st = ctx->stream;
    WS(y32, float2, WS_Y1, (size_t)npw * nband);
    WS(h32, float2, WS_Y2, (size_t)npw * nband);
    WS(HY, double2, WS_HY, (size_t)npw * nband);
    WS(rq, double2, WS_RQ, (size_t)3 * nband + 8);
    CU_TRY(la_to_c64(psi, ldpsi, y32, npw, npw, nband, st), "to c64");
    PW_TRY(apply_impl<float>(ctx, y32, npw, nband, h32, nullptr, npw));
    CU_TRY(la_to_c128(h32, npw, HY, npw, npw, nband, st), "to c128");
    CU_TRY(la_coldot(psi, ldpsi, HY, npw, npw, nband, rq, st), "rq num");
    const double2* SY = psi;
    int64_t lds = ldpsi;
    if (ctx->has_q) {
      WS(SYb, double2, WS_SY, (size_t)npw * nband);
      PW_TRY(apply_s64(ctx, psi, ldpsi, nband, SYb, npw));
      SY = SYb;
      lds = npw;
    }
    CU_TRY(la_coldot(psi, ldpsi, SY, lds, npw, nband, rq + nband, st), "rq den");
    double* mm = (double*)(rq + 2 * nband);
    double* rqv = (double*)(rq + 2 * nband + 1);
    CU_TRY(la_rq_minmax(rq, rq + nband, nband, rqv, mm, st), "rq minmax");
    double h[2];
    CU_TRY(cudaMemcpyAsync(h, mm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "rq copy");
    CU_TRY(cudaStreamSynchronize(st), "rq sync");
    rqmin = h[0];
    a = h[1];
  } else {
    PW_TRY(bounds_impl(ctx, psi, ldpsi, nband, lanczos_steps, (const double2*)v0, &rqmin, &a, &upper));
  }
  if (bounds) { bounds[0] = upper; bounds[1] = a; }
  for (int c = 0; c < cycles; ++c) {
    if (precision == PW_FP64) {
      PW_TRY(filter_impl<double>(ctx, psi, ldpsi, nband, degree, a, upper));
    } else {
      WS(y32, float2, WS_Y32, (size_t)ctx->npw * nband);
      CU_TRY(la_to_c64(psi, ldpsi, y32, ctx->npw, ctx->npw, nband, ctx->stream), "to c64");
      PW_TRY(filter_impl<float>(ctx, y32, ctx->npw, nband, degree, a, upper));
      CU_TRY(la_to_c128(y32, ctx->npw, psi, ldpsi, ctx->npw, nband, ctx->stream), "to c128");
    }
    PW_TRY(rr_impl(ctx, psi, ldpsi, nband, nullptr, eig, resid));
    a = eig[nband - 1];
  }
  return PW_OK;
}

PW_API int pw_density_grad(pw_ctx* ctx, const void* a, const void* b, int64_t ld, int nband, const double* w,
                           double* out, int accumulate) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_block(ctx, a, ld, nband));
  if (!out) return set_error(PW_EINVAL, "NULL output grid");
  if (nband > 0 && !w) return set_error(PW_EINVAL, "NULL weights");
  const cudaStream_t st = ctx->stream;
  const size_t ntot = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  WS(den, double, WS_DEN, ntot + (size_t)nband + 8);
  double* wd = den + ntot;
  CU_TRY(cudaMemsetAsync(den, 0, sizeof(double) * ntot, st), "density reset");
  if (nband > 0) {
    CU_TRY(cudaMemcpyAsync(wd, w, sizeof(double) * nband, cudaMemcpyHostToDevice, st), "weights");
    const int bb = std::max(1, band_batch(ctx, nband) / 2);
    const int64_t hb_bs = (int64_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2];
    WS(hb, double2, WS_HB, hb_bs * bb * 2);
    CU_TRY(launch_density<double>(ctx->plan, ctx->tw64, ctx->sp, (const double2*)a, (const double2*)b, ld, nband, wd,
                                  den, hb, bb, st), "density");
  }
  CU_TRY(setup_unperm(den, ctx->n, ctx->rho_perm, out, accumulate, st), "density unpermute");
  CU_TRY(cudaStreamSynchronize(st), "density sync");
  return PW_OK;
}

PW_API int pw_autotune(pw_ctx* ctx, int nband, int precision, double* best_ms) {
  PW_TRY(check_ctx(ctx));
  if (nband <= 0) return set_error(PW_EINVAL, "nband must be positive");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  const int slot = precision == PW_MIXED ? 0 : 1;
  const size_t elem = precision == PW_MIXED ? 8 : 16;
  const cudaStream_t st = ctx->stream;
  const size_t per = (size_t)ctx->sp.nplane * ctx->n[1] * ctx->n[2] * elem;
  // candidate batch footprints (bytes of half-box planes per launch)
  const size_t cand[7] = {(size_t)16 << 20, (size_t)48 << 20, (size_t)128 << 20, (size_t)256 << 20,
                          (size_t)512 << 20, (size_t)1024 << 20, (size_t)2048 << 20};
  WS(xin, unsigned char, WS_Y1, elem * (size_t)ctx->npw * nband);
  WS(xout, unsigned char, WS_Y2, elem * (size_t)ctx->npw * nband);
  CU_TRY(cudaMemsetAsync(xin, 0, elem * (size_t)ctx->npw * nband, st), "autotune input");
  size_t max_hb = 0;
  for (size_t c : cand) max_hb = std::max(max_hb, std::min<size_t>(std::max<size_t>(c / std::max<size_t>(per, 1), 1), nband) * per);
  WS(hb, unsigned char, WS_HB, max_hb);
  // events and the profiling switch are restored on every exit path
  struct Guard {
    pw_ctx* c;
    bool prof;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Guard() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      c->prof_on = prof;
    }
  } g{ctx, ctx->prof_on};
  ctx->prof_on = false;  // the launches get the context for its kernel-form field only
  CU_TRY(cudaEventCreate(&g.e0), "event");
  CU_TRY(cudaEventCreate(&g.e1), "event");
  double best = 1e30;
  size_t best_c = ctx->fft_batch_bytes[slot];
  int best_v = ctx->fft_variant[slot];
  std::vector<std::pair<float, int>> form_times;  // (time, variant) of the form sweep
  auto consider = [&](size_t c, int v, int reps = 5) -> int {
    const int bb = (int)std::max<size_t>(1, std::min<size_t>(c / std::max<size_t>(per, 1), nband));
    if (c != cand[0] && bb * per > c && bb == 1) return PW_OK;
    ctx->fft_variant[slot] = v;
    float tot = 1e30f;  // the fastest of the timed runs (after a warm-up) resists noise best
    for (int rep = 0; rep < reps; ++rep) {
      CU_TRY(cudaEventRecord(g.e0, st), "autotune event");
      cudaError_t e;
      if (precision == PW_MIXED)
        e = launch_local_apply<float>(ctx->plan, ctx->tw32, ctx->sp, ctx->vperm32, ctx->kin32, (const float2*)xin,
                                      ctx->npw, nband, (float2*)xout, ctx->npw, (float2*)hb, bb, st, ctx);
      else
        e = launch_local_apply<double>(ctx->plan, ctx->tw64, ctx->sp, ctx->vperm64, ctx->kin64, (const double2*)xin,
                                       ctx->npw, nband, (double2*)xout, ctx->npw, (double2*)hb, bb, st, ctx);
      CU_TRY(e, "autotune");
      CU_TRY(cudaEventRecord(g.e1, st), "autotune event");
      CU_TRY(cudaEventSynchronize(g.e1), "autotune sync");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, g.e0, g.e1);
      if (rep > 0) tot = std::min(tot, ms);  // first repetition warms up
    }
    if (tot < best) { best = tot; best_c = c; best_v = v; }
    form_times.push_back({tot, v});
    return PW_OK;
  };
  // batch size with the current kernel forms, every kernel form at that size (complex64:
  // x-line form + kFormStride * plane form), the batch size again with the forms kept
  for (size_t c : cand) PW_TRY(consider(c, best_v));
  const size_t c1 = best_c;
  if (precision == PW_MIXED) {
    form_times.clear();
    for (int pf = 0; pf < kPlaneForms; ++pf)
      for (int xf = 0; xf < kXlineForms; ++xf) PW_TRY(consider(c1, xf + kFormStride * pf));
    // the plane forms compared again inside two steps of the filter itself, round robin (its
    // projector GEMMs between the passes change what the passes find in L2; the persistent
    // plane forms gain there and not in bare applies), each with the x-line form of the best
    // bare time, and the runner-up x-line form (by its best bare time over the plane forms)
    // with the best plane form, since bare applies rank close x-line forms within their
    // noise; the fastest of all their runs kept
    const int xbest = best_v % kFormStride;
    std::vector<std::pair<float, int>> top;
    for (int pf = 0; pf < kPlaneForms; ++pf) top.push_back({0.f, xbest + kFormStride * pf});
    {
      float t2 = 1e30f;
      int x2 = -1;
      for (const auto& f : form_times) {
        const int xf = f.second % kFormStride;
        if (xf != xbest && f.first < t2) { t2 = f.first; x2 = xf; }
      }
      if (x2 >= 0) top.push_back({0.f, x2 + kFormStride * (best_v / kFormStride)});
    }
    // at the batch size that suits the forms found (the first batch sweep ran with the
    // initial forms, which may prefer other sizes)
    {
      const int vb = best_v;
      for (size_t c : cand) PW_TRY(consider(c, vb));
    }
    const size_t c2 = best_c;
    WS(yf, float2, WS_Y32, (size_t)ctx->npw * nband);
    CU_TRY(cudaMemsetAsync(yf, 0, sizeof(float2) * (size_t)ctx->npw * nband, st), "autotune block");
    ctx->fft_batch_bytes[slot] = c2;
    float fbest = 1e30f;
    int fv = best_v;
    for (int round = 0; round < 3; ++round) {
      for (const auto& f : top) {
        ctx->fft_variant[slot] = f.second;
        if (round == 0) PW_TRY(filter_impl<float>(ctx, yf, ctx->npw, nband, 2, 0.0, 1.0));  // warm-up
        CU_TRY(cudaEventRecord(g.e0, st), "autotune event");
        PW_TRY(filter_impl<float>(ctx, yf, ctx->npw, nband, 2, 0.0, 1.0));
        CU_TRY(cudaEventRecord(g.e1, st), "autotune event");
        CU_TRY(cudaEventSynchronize(g.e1), "autotune sync");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g.e0, g.e1);
        if (ms < fbest) { fbest = ms; fv = f.second; }
      }
    }
    best_v = fv;
    best_c = c2;
    ctx->fft_variant[slot] = fv;
  } else {
    // complex128: line-group planes or sphere rows + column slices (x-line form fixed)
    PW_TRY(consider(c1, 0));
    PW_TRY(consider(c1, 3 * kFormStride));
  }
  const int v1 = best_v;
  for (size_t c : cand) PW_TRY(consider(c, v1));
  ctx->fft_batch_bytes[slot] = best_c;
  ctx->fft_variant[slot] = best_v;
  if (best_ms) *best_ms = best;
  // mixed projection GEMM: time the K splits around the whole-waves rule for the column
  // count the filter uses (nband: P^dagger Y_k without Q, P^dagger W with Q)
  if (precision == PW_MIXED && ctx->nproj > 0) {
    PW_TRY(ensure_tc(ctx));
    const int ncols[2] = {nband, 0};
    for (int cols : ncols) {
      if (cols <= 0) continue;
      __nv_bfloat16* ysp;
      PW_TRY(tc_split(ctx, (const float2*)xin, ctx->npw, ctx->npw, std::min(cols, nband), ctx->kp1, WS_YSPLIT, &ysp));
      if (cols > nband) {  // the second half of the pieces: zeros are as good as data for timing
        WS(ysb, __nv_bfloat16, WS_YSPLIT, (size_t)ctx->tc_pieces * cols * ctx->kp1);
        CU_TRY(cudaMemsetAsync(ysb, 0, sizeof(__nv_bfloat16) * (size_t)ctx->tc_pieces * cols * ctx->kp1, st),
               "autotune pieces");
        ysp = ysb;
      }
      WS(cbuf, float2, WS_C, (size_t)ctx->nproj * cols);
      const int K = 2 * ctx->npw, rule = tc_proj_split(ctx, cols, 1);
      std::vector<int> cands;
      for (int c : {rule, 1, 2, rule / 2, rule - 1, rule + 1, 2 * rule, 3 * rule / 2}) {
        const int cc = tc::split_count(K, std::max(1, c));
        if (std::find(cands.begin(), cands.end(), cc) == cands.end() && cc <= 64) cands.push_back(cc);
      }
      float tbest = 1e30f;
      int sbest = rule;
      for (int cc : cands) {
        float tot = 1e30f;
        for (int rep = 0; rep < 5; ++rep) {
          CU_TRY(cudaEventRecord(g.e0, st), "autotune event");
          PW_TRY(tc_project(ctx, ysp, cols, cbuf, cc));
          CU_TRY(cudaEventRecord(g.e1, st), "autotune event");
          CU_TRY(cudaEventSynchronize(g.e1), "autotune sync");
          float ms = 0.f;
          cudaEventElapsedTime(&ms, g.e0, g.e1);
          if (rep > 0) tot = std::min(tot, ms);
        }
        if (tot < tbest) { tbest = tot; sbest = cc; }
      }
      auto& v = ctx->tc_proj_splits;
      v.erase(std::remove_if(v.begin(), v.end(), [&](const std::pair<int, int>& e) { return e.first == cols; }),
              v.end());
      v.push_back({cols, sbest});
    }
    PW_TRY(check_tc_flag(ctx));
  }
  return PW_OK;
}

PW_API int pw_fft_config(pw_ctx* ctx, int precision, int64_t set_batch_bytes, int set_variant, int64_t* batch_bytes,
                         int* variant) {
  PW_TRY(check_ctx(ctx));
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  const int slot = precision == PW_MIXED ? 0 : 1;
  // complex128 has plane forms 0 and 3 only
  if (set_variant >= kFormStride * kPlaneForms || (set_variant >= 0 && set_variant % kFormStride >= kXlineForms) ||
      (slot == 1 && set_variant > 0 && set_variant != 3 * kFormStride))
    return set_error(PW_EINVAL, "unknown FFT kernel variant %d", set_variant);
  if (batch_bytes) *batch_bytes = (int64_t)ctx->fft_batch_bytes[slot];
  if (variant) *variant = ctx->fft_variant[slot];
  if (set_batch_bytes >= 0) ctx->fft_batch_bytes[slot] = (size_t)set_batch_bytes;
  if (set_variant >= 0) ctx->fft_variant[slot] = set_variant;
  return PW_OK;
}

PW_API int pw_tc_config(pw_ctx* ctx, int set_pieces, int* pieces) {
  PW_TRY(check_ctx(ctx));
  if (pieces) *pieces = ctx->tc_pieces;
  if (set_pieces >= 0) {
    if (set_pieces != 2 && set_pieces != 3) return set_error(PW_EINVAL, "bf16 pieces must be 2 or 3");
    ctx->tc_pieces = set_pieces;  // the operands are rebuilt on the next mixed call
  }
  return PW_OK;
}

PW_API int pw_ctx_sync(pw_ctx* ctx) {
  PW_TRY(check_ctx(ctx));
  PW_TRY(check_tc_flag(ctx));
  CU_TRY(cudaStreamSynchronize(ctx->stream), "context sync");
  return PW_OK;
}

PW_API int pw_ctx_test_wait_expiry(pw_ctx* ctx) {
  PW_TRY(check_ctx(ctx));
  ctx->test_wait_expiry = 1;
  return PW_OK;
}

PW_API int pw_fp64_config(pw_ctx* ctx, int set_mode, int* mode) {
  PW_TRY(check_ctx(ctx));
  if (set_mode > 1) return set_error(PW_EINVAL, "FP64 GEMM mode must be 0 (DFMA) or 1 (tensor-core digits)");
  if (mode) *mode = ctx->fp64_tc;
  if (set_mode >= 0) ctx->fp64_tc = set_mode;
  return PW_OK;
}

PW_API int pw_profile_enable(pw_ctx* ctx, int on) {
  PW_TRY(check_ctx(ctx));
  ctx->prof_on = (on != 0);
  return PW_OK;
}

PW_API int pw_profile_read(pw_ctx* ctx, double* ms, int64_t* launches) {
  PW_TRY(check_ctx(ctx));
  CU_TRY(cudaStreamSynchronize(ctx->stream), "profile sync");
  for (auto& r : ctx->prof_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ctx->prof_ms[r.cls] += t;
      ctx->prof_n[r.cls] += 1;
    }
  }
  ctx->prof_recs.clear();
  ctx->ev_used = 0;
  for (int i = 0; i < PW_PROF_NCLASS; ++i) {
    if (ms) ms[i] = ctx->prof_ms[i];
    if (launches) launches[i] = ctx->prof_n[i];
    ctx->prof_ms[i] = 0;
    ctx->prof_n[i] = 0;
    ctx->prof_open[i] = nullptr;
  }
  return PW_OK;
}

PW_API uint64_t pw_kernel_launches(void) { return g_launches.load(); }

PW_API int pw_batch_create(pw_ctx* const* ctxs, int nk, void* stream, pw_batch** out) {
  if (!ctxs || !out || nk <= 0) return set_error(PW_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int k = 0; k < nk; ++k) PW_TRY(check_ctx(ctxs[k]));
  pw_batch* bt = new (std::nothrow) pw_batch();
  if (!bt) return set_error(PW_ENOMEM, "host allocation");
  bt->ctx.assign(ctxs, ctxs + nk);
  bt->stream = (cudaStream_t)stream;
  bt->host_ce.assign(2 * nk, 0.0);
  cudaError_t e = cudaMalloc(&bt->dev_ce, sizeof(double) * 2 * nk);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->ev_out, cudaEventDisableTiming);
  const int ns = std::min(kBatchStreams, nk);
  for (int i = 0; i < ns && e == cudaSuccess; ++i) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) bt->side.push_back(s);
  }
  for (int i = 0; i < ns + 1 && e == cudaSuccess; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) bt->ev.push_back(ev);
  }
  if (e != cudaSuccess) {
    pw_batch_destroy(bt);
    return cuda_status(e, "batch creation");
  }
  *out = bt;
  return PW_OK;
}

PW_API int pw_batch_destroy(pw_batch* bt) {
  if (!bt) return PW_OK;
  if (bt->cap) cudaStreamSynchronize(bt->cap);
  batch_free_graph(bt);
  if (bt->cap) cudaStreamDestroy(bt->cap);
  if (bt->ev_in) cudaEventDestroy(bt->ev_in);
  if (bt->ev_out) cudaEventDestroy(bt->ev_out);
  for (cudaStream_t s : bt->side) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  for (cudaEvent_t ev : bt->ev) cudaEventDestroy(ev);
  for (void* p : bt->y32) if (p) cudaFree(p);
  if (bt->dev_ce) cudaFree(bt->dev_ce);
  delete bt;
  return PW_OK;
}

PW_API int pw_batch_filter(pw_batch* bt, void* const* psi, const int64_t* ld, int nband, int degree, const double* a,
                           const double* b, int precision) {
  if (!bt || !psi || !ld || !a || !b) return set_error(PW_EINVAL, "NULL argument");
  if (bt->poisoned) return set_error(PW_ECUDA, "batch poisoned by an earlier CUDA error");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  if (degree < 0 || nband < 0) return set_error(PW_EINVAL, "negative degree or nband");
  for (size_t k = 0; k < bt->ctx.size(); ++k) {
    PW_TRY(check_ctx(bt->ctx[k]));
    PW_TRY(check_block(bt->ctx[k], psi[k], ld[k], nband));
  }
  if (degree == 0 || nband == 0) return PW_OK;
  return batch_filter_impl(bt, psi, ld, nband, degree, a, b, precision);
}

PW_API int pw_batch_chebfi_solve(pw_batch* bt, void* const* psi, const int64_t* ld, int nband, int degree, int cycles,
                                 int lanczos_steps, void* const* v0, int precision, double* eig, double* resid) {
  if (!bt || !psi || !ld || !eig) return set_error(PW_EINVAL, "NULL argument");
  if (precision != PW_FP64 && precision != PW_MIXED) return set_error(PW_EINVAL, "unknown precision");
  const int nk = (int)bt->ctx.size();
  for (int k = 0; k < nk; ++k) {
    PW_TRY(check_ctx(bt->ctx[k]));
    PW_TRY(check_block(bt->ctx[k], psi[k], ld[k], nband));
  }
  if (nband == 0) return PW_OK;
  std::vector<double> a(nk), b(nk);
  for (int k = 0; k < nk; ++k) {
    pw_ctx* ctx = bt->ctx[k];
    const cudaStream_t saved = ctx->stream;
    ctx->stream = bt->stream;
    double lo = 0;
    const int s = bounds_impl(ctx, (const double2*)psi[k], ld[k], nband, lanczos_steps,
                              v0 ? (const double2*)v0[k] : nullptr, &lo, &a[k], &b[k]);
    ctx->stream = saved;
    if (s != PW_OK) return s;
  }
  std::vector<void*> fpsi(nk);
  std::vector<int64_t> fld(nk);
  if (precision == PW_MIXED) {
    bt->y32.resize(nk, nullptr);
    bt->y32_bytes.resize(nk, 0);
    for (int k = 0; k < nk; ++k) {
      const size_t need = sizeof(float2) * (size_t)bt->ctx[k]->npw * nband;
      if (bt->y32_bytes[k] < need) {
        if (bt->y32[k]) cudaFree(bt->y32[k]);
        cudaError_t e = cudaMalloc(&bt->y32[k], need);
        if (e != cudaSuccess) { bt->y32[k] = nullptr; bt->y32_bytes[k] = 0; return cuda_status(e, "batch c64 buffer"); }
        bt->y32_bytes[k] = need;
      }
      fpsi[k] = bt->y32[k];
      fld[k] = bt->ctx[k]->npw;
    }
  } else {
    for (int k = 0; k < nk; ++k) { fpsi[k] = psi[k]; fld[k] = ld[k]; }
  }
  for (int c = 0; c < cycles; ++c) {
    if (precision == PW_MIXED)
      for (int k = 0; k < nk; ++k) {
        cudaError_t e = la_to_c64((const double2*)psi[k], ld[k], (float2*)fpsi[k], fld[k], bt->ctx[k]->npw, nband,
                                  bt->stream);
        if (e != cudaSuccess) { bt->poisoned = true; return cuda_status(e, "to c64"); }
      }
    PW_TRY(batch_filter_impl(bt, fpsi.data(), fld.data(), nband, degree, a.data(), b.data(), precision));
    if (precision == PW_MIXED)
      for (int k = 0; k < nk; ++k) {
        cudaError_t e = la_to_c128((const float2*)fpsi[k], fld[k], (double2*)psi[k], ld[k], bt->ctx[k]->npw, nband,
                                   bt->stream);
        if (e != cudaSuccess) { bt->poisoned = true; return cuda_status(e, "to c128"); }
      }
    for (int k = 0; k < nk; ++k) {
      pw_ctx* ctx = bt->ctx[k];
      const cudaStream_t saved = ctx->stream;
      ctx->stream = bt->stream;
      const int s = rr_impl(ctx, (double2*)psi[k], ld[k], nband, nullptr, eig + (size_t)k * nband,
                            resid ? resid + (size_t)k * nband : nullptr);
      ctx->stream = saved;
      if (s != PW_OK) return s;
      a[k] = eig[(size_t)k * nband + nband - 1];
    }
  }
  return PW_OK;
}

PW_API const char* pw_strerror(int status) {
  switch (status) {
    case PW_OK: return "ok";
    case PW_EINVAL: return "invalid argument";
    case PW_ENOMEM: return "out of device memory";
    case PW_ECUDA: return "CUDA error";
    case PW_ENOTSPD: return "matrix not positive definite";
    case PW_ETIMEDOUT: return "device wait timed out";
    case PW_ENOTCONV: return "eigensolver did not converge";
    case PW_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

PW_API const char* pw_last_error(void) { return g_err; }

}  // extern "C"
