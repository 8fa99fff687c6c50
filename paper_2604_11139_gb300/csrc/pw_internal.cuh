// Internal declarations shared by the CUDA translation units of libpwcheb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pw.h"

struct pw_ctx;

namespace pw {

// ---------------------------------------------------------------------------
// complex helpers (interleaved re/im, double2 / float2)
// ---------------------------------------------------------------------------
template <typename T> struct CT;
template <> struct CT<double> { using type = double2; };
template <> struct CT<float> { using type = float2; };
template <typename T> using cplx = typename CT<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C{}.x) re, decltype(C{}.x) im) {
  C c; c.x = re; c.y = im; return c;
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by s*i (s = +1 or -1)
template <int S> __host__ __device__ __forceinline__ double2 cmuli(double2 a) {
  return make_double2(-S * a.y, S * a.x);
}
template <int S> __host__ __device__ __forceinline__ float2 cmuli(float2 a) {
  return make_float2(-S * a.y, S * a.x);
}
template <typename C> __host__ __device__ __forceinline__ C czero() { C c; c.x = 0; c.y = 0; return c; }

// ---------------------------------------------------------------------------
// FFT plan: one mixed-radix in-place plan per box dimension.  Inverse
// transforms run decimation-in-frequency (natural -> digit-reversed order),
// forward transforms decimation-in-time with the stages reversed
// (digit-reversed -> natural), so no permutation pass is ever needed; the
// potential grid is stored permuted instead.
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 8;
// FFT pass-kernel variant = x-line form (0-10) + kFormStride * plane form (0-6)
constexpr int kFormStride = 16;
constexpr int kXlineForms = 11, kPlaneForms = 7;
struct FftDim {
  int n, nst;
  int radix[kMaxStages];
  int L[kMaxStages];      // block length at each stage (n, n/r1, ...)
  int tw_off[kMaxStages]; // offset of the stage's twiddles in the table
  int tw_base, tw_count;  // this dimension's contiguous range of the table
};
struct FftPlan {
  int n[3];
  FftDim d[3];
};

// Radix plan of one FFT length, shared by host and device code.  Stages use the
// in-register radices {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2}; the plan has the fewest
// stages, then the smallest largest radix, then the largest leading radices.
struct CPlan {
  int nst;
  int radix[kMaxStages];
  int L[kMaxStages];
};
__host__ __device__ constexpr int radix_at(int i) {
  return i == 0 ? 16 : i == 1 ? 15 : i == 2 ? 12 : i == 3 ? 10 : i == 4 ? 9 : i == 5 ? 8 : i == 6 ? 6 : i == 7 ? 5
       : i == 8 ? 4 : i == 9 ? 3 : 2;
}
__host__ __device__ constexpr bool is_radix(int f) {
  for (int i = 0; i < 11; ++i)
    if (radix_at(i) == f) return true;
  return false;
}
__host__ __device__ constexpr CPlan make_cplan(int n) {
  CPlan p{};
  p.nst = 0;
  int f[kMaxStages] = {0, 0, 0, 0, 0, 0, 0, 0};
  int nf = 0;
  if (n > 1 && is_radix(n)) {
    f[0] = n;
    nf = 1;
  }
  if (nf == 0 && n > 1) {
    int bmax = 1 << 30;
    for (int i = 0; i < 11; ++i) {
      const int a = radix_at(i);
      if (n % a || !is_radix(n / a)) continue;
      const int b = n / a, mx = a > b ? a : b;
      if (mx < bmax || (mx == bmax && a > f[0])) { bmax = mx; f[0] = a; f[1] = b; nf = 2; }
    }
  }
  if (nf == 0 && n > 1) {
    int bmax = 1 << 30;
    for (int i = 0; i < 11; ++i)
      for (int j = 0; j < 11; ++j) {
        const int a = radix_at(i), b = radix_at(j);
        if (n % (a * b) || !is_radix(n / (a * b))) continue;
        const int c = n / (a * b);
        int mx = a > b ? a : b;
        mx = mx > c ? mx : c;
        if (mx < bmax || (mx == bmax && (a > f[0] || (a == f[0] && b > f[1])))) {
          bmax = mx; f[0] = a; f[1] = b; f[2] = c; nf = 3;
        }
      }
  }
  if (nf == 0 && n > 1) {  // longer lengths: greedy over the radix set
    int m = n;
    for (int i = 0; i < 11 && m > 1; ++i)
      while (m > 1 && m % radix_at(i) == 0 && nf < kMaxStages) { f[nf++] = radix_at(i); m /= radix_at(i); }
    if (m != 1) nf = -1;
  }
  p.nst = nf;
  int L = n;
  for (int s = 0; s < nf; ++s) { p.radix[s] = f[s]; p.L[s] = L; L /= f[s]; }
  return p;
}

// plane-wave sphere decomposition: planes (fixed h) -> rows (fixed h,k) -> runs of l
struct SphereDev {
  int npw, nplane, nrow, max_rows;
  int max_plane_g;        // largest coefficient count of one x-plane (its contiguous block)
  const int* plane_h;     // [nplane] Miller h
  const int* plane_row0;  // [nplane+1]
  const int* row_k;       // [nrow]
  const int* row_l0;      // [nrow] first l of the run
  const int* row_cnt;     // [nrow]
  const int* row_g0;      // [nrow] sphere index of the run's first element
};

// epilogue applied by the local-potential exit pass and by the GEMMs
enum EpiMode {
  EPI_STORE = 0,   // out = alpha * v
  EPI_ACCUM = 1,   // out = out + alpha * v
  EPI_CHEB = 2,    // out = alpha * (out + v - shift * yk) - beta * ykm1   (out holds W)
  EPI_KIN = 3      // out = kin * y + v  (local pass only)
};

template <typename T> struct Epi {
  int mode;
  cplx<T>* out;
  int64_t ldo;
  T alpha, beta, shift;
  const cplx<T>* yk;
  const cplx<T>* ykm1;
  int64_t ldy, ldy2;
  // optional device {c, e}: when set, shift = c and alpha = (first ? 1 : 2) / e are read on
  // the device, so a captured graph stays valid when the filter interval changes
  const double* dev_ce;
  int first;
};

// ---------------------------------------------------------------------------
// launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_local_apply(const FftPlan& plan, const cplx<T>* tw, const SphereDev& sp,
                               const T* vperm, const T* kin, const cplx<T>* psi, int64_t ldpsi,
                               int nband, cplx<T>* out, int64_t ldout, cplx<T>* hb, int band_batch,
                               cudaStream_t st, ::pw_ctx* prof);

// Recurrence step fused into FFT pass 3 (complex64, S = I):
//   y_{k+1} = alpha (kin y_k + (V y_k) + pz - shift y_k) - beta y_{k-1}
// pz = P D P^dagger y_k from the back-projection GEMM (ld ldpz); ykm1 may be NULL; with
// dev_ce, shift = c and alpha = (first ? 1 : 2) / e are read from the device.  split (may be
// NULL) receives the bf16 pieces of y_{k+1}: piece p of band b, real row r (2g: Re, 2g+1: Im)
// at split[p * split_piece_stride + b * split_ld + r].
struct Pass3Rec {
  const float2* pz;
  int64_t ldpz;
  const float2* ykm1;
  int64_t ldykm1;
  float alpha, beta, shift;
  const double* dev_ce;
  int first;
  void* split;  // __nv_bfloat16*
  int64_t split_ld, split_piece_stride;
  int pieces;
};
// H-apply local part with the fused recurrence of Pass3Rec (out = y_{k+1}); requires the
// warp-group plane kernels for this box (plane form 2 of the context's complex64 variant),
// else returns cudaErrorNotSupported before launching anything.
cudaError_t launch_local_apply_rec(const FftPlan& plan, const float2* tw, const SphereDev& sp, const float* vperm,
                                   const float* kin, const float2* psi, int64_t ldpsi, int nband, float2* out,
                                   int64_t ldout, float2* hb, int band_batch, cudaStream_t st, ::pw_ctx* prof,
                                   const Pass3Rec& rec);
bool local_apply_rec_supported(const FftPlan& plan, const ::pw_ctx* prof);

// fills the constant twiddles of the composite in-register radices on the current device
cudaError_t fft_set_constants();

template <typename T>
cudaError_t launch_density(const FftPlan& plan, const cplx<T>* tw, const SphereDev& sp,
                           const cplx<T>* a, const cplx<T>* b, int64_t ld, int nband, const T* w_dev,
                           double* out_perm, cplx<T>* hb, int band_batch, cudaStream_t st);

// Structure a GEMM may skip work for:
//  GEMM_LOWER_OUT: M == N and only the 64 x 64 output tiles on or below the diagonal are computed
//    and stored (a Hermitian Gram matrix; the tiles above the diagonal are left as they were);
//  GEMM_B_UPPER: op(B)[k][n] == 0 for k > n (B = L^dagger with L lower triangular), so the K range
//    of an output tile stops at its last column (N <= K).
enum { GEMM_FULL = 0, GEMM_LOWER_OUT = 1, GEMM_B_UPPER = 2 };

// op(A) is M x K, op(B) is K x N; ta/tb: 0 = as stored (column-major), 1 = conjugate transpose.
// nsplit > 1 splits K and reduces through `ws` (nsplit*M*N complex) before the epilogue.
template <typename T>
cudaError_t launch_cgemm(int ta, int tb, int M, int N, int K, const cplx<T>* A, int64_t lda,
                         const cplx<T>* B, int64_t ldb, const Epi<T>& epi, int nsplit, cplx<T>* ws,
                         cudaStream_t st, int tri = GEMM_FULL);

// real block-diagonal (or dense) D times complex C: Z = D C (nproj x nband)
template <typename T>
cudaError_t launch_dblock(int nproj, int nband, const T* D, const int* blk0, const int* blklen,
                          const cplx<T>* Cm, int64_t ldc, cplx<T>* Z, int64_t ldz, cudaStream_t st);

// workspace slots of a context (pw_ctx::ws)
enum WsSlot {
  WS_HB = 0, WS_C, WS_Z, WS_SPLIT, WS_Y1, WS_Y2, WS_CW,      // H-apply and filter
  WS_YSPLIT, WS_WSPLIT, WS_ZSPLIT, WS_TCPART, WS_TCERR,      // tensor-core mixed path
  WS_HY, WS_SY, WS_ROT, WS_Y32,                              // Rayleigh-Ritz / solve
  WS_GRAM, WS_GRAM2, WS_LINV, WS_TMP, WS_U, WS_JAC, WS_EIG,  // subspace matrices
  WS_LZ, WS_RQ, WS_DEN, WS_SCAL, WS_VPOT, WS_PZ,
  WS_OZA, WS_OZB, WS_OZPART, WS_OZAMAX, WS_OZEXP, WS_SCF,
  WS_LOBZ, WS_LOBT, WS_LOBB, WS_LOBR, WS_LOBD, WS_SLICEC, WS_SLICEA, WS_EIGMIX, WS_NUM
};
}  // namespace pw

// the context (opaque to C callers)
struct pw_ctx {
  cudaStream_t stream = nullptr;
  int n[3] = {0, 0, 0};
  int npw = 0, nproj = 0, natom = 0, nchan = 0;
  bool has_q = false;
  double lattice[9], kpt[3], ecut = 0;
  std::vector<int> miller;     // 3*npw
  std::vector<double> kin_h;   // npw
  pw::FftPlan plan;
  pw::SphereDev sp;
  // device memory owned by the context
  std::vector<void*> owned;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  double* kin64 = nullptr;
  float* kin32 = nullptr;
  double* vperm64 = nullptr;
  float* vperm32 = nullptr;
  int* rho_perm[3] = {nullptr, nullptr, nullptr};  // digit-reversal maps per dimension
  // x-line forms 5 and 6 run the two-stage x plan with its radices in the other order: the
  // x digit reversal of that order and V_loc / n1n2n3 permuted with it (complex64 path);
  // NULL when the x plan has no such alternative
  int* rho_x_sw = nullptr;
  float* vperm32_sw = nullptr;
  double2* P64 = nullptr;   // npw x nproj
  float2* P32 = nullptr;
  double* D64 = nullptr;    // nproj x nproj column-major
  float* D32 = nullptr;
  int* blk0 = nullptr;      // per projector: first index of its D block
  int* blklen = nullptr;
  std::vector<int> blk0_h, blklen_h;  // host copies of the D block structure
  uint64_t param_gen = 0;   // bumped whenever V_loc or D is replaced
  double* Q64 = nullptr;
  int* qblk0 = nullptr;     // per projector: first index of its Q block
  int* qblklen = nullptr;
  double2* K64 = nullptr;   // Woodbury K = (Q^-1 + P^dagger P)^-1
  double2* E64 = nullptr;   // E = (I - K P^dagger P) D
  float2* K32 = nullptr;
  float2* E32 = nullptr;
  double2* B64 = nullptr;   // P^dagger P (with Q: the filter's projector-space recurrence)
  float2* B32 = nullptr;
  // tensor-core operands of the mixed path: bf16 pieces of the real-ified P (built on first use)
  int tc_pieces = 3;         // bf16 pieces per operand (2: 3 products, 3: 6 products)
  int tc_built_pieces = 0;   // pieces the operands below were built with (0 = not built)
  void* tcA1 = nullptr;      // [pieces][2 nproj][kp1]
  void* tcA2 = nullptr;      // [pieces][2 npw][kp2]
  int64_t kp1 = 0, kp2 = 0;  // pitches (elements): 2 npw and 2 nproj rounded up to 64
  int* tc_err = nullptr;     // device flag set by a tensor-core kernel whose bounded wait expired
  // kernel-class timing (pw_profile_*)
  struct ProfRec { int cls; cudaEvent_t a, b; };
  bool prof_on = false;
  int prof_suspend = 0;  // >0 inside a Rayleigh-Ritz region: inner classes are not recorded
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<ProfRec> prof_recs;
  cudaEvent_t prof_open[PW_PROF_NCLASS] = {};
  double prof_ms[PW_PROF_NCLASS] = {};
  int64_t prof_n[PW_PROF_NCLASS] = {};
  // grow-only workspaces
  struct Buf { void* p = nullptr; size_t bytes = 0; };
  Buf ws[pw::WS_NUM];
  bool poisoned = false;
  uint64_t ws_gen = 0;  // bumped whenever a workspace is (re)allocated (captured graphs check it)
  // tuning: bytes of half-box planes per FFT band batch (complex64, complex128); set by pw_autotune
  size_t fft_batch_bytes[2] = {(size_t)48 << 20, (size_t)256 << 20};
  // FFT pass kernel forms per precision, variant = xline form + 8 * plane form.  x-line
  // forms: 0 line groups of 1-8 threads with shared-memory twiddles, 1 one thread per line
  // with compile-time twiddles, 2 groups of warps per 32 lines (lane = line) with
  // compile-time twiddles, 3 the same with run-time butterfly indices and table twiddles,
  // 4 as 3 with several bands per CTA (V kept in registers); plane forms: 0 line groups,
  // 1 one thread per line, 2 groups of warps per 32 lines with table twiddles.  Forms other
  // than 0 cover two-stage plans in complex64 only (otherwise form 0 runs); set by pw_autotune
  // FFT pass-kernel forms (complex64, complex128): complex128 defaults to the sphere-row +
  // column-slice plane kernels (plane form 3), which fall back to line groups where they do
  // not apply (1.2x the line-group form on the 120^3 box)
  int fft_variant[2] = {0, 3 * pw::kFormStride};
  int last_sweeps = 0;  // Jacobi sweeps of the last Rayleigh-Ritz step
  // K splits of the mixed projection GEMM per column count, chosen by pw_autotune (columns ->
  // splits); other column counts use the whole-waves rule
  std::vector<std::pair<int, int>> tc_proj_splits;
  // FP64 GEMMs: 1 = FP64-accurate digit-sliced tensor-core GEMMs where a product is large
  // enough (zgemm_tc.cu), 0 = DFMA GEMMs everywhere (pw_fp64_config)
  int fp64_tc = 1;
  // digit planes of P^dagger (A form, rows 2 nproj, K 2 npw) and of P (A form, rows 2 npw,
  // K 2 nproj) for the FP64 projector products, built on first use, with their row exponents
  void* ozPH = nullptr;
  void* ozP = nullptr;
  int* ozPH_exp = nullptr;
  int* ozP_exp = nullptr;
  // test hook: the next tensor-core GEMM issues no copies and waits briefly (its first wait
  // expires), so that the bounded-wait failure path can be exercised without a fault
  int test_wait_expiry = 0;
};

namespace pw {
void* ws_get(pw_ctx* c, int slot, size_t bytes, int* status);
// process-wide count of kernel launches issued by this library (diagnostics)
void count_launch();
// open / close a timed region of class `cls` on the context's stream (no-ops when off or ctx NULL)
void prof_begin(pw_ctx* c, int cls);
void prof_end(pw_ctx* c, int cls);
int set_error(int status, const char* fmt, ...);
int cuda_status(cudaError_t e, const char* where);
}  // namespace pw
