/*
 * pw.h -- C ABI of the GB300 Chebyshev-filtered plane-wave Hamiltonian library.
 *
 * The problem is the Kohn-Sham generalised eigenproblem H psi_i = lambda_i S psi_i
 * of arxiv 2604.11139 Sec. 3.1: N plane waves (the sphere |k+G|^2/2 <= E_cut),
 * M bands, H = T + V_loc + sum_ij |p_i> D_ij <p_j| (Sec. 4.2, nonlocal operator),
 * S = I + sum_ij |p_i> Q_ij <p_j| (PAW overlap, Sec. 3.1).  The library applies H
 * matrix-free (Sec. 3.2), runs the degree-m Chebyshev filter of Alg. 7 / Alg. 12
 * and the Rayleigh-Ritz step of Alg. 5, all in hand-written CUDA kernels for one
 * GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 *  - Wave-function blocks are column-major N x M complex matrices (interleaved
 *    re/im), band j at offset j*ld elements, ld >= npw (strided bands, Sec. 2.1).
 *    Rows follow the context's canonical plane-wave order (pw_ctx_gvectors).
 *    Element type: complex128 for PW_FP64 entry points, complex64 where a
 *    PW_MIXED precision is requested.  Blocks are DEVICE pointers owned by the
 *    caller unless stated otherwise.
 *  - Every call is asynchronous on the context's stream unless it returns host
 *    values (eigenvalues, bounds), in which case it synchronises that stream.
 *  - Workspaces are owned by the context and only grow; after the first call
 *    with a given shape no further device allocation happens.
 *  - Return value: PW_OK (0) or a negative pw_status.  No exception, abort or
 *    exit crosses the ABI.  pw_last_error() gives a one-line description of the
 *    last failure on the calling thread.  After PW_ECUDA the context must be
 *    destroyed.
 */
#ifndef PW_H
#define PW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PW_API __attribute__((visibility("default")))
#else
#define PW_API
#endif

typedef struct pw_ctx pw_ctx;

enum pw_status {
  PW_OK = 0,
  PW_EINVAL = -1,       /* bad argument: shapes, ld < npw, sphere not fitting the box */
  PW_ENOMEM = -2,       /* device allocation failed */
  PW_ECUDA = -3,        /* a CUDA call failed; the context is poisoned */
  PW_ENOTSPD = -4,      /* Cholesky of S_Psi, of Q or of Q^-1 + P^dagger P failed */
  PW_ETIMEDOUT = -5,    /* a bounded device-side wait expired */
  PW_ENOTCONV = -6,     /* subspace eigensolver did not converge */
  PW_EUNSUPPORTED = -7  /* FFT length with a prime factor outside {2,3,5}, etc. */
};

enum pw_precision {
  PW_FP64 = 0,  /* complex128 blocks, FP64 FFT and FP64 projector GEMMs */
  PW_MIXED = 1  /* complex64 blocks and FFTs, BF16-split tensor-core projector
                   GEMMs with FP32 accumulation (filter only) */
};

/* Problem statement (Sec. 3.1 and 4.2).  All pointers are HOST pointers and are
 * only read during pw_ctx_create. */
typedef struct {
  double lattice[9];   /* rows a1, a2, a3 in bohr */
  double kpt[3];       /* k-point in reduced coordinates */
  double ecut;         /* plane-wave cut-off (Ha): sphere |k+G|^2/2 <= ecut */
  int box[3];          /* FFT box n1, n2, n3; each factorises into 2, 3, 5 */
  const double* vloc;  /* n1*n2*n3 real V_loc(r_j), C order (index (j1*n2+j2)*n3+j3) */
  int natom;
  const double* tau;   /* natom*3 cartesian atom positions (bohr) */
  int nchan;           /* projector channels per atom; 4 projectors (s, px, py, pz) each */
  const double* sigma; /* nchan Gaussian widths (bohr) of the projector form factors */
  const double* D;     /* nproj*nproj real symmetric, column-major, nproj = natom*4*nchan
                          (or the nproj below when proj != NULL) */
  const double* Q;     /* nproj*nproj real symmetric positive definite, or NULL (S = I) */
  /* Explicit projectors (Sec. 4.2: the nonlocal operator takes the projector functions
   * <k+G|p_i^R> as data).  proj == NULL: P is generated from natom/tau/nchan/sigma as
   * described at pw_ctx_create, and nproj is ignored.  proj != NULL: P is read from
   * this host array of npw*nproj complex128 values (interleaved re/im), column-major
   * with ld = npw, rows in the canonical plane-wave order of pw_ctx_gvectors (Miller
   * indices (h, k, l) ascending; npw and the order depend only on lattice, kpt, ecut and
   * box, so a caller can read them from a context made with natom = 0); tau, nchan and
   * sigma are then ignored and D (and Q) are nproj x nproj.  The columns are used as
   * given (no normalisation).  PW_EINVAL if nproj < 1 or D is NULL. */
  int nproj;
  const void* proj;
} pw_problem_desc;

/* Builds the plane-wave sphere, the FFT plans, the projector matrix P (Sec. 4.2:
 * P = <G|p_i^R>; unless given explicitly, Gaussian s/p form factors, structure phase
 * exp(-i(k+G).R), unit column norm), the permuted V_loc grid and, when Q != NULL, the
 * Woodbury matrices of S^-1 (Sec. 3.3 Sinv).  Every precision uses the same P: the
 * FP64 path as given, the mixed path its complex64 rounding and its bf16 pieces.
 * stream: a cudaStream_t, or NULL for the legacy default stream.  On success *out owns
 * all device memory it uses. */
PW_API int pw_ctx_create(const pw_problem_desc* desc, void* stream, pw_ctx** out);
PW_API int pw_ctx_destroy(pw_ctx* ctx);
PW_API int pw_ctx_set_stream(pw_ctx* ctx, void* stream);

/* Waits for the work queued on the context's stream and reports device-side failures:
 * PW_ETIMEDOUT if a bounded wait of a tensor-core kernel expired (the context is then
 * poisoned and must be destroyed; the GPU and other contexts stay usable), PW_ECUDA for a
 * CUDA error.  Asynchronous entry points report such failures only at the next call that
 * synchronises (this one, or any that returns host values). */
PW_API int pw_ctx_sync(pw_ctx* ctx);

/* Failure-detection test hook: the next tensor-core GEMM launched for this context issues no
 * copies and gives up its waits after a few thousand polls, so its first bounded wait expires
 * and it leaves through its failure path (records the failing stage, waits for anything it
 * issued, releases tensor memory, returns).  The following pw_ctx_sync returns PW_ETIMEDOUT.
 * No device fault is involved; it exists so that the failure path can be tested. */
PW_API int pw_ctx_test_wait_expiry(pw_ctx* ctx);

/* Sizes: number of plane waves N and projectors N_projs. */
PW_API int pw_ctx_info(const pw_ctx* ctx, int* npw, int* nproj);

/* Canonical plane-wave order: Miller indices (h,k,l) sorted ascending by h, then
 * k, then l (host int32 array 3*npw, row-major), and the kinetic energies
 * |k+G|^2/2 (host, npw doubles).  Either pointer may be NULL. */
PW_API int pw_ctx_gvectors(const pw_ctx* ctx, int32_t* miller, double* kinetic);

/* Copies the projector matrix P in use (generated or given; npw x nproj complex128,
 * column-major, ld = npw) to the device buffer P_out. */
PW_API int pw_ctx_projectors(const pw_ctx* ctx, void* P_out);

/* HX / HX_SX of Sec. 3.3: hpsi = H psi and, if spsi != NULL, spsi = S psi for
 * nband bands.  psi, hpsi, spsi: device blocks of the element type of
 * `precision`, leading dimensions ldpsi and ldout.  psi must not alias the
 * outputs. */
PW_API int pw_hamiltonian_apply(pw_ctx* ctx, const void* psi, int64_t ldpsi, int nband,
                                void* hpsi, void* spsi, int64_t ldout, int precision);

/* Spectrum bounds of Alg. 12 (FP64): Rayleigh quotients
 * lambda_i = (H psi_i)^dagger psi_i / ((S psi_i)^dagger psi_i) of the complex128
 * block psi -> *rq_min, *rq_max (host); and an upper bound of the spectrum of
 * S^-1 H from `lanczos_steps` Lanczos steps on H from the complex128 start
 * vector v0 (npw, device): *upper = theta_max + |beta_k| (host).  With nband = 0
 * only the Lanczos bound is computed; with lanczos_steps = 0 only the quotients. */
PW_API int pw_spectrum_bounds(pw_ctx* ctx, const void* psi, int64_t ld, int nband,
                              int lanczos_steps, const void* v0,
                              double* rq_min, double* rq_max, double* upper);

/* Chebyshev filter of degree m (Alg. 7 / Alg. 12, three-term recurrence):
 * c = (b+a)/2, e = (b-a)/2, Y_0 = psi, Y_1 = (A-c)Y_0/e,
 * Y_{k+1} = (2/e)(A-c)Y_k - Y_{k-1}, A = S^-1 H (Woodbury, Sec. 3.3) or H.
 * psi is overwritten with Y_m.  PW_FP64: complex128 block; PW_MIXED:
 * complex64 block, FP32 FFTs and BF16-split tensor-core projector GEMMs.  With Q a step
 * projects only W = (T + V) Y_k onto the projectors; P^dagger Y_k follows the same
 * recurrence in projector space through the stored P^dagger P. */
PW_API int pw_chebyshev_filter(pw_ctx* ctx, void* psi, int64_t ldpsi, int nband,
                               int degree, double a, double b, int precision);

/* Rayleigh-Ritz on the complex128 block psi (Alg. 5 preceded by S-Ortho, Alg. 9:
 * one Cholesky-QR pass in the S metric, the Cholesky reduction inside Alg. 5 being the
 * second), all FP64: psi <- S-orthonormalised Ritz vectors, eig (host,
 * nband, ascending) <- Ritz values, resid (host, nband, may be NULL) <-
 * ||H psi_i - lambda_i S psi_i||.  hpsi (may be NULL, ld = ldpsi) receives H psi.
 * Returns PW_ENOTSPD if the block is numerically rank deficient. */
PW_API int pw_rayleigh_ritz(pw_ctx* ctx, void* psi, int64_t ldpsi, int nband,
                            void* hpsi, double* eig, double* resid);

/* One full ChebFi solve (Alg. 12): Lanczos upper bound from v0 (device, complex128),
 * cycle-1 cut = max Rayleigh quotient of psi, then `cycles` times
 * [filter (precision) -> Rayleigh-Ritz (FP64)], the cut of each later cycle
 * being the largest Ritz value.  psi: complex128 device block, overwritten with
 * the Ritz vectors.  eig, resid: host arrays of nband (resid may be NULL).
 * bounds (host, may be NULL) receives {upper, first cut}.  With PW_MIXED the Rayleigh
 * quotients of the first cut take their numerators from the complex64 H-apply (their
 * denominators, with Q, from the FP64 S-apply). */
PW_API int pw_chebfi_solve(pw_ctx* ctx, void* psi, int64_t ldpsi, int nband, int degree,
                           int cycles, int lanczos_steps, const void* v0, int precision,
                           double* eig, double* resid, double* bounds);

/* Density / gradient contraction (Alg. 3 density step):
 * out(r_j) (+)= sum_i w_i Re[conj(a_i(r_j)) b_i(r_j)], a_i(r) = sum_G a_iG e^{iG.r_j}
 * (unnormalised inverse DFT), b = a when b == NULL.  a, b: complex128 device
 * blocks (ld); w: host weights (nband); out: device n1*n2*n3 doubles in C order;
 * accumulate != 0 adds to out instead of overwriting it. */
PW_API int pw_density_grad(pw_ctx* ctx, const void* a, const void* b, int64_t ld, int nband,
                           const double* w, double* out, int accumulate);

/* ---- k-point batches (Sec. 2.4: k-points are independent; one launch for all) ----
 * A batch groups contexts of one cell at different k-points (ragged sphere sizes).
 * pw_batch_filter runs the Chebyshev filter of every k-point; the first call for a
 * given (blocks, nband, degree, precision) runs the launches directly and captures
 * them into one CUDA graph (k-points spread over 4 streams), later calls replay that
 * graph with one launch, the filter intervals being read from device memory.
 * A context's workspaces growing (a larger call made on it directly) forces a new
 * capture.  Blocks psi[k] (device, ld[k] >= npw_k) are complex128 for PW_FP64 and
 * complex64 for PW_MIXED; a[k] < b[k] are host arrays.  The contexts must outlive
 * the batch and must not be used concurrently with it; their profiling must be off. */
typedef struct pw_batch pw_batch;
PW_API int pw_batch_create(pw_ctx* const* ctxs, int nk, void* stream, pw_batch** out);
PW_API int pw_batch_destroy(pw_batch* batch);
PW_API int pw_batch_filter(pw_batch* batch, void* const* psi, const int64_t* ld, int nband, int degree,
                           const double* a, const double* b, int precision);
/* ChebFi on every k-point (Alg. 12 per k): Lanczos bounds from v0[k] (complex128,
 * device), `cycles` times [batched filter -> per-k FP64 Rayleigh-Ritz].  psi[k]:
 * complex128 device blocks; eig (host, nk x nband) and resid (host, may be NULL). */
PW_API int pw_batch_chebfi_solve(pw_batch* batch, void* const* psi, const int64_t* ld, int nband, int degree,
                                 int cycles, int lanczos_steps, void* const* v0, int precision, double* eig,
                                 double* resid);

/* ---- differentiation form (S = I): reverse-mode adjoint of ChebFi ----
 * The parameters of H are V_loc(r_j) and D.  pw_ctx_set_vloc / pw_ctx_set_D replace
 * them in a context (V_loc: n1*n2*n3 doubles in C order; D: nproj*nproj doubles,
 * column-major, zero outside the context's D blocks; host or device pointers, read
 * during the call; pw_ctx_set_D needs Q == NULL).
 * pw_local_apply: out = alpha V psi for an arbitrary real potential v on the FFT grid
 * (device, n1*n2*n3 doubles, C order) through the same sphere -> box FFT, multiply and
 * box -> sphere FFT as the local part of H (Sec. 3.2); no kinetic or nonlocal term.
 * psi, out: device blocks of the precision's element type (complex128 / complex64).
 * It is the adjoint of the density (Alg. 3 density step): for
 * rho(r) = sum_i w |psi_i(r)|^2 and a loss gradient rho_bar(r), the gradient of psi_i
 * is pw_local_apply with v = rho_bar and alpha = 2 w n1n2n3. */
PW_API int pw_ctx_set_vloc(pw_ctx* ctx, const double* vloc);
PW_API int pw_ctx_set_D(pw_ctx* ctx, const double* D);
PW_API int pw_local_apply(pw_ctx* ctx, const double* v, double alpha, const void* psi, int64_t ld,
                          int nband, void* out, int64_t ldo, int precision);

/* A differentiation handle holds the tape of `cycles` ChebFi cycles of degree `degree`
 * on nband bands: per cycle the filter iterates (pairs (Y_{js}, Y_{js+1}) of every
 * segment of ckpt steps; ckpt <= 2 keeps them all), P^dagger Y_k, the S-orthonormal
 * block Q, the Rayleigh-Ritz rotation X and (Q^dagger Y_m)^-dagger.  precision PW_MIXED
 * runs the filter and its adjoint in complex64 with BF16-split tensor-core projector
 * GEMMs; the Rayleigh-Ritz step and its adjoint are FP64 in both precisions.  The
 * handle allocates all its device memory at creation (pw_diff_tape_bytes reports it). */
typedef struct pw_diff pw_diff;
PW_API int pw_diff_create(pw_ctx* ctx, int nband, int degree, int cycles, int ckpt, int precision,
                          pw_diff** out);
PW_API int pw_diff_destroy(pw_diff* diff);
PW_API int pw_diff_tape_bytes(const pw_diff* diff, int64_t* bytes);
/* Forward: the ChebFi cycles of pw_chebfi_solve (Alg. 12), recording the tape.  psi:
 * complex128 device block (ld), overwritten with the Ritz vectors.  The filter
 * interval is stop-gradient: bounds_in (host, 1 + cycles doubles: the upper bound b,
 * then the cut a of every cycle) replays given bounds; NULL computes them (Lanczos
 * from v0 with lanczos_steps steps, cycle-1 cut = max Rayleigh quotient of psi, later
 * cuts = largest Ritz value).  eig (host, nband) and bounds_out (host, 1 + cycles) may
 * be NULL. */
PW_API int pw_diff_forward(pw_diff* diff, void* psi, int64_t ld, int lanczos_steps, const void* v0,
                           const double* bounds_in, double* eig, double* bounds_out);
/* Backward: given the adjoints of the last cycle's Ritz values (eig_bar, host, nband,
 * NULL = 0) and Ritz vectors (psi_bar, complex128 device block, NULL = 0), in PyTorch's
 * convention (psi_bar = dL/dRe psi + i dL/dIm psi), writes (accumulate = 0) or adds
 * dL/dV_loc(r_j) to dV (device, n1*n2*n3 doubles, C order) and dL/dD_ab, entries taken
 * as independent, to dD (device, nproj*nproj doubles, column-major); either may be NULL.
 * split < 0 keeps every eigenvector-coupling pair (i, j) of the last cycle; split >= 0
 * keeps only pairs with one band below split and one at or above it, which is exact
 * when the loss does not change under rotations among bands [0, split) and among
 * [split, nband) (e.g. sums of occupied eigenvalues and the occupied density) and
 * avoids dividing by small gaps.  PW_EINVAL if V_loc or D changed since the forward. */
PW_API int pw_diff_backward(pw_diff* diff, const double* eig_bar, const void* psi_bar, int64_t ld,
                            int split, double* dV, double* dD, int accumulate);

/* ---- spectrum slicing (the slice-wise solve the paper's closing section proposes) ----
 * The wanted spectrum is cut into nslice slices [cuts[s], cuts[s+1]] (host, nslice + 1 strictly
 * ascending values); slice s owns the nper bands [s nper, (s+1) nper) of psi.  Each slice's
 * block is filtered by a window polynomial that passes that slice only, and then solved by a
 * small Rayleigh-Ritz step of its own, independent of the other slices.  The paper names the
 * method without formulas; the windows are the standard ones of the slicing literature: the
 * Chebyshev expansion of the slice's indicator function on the spectrum mapped to [-1, 1]
 * (t = (lambda - c)/e, c = (hi + lo)/2, e = (hi - lo)/2; [lo, hi] must contain the spectrum of
 * A = S^-1 H), mu_0 = (acos ta - acos tb)/pi, mu_j = 2 (sin(j acos ta) - sin(j acos tb))/(j pi),
 * damped by the Jackson factors g_j of the degree: p_s(t) = sum_{j <= degree} g_j mu_j T_j(t).
 * pw_slice_filter: psi_s <- p_s(A~) psi_s for every slice, A~ = (A - c)/e.  One recurrence
 * T_{j+1} = 2 A~ T_j - T_{j-1} runs over all nslice nper bands (the H-applies batched over the
 * slices, as in pw_chebyshev_filter) and each band accumulates its own slice's coefficients.
 * psi: device, element type of precision (complex128 / complex64).
 * pw_spectrum_slice: pw_slice_filter (complex64 copy with PW_MIXED), then per slice an FP64
 * S-Ortho + Rayleigh-Ritz step (as pw_rayleigh_ritz) on its nper bands.  psi: complex128,
 * out: the Ritz vectors slice by slice; eig (host, nslice nper): each slice's Ritz values
 * ascending; resid (host, may be NULL): their residual norms.  The caller keeps the values
 * inside each slice.  PW_EINVAL for bad sizes, bounds or cuts; PW_ENOTSPD if a slice's block
 * is numerically rank deficient (more vectors than the window leaves alive: lower nper). */
PW_API int pw_slice_filter(pw_ctx* ctx, void* psi, int64_t ldpsi, int nslice, int nper, int degree, double lo,
                           double hi, const double* cuts, int precision);
PW_API int pw_spectrum_slice(pw_ctx* ctx, void* psi, int64_t ldpsi, int nslice, int nper, int degree, double lo,
                             double hi, const double* cuts, int precision, double* eig, double* resid);

/* ---- LOBPCG (Alg. 11), the vector-oriented solver the paper compares ChebFi with ----
 * nblocks blocks of nband / nblocks consecutive bands, treated one after the other, each with
 * up to nline line minimisations; FP64 throughout (H-apply, Grams, rotations).  Per block i:
 * S-Deflate (Alg. 8) against the finished blocks (i > 1), H and S applied, S-Ortho (Alg. 9),
 * Rayleigh-Ritz (Alg. 10); then per line minimisation the residual W = (H - Lambda S) Psi_i
 * (the loop ends once every residual norm of the block is below tol; tol = 0: never), the
 * diagonal Teter-Payne-Allan preconditioner K_G = p / (p + 16 x^4), p = 27 + 18 x + 12 x^2 +
 * 8 x^3, x = t_G / E_kin(psi) (the paper names K a diagonal preconditioner without giving it),
 * S-Deflate of W, H W and S W, S-Ortho + RR on [Psi_i W_i] (first minimisation) or [Psi_i W_i
 * P_i], keeping the nband / nblocks lowest Ritz pairs: P_i <- the W and P part of the kept
 * vectors, Psi_i <- the Psi part + P_i.  With nblocks > 1 a final S-Ortho + RR over all bands.
 * psi: device complex128 block (ld >= npw), in: the starting bands, out: the S-orthonormal Ritz
 * vectors.  eig (host, nband): Ritz values ascending; resid (host, nband, may be NULL):
 * ||H psi_i - lambda_i S psi_i||; iters (host, nblocks, may be NULL): line minimisations done
 * per block.  PW_EINVAL if nband is not a multiple of nblocks or nline < 0; PW_ENOTSPD if a
 * Gram of S-Ortho is not numerically positive definite (a basis [Psi W P] that has lost rank,
 * typically well past convergence: stop earlier with tol). */
PW_API int pw_lobpcg_solve(pw_ctx* ctx, void* psi, int64_t ldpsi, int nband, int nblocks, int nline, double tol,
                           double* eig, double* resid, int* iters);

/* ---- Gamma-point pairing (time-reversal symmetry at k = 0) ----
 * At k = 0 a function real in r-space has coefficients c(-G) = conj c(G), and H maps such
 * functions to such functions when V_loc, D and Q are real and the projectors satisfy
 * P(-G) = conj P(G) (the generated s/p projectors do; explicit ones must).  Two such bands a,
 * b then travel as one complex band c = a + i b: H is linear, so H c = H a + i H b, and the
 * Chebyshev filter p(A) of pw_chebyshev_filter gives p(A) c = p(A) a + i p(A) b, i.e. the
 * filter of 2 m such bands costs the FFTs and GEMMs of m bands.  In the canonical order the
 * partner -G of index i is npw - 1 - i.
 * pw_gamma_symmetrize: psi <- (psi(G) + conj psi(-G)) / 2, the r-space-real part, in place.
 * pw_gamma_pack: c_j = a_{2j} + i a_{2j+1} for j < nband / 2 (nband even).
 * pw_gamma_unpack: a_{2j}(G) = (c_j(G) + conj c_j(-G)) / 2, a_{2j+1}(G) = (c_j(G) - conj c_j(-G)) / (2 i).
 * Blocks: device, element type of `precision`; nband counts the unpacked bands.  PW_EINVAL
 * unless the context is at k = 0, for odd nband, or for aliasing input and output. */
PW_API int pw_gamma_symmetrize(pw_ctx* ctx, void* psi, int64_t ld, int nband, int precision);
PW_API int pw_gamma_pack(pw_ctx* ctx, const void* a, int64_t lda, int nband, void* c, int64_t ldc, int precision);
PW_API int pw_gamma_unpack(pw_ctx* ctx, const void* c, int64_t ldc, int nband, void* a, int64_t lda, int precision);

/* ---- self-consistent field loop (Alg. 3) ----
 * Alg. 3 repeats: solve H Psi = Lambda S Psi, occupations from Lambda, density from the
 * occupations and Psi, until self-consistent.  The paper leaves open how the density sets the
 * next Hamiltonian; these entry points close the loop with a minimal published model:
 * insulating filling (the lowest nocc states hold 2 electrons each), the Hartree potential
 * V_H(G) = 4 pi rho(G) / |G|^2 (G != 0; neutralising background at G = 0) and Dirac's
 * local-density exchange v_x = -(3 rho / pi)^(1/3) (energy density -(3/4) (3/pi)^(1/3)
 * rho^(4/3); no correlation); the next V_loc is V_in + beta (V_ion + V_H + v_x - V_in).
 *
 * dctx is a "density context": the same cell and FFT box at the Gamma point, no projectors
 * (natom = 0, D empty), E_cut four times the wave functions' (its sphere holds every Fourier
 * component of a density of the E_cut orbitals; its box must hold that sphere).
 *
 * pw_scf_potential: from rho (device, n1*n2*n3 doubles, C order, electrons / bohr^3), V_ion and
 * V_in (device grids), writes V_new (device grid) and out[5] (host): (Omega/n) sum (V_in -
 * V_ion) rho, the Hartree energy (Omega/2n) sum V_H rho, the exchange energy (Omega/n) sum
 * rho e_x, max |V_ion + V_H + v_x - V_in|, and the electron count (Omega/n) sum rho.
 * Synchronises dctx's stream. */
PW_API int pw_scf_potential(pw_ctx* dctx, const double* rho, const double* vion, const double* vin, double beta,
                            double* vnew, double* out);
/* The loop: V_in = V_ion (host or device grid, C order), then up to max_iter times
 * [pw_chebfi_solve(ctx, psi, ..., degree, cycles, 10 Lanczos steps from v0, precision) ->
 * density of the lowest nocc bands (weights 2 / Omega) -> pw_scf_potential -> V_loc of ctx]
 * until max |V_out - V_in| < tol.  psi: complex128 device block (ld), carried from one
 * iteration to the next; eig (host, nband): the last eigenvalues; history (host, 2 max_iter,
 * may be NULL): per iteration the energy sum_i f_i lambda_i - (Omega/n) sum (V_in - V_ion) rho
 * + E_H + E_x and max |V_out - V_in|; *iterations (may be NULL) the iterations run.  On
 * return ctx holds the last input potential.  Allocates 4 grids of scratch for the call.
 * PW_ENOTCONV if tol was not reached. */
PW_API int pw_scf_run(pw_ctx* ctx, pw_ctx* dctx, void* psi, int64_t ld, int nband, int nocc, int degree, int cycles,
                      int max_iter, double beta, double tol, const void* v0, const double* vion, int precision,
                      double* eig, double* history, int* iterations);

/* H psi = (T + V_loc + P D P^dagger) psi in FP64, like pw_hamiltonian_apply with
 * spsi = NULL, but without allocating any device memory.  The paper has no
 * counterpart; this exists for callers that may not call cudaMalloc/cudaFree at
 * apply time (a framework allocator that owns all device memory, a hard memory
 * cap, a loop that cannot absorb cudaFree's device-wide synchronisation).  All
 * scratch lives in one static 32 MiB device array inside the library, held by
 * every GPU that loads it until process exit.  The first call on a device looks
 * up that array's address (cudaGetSymbolAddress); make it before any stream
 * capture.  The address is cached per device for the life of the process, so after a
 * cudaDeviceReset of that device this entry point must not be called again.  Calls
 * share the array: calls that overlap on the GPU race.  Bands are
 * processed in chunks that fit; PW_EINVAL if even one band's scratch (half-box
 * planes + projections) exceeds 32 MiB.  psi, hpsi: complex128 device blocks. */
PW_API int pw_hamiltonian_apply_noalloc(pw_ctx* ctx, const void* psi, int64_t ldpsi, int nband,
                                        void* hpsi, int64_t ldout);

/* Diagnostics.  Per-context timing of kernel classes with CUDA events recorded
 * on the context's stream around each launch (no extra synchronisation while
 * enabled).  pw_profile_read synchronises the stream, returns the accumulated
 * milliseconds and launch counts per class (arrays of PW_PROF_NCLASS) and resets
 * them.  pw_kernel_launches returns the number of kernels this library has
 * launched in the process so far. */
enum pw_prof_class {
  PW_PROF_PLANE_INV = 0,  /* FFT pass 1: sphere -> inverse (z, y) planes */
  PW_PROF_XLINE = 1,      /* FFT pass 2: x-lines, inverse x, V_loc, forward x */
  PW_PROF_PLANE_FWD = 2,  /* FFT pass 3: forward (y, z), gather, kinetic */
  PW_PROF_GEMM_PROJ = 3,  /* C_proj = P^dagger Y (and P^dagger W with S) */
  PW_PROF_GEMM_BACK = 4,  /* Y_{k+1} = alpha (W + P Z - c Y_k) - beta Y_{k-1}, or H psi += P Z */
  PW_PROF_SMALL = 5,      /* projector-space products D C, E C - K C_w */
  PW_PROF_RR = 6,         /* S-Ortho + Rayleigh-Ritz (whole step) */
  PW_PROF_NCLASS = 7
};
/* Autotuner: times the local-potential FFT passes on nband bands for several band
 * batch sizes (the batch's half-box planes from 16 MB to 2 GB) and, for PW_MIXED, the
 * forms of the pass kernels, variant = x-line form + 16 * plane form (0-6).  x-line forms:
 * 0 line groups of 1-8 threads with shared-memory twiddles, 1 one thread per line with
 * compile-time twiddles, 2 groups of warps per 32 lines with compile-time twiddles,
 * 3 the same with run-time butterfly indices and table twiddles, 4 as 3 with several bands
 * per CTA, 5 and 6 as 3 and 4 with the two radices of the x plan in the other order (the
 * radix plan of the x-lines is thus a tuned choice; V_loc is kept permuted for both
 * orders), 7-10 as 3-6 with each band's planes staged into shared memory by asynchronous
 * copies (the several-band forms 8 and 10 double-buffered: band b + 1 in flight while band
 * b is transformed).  Plane forms: 0 line groups, 1 one thread per line, 2 groups of warps per 32
 * lines with table twiddles over the whole plane in shared memory, 3 the same over the
 * plane's sphere rows and 32-column slices (less shared memory per CTA on large boxes),
 * 4 form 3 for the inverse pass and form 2 for the forward pass, 5 as 4 with a persistent
 * forward pass (one CTA per SM walking the planes; the next plane is prefetched into L2 and its
 * blocks of Y_k and t_G into shared memory while the current one is gathered), 6 both passes
 * whole-plane and persistent (pass 1 prefetching the next plane's sphere block into L2).
 * For PW_MIXED the bare-apply ranking is then checked inside two steps of the filter itself:
 * every plane form with the best x-line form, and the runner-up x-line form with the best
 * plane form; the fastest there is kept.
 * PW_FP64 tunes the plane form only (0 or 3, variant 0 or 48; its x-line form is fixed).
 * Forms other than 0 cover box lengths with two-stage radix plans.  Keeps the fastest for
 * `precision` in the context.  Synchronises the stream; *best_ms (may be NULL) receives
 * the best time of one apply. */
PW_API int pw_autotune(pw_ctx* ctx, int nband, int precision, double* best_ms);
/* (pw_autotune, PW_MIXED, continued) It then times the K-split counts of the projection
 * GEMM C = P^dagger Y around the whole-waves rule for nband columns and keeps the fastest;
 * other column counts use the rule. */
/* Reads (*batch_bytes, *variant; either pointer may be NULL) and then, for arguments
 * >= 0, sets the FFT configuration of `precision`: bytes of half-box planes per band
 * batch (>= 1 band is always used) and the pass-kernel forms (as for
 * pw_autotune; non-zero forms apply to PW_MIXED only and fall back to 0 for box
 * lengths they do not cover).  Pass -1 to leave a field unchanged. */
PW_API int pw_fft_config(pw_ctx* ctx, int precision, int64_t set_batch_bytes, int set_variant,
                         int64_t* batch_bytes, int* variant);

/* Reads (*pieces, may be NULL) and then, for set_pieces >= 0, sets the number of bf16
 * pieces per operand of the mixed-precision projector GEMMs: 3 (six products, ~2^-24
 * relative per product, the default) or 2 (three products, ~2^-16).  The tensor-core
 * operands of P are rebuilt on the next mixed-precision call. */
PW_API int pw_tc_config(pw_ctx* ctx, int set_pieces, int* pieces);

/* Reads (*mode, may be NULL) and then, for set_mode >= 0, sets how the FP64 complex GEMMs of
 * the context run (the projector products of the FP64 H-apply and filter, Sec. 4.2, and the
 * Rayleigh-Ritz Grams and rotations, Alg. 5): 1 (the default) as FP64-accurate GEMMs on the
 * bf16 tensor cores by exact digit slicing (each row of op(A) and column of op(B) scaled by a
 * power of two and cut into seven 7-bit integer digits; the 28 digit products with the seven
 * leading weights summed exactly in FP32 per 256-wide K chunk, combined in 64-bit integers and
 * accumulated in FP64; error per product below 2^-44 of the row and column maxima), 0 as DFMA
 * GEMMs.  Products with at most 4 columns (matrix-vector forms) and the M x M x M products of
 * the subspace step always use DFMA. */
PW_API int pw_fp64_config(pw_ctx* ctx, int set_mode, int* mode);

/* Measured FP64 FMA rate of the current GPU (the roofline of DFMA-bound kernels: the DFMA
 * GEMM form and the complex128 FFT passes): a kernel of independent FMA chains on every SM,
 * best of three timed runs on `stream` (a cudaStream_t or NULL) after one warm-up.  *tflops
 * receives 2 x FMAs / second / 1e12, *ms (may be NULL) the kernel time.  Allocates and frees
 * a small device buffer; synchronises the stream. */
PW_API int pw_diag_fp64_fma_rate(void* stream, double* tflops, double* ms);

PW_API int pw_profile_enable(pw_ctx* ctx, int on);
PW_API int pw_profile_read(pw_ctx* ctx, double* ms, int64_t* launches);
PW_API uint64_t pw_kernel_launches(void);

PW_API const char* pw_strerror(int status);
PW_API const char* pw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PW_H */
