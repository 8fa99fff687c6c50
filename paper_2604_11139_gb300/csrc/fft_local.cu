// Local-potential part of the matrix-free H-apply (Sec. 2.1, Alg. 2; Sec. 3.2):
// sphere -> box, inverse 3-D DFT, multiply by V_loc(r), forward 3-D DFT, box -> sphere,
// batched over bands and pruned to the plane-wave sphere.
//
// Three passes per band batch, each a hand-written shared-memory radix FFT:
//   pass 1 (k_plane_inv): one CTA per (x-plane with sphere content, band).  The
//          plane's runs of coefficients are scattered into shared memory, the
//          z-lines that hold coefficients are transformed (inverse DIF), then the
//          y-lines in chunks of z; the plane is written to the half-box buffer.
//   pass 2 (k_xline):     one CTA per chunk of (y,z) lines.  The 2r+1 non-zero
//          planes are placed on x-lines, inverse x-DIF, times V(r) / n1n2n3,
//          forward x-DIT, and only the 2r+1 sphere planes are written back.
//   pass 3 (k_plane_fwd): forward y-DIT on every z chunk, forward z-DIT on the
//          rows holding coefficients, gather to the sphere and the kinetic term:
//          out = |k+G|^2/2 psi + (V psi).
// Inverse transforms are decimation-in-frequency (natural in, digit-reversed
// out) and forward transforms decimation-in-time with reversed stages
// (digit-reversed in, natural out); between them the data stays in the
// digit-reversed (y,z) order and the potential grid is stored permuted to it,
// so no transposition or bit-reversal pass exists.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "pw_internal.cuh"

namespace pw {

// x-line kernel forms 3-10 (run-time butterfly indices, table twiddles): several bands per
// CTA, the radices of the x plan swapped, the planes staged by asynchronous copies
constexpr bool xf_twr(int xf) { return xf >= 3 && xf <= 10; }
constexpr bool xf_multi(int xf) { return xf == 4 || xf == 6 || xf == 8 || xf == 10; }
constexpr bool xf_swap(int xf) { return xf == 5 || xf == 6 || xf == 9 || xf == 10; }
constexpr bool xf_staged(int xf) { return xf >= 7 && xf <= 10; }

// ---- butterfly arithmetic ---------------------------------------------------------
// complex64 sums, differences and real scalings use the paired FP32 instructions of
// sm_100-class SMs (one add, multiply or fused multiply-add for both halves of a float2,
// each half rounded to nearest as the scalar instruction would); complex128 keeps the
// scalar forms.  The products by +-i swap the halves of an operand, which a paired
// instruction cannot do in place, so they stay two scalar instructions (measured on the
// 120^3 plane passes: 6% faster than paired with the swap; all-scalar butterflies are
// slower still).  Every form rounds each result identically.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 bf_add(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float2 bf_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 bf_sub(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ float2 bf_sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 bf_scale(double2 a, double s) { return cscale(a, s); }
__device__ __forceinline__ float2 bf_scale(float2 a, float s) { return __fmul2_rn(a, f2(s, s)); }
// a + s b
__device__ __forceinline__ double2 bf_axpy(double2 a, double s, double2 b) {
  return make_double2(fma(s, b.x, a.x), fma(s, b.y, a.y));
}
__device__ __forceinline__ float2 bf_axpy(float2 a, float s, float2 b) { return __ffma2_rn(b, f2(s, s), a); }
// a + (S i) s b  and  a - (S i) s b
template <int S> __device__ __forceinline__ double2 bf_add_muli(double2 a, double2 b, double s = 1.0) {
  return make_double2(fma(-S * s, b.y, a.x), fma(S * s, b.x, a.y));
}
template <int S> __device__ __forceinline__ float2 bf_add_muli(float2 a, float2 b, float s = 1.f) {
  return f2(__fmaf_rn(-S * s, b.y, a.x), __fmaf_rn(S * s, b.x, a.y));
}
template <int S> __device__ __forceinline__ double2 bf_sub_muli(double2 a, double2 b, double s = 1.0) {
  return make_double2(fma(S * s, b.y, a.x), fma(-S * s, b.x, a.y));
}
template <int S> __device__ __forceinline__ float2 bf_sub_muli(float2 a, float2 b, float s = 1.f) {
  return f2(__fmaf_rn(S * s, b.y, a.x), __fmaf_rn(-S * s, b.x, a.y));
}

// ---- small DFTs: y_m = sum_k x_k exp(S 2 pi i k m / R) -------------------------
template <typename C, int S> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a; a = bf_add(t, b); b = bf_sub(t, b);
}
template <typename C, int S> __device__ __forceinline__ void dft4(C* x) {
  C s02 = bf_add(x[0], x[2]), d02 = bf_sub(x[0], x[2]);
  C s13 = bf_add(x[1], x[3]), d13 = bf_sub(x[1], x[3]);
  x[0] = bf_add(s02, s13); x[2] = bf_sub(s02, s13);
  x[1] = bf_add_muli<S>(d02, d13); x[3] = bf_sub_muli<S>(d02, d13);
}
template <typename C, int S> __device__ __forceinline__ void dft8(C* x) {
  using R = decltype(C{}.x);
  const R h = (R)0.70710678118654752440084436210485;  // cos(pi/4)
  C e[4] = {x[0], x[2], x[4], x[6]};
  C o[4] = {x[1], x[3], x[5], x[7]};
  dft4<C, S>(e); dft4<C, S>(o);
  // o[m] *= w8^m, w8 = exp(S i pi/4): w8 = h (1 + S i), w8^3 = h (-1 + S i)
  const C o1 = bf_scale(bf_add_muli<S>(o[1], o[1]), h);
  const C o3 = bf_scale(bf_sub_muli<S>(o[3], o[3]), -h);
  x[0] = bf_add(e[0], o[0]); x[4] = bf_sub(e[0], o[0]);
  x[1] = bf_add(e[1], o1); x[5] = bf_sub(e[1], o1);
  x[2] = bf_add_muli<S>(e[2], o[2]); x[6] = bf_sub_muli<S>(e[2], o[2]);
  x[3] = bf_add(e[3], o3); x[7] = bf_sub(e[3], o3);
}
template <typename C, int S> __device__ __forceinline__ void dft3(C* x) {
  using R = decltype(C{}.x);
  const R s3 = (R)0.86602540378443864676372317075294;  // sin(pi/3)
  C t = bf_add(x[1], x[2]);
  C d = bf_sub(x[1], x[2]);
  C m = bf_axpy(x[0], (R)-0.5, t);
  x[0] = bf_add(x[0], t);
  x[1] = bf_add_muli<S>(m, d, s3);
  x[2] = bf_sub_muli<S>(m, d, s3);
}
template <typename C, int S> __device__ __forceinline__ void dft5(C* x) {
  using R = decltype(C{}.x);
  const R c1 = (R)0.30901699437494742410229341718282;   // cos(2pi/5)
  const R c2 = (R)-0.80901699437494742410229341718282;  // cos(4pi/5)
  const R s1 = (R)0.95105651629515357211643933337938;   // sin(2pi/5)
  const R s2 = (R)0.58778525229247312916870595463907;   // sin(4pi/5)
  C t1 = bf_add(x[1], x[4]), t2 = bf_add(x[2], x[3]);
  C d1 = bf_sub(x[1], x[4]), d2 = bf_sub(x[2], x[3]);
  C a1 = bf_add(x[0], bf_axpy(bf_scale(t1, c1), c2, t2));
  C a2 = bf_add(x[0], bf_axpy(bf_scale(t1, c2), c1, t2));
  C u1 = bf_axpy(bf_scale(d1, s1), s2, d2);    // b1 = (S i) u1
  C u2 = bf_axpy(bf_scale(d1, s2), -s1, d2);   // b2 = (S i) u2
  x[0] = bf_add(x[0], bf_add(t1, t2));
  x[1] = bf_add_muli<S>(a1, u1); x[4] = bf_sub_muli<S>(a1, u1);
  x[2] = bf_add_muli<S>(a2, u2); x[3] = bf_sub_muli<S>(a2, u2);
}
// exp(-2 pi i m / R) for the composite in-register radices, filled by fft_set_constants
// (host cos/sin in double).  Offsets: R=6: 0, 9: 6, 10: 15, 12: 25, 15: 37, 16: 52.
__constant__ double2 c_wtab64[68];
__constant__ float2 c_wtab32[68];
template <int R> struct WOff;
template <> struct WOff<6> { static constexpr int v = 0; };
template <> struct WOff<9> { static constexpr int v = 6; };
template <> struct WOff<10> { static constexpr int v = 15; };
template <> struct WOff<12> { static constexpr int v = 25; };
template <> struct WOff<15> { static constexpr int v = 37; };
template <> struct WOff<16> { static constexpr int v = 52; };

template <typename C, int S, int R> __device__ __forceinline__ C wconst(int m) {
  C w;
  if constexpr (sizeof(C) == 16) { const double2 t = c_wtab64[WOff<R>::v + m]; w.x = t.x; w.y = t.y; }
  else { const float2 t = c_wtab32[WOff<R>::v + m]; w.x = t.x; w.y = t.y; }
  if (S > 0) w.y = -w.y;
  return w;
}

template <typename C, int S, int R> __device__ __forceinline__ void dftR(C* x);

// R = R1 R2 in registers: R2 DFTs of length R1 (stride R2), constant twiddles w_R^{b k1},
// R1 DFTs of length R2; natural-order output X[k1 + R1 k2].
template <typename C, int S, int R, int R1, int R2> __device__ __forceinline__ void dft_comp(C* x) {
  C t[R];
#pragma unroll
  for (int b = 0; b < R2; ++b) {
    C u[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) u[a] = x[b + R2 * a];
    dftR<C, S, R1>(u);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) t[b + R2 * k1] = (b * k1 == 0) ? u[k1] : cmul(u[k1], wconst<C, S, R>(b * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    C v[R2];
#pragma unroll
    for (int b = 0; b < R2; ++b) v[b] = t[b + R2 * k1];
    dftR<C, S, R2>(v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = v[k2];
  }
}

template <typename C, int S, int R> __device__ __forceinline__ void dftR(C* x) {
  if constexpr (R == 2) dft2<C, S>(x[0], x[1]);
  else if constexpr (R == 3) dft3<C, S>(x);
  else if constexpr (R == 4) dft4<C, S>(x);
  else if constexpr (R == 5) dft5<C, S>(x);
  else if constexpr (R == 8) dft8<C, S>(x);
  else if constexpr (R == 6) dft_comp<C, S, 6, 3, 2>(x);
  else if constexpr (R == 9) dft_comp<C, S, 9, 3, 3>(x);
  else if constexpr (R == 10) dft_comp<C, S, 10, 5, 2>(x);
  else if constexpr (R == 12) dft_comp<C, S, 12, 4, 3>(x);
  else if constexpr (R == 15) dft_comp<C, S, 15, 5, 3>(x);
  else dft_comp<C, S, 16, 4, 4>(x);
}

// one radix-R stage over `nlines` lines (line stride ls, element stride es)
template <typename C, int S, bool DIT, bool LINE_FAST, int R>
__device__ __forceinline__ void fft_stage(C* buf, int nlines, int ls, int es, int n, int L,
                                          const C* __restrict__ tws) {
  const int q = L / R;
  const int nbf = n / R;
  const int total = nlines * nbf;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int line, bf;
    if (LINE_FAST) { line = idx % nlines; bf = idx / nlines; }
    else { bf = idx % nbf; line = idx / nbf; }
    const int blk = bf / q, j = bf - blk * q;
    C* base = buf + line * ls + (blk * L + j) * es;
    C x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = base[m * q * es];
    if (DIT) {
      if (j) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          C w = tws[j * (R - 1) + m - 1];
          if (S > 0) w = cconj(w);
          x[m] = cmul(x[m], w);
        }
      }
      dftR<C, S, R>(x);
    } else {
      dftR<C, S, R>(x);
      if (j) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          C w = tws[j * (R - 1) + m - 1];
          if (S > 0) w = cconj(w);
          x[m] = cmul(x[m], w);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) base[m * q * es] = x[m];
  }
}

// full in-place transform of a batch of lines (any length of the form 2^a 3^b 5^c).  S = +1: inverse (DIF), S = -1:
// forward (DIT, stages reversed).  Ends with a block barrier.
template <typename C, int S, bool LINE_FAST>
__device__ void fft_lines_generic(C* buf, int nlines, int ls, int es, const FftDim& d, const C* __restrict__ tw) {
  constexpr bool DIT = (S < 0);
  for (int s0 = 0; s0 < d.nst; ++s0) {
    const int s = DIT ? (d.nst - 1 - s0) : s0;
    const C* tws = tw + d.tw_off[s];
    switch (d.radix[s]) {
      case 16: fft_stage<C, S, DIT, LINE_FAST, 16>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 15: fft_stage<C, S, DIT, LINE_FAST, 15>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 12: fft_stage<C, S, DIT, LINE_FAST, 12>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 10: fft_stage<C, S, DIT, LINE_FAST, 10>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 9: fft_stage<C, S, DIT, LINE_FAST, 9>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 8: fft_stage<C, S, DIT, LINE_FAST, 8>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 6: fft_stage<C, S, DIT, LINE_FAST, 6>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 5: fft_stage<C, S, DIT, LINE_FAST, 5>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 4: fft_stage<C, S, DIT, LINE_FAST, 4>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      case 3: fft_stage<C, S, DIT, LINE_FAST, 3>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
      default: fft_stage<C, S, DIT, LINE_FAST, 2>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
    }
    __syncthreads();
  }
}


// ---- the same transform with the length known at compile time --------------------
// The radix plan is the one the host builds (greedy 8, 4, 5, 3, 2), so the stage
// twiddle offsets in FftDim apply unchanged.  All index arithmetic is by
// compile-time constants; one barrier per stage.
template <typename C, int S, bool DIT, bool LINE_FAST, int LF, int N, int R, int L>
__device__ __forceinline__ void stage_c(C* buf, int nlines, int ls, int es, const C* __restrict__ tws) {
  constexpr int Q = L / R, NBF = N / R;
  const int total = LINE_FAST ? LF * NBF : nlines * NBF;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int line, bf;
    if (LINE_FAST) {
      line = idx % LF;
      bf = idx / LF;
      if (line >= nlines) continue;
    } else {
      bf = idx % NBF;
      line = idx / NBF;
    }
    const int blk = bf / Q, j = bf - blk * Q;
    C* base = buf + line * ls + (blk * L + j) * es;
    C x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = base[m * Q * es];
    if (DIT) {
      if (Q > 1 && j) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          C w = tws[j * (R - 1) + m - 1];
          if (S > 0) w = cconj(w);
          x[m] = cmul(x[m], w);
        }
      }
      dftR<C, S, R>(x);
    } else {
      dftR<C, S, R>(x);
      if (Q > 1 && j) {
#pragma unroll
        for (int m = 1; m < R; ++m) {
          C w = tws[j * (R - 1) + m - 1];
          if (S > 0) w = cconj(w);
          x[m] = cmul(x[m], w);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) base[m * Q * es] = x[m];
  }
}

template <typename C, int S, bool LINE_FAST, int LF, int N, int S0>
__device__ __forceinline__ void stages_c(C* buf, int nlines, int ls, int es, const C* __restrict__ tw,
                                         const FftDim& d) {
  constexpr CPlan P = make_cplan(N);
  if constexpr (S0 < P.nst) {
    constexpr bool DIT = (S < 0);
    constexpr int s = DIT ? P.nst - 1 - S0 : S0;
    stage_c<C, S, DIT, LINE_FAST, LF, N, P.radix[s], P.L[s]>(buf, nlines, ls, es, tw + d.tw_off[s]);
    __syncthreads();
    stages_c<C, S, LINE_FAST, LF, N, S0 + 1>(buf, nlines, ls, es, tw, d);
  }
}

template <typename C, int S, bool LINE_FAST, int LF, int N>
__device__ __noinline__ void fft_n(C* buf, int nlines, int ls, int es, const C* __restrict__ tw, FftDim d) {
  stages_c<C, S, LINE_FAST, LF, N, 0>(buf, nlines, ls, es, tw, d);
}

// dispatch: specialised lengths of the bundled workloads, generic otherwise.  Ends with a barrier.
template <typename C, int S, bool LINE_FAST, int LF = 1>
__device__ void fft_lines(C* buf, int nlines, int ls, int es, const FftDim& d, const C* __restrict__ tw) {
  if (!LINE_FAST || es == LF) {
    switch (d.n) {
      case 16: fft_n<C, S, LINE_FAST, LF, 16>(buf, nlines, ls, es, tw, d); return;
      case 18: fft_n<C, S, LINE_FAST, LF, 18>(buf, nlines, ls, es, tw, d); return;
      case 20: fft_n<C, S, LINE_FAST, LF, 20>(buf, nlines, ls, es, tw, d); return;
      case 24: fft_n<C, S, LINE_FAST, LF, 24>(buf, nlines, ls, es, tw, d); return;
      case 30: fft_n<C, S, LINE_FAST, LF, 30>(buf, nlines, ls, es, tw, d); return;
      case 64: fft_n<C, S, LINE_FAST, LF, 64>(buf, nlines, ls, es, tw, d); return;
      case 72: fft_n<C, S, LINE_FAST, LF, 72>(buf, nlines, ls, es, tw, d); return;
      case 90: fft_n<C, S, LINE_FAST, LF, 90>(buf, nlines, ls, es, tw, d); return;
      case 96: fft_n<C, S, LINE_FAST, LF, 96>(buf, nlines, ls, es, tw, d); return;
      case 120: fft_n<C, S, LINE_FAST, LF, 120>(buf, nlines, ls, es, tw, d); return;
      default: break;
    }
  }
  fft_lines_generic<C, S, LINE_FAST>(buf, nlines, ls, es, d, tw);
}

__device__ __forceinline__ int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
// (s + d) mod N for 0 <= s, d < N: one conditional subtraction (the gathers step l0 + idx
// by 32 as wrap_n<N3>(l, 32 % N3) instead of a division each)
template <int N> __device__ __forceinline__ int wrap_n(int s, int d) { const int v = s + d; return v >= N ? v - N : v; }

// ---- line-group engine: each line is transformed by a group of TL threads of one warp
// (TL a power of two dividing the butterfly count of every stage), butterflies of a
// stage spread over the group, stages separated by __syncwarp only.  Same radix plan,
// twiddle table and digit-reversed ordering as the block-wide stages above.
constexpr int cgcd(int a, int b) { return b ? cgcd(b, a % b) : a; }
template <int N> struct LineCfg {
  static constexpr CPlan P = make_cplan(N);
  static constexpr int g01 = P.nst >= 2 ? cgcd(N / P.radix[0], N / P.radix[1]) : N / P.radix[0];
  static constexpr int g = P.nst >= 3 ? cgcd(g01, N / P.radix[2]) : g01;
  static constexpr int TL = (g % 8 == 0) ? 8 : (g % 4 == 0) ? 4 : (g % 2 == 0) ? 2 : 1;
  static constexpr int NP = N + ((TL - N) % 16 + 16) % 16;  // padded line pitch (bank spread)
  static constexpr int LPC = 64;                           // lines per CTA
  static constexpr int THREADS = LPC * TL;
};

// twt: this dimension's twiddle table (stage s at twt + tw_off[s] - tw_base), normally a
// shared-memory copy.  mask: lanes of the warp taking part (all lanes of active groups).
template <typename C, int S, int N, int TL, int S0>
__device__ __forceinline__ void line_stages(C* line, int t, const C* twt, const FftDim& d, unsigned mask) {
  constexpr CPlan P = make_cplan(N);
  if constexpr (S0 < P.nst) {
    constexpr bool DIT = (S < 0);
    constexpr int s = DIT ? P.nst - 1 - S0 : S0;
    constexpr int R = P.radix[s], L = P.L[s], Q = L / R, NB = N / R;
    static_assert(NB % TL == 0, "butterflies must split evenly over the line group");
    const C* tws = twt + (d.tw_off[s] - d.tw_base);
#pragma unroll
    for (int i = 0; i < NB / TL; ++i) {
      const int bf = t + TL * i;
      const int blk = bf / Q, j = bf - blk * Q;
      C* base = line + blk * L + j;
      C x[R];
#pragma unroll
      for (int m = 0; m < R; ++m) x[m] = base[m * Q];
      if (DIT) {
        if (Q > 1 && j) {
#pragma unroll
          for (int m = 1; m < R; ++m) {
            C w = tws[j * (R - 1) + m - 1];
            if (S > 0) w = cconj(w);
            x[m] = cmul(x[m], w);
          }
        }
        dftR<C, S, R>(x);
      } else {
        dftR<C, S, R>(x);
        if (Q > 1 && j) {
#pragma unroll
          for (int m = 1; m < R; ++m) {
            C w = tws[j * (R - 1) + m - 1];
            if (S > 0) w = cconj(w);
            x[m] = cmul(x[m], w);
          }
        }
      }
#pragma unroll
      for (int m = 0; m < R; ++m) base[m * Q] = x[m];
    }
    __syncwarp(mask);
    line_stages<C, S, N, TL, S0 + 1>(line, t, twt, d, mask);
  }
}

// copy one dimension's twiddles to shared memory (caller synchronises)
template <typename C>
__device__ __forceinline__ void load_tw(C* dst, const C* __restrict__ tw, const FftDim& d) {
  for (int i = threadIdx.x; i < d.tw_count; i += blockDim.x) dst[i] = tw[d.tw_base + i];
}

// Transform `nlines` lines (line k at buf + k * pitch, unit element stride) with groups of
// TL threads; all threads of the block call this (it contains no block barrier).
template <typename C, int S, int N, int TL>
__device__ __forceinline__ void lines_lg(C* buf, int pitch, int nlines, const C* twt, const FftDim& d) {
  const int g = threadIdx.x / TL, t = threadIdx.x % TL, ng = blockDim.x / TL;
  for (int k0 = 0; k0 < nlines; k0 += ng) {
    const int k = k0 + g;
    const unsigned mask = __ballot_sync(0xffffffffu, k < nlines);
    if (k < nlines) line_stages<C, S, N, TL, 0>(buf + k * pitch, t, twt, d, mask);
  }
}

// x-line pass with the line-group engine: inverse x (DIF), times V / n1n2n3 at the
// digit-reversed positions, forward x (DIT); only the sphere planes are read and written.
template <typename T, int N1>
__global__ void __launch_bounds__(LineCfg<N1>::THREADS) k_xline_lg(cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                                   const T* __restrict__ vperm, SphereDev sp,
                                                                   FftPlan plan, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using LC = LineCfg<N1>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);  // [LPC][NP]
  C* twt = X + LC::LPC * LC::NP;
  const int nyz = plan.n[1] * plan.n[2];
  const int yz0 = blockIdx.x * LC::LPC, b = blockIdx.y;
  const int ln = min(LC::LPC, nyz - yz0);
  for (int i = threadIdx.x; i < LC::LPC * LC::NP; i += blockDim.x) X[i] = czero<C>();
  load_tw(twt, tw, plan.d[0]);
  __syncthreads();
  C* base = hb + (int64_t)b * hb_bs;
  for (int i = threadIdx.x; i < sp.nplane * ln; i += blockDim.x) {
    const int p = i / ln, l = i - p * ln;
    X[l * LC::NP + pmod(sp.plane_h[p], N1)] = base[(int64_t)p * nyz + yz0 + l];
  }
  __syncthreads();
  const int l = threadIdx.x / LC::TL, t = threadIdx.x % LC::TL;
  C* line = X + l * LC::NP;
  line_stages<C, +1, N1, LC::TL, 0>(line, t, twt, plan.d[0], 0xffffffffu);
  if (l < ln) {
#pragma unroll 4
    for (int m = t; m < N1; m += LC::TL) line[m] = cscale(line[m], vperm[(int64_t)m * nyz + yz0 + l]);
  }
  __syncwarp();
  line_stages<C, -1, N1, LC::TL, 0>(line, t, twt, plan.d[0], 0xffffffffu);
  __syncthreads();
  for (int i = threadIdx.x; i < sp.nplane * ln; i += blockDim.x) {
    const int p = i / ln, l2 = i - p * ln;
    base[(int64_t)p * nyz + yz0 + l2] = X[l2 * LC::NP + pmod(sp.plane_h[p], N1)];
  }
}

// x-line pass fused in registers (2-stage plans N1 = R1 R2): the first inverse stage
// reads the sphere planes straight from the half-box buffer, the last inverse stage,
// the V multiply and the first forward stage share registers, and the last forward
// stage writes only the sphere planes back.  Shared memory holds each line once
// between stages (two exchanges per line instead of a full staging per stage).
template <typename T, int N1>
__global__ void __launch_bounds__(LineCfg<N1>::THREADS) k_xline_fused(cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                                      const T* __restrict__ vperm, SphereDev sp,
                                                                      FftPlan plan,
                                                                      const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using LC = LineCfg<N1>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  constexpr int R1 = P.radix[0], R2 = P.radix[1], Q1 = R2;  // stage 1: L = N1, stride R2
  constexpr int TL = LC::TL, NB1 = N1 / R1, NB2 = N1 / R2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);  // [LPC][NP]
  C* twt = X + LC::LPC * LC::NP;
  const int nyz = plan.n[1] * plan.n[2];
  const int yz0 = blockIdx.x * LC::LPC, b = blockIdx.y;
  const int ln = min(LC::LPC, nyz - yz0);
  // The x-line operation (inverse DFT, times V, forward DFT) is a convolution in x-frequency
  // and so commutes with a shift of the frequencies: plane p (Miller index h0 + p) is placed
  // at frequency p instead of h0 + p, and output p is again plane p.
  const int np = sp.nplane;
  auto pidx = [&](int x) { return x < np ? x : -1; };
  load_tw(twt, tw, plan.d[0]);
  __syncthreads();
  const C* tw1 = twt + (plan.d[0].tw_off[0] - plan.d[0].tw_base);
  const int l = threadIdx.x / TL, t = threadIdx.x % TL;
  const bool live = l < ln;
  C* line = X + l * LC::NP;
  C* hbb = hb + (int64_t)b * hb_bs + yz0 + l;
  // stage 1 of the inverse transform (DIF radix R1, stride Q1): inputs from the planes
#pragma unroll
  for (int i = 0; i < NB1 / TL; ++i) {
    const int j = t + TL * i;
    C x[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int p = pidx(j + Q1 * a);
      x[a] = (live && p >= 0) ? hbb[(int64_t)p * nyz] : czero<C>();
    }
    dftR<C, +1, R1>(x);
    if (j) {
#pragma unroll
      for (int m = 1; m < R1; ++m) x[m] = cmul(x[m], cconj(tw1[j * (R1 - 1) + m - 1]));
    }
#pragma unroll
    for (int m = 0; m < R1; ++m) line[j + Q1 * m] = x[m];
  }
  __syncwarp();
  // stage 2 inverse (radix R2 on contiguous blocks), times V at the digit-reversed
  // positions, stage 2 forward (DIT: first stage, no twiddles since its block length is R2)
  const T* vb = vperm + yz0 + l;
#pragma unroll
  for (int i = 0; i < NB2 / TL; ++i) {
    const int blk = t + TL * i;
    C x[R2];
#pragma unroll
    for (int m = 0; m < R2; ++m) x[m] = line[blk * R2 + m];
    dftR<C, +1, R2>(x);
#pragma unroll
    for (int m = 0; m < R2; ++m) x[m] = cscale(x[m], live ? vb[(int64_t)(blk * R2 + m) * nyz] : (T)0);
    dftR<C, -1, R2>(x);
#pragma unroll
    for (int m = 0; m < R2; ++m) line[blk * R2 + m] = x[m];
  }
  __syncwarp();
  // stage 1 forward (DIT radix R1): twiddles, DFT, write the sphere planes
#pragma unroll
  for (int i = 0; i < NB1 / TL; ++i) {
    const int j = t + TL * i;
    C x[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) x[m] = line[j + Q1 * m];
    if (j) {
#pragma unroll
      for (int m = 1; m < R1; ++m) x[m] = cmul(x[m], tw1[j * (R1 - 1) + m - 1]);
    }
    dftR<C, -1, R1>(x);
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int p = pidx(j + Q1 * a);
      if (live && p >= 0) hbb[(int64_t)p * nyz] = x[a];
    }
  }
}

template <typename T, int N1>
static cudaError_t launch_xline_fused(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp,
                                      const FftPlan& plan, const cplx<T>* tw, int nb, cudaStream_t st) {
  using LC = LineCfg<N1>;
  const size_t sm = sizeof(cplx<T>) * ((size_t)LC::LPC * LC::NP + plan.d[0].tw_count);
  cudaError_t e = cudaFuncSetAttribute(k_xline_fused<T, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  const int nyz = plan.n[1] * plan.n[2];
  k_xline_fused<T, N1><<<dim3((nyz + LC::LPC - 1) / LC::LPC, nb), LC::THREADS, sm, st>>>(hb, hb_bs, vperm, sp, plan, tw); count_launch();
  return cudaGetLastError();
}

template <typename T, int N1>
static cudaError_t launch_xline_lg(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp,
                                   const FftPlan& plan, const cplx<T>* tw, int nb, cudaStream_t st) {
  using LC = LineCfg<N1>;
  const size_t sm = sizeof(cplx<T>) * ((size_t)LC::LPC * LC::NP + plan.d[0].tw_count);
  cudaError_t e = cudaFuncSetAttribute(k_xline_lg<T, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  const int nyz = plan.n[1] * plan.n[2];
  k_xline_lg<T, N1><<<dim3((nyz + LC::LPC - 1) / LC::LPC, nb), LC::THREADS, sm, st>>>(hb, hb_bs, vperm, sp, plan, tw); count_launch();
  return cudaGetLastError();
}

// returns cudaErrorNotSupported when n1 has no line-group instantiation
template <typename T>
static cudaError_t xline_lg(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp, const FftPlan& plan,
                            const cplx<T>* tw, int nb, cudaStream_t st) {
  switch (plan.n[0]) {
    case 24: return launch_xline_fused<T, 24>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    case 64: return launch_xline_fused<T, 64>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    case 72: return launch_xline_fused<T, 72>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    case 90: return launch_xline_fused<T, 90>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    case 96: return launch_xline_fused<T, 96>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    case 120: return launch_xline_fused<T, 120>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    default: return cudaErrorNotSupported;
  }
}


constexpr int kThreads = 256;

// ---- pass 1: sphere plane -> inverse (z, y) -> half-box plane ---------------------
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_plane_inv(const cplx<T>* __restrict__ psi, int64_t ldpsi,
                                                        cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                        SphereDev sp, FftPlan plan,
                                                        const cplx<T>* __restrict__ tw, int cz) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  const int n2 = plan.n[1], n3 = plan.n[2], n2p = n2 + 1;
  C* Wb = R + sp.max_rows * n3;
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* src = psi + (int64_t)b * ldpsi;
  for (int i = threadIdx.x; i < nr * n3; i += blockDim.x) R[i] = czero<C>();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = warp; row < nr; row += nw) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    for (int t = lane; t < cnt; t += 32) R[row * n3 + pmod(l0 + t, n3)] = src[g0 + t];
  }
  __syncthreads();
  fft_lines<C, +1, false>(R, nr, n3, 1, plan.d[2], tw);
  C* dst = hb + (int64_t)b * hb_bs + (int64_t)p * n2 * n3;
  for (int zc0 = 0; zc0 < n3; zc0 += cz) {
    const int czn = min(cz, n3 - zc0);
    for (int i = threadIdx.x; i < czn * n2p; i += blockDim.x) Wb[i] = czero<C>();
    __syncthreads();
    for (int i = threadIdx.x; i < nr * czn; i += blockDim.x) {
      const int row = i / czn, zc = i - row * czn;
      Wb[zc * n2p + pmod(sp.row_k[r0 + row], n2)] = R[row * n3 + zc0 + zc];
    }
    __syncthreads();
    fft_lines<C, +1, false>(Wb, czn, n2p, 1, plan.d[1], tw);
    for (int i = threadIdx.x; i < n2 * czn; i += blockDim.x) {
      const int y = i / czn, zc = i - y * czn;
      dst[(int64_t)y * n3 + zc0 + zc] = Wb[zc * n2p + y];
    }
    __syncthreads();
  }
}

// ---- pass 2: x-lines: inverse x, times V, forward x ---------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_xline(cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                    const T* __restrict__ vperm, SphereDev sp,
                                                    FftPlan plan, const cplx<T>* __restrict__ tw, int lyz) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);  // [n1][lyz]
  const int n1 = plan.n[0], nyz = plan.n[1] * plan.n[2];
  const int yz0 = blockIdx.x * lyz, b = blockIdx.y;
  const int ln = min(lyz, nyz - yz0);
  for (int i = threadIdx.x; i < n1 * lyz; i += blockDim.x) X[i] = czero<C>();
  __syncthreads();
  C* base = hb + (int64_t)b * hb_bs;
  for (int i = threadIdx.x; i < sp.nplane * ln; i += blockDim.x) {
    const int p = i / ln, l = i - p * ln;
    X[pmod(sp.plane_h[p], n1) * lyz + l] = base[(int64_t)p * nyz + yz0 + l];
  }
  __syncthreads();
  fft_lines<C, +1, true, 32>(X, ln, 1, lyz, plan.d[0], tw);
  for (int i = threadIdx.x; i < n1 * ln; i += blockDim.x) {
    const int x = i / ln, l = i - x * ln;
    X[x * lyz + l] = cscale(X[x * lyz + l], vperm[(int64_t)x * nyz + yz0 + l]);
  }
  __syncthreads();
  fft_lines<C, -1, true, 32>(X, ln, 1, lyz, plan.d[0], tw);
  for (int i = threadIdx.x; i < sp.nplane * ln; i += blockDim.x) {
    const int p = i / ln, l = i - p * ln;
    base[(int64_t)p * nyz + yz0 + l] = X[pmod(sp.plane_h[p], n1) * lyz + l];
  }
}

// ---- pass 3: half-box plane -> forward (y, z) -> sphere, + kinetic ------------------
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_plane_fwd(const cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                        SphereDev sp, FftPlan plan,
                                                        const cplx<T>* __restrict__ tw, int cz,
                                                        const T* __restrict__ kin,
                                                        const cplx<T>* __restrict__ psi, int64_t ldpsi,
                                                        cplx<T>* __restrict__ out, int64_t ldout) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  const int n2 = plan.n[1], n3 = plan.n[2], n2p = n2 + 1;
  C* Wb = R + sp.max_rows * n3;
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* srcp = hb + (int64_t)b * hb_bs + (int64_t)p * n2 * n3;
  for (int zc0 = 0; zc0 < n3; zc0 += cz) {
    const int czn = min(cz, n3 - zc0);
    for (int i = threadIdx.x; i < n2 * czn; i += blockDim.x) {
      const int y = i / czn, zc = i - y * czn;
      Wb[zc * n2p + y] = srcp[(int64_t)y * n3 + zc0 + zc];
    }
    __syncthreads();
    fft_lines<C, -1, false>(Wb, czn, n2p, 1, plan.d[1], tw);
    for (int i = threadIdx.x; i < nr * czn; i += blockDim.x) {
      const int row = i / czn, zc = i - row * czn;
      R[row * n3 + zc0 + zc] = Wb[zc * n2p + pmod(sp.row_k[r0 + row], n2)];
    }
    __syncthreads();
  }
  fft_lines<C, -1, false>(R, nr, n3, 1, plan.d[2], tw);
  const C* y = psi + (int64_t)b * ldpsi;
  C* o = out + (int64_t)b * ldout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = warp; row < nr; row += nw) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    for (int t = lane; t < cnt; t += 32) {
      const int g = g0 + t;
      const C v = R[row * n3 + pmod(l0 + t, n3)];
      const C yy = y[g];
      const T k = kin[g];
      o[g] = mk<C>(k * yy.x + v.x, k * yy.y + v.y);
    }
  }
}

// ---- density: inverse x-lines for a and b, accumulate w Re(conj(a) b) ---------------
template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_xline_density(const cplx<T>* __restrict__ hba,
                                                            const cplx<T>* __restrict__ hbb, int64_t hb_bs,
                                                            int nb, const T* __restrict__ w, SphereDev sp,
                                                            FftPlan plan, const cplx<T>* __restrict__ tw,
                                                            int lyz, double* __restrict__ out_perm) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* X = reinterpret_cast<C*>(smem_raw);  // [n1][lyz]
  C* Y = X + plan.n[0] * lyz;
  const int n1 = plan.n[0], nyz = plan.n[1] * plan.n[2];
  const int yz0 = blockIdx.x * lyz;
  const int ln = min(lyz, nyz - yz0);
  const bool two = (hbb != nullptr);
  // per-thread accumulators for the points this thread owns: i = tid + k*blockDim
  double acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.0;
  for (int b = 0; b < nb; ++b) {
    for (int i = threadIdx.x; i < n1 * lyz; i += blockDim.x) {
      X[i] = czero<C>();
      if (two) Y[i] = czero<C>();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sp.nplane * ln; i += blockDim.x) {
      const int p = i / ln, l = i - p * ln;
      const int64_t off = (int64_t)b * hb_bs + (int64_t)p * nyz + yz0 + l;
      X[pmod(sp.plane_h[p], n1) * lyz + l] = hba[off];
      if (two) Y[pmod(sp.plane_h[p], n1) * lyz + l] = hbb[off];
    }
    __syncthreads();
    fft_lines<C, +1, true, 8>(X, ln, 1, lyz, plan.d[0], tw);
    if (two) fft_lines<C, +1, true, 8>(Y, ln, 1, lyz, plan.d[0], tw);
    const C* Bv = two ? Y : X;
    const double wb = (double)w[b];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      if (i < n1 * ln) {
        const int x = i / ln, l = i - x * ln;
        const C av = X[x * lyz + l], bv = Bv[x * lyz + l];
        acc[k] += wb * ((double)av.x * (double)bv.x + (double)av.y * (double)bv.y);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = threadIdx.x + k * blockDim.x;
    if (i < n1 * ln) {
      const int x = i / ln, l = i - x * ln;
      out_perm[(int64_t)x * nyz + yz0 + l] += acc[k];
    }
  }
}

// ---- plane passes with the line-group engine ------------------------------------
template <typename T> struct PlaneCh { static constexpr int v = (sizeof(T) == 4) ? 64 : 32; };

template <typename T, int N2, int N3>
__global__ void __launch_bounds__(256) k_plane_inv_lg(const cplx<T>* __restrict__ psi, int64_t ldpsi,
                                                      cplx<T>* __restrict__ hb, int64_t hb_bs, SphereDev sp,
                                                      FftPlan plan, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int NP2 = LineCfg<N2>::NP, NP3 = LineCfg<N3>::NP, CH = PlaneCh<T>::v;
  constexpr int TL2 = LineCfg<N2>::TL, TL3 = LineCfg<N3>::TL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);  // [max_rows][NP3]
  C* W = R + sp.max_rows * NP3;           // [CH][NP2]
  C* tw2 = W + CH * NP2;
  C* tw3 = tw2 + plan.d[1].tw_count;
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* src = psi + (int64_t)b * ldpsi;
  for (int i = threadIdx.x; i < nr * NP3; i += blockDim.x) R[i] = czero<C>();
  load_tw(tw2, tw, plan.d[1]);
  load_tw(tw3, tw, plan.d[2]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = warp; row < nr; row += nw) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    for (int t = lane; t < cnt; t += 32) R[row * NP3 + pmod(l0 + t, N3)] = src[g0 + t];
  }
  __syncthreads();
  lines_lg<C, +1, N3, TL3>(R, NP3, nr, tw3, plan.d[2]);
  __syncthreads();
  C* dst = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  for (int zc0 = 0; zc0 < N3; zc0 += CH) {
    const int czn = min(CH, N3 - zc0);
    for (int i = threadIdx.x; i < czn * NP2; i += blockDim.x) W[i] = czero<C>();
    __syncthreads();
    for (int i = threadIdx.x; i < nr * czn; i += blockDim.x) {
      const int row = i / czn, zc = i - row * czn;
      W[zc * NP2 + pmod(sp.row_k[r0 + row], N2)] = R[row * NP3 + zc0 + zc];
    }
    __syncthreads();
    lines_lg<C, +1, N2, TL2>(W, NP2, czn, tw2, plan.d[1]);
    __syncthreads();
    for (int i = threadIdx.x; i < N2 * czn; i += blockDim.x) {
      const int y = i / czn, zc = i - y * czn;
      dst[(int64_t)y * N3 + zc0 + zc] = W[zc * NP2 + y];
    }
    __syncthreads();
  }
}

template <typename T, int N2, int N3>
__global__ void __launch_bounds__(256) k_plane_fwd_lg(const cplx<T>* __restrict__ hb, int64_t hb_bs, SphereDev sp,
                                                      FftPlan plan, const cplx<T>* __restrict__ tw,
                                                      const T* __restrict__ kin, const cplx<T>* __restrict__ psi,
                                                      int64_t ldpsi, cplx<T>* __restrict__ out, int64_t ldout) {
  using C = cplx<T>;
  constexpr int NP2 = LineCfg<N2>::NP, NP3 = LineCfg<N3>::NP, CH = PlaneCh<T>::v;
  constexpr int TL2 = LineCfg<N2>::TL, TL3 = LineCfg<N3>::TL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  C* W = R + sp.max_rows * NP3;
  C* tw2 = W + CH * NP2;
  C* tw3 = tw2 + plan.d[1].tw_count;
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* srcp = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  load_tw(tw2, tw, plan.d[1]);
  load_tw(tw3, tw, plan.d[2]);
  for (int zc0 = 0; zc0 < N3; zc0 += CH) {
    const int czn = min(CH, N3 - zc0);
    for (int i = threadIdx.x; i < N2 * czn; i += blockDim.x) {
      const int y = i / czn, zc = i - y * czn;
      W[zc * NP2 + y] = srcp[(int64_t)y * N3 + zc0 + zc];
    }
    __syncthreads();
    lines_lg<C, -1, N2, TL2>(W, NP2, czn, tw2, plan.d[1]);
    __syncthreads();
    for (int i = threadIdx.x; i < nr * czn; i += blockDim.x) {
      const int row = i / czn, zc = i - row * czn;
      R[row * NP3 + zc0 + zc] = W[zc * NP2 + pmod(sp.row_k[r0 + row], N2)];
    }
    __syncthreads();
  }
  lines_lg<C, -1, N3, TL3>(R, NP3, nr, tw3, plan.d[2]);
  __syncthreads();
  const C* y = psi + (int64_t)b * ldpsi;
  C* o = out + (int64_t)b * ldout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = warp; row < nr; row += nw) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    for (int t = lane; t < cnt; t += 32) {
      const int g = g0 + t;
      const C v = R[row * NP3 + pmod(l0 + t, N3)];
      const C yy = y[g];
      const T k = kin[g];
      o[g] = mk<C>(k * yy.x + v.x, k * yy.y + v.y);
    }
  }
}

// ---- plane passes fused in registers (2-stage plans for n2 and n3) -----------------
// Pass 1: z-lines read their run of sphere coefficients straight into the first stage,
// y-lines read the transformed rows straight from shared memory (zeros elsewhere) and the
// last y stage writes the half-box plane.  Pass 3 mirrors it: the first y stage reads
// the half-box plane, the last y stage fills only the rows holding coefficients, and the
// last z stage gathers the sphere coefficients with the kinetic term.
constexpr int kYGroups = 64;  // y-lines in flight per CTA

template <typename T, int N2, int N3> struct PlaneF {
  static constexpr CPlan P2 = make_cplan(N2), P3 = make_cplan(N3);
  static constexpr int TL2 = LineCfg<N2>::TL, TL3 = LineCfg<N3>::TL;
  static constexpr int NP2 = LineCfg<N2>::NP, NP3 = LineCfg<N3>::NP;
  static constexpr bool ok = (P2.nst == 2 && P3.nst == 2);
};

template <typename T, int N2, int N3>
__global__ void __launch_bounds__(256) k_plane_inv_f(const cplx<T>* __restrict__ psi, int64_t ldpsi,
                                                     cplx<T>* __restrict__ hb, int64_t hb_bs, SphereDev sp,
                                                     FftPlan plan, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using PF = PlaneF<T, N2, N3>;
  constexpr int TL2 = PF::TL2, TL3 = PF::TL3, NP2 = PF::NP2, NP3 = PF::NP3;
  constexpr int Z1 = PF::P3.radix[0], Z2 = PF::P3.radix[1];  // z stages: radix Z1 stride Z2, then blocks of Z2
  constexpr int Y1 = PF::P2.radix[0], Y2 = PF::P2.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);        // [max_rows][NP3]
  C* Wl = R + sp.max_rows * NP3;                // [kYGroups][NP2]
  C* tw2 = Wl + kYGroups * NP2;
  C* tw3 = tw2 + plan.d[1].tw_count;
  int* ymap = reinterpret_cast<int*>(tw3 + plan.d[2].tw_count);  // y -> row or -1
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* src = psi + (int64_t)b * ldpsi;
  load_tw(tw2, tw, plan.d[1]);
  load_tw(tw3, tw, plan.d[2]);
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  const C* tz1 = tw3 + (plan.d[2].tw_off[0] - plan.d[2].tw_base);
  const C* ty1 = tw2 + (plan.d[1].tw_off[0] - plan.d[1].tw_base);
  // z-lines: one row per group of TL3 threads
  {
    const int g = threadIdx.x / TL3, t = threadIdx.x % TL3, ng = blockDim.x / TL3;
    for (int r00 = 0; r00 < nr; r00 += ng) {
      const int row = r00 + g;
      const bool has = row < nr;
      const unsigned mask = __ballot_sync(0xffffffffu, has);
      if (has) {
        const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
        C* line = R + row * NP3;
#pragma unroll
        for (int i = 0; i < (N3 / Z1) / TL3; ++i) {
          const int j = t + TL3 * i;
          C x[Z1];
#pragma unroll
          for (int a = 0; a < Z1; ++a) {
            const int idx = pmod(j + Z2 * a - l0, N3);
            x[a] = idx < cnt ? src[g0 + idx] : czero<C>();
          }
          dftR<C, +1, Z1>(x);
          if (j) {
#pragma unroll
            for (int m = 1; m < Z1; ++m) x[m] = cmul(x[m], cconj(tz1[j * (Z1 - 1) + m - 1]));
          }
#pragma unroll
          for (int m = 0; m < Z1; ++m) line[j + Z2 * m] = x[m];
        }
        __syncwarp(mask);
#pragma unroll
        for (int i = 0; i < (N3 / Z2) / TL3; ++i) {
          const int blk = t + TL3 * i;
          C x[Z2];
#pragma unroll
          for (int m = 0; m < Z2; ++m) x[m] = line[blk * Z2 + m];
          dftR<C, +1, Z2>(x);
#pragma unroll
          for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = x[m];
        }
      }
    }
  }
  __syncthreads();
  // y-lines: one column per group of TL2 threads, up to kYGroups columns per wave (fewer
  // when the block has fewer groups, e.g. 32 groups of 8 threads)
  C* dst = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  {
    const int g = threadIdx.x / TL2, t = threadIdx.x % TL2;
    const int wave = min(kYGroups, (int)blockDim.x / TL2);
    const bool in_wave = g < wave;
    C* line = Wl + g * NP2;
    for (int c0 = 0; c0 < N3; c0 += wave) {
      const int col = c0 + g;
      const bool has = in_wave && col < N3;
      const unsigned mask = __ballot_sync(0xffffffffu, has);
      if (has) {
#pragma unroll
        for (int i = 0; i < (N2 / Y1) / TL2; ++i) {
          const int j = t + TL2 * i;
          C x[Y1];
#pragma unroll
          for (int a = 0; a < Y1; ++a) {
            const int r = ymap[j + Y2 * a];
            x[a] = r >= 0 ? R[r * NP3 + col] : czero<C>();
          }
          dftR<C, +1, Y1>(x);
          if (j) {
#pragma unroll
            for (int m = 1; m < Y1; ++m) x[m] = cmul(x[m], cconj(ty1[j * (Y1 - 1) + m - 1]));
          }
#pragma unroll
          for (int m = 0; m < Y1; ++m) line[j + Y2 * m] = x[m];
        }
        __syncwarp(mask);
#pragma unroll
        for (int i = 0; i < (N2 / Y2) / TL2; ++i) {
          const int blk = t + TL2 * i;
          C x[Y2];
#pragma unroll
          for (int m = 0; m < Y2; ++m) x[m] = line[blk * Y2 + m];
          dftR<C, +1, Y2>(x);
#pragma unroll
          for (int m = 0; m < Y2; ++m) dst[(int64_t)(blk * Y2 + m) * N3 + col] = x[m];
        }
        __syncwarp(mask);
      }
    }
  }
}

template <typename T, int N2, int N3>
__global__ void __launch_bounds__(256) k_plane_fwd_f(const cplx<T>* __restrict__ hb, int64_t hb_bs, SphereDev sp,
                                                     FftPlan plan, const cplx<T>* __restrict__ tw,
                                                     const T* __restrict__ kin, const cplx<T>* __restrict__ psi,
                                                     int64_t ldpsi, cplx<T>* __restrict__ out, int64_t ldout) {
  using C = cplx<T>;
  using PF = PlaneF<T, N2, N3>;
  constexpr int TL2 = PF::TL2, TL3 = PF::TL3, NP2 = PF::NP2, NP3 = PF::NP3;
  constexpr int Z1 = PF::P3.radix[0], Z2 = PF::P3.radix[1];
  constexpr int Y1 = PF::P2.radix[0], Y2 = PF::P2.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  C* Wl = R + sp.max_rows * NP3;
  C* tw2 = Wl + kYGroups * NP2;
  C* tw3 = tw2 + plan.d[1].tw_count;
  int* ymap = reinterpret_cast<int*>(tw3 + plan.d[2].tw_count);
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* srcp = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  load_tw(tw2, tw, plan.d[1]);
  load_tw(tw3, tw, plan.d[2]);
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  __syncthreads();
  const C* tz1 = tw3 + (plan.d[2].tw_off[0] - plan.d[2].tw_base);
  const C* ty1 = tw2 + (plan.d[1].tw_off[0] - plan.d[1].tw_base);
  // y-lines (forward DIT: blocks of Y2 first, read from the half-box plane)
  {
    const int g = threadIdx.x / TL2, t = threadIdx.x % TL2;
    const int wave = min(kYGroups, (int)blockDim.x / TL2);
    const bool in_wave = g < wave;
    C* line = Wl + g * NP2;
    for (int c0 = 0; c0 < N3; c0 += wave) {
      const int col = c0 + g;
      const bool has = in_wave && col < N3;
      const unsigned mask = __ballot_sync(0xffffffffu, has);
      if (has) {
#pragma unroll
        for (int i = 0; i < (N2 / Y2) / TL2; ++i) {
          const int blk = t + TL2 * i;
          C x[Y2];
#pragma unroll
          for (int m = 0; m < Y2; ++m) x[m] = srcp[(int64_t)(blk * Y2 + m) * N3 + col];
          dftR<C, -1, Y2>(x);
#pragma unroll
          for (int m = 0; m < Y2; ++m) line[blk * Y2 + m] = x[m];
        }
        __syncwarp(mask);
#pragma unroll
        for (int i = 0; i < (N2 / Y1) / TL2; ++i) {
          const int j = t + TL2 * i;
          C x[Y1];
#pragma unroll
          for (int m = 0; m < Y1; ++m) x[m] = line[j + Y2 * m];
          if (j) {
#pragma unroll
            for (int m = 1; m < Y1; ++m) x[m] = cmul(x[m], ty1[j * (Y1 - 1) + m - 1]);
          }
          dftR<C, -1, Y1>(x);
#pragma unroll
          for (int a = 0; a < Y1; ++a) {
            const int r = ymap[j + Y2 * a];
            if (r >= 0) R[r * NP3 + col] = x[a];
          }
        }
        __syncwarp(mask);
      }
    }
  }
  __syncthreads();
  // z-lines: blocks of Z2 in place, then the radix-Z1 stage straight to the sphere
  const C* yv = psi + (int64_t)b * ldpsi;
  C* o = out + (int64_t)b * ldout;
  {
    const int g = threadIdx.x / TL3, t = threadIdx.x % TL3, ng = blockDim.x / TL3;
    for (int r00 = 0; r00 < nr; r00 += ng) {
      const int row = r00 + g;
      const bool has = row < nr;
      const unsigned mask = __ballot_sync(0xffffffffu, has);
      if (has) {
        C* line = R + row * NP3;
#pragma unroll
        for (int i = 0; i < (N3 / Z2) / TL3; ++i) {
          const int blk = t + TL3 * i;
          C x[Z2];
#pragma unroll
          for (int m = 0; m < Z2; ++m) x[m] = line[blk * Z2 + m];
          dftR<C, -1, Z2>(x);
#pragma unroll
          for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = x[m];
        }
        __syncwarp(mask);
        const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
#pragma unroll
        for (int i = 0; i < (N3 / Z1) / TL3; ++i) {
          const int j = t + TL3 * i;
          C x[Z1];
#pragma unroll
          for (int m = 0; m < Z1; ++m) x[m] = line[j + Z2 * m];
          if (j) {
#pragma unroll
            for (int m = 1; m < Z1; ++m) x[m] = cmul(x[m], tz1[j * (Z1 - 1) + m - 1]);
          }
          dftR<C, -1, Z1>(x);
#pragma unroll
          for (int a = 0; a < Z1; ++a) {
            const int idx = pmod(j + Z2 * a - l0, N3);
            if (idx < cnt) {
              const int gg = g0 + idx;
              const C yy = yv[gg];
              const T k = kin[gg];
              o[gg] = mk<C>(k * yy.x + x[a].x, k * yy.y + x[a].y);
            }
          }
        }
      }
    }
  }
}

template <typename T, int N2, int N3>
static size_t plane_f_smem(const SphereDev& sp, const FftPlan& plan) {
  using PF = PlaneF<T, N2, N3>;
  return sizeof(cplx<T>) * ((size_t)sp.max_rows * PF::NP3 + (size_t)kYGroups * PF::NP2 + plan.d[1].tw_count +
                            plan.d[2].tw_count) + sizeof(int) * N2;
}

template <typename T, int N2, int N3>
static size_t plane_lg_smem(const SphereDev& sp, const FftPlan& plan) {
  return sizeof(cplx<T>) * ((size_t)sp.max_rows * LineCfg<N3>::NP + (size_t)PlaneCh<T>::v * LineCfg<N2>::NP +
                            plan.d[1].tw_count + plan.d[2].tw_count);
}

template <typename T, int N2, int N3>
static cudaError_t plane_lg_pair(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                                 const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, const T* kin,
                                 cplx<T>* out, int64_t ldout, int nb, cudaStream_t st) {
  cudaError_t e;
  if constexpr (PlaneF<T, N2, N3>::ok) {
    const size_t smf = plane_f_smem<T, N2, N3>(sp, plan);
    if (smf <= 227 * 1024) {
      if (which == 0) {
        if ((e = cudaFuncSetAttribute(k_plane_inv_f<T, N2, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smf)))
          return e;
        k_plane_inv_f<T, N2, N3><<<dim3(sp.nplane, nb), 256, smf, st>>>(psi, ldpsi, hb, hb_bs, sp, plan, tw); count_launch();
      } else {
        if ((e = cudaFuncSetAttribute(k_plane_fwd_f<T, N2, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smf)))
          return e;
        k_plane_fwd_f<T, N2, N3><<<dim3(sp.nplane, nb), 256, smf, st>>>(hb, hb_bs, sp, plan, tw, kin, psi, ldpsi, out,
                                                                       ldout); count_launch();
      }
      return cudaGetLastError();
    }
  }
  const size_t sm = plane_lg_smem<T, N2, N3>(sp, plan);
  if (which == 0) {
    if ((e = cudaFuncSetAttribute(k_plane_inv_lg<T, N2, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
      return e;
    k_plane_inv_lg<T, N2, N3><<<dim3(sp.nplane, nb), 256, sm, st>>>(psi, ldpsi, hb, hb_bs, sp, plan, tw); count_launch();
  } else {
    if ((e = cudaFuncSetAttribute(k_plane_fwd_lg<T, N2, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
      return e;
    k_plane_fwd_lg<T, N2, N3><<<dim3(sp.nplane, nb), 256, sm, st>>>(hb, hb_bs, sp, plan, tw, kin, psi, ldpsi, out,
                                                                    ldout); count_launch();
  }
  return cudaGetLastError();
}

// which = 0: pass 1, 1: pass 3.  cudaErrorNotSupported when (n2, n3) has no instantiation
// or the shared-memory footprint does not fit.
template <typename T>
static cudaError_t plane_lg(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                            const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, const T* kin, cplx<T>* out,
                            int64_t ldout, int nb, cudaStream_t st) {
  const int n2 = plan.n[1], n3 = plan.n[2];
#define PW_PLANE_CASE(A, B)                                                                              \
  if (n2 == A && n3 == B) {                                                                              \
    if (plane_lg_smem<T, A, B>(sp, plan) > 227 * 1024) return cudaErrorNotSupported;                     \
    return plane_lg_pair<T, A, B>(which, psi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out, ldout, nb, st); \
  }
  PW_PLANE_CASE(24, 24)
  PW_PLANE_CASE(64, 64)
  PW_PLANE_CASE(72, 90)
  PW_PLANE_CASE(96, 96)
  PW_PLANE_CASE(120, 120)
#undef PW_PLANE_CASE
  return cudaErrorNotSupported;
}

// ---- one thread per line ----------------------------------------------------------
// Each thread transforms whole lines: its line lives in shared memory as a column
// (element e of the thread's line at buf[e * blockDim.x + threadIdx.x], or a padded plane
// row or column), so every shared access of a warp hits 32 consecutive words and no
// barrier separates the stages.  The butterfly index of every stage is a compile-time
// constant, so the twiddles are immediate constants: no twiddle table is read.

// exp(-2 pi i n / d) at compile time: exact reduction of n/d to an octant, then Taylor
// series of sin and cos on [0, pi/4] (13 terms: truncation below 1e-24).
struct CxW { double re, im; };
__host__ __device__ constexpr double cx_sinp(double x) {
  double t = x, s = x;
  for (int k = 1; k <= 13; ++k) { t *= -(x * x) / ((2.0 * k) * (2.0 * k + 1.0)); s += t; }
  return s;
}
__host__ __device__ constexpr double cx_cosp(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k <= 13; ++k) { t *= -(x * x) / ((2.0 * k - 1.0) * (2.0 * k)); s += t; }
  return s;
}
__host__ __device__ constexpr CxW cx_w(long n, long d) {
  n %= d;
  if (n < 0) n += d;
  constexpr double q = 0.78539816339744830961566084581987572;  // pi / 4
  const long o = (8 * n) / d;                                  // octant of 2 pi n / d
  const double phi = q * ((double)(8 * n - o * d) / (double)d);          // theta - o pi/4
  const double psi = q * ((double)((o + 1) * d - 8 * n) / (double)d);    // (o+1) pi/4 - theta
  double c = 0, s = 0;  // cos theta, sin theta
  switch (o) {
    case 0: c = cx_cosp(phi); s = cx_sinp(phi); break;
    case 1: c = cx_sinp(psi); s = cx_cosp(psi); break;
    case 2: c = -cx_sinp(phi); s = cx_cosp(phi); break;
    case 3: c = -cx_cosp(psi); s = cx_sinp(psi); break;
    case 4: c = -cx_cosp(phi); s = -cx_sinp(phi); break;
    case 5: c = -cx_sinp(psi); s = -cx_cosp(psi); break;
    case 6: c = cx_sinp(phi); s = -cx_cosp(phi); break;
    default: c = cx_cosp(psi); s = -cx_sinp(psi); break;
  }
  return CxW{c, -s};
}

// x * exp(S 2 pi i NUM / DEN)
template <typename C, int S, long NUM, long DEN> __device__ __forceinline__ C twmul(C x) {
  constexpr long n = ((NUM % DEN) + DEN) % DEN;
  if constexpr (n == 0) {
    return x;
  } else if constexpr ((4 * n) % DEN == 0) {
    constexpr int k = (int)(4 * n / DEN);  // (S i)^k
    if constexpr (k == 1) return cmuli<S>(x);
    else if constexpr (k == 2) return mk<C>(-x.x, -x.y);
    else return cmuli<-S>(x);
  } else {
    using R = decltype(C{}.x);
    constexpr CxW w = cx_w(n, DEN);  // exp(-2 pi i n / DEN)
    constexpr R wr = (R)w.re, wi = (R)(S < 0 ? w.im : -w.im);
    return mk<C>(x.x * wr - x.y * wi, x.x * wi + x.y * wr);
  }
}

template <typename F, int... I> __device__ __forceinline__ void sfor_seq(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
// f(std::integral_constant<int, i>) for i = 0 .. N-1, unrolled at compile time
template <int N, typename F> __device__ __forceinline__ void sfor(F&& f) {
  sfor_seq(f, std::make_integer_sequence<int, N>{});
}

// Keeps the compiler from hoisting the next butterfly's loads above this one's stores:
// bounds the live registers of the fully unrolled stages (otherwise every load of a
// stage is scheduled first and the kernel spills).
__device__ __forceinline__ void sched_fence() { asm volatile("" ::: "memory"); }

// x[m] *= exp(S 2 pi i J m / N) for m = 1 .. R-1
template <typename C, int S, int N, int J, int R> __device__ __forceinline__ void tw_stage(C* x) {
  sfor<R>([&](auto mc) {
    constexpr int M = decltype(mc)::value;
    x[M] = twmul<C, S, (long)J * M, N>(x[M]);
  });
}

constexpr int kTplX = 64;  // threads (= x-lines) per CTA of the x-line pass

// x-line pass, one thread per (y,z) line: inverse x (DIF, first stage reads the sphere
// planes), times V, forward x (DIT, last stage writes the sphere planes).
template <typename T, int N1>
__global__ void __launch_bounds__(kTplX) k_xline_tpl(cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                     const T* __restrict__ vperm, SphereDev sp, FftPlan plan) {
  using C = cplx<T>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  constexpr int R1 = P.radix[0], R2 = P.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw) + threadIdx.x;  // element e at S[e * kTplX]
  const int nyz = plan.n[1] * plan.n[2];
  const int yz = blockIdx.x * kTplX + threadIdx.x, b = blockIdx.y;
  const bool live = yz < nyz;
  const int np = sp.nplane;
  C* hbl = hb + (int64_t)b * hb_bs + (live ? yz : 0);
  // stage 1 of the inverse transform (radix R1, stride R2)
  sfor<R2>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    C x[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int p = J + R2 * a;  // plane p at x-frequency p (shift invariance, see k_xline_fused)
      x[a] = (live && p < np) ? hbl[(int64_t)p * nyz] : czero<C>();
    }
    dftR<C, +1, R1>(x);
    tw_stage<C, +1, N1, J, R1>(x);
#pragma unroll
    for (int m = 0; m < R1; ++m) S[(J + R2 * m) * kTplX] = x[m];
    sched_fence();
  });
  // stage 2 inverse (radix R2, contiguous blocks), V at the digit-reversed positions,
  // stage 2 forward
  const T* vb = vperm + (live ? yz : 0);
#pragma unroll
  for (int blk = 0; blk < R1; ++blk) {
    C y[R2];
#pragma unroll
    for (int m = 0; m < R2; ++m) y[m] = S[(blk * R2 + m) * kTplX];
    dftR<C, +1, R2>(y);
#pragma unroll
    for (int m = 0; m < R2; ++m) y[m] = cscale(y[m], live ? vb[(int64_t)(blk * R2 + m) * nyz] : (T)0);
    dftR<C, -1, R2>(y);
#pragma unroll
    for (int m = 0; m < R2; ++m) S[(blk * R2 + m) * kTplX] = y[m];
    sched_fence();
  }
  // stage 1 of the forward transform (DIT: twiddles, then radix R1): the sphere planes
  sfor<R2>([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    C x[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) x[m] = S[(J + R2 * m) * kTplX];
    tw_stage<C, -1, N1, J, R1>(x);
    dftR<C, -1, R1>(x);
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int p = J + R2 * a;
      if (live && p < np) hbl[(int64_t)p * nyz] = x[a];
    }
    sched_fence();
  });
}

// x-line pass with a group of TW warps per 32 lines: lane = line, warp t of the group takes
// the butterflies (and blocks) with index = t mod TW.  The warp index is uniform, so the
// butterfly indices, and with them the twiddles, are still compile-time constants, while
// each thread holds only 1/TW of a line: more warps per SM than one thread per line.
template <typename C, int S, int N1, int R1, int R2, int T0, int TW>
__device__ __forceinline__ void xw_stage1_inv(C* L, const C* hbl, int nyz, int h0, int np, bool live) {
  sfor<R2 / TW>([&](auto ic) {
    constexpr int J = T0 + TW * decltype(ic)::value;
    C x[R1];
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int p = J + R2 * a;  // plane p at x-frequency p (shift invariance, see k_xline_fused)
      x[a] = (live && p < np) ? hbl[(int64_t)p * nyz] : czero<C>();
    }
    dftR<C, +1, R1>(x);
    tw_stage<C, +1, N1, J, R1>(x);
#pragma unroll
    for (int m = 0; m < R1; ++m) L[(J + R2 * m) * 32] = x[m];
    sched_fence();
  });
}
template <typename C, int S, int N1, int R1, int R2, int T0, int TW>
__device__ __forceinline__ void xw_stage1_fwd(const C* L, C* hbl, int nyz, int h0, int np, bool live) {
  sfor<R2 / TW>([&](auto ic) {
    constexpr int J = T0 + TW * decltype(ic)::value;
    C x[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) x[m] = L[(J + R2 * m) * 32];
    tw_stage<C, -1, N1, J, R1>(x);
    dftR<C, -1, R1>(x);
#pragma unroll
    for (int a = 0; a < R1; ++a) {
      const int p = J + R2 * a;
      if (live && p < np) hbl[(int64_t)p * nyz] = x[a];
    }
    sched_fence();
  });
}

// The same with run-time butterfly indices (one code path for all warps of the group,
// which keeps the kernel small for the larger radices) and twiddles read from the stage
// table with warp-uniform indices.
// Twiddle w_N^(J m) of butterfly J, output m, read from the host's stage table of the first
// stage, [j][m] = w_N^(j m) for j < R2, 1 <= m < R1 at j (R1 - 1) + m - 1: TA = R1 - 1, TB = 1.
// With the radix order swapped the same table serves by symmetry of J m: TA = 1, TB = R1' - 1
// (R1' the table's own first radix).
template <typename C, int S, int R1, int R2, int TA = R1 - 1, int TB = 1>
__device__ __forceinline__ void xw_bf_inv(C* L, const C* hbl, const C* __restrict__ tw1, int J, int nyz, int h0,
                                          int np, int n1, bool live) {
  C x[R1];
#pragma unroll
  for (int a = 0; a < R1; ++a) {
    const int p = J + R2 * a;  // plane p at x-frequency p (shift invariance, see k_xline_fused)
    x[a] = (live && p < np) ? hbl[(int64_t)p * nyz] : czero<C>();
  }
  dftR<C, +1, R1>(x);
  if (J) {
#pragma unroll
    for (int m = 1; m < R1; ++m) x[m] = cmul(x[m], cconj(__ldg(&tw1[J * TA + m * TB - 1])));
  }
#pragma unroll
  for (int m = 0; m < R1; ++m) L[(J + R2 * m) * 32] = x[m];
}
template <typename C, int S, int R1, int R2, int TA = R1 - 1, int TB = 1>
__device__ __forceinline__ void xw_bf_fwd(const C* L, C* hbl, const C* __restrict__ tw1, int J, int nyz, int h0,
                                          int np, int n1, bool live) {
  C x[R1];
#pragma unroll
  for (int m = 0; m < R1; ++m) x[m] = L[(J + R2 * m) * 32];
  if (J) {
#pragma unroll
    for (int m = 1; m < R1; ++m) x[m] = cmul(x[m], __ldg(&tw1[J * TA + m * TB - 1]));
  }
  dftR<C, -1, R1>(x);
  // plane p = J + R2 a at hbl + p nyz, stepped by a running pointer
  C* o = hbl + (int64_t)J * nyz;
  const int64_t so = (int64_t)R2 * nyz;
  const int na = live ? (np - J + R2 - 1) / R2 : 0;  // planes J + R2 a < np
#pragma unroll
  for (int a = 0; a < R1; ++a, o += so) {
    if (a < na) *o = x[a];
  }
}

// Asynchronous global -> shared copies (LDGSTS) of the x-line forms: the CTA issues every
// load of its lines at once and the data bypasses the registers, so the memory system sees
// many requests in flight per SM while the butterflies of other CTAs run.
template <int B>
__device__ __forceinline__ void cp_async_el(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copies one band's np planes of the CTA's 32 lines into the line buffer Lb (element p of
// lane l at Lb[p * 32 + l], which is where the first stage reads and writes it); lanes past
// the end of the yz range are not copied (their results are never stored).
// (blockDim.x a multiple of 32: warp w copies the planes p with p mod (warp count) = w, lane l
// its line l, by pointer increments)
template <typename C>
__device__ __forceinline__ void xw_stage_planes(C* Lb, const C* hbb, int yz0, int nyz, int np) {
  const int nl = min(32, nyz - yz0);
  const int l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l < nl) {
    int p = threadIdx.x >> 5;
    const C* src = hbb + (int64_t)p * nyz + yz0 + l;
    C* dst = Lb + p * 32 + l;
    const int64_t ss = (int64_t)nw * nyz;
    for (; p < np; p += nw, src += ss, dst += nw * 32) cp_async_el<sizeof(C)>(dst, src);
  }
  cp_async_commit();
}

// First inverse stage on lines already staged in shared memory, in place: butterfly J reads
// and writes the slots J + R2 a, a < R1 (slots p >= np hold no plane and read as zero)
template <typename C, int R1, int R2, int TA = R1 - 1, int TB = 1>
__device__ __forceinline__ void xw_bf_inv_s(C* L, const C* __restrict__ tw1, int J, int np) {
  C x[R1];
#pragma unroll
  for (int a = 0; a < R1; ++a) {
    const int p = J + R2 * a;
    x[a] = p < np ? L[p * 32] : czero<C>();
  }
  dftR<C, +1, R1>(x);
  if (J) {
#pragma unroll
    for (int m = 1; m < R1; ++m) x[m] = cmul(x[m], cconj(__ldg(&tw1[J * TA + m * TB - 1])));
  }
#pragma unroll
  for (int m = 0; m < R1; ++m) L[(J + R2 * m) * 32] = x[m];
}

// Staged form: the planes arrive by asynchronous copies and the V values of the thread's
// second-stage blocks are loaded into registers while they are in flight.
template <typename T, int N1, int TW, bool SW = false>
__global__ void __launch_bounds__(32 * TW, 24 / TW) k_xline_tws(cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                      const T* __restrict__ vperm, SphereDev sp, FftPlan plan,
                                                      const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  constexpr int R1 = SW ? P.radix[1] : P.radix[0], R2 = SW ? P.radix[0] : P.radix[1];
  constexpr int TA = SW ? 1 : R1 - 1, TB = SW ? R2 - 1 : 1;
  constexpr int NBK = (R1 + TW - 1) / TW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  C* L0 = reinterpret_cast<C*>(smem_raw);
  C* L = L0 + lane;
  const int nyz = plan.n[1] * plan.n[2];
  const int yz0 = blockIdx.x * 32, yz = yz0 + lane, b = blockIdx.y;
  const bool live = yz < nyz;
  const int np = sp.nplane;
  const C* tw1 = tw + plan.d[0].tw_off[0];
  C* hbb = hb + (int64_t)b * hb_bs;
  xw_stage_planes<C>(L0, hbb, yz0, nyz, np);
  T vr[NBK][R2];
  {
    const T* vb = vperm + (live ? yz : 0);
#pragma unroll
    for (int i = 0; i < NBK; ++i) {
      const int blk = t + TW * i;
#pragma unroll
      for (int m = 0; m < R2; ++m) vr[i][m] = (live && blk < R1) ? vb[(int64_t)(blk * R2 + m) * nyz] : (T)0;
    }
  }
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll 1
  for (int J = t; J < R2; J += TW) xw_bf_inv_s<C, R1, R2, TA, TB>(L, tw1, J, np);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NBK; ++i) {
    const int blk = t + TW * i;
    if (blk < R1) {
      C y[R2];
#pragma unroll
      for (int m = 0; m < R2; ++m) y[m] = L[(blk * R2 + m) * 32];
      dftR<C, +1, R2>(y);
#pragma unroll
      for (int m = 0; m < R2; ++m) y[m] = cscale(y[m], vr[i][m]);
      dftR<C, -1, R2>(y);
#pragma unroll
      for (int m = 0; m < R2; ++m) L[(blk * R2 + m) * 32] = y[m];
    }
  }
  __syncthreads();
  C* hbl = hbb + (live ? yz : 0);
#pragma unroll 1
  for (int J = t; J < R2; J += TW) xw_bf_fwd<C, -1, R1, R2, TA, TB>(L, hbl, tw1, J, nyz, 0, np, N1, live);
}

// Staged form with several bands per CTA and two line buffers: the copies of band b + 1 are
// in flight while band b is transformed; the V values stay in registers for all bands.
template <typename T, int N1, int TW, bool SW = false>
__global__ void __launch_bounds__(32 * TW, 12 / TW) k_xline_twd(cplx<T>* __restrict__ hb, int64_t hb_bs, int nb,
                                                      int bper, const T* __restrict__ vperm, SphereDev sp,
                                                      FftPlan plan, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  constexpr int R1 = SW ? P.radix[1] : P.radix[0], R2 = SW ? P.radix[0] : P.radix[1];
  constexpr int TA = SW ? 1 : R1 - 1, TB = SW ? R2 - 1 : 1;
  constexpr int NBK = (R1 + TW - 1) / TW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  C* Lbuf = reinterpret_cast<C*>(smem_raw);  // two buffers of N1 * 32
  const int nyz = plan.n[1] * plan.n[2];
  const int yz0 = blockIdx.x * 32, yz = yz0 + lane;
  const bool live = yz < nyz;
  const int np = sp.nplane;
  const C* tw1 = tw + plan.d[0].tw_off[0];
  const int b_lo = blockIdx.y * bper, b_hi = min(nb, b_lo + bper);
  if (b_lo >= b_hi) return;
  xw_stage_planes<C>(Lbuf, hb + (int64_t)b_lo * hb_bs, yz0, nyz, np);
  T vr[NBK][R2];
  {
    const T* vb = vperm + (live ? yz : 0);
#pragma unroll
    for (int i = 0; i < NBK; ++i) {
      const int blk = t + TW * i;
#pragma unroll
      for (int m = 0; m < R2; ++m) vr[i][m] = (live && blk < R1) ? vb[(int64_t)(blk * R2 + m) * nyz] : (T)0;
    }
  }
#pragma unroll 1
  for (int b = b_lo; b < b_hi; ++b) {
    C* Lc = Lbuf + ((b - b_lo) & 1) * (N1 * 32);
    if (b + 1 < b_hi) {
      // the other buffer was released by the barrier that ended the previous band
      xw_stage_planes<C>(Lbuf + ((b + 1 - b_lo) & 1) * (N1 * 32), hb + (int64_t)(b + 1) * hb_bs, yz0, nyz, np);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    C* L = Lc + lane;
#pragma unroll 1
    for (int J = t; J < R2; J += TW) xw_bf_inv_s<C, R1, R2, TA, TB>(L, tw1, J, np);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NBK; ++i) {
      const int blk = t + TW * i;
      if (blk < R1) {
        C y[R2];
#pragma unroll
        for (int m = 0; m < R2; ++m) y[m] = L[(blk * R2 + m) * 32];
        dftR<C, +1, R2>(y);
#pragma unroll
        for (int m = 0; m < R2; ++m) y[m] = cscale(y[m], vr[i][m]);
        dftR<C, -1, R2>(y);
#pragma unroll
        for (int m = 0; m < R2; ++m) L[(blk * R2 + m) * 32] = y[m];
      }
    }
    __syncthreads();
    C* hbl = hb + (int64_t)b * hb_bs + (live ? yz : 0);
#pragma unroll 1
    for (int J = t; J < R2; J += TW) xw_bf_fwd<C, -1, R1, R2, TA, TB>(L, hbl, tw1, J, nyz, 0, np, N1, live);
    __syncthreads();  // this buffer is staged again two bands later
  }
}

template <typename T, int N1, int TW, bool SW = false>
__global__ void __launch_bounds__(32 * TW, 24 / TW) k_xline_twr(cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                      const T* __restrict__ vperm, SphereDev sp, FftPlan plan,
                                                      const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  // SW: the two radices in the other order (same twiddle table, transposed index)
  constexpr int R1 = SW ? P.radix[1] : P.radix[0], R2 = SW ? P.radix[0] : P.radix[1];
  constexpr int TA = SW ? 1 : R1 - 1, TB = SW ? R2 - 1 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  C* L = reinterpret_cast<C*>(smem_raw) + lane;
  const int nyz = plan.n[1] * plan.n[2];
  const int yz = blockIdx.x * 32 + lane, b = blockIdx.y;
  const bool live = yz < nyz;
  const int h0 = sp.plane_h[0], np = sp.nplane;
  const C* tw1 = tw + plan.d[0].tw_off[0];
  C* hbl = hb + (int64_t)b * hb_bs + (live ? yz : 0);
#pragma unroll 1
  for (int J = t; J < R2; J += TW) xw_bf_inv<C, +1, R1, R2, TA, TB>(L, hbl, tw1, J, nyz, h0, np, N1, live);
  __syncthreads();
  const T* vb = vperm + (live ? yz : 0);
#pragma unroll 1
  for (int blk = t; blk < R1; blk += TW) {
    C y[R2];
#pragma unroll
    for (int m = 0; m < R2; ++m) y[m] = L[(blk * R2 + m) * 32];
    dftR<C, +1, R2>(y);
#pragma unroll
    for (int m = 0; m < R2; ++m) y[m] = cscale(y[m], live ? vb[(int64_t)(blk * R2 + m) * nyz] : (T)0);
    dftR<C, -1, R2>(y);
#pragma unroll
    for (int m = 0; m < R2; ++m) L[(blk * R2 + m) * 32] = y[m];
  }
  __syncthreads();
#pragma unroll 1
  for (int J = t; J < R2; J += TW) xw_bf_fwd<C, -1, R1, R2, TA, TB>(L, hbl, tw1, J, nyz, h0, np, N1, live);
}

// The same with several bands per CTA: the V values of the CTA's lines stay in registers.
template <typename T, int N1, int TW, bool SW = false>
__global__ void __launch_bounds__(32 * TW, 24 / TW) k_xline_twm(cplx<T>* __restrict__ hb, int64_t hb_bs, int nb,
                                                      int bper, const T* __restrict__ vperm, SphereDev sp,
                                                      FftPlan plan, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  // SW: the two radices in the other order (same twiddle table, transposed index)
  constexpr int R1 = SW ? P.radix[1] : P.radix[0], R2 = SW ? P.radix[0] : P.radix[1];
  constexpr int TA = SW ? 1 : R1 - 1, TB = SW ? R2 - 1 : 1;
  constexpr int NBK = (R1 + TW - 1) / TW;  // stage-2 blocks per warp (at most)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  C* L = reinterpret_cast<C*>(smem_raw) + lane;
  const int nyz = plan.n[1] * plan.n[2];
  const int yz = blockIdx.x * 32 + lane;
  const bool live = yz < nyz;
  const int h0 = sp.plane_h[0], np = sp.nplane;
  const C* tw1 = tw + plan.d[0].tw_off[0];
  // this thread's V values, read once for all the CTA's bands
  T vr[NBK][R2];
  {
    const T* vb = vperm + (live ? yz : 0);
#pragma unroll
    for (int i = 0; i < NBK; ++i) {
      const int blk = t + TW * i;
#pragma unroll
      for (int m = 0; m < R2; ++m) vr[i][m] = (live && blk < R1) ? vb[(int64_t)(blk * R2 + m) * nyz] : (T)0;
    }
  }
  const int b_lo = blockIdx.y * bper, b_hi = min(nb, b_lo + bper);
#pragma unroll 1
  for (int b = b_lo; b < b_hi; ++b) {
    C* hbl = hb + (int64_t)b * hb_bs + (live ? yz : 0);
#pragma unroll 1
    for (int J = t; J < R2; J += TW) xw_bf_inv<C, +1, R1, R2, TA, TB>(L, hbl, tw1, J, nyz, h0, np, N1, live);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NBK; ++i) {
      const int blk = t + TW * i;
      if (blk < R1) {
        C y[R2];
#pragma unroll
        for (int m = 0; m < R2; ++m) y[m] = L[(blk * R2 + m) * 32];
        dftR<C, +1, R2>(y);
#pragma unroll
        for (int m = 0; m < R2; ++m) y[m] = cscale(y[m], vr[i][m]);
        dftR<C, -1, R2>(y);
#pragma unroll
        for (int m = 0; m < R2; ++m) L[(blk * R2 + m) * 32] = y[m];
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int J = t; J < R2; J += TW) xw_bf_fwd<C, -1, R1, R2, TA, TB>(L, hbl, tw1, J, nyz, h0, np, N1, live);
    __syncthreads();  // the next band's first stage overwrites the lines
  }
}

template <typename T, int N1, int TW>
__global__ void __launch_bounds__(32 * TW) k_xline_tw(cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                     const T* __restrict__ vperm, SphereDev sp, FftPlan plan) {
  using C = cplx<T>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  constexpr int R1 = P.radix[0], R2 = P.radix[1];
  static_assert(R1 % TW == 0 && R2 % TW == 0, "butterflies must split evenly over the warps");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  C* L = reinterpret_cast<C*>(smem_raw) + lane;  // element e of this lane's line at L[e * 32]
  const int nyz = plan.n[1] * plan.n[2];
  const int yz = blockIdx.x * 32 + lane, b = blockIdx.y;
  const bool live = yz < nyz;
  const int h0 = sp.plane_h[0], np = sp.nplane;
  C* hbl = hb + (int64_t)b * hb_bs + (live ? yz : 0);
  sfor<TW>([&](auto tc) {
    if (t == decltype(tc)::value) xw_stage1_inv<C, +1, N1, R1, R2, decltype(tc)::value, TW>(L, hbl, nyz, h0, np, live);
  });
  __syncthreads();
  const T* vb = vperm + (live ? yz : 0);
#pragma unroll 1
  for (int blk = t; blk < R1; blk += TW) {
    C y[R2];
#pragma unroll
    for (int m = 0; m < R2; ++m) y[m] = L[(blk * R2 + m) * 32];
    dftR<C, +1, R2>(y);
#pragma unroll
    for (int m = 0; m < R2; ++m) y[m] = cscale(y[m], live ? vb[(int64_t)(blk * R2 + m) * nyz] : (T)0);
    dftR<C, -1, R2>(y);
#pragma unroll
    for (int m = 0; m < R2; ++m) L[(blk * R2 + m) * 32] = y[m];
  }
  __syncthreads();
  sfor<TW>([&](auto tc) {
    if (t == decltype(tc)::value) xw_stage1_fwd<C, -1, N1, R1, R2, decltype(tc)::value, TW>(L, hbl, nyz, h0, np, live);
  });
}

template <typename T, int N1, int TW>
static cudaError_t launch_xline_tw(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp,
                                   const FftPlan& plan, int nb, cudaStream_t st) {
  const size_t sm = sizeof(cplx<T>) * (size_t)N1 * 32;
  cudaError_t e = cudaFuncSetAttribute(k_xline_tw<T, N1, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  if ((e = cudaFuncSetAttribute(k_xline_tw<T, N1, TW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100))) return e;
  const int nyz = plan.n[1] * plan.n[2];
  k_xline_tw<T, N1, TW><<<dim3((nyz + 31) / 32, nb), 32 * TW, sm, st>>>(hb, hb_bs, vperm, sp, plan); count_launch();
  return cudaGetLastError();
}

template <typename T, int N1, int TW, bool SW = false>
static cudaError_t launch_xline_twr(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp,
                                    const FftPlan& plan, const cplx<T>* tw, int nb, bool multi, cudaStream_t st,
                                    bool staged = false) {
  const size_t sm = sizeof(cplx<T>) * (size_t)N1 * 32;
  const int nyz = plan.n[1] * plan.n[2];
  const int gx = (nyz + 31) / 32;
  cudaError_t e;
  if (staged && !multi) {
    if ((e = cudaFuncSetAttribute(k_xline_tws<T, N1, TW, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
      return e;
    if ((e = cudaFuncSetAttribute(k_xline_tws<T, N1, TW, SW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
      return e;
    k_xline_tws<T, N1, TW, SW><<<dim3(gx, nb), 32 * TW, sm, st>>>(hb, hb_bs, vperm, sp, plan, tw); count_launch();
    return cudaGetLastError();
  }
  if (staged) {
    const size_t sm2 = 2 * sm;
    if ((e = cudaFuncSetAttribute(k_xline_twd<T, N1, TW, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)))
      return e;
    if ((e = cudaFuncSetAttribute(k_xline_twd<T, N1, TW, SW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
      return e;
    // a few bands per CTA, about three waves of CTAs
    const int bper = std::max(2, (int)(((int64_t)nb * gx + 152 * 9 - 1) / (152 * 9)));
    const int splits = (nb + bper - 1) / bper;
    k_xline_twd<T, N1, TW, SW><<<dim3(gx, splits), 32 * TW, sm2, st>>>(hb, hb_bs, nb, bper, vperm, sp, plan, tw);
    count_launch();
    return cudaGetLastError();
  }
  if (!multi) {
    if ((e = cudaFuncSetAttribute(k_xline_twr<T, N1, TW, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
      return e;
    if ((e = cudaFuncSetAttribute(k_xline_twr<T, N1, TW, SW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
      return e;
    k_xline_twr<T, N1, TW, SW><<<dim3(gx, nb), 32 * TW, sm, st>>>(hb, hb_bs, vperm, sp, plan, tw); count_launch();
    return cudaGetLastError();
  }
  if ((e = cudaFuncSetAttribute(k_xline_twm<T, N1, TW, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
    return e;
  if ((e = cudaFuncSetAttribute(k_xline_twm<T, N1, TW, SW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
    return e;
  // several bands per CTA (the V values stay in registers), about six waves of CTAs
  const int bper = std::max(1, (int)(((int64_t)nb * gx + 152 * 36 - 1) / (152 * 36)));
  const int splits = (nb + bper - 1) / bper;
  k_xline_twm<T, N1, TW, SW><<<dim3(gx, splits), 32 * TW, sm, st>>>(hb, hb_bs, nb, bper, vperm, sp, plan, tw);
  count_launch();
  return cudaGetLastError();
}

// groups of warps per 32 x-lines, run-time butterfly indices (any two-stage plan)
template <typename T>
static cudaError_t xline_twr(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp, const FftPlan& plan,
                             const cplx<T>* tw, int nb, bool multi, cudaStream_t st, bool swap = false,
                             bool staged = false) {
#define PW_TWR_CASE(N)                                                                                   \
  case N:                                                                                                \
    return swap ? launch_xline_twr<T, N, 4, true>(hb, hb_bs, vperm, sp, plan, tw, nb, multi, st, staged)  \
                : launch_xline_twr<T, N, 4, false>(hb, hb_bs, vperm, sp, plan, tw, nb, multi, st, staged);
  switch (plan.n[0]) {
    PW_TWR_CASE(24)
    PW_TWR_CASE(72)
    PW_TWR_CASE(90)
    PW_TWR_CASE(96)
    PW_TWR_CASE(120)
    case 64: return launch_xline_twr<T, 64, 4>(hb, hb_bs, vperm, sp, plan, tw, nb, multi, st, staged);  // 8 x 8
    default: return cudaErrorNotSupported;
  }
#undef PW_TWR_CASE
}

// groups of warps per line where the butterfly counts allow (otherwise not supported)
template <typename T>
static cudaError_t xline_tw(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp, const FftPlan& plan,
                            int nb, cudaStream_t st) {
  switch (plan.n[0]) {
    case 24: return launch_xline_tw<T, 24, 2>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 64: return launch_xline_tw<T, 64, 4>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 96: return launch_xline_tw<T, 96, 4>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 120: return launch_xline_tw<T, 120, 2>(hb, hb_bs, vperm, sp, plan, nb, st);
    default: return cudaErrorNotSupported;
  }
}

// Plane passes, one thread per line.  The CTA holds its x-plane as F[N2][N3 + 1] (odd
// pitch: row and column accesses of a warp are conflict-free); the z-lines of the rows
// holding coefficients and the y-lines of all N3 columns are transformed in place.
template <int N2, int N3> struct PlaneT {
  static constexpr CPlan P2 = make_cplan(N2), P3 = make_cplan(N3);
  static constexpr int FP = N3 + 1;
  static constexpr bool ok = (P2.nst == 2 && P3.nst == 2);
  static constexpr int THREADS = ((N3 + 31) / 32) * 32;
};

template <typename T, int N2, int N3>
__global__ void __launch_bounds__(PlaneT<N2, N3>::THREADS) k_plane_inv_tpl(const cplx<T>* __restrict__ psi,
                                                                            int64_t ldpsi, cplx<T>* __restrict__ hb,
                                                                            int64_t hb_bs, SphereDev sp) {
  using C = cplx<T>;
  using PT = PlaneT<N2, N3>;
  constexpr int FP = PT::FP;
  constexpr int Y1 = PT::P2.radix[0], Y2 = PT::P2.radix[1];
  constexpr int Z1 = PT::P3.radix[0], Z2 = PT::P3.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* F = reinterpret_cast<C*>(smem_raw);
  int* ymap = reinterpret_cast<int*>(F + N2 * FP);  // y -> sphere row of the plane, or -1
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* src = psi + (int64_t)b * ldpsi;
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  // z-lines: one thread per sphere row, in place on its plane row
  for (int row = threadIdx.x; row < nr; row += blockDim.x) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    C* line = F + pmod(sp.row_k[r0 + row], N2) * FP;
    sfor<Z2>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      C x[Z1];
#pragma unroll
      for (int a = 0; a < Z1; ++a) {
        const int idx = pmod(J + Z2 * a - l0, N3);
        x[a] = idx < cnt ? src[g0 + idx] : czero<C>();
      }
      dftR<C, +1, Z1>(x);
      tw_stage<C, +1, N3, J, Z1>(x);
#pragma unroll
      for (int m = 0; m < Z1; ++m) line[J + Z2 * m] = x[m];
      sched_fence();
    });
#pragma unroll
    for (int blk = 0; blk < Z1; ++blk) {
      C y[Z2];
#pragma unroll
      for (int m = 0; m < Z2; ++m) y[m] = line[blk * Z2 + m];
      dftR<C, +1, Z2>(y);
#pragma unroll
      for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = y[m];
      sched_fence();
    }
  }
  __syncthreads();
  // y-lines: one thread per column, in place; rows without coefficients read as zero
  C* dst = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  for (int c = threadIdx.x; c < N3; c += blockDim.x) {
    C* col = F + c;
    sfor<Y2>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      C x[Y1];
#pragma unroll
      for (int a = 0; a < Y1; ++a) x[a] = ymap[J + Y2 * a] >= 0 ? col[(J + Y2 * a) * FP] : czero<C>();
      dftR<C, +1, Y1>(x);
      tw_stage<C, +1, N2, J, Y1>(x);
#pragma unroll
      for (int m = 0; m < Y1; ++m) col[(J + Y2 * m) * FP] = x[m];
      sched_fence();
    });
#pragma unroll
    for (int blk = 0; blk < Y1; ++blk) {
      C y[Y2];
#pragma unroll
      for (int m = 0; m < Y2; ++m) y[m] = col[(blk * Y2 + m) * FP];
      dftR<C, +1, Y2>(y);
#pragma unroll
      for (int m = 0; m < Y2; ++m) dst[(int64_t)(blk * Y2 + m) * N3 + c] = y[m];
      sched_fence();
    }
  }
}

template <typename T, int N2, int N3>
__global__ void __launch_bounds__(PlaneT<N2, N3>::THREADS) k_plane_fwd_tpl(const cplx<T>* __restrict__ hb,
                                                                            int64_t hb_bs, SphereDev sp,
                                                                            const T* __restrict__ kin,
                                                                            const cplx<T>* __restrict__ psi,
                                                                            int64_t ldpsi, cplx<T>* __restrict__ out,
                                                                            int64_t ldout) {
  using C = cplx<T>;
  using PT = PlaneT<N2, N3>;
  constexpr int FP = PT::FP;
  constexpr int Y1 = PT::P2.radix[0], Y2 = PT::P2.radix[1];
  constexpr int Z1 = PT::P3.radix[0], Z2 = PT::P3.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* F = reinterpret_cast<C*>(smem_raw);
  int* ymap = reinterpret_cast<int*>(F + N2 * FP);
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* srcp = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  __syncthreads();
  // y-lines (forward DIT: radix Y2 blocks read from the half-box plane, then radix Y1
  // with twiddles); only the rows holding coefficients are stored
  for (int c = threadIdx.x; c < N3; c += blockDim.x) {
    C* col = F + c;
#pragma unroll
    for (int blk = 0; blk < Y1; ++blk) {
      C y[Y2];
#pragma unroll
      for (int m = 0; m < Y2; ++m) y[m] = srcp[(int64_t)(blk * Y2 + m) * N3 + c];
      dftR<C, -1, Y2>(y);
#pragma unroll
      for (int m = 0; m < Y2; ++m) col[(blk * Y2 + m) * FP] = y[m];
      sched_fence();
    }
    sfor<Y2>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      C x[Y1];
#pragma unroll
      for (int m = 0; m < Y1; ++m) x[m] = col[(J + Y2 * m) * FP];
      tw_stage<C, -1, N2, J, Y1>(x);
      dftR<C, -1, Y1>(x);
#pragma unroll
      for (int a = 0; a < Y1; ++a)
        if (ymap[J + Y2 * a] >= 0) col[(J + Y2 * a) * FP] = x[a];
      sched_fence();
    });
  }
  __syncthreads();
  // z-lines of the rows holding coefficients: gather with the kinetic term
  const C* yv = psi + (int64_t)b * ldpsi;
  C* o = out + (int64_t)b * ldout;
  for (int row = threadIdx.x; row < nr; row += blockDim.x) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    C* line = F + pmod(sp.row_k[r0 + row], N2) * FP;
#pragma unroll
    for (int blk = 0; blk < Z1; ++blk) {
      C y[Z2];
#pragma unroll
      for (int m = 0; m < Z2; ++m) y[m] = line[blk * Z2 + m];
      dftR<C, -1, Z2>(y);
#pragma unroll
      for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = y[m];
      sched_fence();
    }
    sfor<Z2>([&](auto jc) {
      constexpr int J = decltype(jc)::value;
      C x[Z1];
#pragma unroll
      for (int m = 0; m < Z1; ++m) x[m] = line[J + Z2 * m];
      tw_stage<C, -1, N3, J, Z1>(x);
      dftR<C, -1, Z1>(x);
#pragma unroll
      for (int a = 0; a < Z1; ++a) {
        const int idx = pmod(J + Z2 * a - l0, N3);
        if (idx < cnt) {
          const int g = g0 + idx;
          const C yy = yv[g];
          const T k = kin[g];
          o[g] = mk<C>(k * yy.x + x[a].x, k * yy.y + x[a].y);
        }
      }
      sched_fence();
    });
  }
}

// Plane passes with groups of TW warps per 32 lines (lane = line; the warps of a group take
// the butterflies with index = warp mod TW; run-time indices, twiddles read from the
// stage tables with warp-uniform indices).  The CTA holds the x-plane as F[N2][N3 + 1] and
// has one group per 32 columns; the z-lines of the sphere rows go in chunks of 32 rows.
template <int N2, int N3, int TW> struct PlaneW {
  static constexpr CPlan P2 = make_cplan(N2), P3 = make_cplan(N3);
  static constexpr int FP = N3 + 1;
  static constexpr int NG = (N3 + 31) / 32;
  static constexpr int THREADS = 32 * TW * NG;
  static constexpr bool ok = (P2.nst == 2 && P3.nst == 2);
};
// byte offset of pass 3's prefetched blocks: after the plane and the row map, 16-aligned
template <typename C, int N2, int N3, int TW>
__host__ __device__ constexpr size_t plane_wg_stage_off() {
  return ((sizeof(C) * (size_t)N2 * PlaneW<N2, N3, TW>::FP + sizeof(int) * N2) + 15) / 16 * 16;
}

// One (plane p, band b) item of pass 1 with the whole plane in shared memory; `before_y`
// runs between the z-lines and the y-lines (the persistent form prefetches there).
template <typename T, int N2, int N3, int TW, typename G>
__device__ __forceinline__ void plane_inv_wg_item(int p, int b, const cplx<T>* __restrict__ psi, int64_t ldpsi,
                                                  cplx<T>* __restrict__ hb, int64_t hb_bs, const SphereDev& sp,
                                                  const FftPlan& plan, const cplx<T>* __restrict__ tw, G&& before_y) {
  using C = cplx<T>;
  using PW = PlaneW<N2, N3, TW>;
  constexpr int FP = PW::FP, NG = PW::NG;
  constexpr int Y1 = PW::P2.radix[0], Y2 = PW::P2.radix[1];
  constexpr int Z1 = PW::P3.radix[0], Z2 = PW::P3.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* F = reinterpret_cast<C*>(smem_raw);
  int* ymap = reinterpret_cast<int*>(F + N2 * FP);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = w / TW, t = w % TW;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* src = psi + (int64_t)b * ldpsi;
  const C* twy = tw + plan.d[1].tw_off[0];
  const C* twz = tw + plan.d[2].tw_off[0];
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  // z-lines, chunks of 32 * NG rows (the chunk count is the same for every thread); the
  // first stage reads the row's run of coefficients straight from the block (staging the
  // plane's block first measured slower: with one CTA per SM nothing overlaps the wait)
  // the rows are spread over every warp of the CTA: ngz groups of 32 rows (as many as the
  // plane needs), each group's butterflies over nwz = TW NG / ngz warps
  const int ngz = max(1, min(NG, (nr + 31) / 32)), nwz = (TW * NG) / ngz;
  const int gz = w / nwz, tz = w % nwz;
  for (int c0 = 0; c0 < nr; c0 += 32 * ngz) {
    const int row = c0 + gz * 32 + lane;
    const bool live = gz < ngz && row < nr;
    int g0 = 0, cnt = 0, l0 = 0;
    C* line = F;
    if (live) {
      g0 = sp.row_g0[r0 + row]; cnt = sp.row_cnt[r0 + row]; l0 = sp.row_l0[r0 + row];
      line = F + pmod(sp.row_k[r0 + row], N2) * FP;
    }
    if (live) {
#pragma unroll 1
      for (int J = tz; J < Z2; J += nwz) {
        C x[Z1];
#pragma unroll
        for (int a = 0; a < Z1; ++a) {
          const int idx = pmod(J + Z2 * a - l0, N3);
          x[a] = idx < cnt ? src[g0 + idx] : czero<C>();
        }
        dftR<C, +1, Z1>(x);
        if (J) {
#pragma unroll
          for (int m = 1; m < Z1; ++m) x[m] = cmul(x[m], cconj(__ldg(&twz[J * (Z1 - 1) + m - 1])));
        }
#pragma unroll
        for (int m = 0; m < Z1; ++m) line[J + Z2 * m] = x[m];
      }
    }
    __syncthreads();
    if (live) {
#pragma unroll 1
      for (int blk = tz; blk < Z1; blk += nwz) {
        C y[Z2];
#pragma unroll
        for (int m = 0; m < Z2; ++m) y[m] = line[blk * Z2 + m];
        dftR<C, +1, Z2>(y);
#pragma unroll
        for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = y[m];
      }
    }
  }
  __syncthreads();
  before_y();
  // y-lines: column c = 32 g + lane; rows without coefficients read as zero
  const int c = g * 32 + lane;
  const bool livec = c < N3;
  C* col = F + (livec ? c : 0);
  if (livec) {
#pragma unroll 1
    for (int J = t; J < Y2; J += TW) {
      C x[Y1];
#pragma unroll
      for (int a = 0; a < Y1; ++a) x[a] = ymap[J + Y2 * a] >= 0 ? col[(J + Y2 * a) * FP] : czero<C>();
      dftR<C, +1, Y1>(x);
      if (J) {
#pragma unroll
        for (int m = 1; m < Y1; ++m) x[m] = cmul(x[m], cconj(__ldg(&twy[J * (Y1 - 1) + m - 1])));
      }
#pragma unroll
      for (int m = 0; m < Y1; ++m) col[(J + Y2 * m) * FP] = x[m];
    }
  }
  __syncthreads();
  C* dst = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  if (livec) {
#pragma unroll 1
    for (int blk = t; blk < Y1; blk += TW) {
      C y[Y2];
#pragma unroll
      for (int m = 0; m < Y2; ++m) y[m] = col[(blk * Y2 + m) * FP];
      dftR<C, +1, Y2>(y);
#pragma unroll
      for (int m = 0; m < Y2; ++m) dst[(int64_t)(blk * Y2 + m) * N3 + c] = y[m];
    }
  }
}

template <typename T, int N2, int N3, int TW>
__global__ void __launch_bounds__(PlaneW<N2, N3, TW>::THREADS) k_plane_inv_wg(const cplx<T>* __restrict__ psi,
                                                                               int64_t ldpsi, cplx<T>* __restrict__ hb,
                                                                               int64_t hb_bs, SphereDev sp, FftPlan plan,
                                                                               const cplx<T>* __restrict__ tw) {
  plane_inv_wg_item<T, N2, N3, TW>(blockIdx.x, blockIdx.y, psi, ldpsi, hb, hb_bs, sp, plan, tw, [] {});
}

// Persistent form: one CTA per resident slot walks the (plane, band) items; during an item's
// y-lines the next item's block of sphere coefficients is prefetched into L2 (one bulk
// prefetch, its start rounded down and its end rounded down to 16 bytes).
template <typename T, int N2, int N3, int TW>
__global__ void __launch_bounds__(PlaneW<N2, N3, TW>::THREADS) k_plane_inv_wgp(const cplx<T>* __restrict__ psi,
                                                                                int64_t ldpsi, cplx<T>* __restrict__ hb,
                                                                                int64_t hb_bs, SphereDev sp,
                                                                                FftPlan plan,
                                                                                const cplx<T>* __restrict__ tw, int nb) {
  using C = cplx<T>;
  const int nitems = sp.nplane * nb;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int nxt = it + gridDim.x;
    plane_inv_wg_item<T, N2, N3, TW>(it % sp.nplane, it / sp.nplane, psi, ldpsi, hb, hb_bs, sp, plan, tw, [&] {
      if (nxt < nitems && threadIdx.x == 0) {
        const int pn = nxt % sp.nplane, bn = nxt / sp.nplane;
        const int r0 = sp.plane_row0[pn], nr = sp.plane_row0[pn + 1] - r0;
        if (nr > 0) {
          const int g0 = sp.row_g0[r0], g1 = sp.row_g0[r0 + nr - 1] + sp.row_cnt[r0 + nr - 1];
          const uintptr_t a0 = (uintptr_t)(psi + (int64_t)bn * ldpsi + g0) & ~(uintptr_t)15;
          const uintptr_t a1 = (uintptr_t)(psi + (int64_t)bn * ldpsi + g1) & ~(uintptr_t)15;
          if (a1 > a0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((unsigned)(a1 - a0)) : "memory");
        }
      }
    });
    __syncthreads();  // the plane and the row map are reused by the next item
  }
}

// One (plane p, band b) item of pass 3 with the whole plane in shared memory.  Sy and Sk
// receive the plane's blocks of Y_k and t_G by asynchronous copies that the caller issued
// (committed as the group before any it issues in `before_gather`); `before_gather` runs
// after the z-lines and waits for them.
template <typename T, int N2, int N3, int TW, bool REC, typename G>
__device__ __forceinline__ void plane_fwd_wg_item(int p, int b, const cplx<T>* __restrict__ hb, int64_t hb_bs,
                                                  const SphereDev& sp, const FftPlan& plan,
                                                  const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ psi,
                                                  int64_t ldpsi, cplx<T>* __restrict__ out, int64_t ldout,
                                                  const Pass3Rec& rec, cplx<T>* Sy, T* Sk, G&& before_gather) {
  using C = cplx<T>;
  using PW = PlaneW<N2, N3, TW>;
  constexpr int FP = PW::FP, NG = PW::NG;
  constexpr int Y1 = PW::P2.radix[0], Y2 = PW::P2.radix[1];
  constexpr int Z1 = PW::P3.radix[0], Z2 = PW::P3.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* F = reinterpret_cast<C*>(smem_raw);
  int* ymap = reinterpret_cast<int*>(F + N2 * FP);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = w / TW, t = w % TW;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* srcp = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  const C* twy = tw + plan.d[1].tw_off[0];
  const C* twz = tw + plan.d[2].tw_off[0];
  const int pg0 = nr > 0 ? sp.row_g0[r0] : 0;
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  // y-lines: radix Y2 blocks read from the half-box plane, then radix Y1 with twiddles;
  // only the rows holding coefficients are stored
  const int c = g * 32 + lane;
  const bool livec = c < N3;
  C* col = F + (livec ? c : 0);
  if (livec) {
#pragma unroll 1
    for (int blk = t; blk < Y1; blk += TW) {
      C y[Y2];
#pragma unroll
      for (int m = 0; m < Y2; ++m) y[m] = srcp[(int64_t)(blk * Y2 + m) * N3 + c];
      dftR<C, -1, Y2>(y);
#pragma unroll
      for (int m = 0; m < Y2; ++m) col[(blk * Y2 + m) * FP] = y[m];
    }
  }
  __syncthreads();
  if (livec) {
#pragma unroll 1
    for (int J = t; J < Y2; J += TW) {
      C x[Y1];
#pragma unroll
      for (int m = 0; m < Y1; ++m) x[m] = col[(J + Y2 * m) * FP];
      if (J) {
#pragma unroll
        for (int m = 1; m < Y1; ++m) x[m] = cmul(x[m], __ldg(&twy[J * (Y1 - 1) + m - 1]));
      }
      dftR<C, -1, Y1>(x);
#pragma unroll
      for (int a = 0; a < Y1; ++a)
        if (ymap[J + Y2 * a] >= 0) col[(J + Y2 * a) * FP] = x[a];
    }
  }
  __syncthreads();
  // z-lines of the rows holding coefficients, chunks of 32 * NG rows: gather with the
  // kinetic term
  C* o = out + (int64_t)b * ldout;
  T ra = 0, rs = 0;  // recurrence alpha and shift
  if constexpr (REC) {
    ra = (T)rec.alpha;
    rs = (T)rec.shift;
    if (rec.dev_ce) {
      rs = (T)rec.dev_ce[0];
      ra = (T)((rec.first ? 1.0 : 2.0) / rec.dev_ce[1]);
    }
  }
  // (spreading these rows over all the CTA's warps, as pass 1 does, measured slower here)
  for (int c0 = 0; c0 < nr; c0 += 32 * NG) {
    const int row = c0 + g * 32 + lane;
    const bool live = row < nr;
    C* line = live ? F + pmod(sp.row_k[r0 + row], N2) * FP : F;
    if (live) {
#pragma unroll 1
      for (int blk = t; blk < Z1; blk += TW) {
        C y[Z2];
#pragma unroll
        for (int m = 0; m < Z2; ++m) y[m] = line[blk * Z2 + m];
        dftR<C, -1, Z2>(y);
#pragma unroll
        for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = y[m];
      }
    }
    __syncthreads();
    if (live) {
#pragma unroll 1
      for (int J = t; J < Z2; J += TW) {
        C x[Z1];
#pragma unroll
        for (int m = 0; m < Z1; ++m) x[m] = line[J + Z2 * m];
        if (J) {
#pragma unroll
          for (int m = 1; m < Z1; ++m) x[m] = cmul(x[m], __ldg(&twz[J * (Z1 - 1) + m - 1]));
        }
        dftR<C, -1, Z1>(x);
#pragma unroll
        for (int a = 0; a < Z1; ++a) line[J + Z2 * a] = x[a];
      }
    }
    __syncthreads();
  }
  // gather the plane's coefficients, one warp per row (coalesced reads and writes), with the
  // kinetic term (and the recurrence); Y_k and t_G from the prefetched blocks
  before_gather();
  __syncthreads();
  for (int row = w; row < nr; row += blockDim.x >> 5) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    const C* line = F + pmod(sp.row_k[r0 + row], N2) * FP;
    int lz = pmod(l0 + lane, N3);
    for (int idx = lane; idx < cnt; idx += 32, lz = wrap_n<N3>(lz, 32 % N3)) {
      const C v = line[lz];
      const int gg = g0 + idx;
      const C yy = Sy[gg - pg0];
      const T k = Sk[gg - pg0];
      if constexpr (!REC) {
        o[gg] = mk<C>(k * yy.x + v.x, k * yy.y + v.y);
      } else {
        const C pz = ((const C*)rec.pz)[(int64_t)b * rec.ldpz + gg];
        C r = mk<C>(ra * (k * yy.x + v.x + pz.x - rs * yy.x), ra * (k * yy.y + v.y + pz.y - rs * yy.y));
        if (rec.ykm1) {
          const C ym = ((const C*)rec.ykm1)[(int64_t)b * rec.ldykm1 + gg];
          r.x -= (T)rec.beta * ym.x;
          r.y -= (T)rec.beta * ym.y;
        }
        o[gg] = r;
        if (rec.split) {
          __nv_bfloat16* sb = (__nv_bfloat16*)rec.split + (int64_t)b * rec.split_ld + 2 * (int64_t)gg;
          float re = (float)r.x, im = (float)r.y;
          for (int pc = 0; pc < rec.pieces; ++pc) {
            const __nv_bfloat16 hr = __float2bfloat16_rn(re), hi = __float2bfloat16_rn(im);
            __nv_bfloat162 two;
            two.x = hr;
            two.y = hi;
            *reinterpret_cast<__nv_bfloat162*>(sb + (int64_t)pc * rec.split_piece_stride) = two;
            re -= __bfloat162float(hr);
            im -= __bfloat162float(hi);
          }
        }
      }
    }
  }
}

// copies of a plane's blocks of Y_k (band b) and of t_G into Sy, Sk (one committed group)
template <typename C, typename T>
__device__ __forceinline__ void plane_fwd_stage(const SphereDev& sp, int p, int b, const C* psi, int64_t ldpsi,
                                                const T* kin, C* Sy, T* Sk) {
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const int pg0 = nr > 0 ? sp.row_g0[r0] : 0;
  const int pcnt = nr > 0 ? sp.row_g0[r0 + nr - 1] + sp.row_cnt[r0 + nr - 1] - pg0 : 0;
  const C* yb = psi + (int64_t)b * ldpsi + pg0;
  for (int i = threadIdx.x; i < pcnt; i += blockDim.x) {
    cp_async_el<sizeof(C)>(Sy + i, yb + i);
    cp_async_el<sizeof(T)>(Sk + i, kin + pg0 + i);
  }
  cp_async_commit();
}

// one CTA per (plane, band): the plane's blocks of Y_k and t_G are copied while the y- and
// z-lines are transformed
template <typename T, int N2, int N3, int TW, bool REC>
__global__ void __launch_bounds__(PlaneW<N2, N3, TW>::THREADS) k_plane_fwd_wg(const cplx<T>* __restrict__ hb,
                                                                               int64_t hb_bs, SphereDev sp, FftPlan plan,
                                                                               const cplx<T>* __restrict__ tw,
                                                                               const T* __restrict__ kin,
                                                                               const cplx<T>* __restrict__ psi,
                                                                               int64_t ldpsi, cplx<T>* __restrict__ out,
                                                                               int64_t ldout, Pass3Rec rec) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Sy = reinterpret_cast<C*>(smem_raw + plane_wg_stage_off<C, N2, N3, TW>());
  T* Sk = reinterpret_cast<T*>(Sy + sp.max_plane_g);
  const int p = blockIdx.x, b = blockIdx.y;
  plane_fwd_stage<C, T>(sp, p, b, psi, ldpsi, kin, Sy, Sk);
  plane_fwd_wg_item<T, N2, N3, TW, REC>(p, b, hb, hb_bs, sp, plan, tw, psi, ldpsi, out, ldout, rec, Sy, Sk,
                                        [] { cp_async_wait<0>(); });
}

// Persistent form: one CTA per SM walks the (plane, band) items; while an item's coefficients
// are gathered, the next item's half-box plane is prefetched into L2 (one bulk prefetch of the
// contiguous plane) and its blocks of Y_k and t_G are copied into the other of two buffers.
template <typename T, int N2, int N3, int TW, bool REC>
__global__ void __launch_bounds__(PlaneW<N2, N3, TW>::THREADS) k_plane_fwd_wgp(const cplx<T>* __restrict__ hb,
                                                                                int64_t hb_bs, SphereDev sp,
                                                                                FftPlan plan,
                                                                                const cplx<T>* __restrict__ tw,
                                                                                const T* __restrict__ kin,
                                                                                const cplx<T>* __restrict__ psi,
                                                                                int64_t ldpsi, cplx<T>* __restrict__ out,
                                                                                int64_t ldout, Pass3Rec rec, int nb) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Sy0 = reinterpret_cast<C*>(smem_raw + plane_wg_stage_off<C, N2, N3, TW>());
  T* Sk0 = reinterpret_cast<T*>(Sy0 + 2 * (size_t)sp.max_plane_g);
  const int nitems = sp.nplane * nb;
  int buf = 0;
  if ((int)blockIdx.x < nitems)
    plane_fwd_stage<C, T>(sp, blockIdx.x % sp.nplane, blockIdx.x / sp.nplane, psi, ldpsi, kin, Sy0, Sk0);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x, buf ^= 1) {
    const int p = it % sp.nplane, b = it / sp.nplane;
    const int nxt = it + gridDim.x;
    C* Sy = Sy0 + (size_t)buf * sp.max_plane_g;
    T* Sk = Sk0 + (size_t)buf * sp.max_plane_g;
    plane_fwd_wg_item<T, N2, N3, TW, REC>(p, b, hb, hb_bs, sp, plan, tw, psi, ldpsi, out, ldout, rec, Sy, Sk, [&] {
      if (nxt < nitems) {
        const int pn = nxt % sp.nplane, bn = nxt / sp.nplane;
        if (threadIdx.x == 0) {
          const C* plane = hb + (int64_t)bn * hb_bs + (int64_t)pn * N2 * N3;
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(plane), "r"((unsigned)(sizeof(C) * N2 * N3))
                       : "memory");
        }
        // the other buffer was released by the barrier that ended the previous item
        plane_fwd_stage<C, T>(sp, pn, bn, psi, ldpsi, kin, Sy0 + (size_t)(buf ^ 1) * sp.max_plane_g,
                              Sk0 + (size_t)(buf ^ 1) * sp.max_plane_g);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    });
    __syncthreads();  // the plane, the row map and this buffer are reused two items later
  }
}

template <typename T, int N2, int N3, int TW>
static size_t plane_wg_smem(const SphereDev& sp, int which, bool persist = false) {
  // plane, row map; pass 3 also the prefetched blocks of Y_k and t_G of its plane (two of each
  // in the persistent form)
  return which ? plane_wg_stage_off<cplx<T>, N2, N3, TW>() +
                     (persist ? 2 : 1) * (sizeof(cplx<T>) + sizeof(T)) * (size_t)sp.max_plane_g
               : sizeof(cplx<T>) * (size_t)N2 * PlaneW<N2, N3, TW>::FP + sizeof(int) * N2;
}

template <typename T, int N2, int N3, int TW>
static cudaError_t plane_wg_pair(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                                 const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, const T* kin,
                                 cplx<T>* out, int64_t ldout, int nb, cudaStream_t st, const Pass3Rec* rec,
                                 bool persist) {
  using PW = PlaneW<N2, N3, TW>;
  if constexpr (!PW::ok) {
    return cudaErrorNotSupported;
  } else {
    const size_t sm = plane_wg_smem<T, N2, N3, TW>(sp, which, persist && which == 1);
    if (sm > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e;
    if (which == 1 && persist) {
      int nsm = 152, dev = 0;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      // as many resident CTAs as the SMs hold (one on 120 x 120 planes, more on smaller ones)
      auto grid_of = [&](const void* fn) {
        int per = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, PW::THREADS, sm) != cudaSuccess || per < 1) per = 1;
        return std::max(1, std::min(sp.nplane * nb, nsm * per));
      };
      if (rec) {
        if constexpr (std::is_same<T, float>::value) {
          if ((e = cudaFuncSetAttribute(k_plane_fwd_wgp<T, N2, N3, TW, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
            return e;
          const int grid = grid_of((const void*)k_plane_fwd_wgp<T, N2, N3, TW, true>);
          k_plane_fwd_wgp<T, N2, N3, TW, true><<<grid, PW::THREADS, sm, st>>>(hb, hb_bs, sp, plan, tw, kin, psi,
                                                                             ldpsi, out, ldout, *rec, nb);
          count_launch();
        } else {
          return cudaErrorNotSupported;
        }
      } else {
        if ((e = cudaFuncSetAttribute(k_plane_fwd_wgp<T, N2, N3, TW, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
          return e;
        const int grid = grid_of((const void*)k_plane_fwd_wgp<T, N2, N3, TW, false>);
        k_plane_fwd_wgp<T, N2, N3, TW, false><<<grid, PW::THREADS, sm, st>>>(hb, hb_bs, sp, plan, tw, kin, psi,
                                                                            ldpsi, out, ldout, Pass3Rec{}, nb);
        count_launch();
      }
      return cudaGetLastError();
    }
    if (which == 0 && persist) {
      int nsm = 152, dev = 0, per = 1;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if ((e = cudaFuncSetAttribute(k_plane_inv_wgp<T, N2, N3, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm)))
        return e;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_plane_inv_wgp<T, N2, N3, TW>, PW::THREADS, sm) !=
              cudaSuccess || per < 1)
        per = 1;
      const int grid = std::max(1, std::min(sp.nplane * nb, nsm * per));
      k_plane_inv_wgp<T, N2, N3, TW><<<grid, PW::THREADS, sm, st>>>(psi, ldpsi, hb, hb_bs, sp, plan, tw, nb);
      count_launch();
      return cudaGetLastError();
    }
    if (which == 0) {
      if ((e = cudaFuncSetAttribute(k_plane_inv_wg<T, N2, N3, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm)))
        return e;
      if ((e = cudaFuncSetAttribute(k_plane_inv_wg<T, N2, N3, TW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    100)))
        return e;
      k_plane_inv_wg<T, N2, N3, TW><<<dim3(sp.nplane, nb), PW::THREADS, sm, st>>>(psi, ldpsi, hb, hb_bs, sp, plan,
                                                                                 tw); count_launch();
    } else {
      if (rec) {
        if constexpr (std::is_same<T, float>::value) {
          if ((e = cudaFuncSetAttribute(k_plane_fwd_wg<T, N2, N3, TW, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
            return e;
          if ((e = cudaFuncSetAttribute(k_plane_fwd_wg<T, N2, N3, TW, true>,
                                        cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
            return e;
          k_plane_fwd_wg<T, N2, N3, TW, true><<<dim3(sp.nplane, nb), PW::THREADS, sm, st>>>(
              hb, hb_bs, sp, plan, tw, kin, psi, ldpsi, out, ldout, *rec); count_launch();
        } else {
          return cudaErrorNotSupported;
        }
      } else {
        if ((e = cudaFuncSetAttribute(k_plane_fwd_wg<T, N2, N3, TW, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
          return e;
        if ((e = cudaFuncSetAttribute(k_plane_fwd_wg<T, N2, N3, TW, false>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
          return e;
        k_plane_fwd_wg<T, N2, N3, TW, false><<<dim3(sp.nplane, nb), PW::THREADS, sm, st>>>(
            hb, hb_bs, sp, plan, tw, kin, psi, ldpsi, out, ldout, Pass3Rec{}); count_launch();
      }
    }
    return cudaGetLastError();
  }
}

template <typename T>
static cudaError_t plane_wg(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                            const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, const T* kin, cplx<T>* out,
                            int64_t ldout, int nb, cudaStream_t st, const Pass3Rec* rec = nullptr,
                            bool persist = false) {
  const int n2 = plan.n[1], n3 = plan.n[2];
#define PW_WG_CASE(A, B, TWN)                                                                                  \
  if (n2 == A && n3 == B)                                                                                      \
    return plane_wg_pair<T, A, B, TWN>(which, psi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out, ldout, nb, st, rec, \
                                       persist);
  PW_WG_CASE(24, 24, 4)
  PW_WG_CASE(64, 64, 4)
  PW_WG_CASE(72, 90, 4)
  PW_WG_CASE(96, 96, 4)
  PW_WG_CASE(120, 120, 8)
#undef PW_WG_CASE
  return cudaErrorNotSupported;
}

// Plane passes with a compact row buffer and 32-column slices (plane form 3).  The CTA keeps
// only the plane's sphere rows R[nr][N3 + 1] (the z-lines) and one slice S[N2][33] of 32
// y-columns at a time, instead of the whole N2 x N3 plane: on a 120^3 box that is 88 KB
// instead of 117 KB, so that two CTAs share an SM and one CTA's loads overlap the other's
// butterflies.  Lane = line in both stages, the TW warps of the CTA split the butterflies by
// index mod TW; the y-lines of a slice go through S, the z-lines stay in R.
template <int N2, int N3, int TW> struct PlaneR {
  static constexpr CPlan P2 = make_cplan(N2), P3 = make_cplan(N3);
  static constexpr int FR = N3 + 1;
  static constexpr int SP = 33;
  static constexpr int NSL = (N3 + 31) / 32;
  static constexpr int THREADS = 32 * TW;
  static constexpr bool ok = (P2.nst == 2 && P3.nst == 2);
};

template <typename T, int N2, int N3, int TW>
__global__ void __launch_bounds__(PlaneR<N2, N3, TW>::THREADS) k_plane_inv_rs(const cplx<T>* __restrict__ psi,
                                                                               int64_t ldpsi, cplx<T>* __restrict__ hb,
                                                                               int64_t hb_bs, SphereDev sp, FftPlan plan,
                                                                               const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using PR = PlaneR<N2, N3, TW>;
  constexpr int FR = PR::FR, SP = PR::SP;
  constexpr int Y1 = PR::P2.radix[0], Y2 = PR::P2.radix[1];
  constexpr int Z1 = PR::P3.radix[0], Z2 = PR::P3.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  C* S = R + (size_t)sp.max_rows * FR;
  int* ymap = reinterpret_cast<int*>(S + N2 * SP);
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* src = psi + (int64_t)b * ldpsi;
  const C* twy = tw + plan.d[1].tw_off[0];
  const C* twz = tw + plan.d[2].tw_off[0];
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  // z-lines of the sphere rows into R, 32 rows at a time; the first stage reads the row's run
  // of coefficients straight from the block
  for (int c0 = 0; c0 < nr; c0 += 32) {
    const int row = c0 + lane;
    const bool live = row < nr;
    C* line = R + (size_t)(live ? row : 0) * FR;
    if (live) {
      const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
#pragma unroll 1
      for (int J = t; J < Z2; J += TW) {
        C x[Z1];
#pragma unroll
        for (int a = 0; a < Z1; ++a) {
          const int idx = pmod(J + Z2 * a - l0, N3);
          x[a] = idx < cnt ? src[g0 + idx] : czero<C>();
        }
        dftR<C, +1, Z1>(x);
        if (J) {
#pragma unroll
          for (int m = 1; m < Z1; ++m) x[m] = cmul(x[m], cconj(__ldg(&twz[J * (Z1 - 1) + m - 1])));
        }
#pragma unroll
        for (int m = 0; m < Z1; ++m) line[J + Z2 * m] = x[m];
      }
    }
    __syncthreads();
    if (live) {
#pragma unroll 1
      for (int blk = t; blk < Z1; blk += TW) {
        C y[Z2];
#pragma unroll
        for (int m = 0; m < Z2; ++m) y[m] = line[blk * Z2 + m];
        dftR<C, +1, Z2>(y);
#pragma unroll
        for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = y[m];
      }
    }
  }
  __syncthreads();
  // y-lines, one slice of 32 columns at a time; rows without coefficients read as zero
  C* dst = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  C* col = S + lane;
#pragma unroll 1
  for (int sc = 0; sc < PR::NSL; ++sc) {
    const int c = sc * 32 + lane;
    const bool livec = c < N3;
#pragma unroll 1
    for (int J = t; J < Y2; J += TW) {
      C x[Y1];
#pragma unroll
      for (int a = 0; a < Y1; ++a) {
        const int i = ymap[J + Y2 * a];
        x[a] = (livec && i >= 0) ? R[(size_t)i * FR + c] : czero<C>();
      }
      dftR<C, +1, Y1>(x);
      if (J) {
#pragma unroll
        for (int m = 1; m < Y1; ++m) x[m] = cmul(x[m], cconj(__ldg(&twy[J * (Y1 - 1) + m - 1])));
      }
#pragma unroll
      for (int m = 0; m < Y1; ++m) col[(J + Y2 * m) * SP] = x[m];
    }
    __syncthreads();
#pragma unroll 1
    for (int blk = t; blk < Y1; blk += TW) {
      C y[Y2];
#pragma unroll
      for (int m = 0; m < Y2; ++m) y[m] = col[(blk * Y2 + m) * SP];
      dftR<C, +1, Y2>(y);
      if (livec) {
#pragma unroll
        for (int m = 0; m < Y2; ++m) dst[(int64_t)(blk * Y2 + m) * N3 + c] = y[m];
      }
    }
    __syncthreads();
  }
}

template <typename T, int N2, int N3, int TW, bool REC>
__global__ void __launch_bounds__(PlaneR<N2, N3, TW>::THREADS) k_plane_fwd_rs(const cplx<T>* __restrict__ hb,
                                                                               int64_t hb_bs, SphereDev sp, FftPlan plan,
                                                                               const cplx<T>* __restrict__ tw,
                                                                               const T* __restrict__ kin,
                                                                               const cplx<T>* __restrict__ psi,
                                                                               int64_t ldpsi, cplx<T>* __restrict__ out,
                                                                               int64_t ldout, Pass3Rec rec) {
  using C = cplx<T>;
  using PR = PlaneR<N2, N3, TW>;
  constexpr int FR = PR::FR, SP = PR::SP;
  constexpr int Y1 = PR::P2.radix[0], Y2 = PR::P2.radix[1];
  constexpr int Z1 = PR::P3.radix[0], Z2 = PR::P3.radix[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  C* S = R + (size_t)sp.max_rows * FR;
  int* ymap = reinterpret_cast<int*>(S + N2 * SP);
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  const int p = blockIdx.x, b = blockIdx.y;
  const int r0 = sp.plane_row0[p], nr = sp.plane_row0[p + 1] - r0;
  const C* srcp = hb + (int64_t)b * hb_bs + (int64_t)p * N2 * N3;
  const C* twy = tw + plan.d[1].tw_off[0];
  const C* twz = tw + plan.d[2].tw_off[0];
  for (int i = threadIdx.x; i < N2; i += blockDim.x) ymap[i] = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < nr; i += blockDim.x) ymap[pmod(sp.row_k[r0 + i], N2)] = i;
  __syncthreads();
  // y-lines, one slice of 32 columns at a time: radix Y2 blocks read from the half-box plane,
  // then radix Y1 with twiddles; only the sphere rows are kept (in R)
  C* col = S + lane;
#pragma unroll 1
  for (int sc = 0; sc < PR::NSL; ++sc) {
    const int c = sc * 32 + lane;
    const bool livec = c < N3;
#pragma unroll 1
    for (int blk = t; blk < Y1; blk += TW) {
      C y[Y2];
#pragma unroll
      for (int m = 0; m < Y2; ++m) y[m] = livec ? srcp[(int64_t)(blk * Y2 + m) * N3 + c] : czero<C>();
      dftR<C, -1, Y2>(y);
#pragma unroll
      for (int m = 0; m < Y2; ++m) col[(blk * Y2 + m) * SP] = y[m];
    }
    __syncthreads();
#pragma unroll 1
    for (int J = t; J < Y2; J += TW) {
      C x[Y1];
#pragma unroll
      for (int m = 0; m < Y1; ++m) x[m] = col[(J + Y2 * m) * SP];
      if (J) {
#pragma unroll
        for (int m = 1; m < Y1; ++m) x[m] = cmul(x[m], __ldg(&twy[J * (Y1 - 1) + m - 1]));
      }
      dftR<C, -1, Y1>(x);
#pragma unroll
      for (int a = 0; a < Y1; ++a) {
        const int i = ymap[J + Y2 * a];
        if (livec && i >= 0) R[(size_t)i * FR + c] = x[a];
      }
    }
    __syncthreads();
  }
  // z-lines of the sphere rows, 32 rows at a time, in place in R
  for (int c0 = 0; c0 < nr; c0 += 32) {
    const int row = c0 + lane;
    const bool live = row < nr;
    C* line = R + (size_t)(live ? row : 0) * FR;
    if (live) {
#pragma unroll 1
      for (int blk = t; blk < Z1; blk += TW) {
        C y[Z2];
#pragma unroll
        for (int m = 0; m < Z2; ++m) y[m] = line[blk * Z2 + m];
        dftR<C, -1, Z2>(y);
#pragma unroll
        for (int m = 0; m < Z2; ++m) line[blk * Z2 + m] = y[m];
      }
    }
    __syncthreads();
    if (live) {
#pragma unroll 1
      for (int J = t; J < Z2; J += TW) {
        C x[Z1];
#pragma unroll
        for (int m = 0; m < Z1; ++m) x[m] = line[J + Z2 * m];
        if (J) {
#pragma unroll
          for (int m = 1; m < Z1; ++m) x[m] = cmul(x[m], __ldg(&twz[J * (Z1 - 1) + m - 1]));
        }
        dftR<C, -1, Z1>(x);
#pragma unroll
        for (int a = 0; a < Z1; ++a) line[J + Z2 * a] = x[a];
      }
    }
    __syncthreads();
  }
  // gather the plane's coefficients, one warp per row (coalesced reads and writes), with the
  // kinetic term (and the recurrence)
  const C* yv = psi + (int64_t)b * ldpsi;
  C* o = out + (int64_t)b * ldout;
  T ra = 0, rs = 0;  // recurrence alpha and shift
  if constexpr (REC) {
    ra = (T)rec.alpha;
    rs = (T)rec.shift;
    if (rec.dev_ce) {
      rs = (T)rec.dev_ce[0];
      ra = (T)((rec.first ? 1.0 : 2.0) / rec.dev_ce[1]);
    }
  }
  for (int row = t; row < nr; row += TW) {
    const int g0 = sp.row_g0[r0 + row], cnt = sp.row_cnt[r0 + row], l0 = sp.row_l0[r0 + row];
    const C* line = R + (size_t)row * FR;
    int lz = pmod(l0 + lane, N3);
    for (int idx = lane; idx < cnt; idx += 32, lz = wrap_n<N3>(lz, 32 % N3)) {
      const C v = line[lz];
      const int gg = g0 + idx;
      const C yy = yv[gg];
      const T k = kin[gg];
      if constexpr (!REC) {
        o[gg] = mk<C>(k * yy.x + v.x, k * yy.y + v.y);
      } else {
        const C pz = ((const C*)rec.pz)[(int64_t)b * rec.ldpz + gg];
        C r = mk<C>(ra * (k * yy.x + v.x + pz.x - rs * yy.x), ra * (k * yy.y + v.y + pz.y - rs * yy.y));
        if (rec.ykm1) {
          const C ym = ((const C*)rec.ykm1)[(int64_t)b * rec.ldykm1 + gg];
          r.x -= (T)rec.beta * ym.x;
          r.y -= (T)rec.beta * ym.y;
        }
        o[gg] = r;
        if (rec.split) {
          __nv_bfloat16* sb = (__nv_bfloat16*)rec.split + (int64_t)b * rec.split_ld + 2 * (int64_t)gg;
          float re = (float)r.x, im = (float)r.y;
          for (int pc = 0; pc < rec.pieces; ++pc) {
            const __nv_bfloat16 hr = __float2bfloat16_rn(re), hi = __float2bfloat16_rn(im);
            __nv_bfloat162 two;
            two.x = hr;
            two.y = hi;
            *reinterpret_cast<__nv_bfloat162*>(sb + (int64_t)pc * rec.split_piece_stride) = two;
            re -= __bfloat162float(hr);
            im -= __bfloat162float(hi);
          }
        }
      }
    }
  }
}

template <typename T, int N2, int N3, int TW>
static size_t plane_rs_smem(const SphereDev& sp) {
  return sizeof(cplx<T>) * ((size_t)sp.max_rows * PlaneR<N2, N3, TW>::FR + (size_t)N2 * PlaneR<N2, N3, TW>::SP) +
         sizeof(int) * N2;
}

template <typename T, int N2, int N3, int TW>
static cudaError_t plane_rs_pair(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                                 const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, const T* kin,
                                 cplx<T>* out, int64_t ldout, int nb, cudaStream_t st, const Pass3Rec* rec) {
  using PR = PlaneR<N2, N3, TW>;
  constexpr bool kF32 = std::is_same<T, float>::value;
  if constexpr (!PR::ok) {
    return cudaErrorNotSupported;
  } else {
    // complex128 planes take twice the shared memory (174 KB on 120^3) and no fused recurrence
    if (!kF32 && rec) return cudaErrorNotSupported;
    const size_t sm = plane_rs_smem<T, N2, N3, TW>(sp);
    if (sm > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e;
    const dim3 grid(sp.nplane, nb);
    if (which == 0) {
      if ((e = cudaFuncSetAttribute(k_plane_inv_rs<T, N2, N3, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm)))
        return e;
      k_plane_inv_rs<T, N2, N3, TW><<<grid, PR::THREADS, sm, st>>>(psi, ldpsi, hb, hb_bs, sp, plan, tw); count_launch();
    } else if (rec) {
      if constexpr (kF32) {
        if ((e = cudaFuncSetAttribute(k_plane_fwd_rs<T, N2, N3, TW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm)))
          return e;
        k_plane_fwd_rs<T, N2, N3, TW, true><<<grid, PR::THREADS, sm, st>>>(hb, hb_bs, sp, plan, tw, kin, psi, ldpsi,
                                                                          out, ldout, *rec); count_launch();
      }
    } else {
      if ((e = cudaFuncSetAttribute(k_plane_fwd_rs<T, N2, N3, TW, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm)))
        return e;
      k_plane_fwd_rs<T, N2, N3, TW, false><<<grid, PR::THREADS, sm, st>>>(hb, hb_bs, sp, plan, tw, kin, psi, ldpsi,
                                                                         out, ldout, Pass3Rec{}); count_launch();
    }
    return cudaGetLastError();
  }
}

template <typename T>
static cudaError_t plane_rs(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                            const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, const T* kin, cplx<T>* out,
                            int64_t ldout, int nb, cudaStream_t st, const Pass3Rec* rec = nullptr) {
  const int n2 = plan.n[1], n3 = plan.n[2];
#define PW_RS_CASE(A, B, TWN)                                                                                  \
  if (n2 == A && n3 == B)                                                                                      \
    return plane_rs_pair<T, A, B, TWN>(which, psi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out, ldout, nb, st, rec);
  PW_RS_CASE(64, 64, 8)
  PW_RS_CASE(72, 90, 8)
  PW_RS_CASE(96, 96, 8)
  PW_RS_CASE(120, 120, 8)
#undef PW_RS_CASE
  return cudaErrorNotSupported;
}

static bool plane_wg_covers(const FftPlan& plan) {
  const int n2 = plan.n[1], n3 = plan.n[2];
  return (n2 == 24 && n3 == 24) || (n2 == 64 && n3 == 64) || (n2 == 72 && n3 == 90) || (n2 == 96 && n3 == 96) ||
         (n2 == 120 && n3 == 120);
}

template <typename T, int N1>
static cudaError_t launch_xline_tpl(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp,
                                    const FftPlan& plan, int nb, cudaStream_t st) {
  const size_t sm = sizeof(cplx<T>) * (size_t)N1 * kTplX;
  if (sm > 227 * 1024) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(k_xline_tpl<T, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  if ((e = cudaFuncSetAttribute(k_xline_tpl<T, N1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100))) return e;
  const int nyz = plan.n[1] * plan.n[2];
  k_xline_tpl<T, N1><<<dim3((nyz + kTplX - 1) / kTplX, nb), kTplX, sm, st>>>(hb, hb_bs, vperm, sp, plan); count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t xline_tpl(cplx<T>* hb, int64_t hb_bs, const T* vperm, const SphereDev& sp, const FftPlan& plan,
                             int nb, cudaStream_t st) {
  switch (plan.n[0]) {
    case 24: return launch_xline_tpl<T, 24>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 64: return launch_xline_tpl<T, 64>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 72: return launch_xline_tpl<T, 72>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 90: return launch_xline_tpl<T, 90>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 96: return launch_xline_tpl<T, 96>(hb, hb_bs, vperm, sp, plan, nb, st);
    case 120: return launch_xline_tpl<T, 120>(hb, hb_bs, vperm, sp, plan, nb, st);
    default: return cudaErrorNotSupported;
  }
}

template <typename T, int N2, int N3>
static size_t plane_tpl_smem() {
  return sizeof(cplx<T>) * (size_t)N2 * PlaneT<N2, N3>::FP + sizeof(int) * N2;
}

template <typename T, int N2, int N3>
static cudaError_t plane_tpl_pair(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                                  const SphereDev& sp, const T* kin, cplx<T>* out, int64_t ldout, int nb,
                                  cudaStream_t st) {
  using PT = PlaneT<N2, N3>;
  if constexpr (!PT::ok) {
    return cudaErrorNotSupported;
  } else {
    const size_t sm = plane_tpl_smem<T, N2, N3>();
    if (sm > 227 * 1024 || sp.max_rows > PT::THREADS * 4) return cudaErrorNotSupported;
    cudaError_t e;
    if (which == 0) {
      if ((e = cudaFuncSetAttribute(k_plane_inv_tpl<T, N2, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
        return e;
      if ((e = cudaFuncSetAttribute(k_plane_inv_tpl<T, N2, N3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
        return e;
      k_plane_inv_tpl<T, N2, N3><<<dim3(sp.nplane, nb), PT::THREADS, sm, st>>>(psi, ldpsi, hb, hb_bs, sp); count_launch();
    } else {
      if ((e = cudaFuncSetAttribute(k_plane_fwd_tpl<T, N2, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
        return e;
      if ((e = cudaFuncSetAttribute(k_plane_fwd_tpl<T, N2, N3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)))
        return e;
      k_plane_fwd_tpl<T, N2, N3><<<dim3(sp.nplane, nb), PT::THREADS, sm, st>>>(hb, hb_bs, sp, kin, psi, ldpsi, out,
                                                                             ldout); count_launch();
    }
    return cudaGetLastError();
  }
}

template <typename T>
static cudaError_t plane_tpl(int which, const cplx<T>* psi, int64_t ldpsi, cplx<T>* hb, int64_t hb_bs,
                             const SphereDev& sp, const FftPlan& plan, const T* kin, cplx<T>* out, int64_t ldout,
                             int nb, cudaStream_t st) {
  const int n2 = plan.n[1], n3 = plan.n[2];
#define PW_TPL_CASE(A, B) \
  if (n2 == A && n3 == B) return plane_tpl_pair<T, A, B>(which, psi, ldpsi, hb, hb_bs, sp, kin, out, ldout, nb, st);
  PW_TPL_CASE(24, 24)
  PW_TPL_CASE(64, 64)
  PW_TPL_CASE(72, 90)
  PW_TPL_CASE(96, 96)
  PW_TPL_CASE(120, 120)
#undef PW_TPL_CASE
  return cudaErrorNotSupported;
}

// ---- launchers ------------------------------------------------------------------
cudaError_t fft_set_constants() {
  const int Rs[6] = {6, 9, 10, 12, 15, 16};
  double2 t64[68];
  float2 t32[68];
  int o = 0;
  for (int r : Rs)
    for (int m = 0; m < r; ++m, ++o) {
      const double ang = -2.0 * 3.14159265358979323846264338327950288 * (double)m / (double)r;
      t64[o] = make_double2(cos(ang), sin(ang));
      t32[o] = make_float2((float)t64[o].x, (float)t64[o].y);
    }
  cudaError_t e = cudaMemcpyToSymbol(c_wtab64, t64, sizeof(t64));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wtab32, t32, sizeof(t32));
  return e;
}

static int pick_cz(int n3) { return n3 < 16 ? n3 : 16; }

template <typename T>
static size_t plane_smem(const FftPlan& plan, const SphereDev& sp, int cz) {
  return sizeof(cplx<T>) * ((size_t)sp.max_rows * plan.n[2] + (size_t)cz * (plan.n[1] + 1));
}

template <typename T>
cudaError_t launch_local_apply(const FftPlan& plan, const cplx<T>* tw, const SphereDev& sp,
                               const T* vperm, const T* kin, const cplx<T>* psi, int64_t ldpsi,
                               int nband, cplx<T>* out, int64_t ldout, cplx<T>* hb, int band_batch,
                               cudaStream_t st, ::pw_ctx* prof) {
  if (nband <= 0) return cudaSuccess;
  const int cz = pick_cz(plan.n[2]);
  const int lyz = 32;
  const size_t sm1 = plane_smem<T>(plan, sp, cz);
  const size_t sm2 = sizeof(cplx<T>) * (size_t)plan.n[0] * lyz;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_plane_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1))) return e;
  if ((e = cudaFuncSetAttribute(k_plane_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1))) return e;
  if ((e = cudaFuncSetAttribute(k_xline<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2))) return e;
  const int64_t hb_bs = (int64_t)sp.nplane * plan.n[1] * plan.n[2];
  const int nyz = plan.n[1] * plan.n[2];
  // one-thread-per-line kernels: complex64 only (a complex128 line per thread needs twice
  // the shared memory per CTA), when the context selected them
  // kernel forms (complex64): x-line form = variant % 16 (0 line groups, 1 one thread per
  // line, 2 warp groups with compile-time twiddles, 3 warp groups with table twiddles, 4 the
  // same with several bands per CTA, 5 and 6 as 3 and 4 with the two radices of the line's
  // plan in the other order, 7-10 as 3-6 with the planes staged by asynchronous copies, the
  // multi-band forms double-buffered), plane form = variant / 16 (0 line groups, 1 one thread
  // per line, 2 warp groups over the whole plane, 3 warp groups over sphere rows and 32-column
  // slices, 4 = 3 for pass 1 and 2 for pass 3)
  // complex128: only the plane form is selectable (0 line groups, 3 sphere rows + column
  // slices); the x-line pass keeps the line-group form
  const int fv = prof ? prof->fft_variant[std::is_same<T, float>::value ? 0 : 1] : 0;
  int xf = std::is_same<T, float>::value ? fv % kFormStride : 0;
  const int pf = fv / kFormStride;
  // the swapped-radix x-line forms need V permuted for that order: the context's potential
  // has such a copy, an arbitrary potential (pw_local_apply) takes the unswapped form; the
  // fallbacks for lengths those forms do not cover keep the usual permutation
  const T* vperm_x = vperm;
  if (xf_swap(xf)) {
    if (prof && prof->vperm32_sw && (const void*)vperm == (const void*)prof->vperm32)
      vperm_x = (const T*)prof->vperm32_sw;
    else xf -= 2;
  }
  // plane form 4: pass 1 over sphere rows + column slices, pass 3 over the whole plane; 5 the
  // same with the persistent pass 3 (next plane prefetched); 6 both passes whole-plane and
  // persistent
  const bool tpl = pf == 1, pwg = pf == 2 || pf == 6, prs = pf == 3, pmix = pf == 4 || pf == 5;
  const bool ppers = pf == 5 || pf == 6, ipers = pf == 6;
  const bool xtw = xf == 2, xtwr = xf_twr(xf);
  for (int b0 = 0; b0 < nband; b0 += band_batch) {
    const int nb = min(band_batch, nband - b0);
    prof_begin(prof, PW_PROF_PLANE_INV);
    e = cudaErrorNotSupported;
    if constexpr (std::is_same<T, float>::value) {
      if (tpl) e = plane_tpl<T>(0, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, kin, nullptr, 0, nb, st);
      if (pwg) e = plane_wg<T>(0, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, nullptr, 0, nb, st, nullptr,
                               ipers);
    }
    if (prs || pmix) e = plane_rs<T>(0, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, nullptr, 0, nb, st);
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      e = plane_lg<T>(0, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, nullptr, 0, nb, st);
    }
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      k_plane_inv<T><<<dim3(sp.nplane, nb), kThreads, sm1, st>>>(psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, cz); count_launch();
    } else if (e != cudaSuccess) {
      return e;
    }
    prof_end(prof, PW_PROF_PLANE_INV);
    prof_begin(prof, PW_PROF_XLINE);
    e = cudaErrorNotSupported;
    if constexpr (std::is_same<T, float>::value) {
      if (xtw) e = xline_tw<T>(hb, hb_bs, vperm, sp, plan, nb, st);
      if (xtwr)
        e = xline_twr<T>(hb, hb_bs, xf_swap(xf) ? vperm_x : vperm, sp, plan, tw, nb, xf_multi(xf), st, xf_swap(xf),
                         xf_staged(xf));
      if (xf == 1) {
        (void)cudaGetLastError();
        e = xline_tpl<T>(hb, hb_bs, vperm, sp, plan, nb, st);
      }
    }
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      e = xline_lg<T>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    }
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      k_xline<T><<<dim3((nyz + lyz - 1) / lyz, nb), kThreads, sm2, st>>>(hb, hb_bs, vperm, sp, plan, tw, lyz); count_launch();
    } else if (e != cudaSuccess) {
      return e;
    }
    prof_end(prof, PW_PROF_XLINE);
    prof_begin(prof, PW_PROF_PLANE_FWD);
    e = cudaErrorNotSupported;
    if constexpr (std::is_same<T, float>::value) {
      if (tpl) e = plane_tpl<T>(1, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, kin, out + b0 * ldout, ldout, nb, st);
      if (pwg || pmix)
        e = plane_wg<T>(1, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out + b0 * ldout, ldout, nb, st,
                        nullptr, ppers);
    }
    if (prs)
      e = plane_rs<T>(1, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out + b0 * ldout, ldout, nb, st);
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      e = plane_lg<T>(1, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out + b0 * ldout, ldout, nb, st);
    }
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      k_plane_fwd<T><<<dim3(sp.nplane, nb), kThreads, sm1, st>>>(hb, hb_bs, sp, plan, tw, cz, kin,
                                                                  psi + b0 * ldpsi, ldpsi, out + b0 * ldout, ldout); count_launch();
    } else if (e != cudaSuccess) {
      return e;
    }
    prof_end(prof, PW_PROF_PLANE_FWD);
  }
  return cudaGetLastError();
}

static bool plane_rs_covers(const FftPlan& plan) {
  const int n2 = plan.n[1], n3 = plan.n[2];
  return (n2 == 64 && n3 == 64) || (n2 == 72 && n3 == 90) || (n2 == 96 && n3 == 96) || (n2 == 120 && n3 == 120);
}

bool local_apply_rec_supported(const FftPlan& plan, const ::pw_ctx* prof) {
  if (!prof) return false;
  const int pf = prof->fft_variant[0] / kFormStride;
  return ((pf == 2 || pf == 6) && plane_wg_covers(plan)) || (pf == 3 && plane_rs_covers(plan)) ||
         ((pf == 4 || pf == 5) && plane_wg_covers(plan) && plane_rs_covers(plan));
}

cudaError_t launch_local_apply_rec(const FftPlan& plan, const float2* tw, const SphereDev& sp, const float* vperm,
                                   const float* kin, const float2* psi, int64_t ldpsi, int nband, float2* out,
                                   int64_t ldout, float2* hb, int band_batch, cudaStream_t st, ::pw_ctx* prof,
                                   const Pass3Rec& rec) {
  using T = float;
  if (!local_apply_rec_supported(plan, prof)) return cudaErrorNotSupported;
  if (nband <= 0) return cudaSuccess;
  int xf = prof->fft_variant[0] % kFormStride;
  const float* vperm_x = vperm;
  if (xf_swap(xf)) {
    if (prof->vperm32_sw && vperm == prof->vperm32) vperm_x = prof->vperm32_sw;
    else xf -= 2;
  }
  const int pfr = prof->fft_variant[0] / kFormStride;
  const bool prs = pfr == 3, inv_rs = pfr == 3 || pfr == 4 || pfr == 5, fwd_pers = pfr == 5 || pfr == 6;
  const bool inv_pers = pfr == 6;
  const int64_t hb_bs = (int64_t)sp.nplane * plan.n[1] * plan.n[2];
  const int nyz = plan.n[1] * plan.n[2];
  const int lyz = 32;
  const size_t sm2 = sizeof(cplx<T>) * (size_t)plan.n[0] * lyz;
  cudaError_t e;
  for (int b0 = 0; b0 < nband; b0 += band_batch) {
    const int nb = min(band_batch, nband - b0);
    prof_begin(prof, PW_PROF_PLANE_INV);
    e = inv_rs ? plane_rs<T>(0, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, nullptr, 0, nb, st, nullptr)
               : plane_wg<T>(0, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, nullptr, 0, nb, st, nullptr,
                             inv_pers);
    if (e) return e;
    prof_end(prof, PW_PROF_PLANE_INV);
    prof_begin(prof, PW_PROF_XLINE);
    e = cudaErrorNotSupported;
    if (xf == 2) e = xline_tw<T>(hb, hb_bs, vperm, sp, plan, nb, st);
    if (xf_twr(xf))
      e = xline_twr<T>(hb, hb_bs, xf_swap(xf) ? vperm_x : vperm, sp, plan, tw, nb, xf_multi(xf), st, xf_swap(xf),
                       xf_staged(xf));
    if (xf == 1) e = xline_tpl<T>(hb, hb_bs, vperm, sp, plan, nb, st);
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      e = xline_lg<T>(hb, hb_bs, vperm, sp, plan, tw, nb, st);
    }
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      if ((e = cudaFuncSetAttribute(k_xline<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2))) return e;
      k_xline<T><<<dim3((nyz + lyz - 1) / lyz, nb), kThreads, sm2, st>>>(hb, hb_bs, vperm, sp, plan, tw, lyz); count_launch();
      e = cudaGetLastError();
    }
    if (e) return e;
    prof_end(prof, PW_PROF_XLINE);
    prof_begin(prof, PW_PROF_PLANE_FWD);
    Pass3Rec r = rec;
    r.pz = rec.pz + b0 * rec.ldpz;
    if (rec.ykm1) r.ykm1 = rec.ykm1 + b0 * rec.ldykm1;
    if (rec.split) r.split = (__nv_bfloat16*)rec.split + b0 * rec.split_ld;
    e = prs ? plane_rs<T>(1, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out + b0 * ldout, ldout, nb, st,
                          &r)
            : plane_wg<T>(1, psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, kin, out + b0 * ldout, ldout, nb, st,
                          &r, fwd_pers);
    if (e) return e;
    prof_end(prof, PW_PROF_PLANE_FWD);
  }
  return cudaGetLastError();
}

// Density x-lines with groups of TW warps per 32 lines (lane = line), two-stage plans: each
// CTA takes 32 (y,z) lines and a share of the bands (blockIdx.y), transforms a (and b) per
// band, accumulates w_b Re[conj(a) b] per point in registers and adds its sums to the
// permuted grid atomically.  The planes sit at x-frequency p (a common shift of a and b
// multiplies both by the same phase, which the product cancels).
template <typename T, int N1, int TW>
__global__ void __launch_bounds__(32 * TW) k_xdens_wg(const cplx<T>* __restrict__ hba, const cplx<T>* __restrict__ hbb,
                                                     int64_t hb_bs, int nb, int bper, const T* __restrict__ w,
                                                     SphereDev sp, FftPlan plan, const cplx<T>* __restrict__ tw,
                                                     double* __restrict__ out_perm) {
  using C = cplx<T>;
  constexpr CPlan P = make_cplan(N1);
  static_assert(P.nst == 2, "two-stage plan expected");
  constexpr int R1 = P.radix[0], R2 = P.radix[1];
  constexpr int NBK = (R1 + TW - 1) / TW;  // stage-2 blocks per warp (at most)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  C* La = reinterpret_cast<C*>(smem_raw) + lane;
  C* Lb = La + N1 * 32;
  const int nyz = plan.n[1] * plan.n[2];
  const int yz = blockIdx.x * 32 + lane;
  const bool live = yz < nyz;
  const int np = sp.nplane;
  const bool two = hbb != nullptr;
  const C* tw1 = tw + plan.d[0].tw_off[0];
  double acc[NBK][R2];
#pragma unroll
  for (int i = 0; i < NBK; ++i)
#pragma unroll
    for (int m = 0; m < R2; ++m) acc[i][m] = 0.0;
  const int b_lo = blockIdx.y * bper, b_hi = min(nb, b_lo + bper);
  for (int b = b_lo; b < b_hi; ++b) {
    const C* ha = hba + (int64_t)b * hb_bs + (live ? yz : 0);
    const C* hbp = two ? hbb + (int64_t)b * hb_bs + (live ? yz : 0) : nullptr;
#pragma unroll 1
    for (int J = t; J < R2; J += TW) {
      for (int which = 0; which < (two ? 2 : 1); ++which) {
        const C* src = which ? hbp : ha;
        C* L = which ? Lb : La;
        C x[R1];
#pragma unroll
        for (int a = 0; a < R1; ++a) {
          const int p = J + R2 * a;
          x[a] = (live && p < np) ? src[(int64_t)p * nyz] : czero<C>();
        }
        dftR<C, +1, R1>(x);
        if (J) {
#pragma unroll
          for (int m = 1; m < R1; ++m) x[m] = cmul(x[m], cconj(__ldg(&tw1[J * (R1 - 1) + m - 1])));
        }
#pragma unroll
        for (int m = 0; m < R1; ++m) L[(J + R2 * m) * 32] = x[m];
      }
    }
    __syncthreads();
    const double wb = (double)w[b];
#pragma unroll
    for (int i = 0; i < NBK; ++i) {
      const int blk = t + TW * i;
      if (blk < R1) {
        C ya[R2], yb[R2];
#pragma unroll
        for (int m = 0; m < R2; ++m) ya[m] = La[(blk * R2 + m) * 32];
        dftR<C, +1, R2>(ya);
        if (two) {
#pragma unroll
          for (int m = 0; m < R2; ++m) yb[m] = Lb[(blk * R2 + m) * 32];
          dftR<C, +1, R2>(yb);
        }
#pragma unroll
        for (int m = 0; m < R2; ++m) {
          const C bv = two ? yb[m] : ya[m];
          acc[i][m] += wb * ((double)ya[m].x * (double)bv.x + (double)ya[m].y * (double)bv.y);
        }
      }
    }
    __syncthreads();
  }
  if (live && b_hi > b_lo) {
#pragma unroll
    for (int i = 0; i < NBK; ++i) {
      const int blk = t + TW * i;
      if (blk < R1) {
#pragma unroll
        for (int m = 0; m < R2; ++m) atomicAdd(&out_perm[(int64_t)(blk * R2 + m) * nyz + yz], acc[i][m]);
      }
    }
  }
}

template <typename T, int N1>
static cudaError_t launch_xdens_wg(const cplx<T>* hba, const cplx<T>* hbb, int64_t hb_bs, int nb, const T* w,
                                   const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, double* out_perm,
                                   cudaStream_t st) {
  constexpr int TW = 4;
  const size_t sm = sizeof(cplx<T>) * (size_t)N1 * 32 * (hbb ? 2 : 1);
  cudaError_t e = cudaFuncSetAttribute(k_xdens_wg<T, N1, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  if ((e = cudaFuncSetAttribute(k_xdens_wg<T, N1, TW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100))) return e;
  const int nyz = plan.n[1] * plan.n[2];
  const int gx = (nyz + 31) / 32;
  // enough CTAs for a few waves of the 152 SMs: split the bands
  int splits = std::max(1, std::min(nb, (152 * 6 + gx - 1) / gx));
  const int bper = (nb + splits - 1) / splits;
  splits = (nb + bper - 1) / bper;
  k_xdens_wg<T, N1, TW><<<dim3(gx, splits), 32 * TW, sm, st>>>(hba, hbb, hb_bs, nb, bper, w, sp, plan, tw, out_perm); count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t xdens_wg(const cplx<T>* hba, const cplx<T>* hbb, int64_t hb_bs, int nb, const T* w,
                            const SphereDev& sp, const FftPlan& plan, const cplx<T>* tw, double* out_perm,
                            cudaStream_t st) {
  switch (plan.n[0]) {
    case 24: return launch_xdens_wg<T, 24>(hba, hbb, hb_bs, nb, w, sp, plan, tw, out_perm, st);
    case 64: return launch_xdens_wg<T, 64>(hba, hbb, hb_bs, nb, w, sp, plan, tw, out_perm, st);
    case 72: return launch_xdens_wg<T, 72>(hba, hbb, hb_bs, nb, w, sp, plan, tw, out_perm, st);
    case 90: return launch_xdens_wg<T, 90>(hba, hbb, hb_bs, nb, w, sp, plan, tw, out_perm, st);
    case 96: return launch_xdens_wg<T, 96>(hba, hbb, hb_bs, nb, w, sp, plan, tw, out_perm, st);
    case 120: return launch_xdens_wg<T, 120>(hba, hbb, hb_bs, nb, w, sp, plan, tw, out_perm, st);
    default: return cudaErrorNotSupported;
  }
}

template <typename T>
cudaError_t launch_density(const FftPlan& plan, const cplx<T>* tw, const SphereDev& sp,
                           const cplx<T>* a, const cplx<T>* b, int64_t ld, int nband, const T* w_dev,
                           double* out_perm, cplx<T>* hb, int band_batch, cudaStream_t st) {
  if (nband <= 0) return cudaSuccess;
  const int cz = pick_cz(plan.n[2]);
  const int lyz = 8;  // 8 accumulators per thread cover n1*lyz <= 2048 points
  if (plan.n[0] * lyz > 8 * kThreads) return cudaErrorInvalidValue;
  const size_t sm1 = plane_smem<T>(plan, sp, cz);
  const size_t sm2 = sizeof(cplx<T>) * (size_t)plan.n[0] * lyz * 2;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_plane_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1))) return e;
  if ((e = cudaFuncSetAttribute(k_xline_density<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2))) return e;
  const int64_t hb_bs = (int64_t)sp.nplane * plan.n[1] * plan.n[2];
  const int nyz = plan.n[1] * plan.n[2];
  cplx<T>* hbb = b ? hb + hb_bs * band_batch : nullptr;
  for (int b0 = 0; b0 < nband; b0 += band_batch) {
    const int nb = min(band_batch, nband - b0);
    // pass 1 for a (and b): warp-group plane kernels where they cover the box
    for (int which = 0; which < (b ? 2 : 1); ++which) {
      const cplx<T>* src = (which ? b : a) + b0 * ld;
      cplx<T>* dst = which ? hbb : hb;
      e = plane_wg<T>(0, src, ld, dst, hb_bs, sp, plan, tw, nullptr, nullptr, 0, nb, st);
      if (e == cudaErrorNotSupported) {
        (void)cudaGetLastError();
        k_plane_inv<T><<<dim3(sp.nplane, nb), kThreads, sm1, st>>>(src, ld, dst, hb_bs, sp, plan, tw, cz); count_launch();
        e = cudaGetLastError();
      }
      if (e) return e;
    }
    e = xdens_wg<T>(hb, hbb, hb_bs, nb, w_dev + b0, sp, plan, tw, out_perm, st);
    if (e == cudaErrorNotSupported) {
      (void)cudaGetLastError();
      k_xline_density<T><<<(nyz + lyz - 1) / lyz, kThreads, sm2, st>>>(hb, hbb, hb_bs, nb, w_dev + b0, sp, plan,
                                                                       tw, lyz, out_perm); count_launch();
      e = cudaGetLastError();
    }
    if (e) return e;
  }
  return cudaGetLastError();
}

template cudaError_t launch_local_apply<double>(const FftPlan&, const double2*, const SphereDev&, const double*,
                                                const double*, const double2*, int64_t, int, double2*, int64_t,
                                                double2*, int, cudaStream_t, ::pw_ctx*);
template cudaError_t launch_local_apply<float>(const FftPlan&, const float2*, const SphereDev&, const float*,
                                               const float*, const float2*, int64_t, int, float2*, int64_t,
                                               float2*, int, cudaStream_t, ::pw_ctx*);
template cudaError_t launch_density<double>(const FftPlan&, const double2*, const SphereDev&, const double2*,
                                            const double2*, int64_t, int, const double*, double*, double2*, int,
                                            cudaStream_t);
template cudaError_t launch_density<float>(const FftPlan&, const float2*, const SphereDev&, const float2*,
                                           const float2*, int64_t, int, const float*, double*, float2*, int,
                                           cudaStream_t);

}  // namespace pw
