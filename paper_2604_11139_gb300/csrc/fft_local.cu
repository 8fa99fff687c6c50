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
#include "pw_internal.cuh"

namespace pw {

// ---- small DFTs: y_m = sum_k x_k exp(S 2 pi i k m / R) -------------------------
template <typename C, int S> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a; a = cadd(t, b); b = csub(t, b);
}
template <typename C, int S> __device__ __forceinline__ void dft4(C* x) {
  C s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
  C s13 = cadd(x[1], x[3]), d13 = cmuli<S>(csub(x[1], x[3]));
  x[0] = cadd(s02, s13); x[2] = csub(s02, s13);
  x[1] = cadd(d02, d13); x[3] = csub(d02, d13);
}
template <typename C, int S> __device__ __forceinline__ void dft8(C* x) {
  using R = decltype(C{}.x);
  const R h = (R)0.70710678118654752440084436210485;  // cos(pi/4)
  C e[4] = {x[0], x[2], x[4], x[6]};
  C o[4] = {x[1], x[3], x[5], x[7]};
  dft4<C, S>(e); dft4<C, S>(o);
  // o[m] *= w8^m, w8 = exp(S i pi/4)
  C o1 = o[1]; o[1] = mk<C>(h * (o1.x - S * o1.y), h * (o1.y + S * o1.x));
  o[2] = cmuli<S>(o[2]);
  C o3 = o[3]; o[3] = mk<C>(h * (-o3.x - S * o3.y), h * (-o3.y + S * o3.x));
#pragma unroll
  for (int m = 0; m < 4; ++m) { x[m] = cadd(e[m], o[m]); x[m + 4] = csub(e[m], o[m]); }
}
template <typename C, int S> __device__ __forceinline__ void dft3(C* x) {
  using R = decltype(C{}.x);
  const R s3 = (R)0.86602540378443864676372317075294;  // sin(pi/3)
  C t = cadd(x[1], x[2]);
  C d = cmuli<S>(csub(x[1], x[2]));
  C m = csub(x[0], cscale(t, (R)0.5));
  x[0] = cadd(x[0], t);
  x[1] = cadd(m, cscale(d, s3));
  x[2] = csub(m, cscale(d, s3));
}
template <typename C, int S> __device__ __forceinline__ void dft5(C* x) {
  using R = decltype(C{}.x);
  const R c1 = (R)0.30901699437494742410229341718282;   // cos(2pi/5)
  const R c2 = (R)-0.80901699437494742410229341718282;  // cos(4pi/5)
  const R s1 = (R)0.95105651629515357211643933337938;   // sin(2pi/5)
  const R s2 = (R)0.58778525229247312916870595463907;   // sin(4pi/5)
  C t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
  C d1 = csub(x[1], x[4]), d2 = csub(x[2], x[3]);
  C a1 = cadd(x[0], cadd(cscale(t1, c1), cscale(t2, c2)));
  C a2 = cadd(x[0], cadd(cscale(t1, c2), cscale(t2, c1)));
  C b1 = cmuli<S>(cadd(cscale(d1, s1), cscale(d2, s2)));
  C b2 = cmuli<S>(csub(cscale(d1, s2), cscale(d2, s1)));
  x[0] = cadd(x[0], cadd(t1, t2));
  x[1] = cadd(a1, b1); x[4] = csub(a1, b1);
  x[2] = cadd(a2, b2); x[3] = csub(a2, b2);
}
template <typename C, int S, int R> __device__ __forceinline__ void dftR(C* x) {
  if constexpr (R == 2) dft2<C, S>(x[0], x[1]);
  else if constexpr (R == 3) dft3<C, S>(x);
  else if constexpr (R == 4) dft4<C, S>(x);
  else if constexpr (R == 5) dft5<C, S>(x);
  else dft8<C, S>(x);
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
      case 8: fft_stage<C, S, DIT, LINE_FAST, 8>(buf, nlines, ls, es, d.n, d.L[s], tws); break;
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
struct CPlan {
  int nst;
  int radix[kMaxStages];
  int L[kMaxStages];
};
constexpr CPlan make_cplan(int n) {
  CPlan p{};
  p.nst = 0;
  int m = n;
  const int order[5] = {8, 4, 5, 3, 2};
  for (int i = 0; i < 5; ++i) {
    const int r = order[i];
    while (m > 1 && m % r == 0) {
      p.radix[p.nst++] = r;
      m /= r;
    }
  }
  int L = n;
  for (int s = 0; s < p.nst; ++s) {
    p.L[s] = L;
    L /= p.radix[s];
  }
  return p;
}

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

constexpr int kThreads = 256;

// ---- pass 1: sphere plane -> inverse (z, y) -> half-box plane ---------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_plane_inv(const cplx<T>* __restrict__ psi, int64_t ldpsi,
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
__global__ void __launch_bounds__(kThreads) k_xline(cplx<T>* __restrict__ hb, int64_t hb_bs,
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
__global__ void __launch_bounds__(kThreads) k_plane_fwd(const cplx<T>* __restrict__ hb, int64_t hb_bs,
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
__global__ void __launch_bounds__(kThreads) k_xline_density(const cplx<T>* __restrict__ hba,
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

// ---- launchers ------------------------------------------------------------------
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
  for (int b0 = 0; b0 < nband; b0 += band_batch) {
    const int nb = min(band_batch, nband - b0);
    prof_begin(prof, PW_PROF_PLANE_INV);
    k_plane_inv<T><<<dim3(sp.nplane, nb), kThreads, sm1, st>>>(psi + b0 * ldpsi, ldpsi, hb, hb_bs, sp, plan, tw, cz); count_launch();
    prof_end(prof, PW_PROF_PLANE_INV);
    prof_begin(prof, PW_PROF_XLINE);
    k_xline<T><<<dim3((nyz + lyz - 1) / lyz, nb), kThreads, sm2, st>>>(hb, hb_bs, vperm, sp, plan, tw, lyz); count_launch();
    prof_end(prof, PW_PROF_XLINE);
    prof_begin(prof, PW_PROF_PLANE_FWD);
    k_plane_fwd<T><<<dim3(sp.nplane, nb), kThreads, sm1, st>>>(hb, hb_bs, sp, plan, tw, cz, kin,
                                                                psi + b0 * ldpsi, ldpsi, out + b0 * ldout, ldout); count_launch();
    prof_end(prof, PW_PROF_PLANE_FWD);
  }
  return cudaGetLastError();
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
    k_plane_inv<T><<<dim3(sp.nplane, nb), kThreads, sm1, st>>>(a + b0 * ld, ld, hb, hb_bs, sp, plan, tw, cz); count_launch();
    if (b) { k_plane_inv<T><<<dim3(sp.nplane, nb), kThreads, sm1, st>>>(b + b0 * ld, ld, hbb, hb_bs, sp, plan, tw, cz); count_launch(); }
    k_xline_density<T><<<(nyz + lyz - 1) / lyz, kThreads, sm2, st>>>(hb, hbb, hb_bs, nb, w_dev + b0, sp, plan,
                                                                     tw, lyz, out_perm); count_launch();
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
