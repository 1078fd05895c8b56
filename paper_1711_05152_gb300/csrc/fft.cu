// Bluestein prime-length DFTs over FFTs of length 2^k or 3 * 2^k.
//
// A length-M DFT X[r] = sum_j x[j] exp(-2 pi i j r / M) (Algorithm 2, one
// lattice) is rewritten with j r = (j^2 + r^2 - (r - j)^2) / 2 as
//   X[r] = w[r] * sum_j (x[j] w[j]) conj(w[r - j]),   w[n] = exp(-pi i n^2 / M),
// a linear convolution evaluated by power-of-two FFTs of length P >= 2M - 1.
// The chirp phase uses n^2 mod 2M reduced in exact integers.
//
// On GB300 the FP64 pipe (about 2 FMA per clock per SM) bounds these
// transforms, so the kernels read chirps, filters and twiddles from tables
// instead of recomputing them, and never spend FP64 work on index math.  The
// same kernels also run in double-float arithmetic (arith.cuh), which moves
// the butterflies to the FP32 pipes (about 60 times the FP64 rate).
//
// Structure: P <= 4096 runs in one CTA per transform (everything in shared
// memory).  Larger P uses the 4-step split P = P1 * P2 without transposes:
//   pass 1 (columns): FFT_P1 over n1 of x[n1 P2 + n2], times w_P^(n2 k1),
//                     stored at k1 P2 + n2;
//   pass 2 (rows):    FFT_P2 over n2 (giving X[k1 + P1 k2] at k1 P2 + k2),
//                     times the filter spectrum (stored in the same order),
//                     inverse FFT_P2, times w_P^(-n2 k1);
//   pass 3 (columns): inverse FFT_P1 over k1, natural order x[n1 P2 + n2].
// Each sub-FFT is a mixed-radix (8, 4, 2, 3) Stockham autosort FFT in shared
// memory (Govindaraju et al., SC'08 formulation).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include <cmath>

#include "arith.cuh"
#include "fft.cuh"
#include "prof.cuh"

namespace mr1l {

// ---------------------------------------------------------------------------
// Register DFTs of size 2, 3, 4, 8 (forward: exp(-2 pi i / R); INV: conjugate)
// over an arithmetic O (OpsF64 or OpsDF).
// ---------------------------------------------------------------------------
template <int R, bool INV, class O>
struct RegDft;

template <bool INV, class O>
struct RegDft<2, INV, O> {
  typedef typename O::V V;
  static __device__ __forceinline__ void run(V* v) {
    V a = v[0], b = v[1];
    v[0] = O::add(a, b);
    v[1] = O::sub(a, b);
  }
};

template <bool INV, class O>
struct RegDft<4, INV, O> {
  typedef typename O::V V;
  static __device__ __forceinline__ void run(V* v) {
    V t0 = O::add(v[0], v[2]), t1 = O::sub(v[0], v[2]);
    V t2 = O::add(v[1], v[3]), t3 = O::template mi<INV>(O::sub(v[1], v[3]));
    v[0] = O::add(t0, t2);
    v[2] = O::sub(t0, t2);
    v[1] = O::add(t1, t3);
    v[3] = O::sub(t1, t3);
  }
};

// 1/sqrt(2) and sqrt(3)/2 as FP64 and as FP32 pairs hi + lo (hi = the FP32
// rounding, lo = the FP32 rounding of the remainder)
#define MR1L_INV_SQRT2 0.70710678118654752440, 0x1.6a09e6p-1f, 0x1.9fcef4p-27f
#define MR1L_SQRT3_2 0.86602540378443864676, 0x1.bb67aep-1f, 0x1.0b0996p-26f

// w8 = exp(-+ 2 pi i / 8): w8 x = (x + mi(x)) / sqrt2, w8^3 x = (mi(x) - x) / sqrt2
template <bool INV, class O>
__device__ __forceinline__ typename O::V w8_1(typename O::V x) {
  return O::scalec(O::add(x, O::template mi<INV>(x)), MR1L_INV_SQRT2);
}
template <bool INV, class O>
__device__ __forceinline__ typename O::V w8_3(typename O::V x) {
  return O::scalec(O::sub(O::template mi<INV>(x), x), MR1L_INV_SQRT2);
}

template <bool INV, class O>
struct RegDft<8, INV, O> {
  typedef typename O::V V;
  static __device__ __forceinline__ void run(V* v) {
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    RegDft<4, INV, O>::run(e);
    RegDft<4, INV, O>::run(o);
    V o1 = w8_1<INV, O>(o[1]);
    V o2 = O::template mi<INV>(o[2]);
    V o3 = w8_3<INV, O>(o[3]);
    v[0] = O::add(e[0], o[0]);
    v[4] = O::sub(e[0], o[0]);
    v[1] = O::add(e[1], o1);
    v[5] = O::sub(e[1], o1);
    v[2] = O::add(e[2], o2);
    v[6] = O::sub(e[2], o2);
    v[3] = O::add(e[3], o3);
    v[7] = O::sub(e[3], o3);
  }
};

// Radix 3: X0 = a + b + c, X1,2 = a - (b + c)/2 -+ i (sqrt(3)/2)(b - c) (forward).
template <bool INV, class O>
struct RegDft<3, INV, O> {
  typedef typename O::V V;
  static __device__ __forceinline__ void run(V* v) {
    V t1 = O::add(v[1], v[2]), t2 = O::sub(v[1], v[2]);
    V a = v[0];
    v[0] = O::add(a, t1);
    V m1 = O::sub(a, O::half(t1));
    V m2 = O::scalec(O::template mi<INV>(t2), MR1L_SQRT3_2);
    v[1] = O::add(m1, m2);
    v[2] = O::sub(m1, m2);
  }
};

// Radix-8 DFT of a sequence whose inputs 4..7 are zero (the first stage of a
// zero-padded Bluestein input): v[0..3] in, v[0..7] out.
template <bool INV, class O>
__device__ __forceinline__ void reg_dft8_half(typename O::V* v) {
  typedef typename O::V V;
  V e0 = O::add(v[0], v[2]), e2 = O::sub(v[0], v[2]);
  V m2 = O::template mi<INV>(v[2]);
  V e1 = O::add(v[0], m2), e3 = O::sub(v[0], m2);
  V o0 = O::add(v[1], v[3]), o2 = O::sub(v[1], v[3]);
  V m3 = O::template mi<INV>(v[3]);
  V o1 = O::add(v[1], m3), o3 = O::sub(v[1], m3);
  o1 = w8_1<INV, O>(o1);
  o2 = O::template mi<INV>(o2);
  o3 = w8_3<INV, O>(o3);
  v[0] = O::add(e0, o0);
  v[4] = O::sub(e0, o0);
  v[1] = O::add(e1, o1);
  v[5] = O::sub(e1, o1);
  v[2] = O::add(e2, o2);
  v[6] = O::sub(e2, o2);
  v[3] = O::add(e3, o3);
  v[7] = O::sub(e3, o3);
}

// ---------------------------------------------------------------------------
// Twiddled radix-8, -4 and -2 butterflies in multiply-add form (FP64), after
// Goedecker, "Fast radix 2, 3, 4, and 5 kernels for fast Fourier
// transformations on computers with overlapping multiply-add instructions",
// SIAM J. Sci. Comput. 18 (1997).  A twiddle w = s (1 + i t) is held as the
// pair (s, t); then the two outputs x +- w y cost two FMAs for u = (1 + i t) y
// and four for x +- s u, against four for the product and four for the sums.
// The butterfly on inputs v_r w^r (w = exp(-+2 pi i k / (R Ns))) is split into
// radix-2 levels that factor the twiddles out, so that each of its radix-2
// steps has that form:
//   radix 8: level 1 pairs (v_r, v_r+4) under w^4; level 2 under w^2 and
//            -+i w^2; level 3 under w, w8 w, -+i w, -+i w8 w
//            (w8 = exp(-+2 pi i / 8)): 72 FMAs against 80 instructions
//            (28 for the seven products, 52 for the DFT);
//   radix 4: w^2, then w and -+i w: 24 against 28;  radix 2: 6 against 8.
// Multiplying by -+i is a swap of components.  The first-level twiddle (angle
// pi k / Ns) reaches pi / 2 at k = Ns / 2; from there on ("turned") the
// butterfly swaps the components of y and of one output pair instead, with
// the table's (s, t) taken for i w (fma_bfly_turnable), so that no negated
// value has to be materialised.
// ---------------------------------------------------------------------------
// (1 + i t) y
__device__ __forceinline__ cplx fma_rot(cplx y, double t) { return cmake(fma(-t, y.y, y.x), fma(t, y.x, y.y)); }
// p = x + s u, m = x - s u
__device__ __forceinline__ void fma_bfly(cplx x, double s, cplx u, cplx& p, cplx& m) {
  p = cmake(fma(s, u.x, x.x), fma(s, u.y, x.y));
  m = cmake(fma(-s, u.x, x.x), fma(-s, u.y, x.y));
}

// p, m = x +- w y for the first-level twiddle w = (s, t).  Not turned:
// w = s (1 + i t).  Turned (forward): i w = s (1 - i t), i.e. w y = s ((a -
// t b) - i (b + t a)) with (a, b) = (Im y, Re y); the inverse takes the
// conjugate (t -> -t, the sign on the real part instead).  The swaps are
// register selects.
template <bool INV>
__device__ __forceinline__ void fma_bfly_turnable(cplx x, cplx T, cplx y, bool turned, cplx& p, cplx& m) {
  const double t = INV ? -T.y : T.y;
  const double a = turned ? y.y : y.x, b = turned ? y.x : y.y;
  const double ux = fma(-t, b, a), uy = fma(t, a, b);
  const double px = fma(T.x, ux, x.x), mx = fma(-T.x, ux, x.x);
  const double py = fma(T.x, uy, x.y), my = fma(-T.x, uy, x.y);
  if (INV) {
    p = cmake(turned ? mx : px, py);
    m = cmake(turned ? px : mx, my);
  } else {
    p = cmake(px, turned ? my : py);
    m = cmake(mx, turned ? py : my);
  }
}

template <int R, bool INV>
struct FmaDft;

template <bool INV>
struct FmaDft<8, INV> {
  // e = (s, t) of w^4 (turned when half), w^2, w, w8 w
  static __device__ __forceinline__ void run(cplx* v, const cplx* e, bool half) {
    const cplx T4 = e[0], T2 = e[1], T1 = e[2], TW = e[3];
    const double t2 = INV ? -T2.y : T2.y, t1 = INV ? -T1.y : T1.y, tw = INV ? -TW.y : TW.y;
    cplx a[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) fma_bfly_turnable<INV>(v[q], T4, v[q + 4], half, a[q], a[q + 4]);  // under w^4
    // even half (a0, a2 | a4, a6), odd half (a1, a3 | a5, a7)
    cplx E0, E1, E2, E3, o0, o1, o2, o3;
    fma_bfly(a[0], T2.x, fma_rot(a[2], t2), E0, E2);
    fma_bfly(a[4], T2.x, mul_mi<INV>(fma_rot(a[6], t2)), E1, E3);
    fma_bfly(a[1], T2.x, fma_rot(a[3], t2), o0, o2);
    fma_bfly(a[5], T2.x, mul_mi<INV>(fma_rot(a[7], t2)), o1, o3);
    fma_bfly(E0, T1.x, fma_rot(o0, t1), v[0], v[4]);
    fma_bfly(E1, TW.x, fma_rot(o1, tw), v[1], v[5]);
    fma_bfly(E2, T1.x, mul_mi<INV>(fma_rot(o2, t1)), v[2], v[6]);
    fma_bfly(E3, TW.x, mul_mi<INV>(fma_rot(o3, tw)), v[3], v[7]);
  }
};

template <bool INV>
struct FmaDft<4, INV> {
  // e = (s, t) of w^2 (turned when half), w
  static __device__ __forceinline__ void run(cplx* v, const cplx* e, bool half) {
    const cplx T2 = e[0], T1 = e[1];
    const double t1 = INV ? -T1.y : T1.y;
    cplx A0, A1, B0, B1;
    fma_bfly_turnable<INV>(v[0], T2, v[2], half, A0, A1);
    fma_bfly_turnable<INV>(v[1], T2, v[3], half, B0, B1);
    fma_bfly(A0, T1.x, fma_rot(B0, t1), v[0], v[2]);
    fma_bfly(A1, T1.x, mul_mi<INV>(fma_rot(B1, t1)), v[1], v[3]);
  }
};

template <bool INV>
struct FmaDft<2, INV> {
  // e = (s, t) of w (turned when half)
  static __device__ __forceinline__ void run(cplx* v, const cplx* e, bool half) {
    cplx p, m;
    fma_bfly_turnable<INV>(v[0], e[0], v[1], half, p, m);
    v[0] = p;
    v[1] = m;
  }
};

template <class O, int R>
struct FmaForm {
  static constexpr bool value = std::is_same<O, OpsF64>::value && (R == 2 || R == 4 || R == 8);
};
template <class O>
struct FmaTab {  // the multiply-add twiddles: FP64 only
  static __device__ __forceinline__ const cplx* of(const typename O::V*) { return nullptr; }
};
template <>
struct FmaTab<OpsF64> {
  static __device__ __forceinline__ const cplx* of(const cplx* twn) { return twn + kSmallTw; }
};
template <int R>
__device__ __forceinline__ int fma_off(int Ns, int k) {
  return R == 8 ? 4 * (Ns - 1 + k) : R == 4 ? 4 * kFmaSpan + 2 * (Ns - 1 + k) : 6 * kFmaSpan + (Ns - 1 + k);
}

// The DFT of one radix-R butterfly of a stage with stride Ns, including the
// stage twiddles w^r (w = exp(-+2 pi i k / (R Ns)), none when Ns = 1).
template <int R, bool INV, class O>
__device__ __forceinline__ void twiddled_dft(typename O::V* v, int n, int Ns, int k, const typename O::V* twn_n,
                                             const cplx* ft) {
  if constexpr (FmaForm<O, R>::value) {
    if (Ns > 1) {
      FmaDft<R, INV>::run(v, ft + fma_off<R>(Ns, k), 2 * k >= Ns);
      return;
    }
  } else {
    if (Ns > 1) {
      const int step = k * (n / (Ns * R));
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const typename O::V w = twn_n[r * step];
        v[r] = INV ? O::mulc(v[r], w) : O::mul(v[r], w);
      }
    }
  }
  RegDft<R, INV, O>::run(v);
}

// ---------------------------------------------------------------------------
// One Stockham stage of radix R over nseq sequences of length n in shared
// memory; element i of sequence b sits at s[b * bs + i * is].  The block has
// nseq * n / 8 threads (or more, which idle); each thread runs up to
// ceil(8 / R) butterflies of the stage.
//   COLS: sequence index fastest across threads (column tiles, bs == 1)
//   else: element index fastest (row tiles, is == 1)
// HALF (first radix-8 stage only): inputs r >= 4 are known zeros.
// ---------------------------------------------------------------------------
// Shared-memory tiles of the 4-step passes are stored swizzled: element e of
// a tile at e ^ ((e >> 3) & 7).  The first stage of a sub-FFT writes 8
// consecutive elements per thread, a 128-byte stride between the lanes of a
// warp when a tile holds one sequence, which unswizzled hits one 16-byte bank
// group 8 times per 128-byte wavefront; the swizzle spreads those lanes over
// the 8 groups and only permutes elements within each aligned group of 8, so
// the stride-1 accesses of the other stages stay conflict-free.  (Tiles hold
// a multiple of 8 elements.)
__device__ __forceinline__ int tile_swz(int e) { return e ^ ((e >> 3) & 7); }

template <int R, bool INV, bool COLS, class O, bool HALF = false>
__device__ __forceinline__ void stockham_stage(typename O::V* s, int n, int Ns, int nseq, int bs, int is,
                                               const typename O::V* twn_n, const cplx* ft) {
  // COLS tiles (the column passes) are swizzled, the one-CTA transforms not
  auto at = [](int e) { return COLS ? tile_swz(e) : e; };
  typedef typename O::V V;
  constexpr int CNT = (8 + R - 1) / R;
  const int nb = n / R;
  const int total = nseq * nb;
  V v[CNT][R];
  int base[CNT];
  bool act[CNT];
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    int idx = threadIdx.x + c * blockDim.x;
    act[c] = idx < total;
    int b, j;
    if (COLS) {
      b = idx % nseq;
      j = idx / nseq;
    } else {
      b = idx / nb;
      j = idx - b * nb;
    }
    int k = j % Ns;
    base[c] = b * bs + ((j - k) * R + k) * is;
    if (act[c] && HALF) {
      const int e0 = b * bs + j * is;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[c][r] = s[at(e0 + r * nb * is)];
      reg_dft8_half<INV, O>(v[c]);
    } else if (act[c]) {
      const int e0 = b * bs + j * is;
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = s[at(e0 + r * nb * is)];
      twiddled_dft<R, INV, O>(v[c], n, Ns, k, twn_n, ft);
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    if (act[c]) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[at(base[c] + r * Ns * is)] = O::norm(v[c][r]);
    }
  }
  __syncthreads();
}

// Twiddles exp(-2 pi i e / n) of a sub-FFT length n (2^a or 3 * 2^a).
template <class T>
__device__ __forceinline__ const T* twiddles_of(const T* twn, int n) {
  return (n & (n - 1)) == 0 ? twn + n : twn + kSmallTwPow2 + n - 3;
}

// Full in-smem FFT of length n = 2^a or 3 * 2^a: radix-8 stages, one radix-4
// or radix-2 stage for the rest of 2^a, then radix 3.  Natural order in and
// out.  HALF_FIRST: the upper half of every input sequence is zero (needs
// 8 | n).
template <bool INV, bool COLS, class O, bool HALF_FIRST = false>
__device__ __forceinline__ void smem_fft(typename O::V* s, int n, int nseq, int bs, int is,
                                         const typename O::V* twn) {
  const typename O::V* twn_n = twiddles_of(twn, n);
  const cplx* ft = FmaTab<O>::of(twn);
  const bool three = (n % 3) == 0;
  int rem = 31 - __clz(three ? n / 3 : n);  // log2 of the power-of-two part
  int Ns = 1;
  if (HALF_FIRST && rem >= 3) {
    stockham_stage<8, INV, COLS, O, true>(s, n, Ns, nseq, bs, is, twn_n, ft);
    Ns <<= 3;
    rem -= 3;
  }
  while (rem >= 3) {
    stockham_stage<8, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n, ft);
    Ns <<= 3;
    rem -= 3;
  }
  if (rem == 2) {
    stockham_stage<4, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n, ft);
    Ns <<= 2;
  }
  if (rem == 1) {
    stockham_stage<2, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n, ft);
    Ns <<= 1;
  }
  if (three) stockham_stage<3, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n, ft);
}

// ---------------------------------------------------------------------------
// Tables in the arithmetic's format
// ---------------------------------------------------------------------------
template <class O>
struct Tab;
template <>
struct Tab<OpsF64> {
  static __device__ __forceinline__ const cplx* w(const BlueGeom& g) { return g.w; }
  static __device__ __forceinline__ const cplx* ws(const BlueGeom& g) { return g.ws; }
  static __device__ __forceinline__ const cplx* tw(const BlueGeom& g) { return g.tw; }
  static __device__ __forceinline__ const cplx* twr(const BlueGeom& g) { return g.twr; }
  static __device__ __forceinline__ const cplx* twc(const BlueGeom& g) { return g.twc; }
  static __device__ __forceinline__ const cplx* twn(const BlueGeom& g) { return g.twn; }
  static __device__ __forceinline__ cplx* Bh(const BlueGeom& g) { return g.Bh; }
};
template <>
struct Tab<OpsDF> {
  static __device__ __forceinline__ const float4* w(const BlueGeom& g) { return g.w_df; }
  static __device__ __forceinline__ const float4* ws(const BlueGeom& g) { return g.ws_df; }
  static __device__ __forceinline__ const float4* tw(const BlueGeom& g) { return g.tw_df; }
  static __device__ __forceinline__ const float4* twr(const BlueGeom& g) { return g.twr_df; }
  static __device__ __forceinline__ const float4* twc(const BlueGeom& g) { return g.twc_df; }
  static __device__ __forceinline__ const float4* twn(const BlueGeom& g) { return g.twn_df; }
  static __device__ __forceinline__ float4* Bh(const BlueGeom& g) { return (float4*)g.Bh; }
};

// ---------------------------------------------------------------------------
// Sources and sinks
// ---------------------------------------------------------------------------
template <int MODE, class O>
__device__ __forceinline__ typename O::V load_input(const BlueGeom& g, const BlueIO& io, int h, int M,
                                                    int64_t off, int64_t n) {
  if (MODE == kModeFilter) {
    if (n < M) return O::conj(Tab<O>::w(g)[off + n]);
    if (n > g.P - M) return O::conj(Tab<O>::w(g)[off + (g.P - n)]);
    return O::zero();
  }
  if (n >= M) return O::zero();
  cplx y = io.in[h * io.in_stride + off + n];
  if (MODE == kModeEval && y.x == 0.0 && y.y == 0.0) return O::zero();  // sparse bins: skip the chirp
  if (MODE == kModeRecon && io.add_in) y = cadd(y, io.add_in[h * io.in_stride + off + n]);
  typename O::V x = O::from(y);
  if (MODE == kModeRecon) return O::mul(x, Tab<O>::ws(g)[off + n]);
  return O::mul(O::conj(x), Tab<O>::w(g)[off + n]);
}

template <int MODE, class O>
__device__ __forceinline__ void store_output(const BlueGeom& g, const BlueIO& io, int h, int64_t off, int64_t n,
                                             typename O::V v) {
  if (MODE == kModeRecon) {
    io.out[h * io.out_stride + off + n] = O::to(v);
  } else {
    const typename O::V* wt = io.out_scaled ? Tab<O>::ws(g) : Tab<O>::w(g);
    io.out[h * io.out_stride + off + n] = O::to(O::conj(O::mul(wt[off + n], v)));
  }
}

// ---------------------------------------------------------------------------
// P <= 4096: the whole convolution in one CTA.
// ---------------------------------------------------------------------------
template <int MODE, class O>
__global__ void __launch_bounds__(512) blue_small_kernel(BlueGeom g, BlueIO io) {
  typedef typename O::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = (V*)smraw;
  const int gi = blockIdx.x;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, M = g.M[l];
  const int64_t off = g.off[l];
  // zero padding: for RECON / EVAL the input vanishes from M <= P/2 on, so the
  // upper half is never loaded and the first radix-8 stage skips it
  const bool half = MODE != kModeFilter && (P % 8) == 0;
  const int nload = half ? P / 2 : P;
  for (int n = threadIdx.x; n < nload; n += blockDim.x) sm[n] = load_input<MODE, O>(g, io, h, M, off, n);
  __syncthreads();
  if (half)
    smem_fft<false, false, O, true>(sm, P, 1, 0, 1, Tab<O>::twn(g));
  else
    smem_fft<false, false, O>(sm, P, 1, 0, 1, Tab<O>::twn(g));
  V* Bh = Tab<O>::Bh(g) + (int64_t)l * P;
  if constexpr (MODE == kModeFilter) {
    const double sc = 1.0 / (double)P;
    const float sh = __double2float_rn(sc), sl = __double2float_rn(sc - (double)sh);
    for (int n = threadIdx.x; n < P; n += blockDim.x) Bh[n] = O::scalec(sm[n], sc, sh, sl);
  } else {
    for (int n = threadIdx.x; n < P; n += blockDim.x) sm[n] = O::mul(sm[n], Bh[n]);
    __syncthreads();
    smem_fft<true, false, O>(sm, P, 1, 0, 1, Tab<O>::twn(g));
    for (int n = threadIdx.x; n < M; n += blockDim.x) store_output<MODE, O>(g, io, h, off, n, sm[n]);
  }
}

// ---------------------------------------------------------------------------
// 4-step passes
// ---------------------------------------------------------------------------
// A CTA transforms a tile of `tile` complex elements (tile / 8 threads): CB
// columns of length P1 or RB rows of length P2, CB and RB powers of two (so
// they divide P2 and P1); a single column or row longer than the tile takes a
// tile of its own length.  The tile size is picked per (P, mode, arithmetic)
// by the tile tuner below from kTileCands; 2048 (32 KB of shared memory,
// 256 threads, three CTAs per SM) is the default.
constexpr int kTileElems = 2048;
constexpr int kTileCands[3] = {1024, 2048, 4096};
__host__ __device__ __forceinline__ int col_tile(int P1, int tile) {
  int cb = tile / P1;  // P1 = 3 * 2^a gives a tile of 3/4 x tile
  if (cb > 16) cb = 16;
  if (cb < 1) cb = 1;
  int p = 1;
  while (2 * p <= cb) p *= 2;
  return p;
}
__host__ __device__ __forceinline__ int row_tile(int P2, int P1, int tile) {
  int rb = tile / P2;
  int p = 1;  // power of two dividing P1 (= 2^a or 3 * 2^a)
  while (2 * p <= rb && P1 % (2 * p) == 0) p *= 2;
  return p;
}

// Register budget of the 4-step kernels: the double-float passes wait on
// memory more than on arithmetic, so they are held to 64 registers (two
// 512-thread or four 256-thread CTAs per SM; a few bytes spill) for the
// occupancy; the FP64 column passes otherwise keep what the compiler picks
// (up to 128).  The largest lengths (2^25, 3 * 2^23) have single columns of 6144 or rows of
// 8192 elements, one CTA of up to 1024 threads each (NT = 1024: at most 64
// registers, so the FP64 kernels spill a little there).
// At P = 3 * 2^21 (columns of 3072 in CTAs of 384 threads, rows of 2048 in
// CTAs of 256 or, two rows each, 512) the FP64 passes have register-capped
// forms that fit one more CTA per SM: the evaluation column pass 80
// registers (two CTAs instead of one, -29 %), the rows 80 in CTAs of 256
// (three instead of two) and 64 in CTAs of 512 (two instead of one; also
// the rows of 4096 at P = 2^23), the inverse column pass 56 (three instead
// of two, 16 bytes spill, -3 %).  With the caps the tile tuner picks two
// rows per CTA at that length (rows -2 %).  The same cap measured slower for
// the reconstruct column pass (its chirp products need the registers) and in
// double-float (more spills).
template <class O>
struct MinBlocks {
  static constexpr int value = std::is_same<O, OpsDF>::value ? 2 : 1;
};
template <class O, int NT>
struct ColFwdBlocks {
  static constexpr int value = NT == 512 ? MinBlocks<O>::value : NT == 384 ? 2 : 1;
};
template <class O, int NT>
struct RowBlocks {
  static constexpr int value = NT == 512 ? 2 : NT == 256 ? 3 : 1;
};
template <class O, int NT>
struct ColInvBlocks {
  static constexpr int value = NT == 512 ? MinBlocks<O>::value : NT == 384 ? 3 : 1;
};

// Pass 1: columns, forward, with the 4-step twiddle.
template <int MODE, class O, int NT = 512>
__global__ void __launch_bounds__(NT, (ColFwdBlocks<O, NT>::value)) blue_col_fwd_kernel(BlueGeom g, BlueIO io) {
  typedef typename O::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = (V*)smraw;
  const int gi = blockIdx.y;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, P1 = g.P1, P2 = g.P2, CB = col_tile(P1, g.ctile);
  const int M = g.M[l];
  const int64_t off = g.off[l];
  const int n2_0 = blockIdx.x * CB;
  // RECON / EVAL: rows n1 >= P1/2 hold n >= P/2 >= M, i.e. zero padding
  const int rows = MODE == kModeFilter ? P1 : P1 / 2;
  V* work = (V*)io.work + (int64_t)gi * P;
  // 4-step twiddle w_P^(n2 k1), in column order (twc[n2 P1 + k1]): the tile's
  // columns read it contiguously
  const V* twc = Tab<O>::twc(g) + (int64_t)n2_0 * P1;
  // Evaluation inputs are often sparse (the bins of a few planted
  // frequencies).  A column with at most kColNz non-zeros is transformed
  // directly from its non-zeros, whatever the tiling; the column FFT runs
  // only when some column of the tile has more.  So every column gets the
  // same arithmetic under every tile size.  The direct sums split by n1 mod 8:
  // for k1 < P1/8, S_j = sum_{n1 = j mod 8} x[n1] w_P1^(n1 k1) (ascending n1)
  // and X[k1 + m P1/8] = sum_j S_j w_8^(j m), an 8-point DFT of the partial
  // sums: 4 nz / 8 + 6.5 FP64 instructions per output instead of 4 nz.  A
  // column with at most two non-zeros keeps the plain sums.
  constexpr int kColNz = 24;
  __shared__ int nzc[16];
  __shared__ short nzi[16][kColNz];
  __shared__ V nzv[16][kColNz];
  __shared__ unsigned char nzo[16][9];  // slots of n1 = j mod 8 at [nzo[b][j], nzo[b][j + 1])
  __shared__ int over;
  const V* twP1 = twiddles_of(Tab<O>::twn(g), P1);
  const bool p1_pow2 = (P1 & (P1 - 1)) == 0;
  auto tw1 = [&](int e) { return twP1[p1_pow2 ? (e & (P1 - 1)) : e % P1]; };
  // outputs of the sparse columns into sm (k1-major, CB columns per row)
  auto sparse_cols = [&]() {
    const int P1_8 = P1 >> 3;
    for (int e = threadIdx.x; e < P1_8 * CB; e += blockDim.x) {
      const int b = e / P1_8, k1 = e - b * P1_8;
      const int nz = nzc[b];
      if (nz > kColNz) continue;
      V out[8];
      if (nz <= 2) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int kk = k1 + m * P1_8;
          V acc = O::zero();
          for (int q = 0; q < nz; ++q) acc = O::mac(acc, nzv[b][q], tw1(nzi[b][q] * kk));
          out[m] = acc;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          V acc = O::zero();
          for (int q = nzo[b][j]; q < nzo[b][j + 1]; ++q) acc = O::mac(acc, nzv[b][q], tw1(nzi[b][q] * k1));
          out[j] = acc;
        }
        RegDft<8, false, O>::run(out);
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) sm[tile_swz((k1 + m * P1_8) * CB + b)] = out[m];
    }
  };

  if (MODE == kModeEval) {
    if (threadIdx.x < 16) nzc[threadIdx.x] = 0;
    if (threadIdx.x == 0) over = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < rows * CB; e += blockDim.x) {
      int i = e / CB, b = e - i * CB;
      V x = load_input<MODE, O>(g, io, h, M, off, (int64_t)i * P2 + n2_0 + b);
      sm[tile_swz(e)] = x;
      if (O::nonzero(x)) {
        int slot = atomicAdd(&nzc[b], 1);
        if (slot < kColNz) {
          nzi[b][slot] = (short)i;
          nzv[b][slot] = x;
        } else {
          over = 1;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < CB && nzc[threadIdx.x] <= kColNz) {  // slots by (n1 mod 8, n1)
      const int b = threadIdx.x;
      auto key = [](short i) { return ((i & 7) << 16) | i; };
      for (int q = 1; q < nzc[b]; ++q) {
        const short iq = nzi[b][q];
        const V vq = nzv[b][q];
        int r = q;
        for (; r > 0 && key(nzi[b][r - 1]) > key(iq); --r) {
          nzi[b][r] = nzi[b][r - 1];
          nzv[b][r] = nzv[b][r - 1];
        }
        nzi[b][r] = iq;
        nzv[b][r] = vq;
      }
      int q = 0;
      for (int j = 0; j < 8; ++j) {
        nzo[b][j] = (unsigned char)q;
        while (q < nzc[b] && (nzi[b][q] & 7) == j) ++q;
      }
      nzo[b][8] = (unsigned char)q;
    }
    __syncthreads();
    if (!over) {
      // the sums run column by column across the threads, so that a warp's
      // loops over the non-zeros of its column do not diverge; the store
      // then goes row by row through shared memory
      sparse_cols();
      __syncthreads();
      for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
        int k1 = e / CB, b = e - k1 * CB;
        int n2 = n2_0 + b;
        work[(int64_t)k1 * P2 + n2] = O::mul(sm[tile_swz(e)], twc[b * P1 + k1]);
      }
      return;
    }
  } else {
    for (int e = threadIdx.x; e < rows * CB; e += blockDim.x) {
      int i = e / CB, b = e - i * CB;
      sm[tile_swz(e)] = load_input<MODE, O>(g, io, h, M, off, (int64_t)i * P2 + n2_0 + b);
    }
    __syncthreads();
  }
  if (MODE == kModeFilter)
    smem_fft<false, true, O>(sm, P1, CB, 1, CB, Tab<O>::twn(g));
  else
    smem_fft<false, true, O, true>(sm, P1, CB, 1, CB, Tab<O>::twn(g));
  if (MODE == kModeEval) {  // the sparse columns of a mixed tile
    __syncthreads();
    sparse_cols();
    __syncthreads();
  }
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int k1 = e / CB, b = e - k1 * CB;
    int n2 = n2_0 + b;
    work[(int64_t)k1 * P2 + n2] = O::mul(sm[tile_swz(e)], twc[b * P1 + k1]);
  }
}

// ---------------------------------------------------------------------------
// Row tiles with fused sources and sinks.  A row pass transforms rows of
// length P2 = 2^b (b >= 6) element-fastest across threads.  Its first stage
// reads the work tile straight from global memory, the filter product rides on
// the last forward stage, and the twiddle product and the store ride on the
// last inverse stage, which saves three passes over shared memory and their
// barriers.
// ---------------------------------------------------------------------------
// Shared-memory rows are swizzled like the column tiles (tile_swz).
__device__ __forceinline__ int row_swz(int i) { return tile_swz(i); }

template <class O>
struct RowSmem {
  typename O::V* s;
  int P2;
  __device__ __forceinline__ typename O::V ld(int b, int i) const { return s[b * P2 + row_swz(i)]; }
  __device__ __forceinline__ void st(int b, int i, typename O::V v) const { s[b * P2 + row_swz(i)] = O::norm(v); }
};
template <class O>
struct RowLoad {  // the work tile in global memory
  const typename O::V* p;
  int P2;
  __device__ __forceinline__ typename O::V ld(int b, int i) const { return p[b * P2 + i]; }
};
template <class O>
struct RowTimesFilter {  // shared memory <- v * filter spectrum
  typename O::V* s;
  const typename O::V* Bh;
  int P2;
  __device__ __forceinline__ void st(int b, int i, typename O::V v) const {
    s[b * P2 + row_swz(i)] = O::mul(v, Bh[b * P2 + i]);
  }
};
template <class O>
struct RowStoreTwiddled {  // work tile <- v conj(w_P^(n2 k1)), twiddles in row order
  typename O::V* p;
  const typename O::V* twr;  // rows of the tile: twr[b P2 + n2] = w_P^(n2 (k1_0 + b))
  int P2;
  __device__ __forceinline__ void st(int b, int i, typename O::V v) const {
    p[b * P2 + i] = O::mulc(v, twr[b * P2 + i]);
  }
};
template <class O>
struct RowStoreScaled {  // filter spectrum <- v / P
  typename O::V* p;
  int P2;
  double sc;
  float sh, sl;
  __device__ __forceinline__ void st(int b, int i, typename O::V v) const { p[b * P2 + i] = O::scalec(v, sc, sh, sl); }
};

// One radix-R Stockham stage over nrows rows of length n, element-fastest;
// element i of row b is read as src.ld(b, i) and written as dst.st(b, i, v).
template <int R, bool INV, class O, class Src, class Dst>
__device__ __forceinline__ void row_stage(int n, int Ns, int nrows, const typename O::V* twn_n, const cplx* ft,
                                          const Src& src, const Dst& dst) {
  typedef typename O::V V;
  constexpr int CNT = (8 + R - 1) / R;
  const int nb = n / R;
  const int total = nrows * nb;
  V v[CNT][R];
  int rb[CNT], ob[CNT];
  bool act[CNT];
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    const int idx = threadIdx.x + c * blockDim.x;
    act[c] = idx < total;
    const int b = idx / nb, j = idx - b * nb, k = j % Ns;
    rb[c] = b;
    ob[c] = (j - k) * R + k;
    if (act[c]) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = src.ld(b, j + r * nb);
      twiddled_dft<R, INV, O>(v[c], n, Ns, k, twn_n, ft);
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    if (act[c]) {
#pragma unroll
      for (int r = 0; r < R; ++r) dst.st(rb[c], ob[c] + r * Ns, v[c][r]);
    }
  }
  __syncthreads();
}

// FFT of nrows rows of length P2 = 2^b (b >= 6): radix-8 stages, then one
// radix-4 or radix-2 stage; input through src, output through dst, the stages
// in between in the shared-memory tile sm.
template <bool INV, class O, class Src, class Dst>
__device__ __forceinline__ void row_fft_io(typename O::V* sm, int P2, int nrows, const typename O::V* twn,
                                           const Src& src, const Dst& dst) {
  const typename O::V* tw = twiddles_of(twn, P2);
  const cplx* ft = FmaTab<O>::of(twn);
  const RowSmem<O> smio{sm, P2};
  const int b = 31 - __clz(P2), n8 = b / 3, tail = b % 3;
  row_stage<8, INV, O>(P2, 1, nrows, tw, ft, src, smio);
  int Ns = 8;
  const int mid = n8 - 1 - (tail == 0 ? 1 : 0);
  for (int i = 0; i < mid; ++i) {
    row_stage<8, INV, O>(P2, Ns, nrows, tw, ft, smio, smio);
    Ns <<= 3;
  }
  if (tail == 0)
    row_stage<8, INV, O>(P2, Ns, nrows, tw, ft, smio, dst);
  else if (tail == 2)
    row_stage<4, INV, O>(P2, Ns, nrows, tw, ft, smio, dst);
  else
    row_stage<2, INV, O>(P2, Ns, nrows, tw, ft, smio, dst);
}

// Pass 2: rows.  FILTER: forward FFT scaled by 1/P into Bh.  Otherwise forward
// FFT, times Bh, inverse FFT, times conj(w_P^(n2 k1)), with the loads and
// stores fused into the first and last stages (row_fft_io).
template <bool FILTER, class O, int NT = 512>
__global__ void __launch_bounds__(NT, (RowBlocks<O, NT>::value)) blue_row_kernel(BlueGeom g, BlueIO io) {
  typedef typename O::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = (V*)smraw;
  const int gi = blockIdx.y;
  const int l = gi % g.L;
  const int P = g.P, P2 = g.P2, RB = row_tile(P2, g.P1, g.rtile);
  const int k1_0 = blockIdx.x * RB;
  V* work = (V*)io.work + (int64_t)gi * P + (int64_t)k1_0 * P2;
  V* Bh = Tab<O>::Bh(g) + (int64_t)l * P + (int64_t)k1_0 * P2;
  const RowLoad<O> src{work, P2};
  if (FILTER) {
    const double sc = 1.0 / (double)P;
    const float sh = __double2float_rn(sc), sl = __double2float_rn(sc - (double)sh);
    row_fft_io<false, O>(sm, P2, RB, Tab<O>::twn(g), src, RowStoreScaled<O>{Bh, P2, sc, sh, sl});
    return;
  }
  row_fft_io<false, O>(sm, P2, RB, Tab<O>::twn(g), src, RowTimesFilter<O>{sm, Bh, P2});
  row_fft_io<true, O>(sm, P2, RB, Tab<O>::twn(g), RowSmem<O>{sm, P2},
                      RowStoreTwiddled<O>{work, Tab<O>::twr(g) + (int64_t)k1_0 * P2, P2});
}

// Pass 3: columns, inverse; natural-order output n = n1 P2 + n2 for n < M.
template <int MODE, class O, int NT = 512>
__global__ void __launch_bounds__(NT, (ColInvBlocks<O, NT>::value)) blue_col_inv_kernel(BlueGeom g, BlueIO io) {
  typedef typename O::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = (V*)smraw;
  const int gi = blockIdx.y;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, P1 = g.P1, P2 = g.P2, CB = col_tile(P1, g.ctile);
  const int M = g.M[l];
  const int64_t off = g.off[l];
  const int n2_0 = blockIdx.x * CB;
  const V* work = (const V*)io.work + (int64_t)gi * P;
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int k1 = e / CB, b = e - k1 * CB;
    sm[tile_swz(e)] = work[(int64_t)k1 * P2 + n2_0 + b];
  }
  __syncthreads();
  smem_fft<true, true, O>(sm, P1, CB, 1, CB, Tab<O>::twn(g));
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int n1 = e / CB, b = e - n1 * CB;
    int64_t n = (int64_t)n1 * P2 + n2_0 + b;
    if (n < M) store_output<MODE, O>(g, io, h, off, n, sm[tile_swz(e)]);
  }
}

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------
__global__ void twiddle_kernel(cplx* tw, int64_t P) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= P) return;
  double s, c;
  sincospi(2.0 * (double)e / (double)P, &s, &c);  // 2e/P is exact
  tw[e] = cmake(c, -s);
}

__global__ void small_twiddle_kernel(cplx* tw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 || i >= kSmallTw) return;
  int n, e;
  if (i < kSmallTwPow2) {  // n = 2^a at [n, 2n)
    n = 1 << (31 - __clz(i));
    e = i - n;
  } else {                 // n = 3 * 2^a at [kSmallTwPow2 + n - 3, kSmallTwPow2 + 2n - 3)
    int j = i - kSmallTwPow2 + 3;      // in [n, 2n) for n = 3 * 2^a
    int a = 31 - __clz(j / 3);
    n = 3 << a;
    e = j - n;
  }
  double sn, cs;
  sincospi(2.0 * (double)e / (double)n, &sn, &cs);
  tw[i] = cmake(cs, -sn);
}

// The multiply-add twiddles (s, t), w = s (1 + i t), of the stage stride Ns
// and butterfly k < Ns; angles are exact multiples of pi / (4 Ns):
//   radix 8: w^4 (pi k / Ns, turned past pi / 2), w^2, w, w8 w
//   radix 4: w^2 (pi k / Ns, turned), w;     radix 2: w (pi k / Ns, turned)
// (w = exp(-2 pi i k / (R Ns))).  "Turned" entries, 2 k >= Ns, hold
// i w = s (1 - i t) as s = sin, t = -cos / sin of the angle; the others
// w = s (1 + i t) as s = cos, t = -tan (s > 0 in both).
__global__ void fma_twiddle_kernel(cplx* ft) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kFmaTw) return;
  int per, rel, R;
  if (i < 4 * kFmaSpan) {
    R = 8, per = 4, rel = i;
  } else if (i < 6 * kFmaSpan) {
    R = 4, per = 2, rel = i - 4 * kFmaSpan;
  } else {
    R = 2, per = 1, rel = i - 6 * kFmaSpan;
  }
  const int idx = rel / per, which = rel - idx * per;  // idx = Ns - 1 + k
  const int Ns = 1 << (31 - __clz(idx + 1)), k = idx + 1 - Ns;
  // angle / pi of the entry (forward sign taken below)
  double f;
  bool turned = false;
  if (which == 0) {
    f = (double)k / (double)Ns;  // w^4, w^2 or w of radix 8, 4, 2: pi k / Ns
    turned = 2 * k >= Ns;
  } else if (R == 8) {
    f = which == 1 ? (double)k / (2.0 * Ns) : which == 2 ? (double)k / (4.0 * Ns) : (double)(k + Ns) / (4.0 * Ns);
  } else {
    f = (double)k / (2.0 * Ns);  // radix 4: w
  }
  double sn, cs;
  sincospi(f, &sn, &cs);  // w = cs - i sn
  ft[i] = turned ? cmake(sn, -cs / sn) : cmake(cs, -sn / cs);
}

// Chirp w[n] = exp(-pi i q / M), q = n^2 mod 2M (exact), as the product of two
// tabulated factors exp(-pi i (q >> 12) 4096 / M) * exp(-pi i (q & 4095) / M):
// per-lattice tables of kChirpLo and kChirpSeedLen - kChirpLo entries (2M <=
// 2^25 leaves at most 8192 high parts), filled by sincospi of exactly reduced
// arguments, so that a
// sample costs one complex product instead of a sine and a cosine.
constexpr int kChirpLo = 4096;

__global__ void chirp_seed_kernel(cplx* seed, const int* Ms) {
  const int l = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kChirpSeedLen) return;
  const int64_t M = Ms[l];
  const int64_t e = i < kChirpLo ? i : ((int64_t)(i - kChirpLo) * kChirpLo) % (2 * M);  // phase index mod 2M
  double sn, cs;
  sincospi((double)e / (double)M, &sn, &cs);
  seed[(int64_t)l * kChirpSeedLen + i] = cmake(cs, -sn);
}

__global__ void chirp_kernel(cplx* w, cplx* ws, float4* w_df, float4* ws_df, const int64_t* off, const int* Ms,
                             const cplx* seed) {
  __shared__ double inv_M;
  const int l = blockIdx.y;
  const int M = Ms[l];
  if (threadIdx.x == 0) inv_M = 1.0 / (double)M;
  __syncthreads();
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= M) return;
  const uint64_t q = ((uint64_t)n * (uint64_t)n) % (uint64_t)(2 * (int64_t)M);  // exact n^2 mod 2M
  const cplx* sd = seed + (int64_t)l * kChirpSeedLen;
  const cplx v = cmul(sd[kChirpLo + (q >> 12)], sd[q & (kChirpLo - 1)]);
  const cplx vs = cmake(v.x * inv_M, v.y * inv_M);
  w[off[l] + n] = v;
  ws[off[l] + n] = vs;
  if (w_df) {  // double-float copies for the double-float passes
    w_df[off[l] + n] = OpsDF::from(v);
    ws_df[off[l] + n] = OpsDF::from(vs);
  }
}

namespace {
std::mutex g_tw_mu;
std::map<std::pair<int, int>, cplx*> g_tw;  // (device, P) -> table
std::map<int, cplx*> g_twn;                 // device -> small tables
}  // namespace

const cplx* twiddle_table(int Pn, cudaStream_t s) {
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto key = std::make_pair(dev, Pn);
  auto it = g_tw.find(key);
  if (it != g_tw.end()) return it->second;
  int64_t P = Pn;
  cplx* p = nullptr;
  MR1L_CUDA(cudaMalloc(&p, P * sizeof(cplx)));
  MR1L_LAUNCH("twiddle_kernel", s, 0, 16.0 * P, twiddle_kernel<<<cdiv(P, 256), 256, 0, s>>>(p, P));
  MR1L_CUDA(cudaStreamSynchronize(s));
  g_tw[key] = p;
  return p;
}

const cplx* small_twiddles(cudaStream_t s) {
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto it = g_twn.find(dev);
  if (it != g_twn.end()) return it->second;
  cplx* p = nullptr;
  MR1L_CUDA(cudaMalloc(&p, (kSmallTw + kFmaTw) * sizeof(cplx)));
  MR1L_CUDA(cudaMemsetAsync(p, 0, kSmallTw * sizeof(cplx), s));
  MR1L_LAUNCH("small_twiddle_kernel", s, 0, 16.0 * kSmallTw,
              small_twiddle_kernel<<<cdiv(kSmallTw, 256), 256, 0, s>>>(p));
  MR1L_LAUNCH("fma_twiddle_kernel", s, 0, 16.0 * kFmaTw,
              fma_twiddle_kernel<<<cdiv(kFmaTw, 256), 256, 0, s>>>(p + kSmallTw));
  MR1L_CUDA(cudaStreamSynchronize(s));
  g_twn[dev] = p;
  return p;
}

__global__ void to_df_kernel(const cplx* src, float4* dst, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = OpsDF::from(src[i]);
}

void to_double_float(const cplx* src, float4* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  MR1L_LAUNCH("to_df_kernel", s, 0, 32.0 * n, to_df_kernel<<<cdiv(n, 256), 256, 0, s>>>(src, dst, n));
}

namespace {
std::map<std::pair<int, int>, float4*> g_tw_df;  // (device, P) -> table
std::map<int, float4*> g_twn_df;
}  // namespace

const float4* twiddle_table_df(int Pn, cudaStream_t s) {
  const cplx* src = twiddle_table(Pn, s);
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto key = std::make_pair(dev, Pn);
  auto it = g_tw_df.find(key);
  if (it != g_tw_df.end()) return it->second;
  float4* p = nullptr;
  MR1L_CUDA(cudaMalloc(&p, (size_t)Pn * sizeof(float4)));
  to_double_float(src, p, Pn, s);
  MR1L_CUDA(cudaStreamSynchronize(s));
  g_tw_df[key] = p;
  return p;
}

// The 4-step twiddles w_P^(n2 k1) (k1 < P1, n2 < P2) copied from the P-point
// table in row order (entry k1 P2 + n2) or column order (entry n2 P1 + k1).
template <class T, bool COLS>
__global__ void ordered_twiddle_kernel(const T* tw, T* out, int P2, int64_t P) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= P) return;
  const int64_t P1 = P / P2;
  const int64_t k1 = COLS ? e % P1 : e / P2, n2 = COLS ? e / P1 : e % P2;
  out[e] = tw[n2 * k1];  // n2 k1 < P2 P1 = P
}

namespace {
// (device, P, column order) -> table
std::map<std::tuple<int, int, int>, cplx*> g_two;
std::map<std::tuple<int, int, int>, float4*> g_two_df;

template <class T, bool COLS>
const T* ordered_twiddles(std::map<std::tuple<int, int, int>, T*>& cache, const T* src, int Pn, int P2,
                          cudaStream_t s) {
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto key = std::make_tuple(dev, Pn, COLS ? 1 : 0);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  T* p = nullptr;
  MR1L_CUDA(cudaMalloc(&p, (size_t)Pn * sizeof(T)));
  MR1L_LAUNCH("ordered_twiddle_kernel", s, 0, 2.0 * sizeof(T) * Pn,
              ordered_twiddle_kernel<T, COLS><<<cdiv(Pn, 256), 256, 0, s>>>(src, p, P2, (int64_t)Pn));
  MR1L_CUDA(cudaStreamSynchronize(s));
  cache[key] = p;
  return p;
}
}  // namespace

const cplx* row_twiddle_table(int Pn, int P2, cudaStream_t s) {
  return ordered_twiddles<cplx, false>(g_two, twiddle_table(Pn, s), Pn, P2, s);
}
const cplx* col_twiddle_table(int Pn, int P2, cudaStream_t s) {
  return ordered_twiddles<cplx, true>(g_two, twiddle_table(Pn, s), Pn, P2, s);
}
const float4* row_twiddle_table_df(int Pn, int P2, cudaStream_t s) {
  return ordered_twiddles<float4, false>(g_two_df, twiddle_table_df(Pn, s), Pn, P2, s);
}
const float4* col_twiddle_table_df(int Pn, int P2, cudaStream_t s) {
  return ordered_twiddles<float4, true>(g_two_df, twiddle_table_df(Pn, s), Pn, P2, s);
}

const float4* small_twiddles_df(cudaStream_t s) {
  const cplx* src = small_twiddles(s);
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto it = g_twn_df.find(dev);
  if (it != g_twn_df.end()) return it->second;
  float4* p = nullptr;
  MR1L_CUDA(cudaMalloc(&p, kSmallTw * sizeof(float4)));
  to_double_float(src, p, kSmallTw, s);
  MR1L_CUDA(cudaStreamSynchronize(s));
  g_twn_df[dev] = p;
  return p;
}

int blue_length(int64_t n) {
  int64_t p2 = 1;
  while (p2 < n) p2 <<= 1;
  int64_t p3 = 3;
  while (p3 < n) p3 <<= 1;
  if (p2 < 4) p2 = 4;
  int64_t best = 0;
  if (p2 <= (int64_t(1) << 25)) best = p2;
  if (p3 <= 3 * (int64_t(1) << 23) && (best == 0 || p3 < best)) best = p3;
  return (int)best;
}

void blue_split(BlueGeom& g, int P) {
  MR1L_REQUIRE(P >= 3 && P == blue_length(P), "unsupported Bluestein length");
  g.P = P;
  if (P <= kSmallMax) {
    g.P1 = 1;
    g.P2 = P;
    return;
  }
  // P2 = 2^b, P1 = P / P2 (2^a or 3 * 2^a), P1 about P2
  const bool three = P % 3 == 0;
  int k = 31 - __builtin_clz((unsigned)(three ? P / 3 : P));
  int b = three ? (k + 2) / 2 : k - k / 2;
  g.P2 = 1 << b;
  g.P1 = P / g.P2;
}

void chirp_tables(const BlueGeom& g, int64_t max_M, cplx* seed, cudaStream_t s) {
  MR1L_LAUNCH("chirp_seed_kernel", s, 0, 16.0 * kChirpSeedLen * g.L,
              chirp_seed_kernel<<<dim3(cdiv(kChirpSeedLen, 256), g.L), 256, 0, s>>>(seed, g.M));
  dim3 grid(cdiv(max_M, 256), g.L);
  MR1L_LAUNCH("chirp_kernel", s, 0, 32.0 * g.sum_M,
              chirp_kernel<<<grid, 256, 0, s>>>(const_cast<cplx*>(g.w), const_cast<cplx*>(g.ws),
                                                const_cast<float4*>(g.w_df), const_cast<float4*>(g.ws_df), g.off,
                                                g.M, seed));
}

template <typename K>
static void set_smem(K kernel, size_t bytes) {
  // the 48 KB default bounds static + dynamic shared memory together, and the
  // column kernels hold up to about 7 KB of static shared memory
  if (bytes > 32 * 1024) MR1L_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

static int threads_for(int elems) {
  int t = elems / 8;
  if (t < 32) t = 32;
  return t;
}

static double fft_flops(double n) { return n > 1 ? 5.0 * n * std::log2(n) : 0.0; }

// Algorithmic work of one launch (FFT flops by the 5 n log2 n convention plus
// 6 flops per complex multiply; bytes that the pass must move).
template <int MODE, class O>
static const char* pass_name(const char* pass, std::string& nm) {
  const bool df = std::is_same<O, OpsDF>::value;
  const char* sfx = MODE == kModeFilter ? "filter" : (MODE == kModeRecon ? "recon" : "eval");
  nm = std::string("blue_") + pass + "_" + sfx + (df ? "_df" : "");
  return nm.c_str();
}

// One pass: the dynamic shared-memory size set on the kernel (and, for forms
// that need room for three CTAs, the largest shared-memory carveout), then
// the launch under its profiling name.
template <typename K>
static void run_pass(K kern, const char* name, dim3 grid, int threads, size_t smem, bool carveout, double flops,
                     double bytes, const BlueGeom& g, const BlueIO& io, cudaStream_t s) {
  set_smem(kern, smem);
  if (carveout)
    MR1L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
  MR1L_LAUNCH(name, s, flops, bytes, kern<<<grid, threads, smem, s>>>(g, io));
}

// The 4-step passes with the tiles in g.ctile / g.rtile.  ev (optional):
// events recorded before the column pass and after each pass.  The FP64
// passes at the block sizes of P = 3 * 2^21 (columns of 3072: 384 threads;
// one row of 2048: 256 threads) use their register-capped forms, as do all
// FP64 rows in CTAs of 512 threads.
template <int MODE, class O>
static void launch_passes(const BlueGeom& g, const BlueIO& io, int ntrans, cudaStream_t s, cudaEvent_t* ev) {
  constexpr bool f64 = std::is_same<O, OpsF64>::value;
  constexpr int kCf = f64 && MODE == kModeEval ? 384 : 512, kR = f64 ? 256 : 512,
                kCi = f64 && MODE != kModeFilter ? 384 : 512;
  const double P = g.P, nr = (double)ntrans / g.L, sumM = (double)g.sum_M;
  const double cb = sizeof(cplx);
  std::string nm;
  int CB = col_tile(g.P1, g.ctile), RB = row_tile(g.P2, g.P1, g.rtile);
  MR1L_REQUIRE(g.P2 % CB == 0 && g.P1 % RB == 0, "tile does not divide the 4-step split");
  size_t smem_c = (size_t)g.P1 * CB * sizeof(cplx);
  size_t smem_r = (size_t)RB * g.P2 * sizeof(cplx);
  dim3 gc(g.P2 / CB, ntrans), gr(g.P1 / RB, ntrans);
  const double P1 = g.P1, P2 = g.P2;
  const int tc = threads_for(g.P1 * CB), tr = threads_for(RB * g.P2);
  MR1L_REQUIRE(tc <= 1024 && tr <= 1024, "4-step tile larger than one CTA");
  if (ev) MR1L_CUDA(cudaEventRecord(ev[0], s));

  const char* name = pass_name<MODE, O>("col_fwd", nm);
  const double fl_cf = ntrans * (P2 * fft_flops(P1) + 6 * P) + nr * 6 * sumM;
  const double by_cf = nr * sumM * cb * 2 + ntrans * P * cb;
  if (kCf == 384 && tc == 384)
    run_pass(blue_col_fwd_kernel<MODE, O, kCf>, name, gc, tc, smem_c, false, fl_cf, by_cf, g, io, s);
  else if (tc <= 512)
    run_pass(blue_col_fwd_kernel<MODE, O>, name, gc, tc, smem_c, false, fl_cf, by_cf, g, io, s);
  else
    run_pass(blue_col_fwd_kernel<MODE, O, 1024>, name, gc, tc, smem_c, false, fl_cf, by_cf, g, io, s);
  if (ev) MR1L_CUDA(cudaEventRecord(ev[1], s));

  name = pass_name<MODE, O>("row", nm);
  if (MODE == kModeFilter) {
    const double fl = ntrans * P1 * fft_flops(P2), by = ntrans * P * cb * 2;
    if (tr <= 512)
      run_pass(blue_row_kernel<true, O>, name, gr, tr, smem_r, false, fl, by, g, io, s);
    else
      run_pass(blue_row_kernel<true, O, 1024>, name, gr, tr, smem_r, false, fl, by, g, io, s);
    if (ev) {
      MR1L_CUDA(cudaEventRecord(ev[2], s));
      MR1L_CUDA(cudaEventRecord(ev[3], s));
    }
    return;
  }
  const double fl_r = ntrans * (2 * P1 * fft_flops(P2) + 12 * P), by_r = ntrans * P * cb * 3;
  if (kR == 256 && tr == 256)
    run_pass(blue_row_kernel<false, O, kR>, name, gr, tr, smem_r, false, fl_r, by_r, g, io, s);
  else if (tr <= 512)
    run_pass(blue_row_kernel<false, O>, name, gr, tr, smem_r, false, fl_r, by_r, g, io, s);
  else
    run_pass(blue_row_kernel<false, O, 1024>, name, gr, tr, smem_r, false, fl_r, by_r, g, io, s);
  if (ev) MR1L_CUDA(cudaEventRecord(ev[2], s));

  name = pass_name<MODE, O>("col_inv", nm);
  const double fl_ci = ntrans * P2 * fft_flops(P1) + (MODE == kModeEval ? nr * 6 * sumM : 0.0);
  const double by_ci = ntrans * P * cb + nr * sumM * cb * (MODE == kModeEval ? 2 : 1);
  if (kCi == 384 && tc == 384)  // three CTAs of 48 KB dynamic and up to 7 KB static shared memory
    run_pass(blue_col_inv_kernel<MODE, O, kCi>, name, gc, tc, smem_c, true, fl_ci, by_ci, g, io, s);
  else if (tc <= 512)
    run_pass(blue_col_inv_kernel<MODE, O>, name, gc, tc, smem_c, false, fl_ci, by_ci, g, io, s);
  else
    run_pass(blue_col_inv_kernel<MODE, O, 1024>, name, gc, tc, smem_c, false, fl_ci, by_ci, g, io, s);
  if (ev) MR1L_CUDA(cudaEventRecord(ev[3], s));
}

// ---------------------------------------------------------------------------
// Tile tuner.  The first 4-step transform of each (device, P, mode,
// arithmetic) runs the three passes once with the default tiles, then once
// per distinct candidate tiling, timed with events on its own stream, and
// keeps the fastest column tile (column
// passes together) and row tile; later transforms reuse the choice.  Every
// tiling computes the same operations in the same order, so the outputs are
// identical bit for bit and the last trial's output stands.  The trials
// synchronise the stream once; a stream being captured, or a caller that
// disables tuning (BlueIO::no_tune, mr1l_tune_enable(0)), gets the default.
// MR1L_TILES=<col>,<row> in the environment fixes the tiles instead.
// ---------------------------------------------------------------------------
struct TileChoice {
  int ctile, rtile;
  float col_ms, row_ms;
};
static std::mutex g_tile_mu;
static std::map<std::tuple<int, int, int, int>, TileChoice> g_tiles;  // (device, P, mode, df)
static std::atomic<int> g_tune_on{-1};                                // -1: read MR1L_TILE_TUNE
static int g_forced[2] = {-1, -1};                                    // MR1L_TILES=<col>,<row>

static bool tuning_enabled() {
  int on = g_tune_on.load();
  if (on < 0) {
    const char* e = std::getenv("MR1L_TILE_TUNE");
    int want = (e && e[0] == '0') ? 0 : 1;
    g_tune_on.compare_exchange_strong(on, want);  // an explicit mr1l_tune_enable wins
    on = g_tune_on.load();
  }
  return on != 0;
}

// Tiles fixed by the environment (MR1L_TILES=<col>,<row>, each one of the
// candidates), for reproducible profiles; {0, 0} when unset.
static std::pair<int, int> forced_tiles() {
  std::lock_guard<std::mutex> lk(g_tile_mu);
  if (g_forced[0] < 0) {
    g_forced[0] = g_forced[1] = 0;
    const char* e = std::getenv("MR1L_TILES");
    int c = 0, r = 0;
    if (e && std::sscanf(e, "%d,%d", &c, &r) == 2) {
      auto ok = [](int t) { return std::find(std::begin(kTileCands), std::end(kTileCands), t) != std::end(kTileCands); };
      MR1L_REQUIRE(ok(c) && ok(r), "MR1L_TILES must name two of the tile sizes 1024, 2048, 4096");
      g_forced[0] = c;
      g_forced[1] = r;
    }
  }
  return {g_forced[0], g_forced[1]};
}

struct EventSet {
  std::vector<cudaEvent_t> ev;
  explicit EventSet(size_t n) : ev(n, nullptr) {
    for (auto& e : ev) MR1L_CUDA(cudaEventCreate(&e));
  }
  ~EventSet() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  }
};

template <int MODE, class O>
static void launch_first_last(const BlueGeom& g, const BlueIO& io, int ntrans, cudaStream_t s) {
  if (g.P <= kSmallMax) {
    const double P = g.P, nr = (double)ntrans / g.L, sumM = (double)g.sum_M;
    const double cb = sizeof(cplx);
    std::string nm;
    size_t smem = (size_t)g.P * sizeof(cplx);
    set_smem(blue_small_kernel<MODE, O>, smem);
    double fl = ntrans * (MODE == kModeFilter ? fft_flops(P) : 2 * fft_flops(P) + 6 * P) + nr * 6 * sumM;
    double by = MODE == kModeFilter ? g.L * P * cb + sumM * cb : nr * sumM * cb * 3 + ntrans * P * cb;
    MR1L_LAUNCH((pass_name<MODE, O>("small", nm)), s, fl, by,
                blue_small_kernel<MODE, O><<<ntrans, threads_for(g.P), smem, s>>>(g, io));
    return;
  }
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, g.P, MODE, (int)std::is_same<O, OpsDF>::value);
  BlueGeom gg = g;
  gg.ctile = gg.rtile = kTileElems;
  const auto forced = forced_tiles();
  if (forced.first) {
    gg.ctile = forced.first;
    gg.rtile = forced.second;
    launch_passes<MODE, O>(gg, io, ntrans, s, nullptr);
    return;
  }
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tiles.find(key);
    if (it != g_tiles.end()) {
      gg.ctile = it->second.ctile;
      gg.rtile = it->second.rtile;
      launch_passes<MODE, O>(gg, io, ntrans, s, nullptr);
      return;
    }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MR1L_CUDA(cudaStreamIsCapturing(s, &cap));
  if (io.no_tune || !tuning_enabled() || cap != cudaStreamCaptureStatusNone) {
    launch_passes<MODE, O>(gg, io, ntrans, s, nullptr);
    return;
  }
  // distinct candidate tilings (equal CB and RB give the same launch)
  std::vector<int> cands;
  std::vector<std::pair<int, int>> seen;
  for (int t : kTileCands) {
    auto cr = std::make_pair(col_tile(g.P1, t), row_tile(g.P2, g.P1, t));
    if (std::find(seen.begin(), seen.end(), cr) == seen.end()) {
      seen.push_back(cr);
      cands.push_back(t);
    }
  }
  // one untimed run first: it pays the kernels' first-launch costs and leaves
  // every timed trial the same cache state
  launch_passes<MODE, O>(gg, io, ntrans, s, nullptr);
  EventSet es(4 * cands.size());
  for (size_t i = 0; i < cands.size(); ++i) {
    gg.ctile = gg.rtile = cands[i];
    launch_passes<MODE, O>(gg, io, ntrans, s, &es.ev[4 * i]);
  }
  MR1L_CUDA(cudaEventSynchronize(es.ev.back()));
  TileChoice best{kTileElems, kTileElems, 1e30f, 1e30f};
  for (size_t i = 0; i < cands.size(); ++i) {
    float c1 = 0, r = 0, c2 = 0;
    MR1L_CUDA(cudaEventElapsedTime(&c1, es.ev[4 * i], es.ev[4 * i + 1]));
    MR1L_CUDA(cudaEventElapsedTime(&r, es.ev[4 * i + 1], es.ev[4 * i + 2]));
    MR1L_CUDA(cudaEventElapsedTime(&c2, es.ev[4 * i + 2], es.ev[4 * i + 3]));
    if (c1 + c2 < best.col_ms) {
      best.col_ms = c1 + c2;
      best.ctile = cands[i];
    }
    if (r < best.row_ms) {
      best.row_ms = r;
      best.rtile = cands[i];
    }
  }
  std::lock_guard<std::mutex> lk(g_tile_mu);
  g_tiles.emplace(key, best);
}

void tune_enable(int on) { g_tune_on.store(on ? 1 : 0); }

void tune_reset() {
  std::lock_guard<std::mutex> lk(g_tile_mu);
  g_tiles.clear();
}

std::string tune_json() {
  std::lock_guard<std::mutex> lk(g_tile_mu);
  static const char* modes[3] = {"filter", "recon", "eval"};
  std::string out = "[";
  char buf[256];
  for (const auto& kv : g_tiles) {
    std::snprintf(buf, sizeof buf,
                  "%s{\"device\": %d, \"P\": %d, \"mode\": \"%s\", \"df\": %d, \"col_tile\": %d, \"row_tile\": %d, "
                  "\"col_ms\": %.4f, \"row_ms\": %.4f}",
                  out.size() > 1 ? ", " : "", std::get<0>(kv.first), std::get<1>(kv.first),
                  modes[std::get<2>(kv.first)], std::get<3>(kv.first), kv.second.ctile, kv.second.rtile,
                  kv.second.col_ms, kv.second.row_ms);
    out += buf;
  }
  return out + "]";
}

void blue_filter(const BlueGeom& g, cudaStream_t s) {
  // the filter pass needs P complex of scratch per lattice: use Bh itself as
  // the 4-step work buffer (pass 1 writes it, pass 2 overwrites it in place
  // row by row; each row is read completely before it is written)
  BlueIO io{};
  io.work = g.Bh;
  if (g.df)
    launch_first_last<kModeFilter, OpsDF>(g, io, g.L, s);
  else
    launch_first_last<kModeFilter, OpsF64>(g, io, g.L, s);
}

// ---------------------------------------------------------------------------
// Lattice noise: y[h][off_l + j] += sigma/sqrt(2) (g1 + i g2) by Box-Muller on
// the Philox words of sample j (purpose 5; node 0 shared by all lattices):
// u1 = Q 2^-53 with Q = (a >> 11) + 1 in [1, 2^53], u2 = B 2^-53 with
// B = b >> 11, g1 + i g2 = sqrt(-2 ln u1) e^{2 pi i u2}.
//
// The draws are evaluated in double-float arithmetic (arith.cuh) on the FP32
// pipes, from the integers Q and B, with table-driven functions:
//   ln u1 = E ln2 + ln c_k + log1p(r): Q = 2^e m with m in [3/4, 3/2),
//     E = e - 53, c_k = 1 + k / 4096 with k = trunc(4096 (m - 1)) (so c = 1 for
//     m near 1 and the result keeps its relative accuracy there),
//     r = (m - c_k) / c_k where 2^e (m - c_k) is an exact integer, |r| < 2^-11.5,
//     log1p(r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 (Tang's table-driven
//     logarithm, ACM TOMS 16(4), 1990);
//   sqrt by one Newton correction of the FP32 square root in double-float;
//   2 pi u2 = 2 pi q / 256 + x with q = B >> 45 and x in [0, 2 pi / 256) from
//     the low 45 bits (exact in double-float); sin x and cos x by their Taylor
//     series to degrees 7 and 8, combined with the tabulated sin / cos of
//     2 pi q / 256 by the angle-addition formulas.
// Terms of the series below about 2^-22 relative are summed in plain FP32.
// The result is within about 2^-46 of |g1 + i g2| (the FP64 draws of the
// oracle differ from it by no more than that); only the final conversion to
// FP64 uses the FP64 pipe.
// ---------------------------------------------------------------------------
constexpr int kLnCells = 4096;                   // cells per unit of m
constexpr int kLnTab = 3 * kLnCells / 4;          // k in [-kLnCells/4, kLnCells/2)
constexpr int kScTab = 256;

struct NoiseTables {
  float4 ln[kLnTab];  // (ln c).hi, (ln c).lo, (1/c).hi, (1/c).lo for c = 1 + (i - kLnCells/4) / kLnCells
  float4 sc[kScTab];  // sin.hi, sin.lo, cos.hi, cos.lo of 2 pi i / kScTab
};

__device__ __forceinline__ float2 split_df(double x) {
  float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

__global__ void noise_tables_kernel(NoiseTables* t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kLnTab) {
    double c = 1.0 + (double)(i - kLnCells / 4) / (double)kLnCells;  // exact
    float2 lc = split_df(log(c)), ic = split_df(1.0 / c);
    t->ln[i] = make_float4(lc.x, lc.y, ic.x, ic.y);
  }
  if (i < kScTab) {
    double sn, cs;
    sincospi(2.0 * (double)i / kScTab, &sn, &cs);
    float2 a = split_df(sn), b = split_df(cs);
    t->sc[i] = make_float4(a.x, a.y, b.x, b.y);
  }
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // |e| <= 126

// ln(Q 2^-53) for Q in [1, 2^53] as a double-float (<= 0)
__device__ __forceinline__ void ln_q53(uint64_t Q, const NoiseTables* T, float& lh, float& ll) {
  int e = 63 - __clzll((long long)Q);           // Q in [2^e, 2^(e+1))
  if (e > 0 && (Q >> (e - 1)) >= 3) ++e;        // m = Q / 2^e in [3/4, 3/2)
  const long long num = (long long)Q - (1LL << e);  // 2^e (m - 1)
  int k;
  long long D;                                   // 2^e (m - c_k), exact
  if (e >= 12) {
    const int sh = e - 12;
    const long long a = num < 0 ? -num : num;
    const long long kq = a >> sh;                // trunc(4096 |m - 1|)
    k = (int)(num < 0 ? -kq : kq);
    D = num - (long long)k * (1LL << sh);
  } else {
    k = (int)(num * (1LL << (12 - e)));          // m is a cell point
    D = 0;
  }
  // D (|D| < 2^42) as an exact double-float, scaled by 2^-e
  const long long dq = D / (1LL << 21);          // truncates: dq and the rest share D's sign
  float dh, dl;
  two_sum((float)(int)dq * 2097152.0f, (float)(int)(D - dq * (1LL << 21)), dh, dl);
  const float sc = pow2f(-e);
  const float4 tk = __ldg(&T->ln[k + kLnCells / 4]);
  float rh, rl;
  dw_mul(dh * sc, dl * sc, tk.z, tk.w, rh, rl);  // r = (m - c) / c
  // log1p(r): r - r^2/2 in double-float, the rest in FP32
  const float p = __fmul_rn(rh, rh);
  float pe = __fmaf_rn(rh, rh, -p);
  pe = __fmaf_rn(2.0f * rh, rl, pe);
  float tail = __fmaf_rn(rh, 0.2f, -0.25f);
  tail = __fmaf_rn(rh, tail, 0.33333334f);
  tail = __fmul_rn(__fmul_rn(rh, p), tail);
  float ah, al;
  dw_add(rh, rl, -0.5f * p, -0.5f * pe, ah, al);
  dw_add(ah, al, tail, 0.0f, ah, al);
  // + E ln2 + ln c
  float eh, el;
  dw_mul((float)(e - 53), 0.0f, 0x1.62e430p-1f, -0x1.05c610p-29f, eh, el);
  dw_add(eh, el, tk.x, tk.y, eh, el);
  dw_add(eh, el, ah, al, lh, ll);
}

// sqrt of a non-negative double-float
__device__ __forceinline__ void dw_sqrt(float xh, float xl, float& sh, float& sl) {
  const float s = __fsqrt_rn(xh);
  if (!(s > 0.0f)) {
    sh = 0.0f;
    sl = 0.0f;
    return;
  }
  const float p = __fmul_rn(s, s), pe = __fmaf_rn(s, s, -p);  // s^2 = p + pe
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(xh, p), pe), xl);
  fast_two_sum(s, __fmul_rn(d, __frcp_rn(2.0f * s)), sh, sl);
}

// (sin, cos) of 2 pi B 2^-53 for B in [0, 2^53), as double-floats
__device__ __forceinline__ void sincos_b53(uint64_t B, const NoiseTables* T, float2& sn, float2& cs) {
  const int q = (int)(B >> 45);
  const uint64_t F = B & ((1ull << 45) - 1);     // x = 2 pi F 2^-45 / 256
  float fh, fl;
  two_sum((float)(uint32_t)(F >> 21) * 0x1p-24f, (float)(uint32_t)(F & 0x1fffff) * 0x1p-45f, fh, fl);
  float th, tl;
  dw_mul(fh, fl, 0x1.921fb6p-6f, -0x1.777a5cp-31f, th, tl);  // 2 pi / 256
  float zh, zl;
  dw_mul(th, tl, th, tl, zh, zl);                // x^2
  // sin x = x (1 - x^2/6 + x^4/120 - x^6/5040)
  float ts = __fmaf_rn(zh, -1.0f / 5040.0f, 1.0f / 120.0f);
  ts = __fmul_rn(__fmul_rn(zh, zh), ts);
  float ah, al;
  dw_mul(zh, zl, 0x1.555556p-3f, -0x1.555556p-28f, ah, al);  // x^2 / 6
  dw_add(1.0f, 0.0f, -ah, -al, ah, al);
  dw_add(ah, al, ts, 0.0f, ah, al);
  float sxh, sxl;
  dw_mul(th, tl, ah, al, sxh, sxl);
  // cos x = 1 - x^2/2 + x^4/24 - x^6/720 + x^8/40320
  float tc = __fmaf_rn(zh, 1.0f / 40320.0f, -1.0f / 720.0f);
  tc = __fmaf_rn(zh, tc, 1.0f / 24.0f);
  tc = __fmul_rn(__fmul_rn(zh, zh), tc);
  float cxh, cxl;
  dw_add(1.0f, 0.0f, -0.5f * zh, -0.5f * zl, cxh, cxl);
  dw_add(cxh, cxl, tc, 0.0f, cxh, cxl);
  const float4 tq = __ldg(&T->sc[q]);            // sin, cos of 2 pi q / 256
  dw_dot2(tq.x, tq.y, cxh, cxl, tq.z, tq.w, sxh, sxl, 1.0f, sn.x, sn.y);
  dw_dot2(tq.z, tq.w, cxh, cxl, tq.x, tq.y, sxh, sxl, -1.0f, cs.x, cs.y);
}

__global__ void __launch_bounds__(256) lattice_noise_kernel(BlueGeom g, BlueIO io, const NoiseTables* T, float sch,
                                                           float scl) {
  const int l = blockIdx.y, h = blockIdx.z;
  const int M = g.M[l];
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  U64Pair u = philox_u64(io.noise_seed, kNoiseLattice, (uint32_t)io.noise_t, (uint32_t)j, j == 0 ? 0u : (uint32_t)l,
                         (uint32_t)(io.noise_rep + h * io.noise_rep_per_rhs));
  float lh, ll, Rh, Rl;
  ln_q53((u.a >> 11) + 1, T, lh, ll);
  dw_sqrt(-2.0f * lh, -2.0f * ll, Rh, Rl);
  float2 sn, cs;
  sincos_b53(u.b >> 11, T, sn, cs);
  dw_mul(Rh, Rl, sch, scl, Rh, Rl);
  float reh, rel, imh, iml;
  dw_mul(Rh, Rl, cs.x, cs.y, reh, rel);
  dw_mul(Rh, Rl, sn.x, sn.y, imh, iml);
  const cplx e = cmake((double)reh + (double)rel, (double)imh + (double)iml);
  cplx* y = io.out + h * io.out_stride + g.off[l] + j;
  *y = io.noise_write ? e : cadd(*y, e);
}

static std::mutex g_noise_mu;
static std::map<int, NoiseTables*> g_noise_tabs;

static const NoiseTables* noise_tables(cudaStream_t s) {
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noise_mu);
  auto it = g_noise_tabs.find(dev);
  if (it != g_noise_tabs.end()) return it->second;
  NoiseTables* t = nullptr;
  MR1L_CUDA(cudaMalloc(&t, sizeof(NoiseTables)));
  MR1L_LAUNCH("noise_tables_kernel", s, 0, (double)sizeof(NoiseTables),
              noise_tables_kernel<<<cdiv(kLnTab, 256), 256, 0, s>>>(t));
  MR1L_CUDA(cudaStreamSynchronize(s));
  g_noise_tabs[dev] = t;
  return t;
}

void add_lattice_noise(const BlueGeom& g, const BlueIO& io, int nrhs, cudaStream_t s) {
  if (io.noise_scale == 0.0 || nrhs == 0) return;
  int maxM = (int)std::min<int64_t>(g.sum_M, g.P / 2 + 1);
  dim3 grid(cdiv(maxM, 256), g.L, nrhs);
  const NoiseTables* tabs = noise_tables(s);
  const float sch = static_cast<float>(io.noise_scale);
  const float scl = static_cast<float>(io.noise_scale - (double)sch);
  MR1L_LAUNCH("lattice_noise_kernel", s, 0, 32.0 * nrhs * g.sum_M,
              lattice_noise_kernel<<<grid, 256, 0, s>>>(g, io, tabs, sch, scl));
}

void blue_run(const BlueGeom& g, const BlueIO& io, int mode, int nrhs, cudaStream_t s) {
  int ntrans = g.L * nrhs;
  if (ntrans == 0) return;
  if (mode == kModeRecon) {
    if (g.df)
      launch_first_last<kModeRecon, OpsDF>(g, io, ntrans, s);
    else
      launch_first_last<kModeRecon, OpsF64>(g, io, ntrans, s);
    return;
  }
  if (g.df)
    launch_first_last<kModeEval, OpsDF>(g, io, ntrans, s);
  else
    launch_first_last<kModeEval, OpsF64>(g, io, ntrans, s);
  add_lattice_noise(g, io, nrhs, s);
}

}  // namespace mr1l
