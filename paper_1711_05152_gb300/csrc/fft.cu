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
#include <map>
#include <mutex>
#include <string>
#include <type_traits>

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
// One Stockham stage of radix R over nseq sequences of length n in shared
// memory; element i of sequence b sits at s[b * bs + i * is].  The block has
// nseq * n / 8 threads (or more, which idle); each thread runs up to
// ceil(8 / R) butterflies of the stage.
//   COLS: sequence index fastest across threads (column tiles, bs == 1)
//   else: element index fastest (row tiles, is == 1)
// HALF (first radix-8 stage only): inputs r >= 4 are known zeros.
// ---------------------------------------------------------------------------
template <int R, bool INV, bool COLS, class O, bool HALF = false>
__device__ __forceinline__ void stockham_stage(typename O::V* s, int n, int Ns, int nseq, int bs, int is,
                                               const typename O::V* twn_n) {
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
      const V* src = s + b * bs + j * is;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[c][r] = src[r * nb * is];
      reg_dft8_half<INV, O>(v[c]);
    } else if (act[c]) {
      const V* src = s + b * bs + j * is;
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = src[r * nb * is];
      if (Ns > 1) {
        int step = k * (n / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r) {
          V w = twn_n[r * step];
          v[c][r] = INV ? O::mulc(v[c][r], w) : O::mul(v[c][r], w);
        }
      }
      RegDft<R, INV, O>::run(v[c]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    if (act[c]) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[base[c] + r * Ns * is] = v[c][r];
    }
  }
  __syncthreads();
}

// Twiddles exp(-2 pi i e / n) of a sub-FFT length n (2^a or 3 * 2^a).
template <class T>
__device__ __forceinline__ const T* twiddles_of(const T* twn, int n) {
  return (n & (n - 1)) == 0 ? twn + n : twn + 8192 + n - 3;
}

// Full in-smem FFT of length n = 2^a or 3 * 2^a: radix-8 stages, one radix-4
// or radix-2 stage for the rest of 2^a, then radix 3.  Natural order in and
// out.  HALF_FIRST: the upper half of every input sequence is zero (needs
// 8 | n).
template <bool INV, bool COLS, class O, bool HALF_FIRST = false>
__device__ __forceinline__ void smem_fft(typename O::V* s, int n, int nseq, int bs, int is,
                                         const typename O::V* twn) {
  const typename O::V* twn_n = twiddles_of(twn, n);
  const bool three = (n % 3) == 0;
  int rem = 31 - __clz(three ? n / 3 : n);  // log2 of the power-of-two part
  int Ns = 1;
  if (HALF_FIRST && rem >= 3) {
    stockham_stage<8, INV, COLS, O, true>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 3;
    rem -= 3;
  }
  while (rem >= 3) {
    stockham_stage<8, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 3;
    rem -= 3;
  }
  if (rem == 2) {
    stockham_stage<4, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 2;
  }
  if (rem == 1) {
    stockham_stage<2, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 1;
  }
  if (three) stockham_stage<3, INV, COLS, O>(s, n, Ns, nseq, bs, is, twn_n);
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
  static __device__ __forceinline__ const cplx* twn(const BlueGeom& g) { return g.twn; }
  static __device__ __forceinline__ cplx* Bh(const BlueGeom& g) { return g.Bh; }
};
template <>
struct Tab<OpsDF> {
  static __device__ __forceinline__ const float4* w(const BlueGeom& g) { return g.w_df; }
  static __device__ __forceinline__ const float4* ws(const BlueGeom& g) { return g.ws_df; }
  static __device__ __forceinline__ const float4* tw(const BlueGeom& g) { return g.tw_df; }
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
  if (MODE == kModeRecon && io.add_in) y = cadd(y, io.add_in[h * io.in_stride + off + n]);
  typename O::V x = O::from(y);
  if (MODE == kModeRecon) return O::mul(x, Tab<O>::ws(g)[off + n]);
  return O::mul(O::conj(x), Tab<O>::w(g)[off + n]);
}

template <int MODE, class O>
__device__ __forceinline__ void store_output(const BlueGeom& g, const BlueIO& io, int h, int64_t off, int64_t n,
                                             typename O::V v) {
  if (MODE == kModeRecon)
    io.out[h * io.out_stride + off + n] = O::to(v);
  else
    io.out[h * io.out_stride + off + n] = O::to(O::conj(O::mul(Tab<O>::w(g)[off + n], v)));
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
  if (MODE == kModeFilter) {
    const double sc = 1.0 / (double)P;
    const float sh = __double2float_rn(sc), sl = __double2float_rn(sc - (double)sh);
    for (int n = threadIdx.x; n < P; n += blockDim.x) Bh[n] = O::scalec(sm[n], sc, sh, sl);
    return;
  }
  for (int n = threadIdx.x; n < P; n += blockDim.x) sm[n] = O::mul(sm[n], Bh[n]);
  __syncthreads();
  smem_fft<true, false, O>(sm, P, 1, 0, 1, Tab<O>::twn(g));
  for (int n = threadIdx.x; n < M; n += blockDim.x) store_output<MODE, O>(g, io, h, off, n, sm[n]);
}

// ---------------------------------------------------------------------------
// 4-step passes
// ---------------------------------------------------------------------------
// Tiles of 2048 complex (32 KB shared memory, 256 threads) so that three CTAs
// share an SM and hide each other's load and barrier phases; a single
// column or row of more than 2048 takes a tile of its own length.
constexpr int kTileElems = 2048;
__host__ __device__ __forceinline__ int col_tile(int P1) {
  int cb = kTileElems / P1;  // P1 = 3 * 2^a gives a tile of 3/4 x 2048
  if (cb > 16) cb = 16;
  if (cb < 1) cb = 1;
  int p = 1;  // power of two, so it divides P2
  while (2 * p <= cb) p *= 2;
  return p;
}
__host__ __device__ __forceinline__ int row_tile(int P2) {
  int rb = kTileElems / P2;
  return rb < 1 ? 1 : rb;
}

// Pass 1: columns, forward, with the 4-step twiddle.
template <int MODE, class O>
__global__ void __launch_bounds__(512) blue_col_fwd_kernel(BlueGeom g, BlueIO io) {
  typedef typename O::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = (V*)smraw;
  const int gi = blockIdx.y;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, P1 = g.P1, P2 = g.P2, CB = col_tile(P1);
  const int M = g.M[l];
  const int64_t off = g.off[l];
  const int n2_0 = blockIdx.x * CB;
  // RECON / EVAL: rows n1 >= P1/2 hold n >= P/2 >= M, i.e. zero padding
  const int rows = MODE == kModeFilter ? P1 : P1 / 2;
  V* work = (V*)io.work + (int64_t)gi * P;
  // 4-step twiddle w_P^(n2 k1): n2 < P2 and k1 < P1, so n2 k1 < P indexes the
  // table without reduction
  const V* tw = Tab<O>::tw(g);
  if (MODE == kModeEval) {
    // Evaluation inputs are often sparse (the bins of a few planted
    // frequencies).  Columns with at most kColNz non-zeros are transformed as
    // direct sums X[k1] = sum_nz x[n1] w_P1^(n1 k1), cheaper than the FFT.
    constexpr int kColNz = 8;
    __shared__ int nzc[16];
    __shared__ short nzi[16][kColNz];
    __shared__ int over;
    if (threadIdx.x < 16) nzc[threadIdx.x] = 0;
    if (threadIdx.x == 0) over = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < rows * CB; e += blockDim.x) {
      int i = e / CB, b = e - i * CB;
      V x = load_input<MODE, O>(g, io, h, M, off, (int64_t)i * P2 + n2_0 + b);
      sm[e] = x;
      if (O::nonzero(x)) {
        int slot = atomicAdd(&nzc[b], 1);
        if (slot < kColNz) nzi[b][slot] = (short)i;
        else over = 1;
      }
    }
    __syncthreads();
    if (!over) {
      const V* twP1 = twiddles_of(Tab<O>::twn(g), P1);
      for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
        int k1 = e / CB, b = e - k1 * CB;
        V acc = O::zero();
        for (int q = 0; q < nzc[b]; ++q) {
          int n1 = nzi[b][q];
          acc = O::add(acc, O::mul(sm[n1 * CB + b], twP1[(n1 * k1) % P1]));
        }
        int n2 = n2_0 + b;
        work[(int64_t)k1 * P2 + n2] = O::mul(acc, tw[n2 * k1]);
      }
      return;
    }
  } else {
    for (int e = threadIdx.x; e < rows * CB; e += blockDim.x) {
      int i = e / CB, b = e - i * CB;
      sm[e] = load_input<MODE, O>(g, io, h, M, off, (int64_t)i * P2 + n2_0 + b);
    }
    __syncthreads();
  }
  if (MODE == kModeFilter)
    smem_fft<false, true, O>(sm, P1, CB, 1, CB, Tab<O>::twn(g));
  else
    smem_fft<false, true, O, true>(sm, P1, CB, 1, CB, Tab<O>::twn(g));
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int k1 = e / CB, b = e - k1 * CB;
    int n2 = n2_0 + b;
    work[(int64_t)k1 * P2 + n2] = O::mul(sm[e], tw[n2 * k1]);
  }
}

// Pass 2: rows.  FILTER: forward FFT scaled by 1/P into Bh.  Otherwise forward
// FFT, times Bh, inverse FFT, times conj(w_P^(n2 k1)).
template <bool FILTER, class O>
__global__ void __launch_bounds__(512) blue_row_kernel(BlueGeom g, BlueIO io) {
  typedef typename O::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = (V*)smraw;
  const int gi = blockIdx.y;
  const int l = gi % g.L;
  const int P = g.P, P2 = g.P2, RB = row_tile(P2);
  const int k1_0 = blockIdx.x * RB;
  V* work = (V*)io.work + (int64_t)gi * P + (int64_t)k1_0 * P2;
  for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) sm[e] = work[e];
  __syncthreads();
  smem_fft<false, false, O>(sm, P2, RB, P2, 1, Tab<O>::twn(g));
  V* Bh = Tab<O>::Bh(g) + (int64_t)l * P + (int64_t)k1_0 * P2;
  if (FILTER) {
    const double sc = 1.0 / (double)P;
    const float sh = __double2float_rn(sc), sl = __double2float_rn(sc - (double)sh);
    for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) Bh[e] = O::scalec(sm[e], sc, sh, sl);
    return;
  }
  for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) sm[e] = O::mul(sm[e], Bh[e]);
  __syncthreads();
  smem_fft<true, false, O>(sm, P2, RB, P2, 1, Tab<O>::twn(g));
  const V* tw = Tab<O>::tw(g);
  for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) {
    int b = e / P2, n2 = e - b * P2;
    int k1 = k1_0 + b;
    work[e] = O::mulc(sm[e], tw[n2 * k1]);
  }
}

// Pass 3: columns, inverse; natural-order output n = n1 P2 + n2 for n < M.
template <int MODE, class O>
__global__ void __launch_bounds__(512) blue_col_inv_kernel(BlueGeom g, BlueIO io) {
  typedef typename O::V V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = (V*)smraw;
  const int gi = blockIdx.y;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, P1 = g.P1, P2 = g.P2, CB = col_tile(P1);
  const int M = g.M[l];
  const int64_t off = g.off[l];
  const int n2_0 = blockIdx.x * CB;
  const V* work = (const V*)io.work + (int64_t)gi * P;
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int k1 = e / CB, b = e - k1 * CB;
    sm[e] = work[(int64_t)k1 * P2 + n2_0 + b];
  }
  __syncthreads();
  smem_fft<true, true, O>(sm, P1, CB, 1, CB, Tab<O>::twn(g));
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int n1 = e / CB, b = e - n1 * CB;
    int64_t n = (int64_t)n1 * P2 + n2_0 + b;
    if (n < M) store_output<MODE, O>(g, io, h, off, n, sm[e]);
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
  if (i < 8192) {  // n = 2^a at [n, 2n)
    n = 1 << (31 - __clz(i));
    e = i - n;
  } else {         // n = 3 * 2^a at [8192 + n - 3, 8192 + 2n - 3)
    int j = i - 8192 + 3;              // in [n, 2n) for n = 3 * 2^a
    int a = 31 - __clz(j / 3);
    n = 3 << a;
    e = j - n;
  }
  double sn, cs;
  sincospi(2.0 * (double)e / (double)n, &sn, &cs);
  tw[i] = cmake(cs, -sn);
}

__global__ void chirp_kernel(cplx* w, cplx* ws, float4* w_df, float4* ws_df, const int64_t* off, const int* Ms,
                             int L) {
  int l = blockIdx.y;
  int M = Ms[l];
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= M) return;
  uint64_t q = ((uint64_t)n * (uint64_t)n) % (uint64_t)(2 * (int64_t)M);  // exact n^2 mod 2M
  double s, c;
  sincospi((double)q / (double)M, &s, &c);
  cplx v = cmake(c, -s);  // exp(-pi i q / M)
  double inv = 1.0 / (double)M;
  cplx vs = cmake(c * inv, -s * inv);
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
  MR1L_CUDA(cudaMalloc(&p, kSmallTw * sizeof(cplx)));
  MR1L_CUDA(cudaMemsetAsync(p, 0, kSmallTw * sizeof(cplx), s));
  MR1L_LAUNCH("small_twiddle_kernel", s, 0, 16.0 * kSmallTw,
              small_twiddle_kernel<<<cdiv(kSmallTw, 256), 256, 0, s>>>(p));
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
  if (p2 <= (int64_t(1) << 24)) best = p2;
  if (p3 <= 3 * (int64_t(1) << 22) && (best == 0 || p3 < best)) best = p3;
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

void chirp_tables(const BlueGeom& g, int64_t max_M, cudaStream_t s) {
  dim3 grid(cdiv(max_M, 256), g.L);
  MR1L_LAUNCH("chirp_kernel", s, 0, 32.0 * g.sum_M,
              chirp_kernel<<<grid, 256, 0, s>>>(const_cast<cplx*>(g.w), const_cast<cplx*>(g.ws), const_cast<float4*>(g.w_df),
                                    const_cast<float4*>(g.ws_df), g.off, g.M, g.L));
}

template <typename K>
static void set_smem(K kernel, size_t bytes) {
  // the 48 KB default bounds static + dynamic shared memory together, and the
  // column kernels hold a few hundred bytes of static shared memory
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
static void launch_first_last(const BlueGeom& g, const BlueIO& io, int ntrans, cudaStream_t s) {
  const bool df = std::is_same<O, OpsDF>::value;
  const double P = g.P, nr = (double)ntrans / g.L, sumM = (double)g.sum_M;
  const double cb = sizeof(cplx);
  const char* sfx = MODE == kModeFilter ? "filter" : (MODE == kModeRecon ? "recon" : "eval");
  std::string nm;
  auto name = [&](const char* pass) {
    nm = std::string("blue_") + pass + "_" + sfx + (df ? "_df" : "");
    return nm.c_str();
  };
  if (g.P <= kSmallMax) {
    size_t smem = (size_t)g.P * sizeof(cplx);
    set_smem(blue_small_kernel<MODE, O>, smem);
    double fl = ntrans * (MODE == kModeFilter ? fft_flops(P) : 2 * fft_flops(P) + 6 * P) + nr * 6 * sumM;
    double by = MODE == kModeFilter ? g.L * P * cb + sumM * cb : nr * sumM * cb * 3 + ntrans * P * cb;
    MR1L_LAUNCH(name("small"), s, fl, by, blue_small_kernel<MODE, O><<<ntrans, threads_for(g.P), smem, s>>>(g, io));
    return;
  }
  int CB = col_tile(g.P1), RB = row_tile(g.P2);
  size_t smem_c = (size_t)g.P1 * CB * sizeof(cplx);
  size_t smem_r = (size_t)RB * g.P2 * sizeof(cplx);
  dim3 gc(g.P2 / CB, ntrans), gr(g.P1 / RB, ntrans);
  const double P1 = g.P1, P2 = g.P2;
  set_smem(blue_col_fwd_kernel<MODE, O>, smem_c);
  MR1L_LAUNCH(name("col_fwd"), s, ntrans * (P2 * fft_flops(P1) + 6 * P) + nr * 6 * sumM,
              nr * sumM * cb * 2 + ntrans * P * cb,
              blue_col_fwd_kernel<MODE, O><<<gc, threads_for(g.P1 * CB), smem_c, s>>>(g, io));
  if (MODE == kModeFilter) {
    set_smem(blue_row_kernel<true, O>, smem_r);
    MR1L_LAUNCH(name("row"), s, ntrans * P1 * fft_flops(P2), ntrans * P * cb * 2,
                blue_row_kernel<true, O><<<gr, threads_for(RB * g.P2), smem_r, s>>>(g, io));
    return;
  }
  set_smem(blue_row_kernel<false, O>, smem_r);
  MR1L_LAUNCH(name("row"), s, ntrans * (2 * P1 * fft_flops(P2) + 12 * P), ntrans * P * cb * 3,
              blue_row_kernel<false, O><<<gr, threads_for(RB * g.P2), smem_r, s>>>(g, io));
  set_smem(blue_col_inv_kernel<MODE, O>, smem_c);
  MR1L_LAUNCH(name("col_inv"), s, ntrans * P2 * fft_flops(P1) + (MODE == kModeEval ? nr * 6 * sumM : 0.0),
              ntrans * P * cb + nr * sumM * cb * (MODE == kModeEval ? 2 : 1),
              blue_col_inv_kernel<MODE, O><<<gc, threads_for(g.P1 * CB), smem_c, s>>>(g, io));
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
// the Philox words of sample j (purpose 5; node 0 shared by all lattices).
//
// The logarithm and the sine/cosine are table driven so that the FP64 pipe
// does little work per sample:
//   ln u = E ln2 + ln c_k + log1p(r),  u = 2^E m with m in [3/4, 3/2),
//     c_k = 1 + trunc(128 (m - 1)) / 128 (so c = 1 for m near 1 and the result
//     keeps its relative accuracy there), r = (m - c_k) / c_k with m - c_k
//     exact, |r| < 1/96, log1p by its Taylor series to degree 9 (Tang's
//     table-driven logarithm, ACM TOMS 16(4), 1990);
//   2 pi u = 2 pi q / 256 + x,  x in [0, 2 pi / 256): sin and cos of x by
//     their Taylor series (degrees 7 and 8), combined with the tabulated
//     sin / cos of 2 pi q / 256 by the angle-addition formulas.
// Both stay within a few units in the last place of FP64.
// ---------------------------------------------------------------------------
constexpr int kLnTab = 96, kScTab = 256;

struct NoiseTables {
  double inv_c[kLnTab], ln_c[kLnTab];
  double sn[kScTab], cs[kScTab];
};

__global__ void noise_tables_kernel(NoiseTables* t) {
  int i = threadIdx.x;
  if (i < kLnTab) {
    double c = 1.0 + (double)(i - 32) / 128.0;  // exact
    t->inv_c[i] = 1.0 / c;
    t->ln_c[i] = log(c);
  }
  if (i < kScTab) {
    double sn, cs;
    sincospi(2.0 * (double)i / kScTab, &sn, &cs);
    t->sn[i] = sn;
    t->cs[i] = cs;
  }
}

// ln u for u in (0, 1] (normal doubles)
__device__ __forceinline__ double ln_unit(double u, const NoiseTables& T) {
  const double LN2 = 0.69314718055994530942;
  long long b = __double_as_longlong(u);
  int E = (int)((b >> 52) & 0x7ff) - 1023;
  double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);  // [1, 2)
  if (m >= 1.5) {
    m *= 0.5;  // exact
    E += 1;
  }
  const double d = m - 1.0;                     // exact
  const int k = 32 + (int)trunc(d * 128.0);     // table cell, c_k = 1 + (k - 32) / 128
  const double c = 1.0 + (double)(k - 32) * 0.0078125;
  const double r = (m - c) * T.inv_c[k];        // m - c exact
  // log1p(r) = r - r^2/2 + r^3/3 - ... + r^9/9
  double p = fma(r, 1.0 / 9.0, -1.0 / 8.0);
  p = fma(r, p, 1.0 / 7.0);
  p = fma(r, p, -1.0 / 6.0);
  p = fma(r, p, 1.0 / 5.0);
  p = fma(r, p, -1.0 / 4.0);
  p = fma(r, p, 1.0 / 3.0);
  p = fma(r, p, -0.5);
  p = fma(r * r, p, r);
  return fma((double)E, LN2, T.ln_c[k] + p);
}

// (sin, cos) of 2 pi u for u in [0, 1) on the 2^-53 grid
__device__ __forceinline__ void sincos_2pi(double u, const NoiseTables& T, double& s, double& c) {
  const double K = 0.024543692606170259675;  // 2 pi / 256
  double v = u * kScTab;                     // exact
  double q = floor(v);
  int iq = (int)q;
  double x = (v - q) * K;
  double x2 = x * x;
  double ps = fma(x2, -1.0 / 5040.0, 1.0 / 120.0);
  ps = fma(x2, ps, -1.0 / 6.0);
  double sx = fma(x * x2, ps, x);
  double pc = fma(x2, 1.0 / 40320.0, -1.0 / 720.0);
  pc = fma(x2, pc, 1.0 / 24.0);
  pc = fma(x2, pc, -0.5);
  double cx = fma(x2, pc, 1.0);
  double sq = T.sn[iq], cq = T.cs[iq];
  s = fma(sq, cx, cq * sx);
  c = fma(cq, cx, -sq * sx);
}

__global__ void __launch_bounds__(256) lattice_noise_kernel(BlueGeom g, BlueIO io, const NoiseTables* tabs) {
  __shared__ NoiseTables T;
  for (int i = threadIdx.x; i < (int)(sizeof(NoiseTables) / sizeof(double)); i += blockDim.x)
    ((double*)&T)[i] = ((const double*)tabs)[i];
  __syncthreads();
  const int l = blockIdx.y, h = blockIdx.z;
  const int M = g.M[l];
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  U64Pair u = philox_u64(io.noise_seed, kNoiseLattice, (uint32_t)io.noise_t, (uint32_t)j, j == 0 ? 0u : (uint32_t)l,
                         (uint32_t)(io.noise_rep + h * io.noise_rep_per_rhs));
  double u1 = ((double)(u.a >> 11) + 1.0) * 0x1.0p-53;
  double u2 = (double)(u.b >> 11) * 0x1.0p-53;
  double R = sqrt(fmax(-2.0 * ln_unit(u1, T), 0.0));  // ln 1 may round to a tiny positive value
  double sn, cs;
  sincos_2pi(u2, T, sn, cs);
  cplx* y = io.out + h * io.out_stride + g.off[l] + j;
  const double sc = io.noise_scale;
  const cplx e = cmake(sc * (R * cs), sc * (R * sn));
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
  MR1L_LAUNCH("noise_tables_kernel", s, 0, (double)sizeof(NoiseTables), noise_tables_kernel<<<1, 256, 0, s>>>(t));
  MR1L_CUDA(cudaStreamSynchronize(s));
  g_noise_tabs[dev] = t;
  return t;
}

void add_lattice_noise(const BlueGeom& g, const BlueIO& io, int nrhs, cudaStream_t s) {
  if (io.noise_scale == 0.0 || nrhs == 0) return;
  int maxM = (int)std::min<int64_t>(g.sum_M, g.P / 2 + 1);
  dim3 grid(cdiv(maxM, 256), g.L, nrhs);
  const NoiseTables* tabs = noise_tables(s);
  MR1L_LAUNCH("lattice_noise_kernel", s, 0, 32.0 * nrhs * g.sum_M, lattice_noise_kernel<<<grid, 256, 0, s>>>(g, io, tabs));
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
