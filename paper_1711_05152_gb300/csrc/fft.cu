// Bluestein prime-length DFTs over power-of-two FP64 FFTs.
//
// A length-M DFT X[r] = sum_j x[j] exp(-2 pi i j r / M) (Algorithm 2, one
// lattice) is rewritten with j r = (j^2 + r^2 - (r - j)^2) / 2 as
//   X[r] = w[r] * sum_j (x[j] w[j]) conj(w[r - j]),   w[n] = exp(-pi i n^2 / M),
// a linear convolution evaluated by power-of-two FFTs of length P >= 2M - 1.
// The chirp phase uses n^2 mod 2M reduced in exact integers.
//
// On GB300 the FP64 pipe (about 2 FMA per clock per SM) bounds these
// transforms, so the kernels read chirps, filters and twiddles from tables
// instead of recomputing them, and never spend FP64 work on index math.
//
// Structure: P <= 4096 runs in one CTA per transform (everything in shared
// memory).  Larger P uses the 4-step split P = P1 * P2 without transposes:
//   pass 1 (columns): FFT_P1 over n1 of x[n1 P2 + n2], times w_P^(n2 k1),
//                     stored at k1 P2 + n2;
//   pass 2 (rows):    FFT_P2 over n2 (giving X[k1 + P1 k2] at k1 P2 + k2),
//                     times the filter spectrum (stored in the same order),
//                     inverse FFT_P2, times w_P^(-n2 k1);
//   pass 3 (columns): inverse FFT_P1 over k1, natural order x[n1 P2 + n2].
// Each sub-FFT is a mixed-radix (8, 4, 2) Stockham autosort FFT in shared
// memory (Govindaraju et al., SC'08 formulation).
#include <map>
#include <mutex>

#include <cmath>

#include "fft.cuh"
#include "prof.cuh"

namespace mr1l {

// ---------------------------------------------------------------------------
// Register DFTs of size 2, 4, 8 (forward: exp(-2 pi i / R); INV: conjugate).
// ---------------------------------------------------------------------------
template <int R, bool INV>
struct RegDft;

template <bool INV>
struct RegDft<2, INV> {
  static __device__ __forceinline__ void run(cplx* v) {
    cplx a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct RegDft<4, INV> {
  static __device__ __forceinline__ void run(cplx* v) {
    cplx t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    cplx t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV>
struct RegDft<8, INV> {
  static __device__ __forceinline__ void run(cplx* v) {
    const double h = 0.70710678118654752440;  // 1/sqrt(2)
    cplx e[4] = {v[0], v[2], v[4], v[6]};
    cplx o[4] = {v[1], v[3], v[5], v[7]};
    RegDft<4, INV>::run(e);
    RegDft<4, INV>::run(o);
    // X_k = E_k + w8^k O_k, X_{k+4} = E_k - w8^k O_k; the 1/sqrt(2) of w8 and
    // w8^3 is folded into fused multiply-adds
    cplx a = o[1], c = o[3];
    double a1x, a1y, a3x, a3y;  // w8 O_1 and w8^3 O_3 without the factor h
    if (!INV) {
      a1x = a.x + a.y;
      a1y = a.y - a.x;
      a3x = c.y - c.x;
      a3y = -(c.x + c.y);
    } else {
      a1x = a.x - a.y;
      a1y = a.x + a.y;
      a3x = -(c.x + c.y);
      a3y = c.x - c.y;
    }
    cplx o2 = mul_mi<INV>(o[2]);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cmake(fma(h, a1x, e[1].x), fma(h, a1y, e[1].y));
    v[5] = cmake(fma(-h, a1x, e[1].x), fma(-h, a1y, e[1].y));
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cmake(fma(h, a3x, e[3].x), fma(h, a3y, e[3].y));
    v[7] = cmake(fma(-h, a3x, e[3].x), fma(-h, a3y, e[3].y));
  }
};

// Radix 3: X0 = a + b + c, X1,2 = a - (b + c)/2 -+ i (sqrt(3)/2)(b - c) (forward).
template <bool INV>
struct RegDft<3, INV> {
  static __device__ __forceinline__ void run(cplx* v) {
    const double s3 = 0.86602540378443864676;  // sqrt(3)/2
    cplx t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    cplx a = v[0];
    v[0] = cadd(a, t1);
    cplx m1 = cmake(fma(-0.5, t1.x, a.x), fma(-0.5, t1.y, a.y));
    // forward: -i s3 t2 ; inverse: +i s3 t2
    cplx m2 = INV ? cmake(-s3 * t2.y, s3 * t2.x) : cmake(s3 * t2.y, -s3 * t2.x);
    v[1] = cadd(m1, m2);
    v[2] = csub(m1, m2);
  }
};

// Radix-8 DFT of a sequence whose inputs 4..7 are zero (the first stage of a
// zero-padded Bluestein input): v[0..3] in, v[0..7] out, 36 FP64 operations
// instead of 52.
template <bool INV>
__device__ __forceinline__ void reg_dft8_half(cplx* v) {
  const double h = 0.70710678118654752440;
  cplx e0 = cadd(v[0], v[2]), e2 = csub(v[0], v[2]);
  cplx m2 = mul_mi<INV>(v[2]);
  cplx e1 = cadd(v[0], m2), e3 = csub(v[0], m2);
  cplx o0 = cadd(v[1], v[3]), o2 = csub(v[1], v[3]);
  cplx m3 = mul_mi<INV>(v[3]);
  cplx o1 = cadd(v[1], m3), o3 = csub(v[1], m3);
  double a1x, a1y, a3x, a3y;
  if (!INV) {
    a1x = o1.x + o1.y;
    a1y = o1.y - o1.x;
    a3x = o3.y - o3.x;
    a3y = -(o3.x + o3.y);
  } else {
    a1x = o1.x - o1.y;
    a1y = o1.x + o1.y;
    a3x = -(o3.x + o3.y);
    a3y = o3.x - o3.y;
  }
  o2 = mul_mi<INV>(o2);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cmake(fma(h, a1x, e1.x), fma(h, a1y, e1.y));
  v[5] = cmake(fma(-h, a1x, e1.x), fma(-h, a1y, e1.y));
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cmake(fma(h, a3x, e3.x), fma(h, a3y, e3.y));
  v[7] = cmake(fma(-h, a3x, e3.x), fma(-h, a3y, e3.y));
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
template <int R, bool INV, bool COLS, bool HALF = false>
__device__ __forceinline__ void stockham_stage(cplx* s, int n, int Ns, int nseq, int bs, int is,
                                               const cplx* twn_n) {
  constexpr int CNT = (8 + R - 1) / R;
  const int nb = n / R;
  const int total = nseq * nb;
  cplx v[CNT][R];
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
      const cplx* src = s + b * bs + j * is;
#pragma unroll
      for (int r = 0; r < 4; ++r) v[c][r] = src[r * nb * is];
      reg_dft8_half<INV>(v[c]);
    } else if (act[c]) {
      const cplx* src = s + b * bs + j * is;
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = src[r * nb * is];
      if (Ns > 1) {
        int step = k * (n / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cplx w = twn_n[r * step];
          v[c][r] = INV ? cmulc(v[c][r], w) : cmul(v[c][r], w);
        }
      }
      RegDft<R, INV>::run(v[c]);
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
__device__ __forceinline__ const cplx* twiddles_of(const cplx* twn, int n) {
  return (n & (n - 1)) == 0 ? twn + n : twn + 8192 + n - 3;
}

// Full in-smem FFT of length n = 2^a or 3 * 2^a: radix-8 stages, one radix-4
// or radix-2 stage for the rest of 2^a, then radix 3.  Natural order in and
// out.  HALF_FIRST: the upper half of every input sequence is zero (needs
// 8 | n).
template <bool INV, bool COLS, bool HALF_FIRST = false>
__device__ __forceinline__ void smem_fft(cplx* s, int n, int nseq, int bs, int is, const cplx* twn) {
  const cplx* twn_n = twiddles_of(twn, n);
  const bool three = (n % 3) == 0;
  int rem = 31 - __clz(three ? n / 3 : n);  // log2 of the power-of-two part
  int Ns = 1;
  if (HALF_FIRST && rem >= 3) {
    stockham_stage<8, INV, COLS, true>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 3;
    rem -= 3;
  }
  while (rem >= 3) {
    stockham_stage<8, INV, COLS>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 3;
    rem -= 3;
  }
  if (rem == 2) {
    stockham_stage<4, INV, COLS>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 2;
  }
  if (rem == 1) {
    stockham_stage<2, INV, COLS>(s, n, Ns, nseq, bs, is, twn_n);
    Ns <<= 1;
  }
  if (three) stockham_stage<3, INV, COLS>(s, n, Ns, nseq, bs, is, twn_n);
}

// ---------------------------------------------------------------------------
// Sources and sinks
// ---------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ cplx load_input(const BlueGeom& g, const BlueIO& io, int l, int h, int M,
                                           int64_t off, int64_t n) {
  if (MODE == kModeFilter) {
    if (n < M) return cconj(g.w[off + n]);
    if (n > g.P - M) return cconj(g.w[off + (g.P - n)]);
    return cmake(0.0, 0.0);
  }
  if (n >= M) return cmake(0.0, 0.0);
  cplx x = io.in[h * io.in_stride + off + n];
  if (MODE == kModeRecon) return cmul(x, g.ws[off + n]);
  return cmul(cconj(x), g.w[off + n]);
}

__device__ __forceinline__ cplx lattice_noise(uint64_t seed, int t, int rep, int l, int64_t j, double scale) {
  U64Pair u = philox_u64(seed, kNoiseLattice, (uint32_t)t, (uint32_t)j, j == 0 ? 0u : (uint32_t)l,
                         (uint32_t)rep);
  double u1 = ((double)(u.a >> 11) + 1.0) * 0x1.0p-53;
  double u2 = (double)(u.b >> 11) * 0x1.0p-53;
  double R = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return cmake(scale * (R * cs), scale * (R * sn));
}

template <int MODE>
__device__ __forceinline__ void store_output(const BlueGeom& g, const BlueIO& io, int l, int h, int64_t off,
                                             int64_t n, cplx v) {
  if (MODE == kModeRecon) {
    io.out[h * io.out_stride + off + n] = v;
  } else {
    cplx y = cconj(cmul(g.w[off + n], v));
    if (io.noise_scale != 0.0) {
      cplx e = lattice_noise(io.noise_seed, io.noise_t, io.noise_rep + h * io.noise_rep_per_rhs, l, n,
                             io.noise_scale);
      y = cadd(y, e);
    }
    io.out[h * io.out_stride + off + n] = y;
  }
}

// ---------------------------------------------------------------------------
// P <= 4096: the whole convolution in one CTA.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(512) blue_small_kernel(BlueGeom g, BlueIO io) {
  extern __shared__ cplx sm[];
  const int gi = blockIdx.x;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, M = g.M[l];
  const int64_t off = g.off[l];
  // zero padding: for RECON / EVAL the input vanishes from M <= P/2 on, so the
  // upper half is never loaded and the first radix-8 stage skips it
  const bool half = MODE != kModeFilter && (P % 8) == 0;
  const int nload = half ? P / 2 : P;
  for (int n = threadIdx.x; n < nload; n += blockDim.x) sm[n] = load_input<MODE>(g, io, l, h, M, off, n);
  __syncthreads();
  if (half)
    smem_fft<false, false, true>(sm, P, 1, 0, 1, g.twn);
  else
    smem_fft<false, false>(sm, P, 1, 0, 1, g.twn);
  cplx* Bh = g.Bh + (int64_t)l * P;
  if (MODE == kModeFilter) {
    const double sc = 1.0 / (double)P;  // exact: P is a power of two
    for (int n = threadIdx.x; n < P; n += blockDim.x) Bh[n] = cmake(sm[n].x * sc, sm[n].y * sc);
    return;
  }
  for (int n = threadIdx.x; n < P; n += blockDim.x) sm[n] = cmul(sm[n], Bh[n]);
  __syncthreads();
  smem_fft<true, false>(sm, P, 1, 0, 1, g.twn);
  for (int n = threadIdx.x; n < M; n += blockDim.x) store_output<MODE>(g, io, l, h, off, n, sm[n]);
}

// ---------------------------------------------------------------------------
// 4-step passes
// ---------------------------------------------------------------------------
// Tiles of 2048 complex (32 KB shared memory, 256 threads) so that three CTAs
// share an SM and hide each other's load and barrier phases; a single
// column or row of 4096 takes a 4096-element tile.
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
template <int MODE>
__global__ void __launch_bounds__(512) blue_col_fwd_kernel(BlueGeom g, BlueIO io) {
  extern __shared__ cplx sm[];
  const int gi = blockIdx.y;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, P1 = g.P1, P2 = g.P2, CB = col_tile(P1);
  const int M = g.M[l];
  const int64_t off = g.off[l];
  const int n2_0 = blockIdx.x * CB;
  // RECON / EVAL: rows n1 >= P1/2 hold n >= P/2 >= M, i.e. zero padding
  const int rows = MODE == kModeFilter ? P1 : P1 / 2;
  for (int e = threadIdx.x; e < rows * CB; e += blockDim.x) {
    int i = e / CB, b = e - i * CB;
    sm[e] = load_input<MODE>(g, io, l, h, M, off, (int64_t)i * P2 + n2_0 + b);
  }
  __syncthreads();
  if (MODE == kModeFilter)
    smem_fft<false, true>(sm, P1, CB, 1, CB, g.twn);
  else
    smem_fft<false, true, true>(sm, P1, CB, 1, CB, g.twn);
  cplx* work = io.work + (int64_t)gi * P;
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int k1 = e / CB, b = e - k1 * CB;
    int n2 = n2_0 + b;
    cplx w = g.tw[((int64_t)n2 * k1) % P];
    work[(int64_t)k1 * P2 + n2] = cmul(sm[e], w);
  }
}

// Pass 2: rows.  FILTER: forward FFT scaled by 1/P into Bh.  Otherwise forward
// FFT, times Bh, inverse FFT, times conj(w_P^(n2 k1)).
template <bool FILTER>
__global__ void __launch_bounds__(512) blue_row_kernel(BlueGeom g, BlueIO io) {
  extern __shared__ cplx sm[];
  const int gi = blockIdx.y;
  const int l = gi % g.L;
  const int P = g.P, P2 = g.P2, RB = row_tile(P2);
  const int k1_0 = blockIdx.x * RB;
  cplx* work = io.work + (int64_t)gi * P + (int64_t)k1_0 * P2;
  for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) sm[e] = work[e];
  __syncthreads();
  smem_fft<false, false>(sm, P2, RB, P2, 1, g.twn);
  cplx* Bh = g.Bh + (int64_t)l * P + (int64_t)k1_0 * P2;
  if (FILTER) {
    const double sc = 1.0 / (double)P;
    for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) Bh[e] = cmake(sm[e].x * sc, sm[e].y * sc);
    return;
  }
  for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) sm[e] = cmul(sm[e], Bh[e]);
  __syncthreads();
  smem_fft<true, false>(sm, P2, RB, P2, 1, g.twn);
  for (int e = threadIdx.x; e < RB * P2; e += blockDim.x) {
    int b = e / P2, n2 = e - b * P2;
    int k1 = k1_0 + b;
    cplx w = g.tw[((int64_t)n2 * k1) % P];
    work[e] = cmulc(sm[e], w);
  }
}

// Pass 3: columns, inverse; natural-order output n = n1 P2 + n2 for n < M.
template <int MODE>
__global__ void __launch_bounds__(512) blue_col_inv_kernel(BlueGeom g, BlueIO io) {
  extern __shared__ cplx sm[];
  const int gi = blockIdx.y;
  const int l = gi % g.L, h = gi / g.L;
  const int P = g.P, P1 = g.P1, P2 = g.P2, CB = col_tile(P1);
  const int M = g.M[l];
  const int64_t off = g.off[l];
  const int n2_0 = blockIdx.x * CB;
  const cplx* work = io.work + (int64_t)gi * P;
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int k1 = e / CB, b = e - k1 * CB;
    sm[e] = work[(int64_t)k1 * P2 + n2_0 + b];
  }
  __syncthreads();
  smem_fft<true, true>(sm, P1, CB, 1, CB, g.twn);
  for (int e = threadIdx.x; e < P1 * CB; e += blockDim.x) {
    int n1 = e / CB, b = e - n1 * CB;
    int64_t n = (int64_t)n1 * P2 + n2_0 + b;
    if (n < M) store_output<MODE>(g, io, l, h, off, n, sm[e]);
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

__global__ void chirp_kernel(cplx* w, cplx* ws, const int64_t* off, const int* Ms, int L) {
  int l = blockIdx.y;
  int M = Ms[l];
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= M) return;
  uint64_t q = ((uint64_t)n * (uint64_t)n) % (uint64_t)(2 * (int64_t)M);  // exact n^2 mod 2M
  double s, c;
  sincospi((double)q / (double)M, &s, &c);
  cplx v = cmake(c, -s);  // exp(-pi i q / M)
  w[off[l] + n] = v;
  double inv = 1.0 / (double)M;
  ws[off[l] + n] = cmake(c * inv, -s * inv);
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
              chirp_kernel<<<grid, 256, 0, s>>>(const_cast<cplx*>(g.w), const_cast<cplx*>(g.ws), g.off, g.M, g.L));
}

template <typename K>
static void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) MR1L_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

static int threads_for(int elems) {
  int t = elems / 8;
  if (t < 32) t = 32;
  return t;
}

static double fft_flops(double n) { return n > 1 ? 5.0 * n * std::log2(n) : 0.0; }

// Algorithmic work of one launch (FFT flops by the 5 n log2 n convention plus
// 6 flops per complex multiply; bytes that the pass must move).
template <int MODE>
static void launch_first_last(const BlueGeom& g, const BlueIO& io, int ntrans, cudaStream_t s) {
  const double P = g.P, nr = (double)ntrans / g.L, sumM = (double)g.sum_M;
  const double cb = sizeof(cplx);
  if (g.P <= kSmallMax) {
    size_t smem = (size_t)g.P * sizeof(cplx);
    set_smem(blue_small_kernel<MODE>, smem);
    double fl = ntrans * (MODE == kModeFilter ? fft_flops(P) : 2 * fft_flops(P) + 6 * P) + nr * 6 * sumM;
    double by = MODE == kModeFilter ? g.L * P * cb + sumM * cb : nr * sumM * cb * 3 + ntrans * P * cb;
    MR1L_LAUNCH(MODE == kModeFilter ? "blue_small_filter" : (MODE == kModeRecon ? "blue_small_recon" : "blue_small_eval"),
                s, fl, by, blue_small_kernel<MODE><<<ntrans, threads_for(g.P), smem, s>>>(g, io));
    return;
  }
  int CB = col_tile(g.P1), RB = row_tile(g.P2);
  size_t smem_c = (size_t)g.P1 * CB * sizeof(cplx);
  size_t smem_r = (size_t)RB * g.P2 * sizeof(cplx);
  dim3 gc(g.P2 / CB, ntrans), gr(g.P1 / RB, ntrans);
  const double P1 = g.P1, P2 = g.P2;
  set_smem(blue_col_fwd_kernel<MODE>, smem_c);
  MR1L_LAUNCH(MODE == kModeFilter ? "blue_col_fwd_filter" : (MODE == kModeRecon ? "blue_col_fwd_recon" : "blue_col_fwd_eval"),
              s, ntrans * (P2 * fft_flops(P1) + 6 * P) + nr * 6 * sumM, nr * sumM * cb * 2 + ntrans * P * cb,
              blue_col_fwd_kernel<MODE><<<gc, threads_for(g.P1 * CB), smem_c, s>>>(g, io));
  if (MODE == kModeFilter) {
    set_smem(blue_row_kernel<true>, smem_r);
    MR1L_LAUNCH("blue_row_filter", s, ntrans * P1 * fft_flops(P2), ntrans * P * cb * 2,
                blue_row_kernel<true><<<gr, threads_for(RB * g.P2), smem_r, s>>>(g, io));
    return;
  }
  set_smem(blue_row_kernel<false>, smem_r);
  MR1L_LAUNCH(MODE == kModeRecon ? "blue_row_recon" : "blue_row_eval", s,
              ntrans * (2 * P1 * fft_flops(P2) + 12 * P), ntrans * P * cb * 3,
              blue_row_kernel<false><<<gr, threads_for(RB * g.P2), smem_r, s>>>(g, io));
  set_smem(blue_col_inv_kernel<MODE>, smem_c);
  MR1L_LAUNCH(MODE == kModeRecon ? "blue_col_inv_recon" : "blue_col_inv_eval", s,
              ntrans * P2 * fft_flops(P1) + (MODE == kModeEval ? nr * 6 * sumM : 0.0),
              ntrans * P * cb + nr * sumM * cb * (MODE == kModeEval ? 2 : 1),
              blue_col_inv_kernel<MODE><<<gc, threads_for(g.P1 * CB), smem_c, s>>>(g, io));
}

void blue_filter(const BlueGeom& g, cudaStream_t s) {
  // the filter pass needs P complex of scratch per lattice: use Bh itself as
  // the 4-step work buffer (pass 1 writes it, pass 2 overwrites it in place
  // row by row; each row is read completely before it is written)
  BlueIO io{};
  io.work = g.Bh;
  launch_first_last<kModeFilter>(g, io, g.L, s);
}

void blue_run(const BlueGeom& g, const BlueIO& io, int mode, int nrhs, cudaStream_t s) {
  int ntrans = g.L * nrhs;
  if (ntrans == 0) return;
  if (mode == kModeRecon)
    launch_first_last<kModeRecon>(g, io, ntrans, s);
  else
    launch_first_last<kModeEval>(g, io, ntrans, s);
}

}  // namespace mr1l
