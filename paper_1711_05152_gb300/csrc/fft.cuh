// Batched prime-length DFTs by Bluestein convolution over FFTs of length 2^k
// or 3 * 2^k (the per-lattice DFT of Algorithm 2 and of the lattice
// evaluation), in FP64 or in double-float arithmetic on the FP32 pipes.
#pragma once

#include <string>

#include "common.cuh"

namespace mr1l {

// Source/sink of the first and last pass of a Bluestein convolution.
enum BlueMode : int {
  kModeFilter = 0,  // input b[n] = conj(w[n]) (n < M), conj(w[P-n]) (n > P-M), else 0
  kModeRecon = 1,   // input y[n] * w[n] / M, output raw convolution C[n] (n < M)
  kModeEval = 2,    // input conj(B[n]) * w[n], output conj(w[n] C[n]) (+ noise)
};

// Per-transform geometry shared by every pass of one batched launch.
struct BlueGeom {
  int L;            // lattices (transform g has lattice g % L, right-hand side g / L)
  int P;            // convolution length 2^k or 3 * 2^k, P >= 2 max M - 1
  int P1, P2;       // 4-step split P = P1 * P2 (P1 = 2^a or 3 * 2^a, P2 = 2^b) when P > kSmallMax
  const int64_t* off;   // device [L]: offset of lattice l in per-lattice arrays
  const int* M;         // device [L]: lattice sizes
  const cplx* w;        // device [sum M]: chirp exp(-pi i n^2 / M)
  const cplx* ws;       // device [sum M]: chirp / M
  cplx* Bh;             // device [L][P]: filter spectrum FFT_P(b) / P (pass order)
  const cplx* tw;       // device [P]: exp(-2 pi i e / P)
  const cplx* twr;      // device [P1][P2]: exp(-2 pi i n2 k1 / P) at k1 P2 + n2 (the row pass's
                        //   twiddles in the order it stores them; P > kSmallMax only)
  const cplx* twc;      // device [P2][P1]: the same twiddles at n2 P1 + k1 (the column pass's order)
  const cplx* twn;      // device [kSmallTw + kFmaTw]: exp(-2 pi i e / n), n = 2^a <= 8192 at offset n,
                        //   n = 3 * 2^a <= 6144 at offset kSmallTwPow2 + n - 3; then the
                        //   multiply-add twiddles (kFmaTw)
  int64_t sum_M;        // host: sum of the L lattice sizes (for launch accounting)
  // double-float arithmetic (df != 0): the same tables as hi/lo FP32 pairs
  // (float4 = re.hi, re.lo, im.hi, im.lo); Bh then holds float4 data
  int df;
  const float4* w_df;
  const float4* ws_df;
  const float4* tw_df;
  const float4* twr_df;
  const float4* twc_df;
  const float4* twn_df;
  // complex elements per CTA tile of the column / row passes (set per launch
  // by the tile tuner)
  int ctile, rtile;
};

struct BlueIO {
  const cplx* in;       // RECON: samples y; EVAL: bins B (both [nrhs][sum M])
  int64_t in_stride;    // per right-hand side
  cplx* out;            // RECON: C; EVAL: y
  int64_t out_stride;
  cplx* work;           // [nrhs][L][P]
  // RECON: optional second input added to the samples as they are loaded
  // (the measurement noise, computed concurrently on another stream)
  const cplx* add_in;   // [nrhs][sum M] with stride in_stride, or null
  // complex Gaussian noise (Philox purpose 5) written by add_lattice_noise
  double noise_scale;   // sigma / sqrt(2); 0 disables
  int noise_write;      // 1: out = noise; 0: out += noise
  uint64_t noise_seed;
  int noise_t, noise_rep;
  int noise_rep_per_rhs;  // rep index = noise_rep + rhs * noise_rep_per_rhs
  int no_tune;            // 1: never run tiling trials (default tiles unless already tuned)
  int out_scaled;         // EVAL: output chirp divided by M_l (the 1 / M_l of the adjoint)
};

constexpr int kSmallMax = 4096;  // P <= 4096: one CTA holds the whole transform
constexpr int kSmallTwPow2 = 16384;  // power-of-two sub-FFT lengths up to 8192
constexpr int kSmallTw = kSmallTwPow2 + 12288;
// Twiddles of the FP64 multiply-add butterflies, stored after the kSmallTw
// small twiddles in the same allocation as (s, t) pairs (w = s (1 + i t)):
// for radix 8, 4 and 2 and every stage stride Ns = 2^e <= kFmaMaxNs, the
// entries of k < Ns sit at index Ns - 1 + k of the radix's region, 4, 2 and 1
// pairs per index.
constexpr int kFmaMaxNs = 4096;
constexpr int kFmaSpan = 2 * kFmaMaxNs - 1;
constexpr int kFmaTw = 7 * kFmaSpan;

// Device-resident twiddle tables, cached per (device, P).
const cplx* twiddle_table(int P, cudaStream_t s);
const float4* twiddle_table_df(int P, cudaStream_t s);
// The same twiddles in row order for the 4-step split P = P1 x P2 (entry
// k1 P2 + n2 = exp(-2 pi i n2 k1 / P), copied from twiddle_table), cached per
// (device, P).
const cplx* row_twiddle_table(int P, int P2, cudaStream_t s);
const float4* row_twiddle_table_df(int P, int P2, cudaStream_t s);
// ... and in column order (entry n2 P1 + k1).
const cplx* col_twiddle_table(int P, int P2, cudaStream_t s);
const float4* col_twiddle_table_df(int P, int P2, cudaStream_t s);
const float4* small_twiddles_df(cudaStream_t s);

// dst[i] = (hi, lo) split of src[i] for i < n (double-float copies of tables).
void to_double_float(const cplx* src, float4* dst, int64_t n, cudaStream_t s);
const cplx* small_twiddles(cudaStream_t s);

// The smallest supported convolution length P >= n (2^k <= 2^25 or 3 * 2^k <= 3 * 2^23);
// 0 if there is none.
int blue_length(int64_t n);

// Fill geometry split for a given P.
void blue_split(BlueGeom& g, int P);

// Build the filter spectra Bh for all L lattices (needs w).
void blue_filter(const BlueGeom& g, cudaStream_t s);

// Run nrhs * L Bluestein convolutions in mode kModeRecon or kModeEval.
void blue_run(const BlueGeom& g, const BlueIO& io, int mode, int nrhs, cudaStream_t s);

// y += complex Gaussian noise of every lattice sample (io.out, io.noise_*),
// using g.L, g.M, g.off and g.sum_M only.
void add_lattice_noise(const BlueGeom& g, const BlueIO& io, int nrhs, cudaStream_t s);

// Tile tuner: enable/disable trials, forget the choices, and list them as a
// JSON array of {device, P, mode, df, col_tile, row_tile, col_ms, row_ms}.
void tune_enable(int on);
void tune_reset();
std::string tune_json();

// Chirp tables w and ws for every lattice (w[n] = exp(-pi i (n^2 mod 2M)/M)).
// seed: device scratch of g.L * kChirpSeedLen complex (per-lattice factor tables).
constexpr int kChirpSeedLen = 4096 + 8192;
void chirp_tables(const BlueGeom& g, int64_t max_M, cplx* seed, cudaStream_t s);

}  // namespace mr1l
