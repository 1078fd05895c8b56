// Lattice-side kernels of the hot path: residues, collision counting and
// coverage (Algorithm 1 / condition 2.1), the averaged gather (Algorithm 2),
// the lattice bins of evaluation and adjoint, the planted sampler,
// 1-D line detection (steps 1 and 2a of Algorithm 3), thresholded top-s
// selection and compaction.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace mr1l {

// A candidate set: the product prefix x last (Algorithm 3, J_t), or a plain
// set (last == nullptr, nq == 1).  Candidate id c = p * nq + q.
struct CandSet {
  int tp = 0;                     // components stored per prefix row
  int t = 0;                      // components of a candidate (tp + has_last)
  int64_t np = 0, nq = 1;
  const int32_t* pre = nullptr;   // device [np][tp]
  const int32_t* last = nullptr;  // device [nq] or nullptr
  int64_t n() const { return np * nq; }
};

// L rank-1 lattices on the device plus per-candidate residue factors.
struct LatticeDev {
  int L = 0;
  int t = 0;
  const int* M = nullptr;          // [L]
  const int64_t* z = nullptr;      // [L][t]
  uint32_t* pre_res = nullptr;     // [L][np]
  uint32_t* last_res = nullptr;    // [L][nq]
};

// Residues r_l(c) = (pre_res + last_res) mod M_l for all lattices.
void residues(const CandSet& J, const LatticeDev& lat, cudaStream_t s);

// Collision count of every lattice (2-bit saturating bucket state in two
// bitmaps, offsets bm_off[l] in 32-bit words) and the coverage pass:
// umask[c] = bitmask of lattices in which c is collision-free; cover[0] =
// smallest L such that every covered c has a bit below L; cover[1] = number of
// candidates in no I_l; cover[2 + l] = |I_l|; cover[66 + l] = candidates
// whose first collision-free lattice is l (cover holds 130 ints).  seen must
// be zeroed (2 * words) beforehand.
void collide_and_cover(const CandSet& J, const LatticeDev& lat, uint32_t* seen, const int64_t* bm_off,
                       int64_t words, uint64_t* umask, int* cover, cudaStream_t s);

// Algorithm 2 gather: p[h][c] = (1/cnt) sum_{l < Luse, c in I_l} w_l[r] C[h][off_l + r].
// Also writes keys[h][c] = bits(re*re + im*im) (0 where uncovered) and
// atomically maxes them into keymax[h] (must be zeroed beforehand).  pairs =
// sum_{l < Luse} |I_l| (launch accounting only).
void gather(const CandSet& J, const LatticeDev& lat, int Luse, const uint64_t* umask, const BlueGeom& g,
            const cplx* C, int64_t C_stride, int nrhs, cplx* p, int64_t p_stride, uint64_t* keys,
            uint64_t* keymax, int64_t pairs, cudaStream_t s);

// Scatter for evaluation (EVAL): bins[h][off_l + r_l(c)] += c_k over all
// lattices l < Luse (colliding candidates share a bin).  bins must be zeroed.
void scatter(const CandSet& J, const LatticeDev& lat, int Luse, const BlueGeom& g, const cplx* coef,
             int64_t coef_stride, int nrhs, cplx* bins, int64_t bins_stride, cudaStream_t s);

// The adjoint of Algorithm 2 (ADJOINT) in bin order.  adjoint_map (once per
// plan): map[off_l + r] = the candidate collision-free at residue r of
// lattice l (at most one: that is what collision-free means), -1 where there
// is none; inv_cnt[c] = 1 / |{l < Luse : c in I_l}| (0 if uncovered).  map
// must hold -1 everywhere beforehand.  adjoint_bins: cs[h][c] = c_k / cnt_k
// (scratch [nrhs][n]), then every bin bins[h][off_l + j] = cs[h][k] for the
// candidate k of map, else 0 (maxM: the largest M_l, l < Luse); the 1 / M_l
// is applied by the evaluation pass (BlueIO::out_scaled).
void adjoint_map(const CandSet& J, const LatticeDev& lat, int Luse, const uint64_t* umask, const BlueGeom& g,
                 int32_t* map, double* inv_cnt, int64_t pairs, cudaStream_t s);
void adjoint_bins(int Luse, int maxM, const BlueGeom& g, int64_t n, const int32_t* map, const double* inv_cnt,
                  const cplx* coef, int64_t coef_stride, int nrhs, cplx* cs, cplx* bins, int64_t bins_stride,
                  cudaStream_t s);

// Planted sampler, lattice request: weights c_h e^{2 pi i h_(>t).x'} per
// right-hand side (anchors [nrhs][d]) scattered to bin h_(1..t).z_l mod M_l.
// wts: device scratch of nrhs * s_count complex.
void planted_lattice_bins(const int32_t* freqs, const cplx* coeffs, int64_t s_count, int d, int t,
                          const double* anchors_dev, int nrhs, const LatticeDev& lat, int Luse,
                          const BlueGeom& g, cplx* bins, int64_t bins_stride, cplx* wts, cudaStream_t s);

// Planted sampler, line request: y[i][l] = p(x'_1.., l/K, ..x'_d) + noise.
void planted_lines(const int32_t* freqs, const cplx* coeffs, int64_t s_count, int d, int t, int K,
                   const double* anchors_dev, int nlines, double noise_scale, uint64_t noise_seed,
                   int rep0, cplx* bins_scratch, cplx* y, cudaStream_t s);

// Section 5.3 test function f(x) = sum_g prod_{t: group_of[t] = g} N_{m_g}(x_t)
// with N_m(x) = C_m m B_m(m x): per group, the polynomial of B_m on each knot
// interval [q, q+1) in powers of (u - q), scaled by C_m m (host-computed).
constexpr int kBsMaxGroups = 8, kBsMaxOrder = 8, kBsMaxDim = 64;
struct BsplineDev {
  int d, n_groups;
  int group_of[kBsMaxDim];
  int order[kBsMaxGroups];
  double coef[kBsMaxGroups][kBsMaxOrder][kBsMaxOrder];  // [g][q][power]
};
// y[h][off_l + j] = f(x) at node j of lattice l: x_i = (j z_{l,i} mod M_l) / M_l
// for i < t, the anchor component anchors[h][i] for i >= t.
void bspline_lattice(const BsplineDev* S, int t, const double* anchors_dev, int nrhs, const LatticeDev& lat,
                     int Luse, const BlueGeom& g, int max_M, cplx* y, int64_t y_stride, cudaStream_t s);
// y[i][l] = f(anchors[i] with component t-1 replaced by l / K).
void bspline_lines(const BsplineDev* S, int t, int K, const double* anchors_dev, int nlines, cplx* y,
                   cudaStream_t s);

// Line detection: p~_k = (1/K) sum_l y_l e^{-2 pi i l k/K}, k = -N..N, keep
// the (up to) cap largest keys >= threshold per line; sel[k + N] |= 1.
void detect_lines(const cplx* y, int nlines, int N, int64_t cap, double theta2, int rel, uint8_t* sel,
                  cudaStream_t s);

// Selection state of one segment (device memory, see select.cu).
constexpr int kSelBits = 11;                 // radix digit width
constexpr int kSelBins = 1 << kSelBits;
constexpr int kSelPasses = 6;                // digits [52,63) [41,52) [30,41) [19,30) [8,19) [0,8)
struct SelectState {
  uint64_t thr;        // squared-threshold bits
  uint64_t prefix;     // radix-select prefix
  int64_t need;        // how many still to take among keys matching prefix
  int64_t total;       // eligible count (keys >= thr)
  int take_all;        // eligible count <= cap
  int64_t eq_count;    // keys equal to the final prefix
  unsigned int ticket; // CTAs of the current histogram pass that have finished
  uint32_t hist[kSelBins];
};

// Segments of at most kSelSmallMax keys are selected by one CTA each in a
// single launch; longer ones by the multi-CTA digit passes.
constexpr int64_t kSelSmallMax = 65536;

// Thresholded "(up to) cap largest" over nrhs segments of n keys each
// (keys [h][n], keymax [h]); selected ids are OR-ed into flags[c] (uint8)
// (shared across segments).  st: device SelectState [nrhs].
void select_topk(const uint64_t* keys, int64_t n, int nrhs, const uint64_t* keymax, double theta2, int rel,
                 int64_t cap, SelectState* st, uint8_t* flags, cudaStream_t s);

// Selection keys of plain values: keys[h][c] = bits(|p[h][c]|^2) + 1 where
// eligible[c] != 0 (or eligible == nullptr), else 0; keymax[h] their maximum.
void value_keys(const cplx* p, int64_t n, int nrhs, const uint8_t* eligible, uint64_t* keys, uint64_t* keymax,
                cudaStream_t s);

// Compaction of flags[c] into the next prefix list rows (pre x last) and,
// optionally, the coefficients p[c].  Returns the count (synchronises);
// total_host, if given, is pinned host memory for the count's copy.
int64_t compact(const CandSet& J, const uint8_t* flags, int32_t* out_rows, const cplx* p, cplx* out_p,
                int64_t* scratch_counts, int64_t scratch_len, int64_t* total_host, cudaStream_t s);

}  // namespace mr1l
