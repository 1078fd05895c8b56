// Lattice-side kernels: residues, collision counting / coverage, the
// averaged gather of Algorithm 2, scatter into lattice bins, the planted
// sampler and the 1-D line detection of Algorithm 3.
#include "ops.cuh"
#include "prof.cuh"

namespace mr1l {

__device__ __forceinline__ uint32_t residue_of(const LatticeDev& lat, int64_t np, int64_t nq, int l,
                                               int64_t p, int64_t q, uint32_t M) {
  uint32_t r = lat.pre_res[(int64_t)l * np + p] + lat.last_res[(int64_t)l * nq + q];  // < 2^32
  return r >= M ? r - M : r;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Residues k . z_l mod M_l (Section 2.1), exact in int64, canonical in [0, M).
// ---------------------------------------------------------------------------
__global__ void pre_res_kernel(CandSet J, LatticeDev lat) {
  const int l = blockIdx.y;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= J.np) return;
  const int64_t M = lat.M[l];
  const int64_t* z = lat.z + (int64_t)l * lat.t;
  const int32_t* k = J.pre + p * J.tp;
  int64_t acc = 0;
  for (int j = 0; j < J.tp; ++j) acc += (int64_t)k[j] * z[j];
  acc %= M;
  if (acc < 0) acc += M;
  lat.pre_res[(int64_t)l * J.np + p] = (uint32_t)acc;
}

__global__ void last_res_kernel(CandSet J, LatticeDev lat) {
  const int l = blockIdx.y;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= J.nq) return;
  int64_t acc = 0;
  if (J.last) {
    const int64_t M = lat.M[l];
    acc = ((int64_t)J.last[q] * lat.z[(int64_t)l * lat.t + J.tp]) % M;
    if (acc < 0) acc += M;
  }
  lat.last_res[(int64_t)l * J.nq + q] = (uint32_t)acc;
}

void residues(const CandSet& J, const LatticeDev& lat, cudaStream_t s) {
  // algorithmic bytes: the rows read once, the factors written
  if (J.np > 0) {
    MR1L_LAUNCH("pre_res_kernel", s, 0, 4.0 * J.np * (J.tp + lat.L),
                pre_res_kernel<<<dim3(cdiv(J.np, 256), lat.L), 256, 0, s>>>(J, lat));
  }
  MR1L_LAUNCH("last_res_kernel", s, 0, 4.0 * J.nq * (1 + lat.L),
              last_res_kernel<<<dim3(cdiv(J.nq, 256), lat.L), 256, 0, s>>>(J, lat));
}

// ---------------------------------------------------------------------------
// Collision counting: bucket state per residue in two bitmaps (seen once,
// seen at least twice); order-free, so the result is deterministic.
// ---------------------------------------------------------------------------
__global__ void collide_kernel(CandSet J, LatticeDev lat, uint32_t* seen1, uint32_t* seen2,
                               const int64_t* bm_off) {
  const int l = blockIdx.y;
  const int64_t n = J.np * J.nq;
  const uint32_t M = (uint32_t)lat.M[l];
  uint32_t* s1 = seen1 + bm_off[l];
  uint32_t* s2 = seen2 + bm_off[l];
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = c / J.nq, q = c - p * J.nq;
    uint32_t r = residue_of(lat, J.np, J.nq, l, p, q, M);
    uint32_t bit = 1u << (r & 31);
    uint32_t old = atomicOr(s1 + (r >> 5), bit);
    if (old & bit) atomicOr(s2 + (r >> 5), bit);
  }
}

// umask[c]: lattices in which c is collision-free; cover[0] = max over covered
// c of (first covering lattice + 1); cover[1] = uncovered count; cover[2 + l]
// = |I_l| (the number of candidates collision-free in lattice l); cover[66 +
// l] = the number of candidates whose first collision-free lattice is l.
__global__ void cover_kernel(CandSet J, LatticeDev lat, const uint32_t* seen2, const int64_t* bm_off,
                             uint64_t* umask, int* cover) {
  const int64_t n = J.np * J.nq;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned need = 0, unc = 0;
  uint64_t m = 0;
  if (c < n) {
    int64_t p = c / J.nq, q = c - p * J.nq;
    for (int l = 0; l < lat.L; ++l) {
      uint32_t r = residue_of(lat, J.np, J.nq, l, p, q, (uint32_t)lat.M[l]);
      if (!(seen2[bm_off[l] + (r >> 5)] & (1u << (r & 31)))) m |= (uint64_t)1 << l;
    }
    umask[c] = m;
    if (m) need = (unsigned)__ffsll((long long)m);
    else unc = 1;
  }
  need = __reduce_max_sync(0xffffffffu, need);
  unc = __reduce_add_sync(0xffffffffu, unc);
  if ((threadIdx.x & 31) == 0) {
    if (need) atomicMax(cover, (int)need);
    if (unc) atomicAdd(cover + 1, (int)unc);
  }
  // per-lattice sizes |I_l| and first-covering counts: one ballot per
  // lattice and warp
  const int first = m ? __ffsll((long long)m) - 1 : -1;
  for (int l = 0; l < lat.L; ++l) {
    const unsigned b = __ballot_sync(0xffffffffu, (m >> l) & 1);
    const unsigned f = __ballot_sync(0xffffffffu, first == l);
    if ((threadIdx.x & 31) == 0) {
      if (b) atomicAdd(cover + 2 + l, __popc(b));
      if (f) atomicAdd(cover + 2 + 64 + l, __popc(f));
    }
  }
}

void collide_and_cover(const CandSet& J, const LatticeDev& lat, uint32_t* seen, const int64_t* bm_off,
                       int64_t words, uint64_t* umask, int* cover, cudaStream_t s) {
  const int64_t n = J.n();
  MR1L_CUDA(cudaMemsetAsync(cover, 0, (2 + 128) * sizeof(int), s));
  if (n == 0) return;
  int blocks = (int)std::min<int64_t>(cdiv(n, 256), 4096);
  // algorithmic bytes: the residue factors read once, the two bitmaps
  // written once (collide); the factors and the second bitmap read, the masks
  // written (cover)
  const double factors = 4.0 * lat.L * (double)(J.np + J.nq), bitmaps = 4.0 * 2 * words;
  MR1L_LAUNCH("collide_kernel", s, 0, factors + bitmaps,
              collide_kernel<<<dim3(blocks, lat.L), 256, 0, s>>>(J, lat, seen, seen + words, bm_off));
  MR1L_LAUNCH("cover_kernel", s, 0, factors + bitmaps / 2 + 8.0 * n,
              cover_kernel<<<cdiv(n, 256), 256, 0, s>>>(J, lat, seen + words, bm_off, umask, cover));
}

// ---------------------------------------------------------------------------
// Algorithm 2 gather with the fused Bluestein post-chirp.
// keys: bits(|p~|^2) + 1 for covered candidates (order-preserving for
// non-negative doubles), 0 for uncovered ones.
// ---------------------------------------------------------------------------
// One thread per candidate and group of G right-hand sides: the residue,
// mask and chirp of each (candidate, lattice) pair are read once for the
// whole group, and the group's samples at that residue are independent loads
// in flight together.  Per right-hand side the lattices are summed in
// ascending order, whatever G is, so every G gives the same bits.
template <int kGatherRhs>
__global__ void __launch_bounds__(256) gather_kernel(CandSet J, LatticeDev lat, uint64_t lmask, const uint64_t* umask,
                                                     const int64_t* off, const cplx* w, const cplx* C, int64_t C_stride,
                                                     int nrhs, cplx* out, int64_t out_stride, uint64_t* keys,
                                                     uint64_t* keymax) {
  const int h0 = blockIdx.y * kGatherRhs;
  const int nh = min(kGatherRhs, nrhs - h0);
  const int64_t n = J.np * J.nq;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  cplx acc[kGatherRhs];
#pragma unroll
  for (int i = 0; i < kGatherRhs; ++i) acc[i] = cmake(0.0, 0.0);
  int cnt = 0;
  if (c < n) {
    const int64_t p = c / J.nq, q = c - p * J.nq;
    uint64_t m = umask[c] & lmask;
    cnt = __popcll(m);
    const cplx* Ch = C + h0 * C_stride;
    while (m) {
      const int l = __ffsll((long long)m) - 1;
      m &= m - 1;
      const uint32_t r = residue_of(lat, J.np, J.nq, l, p, q, (uint32_t)lat.M[l]);
      const int64_t o = off[l] + r;
      const cplx wo = w[o];
      cplx y[kGatherRhs];
#pragma unroll
      for (int i = 0; i < kGatherRhs; ++i)
        if (i < nh) y[i] = Ch[i * C_stride + o];
      // acc += wo * y as four FMAs (FP64 instructions are the scarce resource)
#pragma unroll
      for (int i = 0; i < kGatherRhs; ++i)
        if (i < nh) {
          acc[i].x = fma(wo.x, y[i].x, fma(-wo.y, y[i].y, acc[i].x));
          acc[i].y = fma(wo.x, y[i].y, fma(wo.y, y[i].x, acc[i].y));
        }
    }
  }
  const double inv = cnt ? __drcp_rn((double)cnt) : 0.0;
#pragma unroll
  for (int i = 0; i < kGatherRhs; ++i) {
    if (i >= nh) break;  // uniform across the block
    const int h = h0 + i;
    uint64_t key = 0;
    if (c < n) {
      cplx res = cmake(0.0, 0.0);
      if (cnt) {
        res = cmake(acc[i].x * inv, acc[i].y * inv);
        const double k2 = __dadd_rn(__dmul_rn(res.x, res.x), __dmul_rn(res.y, res.y));
        key = (uint64_t)__double_as_longlong(k2) + 1;
      }
      out[h * out_stride + c] = res;
      if (keys) keys[h * n + c] = key;
    }
    if (keymax) {
      key = warp_max_u64(key);
      if ((threadIdx.x & 31) == 0 && key) atomicMax((unsigned long long*)(keymax + h), (unsigned long long)key);
    }
  }
}

void gather(const CandSet& J, const LatticeDev& lat, int Luse, const uint64_t* umask, const BlueGeom& g,
            const cplx* C, int64_t C_stride, int nrhs, cplx* p, int64_t p_stride, uint64_t* keys,
            uint64_t* keymax, int64_t pairs, cudaStream_t s) {
  const int64_t n = J.n();
  if (n == 0 || nrhs == 0) return;
  uint64_t lmask = Luse >= 64 ? ~0ull : ((1ull << Luse) - 1);
  // algorithmic bytes: the samples of every right-hand side at every (k, l)
  // with k in I_l and the chirp there, the masks, the coefficients (and keys)
  const double bytes = 16.0 * pairs * (nrhs + 1) + 8.0 * n + (double)nrhs * (keys ? 24.0 : 16.0) * n;
  // the largest group that still leaves about 2^18 threads to hide the
  // latency of the random reads
  auto threads = [&](int G) { return (int64_t)cdiv(n, 256) * 256 * cdiv(nrhs, G); };
  const int G = threads(8) >= (1 << 18) ? 8 : threads(4) >= (1 << 18) ? 4 : threads(2) >= (1 << 18) ? 2 : 1;
#define MR1L_GATHER(GG)                                                                                         \
  MR1L_LAUNCH("gather_kernel", s, 0, bytes,                                                                   \
              gather_kernel<GG><<<dim3(cdiv(n, 256), cdiv(nrhs, GG)), 256, 0, s>>>(                          \
                  J, lat, lmask, umask, g.off, g.w, C, C_stride, nrhs, p, p_stride, keys, keymax))
  if (G == 8)
    MR1L_GATHER(8);
  else if (G == 4)
    MR1L_GATHER(4);
  else if (G == 2)
    MR1L_GATHER(2);
  else
    MR1L_GATHER(1);
#undef MR1L_GATHER
}

// ---------------------------------------------------------------------------
// Scatter into lattice bins for evaluation: all lattices, weight c_k; a bin
// that several candidates share (a collision) sums them, hence the atomics.
// ---------------------------------------------------------------------------
__global__ void scatter_kernel(CandSet J, LatticeDev lat, uint64_t lmask, const int64_t* off, const cplx* coef,
                               int64_t coef_stride, cplx* bins, int64_t bins_stride) {
  const int h = blockIdx.y;
  const int64_t n = J.np * J.nq;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  int64_t p = c / J.nq, q = c - p * J.nq;
  const cplx v = coef[h * coef_stride + c];
  uint64_t m = lmask;
  cplx* B = bins + h * bins_stride;
  while (m) {
    int l = __ffsll((long long)m) - 1;
    m &= m - 1;
    uint32_t r = residue_of(lat, J.np, J.nq, l, p, q, (uint32_t)lat.M[l]);
    double* dst = (double*)(B + off[l] + r);
    atomicAdd(dst, v.x);
    atomicAdd(dst + 1, v.y);
  }
}

void scatter(const CandSet& J, const LatticeDev& lat, int Luse, const BlueGeom& g, const cplx* coef,
             int64_t coef_stride, int nrhs, cplx* bins, int64_t bins_stride, cudaStream_t s) {
  const int64_t n = J.n();
  if (n == 0 || nrhs == 0) return;
  uint64_t lmask = Luse >= 64 ? ~0ull : ((1ull << Luse) - 1);
  // algorithmic bytes: the coefficients in, one complex read-modify-write per
  // (k, l) pair
  const double bytes = (double)nrhs * (16.0 * n + 32.0 * n * (int64_t)Luse);
  MR1L_LAUNCH("scatter_kernel", s, 0, bytes,
              scatter_kernel<<<dim3(cdiv(n, 256), nrhs), 256, 0, s>>>(J, lat, lmask, g.off, coef, coef_stride, bins,
                                                                       bins_stride));
}

// ---------------------------------------------------------------------------
// Adjoint of Algorithm 2 in bin order.  A candidate's coefficient reaches only
// the bins where it is collision-free, and such a bin belongs to that
// candidate alone, so the adjoint is a map from bins to candidates, built once
// per plan (random 4-byte stores).  A transform then scales the coefficients
// by 1 / cnt_k (one dense pass; the 1 / M_l goes into the output chirp of the
// evaluation pass) and writes every bin once, in order, copying its
// candidate's value (a small array that stays in L2): no FP64 instruction in
// the sparse pass, which on this GPU costs a whole warp's issue even with few
// lanes active, and no random read-modify-write of 32-byte sectors.
// ---------------------------------------------------------------------------
__global__ void adjoint_map_kernel(CandSet J, LatticeDev lat, uint64_t lmask, const uint64_t* umask,
                                   const int64_t* off, int32_t* map, double* inv_cnt) {
  const int64_t n = J.np * J.nq;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t p = c / J.nq, q = c - p * J.nq;
  uint64_t m = umask[c] & lmask;
  const int cnt = __popcll(m);
  inv_cnt[c] = cnt ? __drcp_rn((double)cnt) : 0.0;
  while (m) {
    const int l = __ffsll((long long)m) - 1;
    m &= m - 1;
    map[off[l] + residue_of(lat, J.np, J.nq, l, p, q, (uint32_t)lat.M[l])] = (int32_t)c;
  }
}

void adjoint_map(const CandSet& J, const LatticeDev& lat, int Luse, const uint64_t* umask, const BlueGeom& g,
                 int32_t* map, double* inv_cnt, int64_t pairs, cudaStream_t s) {
  const int64_t n = J.n();
  if (n == 0) return;
  MR1L_REQUIRE(n < (int64_t(1) << 31), "too many candidates for the adjoint map");
  uint64_t lmask = Luse >= 64 ? ~0ull : ((1ull << Luse) - 1);
  MR1L_LAUNCH("adjoint_map_kernel", s, 0, 16.0 * n + 4.0 * pairs,
              adjoint_map_kernel<<<cdiv(n, 256), 256, 0, s>>>(J, lat, lmask, umask, g.off, map, inv_cnt));
}

__global__ void adjoint_scale_kernel(const cplx* coef, int64_t coef_stride, int64_t n, const double* inv_cnt,
                                     cplx* cs) {
  const int h = blockIdx.y;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  const cplx v = coef[h * coef_stride + c];
  const double sc = inv_cnt[c];
  cs[h * n + c] = cmake(v.x * sc, v.y * sc);
}

// grid (bins of the largest lattice / 256, lattices, right-hand sides)
__global__ void adjoint_bins_kernel(const int* M, const int64_t* off, const int32_t* map, const cplx* cs, int64_t n,
                                    cplx* bins, int64_t bins_stride) {
  const int l = blockIdx.y, h = blockIdx.z;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M[l]) return;
  const int64_t b = off[l] + j;
  const int32_t c = map[b];
  bins[h * bins_stride + b] = c >= 0 ? cs[h * n + c] : cmake(0.0, 0.0);
}

void adjoint_bins(int Luse, int maxM, const BlueGeom& g, int64_t n, const int32_t* map, const double* inv_cnt,
                  const cplx* coef, int64_t coef_stride, int nrhs, cplx* cs, cplx* bins, int64_t bins_stride,
                  cudaStream_t s) {
  if (nrhs == 0 || Luse == 0) return;
  if (n > 0)
    MR1L_LAUNCH("adjoint_scale_kernel", s, 0, 32.0 * nrhs * n + 8.0 * n,
                adjoint_scale_kernel<<<dim3(cdiv(n, 256), nrhs), 256, 0, s>>>(coef, coef_stride, n, inv_cnt, cs));
  // algorithmic bytes: every bin written once, the map and the scaled
  // coefficients read once
  const double bytes = 16.0 * nrhs * (double)g.sum_M + 4.0 * (double)g.sum_M + 16.0 * nrhs * (double)n;
  MR1L_LAUNCH("adjoint_bins_kernel", s, 0, bytes,
              adjoint_bins_kernel<<<dim3(cdiv(maxM, 256), Luse, nrhs), 256, 0, s>>>(g.M, g.off, map, cs, n, bins,
                                                                                    bins_stride));
}

// ---------------------------------------------------------------------------
// Planted sampler
// ---------------------------------------------------------------------------
// weight c_h exp(2 pi i sum_{j in [j0, j1) \ {skip}} h_j x_j)
__device__ __forceinline__ cplx planted_weight(const int32_t* f, cplx c, const double* x, int j0, int j1,
                                               int skip) {
  double phi = 0.0;
  for (int j = j0; j < j1; ++j)
    if (j != skip) phi += (double)f[j] * x[j];
  phi -= floor(phi);
  double sn, cs;
  sincospi(2.0 * phi, &sn, &cs);
  return cmul(c, cmake(cs, sn));
}

// The weight c_h e^{2 pi i h_(>t).x'} of a planted frequency depends on the
// right-hand side (its anchor) but not on the lattice, and the bin
// h_(1..t).z_l mod M_l on the lattice but not on the right-hand side: the
// weights are computed once per (frequency, rhs), the residues once per
// (frequency, lattice).
__global__ void planted_weights_kernel(const int32_t* freqs, const cplx* coeffs, int64_t s_count, int d, int t,
                                       const double* anchors, cplx* wts) {
  const int h = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= s_count) return;
  wts[h * s_count + i] = planted_weight(freqs + i * d, coeffs[i], anchors + (int64_t)h * d, t, d, -1);
}

// one thread per (planted frequency, lattice): the bin, then one atomic add per rhs
__global__ void planted_lattice_kernel(const int32_t* freqs, int64_t s_count, int d, int t, int nrhs,
                                       const cplx* wts, LatticeDev lat, const int64_t* off, cplx* bins,
                                       int64_t bins_stride) {
  const int l = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= s_count) return;
  const int32_t* f = freqs + i * d;
  const int64_t M = lat.M[l];
  const int64_t* z = lat.z + (int64_t)l * lat.t;
  int64_t acc = 0;
  for (int j = 0; j < t; ++j) acc += (int64_t)f[j] * z[j];
  acc %= M;
  if (acc < 0) acc += M;
  for (int h = 0; h < nrhs; ++h) {
    const cplx wv = wts[h * s_count + i];
    double* dst = (double*)(bins + h * bins_stride + off[l] + acc);
    atomicAdd(dst, wv.x);
    atomicAdd(dst + 1, wv.y);
  }
}

void planted_lattice_bins(const int32_t* freqs, const cplx* coeffs, int64_t s_count, int d, int t,
                          const double* anchors_dev, int nrhs, const LatticeDev& lat, int Luse,
                          const BlueGeom& g, cplx* bins, int64_t bins_stride, cplx* wts, cudaStream_t s) {
  if (s_count == 0) return;
  if (Luse == 0 || nrhs == 0) return;
  // algorithmic bytes: every planted row and coefficient read once, the
  // weights written and read once per lattice, one complex read-modify-write
  // per (frequency, lattice, right-hand side)
  MR1L_LAUNCH("planted_weights_kernel", s, 0, (double)s_count * (4.0 * (d - t) + 16.0 + 16.0 * nrhs),
              planted_weights_kernel<<<dim3(cdiv(s_count, 256), nrhs), 256, 0, s>>>(freqs, coeffs, s_count, d, t,
                                                                                     anchors_dev, wts));
  MR1L_LAUNCH("planted_lattice_kernel", s, 0, (double)s_count * Luse * (4.0 * t + 48.0 * nrhs),
              planted_lattice_kernel<<<dim3(cdiv(s_count, 256), Luse), 256, 0, s>>>(
                  freqs, s_count, d, t, nrhs, wts, lat, g.off, bins, bins_stride));
}

// ---------------------------------------------------------------------------
// Section 5.3 test function (tensor-product B-splines)
// ---------------------------------------------------------------------------
// N_m(x) for x in [0, 1): u = m x on knot interval q, Horner in (u - q)
__device__ __forceinline__ double bspline_factor(const BsplineDev& S, int g, double x) {
  const int m = S.order[g];
  const double u = x * (double)m;
  int q = (int)u;
  if (q > m - 1) q = m - 1;
  const double f = u - (double)q;
  const double* c = S.coef[g][q];
  double v = c[m - 1];
  for (int k = m - 2; k >= 0; --k) v = fma(v, f, c[k]);
  return v;
}

__device__ __forceinline__ void load_bspline(const BsplineDev* src, BsplineDev& dst) {
  const int words = (int)(sizeof(BsplineDev) / sizeof(int));
  for (int i = threadIdx.x; i < words; i += blockDim.x) ((int*)&dst)[i] = ((const int*)src)[i];
  __syncthreads();
}

__global__ void bspline_lattice_kernel(const BsplineDev* Sg, int t, const double* anchors, LatticeDev lat,
                                       const int64_t* off, cplx* y, int64_t y_stride) {
  __shared__ BsplineDev S;
  __shared__ double anchor_prod[kBsMaxGroups];
  load_bspline(Sg, S);
  const int l = blockIdx.y, h = blockIdx.z;
  const double* xa = anchors + (int64_t)h * S.d;
  if (threadIdx.x < S.n_groups) {  // factors of the anchored components, once per block
    double p = 1.0;
    for (int i = t; i < S.d; ++i)
      if (S.group_of[i] == (int)threadIdx.x) p *= bspline_factor(S, threadIdx.x, xa[i]);
    anchor_prod[threadIdx.x] = p;
  }
  __syncthreads();
  const int64_t M = lat.M[l];
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int64_t* z = lat.z + (int64_t)l * lat.t;
  double prod[kBsMaxGroups];
  for (int g = 0; g < S.n_groups; ++g) prod[g] = anchor_prod[g];
  for (int i = 0; i < t; ++i) {
    const int g = S.group_of[i];
    if (g < 0) continue;
    const double x = (double)((j * z[i]) % M) / (double)M;  // j z_i < 2^46, exact
    prod[g] *= bspline_factor(S, g, x);
  }
  double f = 0.0;
  for (int g = 0; g < S.n_groups; ++g) f += prod[g];
  y[h * y_stride + off[l] + j] = cmake(f, 0.0);
}

void bspline_lattice(const BsplineDev* S, int t, const double* anchors_dev, int nrhs, const LatticeDev& lat,
                     int Luse, const BlueGeom& g, int max_M, cplx* y, int64_t y_stride, cudaStream_t s) {
  if (Luse == 0 || nrhs == 0) return;
  MR1L_LAUNCH("bspline_lattice_kernel", s, 0, 16.0 * nrhs * g.sum_M,
              bspline_lattice_kernel<<<dim3(cdiv(max_M, 256), Luse, nrhs), 256, 0, s>>>(S, t, anchors_dev, lat,
                                                                                       g.off, y, y_stride));
}

__global__ void bspline_lines_kernel(const BsplineDev* Sg, int t, int K, const double* anchors, cplx* y) {
  __shared__ BsplineDev S;
  load_bspline(Sg, S);
  const int i = blockIdx.y;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= K) return;
  const double* xa = anchors + (int64_t)i * S.d;
  double prod[kBsMaxGroups];
  for (int g = 0; g < S.n_groups; ++g) prod[g] = 1.0;
  for (int c = 0; c < S.d; ++c) {
    const int g = S.group_of[c];
    if (g < 0) continue;
    const double x = c == t - 1 ? (double)l / (double)K : xa[c];
    prod[g] *= bspline_factor(S, g, x);
  }
  double f = 0.0;
  for (int g = 0; g < S.n_groups; ++g) f += prod[g];
  y[(int64_t)i * K + l] = cmake(f, 0.0);
}

void bspline_lines(const BsplineDev* S, int t, int K, const double* anchors_dev, int nlines, cplx* y,
                   cudaStream_t s) {
  MR1L_LAUNCH("bspline_lines_kernel", s, 0, 16.0 * nlines * K,
              bspline_lines_kernel<<<dim3(cdiv(K, 128), nlines), 128, 0, s>>>(S, t, K, anchors_dev, y));
}

__global__ void planted_line_bins_kernel(const int32_t* freqs, const cplx* coeffs, int64_t s_count, int d, int t,
                                         int K, const double* anchors, cplx* bins) {
  const int i = blockIdx.y;
  const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= s_count) return;
  const int32_t* f = freqs + h * d;
  cplx wv = planted_weight(f, coeffs[h], anchors + (int64_t)i * d, 0, d, t - 1);
  int b = f[t - 1] % K;
  if (b < 0) b += K;
  double* dst = (double*)(bins + (int64_t)i * K + b);
  atomicAdd(dst, wv.x);
  atomicAdd(dst + 1, wv.y);
}

// y_l = sum_r B[r] exp(2 pi i l r / K) + eta_l (Philox purpose 4)
__global__ void planted_line_eval_kernel(const cplx* bins, int K, int t, double noise_scale, uint64_t noise_seed,
                                         int rep0, cplx* y) {
  extern __shared__ cplx sh[];
  cplx* ph = sh;       // exp(2 pi i m / K)
  cplx* B = sh + K;
  const int i = blockIdx.x;
  for (int m = threadIdx.x; m < K; m += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)m / (double)K, &sn, &cs);
    ph[m] = cmake(cs, sn);
    B[m] = bins[(int64_t)i * K + m];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < K; l += blockDim.x) {
    cplx acc = cmake(0.0, 0.0);
    int m = 0;  // l r mod K, advanced by l per step
    for (int r = 0; r < K; ++r) {
      cplx v = cmul(B[r], ph[m]);
      acc.x += v.x;
      acc.y += v.y;
      m += l;
      if (m >= K) m -= K;
    }
    if (noise_scale != 0.0) {
      U64Pair u = philox_u64(noise_seed, kNoiseLine, (uint32_t)t, (uint32_t)l, 0u, (uint32_t)(rep0 + i));
      double u1 = ((double)(u.a >> 11) + 1.0) * 0x1.0p-53;
      double u2 = (double)(u.b >> 11) * 0x1.0p-53;
      double R = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      acc.x += noise_scale * (R * cs);
      acc.y += noise_scale * (R * sn);
    }
    y[(int64_t)i * K + l] = acc;
  }
}

void planted_lines(const int32_t* freqs, const cplx* coeffs, int64_t s_count, int d, int t, int K,
                   const double* anchors_dev, int nlines, double noise_scale, uint64_t noise_seed, int rep0,
                   cplx* bins_scratch, cplx* y, cudaStream_t s) {
  MR1L_CUDA(cudaMemsetAsync(bins_scratch, 0, (size_t)nlines * K * sizeof(cplx), s));
  if (s_count) {
    MR1L_LAUNCH("planted_line_bins_kernel", s, 0, 0, planted_line_bins_kernel<<<dim3(cdiv(s_count, 256), nlines), 256, 0, s>>>(freqs, coeffs, s_count, d, t, K,
                                                                               anchors_dev, bins_scratch));
  }
  size_t smem = 2 * (size_t)K * sizeof(cplx);
  if (smem > 48 * 1024)
    MR1L_CUDA(cudaFuncSetAttribute(planted_line_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MR1L_LAUNCH("planted_line_eval_kernel", s, 0, 0, planted_line_eval_kernel<<<nlines, 256, smem, s>>>(bins_scratch, K, t, noise_scale, noise_seed, rep0, y));
}

// ---------------------------------------------------------------------------
// 1-D detection (steps 1 and 2a): one CTA per line.
// ---------------------------------------------------------------------------
__global__ void detect_lines_kernel(const cplx* y, int N, int64_t cap, double theta2, int rel, uint8_t* sel) {
  extern __shared__ unsigned char shraw[];
  const int K = 2 * N + 1;
  cplx* ph = (cplx*)shraw;          // exp(-2 pi i m / K)
  cplx* Y = ph + K;
  uint64_t* key = (uint64_t*)(Y + K);
  __shared__ uint64_t kmax;
  const int i = blockIdx.x;
  if (threadIdx.x == 0) kmax = 0;
  for (int m = threadIdx.x; m < K; m += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)m / (double)K, &sn, &cs);
    ph[m] = cmake(cs, -sn);
    Y[m] = y[(int64_t)i * K + m];
  }
  __syncthreads();
  for (int a = threadIdx.x; a < K; a += blockDim.x) {
    int k = a - N;
    int km = k < 0 ? k + K : k;
    cplx acc = cmake(0.0, 0.0);
    int m = 0;  // km l mod K, advanced by km per step
    for (int l = 0; l < K; ++l) {
      cplx v = cmul(Y[l], ph[m]);
      acc.x += v.x;
      acc.y += v.y;
      m += km;
      if (m >= K) m -= K;
    }
    double re = acc.x / (double)K, im = acc.y / (double)K;
    double k2 = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
    key[a] = (uint64_t)__double_as_longlong(k2);
    atomicMax((unsigned long long*)&kmax, (unsigned long long)key[a]);
  }
  __syncthreads();
  double thr = rel ? theta2 * __longlong_as_double((long long)kmax) : theta2;
  uint64_t tb = (uint64_t)__double_as_longlong(thr);
  for (int a = threadIdx.x; a < K; a += blockDim.x) {
    uint64_t ka = key[a];
    if (ka < tb) continue;
    int64_t rank = 0;
    for (int b = 0; b < K; ++b) {
      uint64_t kb = key[b];
      rank += (kb > ka) || (kb == ka && b < a);
    }
    if (rank < cap) sel[a] = 1;
  }
}

void detect_lines(const cplx* y, int nlines, int N, int64_t cap, double theta2, int rel, uint8_t* sel,
                  cudaStream_t s) {
  const int K = 2 * N + 1;
  size_t smem = 2 * (size_t)K * sizeof(cplx) + (size_t)K * sizeof(uint64_t);
  if (smem > 48 * 1024)
    MR1L_CUDA(cudaFuncSetAttribute(detect_lines_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MR1L_LAUNCH("detect_lines_kernel", s, 0, 0, detect_lines_kernel<<<nlines, 256, smem, s>>>(y, N, cap, theta2, rel, sel));
}

}  // namespace mr1l
