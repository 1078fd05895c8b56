// Thresholded "(up to) s-largest" selection (steps 2e of Algorithm 3) and
// compaction of the detected set.
//
// Keys are bits(|p~|^2) + 1 for covered candidates and 0 otherwise; for
// non-negative doubles the bit pattern orders like the value, so the
// selection is an integer radix select: six passes of an 11-bit digit
// histogram (multi-CTA, shared-memory privatised), the last CTA of each pass
// picking the digit, then a marking pass.  Ties at the cut are broken by the smaller
// candidate id, as the (lexicographic) candidate order demands.
#include "ops.cuh"
#include "prof.cuh"

namespace mr1l {

__global__ void sel_init_kernel(SelectState* st, const uint64_t* keymax, double theta2, int rel, int nrhs) {
  int h = blockIdx.x;
  if (h >= nrhs) return;
  SelectState& S = st[h];
  if (threadIdx.x == 0) {
    double thr = theta2;
    if (rel) {
      uint64_t km = keymax[h];
      double mx = km ? __longlong_as_double((long long)(km - 1)) : 0.0;
      thr = theta2 * mx;
    }
    S.thr = (uint64_t)__double_as_longlong(thr) + 1;  // covered keys carry +1
    S.prefix = 0;
    S.need = 0;
    S.total = 0;
    S.take_all = 0;
    S.eq_count = 0;
    S.ticket = 0;
  }
  for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) S.hist[i] = 0;
}

__device__ __forceinline__ void sel_digit(int pass, int& lo, int& width) {
  // digits from the top: [52,63) [41,52) [30,41) [19,30) [8,19) [0,8)
  lo = pass < kSelPasses - 1 ? 52 - 11 * pass : 0;
  width = pass < kSelPasses - 1 ? 11 : 8;
}

// The last CTA of a histogram pass picks the digit of the cap-th largest key:
// a parallel suffix scan over the bins (256 threads, 8 bins each).
__device__ void sel_pick(SelectState& S, int64_t cap, int pass) {
  __shared__ int64_t part[256];
  __shared__ int64_t cum_above[256];
  int lo, width;
  sel_digit(pass, lo, width);
  const int nb = 1 << width;
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  // thread i owns bins [i*per, (i+1)*per); scan from the highest bin down
  const int t = threadIdx.x;
  int64_t mine = 0;
  for (int k = 0; k < per; ++k) {
    int b = t * per + k;
    if (b < nb) mine += S.hist[b];
  }
  part[t] = mine;
  __syncthreads();
  if (t == 0) {
    int64_t tot = 0;
    for (int i = blockDim.x - 1; i >= 0; --i) {
      cum_above[i] = tot;
      tot += part[i];
    }
    if (pass == 0) {
      S.total = tot;
      if (tot <= cap) S.take_all = 1;
      else S.need = cap;
    }
  }
  __syncthreads();
  if (!S.take_all) {
    const int64_t need = S.need;
    // exactly one thread's range contains the crossing
    if (cum_above[t] < need && cum_above[t] + part[t] >= need) {
      int64_t cum = cum_above[t];
      for (int k = per - 1; k >= 0; --k) {
        int b = t * per + k;
        if (b >= nb) continue;
        int64_t hc = S.hist[b];
        if (cum + hc >= need) {
          S.prefix |= (uint64_t)b << lo;
          S.need = need - cum;
          S.eq_count = hc;
          break;
        }
        cum += hc;
      }
    }
  }
  __syncthreads();
  for (int i = t; i < nb; i += blockDim.x) S.hist[i] = 0;
  if (t == 0) S.ticket = 0;
}

// One round of digit counting: kSelUnroll keys per thread at c0 + threadIdx.x
// + u * stride (keys past n count as 0, which is below every threshold).
constexpr int kSelUnroll = 8;
__device__ __forceinline__ void sel_count_round(const uint64_t* kh, int64_t n, int64_t c0, int64_t stride,
                                                uint64_t thr, uint64_t hi_mask, uint64_t prefix, int lo, int nb,
                                                uint32_t* hist) {
  uint64_t k[kSelUnroll];
#pragma unroll
  for (int u = 0; u < kSelUnroll; ++u) {
    const int64_t c = c0 + threadIdx.x + u * stride;
    k[u] = c < n ? kh[c] : 0;
  }
#pragma unroll
  for (int u = 0; u < kSelUnroll; ++u) {
    const int bin = (k[u] >= thr && (k[u] & hi_mask) == prefix) ? (int)((k[u] >> lo) & (nb - 1)) : -1;
    const unsigned same = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0 && (int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(same));
  }
}

__global__ void __launch_bounds__(256) sel_hist_kernel(const uint64_t* keys, int64_t n, SelectState* st, int pass,
                                                       int64_t cap) {
  __shared__ uint32_t hist[kSelBins];
  __shared__ bool last;
  const int h = blockIdx.y;
  SelectState& S = st[h];
  if (S.take_all) return;  // uniform per segment
  int lo, width;
  sel_digit(pass, lo, width);
  const int nb = 1 << width;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint64_t thr = S.thr;
  const uint64_t hi_mask = pass == 0 ? 0ull : (~0ull << (lo + width));
  const uint64_t prefix = S.prefix & hi_mask;
  const uint64_t* kh = keys + h * n;
  // keys of similar magnitude share the top digits, so the lanes of a warp
  // that hit the same bin are merged into one shared-memory atomic; the keys
  // of kSelUnroll rounds are loaded before any is counted, so their loads
  // are in flight together
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c0 = blockIdx.x * (int64_t)blockDim.x; c0 < n; c0 += stride * kSelUnroll)  // same trip count per warp
    sel_count_round(kh, n, c0, stride, thr, hi_mask, prefix, lo, nb, hist);
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (hist[i]) atomicAdd(&S.hist[i], hist[i]);
  // last CTA of this segment picks the digit
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&S.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) {
    __threadfence();
    sel_pick(S, cap, pass);
  }
}

__global__ void sel_mark_kernel(const uint64_t* keys, int64_t n, const SelectState* st, uint8_t* flags) {
  const int h = blockIdx.y;
  const SelectState& S = st[h];
  const uint64_t thr = S.thr, T = S.prefix;
  const bool all = S.take_all, eq_all = S.need == S.eq_count;
  const uint64_t* kh = keys + h * n;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = kh[c];
    if (k < thr) continue;
    if (all || k > T || (k == T && eq_all)) flags[c] = 1;
  }
}

// Rare: more keys equal to the cut value than still needed; take the ones
// with the smallest candidate ids (single CTA, ids in ascending order).
__global__ void sel_tie_kernel(const uint64_t* keys, int64_t n, const SelectState* st, uint8_t* flags) {
  const int h = blockIdx.x;
  const SelectState& S = st[h];
  if (S.take_all || S.need == S.eq_count) return;
  const uint64_t T = S.prefix;
  const int64_t need = S.need;
  const uint64_t* kh = keys + h * n;
  __shared__ int64_t base;
  __shared__ int warp_cnt[32];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
    int64_t c = c0 + threadIdx.x;
    bool e = c < n && kh[c] == T;
    unsigned b = __ballot_sync(0xffffffffu, e);
    if (lane == 0) warp_cnt[wid] = __popc(b);
    __syncthreads();
    int64_t before = base;
    for (int w = 0; w < wid; ++w) before += warp_cnt[w];
    before += __popc(b & ((1u << lane) - 1));
    if (e && before < need) flags[c] = 1;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int w = 0; w < nw; ++w) base += warp_cnt[w];
    __syncthreads();
    if (base >= need) break;
  }
}

// ---------------------------------------------------------------------------
// The whole selection of a small segment in one CTA: the same six digit
// passes, the pick of each digit by a block-wide suffix scan over the
// shared-memory histogram, the marking and the tie pass.  One launch per
// selection instead of nine, for segments whose keys one CTA reads six times
// faster than nine dependent launches take to start.
// ---------------------------------------------------------------------------
constexpr int kSelSmallThreads = 1024;

// Exclusive suffix sum over the threads of the block: the sum of v over all
// threads with a larger index.  tmp: shared [kSelSmallThreads / 32].
__device__ __forceinline__ uint32_t block_suffix_excl(uint32_t v, uint32_t* tmp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;  // inclusive suffix within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o < 32) x += y;
  }
  if (lane == 0) tmp[w] = x;  // the warp's total
  __syncthreads();
  uint32_t above = 0;
  for (int u = w + 1; u < nw; ++u) above += tmp[u];
  __syncthreads();
  return above + x - v;
}

__global__ void __launch_bounds__(kSelSmallThreads) sel_small_kernel(const uint64_t* keys, int64_t n,
                                                                      const uint64_t* keymax, double theta2, int rel,
                                                                      int64_t cap, uint8_t* flags) {
  __shared__ uint32_t hist[kSelBins];
  __shared__ uint32_t tmp[kSelSmallThreads / 32];
  __shared__ uint64_t s_prefix;
  __shared__ int64_t s_need, s_eq;
  __shared__ int s_all;
  const int h = blockIdx.x;
  const uint64_t* kh = keys + (int64_t)h * n;
  double thr_d = theta2;
  if (rel) {
    const uint64_t km = keymax[h];
    thr_d = theta2 * (km ? __longlong_as_double((long long)(km - 1)) : 0.0);
  }
  const uint64_t thr = (uint64_t)__double_as_longlong(thr_d) + 1;  // covered keys carry +1
  if (threadIdx.x == 0) {
    s_prefix = 0;
    s_need = cap;
    s_eq = 0;
    s_all = 0;
  }
  for (int pass = 0; pass < kSelPasses; ++pass) {
    int lo, width;
    sel_digit(pass, lo, width);
    const int nb = 1 << width;
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint64_t hi_mask = pass == 0 ? 0ull : (~0ull << (lo + width));
    const uint64_t prefix = s_prefix & hi_mask;
    for (int64_t c0 = 0; c0 < n; c0 += (int64_t)blockDim.x * kSelUnroll)  // same trip count for every warp
      sel_count_round(kh, n, c0, blockDim.x, thr, hi_mask, prefix, lo, nb, hist);
    __syncthreads();
    // thread t owns bins 2t and 2t + 1; find the bin holding the need-th largest
    const int b0 = 2 * threadIdx.x;
    const uint32_t h0 = b0 < nb ? hist[b0] : 0, h1 = b0 + 1 < nb ? hist[b0 + 1] : 0;
    const uint32_t above = block_suffix_excl(h0 + h1, tmp);
    if (pass == 0) {
      // the total number of eligible keys is the suffix sum above thread -1
      if (threadIdx.x == 0 && (int64_t)(above + h0 + h1) <= cap) s_all = 1;
      __syncthreads();
      if (s_all) break;
    }
    const int64_t need = s_need;
    __syncthreads();
    if ((int64_t)above < need && (int64_t)(above + h0 + h1) >= need) {
      if ((int64_t)above + h1 >= need) {
        s_prefix |= (uint64_t)(b0 + 1) << lo;
        s_need = need - above;
        s_eq = h1;
      } else {
        s_prefix |= (uint64_t)b0 << lo;
        s_need = need - above - h1;
        s_eq = h0;
      }
    }
    __syncthreads();
  }
  const bool all = s_all;
  const uint64_t T = s_prefix;
  const int64_t need = s_need;
  const bool eq_all = need == s_eq;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    const uint64_t k = kh[c];
    if (k >= thr && (all || k > T || (k == T && eq_all))) flags[c] = 1;
  }
  if (all || eq_all) return;
  // more keys equal to the cut than still needed: the smallest ids among them
  int64_t base = 0;
  for (int64_t c0 = 0; c0 < n && base < need; c0 += blockDim.x) {
    const int64_t c = c0 + threadIdx.x;
    const bool e = c < n && kh[c] == T;
    const unsigned b = __ballot_sync(0xffffffffu, e);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) tmp[w] = __popc(b);
    __syncthreads();
    int64_t pos = base + __popc(b & ((1u << lane) - 1));
    for (int u = 0; u < w; ++u) pos += tmp[u];
    if (e && pos < need) flags[c] = 1;
    int64_t tot = 0;
    for (int u = 0; u < (int)(blockDim.x >> 5); ++u) tot += tmp[u];
    __syncthreads();
    base += tot;
  }
}

void select_topk(const uint64_t* keys, int64_t n, int nrhs, const uint64_t* keymax, double theta2, int rel,
                 int64_t cap, SelectState* st, uint8_t* flags, cudaStream_t s) {
  if (n == 0 || nrhs == 0 || cap <= 0) return;
  if (n <= kSelSmallMax) {
    MR1L_LAUNCH("sel_small_kernel", s, 0, 8.0 * n * nrhs * (kSelPasses + 1),
                sel_small_kernel<<<nrhs, kSelSmallThreads, 0, s>>>(keys, n, keymax, theta2, rel, cap, flags));
    return;
  }
  MR1L_LAUNCH("sel_init_kernel", s, 0, 0, sel_init_kernel<<<nrhs, 256, 0, s>>>(st, keymax, theta2, rel, nrhs));
  int blocks = (int)std::min<int64_t>(cdiv(n, 2048), 304);
  for (int pass = 0; pass < kSelPasses; ++pass)
    MR1L_LAUNCH("sel_hist_kernel", s, 0, 8.0 * n * nrhs,
                sel_hist_kernel<<<dim3(blocks, nrhs), 256, 0, s>>>(keys, n, st, pass, cap));
  MR1L_LAUNCH("sel_mark_kernel", s, 0, 8.0 * n * nrhs,
              sel_mark_kernel<<<dim3(blocks, nrhs), 256, 0, s>>>(keys, n, st, flags));
  MR1L_LAUNCH("sel_tie_kernel", s, 0, 0, sel_tie_kernel<<<nrhs, 1024, 0, s>>>(keys, n, st, flags));
}

// keys[h][c] = bits(re*re + im*im) + 1 (no fused multiply-add) where c is
// eligible, else 0; keymax[h] = the largest key of segment h (zeroed first)
__global__ void keys_kernel(const cplx* p, int64_t n, const uint8_t* eligible, uint64_t* keys, uint64_t* keymax) {
  const int h = blockIdx.y;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  uint64_t key = 0;
  if (c < n) {
    if (!eligible || eligible[c]) {
      const cplx v = p[(int64_t)h * n + c];
      key = (uint64_t)__double_as_longlong(__dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y))) + 1;
    }
    keys[(int64_t)h * n + c] = key;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t u = __shfl_xor_sync(0xffffffffu, key, o);
    key = u > key ? u : key;
  }
  if ((threadIdx.x & 31) == 0 && key) atomicMax((unsigned long long*)(keymax + h), (unsigned long long)key);
}

void value_keys(const cplx* p, int64_t n, int nrhs, const uint8_t* eligible, uint64_t* keys, uint64_t* keymax,
                cudaStream_t s) {
  MR1L_CUDA(cudaMemsetAsync(keymax, 0, nrhs * sizeof(uint64_t), s));
  if (n == 0 || nrhs == 0) return;
  MR1L_LAUNCH("keys_kernel", s, 0, (double)nrhs * n * 24.0 + (eligible ? (double)n : 0.0),
              keys_kernel<<<dim3(cdiv(n, 256), nrhs), 256, 0, s>>>(p, n, eligible, keys, keymax));
}

// ---------------------------------------------------------------------------
// Compaction
// ---------------------------------------------------------------------------
constexpr int kCompactBlock = 1024;

__global__ void compact_count_kernel(const uint8_t* flags, int64_t n, int64_t* counts) {
  int64_t c = blockIdx.x * (int64_t)kCompactBlock + threadIdx.x;
  int f = c < n ? flags[c] != 0 : 0;
  int tot = __syncthreads_count(f);
  if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

__global__ void compact_scan_kernel(int64_t* counts, int64_t nblocks) {
  __shared__ int64_t buf[kCompactBlock];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nblocks; b0 += kCompactBlock) {
    int64_t b = b0 + threadIdx.x;
    int64_t v = b < nblocks ? counts[b] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kCompactBlock; o <<= 1) {
      int64_t add = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (b < nblocks) counts[b] = carry + buf[threadIdx.x] - v;  // exclusive
    __syncthreads();
    if (threadIdx.x == 0) carry += buf[kCompactBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[nblocks] = carry;
}

__global__ void compact_scatter_kernel(CandSet J, const uint8_t* flags, const int64_t* counts, int32_t* out_rows,
                                       const cplx* p, cplx* out_p) {
  __shared__ int warp_cnt[kCompactBlock / 32];
  const int64_t n = J.np * J.nq;
  const int64_t c = blockIdx.x * (int64_t)kCompactBlock + threadIdx.x;
  const bool f = c < n && flags[c] != 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned b = __ballot_sync(0xffffffffu, f);
  if (lane == 0) warp_cnt[wid] = __popc(b);
  __syncthreads();
  if (!f) return;
  int64_t pos = counts[blockIdx.x];
  for (int w = 0; w < wid; ++w) pos += warp_cnt[w];
  pos += __popc(b & ((1u << lane) - 1));
  const int64_t pi = c / J.nq, q = c - pi * J.nq;
  int32_t* row = out_rows + pos * J.t;
  for (int j = 0; j < J.tp; ++j) row[j] = J.pre[pi * J.tp + j];
  if (J.last) row[J.tp] = J.last[q];
  if (out_p) out_p[pos] = p[c];
}

int64_t compact(const CandSet& J, const uint8_t* flags, int32_t* out_rows, const cplx* p, cplx* out_p,
                int64_t* scratch_counts, int64_t scratch_len, int64_t* total_host, cudaStream_t s) {
  const int64_t n = J.n();
  if (n == 0) return 0;
  const int64_t nblocks = cdiv(n, kCompactBlock);
  MR1L_REQUIRE(scratch_len >= nblocks + 1, "compaction scratch too small");
  MR1L_LAUNCH("compact_count_kernel", s, 0, (double)n + 8.0 * nblocks,
              compact_count_kernel<<<nblocks, kCompactBlock, 0, s>>>(flags, n, scratch_counts));
  MR1L_LAUNCH("compact_scan_kernel", s, 0, 0, compact_scan_kernel<<<1, kCompactBlock, 0, s>>>(scratch_counts, nblocks));
  if (out_rows || out_p) {
    MR1L_LAUNCH("compact_scatter_kernel", s, 0, 0, compact_scatter_kernel<<<nblocks, kCompactBlock, 0, s>>>(J, flags, scratch_counts, out_rows, p, out_p));
  }
  int64_t local = 0;
  int64_t* total = total_host ? total_host : &local;
  MR1L_CUDA(cudaMemcpyAsync(total, scratch_counts + nblocks, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  MR1L_CUDA(cudaStreamSynchronize(s));
  return *total;
}

}  // namespace mr1l
