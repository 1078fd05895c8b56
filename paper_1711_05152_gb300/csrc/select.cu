// Thresholded "(up to) s-largest" selection (steps 2e of Algorithm 3) and
// compaction of the detected set.
//
// Keys are bits(|p~|^2) + 1 for covered candidates and 0 otherwise; for
// non-negative doubles the bit pattern orders like the value, so the
// selection is an integer radix select: eight passes of an 8-bit digit
// histogram (multi-CTA, shared-memory privatised) each followed by a one-CTA
// pick, then a marking pass.  Ties at the cut are broken by the smaller
// candidate id, as the (lexicographic) candidate order demands.
#include "ops.cuh"
#include "prof.cuh"

namespace mr1l {

__global__ void sel_init_kernel(SelectState* st, const uint64_t* keymax, double theta2, int rel, int nrhs) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nrhs) return;
  double thr = theta2;
  if (rel) {
    uint64_t km = keymax[h];
    double mx = km ? __longlong_as_double((long long)(km - 1)) : 0.0;
    thr = theta2 * mx;
  }
  SelectState& S = st[h];
  S.thr = (uint64_t)__double_as_longlong(thr) + 1;  // covered keys carry +1
  S.prefix = 0;
  S.need = 0;
  S.total = 0;
  S.take_all = 0;
  S.eq_count = 0;
  for (int i = 0; i < 256; ++i) S.hist[i] = 0;
}

__global__ void sel_hist_kernel(const uint64_t* keys, int64_t n, SelectState* st, int pass) {
  __shared__ uint32_t hist[256];
  const int h = blockIdx.y;
  SelectState& S = st[h];
  if (S.take_all) return;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int shift = 56 - 8 * pass;
  const uint64_t thr = S.thr;
  const uint64_t hi_mask = pass == 0 ? 0ull : (~0ull << (shift + 8));
  const uint64_t prefix = S.prefix & hi_mask;
  const uint64_t* kh = keys + h * n;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = kh[c];
    if (k >= thr && (k & hi_mask) == prefix) atomicAdd(&hist[(k >> shift) & 255], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (hist[i]) atomicAdd(&S.hist[i], hist[i]);
}

__global__ void sel_pick_kernel(SelectState* st, int64_t cap, int pass) {
  SelectState& S = st[blockIdx.x];
  if (threadIdx.x != 0 || S.take_all) return;
  const int shift = 56 - 8 * pass;
  if (pass == 0) {
    int64_t tot = 0;
    for (int i = 0; i < 256; ++i) tot += S.hist[i];
    S.total = tot;
    if (tot <= cap) {
      S.take_all = 1;
      return;
    }
    S.need = cap;
  }
  int64_t cum = 0;
  for (int dgt = 255; dgt >= 0; --dgt) {
    int64_t hcount = S.hist[dgt];
    if (cum + hcount >= S.need) {
      S.prefix |= (uint64_t)dgt << shift;
      S.need -= cum;
      S.eq_count = hcount;
      break;
    }
    cum += hcount;
  }
  for (int i = 0; i < 256; ++i) S.hist[i] = 0;
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

void select_topk(const uint64_t* keys, int64_t n, int nrhs, const uint64_t* keymax, double theta2, int rel,
                 int64_t cap, SelectState* st, uint8_t* flags, cudaStream_t s) {
  if (n == 0 || nrhs == 0) return;
  MR1L_LAUNCH("sel_init_kernel", s, 0, 0, sel_init_kernel<<<cdiv(nrhs, 64), 64, 0, s>>>(st, keymax, theta2, rel, nrhs));
  int blocks = (int)std::min<int64_t>(cdiv(n, 1024), 304);
  for (int pass = 0; pass < 8; ++pass) {
    MR1L_LAUNCH("sel_hist_kernel", s, 0, 0, sel_hist_kernel<<<dim3(blocks, nrhs), 256, 0, s>>>(keys, n, st, pass));
    MR1L_LAUNCH("sel_pick_kernel", s, 0, 0, sel_pick_kernel<<<nrhs, 32, 0, s>>>(st, cap, pass));
  }
  MR1L_LAUNCH("sel_mark_kernel", s, 0, 0, sel_mark_kernel<<<dim3(blocks, nrhs), 256, 0, s>>>(keys, n, st, flags));
  MR1L_LAUNCH("sel_tie_kernel", s, 0, 0, sel_tie_kernel<<<nrhs, 1024, 0, s>>>(keys, n, st, flags));
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
                int64_t* scratch_counts, int64_t scratch_len, cudaStream_t s) {
  const int64_t n = J.n();
  if (n == 0) return 0;
  const int64_t nblocks = cdiv(n, kCompactBlock);
  MR1L_REQUIRE(scratch_len >= nblocks + 1, "compaction scratch too small");
  MR1L_LAUNCH("compact_count_kernel", s, 0, 0, compact_count_kernel<<<nblocks, kCompactBlock, 0, s>>>(flags, n, scratch_counts));
  MR1L_LAUNCH("compact_scan_kernel", s, 0, 0, compact_scan_kernel<<<1, kCompactBlock, 0, s>>>(scratch_counts, nblocks));
  if (out_rows || out_p) {
    MR1L_LAUNCH("compact_scatter_kernel", s, 0, 0, compact_scatter_kernel<<<nblocks, kCompactBlock, 0, s>>>(J, flags, scratch_counts, out_rows, p, out_p));
  }
  int64_t total = 0;
  MR1L_CUDA(cudaMemcpyAsync(&total, scratch_counts + nblocks, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  MR1L_CUDA(cudaStreamSynchronize(s));
  return total;
}

}  // namespace mr1l
