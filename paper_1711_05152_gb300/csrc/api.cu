// C ABI of the library: plans on multiple rank-1 lattices (Algorithms 1, 2,
// lattice evaluation and adjoint) and the dimension-incremental sparse FFT
// driver (Algorithm 3).  Host code here only orchestrates: every step of the
// transforms runs in the CUDA kernels of fft.cu, lattice.cu and select.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <atomic>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ops.cuh"

namespace mr1l {

// ---------------------------------------------------------------------------
// Last error (per thread)
// ---------------------------------------------------------------------------
static thread_local int tl_code = MR1L_OK;
static thread_local std::string tl_msg;

void set_last_error(int code, const std::string& msg) {
  tl_code = code;
  tl_msg = msg;
}

template <typename F>
static int guarded(F&& f) {
  try {
    f();
    return MR1L_OK;
  } catch (const Error& e) {
    set_last_error(e.code, e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error(MR1L_E_NOMEM, "host allocation failed");
    return MR1L_E_NOMEM;
  } catch (const std::exception& e) {
    set_last_error(MR1L_E_CUDA, e.what());
    return MR1L_E_CUDA;
  }
}

// ---------------------------------------------------------------------------
// The block cache behind DevBuf.  Sizes are rounded up (to 2 MiB from 2 MiB
// on, to 4 KiB below) so that the buffers of repeated solves of one shape
// find their blocks again; a request takes the smallest cached block of at
// least its size and at most twice it.  At most kPoolCacheBytes stay cached
// per device; an allocation that fails empties the cache and retries.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kPoolCacheBytes = size_t(8) << 30;
struct BlockPool {
  std::multimap<size_t, void*> free_blocks;
  size_t cached = 0;       // bytes of the free blocks
  size_t outstanding = 0;  // bytes of blocks handed out and not yet released
  int64_t mallocs = 0;     // cudaMalloc calls that succeeded
};
std::mutex g_pool_mu;
// never destroyed: DevBufs with static storage may release after exit-time destructors run
std::map<int, BlockPool>& pools() {
  static auto* m = new std::map<int, BlockPool>();
  return *m;
}
size_t pool_round(size_t bytes) {
  const size_t g = bytes >= (size_t(2) << 20) ? (size_t(2) << 20) : 4096;
  return (bytes + g - 1) / g * g;
}
// allocation requests still to pass before an injected failure (-1: none)
std::atomic<int64_t> g_fail_after{-1};

// Makes `dev` current for the lifetime of the guard (if it is not already).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace

void* dev_alloc(size_t bytes, size_t* block_bytes, int* device) {
  const size_t want = pool_round(bytes);
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  *device = dev;
  int64_t k = g_fail_after.load();
  while (k >= 0 && !g_fail_after.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 0)
    throw Error(MR1L_E_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected failure)");
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    BlockPool& bp = pools()[dev];
    auto it = bp.free_blocks.lower_bound(want);
    if (it != bp.free_blocks.end() && it->first <= 2 * want) {
      void* p = it->second;
      *block_bytes = it->first;
      bp.cached -= it->first;
      bp.outstanding += it->first;
      bp.free_blocks.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lk(g_pool_mu);
      BlockPool& bp = pools()[dev];
      for (auto& kv : bp.free_blocks) cudaFree(kv.second);
      bp.free_blocks.clear();
      bp.cached = 0;
    }
    MR1L_CUDA(cudaMalloc(&p, want));
  }
  *block_bytes = want;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  BlockPool& bp = pools()[dev];
  bp.outstanding += want;
  ++bp.mallocs;
  return p;
}

void dev_free(void* p, size_t block_bytes, int device) {
  if (!p) return;
  // the block's own device: its queued work may still read the block, and its
  // cache is the one that may hand the block out again
  DeviceGuard guard(device);
  const bool idle = cudaDeviceSynchronize() == cudaSuccess;
  if (!idle) cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_pool_mu);
  BlockPool& bp = pools()[device];
  bp.outstanding -= std::min(bp.outstanding, block_bytes);
  if (idle && bp.cached + block_bytes <= kPoolCacheBytes) {
    bp.free_blocks.emplace(block_bytes, p);
    bp.cached += block_bytes;
    return;
  }
  cudaFree(p);
}

// ---------------------------------------------------------------------------
// Algorithm 1 host logic: Lmax, lambda, the prime set of Eq. 2.2, z draws.
// ---------------------------------------------------------------------------
static bool is_prime_u64(int64_t p) {
  if (p < 2) return false;
  if (p % 2 == 0) return p == 2;
  if (p % 3 == 0) return p == 3;
  for (int64_t f = 5; f * f <= p; f += 6)
    if (p % f == 0 || p % (f + 2) == 0) return false;
  return true;
}

static void lmax_lambda(int64_t n, double c, double gamma, int& Lmax, double& lam) {
  Lmax = (int)std::ceil(c * c / ((c - 1.0) * (c - 1.0)) * (std::log((double)n) - std::log(gamma)) / 2.0);
  lam = c * (double)(n - 1);
}

// Rows of the candidate set on the host (only needed for the injectivity
// test of small primes; rows are produced on demand from prefix x last).
struct HostRows {
  const int32_t* pre;
  int tp;
  int64_t np;
  const int32_t* last;  // may be null
  int64_t nq;
  // >= 0: a known upper bound on the component ranges, used instead of
  // scanning the rows (pre may then be null while no prime at or below the
  // bound needs the explicit injectivity test)
  int64_t range_bound = -1;
  int t() const { return tp + (last ? 1 : 0); }
  int64_t n() const { return np * nq; }
  void row(int64_t c, int32_t* out) const {
    int64_t p = c / nq, q = c - p * nq;
    for (int j = 0; j < tp; ++j) out[j] = pre[p * tp + j];
    if (last) out[tp] = last[q];
  }
  // the largest component range max_j (max k_j - min k_j) over J: J is the
  // product prefix x last, so each component ranges over its own factor
  // (O(np tp + nq), not O(np nq t))
  int64_t expansion() const {
    int64_t e = 0;
    if (np == 0 || nq == 0) return 0;
    if (range_bound >= 0) return range_bound;
    for (int j = 0; j < tp; ++j) {
      int64_t lo = INT64_MAX, hi = INT64_MIN;
      for (int64_t p = 0; p < np; ++p) {
        lo = std::min<int64_t>(lo, pre[p * tp + j]);
        hi = std::max<int64_t>(hi, pre[p * tp + j]);
      }
      e = std::max(e, hi - lo);
    }
    if (last) {
      int64_t lo = INT64_MAX, hi = INT64_MIN;
      for (int64_t q = 0; q < nq; ++q) {
        lo = std::min<int64_t>(lo, last[q]);
        hi = std::max<int64_t>(hi, last[q]);
      }
      e = std::max(e, hi - lo);
    }
    return e;
  }
};

// k -> k mod p componentwise injective on J (membership in P^J)
static bool injective_mod(const HostRows& J, int64_t p) {
  const int64_t n = J.n();
  if (n <= 1) return true;
  const int t = J.t();
  // expansion: a prime above every component range is injective
  if (p > J.expansion()) return true;
  std::vector<int32_t> row(t);
  std::vector<std::vector<int64_t>> red(n, std::vector<int64_t>(t));
  for (int64_t c = 0; c < n; ++c) {
    J.row(c, row.data());
    for (int j = 0; j < t; ++j) red[c][j] = ((row[j] % p) + p) % p;
  }
  std::sort(red.begin(), red.end());
  return std::adjacent_find(red.begin(), red.end()) == red.end();
}

static std::vector<int> prime_set(const HostRows& J, double lam, int Lmax) {
  std::vector<int> out;
  int64_t p = (int64_t)std::floor(lam) + 1;
  bool checked_expansion = false;
  int64_t expansion_ok_from = INT64_MAX;
  while ((int)out.size() < Lmax) {
    if (is_prime_u64(p)) {
      bool ok;
      if (checked_expansion && p >= expansion_ok_from) {
        ok = true;
      } else {
        ok = injective_mod(J, p);
        // once a prime beyond the expansion is reached all larger ones pass
        if (!checked_expansion) {
          checked_expansion = true;
          expansion_ok_from = J.expansion() + 1;
        }
      }
      if (ok) {
        MR1L_REQUIRE(p < (int64_t(1) << 31), "lattice size exceeds 2^31");
        out.push_back((int)p);
      }
    }
    ++p;
  }
  return out;
}

// z_l of a search: Philox counter (j, l, attempt + r_l 2^16, 3 << 24 | t),
// r_l the replacement draw of lattice l under the redraw rule (0 otherwise)
static void draw_z(uint64_t seed, int t, int attempt, const std::vector<int>& M, std::vector<int64_t>& z,
                   const std::vector<int>* redraws = nullptr) {
  z.assign(M.size() * t, 0);
  for (size_t l = 0; l < M.size(); ++l)
    for (int j = 0; j < t; ++j) {
      const uint32_t c2 = (uint32_t)attempt + (redraws ? (uint32_t)(*redraws)[l] << 16 : 0u);
      U64Pair u = philox_u64(seed, kZvec, (uint32_t)t, (uint32_t)j, (uint32_t)l, c2);
      z[l * t + j] = 1 + (int64_t)(u.a % (uint64_t)(M[l] - 1));
    }
}

// ---------------------------------------------------------------------------
// Lattice workspace: residues, collisions, coverage, Bluestein tables.
// ---------------------------------------------------------------------------
// Filter spectra a run has computed, by (M, P).  A lattice's spectrum depends
// on its size and the Bluestein length only, and the increments of one run
// repeat lattice sizes: Algorithm 1 takes the smallest admissible primes above
// lambda = 2 (|J| - 1), the same list for every increment with as many
// candidates.  Bounded by kFilterCacheBytes; MR1L_FILTER_CACHE=0 turns it off.
struct FilterCache {
  static constexpr size_t kFilterCacheBytes = size_t(2) << 30;
  std::map<std::pair<int, int>, const cplx*> spectra;
  // spectra are carved from a few large slabs: one block per slab, not per
  // spectrum
  static constexpr size_t kSlabElems = (size_t(256) << 20) / sizeof(cplx);
  std::vector<std::unique_ptr<DevBuf<cplx>>> slabs;
  size_t slab_used = 0, slab_cap = 0, bytes = 0;
  const cplx* find(int M, int P) const {
    auto it = spectra.find({M, P});
    return it == spectra.end() ? nullptr : it->second;
  }
  void put(int M, int P, const cplx* src, cudaStream_t s) {
    const size_t n = (size_t)P, b = n * sizeof(cplx);
    if (bytes + b > kFilterCacheBytes || spectra.count({M, P})) return;
    if (slabs.empty() || slab_used + n > slab_cap) {
      slabs.push_back(std::make_unique<DevBuf<cplx>>());
      slab_cap = std::max(n, kSlabElems);
      slabs.back()->reserve(slab_cap);
      slab_used = 0;
    }
    cplx* dst = slabs.back()->get() + slab_used;
    slab_used += n;
    MR1L_CUDA(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, s));
    bytes += b;
    spectra[{M, P}] = dst;
  }
  static bool enabled() {
    const char* e = std::getenv("MR1L_FILTER_CACHE");
    return !(e && e[0] == '0');
  }
};

struct Staging;
static void stage_h2d(Staging* st, void* dst, const void* src, size_t bytes, cudaStream_t s);
static void stage_reset(Staging* st);
// the coverage result of a search: [0] Lneed, [1] uncovered, [2 + l] |I_l|,
// [kCoverFirst + l] candidates whose first collision-free lattice is l
constexpr int kCoverFirst = 2 + 64, kCoverInts = 2 + 128;

struct LatticeWork {
  int t = 0, L = 0, Luse = 0;
  Staging* stage = nullptr;  // pinned staging of the host-to-device copies (optional)
  int* cover_host = nullptr;  // pinned [2] for the coverage result (optional)
  std::vector<int> Mh;
  std::vector<int64_t> zh, offh;
  int64_t words = 0, sumM_all = 0, sumM = 0;
  int Lneed = 0, n_uncovered = 0;
  std::vector<int64_t> I_size;       // |I_l| per lattice
  std::vector<int64_t> first_count;  // candidates whose first collision-free lattice is l
  // sum of |I_l| over the lattices in use (pairs (k, l) with k in I_l)
  int64_t pairs() const {
    int64_t p = 0;
    for (int l = 0; l < Luse && l < (int)I_size.size(); ++l) p += I_size[l];
    return p;
  }
  DevBuf<int> M;
  DevBuf<int64_t> z, off, bm_off;
  DevBuf<uint32_t> pre_res, last_res, seen;
  DevBuf<uint64_t> umask;
  DevBuf<int> cover;
  DevBuf<cplx> w, ws, Bh, chirp_seed;
  DevBuf<float4> w_df, ws_df;
  // filter spectra of the lattices a FilterCache does not hold
  std::vector<int> sub_Mh;
  std::vector<int64_t> sub_offh;
  DevBuf<int> sub_M;
  DevBuf<int64_t> sub_off;
  DevBuf<cplx> sub_Bh;
  int df = 0;  // Bluestein butterflies in double-float arithmetic
  BlueGeom geom{};
  LatticeDev dev() {
    LatticeDev d;
    d.L = L;
    d.t = t;
    d.M = M.get();
    d.z = z.get();
    d.pre_res = pre_res.get();
    d.last_res = last_res.get();
    return d;
  }

  // Residues, collision counts and coverage of lattices (M, z) on J.
  void load(const CandSet& J, const std::vector<int>& Ms, const std::vector<int64_t>& zs, int t_, cudaStream_t s) {
    t = t_;
    L = (int)Ms.size();
    MR1L_REQUIRE(L >= 1 && L <= 64, "number of lattices must be in [1, 64]");
    Mh = Ms;
    zh = zs;
    offh.assign(L, 0);
    std::vector<int64_t> bm(L, 0);
    sumM_all = 0;
    words = 0;
    for (int l = 0; l < L; ++l) {
      offh[l] = sumM_all;
      bm[l] = words;
      sumM_all += Mh[l];
      words += (Mh[l] + 31) / 32;
    }
    M.reserve(L);
    z.reserve((size_t)L * t);
    off.reserve(L);
    bm_off.reserve(L);
    stage_h2d(stage, M.get(), Mh.data(), L * sizeof(int), s);
    stage_h2d(stage, z.get(), zh.data(), (size_t)L * t * sizeof(int64_t), s);
    stage_h2d(stage, off.get(), offh.data(), L * sizeof(int64_t), s);
    stage_h2d(stage, bm_off.get(), bm.data(), L * sizeof(int64_t), s);
    pre_res.reserve((size_t)L * std::max<int64_t>(J.np, 1));
    last_res.reserve((size_t)L * std::max<int64_t>(J.nq, 1));
    seen.reserve(2 * words);
    umask.reserve(std::max<int64_t>(J.n(), 1));
    cover.reserve(kCoverInts);
    MR1L_CUDA(cudaMemsetAsync(seen.get(), 0, 2 * words * sizeof(uint32_t), s));
    residues(J, dev(), s);
    collide_and_cover(J, dev(), seen.get(), bm_off.get(), words, umask.get(), cover.get(), s);
    int hc_local[kCoverInts];
    int* hc = cover_host ? cover_host : hc_local;
    MR1L_CUDA(cudaMemcpyAsync(hc, cover.get(), kCoverInts * sizeof(int), cudaMemcpyDeviceToHost, s));
    MR1L_CUDA(cudaStreamSynchronize(s));
    Lneed = hc[0];
    n_uncovered = hc[1];
    I_size.assign(hc + 2, hc + 2 + L);
    first_count.assign(hc + kCoverFirst, hc + kCoverFirst + L);
  }

  // Chirp and filter tables of lattices 0..Luse-1; filter spectra found in
  // cache are copied instead of computed, and new ones are added to it.
  void tables(int Luse_, cudaStream_t s, FilterCache* cache = nullptr) {
    Luse = Luse_;
    int maxM = 0;
    sumM = 0;
    for (int l = 0; l < Luse; ++l) {
      maxM = std::max(maxM, Mh[l]);
      sumM += Mh[l];
    }
    const int P = blue_length(2 * (int64_t)maxM - 1);
    MR1L_REQUIRE(P > 0, "lattice size too large for the Bluestein FFT (2 M - 1 > 2^25)");
    geom = BlueGeom{};
    blue_split(geom, P);
    geom.L = Luse;
    geom.off = off.get();
    geom.M = M.get();
    w.reserve(std::max<int64_t>(sumM, 1));
    ws.reserve(std::max<int64_t>(sumM, 1));
    Bh.reserve((size_t)Luse * geom.P);
    geom.w = w.get();
    geom.ws = ws.get();
    geom.Bh = Bh.get();
    geom.tw = twiddle_table(P, s);
    if (P > kSmallMax) {
      geom.twr = row_twiddle_table(P, geom.P2, s);
      geom.twc = col_twiddle_table(P, geom.P2, s);
    }
    geom.twn = small_twiddles(s);
    geom.sum_M = sumM;
    geom.df = df;
    if (df) {
      w_df.reserve(std::max<int64_t>(sumM, 1));
      ws_df.reserve(std::max<int64_t>(sumM, 1));
      geom.w_df = w_df.get();
      geom.ws_df = ws_df.get();
      geom.tw_df = twiddle_table_df(P, s);
      if (P > kSmallMax) {
        geom.twr_df = row_twiddle_table_df(P, geom.P2, s);
        geom.twc_df = col_twiddle_table_df(P, geom.P2, s);
      }
      geom.twn_df = small_twiddles_df(s);
    }
    chirp_seed.reserve((size_t)Luse * kChirpSeedLen);
    chirp_tables(geom, maxM, chirp_seed.get(), s);  // writes the double-float copies as well when df
    if (!cache) {
      blue_filter(geom, s);
      return;
    }
    const size_t pb = (size_t)P * sizeof(cplx);
    std::vector<int> miss;
    for (int l = 0; l < Luse; ++l) {
      if (const cplx* hit = cache->find(Mh[l], P))
        MR1L_CUDA(cudaMemcpyAsync(Bh.get() + (size_t)l * P, hit, pb, cudaMemcpyDeviceToDevice, s));
      else
        miss.push_back(l);
    }
    if (miss.empty()) return;
    if ((int)miss.size() == Luse) {
      blue_filter(geom, s);
    } else {
      // the missing lattices as a geometry of their own (sizes, chirp offsets),
      // spectra into scratch, then into place
      const int nm = (int)miss.size();
      sub_Mh.resize(nm);
      sub_offh.resize(nm);
      for (int i = 0; i < nm; ++i) {
        sub_Mh[i] = Mh[miss[i]];
        sub_offh[i] = offh[miss[i]];
      }
      sub_M.reserve(nm);
      sub_off.reserve(nm);
      sub_Bh.reserve((size_t)nm * P);
      stage_h2d(stage, sub_M.get(), sub_Mh.data(), nm * sizeof(int), s);
      stage_h2d(stage, sub_off.get(), sub_offh.data(), nm * sizeof(int64_t), s);
      BlueGeom gs = geom;
      gs.L = nm;
      gs.M = sub_M.get();
      gs.off = sub_off.get();
      gs.Bh = sub_Bh.get();
      blue_filter(gs, s);
      for (int i = 0; i < nm; ++i)
        MR1L_CUDA(cudaMemcpyAsync(Bh.get() + (size_t)miss[i] * P, sub_Bh.get() + (size_t)i * P, pb,
                                  cudaMemcpyDeviceToDevice, s));
    }
    for (int l : miss) cache->put(Mh[l], P, Bh.get() + (size_t)l * P, s);
  }
};

// Step 2b of Algorithm 3: Algorithm 1 on J with the prime sizes `primes`,
// repeated up to b times until condition (2.1) holds.  The GPU evaluates all
// lattices of a search at once; with `redraw` (the rule of the remark after
// Algorithm 1) a lattice that covers no candidate the earlier ones leave
// uncovered has its z drawn again (at most kRedrawCap times) and the search is
// evaluated again: lattices before it are unchanged, so the kept lattices are
// those of the one-lattice-at-a-time rule.  Returns the searches used; lw
// holds the last one.
constexpr int kRedrawCap = 64;
static int search_lattices(LatticeWork& lw, const CandSet& J, const std::vector<int>& primes, uint64_t seed, int t,
                           int b, bool redraw, cudaStream_t s, Staging* stage) {
  std::vector<int64_t> zs;
  int attempts = 0;
  for (int a = 0; a < b; ++a) {
    std::vector<int> rd(primes.size(), 0);
    for (;;) {
      draw_z(seed, t, a, primes, zs, &rd);
      lw.load(J, primes, zs, t, s);
      if (stage) stage_reset(stage);  // load() synchronised the stream
      if (!redraw) break;
      const int limit = lw.n_uncovered == 0 ? lw.Lneed : (int)primes.size();
      int idle = -1;
      for (int l = 0; l < limit; ++l)
        if (lw.first_count[l] == 0 && rd[l] < kRedrawCap) {
          idle = l;
          break;
        }
      if (idle < 0) break;
      ++rd[idle];
    }
    attempts = a + 1;
    if (lw.n_uncovered == 0) break;
  }
  return attempts;
}

// Validation shared by the plan constructors.
static void validate_set(const int32_t* I, int64_t nI, int t) {
  MR1L_REQUIRE(I != nullptr || nI == 0, "I is null");
  MR1L_REQUIRE(nI >= 1, "the frequency set must not be empty");
  MR1L_REQUIRE(t >= 1 && t <= 64, "t must be in [1, 64]");
  for (int64_t i = 0; i < nI * t; ++i) MR1L_REQUIRE(I[i] > -32768 && I[i] < 32768, "|k_j| must be < 2^15");
  std::vector<int64_t> idx(nI);
  for (int64_t i = 0; i < nI; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    return std::lexicographical_compare(I + a * t, I + a * t + t, I + b * t, I + b * t + t);
  });
  for (int64_t i = 1; i < nI; ++i)
    MR1L_REQUIRE(!std::equal(I + idx[i - 1] * t, I + idx[i - 1] * t + t, I + idx[i] * t),
                 "frequencies must be pairwise distinct");
}

}  // namespace mr1l

using namespace mr1l;

// ---------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------
struct mr1l_plan_s {
  int64_t nI = 0;
  int t = 0;
  int flags = 0;
  int attempts = 0;
  DevBuf<int32_t> I;
  LatticeWork lw;
  // grow-only transform scratch
  DevBuf<cplx> C, bins, work;
  // the adjoint's bin -> candidate map and per-candidate 1 / cnt, built once
  DevBuf<int32_t> adj_map;
  DevBuf<double> adj_inv;
  DevBuf<cplx> adj_coef;  // scratch: the coefficients scaled by 1 / cnt_k
  bool adj_ready = false;
  CandSet cand() const {
    CandSet J;
    J.tp = t;
    J.t = t;
    J.np = nI;
    J.nq = 1;
    J.pre = I.get();
    J.last = nullptr;
    return J;
  }
};

static void plan_finish(mr1l_plan_t* p, int Luse, cudaStream_t s) {
  p->lw.tables(Luse, s);
  MR1L_CUDA(cudaStreamSynchronize(s));
}

extern "C" int mr1l_last_error(char* buf, size_t len) {
  if (buf && len) {
    size_t k = std::min(len - 1, tl_msg.size());
    std::memcpy(buf, tl_msg.data(), k);
    buf[k] = 0;
  }
  return tl_code;
}

extern "C" int mr1l_version(void) { return 100; }

extern "C" int mr1l_pool_stats(int device, int64_t* outstanding, int64_t* cached, int64_t* mallocs) {
  return guarded([&] {
    MR1L_REQUIRE(device >= 0, "device must be >= 0");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = pools().find(device);
    if (outstanding) *outstanding = it == pools().end() ? 0 : (int64_t)it->second.outstanding;
    if (cached) *cached = it == pools().end() ? 0 : (int64_t)it->second.cached;
    if (mallocs) *mallocs = it == pools().end() ? 0 : it->second.mallocs;
  });
}

extern "C" int mr1l_inject_alloc_failure(int64_t after) {
  return guarded([&] {
    MR1L_REQUIRE(after >= -1, "after must be >= -1");
    g_fail_after.store(after);
  });
}

extern "C" int mr1l_plan(const int32_t* I, int64_t nI, int t, int L, const int64_t* M, const int64_t* z, int flags,
                         void* stream, mr1l_plan_t** out) {
  return guarded([&] {
    MR1L_REQUIRE(out != nullptr, "out is null");
    *out = nullptr;
    validate_set(I, nI, t);
    MR1L_REQUIRE(L >= 1 && L <= 64, "L must be in [1, 64]");
    MR1L_REQUIRE(M != nullptr && z != nullptr, "M or z is null");
    std::vector<int> Ms(L);
    for (int l = 0; l < L; ++l) {
      MR1L_REQUIRE(M[l] >= 2 && M[l] < (int64_t(1) << 31), "M_l must be in [2, 2^31)");
      MR1L_REQUIRE(is_prime_u64(M[l]), "M_l must be prime");
      for (int k = 0; k < l; ++k) MR1L_REQUIRE(M[k] != M[l], "lattice sizes must be distinct");
      Ms[l] = (int)M[l];
    }
    std::vector<int64_t> zs((size_t)L * t);
    for (int l = 0; l < L; ++l)
      for (int j = 0; j < t; ++j) {
        MR1L_REQUIRE(z[l * t + j] >= 0 && z[l * t + j] < M[l], "z_l must lie in [0, M_l)");
        zs[l * t + j] = z[l * t + j];
      }
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<mr1l_plan_t> p(new mr1l_plan_t());
    p->nI = nI;
    p->t = t;
    p->flags = flags;
    p->attempts = 1;
    p->I.reserve(nI * t);
    p->lw.df = (flags & MR1L_FFT_DF) ? 1 : 0;
    MR1L_CUDA(cudaMemcpyAsync(p->I.get(), I, nI * t * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    p->lw.load(p->cand(), Ms, zs, t, s);
    if ((flags & MR1L_STRICT) && p->lw.n_uncovered)
      throw Error(MR1L_E_NOT_RECONSTRUCTING, "the lattices do not satisfy condition (2.1) for I");
    plan_finish(p.get(), L, s);
    *out = p.release();
  });
}

extern "C" int mr1l_plan_search(const int32_t* I, int64_t nI, int t, double c, double gamma, int b, uint64_t seed,
                                int flags, void* stream, mr1l_plan_t** out) {
  return guarded([&] {
    MR1L_REQUIRE(out != nullptr, "out is null");
    *out = nullptr;
    validate_set(I, nI, t);
    MR1L_REQUIRE(c > 1.0 && gamma > 0.0 && gamma < 1.0, "need c > 1 and 0 < gamma < 1");
    MR1L_REQUIRE(b >= 1, "b must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<mr1l_plan_t> p(new mr1l_plan_t());
    p->nI = nI;
    p->t = t;
    p->flags = flags;
    p->lw.df = (flags & MR1L_FFT_DF) ? 1 : 0;
    p->I.reserve(nI * t);
    MR1L_CUDA(cudaMemcpyAsync(p->I.get(), I, nI * t * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int Lmax;
    double lam;
    lmax_lambda(nI, c, gamma, Lmax, lam);
    MR1L_REQUIRE(Lmax >= 1 && Lmax <= 64, "Lmax out of range");
    HostRows rows{I, t, nI, nullptr, 1};
    std::vector<int> primes = prime_set(rows, lam, Lmax);
    p->attempts = search_lattices(p->lw, p->cand(), primes, seed, t, b, (flags & MR1L_REDRAW) != 0, s, nullptr);
    int Luse = p->lw.n_uncovered == 0 ? p->lw.Lneed : Lmax;
    if (p->lw.n_uncovered && (flags & MR1L_STRICT))
      throw Error(MR1L_E_NOT_RECONSTRUCTING, "no reconstructing lattice after b searches");
    if (Luse < Lmax) {
      // drop the lattices beyond the first full coverage (Algorithm 1 stops there)
      std::vector<int> Ms(primes.begin(), primes.begin() + Luse);
      std::vector<int64_t> z2(p->lw.zh.begin(), p->lw.zh.begin() + (size_t)Luse * t);
      p->lw.load(p->cand(), Ms, z2, t, s);
    }
    plan_finish(p.get(), p->lw.L, s);
    *out = p.release();
  });
}

extern "C" int mr1l_plan_info(const mr1l_plan_t* plan, int* L, int64_t* M_out, int64_t* z_out, int64_t* nodes,
                              int64_t* sum_M, int64_t* n_uncovered) {
  return guarded([&] {
    MR1L_REQUIRE(plan != nullptr, "plan is null");
    const LatticeWork& lw = plan->lw;
    if (L) *L = lw.L;
    if (M_out)
      for (int l = 0; l < lw.L; ++l) M_out[l] = lw.Mh[l];
    if (z_out)
      for (size_t i = 0; i < lw.zh.size(); ++i) z_out[i] = lw.zh[i];
    if (nodes) *nodes = 1 - lw.L + lw.sumM_all;
    if (sum_M) *sum_M = lw.sumM_all;
    if (n_uncovered) *n_uncovered = lw.n_uncovered;
  });
}

extern "C" int mr1l_plan_masks(const mr1l_plan_t* plan, uint64_t* masks, uint32_t* res) {
  return guarded([&] {
    MR1L_REQUIRE(plan != nullptr, "plan is null");
    const LatticeWork& lw = plan->lw;
    if (masks)
      MR1L_CUDA(cudaMemcpy(masks, lw.umask.get(), plan->nI * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (res) {
      MR1L_CUDA(cudaMemcpy(res, lw.pre_res.get(), (size_t)lw.L * plan->nI * sizeof(uint32_t),
                           cudaMemcpyDeviceToHost));
    }
  });
}

extern "C" void mr1l_destroy(mr1l_plan_t* plan) { delete plan; }

static void reconstruct_impl(mr1l_plan_t* plan, const void* y, int nrhs, void* c, cudaStream_t s) {
  MR1L_REQUIRE(plan != nullptr, "plan is null");
  MR1L_REQUIRE(nrhs >= 0 && nrhs <= 65535 / 64, "nrhs out of range");
  if (nrhs == 0) return;
  MR1L_REQUIRE(y != nullptr && c != nullptr, "null array");
  MR1L_REQUIRE(((uintptr_t)y & 15) == 0 && ((uintptr_t)c & 15) == 0, "arrays must be 16-byte aligned");
  LatticeWork& lw = plan->lw;
  const int64_t sumM = lw.sumM;
  plan->C.reserve((size_t)nrhs * sumM);
  plan->work.reserve((size_t)nrhs * lw.Luse * lw.geom.P);
  BlueIO io{};
  io.in = (const cplx*)y;
  io.in_stride = sumM;
  io.out = plan->C.get();
  io.out_stride = sumM;
  io.work = plan->work.get();
  blue_run(lw.geom, io, kModeRecon, nrhs, s);
  gather(plan->cand(), lw.dev(), lw.Luse, lw.umask.get(), lw.geom, plan->C.get(), sumM, nrhs, (cplx*)c, plan->nI,
         nullptr, nullptr, lw.pairs(), s);
}

static void evaluate_impl(mr1l_plan_t* plan, const void* c, int nrhs, void* y, int mode, cudaStream_t s) {
  MR1L_REQUIRE(plan != nullptr, "plan is null");
  MR1L_REQUIRE(mode == MR1L_EVAL || mode == MR1L_ADJOINT, "mode must be MR1L_EVAL or MR1L_ADJOINT");
  MR1L_REQUIRE(nrhs >= 0 && nrhs <= 65535 / 64, "nrhs out of range");
  if (nrhs == 0) return;
  MR1L_REQUIRE(y != nullptr && c != nullptr, "null array");
  MR1L_REQUIRE(((uintptr_t)y & 15) == 0 && ((uintptr_t)c & 15) == 0, "arrays must be 16-byte aligned");
  LatticeWork& lw = plan->lw;
  const int64_t sumM = lw.sumM;
  plan->bins.reserve((size_t)nrhs * sumM);
  plan->work.reserve((size_t)nrhs * lw.Luse * lw.geom.P);
  if (mode == MR1L_ADJOINT) {
    // the bin -> candidate map of the adjoint, built on the first adjoint
    // transform of the plan
    if (!plan->adj_ready) {
      plan->adj_map.reserve(sumM);
      plan->adj_inv.reserve(plan->nI);
      MR1L_CUDA(cudaMemsetAsync(plan->adj_map.get(), 0xff, sumM * sizeof(int32_t), s));
      adjoint_map(plan->cand(), lw.dev(), lw.Luse, lw.umask.get(), lw.geom, plan->adj_map.get(),
                  plan->adj_inv.get(), lw.pairs(), s);
      plan->adj_ready = true;
    }
    int maxM = 0;
    for (int l = 0; l < lw.Luse; ++l) maxM = std::max(maxM, lw.Mh[l]);
    plan->adj_coef.reserve((size_t)nrhs * plan->nI);
    adjoint_bins(lw.Luse, maxM, lw.geom, plan->nI, plan->adj_map.get(), plan->adj_inv.get(), (const cplx*)c,
                 plan->nI, nrhs, plan->adj_coef.get(), plan->bins.get(), sumM, s);
  } else {
    MR1L_CUDA(cudaMemsetAsync(plan->bins.get(), 0, (size_t)nrhs * sumM * sizeof(cplx), s));
    scatter(plan->cand(), lw.dev(), lw.Luse, lw.geom, (const cplx*)c, plan->nI, nrhs, plan->bins.get(), sumM, s);
  }
  BlueIO io{};
  io.in = plan->bins.get();
  io.in_stride = sumM;
  io.out = (cplx*)y;
  io.out_stride = sumM;
  io.work = plan->work.get();
  io.out_scaled = mode == MR1L_ADJOINT;
  blue_run(lw.geom, io, kModeEval, nrhs, s);
}

extern "C" int mr1l_reconstruct(mr1l_plan_t* plan, const void* y, int nrhs, void* c, void* stream) {
  return guarded([&] { reconstruct_impl(plan, y, nrhs, c, (cudaStream_t)stream); });
}

extern "C" int mr1l_evaluate(mr1l_plan_t* plan, const void* c, int nrhs, void* y, int mode, void* stream) {
  return guarded([&] { evaluate_impl(plan, c, nrhs, y, mode, (cudaStream_t)stream); });
}

// Runs body(i, stream_i) for i < count on up to kBatchStreams streams forked
// from s (they wait for the work already queued on s) and joined back into s.
// Entries with the same plan share a stream, since a plan's scratch buffers
// serve one transform at a time.
constexpr int kBatchStreams = 8;
template <class F>
static void fork_join(mr1l_plan_t* const* plans, int count, cudaStream_t s, F&& body) {
  if (count <= 0) return;
  const int ns = std::min(count, kBatchStreams);
  struct Res {
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> ev;
    ~Res() {
      for (auto e : ev)
        if (e) cudaEventDestroy(e);
      for (auto x : st)
        if (x) cudaStreamDestroy(x);
    }
  } r;
  r.st.assign(ns, nullptr);
  r.ev.assign(ns + 1, nullptr);
  for (auto& e : r.ev) MR1L_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (auto& x : r.st) MR1L_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  MR1L_CUDA(cudaEventRecord(r.ev[ns], s));
  for (auto x : r.st) MR1L_CUDA(cudaStreamWaitEvent(x, r.ev[ns], 0));
  std::map<const mr1l_plan_t*, int> lane;
  int next = 0;
  for (int i = 0; i < count; ++i) {
    auto it = lane.find(plans[i]);
    const int k = it != lane.end() ? it->second : (lane[plans[i]] = next++ % ns);
    body(i, r.st[k]);
  }
  for (int k = 0; k < ns; ++k) {
    MR1L_CUDA(cudaEventRecord(r.ev[k], r.st[k]));
    MR1L_CUDA(cudaStreamWaitEvent(s, r.ev[k], 0));
  }
}

extern "C" int mr1l_reconstruct_batch(mr1l_plan_t* const* plans, int count, const void* const* y, const int* nrhs,
                                      void* const* c, void* stream) {
  return guarded([&] {
    MR1L_REQUIRE(count >= 0, "count must be >= 0");
    if (count == 0) return;
    MR1L_REQUIRE(plans && y && nrhs && c, "null argument");
    fork_join(plans, count, (cudaStream_t)stream,
              [&](int i, cudaStream_t si) { reconstruct_impl(plans[i], y[i], nrhs[i], c[i], si); });
  });
}

extern "C" int mr1l_evaluate_batch(mr1l_plan_t* const* plans, int count, const void* const* c, const int* nrhs,
                                   void* const* y, int mode, void* stream) {
  return guarded([&] {
    MR1L_REQUIRE(count >= 0, "count must be >= 0");
    if (count == 0) return;
    MR1L_REQUIRE(plans && c && nrhs && y, "null argument");
    fork_join(plans, count, (cudaStream_t)stream,
              [&](int i, cudaStream_t si) { evaluate_impl(plans[i], c[i], nrhs[i], y[i], mode, si); });
  });
}

// ---------------------------------------------------------------------------
// Algorithm 3
// ---------------------------------------------------------------------------
namespace mr1l {

// ---------------------------------------------------------------------------
// Section 5.3 test function: polynomial pieces of N_m(x) = C_m m B_m(m x)
// ---------------------------------------------------------------------------
static int64_t binom_i64(int n, int k) {
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
static int64_t ipow_i64(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}
static double factorial_d(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// On [q, q+1), B_m(q + f) = 1/(m-1)! sum_{j<=q} (-1)^j binom(m,j) (q - j + f)^{m-1}
// (truncated-power form), i.e. sum_k a_{q,k} f^k / (m-1)! with the integers
// a_{q,k} = binom(m-1,k) sum_{j<=q} (-1)^j binom(m,j) (q-j)^{m-1-k}.
// C_m^-2 = m B_2m(m) (the autocorrelation of B_m is B_2m), B_2m(m) from the
// same form in integers.
static void bspline_tables(const sfft_sampler& S, int d, BsplineDev& B) {
  std::memset(&B, 0, sizeof(B));
  B.d = d;
  B.n_groups = S.n_groups;
  for (int i = 0; i < d; ++i) B.group_of[i] = S.group_of[i];
  for (int g = 0; g < S.n_groups; ++g) {
    const int m = S.orders[g];
    B.order[g] = m;
    int64_t s2 = 0;
    for (int j = 0; j <= m; ++j) s2 += ((j & 1) ? -1 : 1) * binom_i64(2 * m, j) * ipow_i64(m - j, 2 * m - 1);
    const long double b2m = (long double)s2 / (long double)factorial_d(2 * m - 1);
    const long double Cm = 1.0L / std::sqrt((long double)m * b2m);
    const long double scale = Cm * (long double)m / (long double)factorial_d(m - 1);
    for (int q = 0; q < m; ++q)
      for (int k = 0; k < m; ++k) {
        int64_t a = 0;
        for (int j = 0; j <= q; ++j) a += ((j & 1) ? -1 : 1) * binom_i64(m, j) * ipow_i64(q - j, m - 1 - k);
        B.coef[g][q][k] = (double)((long double)(a * binom_i64(m - 1, k)) * scale);
      }
  }
}

// Pinned host memory for the small copies of a solve.  A copy from pageable
// host memory may wait for the stream (the driver stages it) and a copy to
// pageable memory always does; from and to pinned memory both stay
// asynchronous.  Released blocks are kept per process (at most 64 MiB) since
// cudaHostAlloc is slow.
namespace {
std::mutex g_pinned_mu;
std::multimap<size_t, void*>& pinned_free() {
  static auto* m = new std::multimap<size_t, void*>();
  return *m;
}
size_t g_pinned_cached = 0;
constexpr size_t kPinnedCacheBytes = size_t(64) << 20;
}  // namespace

struct PinnedBuf {
  void* p = nullptr;
  size_t n = 0;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf&) = delete;
  PinnedBuf& operator=(const PinnedBuf&) = delete;
  ~PinnedBuf() { release(); }
  void release() {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (g_pinned_cached + n <= kPinnedCacheBytes) {
      pinned_free().emplace(n, p);
      g_pinned_cached += n;
    } else {
      cudaFreeHost(p);
    }
    p = nullptr;
    n = 0;
  }
  void* reserve(size_t bytes) {
    if (bytes <= n && p) return p;
    release();
    const size_t want = std::max<size_t>(size_t(1) << 16, (bytes + 4095) / 4096 * 4096);
    {
      std::lock_guard<std::mutex> lk(g_pinned_mu);
      auto it = pinned_free().lower_bound(want);
      if (it != pinned_free().end() && it->first <= 4 * want) {
        p = it->second;
        n = it->first;
        g_pinned_cached -= n;
        pinned_free().erase(it);
        return p;
      }
    }
    MR1L_CUDA(cudaHostAlloc(&p, want, cudaHostAllocDefault));
    n = want;
    return p;
  }
};

// Host-to-device staging through a pinned buffer: put() copies the source
// into the buffer and queues the device copy from there.  The buffer is
// reused only after the stream has been synchronised (reset()); when it is
// full, put() synchronises first.
struct Staging {
  PinnedBuf buf;
  size_t used = 0;
  cudaStream_t s = nullptr;
  void h2d(void* dst, const void* src, size_t bytes) {
    if (!bytes) return;
    const size_t need = (bytes + 255) / 256 * 256;
    if (used + need > buf.n) {
      if (used) {
        MR1L_CUDA(cudaStreamSynchronize(s));
        used = 0;
      }
      if (need > buf.n) buf.reserve(std::max(need, size_t(1) << 20));
    }
    char* pin = (char*)buf.p + used;
    used += need;
    std::memcpy(pin, src, bytes);
    MR1L_CUDA(cudaMemcpyAsync(dst, pin, bytes, cudaMemcpyHostToDevice, s));
  }
  void reset() { used = 0; }
};

static void stage_reset(Staging* st) { st->reset(); }

static void stage_h2d(Staging* st, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (st)
    st->h2d(dst, src, bytes);
  else if (bytes)
    MR1L_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
}

// Largest FFT work array of one group of fused repetitions (32 GiB).
constexpr int64_t kRepGroupBytes = int64_t(1) << 35;

struct SfftRun {
  sfft_params P;
  sfft_sampler S;
  cudaStream_t s;
  int K;
  double theta2;
  int rel;
  sfft_stats stats{};
  Staging stage;
  PinnedBuf pin_out;    // device-to-host results (selection flags, counts)
  PinnedBuf cover_pin;  // coverage result of Algorithm 1
  // planted signal on the device (copied, or the caller's device arrays)
  DevBuf<int32_t> freqs_buf;
  DevBuf<cplx> coeffs_buf;
  const int32_t* freqs_ptr = nullptr;
  const cplx* coeffs_ptr = nullptr;
  // Section 5.3 function sampler
  bool bspline = false;
  BsplineDev bs_host;
  DevBuf<BsplineDev> bs_dev;
  // candidate prefix I^(1..t-1) (device rows [np][tp]) and last list I^(t);
  // the host reads the prefix rows back only when it needs them
  DevBuf<int32_t> pre, pre_next, last;
  std::vector<int32_t> pre_h;
  int64_t np = 0;
  int tp = 0;
  // I^(t) of every increment from the 1-D detections (steps 1 and 2a)
  std::vector<std::vector<int32_t>> lines;
  LatticeWork lw;
  std::unique_ptr<FilterCache> filter_cache{FilterCache::enabled() ? new FilterCache : nullptr};
  DevBuf<double> anchors, line_anchors;
  DevBuf<cplx> y, C, bins, work, pvals, coef_out, planted_w;
  DevBuf<uint64_t> keys, keymax;
  DevBuf<SelectState> sel;
  DevBuf<uint8_t> flags, line_sel;
  DevBuf<int64_t> counts;
  DevBuf<cplx> line_y, line_bins;
  std::vector<cudaEvent_t> ev;
  // measurement noise: drawn on a side stream (its arithmetic runs on the FP32
  // pipes) while the main stream runs the sampler's inverse transform on the
  // FP64 pipe, then added to the samples by the reconstruct pass as it loads
  // them
  cudaStream_t side = nullptr;
  cudaEvent_t ev_free = nullptr, ev_noise = nullptr;
  DevBuf<cplx> noise;

  ~SfftRun() {
    for (auto e : ev) cudaEventDestroy(e);
    if (ev_free) cudaEventDestroy(ev_free);
    if (ev_noise) cudaEventDestroy(ev_noise);
    if (side) cudaStreamDestroy(side);
  }

  void sync() {
    MR1L_CUDA(cudaStreamSynchronize(s));
    stage.reset();
  }

  void noise_setup() {
    if (side) return;
    // the noise draws run on the FP32 pipes beside the sampler's FP64
    // transform; a high priority lets their CTAs take the SM slots that the
    // transform's CTAs leave free as soon as they are free
    int lo = 0, hi = 0;
    MR1L_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    MR1L_CUDA(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, hi));
    MR1L_CUDA(cudaEventCreateWithFlags(&ev_free, cudaEventDisableTiming));
    MR1L_CUDA(cudaEventCreateWithFlags(&ev_noise, cudaEventDisableTiming));
  }

  void ev_record() {
    cudaEvent_t e;
    MR1L_CUDA(cudaEventCreate(&e));
    ev.push_back(e);
    MR1L_CUDA(cudaEventRecord(e, s));
  }

  std::vector<double> anchor_rows(uint32_t purpose, int t, int rep0, int count) {
    std::vector<double> a((size_t)count * P.d, 0.0);
    if (P.zero_anchors) return a;
    for (int i = 0; i < count; ++i)
      for (int j = 0; j < P.d; ++j)
        a[(size_t)i * P.d + j] =
            u64_to_unit(philox_u64(P.seed, purpose, (uint32_t)t, (uint32_t)j, 0u, (uint32_t)(rep0 + i)).a);
    return a;
  }

  // Steps 1 and 2a for every increment: I^(t) from r random lines through
  // the t-th coordinate.  They do not depend on the lattice steps, so all d
  // are queued at once (in chunks of increments whose line samples fit
  // kLineChunkBytes, each increment in its own slot so that a user sampler
  // that writes synchronously cannot overwrite lines still being read) and
  // read back with one synchronisation per chunk.
  void detect_all() {
    const int r = P.r, d = P.d;
    constexpr size_t kLineChunkBytes = size_t(256) << 20;
    const size_t per_t = (size_t)r * K * sizeof(cplx);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(d, kLineChunkBytes / per_t));
    line_y.reserve((size_t)chunk * r * K);
    line_bins.reserve((size_t)r * K);
    line_anchors.reserve((size_t)chunk * r * d);
    line_sel.reserve((size_t)d * K);
    uint8_t* hsel = (uint8_t*)pin_out.reserve((size_t)d * K);
    MR1L_CUDA(cudaMemsetAsync(line_sel.get(), 0, (size_t)d * K, s));
    lines.assign(d + 1, {});
    for (int t0 = 1; t0 <= d; t0 += chunk) {
      const int t1 = std::min(d, t0 + chunk - 1);
      for (int t = t0; t <= t1; ++t) {
        const int slot = t - t0;
        cplx* ly = line_y.get() + (size_t)slot * r * K;
        double* la = line_anchors.get() + (size_t)slot * r * d;
        std::vector<double> a = anchor_rows(kAnchorLine, t, 0, r);
        stage.h2d(la, a.data(), a.size() * sizeof(double));
        ev_record();
        if (S.fn) {
          for (int i = 0; i < r; ++i) {
            sfft_request q{};
            q.kind = SFFT_REQ_LINE;
            q.t = t;
            q.rep = i;
            q.d = d;
            q.anchors = a.data() + (size_t)i * d;
            q.K = K;
            int rc = S.fn(S.user, &q, ly + (size_t)i * K, s);
            if (rc != 0) throw Error(MR1L_E_SAMPLER, "sampler callback failed (line request, t = " + std::to_string(t) + ")");
          }
        } else if (bspline) {
          bspline_lines(bs_dev.get(), t, K, la, r, ly, s);
        } else {
          planted_lines(freqs_ptr, coeffs_ptr, S.s, d, t, K, la, r, S.sigma / std::sqrt(2.0), S.noise_seed, 0,
                        line_bins.get(), ly, s);
        }
        ev_record();
        detect_lines(ly, r, P.N, P.s_local, theta2, rel, line_sel.get() + (size_t)(t - 1) * K, s);
      }
      MR1L_CUDA(cudaMemcpyAsync(hsel + (size_t)(t0 - 1) * K, line_sel.get() + (size_t)(t0 - 1) * K,
                                (size_t)(t1 - t0 + 1) * K, cudaMemcpyDeviceToHost, s));
      sync();
      for (int t = t0; t <= t1; ++t)
        for (int a2 = 0; a2 < K; ++a2)
          if (hsel[(size_t)(t - 1) * K + a2]) lines[t].push_back(a2 - P.N);
    }
  }

  // One group of repetitions [rep0, rep0 + nrep): sample, reconstruct, select.
  void passes(const CandSet& J, int t, int rep0, int nrep, int64_t cap) {
    const int64_t n = J.n();
    const int64_t sumM = lw.sumM;
    std::vector<double> a = anchor_rows(kAnchorLattice, t, rep0, nrep);
    anchors.reserve(a.size());
    stage.h2d(anchors.get(), a.data(), a.size() * sizeof(double));
    y.reserve((size_t)nrep * sumM);
    C.reserve((size_t)nrep * sumM);
    work.reserve((size_t)nrep * lw.Luse * lw.geom.P);
    ev_record();
    if (S.fn) {
      std::vector<int64_t> Ml(lw.Mh.begin(), lw.Mh.begin() + lw.Luse);
      for (int i = 0; i < nrep; ++i) {
        sfft_request q{};
        q.kind = SFFT_REQ_LATTICE;
        q.t = t;
        q.rep = rep0 + i;
        q.d = P.d;
        q.anchors = a.data() + (size_t)i * P.d;
        q.L = lw.Luse;
        q.M = Ml.data();
        q.z = lw.zh.data();
        q.sum_M = sumM;
        int rc = S.fn(S.user, &q, y.get() + (size_t)i * sumM, s);
        if (rc != 0)
          throw Error(MR1L_E_SAMPLER, "sampler callback failed (lattice request, t = " + std::to_string(t) + ")");
      }
    } else if (bspline) {
      int maxM = 0;
      for (int l = 0; l < lw.Luse; ++l) maxM = std::max(maxM, lw.Mh[l]);
      bspline_lattice(bs_dev.get(), t, anchors.get(), nrep, lw.dev(), lw.Luse, lw.geom, maxM, y.get(), sumM, s);
    } else {
      const bool noisy = S.sigma > 0;
      if (noisy) {
        // the previous pass has consumed the noise buffer once the main stream
        // reaches this point; draw this pass's noise on the side stream
        noise_setup();
        noise.reserve((size_t)nrep * sumM);
        MR1L_CUDA(cudaEventRecord(ev_free, s));
        MR1L_CUDA(cudaStreamWaitEvent(side, ev_free, 0));
        BlueIO nio{};
        nio.out = noise.get();
        nio.out_stride = sumM;
        nio.noise_scale = S.sigma / std::sqrt(2.0);
        nio.noise_write = 1;
        nio.noise_seed = S.noise_seed;
        nio.noise_t = t;
        nio.noise_rep = rep0;
        nio.noise_rep_per_rhs = 1;
        add_lattice_noise(lw.geom, nio, nrep, side);
        MR1L_CUDA(cudaEventRecord(ev_noise, side));
      }
      bins.reserve((size_t)nrep * sumM);
      MR1L_CUDA(cudaMemsetAsync(bins.get(), 0, (size_t)nrep * sumM * sizeof(cplx), s));
      planted_w.reserve(std::max<int64_t>((int64_t)nrep * S.s, 1));
      planted_lattice_bins(freqs_ptr, coeffs_ptr, S.s, P.d, t, anchors.get(), nrep, lw.dev(), lw.Luse, lw.geom,
                           bins.get(), sumM, planted_w.get(), s);
      BlueIO io{};
      io.in = bins.get();
      io.in_stride = sumM;
      io.out = y.get();
      io.out_stride = sumM;
      io.work = work.get();
      blue_run(lw.geom, io, kModeEval, nrep, s);
      if (noisy) MR1L_CUDA(cudaStreamWaitEvent(s, ev_noise, 0));
    }
    ev_record();
    BlueIO io{};
    io.in = y.get();
    io.in_stride = sumM;
    io.add_in = (!S.fn && !bspline && S.sigma > 0) ? noise.get() : nullptr;
    io.out = C.get();
    io.out_stride = sumM;
    io.work = work.get();
    blue_run(lw.geom, io, kModeRecon, nrep, s);
    pvals.reserve((size_t)nrep * n);
    keys.reserve((size_t)nrep * n);
    keymax.reserve(nrep);
    sel.reserve(nrep);
    MR1L_CUDA(cudaMemsetAsync(keymax.get(), 0, nrep * sizeof(uint64_t), s));
    gather(J, lw.dev(), lw.Luse, lw.umask.get(), lw.geom, C.get(), sumM, nrep, pvals.get(), n, keys.get(),
           keymax.get(), lw.pairs(), s);
    select_topk(keys.get(), n, nrep, keymax.get(), theta2, rel, cap, sel.get(), flags.get(), s);
  }

  // The prefix rows on the host (read back from the device when needed).
  const int32_t* prefix_host() {
    if ((int64_t)pre_h.size() != np * tp) {
      pre_h.resize(np * tp);
      if (np) MR1L_CUDA(cudaMemcpyAsync(pre_h.data(), pre.get(), np * tp * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      sync();
    }
    return pre_h.data();
  }

  void run(sfft_result* res) {
    auto t0 = std::chrono::steady_clock::now();
    const int d = P.d;
    K = 2 * P.N + 1;
    stage.s = s;
    lw.df = P.fft_arith ? 1 : 0;
    lw.stage = &stage;
    lw.cover_host = (int*)cover_pin.reserve(kCoverInts * sizeof(int));
    theta2 = P.theta * P.theta;
    rel = P.theta_mode == SFFT_THETA_REL;
    bspline = !S.fn && S.kind == SFFT_SAMPLER_BSPLINE;
    if (bspline) {
      bspline_tables(S, d, bs_host);
      bs_dev.reserve(1);
      stage.h2d(bs_dev.get(), &bs_host, sizeof(BsplineDev));
    } else if (!S.fn && !S.device_arrays) {
      freqs_buf.reserve(std::max<int64_t>(S.s * d, 1));
      coeffs_buf.reserve(std::max<int64_t>(S.s, 1));
      if (S.s) {
        MR1L_CUDA(cudaMemcpyAsync(freqs_buf.get(), S.freqs, S.s * d * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        MR1L_CUDA(cudaMemcpyAsync(coeffs_buf.get(), S.coeffs, S.s * sizeof(cplx), cudaMemcpyHostToDevice, s));
      }
      freqs_ptr = freqs_buf.get();
      coeffs_ptr = (const cplx*)coeffs_buf.get();
    } else if (!S.fn) {
      freqs_ptr = S.freqs;
      coeffs_ptr = (const cplx*)S.coeffs;
    }
    // steps 1 and 2a for all increments
    detect_all();
    // the component ranges of the 1-D sets bound those of every candidate set
    // (a candidate's j-th component lies in I^(j))
    std::vector<int64_t> range(d + 1, 0);
    for (int t = 1; t <= d; ++t)
      if (!lines[t].empty())
        range[t] = *std::max_element(lines[t].begin(), lines[t].end()) -
                   *std::min_element(lines[t].begin(), lines[t].end());
    const std::vector<int32_t>& I1 = lines[1];
    stats.samples += (int64_t)P.r * K;
    np = (int64_t)I1.size();
    tp = 1;
    pre.reserve(std::max<int64_t>(np, 1));
    stage.h2d(pre.get(), I1.data(), np * sizeof(int32_t));
    pre_h.assign(I1.begin(), I1.end());
    int64_t range_bound = range[1];
    // step 2
    for (int t = 2; t <= d; ++t) {
      const std::vector<int32_t>& It = lines[t];
      sfft_step_stats& st = stats.steps[stats.n_steps++];
      st.t = t;
      st.n_line = (int)It.size();
      st.samples = (int64_t)P.r * K;
      range_bound = std::max(range_bound, range[t]);
      const int rt = t < d ? P.r : 1;
      const int64_t cap = t < d ? P.s_local : P.s;
      const int64_t n = np * (int64_t)It.size();
      st.n_cand = n;
      if (n == 0) {
        np = 0;
        tp = t;
        pre_h.clear();
        stats.samples += st.samples;
        st.covered = 1;
        continue;
      }
      last.reserve(It.size());
      stage.h2d(last.get(), It.data(), It.size() * sizeof(int32_t));
      CandSet J;
      J.tp = tp;
      J.t = t;
      J.np = np;
      J.nq = (int64_t)It.size();
      J.pre = pre.get();
      J.last = last.get();
      // step 2b: Algorithm 1, up to b searches
      int Lmax;
      double lam;
      lmax_lambda(n, 2.0, 0.5, Lmax, lam);
      MR1L_REQUIRE(Lmax >= 1 && Lmax <= 64, "Lmax out of range");
      // primes above the bound on the component ranges are in P^J without a
      // look at the rows; smaller ones are checked on the host rows
      HostRows rows{nullptr, tp, np, It.data(), (int64_t)It.size()};
      if ((int64_t)std::floor(lam) + 1 <= range_bound) rows.pre = prefix_host();
      rows.range_bound = range_bound;
      std::vector<int> primes = prime_set(rows, lam, Lmax);
      const int attempts = search_lattices(lw, J, primes, P.seed, t, P.b, P.redraw != 0, s, &stage);
      const int covered = lw.n_uncovered == 0;
      const int Luse = covered ? lw.Lneed : Lmax;
      lw.tables(Luse, s, filter_cache ? filter_cache.get() : nullptr);
      st.L = Luse;
      st.attempts = attempts;
      st.covered = covered;
      st.sum_M = lw.sumM;
      flags.reserve(n);
      MR1L_CUDA(cudaMemsetAsync(flags.get(), 0, n, s));
      // steps 2c-2e
      if (P.batch_reps) {
        // the repetitions in groups: a launch covers the Luse lattices of each
        // repetition of its group (grid.y = Luse x repetitions <= 65535), and
        // a group's FFT work array stays within kRepGroupBytes (one group for
        // the usual r <= 10)
        const int64_t per_rep = (int64_t)Luse * lw.geom.P * (int64_t)sizeof(cplx);
        const int group = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)rt, 65535 / Luse,
                                                                        kRepGroupBytes / per_rep}));
        for (int i = 0; i < rt; i += group) passes(J, t, i, std::min(group, rt - i), cap);
      } else {
        for (int i = 0; i < rt; ++i) passes(J, t, i, 1, cap);
      }
      st.samples += (int64_t)rt * (1 - Luse + lw.sumM);
      stats.samples += st.samples;
      // compaction: next prefix I^(1..t) on the device (and the coefficients
      // at t = d); only the count comes back
      pre_next.reserve(n * t);
      counts.reserve(cdiv(n, 1024) + 1);
      if (t == d) coef_out.reserve(n);
      int64_t cnt = compact(J, flags.get(), pre_next.get(), t == d ? pvals.get() : nullptr,
                            t == d ? coef_out.get() : nullptr, counts.get(), (int64_t)counts.n,
                            (int64_t*)pin_out.reserve(sizeof(int64_t)), s);
      stage.reset();  // compact() synchronised the stream
      std::swap(pre.p, pre_next.p);
      std::swap(pre.n, pre_next.n);
      std::swap(pre.block, pre_next.block);
      std::swap(pre.device, pre_next.device);
      np = cnt;
      tp = t;
      pre_h.clear();
      st.n_detected = np;
      if (P.t_stop && t == P.t_stop) break;
    }
    std::vector<cplx> coef_h;
    if (tp == d && np) {
      coef_h.resize(np);
      MR1L_CUDA(cudaMemcpyAsync(coef_h.data(), coef_out.get(), np * sizeof(cplx), cudaMemcpyDeviceToHost, s));
    }
    const int32_t* rows_h = prefix_host();
    sync();
    double samp = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      float ms = 0.f;
      MR1L_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
      samp += ms;
    }
    stats.ms_sampling = samp;
    stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const int dout = tp;  // d, or t_stop for a run stopped early
    res->n = np;
    res->d = dout;
    res->freqs = (int32_t*)std::malloc(std::max<int64_t>(np * dout, 1) * sizeof(int32_t));
    res->coeffs = (double*)std::calloc(std::max<int64_t>(np, 1) * 2, sizeof(double));
    if (!res->freqs || !res->coeffs) throw std::bad_alloc();
    if (np) {
      std::memcpy(res->freqs, rows_h, np * dout * sizeof(int32_t));
      if ((int64_t)coef_h.size() == np) std::memcpy(res->coeffs, coef_h.data(), np * sizeof(cplx));
    }
    res->stats = stats;
  }
};

}  // namespace mr1l

static void validate_sfft(const sfft_params* params, const sfft_sampler* sampler) {
  MR1L_REQUIRE(params && sampler, "null argument");
  const sfft_params& P = *params;
  MR1L_REQUIRE(P.d >= 2 && P.d <= SFFT_MAX_STEPS, "d must be in [2, 256]");
  MR1L_REQUIRE(P.N >= 1 && P.N <= 2048, "N must be in [1, 2048]");
  MR1L_REQUIRE(P.s >= 1 && P.s_local >= 1, "s and s_local must be >= 1");
  MR1L_REQUIRE(P.r >= 1 && P.r <= 4096, "r must be in [1, 4096]");
  MR1L_REQUIRE(P.b >= 1, "b must be >= 1");
  MR1L_REQUIRE(P.theta >= 0.0 && std::isfinite(P.theta), "theta must be finite and >= 0");
  MR1L_REQUIRE(P.theta_mode == SFFT_THETA_ABS || P.theta_mode == SFFT_THETA_REL, "bad theta_mode");
  MR1L_REQUIRE(P.t_stop == 0 || (P.t_stop >= 2 && P.t_stop <= P.d), "t_stop must be 0 or in [2, d]");
  MR1L_REQUIRE(P.zero_anchors == 0 || P.zero_anchors == 1, "zero_anchors must be 0 or 1");
  MR1L_REQUIRE(P.redraw == 0 || P.redraw == 1, "redraw must be 0 or 1");
  MR1L_REQUIRE(P.fft_arith == 0 || P.fft_arith == 1, "fft_arith must be 0 (FP64) or 1 (double-float)");
  if (!sampler->fn && sampler->kind == SFFT_SAMPLER_BSPLINE) {
    const sfft_sampler& S = *sampler;
    MR1L_REQUIRE(P.d <= kBsMaxDim, "the B-spline sampler needs d <= 64");
    MR1L_REQUIRE(S.n_groups >= 1 && S.n_groups <= kBsMaxGroups, "n_groups must be in [1, 8]");
    MR1L_REQUIRE(S.group_of && S.orders, "group_of and orders must not be null");
    MR1L_REQUIRE(S.sigma == 0.0, "the B-spline sampler is noiseless (sigma must be 0)");
    for (int i = 0; i < P.d; ++i)
      MR1L_REQUIRE(S.group_of[i] >= -1 && S.group_of[i] < S.n_groups, "group_of entries must be in [-1, n_groups)");
    for (int g = 0; g < S.n_groups; ++g)
      MR1L_REQUIRE(S.orders[g] >= 2 && S.orders[g] <= kBsMaxOrder, "B-spline orders must be in [2, 8]");
  } else if (!sampler->fn) {
    MR1L_REQUIRE(sampler->kind == SFFT_SAMPLER_PLANTED, "unknown sampler kind");
    MR1L_REQUIRE(sampler->s >= 0, "planted s must be >= 0");
    MR1L_REQUIRE(sampler->s == 0 || (sampler->freqs && sampler->coeffs), "planted arrays are null");
    MR1L_REQUIRE(sampler->sigma >= 0.0, "sigma must be >= 0");
    if (!sampler->device_arrays)
      for (int64_t i = 0; i < sampler->s * P.d; ++i)
        MR1L_REQUIRE(sampler->freqs[i] > -32768 && sampler->freqs[i] < 32768, "|h_j| must be < 2^15");
  }
}

static sfft_result* run_one(const sfft_params& P, const sfft_sampler& S, cudaStream_t s) {
  std::unique_ptr<SfftRun> run(new SfftRun());
  run->P = P;
  run->S = S;
  run->s = s;
  std::unique_ptr<sfft_result> res(new sfft_result());
  std::memset(res.get(), 0, sizeof(sfft_result));
  run->run(res.get());
  return res.release();
}

extern "C" int sfft_dimincr(const sfft_params* params, const sfft_sampler* sampler, void* stream, sfft_result** out) {
  return guarded([&] {
    MR1L_REQUIRE(out != nullptr, "null argument");
    *out = nullptr;
    validate_sfft(params, sampler);
    *out = run_one(*params, *sampler, (cudaStream_t)stream);
  });
}

extern "C" int sfft_dimincr_batch(const sfft_params* params, const sfft_sampler* samplers, int count, int concurrency,
                                  sfft_result** out, int* status) {
  return guarded([&] {
    MR1L_REQUIRE(count >= 0 && params && samplers && out && status, "null argument");
    MR1L_REQUIRE(concurrency >= 1 && concurrency <= 256, "concurrency must be in [1, 256]");
    for (int i = 0; i < count; ++i) {
      out[i] = nullptr;
      status[i] = MR1L_OK;
      validate_sfft(params + i, samplers + i);
    }
    int dev = 0;
    MR1L_CUDA(cudaGetDevice(&dev));
    // twiddle tables are built under a lock by whichever worker needs them first
    const int workers = std::min(concurrency, std::max(count, 1));
    std::atomic<int> next{0};
    std::vector<std::string> why(count);  // each failed problem's message (workers' errors are thread-local)
    auto worker = [&]() {
      cudaSetDevice(dev);
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
      for (;;) {
        int i = next.fetch_add(1);
        if (i >= count) break;
        if (!s) {
          status[i] = MR1L_E_CUDA;
          continue;
        }
        status[i] = guarded([&] { out[i] = run_one(params[i], samplers[i], s); });
        if (status[i] != MR1L_OK) why[i] = tl_msg;
      }
      if (s) cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
    for (int i = 0; i < count; ++i)
      if (status[i] != MR1L_OK) throw Error(status[i], "problem " + std::to_string(i) + " failed: " + why[i]);
  });
}

extern "C" int sfft_select(const void* p, int64_t n, int nrhs, const uint8_t* eligible, int64_t cap, double theta,
                           int theta_mode, uint8_t* flags, void* stream) {
  return guarded([&] {
    MR1L_REQUIRE(n >= 0 && nrhs >= 0 && nrhs <= 65535, "need n >= 0 and 0 <= nrhs <= 65535");
    MR1L_REQUIRE(cap >= 0, "cap must be >= 0");
    MR1L_REQUIRE(theta >= 0.0 && std::isfinite(theta), "theta must be finite and >= 0");
    MR1L_REQUIRE(theta_mode == SFFT_THETA_ABS || theta_mode == SFFT_THETA_REL, "bad theta_mode");
    if (n == 0 || nrhs == 0 || cap == 0) return;
    MR1L_REQUIRE(p != nullptr && flags != nullptr, "null array");
    MR1L_REQUIRE(((uintptr_t)p & 15) == 0, "p must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf<uint64_t> keys, keymax;
    DevBuf<SelectState> st;
    keys.reserve((size_t)nrhs * n);
    keymax.reserve(nrhs);
    st.reserve(nrhs);
    value_keys((const cplx*)p, n, nrhs, eligible, keys.get(), keymax.get(), s);
    select_topk(keys.get(), n, nrhs, keymax.get(), theta * theta, theta_mode == SFFT_THETA_REL, cap, st.get(), flags,
                s);
    // the scratch goes back to the block cache, which waits for the device
  });
}

extern "C" int sfft_theorem_params(int d, int64_t supp, double eps, int64_t* r, int* b) {
  return guarded([&] {
    MR1L_REQUIRE(r && b, "null argument");
    MR1L_REQUIRE(d >= 1 && supp >= 1 && eps > 0.0 && eps < 1.0, "need d >= 1, supp >= 1, 0 < eps < 1");
    const double lg = std::log(3.0) + std::log((double)d) - std::log(eps);
    *r = (int64_t)std::ceil(2.0 * (double)supp * (lg + std::log((double)supp)));
    *b = (int)std::ceil(lg / std::log(2.0));
  });
}

extern "C" void sfft_free(sfft_result* res) {
  if (!res) return;
  std::free(res->freqs);
  std::free(res->coeffs);
  delete res;
}

// ---------------------------------------------------------------------------
// Reconstruction without allocation.
//
// Some callers cannot allocate device memory while they run: hosts whose
// device memory is entirely owned by another allocator (a framework's caching
// allocator that has reserved the GPU, a fixed memory budget), and
// latency-critical loops that cannot afford the device-wide synchronisation
// cudaMalloc / cudaFree may cause.  mr1l_reconstruct grows plan-owned scratch
// on demand; this variant instead uses a fixed scratch array compiled into the
// library.  Every GPU that loads the library holds that array (32 MiB) until
// the process exits.
// ---------------------------------------------------------------------------
namespace mr1l {

constexpr int64_t kNoallocScratchElems = int64_t(1) << 21;  // complex128 elements = 32 MiB
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) cplx g_noalloc_scratch[kNoallocScratchElems];

static std::mutex g_noalloc_mu;
static cplx* g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol is only a host-side stand-in, so the address is looked up once
// per device, with that device current.
static cplx* noalloc_scratch() {
  int dev = 0;
  MR1L_CUDA(cudaGetDevice(&dev));
  MR1L_REQUIRE(dev >= 0 && dev < kNoallocMaxDevices, "device index out of range for the fixed scratch");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      throw Error(MR1L_E_CUDA, std::string("cudaGetSymbolAddress(fixed scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = (cplx*)ptr;
  }
  return g_noalloc_addr[dev];
}

}  // namespace mr1l

extern "C" int mr1l_reconstruct_noalloc(mr1l_plan_t* plan, const void* y, int nrhs, void* c, void* stream) {
  return guarded([&] {
    MR1L_REQUIRE(plan != nullptr, "plan is null");
    MR1L_REQUIRE(nrhs >= 0 && nrhs <= 65535 / 64, "nrhs out of range");
    if (nrhs == 0) return;
    MR1L_REQUIRE(y != nullptr && c != nullptr, "null array");
    MR1L_REQUIRE(((uintptr_t)y & 15) == 0 && ((uintptr_t)c & 15) == 0, "arrays must be 16-byte aligned");
    LatticeWork& lw = plan->lw;
    const int64_t sumM = lw.sumM;
    const int64_t need = (int64_t)nrhs * (sumM + (int64_t)lw.Luse * lw.geom.P);
    if (need > kNoallocScratchElems)
      throw Error(MR1L_E_INVAL, "mr1l_reconstruct_noalloc needs " + std::to_string(need) +
                                    " complex scratch elements (nrhs * (sum M + L * P)); the fixed maximum is " +
                                    std::to_string(kNoallocScratchElems));
    cudaStream_t s = (cudaStream_t)stream;
    cplx* scratch = noalloc_scratch();
    // C needs no clearing: every entry the gather reads is written first
    cplx* Cbuf = scratch;
    cplx* work = scratch + (size_t)nrhs * sumM;
    BlueIO io{};
    io.in = (const cplx*)y;
    io.in_stride = sumM;
    io.out = Cbuf;
    io.out_stride = sumM;
    io.work = work;
    io.no_tune = 1;  // tiling trials would synchronise and create events
    blue_run(lw.geom, io, kModeRecon, nrhs, s);
    gather(plan->cand(), lw.dev(), lw.Luse, lw.umask.get(), lw.geom, Cbuf, sumM, nrhs, (cplx*)c, plan->nI,
           nullptr, nullptr, lw.pairs(), s);
  });
}

extern "C" int mr1l_lattice_noise(uint64_t seed, int t, int rep, int L, const int64_t* M, double sigma, void* y,
                                  void* stream) {
  return guarded([&] {
    MR1L_REQUIRE(L >= 1 && L <= 64 && M != nullptr && y != nullptr, "bad arguments");
    MR1L_REQUIRE(((uintptr_t)y & 15) == 0, "y must be 16-byte aligned");
    MR1L_REQUIRE(sigma >= 0.0, "sigma must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> Mh(L);
    std::vector<int64_t> offh(L);
    int64_t sum = 0;
    for (int l = 0; l < L; ++l) {
      MR1L_REQUIRE(M[l] >= 1 && M[l] < (int64_t(1) << 31), "M_l out of range");
      Mh[l] = (int)M[l];
      offh[l] = sum;
      sum += M[l];
    }
    DevBuf<int> Md;
    DevBuf<int64_t> offd;
    Md.reserve(L);
    offd.reserve(L);
    MR1L_CUDA(cudaMemcpyAsync(Md.get(), Mh.data(), L * sizeof(int), cudaMemcpyHostToDevice, s));
    MR1L_CUDA(cudaMemcpyAsync(offd.get(), offh.data(), L * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MR1L_CUDA(cudaMemsetAsync(y, 0, sum * sizeof(cplx), s));
    BlueGeom g{};
    g.L = L;
    g.M = Md.get();
    g.off = offd.get();
    g.sum_M = sum;
    g.P = 2 * (int)*std::max_element(Mh.begin(), Mh.end());
    BlueIO io{};
    io.out = (cplx*)y;
    io.out_stride = sum;
    io.noise_scale = sigma / std::sqrt(2.0);
    io.noise_seed = seed;
    io.noise_t = t;
    io.noise_rep = rep;
    io.noise_rep_per_rhs = 1;
    add_lattice_noise(g, io, 1, s);
    MR1L_CUDA(cudaStreamSynchronize(s));
  });
}

// ---------------------------------------------------------------------------
// Tile tuner control
// ---------------------------------------------------------------------------
extern "C" int mr1l_tune_enable(int on) {
  return guarded([&] { tune_enable(on); });
}

extern "C" int mr1l_tune_reset(void) {
  return guarded([&] { tune_reset(); });
}

extern "C" int mr1l_tune_read(char* buf, size_t len) {
  return guarded([&] {
    const std::string js = tune_json();
    if (!buf || len < js.size() + 1)
      throw Error(MR1L_E_INVAL, "buffer too small for the tile table (" + std::to_string(js.size() + 1) + " bytes)");
    std::memcpy(buf, js.c_str(), js.size() + 1);
  });
}
