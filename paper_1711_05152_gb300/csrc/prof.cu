// Launch counting and optional per-kernel CUDA-event timing (exported as
// mr1l_prof_*).  Events are pooled and reused; timings are read back only by
// mr1l_prof_read, which synchronises the recorded events.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "prof.cuh"

namespace mr1l {

namespace {
struct Rec {
  std::string name;
  cudaEvent_t a, b;
  double flops, bytes;
};
std::mutex g_mu;
bool g_enabled = false;
std::atomic<long long> g_launches{0};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
size_t g_pool_used = 0;
// one open event per stream-name pair (launches are not nested)
std::map<std::pair<cudaStream_t, std::string>, cudaEvent_t> g_open;

cudaEvent_t take_event() {
  if (g_pool_used < g_pool.size()) return g_pool[g_pool_used++];
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  g_pool.push_back(e);
  ++g_pool_used;
  return e;
}
}  // namespace

void prof_begin(const char* name, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_enabled) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = take_event();
  if (!e) return;
  cudaEventRecord(e, s);
  g_open[{s, name}] = e;
}

void prof_end(const char* name, cudaStream_t s, double flops, double bytes) {
  if (!g_enabled) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_open.find({s, name});
  if (it == g_open.end()) return;
  cudaEvent_t e = take_event();
  if (!e) return;
  cudaEventRecord(e, s);
  g_recs.push_back(Rec{name, it->second, e, flops, bytes});
  g_open.erase(it);
}

}  // namespace mr1l

using namespace mr1l;

extern "C" int mr1l_prof_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_enabled = on != 0;
  return MR1L_OK;
}

extern "C" int mr1l_prof_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.clear();
  g_open.clear();
  g_pool_used = 0;
  g_launches.store(0);
  return MR1L_OK;
}

extern "C" long long mr1l_prof_launches(void) { return g_launches.load(); }

extern "C" int mr1l_prof_read(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(g_mu);
  struct Agg {
    long long n = 0;
    double ms = 0, flops = 0, bytes = 0;
  };
  std::map<std::string, Agg> agg;
  for (const Rec& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      set_last_error(MR1L_E_CUDA, "event synchronisation failed");
      return MR1L_E_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    Agg& a = agg[r.name];
    a.n += 1;
    a.ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
  }
  std::string out = "{";
  bool first = true;
  char tmp[512];
  for (auto& kv : agg) {
    snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
             first ? "" : ", ", kv.first.c_str(), kv.second.n, kv.second.ms, kv.second.flops, kv.second.bytes);
    out += tmp;
    first = false;
  }
  out += "}";
  if (!buf || len < out.size() + 1) {
    set_last_error(MR1L_E_INVAL, "buffer too small for the profile (" + std::to_string(out.size() + 1) + " bytes)");
    return MR1L_E_INVAL;
  }
  memcpy(buf, out.c_str(), out.size() + 1);
  return MR1L_OK;
}
