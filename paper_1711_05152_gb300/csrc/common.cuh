// Shared definitions of the mr1l CUDA library: status handling, complex fp64
// helpers, and the library's Philox4x32-10 (Salmon et al., SC'11).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <stdexcept>
#include <string>

#include "../../include/mr1l.h"

namespace mr1l {

// ---------------------------------------------------------------------------
// Status handling: C++ exceptions inside the library, converted to status
// codes at the C boundary.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(int code, const std::string& msg);

#define MR1L_CUDA(call)                                                                 \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::mr1l::Error(e_ == cudaErrorMemoryAllocation ? MR1L_E_NOMEM : MR1L_E_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

#define MR1L_CHECK_LAUNCH(name)                                                           \
  do {                                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess)                                                                \
      throw ::mr1l::Error(MR1L_E_CUDA, std::string(name) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MR1L_REQUIRE(cond, msg)                                      \
  do {                                                               \
    if (!(cond)) throw ::mr1l::Error(MR1L_E_INVAL, std::string(msg)); \
  } while (0)

// ---------------------------------------------------------------------------
// Device memory of plans and workspaces.  Blocks come from a per-device cache
// of released blocks (dev_alloc / dev_free, api.cu): a solve allocates and
// releases dozens of buffers, and cudaMalloc / cudaFree of large blocks cost
// tens to hundreds of microseconds each while the GPU waits.  dev_free
// synchronises the device first, as the cudaFree it replaces does, so a cached
// block is never handed out while queued work may still use it.
// ---------------------------------------------------------------------------
// A block belongs to the device that was current when it was allocated;
// dev_free returns it to that device's cache whatever device is current then.
void* dev_alloc(size_t bytes, size_t* block_bytes, int* device);
void dev_free(void* p, size_t block_bytes, int device);

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  size_t block = 0;  // bytes of the block behind p
  int device = 0;    // device that owns the block
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) dev_free(p, block, device);
    p = nullptr;
    n = 0;
    block = 0;
  }
  // grow-only: keeps the allocation when it is already large enough
  T* reserve(size_t count) {
    if (count <= n && p) return p;
    release();
    size_t bytes = (count ? count : 1) * sizeof(T);
    p = (T*)dev_alloc(bytes, &block, &device);
    n = count;
    return p;
  }
  T* get() const { return p; }
};

// ---------------------------------------------------------------------------
// Complex fp64
// ---------------------------------------------------------------------------
typedef double2 cplx;

__host__ __device__ __forceinline__ cplx cmake(double re, double im) {
  cplx r;
  r.x = re;
  r.y = im;
  return r;
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmake(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmake(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return cmake(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ cplx cmulc(cplx a, cplx b) {
  return cmake(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ cplx cconj(cplx a) { return cmake(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ cplx mul_mi(cplx a) {
  return INV ? cmake(-a.y, a.x) : cmake(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the draw conventions.
//   key = (seed mod 2^32, seed >> 32); counter = (c0, c1, c2, purpose<<24 | t)
//   u64a = x0 | x1 << 32, u64b = x2 | x3 << 32
// ---------------------------------------------------------------------------
enum Purpose : uint32_t {
  kAnchorLine = 1,
  kAnchorLattice = 2,
  kZvec = 3,
  kNoiseLine = 4,
  kNoiseLattice = 5,
};

struct U64Pair {
  uint64_t a, b;
};

__host__ __device__ __forceinline__ void mulhilo32(uint32_t m, uint32_t x, uint32_t& hi, uint32_t& lo) {
  uint64_t p = (uint64_t)m * (uint64_t)x;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

__host__ __device__ __forceinline__ U64Pair philox_u64(uint64_t seed, uint32_t purpose, uint32_t t,
                                                       uint32_t c0, uint32_t c1, uint32_t c2) {
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = (purpose << 24) | (t & 0xFFFFFFu);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, x0, hi0, lo0);
    mulhilo32(0xCD9E8D57u, x2, hi1, lo1);
    uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
    x0 = n0;
    x1 = lo1;
    x2 = n2;
    x3 = lo0;
  }
  U64Pair r;
  r.a = (uint64_t)x0 | ((uint64_t)x1 << 32);
  r.b = (uint64_t)x2 | ((uint64_t)x3 << 32);
  return r;
}

__host__ __device__ __forceinline__ double u64_to_unit(uint64_t u) {
  return (double)(u >> 11) * 0x1.0p-53;
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int ilog2_pow2(int64_t p) {
  int k = 0;
  while ((int64_t(1) << k) < p) ++k;
  return k;
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace mr1l
