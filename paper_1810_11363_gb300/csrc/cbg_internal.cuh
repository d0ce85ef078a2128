// Internal declarations shared by the translation units of libcbg.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "cbg.h"

struct cbg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  void* ws = nullptr;          // library scratch for one-off steps
  size_t ws_bytes = 0;
  bool ws_fixed = false;       // preallocated by the caller's request: never grown
  unsigned int* d_status = nullptr;  // asynchronous data/timeout flags (device word)
  std::string err;
  // histogram launch timing (cbg_profile_*)
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;                // events handed out since the last read (pairs)
  double prof_ms = 0.0;
  int64_t prof_launches = 0;
  cudaStream_t capture_stream = nullptr;   // non-blocking stream used to capture graphs
  std::vector<cudaStream_t> branch_streams;  // branches of a captured batched round
  std::vector<cudaEvent_t> branch_events;
  void* noalloc_scratch = nullptr;   // device address of cbg_histogram_noalloc's array (looked up once)
  bool test_force_wait_timeout = false;   // cbg_test_force_wait_timeout: bounded waits run out
};

namespace cbg {

// Bits of the device status word.
constexpr unsigned STATUS_NONFINITE = 1u;
constexpr unsigned STATUS_BAD_LABEL = 2u;
constexpr unsigned STATUS_TIMEOUT = 4u;
constexpr unsigned STATUS_BAD_BIN = 8u;     // a bin that does not fit a packed layout (4-bit or 1-bit)

cbg_status fail(cbg_ctx* ctx, cbg_status code, const char* fmt, ...);

#define CBG_CUDA(ctx, call)                                                        \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ::cbg::fail((ctx), CBG_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CBG_CHECK_LAUNCH(ctx) CBG_CUDA(ctx, cudaGetLastError())

#define CBG_REQUIRE(ctx, cond, ...)                       \
  do {                                                    \
    if (!(cond)) return ::cbg::fail((ctx), CBG_EINVAL, __VA_ARGS__); \
  } while (0)

// Makes ctx->device current for the scope of a call and restores the previous one.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Bump allocator over a caller- or library-owned buffer.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* p) : base(static_cast<char*>(p)) {}
  template <typename T>
  T* take(size_t count, size_t align = 256) {
    off = (off + align - 1) / align * align;
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

// Event pair around a profiled launch (no-op unless profiling is enabled).
cbg_status prof_begin(cbg_ctx* ctx, cudaEvent_t* a, cudaEvent_t* b);
cbg_status prof_end(cbg_ctx* ctx, cudaEvent_t b);

// Make sure the library workspace holds `bytes`; grows it when allowed.
cbg_status ws_reserve(cbg_ctx* ctx, size_t bytes);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- primitives
// Exclusive prefix sum of uint32 values (wrapping), out may alias nothing.
size_t scan_u32_temp_bytes(int64_t n);
cbg_status scan_u32_exclusive(cbg_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, void* temp);

// Stable LSD radix sort, 8-bit digits over key bits [0, key_bits).
// Keys are 32 or 64 bits; values optional (uint32). Results end in keys_a/vals_a.
size_t radix_temp_bytes(int64_t n);
cbg_status radix_sort_u32(cbg_ctx* ctx, uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a,
                          uint32_t* vals_b, int64_t n, int key_bits, void* temp);
cbg_status radix_sort_u64(cbg_ctx* ctx, uint64_t* keys_a, uint64_t* keys_b, uint32_t* vals_a,
                          uint32_t* vals_b, int64_t n, int key_bits, void* temp);

// Segmented inclusive scan of (count, sum) pairs: heads[i] != 0 starts a segment.
// out_cnt[i] = number of elements in [seg_start, i], out_sum[i] = FP64 sum of vals.
size_t segscan_temp_bytes(int64_t n);
cbg_status segscan_cnt_sum(cbg_ctx* ctx, const uint8_t* heads, const double* vals, int64_t n,
                           uint32_t* out_cnt, double* out_sum, void* temp);

}  // namespace cbg

// ------------------------------------------------------------ device helpers
namespace cbgd {

__device__ __forceinline__ float load_gh(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_gh(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}
// The stored bits of element i, and their value: a load whose value is needed only later
// keeps the raw bits, so that no conversion right after the load waits for it.
__device__ __forceinline__ uint32_t load_gh_bits(const float* p, int64_t i) { return __float_as_uint(__ldg(p + i)); }
__device__ __forceinline__ uint32_t load_gh_bits(const __nv_bfloat16* p, int64_t i) {
  return __ldg(reinterpret_cast<const unsigned short*>(p) + i);
}
template <typename GH>
__device__ __forceinline__ float gh_from_bits(uint32_t b) {
  return __uint_as_float(sizeof(GH) == 2 ? b << 16 : b);   // a BF16 is the high half of an FP32
}
__device__ __forceinline__ void store_gh(float* p, int64_t i, float v) { p[i] = v; }
__device__ __forceinline__ void store_gh(__nv_bfloat16* p, int64_t i, float v) {
  p[i] = __float2bfloat16_rn(v);
}

// SplitMix64 (Steele, Lea & Flood 2014): output i of the generator seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// First and second derivative of the loss in the model value a (FP32): RMSE a - y and 1;
// Logloss sigmoid(a) - y and sigmoid(a) (1 - sigmoid(a)).
__device__ __forceinline__ void loss_grad(int loss, float a, float y, float* g, float* h) {
  if (loss == CBG_LOSS_RMSE) {
    *g = a - y;
    *h = 1.0f;
  } else {
    const float s = 1.0f / (1.0f + expf(-a));
    *g = s - y;
    *h = s * (1.0f - s);
  }
}

// Orderable 32-bit image of a finite float (ascending float order = ascending uint order),
// with -0.0 mapped to +0.0.
__device__ __forceinline__ uint32_t float_order_bits(float x) {
  if (x == 0.0f) x = 0.0f;
  uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_from_order_bits(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(u);
}

}  // namespace cbgd
