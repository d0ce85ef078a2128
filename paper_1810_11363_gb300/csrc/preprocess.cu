// One-off steps of the path: permutation, prior, ordered target statistics (Section 2,
// Eq. 1), quantile borders and uint8 quantisation (Section 5, "Dense numerical
// features").
#include "cbg_internal.cuh"

#include <algorithm>
#include <cmath>

using namespace cbg;

namespace {

constexpr int BLOCK = 256;

__global__ void perm_keys_kernel(uint64_t seed, int64_t n, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    keys[i] = cbgd::splitmix64_at(seed, static_cast<uint64_t>(i));
    vals[i] = static_cast<uint32_t>(i);
  }
}

// ------------------------------------------------------------------ prior
// Per-block partial: count of positive labels (binary) or FP64 label sum (real).
__global__ void prior_partial_kernel(const float* __restrict__ y, int64_t n, int label_kind,
                                     double* __restrict__ partial, unsigned int* __restrict__ status) {
  __shared__ double sh[BLOCK];
  double s = 0.0;
  bool bad = false;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(BLOCK) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * BLOCK) {
    float v = y[i];
    if (label_kind == CBG_LABEL_BINARY) {
      bad |= !(v == 0.0f || v == 1.0f);
      s += (v == 1.0f) ? 1.0 : 0.0;
    } else {
      s += static_cast<double>(v);
    }
  }
  if (bad) atomicOr(status, STATUS_BAD_LABEL);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = BLOCK / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void prior_final_kernel(const double* __restrict__ partial, int nparts, int64_t n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += partial[i];
    *out = __ddiv_rn(s, static_cast<double>(n));
  }
}

// ------------------------------------------------------------ ordered TS
// Several columns at once: element i = c n + p holds column c at permutation position p,
// keyed (c << 32) | id. A stable sort by key keeps positions in order within every
// (column, category) group, so a segmented scan over the sorted elements gives, for every
// element, the count and label sum of the earlier positions of its group.
__global__ void ts_gather_kernel(const uint32_t* __restrict__ cat, const uint32_t* __restrict__ perm, int64_t n,
                                 int64_t total, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t c = i / n, p = i - c * n;
    const uint32_t r = perm[p];
    keys[i] = (static_cast<uint64_t>(c) << 32) | (r < n ? cat[c * n + r] : 0u);
    vals[i] = static_cast<uint32_t>(p);
  }
}

// Sorted by (column, category, position): mark group heads and fetch each element's label.
__global__ void ts_heads_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                const uint32_t* __restrict__ perm, const float* __restrict__ y, int64_t n,
                                int64_t total, int label_kind, uint8_t* __restrict__ heads, double* __restrict__ lab,
                                unsigned int* __restrict__ status) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    heads[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
    const uint32_t r = perm[vals[i]];
    float v = r < n ? y[r] : 0.0f;
    if (label_kind == CBG_LABEL_BINARY && !(v == 0.0f || v == 1.0f)) atomicOr(status, STATUS_BAD_LABEL);
    lab[i] = static_cast<double>(v);
  }
}

// Eq. 1: (S + a*P) / (N + a), FP64 without contraction, rounded to float, scattered to
// rows of the element's column.
__global__ void ts_final_kernel(const uint64_t* __restrict__ keys, const uint8_t* __restrict__ heads,
                                const uint32_t* __restrict__ incl_cnt, const double* __restrict__ incl_sum,
                                const uint32_t* __restrict__ vals, const uint32_t* __restrict__ perm, int64_t n,
                                int64_t total, double prior, double a, int label_kind, float* __restrict__ ts,
                                uint32_t* __restrict__ cnt_before, void* __restrict__ sum_before) {
  const double aP = __dmul_rn(a, prior);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint32_t N = incl_cnt[i] - 1u;
    double S = heads[i] ? 0.0 : incl_sum[i - 1];
    double num = __dadd_rn(S, aP);
    double den = __dadd_rn(static_cast<double>(N), a);
    uint32_t row = perm[vals[i]];
    if (row >= n) continue;
    const int64_t at = static_cast<int64_t>(keys[i] >> 32) * n + row;
    ts[at] = __double2float_rn(__ddiv_rn(num, den));
    if (cnt_before) cnt_before[at] = N;
    if (sum_before) {
      if (label_kind == CBG_LABEL_BINARY)
        static_cast<uint32_t*>(sum_before)[at] = static_cast<uint32_t>(S);
      else
        static_cast<double*>(sum_before)[at] = S;
    }
  }
}

__global__ void border_keys_kernel(const float* __restrict__ x, int64_t n, int64_t total,
                                   uint64_t* __restrict__ keys, unsigned int* __restrict__ status) {
  bool bad = false;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float v = x[i];
    if (!isfinite(v)) {
      bad = true;
      v = 0.0f;
    }
    uint64_t f = static_cast<uint64_t>(i / n);
    keys[i] = (f << 32) | cbgd::float_order_bits(v);
  }
  if (bad) atomicOr(status, STATUS_NONFINITE);
}

// One block per feature: pick v[floor(k*n/(B+1))], keep strictly increasing values below max.
__global__ void border_pick_kernel(const uint64_t* __restrict__ sorted, int64_t n, int max_borders,
                                   float* __restrict__ borders, int32_t* __restrict__ n_borders) {
  __shared__ float cand[256];
  __shared__ int keep_pos[256];
  const int f = blockIdx.x, k = threadIdx.x + 1;   // candidate index 1..B
  const uint64_t* s = sorted + static_cast<int64_t>(f) * n;
  const float vmax = cbgd::float_from_order_bits(static_cast<uint32_t>(s[n - 1]));
  float c = INFINITY;
  if (k <= max_borders) {
    int64_t idx = (static_cast<int64_t>(k) * n) / (max_borders + 1);
    c = cbgd::float_from_order_bits(static_cast<uint32_t>(s[idx]));
  }
  cand[threadIdx.x] = c;
  __syncthreads();
  int keep = 0;
  if (k <= max_borders) keep = (c < vmax) && (k == 1 || c > cand[threadIdx.x - 1]);
  // exclusive scan of keep flags (256 threads)
  keep_pos[threadIdx.x] = keep;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    int v = threadIdx.x >= o ? keep_pos[threadIdx.x - o] : 0;
    __syncthreads();
    keep_pos[threadIdx.x] += v;
    __syncthreads();
  }
  int incl = keep_pos[threadIdx.x];
  int total = keep_pos[255];
  float* b = borders + static_cast<int64_t>(f) * max_borders;
  if (keep) b[incl - 1] = c;
  __syncthreads();
  for (int i = total + threadIdx.x; i < max_borders; i += blockDim.x) b[i] = INFINITY;
  if (threadIdx.x == 0) n_borders[f] = total;
}

// ---------------------------------------------------------------- quantise
constexpr int Q_FEAT = 32;
constexpr int Q_ROWS = 64;

// Block: features [f0, f0+32) x rows [r0, r0+64). bin = #{borders < x} by binary search.
// Bins go to the grouped layout ((f/32)*n + r)*32 + f%32 and optionally to bins_t[f][r].
__global__ void quantize_kernel(const float* __restrict__ x, int64_t n, int F, const float* __restrict__ borders,
                                const int32_t* __restrict__ n_borders, int max_borders, uint8_t* __restrict__ bins,
                                int f_offset, uint8_t* __restrict__ bins_t, unsigned int* __restrict__ status) {
  extern __shared__ float qsh[];                 // [32][max_borders] borders
  __shared__ uint8_t tile[Q_ROWS][Q_FEAT];
  __shared__ int nb[Q_FEAT];
  const int f0 = blockIdx.y * Q_FEAT;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * Q_ROWS;
  const int nf = min(Q_FEAT, F - f0);
  for (int i = threadIdx.x; i < nf * max_borders; i += blockDim.x)
    qsh[i] = borders[static_cast<int64_t>(f0) * max_borders + i];
  if (threadIdx.x < Q_FEAT) nb[threadIdx.x] = threadIdx.x < nf ? min(n_borders[f0 + threadIdx.x], max_borders) : 0;
  __syncthreads();
  const int r = threadIdx.x & (Q_ROWS - 1);
  const int fq = threadIdx.x / Q_ROWS;           // 0..3
  bool bad = false;
  for (int j = 0; j < Q_FEAT / 4; ++j) {
    int fl = fq * (Q_FEAT / 4) + j;
    uint8_t bin = 0;
    if (fl < nf && r0 + r < n) {
      float v = x[static_cast<int64_t>(f0 + fl) * n + r0 + r];
      bad |= !isfinite(v);
      const float* b = qsh + fl * max_borders;
      int lo = 0, hi = nb[fl];
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (b[mid] < v) lo = mid + 1; else hi = mid;
      }
      bin = static_cast<uint8_t>(lo);
    }
    tile[r][fl] = bin;
  }
  if (bad) atomicOr(status, STATUS_NONFINITE);
  __syncthreads();
  for (int i = threadIdx.x; i < Q_ROWS * Q_FEAT; i += blockDim.x) {
    int rr = i / Q_FEAT, fl = i % Q_FEAT;
    int64_t row = r0 + rr;
    if (fl < nf && row < n) {
      int fg = f_offset + f0 + fl;
      bins[((static_cast<int64_t>(fg >> 5)) * n + row) * 32 + (fg & 31)] = tile[rr][fl];
    }
  }
  if (bins_t) {
    for (int i = threadIdx.x; i < Q_ROWS * Q_FEAT; i += blockDim.x) {
      int fl = i / Q_ROWS, rr = i % Q_ROWS;
      int64_t row = r0 + rr;
      if (fl < nf && row < n) bins_t[static_cast<int64_t>(f_offset + f0 + fl) * n + row] = tile[rr][fl];
    }
  }
}

unsigned grid_for(int64_t n, int block = BLOCK) {
  int64_t g = ceil_div(n, block);
  if (g > 65535LL * 16) g = 65535LL * 16;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

}  // namespace

extern "C" {

cbg_status cbg_make_permutation(cbg_ctx* ctx, uint64_t seed, int64_t n, uint32_t* perm) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1], got %lld", (long long)n);
  CBG_REQUIRE(ctx, perm != nullptr, "perm is NULL");
  DeviceGuard guard(ctx->device);
  size_t need = 2 * (n * sizeof(uint64_t) + 256) + (n * sizeof(uint32_t) + 256) + radix_temp_bytes(n) + 256;
  cbg_status st = ws_reserve(ctx, need);
  if (st != CBG_OK) return st;
  Carve cv(ctx->ws);
  uint64_t* ka = cv.take<uint64_t>(n);
  uint64_t* kb = cv.take<uint64_t>(n);
  uint32_t* vb = cv.take<uint32_t>(n);
  void* tmp = cv.take<char>(radix_temp_bytes(n));
  perm_keys_kernel<<<grid_for(n), BLOCK, 0, ctx->stream>>>(seed, n, ka, perm);
  CBG_CHECK_LAUNCH(ctx);
  return radix_sort_u64(ctx, ka, kb, perm, vb, n, 64, tmp);
}

cbg_status cbg_prior(cbg_ctx* ctx, const float* y, int64_t n, int label_kind, double* prior_out) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, y && prior_out, "NULL argument");
  CBG_REQUIRE(ctx, label_kind == CBG_LABEL_BINARY || label_kind == CBG_LABEL_REAL, "bad label_kind");
  DeviceGuard guard(ctx->device);
  const int parts = 1024;
  cbg_status st = ws_reserve(ctx, parts * sizeof(double));
  if (st != CBG_OK) return st;
  double* partial = static_cast<double*>(ctx->ws);
  prior_partial_kernel<<<parts, BLOCK, 0, ctx->stream>>>(y, n, label_kind, partial, ctx->d_status);
  CBG_CHECK_LAUNCH(ctx);
  prior_final_kernel<<<1, 32, 0, ctx->stream>>>(partial, parts, n, prior_out);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

cbg_status cbg_ordered_ts(cbg_ctx* ctx, const uint32_t* cat, const float* y, int64_t n, int32_t C,
                          const uint32_t* perm, double prior, double a, int label_kind, float* ts,
                          uint32_t* cnt_before, void* sum_before) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, C >= 0, "C must be >= 0");
  CBG_REQUIRE(ctx, a > 0.0 && std::isfinite(a), "the prior weight a must be > 0 (Eq. 1)");
  CBG_REQUIRE(ctx, std::isfinite(prior), "the prior must be finite");
  CBG_REQUIRE(ctx, label_kind == CBG_LABEL_BINARY || label_kind == CBG_LABEL_REAL, "bad label_kind");
  if (C == 0) return CBG_OK;
  CBG_REQUIRE(ctx, cat && y && perm && ts, "NULL argument");
  DeviceGuard guard(ctx->device);
  // columns in chunks of at most 2^26 elements, each chunk sorted once by (column, id)
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(C, (int64_t(1) << 26) / n));
  const int64_t cap = chunk * n;
  int cbits = 0;
  while ((int64_t(1) << cbits) < chunk) ++cbits;
  size_t need = 2 * (cap * sizeof(uint64_t) + 256) + 2 * (cap * sizeof(uint32_t) + 256) + (cap + 256) +
                2 * (cap * sizeof(double) + 256) + (cap * sizeof(uint32_t) + 256) + radix_temp_bytes(cap) +
                segscan_temp_bytes(cap) + 512;
  cbg_status st = ws_reserve(ctx, need);
  if (st != CBG_OK) return st;
  Carve cv(ctx->ws);
  uint64_t* ka = cv.take<uint64_t>(cap);
  uint64_t* kb = cv.take<uint64_t>(cap);
  uint32_t* va = cv.take<uint32_t>(cap);
  uint32_t* vb = cv.take<uint32_t>(cap);
  uint8_t* heads = cv.take<uint8_t>(cap);
  double* lab = cv.take<double>(cap);
  double* isum = cv.take<double>(cap);
  uint32_t* icnt = cv.take<uint32_t>(cap);
  void* rtmp = cv.take<char>(radix_temp_bytes(cap));
  void* stmp = cv.take<char>(segscan_temp_bytes(cap));
  for (int64_t c0 = 0; c0 < C; c0 += chunk) {
    const int64_t cc = std::min<int64_t>(chunk, C - c0);
    const int64_t total = cc * n, off = c0 * n;
    ts_gather_kernel<<<grid_for(total), BLOCK, 0, ctx->stream>>>(cat + off, perm, n, total, ka, va);
    CBG_CHECK_LAUNCH(ctx);
    st = radix_sort_u64(ctx, ka, kb, va, vb, total, 32 + cbits, rtmp);
    if (st != CBG_OK) return st;
    ts_heads_kernel<<<grid_for(total), BLOCK, 0, ctx->stream>>>(ka, va, perm, y, n, total, label_kind, heads, lab,
                                                               ctx->d_status);
    CBG_CHECK_LAUNCH(ctx);
    st = segscan_cnt_sum(ctx, heads, lab, total, icnt, isum, stmp);
    if (st != CBG_OK) return st;
    void* sb = nullptr;
    if (sum_before)
      sb = label_kind == CBG_LABEL_BINARY ? static_cast<void*>(static_cast<uint32_t*>(sum_before) + off)
                                          : static_cast<void*>(static_cast<double*>(sum_before) + off);
    ts_final_kernel<<<grid_for(total), BLOCK, 0, ctx->stream>>>(ka, heads, icnt, isum, va, perm, n, total, prior, a,
                                                               label_kind, ts + off,
                                                               cnt_before ? cnt_before + off : nullptr, sb);
    CBG_CHECK_LAUNCH(ctx);
  }
  return CBG_OK;
}

cbg_status cbg_select_borders(cbg_ctx* ctx, const float* x, int64_t n, int32_t F, int32_t max_borders,
                              float* borders, int32_t* n_borders) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, F >= 1 && F <= 65535, "F must be in [1, 65535]");
  CBG_REQUIRE(ctx, max_borders >= 1 && max_borders <= 254, "max_borders must be in [1, 254]");
  CBG_REQUIRE(ctx, x && borders && n_borders, "NULL argument");
  DeviceGuard guard(ctx->device);
  const int64_t total = n * static_cast<int64_t>(F);
  int fbits = 0;
  while ((1LL << fbits) < F) ++fbits;
  size_t need = 2 * (total * sizeof(uint64_t) + 256) + radix_temp_bytes(total) + 256;
  cbg_status st = ws_reserve(ctx, need);
  if (st != CBG_OK) return st;
  Carve cv(ctx->ws);
  uint64_t* ka = cv.take<uint64_t>(total);
  uint64_t* kb = cv.take<uint64_t>(total);
  void* tmp = cv.take<char>(radix_temp_bytes(total));
  border_keys_kernel<<<grid_for(total), BLOCK, 0, ctx->stream>>>(x, n, total, ka, ctx->d_status);
  CBG_CHECK_LAUNCH(ctx);
  st = radix_sort_u64(ctx, ka, kb, nullptr, nullptr, total, 32 + fbits, tmp);
  if (st != CBG_OK) return st;
  border_pick_kernel<<<F, 256, 0, ctx->stream>>>(ka, n, max_borders, borders, n_borders);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

cbg_status cbg_quantize(cbg_ctx* ctx, const float* x, int64_t n, int32_t F, const float* borders,
                        const int32_t* n_borders, int32_t max_borders, uint8_t* bins, int32_t F_pad,
                        int32_t f_offset, uint8_t* bins_t) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, F >= 1, "F must be >= 1");
  CBG_REQUIRE(ctx, max_borders >= 1 && max_borders <= 254, "max_borders must be in [1, 254]");
  CBG_REQUIRE(ctx, F_pad >= 32 && F_pad % 32 == 0, "F_pad must be a positive multiple of 32");
  CBG_REQUIRE(ctx, f_offset >= 0 && f_offset + F <= F_pad, "columns [f_offset, f_offset+F) exceed F_pad");
  CBG_REQUIRE(ctx, x && borders && n_borders && bins, "NULL argument");
  DeviceGuard guard(ctx->device);
  dim3 grid(static_cast<unsigned>(ceil_div(n, Q_ROWS)), static_cast<unsigned>(ceil_div(F, Q_FEAT)));
  CBG_REQUIRE(ctx, grid.y <= 65535, "too many features");
  size_t smem = static_cast<size_t>(Q_FEAT) * max_borders * sizeof(float);
  CBG_CUDA(ctx, cudaFuncSetAttribute(quantize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  quantize_kernel<<<grid, BLOCK, smem, ctx->stream>>>(x, n, F, borders, n_borders, max_borders, bins, f_offset,
                                                     bins_t, ctx->d_status);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

}  // extern "C"
