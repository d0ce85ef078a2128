// Inference path: full-data target statistics of new rows (Section 2, Eq. 1 with every
// training row seen before the new one) and model prediction over many trees
// (Section 4 "Fast scorer": a row's leaf in a tree is given by its binary features,
// the model value is the sum of the leaves' values over trees).
#include "cbg_internal.cuh"

#include <cmath>

using namespace cbg;

namespace {

constexpr int BLOCK = 256;
constexpr int MAX_DEPTH = 10;

unsigned grid_for(int64_t n, int block = BLOCK) {
  int64_t g = ceil_div(n, block);
  if (g > 65535LL * 16) g = 65535LL * 16;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

// keys = category ids in row order, vals = row ids (the sort keeps rows ascending
// within a category, so every segment lists its rows in row order).
__global__ void table_keys_kernel(const uint32_t* __restrict__ cat, int64_t n, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ rows) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    keys[i] = cat[i];
    rows[i] = static_cast<uint32_t>(i);
  }
}

// Segment heads of the sorted ids, the labels in sorted order (FP64), and the heads as
// uint32 for the scan that numbers the segments.
__global__ void table_heads_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rows,
                                   const float* __restrict__ y, int64_t n, int label_kind,
                                   uint8_t* __restrict__ heads, uint32_t* __restrict__ heads32,
                                   double* __restrict__ lab, unsigned* status) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint8_t hd = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
    heads[i] = hd;
    heads32[i] = hd;
    const float v = y[rows[i]];
    if (!isfinite(v)) atomicOr(status, STATUS_NONFINITE);
    if (label_kind == CBG_LABEL_BINARY && v != 0.0f && v != 1.0f) atomicOr(status, STATUS_BAD_LABEL);
    lab[i] = static_cast<double>(v);
  }
}

// The last element of every segment holds the segment's inclusive (count, sum): it
// becomes table entry (number of heads before it).
__global__ void table_write_kernel(const uint32_t* __restrict__ keys, const uint8_t* __restrict__ heads,
                                   const uint32_t* __restrict__ seg_before, const uint32_t* __restrict__ icnt,
                                   const double* __restrict__ isum, int64_t n, uint32_t* __restrict__ ids,
                                   double* __restrict__ sums, uint32_t* __restrict__ cnts,
                                   int32_t* __restrict__ n_unique) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool tail = i == n - 1 || heads[i + 1];
    if (!tail) continue;
    const uint32_t u = seg_before[i] + heads[i] - 1u;   // segments that start at or before i, minus one
    ids[u] = keys[i];
    sums[u] = isum[i];
    cnts[u] = icnt[i];
    if (i == n - 1) *n_unique = static_cast<int32_t>(u + 1u);
  }
}

__global__ void ts_apply_kernel(const uint32_t* __restrict__ ids, const double* __restrict__ sums,
                                const uint32_t* __restrict__ cnts, const int32_t* __restrict__ n_unique,
                                const uint32_t* __restrict__ cat_new, int64_t m, double prior, double a,
                                float* __restrict__ ts) {
  const int32_t U = *n_unique;
  const double ap = __dmul_rn(a, prior);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t c = cat_new[i];
    int lo = 0, hi = U;   // first index with ids[idx] >= c
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ids[mid] < c) lo = mid + 1; else hi = mid;
    }
    double S = 0.0, N = 0.0;
    if (lo < U && ids[lo] == c) {
      S = sums[lo];
      N = static_cast<double>(cnts[lo]);
    }
    ts[i] = __double2float_rn(__ddiv_rn(__dadd_rn(S, ap), __dadd_rn(N, a)));
  }
}

// float(lr * v) for every leaf of every tree, and the splits packed as (feature, border).
// A level without a split (feature -1, or one outside [0, F)) becomes (0, 255): no bin is
// above 255, so every row takes its 0 side without a test in the hot loop.
__global__ void predict_prep_kernel(const cbg_split* __restrict__ splits, const double* __restrict__ values,
                                    int64_t n_values, int64_t n_splits, int F, double lr, float* __restrict__ inc,
                                    int2* __restrict__ fk) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_values;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    inc[i] = static_cast<float>(lr * values[i]);
    if (i < n_splits) {
      const int f = splits[i].feature;
      fk[i] = (f >= 0 && f < F) ? make_int2(f, splits[i].border) : make_int2(0, 255);
    }
  }
}

// One thread per row, every tree in order. The splits and increments of a chunk of trees
// are staged in shared memory by the whole block; the rows of a block read each split's
// bin column as consecutive bytes (column-major bins). All blocks sweep the trees in the
// same order, so the feature columns the current chunk needs stay in L2. One row per
// thread leaves few warps per SM (10^5 rows: 20), so the tree loop is unrolled by 4 to
// keep 4 x depth independent bin loads of a thread in flight.
constexpr int PRED_THREADS = 256;
constexpr int PRED_SMEM_FLOATS = 8192;   // increments of one chunk: trees x 2^depth

template <int D>
__global__ void __launch_bounds__(PRED_THREADS) predict_kernel(const uint8_t* __restrict__ bins_t, int64_t n,
                                                               int F, const int2* __restrict__ fk,
                                                               const float* __restrict__ inc, int trees,
                                                               float* __restrict__ pred) {
  constexpr int L = 1 << D;
  constexpr int TC = PRED_SMEM_FLOATS / L < 512 ? PRED_SMEM_FLOATS / L : 512;   // trees per chunk
  __shared__ float s_inc[TC * L];
  __shared__ int2 s_fk[TC * D];
  const int64_t r = blockIdx.x * static_cast<int64_t>(PRED_THREADS) + threadIdx.x;
  const bool live = r < n;
  const uint8_t* col = bins_t + (live ? r : 0);
  float acc = live ? pred[r] : 0.f;
  for (int t0 = 0; t0 < trees; t0 += TC) {
    const int tc = min(TC, trees - t0);
    __syncthreads();
    for (int i = threadIdx.x; i < tc * L; i += PRED_THREADS) s_inc[i] = inc[static_cast<int64_t>(t0) * L + i];
    for (int i = threadIdx.x; i < tc * D; i += PRED_THREADS) s_fk[i] = fk[static_cast<int64_t>(t0) * D + i];
    __syncthreads();
    if (!live) continue;
#pragma unroll 4
    for (int t = 0; t < tc; ++t) {
      int leaf = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int2 s = s_fk[t * D + d];
        if (__ldg(col + static_cast<int64_t>(s.x) * n) > s.y) leaf |= 1 << d;
      }
      acc += s_inc[t * L + leaf];
    }
  }
  if (live) pred[r] = acc;
}

template <int D>
cbg_status launch_predict(cbg_ctx* ctx, const cbg_predict_args* a, const int2* fk, const float* inc) {
  const unsigned grid = static_cast<unsigned>(ceil_div(a->n, PRED_THREADS));
  predict_kernel<D><<<grid, PRED_THREADS, 0, ctx->stream>>>(a->bins_t, a->n, a->F, fk, inc, a->trees, a->pred);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

}  // namespace

extern "C" {

cbg_status cbg_ts_table(cbg_ctx* ctx, const uint32_t* cat, const float* y, int64_t n, int label_kind,
                        uint32_t* ids, double* sums, uint32_t* cnts, int32_t* n_unique) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, label_kind == CBG_LABEL_BINARY || label_kind == CBG_LABEL_REAL, "bad label_kind");
  CBG_REQUIRE(ctx, cat && y && ids && sums && cnts && n_unique, "NULL argument");
  DeviceGuard guard(ctx->device);
  const size_t need = 5 * (n * sizeof(uint32_t) + 256) + (n + 256) + 2 * (n * sizeof(double) + 256) +
                      (n * sizeof(uint32_t) + 256) + radix_temp_bytes(n) + segscan_temp_bytes(n) +
                      scan_u32_temp_bytes(n) + 1024;
  cbg_status st = ws_reserve(ctx, need);
  if (st != CBG_OK) return st;
  Carve cv(ctx->ws);
  uint32_t* ka = cv.take<uint32_t>(n);
  uint32_t* kb = cv.take<uint32_t>(n);
  uint32_t* va = cv.take<uint32_t>(n);
  uint32_t* vb = cv.take<uint32_t>(n);
  uint32_t* heads32 = cv.take<uint32_t>(n);
  uint8_t* heads = cv.take<uint8_t>(n);
  double* lab = cv.take<double>(n);
  double* isum = cv.take<double>(n);
  uint32_t* icnt = cv.take<uint32_t>(n);
  void* rtmp = cv.take<char>(radix_temp_bytes(n));
  void* stmp = cv.take<char>(segscan_temp_bytes(n));
  void* qtmp = cv.take<char>(scan_u32_temp_bytes(n));
  table_keys_kernel<<<grid_for(n), BLOCK, 0, ctx->stream>>>(cat, n, ka, va);
  CBG_CHECK_LAUNCH(ctx);
  st = radix_sort_u32(ctx, ka, kb, va, vb, n, 32, rtmp);
  if (st != CBG_OK) return st;
  table_heads_kernel<<<grid_for(n), BLOCK, 0, ctx->stream>>>(ka, va, y, n, label_kind, heads, heads32, lab,
                                                             ctx->d_status);
  CBG_CHECK_LAUNCH(ctx);
  st = segscan_cnt_sum(ctx, heads, lab, n, icnt, isum, stmp);
  if (st != CBG_OK) return st;
  st = scan_u32_exclusive(ctx, heads32, kb, n, qtmp);   // kb: heads before each position
  if (st != CBG_OK) return st;
  table_write_kernel<<<grid_for(n), BLOCK, 0, ctx->stream>>>(ka, heads, kb, icnt, isum, n, ids, sums, cnts,
                                                             n_unique);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

cbg_status cbg_ts_apply(cbg_ctx* ctx, const uint32_t* ids, const double* sums, const uint32_t* cnts,
                        const int32_t* n_unique, const uint32_t* cat_new, int64_t m, double prior, double a,
                        float* ts) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, m >= 0 && m <= INT32_MAX, "m must be in [0, 2^31-1]");
  CBG_REQUIRE(ctx, a > 0.0 && std::isfinite(a), "the prior weight a must be > 0 (Eq. 1)");
  CBG_REQUIRE(ctx, std::isfinite(prior), "the prior must be finite");
  if (m == 0) return CBG_OK;
  CBG_REQUIRE(ctx, ids && sums && cnts && n_unique && cat_new && ts, "NULL argument");
  DeviceGuard guard(ctx->device);
  ts_apply_kernel<<<grid_for(m), BLOCK, 0, ctx->stream>>>(ids, sums, cnts, n_unique, cat_new, m, prior, a, ts);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

cbg_status cbg_predict(cbg_ctx* ctx, const cbg_predict_args* a) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, a != nullptr, "args is NULL");
  CBG_REQUIRE(ctx, a->n >= 0 && a->n <= INT32_MAX, "n must be in [0, 2^31-1]");
  CBG_REQUIRE(ctx, a->F >= 1, "F must be >= 1");
  CBG_REQUIRE(ctx, a->depth >= 1 && a->depth <= MAX_DEPTH, "depth must be in [1, 10]");
  CBG_REQUIRE(ctx, a->trees >= 0, "trees must be >= 0");
  if (a->n == 0 || a->trees == 0) return CBG_OK;
  CBG_REQUIRE(ctx, a->bins_t && a->splits && a->leaf_values && a->pred, "NULL argument");
  DeviceGuard guard(ctx->device);
  const int64_t n_values = static_cast<int64_t>(a->trees) << a->depth;
  const int64_t n_splits = static_cast<int64_t>(a->trees) * a->depth;
  const size_t need = n_values * sizeof(float) + 256 + n_splits * sizeof(int2) + 256;
  cbg_status st = ws_reserve(ctx, need);
  if (st != CBG_OK) return st;
  Carve cv(ctx->ws);
  float* inc = cv.take<float>(n_values);
  int2* fk = cv.take<int2>(n_splits);
  predict_prep_kernel<<<grid_for(n_values), BLOCK, 0, ctx->stream>>>(a->splits, a->leaf_values, n_values, n_splits,
                                                                     a->F, a->lr, inc, fk);
  CBG_CHECK_LAUNCH(ctx);
  switch (a->depth) {
    case 1: return launch_predict<1>(ctx, a, fk, inc);
    case 2: return launch_predict<2>(ctx, a, fk, inc);
    case 3: return launch_predict<3>(ctx, a, fk, inc);
    case 4: return launch_predict<4>(ctx, a, fk, inc);
    case 5: return launch_predict<5>(ctx, a, fk, inc);
    case 6: return launch_predict<6>(ctx, a, fk, inc);
    case 7: return launch_predict<7>(ctx, a, fk, inc);
    case 8: return launch_predict<8>(ctx, a, fk, inc);
    case 9: return launch_predict<9>(ctx, a, fk, inc);
    default: return launch_predict<10>(ctx, a, fk, inc);
  }
}

}  // extern "C"
