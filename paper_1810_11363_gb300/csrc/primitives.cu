// Scan, segmented scan and stable LSD radix sort used by the one-off steps of the path
// (permutation, ordered target statistics, border selection). Written for this
// library: 3-phase (reduce, scan of tile aggregates, down-sweep) so no kernel waits
// on another block.
#include "cbg_internal.cuh"

namespace cbg {
namespace {

constexpr int BLOCK = 256;
constexpr int ITEMS = 8;
constexpr int TILE = BLOCK * ITEMS;   // 2048 elements per tile

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// --------------------------------------------------------------- u32 scan
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* sh, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < BLOCK / 32 ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < BLOCK / 32) sh[lane] = w;
  }
  __syncthreads();
  uint32_t before = (warp > 0 ? sh[warp - 1] : 0u) + x - v;
  *total = sh[BLOCK / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t sh[BLOCK / 32];
  int64_t base = static_cast<int64_t>(blockIdx.x) * TILE;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    int64_t idx = base + static_cast<int64_t>(i) * BLOCK + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  uint32_t total;
  block_excl_scan_u32(s, sh, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums, in place.
__global__ void scan_top_kernel(uint32_t* __restrict__ sums, int64_t m) {
  __shared__ uint32_t sh[BLOCK / 32];
  uint32_t carry = 0;
  for (int64_t base = 0; base < m; base += BLOCK) {
    int64_t idx = base + threadIdx.x;
    uint32_t v = idx < m ? sums[idx] : 0u;
    uint32_t total;
    uint32_t before = block_excl_scan_u32(v, sh, &total);
    if (idx < m) sums[idx] = carry + before;
    carry += total;
  }
}

__global__ void scan_down_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                                 const uint32_t* __restrict__ offs) {
  __shared__ uint32_t sh[BLOCK / 32];
  int64_t base = static_cast<int64_t>(blockIdx.x) * TILE + static_cast<int64_t>(threadIdx.x) * ITEMS;
  uint32_t v[ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    s += v[i];
  }
  uint32_t total;
  uint32_t run = block_excl_scan_u32(s, sh, &total) + offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

// --------------------------------------------------------------- radix sort
template <typename K>
__global__ void radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift,
                                  uint32_t* __restrict__ counts, int64_t num_tiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = static_cast<int64_t>(blockIdx.x) * TILE;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    int64_t idx = base + static_cast<int64_t>(i) * BLOCK + threadIdx.x;
    if (idx < n) atomicAdd(&h[static_cast<uint32_t>(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[static_cast<int64_t>(threadIdx.x) * num_tiles + blockIdx.x] = h[threadIdx.x];
}

template <typename K, bool HAS_VAL>
__global__ void radix_scatter_kernel(const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                                     int64_t n, int shift, const uint32_t* __restrict__ offsets,
                                     int64_t num_tiles, K* __restrict__ keys_out,
                                     uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t running[256];
  __shared__ uint32_t total[256];
  __shared__ uint32_t wcnt[BLOCK / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  running[tid] = offsets[static_cast<int64_t>(tid) * num_tiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < BLOCK / 32; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * TILE;
  for (int i = 0; i < ITEMS; ++i) {
    int64_t idx = base + static_cast<int64_t>(i) * BLOCK + tid;
    bool valid = idx < n;
    K k = valid ? keys_in[idx] : K(0);
    uint32_t v = (HAS_VAL && valid) ? vals_in[idx] : 0u;
    uint32_t d = valid ? (static_cast<uint32_t>(k >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lanemask_lt());
    bool leader = (__ffs(peers) - 1) == lane;
    if (valid && leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < BLOCK / 32; ++w) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      total[tid] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = running[d] + wcnt[warp][d] + rank;
      keys_out[pos] = k;
      if (HAS_VAL) vals_out[pos] = v;
    }
    __syncthreads();
    running[tid] += total[tid];
#pragma unroll
    for (int w = 0; w < BLOCK / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
  }
}

template <typename K>
cbg_status radix_sort_impl(cbg_ctx* ctx, K* keys_a, K* keys_b, uint32_t* vals_a, uint32_t* vals_b,
                           int64_t n, int key_bits, void* temp) {
  if (n <= 1) return CBG_OK;
  const int64_t num_tiles = ceil_div(n, TILE);
  const int64_t m = 256 * num_tiles;
  Carve cv(temp);
  uint32_t* counts = cv.take<uint32_t>(m);
  uint32_t* offsets = cv.take<uint32_t>(m);
  void* scan_tmp = cv.take<char>(scan_u32_temp_bytes(m));
  const int passes = (key_bits + 7) / 8;
  K* kin = keys_a;
  K* kout = keys_b;
  uint32_t* vin = vals_a;
  uint32_t* vout = vals_b;
  const bool has_val = vals_a != nullptr;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    radix_hist_kernel<K><<<static_cast<unsigned>(num_tiles), BLOCK, 0, ctx->stream>>>(kin, n, shift, counts, num_tiles);
    CBG_CHECK_LAUNCH(ctx);
    cbg_status st = scan_u32_exclusive(ctx, counts, offsets, m, scan_tmp);
    if (st != CBG_OK) return st;
    if (has_val)
      radix_scatter_kernel<K, true><<<static_cast<unsigned>(num_tiles), BLOCK, 0, ctx->stream>>>(
          kin, vin, n, shift, offsets, num_tiles, kout, vout);
    else
      radix_scatter_kernel<K, false><<<static_cast<unsigned>(num_tiles), BLOCK, 0, ctx->stream>>>(
          kin, nullptr, n, shift, offsets, num_tiles, kout, nullptr);
    CBG_CHECK_LAUNCH(ctx);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if (kin != keys_a) {
    CBG_CUDA(ctx, cudaMemcpyAsync(keys_a, kin, n * sizeof(K), cudaMemcpyDeviceToDevice, ctx->stream));
    if (has_val)
      CBG_CUDA(ctx, cudaMemcpyAsync(vals_a, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return CBG_OK;
}

// ---------------------------------------------------- segmented (cnt, sum) scan
struct Seg {
  uint32_t flag;
  uint32_t cnt;
  double sum;
};

__device__ __forceinline__ Seg seg_op(const Seg& a, const Seg& b) {
  Seg r;
  r.flag = a.flag | b.flag;
  r.cnt = b.flag ? b.cnt : a.cnt + b.cnt;
  r.sum = b.flag ? b.sum : __dadd_rn(a.sum, b.sum);
  return r;
}

__device__ __forceinline__ Seg seg_shfl_up(const Seg& s, int o) {
  Seg r;
  r.flag = __shfl_up_sync(0xffffffffu, s.flag, o);
  r.cnt = __shfl_up_sync(0xffffffffu, s.cnt, o);
  r.sum = __shfl_up_sync(0xffffffffu, s.sum, o);
  return r;
}

// Inclusive block scan; returns the exclusive prefix of this thread (identity for thread 0
// is flag=0,cnt=0,sum=0) and the block aggregate.
__device__ Seg block_seg_scan(const Seg& v, Seg* sh, Seg* agg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Seg x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Seg y = seg_shfl_up(x, o);
    if (lane >= o) x = seg_op(y, x);
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    Seg w = lane < BLOCK / 32 ? sh[lane] : Seg{0u, 0u, 0.0};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Seg y = seg_shfl_up(w, o);
      if (lane >= o) w = seg_op(y, w);
    }
    if (lane < BLOCK / 32) sh[lane] = w;
  }
  __syncthreads();
  // exclusive prefix within the warp
  Seg xe = seg_shfl_up(x, 1);
  if (lane == 0) xe = Seg{0u, 0u, 0.0};
  Seg before = xe;
  if (warp > 0) before = (lane == 0) ? sh[warp - 1] : seg_op(sh[warp - 1], xe);
  *agg = sh[BLOCK / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void segscan_reduce_kernel(const uint8_t* __restrict__ heads, const double* __restrict__ vals,
                                      int64_t n, Seg* __restrict__ aggs) {
  __shared__ Seg sh[BLOCK / 32];
  int64_t base = static_cast<int64_t>(blockIdx.x) * TILE + static_cast<int64_t>(threadIdx.x) * ITEMS;
  Seg s{0u, 0u, 0.0};
  for (int i = 0; i < ITEMS; ++i) {
    int64_t idx = base + i;
    if (idx < n) s = seg_op(s, Seg{heads[idx] ? 1u : 0u, 1u, vals[idx]});
  }
  Seg agg;
  block_seg_scan(s, sh, &agg);
  if (threadIdx.x == 0) aggs[blockIdx.x] = agg;
}

// One block: exclusive scan of tile aggregates in place (carry into each tile).
__global__ void segscan_top_kernel(Seg* __restrict__ aggs, int64_t m) {
  __shared__ Seg sh[BLOCK / 32];
  Seg carry{0u, 0u, 0.0};
  for (int64_t base = 0; base < m; base += BLOCK) {
    int64_t idx = base + threadIdx.x;
    Seg v = idx < m ? aggs[idx] : Seg{0u, 0u, 0.0};
    Seg agg;
    Seg before = block_seg_scan(v, sh, &agg);
    if (idx < m) aggs[idx] = seg_op(carry, before);
    carry = seg_op(carry, agg);
  }
}

__global__ void segscan_down_kernel(const uint8_t* __restrict__ heads, const double* __restrict__ vals,
                                    int64_t n, const Seg* __restrict__ carries,
                                    uint32_t* __restrict__ out_cnt, double* __restrict__ out_sum) {
  __shared__ Seg sh[BLOCK / 32];
  int64_t base = static_cast<int64_t>(blockIdx.x) * TILE + static_cast<int64_t>(threadIdx.x) * ITEMS;
  Seg e[ITEMS];
  Seg s{0u, 0u, 0.0};
  for (int i = 0; i < ITEMS; ++i) {
    int64_t idx = base + i;
    e[i] = idx < n ? Seg{heads[idx] ? 1u : 0u, 1u, vals[idx]} : Seg{0u, 0u, 0.0};
    s = seg_op(s, e[i]);
  }
  Seg agg;
  Seg run = seg_op(carries[blockIdx.x], block_seg_scan(s, sh, &agg));
  for (int i = 0; i < ITEMS; ++i) {
    int64_t idx = base + i;
    run = seg_op(run, e[i]);
    if (idx < n) {
      out_cnt[idx] = run.cnt;
      out_sum[idx] = run.sum;
    }
  }
}

}  // namespace

size_t scan_u32_temp_bytes(int64_t n) { return (ceil_div(n, TILE) + 64) * sizeof(uint32_t) + 256; }

cbg_status scan_u32_exclusive(cbg_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, void* temp) {
  if (n <= 0) return CBG_OK;
  const int64_t tiles = ceil_div(n, TILE);
  uint32_t* sums = static_cast<uint32_t*>(temp);
  scan_reduce_kernel<<<static_cast<unsigned>(tiles), BLOCK, 0, ctx->stream>>>(in, n, sums);
  CBG_CHECK_LAUNCH(ctx);
  scan_top_kernel<<<1, BLOCK, 0, ctx->stream>>>(sums, tiles);
  CBG_CHECK_LAUNCH(ctx);
  scan_down_kernel<<<static_cast<unsigned>(tiles), BLOCK, 0, ctx->stream>>>(in, out, n, sums);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

size_t radix_temp_bytes(int64_t n) {
  const int64_t m = 256 * ceil_div(n, TILE);
  return 2 * (m * sizeof(uint32_t) + 256) + scan_u32_temp_bytes(m) + 256;
}

cbg_status radix_sort_u32(cbg_ctx* ctx, uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a,
                          uint32_t* vals_b, int64_t n, int key_bits, void* temp) {
  return radix_sort_impl<uint32_t>(ctx, keys_a, keys_b, vals_a, vals_b, n, key_bits, temp);
}

cbg_status radix_sort_u64(cbg_ctx* ctx, uint64_t* keys_a, uint64_t* keys_b, uint32_t* vals_a,
                          uint32_t* vals_b, int64_t n, int key_bits, void* temp) {
  return radix_sort_impl<uint64_t>(ctx, keys_a, keys_b, vals_a, vals_b, n, key_bits, temp);
}

size_t segscan_temp_bytes(int64_t n) { return (ceil_div(n, TILE) + 64) * sizeof(Seg) + 256; }

cbg_status segscan_cnt_sum(cbg_ctx* ctx, const uint8_t* heads, const double* vals, int64_t n,
                           uint32_t* out_cnt, double* out_sum, void* temp) {
  if (n <= 0) return CBG_OK;
  const int64_t tiles = ceil_div(n, TILE);
  Seg* aggs = static_cast<Seg*>(temp);
  segscan_reduce_kernel<<<static_cast<unsigned>(tiles), BLOCK, 0, ctx->stream>>>(heads, vals, n, aggs);
  CBG_CHECK_LAUNCH(ctx);
  segscan_top_kernel<<<1, BLOCK, 0, ctx->stream>>>(aggs, tiles);
  CBG_CHECK_LAUNCH(ctx);
  segscan_down_kernel<<<static_cast<unsigned>(tiles), BLOCK, 0, ctx->stream>>>(heads, vals, n, aggs,
                                                                              out_cnt, out_sum);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

}  // namespace cbg
