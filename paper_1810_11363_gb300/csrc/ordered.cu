// Ordered boosting (Section 3 "Fighting Gradient Bias", Algorithm 1) with the log-scale
// supporting models M'_i, on the GPU.
//
// Every permutation sigma_q keeps its data in its own position order: bins (grouped and
// [F][n]), labels, and its supporting values. The structure of a tree is searched by the
// ordinary level pipeline on permutation r's position-ordered data with the ordered
// gradients (position k takes its model value from M'_{r, floor(log2 k)}; position 0 from
// the start value 0), so the gradient gather is a contiguous read. The final model's leaf
// values are Newton steps on the plain gradients of every row (the second phase, done the
// classic way) with leaf indices on the final model's own row-order bins; every supporting
// model of every permutation takes the same structure and Newton leaf values from its own
// first 2^i positions.
//
// Supporting values of one permutation (FP32, `sup_len(n) = 2^(I+1) + n` floats used,
// I = floor(log2(n-1)), I = 0 for n = 1, rows of the [s] array padded to a multiple of 64
// floats): model i occupies [2^(i+1), 2^(i+2)) -- the last model [2^(I+1), 2^(I+1) + n) --
// and holds position j at 2^(i+1) + j. Elements 0 and 1 are unused. With this layout a model's range starts at a power of two, so a block of 2^b
// consecutive elements past the first block lies inside one model, and model i's training
// positions p < 2^i are the first half of its range.
#include <algorithm>
#include <cmath>

#include "cbg_internal.cuh"

using namespace cbg;

namespace {

constexpr int OB_THREADS = 256;
constexpr int64_t OB_ITEMS = 2048;     // items per block of the supporting-model kernels
constexpr int OB_MAX_DEPTH = 10;

__host__ __device__ __forceinline__ int ilog2(int64_t k) {   // floor(log2 k), k >= 1
#ifdef __CUDA_ARCH__
  return 63 - __clzll(static_cast<unsigned long long>(k));
#else
  int r = 0;
  while ((int64_t(1) << (r + 1)) <= k) ++r;
  return r;
#endif
}

int top_model(int64_t n) { return n > 1 ? ilog2(n - 1) : 0; }
int64_t sup_len_of(int64_t n) { return (int64_t(2) << top_model(n)) + n; }
int64_t pad64(int64_t x) { return (x + 63) / 64 * 64; }
int64_t sup_stride_of(int64_t n) { return pad64(sup_len_of(n)); }

// ------------------------------------------------------------- row permutation
// out[g][k][0..31] = in[g][sigma[k]][0..31] for the grouped layout, two 16-byte halves
// per row.
__global__ void permute_grouped_kernel(const uint32_t* __restrict__ perm, int64_t n, int64_t groups,
                                       const uint4* __restrict__ in, uint4* __restrict__ out) {
  const int64_t total = groups * n * 2;
  for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
       x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t gk = x >> 1;
    const int64_t g = gk / n, k = gk - g * n;
    out[x] = in[((g * n + perm[k]) << 1) + (x & 1)];
  }
}

// out[f][k] = in[f][sigma[k]] (bytes), and y_out[k] = y[sigma[k]] from the f = 0 pass.
__global__ void permute_columns_kernel(const uint32_t* __restrict__ perm, int64_t n, int F,
                                       const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                       const float* __restrict__ y, float* __restrict__ y_out) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t src = perm[k];
    if (y_out) y_out[k] = y[src];
    if (in)
      for (int f = 0; f < F; ++f) out[f * n + k] = in[f * n + src];
  }
}

// ------------------------------------------------------------ ordered gradients
// Position k >= 1 of permutation r takes its gradient at M'_{r, floor(log2 k)}(x_k),
// stored at element 2^(floor(log2 k)+1) + k; position 0 at the start value 0.
template <typename GH>
__global__ void ordered_grad_kernel(const float* __restrict__ sup, const float* __restrict__ y_pos, int64_t n,
                                    int loss, GH* __restrict__ g, GH* __restrict__ h) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float a = k == 0 ? 0.0f : sup[(int64_t(2) << ilog2(k)) + k];
    float gi, hi;
    cbgd::loss_grad(loss, a, y_pos[k], &gi, &hi);
    cbgd::store_gh(g, k, gi);
    cbgd::store_gh(h, k, hi);
  }
}

// Leaf of row (or position) r from the splits: from the [F][n] bins when given, else the
// grouped layout.
__device__ __forceinline__ int leaf_of(const uint8_t* __restrict__ bins_t, const uint8_t* __restrict__ bins,
                                       int64_t n, int64_t r, const int* sf, const int* sk, int depth) {
  int l = 0;
  for (int d = 0; d < depth; ++d) {
    const int f = sf[d];
    if (f < 0) continue;
    const int b = bins_t ? bins_t[static_cast<int64_t>(f) * n + r]
                         : bins[((static_cast<int64_t>(f >> 5) * n + r) << 5) + (f & 31)];
    if (b > sk[d]) l += 1 << d;
  }
  return l;
}

__device__ __forceinline__ void load_splits(const cbg_split* __restrict__ sp, int depth, int* sf, int* sk) {
  if (threadIdx.x < depth) {
    sf[threadIdx.x] = sp[threadIdx.x].feature;
    sk[threadIdx.x] = sp[threadIdx.x].border;
  }
}

// Per-leaf (G, H) accumulation used by the totals kernels: every warp adds into its own
// FP32 copy in shared memory (red.shared.add.f32, contention only within the warp), and
// the block sums the warps' copies in FP64 before one FP64 atomic per (leaf, statistic)
// into the global totals. A warp's copy sums at most OB_ITEMS / 8 items.
constexpr int OB_WARPS = OB_THREADS / 32;
constexpr int OB_UNROLL = static_cast<int>(OB_ITEMS / OB_THREADS);   // items per thread and block

__device__ __forceinline__ void zero_acc(float* s_acc, int L) {
  for (int x = threadIdx.x; x < OB_WARPS * 2 * L; x += blockDim.x) s_acc[x] = 0.0f;
}

__device__ __forceinline__ void flush_acc(const float* s_acc, int L, double* __restrict__ out) {
  for (int x = threadIdx.x; x < 2 * L; x += blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < OB_WARPS; ++w) v += static_cast<double>(s_acc[w * 2 * L + x]);
    if (v != 0.0) atomicAdd(&out[x], v);
  }
}

// Leaves of the 4 consecutive rows x0..x0+3 from [F][n] bins with one 32-bit load per
// split (x0 % 4 == 0, n % 4 == 0 and a 4-byte aligned base, so every load is aligned).
__device__ __forceinline__ void leaf4(const uint8_t* __restrict__ bins_t, int64_t n, int64_t x0, const int* sf,
                                      const int* sk, int depth, int* l) {
  l[0] = l[1] = l[2] = l[3] = 0;
  for (int d = 0; d < depth; ++d) {
    const int f = sf[d];
    if (f < 0) continue;
    const uint32_t w = *reinterpret_cast<const uint32_t*>(bins_t + static_cast<int64_t>(f) * n + x0);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (static_cast<int>((w >> (8 * j)) & 0xffu) > sk[d]) l[j] += 1 << d;
  }
}

// --------------------------------------------------- final model: leaf totals
// (G, H) per leaf of the plain gradients at pred, leaves from the splits on the final
// model's row-order bins; leaf indices are written for the update that follows. Each
// block takes OB_ITEMS consecutive rows per round, OB_UNROLL per thread: with VEC, two
// runs of 4 consecutive rows read with 32-bit (bins) and 128-bit (pred, y) loads.
template <bool VEC>
__global__ void rows_totals_kernel(const uint8_t* __restrict__ bins_t, const uint8_t* __restrict__ bins, int64_t n,
                                   const cbg_split* __restrict__ sp, int depth, const float* __restrict__ y,
                                   const float* __restrict__ pred, int loss, double* __restrict__ tot,
                                   uint16_t* __restrict__ leaf_out) {
  extern __shared__ float s_acc[];
  __shared__ int sf[OB_MAX_DEPTH], sk[OB_MAX_DEPTH];
  const int L = 1 << depth;
  zero_acc(s_acc, L);
  load_splits(sp, depth, sf, sk);
  __syncthreads();
  float* acc = s_acc + (threadIdx.x >> 5) * 2 * L;
  for (int64_t r0 = blockIdx.x * OB_ITEMS; r0 < n; r0 += static_cast<int64_t>(gridDim.x) * OB_ITEMS) {
    int l[OB_UNROLL];
    float a[OB_UNROLL], yv[OB_UNROLL];
    if (VEC) {
#pragma unroll
      for (int c = 0; c < OB_UNROLL / 4; ++c) {
        const int64_t x0 = r0 + 4 * threadIdx.x + c * 4 * OB_THREADS;
        if (x0 < n) {
          leaf4(bins_t, n, x0, sf, sk, depth, l + 4 * c);
          const float4 p4 = *reinterpret_cast<const float4*>(pred + x0);
          const float4 y4 = *reinterpret_cast<const float4*>(y + x0);
          a[4 * c] = p4.x, a[4 * c + 1] = p4.y, a[4 * c + 2] = p4.z, a[4 * c + 3] = p4.w;
          yv[4 * c] = y4.x, yv[4 * c + 1] = y4.y, yv[4 * c + 2] = y4.z, yv[4 * c + 3] = y4.w;
          *reinterpret_cast<ushort4*>(leaf_out + x0) =
              make_ushort4(static_cast<uint16_t>(l[4 * c]), static_cast<uint16_t>(l[4 * c + 1]),
                           static_cast<uint16_t>(l[4 * c + 2]), static_cast<uint16_t>(l[4 * c + 3]));
        } else {
          l[4 * c] = l[4 * c + 1] = l[4 * c + 2] = l[4 * c + 3] = -1;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < OB_UNROLL; ++k) {
        const int64_t r = r0 + threadIdx.x + k * OB_THREADS;
        l[k] = -1;
        if (r < n) {
          l[k] = leaf_of(bins_t, bins, n, r, sf, sk, depth);
          a[k] = pred[r];
          yv[k] = y[r];
          leaf_out[r] = static_cast<uint16_t>(l[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < OB_UNROLL; ++k) {
      if (l[k] < 0) continue;
      float g, h;
      cbgd::loss_grad(loss, a[k], yv[k], &g, &h);
      atomicAdd(&acc[2 * l[k]], g);
      atomicAdd(&acc[2 * l[k] + 1], h);
    }
  }
  __syncthreads();
  flush_acc(s_acc, L, tot);
}

// ------------------------------------------ supporting models: leaf by position
// leaf_pos[q][k] (row stride lp_stride) for every permutation q, from the splits on q's
// position-ordered bins; OB_UNROLL positions per thread and round (with VEC, two runs of 4
// read with 32-bit loads and written with one 64-bit store each).
template <bool VEC>
__global__ void leaf_pos_kernel(const uint8_t* __restrict__ bins_t_pos, const uint8_t* __restrict__ bins_pos,
                                int64_t n, int F, int F_pad, const cbg_split* __restrict__ sp, int depth,
                                uint16_t* __restrict__ leaf_pos, int64_t lp_stride) {
  __shared__ int sf[OB_MAX_DEPTH], sk[OB_MAX_DEPTH];
  load_splits(sp, depth, sf, sk);
  __syncthreads();
  const int q = blockIdx.y;
  const uint8_t* bt = bins_t_pos ? bins_t_pos + static_cast<int64_t>(q) * F * n : nullptr;
  const uint8_t* bg = bins_pos + static_cast<int64_t>(q) * F_pad * n;
  uint16_t* lq = leaf_pos + static_cast<int64_t>(q) * lp_stride;
  for (int64_t k0 = blockIdx.x * OB_ITEMS; k0 < n; k0 += static_cast<int64_t>(gridDim.x) * OB_ITEMS) {
    if (VEC) {
      int l[OB_UNROLL];
#pragma unroll
      for (int c = 0; c < OB_UNROLL / 4; ++c) {
        const int64_t x0 = k0 + 4 * threadIdx.x + c * 4 * OB_THREADS;
        if (x0 < n) leaf4(bt, n, x0, sf, sk, depth, l + 4 * c);
      }
#pragma unroll
      for (int c = 0; c < OB_UNROLL / 4; ++c) {
        const int64_t x0 = k0 + 4 * threadIdx.x + c * 4 * OB_THREADS;
        if (x0 < n)
          *reinterpret_cast<ushort4*>(lq + x0) =
              make_ushort4(static_cast<uint16_t>(l[4 * c]), static_cast<uint16_t>(l[4 * c + 1]),
                           static_cast<uint16_t>(l[4 * c + 2]), static_cast<uint16_t>(l[4 * c + 3]));
      }
    } else {
      int l[OB_UNROLL];
#pragma unroll
      for (int k = 0; k < OB_UNROLL; ++k) {
        const int64_t x = k0 + threadIdx.x + k * OB_THREADS;
        l[k] = x < n ? leaf_of(bt, bg, n, x, sf, sk, depth) : -1;
      }
#pragma unroll
      for (int k = 0; k < OB_UNROLL; ++k)
        if (l[k] >= 0) lq[k0 + threadIdx.x + k * OB_THREADS] = static_cast<uint16_t>(l[k]);
    }
  }
}

// ------------------------------------------------- supporting models: totals
// Training items of permutation q are u in [1, 2^(I+1)): model i = floor(log2 u), position
// p = u - 2^i, value at element u + 2^i. Block b > 0 covers u in [b B, (b+1) B), all in one
// model (B = OB_ITEMS, a power of two); block 0 (the models with fewer than B training
// positions) adds its few items straight to the FP64 totals.
__global__ void sup_totals_kernel(const float* __restrict__ sup, int64_t sup_stride, const float* __restrict__ y_pos,
                                  const uint16_t* __restrict__ leaf_pos, int64_t lp_stride, int64_t n, int n_models,
                                  int depth, int loss, double* __restrict__ tot) {
  extern __shared__ float s_acc[];
  const int L = 1 << depth;
  const int q = blockIdx.y;
  const float* sq = sup + static_cast<int64_t>(q) * sup_stride;
  const float* yq = y_pos + static_cast<int64_t>(q) * n;
  const uint16_t* lq = leaf_pos + static_cast<int64_t>(q) * lp_stride;
  double* tq = tot + static_cast<int64_t>(q) * n_models * L * 2;
  const int64_t u_end = min((blockIdx.x + 1) * OB_ITEMS, int64_t(1) << n_models);
  if (blockIdx.x == 0) {
    for (int64_t u = 1 + threadIdx.x; u < u_end; u += blockDim.x) {
      const int i = ilog2(u);
      const int64_t p = u - (int64_t(1) << i);
      float g, h;
      cbgd::loss_grad(loss, sq[u + (int64_t(1) << i)], yq[p], &g, &h);
      double* t = tq + (static_cast<int64_t>(i) * L + lq[p]) * 2;
      atomicAdd(t, static_cast<double>(g));
      atomicAdd(t + 1, static_cast<double>(h));
    }
    return;
  }
  const int64_t u0 = blockIdx.x * OB_ITEMS;
  const int i = ilog2(u0);
  const int64_t half = int64_t(1) << i;
  zero_acc(s_acc, L);
  __syncthreads();
  float* acc = s_acc + (threadIdx.x >> 5) * 2 * L;
  float a[OB_UNROLL], yv[OB_UNROLL];
  int l[OB_UNROLL];
#pragma unroll
  for (int k = 0; k < OB_UNROLL; ++k) {
    const int64_t u = u0 + threadIdx.x + k * OB_THREADS;
    l[k] = -1;
    if (u < u_end) {
      a[k] = sq[u + half];
      yv[k] = yq[u - half];
      l[k] = lq[u - half];
    }
  }
#pragma unroll
  for (int k = 0; k < OB_UNROLL; ++k) {
    if (l[k] < 0) continue;
    float g, h;
    cbgd::loss_grad(loss, a[k], yv[k], &g, &h);
    atomicAdd(&acc[2 * l[k]], g);
    atomicAdd(&acc[2 * l[k] + 1], h);
  }
  __syncthreads();
  flush_acc(s_acc, L, tq + static_cast<int64_t>(i) * L * 2);
}

__device__ __forceinline__ float newton_step_lr(const double* t, double l2, double lr) {
  const double den = t[1] + l2;
  const double v = den == 0.0 ? 0.0 : -t[0] / den;
  return static_cast<float>(lr * v);
}

// -------------------------------------------------- supporting models: update
// Element e in [2, sup_len) belongs to model i = floor(log2 e) - 1 at position
// j = e - 2^(i+1); it gains float(lr v) of its leaf, v = -G/(H + l2) (0 when H + l2 = 0).
__global__ void sup_apply_kernel(float* __restrict__ sup, int64_t sup_stride, int64_t sup_len,
                                 const uint16_t* __restrict__ leaf_pos, int64_t lp_stride, int n_models, int depth,
                                 const double* __restrict__ tot, double l2, double lr) {
  extern __shared__ float s_lrv[];
  const int L = 1 << depth;
  const int q = blockIdx.y;
  float* sq = sup + static_cast<int64_t>(q) * sup_stride;
  const uint16_t* lq = leaf_pos + static_cast<int64_t>(q) * lp_stride;
  const double* tq = tot + static_cast<int64_t>(q) * n_models * L * 2;
  const int64_t e_end = min((blockIdx.x + 1) * OB_ITEMS, sup_len);
  if (blockIdx.x == 0) {
    for (int64_t e = 2 + threadIdx.x; e < e_end; e += blockDim.x) {
      const int i = ilog2(e) - 1;
      const int64_t j = e - (int64_t(2) << i);
      sq[e] += newton_step_lr(tq + (static_cast<int64_t>(i) * L + lq[j]) * 2, l2, lr);
    }
    return;
  }
  const int64_t e0 = blockIdx.x * OB_ITEMS;
  const int i = ilog2(e0) - 1;
  const int64_t base = int64_t(2) << i;
  for (int l = threadIdx.x; l < L; l += blockDim.x)
    s_lrv[l] = newton_step_lr(tq + (static_cast<int64_t>(i) * L + l) * 2, l2, lr);
  __syncthreads();
  float v[OB_UNROLL];
  int l[OB_UNROLL];
#pragma unroll
  for (int k = 0; k < OB_UNROLL; ++k) {
    const int64_t e = e0 + threadIdx.x + k * OB_THREADS;
    l[k] = -1;
    if (e < e_end) {
      v[k] = sq[e];
      l[k] = lq[e - base];
    }
  }
#pragma unroll
  for (int k = 0; k < OB_UNROLL; ++k)
    if (l[k] >= 0) sq[e0 + threadIdx.x + k * OB_THREADS] = v[k] + s_lrv[l[k]];
}

// Copies one tree's splits and leaf values from the graph's fixed scratch to slot t of the
// model (t read from, then advanced in, a device counter), so that a captured tree can be
// replayed for every tree of its permutation.
__global__ void ordered_record_kernel(const cbg_split* __restrict__ sp_tmp, const double* __restrict__ v_tmp, int depth,
                                      cbg_split* __restrict__ splits, double* __restrict__ values,
                                      unsigned* __restrict__ counter, int trees) {
  __shared__ unsigned t;
  if (threadIdx.x == 0) t = *counter;
  __syncthreads();
  if (t < static_cast<unsigned>(trees)) {
    const int L = 1 << depth;
    for (int i = threadIdx.x; i < depth; i += blockDim.x) splits[static_cast<int64_t>(t) * depth + i] = sp_tmp[i];
    for (int i = threadIdx.x; i < L; i += blockDim.x) values[static_cast<int64_t>(t) * L + i] = v_tmp[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = t + 1;
}

unsigned stride_grid(int64_t n) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, OB_THREADS), 152LL * 16)));
}

struct Work {
  uint16_t* leaf_pos;   // [s][pad64(n)]
  uint16_t* leaf_rows;  // [n]
  double* tot_final;    // [L][2]
  double* tot_sup;      // [s][n_models][L][2], directly after tot_final
  cbg_split* sp_tmp;    // [depth] a captured tree's splits
  double* v_tmp;        // [L] a captured tree's leaf values
  unsigned* counter;    // slot of the next recorded tree
  size_t bytes;
};

Work carve_work(void* base, int64_t n, int s, int depth) {
  Carve c(base);
  Work w;
  const int L = 1 << depth;
  w.leaf_pos = c.take<uint16_t>(static_cast<size_t>(s) * pad64(n));
  w.leaf_rows = c.take<uint16_t>(static_cast<size_t>(n));
  w.tot_final = c.take<double>(static_cast<size_t>(2 * L));
  w.tot_sup = c.take<double>(static_cast<size_t>(s) * (top_model(n) + 1) * L * 2, 8);
  w.sp_tmp = c.take<cbg_split>(OB_MAX_DEPTH);
  w.v_tmp = c.take<double>(static_cast<size_t>(L));
  w.counter = c.take<unsigned>(1);
  w.bytes = c.off;
  return w;
}

}  // namespace

extern "C" {

cbg_status cbg_ordered_sup_len(int64_t n, int64_t* len) {
  if (!len || n < 1 || n > INT32_MAX) return CBG_EINVAL;
  *len = sup_stride_of(n);
  return CBG_OK;
}

cbg_status cbg_ordered_work_bytes(int64_t n, int32_t s, int32_t depth, size_t* bytes) {
  if (!bytes || n < 1 || n > INT32_MAX || s < 1 || depth < 1 || depth > OB_MAX_DEPTH) return CBG_EINVAL;
  *bytes = carve_work(nullptr, n, s, depth).bytes;
  return CBG_OK;
}

cbg_status cbg_permute_rows(cbg_ctx* ctx, const uint32_t* perm, int64_t n, int32_t F, int32_t F_pad,
                            const uint8_t* bins, const uint8_t* bins_t, const float* y, uint8_t* bins_pos,
                            uint8_t* bins_t_pos, float* y_pos) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, perm != nullptr && n >= 1 && n <= INT32_MAX, "need perm and n in [1, 2^31-1]");
  CBG_REQUIRE(ctx, !bins || (F_pad >= 32 && F_pad % 32 == 0 && bins_pos), "grouped bins need F_pad % 32 == 0 and an output");
  CBG_REQUIRE(ctx, !bins || ((reinterpret_cast<uintptr_t>(bins) | reinterpret_cast<uintptr_t>(bins_pos)) & 15) == 0,
              "grouped bins must be 16-byte aligned");
  CBG_REQUIRE(ctx, !bins_t || (F >= 1 && bins_t_pos), "bins_t needs F >= 1 and an output");
  CBG_REQUIRE(ctx, !y || y_pos, "y needs an output");
  DeviceGuard guard(ctx->device);
  if (bins) {
    const int64_t groups = F_pad / 32;
    permute_grouped_kernel<<<stride_grid(groups * n * 2), OB_THREADS, 0, ctx->stream>>>(
        perm, n, groups, reinterpret_cast<const uint4*>(bins),
        reinterpret_cast<uint4*>(bins_pos));
    CBG_CHECK_LAUNCH(ctx);
  }
  if (bins_t || y) {
    permute_columns_kernel<<<stride_grid(n), OB_THREADS, 0, ctx->stream>>>(perm, n, F, bins_t, bins_t_pos, y, y_pos);
    CBG_CHECK_LAUNCH(ctx);
  }
  return CBG_OK;
}

}  // extern "C"

namespace {

// One iteration of ordered boosting on permutation r; splits to sp, leaf values to vals.
cbg_status ordered_tree(cbg_ctx* ctx, const cbg_ordered_args* a, const Work& w, int r, cbg_split* sp, double* vals) {
  const cbg_tree_shape* sh = a->shape;
  const int64_t n = sh->n;
  const int D = a->depth;
  const int L = 1 << D;
  const int n_models = top_model(n) + 1;
  const int64_t sup_len = sup_len_of(n);
  const int64_t sup_stride = sup_stride_of(n);
  const int64_t lp_stride = pad64(n);
  const int64_t plane = static_cast<int64_t>(sh->F_pad) * n;
  const unsigned grid_n = stride_grid(n);
  const unsigned grid_rows = static_cast<unsigned>(std::min<int64_t>(ceil_div(n, OB_ITEMS), 152LL * 8));
  const dim3 grid_tot(static_cast<unsigned>(ceil_div(int64_t(1) << n_models, OB_ITEMS)), a->s);
  const dim3 grid_app(static_cast<unsigned>(ceil_div(sup_len, OB_ITEMS)), a->s);
  const dim3 grid_leaf(static_cast<unsigned>(std::min<int64_t>(ceil_div(n, OB_ITEMS), 152LL * 8 / a->s + 1)), a->s);
  const size_t tot_bytes = sizeof(double) * 2 * L * (1 + static_cast<size_t>(a->s) * n_models);
  const size_t acc_bytes = sizeof(float) * OB_WARPS * 2 * L;
  const float* sup_r = a->sup + r * sup_stride;
  const float* y_r = a->y_pos + r * n;
  if (a->gh_dtype == CBG_F32)
    ordered_grad_kernel<float><<<grid_n, OB_THREADS, 0, ctx->stream>>>(sup_r, y_r, n, a->loss, static_cast<float*>(a->g),
                                                                       static_cast<float*>(a->h));
  else
    ordered_grad_kernel<__nv_bfloat16><<<grid_n, OB_THREADS, 0, ctx->stream>>>(
        sup_r, y_r, n, a->loss, static_cast<__nv_bfloat16*>(a->g), static_cast<__nv_bfloat16*>(a->h));
  CBG_CHECK_LAUNCH(ctx);
  // the structure, on permutation r's position-ordered data
  cbg_status st = cbg_tree_begin(ctx, sh, a->state, a->state_bytes, a->leaf);
  if (st != CBG_OK) return st;
  for (int d = 0; d < D; ++d) {
    cbg_level_args la{};
    la.shape = sh;
    la.state = a->state;
    la.state_bytes = a->state_bytes;
    la.bins = a->bins_pos + r * plane;
    la.bins_t = a->bins_t_pos ? a->bins_t_pos + static_cast<int64_t>(r) * sh->F * n : nullptr;
    la.n_borders = a->n_borders;
    la.g = a->g;
    la.h = a->h;
    la.gh_dtype = a->gh_dtype;
    la.depth = d;
    la.l2 = a->l2;
    la.force_feature = -1;
    la.force_border = -1;
    la.leaf = a->leaf;
    la.splits = sp;
    la.child_totals = a->child_totals;
    la.last_level = d == D - 1;
    st = cbg_build_level(ctx, &la);
    if (st != CBG_OK) return st;
  }
  // the final model: plain gradients of every row, leaf values, prediction update
  CBG_CUDA(ctx, cudaMemsetAsync(w.tot_final, 0, tot_bytes, ctx->stream));
  const bool vec_rows = a->bins_t && n % 4 == 0 && ((reinterpret_cast<uintptr_t>(a->bins_t) |
                                                      reinterpret_cast<uintptr_t>(a->y) |
                                                      reinterpret_cast<uintptr_t>(a->pred)) & 15) == 0;
  if (vec_rows)
    rows_totals_kernel<true><<<grid_rows, OB_THREADS, acc_bytes, ctx->stream>>>(a->bins_t, a->bins, n, sp, D, a->y,
                                                                               a->pred, a->loss, w.tot_final,
                                                                               w.leaf_rows);
  else
    rows_totals_kernel<false><<<grid_rows, OB_THREADS, acc_bytes, ctx->stream>>>(a->bins_t, a->bins, n, sp, D, a->y,
                                                                                a->pred, a->loss, w.tot_final,
                                                                                w.leaf_rows);
  CBG_CHECK_LAUNCH(ctx);
  cbg_apply_args aa{};
  aa.bins = a->bins;
  aa.n = n;
  aa.F_pad = sh->F_pad;
  aa.splits = sp;
  aa.depth = D;
  aa.leaf_totals = w.tot_final;
  aa.l2 = a->l2;
  aa.lr = a->lr;
  aa.leaf_in = w.leaf_rows;
  aa.pred = a->pred;
  aa.leaf_values_out = vals;
  st = cbg_apply_tree(ctx, &aa);
  if (st != CBG_OK) return st;
  // the supporting models of every permutation
  const bool vec_pos = a->bins_t_pos && n % 4 == 0 && (reinterpret_cast<uintptr_t>(a->bins_t_pos) & 3) == 0;
  if (vec_pos)
    leaf_pos_kernel<true><<<grid_leaf, OB_THREADS, 0, ctx->stream>>>(a->bins_t_pos, a->bins_pos, n, sh->F, sh->F_pad,
                                                                    sp, D, w.leaf_pos, lp_stride);
  else
    leaf_pos_kernel<false><<<grid_leaf, OB_THREADS, 0, ctx->stream>>>(a->bins_t_pos, a->bins_pos, n, sh->F, sh->F_pad,
                                                                     sp, D, w.leaf_pos, lp_stride);
  CBG_CHECK_LAUNCH(ctx);
  sup_totals_kernel<<<grid_tot, OB_THREADS, acc_bytes, ctx->stream>>>(a->sup, sup_stride, a->y_pos, w.leaf_pos,
                                                                     lp_stride, n, n_models, D, a->loss, w.tot_sup);
  CBG_CHECK_LAUNCH(ctx);
  sup_apply_kernel<<<grid_app, OB_THREADS, sizeof(float) * L, ctx->stream>>>(a->sup, sup_stride, sup_len, w.leaf_pos,
                                                                            lp_stride, n_models, D, w.tot_sup, a->l2,
                                                                            a->lr);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

// Captures one tree of permutation r (outputs to the work scratch, then the record kernel)
// as a graph. The caller's stream may be the legacy default stream, which cannot be
// captured: the capture runs on a library-owned stream.
cbg_status capture_tree(cbg_ctx* ctx, const cbg_ordered_args* a, const Work& w, int r, cudaGraphExec_t* exec) {
  if (!ctx->capture_stream) CBG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  cudaStream_t user_stream = ctx->stream;
  ctx->stream = ctx->capture_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    ctx->stream = user_stream;
    return fail(ctx, CBG_ECUDA, "cudaStreamBeginCapture failed: %s", cudaGetErrorString(ce));
  }
  cbg_status st = ordered_tree(ctx, a, w, r, w.sp_tmp, w.v_tmp);
  if (st == CBG_OK) {
    ordered_record_kernel<<<1, 256, 0, ctx->stream>>>(w.sp_tmp, w.v_tmp, a->depth, a->splits, a->leaf_values, w.counter,
                                                      a->trees);
    if (cudaGetLastError() != cudaSuccess) st = fail(ctx, CBG_ECUDA, "record kernel launch failed during capture");
  }
  ce = cudaStreamEndCapture(ctx->stream, &graph);
  ctx->stream = user_stream;
  if (st != CBG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "stream capture of a tree failed: %s", cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
  return CBG_OK;
}

}  // namespace

extern "C" {

cbg_status cbg_boost_ordered(cbg_ctx* ctx, const cbg_ordered_args* a) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, a != nullptr && a->shape != nullptr, "args is NULL");
  const cbg_tree_shape* sh = a->shape;
  const int64_t n = sh->n;
  const int D = a->depth;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, D >= 1 && D <= sh->max_depth && D <= OB_MAX_DEPTH, "depth outside [1, max_depth]");
  CBG_REQUIRE(ctx, a->s >= 1, "need at least one permutation");
  CBG_REQUIRE(ctx, a->trees >= 0 && a->first_tree >= 0, "trees and first_tree must be >= 0");
  CBG_REQUIRE(ctx, a->loss == CBG_LOSS_RMSE || a->loss == CBG_LOSS_LOGLOSS, "bad loss");
  CBG_REQUIRE(ctx, a->gh_dtype == CBG_F32 || a->gh_dtype == CBG_BF16, "bad gh_dtype");
  CBG_REQUIRE(ctx, a->bins_pos && a->y_pos && a->bins && a->y && a->pred && a->sup && a->g && a->h && a->leaf &&
                       a->splits && a->leaf_values && a->child_totals && a->work,
              "NULL argument");
  const Work w = carve_work(a->work, n, a->s, D);
  CBG_REQUIRE(ctx, a->work_bytes >= w.bytes, "work holds %zu bytes, %zu needed", a->work_bytes, w.bytes);
  DeviceGuard guard(ctx->device);
  const int L = 1 << D;
  const int acc_bytes = static_cast<int>(sizeof(float)) * OB_WARPS * 2 * L;   // 64 KB at depth 10
  if (acc_bytes > 48 * 1024) {
    CBG_CUDA(ctx, cudaFuncSetAttribute(rows_totals_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, acc_bytes));
    CBG_CUDA(ctx, cudaFuncSetAttribute(rows_totals_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, acc_bytes));
    CBG_CUDA(ctx, cudaFuncSetAttribute(sup_totals_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, acc_bytes));
  }
  if (!a->use_graph || a->trees <= 1) {
    for (int t = 0; t < a->trees; ++t) {
      cbg_status st = ordered_tree(ctx, a, w, (a->first_tree + t) % a->s, a->splits + static_cast<int64_t>(t) * D,
                                   a->leaf_values + static_cast<int64_t>(t) * L);
      if (st != CBG_OK) return st;
    }
    return CBG_OK;
  }
  // Graph replay: the first tree runs directly (its launch-geometry queries fill the
  // caches a capture cannot query), then one captured tree per permutation is replayed.
  CBG_CUDA(ctx, cudaMemsetAsync(w.counter, 0, sizeof(unsigned), ctx->stream));
  cbg_status st = ordered_tree(ctx, a, w, a->first_tree % a->s, w.sp_tmp, w.v_tmp);
  if (st != CBG_OK) return st;
  ordered_record_kernel<<<1, 256, 0, ctx->stream>>>(w.sp_tmp, w.v_tmp, D, a->splits, a->leaf_values, w.counter,
                                                    a->trees);
  CBG_CHECK_LAUNCH(ctx);
  std::vector<cudaGraphExec_t> exec(a->s, nullptr);
  cudaError_t ce = cudaSuccess;
  for (int t = 1; t < a->trees && st == CBG_OK; ++t) {
    const int r = (a->first_tree + t) % a->s;
    if (!exec[r]) st = capture_tree(ctx, a, w, r, &exec[r]);
    if (st == CBG_OK) {
      ce = cudaGraphLaunch(exec[r], ctx->stream);
      if (ce != cudaSuccess) st = fail(ctx, CBG_ECUDA, "graph launch failed: %s", cudaGetErrorString(ce));
    }
  }
  for (cudaGraphExec_t e : exec)
    if (e) cudaGraphExecDestroy(e);   // freed once the queued launches complete
  return st;
}

}  // extern "C"
