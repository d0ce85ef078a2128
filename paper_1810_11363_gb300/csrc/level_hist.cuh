// Histogram of one tree level: the work-unit plan, the cluster histogram kernel (FP32
// accumulation in shared memory, reduced across the CTAs of a cluster through
// distributed shared memory), the FP64 reduction of the unit partials with sibling
// subtraction, and the launch geometry. Shared by the level builder (tree.cu) and the
// allocation-free root histogram (noalloc.cu).
#pragma once

#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <tuple>

#include "cbg_internal.cuh"

namespace {

constexpr int GROUP = 32;          // features per group / histogram slab
constexpr int MAX_DEPTH = 10;
constexpr int MAX_HLEAVES = 1 << (MAX_DEPTH - 1);  // leaves histogrammed at the last level

struct Plan {
  int n_small;                      // leaves histogrammed directly at this level
  int total_units;                  // sum of chunks over those leaves
  int level_leaves;                 // 2^d
  int pad;
  int small_leaf[MAX_HLEAVES];
  int large_leaf[MAX_HLEAVES];      // sibling obtained by subtraction (-1: none)
  int parent[MAX_HLEAVES];          // index of the parent in the previous histogram
  int unit_begin[MAX_HLEAVES + 1];
  int chunk_rows[MAX_HLEAVES];
  int seg_start[MAX_HLEAVES];
  int seg_cnt[MAX_HLEAVES];
};

size_t hist_smem_bytes(int nb_alloc) { return static_cast<size_t>(2) * nb_alloc * GROUP * sizeof(float); }

// What the histogram launch needs to know about a problem. kind 0: warp-private
// histograms without atomics (default); kind 1: one shared histogram per CTA updated with
// shared-memory float reductions.
struct HistConfig {
  int64_t n;
  int G, F, max_bins, nb_alloc, threads, cluster, kind = 0;
};

// Warps per CTA of the warp-private kernel: as many (G, H) float2 histograms of
// max_bins x 32 as fit in one SM's shared memory, at most 16.
// Every warp of the warp-private kernel holds a (G, H) float2 histogram of 16 features x
// max_bins; warps come in pairs (the two halves of a 32-feature group).
constexpr int WP_FEATS = 16;
inline int wp_warps(int max_bins, int requested_threads) {
  const int fit = static_cast<int>((227 * 1024) / (static_cast<size_t>(max_bins) * WP_FEATS * sizeof(float2)));
  int w = fit < 16 ? fit : 16;
  if (requested_threads > 0 && requested_threads / 32 < w) w = requested_threads / 32;
  w &= ~1;
  return w < 2 ? 2 : w;
}
inline size_t wp_smem_bytes(int max_bins, int warps) {
  return static_cast<size_t>(warps) * max_bins * WP_FEATS * sizeof(float2);
}

// ------------------------------------------------------------------ histogram
__device__ __forceinline__ void red_add(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Persistent kernel over work units (leaf chunk x feature group), launched as thread-block
// clusters of cs CTAs. Each CTA of a cluster accumulates the (G, H) histogram of its
// sub-chunk of rows in its own shared memory (FP32, red.shared.add). After a cluster
// barrier, CTA r sums its slice of bins across the cs CTAs through distributed shared
// memory and writes it to the unit's FP32 partial, so one partial is written per cluster
// and unit. Lane (j, c): row j of 16, 16-feature chunk c of the group; iteration l
// updates feature 16c + (l + j) % 16, so the 32 lanes hit 32 different features and banks
// (the rotation of the paper's Section 4 example, applied to 16-byte loads). Chunks that
// hold only padding features are skipped.
// MODE 0: G and H in two planes [2][NB][32], each updated with red.shared.add.f32.
// MODE 1: (G, H) interleaved as float2 [NB][32], updated with one 64-bit compare-and-swap
// loop per (row, feature); on sm_103a the FP32 shared reduction is itself a
// compare-and-swap loop, so this halves the atomic operations.
__device__ __forceinline__ void cas_add2(float2* p, float gx, float hy) {
  unsigned long long* a = reinterpret_cast<unsigned long long*>(p);
  unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(a);
  while (true) {
    float2 o;
    memcpy(&o, &old, 8);
    const float2 nw = make_float2(o.x + gx, o.y + hy);
    unsigned long long nv;
    memcpy(&nv, &nw, 8);
    const unsigned long long prev = atomicCAS(a, old, nv);
    if (prev == old) break;
    old = prev;
  }
}

template <typename GH, int NB, int MODE>
__global__ void __launch_bounds__(512, 3) level_hist_kernel(const uint8_t* __restrict__ bins, int64_t n, int G, int F,
                                                         const uint32_t* __restrict__ order,
                                                         const GH* __restrict__ g, const GH* __restrict__ h,
                                                         const Plan* __restrict__ plan, int max_bins,
                                                         float* __restrict__ partials) {
  namespace cgr = cooperative_groups;
  extern __shared__ __align__(16) float hsh[];   // [2][NB][32]
  constexpr int PLANE = NB * GROUP;
  constexpr int MAX_CS = 16;
  cgr::cluster_group cl = cgr::this_cluster();
  const int cs = static_cast<int>(cl.num_blocks());
  const int rank = static_cast<int>(cl.block_rank());
  const int cid = blockIdx.x / cs, ncl = gridDim.x / cs;
  const float* peer[MAX_CS];
  for (int r = 0; r < cs && r < MAX_CS; ++r) peer[r] = cl.map_shared_rank(hsh, r);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int j = lane >> 1, c = lane & 1;
  const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(hsh));
  uint32_t off[16];
#pragma unroll
  for (int l = 0; l < 16; ++l) off[l] = sbase + 4u * static_cast<uint32_t>(c * 16 + ((l + j) & 15));
  const int total_items = plan->total_units * G;
  const int n_small = plan->n_small;
  for (int item = cid; item < total_items; item += ncl) {
    const int unit = item / G, grp = item - unit * G;
    // leaf of this unit: last jj with unit_begin[jj] <= unit
    int lo = 0, hi = n_small - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (plan->unit_begin[mid] <= unit) lo = mid; else hi = mid - 1;
    }
    const int jj = lo;
    const int chunk = unit - plan->unit_begin[jj];
    const int seg_s = plan->seg_start[jj], seg_c = plan->seg_cnt[jj];
    const int cr = plan->chunk_rows[jj];
    const int p0 = seg_s + (chunk * cs + rank) * cr;
    const int p1 = min(seg_s + seg_c, p0 + cr);
    for (int i = threadIdx.x; i < 2 * PLANE / 4; i += blockDim.x)
      reinterpret_cast<float4*>(hsh)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const bool active = grp * GROUP + c * 16 < F;
    const uint8_t* gbase = bins + static_cast<int64_t>(grp) * n * GROUP + c * 16;
    if (active) {
      for (int pos = p0 + warp * 16 + j; pos < p1; pos += nw * 16) {
        const uint32_t row = order ? order[pos] : static_cast<uint32_t>(pos);
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(gbase + static_cast<int64_t>(row) * GROUP));
        const float gv = cbgd::load_gh(g, row), hv = cbgd::load_gh(h, row);
        // rotate the 16 bytes so that byte l of R is byte (l + j) % 16 of v
        uint32_t w0 = v.x, w1 = v.y, w2 = v.z, w3 = v.w;
        const int q = (j >> 2) & 3, r = j & 3;
        if (q & 2) {
          uint32_t t = w0; w0 = w2; w2 = t;
          t = w1; w1 = w3; w3 = t;
        }
        if (q & 1) {
          uint32_t t = w0; w0 = w1; w1 = w2; w2 = w3; w3 = t;
        }
        uint32_t R[4];
        R[0] = __funnelshift_r(w0, w1, 8 * r);
        R[1] = __funnelshift_r(w1, w2, 8 * r);
        R[2] = __funnelshift_r(w2, w3, 8 * r);
        R[3] = __funnelshift_r(w3, w0, 8 * r);
#pragma unroll
        for (int l = 0; l < 16; ++l) {
          const uint32_t b = (R[l >> 2] >> (8 * (l & 3))) & (NB - 1);
          if (MODE == 0) {
            const uint32_t a = off[l] + b * (GROUP * 4);
            red_add(a, gv);
            red_add(a + PLANE * 4, hv);
          } else {
            // off[l] - sbase is 4 x (feature within the group)
            const uint32_t f = (off[l] - sbase) >> 2;
            cas_add2(reinterpret_cast<float2*>(hsh) + b * GROUP + f, gv, hv);
          }
        }
      }
    }
    cl.sync();
    // this CTA's slice of bins, summed over the cluster's CTAs in rank order
    const int bs = (max_bins + cs - 1) / cs;
    const int b0 = rank * bs;
    const int nbs = max(0, min(max_bins, b0 + bs) - b0);
    float* dst = partials + static_cast<int64_t>(item) * (2 * max_bins * GROUP);
    for (int i = threadIdx.x; i < 2 * nbs * GROUP; i += blockDim.x) {
      const int st = i / (nbs * GROUP), rem = i - st * (nbs * GROUP);
      const int e = MODE == 0 ? st * PLANE + b0 * GROUP + rem : (b0 * GROUP + rem) * 2 + st;
      float v = 0.f;
      for (int r = 0; r < cs; ++r) v += peer[r][e];
      dst[st * (max_bins * GROUP) + b0 * GROUP + rem] = v;
    }
    cl.sync();
  }
}

// Warp-private histogram, no atomics (the paper's Section 4 scheme: per-warp partial
// histograms of a few features, updated without atomic operations; here 16 features and
// two rows per warp instruction). A warp owns half of a 32-feature group: a (G, H) float2
// histogram [max_bins][16] in shared memory that no other warp touches. Lane (r, f)
// handles feature f of row 2p + r of each row pair p, so one instruction updates 32
// (row, feature) cells with plain shared loads and stores. The two lanes of a feature
// may hit the same bin: the r = 1 lane then hands its (g, h) to the r = 0 lane (one
// shuffle) and skips, so the 32 addresses of an instruction are distinct and the
// update is race-free; successive row pairs are ordered by the warp's program order.
// Both lanes of a feature share a bank pair, but a 64-bit access is served per half
// warp, so there is no conflict. A warp walks rows in blocks of 32: lane i fetches the
// row id and (g, h) of row i, every lane its feature's bin byte of its 16 rows; the bytes
// of the next block are in flight while the current block is applied. Warp 2s + h takes
// half h of the group on the s-th share of the CTA's rows; the CTAs of a cluster split
// the unit's rows, and at the end CTA r sums its slice of bins over every warp of every
// CTA of the cluster (distributed shared memory) into the unit's FP32 partial.
template <typename GH>
__global__ void __launch_bounds__(512, 1) level_hist_wp_kernel(const uint8_t* __restrict__ bins, int64_t n, int G,
                                                               int F, const uint32_t* __restrict__ order,
                                                               const GH* __restrict__ g, const GH* __restrict__ h,
                                                               const Plan* __restrict__ plan, int max_bins,
                                                               float* __restrict__ partials) {
  namespace cgr = cooperative_groups;
  extern __shared__ __align__(16) float2 wsh[];   // [W][max_bins][16]
  constexpr int MAX_CS = 16;
  constexpr unsigned FULL = 0xffffffffu;
  cgr::cluster_group cl = cgr::this_cluster();
  const int cs = static_cast<int>(cl.num_blocks());
  const int rank = static_cast<int>(cl.block_rank());
  const int cid = blockIdx.x / cs, ncl = gridDim.x / cs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int half = warp & 1, share = warp >> 1, shares = W >> 1;
  const int r = lane >> 4, f = lane & 15;
  const int per_warp = max_bins * WP_FEATS;
  float2* my = wsh + static_cast<int64_t>(warp) * per_warp;
  const int maxb1 = max_bins - 1;
  const float2* peer[MAX_CS];
  for (int c = 0; c < cs && c < MAX_CS; ++c) peer[c] = cl.map_shared_rank(wsh, c);
  const int total_items = plan->total_units * G;
  const int n_small = plan->n_small;
  for (int item = cid; item < total_items; item += ncl) {
    const int unit = item / G, grp = item - unit * G;
    int lo = 0, hi = n_small - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (plan->unit_begin[mid] <= unit) lo = mid; else hi = mid - 1;
    }
    const int jj = lo;
    const int chunk = unit - plan->unit_begin[jj];
    const int seg_s = plan->seg_start[jj], seg_c = plan->seg_cnt[jj];
    const int cr = plan->chunk_rows[jj];
    const int p0 = seg_s + (chunk * cs + rank) * cr;
    const int p1 = min(seg_s + seg_c, p0 + cr);
    for (int i = lane; i < per_warp; i += 32) my[i] = make_float2(0.f, 0.f);
    __syncwarp();
    const int nblk = p1 > p0 ? (p1 - p0 + 31) / 32 : 0;
    const bool active = grp * GROUP + half * WP_FEATS < F;   // a half holding only padding is skipped
    const uint8_t* gb = bins + static_cast<int64_t>(grp) * n * GROUP + half * WP_FEATS + f;
    auto load_rows = [&](int k, uint32_t& row, float& gv, float& hv) {
      const int blk = share + k * shares;
      const int pos = p0 + blk * 32 + lane;
      if (blk < nblk && pos < p1) {
        row = order ? order[pos] : static_cast<uint32_t>(pos);
        gv = cbgd::load_gh(g, row);
        hv = cbgd::load_gh(h, row);
      } else {
        row = 0;       // a valid address; zero (g, h) make its updates no-ops
        gv = 0.f;
        hv = 0.f;
      }
    };
    auto load_bins = [&](uint32_t row_lane, uint8_t (&raw)[16]) {
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const uint32_t rr = __shfl_sync(FULL, row_lane, 2 * p + r);
        raw[p] = __ldg(gb + static_cast<int64_t>(rr) * GROUP);
      }
    };
    auto process = [&](const uint8_t (&raw)[16], float gl, float hl) {
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const int b = min(static_cast<int>(raw[p]), maxb1);
        const int bp = __shfl_xor_sync(FULL, b, 16);
        float gv = __shfl_sync(FULL, gl, 2 * p + r);
        float hv = __shfl_sync(FULL, hl, 2 * p + r);
        const float gp = __shfl_xor_sync(FULL, gv, 16);
        const float hp = __shfl_xor_sync(FULL, hv, 16);
        const bool dup = b == bp;
        if (dup && r == 0) {
          gv += gp;
          hv += hp;
        }
        if (!(dup && r == 1)) {
          float2* a = my + b * WP_FEATS + f;
          float2 o = *a;
          o.x += gv;
          o.y += hv;
          *a = o;
        }
      }
    };
    const int my_blocks = nblk > share ? (nblk - share + shares - 1) / shares : 0;
    if (active && my_blocks > 0) {
      uint32_t rowA, rowB, rowC;
      float gA, hA, gB, hB, gC, hC;
      uint8_t rawA[16], rawB[16];
      load_rows(0, rowA, gA, hA);
      load_rows(1, rowB, gB, hB);
      load_bins(rowA, rawA);
      for (int k = 0; k < my_blocks; ++k) {
        load_rows(k + 2, rowC, gC, hC);
        if (k + 1 < my_blocks) load_bins(rowB, rawB);
        process(rawA, gA, hA);
#pragma unroll
        for (int i = 0; i < 16; ++i) rawA[i] = rawB[i];
        gA = gB; hA = hB; rowB = rowC; gB = gC; hB = hC;
      }
    }
    cl.sync();
    const int bs = (max_bins + cs - 1) / cs;
    const int b0 = rank * bs;
    const int nbs = max(0, min(max_bins, b0 + bs) - b0);
    float* dst = partials + static_cast<int64_t>(item) * (2 * max_bins * GROUP);
    for (int i = threadIdx.x; i < nbs * GROUP; i += blockDim.x) {
      const int b = b0 + i / GROUP, f32 = i % GROUP;
      const int hw = f32 / WP_FEATS, fl = f32 % WP_FEATS;
      const int64_t e = static_cast<int64_t>(b) * WP_FEATS + fl;
      float sx = 0.f, sy = 0.f;
      for (int c = 0; c < cs; ++c)
        for (int sh = 0; sh < shares; ++sh) {
          const float2 v = peer[c][static_cast<int64_t>(2 * sh + hw) * per_warp + e];
          sx += v.x;
          sy += v.y;
        }
      dst[b * GROUP + f32] = sx;
      dst[max_bins * GROUP + b * GROUP + f32] = sy;
    }
    cl.sync();
  }
}

// ------------------------------------------------------------ reduce + subtract
// One thread per (direct leaf jj, feature f, stat, bin): FP64 sum of the item partials,
// written to the leaf; the sibling gets parent - direct. For the feature the parent was
// split on, both children follow exactly from the parent (bins <= k stay in child 0, the
// rest in child 1), so their empty bins are exact zeros rather than rounding residue.
__global__ void reduce_kernel(const Plan* __restrict__ plan, const float* __restrict__ partials, int G, int F,
                              int max_bins, const double* __restrict__ hist_prev, double* __restrict__ hist_cur,
                              const cbg_split* __restrict__ splits, int depth) {
  const int jj = blockIdx.y;
  if (jj >= plan->n_small) return;
  const int per_leaf = G * 2 * max_bins * GROUP;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= per_leaf) return;
  const int grp = e / (2 * max_bins * GROUP);
  const int rem = e - grp * (2 * max_bins * GROUP);
  const int st = rem / (max_bins * GROUP);
  const int rem2 = rem - st * (max_bins * GROUP);
  const int b = rem2 / GROUP, fl = rem2 - b * GROUP;
  const int f = grp * GROUP + fl;
  if (f >= F) return;
  const int leaf = plan->small_leaf[jj];
  const int large = plan->large_leaf[jj];
  const int64_t cell = ((static_cast<int64_t>(leaf) * F + f) * max_bins + b) * 2 + st;
  if (large >= 0 && depth > 0 && splits[depth - 1].feature == f) {
    const int k = splits[depth - 1].border;
    const int64_t pcell = ((static_cast<int64_t>(plan->parent[jj]) * F + f) * max_bins + b) * 2 + st;
    const int64_t lcell = ((static_cast<int64_t>(large) * F + f) * max_bins + b) * 2 + st;
    const double pv = hist_prev[pcell];
    const bool small_is_child0 = leaf < (1 << (depth - 1));
    const bool in_child0 = b <= k;
    hist_cur[cell] = (in_child0 == small_is_child0) ? pv : 0.0;
    hist_cur[lcell] = (in_child0 == small_is_child0) ? 0.0 : pv;
    return;
  }
  const int u0 = plan->unit_begin[jj], u1 = plan->unit_begin[jj + 1];
  double s = 0.0;
  for (int u = u0; u < u1; ++u)
    s += static_cast<double>(partials[(static_cast<int64_t>(u) * G + grp) * (2 * max_bins * GROUP) + rem]);
  hist_cur[cell] = s;
  if (large >= 0) {
    const int64_t pcell = ((static_cast<int64_t>(plan->parent[jj]) * F + f) * max_bins + b) * 2 + st;
    const int64_t lcell = ((static_cast<int64_t>(large) * F + f) * max_bins + b) * 2 + st;
    hist_cur[lcell] = hist_prev[pcell] - s;
  }
}

// Launch geometry of the histogram kernel for one (bins allocation, threads, cluster
// size, gh type): the cluster size actually used and the number of co-resident
// clusters. Queried once per geometry through the occupancy API and cached.
struct HistGeom {
  int cs = 1;
  int clusters = 0;
};

template <typename GH, int NB, int MODE>
cbg_status hist_geom_for(cbg_ctx* ctx, const HistConfig& L, HistGeom* out) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, HistGeom> cache;
  const auto key = std::make_tuple(ctx->device, NB, L.threads, L.cluster, static_cast<int>(sizeof(GH)));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return CBG_OK;
    }
  }
  auto kern = level_hist_kernel<GH, NB, MODE>;
  const size_t smem = hist_smem_bytes(NB);
  CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  HistGeom geom;
  for (int cs = L.cluster; cs >= 1; cs >>= 1) {
    if (cs > 8) CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(cs * ctx->num_sms));
    cfg.blockDim = dim3(static_cast<unsigned>(L.threads));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) {
      cudaGetLastError();
      clusters = 0;
    }
    if (clusters > 0) {
      geom.cs = cs;
      geom.clusters = clusters;
      break;
    }
  }
  if (geom.clusters == 0) return ::cbg::fail(ctx, CBG_EUNSUPPORTED, "no co-resident histogram cluster fits on this device");
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = geom;
  *out = geom;
  return CBG_OK;
}

template <typename GH, int MODE>
cbg_status hist_geom_mode(cbg_ctx* ctx, const HistConfig& L, HistGeom* g) {
  switch (L.nb_alloc) {
    case 2: return hist_geom_for<GH, 2, MODE>(ctx, L, g);
    case 4: return hist_geom_for<GH, 4, MODE>(ctx, L, g);
    case 8: return hist_geom_for<GH, 8, MODE>(ctx, L, g);
    case 16: return hist_geom_for<GH, 16, MODE>(ctx, L, g);
    case 32: return hist_geom_for<GH, 32, MODE>(ctx, L, g);
    case 64: return hist_geom_for<GH, 64, MODE>(ctx, L, g);
    case 128: return hist_geom_for<GH, 128, MODE>(ctx, L, g);
    case 256: return hist_geom_for<GH, 256, MODE>(ctx, L, g);
    default: return ::cbg::fail(ctx, CBG_EINVAL, "unsupported bin allocation %d", L.nb_alloc);
  }
}

template <typename GH>
cbg_status hist_geom(cbg_ctx* ctx, const HistConfig& L, HistGeom* g) {
  return L.kind == 3 ? hist_geom_mode<GH, 1>(ctx, L, g) : hist_geom_mode<GH, 0>(ctx, L, g);
}

template <typename GH>
cbg_status wp_geom(cbg_ctx* ctx, const HistConfig& L, HistGeom* out) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, HistGeom> cache;
  const int warps = wp_warps(L.max_bins, L.threads);
  const auto key = std::make_tuple(ctx->device, L.max_bins, warps, L.cluster, static_cast<int>(sizeof(GH)));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return CBG_OK;
    }
  }
  auto kern = level_hist_wp_kernel<GH>;
  const size_t smem = wp_smem_bytes(L.max_bins, warps);
  // one attribute for every histogram size this kernel is launched with
  CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  HistGeom geom;
  // the cluster size (<= the requested one) that keeps the most CTAs co-resident
  for (int cs = L.cluster; cs >= 1; cs >>= 1) {
    if (cs > 8) CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(cs * ctx->num_sms));
    cfg.blockDim = dim3(static_cast<unsigned>(32 * warps));
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) {
      cudaGetLastError();
      clusters = 0;
    }
    if (clusters * cs > geom.clusters * geom.cs) {
      geom.cs = cs;
      geom.clusters = clusters;
    }
  }
  if (geom.clusters == 0) return ::cbg::fail(ctx, CBG_EUNSUPPORTED, "no co-resident histogram cluster fits on this device");
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = geom;
  *out = geom;
  return CBG_OK;
}

// The cluster size the plan must chunk for (identical for FP32 and BF16 gradients).
cbg_status hist_cluster_size(cbg_ctx* ctx, const HistConfig& L, int* cs) {
  HistGeom g;
  cbg_status st = L.kind == 0 ? wp_geom<float>(ctx, L, &g) : hist_geom<float>(ctx, L, &g);
  if (st != CBG_OK) return st;
  *cs = g.cs;
  return CBG_OK;
}

template <typename GH, int NB, int MODE>
cbg_status launch_hist_nb(cbg_ctx* ctx, const HistConfig& L, const uint8_t* bins, const uint32_t* order, const GH* g,
                          const GH* h, const Plan* plan, float* partials, int cs_plan) {
  HistGeom geom;
  cbg_status st = hist_geom_for<GH, NB, MODE>(ctx, L, &geom);
  if (st != CBG_OK) return st;
  if (geom.cs != cs_plan) return ::cbg::fail(ctx, CBG_ECUDA, "histogram cluster size changed between plan and launch");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(geom.cs * geom.clusters));
  cfg.blockDim = dim3(static_cast<unsigned>(L.threads));
  cfg.dynamicSmemBytes = hist_smem_bytes(NB);
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(geom.cs);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CBG_CUDA(ctx, cudaLaunchKernelEx(&cfg, level_hist_kernel<GH, NB, MODE>, bins, L.n, L.G, L.F, order, g, h, plan,
                                   L.max_bins, partials));
  return CBG_OK;
}

template <typename GH>
cbg_status launch_hist(cbg_ctx* ctx, const HistConfig& L, const uint8_t* bins, const uint32_t* order, const void* g,
                       const void* h, const Plan* plan, float* partials) {
  int cs = 1;
  cbg_status st = hist_cluster_size(ctx, L, &cs);
  if (st != CBG_OK) return st;
  const GH* gg = static_cast<const GH*>(g);
  const GH* hh = static_cast<const GH*>(h);
  if (L.kind == 0) {
    HistGeom geom;
    st = wp_geom<GH>(ctx, L, &geom);
    if (st != CBG_OK) return st;
    if (geom.cs != cs) return ::cbg::fail(ctx, CBG_ECUDA, "histogram cluster size changed between plan and launch");
    const int warps = wp_warps(L.max_bins, L.threads);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(geom.cs * geom.clusters));
    cfg.blockDim = dim3(static_cast<unsigned>(32 * warps));
    cfg.dynamicSmemBytes = wp_smem_bytes(L.max_bins, warps);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(geom.cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CBG_CUDA(ctx, cudaLaunchKernelEx(&cfg, level_hist_wp_kernel<GH>, bins, L.n, L.G, L.F, order, gg, hh, plan,
                                     L.max_bins, partials));
    return CBG_OK;
  }
  if (L.kind == 3) {
    switch (L.nb_alloc) {
      case 2: return launch_hist_nb<GH, 2, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 4: return launch_hist_nb<GH, 4, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 8: return launch_hist_nb<GH, 8, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 16: return launch_hist_nb<GH, 16, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 32: return launch_hist_nb<GH, 32, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 64: return launch_hist_nb<GH, 64, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 128: return launch_hist_nb<GH, 128, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 256: return launch_hist_nb<GH, 256, 1>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      default: return ::cbg::fail(ctx, CBG_EINVAL, "unsupported bin allocation %d", L.nb_alloc);
    }
  }
  switch (L.nb_alloc) {
    case 2: return launch_hist_nb<GH, 2, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 4: return launch_hist_nb<GH, 4, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 8: return launch_hist_nb<GH, 8, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 16: return launch_hist_nb<GH, 16, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 32: return launch_hist_nb<GH, 32, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 64: return launch_hist_nb<GH, 64, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 128: return launch_hist_nb<GH, 128, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 256: return launch_hist_nb<GH, 256, 0>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    default: return ::cbg::fail(ctx, CBG_EINVAL, "unsupported bin allocation %d", L.nb_alloc);
  }
}

}  // namespace
