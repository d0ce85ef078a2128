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

// What the histogram launch needs to know about a problem.
struct HistConfig {
  int64_t n;
  int G, F, max_bins, nb_alloc, threads, cluster;
};

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
template <typename GH, int NB>
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
          const uint32_t a = off[l] + b * (GROUP * 4);
          red_add(a, gv);
          red_add(a + PLANE * 4, hv);
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
      const int e = st * PLANE + b0 * GROUP + rem;
      float v = 0.f;
      for (int r = 0; r < cs; ++r) v += peer[r][e];
      dst[st * (max_bins * GROUP) + b0 * GROUP + rem] = v;
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

template <typename GH, int NB>
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
  auto kern = level_hist_kernel<GH, NB>;
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

template <typename GH>
cbg_status hist_geom(cbg_ctx* ctx, const HistConfig& L, HistGeom* g) {
  switch (L.nb_alloc) {
    case 2: return hist_geom_for<GH, 2>(ctx, L, g);
    case 4: return hist_geom_for<GH, 4>(ctx, L, g);
    case 8: return hist_geom_for<GH, 8>(ctx, L, g);
    case 16: return hist_geom_for<GH, 16>(ctx, L, g);
    case 32: return hist_geom_for<GH, 32>(ctx, L, g);
    case 64: return hist_geom_for<GH, 64>(ctx, L, g);
    case 128: return hist_geom_for<GH, 128>(ctx, L, g);
    case 256: return hist_geom_for<GH, 256>(ctx, L, g);
    default: return ::cbg::fail(ctx, CBG_EINVAL, "unsupported bin allocation %d", L.nb_alloc);
  }
}

// The cluster size the plan must chunk for (identical for FP32 and BF16 gradients).
cbg_status hist_cluster_size(cbg_ctx* ctx, const HistConfig& L, int* cs) {
  HistGeom g;
  cbg_status st = hist_geom<float>(ctx, L, &g);
  if (st != CBG_OK) return st;
  *cs = g.cs;
  return CBG_OK;
}

template <typename GH, int NB>
cbg_status launch_hist_nb(cbg_ctx* ctx, const HistConfig& L, const uint8_t* bins, const uint32_t* order, const GH* g,
                          const GH* h, const Plan* plan, float* partials, int cs_plan) {
  HistGeom geom;
  cbg_status st = hist_geom_for<GH, NB>(ctx, L, &geom);
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
  CBG_CUDA(ctx, cudaLaunchKernelEx(&cfg, level_hist_kernel<GH, NB>, bins, L.n, L.G, L.F, order, g, h, plan,
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
  switch (L.nb_alloc) {
    case 2: return launch_hist_nb<GH, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 4: return launch_hist_nb<GH, 4>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 8: return launch_hist_nb<GH, 8>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 16: return launch_hist_nb<GH, 16>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 32: return launch_hist_nb<GH, 32>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 64: return launch_hist_nb<GH, 64>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 128: return launch_hist_nb<GH, 128>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    case 256: return launch_hist_nb<GH, 256>(ctx, L, bins, order, gg, hh, plan, partials, cs);
    default: return ::cbg::fail(ctx, CBG_EINVAL, "unsupported bin allocation %d", L.nb_alloc);
  }
}

}  // namespace
