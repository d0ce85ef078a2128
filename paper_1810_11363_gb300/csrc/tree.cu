// Per-tree hot path: gradients, per-level histograms, split scoring, leaf update and row
// partition, leaf values and prediction update (Sections 3 and 4 of the paper).
//
// Data layout in HBM
//   bins      grouped uint8: feature f of row r at ((f/32)*n + r)*32 + f%32, so one
//             32-feature group of one row is one 32-byte sector.
//   order     uint32 [n]: rows grouped by leaf (stable), rebuilt every level.
//   hist      FP64 [2^d][F][max_bins][2] (G, H) per level; the previous level's
//             histogram is kept to obtain one sibling of each pair by subtraction.
//   partials  FP32 [item][2][max_bins][32]: one shared-memory histogram per work item.
#include "cbg_internal.cuh"
#include "level_hist.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

using namespace cbg;

namespace {

constexpr int PT = 2048;           // positions per partition tile (256 threads x 8)
constexpr int PT_THREADS = 256;
constexpr int PT_PER_THREAD = PT / PT_THREADS;   // consecutive positions of a thread


struct Segs {                       // row segments of the leaves of one level
  int start[1 << MAX_DEPTH];
  int cnt[1 << MAX_DEPTH];
  int order[1 << MAX_DEPTH];        // leaf ids in memory order of their segments
  unsigned ones[1 << MAX_DEPTH];    // rows of the leaf sent to the "1" side
  unsigned ones_before[1 << MAX_DEPTH];
};

struct BestF {
  double score;
  int k;
  int pad;
};

struct Layout {
  int64_t n;
  int F, F_pad, G, max_bins, nb_alloc, D;
  int rows_per_item, threads, blocks_per_sm, cluster, kind;
  int64_t max_items;
  int64_t n_ptiles;
  size_t hist_elems;                // per hist buffer (doubles)
  size_t part_elems_item;           // floats per partial item
  // byte offsets
  size_t o_order_a, o_order_b, o_flags, o_tcnt, o_toff, o_seg_a, o_seg_b, o_plan, o_hist_a, o_hist_b,
      o_part, o_best, o_misc, o_count, o_hdf, o_gsplit, o_gvals, o_gp_a, o_gp_b, o_hp_a, o_hp_b,
      total;
};

int pow2_at_least(int v) {
  int p = 2;
  while (p < v) p <<= 1;
  return p;
}


cbg_status make_layout(cbg_ctx* ctx, const cbg_tree_shape* s, Layout* L) {
  CBG_REQUIRE(ctx, s != nullptr, "shape is NULL");
  CBG_REQUIRE(ctx, s->n >= 1 && s->n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, s->F >= 1, "F must be >= 1");
  CBG_REQUIRE(ctx, s->F_pad >= s->F && s->F_pad % GROUP == 0, "F_pad must be a multiple of 32 and >= F");
  CBG_REQUIRE(ctx, s->max_bins >= 1 && s->max_bins <= 256, "max_bins must be in [1, 256]");
  CBG_REQUIRE(ctx, s->max_depth >= 1 && s->max_depth <= MAX_DEPTH, "max_depth must be in [1, 10]");
  const cbg_tiles& t = s->tiles;
  CBG_REQUIRE(ctx, t.slab_chunks == 0 || t.slab_chunks == 2, "slab_chunks must be 0 (default) or 2");
  CBG_REQUIRE(ctx, t.rows_per_item >= 0 && t.threads >= 0 && t.blocks_per_sm >= 0, "negative tile field");
  CBG_REQUIRE(ctx, t.threads % 32 == 0 && t.threads <= 512, "threads must be a multiple of 32, <= 512");
  L->n = s->n;
  L->F = s->F;
  L->F_pad = s->F_pad;
  L->G = s->F_pad / GROUP;
  L->max_bins = std::max(2, s->max_bins);
  L->nb_alloc = pow2_at_least(L->max_bins);
  L->D = s->max_depth;
  CBG_REQUIRE(ctx, t.cluster >= 0 && t.cluster <= 16, "cluster must be in [0, 16]");
  CBG_REQUIRE(ctx, t.kernel >= 0 && t.kernel <= 9, "kernel must be 0 (default), 1 (shared reductions), 2 "
              "(warp-private, 16 features per warp), 3 (64-bit compare-and-swap), 4 (lane per feature), 5 (lane "
              "per feature, one statistic per warp), 6 (lane per feature over 4-bit packed bins), 7 (shared "
              "integer reductions of fixed-point values), 8 (lane per feature with loader warps) or 9 (1-bit "
              "binary features)");
  CBG_REQUIRE(ctx, t.kernel != 6 || s->max_bins <= 16, "the 4-bit packed kernel needs max_bins <= 16");
  CBG_REQUIRE(ctx, t.kernel != 9 || s->max_bins <= 2, "the 1-bit kernel needs max_bins <= 2");
  L->kind = t.kernel == 2 ? 0 : (t.kernel >= 3 ? t.kernel : 1);
  const bool lane_kind = L->kind == 4 || L->kind == 5 || L->kind == 6 || L->kind == 8 || L->kind == 9;
  const bool fixed_kind = L->kind == 7;
  L->rows_per_item = t.rows_per_item > 0 ? t.rows_per_item : (lane_kind ? 8192 : fixed_kind ? 4096 : 2048);
  L->cluster = t.cluster > 0 ? t.cluster : (lane_kind ? 2 : fixed_kind ? 4 : 8);
  L->threads = t.threads > 0 ? t.threads : 512;
  const int fit = static_cast<int>(SMEM_DYN_BUDGET / hist_smem_bytes(L->nb_alloc));
  L->blocks_per_sm = std::max(1, std::min(t.blocks_per_sm > 0 ? t.blocks_per_sm : 3, fit));
  const int hleaves = 1 << (L->D - 1);
  L->max_items = static_cast<int64_t>(L->G) * (ceil_div(L->n, L->rows_per_item) + hleaves + 1);
  L->n_ptiles = ceil_div(L->n, PT);
  L->hist_elems = static_cast<size_t>(hleaves) * L->F * L->max_bins * 2;
  L->part_elems_item = static_cast<size_t>(2) * L->max_bins * GROUP;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) / 256 * 256;
    size_t o = off;
    off += bytes;
    return o;
  };
  L->o_order_a = take(L->n * 4);
  L->o_order_b = take(L->n * 4);
  L->o_flags = take(L->n);
  L->o_tcnt = take((L->n_ptiles + 1) * 4);
  L->o_toff = take((L->n_ptiles + 1) * 4);
  L->o_seg_a = take(sizeof(Segs));
  L->o_seg_b = take(sizeof(Segs));
  L->o_plan = take(sizeof(Plan));
  L->o_hist_a = take(L->hist_elems * 8);
  L->o_hist_b = take(L->hist_elems * 8);
  L->o_part = take(static_cast<size_t>(L->max_items) * L->part_elems_item * 4);
  L->o_hdf = take(L->hist_elems * sizeof(float2));   // (hi, lo) FP32 copy of the current level's histogram
  L->o_best = take(static_cast<size_t>(L->F) * sizeof(BestF) + 64);
  L->o_misc = take(256);
  L->o_count = take(256);
  L->o_gsplit = take(sizeof(cbg_split) * MAX_DEPTH + 256);   // per-tree outputs while replaying a graph
  L->o_gvals = take(sizeof(double) * (static_cast<size_t>(1) << L->D));
  // (g, h) in the row order of each level (position order), for the kernel that reads
  // them by position; 4 bytes per row covers both FP32 and BF16
  L->o_gp_a = take(L->n * 4);
  L->o_gp_b = take(L->n * 4);
  L->o_hp_a = take(L->n * 4);
  L->o_hp_b = take(L->n * 4);
  L->total = take(0) + 256;
  return CBG_OK;
}

HistConfig hist_config(const Layout& L) {
  HistConfig c;
  c.n = L.n;
  c.G = L.G;
  c.F = L.F;
  c.max_bins = L.max_bins;
  c.nb_alloc = L.nb_alloc;
  c.threads = L.threads;
  c.cluster = L.cluster;
  c.kind = L.kind;
  return c;
}

template <typename T>
T* at(void* state, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(state) + off);
}

struct Misc {
  unsigned done;        // blocks finished in the argmax kernel (reset by the last one)
  unsigned done_part;   // blocks finished in the partition-flags kernel (reset by the last one)
  double forced_score;
};

// ------------------------------------------------------------------ gradients
template <typename GH>
__global__ void gradients_kernel(int loss, const float* __restrict__ y, const float* __restrict__ pred, int64_t n,
                                 GH* __restrict__ g, GH* __restrict__ h) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float p = pred[i], yi = y[i], gi, hi;
    if (loss == CBG_LOSS_RMSE) {
      gi = p - yi;
      hi = 1.0f;
    } else {
      float s = 1.0f / (1.0f + expf(-p));
      gi = s - yi;
      hi = s * (1.0f - s);
    }
    cbgd::store_gh(g, i, gi);
    cbgd::store_gh(h, i, hi);
  }
}

unsigned grid_stride_blocks(int64_t n, int block) {
  int64_t g = ceil_div(n, block);
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(g, 152LL * 64)));
}

// ------------------------------------------------------------------ tree begin
// The root's plan and segment (one thread): every row in leaf 0, chunked into units.
// Rows of one work unit (its cs CTAs together) for a level whose directly computed
// leaves hold `rows` rows: rows_per_item per CTA of the unit, or more when the level has
// so many rows that this would give more than target_units units (larger units then
// write fewer partials, and the launch's queue still has several items per cluster).
// target_units = 0 keeps rows_per_item x cs.
__device__ __forceinline__ int unit_rows(long long rows, int rows_per_item, int cs, int target_units) {
  const long long floor_rows = static_cast<long long>(rows_per_item) * cs;
  if (target_units <= 0) return static_cast<int>(floor_rows);
  const long long r = (rows + target_units - 1) / target_units;
  return static_cast<int>(r > floor_rows ? r : floor_rows);
}

__device__ void tree_begin_body(Plan* plan, Segs* seg, int n, int rows_per_item, int cs, int target_units,
                                unsigned long long* rows_hist) {
  *rows_hist += static_cast<unsigned long long>(n);
  const int per_unit = unit_rows(n, rows_per_item, cs, target_units);
  int chunks = (n + per_unit - 1) / per_unit;
  if (chunks < 1) chunks = 1;
  plan->queue = 0;
  plan->rqueue = 0;
  plan->done[0] = 0;
  plan->n_small = 1;
  plan->total_units = chunks;
  plan->level_leaves = 1;
  plan->small_leaf[0] = 0;
  plan->large_leaf[0] = -1;
  plan->parent[0] = -1;
  plan->unit_begin[0] = 0;
  plan->unit_begin[1] = chunks;
  plan->chunk_rows[0] = (n + chunks * cs - 1) / (chunks * cs);
  plan->seg_start[0] = 0;
  plan->seg_cnt[0] = n;
  seg->start[0] = 0;
  seg->cnt[0] = n;
  seg->order[0] = 0;
}

__global__ void tree_begin_kernel(Plan* plan, Segs* seg, int n, int rows_per_item, int cs, int target_units,
                                  unsigned long long* rows_hist) {
  if (threadIdx.x == 0 && blockIdx.x == 0) tree_begin_body(plan, seg, n, rows_per_item, cs, target_units, rows_hist);
}

// ----------------------------------------------------------------- scoring
// GB300 runs FP64 at a small fraction of the FP32 rate, so FP64 is kept to what the
// precision needs: prefix sums over bins in FP64, then the candidate terms
// G^2/(H + l2) in FP32 and their sum over leaves with compensated FP32 addition.

__device__ __forceinline__ float score_term_f(float G, float H, float l2) {
  const float den = H + l2;
  return den == 0.0f ? 0.0f : G * G / den;
}

// Compensated FP32 pair (hi + lo): about 2^-44 relative precision on the FP32 pipe.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return DF{hi, e - (hi - s)};
}

__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }

__device__ __forceinline__ DF df_shfl_up(DF v, int o) {
  return DF{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ DF df_shfl(DF v, int src) {
  return DF{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

__device__ __forceinline__ bool better(double s, int k, double bs, int bk) {
  return s > bs || (s == bs && k < bk);
}

// Split scoring of one level in one kernel, a block per feature (Sections 3-4: one split
// per level, scored over every leaf of the level). It reads the compensated FP32 copy
// (hi, lo) of the FP64 histogram that the reduction writes, so it runs on the FP32 pipe
// alone (GB300 executes FP64 at 1/64 of the FP32 rate).
//  - A block has min(16, 2^d) warps; warp w takes leaves w, w + warps, ... For each it
//    forms compensated prefix sums
//    over bins (lane i owns bins [8i, 8i + 8), then a warp scan), so G_L(k), H_L(k) and
//    the leaf totals come out at about 2^-44 relative, and adds the FP32 term
//    G_L^2/(H_L+l2) + G_R^2/(H_R+l2) of every border to its own compensated accumulators.
//  - The warps' accumulators are added in warp order (compensated); the block keeps its
//    best border.
//  - The last block to finish picks the best feature (ties to the smallest f, then k) and
//    writes the split.
constexpr int SC_MAX_WARPS = 16;
constexpr int SC_BINS_PER_LANE = 8;   // 32 lanes x 8 = 256 bins

template <int SC_WARPS>
__device__ __forceinline__ void score_level_body(const float2* __restrict__ hist_df, int level_leaves, int F, int max_bins,
                       const int32_t* __restrict__ n_borders, double l2, BestF* __restrict__ best, Misc* misc,
                       int force_f, int force_k, int depth, cbg_split* __restrict__ splits, int bid, int nblk,
                       const cbg_split* __restrict__ chal) {
  constexpr int NT = SC_WARPS * 32;
  __shared__ DF s_acc[SC_WARPS][256];
  __shared__ double r_s[NT];
  __shared__ int r_f[NT], r_k[NT];
  __shared__ bool is_last;
  const int f = bid, K = max_bins - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = min(n_borders[f], K);
  const float l2f = static_cast<float>(l2);
  DF acc[SC_BINS_PER_LANE];
#pragma unroll
  for (int i = 0; i < SC_BINS_PER_LANE; ++i) acc[i] = DF{0.f, 0.f};
  if (nb > 0) {
    for (int l = warp; l < level_leaves; l += SC_WARPS) {
      const float4* hl = reinterpret_cast<const float4*>(hist_df + (static_cast<int64_t>(l) * F + f) * max_bins * 2);
      DF g[SC_BINS_PER_LANE], h[SC_BINS_PER_LANE];
      DF sg{0.f, 0.f}, sh{0.f, 0.f};
#pragma unroll
      for (int i = 0; i < SC_BINS_PER_LANE; ++i) {
        const int b = lane * SC_BINS_PER_LANE + i;
        const float4 v = b < max_bins ? hl[b] : make_float4(0.f, 0.f, 0.f, 0.f);   // (G hi, G lo, H hi, H lo)
        sg = df_add(sg, DF{v.x, v.y});
        sh = df_add(sh, DF{v.z, v.w});
        g[i] = sg;   // inclusive prefix within the lane
        h[i] = sh;
      }
      DF ig = sg, ih = sh;   // inclusive scan of the lane totals
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const DF ug = df_shfl_up(ig, o), uh = df_shfl_up(ih, o);
        if (lane >= o) {
          ig = df_add(ug, ig);
          ih = df_add(uh, ih);
        }
      }
      const DF tg = df_shfl(ig, 31), th = df_shfl(ih, 31);
      DF eg = df_shfl_up(ig, 1), eh = df_shfl_up(ih, 1);
      if (lane == 0) eg = eh = DF{0.f, 0.f};
#pragma unroll
      for (int i = 0; i < SC_BINS_PER_LANE; ++i) {
        const int k = lane * SC_BINS_PER_LANE + i;
        if (k < nb) {
          const DF GL = df_add(eg, g[i]), HL = df_add(eh, h[i]);
          const DF GR = df_sub(tg, GL), HR = df_sub(th, HL);
          const float t = score_term_f(GL.hi + GL.lo, HL.hi + HL.lo, l2f) +
                          score_term_f(GR.hi + GR.lo, HR.hi + HR.lo, l2f);
          acc[i] = df_add(acc[i], DF{t, 0.f});
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < SC_BINS_PER_LANE; ++i) s_acc[warp][lane * SC_BINS_PER_LANE + i] = acc[i];
  __syncthreads();
  double bs = -INFINITY;
  int bk = -1;
  for (int k = threadIdx.x; k < nb; k += NT) {
    DF t = s_acc[0][k];
    for (int w = 1; w < SC_WARPS; ++w) t = df_add(t, s_acc[w][k]);
    const double sc = static_cast<double>(t.hi) + static_cast<double>(t.lo);
    if (f == force_f && k == force_k) misc->forced_score = sc;
    if (bk < 0 || better(sc, k, bs, bk)) {
      bs = sc;
      bk = k;
    }
  }
  __threadfence();   // the forced-score store must be visible before this block is counted
  r_s[threadIdx.x] = bs;
  r_k[threadIdx.x] = bk;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const int ok = r_k[threadIdx.x + o];
      if (ok >= 0 && (r_k[threadIdx.x] < 0 || better(r_s[threadIdx.x + o], ok, r_s[threadIdx.x], r_k[threadIdx.x]))) {
        r_s[threadIdx.x] = r_s[threadIdx.x + o];
        r_k[threadIdx.x] = ok;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    best[f].score = r_s[0];
    best[f].k = r_k[0];
    __threadfence();
    const unsigned ticket = atomicAdd(&misc->done, 1u);
    is_last = (ticket == nblk - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // last block: global argmax over features
  double gbs = -INFINITY;
  int gbf = -1, gbk = -1;
  for (int ff = threadIdx.x; ff < F; ff += NT) {
    const double sc = __ldcg(&best[ff].score);
    const int k = __ldcg(&best[ff].k);
    if (k >= 0 && (gbf < 0 || sc > gbs || (sc == gbs && ff < gbf))) {
      gbs = sc;
      gbf = ff;
      gbk = k;
    }
  }
  r_s[threadIdx.x] = gbs;
  r_f[threadIdx.x] = gbf;
  r_k[threadIdx.x] = gbk;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const int of = r_f[threadIdx.x + o];
      const double os = r_s[threadIdx.x + o];
      const int mf = r_f[threadIdx.x];
      if (of >= 0 && (mf < 0 || os > r_s[threadIdx.x] || (os == r_s[threadIdx.x] && of < mf))) {
        r_s[threadIdx.x] = os;
        r_f[threadIdx.x] = of;
        r_k[threadIdx.x] = r_k[threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int cf = r_f[0], ck = r_k[0];
    double cs = r_s[0];
    if (force_f >= 0) {
      cf = force_f;
      ck = force_k;
      cs = *(volatile double*)&misc->forced_score;
    } else if (chal != nullptr && chal->feature >= 0 && (cf < 0 || chal->score > cs)) {
      // a split on a column outside bins (a feature combination) with a strictly higher score
      cf = chal->feature;
      ck = chal->border;
      cs = chal->score;
    }
    splits[depth].feature = cf;
    splits[depth].border = cf >= 0 ? ck : -1;
    splits[depth].score = cf >= 0 ? cs : -INFINITY;
    misc->done = 0;
  }
}

template <int SC_WARPS>
__global__ void __launch_bounds__(SC_WARPS * 32)
    score_level_kernel(const float2* __restrict__ hist_df, int level_leaves, int F, int max_bins,
                       const int32_t* __restrict__ n_borders, double l2, BestF* __restrict__ best, Misc* misc,
                       int force_f, int force_k, int depth, cbg_split* __restrict__ splits,
                       const cbg_split* __restrict__ chal) {
  score_level_body<SC_WARPS>(hist_df, level_leaves, F, max_bins, n_borders, l2, best, misc, force_f, force_k, depth, splits, blockIdx.x, gridDim.x, chal);
}

// FP64 child totals of the level's split for leaf l, one warp: bins <= k stay in leaf l,
// the rest go to l + 2^d (every row stays in l when no split exists).
__device__ void child_totals_warp(const double* __restrict__ hist, int l, int level_leaves, int F, int max_bins,
                                  int sf, int sk, double* __restrict__ child_totals) {
  const int lane = threadIdx.x & 31;
  const int cf = sf >= 0 ? sf : 0;
  const double2* hl = reinterpret_cast<const double2*>(hist + (static_cast<int64_t>(l) * F + cf) * max_bins * 2);
  double g0 = 0.0, h0 = 0.0, g1 = 0.0, h1 = 0.0;
  for (int b = lane; b < max_bins; b += 32) {
    const double2 v = hl[b];
    if (sf < 0 || b <= sk) {
      g0 += v.x;
      h0 += v.y;
    } else {
      g1 += v.x;
      h1 += v.y;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    g0 += __shfl_down_sync(0xffffffffu, g0, o);
    h0 += __shfl_down_sync(0xffffffffu, h0, o);
    g1 += __shfl_down_sync(0xffffffffu, g1, o);
    h1 += __shfl_down_sync(0xffffffffu, h1, o);
  }
  if (lane == 0) {
    child_totals[2 * l] = g0;
    child_totals[2 * l + 1] = h0;
    child_totals[2 * (l + level_leaves)] = g1;
    child_totals[2 * (l + level_leaves) + 1] = h1;
  }
}

// ---------------------------------------------------------------- partition
__device__ __forceinline__ int split_bit(const uint8_t* bins, const uint8_t* bins_t, int64_t n, uint32_t row,
                                         int f, int k) {
  if (f < 0) return 0;
  uint8_t b = bins_t ? bins_t[static_cast<int64_t>(f) * n + row]
                     : bins[(static_cast<int64_t>(f >> 5) * n + row) * GROUP + (f & 31)];
  return b > k ? 1 : 0;
}

// Plan of the next level, run by one block: exclusive scan of the tile ones, ones before
// every segment, the child segments, and the work units of the next level (the smaller
// child of each pair is histogrammed directly, the other by subtraction).
__device__ void plan_next_level(uint32_t* __restrict__ tile_cnt, int64_t n_ptiles, Segs* __restrict__ cur,
                                Segs* __restrict__ nxt, Plan* __restrict__ plan, int depth, int rows_per_item,
                                int cs, int target_units, unsigned long long* __restrict__ rows_hist) {
  __shared__ uint32_t sh[PT_THREADS / 32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < n_ptiles; b0 += blockDim.x) {
    const int64_t idx = b0 + threadIdx.x;
    uint32_t v = idx < n_ptiles ? __ldcg(tile_cnt + idx) : 0u;
    uint32_t x = v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int w = 0; w < PT_THREADS / 32; ++w) {
        uint32_t t = sh[w];
        sh[w] = run;
        run += t;
      }
    }
    __syncthreads();
    uint32_t excl = carry + sh[warp] + x - v;
    __syncthreads();
    if (idx < n_ptiles) tile_cnt[idx] = excl;   // now the tile offsets
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  __syncthreads();
  // per-parent data, staged in shared memory by all threads: parents in memory order
  // (i) for the ones-before scan, and by leaf id (p) for the child pairs
  constexpr int PER_T = (1 << (MAX_DEPTH - 1)) / PT_THREADS;   // parents per thread
  __shared__ uint32_t s_ones_by_leaf[1 << (MAX_DEPTH - 1)];
  __shared__ uint32_t s_wsum[PT_THREADS / 32];
  const int L = 1 << depth;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < L; i += blockDim.x) s_ones_by_leaf[i] = __ldcg(&cur->ones[i]);
  __syncthreads();
  // block exclusive scan over parents i in memory order (PER_T consecutive per thread)
  auto block_scan = [&](uint32_t (&v)[PER_T], uint32_t& total) {
    uint32_t t = 0;
#pragma unroll
    for (int q = 0; q < PER_T; ++q) t += v[q];
    uint32_t x = t;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    total = 0;
    for (int w = 0; w < PT_THREADS / 32; ++w) {
      if (w < warp) before += s_wsum[w];
      total += s_wsum[w];
    }
    __syncthreads();
    uint32_t run = before + x - t;
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const uint32_t vq = v[q];
      v[q] = run;
      run += vq;
    }
  };
  {
    uint32_t v[PER_T];
    int leaf_of[PER_T];
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const int i = threadIdx.x * PER_T + q;
      leaf_of[q] = i < L ? cur->order[i] : -1;
      v[q] = i < L ? s_ones_by_leaf[leaf_of[q]] : 0u;
    }
    uint32_t total;
    block_scan(v, total);
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const int i = threadIdx.x * PER_T + q;
      if (i >= L) continue;
      const int l = leaf_of[q];
      cur->ones_before[l] = v[q];
      const int st = cur->start[l], c = cur->cnt[l];
      const int c1 = static_cast<int>(s_ones_by_leaf[l]);
      const int c0 = c - c1;
      nxt->start[l] = st;
      nxt->cnt[l] = c0;
      nxt->start[l + L] = st + c0;
      nxt->cnt[l + L] = c1;
      nxt->order[2 * i] = l;
      nxt->order[2 * i + 1] = l + L;
      nxt->ones[l] = 0;
      nxt->ones[l + L] = 0;
    }
  }
  // pair p = children p and p + L of parent p; the smaller one is histogrammed directly.
  // Its rows are cut into units of about the same size over the whole level; the pairs
  // are listed by decreasing rows per CTA, so that a launch hands out its largest work
  // items first.
  {
    __shared__ int s_cr[1 << (MAX_DEPTH - 1)];         // rows per CTA of pair p
    __shared__ int s_chunks_by_rank[1 << (MAX_DEPTH - 1)];
    __shared__ int s_pair_by_rank[1 << (MAX_DEPTH - 1)];
    __shared__ unsigned long long s_rows;
    if (threadIdx.x == 0) s_rows = 0;
    __syncthreads();
    unsigned long long rows = 0;
    for (int p = threadIdx.x; p < L; p += blockDim.x) {
      const int c1 = static_cast<int>(s_ones_by_leaf[p]);
      rows += static_cast<unsigned long long>(min(cur->cnt[p] - c1, c1));
    }
    if (rows) atomicAdd(&s_rows, rows);
    __syncthreads();
    const int per_unit = unit_rows(static_cast<long long>(s_rows), rows_per_item, cs, target_units);
    for (int p = threadIdx.x; p < L; p += blockDim.x) {
      const int c1 = static_cast<int>(s_ones_by_leaf[p]);
      const int m = min(cur->cnt[p] - c1, c1);
      const int chunks = m > per_unit ? (m + per_unit - 1) / per_unit : 1;
      s_cr[p] = m > 0 ? (m + chunks * cs - 1) / (chunks * cs) : 0;
    }
    __syncthreads();
    // rank of pair p: pairs with more rows per CTA first, then by index
    for (int p = threadIdx.x; p < L; p += blockDim.x) {
      const int cr = s_cr[p];
      int rank = 0;
      for (int q = 0; q < L; ++q) rank += (s_cr[q] > cr || (s_cr[q] == cr && q < p)) ? 1 : 0;
      const int c1 = static_cast<int>(s_ones_by_leaf[p]);
      const int m = min(cur->cnt[p] - c1, c1);
      s_chunks_by_rank[rank] = m > per_unit ? (m + per_unit - 1) / per_unit : 1;
      s_pair_by_rank[rank] = p;
    }
    __syncthreads();
    uint32_t v[PER_T];
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const int r = threadIdx.x * PER_T + q;
      v[q] = r < L ? static_cast<uint32_t>(s_chunks_by_rank[r]) : 0u;
    }
    uint32_t units;
    block_scan(v, units);
#pragma unroll
    for (int q = 0; q < PER_T; ++q) {
      const int r = threadIdx.x * PER_T + q;
      if (r >= L) continue;
      const int p = s_pair_by_rank[r];
      const int c = cur->cnt[p];
      const int c1 = static_cast<int>(s_ones_by_leaf[p]);
      const int c0 = c - c1;
      const bool small_is_a = c0 <= c1;   // ties go to child p
      plan->done[r] = 0;
      plan->small_leaf[r] = small_is_a ? p : p + L;
      plan->large_leaf[r] = small_is_a ? p + L : p;
      plan->parent[r] = p;
      plan->unit_begin[r] = static_cast<int>(v[q]);
      plan->chunk_rows[r] = s_cr[p] > 0 ? s_cr[p] : 1;
      plan->seg_start[r] = small_is_a ? cur->start[p] : cur->start[p] + c0;
      plan->seg_cnt[r] = min(c0, c1);
    }
    if (threadIdx.x == 0) {
      atomicAdd(rows_hist, s_rows);
      plan->unit_begin[L] = static_cast<int>(units);
      plan->n_small = L;
      plan->total_units = static_cast<int>(units);
      plan->level_leaves = 2 * L;
      plan->queue = 0;
      plan->rqueue = 0;
    }
  }
}

// The leaf segments of a level in memory order, staged in shared memory: seg_pos[i] is
// the first position of the i-th segment and seg_leaf[i] its leaf. Positions are grouped
// by leaf, so the leaf of a position is found here instead of being read per row.
__device__ void load_seg_table(const Segs* __restrict__ seg, int L, int* seg_pos, int* seg_leaf) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    const int l = seg->order[i];
    seg_leaf[i] = l;
    seg_pos[i] = seg->start[l];
  }
}

// The segment holding position pos: the last i with seg_pos[i] <= pos. An empty segment
// starts where the next one does and comes before it, so it is never the last such i.
__device__ __forceinline__ int seg_find(const int* seg_pos, int L, int64_t pos) {
  int lo = 0, hi = L - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_pos[mid] <= pos) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Row ids of positions base .. base + PT_PER_THREAD - 1 (identity without an order; rows
// past n read as 0 and are not used), in two 16-byte loads where they are whole.
__device__ __forceinline__ void load_rows(const uint32_t* __restrict__ order, int64_t n, int64_t base,
                                          uint32_t (&rows)[PT_PER_THREAD]) {
  static_assert(PT_PER_THREAD == 8, "two 16-byte loads per thread");
  if (order && base + PT_PER_THREAD <= n) {   // order buffers are 256-byte aligned, base a multiple of 8
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(order + base));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(order + base) + 1);
    rows[0] = a.x; rows[1] = a.y; rows[2] = a.z; rows[3] = a.w;
    rows[4] = b.x; rows[5] = b.y; rows[6] = b.z; rows[7] = b.w;
  } else {
#pragma unroll
    for (int i = 0; i < PT_PER_THREAD; ++i)
      rows[i] = base + i >= n ? 0u : order ? __ldg(order + base + i) : static_cast<uint32_t>(base + i);
  }
}

// A: the FP64 child totals of the level's split (one warp per leaf); per position (8
// consecutive positions per thread), the split bit of its row; leaf += 2^d * bit. Unless this is the last level: ones per tile and per leaf (run-length counted
// in shared memory, since positions are grouped by leaf), and the last block to finish
// plans the next level.
__device__ __forceinline__ void part_flags_body(const uint8_t* __restrict__ bins, const uint8_t* __restrict__ bins_t, int64_t n,
                                  const uint32_t* __restrict__ order, const cbg_split* __restrict__ splits, int depth,
                                  uint16_t* __restrict__ leaf, uint8_t* __restrict__ flags,
                                  uint32_t* __restrict__ tile_cnt, Segs* seg, int write_flags, int64_t n_ptiles,
                                  Segs* __restrict__ nxt, Plan* __restrict__ plan, int rows_per_item, int cs,
                                  int target_units,
                                  unsigned long long* __restrict__ rows_hist, Misc* misc,
                                  const double* __restrict__ hist, int F, int max_bins,
                                  double* __restrict__ child_totals, int bid, int nblk,
                                  const uint8_t* __restrict__ chal_bins, const double* __restrict__ chal_hist,
                                  int chal_max_bins) {
  __shared__ uint32_t wsum[PT_THREADS / 32];
  __shared__ uint32_t sh_ones[1 << MAX_DEPTH];
  __shared__ int sh_pos[1 << (MAX_DEPTH - 1)], sh_leaf[1 << (MAX_DEPTH - 1)];
  __shared__ bool is_last;
  const int L = 1 << depth;
  if (write_flags)
    for (int i = threadIdx.x; i < L; i += blockDim.x) sh_ones[i] = 0;
  load_seg_table(seg, L, sh_pos, sh_leaf);
  __syncthreads();
  const int f = splits[depth].feature, k = splits[depth].border;
  // a feature index >= F is the challenger's column (outside bins), with its own histogram
  const bool chal = f >= F && chal_bins != nullptr;
  // the FP64 child totals of the split, one warp per leaf of the level
  for (int l = bid * (PT_THREADS / 32) + (threadIdx.x >> 5); l < L; l += nblk * (PT_THREADS / 32)) {
    if (chal)
      child_totals_warp(chal_hist, l, L, 1, chal_max_bins, 0, k, child_totals);
    else
      child_totals_warp(hist, l, L, F, max_bins, f, k, child_totals);
  }
  const int64_t base = static_cast<int64_t>(bid) * PT + static_cast<int64_t>(threadIdx.x) * PT_PER_THREAD;
  int si = seg_find(sh_pos, L, base);
  uint32_t cnt = 0, run = 0;
  int cur = -1;
  // all row ids of the thread's positions, then all their split bits, so that the loads
  // of each kind are in flight together
  uint32_t rows[PT_PER_THREAD];
  load_rows(order, n, base, rows);
  int bits[PT_PER_THREAD];
#pragma unroll
  for (int i = 0; i < PT_PER_THREAD; ++i)
    bits[i] = base + i >= n ? 0 : chal ? (chal_bins[rows[i]] > k ? 1 : 0) : split_bit(bins, bins_t, n, rows[i], f, k);
  uint32_t fw[PT_PER_THREAD / 4] = {};
#pragma unroll
  for (int i = 0; i < PT_PER_THREAD; ++i) {
    const int64_t pos = base + i;
    if (pos < n) {
      const int bit = bits[i];
      while (si + 1 < L && sh_pos[si + 1] <= pos) ++si;
      const int lf = sh_leaf[si];
      if (bit) leaf[rows[i]] = static_cast<uint16_t>(lf + L);   // rows of leaf lf already hold lf
      if (write_flags) {
        fw[i / 4] |= static_cast<uint32_t>(bit) << (8 * (i % 4));
        if (lf != cur) {
          if (run) atomicAdd(&sh_ones[cur], run);
          cur = lf;
          run = 0;
        }
        run += bit;
        cnt += bit;
      }
    }
  }
  if (write_flags) {
    if (base + PT_PER_THREAD <= n) {
      *reinterpret_cast<uint2*>(flags + base) = make_uint2(fw[0], fw[1]);   // base is a multiple of 8
    } else {
#pragma unroll
      for (int i = 0; i < PT_PER_THREAD; ++i)
        if (base + i < n) flags[base + i] = static_cast<uint8_t>((fw[i / 4] >> (8 * (i % 4))) & 1u);
    }
  }
  if (!write_flags) return;
  if (run) atomicAdd(&sh_ones[cur], run);
  const int lane = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if (lane == 0) wsum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < PT_THREADS / 32; ++w) s += wsum[w];
    tile_cnt[bid] = s;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x)
    if (sh_ones[i]) atomicAdd(&seg->ones[i], sh_ones[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(&misc->done_part, 1u) == nblk - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  plan_next_level(tile_cnt, n_ptiles, seg, nxt, plan, depth, rows_per_item, cs, target_units, rows_hist);
  if (threadIdx.x == 0) misc->done_part = 0;
}

__global__ void part_flags_kernel(const uint8_t* __restrict__ bins, const uint8_t* __restrict__ bins_t, int64_t n,
                                  const uint32_t* __restrict__ order, const cbg_split* __restrict__ splits, int depth,
                                  uint16_t* __restrict__ leaf, uint8_t* __restrict__ flags,
                                  uint32_t* __restrict__ tile_cnt, Segs* seg, int write_flags, int64_t n_ptiles,
                                  Segs* __restrict__ nxt, Plan* __restrict__ plan, int rows_per_item, int cs,
                                  int target_units,
                                  unsigned long long* __restrict__ rows_hist, Misc* misc,
                                  const double* __restrict__ hist, int F, int max_bins,
                                  double* __restrict__ child_totals, const uint8_t* __restrict__ chal_bins,
                                  const double* __restrict__ chal_hist, int chal_max_bins) {
  part_flags_body(bins, bins_t, n, order, splits, depth, leaf, flags, tile_cnt, seg, write_flags, n_ptiles, nxt, plan,
                  rows_per_item, cs, target_units, rows_hist, misc, hist, F, max_bins, child_totals, blockIdx.x,
                  gridDim.x, chal_bins, chal_hist, chal_max_bins);
}

// C: stable partition of every segment: the row at position i moves to
// start + (zeros before it) or start + zeros + (ones before it).
__device__ __forceinline__ void part_scatter_body(const uint32_t* __restrict__ order, const uint8_t* __restrict__ flags, int64_t n,
                                    const uint32_t* __restrict__ tile_off, const Segs* __restrict__ cur, int depth,
                                    uint32_t* __restrict__ order_out,
                                    const void* __restrict__ g_in, const void* __restrict__ h_in,
                                    void* __restrict__ g_out, void* __restrict__ h_out, int gh_bytes, int bid, int nblk) {
  __shared__ uint32_t sh[PT_THREADS / 32];
  __shared__ int sh_pos[1 << (MAX_DEPTH - 1)], sh_leaf[1 << (MAX_DEPTH - 1)];
  __shared__ uint32_t sh_ob[1 << (MAX_DEPTH - 1)];   // per segment: ones before it (level order)
  __shared__ int sh_zeros[1 << (MAX_DEPTH - 1)];     // per segment: rows of its "0" side
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int L = 1 << depth;
  load_seg_table(cur, L, sh_pos, sh_leaf);
  for (int i = threadIdx.x; i < L; i += blockDim.x) {   // the same thread wrote sh_leaf[i]
    const int l = sh_leaf[i];
    sh_ob[i] = cur->ones_before[l];
    sh_zeros[i] = cur->cnt[l] - static_cast<int>(cur->ones[l]);
  }
  const int64_t base = static_cast<int64_t>(bid) * PT + static_cast<int64_t>(threadIdx.x) * PT_PER_THREAD;
  const bool whole = base + PT_PER_THREAD <= n;
  uint8_t fl[PT_PER_THREAD];
  uint32_t s = 0;
  if (whole) {   // the flags buffer is 256-byte aligned and base a multiple of 8
    const uint2 w = *reinterpret_cast<const uint2*>(flags + base);
#pragma unroll
    for (int i = 0; i < PT_PER_THREAD; ++i) fl[i] = static_cast<uint8_t>(((i < 4 ? w.x : w.y) >> (8 * (i % 4))) & 0xffu);
  } else {
#pragma unroll
    for (int i = 0; i < PT_PER_THREAD; ++i) fl[i] = (base + i < n) ? flags[base + i] : 0;
  }
#pragma unroll
  for (int i = 0; i < PT_PER_THREAD; ++i) s += fl[i];
  // the row ids and (g, h) of the thread's positions, loaded together ahead of the stores
  uint32_t rows[PT_PER_THREAD];
  load_rows(order, n, base, rows);
  uint32_t gv[PT_PER_THREAD], hv[PT_PER_THREAD];
  if (gh_bytes == 4) {
    const uint32_t* gi = static_cast<const uint32_t*>(g_in);
    const uint32_t* hi = static_cast<const uint32_t*>(h_in);
    if (whole && ((reinterpret_cast<uintptr_t>(gi + base) | reinterpret_cast<uintptr_t>(hi + base)) & 15) == 0) {
      const uint4 g0 = *reinterpret_cast<const uint4*>(gi + base), g1 = *(reinterpret_cast<const uint4*>(gi + base) + 1);
      const uint4 h0 = *reinterpret_cast<const uint4*>(hi + base), h1 = *(reinterpret_cast<const uint4*>(hi + base) + 1);
      gv[0] = g0.x; gv[1] = g0.y; gv[2] = g0.z; gv[3] = g0.w; gv[4] = g1.x; gv[5] = g1.y; gv[6] = g1.z; gv[7] = g1.w;
      hv[0] = h0.x; hv[1] = h0.y; hv[2] = h0.z; hv[3] = h0.w; hv[4] = h1.x; hv[5] = h1.y; hv[6] = h1.z; hv[7] = h1.w;
    } else {
#pragma unroll
      for (int i = 0; i < PT_PER_THREAD; ++i) {
        gv[i] = base + i < n ? gi[base + i] : 0u;
        hv[i] = base + i < n ? hi[base + i] : 0u;
      }
    }
  } else if (gh_bytes == 2) {
    const uint16_t* gi = static_cast<const uint16_t*>(g_in);
    const uint16_t* hi = static_cast<const uint16_t*>(h_in);
#pragma unroll
    for (int i = 0; i < PT_PER_THREAD; ++i) {
      gv[i] = base + i < n ? gi[base + i] : 0u;
      hv[i] = base + i < n ? hi[base + i] : 0u;
    }
  }
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < PT_THREADS / 32; ++w) {
      uint32_t t = sh[w];
      sh[w] = run;
      run += t;
    }
  }
  __syncthreads();
  uint32_t ones_before = tile_off[bid] + sh[warp] + x - s;
  int si = seg_find(sh_pos, L, base);
#pragma unroll
  for (int i = 0; i < PT_PER_THREAD; ++i) {
    const int64_t pos = base + i;
    if (pos < n) {
      const uint32_t row = rows[i];
      while (si + 1 < L && sh_pos[si + 1] <= pos) ++si;
      const int start = sh_pos[si];
      const uint32_t ob = ones_before - sh_ob[si];   // ones of the segment before pos
      const int zeros_total = sh_zeros[si];
      int dst;
      if (fl[i])
        dst = start + zeros_total + static_cast<int>(ob);
      else
        dst = start + static_cast<int>(pos - start) - static_cast<int>(ob);
      if (dst >= 0 && dst < n) {
        order_out[dst] = row;
        if (gh_bytes == 4) {
          static_cast<uint32_t*>(g_out)[dst] = gv[i];
          static_cast<uint32_t*>(h_out)[dst] = hv[i];
        } else if (gh_bytes == 2) {
          static_cast<uint16_t*>(g_out)[dst] = static_cast<uint16_t>(gv[i]);
          static_cast<uint16_t*>(h_out)[dst] = static_cast<uint16_t>(hv[i]);
        }
      }
    }
    ones_before += fl[i];
  }
}

__global__ void part_scatter_kernel(const uint32_t* __restrict__ order, const uint8_t* __restrict__ flags, int64_t n,
                                    const uint32_t* __restrict__ tile_off, const Segs* __restrict__ cur, int depth,
                                    uint32_t* __restrict__ order_out,
                                    const void* __restrict__ g_in, const void* __restrict__ h_in,
                                    void* __restrict__ g_out, void* __restrict__ h_out, int gh_bytes) {
  part_scatter_body(order, flags, n, tile_off, cur, depth, order_out, g_in, h_in, g_out, h_out, gh_bytes, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------- apply
template <typename GH>
__device__ __forceinline__ void apply_body(const uint8_t* __restrict__ bins, int64_t n, int groups, const cbg_split* __restrict__ splits,
                             int depth, const double* __restrict__ leaf_totals, const double* __restrict__ values_in,
                             double l2, double lr, const uint16_t* __restrict__ leaf_in, uint16_t* __restrict__ leaf_out,
                             float* __restrict__ pred, double* __restrict__ values_out, const float* __restrict__ y,
                             int loss, GH* __restrict__ g, GH* __restrict__ h, int bid, int nblk) {
  __shared__ float lrv[1 << MAX_DEPTH];
  __shared__ int sf[MAX_DEPTH], sk[MAX_DEPTH];
  const int L = 1 << depth;
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    double v;
    if (leaf_totals) {
      const double den = leaf_totals[2 * l + 1] + l2;
      v = den == 0.0 ? 0.0 : -leaf_totals[2 * l] / den;
    } else {
      v = values_in[l];
    }
    lrv[l] = static_cast<float>(lr * v);
    if (values_out && bid == 0) values_out[l] = v;
  }
  if (threadIdx.x < depth) {
    sf[threadIdx.x] = splits[threadIdx.x].feature;
    sk[threadIdx.x] = splits[threadIdx.x].border;
  }
  __syncthreads();
  for (int64_t r = bid * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(nblk) * blockDim.x) {
    int l;
    if (leaf_in) {
      l = leaf_in[r] & (L - 1);
    } else {
      l = 0;
      for (int i = 0; i < depth; ++i) {
        const int f = sf[i];
        if (f >= 0 && (f >> 5) < groups && bins[(static_cast<int64_t>(f >> 5) * n + r) * GROUP + (f & 31)] > sk[i])
          l += 1 << i;
      }
    }
    if (leaf_out) leaf_out[r] = static_cast<uint16_t>(l);
    const float p = pred[r] + lrv[l];
    pred[r] = p;
    if (g) {
      const float yi = y[r];
      float gi, hi;
      if (loss == CBG_LOSS_RMSE) {
        gi = p - yi;
        hi = 1.0f;
      } else {
        const float s = 1.0f / (1.0f + expf(-p));
        gi = s - yi;
        hi = s * (1.0f - s);
      }
      cbgd::store_gh(g, r, gi);
      cbgd::store_gh(h, r, hi);
    }
  }
}

template <typename GH>
__global__ void apply_kernel(const uint8_t* __restrict__ bins, int64_t n, int groups, const cbg_split* __restrict__ splits,
                             int depth, const double* __restrict__ leaf_totals, const double* __restrict__ values_in,
                             double l2, double lr, const uint16_t* __restrict__ leaf_in, uint16_t* __restrict__ leaf_out,
                             float* __restrict__ pred, double* __restrict__ values_out, const float* __restrict__ y,
                             int loss, GH* __restrict__ g, GH* __restrict__ h) {
  apply_body<GH>(bins, n, groups, splits, depth, leaf_totals, values_in, l2, lr, leaf_in, leaf_out, pred, values_out, y, loss, g, h, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------- host helpers
// Copies one tree's splits and leaf values from the graph's fixed scratch to tree slot t of
// the model (t read from, then advanced in, a device counter), so one captured tree can be
// replayed for every tree of the run.
__device__ __forceinline__ void record_tree_body(const cbg_split* __restrict__ sp_tmp, const double* __restrict__ v_tmp,
                                                 int depth, cbg_split* __restrict__ splits, double* __restrict__ values,
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

__global__ void record_tree_kernel(const cbg_split* __restrict__ sp_tmp, const double* __restrict__ v_tmp, int depth,
                                   cbg_split* __restrict__ splits, double* __restrict__ values,
                                   unsigned* __restrict__ counter, int trees) {
  record_tree_body(sp_tmp, v_tmp, depth, splits, values, counter, trees);
}

// ---------------------------------------------------------------- batched form
// Everything the level kernels need for one problem of a batched round, with the buffers
// of one level (the ping-pong buffers alternate between levels). A block map gives every
// block of a batched launch its problem and its block index within that problem.
struct LevelProblem {
  const uint8_t* bins;
  const uint8_t* bins_t;
  int64_t n;
  int F, G, max_bins, rows_per_item, cs;
  int target_units;           // work units per level of a histogram launch (0: rows_per_item x cs each)
  int64_t n_ptiles;
  int apply_blocks;
  const int32_t* n_borders;
  const float* y;
  int loss;
  float* pred;
  void* g;
  void* h;
  uint16_t* leaf;
  cbg_split* sp;              // the tree's splits (graph scratch)
  double* vals;               // the tree's leaf values (graph scratch)
  double* child_totals;
  cbg_split* splits_out;      // model slots [T][D]
  double* values_out;         // model slots [T][2^D]
  unsigned* counter;
  Plan* plan;
  float* partials;
  float2* hist_df;
  BestF* best;
  Misc* misc;
  uint8_t* flags;
  uint32_t* tcnt;
  unsigned long long* rows_hist;
  Segs* seg_root;
  Segs* seg_cur;
  Segs* seg_nxt;
  const uint32_t* order_cur;
  uint32_t* order_nxt;
  double* hist_cur;
  const double* hist_prev;
};

constexpr int BEGIN_ROWS = 4096;   // leaf entries zeroed per block of the batched tree start

__global__ void begin_batched_kernel(const LevelProblem* __restrict__ tab, const int2* __restrict__ map) {
  const int2 m = map[blockIdx.x];
  const LevelProblem& P = tab[m.x];
  const int64_t r0 = static_cast<int64_t>(m.y) * BEGIN_ROWS;
  const int64_t r1 = min(P.n, r0 + BEGIN_ROWS);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) P.leaf[r] = 0;
  if (m.y != 0) return;
  uint32_t* sw = reinterpret_cast<uint32_t*>(P.seg_root);
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(Segs) / 4); i += blockDim.x) sw[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    P.misc->done = 0;
    P.misc->done_part = 0;
    P.misc->forced_score = 0.0;
    tree_begin_body(P.plan, P.seg_root, static_cast<int>(P.n), P.rows_per_item, P.cs, P.target_units, P.rows_hist);
  }
}


template <int SC_WARPS>
__global__ void __launch_bounds__(SC_WARPS * 32) score_batched_kernel(const LevelProblem* __restrict__ tab,
                                                                      const int2* __restrict__ map, int level_leaves,
                                                                      double l2, int depth) {
  const int2 m = map[blockIdx.x];
  const LevelProblem& P = tab[m.x];
  score_level_body<SC_WARPS>(P.hist_df, level_leaves, P.F, P.max_bins, P.n_borders, l2, P.best, P.misc, -1, -1, depth,
                             P.sp, m.y, P.F, nullptr);
}

__global__ void flags_batched_kernel(const LevelProblem* __restrict__ tab, const int2* __restrict__ map, int depth,
                                     int write_flags) {
  const int2 m = map[blockIdx.x];
  const LevelProblem& P = tab[m.x];
  part_flags_body(P.bins, P.bins_t, P.n, P.order_cur, P.sp, depth, P.leaf, P.flags, P.tcnt, P.seg_cur, write_flags,
                  P.n_ptiles, P.seg_nxt, P.plan, P.rows_per_item, P.cs, P.target_units, P.rows_hist, P.misc,
                  P.hist_cur, P.F,
                  P.max_bins, P.child_totals, m.y, static_cast<int>(P.n_ptiles), nullptr, nullptr, 0);
}

__global__ void scatter_batched_kernel(const LevelProblem* __restrict__ tab, const int2* __restrict__ map, int depth) {
  const int2 m = map[blockIdx.x];
  const LevelProblem& P = tab[m.x];
  part_scatter_body(P.order_cur, P.flags, P.n, P.tcnt, P.seg_cur, depth, P.order_nxt, nullptr, nullptr, nullptr,
                    nullptr, 0, m.y, static_cast<int>(P.n_ptiles));
}

template <typename GH>
__global__ void apply_batched_kernel(const LevelProblem* __restrict__ tab, const int2* __restrict__ map, int depth,
                                     double l2, double lr) {
  const int2 m = map[blockIdx.x];
  const LevelProblem& P = tab[m.x];
  apply_body<GH>(P.bins, P.n, P.G, P.sp, depth, P.child_totals, nullptr, l2, lr, P.leaf, nullptr, P.pred, P.vals, P.y,
                 P.loss, static_cast<GH*>(P.g), static_cast<GH*>(P.h), m.y, P.apply_blocks);
}

__global__ void record_batched_kernel(const LevelProblem* __restrict__ tab, int depth, int trees) {
  const LevelProblem& P = tab[blockIdx.x];
  record_tree_body(P.sp, P.vals, depth, P.splits_out, P.values_out, P.counter, trees);
}

cbg_status check_state(cbg_ctx* ctx, const Layout& L, void* state, size_t bytes) {
  CBG_REQUIRE(ctx, state != nullptr, "state is NULL");
  CBG_REQUIRE(ctx, reinterpret_cast<uintptr_t>(state) % 256 == 0, "state must be 256-byte aligned");
  if (bytes < L.total) return fail(ctx, CBG_ENOMEM, "tree state of %zu bytes is smaller than the %zu needed", bytes, L.total);
  return CBG_OK;
}

}  // namespace

extern "C" {

cbg_status cbg_gradients(cbg_ctx* ctx, int loss, const float* y, const float* pred, int64_t n, int gh_dtype,
                         void* g, void* h) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, loss == CBG_LOSS_RMSE || loss == CBG_LOSS_LOGLOSS, "bad loss");
  CBG_REQUIRE(ctx, gh_dtype == CBG_F32 || gh_dtype == CBG_BF16, "bad gh_dtype");
  CBG_REQUIRE(ctx, y && pred && g && h, "NULL argument");
  DeviceGuard guard(ctx->device);
  const unsigned grid = grid_stride_blocks(n, 256);
  if (gh_dtype == CBG_F32)
    gradients_kernel<float><<<grid, 256, 0, ctx->stream>>>(loss, y, pred, n, static_cast<float*>(g), static_cast<float*>(h));
  else
    gradients_kernel<__nv_bfloat16><<<grid, 256, 0, ctx->stream>>>(loss, y, pred, n, static_cast<__nv_bfloat16*>(g),
                                                                   static_cast<__nv_bfloat16*>(h));
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

cbg_status cbg_tree_state_bytes(const cbg_tree_shape* shape, size_t* bytes) {
  if (!bytes) return CBG_EINVAL;
  Layout L;
  cbg_status st = make_layout(nullptr, shape, &L);
  if (st != CBG_OK) return st;
  *bytes = L.total;
  return CBG_OK;
}

cbg_status cbg_tree_begin(cbg_ctx* ctx, const cbg_tree_shape* shape, void* state, size_t state_bytes, uint16_t* leaf) {
  if (!ctx) return CBG_EINVAL;
  Layout L;
  cbg_status st = make_layout(ctx, shape, &L);
  if (st != CBG_OK) return st;
  st = check_state(ctx, L, state, state_bytes);
  if (st != CBG_OK) return st;
  CBG_REQUIRE(ctx, leaf != nullptr, "leaf is NULL");
  DeviceGuard guard(ctx->device);
  CBG_CUDA(ctx, cudaMemsetAsync(leaf, 0, L.n * sizeof(uint16_t), ctx->stream));
  CBG_CUDA(ctx, cudaMemsetAsync(at<char>(state, L.o_seg_a), 0, sizeof(Segs), ctx->stream));
  CBG_CUDA(ctx, cudaMemsetAsync(at<char>(state, L.o_misc), 0, sizeof(Misc), ctx->stream));
  int cs = 1, clusters = 1;
  st = hist_cluster_geom(ctx, hist_config(L), &cs, &clusters);
  if (st != CBG_OK) return st;
  tree_begin_kernel<<<1, 32, 0, ctx->stream>>>(at<Plan>(state, L.o_plan), at<Segs>(state, L.o_seg_a),
                                               static_cast<int>(L.n), L.rows_per_item, cs,
                                               hist_target_units(clusters, L.G),
                                               at<unsigned long long>(state, L.o_count));
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

namespace {
cbg_status build_level_impl(cbg_ctx* ctx, const cbg_level_args* a, bool do_hist);
}

cbg_status cbg_build_level(cbg_ctx* ctx, const cbg_level_args* a) { return build_level_impl(ctx, a, true); }

namespace {

// One level; do_hist = false when the histogram of this level was computed by a batched
// launch over many problems (cbg_boost_batched).
cbg_status build_level_impl(cbg_ctx* ctx, const cbg_level_args* a, bool do_hist) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, a != nullptr, "args is NULL");
  Layout L;
  cbg_status st = make_layout(ctx, a->shape, &L);
  if (st != CBG_OK) return st;
  st = check_state(ctx, L, a->state, a->state_bytes);
  if (st != CBG_OK) return st;
  const int d = a->depth;
  CBG_REQUIRE(ctx, d >= 0 && d < L.D, "depth %d outside [0, max_depth)", d);
  CBG_REQUIRE(ctx, a->bins && a->n_borders && a->g && a->h && a->leaf && a->splits && a->child_totals, "NULL argument");
  CBG_REQUIRE(ctx, (L.kind != 4 && L.kind != 5 && L.kind != 8) || (reinterpret_cast<uintptr_t>(a->bins) & 15) == 0,
              "bins must be 16-byte aligned for the lane-per-feature histogram kernel");
  CBG_REQUIRE(ctx, L.kind != 6 || (a->bins4 != nullptr && (reinterpret_cast<uintptr_t>(a->bins4) & 15) == 0),
              "the 4-bit packed histogram kernel needs bins4 (16-byte aligned, cbg_pack_bins4)");
  CBG_REQUIRE(ctx, L.kind != 9 || (a->bits1 != nullptr && (reinterpret_cast<uintptr_t>(a->bits1) & 15) == 0),
              "the 1-bit histogram kernel needs bits1 (16-byte aligned, cbg_pack_bits1)");
  CBG_REQUIRE(ctx, a->gh_dtype == CBG_F32 || a->gh_dtype == CBG_BF16, "bad gh_dtype");
  CBG_REQUIRE(ctx, a->l2 >= 0.0 && std::isfinite(a->l2), "l2 must be finite and >= 0");
  CBG_REQUIRE(ctx, a->force_feature < L.F, "force_feature out of range");
  CBG_REQUIRE(ctx, a->force_feature < 0 || (a->force_border >= 0 && a->force_border < L.max_bins - 1),
              "force_border out of range");
  CBG_REQUIRE(ctx, !a->challenger || (a->challenger_bins && a->challenger_hist && a->challenger_max_bins >= 2 &&
                                      a->challenger_max_bins <= 256),
              "a challenger needs its bins, its histogram and 2 <= challenger_max_bins <= 256");
  DeviceGuard guard(ctx->device);
  void* S = a->state;
  Plan* plan = at<Plan>(S, L.o_plan);
  Segs* seg_cur = at<Segs>(S, d % 2 == 0 ? L.o_seg_a : L.o_seg_b);
  Segs* seg_nxt = at<Segs>(S, d % 2 == 0 ? L.o_seg_b : L.o_seg_a);
  const uint32_t* order_cur = d == 0 ? nullptr : at<uint32_t>(S, d % 2 == 1 ? L.o_order_a : L.o_order_b);
  uint32_t* order_nxt = at<uint32_t>(S, (d + 1) % 2 == 1 ? L.o_order_a : L.o_order_b);
  double* hist_cur = at<double>(S, d % 2 == 0 ? L.o_hist_a : L.o_hist_b);
  const double* hist_prev = at<double>(S, d % 2 == 0 ? L.o_hist_b : L.o_hist_a);
  float* partials = at<float>(S, L.o_part);
  float2* hist_df = at<float2>(S, L.o_hdf);
  BestF* best = at<BestF>(S, L.o_best);
  Misc* misc = at<Misc>(S, L.o_misc);
  uint8_t* flags = at<uint8_t>(S, L.o_flags);
  uint32_t* tcnt = at<uint32_t>(S, L.o_tcnt);

  // 1. histogram of the directly computed leaves
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  CBG_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &capturing));
  if (do_hist && capturing == cudaStreamCaptureStatusNone) st = prof_begin(ctx, &ev0, &ev1);
  if (st != CBG_OK) return st;
  // the lane-per-feature kernels and the fixed-point kernel read (g, h) by position: the
  // caller's arrays at the root (positions are rows), then the copies the previous level's
  // partition moved along (for the FP32 shared-reduction kernel, which is bound by its
  // compare-and-swap loops, the copy costs the partition more than it saves; the loader-
  // warp kernel, whose loaders could gather by row from L2, lost a third of its speed so)
  const bool by_pos = L.kind == 4 || L.kind == 5 || L.kind == 6 || L.kind == 7 || L.kind == 8 || L.kind == 9;
  const uint8_t* hist_bins = L.kind == 6   ? a->bins4
                             : L.kind == 9 ? reinterpret_cast<const uint8_t*>(a->bits1)
                                           : a->bins;
  const void* g_pos = d == 0 ? a->g : at<char>(S, d % 2 == 1 ? L.o_gp_a : L.o_gp_b);
  const void* h_pos = d == 0 ? a->h : at<char>(S, d % 2 == 1 ? L.o_hp_a : L.o_hp_b);
  void* g_pos_nxt = at<char>(S, (d + 1) % 2 == 1 ? L.o_gp_a : L.o_gp_b);
  void* h_pos_nxt = at<char>(S, (d + 1) % 2 == 1 ? L.o_hp_a : L.o_hp_b);
  const void* g_hist = by_pos ? g_pos : a->g;
  const void* h_hist = by_pos ? h_pos : a->h;
  if (do_hist) {
    st = a->gh_dtype == CBG_F32
             ? launch_hist<float>(ctx, hist_config(L), hist_bins, order_cur, g_hist, h_hist, plan, partials)
             : launch_hist<__nv_bfloat16>(ctx, hist_config(L), hist_bins, order_cur, g_hist, h_hist, plan, partials);
    if (st != CBG_OK) return st;
    st = prof_end(ctx, ev1);
    if (st != CBG_OK) return st;
  }
  // 2. FP64 reduction of the partials + sibling subtraction
  {
    reduce_kernel<<<reduce_grid(L.G, L.max_bins, d == 0 ? 1 : (1 << (d - 1))), RD_THREADS, 0, ctx->stream>>>(
        plan, partials, L.G, L.F, L.max_bins, hist_prev, hist_cur, a->splits, d, hist_df, a->n_borders);
    CBG_CHECK_LAUNCH(ctx);
  }
  // 3. split scores and argmax
  const int level_leaves = 1 << d;
  {
    auto launch = [&](auto warps) {
      constexpr int W = decltype(warps)::value;
      score_level_kernel<W><<<L.F, W * 32, 0, ctx->stream>>>(hist_df, level_leaves, L.F, L.max_bins, a->n_borders,
                                                           a->l2, best, misc, a->force_feature, a->force_border, d,
                                                           a->splits, a->challenger);
    };
    if (level_leaves >= SC_MAX_WARPS) launch(std::integral_constant<int, SC_MAX_WARPS>{});
    else if (level_leaves >= 8) launch(std::integral_constant<int, 8>{});
    else if (level_leaves >= 4) launch(std::integral_constant<int, 4>{});
    else if (level_leaves >= 2) launch(std::integral_constant<int, 2>{});
    else launch(std::integral_constant<int, 1>{});
    CBG_CHECK_LAUNCH(ctx);
  }
  if (a->hist_out)
    CBG_CUDA(ctx, cudaMemcpyAsync(a->hist_out, hist_cur,
                                  static_cast<size_t>(level_leaves) * L.F * L.max_bins * 2 * sizeof(double),
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  // 4. leaf update and (unless this is the last level) the row partition of the next level
  const bool last = a->last_level || d == L.D - 1;
  int cs = 1, clusters = 1;
  if (!last) {
    st = hist_cluster_geom(ctx, hist_config(L), &cs, &clusters);
    if (st != CBG_OK) return st;
  }
  part_flags_kernel<<<static_cast<unsigned>(L.n_ptiles), PT_THREADS, 0, ctx->stream>>>(
      a->bins, a->bins_t, L.n, order_cur, a->splits, d, a->leaf, flags, tcnt, seg_cur, last ? 0 : 1, L.n_ptiles,
      seg_nxt, plan, L.rows_per_item, cs, hist_target_units(clusters, L.G), at<unsigned long long>(S, L.o_count),
      misc, hist_cur, L.F, L.max_bins,
      a->child_totals, a->challenger ? a->challenger_bins : nullptr, a->challenger_hist, a->challenger_max_bins);
  CBG_CHECK_LAUNCH(ctx);
  if (!last) {
    part_scatter_kernel<<<static_cast<unsigned>(L.n_ptiles), PT_THREADS, 0, ctx->stream>>>(
        order_cur, flags, L.n, tcnt, seg_cur, d, order_nxt, g_pos, h_pos, g_pos_nxt, h_pos_nxt,
        by_pos ? (a->gh_dtype == CBG_F32 ? 4 : 2) : 0);
    CBG_CHECK_LAUNCH(ctx);
  }
  return CBG_OK;
}

}  // namespace

cbg_status cbg_tree_rows_histogrammed(cbg_ctx* ctx, const cbg_tree_shape* shape, void* state, int reset,
                                      int64_t* rows) {
  if (!ctx) return CBG_EINVAL;
  Layout L;
  cbg_status st = make_layout(ctx, shape, &L);
  if (st != CBG_OK) return st;
  CBG_REQUIRE(ctx, state != nullptr && rows != nullptr, "NULL argument");
  DeviceGuard guard(ctx->device);
  unsigned long long v = 0;
  CBG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  CBG_CUDA(ctx, cudaMemcpy(&v, at<char>(state, L.o_count), sizeof(v), cudaMemcpyDeviceToHost));
  *rows = static_cast<int64_t>(v);
  if (reset) CBG_CUDA(ctx, cudaMemset(at<char>(state, L.o_count), 0, sizeof(v)));
  return CBG_OK;
}

cbg_status cbg_apply_tree(cbg_ctx* ctx, const cbg_apply_args* a) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, a != nullptr, "args is NULL");
  CBG_REQUIRE(ctx, a->n >= 1 && a->n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, a->depth >= 1 && a->depth <= MAX_DEPTH, "depth must be in [1, 10]");
  CBG_REQUIRE(ctx, a->pred != nullptr, "pred is NULL");
  CBG_REQUIRE(ctx, a->leaf_totals || a->leaf_values_in, "need leaf_totals or leaf_values_in");
  CBG_REQUIRE(ctx, a->leaf_in || (a->bins && a->splits), "need leaf_in or bins + splits");
  CBG_REQUIRE(ctx, a->leaf_in || (a->F_pad >= 32 && a->F_pad % 32 == 0), "F_pad must be a multiple of 32");
  CBG_REQUIRE(ctx, a->l2 >= 0.0, "l2 must be >= 0");
  const bool grads = a->g != nullptr;
  CBG_REQUIRE(ctx, !grads || (a->h && a->y), "fused gradients need y, g and h");
  CBG_REQUIRE(ctx, !grads || a->loss == CBG_LOSS_RMSE || a->loss == CBG_LOSS_LOGLOSS, "bad loss");
  CBG_REQUIRE(ctx, !grads || a->gh_dtype == CBG_F32 || a->gh_dtype == CBG_BF16, "bad gh_dtype");
  DeviceGuard guard(ctx->device);
  const unsigned grid = grid_stride_blocks(a->n, 256);
  if (!grads || a->gh_dtype == CBG_F32)
    apply_kernel<float><<<grid, 256, 0, ctx->stream>>>(a->bins, a->n, a->F_pad / GROUP, a->splits, a->depth, a->leaf_totals,
                                                       a->leaf_values_in, a->l2, a->lr, a->leaf_in, a->leaf_out,
                                                       a->pred, a->leaf_values_out, a->y, a->loss,
                                                       static_cast<float*>(a->g), static_cast<float*>(a->h));
  else
    apply_kernel<__nv_bfloat16><<<grid, 256, 0, ctx->stream>>>(
        a->bins, a->n, a->F_pad / GROUP, a->splits, a->depth, a->leaf_totals, a->leaf_values_in, a->l2, a->lr, a->leaf_in,
        a->leaf_out, a->pred, a->leaf_values_out, a->y, a->loss, static_cast<__nv_bfloat16*>(a->g),
        static_cast<__nv_bfloat16*>(a->h));
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

namespace {

// One boosting iteration: tree_begin, D levels, leaf values + prediction update + next
// gradients. Splits go to sp, leaf values to vals.
cbg_status boost_one_tree(cbg_ctx* ctx, const cbg_boost_args* a, cbg_split* sp, double* vals) {
  const int D = a->depth;
  cbg_status st = cbg_tree_begin(ctx, a->shape, a->state, a->state_bytes, a->leaf);
  if (st != CBG_OK) return st;
  for (int d = 0; d < D; ++d) {
    cbg_level_args la{};
    la.shape = a->shape;
    la.state = a->state;
    la.state_bytes = a->state_bytes;
    la.bins = a->bins;
    la.bins_t = a->bins_t;
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
    la.hist_out = nullptr;
    la.last_level = d == D - 1;
    la.bins4 = a->bins4;
    la.bits1 = a->bits1;
    st = cbg_build_level(ctx, &la);
    if (st != CBG_OK) return st;
  }
  cbg_apply_args aa{};
  aa.bins = a->bins;
  aa.n = a->shape->n;
  aa.F_pad = a->shape->F_pad;
  aa.splits = sp;
  aa.depth = D;
  aa.leaf_totals = a->child_totals;
  aa.l2 = a->l2;
  aa.lr = a->lr;
  aa.leaf_in = a->leaf;
  aa.pred = a->pred;
  aa.leaf_values_out = vals;
  aa.y = a->y;
  aa.loss = a->loss;
  aa.gh_dtype = a->gh_dtype;
  aa.g = a->g;
  aa.h = a->h;
  return cbg_apply_tree(ctx, &aa);
}

}  // namespace

cbg_status cbg_boost(cbg_ctx* ctx, const cbg_boost_args* a) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, a != nullptr && a->shape != nullptr, "args is NULL");
  CBG_REQUIRE(ctx, a->depth >= 1 && a->depth <= a->shape->max_depth, "depth outside [1, max_depth]");
  CBG_REQUIRE(ctx, a->trees >= 0, "trees must be >= 0");
  CBG_REQUIRE(ctx, a->pred && a->y && a->g && a->h && a->leaf && a->splits && a->leaf_values && a->child_totals,
              "NULL argument");
  DeviceGuard guard(ctx->device);
  const int D = a->depth;
  const int64_t n = a->shape->n;
  cbg_status st = cbg_gradients(ctx, a->loss, a->y, a->pred, n, a->gh_dtype, a->g, a->h);
  if (st != CBG_OK) return st;
  if (!a->use_graph || a->trees <= 1) {
    for (int t = 0; t < a->trees; ++t) {
      st = boost_one_tree(ctx, a, a->splits + static_cast<int64_t>(t) * D,
                          a->leaf_values + static_cast<int64_t>(t) * (1 << D));
      if (st != CBG_OK) return st;
    }
    return CBG_OK;
  }
  // Graph replay: capture one tree (outputs to fixed scratch + a record kernel) and launch
  // it once per tree. Launch-geometry queries are made before the capture begins.
  Layout L;
  st = make_layout(ctx, a->shape, &L);
  if (st != CBG_OK) return st;
  st = check_state(ctx, L, a->state, a->state_bytes);
  if (st != CBG_OK) return st;
  st = a->gh_dtype == CBG_F32 ? hist_warm<float>(ctx, hist_config(L)) : hist_warm<__nv_bfloat16>(ctx, hist_config(L));
  if (st != CBG_OK) return st;
  cbg_split* sp_tmp = at<cbg_split>(a->state, L.o_gsplit);
  double* v_tmp = at<double>(a->state, L.o_gvals);
  unsigned* counter = reinterpret_cast<unsigned*>(at<char>(a->state, L.o_gsplit) + sizeof(cbg_split) * MAX_DEPTH);
  CBG_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream));
  // The caller's stream may be the legacy default stream, which cannot be captured: the
  // tree is captured on a library-owned stream and the graph is launched on the caller's.
  if (!ctx->capture_stream) CBG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  cudaStream_t user_stream = ctx->stream;
  ctx->stream = ctx->capture_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    ctx->stream = user_stream;
    return fail(ctx, CBG_ECUDA, "cudaStreamBeginCapture failed: %s", cudaGetErrorString(ce));
  }
  st = boost_one_tree(ctx, a, sp_tmp, v_tmp);
  if (st == CBG_OK) {
    record_tree_kernel<<<1, 256, 0, ctx->stream>>>(sp_tmp, v_tmp, D, a->splits, a->leaf_values, counter, a->trees);
    if (cudaGetLastError() != cudaSuccess) st = fail(ctx, CBG_ECUDA, "record kernel launch failed during capture");
  }
  ce = cudaStreamEndCapture(ctx->stream, &graph);
  ctx->stream = user_stream;
  if (st != CBG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "stream capture of a tree failed: %s", cudaGetErrorString(ce));
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
  for (int t = 0; t < a->trees; ++t) {
    ce = cudaGraphLaunch(exec, ctx->stream);
    if (ce != cudaSuccess) break;
  }
  cudaGraphExecDestroy(exec);   // freed once the queued launches complete
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "graph launch failed: %s", cudaGetErrorString(ce));
  return CBG_OK;
}


cbg_status cbg_boost_batched(cbg_ctx* ctx, const cbg_problem* problems, int32_t n_problems, int32_t gh_dtype,
                             int32_t depth, int32_t trees, double lr, double l2, int32_t branches) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, problems != nullptr && n_problems >= 1, "need at least one problem");
  CBG_REQUIRE(ctx, depth >= 1 && depth <= MAX_DEPTH, "depth must be in [1, 10]");
  CBG_REQUIRE(ctx, trees >= 0, "trees must be >= 0");
  CBG_REQUIRE(ctx, gh_dtype == CBG_F32 || gh_dtype == CBG_BF16, "bad gh_dtype");
  CBG_REQUIRE(ctx, branches >= 0, "branches must be >= 0");
  DeviceGuard guard(ctx->device);
  const int nb = branches > 0 ? std::min(branches, n_problems) : std::min(n_problems, 32);
  std::vector<cbg_boost_args> args(n_problems);
  for (int i = 0; i < n_problems; ++i) {
    const cbg_problem& p = problems[i];
    cbg_boost_args& a = args[i];
    a = cbg_boost_args{};
    a.shape = &p.shape;
    a.state = p.state;
    a.state_bytes = p.state_bytes;
    a.bins = p.bins;
    a.bins_t = p.bins_t;
    a.n_borders = p.n_borders;
    a.y = p.y;
    a.loss = p.loss;
    a.gh_dtype = gh_dtype;
    a.depth = depth;
    a.trees = trees;
    a.lr = lr;
    a.l2 = l2;
    a.pred = p.pred;
    a.g = p.g;
    a.h = p.h;
    a.leaf = p.leaf;
    a.splits = p.splits;
    a.leaf_values = p.leaf_values;
    a.child_totals = p.child_totals;
    CBG_REQUIRE(ctx, depth <= p.shape.max_depth, "problem %d: depth exceeds its max_depth", i);
    CBG_REQUIRE(ctx, p.pred && p.y && p.g && p.h && p.leaf && p.splits && p.leaf_values && p.child_totals,
                "problem %d: NULL argument", i);
    Layout L;
    cbg_status st = make_layout(ctx, &p.shape, &L);
    if (st != CBG_OK) return st;
    st = check_state(ctx, L, p.state, p.state_bytes);
    if (st != CBG_OK) return st;
    // launch-geometry queries happen here, before the capture
    st = gh_dtype == CBG_F32 ? hist_warm<float>(ctx, hist_config(L)) : hist_warm<__nv_bfloat16>(ctx, hist_config(L));
    if (st != CBG_OK) return st;
    st = cbg_gradients(ctx, p.loss, p.y, p.pred, p.shape.n, gh_dtype, p.g, p.h);
    if (st != CBG_OK) return st;
    unsigned* counter = reinterpret_cast<unsigned*>(at<char>(p.state, L.o_gsplit) + sizeof(cbg_split) * MAX_DEPTH);
    CBG_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream));
  }
  if (trees == 0) return CBG_OK;
  // When every problem uses the shared-reduction kernel with the same tiling (the plans are
  // chunked for one cluster size), every kernel of a round is one launch over all problems,
  // the level's histograms and FP64 reductions in one persistent launch; otherwise each
  // problem's tree runs on one of the graph's parallel branches.
  bool batch_hist = n_problems <= HIST_MAX_BATCH;
  Layout L0;
  {
    cbg_status st = make_layout(ctx, &problems[0].shape, &L0);
    if (st != CBG_OK) return st;
  }
  int nb_alloc = 2, cs_plan = 1;
  for (int i = 0; i < n_problems && batch_hist; ++i) {
    Layout L;
    cbg_status st = make_layout(ctx, &problems[i].shape, &L);
    if (st != CBG_OK) return st;
    batch_hist = L.kind == 1 && L.cluster == L0.cluster && L.rows_per_item == L0.rows_per_item &&
                 L.threads == L0.threads;
    nb_alloc = std::max(nb_alloc, L.nb_alloc);
  }
  std::vector<HistProblem*> tables;        // histogram tables, one per level
  std::vector<LevelProblem*> ltables;      // level tables, one per level
  int2 *begin_map = nullptr, *score_map = nullptr, *tile_map = nullptr, *apply_map = nullptr;
  int begin_blocks = 0, score_blocks = 0, tile_blocks = 0, apply_blocks = 0;
  if (batch_hist) {
    cbg_status st = hist_cluster_size(ctx, hist_config(L0), &cs_plan);
    if (st != CBG_OK) return st;
    st = gh_dtype == CBG_F32 ? launch_hist_batched<float>(ctx, nb_alloc, nullptr, n_problems, L0.threads, cs_plan, true)
                             : launch_hist_batched<__nv_bfloat16>(ctx, nb_alloc, nullptr, n_problems, L0.threads,
                                                                  cs_plan, true);
    batch_hist = st == CBG_OK;
  }
  if (batch_hist) {
    // host copies of every table and block map, then one upload into the workspace
    std::vector<Layout> Ls(n_problems);
    std::vector<int> target_units(n_problems, 0);
    for (int i = 0; i < n_problems; ++i) {
      make_layout(ctx, &problems[i].shape, &Ls[i]);
      int cs_i = 1, clusters_i = 1;
      if (hist_cluster_geom(ctx, hist_config(Ls[i]), &cs_i, &clusters_i) == CBG_OK)
        target_units[i] = hist_target_units(clusters_i, Ls[i].G);
    }
    std::vector<std::vector<HistProblem>> hts(depth, std::vector<HistProblem>(n_problems));
    std::vector<std::vector<LevelProblem>> lts(depth, std::vector<LevelProblem>(n_problems));
    std::vector<int2> bmap, smap, tmap, amap;
    for (int i = 0; i < n_problems; ++i) {
      const cbg_problem& p = problems[i];
      const Layout& L = Ls[i];
      void* S = p.state;
      const int apply_grid = static_cast<int>(grid_stride_blocks(L.n, 256));
      for (int b = 0; b < static_cast<int>(ceil_div(L.n, BEGIN_ROWS)); ++b) bmap.push_back(make_int2(i, b));
      for (int b = 0; b < L.F; ++b) smap.push_back(make_int2(i, b));
      for (int64_t b = 0; b < L.n_ptiles; ++b) tmap.push_back(make_int2(i, static_cast<int>(b)));
      for (int b = 0; b < apply_grid; ++b) amap.push_back(make_int2(i, b));
      for (int d = 0; d < depth; ++d) {
        hts[d][i] = HistProblem{p.bins, L.n, L.G, L.F,
                                d == 0 ? nullptr : at<uint32_t>(S, d % 2 == 1 ? L.o_order_a : L.o_order_b),
                                p.g, p.h, at<Plan>(S, L.o_plan), L.max_bins, at<float>(S, L.o_part)};
        LevelProblem& q = lts[d][i];
        q = LevelProblem{};
        q.bins = p.bins;
        q.bins_t = p.bins_t;
        q.n = L.n;
        q.F = L.F;
        q.G = L.G;
        q.max_bins = L.max_bins;
        q.rows_per_item = L.rows_per_item;
        q.cs = cs_plan;
        q.target_units = target_units[i];   // the units a single-problem run would cut the level into
        q.n_ptiles = L.n_ptiles;
        q.apply_blocks = apply_grid;
        q.n_borders = p.n_borders;
        q.y = p.y;
        q.loss = p.loss;
        q.pred = p.pred;
        q.g = p.g;
        q.h = p.h;
        q.leaf = p.leaf;
        q.sp = at<cbg_split>(S, L.o_gsplit);
        q.vals = at<double>(S, L.o_gvals);
        q.child_totals = p.child_totals;
        q.splits_out = p.splits;
        q.values_out = p.leaf_values;
        q.counter = reinterpret_cast<unsigned*>(at<char>(S, L.o_gsplit) + sizeof(cbg_split) * MAX_DEPTH);
        q.plan = at<Plan>(S, L.o_plan);
        q.partials = at<float>(S, L.o_part);
        q.hist_df = at<float2>(S, L.o_hdf);
        q.best = at<BestF>(S, L.o_best);
        q.misc = at<Misc>(S, L.o_misc);
        q.flags = at<uint8_t>(S, L.o_flags);
        q.tcnt = at<uint32_t>(S, L.o_tcnt);
        q.rows_hist = at<unsigned long long>(S, L.o_count);
        q.seg_root = at<Segs>(S, L.o_seg_a);
        q.seg_cur = at<Segs>(S, d % 2 == 0 ? L.o_seg_a : L.o_seg_b);
        q.seg_nxt = at<Segs>(S, d % 2 == 0 ? L.o_seg_b : L.o_seg_a);
        q.order_cur = d == 0 ? nullptr : at<uint32_t>(S, d % 2 == 1 ? L.o_order_a : L.o_order_b);
        q.order_nxt = at<uint32_t>(S, (d + 1) % 2 == 1 ? L.o_order_a : L.o_order_b);
        q.hist_cur = at<double>(S, d % 2 == 0 ? L.o_hist_a : L.o_hist_b);
        q.hist_prev = at<double>(S, d % 2 == 0 ? L.o_hist_b : L.o_hist_a);
        // the level's FP64 reduction runs inside the batched histogram launch
        hts[d][i].hist_prev = q.hist_prev;
        hts[d][i].hist_cur = q.hist_cur;
        hts[d][i].splits = q.sp;
        hts[d][i].hist_df = q.hist_df;
        hts[d][i].n_borders = q.n_borders;
      }
    }
    size_t need = 4096;
    auto bytes = [](size_t v) { return (v + 255) / 256 * 256; };
    need += depth * (bytes(sizeof(HistProblem) * n_problems) + bytes(sizeof(LevelProblem) * n_problems));
    need += bytes(sizeof(int2) * bmap.size()) + bytes(sizeof(int2) * smap.size()) + bytes(sizeof(int2) * tmap.size()) +
            bytes(sizeof(int2) * amap.size());
    cbg_status st = ws_reserve(ctx, need);
    if (st != CBG_OK) return st;
    Carve cv(ctx->ws);
    auto upload = [&](const void* host, size_t n_bytes, void* dev) -> cbg_status {
      CBG_CUDA(ctx, cudaMemcpyAsync(dev, host, n_bytes, cudaMemcpyHostToDevice, ctx->stream));
      return CBG_OK;
    };
    for (int d = 0; d < depth && st == CBG_OK; ++d) {
      tables.push_back(cv.take<HistProblem>(n_problems));
      st = upload(hts[d].data(), sizeof(HistProblem) * n_problems, tables.back());
      if (st != CBG_OK) break;
      ltables.push_back(cv.take<LevelProblem>(n_problems));
      st = upload(lts[d].data(), sizeof(LevelProblem) * n_problems, ltables.back());
      if (st != CBG_OK) break;
    }
    begin_map = cv.take<int2>(bmap.size());
    score_map = cv.take<int2>(smap.size());
    tile_map = cv.take<int2>(tmap.size());
    apply_map = cv.take<int2>(amap.size());
    if (st == CBG_OK) st = upload(bmap.data(), sizeof(int2) * bmap.size(), begin_map);
    if (st == CBG_OK) st = upload(smap.data(), sizeof(int2) * smap.size(), score_map);
    if (st == CBG_OK) st = upload(tmap.data(), sizeof(int2) * tmap.size(), tile_map);
    if (st == CBG_OK) st = upload(amap.data(), sizeof(int2) * amap.size(), apply_map);
    if (st != CBG_OK) return st;
    begin_blocks = static_cast<int>(bmap.size());
    score_blocks = static_cast<int>(smap.size());
    tile_blocks = static_cast<int>(tmap.size());
    apply_blocks = static_cast<int>(amap.size());
    CBG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // the host staging vectors go out of scope
  }
  if (!ctx->capture_stream) CBG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  while (static_cast<int>(ctx->branch_streams.size()) < nb) {
    cudaStream_t st;
    CBG_CUDA(ctx, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ctx->branch_streams.push_back(st);
  }
  while (static_cast<int>(ctx->branch_events.size()) < nb + 1) {
    cudaEvent_t e;
    CBG_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->branch_events.push_back(e);
  }
  cudaStream_t user_stream = ctx->stream;
  cudaStream_t origin = ctx->capture_stream;
  cudaGraph_t graph = nullptr;
  CBG_CUDA(ctx, cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
  cbg_status st = CBG_OK;
  cudaError_t ce = cudaEventRecord(ctx->branch_events[nb], origin);
  for (int b = 0; b < nb && ce == cudaSuccess; ++b) ce = cudaStreamWaitEvent(ctx->branch_streams[b], ctx->branch_events[nb], 0);
  if (ce != cudaSuccess) st = fail(ctx, CBG_ECUDA, "forking the batched round failed: %s", cudaGetErrorString(ce));
  // join every branch into the origin stream, and fork the origin again
  auto join = [&]() {
    for (int b = 0; b < nb && st == CBG_OK; ++b) {
      ce = cudaEventRecord(ctx->branch_events[b], ctx->branch_streams[b]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(origin, ctx->branch_events[b], 0);
      if (ce != cudaSuccess) st = fail(ctx, CBG_ECUDA, "joining the batched round failed: %s", cudaGetErrorString(ce));
    }
  };
  auto fork = [&]() {
    if (st != CBG_OK) return;
    ce = cudaEventRecord(ctx->branch_events[nb], origin);
    for (int b = 0; b < nb && ce == cudaSuccess; ++b)
      ce = cudaStreamWaitEvent(ctx->branch_streams[b], ctx->branch_events[nb], 0);
    if (ce != cudaSuccess) st = fail(ctx, CBG_ECUDA, "forking the batched round failed: %s", cudaGetErrorString(ce));
  };
  auto record = [&](int i) {
    Layout L;
    st = make_layout(ctx, &problems[i].shape, &L);
    if (st != CBG_OK) return;
    cbg_split* sp_tmp = at<cbg_split>(problems[i].state, L.o_gsplit);
    double* v_tmp = at<double>(problems[i].state, L.o_gvals);
    unsigned* counter = reinterpret_cast<unsigned*>(at<char>(problems[i].state, L.o_gsplit) + sizeof(cbg_split) * MAX_DEPTH);
    record_tree_kernel<<<1, 256, 0, ctx->stream>>>(sp_tmp, v_tmp, depth, problems[i].splits, problems[i].leaf_values,
                                                   counter, trees);
    if (cudaGetLastError() != cudaSuccess) st = fail(ctx, CBG_ECUDA, "record kernel launch failed during capture");
  };
  if (!batch_hist) {
    for (int i = 0; i < n_problems && st == CBG_OK; ++i) {
      Layout L;
      st = make_layout(ctx, &problems[i].shape, &L);
      if (st != CBG_OK) break;
      ctx->stream = ctx->branch_streams[i % nb];
      st = boost_one_tree(ctx, &args[i], at<cbg_split>(problems[i].state, L.o_gsplit),
                          at<double>(problems[i].state, L.o_gvals));
      if (st == CBG_OK) record(i);
    }
  } else {
    // every kernel of the round is one launch over all problems, on the origin stream
    join();
    ctx->stream = origin;
    auto launched = [&](const char* what) {
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess && st == CBG_OK) st = fail(ctx, CBG_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    };
    begin_batched_kernel<<<begin_blocks, 256, 0, origin>>>(ltables[0], begin_map);
    launched("batched tree start");
    for (int d = 0; d < depth && st == CBG_OK; ++d) {
      // histograms and their FP64 reduction, one persistent launch for every problem
      const int wait_extra = ctx->test_force_wait_timeout ? 1 : 0;
      const unsigned wait_limit = ctx->test_force_wait_timeout ? 4096u : BATCH_WAIT_LIMIT;
      st = gh_dtype == CBG_F32
               ? launch_hist_batched<float>(ctx, nb_alloc, tables[d], n_problems, L0.threads, cs_plan, false, d,
                                            wait_extra, wait_limit)
               : launch_hist_batched<__nv_bfloat16>(ctx, nb_alloc, tables[d], n_problems, L0.threads, cs_plan,
                                                    false, d, wait_extra, wait_limit);
      if (st != CBG_OK) break;
      const int level_leaves = 1 << d;
      auto score = [&](auto warps) {
        constexpr int W = decltype(warps)::value;
        score_batched_kernel<W><<<score_blocks, W * 32, 0, origin>>>(ltables[d], score_map, level_leaves, l2, d);
      };
      if (level_leaves >= SC_MAX_WARPS) score(std::integral_constant<int, SC_MAX_WARPS>{});
      else if (level_leaves >= 8) score(std::integral_constant<int, 8>{});
      else if (level_leaves >= 4) score(std::integral_constant<int, 4>{});
      else if (level_leaves >= 2) score(std::integral_constant<int, 2>{});
      else score(std::integral_constant<int, 1>{});
      launched("batched scoring");
      const bool last = d == depth - 1;
      flags_batched_kernel<<<tile_blocks, PT_THREADS, 0, origin>>>(ltables[d], tile_map, d, last ? 0 : 1);
      launched("batched partition flags");
      if (!last) {
        scatter_batched_kernel<<<tile_blocks, PT_THREADS, 0, origin>>>(ltables[d], tile_map, d);
        launched("batched partition scatter");
      }
    }
    if (st == CBG_OK) {
      if (gh_dtype == CBG_F32)
        apply_batched_kernel<float><<<apply_blocks, 256, 0, origin>>>(ltables[0], apply_map, depth, l2, lr);
      else
        apply_batched_kernel<__nv_bfloat16><<<apply_blocks, 256, 0, origin>>>(ltables[0], apply_map, depth, l2, lr);
      launched("batched apply");
      record_batched_kernel<<<n_problems, 256, 0, origin>>>(ltables[0], depth, trees);
      launched("batched record");
    }
    fork();
  }
  join();
  ctx->stream = origin;
  ce = cudaStreamEndCapture(origin, &graph);
  ctx->stream = user_stream;
  if (st != CBG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "capture of the batched round failed: %s", cudaGetErrorString(ce));
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "instantiating the batched round failed: %s", cudaGetErrorString(ce));
  for (int t = 0; t < trees; ++t) {
    ce = cudaGraphLaunch(exec, user_stream);
    if (ce != cudaSuccess) break;
  }
  cudaGraphExecDestroy(exec);
  if (ce != cudaSuccess) return fail(ctx, CBG_ECUDA, "batched round launch failed: %s", cudaGetErrorString(ce));
  return CBG_OK;
}

}  // extern "C"

cbg_status cbg_pack_bits1(cbg_ctx* ctx, const uint8_t* bins, int64_t n, int32_t F_pad, uint32_t* bits1) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, F_pad >= GROUP && F_pad % GROUP == 0, "F_pad must be a positive multiple of 32");
  CBG_REQUIRE(ctx, bins && bits1, "NULL argument");
  CBG_REQUIRE(ctx, ((reinterpret_cast<uintptr_t>(bins) | reinterpret_cast<uintptr_t>(bits1)) & 15) == 0,
              "bins and bits1 must be 16-byte aligned");
  DeviceGuard guard(ctx->device);
  const int G = F_pad / GROUP;
  pack_bits1_kernel<<<grid_stride_blocks(static_cast<int64_t>(G) * n, 256), 256, 0, ctx->stream>>>(bins, n, G, bits1,
                                                                                                   ctx->d_status);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

cbg_status cbg_pack_bins4(cbg_ctx* ctx, const uint8_t* bins, int64_t n, int32_t F_pad, uint8_t* bins4) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, F_pad >= GROUP && F_pad % GROUP == 0, "F_pad must be a positive multiple of 32");
  CBG_REQUIRE(ctx, bins && bins4, "NULL argument");
  CBG_REQUIRE(ctx, ((reinterpret_cast<uintptr_t>(bins) | reinterpret_cast<uintptr_t>(bins4)) & 15) == 0,
              "bins and bins4 must be 16-byte aligned");
  DeviceGuard guard(ctx->device);
  const int G = F_pad / GROUP;
  pack_bins4_kernel<<<grid_stride_blocks(static_cast<int64_t>((G + 1) / 2) * n * 2, 256), 256, 0, ctx->stream>>>(
      bins, n, G, bins4, ctx->d_status);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

// ------------------------------------------------------------------ autotuner
namespace {

// The tilings the autotuner times: the shared-reduction kernel with clusters of 1, 2, 4
// or 8 and 2048 or 4096 rows per CTA of a unit; on request its fixed-point form with
// clusters of 4 or 8 and 4096 or 8192 rows; the lane-per-feature kernel and its loader-warp
// form with clusters of 2 and 8192 or 16384 rows; its one-statistic-per-warp form with clusters of 2 or 4 and
// 8192 or 16384 rows; the 16-feature warp-private kernel once; with 4-bit packed bins
// (at most 16 bins), the packed lane-per-feature kernel with clusters of 2 and 8192 or
// 16384 rows; with 1-bit packed bins (at most 2 bins), the 1-bit kernel with clusters of
// 2 and 8192 or 32768 rows.
std::vector<cbg_tiles> autotune_candidates(bool packed, bool fixed_point, bool bits) {
  std::vector<cbg_tiles> c;
  auto add = [&](int kernel, int cluster, int rows) {
    cbg_tiles t{};
    t.kernel = kernel;
    t.cluster = cluster;
    t.rows_per_item = rows;
    c.push_back(t);
  };
  for (int cl : {1, 2, 4, 8})
    for (int r : {2048, 4096}) add(1, cl, r);
  if (fixed_point)
    for (int cl : {4, 8})
      for (int r : {4096, 8192}) add(7, cl, r);
  for (int r : {8192, 16384}) add(4, 2, r);
  for (int r : {8192, 16384}) add(8, 2, r);
  for (int cl : {2, 4})
    for (int r : {8192, 16384}) add(5, cl, r);
  add(2, 2, 8192);
  if (packed)
    for (int r : {8192, 16384}) add(6, 2, r);
  if (bits)
    for (int r : {8192, 32768}) add(9, 2, r);
  return c;
}

cbg_status tune_tree(cbg_ctx* ctx, const cbg_tree_shape* s, const cbg_autotune_args* a) {
  cbg_status st = cbg_tree_begin(ctx, s, a->state, a->state_bytes, a->leaf);
  if (st != CBG_OK) return st;
  for (int d = 0; d < a->depth; ++d) {
    cbg_level_args la{};
    la.shape = s;
    la.state = a->state;
    la.state_bytes = a->state_bytes;
    la.bins = a->bins;
    la.bins_t = a->bins_t;
    la.n_borders = a->n_borders;
    la.g = a->g;
    la.h = a->h;
    la.gh_dtype = a->gh_dtype;
    la.depth = d;
    la.l2 = a->l2;
    la.force_feature = -1;
    la.force_border = -1;
    la.leaf = a->leaf;
    la.splits = a->splits;
    la.child_totals = a->child_totals;
    la.last_level = d == a->depth - 1;
    la.bins4 = a->bins4;
    la.bits1 = a->bits1;
    st = cbg_build_level(ctx, &la);
    if (st != CBG_OK) return st;
  }
  return CBG_OK;
}

}  // namespace

cbg_status cbg_autotune_state_bytes(const cbg_tree_shape* shape, size_t* bytes) {
  if (!shape || !bytes) return CBG_EINVAL;
  size_t mx = 0;
  for (const cbg_tiles& t : autotune_candidates(shape->max_bins <= 16, true, shape->max_bins <= 2)) {
    cbg_tree_shape s = *shape;
    s.tiles = t;
    Layout L;
    cbg_status st = make_layout(nullptr, &s, &L);
    if (st != CBG_OK) return st;
    mx = std::max(mx, L.total);
  }
  *bytes = mx;
  return CBG_OK;
}

cbg_status cbg_autotune_tiles(cbg_ctx* ctx, const cbg_autotune_args* a, cbg_tiles* best, double* best_ms) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, a != nullptr && a->shape != nullptr && best != nullptr && best_ms != nullptr, "NULL argument");
  CBG_REQUIRE(ctx, a->depth >= 1 && a->depth <= a->shape->max_depth, "depth outside [1, max_depth]");
  CBG_REQUIRE(ctx, a->reps >= 1, "reps must be >= 1");
  DeviceGuard guard(ctx->device);
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  CBG_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &capturing));
  CBG_REQUIRE(ctx, capturing == cudaStreamCaptureStatusNone, "the autotuner cannot run while the stream is captured");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CBG_CUDA(ctx, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, CBG_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(ce));
  }
  double best_t = INFINITY;
  cbg_tiles best_c{};
  cbg_status result = CBG_OK;
  for (const cbg_tiles& cand : autotune_candidates(a->bins4 != nullptr && a->shape->max_bins <= 16,
                                                   a->fixed_point != 0,
                                                   a->bits1 != nullptr && a->shape->max_bins <= 2)) {
    cbg_tree_shape s = *a->shape;
    s.tiles = cand;
    Layout L;
    if (make_layout(ctx, &s, &L) != CBG_OK || L.total > a->state_bytes) continue;
    double total = 0.0;
    bool ok = true;
    for (int r = 0; r <= a->reps && ok; ++r) {
      if ((ce = cudaEventRecord(e0, ctx->stream)) != cudaSuccess) break;
      ok = tune_tree(ctx, &s, a) == CBG_OK;
      if (!ok) break;
      if ((ce = cudaEventRecord(e1, ctx->stream)) != cudaSuccess) break;
      if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.f;
      if ((ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (r > 0) total += ms;
    }
    if (ce != cudaSuccess) {
      result = fail(ctx, CBG_ECUDA, "autotuner timing: %s", cudaGetErrorString(ce));
      break;
    }
    if (!ok) {           // a candidate this device or these inputs cannot run
      cudaGetLastError();  // its API error must not surface in the caller's next launch check
      continue;
    }
    const double t = total / a->reps;
    if (t < best_t) {
      best_t = t;
      best_c = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != CBG_OK) return result;
  if (!(best_t < INFINITY)) return fail(ctx, CBG_EINVAL, "no autotuner candidate could run on these inputs");
  *best = best_c;
  *best_ms = best_t;
  return CBG_OK;
}
