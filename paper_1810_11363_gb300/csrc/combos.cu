// Greedy categorical feature combinations (Section 2 "Feature combinations"; Section 5
// "Categorical features": a combination is turned into numbers on the fly by a radix sort
// of its values and a segmented scan, the same machinery as the single columns' TS).
//
// Per level d >= 1 of a tree the host lists the candidates: every item set present in the
// tree (a categorical column, a float split taken as a two-valued column, or a chosen
// combination) joined with every categorical column it lacks, up to max_complexity items,
// without repeats, in lexicographic order of their sorted items. On the GPU, for all
// candidates at once:
//   1. combo_ids_kernel: a SplitMix64 chain over the items' values of every row;
//   2. cbg_ordered_ts, cbg_select_borders, cbg_quantize on the [Nc][n] id columns (only for
//      candidates new to the tree: the columns of earlier levels' candidates are kept);
//   3. cand_hist_kernel: FP64 (G, H) histograms of every candidate over the current leaves
//      (FP32 per block of rows in shared memory, FP64 across blocks);
//   4. cand_score_kernel: the best border of every candidate (Section 3 score, FP64);
//   5. cand_select_kernel / cand_copy_kernel: the best candidate becomes the challenger of
//      the level: cbg_build_level takes it over the best ordinary split only with a
//      strictly higher score, reading its bins and histogram from the copies.
// A chosen combination is recorded as feature F + j (the j-th combination of the tree).
#include <algorithm>
#include <cmath>
#include <set>
#include <type_traits>
#include <vector>

#include "cbg_internal.cuh"

using namespace cbg;

namespace {

constexpr int CB_THREADS = 256;
constexpr int CB_MAX_ITEMS = 16;
constexpr int CB_MAX_DEPTH = 10;
constexpr int64_t CB_HIST_ROWS = 16384;        // rows per block of the candidate histograms
constexpr int CB_HIST_SMEM = 96 * 1024;         // shared (G, H) cells of one block, at most

struct Item {
  int kind, a, b;
  bool operator<(const Item& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (a != o.a) return a < o.a;
    return b < o.b;
  }
  bool operator==(const Item& o) const { return kind == o.kind && a == o.a && b == o.b; }
};

__global__ void combo_ids_kernel(const int* __restrict__ items, const int* __restrict__ n_items, int mc,
                                 const uint32_t* __restrict__ cat, const uint8_t* __restrict__ bins_t, int64_t n,
                                 uint32_t* __restrict__ ids) {
  __shared__ int it[3 * CB_MAX_ITEMS];
  const int j = blockIdx.y;
  const int m = n_items[j];
  if (threadIdx.x < 3 * m) it[threadIdx.x] = items[static_cast<int64_t>(j) * mc * 3 + threadIdx.x];
  __syncthreads();
  uint32_t* out = ids + static_cast<int64_t>(j) * n;
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint64_t h = 0;
    for (int i = 0; i < m; ++i) {
      const int64_t col = static_cast<int64_t>(it[3 * i + 1]) * n + r;
      const uint64_t v = it[3 * i] == 0 ? cat[col] : (bins_t[col] > it[3 * i + 2] ? 1u : 0u);
      h = cbgd::splitmix64_at(h, v);
    }
    out[r] = static_cast<uint32_t>(h ^ (h >> 32));
  }
}

// hist[j][l][b][2] += (g, h) of the rows of leaf l with bin b of the level's candidate j,
// whose column is slot slots[j] of the tree's candidate cache. COPIES > 0: the block's rows
// are summed in FP32 shared cells first, COPIES copies of the level_leaves * cmb float2
// cells (one per group of 256 / COPIES threads, so that fewer threads contend for a cell;
// with few cells and skewed bins the contention, not the row count, sets the time), added
// in copy order; COPIES = 0: FP64 global atomics per row.
template <typename GH, int COPIES>
__global__ void cand_hist_kernel(const uint8_t* __restrict__ cbins_t, const int* __restrict__ slots, int64_t n,
                                 const uint16_t* __restrict__ leaf, int level_leaves, const GH* __restrict__ g,
                                 const GH* __restrict__ h, int cmb, double* __restrict__ hist) {
  extern __shared__ float2 s_h[];
  const int j = blockIdx.y;
  const int cells = level_leaves * cmb;
  const uint8_t* col = cbins_t + static_cast<int64_t>(slots[j]) * n;
  double* hj = hist + static_cast<int64_t>(j) * cells * 2;
  const int64_t r0 = blockIdx.x * CB_HIST_ROWS;
  const int64_t r1 = min(r0 + CB_HIST_ROWS, n);
  float2* mine = s_h;
  if (COPIES > 0) {
    for (int c = threadIdx.x; c < COPIES * cells; c += blockDim.x) s_h[c] = make_float2(0.f, 0.f);
    mine = s_h + (threadIdx.x * COPIES / blockDim.x) * cells;
    __syncthreads();
  }
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int c = (leaf[r] & (level_leaves - 1)) * cmb + col[r];
    const float gv = cbgd::load_gh(g, r), hv = cbgd::load_gh(h, r);
    if (COPIES > 0) {
      atomicAdd(&mine[c].x, gv);
      atomicAdd(&mine[c].y, hv);
    } else {
      atomicAdd(&hj[2 * c], static_cast<double>(gv));
      atomicAdd(&hj[2 * c + 1], static_cast<double>(hv));
    }
  }
  if (COPIES > 0) {
    __syncthreads();
    for (int c = threadIdx.x; c < cells; c += blockDim.x) {
      float2 v = s_h[c];
      for (int k = 1; k < COPIES; ++k) {
        v.x += s_h[k * cells + c].x;
        v.y += s_h[k * cells + c].y;
      }
      if (v.x != 0.f) atomicAdd(&hj[2 * c], static_cast<double>(v.x));
      if (v.y != 0.f) atomicAdd(&hj[2 * c + 1], static_cast<double>(v.y));
    }
  }
}

__device__ __forceinline__ double score_term(double G, double H, double l2) {
  const double den = H + l2;
  return den == 0.0 ? 0.0 : G * G / den;
}

// Best border of candidate j (one block, thread k scores border k): the sum over leaves of
// G_L^2/(H_L+l2) + G_R^2/(H_R+l2), left sums in increasing bin order and right sums from the
// top bin down; ties to the smallest border. best[j] = (score, k) or (-inf, -1).
__global__ void cand_score_kernel(const double* __restrict__ hist, const int32_t* __restrict__ nb,
                                  const int* __restrict__ slots, int level_leaves, int cmb, double l2,
                                  double2* __restrict__ best) {
  __shared__ double row[256][2];
  __shared__ double r_s[CB_THREADS];
  __shared__ int r_k[CB_THREADS];
  const int j = blockIdx.x;
  const int nbj = min(nb[slots[j]], cmb - 1);
  const double* hj = hist + static_cast<int64_t>(j) * level_leaves * cmb * 2;
  const int k = threadIdx.x;
  double sc = 0.0;
  for (int l = 0; l < level_leaves; ++l) {
    __syncthreads();
    for (int b = threadIdx.x; b < cmb; b += blockDim.x) {
      row[b][0] = hj[(static_cast<int64_t>(l) * cmb + b) * 2];
      row[b][1] = hj[(static_cast<int64_t>(l) * cmb + b) * 2 + 1];
    }
    __syncthreads();
    if (k < nbj) {
      double GL = 0.0, HL = 0.0, GR = 0.0, HR = 0.0;
      for (int b = 0; b <= k; ++b) {
        GL += row[b][0];
        HL += row[b][1];
      }
      for (int b = cmb - 1; b > k; --b) {
        GR += row[b][0];
        HR += row[b][1];
      }
      sc += score_term(GL, HL, l2) + score_term(GR, HR, l2);
    }
  }
  r_s[threadIdx.x] = k < nbj ? sc : -INFINITY;
  r_k[threadIdx.x] = k < nbj ? k : -1;
  __syncthreads();
  for (int o = CB_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const int ok = r_k[threadIdx.x + o];
      const double os = r_s[threadIdx.x + o];
      const int mk = r_k[threadIdx.x];
      if (ok >= 0 && (mk < 0 || os > r_s[threadIdx.x] || (os == r_s[threadIdx.x] && ok < mk))) {
        r_s[threadIdx.x] = os;
        r_k[threadIdx.x] = ok;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) best[j] = make_double2(r_s[0], static_cast<double>(r_k[0]));
}

// The best candidate (strictly higher score; ties to the first) becomes the challenger
// split {feature, border, score}; feature -1 when no candidate has a border.
__global__ void cand_select_kernel(const double2* __restrict__ best, int n_cand, int feature,
                                   cbg_split* __restrict__ chal, int* __restrict__ chal_idx) {
  if (threadIdx.x != 0) return;
  int bj = -1;
  double bs = -INFINITY;
  for (int j = 0; j < n_cand; ++j) {
    const double2 v = best[j];
    if (v.y >= 0.0 && (bj < 0 || v.x > bs)) {
      bj = j;
      bs = v.x;
    }
  }
  chal->feature = bj >= 0 ? feature : -1;
  chal->border = bj >= 0 ? static_cast<int>(best[bj].y) : -1;
  chal->score = bs;
  *chal_idx = bj;
}

// Copies the winning candidate's bins column and histogram next to the challenger split.
__global__ void cand_copy_kernel(const int* __restrict__ chal_idx, const int* __restrict__ slots,
                                 const uint8_t* __restrict__ cbins_t, int64_t n, const double* __restrict__ hist,
                                 int64_t hist_elems, uint8_t* __restrict__ chal_bins, double* __restrict__ chal_hist) {
  const int j = *chal_idx;
  if (j < 0) return;
  const uint8_t* col = cbins_t + static_cast<int64_t>(slots[j]) * n;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n; r += stride)
    chal_bins[r] = col[r];
  const double* hj = hist + static_cast<int64_t>(j) * hist_elems;
  for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < hist_elems; x += stride)
    chal_hist[x] = hj[x];
}

struct ComboWork {
  int* items;          // [Nc_max][mc][3]
  int* n_items;        // [Nc_max]
  uint32_t* ids;       // [Nc_max][n]
  float* ts;           // [Nc_max][n]
  float* borders;      // [Nc_max][max_borders]
  int32_t* nb;         // [Nc_max]
  uint8_t* cbins;      // grouped [pad32(Nc_max) / 32][n][32]
  uint8_t* cbins_t;    // [Nc_max][n]
  double* hist;        // [Nc_max][2^(depth-1)][cmb][2]
  double2* best;       // [Nc_max]
  int* slots;          // [Nc_max] cache slot of each candidate of the level
  cbg_split* chal;
  int* chal_idx;
  uint8_t* chal_bins;  // [n]
  double* chal_hist;   // [2^(depth-1)][cmb][2]
  size_t bytes;
};

int max_candidates(int C, int depth) { return std::max(1, (depth - 1) * C); }

ComboWork carve_combo(void* base, int64_t n, int C, int depth, int max_borders, int mc) {
  Carve c(base);
  ComboWork w;
  const int nc = max_candidates(C, depth);
  const int cmb = max_borders + 1;
  const size_t lh = static_cast<size_t>(1) << (depth - 1);
  w.items = c.take<int>(static_cast<size_t>(nc) * mc * 3);
  w.n_items = c.take<int>(nc);
  w.ids = c.take<uint32_t>(static_cast<size_t>(nc) * n);
  w.ts = c.take<float>(static_cast<size_t>(nc) * n);
  w.borders = c.take<float>(static_cast<size_t>(nc) * max_borders);
  w.nb = c.take<int32_t>(nc);
  w.cbins = c.take<uint8_t>(static_cast<size_t>((nc + 31) / 32 * 32) * n);
  w.cbins_t = c.take<uint8_t>(static_cast<size_t>(nc) * n);
  w.hist = c.take<double>(static_cast<size_t>(nc) * lh * cmb * 2);
  w.best = c.take<double2>(nc);
  w.slots = c.take<int>(nc);
  w.chal = c.take<cbg_split>(1);
  w.chal_idx = c.take<int>(1);
  w.chal_bins = c.take<uint8_t>(static_cast<size_t>(n));
  w.chal_hist = c.take<double>(lh * cmb * 2);
  w.bytes = c.off;
  return w;
}

unsigned grid_for(int64_t n, int per_y) {
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, CB_THREADS), 152LL * 8 / per_y + 1)));
}

// Candidates of level d: every present set joined with every categorical column it lacks.
std::vector<std::vector<Item>> candidates(const std::vector<std::vector<Item>>& present, int C, int mc) {
  std::set<std::vector<Item>> out;
  for (const auto& p : present)
    for (int c = 0; c < C; ++c) {
      const Item it{0, c, 0};
      if (std::find(p.begin(), p.end(), it) != p.end() || static_cast<int>(p.size()) + 1 > mc) continue;
      std::vector<Item> q = p;
      q.push_back(it);
      std::sort(q.begin(), q.end());
      out.insert(q);
    }
  return std::vector<std::vector<Item>>(out.begin(), out.end());
}

// The columns of a tree's candidates are cached: a candidate's ids, TS, borders and bins
// depend only on its items, so each is computed once per tree, at the first level that
// lists it, into the next free slot (slots are handed out in order, so the new columns of a
// level are contiguous). The histograms, scores and the choice run over all of the level's
// candidates. Runs steps 1-5 of the file comment; the challenger is left in w.chal.
struct CandidateCache {
  std::vector<std::vector<Item>> by_slot;
  int find(const std::vector<Item>& q) const {
    for (size_t i = 0; i < by_slot.size(); ++i)
      if (by_slot[i] == q) return static_cast<int>(i);
    return -1;
  }
};

cbg_status challenger_for_level(cbg_ctx* ctx, const cbg_combo_args* a, const ComboWork& w, CandidateCache& cache,
                                const std::vector<std::vector<Item>>& cands, int d, int feature,
                                std::vector<int>* slots_out) {
  const int64_t n = a->shape->n;
  const int nc = static_cast<int>(cands.size());
  const int mc = a->max_complexity;
  const int cmb = a->max_borders + 1;
  const int level_leaves = 1 << d;
  std::vector<int>& slots = *slots_out;
  slots.assign(nc, -1);
  const int slot0 = static_cast<int>(cache.by_slot.size());
  std::vector<int> items, n_items;
  for (int j = 0; j < nc; ++j) {
    slots[j] = cache.find(cands[j]);
    if (slots[j] >= 0) continue;
    slots[j] = static_cast<int>(cache.by_slot.size());
    cache.by_slot.push_back(cands[j]);
    n_items.push_back(static_cast<int>(cands[j].size()));
    for (int i = 0; i < mc; ++i) {
      const bool used = i < static_cast<int>(cands[j].size());
      items.push_back(used ? cands[j][i].kind : -1);
      items.push_back(used ? cands[j][i].a : -1);
      items.push_back(used ? cands[j][i].b : -1);
    }
  }
  const int n_new = static_cast<int>(n_items.size());
  CBG_REQUIRE(ctx, slot0 + n_new <= max_candidates(a->C, a->depth), "candidate cache overflow");
  if (n_new > 0) {
    CBG_CUDA(ctx, cudaMemcpyAsync(w.items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice,
                                  ctx->stream));
    CBG_CUDA(ctx, cudaMemcpyAsync(w.n_items, n_items.data(), n_items.size() * sizeof(int), cudaMemcpyHostToDevice,
                                  ctx->stream));
    uint32_t* ids = w.ids + static_cast<int64_t>(slot0) * n;
    float* ts = w.ts + static_cast<int64_t>(slot0) * n;
    combo_ids_kernel<<<dim3(grid_for(n, n_new), n_new), CB_THREADS, 0, ctx->stream>>>(w.items, w.n_items, mc, a->cat,
                                                                                      a->bins_t, n, ids);
    CBG_CHECK_LAUNCH(ctx);
    cbg_status st = cbg_ordered_ts(ctx, ids, a->y, n, n_new, a->perm, a->prior, a->a, a->label_kind, ts, nullptr,
                                   nullptr);
    if (st != CBG_OK) return st;
    st = cbg_select_borders(ctx, ts, n, n_new, a->max_borders, w.borders + static_cast<int64_t>(slot0) * a->max_borders,
                            w.nb + slot0);
    if (st != CBG_OK) return st;
    st = cbg_quantize(ctx, ts, n, n_new, w.borders + static_cast<int64_t>(slot0) * a->max_borders, w.nb + slot0,
                      a->max_borders, w.cbins, (n_new + 31) / 32 * 32, 0, w.cbins_t + static_cast<int64_t>(slot0) * n);
    if (st != CBG_OK) return st;
  }
  CBG_CUDA(ctx, cudaMemcpyAsync(w.slots, slots.data(), slots.size() * sizeof(int), cudaMemcpyHostToDevice,
                                ctx->stream));
  const int64_t hist_elems = static_cast<int64_t>(level_leaves) * cmb * 2;
  CBG_CUDA(ctx, cudaMemsetAsync(w.hist, 0, sizeof(double) * hist_elems * nc, ctx->stream));
  const dim3 hgrid(static_cast<unsigned>(ceil_div(n, CB_HIST_ROWS)), nc);
  const int cell_bytes = static_cast<int>(sizeof(float2)) * level_leaves * cmb;
  const bool f32 = a->gh_dtype == CBG_F32;
  auto launch = [&](auto copies) {
    constexpr int K = decltype(copies)::value;
    const int smem = K > 0 ? K * cell_bytes : 0;
    if (f32)
      cand_hist_kernel<float, K><<<hgrid, CB_THREADS, smem, ctx->stream>>>(
          w.cbins_t, w.slots, n, a->leaf, level_leaves, static_cast<const float*>(a->g),
          static_cast<const float*>(a->h), cmb, w.hist);
    else
      cand_hist_kernel<__nv_bfloat16, K><<<hgrid, CB_THREADS, smem, ctx->stream>>>(
          w.cbins_t, w.slots, n, a->leaf, level_leaves, static_cast<const __nv_bfloat16*>(a->g),
          static_cast<const __nv_bfloat16*>(a->h), cmb, w.hist);
  };
  if (8 * cell_bytes <= CB_HIST_SMEM) launch(std::integral_constant<int, 8>{});
  else if (cell_bytes <= CB_HIST_SMEM) launch(std::integral_constant<int, 1>{});
  else launch(std::integral_constant<int, 0>{});
  CBG_CHECK_LAUNCH(ctx);
  cand_score_kernel<<<nc, CB_THREADS, 0, ctx->stream>>>(w.hist, w.nb, w.slots, level_leaves, cmb, a->l2, w.best);
  CBG_CHECK_LAUNCH(ctx);
  cand_select_kernel<<<1, 32, 0, ctx->stream>>>(w.best, nc, feature, w.chal, w.chal_idx);
  CBG_CHECK_LAUNCH(ctx);
  cand_copy_kernel<<<grid_for(n, 1), CB_THREADS, 0, ctx->stream>>>(w.chal_idx, w.slots, w.cbins_t, n, w.hist,
                                                                  hist_elems, w.chal_bins, w.chal_hist);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}

}  // namespace

extern "C" {

cbg_status cbg_combo_work_bytes(int64_t n, int32_t C, int32_t depth, int32_t max_borders, int32_t max_complexity,
                                size_t* bytes) {
  if (!bytes || n < 1 || n > INT32_MAX || C < 0 || depth < 1 || depth > CB_MAX_DEPTH || max_borders < 1 ||
      max_borders > 254 || max_complexity < 1 || max_complexity > CB_MAX_ITEMS)
    return CBG_EINVAL;
  *bytes = carve_combo(nullptr, n, C, depth, max_borders, max_complexity).bytes;
  return CBG_OK;
}

cbg_status cbg_combo_ids(cbg_ctx* ctx, const cbg_combo_item* items, int32_t n_items, const uint32_t* cat, int32_t C,
                         const uint8_t* bins_t, int32_t F, int64_t n, uint32_t* ids) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, items != nullptr && n_items >= 1 && n_items <= CB_MAX_ITEMS, "need 1..16 items");
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX && ids != nullptr, "need n in [1, 2^31-1] and ids");
  std::vector<int> flat(3 * static_cast<size_t>(n_items));
  for (int i = 0; i < n_items; ++i) {
    const cbg_combo_item& it = items[i];
    CBG_REQUIRE(ctx, (it.kind == 0 && it.a >= 0 && it.a < C && cat) || (it.kind == 1 && it.a >= 0 && it.a < F && bins_t),
                "item %d names no column of cat or bins_t", i);
    bool ordered = true;
    if (i > 0) {
      Item prev, cur;
      prev.kind = items[i - 1].kind;
      prev.a = items[i - 1].a;
      prev.b = items[i - 1].b;
      cur.kind = it.kind;
      cur.a = it.a;
      cur.b = it.b;
      ordered = prev < cur;
    }
    CBG_REQUIRE(ctx, ordered, "items must be sorted by (kind, a, b) without repeats");
    flat[3 * i] = it.kind;
    flat[3 * i + 1] = it.a;
    flat[3 * i + 2] = it.b;
  }
  DeviceGuard guard(ctx->device);
  cbg_status st = ws_reserve(ctx, 4096);
  if (st != CBG_OK) return st;
  int* d_items = static_cast<int*>(ctx->ws);
  int* d_n = d_items + 3 * CB_MAX_ITEMS;
  CBG_CUDA(ctx, cudaMemcpyAsync(d_items, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CBG_CUDA(ctx, cudaMemcpyAsync(d_n, &n_items, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  combo_ids_kernel<<<dim3(grid_for(n, 1), 1), CB_THREADS, 0, ctx->stream>>>(d_items, d_n, n_items, cat, bins_t, n, ids);
  CBG_CHECK_LAUNCH(ctx);
  // the host arrays above must outlive the copies: wait for them
  CBG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return CBG_OK;
}

cbg_status cbg_boost_combos(cbg_ctx* ctx, const cbg_combo_args* a) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, a != nullptr && a->shape != nullptr, "args is NULL");
  const cbg_tree_shape* sh = a->shape;
  const int64_t n = sh->n;
  const int D = a->depth;
  const int F = sh->F;
  const int C = a->C;
  const int mc = a->max_complexity;
  CBG_REQUIRE(ctx, n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31-1]");
  CBG_REQUIRE(ctx, D >= 1 && D <= sh->max_depth && D <= CB_MAX_DEPTH, "depth outside [1, max_depth]");
  CBG_REQUIRE(ctx, C >= 0 && a->F_float >= 0 && a->F_float + C == F, "F must equal F_float + C");
  CBG_REQUIRE(ctx, a->max_borders >= 1 && a->max_borders <= 254, "max_borders must be in [1, 254]");
  CBG_REQUIRE(ctx, mc >= 1 && mc <= CB_MAX_ITEMS, "max_complexity must be in [1, 16]");
  CBG_REQUIRE(ctx, a->trees >= 0, "trees must be >= 0");
  CBG_REQUIRE(ctx, a->bins && a->bins_t && a->n_borders && a->y && a->pred && a->g && a->h && a->leaf && a->splits &&
                       a->leaf_values && a->child_totals && a->work && (C == 0 || (a->cat && a->perm)),
              "NULL argument");
  CBG_REQUIRE(ctx, a->combo_items && a->combo_nb && a->combo_borders, "NULL host output");
  const ComboWork w = carve_combo(a->work, n, C, D, a->max_borders, mc);
  CBG_REQUIRE(ctx, a->work_bytes >= w.bytes, "work holds %zu bytes, %zu needed", a->work_bytes, w.bytes);
  DeviceGuard guard(ctx->device);
  const int cmb = a->max_borders + 1;
  if (static_cast<int>(sizeof(float2)) * (1 << (D - 1)) * cmb <= CB_HIST_SMEM) {
    CBG_CUDA(ctx, cudaFuncSetAttribute(cand_hist_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       CB_HIST_SMEM));
    CBG_CUDA(ctx, cudaFuncSetAttribute(cand_hist_kernel<__nv_bfloat16, 1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, CB_HIST_SMEM));
    CBG_CUDA(ctx, cudaFuncSetAttribute(cand_hist_kernel<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       CB_HIST_SMEM));
    CBG_CUDA(ctx, cudaFuncSetAttribute(cand_hist_kernel<__nv_bfloat16, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, CB_HIST_SMEM));
  }
  const int L = 1 << D;
  cbg_status st = cbg_gradients(ctx, a->loss, a->y, a->pred, n, a->gh_dtype, a->g, a->h);
  if (st != CBG_OK) return st;
  for (int t = 0; t < a->trees; ++t) {
    cbg_split* sp = a->splits + static_cast<int64_t>(t) * D;
    st = cbg_tree_begin(ctx, sh, a->state, a->state_bytes, a->leaf);
    if (st != CBG_OK) return st;
    std::vector<std::vector<Item>> present;
    CandidateCache cache;
    std::vector<int> slots;
    int n_combo = 0;
    for (int d = 0; d < D; ++d) {
      const int64_t rec = static_cast<int64_t>(t) * D + d;
      for (int i = 0; i < mc; ++i) a->combo_items[rec * mc + i] = cbg_combo_item{-1, -1, -1};
      a->combo_nb[rec] = 0;
      std::fill(a->combo_borders + rec * a->max_borders, a->combo_borders + (rec + 1) * a->max_borders, 0.0f);
      std::vector<std::vector<Item>> cands;
      if (d >= 1 && C > 0) cands = candidates(present, C, mc);
      if (!cands.empty()) {
        st = challenger_for_level(ctx, a, w, cache, cands, d, F + n_combo, &slots);
        if (st != CBG_OK) return st;
      }
      cbg_level_args la{};
      la.shape = sh;
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
      la.last_level = d == D - 1;
      if (!cands.empty()) {
        la.challenger = w.chal;
        la.challenger_bins = w.chal_bins;
        la.challenger_hist = w.chal_hist;
        la.challenger_max_bins = cmb;
      }
      st = cbg_build_level(ctx, &la);
      if (st != CBG_OK) return st;
      // the split taken decides the items present at the next level
      cbg_split got;
      int win = -1;
      CBG_CUDA(ctx, cudaMemcpyAsync(&got, sp + d, sizeof(got), cudaMemcpyDeviceToHost, ctx->stream));
      if (!cands.empty())
        CBG_CUDA(ctx, cudaMemcpyAsync(&win, w.chal_idx, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CBG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (got.feature >= F) {
        CBG_REQUIRE(ctx, win >= 0 && got.feature == F + n_combo, "combination split without a candidate");
        const auto& q = cands[win];
        for (size_t i = 0; i < q.size(); ++i) a->combo_items[rec * mc + i] = cbg_combo_item{q[i].kind, q[i].a, q[i].b};
        int32_t nb = 0;
        const int slot = slots[win];
        CBG_CUDA(ctx, cudaMemcpy(&nb, w.nb + slot, sizeof(nb), cudaMemcpyDeviceToHost));
        a->combo_nb[rec] = nb;
        if (nb > 0)
          CBG_CUDA(ctx, cudaMemcpy(a->combo_borders + rec * a->max_borders,
                                   w.borders + static_cast<int64_t>(slot) * a->max_borders, sizeof(float) * nb,
                                   cudaMemcpyDeviceToHost));
        if (std::find(present.begin(), present.end(), q) == present.end()) present.push_back(q);
        ++n_combo;
      } else if (got.feature >= 0) {
        Item it;
        if (got.feature < a->F_float) {
          it.kind = 1;
          it.a = got.feature;
          it.b = got.border;
        } else {
          it.kind = 0;
          it.a = got.feature - a->F_float;
          it.b = 0;
        }
        const std::vector<Item> p(1, it);
        if (std::find(present.begin(), present.end(), p) == present.end()) present.push_back(p);
      }
    }
    cbg_apply_args aa{};
    aa.bins = a->bins;
    aa.n = n;
    aa.F_pad = sh->F_pad;
    aa.splits = sp;
    aa.depth = D;
    aa.leaf_totals = a->child_totals;
    aa.l2 = a->l2;
    aa.lr = a->lr;
    aa.leaf_in = a->leaf;
    aa.pred = a->pred;
    aa.leaf_values_out = a->leaf_values + static_cast<int64_t>(t) * L;
    aa.y = a->y;
    aa.loss = a->loss;
    aa.gh_dtype = a->gh_dtype;
    aa.g = a->g;
    aa.h = a->h;
    st = cbg_apply_tree(ctx, &aa);
    if (st != CBG_OK) return st;
  }
  return CBG_OK;
}

}  // extern "C"
