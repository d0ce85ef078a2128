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
#include <type_traits>

#include "cbg_internal.cuh"

namespace {

constexpr int GROUP = 32;          // features per group / histogram slab
// Shared memory a CTA may take: the 227 KB opt-in limit less 1 KB kept for the kernels'
// static shared variables (the work-queue slot, cluster bookkeeping).
constexpr int SMEM_DYN_BUDGET = 227 * 1024 - 1024;
constexpr int MAX_DEPTH = 10;
constexpr int MAX_HLEAVES = 1 << (MAX_DEPTH - 1);  // leaves histogrammed at the last level

// Work of one level's histogram launch. The directly computed leaves are listed by
// decreasing rows per CTA (largest work items first), each split into chunk units; work
// item u * G + g is unit u of feature group g. Every cluster of a launch takes its next
// item from `queue` (reset to 0 by whoever writes the plan and by the reduction that
// follows the launch), so the items spread over the clusters as they finish.
struct Plan {
  int n_small;                      // leaves histogrammed directly at this level
  int total_units;                  // sum of chunks over those leaves
  int level_leaves;                 // 2^d
  int queue;                        // next work item of the running histogram launch
  int rqueue;                       // batched form: next reduction chunk of the running launch
  int done[MAX_HLEAVES];            // batched form: work items of leaf jj whose partials are written
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
// histograms of 16 features per warp; kind 1: one shared histogram per CTA updated with
// shared-memory float reductions; kind 3: the same with 64-bit compare-and-swap; kind 4:
// lane-per-feature warp histograms with batched updates; kind 5: the same with G and H
// in separate warps; kind 6: kind 4 over 4-bit packed bins; kind 7: kind 1 with int32
// fixed-point cells and integer reductions. Kinds 4-7 read (g, h) by position, the
// others by row.
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
  const int fit = static_cast<int>(SMEM_DYN_BUDGET / (static_cast<size_t>(max_bins) * WP_FEATS * sizeof(float2)));
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
// Signed int32 reduction: two's-complement addition is the unsigned one.
__device__ __forceinline__ void red_add_s32(uint32_t addr, int v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Fixed-point scale of the integer histogram: the largest e with 2^e * bound < 2^30, where
// bound >= the sum of |v| over a CTA's rows (the float sum, inflated by 0.1% to cover its
// rounding). Then every cell's sum of the rounded v * 2^e stays below 2^30 + rows < 2^31 in
// magnitude. e is clamped to [-120, 120]; an all-zero chunk takes e = 0.
__device__ __forceinline__ int fixed_scale_exp(float abs_sum) {
  const float b = abs_sum * 1.001f;
  if (!(b > 0.f)) return 0;
  if (!(b < 1e30f)) return -120;
  int k;
  frexpf(b, &k);   // b < 2^k
  const int e = 30 - k;
  return e < -120 ? -120 : (e > 120 ? 120 : e);
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }          // |e| <= 126

// The 32-bit finaliser of MurmurHash3 (Appleby): a bijection that mixes every input bit.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// floor(x + u) for u in [0, 1): dithered rounding of a fixed-point value. Values that
// repeat across rows (after a few trees g takes one value per leaf and label) would all
// round the same way under round-to-nearest, and their errors would add up linearly; a
// dither drawn per row makes the errors independent with mean zero. x - floor(x) is exact
// in FP32 for x >= 0 and for negative x with |x| not below 2^-24 |floor(x)|; a tinier
// negative x gives 1 + x = 1 after rounding and so always rounds to 0 (no dither there).
// The sum with u rounds too, which moves the result only when that sum lies within an
// ulp of 1. In every case the error is below one unit.
__device__ __forceinline__ int dither_round(float x, float u) {
  const float xi = floorf(x);
  return __float2int_rz(xi) + ((x - xi) + u >= 1.f ? 1 : 0);
}
__device__ __forceinline__ double pow2d(int e) {   // |e| <= 1022
  return __longlong_as_double(static_cast<long long>(1023 + e) << 52);
}

// Persistent kernel over work units (leaf chunk x feature group), launched as thread-block
// clusters of cs CTAs. Each CTA of a cluster accumulates the (G, H) histogram of its
// sub-chunk of rows in its own shared memory (FP32, red.shared.add). After a cluster
// barrier, CTA r sums its slice of bins across the cs CTAs through distributed shared
// memory and writes it to the unit's FP32 partial, so one partial is written per cluster
// and unit. Lane (j, c): row j of 16, 16-feature chunk c of the group; iteration l
// updates feature 16c + (l + j) % 16, so the 32 lanes hit 32 different features and banks
// (the rotation of the paper's Section 5 example, applied to 16-byte loads). Chunks that
// hold only padding features are skipped.
// MODE 0: G and H in two planes [2][NB][32], each updated with red.shared.add.f32.
// MODE 1: (G, H) interleaved as float2 [NB][32], updated with one 64-bit compare-and-swap
// loop per (row, feature); on sm_103a the FP32 shared reduction is itself a
// compare-and-swap loop, so this halves the atomic operations.
// MODE 2: G and H in two int32 planes, updated with the native integer reduction
// red.shared.add.u32 of fixed-point values floor(g * 2^eg + u), floor(h * 2^eh + u'), u
// and u' dithers hashed from the position, with (g, h) read by position (the copies the
// partition moves along with the rows). A pre-pass over the CTA's rows sums |g| and |h|,
// and each scale is the largest power of two that keeps every cell below 2^31
// (fixed_scale_exp). Integer sums are exact, so the CTA's histogram does not depend on
// the order of its updates. The cluster step converts each CTA's cells with its own scale
// (exact in FP64), sums them in rank order and rounds once to the FP32 partial. Per row
// the error is below 2^-e <= 2.002 * (sum of |g| over the CTA's rows) * 2^-30, with mean
// zero; integer-valued g with e >= 0 is exact.
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

// One problem's inputs to a histogram launch (the batched form passes a table of them).
struct HistProblem {
  const uint8_t* bins;
  int64_t n;
  int G, F;
  const uint32_t* order;    // row order of the level (NULL: identity)
  const void* g;            // gradients / hessians (by row), GH
  const void* h;
  const Plan* plan;
  int max_bins;
  float* partials;
  // the batched form also reduces the partials into the level's FP64 histogram
  const double* hist_prev;
  double* hist_cur;
  const cbg_split* splits;
  float2* hist_df;
  const int32_t* n_borders;
};

// One work item (unit x group) of one problem, for this CTA of the cluster: accumulate
// the item's rows into the CTA's shared histogram, then sum this CTA's slice of bins over
// the cluster (distributed shared memory) into the item's FP32 partial.
// Work-item queue of a single-problem launch: thread 0 of cluster rank 0 takes the next
// item and writes it into the same shared slot of every CTA of the cluster (distributed
// shared memory); each CTA then reads only its own slot. The writes happen between the
// two cluster barriers of an item (every CTA has read the current item before the first
// and reads the next one after the second), and no CTA touches another CTA's shared
// memory after the last barrier, so a CTA may exit as soon as it finds the queue empty.
// Before the first take the cluster synchronises once, so that every CTA has started.
__device__ __forceinline__ void queue_take(const Plan* plan, int* slot, int cs) {
  const int v = atomicAdd(&const_cast<Plan*>(plan)->queue, 1);   // the launch's counter (see Plan::queue)
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  for (int r = 0; r < cs; ++r) *cl.map_shared_rank(slot, r) = v;
}
__device__ __forceinline__ int queue_read(const int* slot) { return *reinterpret_cast<const volatile int*>(slot); }

template <typename GH, int NB, int MODE>
__device__ __forceinline__ void hist_item(const HistProblem& P, int item, int cs, int rank, float* hsh,
                                          const float* const* peer, uint32_t sbase, int* next_slot = nullptr,
                                          const Plan* queue_plan = nullptr, bool signal_done = false) {
  namespace cgr = cooperative_groups;
  constexpr int PLANE = NB * GROUP;
  __shared__ int s_exp[2];   // MODE 2: this CTA's fixed-point exponents of G and H
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int j = lane >> 1, c = lane & 1;
  const uint32_t cbase = sbase + 64u * static_cast<uint32_t>(c);   // lane (j, c) updates feature 16c + (l + j) % 16 at step l
  const Plan* plan = P.plan;
  const int G = P.G;
  const int unit = item / G, grp = item - unit * G;
  // leaf of this unit: last jj with unit_begin[jj] <= unit
  int lo = 0, hi = plan->n_small - 1;
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
  // zero the rows the problem's bins use (rows at or above max_bins are never read)
  if (MODE != 1) {   // two planes [NB][32] (float, or int32 for MODE 2)
    const int rows4 = P.max_bins * GROUP / 4;   // float4 per plane
    for (int i = threadIdx.x; i < 2 * rows4; i += blockDim.x) {
      const int st = i / rows4;
      reinterpret_cast<float4*>(hsh + st * PLANE)[i - st * rows4] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else {           // interleaved [NB][32] float2
    for (int i = threadIdx.x; i < P.max_bins * GROUP / 2; i += blockDim.x)
      reinterpret_cast<float4*>(hsh)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const GH* g = static_cast<const GH*>(P.g);
  const GH* h = static_cast<const GH*>(P.h);
  const uint32_t* order = P.order;
  float scale_g = 1.f, scale_h = 1.f;
  if constexpr (MODE == 2) {
    // pre-pass: sums of |g| and |h| over this CTA's rows, reduced in a fixed order
    __shared__ float s_abs[2][32];
    float ag = 0.f, ah = 0.f;
#pragma unroll 4
    for (int pos = p0 + static_cast<int>(threadIdx.x); pos < p1; pos += blockDim.x) {
      ag += fabsf(cbgd::load_gh(g, pos));   // (g, h) by position
      ah += fabsf(cbgd::load_gh(h, pos));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ag += __shfl_down_sync(0xffffffffu, ag, o);
      ah += __shfl_down_sync(0xffffffffu, ah, o);
    }
    if (lane == 0) {
      s_abs[0][warp] = ag;
      s_abs[1][warp] = ah;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float tg = 0.f, th = 0.f;
      for (int w = 0; w < nw; ++w) {
        tg += s_abs[0][w];
        th += s_abs[1][w];
      }
      s_exp[0] = fixed_scale_exp(tg);
      s_exp[1] = fixed_scale_exp(th);
    }
    __syncthreads();
    scale_g = pow2f(s_exp[0]);
    scale_h = pow2f(s_exp[1]);
  }
  __syncthreads();
  const bool active = grp * GROUP + c * 16 < P.F;
  const uint8_t* gbase = P.bins + static_cast<int64_t>(grp) * P.n * GROUP + c * 16;
  if (active) {
    // software-pipelined over rows: the row id two rows ahead, and the next row's bin record
    // and (g, h), are loaded before this row's 32 reductions issue, so their latency
    // overlaps the shared-memory work. MODE 2 reads (g, h) by position.
    const int stride = nw * 16;
    int pos = p0 + warp * 16 + j;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    float gv = 0.f, hv = 0.f;
    uint32_t rn = 0;   // row id at pos + stride
    if (pos < p1) {
      const uint32_t row = order ? order[pos] : static_cast<uint32_t>(pos);
      v = __ldg(reinterpret_cast<const uint4*>(gbase + static_cast<int64_t>(row) * GROUP));
      gv = cbgd::load_gh(g, MODE == 2 ? static_cast<uint32_t>(pos) : row);
      hv = cbgd::load_gh(h, MODE == 2 ? static_cast<uint32_t>(pos) : row);
      if (pos + stride < p1) rn = order ? order[pos + stride] : static_cast<uint32_t>(pos + stride);
    }
    for (; pos < p1; pos += stride) {
      const int nxt = pos + stride, nn = nxt + stride;
      uint32_t rnn = 0;
      if (nn < p1) rnn = order ? order[nn] : static_cast<uint32_t>(nn);
      uint4 vn = make_uint4(0u, 0u, 0u, 0u);
      float gn = 0.f, hn = 0.f;
      if (nxt < p1) {
        vn = __ldg(reinterpret_cast<const uint4*>(gbase + static_cast<int64_t>(rn) * GROUP));
        gn = cbgd::load_gh(g, MODE == 2 ? static_cast<uint32_t>(nxt) : rn);
        hn = cbgd::load_gh(h, MODE == 2 ? static_cast<uint32_t>(nxt) : rn);
      }
      int qg = 0, qh = 0;
      if (MODE == 2) {
        // dithers of this position (the same for every feature group of the level)
        const uint32_t d1 = fmix32(static_cast<uint32_t>(pos) * 0x9e3779b9u + 0x7f4a7c15u);
        const uint32_t d2 = fmix32(d1);
        qg = dither_round(gv * scale_g, static_cast<float>(d1 >> 8) * 0x1p-24f);   // gv * 2^e is exact
        qh = dither_round(hv * scale_h, static_cast<float>(d2 >> 8) * 0x1p-24f);
      }
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
        const uint32_t fo = 4u * static_cast<uint32_t>((l + j) & 15);   // 4 x feature within the chunk
        if (MODE == 0) {
          const uint32_t a = cbase + fo + b * (GROUP * 4);
          red_add(a, gv);
          red_add(a + PLANE * 4, hv);
        } else if (MODE == 2) {
          const uint32_t a = cbase + fo + b * (GROUP * 4);
          red_add_s32(a, qg);
          red_add_s32(a + PLANE * 4, qh);
        } else {
          const uint32_t f = static_cast<uint32_t>(c * 16) + (fo >> 2);
          cas_add2(reinterpret_cast<float2*>(hsh) + b * GROUP + f, gv, hv);
        }
      }
      v = vn;
      gv = gn;
      hv = hn;
      rn = rnn;
    }
  }
  cgr::this_cluster().sync();
  if (next_slot != nullptr && rank == 0 && threadIdx.x == 0)
    queue_take(queue_plan != nullptr ? queue_plan : P.plan, next_slot, cs);
  // this CTA's slice of bins, summed over the cluster's CTAs in rank order
  const int max_bins = P.max_bins;
  const int bs = (max_bins + cs - 1) / cs;
  const int b0 = rank * bs;
  const int nbs = max(0, min(max_bins, b0 + bs) - b0);
  float* dst = P.partials + static_cast<int64_t>(item) * (2 * max_bins * GROUP);
  if constexpr (MODE == 2) {
    // each peer's cells back to real units with that peer's scales (exact in FP64)
    __shared__ double s_inv[2][16];
    if (static_cast<int>(threadIdx.x) < cs) {
      const int* e = cgr::this_cluster().map_shared_rank(s_exp, static_cast<int>(threadIdx.x));
      s_inv[0][threadIdx.x] = pow2d(-e[0]);
      s_inv[1][threadIdx.x] = pow2d(-e[1]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * nbs * GROUP; i += blockDim.x) {
      const int st = i / (nbs * GROUP), rem = i - st * (nbs * GROUP);
      const int e = st * PLANE + b0 * GROUP + rem;
      double v = 0.0;
#pragma unroll 4
      for (int r = 0; r < cs; ++r) v += static_cast<double>(reinterpret_cast<const int*>(peer[r])[e]) * s_inv[st][r];
      dst[st * (max_bins * GROUP) + b0 * GROUP + rem] = static_cast<float>(v);
    }
  } else {
    for (int i = threadIdx.x; i < 2 * nbs * GROUP; i += blockDim.x) {
      const int st = i / (nbs * GROUP), rem = i - st * (nbs * GROUP);
      const int e = MODE == 0 ? st * PLANE + b0 * GROUP + rem : (b0 * GROUP + rem) * 2 + st;
      float v = 0.f;
#pragma unroll 4
      for (int r = 0; r < cs; ++r) v += peer[r][e];
      dst[st * (max_bins * GROUP) + b0 * GROUP + rem] = v;
    }
  }
  if (signal_done) __threadfence();   // this CTA's partial slice, visible before the count below
  cgr::this_cluster().sync();
  // every CTA of the cluster has written its slice: one more item of leaf jj is complete
  if (signal_done && rank == 0 && threadIdx.x == 0) atomicAdd(&const_cast<Plan*>(plan)->done[jj], 1);
}

// Cluster geometry shared by the single-problem and batched kernels: rank, cluster index,
// and the peers' shared histograms.
struct HistCta {
  int cs, rank, cid, ncl;
  const float* peer[16];
  uint32_t sbase;
  __device__ explicit HistCta(float* hsh) {
    namespace cgr = cooperative_groups;
    cgr::cluster_group cl = cgr::this_cluster();
    cs = static_cast<int>(cl.num_blocks());
    rank = static_cast<int>(cl.block_rank());
    cid = blockIdx.x / cs;
    ncl = gridDim.x / cs;
    for (int r = 0; r < cs && r < 16; ++r) peer[r] = cl.map_shared_rank(hsh, r);
    sbase = static_cast<uint32_t>(__cvta_generic_to_shared(hsh));
  }
};

template <typename GH, int NB, int MODE>
__global__ void __launch_bounds__(512, 3) level_hist_kernel(const uint8_t* __restrict__ bins, int64_t n, int G, int F,
                                                         const uint32_t* __restrict__ order,
                                                         const GH* __restrict__ g, const GH* __restrict__ h,
                                                         const Plan* __restrict__ plan, int max_bins,
                                                         float* __restrict__ partials) {
  extern __shared__ __align__(16) float hsh[];   // [2][NB][32]
  __shared__ int s_next;
  HistCta k(hsh);
  const HistProblem P{bins, n, G, F, order, g, h, plan, max_bins, partials};
  const int total_items = plan->total_units * G;
  cooperative_groups::this_cluster().sync();
  if (k.rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, k.cs);
  cooperative_groups::this_cluster().sync();
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next))
    hist_item<GH, NB, MODE>(P, item, k.cs, k.rank, hsh, k.peer, k.sbase, &s_next);
}

// Warp-private histogram, no atomics (the paper's Section 5 scheme: per-warp partial
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
  __shared__ int s_next;   // this cluster's next work item (rank 0's slot)
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
  cl.sync();
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next)) {
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
    if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
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

// ------------------------------------------- lane-per-feature warp histograms
// The warp-private scheme of the paper's Section 5 with one feature per lane: a warp owns
// the (G, H) float2 histogram [max_bins][32] of one 32-feature group, and lane f updates
// column f for every row, so the 32 addresses of an update are always distinct and no
// atomics are needed. Rows come in blocks of 32 staged in shared memory: lane i fetches
// the row id and the position-ordered (g, h) of row i four blocks ahead and copies the
// row's 32-byte bin record with cp.async two blocks ahead. Within a block the rows are
// updated in batches of LH_BATCH: the histogram loads of a batch are issued before its
// stores, and rows of the batch that share a cell are summed before they are added to it,
// so one shared-memory round trip serves a whole batch (lane_batched_updates). A 255-bin warp histogram is 64 KB, so an SM holds 3 such
// warps; the batches give each warp the instruction-level parallelism it needs.
// At the end of a work unit the warps of a CTA are summed into warp 0's histogram, and
// CTA r of the cluster sums its slice of bins over the cluster (distributed shared
// memory) into the unit's FP32 partial.
constexpr int LH_ROWS = 32;       // rows per block: one per lane for row ids and (g, h)
constexpr int LH_STAGES = 3;      // bin-record buffers per warp: blocks j, j + 1, j + 2
constexpr int LH_AHEAD = 4;       // blocks of lookahead for row ids and (g, h)
constexpr int LH_MAX_WARPS = 16;
constexpr int LH_BATCH = 4;       // rows whose histogram loads are issued before their stores

// Histogram accesses of the lane kernel. Volatile keeps them in program order among
// themselves (a load issued ahead of a store to the same cell must stay ahead of it, the
// batched updates rely on that); without a memory clobber the staging-buffer loads around
// them remain free to be scheduled early.
__device__ __forceinline__ float2 lds_f2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_f2(uint32_t addr, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y));
}

// Histogram updates of N consecutive staged rows of one lane, for C update chains whose
// cells are disjoint (chain c: cell addresses a[c][i]; rows row0 + i take their (g, h)
// from the staged pairs gh4, two rows per float4; row0 is even). A warp's shared load
// waits for that warp's own earlier shared stores, so an update loop that loads a row's
// cell after the previous row's store pays one full shared-memory round trip per row.
// Here the loads of LH_BATCH rows (of every chain) are issued before any of their stores.
// Rows of a batch that share a cell loaded the same value, so each row adds to its loaded
// value the sum of its own (g, h) and those of the earlier rows of the batch in that cell,
// and the last of them stores the cell's new value (the stores go in row order). The sums
// depend only on the addresses and the staged pairs, not on the loads, which keeps the
// dependent chain behind each load to one addition.
template <int N, int C>
__device__ __forceinline__ void lane_batched_updates(const uint32_t (&a)[C][N], const float4* __restrict__ gh4, int row0,
                                                     const bool (&act)[C]) {
  static_assert(N % LH_BATCH == 0, "rows must fill whole batches");
#pragma unroll
  for (int i0 = 0; i0 < N; i0 += LH_BATCH) {
    float2 v[C][LH_BATCH];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int j = 0; j < LH_BATCH; ++j) v[c][j] = act[c] ? lds_f2(a[c][i0 + j]) : make_float2(0.f, 0.f);
    float gx[LH_BATCH], hy[LH_BATCH];
#pragma unroll
    for (int j = 0; j < LH_BATCH; ++j) {
      const float4 gq = gh4[(row0 + i0 + j) >> 1];
      gx[j] = ((i0 + j) & 1) ? gq.z : gq.x;
      hy[j] = ((i0 + j) & 1) ? gq.w : gq.y;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int j = 0; j < LH_BATCH; ++j) {
        float sx = gx[j], sy = hy[j];
#pragma unroll
        for (int q = 0; q < j; ++q)
          if (a[c][i0 + q] == a[c][i0 + j]) {
            sx += gx[q];
            sy += hy[q];
          }
        v[c][j].x += sx;
        v[c][j].y += sy;
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int j = 0; j < LH_BATCH; ++j)
        if (act[c]) sts_f2(a[c][i0 + j], v[c][j]);
  }
}

inline size_t lh_warp_bytes(int max_bins) {
  return static_cast<size_t>(max_bins) * GROUP * sizeof(float2) + static_cast<size_t>(LH_STAGES) * LH_ROWS * GROUP +
         LH_ROWS * sizeof(float2);
}
inline int lh_warps(int max_bins, int requested_threads) {
  int w = static_cast<int>(SMEM_DYN_BUDGET / lh_warp_bytes(max_bins));
  if (w > LH_MAX_WARPS) w = LH_MAX_WARPS;
  if (requested_threads > 0 && requested_threads / 32 < w) w = requested_threads / 32;
  return w < 1 ? 1 : w;
}
inline size_t lh_smem_bytes(int max_bins, int warps) { return static_cast<size_t>(warps) * lh_warp_bytes(max_bins); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename GH>
__global__ void __launch_bounds__(LH_MAX_WARPS * 32, 1)
    level_hist_lane_kernel(const uint8_t* __restrict__ bins, int64_t n, int G, int F, const uint32_t* __restrict__ order,
                           const GH* __restrict__ gpos, const GH* __restrict__ hpos, const Plan* __restrict__ plan,
                           int max_bins, float* __restrict__ partials) {
  namespace cgr = cooperative_groups;
  extern __shared__ __align__(16) unsigned char lsh[];
  constexpr int MAX_CS = 16;
  constexpr uint32_t NONE = 0xffffffffu;
  cgr::cluster_group cl = cgr::this_cluster();
  const int cs = static_cast<int>(cl.num_blocks());
  const int rank = static_cast<int>(cl.block_rank());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int per_warp = max_bins * GROUP;   // float2 cells of one warp histogram
  float2* hist_all = reinterpret_cast<float2*>(lsh);
  float2* my = hist_all + static_cast<int64_t>(warp) * per_warp;
  unsigned char* stages = lsh + static_cast<size_t>(W) * per_warp * sizeof(float2);
  unsigned char* my_stage = stages + static_cast<size_t>(warp) * LH_STAGES * LH_ROWS * GROUP;
  float2* my_gh = reinterpret_cast<float2*>(stages + static_cast<size_t>(W) * LH_STAGES * LH_ROWS * GROUP) +
                  warp * LH_ROWS;
  const uint32_t stage_s = static_cast<uint32_t>(__cvta_generic_to_shared(my_stage));
  const uint32_t hbase = static_cast<uint32_t>(__cvta_generic_to_shared(my + lane));
  const int maxb1 = max_bins - 1;
  const float2* peer0[MAX_CS];
  for (int r = 0; r < cs && r < MAX_CS; ++r) peer0[r] = cl.map_shared_rank(hist_all, r);
  const int total_items = plan->total_units * G;
  const int n_small = plan->n_small;
  __shared__ int s_next;   // this cluster's next work item (rank 0's slot)
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
  cl.sync();
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next)) {
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
    {
      float4* z = reinterpret_cast<float4*>(my);
      for (int i = lane; i < per_warp / 2; i += 32) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    const int nblk = p1 > p0 ? (p1 - p0 + LH_ROWS - 1) / LH_ROWS : 0;
    const int my_blocks = nblk > warp ? (nblk - warp + W - 1) / W : 0;
    const bool act = lane < F - grp * GROUP;   // lanes of padding features do no updates
    const uint8_t* gb = bins + static_cast<int64_t>(grp) * n * GROUP;
    if (my_blocks > 0) {
      uint32_t rid[LH_AHEAD + 1];
      float gr[LH_AHEAD + 1], hr[LH_AHEAD + 1];
      auto fetch = [&](int j, uint32_t& row, float& gv, float& hv) {
        const int pos = p0 + (warp + j * W) * LH_ROWS + lane;
        if (j < my_blocks && pos < p1) {
          row = order ? __ldg(order + pos) : static_cast<uint32_t>(pos);
          gv = cbgd::load_gh(gpos, pos);
          hv = cbgd::load_gh(hpos, pos);
        } else {
          row = NONE;   // a row past the end: zero record, zero (g, h)
          gv = 0.f;
          hv = 0.f;
        }
      };
      auto copy_bins = [&](int j, uint32_t row) {
        const uint32_t dst = stage_s + static_cast<uint32_t>(((j % LH_STAGES) * LH_ROWS + lane) * GROUP);
        if (row != NONE) {
          const uint8_t* src = gb + static_cast<int64_t>(row) * GROUP;
          cp_async16(dst, src);
          cp_async16(dst + 16, src + 16);
        } else {
          asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n\tst.shared.v4.u32 [%2], {%1, %1, %1, %1};" ::"r"(dst),
                       "r"(0u), "r"(dst + 16u)
                       : "memory");
        }
      };
#pragma unroll
      for (int q = 0; q < LH_AHEAD; ++q) fetch(q, rid[q], gr[q], hr[q]);
      copy_bins(0, rid[0]);
      cp_async_commit();
      if (1 < my_blocks) copy_bins(1, rid[1]);
      cp_async_commit();
      for (int j = 0; j < my_blocks; ++j) {
        fetch(j + LH_AHEAD, rid[LH_AHEAD], gr[LH_AHEAD], hr[LH_AHEAD]);
        if (j + 2 < my_blocks) copy_bins(j + 2, rid[2]);
        cp_async_commit();
        my_gh[lane] = make_float2(gr[0], hr[0]);
        cp_async_wait<2>();
        __syncwarp();
        if (act) {
          const unsigned char* sb = my_stage + (j % LH_STAGES) * LH_ROWS * GROUP + lane;
          const float4* gh4 = reinterpret_cast<const float4*>(my_gh);
          // shared-memory offsets (bytes) of the 32 rows' cells, loaded up front so that
          // only the histogram loads remain on the chain
          uint32_t a[1][LH_ROWS];
#pragma unroll
          for (int i = 0; i < LH_ROWS; ++i)
            a[0][i] = hbase + static_cast<uint32_t>(min(static_cast<int>(sb[i * GROUP]), maxb1)) * (GROUP * 8u);
          const bool on[1] = {true};
          lane_batched_updates<LH_ROWS, 1>(a, gh4, 0, on);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < LH_AHEAD; ++q) {
          rid[q] = rid[q + 1];
          gr[q] = gr[q + 1];
          hr[q] = hr[q + 1];
        }
      }
      cp_async_wait<0>();
    }
    __syncthreads();
    // the CTA's warps, summed in warp order into warp 0's histogram
    if (W > 1) {
      for (int e = threadIdx.x; e < per_warp; e += blockDim.x) {
        float2 s = hist_all[e];
        for (int w = 1; w < W; ++w) {
          const float2 v = hist_all[static_cast<int64_t>(w) * per_warp + e];
          s.x += v.x;
          s.y += v.y;
        }
        hist_all[e] = s;
      }
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
    // this CTA's slice of bins, summed over the cluster's CTAs in rank order
    const int bs = (max_bins + cs - 1) / cs;
    const int b0 = rank * bs;
    const int nbs = max(0, min(max_bins, b0 + bs) - b0);
    float* dst = partials + static_cast<int64_t>(item) * (2 * max_bins * GROUP);
    for (int i = threadIdx.x; i < nbs * GROUP; i += blockDim.x) {
      const int e = b0 * GROUP + i;
      float sx = 0.f, sy = 0.f;
      for (int r = 0; r < cs; ++r) {
        const float2 v = peer0[r][e];
        sx += v.x;
        sy += v.y;
      }
      dst[e] = sx;
      dst[max_bins * GROUP + e] = sy;
    }
    cl.sync();
  }
}

// ------------------------- lane-per-feature with loader warps (warp specialised)
// The lane kernel's warps stage their own rows: with one warp per scheduler, the time a
// warp spends fetching row ids, copying bin records and waiting for them adds to the time
// of its histogram updates instead of overlapping it. Here a CTA has W compute warps, each
// with its private [max_bins][32] (G, H) table updated as in the lane kernel, and W loader
// warps: warp W + w stages every block of 32 rows of compute warp w. Block b of a work item
// goes to compute warp b % W, and every work item is padded to a multiple of W blocks. A
// loader fetches row ids and position-ordered (g, h) into registers a batch of LD_AHEAD
// blocks ahead and writes a block into one of its warp's LD_STAGES buffers: the rows'
// 32-byte bin records with cp.async, the (g, h) pairs with plain stores. Two mbarriers per
// buffer hand it over: `full` (32 arrivals, one per loader lane, each also waiting for
// that lane's copies) and `empty` (one arrival by the compute warp once it has read the
// buffer). One loader for all compute warps (its chain of shared-memory round trips
// queues behind the compute warps' histogram traffic) fell behind them.
// Every wait polls a bounded number of times: a wait that runs out records STATUS_TIMEOUT
// in `status` and raises the CTA's abort flag, after which the CTA's waits all give up at
// once and skip their work, so every warp still reaches the barriers of the work item and
// the launch ends. For a test of that path, test_stall != 0 makes the loaders skip their
// arrivals on `full` (the compute warps then wait for a phase that never completes) and
// wait_limit sets the polls of a wait.
constexpr int LD_STAGES = 4;                  // buffers per compute warp
constexpr int LD_AHEAD = 8;                   // blocks per batch of row-id and (g, h) loads of the loader
constexpr unsigned LD_WAIT_LIMIT = 1u << 24;  // polls of one mbarrier wait (about a second at most)

inline size_t ld_warp_bytes(int max_bins) {
  return static_cast<size_t>(max_bins) * GROUP * sizeof(float2) +
         static_cast<size_t>(LD_STAGES) * (LH_ROWS * GROUP + LH_ROWS * sizeof(float2) + 2 * sizeof(uint64_t));
}
inline int ld_warps(int max_bins, int requested_threads) {   // compute warps (as many loaders come on top)
  int w = static_cast<int>(SMEM_DYN_BUDGET / ld_warp_bytes(max_bins));
  if (w > LH_MAX_WARPS / 2) w = LH_MAX_WARPS / 2;
  if (requested_threads > 0 && requested_threads / 64 < w) w = requested_threads / 64;
  return w < 1 ? 1 : w;
}
inline size_t ld_smem_bytes(int max_bins, int warps) { return static_cast<size_t>(warps) * ld_warp_bytes(max_bins); }

// Waits until the mbarrier at shared address `bar` has completed the phase of the given
// parity. Every lane of the warp calls it; false (for the whole warp) if the CTA aborts or
// the wait runs out (which starts the abort).
__device__ __forceinline__ bool ld_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, unsigned* status,
                                        unsigned limit) {
  bool ok = false;
  for (unsigned polls = 0;; ++polls) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) {
      ok = true;
      break;
    }
    if (*abort_flag) break;
    if (polls >= limit) {
      atomicOr(status, ::cbg::STATUS_TIMEOUT);
      *abort_flag = 1;
      break;
    }
  }
  return __all_sync(0xffffffffu, ok) != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// One arrival on `bar` once every cp.async this thread has issued so far has completed.
__device__ __forceinline__ void mbar_arrive_after_copies(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
// Whether the mbarrier at `bar` has completed the phase of the given parity (one poll).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

template <typename GH>
__global__ void __launch_bounds__(LH_MAX_WARPS * 32, 1)
    level_hist_lane_ld_kernel(const uint8_t* __restrict__ bins, int64_t n, int G, int F,
                              const uint32_t* __restrict__ order, const GH* __restrict__ gpos,
                              const GH* __restrict__ hpos, const Plan* __restrict__ plan, int max_bins,
                              float* __restrict__ partials, unsigned* __restrict__ status, int test_stall,
                              unsigned wait_limit) {
  namespace cgr = cooperative_groups;
  extern __shared__ __align__(16) unsigned char lsh[];
  constexpr int MAX_CS = 16;
  constexpr uint32_t NONE = 0xffffffffu;
  constexpr uint32_t FULL_MASK = 0xffffffffu;
  cgr::cluster_group cl = cgr::this_cluster();
  const int cs = static_cast<int>(cl.num_blocks());
  const int rank = static_cast<int>(cl.block_rank());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = (blockDim.x >> 5) / 2;   // compute warps 0..W-1; warp W + w loads for warp w
  const int per_warp = max_bins * GROUP;
  float2* hist_all = reinterpret_cast<float2*>(lsh);
  unsigned char* recs = lsh + static_cast<size_t>(W) * per_warp * sizeof(float2);
  float2* ghs = reinterpret_cast<float2*>(recs + static_cast<size_t>(W) * LD_STAGES * LH_ROWS * GROUP);
  const uint32_t recs_s = static_cast<uint32_t>(__cvta_generic_to_shared(recs));
  const uint32_t full_s = static_cast<uint32_t>(__cvta_generic_to_shared(ghs + W * LD_STAGES * LH_ROWS));
  const uint32_t empty_s = full_s + static_cast<uint32_t>(W * LD_STAGES * sizeof(uint64_t));
  const int maxb1 = max_bins - 1;
  const float2* peer0[MAX_CS];
  for (int r = 0; r < cs && r < MAX_CS; ++r) peer0[r] = cl.map_shared_rank(hist_all, r);
  const int total_items = plan->total_units * G;
  const int n_small = plan->n_small;
  __shared__ int s_next;    // this cluster's next work item
  __shared__ int s_abort;   // a wait of this CTA ran out
  if (threadIdx.x < 2 * W * LD_STAGES) {
    const uint32_t bar = full_s + threadIdx.x * static_cast<uint32_t>(sizeof(uint64_t));
    // full: one arrival per loader lane, each once that lane's copies have landed;
    // empty: one by the compute warp
    const uint32_t count = threadIdx.x < W * LD_STAGES ? 32u : 1u;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n\tfence.mbarrier_init.release.cluster;" ::"r"(bar),
                 "r"(count)
                 : "memory");
  }
  if (threadIdx.x == 0) s_abort = 0;
  // Blocks each compute warp has taken so far in this launch: every work item is padded
  // to a multiple of W blocks (the padding blocks have no rows), so the count is the same
  // for every warp.
  uint32_t U = 0;
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
  cl.sync();
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next)) {
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
    const int nblk = p1 > p0 ? (p1 - p0 + LH_ROWS - 1) / LH_ROWS : 0;
    const int rounds = (nblk + W - 1) / W;   // blocks per warp; block b = j W + w is warp w's j-th
    if (warp < W) {   // ---- compute warp
      float2* my = hist_all + static_cast<int64_t>(warp) * per_warp;
      const uint32_t hbase = static_cast<uint32_t>(__cvta_generic_to_shared(my + lane));
      {
        float4* z = reinterpret_cast<float4*>(my);
        for (int i = lane; i < per_warp / 2; i += 32) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncwarp();
      const bool act = lane < F - grp * GROUP;   // lanes of padding features do no updates
      for (int j = 0; j < rounds; ++j) {
        const uint32_t k = U + static_cast<uint32_t>(j);
        const int slot = warp * LD_STAGES + static_cast<int>(k % LD_STAGES);
        const bool ok = ld_wait(full_s + slot * 8u, (k / LD_STAGES) & 1u, &s_abort, status, wait_limit);
        if (ok && act && j * W + warp < nblk) {
          const unsigned char* sb = recs + slot * (LH_ROWS * GROUP) + lane;
          const float4* gh4 = reinterpret_cast<const float4*>(ghs + slot * LH_ROWS);
          uint32_t a[1][LH_ROWS];
#pragma unroll
          for (int i = 0; i < LH_ROWS; ++i)
            a[0][i] = hbase + static_cast<uint32_t>(min(static_cast<int>(sb[i * GROUP]), maxb1)) * (GROUP * 8u);
          const bool on[1] = {true};
          lane_batched_updates<LH_ROWS, 1>(a, gh4, 0, on);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty_s + slot * 8u);
      }
    } else {   // ---- loader warp W + w, for compute warp w
      const int w = warp - W;
      const uint8_t* gb = bins + static_cast<int64_t>(grp) * n * GROUP;
      // row ids and (g, h) of the next LD_AHEAD blocks load while the current LD_AHEAD
      // blocks are handed out; the registers are moved only once per batch, after the
      // loads have had a whole batch of hand-overs to arrive
      // (g, h) stay raw bits until the hand-over converts them
      uint32_t rc[LD_AHEAD], rn[LD_AHEAD];
      uint32_t gc[LD_AHEAD], hc[LD_AHEAD], gn[LD_AHEAD], hn[LD_AHEAD];
      auto fetch = [&](int j, uint32_t& row, uint32_t& gv, uint32_t& hv) {   // warp w's j-th block
        const int b = j * W + w;
        const int pos = p0 + b * LH_ROWS + lane;
        if (b < nblk && pos < p1) {
          row = order ? __ldg(order + pos) : static_cast<uint32_t>(pos);
          gv = cbgd::load_gh_bits(gpos, pos);
          hv = cbgd::load_gh_bits(hpos, pos);
        } else {
          row = NONE;   // a row past the end: (g, h) = 0, and its record is not copied
          gv = 0u;
          hv = 0u;
        }
      };
#pragma unroll
      for (int q = 0; q < LD_AHEAD; ++q) fetch(q, rc[q], gc[q], hc[q]);
      for (int j0 = 0; j0 < rounds; j0 += LD_AHEAD) {
#pragma unroll
        for (int q = 0; q < LD_AHEAD; ++q) fetch(j0 + LD_AHEAD + q, rn[q], gn[q], hn[q]);
        // one poll of the `empty` barrier of each of the batch's first LD_STAGES blocks, a
        // lane each (a later block's buffer is last filled within this batch, and its poll
        // could see the phase before last, which has the same parity: it is left to the
        // wait below)
        bool free_l = false;
        if (lane < LD_AHEAD && lane < LD_STAGES && j0 + lane < rounds) {
          const uint32_t k = U + static_cast<uint32_t>(j0 + lane);
          free_l = mbar_test(empty_s + (w * LD_STAGES + static_cast<int>(k % LD_STAGES)) * 8u,
                             ((k / LD_STAGES) & 1u) ^ 1u);
        }
        const uint32_t free_mask = __ballot_sync(FULL_MASK, free_l);
#pragma unroll
        for (int q = 0; q < LD_AHEAD; ++q) {
          if (j0 + q < rounds) {
            const uint32_t k = U + static_cast<uint32_t>(j0 + q);
            const int slot = w * LD_STAGES + static_cast<int>(k % LD_STAGES);
            // a fresh mbarrier counts as having completed the phase before its first, so
            // the first LD_STAGES blocks find their buffers free
            const bool ok = ((free_mask >> q) & 1u) ||
                            ld_wait(empty_s + slot * 8u, ((k / LD_STAGES) & 1u) ^ 1u, &s_abort, status, wait_limit);
            if (ok) {
              // rows past the end keep whatever record the buffer held: with (g, h) = 0
              // their clamped bins add zero to some cell
              if (rc[q] != NONE) {
                const uint32_t dst = recs_s + static_cast<uint32_t>((slot * LH_ROWS + lane) * GROUP);
                const uint8_t* src = gb + static_cast<int64_t>(rc[q]) * GROUP;
                cp_async16(dst, src);
                cp_async16(dst + 16, src + 16);
              }
              ghs[slot * LH_ROWS + lane] = make_float2(cbgd::gh_from_bits<GH>(gc[q]), cbgd::gh_from_bits<GH>(hc[q]));
              if (!test_stall) {
                mbar_arrive_after_copies(full_s + slot * 8u);
                mbar_arrive(full_s + slot * 8u);
              }
            }
          }
        }
#pragma unroll
        for (int q = 0; q < LD_AHEAD; ++q) {
          rc[q] = rn[q];
          gc[q] = gn[q];
          hc[q] = hn[q];
        }
      }
      cp_async_wait<0>();
    }
    U += static_cast<uint32_t>(rounds);
    __syncthreads();
    // the CTA's warps, summed in warp order into warp 0's histogram
    if (W > 1) {
      for (int e = threadIdx.x; e < per_warp; e += blockDim.x) {
        float2 s = hist_all[e];
        for (int v = 1; v < W; ++v) {
          const float2 x = hist_all[static_cast<int64_t>(v) * per_warp + e];
          s.x += x.x;
          s.y += x.y;
        }
        hist_all[e] = s;
      }
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
    // this CTA's slice of bins, summed over the cluster's CTAs in rank order
    const int bs = (max_bins + cs - 1) / cs;
    const int b0 = rank * bs;
    const int nbs = max(0, min(max_bins, b0 + bs) - b0);
    float* dst = partials + static_cast<int64_t>(item) * (2 * max_bins * GROUP);
    for (int i = threadIdx.x; i < nbs * GROUP; i += blockDim.x) {
      const int e = b0 * GROUP + i;
      float sx = 0.f, sy = 0.f;
      for (int r = 0; r < cs; ++r) {
        const float2 v = peer0[r][e];
        sx += v.x;
        sy += v.y;
      }
      dst[e] = sx;
      dst[max_bins * GROUP + e] = sy;
    }
    cl.sync();
  }
}

// ------------------------------------ lane-per-feature over 4-bit packed bins
// The packed layout of Section 5 for features with at most 16 bins: byte i of a row's
// 32-byte record in packed group q holds feature 64q + i in its low nibble and feature
// 64q + 32 + i in its high nibble (bins4 [ceil(G/2)][n][32], 64 features per record, half
// the bytes of the uint8 layout). The kernel is the lane kernel above with two update
// chains per lane: lane i owns column i of both 32-feature halves, in a warp histogram
// [max_bins][2][32] float2 whose halves are exactly the histograms of uint8 groups 2q and
// 2q + 1, so the partials and the reduction are unchanged. A 32-row block is worked in
// two halves of 16 rows to bound the registers of the precomputed cell addresses.
constexpr int L4_SUB = 16;

inline size_t l4_warp_bytes(int max_bins) {
  return static_cast<size_t>(max_bins) * 2 * GROUP * sizeof(float2) + static_cast<size_t>(LH_STAGES) * LH_ROWS * GROUP +
         LH_ROWS * sizeof(float2);
}
inline int l4_warps(int max_bins, int requested_threads) {
  int w = static_cast<int>(SMEM_DYN_BUDGET / l4_warp_bytes(max_bins));
  if (w > LH_MAX_WARPS) w = LH_MAX_WARPS;
  if (requested_threads > 0 && requested_threads / 32 < w) w = requested_threads / 32;
  return w < 1 ? 1 : w;
}
inline size_t l4_smem_bytes(int max_bins, int warps) { return static_cast<size_t>(warps) * l4_warp_bytes(max_bins); }

template <typename GH>
__global__ void __launch_bounds__(LH_MAX_WARPS * 32, 1)
    level_hist_lane4_kernel(const uint8_t* __restrict__ bins4, int64_t n, int G, int F,
                            const uint32_t* __restrict__ order, const GH* __restrict__ gpos,
                            const GH* __restrict__ hpos, const Plan* __restrict__ plan, int max_bins,
                            float* __restrict__ partials) {
  namespace cgr = cooperative_groups;
  extern __shared__ __align__(16) unsigned char l4sh[];
  constexpr int MAX_CS = 16;
  constexpr uint32_t NONE = 0xffffffffu;
  cgr::cluster_group cl = cgr::this_cluster();
  const int cs = static_cast<int>(cl.num_blocks());
  const int rank = static_cast<int>(cl.block_rank());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int G4 = (G + 1) / 2;
  const int per_warp = max_bins * 2 * GROUP;   // float2 cells of one warp histogram
  float2* hist_all = reinterpret_cast<float2*>(l4sh);
  float2* my = hist_all + static_cast<int64_t>(warp) * per_warp;
  unsigned char* stages = l4sh + static_cast<size_t>(W) * per_warp * sizeof(float2);
  unsigned char* my_stage = stages + static_cast<size_t>(warp) * LH_STAGES * LH_ROWS * GROUP;
  float2* my_gh = reinterpret_cast<float2*>(stages + static_cast<size_t>(W) * LH_STAGES * LH_ROWS * GROUP) +
                  warp * LH_ROWS;
  const uint32_t stage_s = static_cast<uint32_t>(__cvta_generic_to_shared(my_stage));
  const uint32_t hbase_lo = static_cast<uint32_t>(__cvta_generic_to_shared(my + lane));
  const uint32_t hbase_hi = hbase_lo + GROUP * 8u;
  const uint32_t bin_stride = 2u * GROUP * 8u;   // bytes between bins of one column
  const int maxb1 = max_bins - 1;
  const float2* peer0[MAX_CS];
  for (int r = 0; r < cs && r < MAX_CS; ++r) peer0[r] = cl.map_shared_rank(hist_all, r);
  const int total_items = plan->total_units * G4;
  const int n_small = plan->n_small;
  __shared__ int s_next;   // this cluster's next work item (rank 0's slot)
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
  cl.sync();
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next)) {
    const int unit = item / G4, q4 = item - unit * G4;
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
    {
      float4* z = reinterpret_cast<float4*>(my);
      for (int i = lane; i < per_warp / 2; i += 32) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    const int nblk = p1 > p0 ? (p1 - p0 + LH_ROWS - 1) / LH_ROWS : 0;
    const int my_blocks = nblk > warp ? (nblk - warp + W - 1) / W : 0;
    const bool act_lo = lane < F - q4 * 2 * GROUP;            // lanes of padding features do no updates
    const bool act_hi = lane < F - q4 * 2 * GROUP - GROUP;
    const uint8_t* gb = bins4 + static_cast<int64_t>(q4) * n * GROUP;
    if (my_blocks > 0) {
      uint32_t rid[LH_AHEAD + 1];
      float gr[LH_AHEAD + 1], hr[LH_AHEAD + 1];
      auto fetch = [&](int j, uint32_t& row, float& gv, float& hv) {
        const int pos = p0 + (warp + j * W) * LH_ROWS + lane;
        if (j < my_blocks && pos < p1) {
          row = order ? __ldg(order + pos) : static_cast<uint32_t>(pos);
          gv = cbgd::load_gh(gpos, pos);
          hv = cbgd::load_gh(hpos, pos);
        } else {
          row = NONE;   // a row past the end: zero record, zero (g, h)
          gv = 0.f;
          hv = 0.f;
        }
      };
      auto copy_bins = [&](int j, uint32_t row) {
        const uint32_t dst = stage_s + static_cast<uint32_t>(((j % LH_STAGES) * LH_ROWS + lane) * GROUP);
        if (row != NONE) {
          const uint8_t* src = gb + static_cast<int64_t>(row) * GROUP;
          cp_async16(dst, src);
          cp_async16(dst + 16, src + 16);
        } else {
          asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n\tst.shared.v4.u32 [%2], {%1, %1, %1, %1};" ::"r"(dst),
                       "r"(0u), "r"(dst + 16u)
                       : "memory");
        }
      };
#pragma unroll
      for (int q = 0; q < LH_AHEAD; ++q) fetch(q, rid[q], gr[q], hr[q]);
      copy_bins(0, rid[0]);
      cp_async_commit();
      if (1 < my_blocks) copy_bins(1, rid[1]);
      cp_async_commit();
      for (int j = 0; j < my_blocks; ++j) {
        fetch(j + LH_AHEAD, rid[LH_AHEAD], gr[LH_AHEAD], hr[LH_AHEAD]);
        if (j + 2 < my_blocks) copy_bins(j + 2, rid[2]);
        cp_async_commit();
        my_gh[lane] = make_float2(gr[0], hr[0]);
        cp_async_wait<2>();
        __syncwarp();
        const unsigned char* sb = my_stage + (j % LH_STAGES) * LH_ROWS * GROUP + lane;
        const float4* gh4 = reinterpret_cast<const float4*>(my_gh);
#pragma unroll
        for (int s0 = 0; s0 < LH_ROWS; s0 += L4_SUB) {
          uint32_t a[2][L4_SUB];
#pragma unroll
          for (int i = 0; i < L4_SUB; ++i) {
            const unsigned byte = sb[(s0 + i) * GROUP];
            a[0][i] = hbase_lo + static_cast<uint32_t>(min(static_cast<int>(byte & 15u), maxb1)) * bin_stride;
            a[1][i] = hbase_hi + static_cast<uint32_t>(min(static_cast<int>(byte >> 4), maxb1)) * bin_stride;
          }
          // the two nibbles' chains (disjoint halves of the warp histogram) in one batch
          const bool on[2] = {act_lo, act_hi};
          lane_batched_updates<L4_SUB, 2>(a, gh4, s0, on);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < LH_AHEAD; ++q) {
          rid[q] = rid[q + 1];
          gr[q] = gr[q + 1];
          hr[q] = hr[q + 1];
        }
      }
      cp_async_wait<0>();
    }
    __syncthreads();
    // the CTA's warps, summed in warp order into warp 0's histogram
    if (W > 1) {
      for (int e = threadIdx.x; e < per_warp; e += blockDim.x) {
        float2 s = hist_all[e];
        for (int w = 1; w < W; ++w) {
          const float2 v = hist_all[static_cast<int64_t>(w) * per_warp + e];
          s.x += v.x;
          s.y += v.y;
        }
        hist_all[e] = s;
      }
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
    // this CTA's slice of bins, summed over the cluster's CTAs in rank order, written as
    // the partials of uint8 groups 2 q4 and 2 q4 + 1
    const int bs = (max_bins + cs - 1) / cs;
    const int b0 = rank * bs;
    const int nbs = max(0, min(max_bins, b0 + bs) - b0);
    for (int i = threadIdx.x; i < nbs * 2 * GROUP; i += blockDim.x) {
      const int b = b0 + i / (2 * GROUP), half = (i / GROUP) & 1, col = i & (GROUP - 1);
      const int grp = 2 * q4 + half;
      if (grp >= G) continue;
      const int e = (b * 2 + half) * GROUP + col;
      float sx = 0.f, sy = 0.f;
      for (int r = 0; r < cs; ++r) {
        const float2 v = peer0[r][e];
        sx += v.x;
        sy += v.y;
      }
      float* dst = partials + (static_cast<int64_t>(unit) * G + grp) * (2 * max_bins * GROUP);
      dst[b * GROUP + col] = sx;
      dst[max_bins * GROUP + b * GROUP + col] = sy;
    }
    cl.sync();
  }
}

// bins4[q][r][i] = bins[2q][r][i] | bins[2q+1][r][i] << 4 (the second group read as 0 past
// the last one); every bin must be below 16.
__global__ void pack_bins4_kernel(const uint8_t* __restrict__ bins, int64_t n, int G, uint8_t* __restrict__ bins4,
                                  unsigned int* __restrict__ status) {
  const int G4 = (G + 1) / 2;
  const int64_t total = static_cast<int64_t>(G4) * n * 2;   // 16-byte halves of the packed records
  bool bad = false;
  for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
       x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t rec = x >> 1, q = rec / n, r = rec - q * n;
    const int half = static_cast<int>(x & 1);
    const uint4 lo = reinterpret_cast<const uint4*>(bins)[((2 * q) * n + r) * 2 + half];
    uint4 hi = make_uint4(0u, 0u, 0u, 0u);
    if (2 * q + 1 < G) hi = reinterpret_cast<const uint4*>(bins)[((2 * q + 1) * n + r) * 2 + half];
    bad |= ((lo.x | lo.y | lo.z | lo.w | hi.x | hi.y | hi.z | hi.w) & 0xf0f0f0f0u) != 0u;
    // bytes of lo stay in the low nibbles, bytes of hi move to the high nibbles
    reinterpret_cast<uint4*>(bins4)[x] = make_uint4(lo.x | (hi.x << 4), lo.y | (hi.y << 4), lo.z | (hi.z << 4),
                                                    lo.w | (hi.w << 4));
  }
  if (bad) atomicOr(status, ::cbg::STATUS_BAD_BIN);
}

// ------------------------------------------------------ 1-bit binary features
// Section 5 ("Dense numerical features") packs binary features 32 to a 32-bit integer
// and builds their histograms 32 features and 2 statistics at a time. Here bits1[q][r]
// (uint32) holds bit i = [bin of feature 32q + i of row r is 1] (cbg_pack_bits1). A
// feature of at most 2 bins has only two cells per leaf, so lane f of a warp keeps both
// of feature f's (G, H) cells of the work item in registers: for every row of a staged
// block of 32 it tests its bit of the row's word and adds the row's (g, h) to bin 1 or
// bin 0. No shared-memory histogram and no atomics; the warps of a CTA, then the CTAs of
// the cluster, are summed in order at the end of the item into the same [stat][bin][32]
// FP32 partial as the other kernels (max_bins = 2), for the FP64 reduction.
constexpr int LB_WARPS = 16;

__global__ void pack_bits1_kernel(const uint8_t* __restrict__ bins, int64_t n, int G, uint32_t* __restrict__ bits1,
                                  unsigned int* __restrict__ status) {
  const int64_t total = static_cast<int64_t>(G) * n;
  bool bad = false;
  for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < total;
       x += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint4* rec = reinterpret_cast<const uint4*>(bins) + 2 * x;   // group q, row r: record x = q n + r
    const uint4 a = rec[0], b = rec[1];
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t word = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      bad |= (w[k] & 0xfefefefeu) != 0u;
      // bytes 0..3 of w[k] (each 0 or 1) are features 4k .. 4k + 3
      const uint32_t nib = (w[k] & 1u) | ((w[k] >> 7) & 2u) | ((w[k] >> 14) & 4u) | ((w[k] >> 21) & 8u);
      word |= nib << (4 * k);
    }
    bits1[x] = word;
  }
  if (bad) atomicOr(status, ::cbg::STATUS_BAD_BIN);
}

template <typename GH>
__global__ void __launch_bounds__(LB_WARPS * 32, 2)
    level_hist_bits_kernel(const uint32_t* __restrict__ bits1, int64_t n, int G, int F,
                           const uint32_t* __restrict__ order, const GH* __restrict__ gpos,
                           const GH* __restrict__ hpos, const Plan* __restrict__ plan, float* __restrict__ partials) {
  namespace cgr = cooperative_groups;
  constexpr int CELLS = 2 * 2 * GROUP;   // [stat][bin][feature]
  __shared__ float4 s_row[LB_WARPS][LH_ROWS];         // (word, g, h, -) of the rows of a warp's block
  __shared__ float s_acc[LB_WARPS][CELLS];            // each warp's cells at the end of an item
  __shared__ float s_cta[CELLS];                      // the CTA's cells, read by the cluster
  __shared__ int s_next;
  cgr::cluster_group cl = cgr::this_cluster();
  const int cs = static_cast<int>(cl.num_blocks());
  const int rank = static_cast<int>(cl.block_rank());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int total_items = plan->total_units * G;
  const int n_small = plan->n_small;
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
  cl.sync();
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next)) {
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
    const int nblk = p1 > p0 ? (p1 - p0 + LH_ROWS - 1) / LH_ROWS : 0;
    const uint32_t* gb = bits1 + static_cast<int64_t>(grp) * n;
    float g0 = 0.f, h0 = 0.f, g1 = 0.f, h1 = 0.f;   // lane f: feature 32 grp + f, bins 0 and 1
    for (int blk = warp; blk < nblk; blk += W) {
      const int pos = p0 + blk * LH_ROWS + lane;
      uint32_t word = 0u;
      float gv = 0.f, hv = 0.f;   // rows past the end add zero
      if (pos < p1) {
        const uint32_t row = order ? __ldg(order + pos) : static_cast<uint32_t>(pos);
        word = __ldg(gb + row);
        gv = cbgd::load_gh(gpos, pos);
        hv = cbgd::load_gh(hpos, pos);
      }
      s_row[warp][lane] = make_float4(__uint_as_float(word), gv, hv, 0.f);
      __syncwarp();
#pragma unroll 4
      for (int j = 0; j < LH_ROWS; ++j) {
        const float4 v = s_row[warp][j];
        if ((__float_as_uint(v.x) >> lane) & 1u) {
          g1 += v.y;
          h1 += v.z;
        } else {
          g0 += v.y;
          h0 += v.z;
        }
      }
      __syncwarp();
    }
    s_acc[warp][0 * 2 * GROUP + 0 * GROUP + lane] = g0;   // [stat][bin][feature]
    s_acc[warp][0 * 2 * GROUP + 1 * GROUP + lane] = g1;
    s_acc[warp][1 * 2 * GROUP + 0 * GROUP + lane] = h0;
    s_acc[warp][1 * 2 * GROUP + 1 * GROUP + lane] = h1;
    __syncthreads();
    // the CTA's warps in warp order
    for (int c = threadIdx.x; c < CELLS; c += blockDim.x) {
      float v = s_acc[0][c];
      for (int w = 1; w < W; ++w) v += s_acc[w][c];
      s_cta[c] = v;
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
    // this CTA's slice of the cells, summed over the cluster's CTAs in rank order
    const int per = (CELLS + cs - 1) / cs;
    float* dst = partials + static_cast<int64_t>(item) * CELLS;
    for (int c = rank * per + threadIdx.x; c < min(CELLS, (rank + 1) * per); c += blockDim.x) {
      float v = 0.f;
      for (int r = 0; r < cs; ++r) v += cl.map_shared_rank(s_cta, r)[c];
      dst[c] = v;
    }
    cl.sync();
  }
}

// ---------------------------------------- lane-per-feature, one statistic per warp
// The lane kernel with G and H split over a pair of warps: warp 2p accumulates G and warp
// 2p + 1 accumulates H of the same rows, each in a private FP32 histogram [max_bins][32]
// (32 KB at 255 bins instead of 64 KB), so twice as many warps fit on an SM to hide the
// shared-memory latency that bounds the one-warp-per-scheduler lane kernel. Both warps of a
// pair stage the same 32-row blocks (the second copy comes from L2); each loads only its
// own statistic. The batched updates and the per-unit reduction are as in the lane kernel:
// the G warps are summed in order into warp 0, the H warps into warp 1.
__device__ __forceinline__ float lds_f(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_f(uint32_t addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

inline size_t lp_warp_bytes(int max_bins) {
  return static_cast<size_t>(max_bins) * GROUP * sizeof(float) + static_cast<size_t>(LH_STAGES) * LH_ROWS * GROUP +
         LH_ROWS * sizeof(float);
}
inline int lp_warps(int max_bins, int requested_threads) {
  int w = static_cast<int>(SMEM_DYN_BUDGET / lp_warp_bytes(max_bins));
  if (w > LH_MAX_WARPS) w = LH_MAX_WARPS;
  if (requested_threads > 0 && requested_threads / 32 < w) w = requested_threads / 32;
  w &= ~1;
  return w < 2 ? 2 : w;
}
inline size_t lp_smem_bytes(int max_bins, int warps) { return static_cast<size_t>(warps) * lp_warp_bytes(max_bins); }

template <typename GH>
__global__ void __launch_bounds__(LH_MAX_WARPS * 32, 1)
    level_hist_pair_kernel(const uint8_t* __restrict__ bins, int64_t n, int G, int F, const uint32_t* __restrict__ order,
                           const GH* __restrict__ gpos, const GH* __restrict__ hpos, const Plan* __restrict__ plan,
                           int max_bins, float* __restrict__ partials) {
  namespace cgr = cooperative_groups;
  extern __shared__ __align__(16) unsigned char psh[];
  constexpr int MAX_CS = 16;
  constexpr uint32_t NONE = 0xffffffffu;
  cgr::cluster_group cl = cgr::this_cluster();
  const int cs = static_cast<int>(cl.num_blocks());
  const int rank = static_cast<int>(cl.block_rank());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int pair = warp >> 1, stat = warp & 1, P = W >> 1;
  const GH* sv = stat == 0 ? gpos : hpos;
  const int per_warp = max_bins * GROUP;   // float cells of one warp histogram
  float* hist_all = reinterpret_cast<float*>(psh);
  float* my = hist_all + static_cast<int64_t>(warp) * per_warp;
  unsigned char* stages = psh + static_cast<size_t>(W) * per_warp * sizeof(float);
  unsigned char* my_stage = stages + static_cast<size_t>(warp) * LH_STAGES * LH_ROWS * GROUP;
  float* my_sv = reinterpret_cast<float*>(stages + static_cast<size_t>(W) * LH_STAGES * LH_ROWS * GROUP) +
                 warp * LH_ROWS;
  const uint32_t stage_s = static_cast<uint32_t>(__cvta_generic_to_shared(my_stage));
  const uint32_t hbase = static_cast<uint32_t>(__cvta_generic_to_shared(my + lane));
  const int maxb1 = max_bins - 1;
  const float* peer0[MAX_CS];
  for (int r = 0; r < cs && r < MAX_CS; ++r) peer0[r] = cl.map_shared_rank(hist_all, r);
  const int total_items = plan->total_units * G;
  const int n_small = plan->n_small;
  __shared__ int s_next;   // this cluster's next work item (rank 0's slot)
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
  cl.sync();
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next)) {
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
    {
      float4* z = reinterpret_cast<float4*>(my);
      for (int i = lane; i < per_warp / 4; i += 32) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    const int nblk = p1 > p0 ? (p1 - p0 + LH_ROWS - 1) / LH_ROWS : 0;
    const int my_blocks = nblk > pair ? (nblk - pair + P - 1) / P : 0;
    const bool act = lane < F - grp * GROUP;
    const uint8_t* gb = bins + static_cast<int64_t>(grp) * n * GROUP;
    if (my_blocks > 0) {
      uint32_t rid[LH_AHEAD + 1];
      float vr[LH_AHEAD + 1];
      auto fetch = [&](int j, uint32_t& row, float& v) {
        const int pos = p0 + (pair + j * P) * LH_ROWS + lane;
        if (j < my_blocks && pos < p1) {
          row = order ? __ldg(order + pos) : static_cast<uint32_t>(pos);
          v = cbgd::load_gh(sv, pos);
        } else {
          row = NONE;   // a row past the end: zero record, zero statistic
          v = 0.f;
        }
      };
      auto copy_bins = [&](int j, uint32_t row) {
        const uint32_t dst = stage_s + static_cast<uint32_t>(((j % LH_STAGES) * LH_ROWS + lane) * GROUP);
        if (row != NONE) {
          const uint8_t* src = gb + static_cast<int64_t>(row) * GROUP;
          cp_async16(dst, src);
          cp_async16(dst + 16, src + 16);
        } else {
          asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n\tst.shared.v4.u32 [%2], {%1, %1, %1, %1};" ::"r"(dst),
                       "r"(0u), "r"(dst + 16u)
                       : "memory");
        }
      };
#pragma unroll
      for (int q = 0; q < LH_AHEAD; ++q) fetch(q, rid[q], vr[q]);
      copy_bins(0, rid[0]);
      cp_async_commit();
      if (1 < my_blocks) copy_bins(1, rid[1]);
      cp_async_commit();
      for (int j = 0; j < my_blocks; ++j) {
        fetch(j + LH_AHEAD, rid[LH_AHEAD], vr[LH_AHEAD]);
        if (j + 2 < my_blocks) copy_bins(j + 2, rid[2]);
        cp_async_commit();
        my_sv[lane] = vr[0];
        cp_async_wait<2>();
        __syncwarp();
        if (act) {
          const unsigned char* sb = my_stage + (j % LH_STAGES) * LH_ROWS * GROUP + lane;
          const float4* s4 = reinterpret_cast<const float4*>(my_sv);
          uint32_t a[LH_ROWS];
#pragma unroll
          for (int i = 0; i < LH_ROWS; ++i)
            a[i] = hbase + static_cast<uint32_t>(min(static_cast<int>(sb[i * GROUP]), maxb1)) * (GROUP * 4u);
          // batches of LH_BATCH rows: loads before stores, repeats take the batch's new value
#pragma unroll
          for (int i0 = 0; i0 < LH_ROWS; i0 += LH_BATCH) {
            float v[LH_BATCH];
#pragma unroll
            for (int q = 0; q < LH_BATCH; ++q) v[q] = lds_f(a[i0 + q]);
#pragma unroll
            for (int q = 0; q < LH_BATCH; ++q) {
              const int i = i0 + q;
#pragma unroll
              for (int e = 0; e < q; ++e)
                if (a[i0 + e] == a[i]) v[q] = v[e];
              const float4 sq = s4[i >> 2];
              v[q] += (i & 3) == 0 ? sq.x : (i & 3) == 1 ? sq.y : (i & 3) == 2 ? sq.z : sq.w;
            }
#pragma unroll
            for (int q = 0; q < LH_BATCH; ++q) sts_f(a[i0 + q], v[q]);
          }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < LH_AHEAD; ++q) {
          rid[q] = rid[q + 1];
          vr[q] = vr[q + 1];
        }
      }
      cp_async_wait<0>();
    }
    __syncthreads();
    // G warps (even) summed in order into warp 0, H warps (odd) into warp 1
    if (P > 1) {
      for (int e = threadIdx.x; e < 2 * per_warp; e += blockDim.x) {
        const int st = e / per_warp, c = e - st * per_warp;
        float sum = hist_all[static_cast<int64_t>(st) * per_warp + c];
        for (int q = 1; q < P; ++q) sum += hist_all[static_cast<int64_t>(2 * q + st) * per_warp + c];
        hist_all[static_cast<int64_t>(st) * per_warp + c] = sum;
      }
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) queue_take(plan, &s_next, cs);
    // this CTA's slice of bins, summed over the cluster's CTAs in rank order
    const int bs = (max_bins + cs - 1) / cs;
    const int b0 = rank * bs;
    const int nbs = max(0, min(max_bins, b0 + bs) - b0);
    float* dst = partials + static_cast<int64_t>(item) * (2 * max_bins * GROUP);
    for (int i = threadIdx.x; i < 2 * nbs * GROUP; i += blockDim.x) {
      const int st = i / (nbs * GROUP), rem = i - st * (nbs * GROUP);
      const int e = st * per_warp + b0 * GROUP + rem;
      float sum = 0.f;
      for (int r = 0; r < cs; ++r) sum += peer0[r][e];
      dst[e] = sum;
    }
    cl.sync();
  }
}

// ------------------------------------------------------------ reduce + subtract
// Every cell of a directly computed leaf gets the FP64 sum of its unit partials; the
// sibling gets parent - direct. For the feature the parent was
// split on, both children follow exactly from the parent (bins <= k stay in child 0, the
// rest in child 1), so their empty bins are exact zeros rather than rounding residue.
// Besides the FP64 histogram, a compensated FP32 copy (hi, lo) of every written cell goes
// to hist_df when it is given, so that split scoring needs no FP64 arithmetic.
__device__ __forceinline__ void put_cell(double* hist, float2* hist_df, int64_t cell, double v) {
  hist[cell] = v;
  if (hist_df) {
    const float hi = __double2float_rn(v);
    hist_df[cell] = make_float2(hi, __double2float_rn(v - static_cast<double>(hi)));
  }
}

// A block takes a tile of 32 features (one group) x RD_BINS bins x 2 statistics of one
// directly computed leaf: threads sum the unit partials of a cell in FP64 in unit order
// (reads coalesced over the group's features), the tile is transposed through shared
// memory, and the cells go out in the histogram's [leaf][f][b][stat] order (writes
// coalesced over bins and statistics).
constexpr int RD_BINS = 4;
constexpr int RD_THREADS = 256;   // 2 x RD_BINS x 32 = 256 cells, one per thread

template <int BINS>
__device__ __forceinline__ void reduce_tile(const Plan* __restrict__ plan, const float* __restrict__ partials, int G, int F, int max_bins,
                  const double* __restrict__ hist_prev, double* __restrict__ hist_cur,
                  const cbg_split* __restrict__ splits, int depth, float2* __restrict__ hist_df, int bx, int by,
                  const int32_t* __restrict__ n_borders, double (*tile)[BINS][2]) {   // tile: shared [GROUP][BINS][2]
  constexpr int RD_BINS = BINS;   // bins of the tile: 2 x BINS x 32 cells
  constexpr int CELLS = 2 * RD_BINS * GROUP;
  const int jj = by;
  if (jj >= plan->n_small) return;
  const int nbt = (max_bins + RD_BINS - 1) / RD_BINS;
  const int grp = bx / nbt, b0 = (bx - grp * nbt) * RD_BINS;
  if (grp >= G) return;
  const int u0 = plan->unit_begin[jj], u1 = plan->unit_begin[jj + 1];
  const int64_t item_elems = static_cast<int64_t>(2) * max_bins * GROUP;
  for (int c = threadIdx.x; c < CELLS; c += blockDim.x) {
    const int fl = c % GROUP, rest = c / GROUP;
    const int st = rest / RD_BINS, bl = rest - st * RD_BINS;
    const int b = b0 + bl;
    const int f = grp * GROUP + fl;
    double s = 0.0;
    // padding features and the bins above a feature's last border hold no rows: their
    // partials are zero, and FP64 additions are scarce on this GPU
    if (b < max_bins && f < F && (n_borders == nullptr || b <= n_borders[f])) {
      const float* src = partials + (static_cast<int64_t>(u0) * G + grp) * item_elems +
                         static_cast<int64_t>(st) * max_bins * GROUP + b * GROUP + fl;
      const int64_t step = G * item_elems;
      // four independent FP64 chains so that the unit loads overlap
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int u = u0;
      for (; u + 4 <= u1; u += 4, src += 4 * step) {
        s0 += static_cast<double>(src[0]);
        s1 += static_cast<double>(src[step]);
        s2 += static_cast<double>(src[2 * step]);
        s3 += static_cast<double>(src[3 * step]);
      }
      for (; u < u1; ++u, src += step) s0 += static_cast<double>(*src);
      s = (s0 + s1) + (s2 + s3);
    }
    tile[fl][bl][st] = s;
  }
  __syncthreads();
  const int leaf = plan->small_leaf[jj];
  const int large = plan->large_leaf[jj];
  const int par = plan->parent[jj];
  const bool exact = large >= 0 && depth > 0 && splits[depth - 1].feature >= grp * GROUP &&
                     splits[depth - 1].feature < (grp + 1) * GROUP;
  for (int c = threadIdx.x; c < CELLS; c += blockDim.x) {
    const int fl = c / (2 * RD_BINS), rem = c - fl * (2 * RD_BINS);
    const int bl = rem >> 1, st = rem & 1;
    const int f = grp * GROUP + fl, b = b0 + bl;
    if (f >= F || b >= max_bins) continue;
    const int64_t cell = ((static_cast<int64_t>(leaf) * F + f) * max_bins + b) * 2 + st;
    if (exact && splits[depth - 1].feature == f) {
      // the children of the parent's split feature follow exactly from the parent
      const int k = splits[depth - 1].border;
      const int64_t pcell = ((static_cast<int64_t>(par) * F + f) * max_bins + b) * 2 + st;
      const int64_t lcell = ((static_cast<int64_t>(large) * F + f) * max_bins + b) * 2 + st;
      const double pv = hist_prev[pcell];
      const bool small_is_child0 = leaf < (1 << (depth - 1));
      const bool in_child0 = b <= k;
      put_cell(hist_cur, hist_df, cell, (in_child0 == small_is_child0) ? pv : 0.0);
      put_cell(hist_cur, hist_df, lcell, (in_child0 == small_is_child0) ? 0.0 : pv);
      continue;
    }
    const double s = tile[fl][bl][st];
    put_cell(hist_cur, hist_df, cell, s);
    if (large >= 0) {
      const int64_t pcell = ((static_cast<int64_t>(par) * F + f) * max_bins + b) * 2 + st;
      const int64_t lcell = ((static_cast<int64_t>(large) * F + f) * max_bins + b) * 2 + st;
      put_cell(hist_cur, hist_df, lcell, hist_prev[pcell] - s);
    }
  }
}

// The reduction's block for the regular launch: a tile of RD_BINS bins, one cell a thread.
__device__ __forceinline__ void reduce_body(const Plan* __restrict__ plan, const float* __restrict__ partials, int G, int F, int max_bins,
                  const double* __restrict__ hist_prev, double* __restrict__ hist_cur,
                  const cbg_split* __restrict__ splits, int depth, float2* __restrict__ hist_df, int bx, int by,
                  const int32_t* __restrict__ n_borders = nullptr) {
  __shared__ double tile[GROUP][RD_BINS][2];
  reduce_tile<RD_BINS>(plan, partials, G, F, max_bins, hist_prev, hist_cur, splits, depth, hist_df, bx, by, n_borders,
                       tile);
}

__global__ void __launch_bounds__(RD_THREADS)
    reduce_kernel(const Plan* __restrict__ plan, const float* __restrict__ partials, int G, int F, int max_bins,
                  const double* __restrict__ hist_prev, double* __restrict__ hist_cur,
                  const cbg_split* __restrict__ splits, int depth, float2* __restrict__ hist_df,
                  const int32_t* __restrict__ n_borders) {
  // the histogram launch that filled the partials has ended: rearm its work queue
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) const_cast<Plan*>(plan)->queue = 0;
  reduce_body(plan, partials, G, F, max_bins, hist_prev, hist_cur, splits, depth, hist_df, blockIdx.x, blockIdx.y,
              n_borders);
}

// The batched form: one persistent launch for a level of many problems, in two phases.
// 1. Clusters take the histogram work items of every problem (unit x group, as in the
//    single-problem kernel, numbered problem after problem) from one queue (the first
//    problem's Plan::queue).
// 2. A CTA whose cluster finds that queue empty turns to the FP64 reduction: it takes
//    chunks of reduction tiles (BATCH_RD_CHUNK tiles of BATCH_RD_BINS bins of a group, the
//    single-problem reduction's blocks made 512 cells wide, of one directly built leaf)
//    from a second queue
//    (Plan::rqueue), on its own. A chunk of leaf jj first waits until every histogram
//    item of jj has written its partials (Plan::done). Those items were all handed out
//    before any cluster reached phase 2 and are held by clusters still running phase 1,
//    so the wait ends; it is bounded all the same: after wait_limit polls it sets
//    STATUS_TIMEOUT in the context's status word (reported by cbg_sync) and skips the
//    chunk, so the launch ends and the context stays usable. wait_extra > 0 raises the
//    count waited for past what can arrive (a test hook that makes every wait run out).
constexpr int HIST_MAX_BATCH = 2048;
constexpr int BATCH_RD_BINS = 8;      // phase-2 tiles: 2 x 8 x 32 = 512 cells, one per thread of a 512-thread CTA
constexpr int BATCH_RD_CHUNK = 4;     // tiles of a phase-2 chunk
constexpr unsigned BATCH_WAIT_LIMIT = 1u << 22;       // polls of about 0.25 us: about 1 s
// Dynamic shared memory of the batched kernel: the histogram, and at least the phase-2
// reduction tile that reuses it.
inline size_t batched_smem_bytes(int nb) {
  const size_t tile = sizeof(double) * GROUP * BATCH_RD_BINS * 2;
  return hist_smem_bytes(nb) > tile ? hist_smem_bytes(nb) : tile;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// first[p] = sum over problems q < p of count(q), a block-wide scan in chunks of blockDim
template <typename Count>
__device__ void batch_prefix(int n_probs, int* first, int* carry, Count count) {
  if (threadIdx.x == 0) *carry = 0;
  __syncthreads();
  for (int base = 0; base < n_probs; base += blockDim.x) {
    const int p = base + threadIdx.x;
    first[p < n_probs ? p + 1 : HIST_MAX_BATCH] = p < n_probs ? count(p) : 0;   // counts, scanned below
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = *carry;
      const int end = min(n_probs, base + static_cast<int>(blockDim.x));
      for (int q = base; q < end; ++q) {
        run += first[q + 1];
        first[q + 1] = run;
      }
      *carry = run;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) first[0] = 0;
  __syncthreads();
}

__device__ __forceinline__ int batch_find(const int* first, int n_probs, int item) {
  int lo = 0, hi = n_probs - 1;   // last p with first[p] <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename GH, int NB>
__global__ void __launch_bounds__(512, 3) level_hist_batched_kernel(const HistProblem* __restrict__ probs, int n_probs,
                                                                    int depth, unsigned* __restrict__ status,
                                                                    int wait_extra, unsigned wait_limit) {
  extern __shared__ __align__(16) float hsh[];   // [2][NB][32]
  __shared__ int s_first[HIST_MAX_BATCH + 1];
  __shared__ int s_carry;
  __shared__ int s_next;
  __shared__ int s_ok;
  namespace cgr = cooperative_groups;
  HistCta k(hsh);
  const Plan* qplan = probs[0].plan;
  // phase 1: histogram items
  batch_prefix(n_probs, s_first, &s_carry, [&](int p) { return probs[p].plan->total_units * probs[p].G; });
  cgr::this_cluster().sync();
  if (k.rank == 0 && threadIdx.x == 0) queue_take(qplan, &s_next, k.cs);
  cgr::this_cluster().sync();
  const int total_items = s_first[n_probs];
  for (int item = queue_read(&s_next); item < total_items; item = queue_read(&s_next)) {
    const int p = batch_find(s_first, n_probs, item);
    hist_item<GH, NB, 0>(probs[p], item - s_first[p], k.cs, k.rank, hsh, k.peer, k.sbase, &s_next, qplan, true);
  }
  // phase 2: reduction chunks, each CTA on its own (no distributed shared memory from here,
  // so the CTA's histogram buffer serves as the reduction's tile)
  __syncthreads();
  auto gx_of = [&](int p) { return probs[p].G * ((probs[p].max_bins + BATCH_RD_BINS - 1) / BATCH_RD_BINS); };
  auto chunks_per_leaf = [&](int p) { return (gx_of(p) + BATCH_RD_CHUNK - 1) / BATCH_RD_CHUNK; };
  batch_prefix(n_probs, s_first, &s_carry, [&](int p) { return probs[p].plan->n_small * chunks_per_leaf(p); });
  const int total_chunks = s_first[n_probs];
  int* const rq = &const_cast<Plan*>(qplan)->rqueue;
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(rq, 1);
    __syncthreads();
    const int c = s_next;
    if (c >= total_chunks) break;
    const int p = batch_find(s_first, n_probs, c);
    const HistProblem& P = probs[p];
    const int cpl = chunks_per_leaf(p), gx = gx_of(p);
    const int local = c - s_first[p];
    const int jj = local / cpl;
    const int b0 = (local - jj * cpl) * BATCH_RD_CHUNK;
    if (threadIdx.x == 0) {
      int ok = 1;
      const int need = (P.plan->unit_begin[jj + 1] - P.plan->unit_begin[jj]) * P.G + wait_extra;
      unsigned polls = 0;
      while (ld_acquire_gpu(&P.plan->done[jj]) < need) {
        if (++polls > wait_limit) {
          atomicOr(status, ::cbg::STATUS_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok)
      for (int bx = b0; bx < min(gx, b0 + BATCH_RD_CHUNK); ++bx) {
        reduce_tile<BATCH_RD_BINS>(P.plan, P.partials, P.G, P.F, P.max_bins, P.hist_prev, P.hist_cur, P.splits, depth,
                                   P.hist_df, bx, jj, P.n_borders,
                                   reinterpret_cast<double (*)[BATCH_RD_BINS][2]>(hsh));   // the histogram's buffer
        __syncthreads();   // every thread has read the shared tile before the next tile overwrites it
      }
    __syncthreads();   // s_next and s_ok are rewritten next round
  }
}

// Grid of reduce_kernel for one level: (bin tiles x groups, directly computed leaves).
inline dim3 reduce_grid(int G, int max_bins, int n_small) {
  return dim3(static_cast<unsigned>(G * ((max_bins + RD_BINS - 1) / RD_BINS)), static_cast<unsigned>(n_small));
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
  return L.kind == 3   ? hist_geom_mode<GH, 1>(ctx, L, g)
         : L.kind == 7 ? hist_geom_mode<GH, 2>(ctx, L, g)
                       : hist_geom_mode<GH, 0>(ctx, L, g);
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
  CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN_BUDGET));
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

// Warps, threads and shared memory of the lane-per-feature kernels (V as for lane_geom):
// `warps` counts the warps that hold histograms; the loader form adds its loader warp.
inline int lane_warps(const HistConfig& L, int V) {
  return V == 1   ? lp_warps(L.max_bins, L.threads)
         : V == 2 ? l4_warps(L.max_bins, L.threads)
         : V == 3 ? ld_warps(L.max_bins, L.threads)
                  : lh_warps(L.max_bins, L.threads);
}
inline int lane_threads_warps(int V, int warps) { return V == 3 ? 2 * warps : warps; }
inline size_t lane_smem(const HistConfig& L, int V, int warps) {
  return V == 1   ? lp_smem_bytes(L.max_bins, warps)
         : V == 2 ? l4_smem_bytes(L.max_bins, warps)
         : V == 3 ? ld_smem_bytes(L.max_bins, warps)
                  : lh_smem_bytes(L.max_bins, warps);
}
template <typename GH>
const void* lane_kernel_fn(int V) {
  return V == 1   ? reinterpret_cast<const void*>(level_hist_pair_kernel<GH>)
         : V == 2 ? reinterpret_cast<const void*>(level_hist_lane4_kernel<GH>)
         : V == 3 ? reinterpret_cast<const void*>(level_hist_lane_ld_kernel<GH>)
                  : reinterpret_cast<const void*>(level_hist_lane_kernel<GH>);
}

// Geometry of the lane-per-feature kernels (V: 0 one warp per 32 features, 1 one statistic
// per warp, 2 the 4-bit packed records, 3 with a loader warp): one CTA per SM
// with as many warp histograms as fit, and the cluster size (<= the requested one) that
// keeps the most CTAs resident.
template <typename GH, int V>
cbg_status lane_geom(cbg_ctx* ctx, const HistConfig& L, HistGeom* out) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, HistGeom> cache;
  const int warps = lane_warps(L, V);
  const auto key = std::make_tuple(ctx->device, L.max_bins, warps, L.cluster, static_cast<int>(sizeof(GH)));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return CBG_OK;
    }
  }
  const void* kern = lane_kernel_fn<GH>(V);
  const size_t smem = lane_smem(L, V, warps);
  CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN_BUDGET));
  HistGeom geom;
  for (int cs = L.cluster; cs >= 1; cs >>= 1) {
    if (cs > 8) CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(cs * ctx->num_sms));
    cfg.blockDim = dim3(static_cast<unsigned>(32 * lane_threads_warps(V, warps)));
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

// Geometry of the 1-bit kernel: 512-thread CTAs with static shared memory only, and the
// cluster size (<= the requested one) that keeps the most CTAs resident.
template <typename GH>
cbg_status bits_geom(cbg_ctx* ctx, const HistConfig& L, HistGeom* out) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, HistGeom> cache;
  const auto key = std::make_tuple(ctx->device, L.cluster, static_cast<int>(sizeof(GH)));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return CBG_OK;
    }
  }
  auto kern = level_hist_bits_kernel<GH>;
  HistGeom geom;
  for (int cs = L.cluster; cs >= 1; cs >>= 1) {
    if (cs > 8) CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(cs * ctx->num_sms));
    cfg.blockDim = dim3(static_cast<unsigned>(32 * LB_WARPS));
    cfg.dynamicSmemBytes = 0;
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

// The cluster size the plan must chunk for, and the clusters of a launch (identical for
// FP32 and BF16 gradients).
cbg_status hist_cluster_geom(cbg_ctx* ctx, const HistConfig& L, int* cs, int* clusters) {
  HistGeom g;
  cbg_status st = L.kind == 0   ? wp_geom<float>(ctx, L, &g)
                  : L.kind == 4 ? lane_geom<float, 0>(ctx, L, &g)
                  : L.kind == 5 ? lane_geom<float, 1>(ctx, L, &g)
                  : L.kind == 6 ? lane_geom<float, 2>(ctx, L, &g)
                  : L.kind == 8 ? lane_geom<float, 3>(ctx, L, &g)
                  : L.kind == 9 ? bits_geom<float>(ctx, L, &g)
                                : hist_geom<float>(ctx, L, &g);
  if (st != CBG_OK) return st;
  *cs = g.cs;
  if (clusters) *clusters = g.clusters;
  return CBG_OK;
}
cbg_status hist_cluster_size(cbg_ctx* ctx, const HistConfig& L, int* cs) { return hist_cluster_geom(ctx, L, cs, nullptr); }

// Work items a level's histogram launch is cut into, per cluster of the launch: enough
// that the clusters, taking items from the queue as they finish, end close together.
constexpr int HIST_ITEMS_PER_CLUSTER = 4;
inline int hist_target_units(int clusters, int G) {
  return (HIST_ITEMS_PER_CLUSTER * clusters + G - 1) / G;
}

// Every occupancy query and function attribute that a launch of this configuration
// needs, made ahead of a graph capture (those calls cannot be captured).
template <typename GH>
cbg_status hist_warm(cbg_ctx* ctx, const HistConfig& L) {
  HistGeom g;
  cbg_status st = L.kind == 0   ? wp_geom<GH>(ctx, L, &g)
                  : L.kind == 4 ? lane_geom<GH, 0>(ctx, L, &g)
                  : L.kind == 5 ? lane_geom<GH, 1>(ctx, L, &g)
                  : L.kind == 6 ? lane_geom<GH, 2>(ctx, L, &g)
                  : L.kind == 8 ? lane_geom<GH, 3>(ctx, L, &g)
                  : L.kind == 9 ? bits_geom<GH>(ctx, L, &g)
                                : hist_geom<GH>(ctx, L, &g);
  if (st != CBG_OK) return st;
  int cs = 1;
  return hist_cluster_size(ctx, L, &cs);
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

// The batched kernel with the cluster size the problems' plans were made for: the number
// of co-resident clusters (cached per geometry); 0 if none fits.
template <typename GH, int NB>
cbg_status batched_clusters(cbg_ctx* ctx, int threads, int cs, int* clusters) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int>, int> cache;
  const auto key = std::make_tuple(ctx->device, threads, cs, static_cast<int>(sizeof(GH)));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *clusters = it->second;
      return CBG_OK;
    }
  }
  auto kern = level_hist_batched_kernel<GH, NB>;
  CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(batched_smem_bytes(NB))));
  if (cs > 8) CBG_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(cs * ctx->num_sms));
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = batched_smem_bytes(NB);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(cs);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = n;
  *clusters = n;
  return CBG_OK;
}

template <typename GH, int NB>
cbg_status launch_hist_batched_nb(cbg_ctx* ctx, const HistProblem* table, int n_probs, int threads, int cs, int depth,
                                  int wait_extra, unsigned wait_limit) {
  int clusters = 0;
  cbg_status st = batched_clusters<GH, NB>(ctx, threads, cs, &clusters);
  if (st != CBG_OK) return st;
  if (clusters <= 0) return ::cbg::fail(ctx, CBG_EUNSUPPORTED, "no co-resident batched histogram cluster of %d fits", cs);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(cs * clusters));
  cfg.blockDim = dim3(static_cast<unsigned>(threads));
  cfg.dynamicSmemBytes = batched_smem_bytes(NB);
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(cs);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CBG_CUDA(ctx, cudaLaunchKernelEx(&cfg, level_hist_batched_kernel<GH, NB>, table, n_probs, depth, ctx->d_status,
                                   wait_extra, wait_limit));
  return CBG_OK;
}

// One histogram-and-reduction launch for level `depth` of many problems (shared-reduction
// kernel): table is a device array of n_probs entries, nb_alloc the largest bin allocation
// among them; wait_extra / wait_limit as for level_hist_batched_kernel.
template <typename GH>
cbg_status launch_hist_batched(cbg_ctx* ctx, int nb_alloc, const HistProblem* table, int n_probs, int threads,
                               int cs, bool query_only = false, int depth = 0, int wait_extra = 0,
                               unsigned wait_limit = BATCH_WAIT_LIMIT) {
  auto run = [&](auto nbc) -> cbg_status {
    constexpr int NB = decltype(nbc)::value;
    if (query_only) {
      int clusters = 0;
      cbg_status st = batched_clusters<GH, NB>(ctx, threads, cs, &clusters);
      if (st != CBG_OK) return st;
      return clusters > 0 ? CBG_OK : CBG_EUNSUPPORTED;
    }
    return launch_hist_batched_nb<GH, NB>(ctx, table, n_probs, threads, cs, depth, wait_extra, wait_limit);
  };
  switch (nb_alloc) {
    case 2: return run(std::integral_constant<int, 2>{});
    case 4: return run(std::integral_constant<int, 4>{});
    case 8: return run(std::integral_constant<int, 8>{});
    case 16: return run(std::integral_constant<int, 16>{});
    case 32: return run(std::integral_constant<int, 32>{});
    case 64: return run(std::integral_constant<int, 64>{});
    case 128: return run(std::integral_constant<int, 128>{});
    case 256: return run(std::integral_constant<int, 256>{});
    default: return ::cbg::fail(ctx, CBG_EINVAL, "unsupported bin allocation %d", nb_alloc);
  }
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
  if (L.kind == 4 || L.kind == 5 || L.kind == 6) {
    const bool pair = L.kind == 5, packed = L.kind == 6;
    HistGeom geom;
    st = pair ? lane_geom<GH, 1>(ctx, L, &geom) : packed ? lane_geom<GH, 2>(ctx, L, &geom) : lane_geom<GH, 0>(ctx, L, &geom);
    if (st != CBG_OK) return st;
    if (geom.cs != cs) return ::cbg::fail(ctx, CBG_ECUDA, "histogram cluster size changed between plan and launch");
    const int warps = pair ? lp_warps(L.max_bins, L.threads)
                    : packed ? l4_warps(L.max_bins, L.threads)
                             : lh_warps(L.max_bins, L.threads);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(geom.cs * geom.clusters));
    cfg.blockDim = dim3(static_cast<unsigned>(32 * warps));
    cfg.dynamicSmemBytes = pair ? lp_smem_bytes(L.max_bins, warps)
                         : packed ? l4_smem_bytes(L.max_bins, warps)
                                  : lh_smem_bytes(L.max_bins, warps);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(geom.cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // for the packed kernel `bins` is the 4-bit layout (bins4)
    CBG_CUDA(ctx, cudaLaunchKernelEx(&cfg,
                                     pair     ? level_hist_pair_kernel<GH>
                                     : packed ? level_hist_lane4_kernel<GH>
                                              : level_hist_lane_kernel<GH>,
                                     bins, L.n, L.G, L.F, order, gg, hh, plan, L.max_bins, partials));
    return CBG_OK;
  }
  if (L.kind == 9) {   // `bins` is the 1-bit layout (bits1)
    HistGeom geom;
    st = bits_geom<GH>(ctx, L, &geom);
    if (st != CBG_OK) return st;
    if (geom.cs != cs) return ::cbg::fail(ctx, CBG_ECUDA, "histogram cluster size changed between plan and launch");
    if (L.max_bins != 2) return ::cbg::fail(ctx, CBG_EINVAL, "the 1-bit histogram kernel needs max_bins = 2");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(geom.cs * geom.clusters));
    cfg.blockDim = dim3(static_cast<unsigned>(32 * LB_WARPS));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(geom.cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CBG_CUDA(ctx, cudaLaunchKernelEx(&cfg, level_hist_bits_kernel<GH>, reinterpret_cast<const uint32_t*>(bins), L.n,
                                     L.G, L.F, order, gg, hh, plan, partials));
    return CBG_OK;
  }
  if (L.kind == 8) {
    HistGeom geom;
    st = lane_geom<GH, 3>(ctx, L, &geom);
    if (st != CBG_OK) return st;
    if (geom.cs != cs) return ::cbg::fail(ctx, CBG_ECUDA, "histogram cluster size changed between plan and launch");
    const int warps = ld_warps(L.max_bins, L.threads);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(geom.cs * geom.clusters));
    cfg.blockDim = dim3(static_cast<unsigned>(32 * lane_threads_warps(3, warps)));
    cfg.dynamicSmemBytes = ld_smem_bytes(L.max_bins, warps);
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(geom.cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CBG_CUDA(ctx, cudaLaunchKernelEx(&cfg, level_hist_lane_ld_kernel<GH>, bins, L.n, L.G, L.F, order, gg, hh, plan,
                                     L.max_bins, partials, ctx->d_status, ctx->test_force_wait_timeout ? 1 : 0,
                                     ctx->test_force_wait_timeout ? 4096u : LD_WAIT_LIMIT));
    return CBG_OK;
  }
  if (L.kind == 7) {
    switch (L.nb_alloc) {
      case 2: return launch_hist_nb<GH, 2, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 4: return launch_hist_nb<GH, 4, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 8: return launch_hist_nb<GH, 8, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 16: return launch_hist_nb<GH, 16, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 32: return launch_hist_nb<GH, 32, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 64: return launch_hist_nb<GH, 64, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 128: return launch_hist_nb<GH, 128, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      case 256: return launch_hist_nb<GH, 256, 2>(ctx, L, bins, order, gg, hh, plan, partials, cs);
      default: return ::cbg::fail(ctx, CBG_EINVAL, "unsupported bin allocation %d", L.nb_alloc);
    }
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
