// Allocation-free root histogram (cbg_histogram_noalloc).
//
// Some callers cannot allocate device memory: code that runs inside a host application
// which owns the whole device memory budget (a framework's caching allocator or a fixed
// arena that a stray cudaMalloc would fragment or overrun), or plugin code that is not
// allowed to call cudaMalloc at all. The regular level builder needs a caller-allocated
// tree state; this entry point needs nothing but its inputs and its output. Its scratch
// (the work-unit plan and the FP32 partial histograms) lives in one file-scope device
// array, which every GPU that loads the library holds until the process exits.
#include "cbg_internal.cuh"
#include "level_hist.cuh"

using namespace cbg;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = static_cast<size_t>(16) << 20;   // 16 MiB per device
constexpr int NOALLOC_ROWS_PER_CTA = 4096;        // rows per CTA while the scratch has room for the units
constexpr int NOALLOC_MAX_ROWS_PER_CTA = 16384;   // beyond this one FP32 cell would sum too many rows
constexpr int64_t NOALLOC_MAX_N = (int64_t(1) << 31) - (int64_t(1) << 20);   // slack for the last chunk's end

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on ctx's device (current while this runs). In host
// code the array's name is only a stand-in. The address is looked up by the first call
// through a context and kept in it; a new context (for example after cudaDeviceReset,
// which may reload the module at another address) looks it up again.
cbg_status scratch_address(cbg_ctx* ctx, void** out) {
  if (!ctx->noalloc_scratch) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(ctx, CBG_ECUDA, "cudaGetSymbolAddress of the histogram scratch failed: %s", cudaGetErrorString(e));
    ctx->noalloc_scratch = p;
  }
  *out = ctx->noalloc_scratch;
  return CBG_OK;
}

// Plan of the single root leaf: all n rows in identity order, `units` work units per
// feature group of cs x chunk_rows rows.
__global__ void root_plan_kernel(Plan* plan, int n, int units, int chunk_rows) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  plan->queue = 0;
  plan->rqueue = 0;
  plan->done[0] = 0;
  plan->n_small = 1;
  plan->total_units = units;
  plan->level_leaves = 1;
  plan->small_leaf[0] = 0;
  plan->large_leaf[0] = -1;
  plan->parent[0] = -1;
  plan->unit_begin[0] = 0;
  plan->unit_begin[1] = units;
  plan->chunk_rows[0] = chunk_rows;
  plan->seg_start[0] = 0;
  plan->seg_cnt[0] = n;
}

}  // namespace

extern "C" cbg_status cbg_histogram_noalloc(cbg_ctx* ctx, const uint8_t* bins, int64_t n, int32_t F, int32_t F_pad,
                                            int32_t max_bins, const void* g, const void* h, int32_t gh_dtype,
                                            double* hist_out) {
  if (!ctx) return CBG_EINVAL;
  CBG_REQUIRE(ctx, n >= 1 && n <= NOALLOC_MAX_N, "n must be in [1, 2^31 - 2^20]");
  CBG_REQUIRE(ctx, F >= 1 && F_pad >= F && F_pad % GROUP == 0, "F_pad must be a multiple of 32 and >= F >= 1");
  CBG_REQUIRE(ctx, max_bins >= 2 && max_bins <= 256, "max_bins must be in [2, 256]");
  CBG_REQUIRE(ctx, gh_dtype == CBG_F32 || gh_dtype == CBG_BF16, "bad gh_dtype");
  CBG_REQUIRE(ctx, bins && g && h && hist_out, "NULL argument");
  DeviceGuard guard(ctx->device);
  HistConfig hc;
  hc.n = n;
  hc.G = F_pad / GROUP;
  hc.F = F;
  hc.max_bins = max_bins;
  hc.nb_alloc = 2;
  while (hc.nb_alloc < max_bins) hc.nb_alloc <<= 1;
  hc.threads = 512;
  hc.cluster = 8;
  hc.kind = 1;
  const size_t plan_bytes = (sizeof(Plan) + 255) / 256 * 256;
  const size_t unit_bytes = static_cast<size_t>(hc.G) * 2 * max_bins * GROUP * sizeof(float);
  if (plan_bytes + unit_bytes > NOALLOC_SCRATCH_BYTES)
    return fail(ctx, CBG_EINVAL,
                "F_pad %d x %d bins needs %zu bytes of partials per work unit; the %zu-byte scratch of "
                "cbg_histogram_noalloc holds at most %zu",
                F_pad, max_bins, unit_bytes, NOALLOC_SCRATCH_BYTES, NOALLOC_SCRATCH_BYTES - plan_bytes);
  void* scratch = nullptr;
  cbg_status st = scratch_address(ctx, &scratch);
  if (st != CBG_OK) return st;
  int cs = 1;
  st = hist_cluster_size(ctx, hc, &cs);
  if (st != CBG_OK) return st;
  const int64_t max_units = static_cast<int64_t>((NOALLOC_SCRATCH_BYTES - plan_bytes) / unit_bytes);
  int64_t units = ceil_div(n, static_cast<int64_t>(cs) * NOALLOC_ROWS_PER_CTA);
  if (units > max_units) units = max_units;
  if (units < 1) units = 1;
  if (ceil_div(n, units * cs) > NOALLOC_MAX_ROWS_PER_CTA)
    return fail(ctx, CBG_EINVAL,
                "n = %lld rows at F_pad %d x %d bins: the scratch holds %lld work units of %d CTAs, which would "
                "put more than %d rows into one CTA's FP32 histogram; at most %lld rows fit",
                static_cast<long long>(n), F_pad, max_bins, static_cast<long long>(max_units), cs,
                NOALLOC_MAX_ROWS_PER_CTA, static_cast<long long>(max_units * cs * NOALLOC_MAX_ROWS_PER_CTA));
  const int chunk_rows = static_cast<int>(ceil_div(n, units * cs));
  Plan* plan = static_cast<Plan*>(scratch);
  float* partials = reinterpret_cast<float*>(static_cast<char*>(scratch) + plan_bytes);
  root_plan_kernel<<<1, 32, 0, ctx->stream>>>(plan, static_cast<int>(n), static_cast<int>(units), chunk_rows);
  CBG_CHECK_LAUNCH(ctx);
  st = gh_dtype == CBG_F32 ? launch_hist<float>(ctx, hc, bins, nullptr, g, h, plan, partials)
                           : launch_hist<__nv_bfloat16>(ctx, hc, bins, nullptr, g, h, plan, partials);
  if (st != CBG_OK) return st;
  reduce_kernel<<<reduce_grid(hc.G, max_bins, 1), RD_THREADS, 0, ctx->stream>>>(plan, partials, hc.G, F, max_bins,
                                                                               nullptr, hist_out, nullptr, 0, nullptr, nullptr);
  CBG_CHECK_LAUNCH(ctx);
  return CBG_OK;
}
