// Context, error reporting and library workspace.
#include "cbg_internal.cuh"

#include <cstring>
#include <new>

namespace cbg {

cbg_status fail(cbg_ctx* ctx, cbg_status code, const char* fmt, ...) {
  if (ctx) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

cbg_status ws_reserve(cbg_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return CBG_OK;
  if (ctx->ws_fixed)
    return fail(ctx, CBG_ENOMEM, "library workspace of %zu bytes is smaller than the %zu needed",
                ctx->ws_bytes, bytes);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CBG_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(ctx, CBG_ENOMEM, "workspace must grow to %zu bytes but the stream is capturing", bytes);
  CBG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) CBG_CUDA(ctx, cudaFree(ctx->ws));
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(ctx, CBG_ENOMEM, "cudaMalloc(%zu) for the library workspace failed: %s", want,
                cudaGetErrorString(e));
  }
  ctx->ws_bytes = want;
  return CBG_OK;
}

cbg_status prof_begin(cbg_ctx* ctx, cudaEvent_t* a, cudaEvent_t* b) {
  *a = *b = nullptr;
  if (!ctx->profile) return CBG_OK;
  while (ctx->ev_pool.size() < 2 * (ctx->ev_used + 1)) {
    cudaEvent_t e;
    CBG_CUDA(ctx, cudaEventCreate(&e));
    ctx->ev_pool.push_back(e);
  }
  *a = ctx->ev_pool[2 * ctx->ev_used];
  *b = ctx->ev_pool[2 * ctx->ev_used + 1];
  ctx->ev_used++;
  CBG_CUDA(ctx, cudaEventRecord(*a, ctx->stream));
  return CBG_OK;
}

cbg_status prof_end(cbg_ctx* ctx, cudaEvent_t b) {
  if (!b) return CBG_OK;
  CBG_CUDA(ctx, cudaEventRecord(b, ctx->stream));
  return CBG_OK;
}

}  // namespace cbg

using namespace cbg;

extern "C" {

const char* cbg_version(void) { return "cbg 0.1 (sm_103a)"; }

cbg_status cbg_ctx_create(int device, void* cuda_stream, size_t workspace_bytes, cbg_ctx** out) {
  if (!out) return CBG_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return CBG_EINVAL;
  }
  cbg_ctx* ctx = new (std::nothrow) cbg_ctx();
  if (!ctx) return CBG_ENOMEM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard guard(device);
  cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(unsigned int));
  if (e == cudaSuccess && workspace_bytes > 0) {
    e = cudaMalloc(&ctx->ws, workspace_bytes);
    if (e == cudaSuccess) {
      ctx->ws_bytes = workspace_bytes;
      ctx->ws_fixed = true;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->ws) cudaFree(ctx->ws);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? CBG_ENOMEM : CBG_ECUDA;
  }
  *out = ctx;
  return CBG_OK;
}

void cbg_ctx_destroy(cbg_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (cudaStream_t st : ctx->branch_streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : ctx->branch_events) cudaEventDestroy(e);
  cudaGetLastError();
  delete ctx;
}

cbg_status cbg_profile_enable(cbg_ctx* ctx, int enable) {
  if (!ctx) return CBG_EINVAL;
  ctx->profile = enable != 0;
  return CBG_OK;
}

cbg_status cbg_profile_read(cbg_ctx* ctx, int reset, double* hist_ms, int64_t* hist_launches) {
  if (!ctx) return CBG_EINVAL;
  DeviceGuard guard(ctx->device);
  CBG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0.f;
    CBG_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]));
    ctx->prof_ms += ms;
    ctx->prof_launches++;
  }
  ctx->ev_used = 0;
  if (hist_ms) *hist_ms = ctx->prof_ms;
  if (hist_launches) *hist_launches = ctx->prof_launches;
  if (reset) {
    ctx->prof_ms = 0.0;
    ctx->prof_launches = 0;
  }
  return CBG_OK;
}

const char* cbg_last_error(const cbg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int cbg_num_sms(const cbg_ctx* ctx) { return ctx ? ctx->num_sms : 0; }

cbg_status cbg_set_stream(cbg_ctx* ctx, void* cuda_stream) {
  if (!ctx) return CBG_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return CBG_OK;
}

cbg_status cbg_test_force_wait_timeout(cbg_ctx* ctx, int enable) {
  if (!ctx) return CBG_EINVAL;
  ctx->test_force_wait_timeout = enable != 0;
  return CBG_OK;
}

cbg_status cbg_sync(cbg_ctx* ctx) {
  if (!ctx) return CBG_EINVAL;
  DeviceGuard guard(ctx->device);
  CBG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  unsigned int status = 0;
  CBG_CUDA(ctx, cudaMemcpy(&status, ctx->d_status, sizeof(status), cudaMemcpyDeviceToHost));
  if (status) {
    CBG_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(unsigned int)));
    if (status & STATUS_TIMEOUT) return fail(ctx, CBG_ETIMEOUT, "a bounded device-side wait ran out");
    if (status & STATUS_NONFINITE) return fail(ctx, CBG_EDATA, "a feature value was NaN or infinite");
    if (status & STATUS_BAD_LABEL) return fail(ctx, CBG_EDATA, "a binary label was not 0 or 1");
    if (status & STATUS_BAD_BIN)
      return fail(ctx, CBG_EDATA, "a bin too large for its packed layout (16 or more in 4 bits, 2 or more in 1 bit)");
    return fail(ctx, CBG_EDATA, "device status 0x%x", status);
  }
  return CBG_OK;
}

}  // extern "C"
