// Context, error reporting, scratch buffers and host/device staging.
#include <cstring>
#include <mutex>
#include <utility>

#include "internal.h"

namespace tmat {

int set_error(tmat_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(tmat_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
  int code = (e == cudaErrorMemoryAllocation) ? TMAT_ENOMEM : TMAT_ECUDA;
  // a non-sticky error (allocation, launch configuration) is cleared so that the next launch
  // check does not report it again; a sticky one stays whatever is done here
  cudaGetLastError();
  return set_error(ctx, code, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

int scratch(tmat_ctx* ctx, const char* name, size_t bytes, void** out) {
  DevBuf& b = ctx->bufs[name];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) {
      TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      TM_CUDA(ctx, cudaFree(b.p));
      b.p = nullptr;
      b.bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    TM_CUDA(ctx, cudaMalloc(&b.p, want));
    b.bytes = want;
  }
  *out = b.p;
  return TMAT_OK;
}

static cudaEvent_t pooled_event(tmat_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

cudaEvent_t timing_begin(tmat_ctx* ctx) {
  if (!ctx->timing || ctx->timing_skip) return nullptr;
  cudaEvent_t e = pooled_event(ctx);
  if (e) cudaEventRecord(e, ctx->stream);
  return e;
}

void timing_end(tmat_ctx* ctx, const char* kind, cudaEvent_t start, double bytes) {
  if (!ctx->timing) return;
  ctx->timed_calls[kind] += 1;
  if (!start) return;
  cudaEvent_t e = pooled_event(ctx);
  if (!e) return;
  cudaEventRecord(e, ctx->stream);
  ctx->timed[kind].push_back({start, e});
  ctx->timed_bytes[kind] += bytes;
}

// The limit is an attribute of the kernel (per device), shared by every context of the
// process: the record is process-wide and the limit only grows, so that one context never
// lowers it below what another has launched with.
int set_smem_limit(tmat_ctx* ctx, const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limits;
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limits[{ctx->device, func}];
  if (cur >= (int)bytes) return TMAT_OK;
  TM_CUDA(ctx, cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = (int)bytes;
  return TMAT_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int stage_in(tmat_ctx* ctx, const char* name, const void* user, size_t bytes, Staged* s) {
  s->user = user;
  s->bytes = bytes;
  s->host = false;
  s->dev = const_cast<void*>(user);
  if (!user) return TMAT_OK;
  if (is_device_ptr(user)) return TMAT_OK;
  s->host = true;
  TM_TRY(scratch(ctx, name, bytes, &s->dev));
  if (bytes) TM_CUDA(ctx, cudaMemcpyAsync(s->dev, user, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return TMAT_OK;
}

int stage_out(tmat_ctx* ctx, const char* name, void* user, size_t bytes, Staged* s) {
  s->user = user;
  s->bytes = bytes;
  s->host = false;
  s->dev = user;
  if (!user) return TMAT_OK;
  if (is_device_ptr(user)) return TMAT_OK;
  s->host = true;
  return scratch(ctx, name, bytes, &s->dev);
}

int aux_stream_ready(tmat_ctx* ctx) {
  if (!ctx->aux_stream) TM_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
  if (!ctx->aux_event) TM_CUDA(ctx, cudaEventCreateWithFlags(&ctx->aux_event, cudaEventDisableTiming));
  return TMAT_OK;
}

int finish_out(tmat_ctx* ctx, Staged* s) {
  if (s->user && s->host && s->bytes) {
    TM_CUDA(ctx, cudaMemcpyAsync(const_cast<void*>(s->user), s->dev, s->bytes, cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return TMAT_OK;
}

}  // namespace tmat

using namespace tmat;

// recorded timing events go back to the pool (destroy_all: release them, at destruction)
static void drop_events(tmat_ctx* ctx, bool destroy_all = false) {
  for (auto& kv : ctx->timed)
    for (auto& pr : kv.second) {
      ctx->event_pool.push_back(pr.first);
      ctx->event_pool.push_back(pr.second);
    }
  ctx->timed.clear();
  ctx->timed_bytes.clear();
  ctx->timed_calls.clear();
  if (destroy_all) {
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    ctx->event_pool.clear();
  }
}


extern "C" int tmat_ctx_create(int device, void* cuda_stream, tmat_ctx** out) {
  if (!out) return TMAT_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TMAT_ECUDA;
  }
  tmat_ctx* c = new tmat_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost(&c->pinned, 4096) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TMAT_ENOMEM;
  }
  *out = c;
  return TMAT_OK;
}

extern "C" int tmat_ctx_set_stream(tmat_ctx* ctx, void* cuda_stream) {
  if (!ctx) return TMAT_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return TMAT_OK;
}

extern "C" int tmat_ctx_destroy(tmat_ctx* ctx) {
  if (!ctx) return TMAT_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->bufs) cudaFree(kv.second.p);
  for (auto& kv : ctx->tables) free_tables(kv.second);
  drop_events(ctx, true);
  if (ctx->flag_event) cudaEventDestroy(ctx->flag_event);
  if (ctx->flag_host) cudaFreeHost(ctx->flag_host);
  if (ctx->aux_stream) {
    cudaStreamSynchronize(ctx->aux_stream);
    cudaStreamDestroy(ctx->aux_stream);
  }
  if (ctx->aux_event) cudaEventDestroy(ctx->aux_event);
  cudaFreeHost(ctx->pinned);
  delete ctx;
  return TMAT_OK;
}

extern "C" const char* tmat_last_error(const tmat_ctx* ctx) { return ctx ? ctx->err : "null context"; }

extern "C" int64_t tmat_ctx_launch_count(const tmat_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int tmat_ctx_set_lattice_fft(tmat_ctx* ctx, int enable) {
  if (!ctx) return TMAT_EINVAL;
  if (enable < 0 || enable > 2) return set_error(ctx, TMAT_EINVAL, "tmat_ctx_set_lattice_fft: enable must be 0, 1 or 2");
  ctx->lattice_fft = enable != 0;
  ctx->fft_quad = enable == 1;
  return TMAT_OK;
}

extern "C" int tmat_ctx_set_tensor_cores(tmat_ctx* ctx, int enable) {
  if (!ctx) return TMAT_EINVAL;
  ctx->tensor_cores = enable != 0;
  ctx->tc_variant = enable == 2 ? 1 : 0;
  return TMAT_OK;
}

extern "C" int tmat_ctx_set_timing(tmat_ctx* ctx, int enable) {
  if (!ctx) return TMAT_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  drop_events(ctx);
  if (enable < 0) return set_error(ctx, TMAT_EINVAL, "tmat_ctx_set_timing: enable must be >= 0");
  ctx->timing = enable != 0;
  ctx->timing_every = enable > 1 ? enable : 1;
  ctx->timing_skip = false;
  ctx->timing_iter = 0;
  return TMAT_OK;
}

extern "C" int tmat_ctx_kernel_calls(tmat_ctx* ctx, const char* kind, int64_t* calls) {
  if (!ctx || !kind || !calls) return TMAT_EINVAL;
  auto it = ctx->timed_calls.find(kind);
  *calls = it == ctx->timed_calls.end() ? 0 : it->second;
  return TMAT_OK;
}

extern "C" int tmat_ctx_kernel_bytes(tmat_ctx* ctx, const char* kind, double* bytes) {
  if (!ctx || !kind || !bytes) return TMAT_EINVAL;
  auto it = ctx->timed_bytes.find(kind);
  *bytes = it == ctx->timed_bytes.end() ? 0.0 : it->second;
  return TMAT_OK;
}

extern "C" int tmat_ctx_kernel_time(tmat_ctx* ctx, const char* kind, int64_t* launches, double* total_ms) {
  if (!ctx || !kind || !launches || !total_ms) return TMAT_EINVAL;
  TM_CUDA(ctx, cudaSetDevice(ctx->device));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *launches = 0;
  *total_ms = 0.0;
  auto it = ctx->timed.find(kind);
  if (it == ctx->timed.end()) return TMAT_OK;
  for (auto& pr : it->second) {
    float ms = 0;
    TM_CUDA(ctx, cudaEventElapsedTime(&ms, pr.first, pr.second));
    *total_ms += ms;
    *launches += 1;
  }
  return TMAT_OK;
}

extern "C" int tmat_ctx_memory(const tmat_ctx* ctx, int64_t* bytes_out) {
  if (!ctx || !bytes_out) return TMAT_EINVAL;
  int64_t b = 0;
  for (const auto& kv : ctx->bufs) b += (int64_t)kv.second.bytes;
  *bytes_out = b;
  return TMAT_OK;
}

extern "C" int tmat_ctx_set_compressed_basis(tmat_ctx* ctx, int enable) {
  if (!ctx) return TMAT_EINVAL;
  ctx->compress_basis = enable != 0;
  return TMAT_OK;
}

extern "C" int tmat_ctx_set_field_precision(tmat_ctx* ctx, int precision) {
  if (!ctx) return TMAT_EINVAL;
  if (precision != TMAT_PREC_FP64 && precision != TMAT_PREC_MIXED)
    return set_error(ctx, TMAT_EINVAL, "tmat_ctx_set_field_precision: TMAT_PREC_FP64 or TMAT_PREC_MIXED");
  ctx->field_mixed = precision == TMAT_PREC_MIXED;
  return TMAT_OK;
}
