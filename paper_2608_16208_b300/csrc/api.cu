// Context, status and error reporting of the C ABI.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>

#include "bie_internal.cuh"

namespace bie {
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

bie_status cuda_fail(cudaError_t e, const char* where) {
  set_error("%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? BIE_ENOMEM : BIE_ECUDA;
}

bie_status check_device(bie_ctx ctx, const char* where) {
  int cur = -1;
  const cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, where);
  if (cur != ctx->device) {
    set_error("%s: the context's device (%d) is not the current device (%d)", where, ctx->device, cur);
    return BIE_EINVAL;
  }
  return BIE_OK;
}

int trace_begin(bie_ctx ctx, int kind) {
  if (!ctx || !ctx->trace) return -1;
  if (!ctx->marks) ctx->marks = new std::vector<TraceMark>();
  TraceMark m;
  m.kind = kind;
  if (cudaEventCreate(&m.e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&m.e1) != cudaSuccess) {
    cudaEventDestroy(m.e0);
    return -1;
  }
  cudaEventRecord(m.e0, ctx->stream);
  ctx->marks->push_back(m);
  return (int)ctx->marks->size() - 1;
}

void trace_end(bie_ctx ctx, int mark) {
  if (mark < 0 || !ctx->marks || mark >= (int)ctx->marks->size()) return;
  cudaEventRecord((*ctx->marks)[mark].e1, ctx->stream);
}

static void trace_clear(bie_ctx ctx) {
  if (!ctx->marks) return;
  for (TraceMark& m : *ctx->marks) {
    cudaEventDestroy(m.e0);
    cudaEventDestroy(m.e1);
  }
  ctx->marks->clear();
}

}  // namespace bie

extern "C" {

bie_status bie_ctx_set_option(bie_ctx ctx, int option, int value) {
  if (!ctx) { bie::set_error("bie_ctx_set_option: NULL context"); return BIE_EINVAL; }
  switch (option) {
    case BIE_OPT_FP64_TRANSFORMS: ctx->fp64_transforms = value ? 1 : 0; return BIE_OK;
    default: bie::set_error("bie_ctx_set_option: unknown option %d", option); return BIE_EINVAL;
  }
}

bie_status bie_ctx_trace(bie_ctx ctx, int enable) {
  if (!ctx) { bie::set_error("bie_ctx_trace: NULL context"); return BIE_EINVAL; }
  ctx->trace = enable ? 1 : 0;
  bie::trace_clear(ctx);
  return BIE_OK;
}

bie_status bie_ctx_trace_read(bie_ctx ctx, double* ms, int* launches) {
  if (!ctx || !ms || !launches) { bie::set_error("bie_ctx_trace_read: invalid arguments"); return BIE_EINVAL; }
  for (int k = 0; k < kTraceKinds; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  if (ctx->marks) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bie::cuda_fail(e, "bie_ctx_trace_read");
    for (const TraceMark& m : *ctx->marks) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, m.e0, m.e1) == cudaSuccess) {
        ms[m.kind] += t;
        launches[m.kind] += 1;
      }
    }
  }
  bie::trace_clear(ctx);
  return BIE_OK;
}


const char* bie_last_error(void) { return bie::g_err; }

bie_status bie_ctx_create(bie_ctx* out, void* cuda_stream) {
  if (!out) {
    bie::set_error("bie_ctx_create: out is NULL");
    return BIE_EINVAL;
  }
  bie_ctx c = new bie_ctx_s();
  c->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { delete c; return bie::cuda_fail(e, "cudaGetDevice"); }
  e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) { delete c; return bie::cuda_fail(e, "cudaDeviceGetAttribute"); }
  e = cudaMalloc(&c->d_status, sizeof(int) * 4);
  if (e != cudaSuccess) { delete c; return bie::cuda_fail(e, "cudaMalloc(status)"); }
  e = cudaMemsetAsync(c->d_status, 0, sizeof(int) * 4, c->stream);
  if (e != cudaSuccess) { cudaFree(c->d_status); delete c; return bie::cuda_fail(e, "cudaMemset(status)"); }
  *out = c;
  return BIE_OK;
}

void bie_ctx_free(bie_ctx ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  bie::trace_clear(ctx);
  delete ctx->marks;
  cudaFree(ctx->pair_scratch);
  cudaFree(ctx->pair_records);
  cudaFree(ctx->band_scratch);
  cudaFree(ctx->d_status);
  delete ctx;
}

bie_status bie_ctx_sync(bie_ctx ctx) {
  if (!ctx) { bie::set_error("bie_ctx_sync: NULL context"); return BIE_EINVAL; }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bie::cuda_fail(e, "cudaStreamSynchronize");
  int st[4];
  e = cudaMemcpy(st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bie::cuda_fail(e, "status readback");
  if (st[0]) {
    bie::set_error("device reported invalid pairs (%d)", st[0]);
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int) * 4, ctx->stream);
    return BIE_EINVAL;
  }
  if (st[1]) {
    bie::set_error("a bounded device wait expired (tensor-core product)");
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int) * 4, ctx->stream);
    return BIE_ETIMEOUT;
  }
  if (st[2]) {
    bie::set_error("O(M) route: %d queries with t == t_s, a non-finite input or a singular banded system", st[2]);
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int) * 4, ctx->stream);
    return BIE_ENAN;
  }
  return BIE_OK;
}

}  // extern "C"
