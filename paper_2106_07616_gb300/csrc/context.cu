// context.cu -- context lifetime, error text, budgeted allocation.
#include <cstring>

#include "abi_guard.cuh"
#include "common.cuh"

namespace rbffd {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = 0; }

bool dev_reserve(rbffd_ctx *ctx, size_t bytes) {
  size_t cur = ctx->used.load();
  do {
    if (ctx->budget && cur + bytes > ctx->budget) {
      set_error("device budget exceeded: %zu + %zu > %zu bytes", cur, bytes, ctx->budget);
      return false;
    }
  } while (!ctx->used.compare_exchange_weak(cur, cur + bytes));
  return true;
}

void dev_release(rbffd_ctx *ctx, size_t bytes) { ctx->used.fetch_sub(bytes); }

int dev_alloc(rbffd_ctx *ctx, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return RBFFD_OK;
  if (!dev_reserve(ctx, bytes)) return RBFFD_ENOMEM;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    dev_release(ctx, bytes);
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return RBFFD_ENOMEM;
  }
  return RBFFD_OK;
}

void dev_free(rbffd_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  dev_release(ctx, bytes);
}

int pinned(rbffd_ctx *ctx, size_t bytes, void **out) {
  if (ctx->pinned_bytes < bytes) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    RBFFD_CK(cudaMallocHost(&ctx->pinned, bytes));
    ctx->pinned_bytes = bytes;
  }
  *out = ctx->pinned;
  return RBFFD_OK;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" const char *rbffd_last_error(void) { return g_err; }

extern "C" int rbffd_ctx_create(rbffd_ctx **out, int device, size_t hbm_budget_bytes,
                                void *cuda_stream) {
  return guarded([&]() -> int {
    if (!out) return RBFFD_EINVAL;
    *out = nullptr;
    int ndev = 0;
    RBFFD_CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
      set_error("device %d out of range (%d devices)", device, ndev);
      return RBFFD_EINVAL;
    }
    RBFFD_CK(cudaSetDevice(device));
    rbffd_ctx *c = new rbffd_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
      delete c;
      set_error("cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
      return RBFFD_ECUDA;
    }
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        delete c;
        set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
        return RBFFD_ECUDA;
      }
      c->own_stream = true;
    }
    *out = c;
    return RBFFD_OK;
  });
}

static void ctx_free(rbffd_ctx *ctx) {
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (int k = 0; k < 8; ++k)
    if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
  delete ctx;
}

namespace rbffd {
void ctx_ref(rbffd_ctx *ctx) { ctx->refs++; }
void ctx_unref(rbffd_ctx *ctx) {
  if (--ctx->refs == 0 && ctx->closing) ctx_free(ctx);
}
}  // namespace rbffd

extern "C" void rbffd_ctx_destroy(rbffd_ctx *ctx) {
  if (!ctx) return;
  ctx->closing = true;
  if (ctx->refs == 0) ctx_free(ctx);
}

namespace rbffd {

__global__ void k_reset_barriers(GridBarrier *bars, int m, int wait_log2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  bars[i].count = 0;
  bars[i].gen = 0;
  bars[i].err = 0;
  bars[i].wait_log2 = wait_log2;
}

int reset_barriers(rbffd_ctx *ctx, GridBarrier *bars, int m) {
  if (m < 1) return RBFFD_OK;
  k_reset_barriers<<<(m + 127) / 128, 128, 0, ctx->stream>>>(bars, m, ctx->wait_log2);
  return after_launch(ctx, "k_reset_barriers");
}

}  // namespace rbffd

extern "C" int rbffd_ctx_set_wait_limit(rbffd_ctx *ctx, int32_t log2_cycles) {
  return guarded([&]() -> int {
    if (!ctx || log2_cycles < 0 || log2_cycles > 40) {
      set_error("rbffd_ctx_set_wait_limit: log2_cycles must be 0 (default) or 1..40");
      return RBFFD_EINVAL;
    }
    ctx->wait_log2 = log2_cycles;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_ctx_set_amg_compose(rbffd_ctx *ctx, int on) {
  return guarded([&]() -> int {
    if (!ctx) return RBFFD_EINVAL;
    ctx->amg_compose = on != 0;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_ctx_set_fgmres_reorth(rbffd_ctx *ctx, int mode) {
  return guarded([&]() -> int {
    if (!ctx || mode < 0 || mode > 2) {
      set_error("rbffd_ctx_set_fgmres_reorth: mode must be 0, 1 or 2");
      return RBFFD_EINVAL;
    }
    ctx->fgmres_reorth = mode;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_ctx_set_amg_device_setup(rbffd_ctx *ctx, int on) {
  return guarded([&]() -> int {
    if (!ctx) return RBFFD_EINVAL;
    ctx->amg_device_setup = on != 0;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_ctx_profile(rbffd_ctx *ctx, int enable) {
  return guarded([&]() -> int {
    if (!ctx) return RBFFD_EINVAL;
    RBFFD_CK(cudaSetDevice(ctx->device));
    if (enable && !ctx->ev[0]) {
      for (int k = 0; k < 8; ++k) RBFFD_CK(cudaEventCreate(&ctx->ev[k]));
    }
    memset(ctx->kst, 0, sizeof(ctx->kst));
    ctx->prof = enable != 0;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_ctx_kernel_stat(const rbffd_ctx *ctx, int32_t which, rbffd_kernel_stat *out) {
  return guarded([&]() -> int {
    if (!ctx || !out || which < 0 || which >= RBFFD_KSTAT_COUNT) return RBFFD_EINVAL;
    *out = ctx->kst[which];
    return RBFFD_OK;
  });
}

extern "C" int64_t rbffd_ctx_launch_count(const rbffd_ctx *ctx) { return ctx ? ctx->launches : 0; }
