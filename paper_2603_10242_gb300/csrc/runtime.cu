// runtime.cu -- errors, device memory accounting and scratch arenas.
#include <stdarg.h>
#include <stdio.h>

#include "runtime.cuh"

namespace ace {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }
const char* last_error() { return g_err; }

int dev_alloc(ace_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return ACE_OK;
    if (ctx->budget && ctx->held + bytes > ctx->budget) {
        set_error("device budget exceeded: holding %zu, need %zu more, budget %zu", ctx->held, bytes, ctx->budget);
        return ACE_E_OOM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return ACE_E_OOM;
    }
    ctx->held += bytes;
    return ACE_OK;
}

void dev_free(ace_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    ctx->held -= bytes;
}

int arena_ensure(ace_ctx* ctx, int slot, size_t bytes) {
    Arena& a = ctx->scratch[slot];
    a.reset();
    if (a.cap >= bytes) return ACE_OK;
    // round up to limit regrowth
    size_t want = bytes + bytes / 8 + (1u << 20);
    ACE_TRY_CUDA(cudaDeviceSynchronize());
    dev_free(ctx, a.base, a.cap);
    a.base = nullptr;
    a.cap = 0;
    void* p = nullptr;
    ACE_TRY(dev_alloc(ctx, &p, want));
    a.base = (char*)p;
    a.cap = want;
    return ACE_OK;
}

int ctx_aux_streams(ace_ctx* ctx) {
    if (ctx->aux[0]) return ACE_OK;
    for (int i = 0; i < 8; i++) ACE_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking));
    for (int i = 0; i < 16; i++) ACE_TRY_CUDA(cudaEventCreateWithFlags(&ctx->ev[i], cudaEventDisableTiming));
    return ACE_OK;
}

}  // namespace ace
