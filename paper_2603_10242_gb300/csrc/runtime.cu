// runtime.cu -- errors, device memory accounting and scratch arenas.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

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

static int grow(ace_ctx* ctx, Arena& a, size_t bytes) {
    a.reset();
    if (a.cap >= bytes) return ACE_OK;
    // round up to limit regrowth; the device is idle before the old block goes
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

int arena_ensure(ace_ctx* ctx, int slot, size_t bytes) { return grow(ctx, ctx->scratch[slot], bytes); }

int slot_arena_ensure(ace_ctx* ctx, int s, int k, size_t bytes) { return grow(ctx, ctx->slots[s].ar[k], bytes); }

int slot_witness_ensure(ace_ctx* ctx, int s, size_t bytes) { return grow(ctx, ctx->slots[s].wit, bytes); }

int slot_ready(ace_ctx* ctx, int s) {
    ProveSlot& sl = ctx->slots[s];
    if (sl.ready) return ACE_OK;
    int least = 0, greatest = 0;
    ACE_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    // greatest is the numerically lowest (highest) priority.  Within a level
    // the main stream (QAP, then the H MSM: the longest chain of a proof) is
    // one step above the auxiliary streams.
    for (int l = 0; l < PRIO_LEVELS; l++) {
        int pm = greatest + 2 * l, pa = pm + 1;
        if (pm > least) pm = least;
        if (pa > least) pa = least;
        ACE_TRY_CUDA(cudaStreamCreateWithPriority(&sl.lv[l].main, cudaStreamNonBlocking, pm));
        for (auto& a : sl.lv[l].aux) ACE_TRY_CUDA(cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, pa));
    }
    ACE_TRY_CUDA(cudaEventCreateWithFlags(&sl.ev_in, cudaEventDisableTiming));
    ACE_TRY_CUDA(cudaEventCreateWithFlags(&sl.ev_start, cudaEventDisableTiming));
    ACE_TRY_CUDA(cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming));
    for (auto& e : sl.ev_aux) ACE_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ACE_TRY_CUDA(cudaEventCreateWithFlags(&sl.ev_sort, cudaEventDisableTiming));
    sl.ready = true;
    return ACE_OK;
}

// ---------------------------------------------------------------------------
// launch counter and profiler
// ---------------------------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(); }

namespace {
const int PROF_MAX = 8192;
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    uint64_t host_units;
    bool dev_units;
};
struct Profiler {
    std::mutex mu;
    bool on = false;
    int device = -1;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfRec> recs;
    uint32_t* d_units = nullptr;
};
Profiler& prof() {
    static Profiler p;
    return p;
}
}  // namespace

bool prof_on() { return prof().on; }

void prof_enable(bool on) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    cudaDeviceSynchronize();
    p.recs.clear();
    int dev = 0;
    cudaGetDevice(&dev);
    if (on && (p.pool.empty() || p.device != dev)) {
        p.pool.resize(2 * PROF_MAX);
        for (auto& e : p.pool) cudaEventCreate(&e);
        cudaMalloc(&p.d_units, PROF_MAX * sizeof(uint32_t));
        p.device = dev;
    }
    if (p.d_units) cudaMemset(p.d_units, 0, PROF_MAX * sizeof(uint32_t));
    p.on = on;
}

int prof_begin(int kind, cudaStream_t st) {
    Profiler& p = prof();
    if (!p.on) return -1;
    std::lock_guard<std::mutex> g(p.mu);
    int slot = (int)p.recs.size();
    if (slot >= PROF_MAX) return -1;
    ProfRec r{kind, p.pool[2 * slot], p.pool[2 * slot + 1], 0, false};
    p.recs.push_back(r);
    cudaEventRecord(r.a, st);
    return slot;
}

void prof_end(int slot, cudaStream_t st, const uint32_t* device_units, uint64_t host_units) {
    if (slot < 0) return;
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    ProfRec& r = p.recs[slot];
    cudaEventRecord(r.b, st);
    r.host_units = host_units;
    if (device_units) {
        r.dev_units = true;
        cudaMemcpyAsync(p.d_units + slot, device_units, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    }
}

int prof_read(int kind, double* ms, uint64_t* launches, uint64_t* units, double* sum_ms) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    ACE_TRY_CUDA(cudaDeviceSynchronize());
    std::vector<uint32_t> du(p.recs.size());
    if (!p.recs.empty()) ACE_TRY_CUDA(cudaMemcpy(du.data(), p.d_units, du.size() * 4, cudaMemcpyDeviceToHost));
    // time = length of the union of the [start, end] intervals of this kind,
    // on the common GPU clock (launches on several streams may overlap)
    std::vector<std::pair<double, double>> iv;
    uint64_t n = 0, u = 0;
    cudaEvent_t origin = nullptr;
    for (size_t i = 0; i < p.recs.size(); i++) {
        const ProfRec& r = p.recs[i];
        if (r.kind != kind) continue;
        if (!origin) origin = r.a;
        float a = 0, b = 0;
        ACE_TRY_CUDA(cudaEventElapsedTime(&a, origin, r.a));
        ACE_TRY_CUDA(cudaEventElapsedTime(&b, origin, r.b));
        iv.push_back({a, b});
        n++;
        u += r.host_units + (r.dev_units ? du[i] : 0);
    }
    if (sum_ms) {
        double total = 0;
        for (auto& x : iv) total += x.second - x.first;
        *sum_ms = total;
    }
    std::sort(iv.begin(), iv.end());
    double t = 0, cs = 0, ce = -1e300;
    for (auto& x : iv) {
        if (x.first > ce) {
            if (ce > cs) t += ce - cs;
            cs = x.first;
            ce = x.second;
        } else if (x.second > ce) {
            ce = x.second;
        }
    }
    if (!iv.empty() && ce > cs) t += ce - cs;
    *ms = t;
    *launches = n;
    *units = u;
    return ACE_OK;
}

}  // namespace ace
