// runtime.cuh -- context, error reporting, device memory and scratch arenas
// shared by the translation units of libace.so.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ace.h"

namespace ace {

// ---- errors -----------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();
const char* last_error();

#define ACE_TRY_CUDA(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) {                                                        \
            ::ace::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e),   \
                             __FILE__, __LINE__);                                       \
            return ACE_E_CUDA;                                                          \
        }                                                                               \
    } while (0)

#define ACE_TRY(expr)                 \
    do {                              \
        int _rc = (expr);             \
        if (_rc != ACE_OK) return _rc; \
    } while (0)

// ---- device memory -------------------------------------------------------------
// A growable device buffer carved by bump allocation.  take() hands out
// 256-byte-aligned pieces; reset() forgets them (the caller guarantees the
// work using them is complete or ordered on the same stream).
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    void reset() { off = 0; }
    void* take(size_t bytes) {
        size_t a = (off + 255) & ~(size_t)255;
        if (a + bytes > cap) return nullptr;
        off = a + bytes;
        return base + a;
    }
};

// Sizing pass: the same carving sequence run without memory to learn the size.
struct Sizer {
    size_t off = 0;
    void* take(size_t bytes) {
        size_t a = (off + 255) & ~(size_t)255;
        off = a + bytes;
        return (void*)(uintptr_t)1;  // non-null marker, never dereferenced
    }
};

struct NttPlan;  // twiddle tables for one size (ntt.cu)

// A proving slot: the streams, events and scratch one proof needs.  Proofs on
// different slots run concurrently; proofs on the same slot run in order.
// Each slot has its streams at PRIO_LEVELS CUDA stream priorities (level 0
// the highest; in a level the main stream above the auxiliary ones): a proof
// runs on one level's streams, so that a server can let the proofs admitted
// first keep the SMs while later ones fill the gaps.
static const int PROVE_ARENAS = 5;  // QAP + H MSM, A, B1, B2, L
static const int MAX_SLOTS = 16;
static const int PRIO_LEVELS = 3;
struct SlotStreams {
    cudaStream_t main = nullptr;
    cudaStream_t aux[5] = {};
};
struct ProveSlot {
    bool ready = false;
    Arena ar[PROVE_ARENAS];
    SlotStreams lv[PRIO_LEVELS];
    cudaEvent_t ev_in = nullptr, ev_start = nullptr, ev_done = nullptr;
    cudaEvent_t ev_aux[5] = {};
    cudaEvent_t ev_sort = nullptr;  // the B query's entries are sorted (B2 reuses B1's)
    Arena wit;  // staging buffer for witnesses that arrive in host memory
};

}  // namespace ace

struct ace_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;  // 0 = unbounded
    size_t held = 0;    // bytes of device memory held by caches and arenas
    std::mutex mu;
    ace::Arena scratch[4];  // scratch of single calls (MSM, NTT, QAP, batch outputs)
    ace::ProveSlot slots[ace::MAX_SLOTS];
    int batch_slots = 2;  // slots a batch spreads its proofs over
    // a batch's proofs run all their stages on their slot's main stream
    // (proofs overlap across slots only); autotuned with batch_slots
    bool batch_one_stream = false;
    // measurement mode: a proof runs every stage on its main stream in turn
    // (ace_debug_serial_proofs), so per-stage times do not overlap
    bool serial = false;
    // autotuned choices (0 = cost model): MSM window bits by log2(n), NTT
    // shared-memory width by log2(N)
    int tuned_msm_c[32] = {};
    int tuned_ntt_smem[32] = {};
    int tuned_ntt_radix[32] = {};  // 2 or 4 (0 = ntt_default_radix)
    std::map<int, ace::NttPlan*> ntt_plans;
    void* g1_fixed_tab = nullptr;  // fixed-base tables for the generators (setup.cu)
    void* g2_fixed_tab = nullptr;
    // proving keys and servers that use this context; ace_ctx_destroy with
    // users left only marks it, and the last user's release frees it
    int users = 0;
    bool closing = false;
};

namespace ace {
int dev_alloc(ace_ctx* ctx, void** p, size_t bytes);
void dev_free(ace_ctx* ctx, void* p, size_t bytes);
// make arena `slot` hold at least `bytes` (synchronises the device if it grows)
int arena_ensure(ace_ctx* ctx, int slot, size_t bytes);
inline cudaStream_t pick_stream(ace_ctx* ctx, ace_stream s) { return s ? (cudaStream_t)s : ctx->stream; }
// users of a context (proving keys, servers): see ace_ctx::users
void ctx_ref(ace_ctx* ctx);
void ctx_unref(ace_ctx* ctx);
// create the streams and events of proving slot s (once)
int slot_ready(ace_ctx* ctx, int s);
// make arena k of slot s hold at least `bytes` (synchronises the device if it grows)
int slot_arena_ensure(ace_ctx* ctx, int s, int k, size_t bytes);
// make slot s's witness staging buffer hold at least `bytes` (synchronises the
// device if it grows)
int slot_witness_ensure(ace_ctx* ctx, int s, size_t bytes);

// ---- launch counting and kernel timing ----------------------------------------
// Every kernel launch of the library bumps a process-wide counter.  When the
// profiler is on, the hot kernels are bracketed with CUDA events on the
// stream they run on, together with their work count (taken from the device
// when only the device knows it).
void note_launch();
uint64_t launch_count();
// kinds: bucket accumulation (G1, G2), NTT passes, sparse products, MSM
// digit sort (digits, scans, scatter, bucket order), MSM bucket reduction
// (segments, tree, final), proof-assembly scalar multiplications
enum ProfKind {
    PROF_G1_BUCKET = 0,
    PROF_G2_BUCKET = 1,
    PROF_NTT = 2,
    PROF_SPMV = 3,
    PROF_SORT = 4,
    PROF_REDUCE = 5,
    PROF_ASSEMBLY = 6,
    PROF_KINDS = 7
};
bool prof_on();
int prof_begin(int kind, cudaStream_t st);  // returns a record slot, or -1 when off / full
// device_units (optional): a u32 on the device copied into the record;
// host_units is added to it
void prof_end(int slot, cudaStream_t st, const uint32_t* device_units, uint64_t host_units);
void prof_enable(bool on);
// ms: length of the union of the intervals; sum_ms (optional): their total length
int prof_read(int kind, double* ms, uint64_t* launches, uint64_t* units, double* sum_ms = nullptr);
}  // namespace ace
