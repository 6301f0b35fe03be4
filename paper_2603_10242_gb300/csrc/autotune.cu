// autotune.cu -- measured choice of the tunable sizes on this device:
// the MSM window bits c per problem size, the NTT pass width (elements per
// block in shared memory) per transform size, and the number of proving
// slots a batch spreads its proofs over.  Candidates are timed with CUDA
// events on synthetic inputs; the winners live in the context and can be
// saved to / loaded from a small JSON file keyed by the GPU's name.
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <string>
#include <vector>

#include "fixed_base.cuh"
#include "msm.cuh"
#include "ntt.cuh"
#include "pk.h"

using namespace ace;

namespace {

// pseudo-random canonical scalars (< 2^253) on the device
__global__ void k_fill_scalars(uint32_t* sc, size_t n, uint32_t seed) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t x = seed ^ (uint32_t)(i * 2654435761u);
    for (int k = 0; k < 8; k++) {
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        sc[8 * i + k] = k == 7 ? (x & 0x0fffffffu) : x;
    }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    float ms() {
        cudaEventSynchronize(b);
        float t = 0;
        cudaEventElapsedTime(&t, a, b);
        return t;
    }
};

int gpu_name(ace_ctx* ctx, std::string& out) {
    cudaDeviceProp p;
    ACE_TRY_CUDA(cudaGetDeviceProperties(&p, ctx->device));
    out = p.name;
    return ACE_OK;
}

}  // namespace

extern "C" {

// Time candidate MSM window sizes (G1, the generic entry point) for
// n = 2^log_min .. 2^log_max on synthetic bases and uniform scalars and keep
// the fastest per size.  report (optional): per size, [log_n, best c,
// best ms, cost-model c, cost-model ms].
int ace_autotune_msm(ace_ctx* ctx, uint32_t log_min, uint32_t log_max, double* report) {
    clear_error();
    if (!ctx || log_min < 6 || log_max > 24 || log_min > log_max) {
        set_error("ace_autotune_msm: sizes must satisfy 6 <= log_min <= log_max <= 24");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    size_t nmax = (size_t)1 << log_max;
    void *d_sc = nullptr, *d_b = nullptr, *d_out = nullptr;
    ACE_TRY(dev_alloc(ctx, &d_sc, nmax * 32));
    int rc = dev_alloc(ctx, &d_b, nmax * sizeof(g1_aff));
    if (rc == ACE_OK) rc = dev_alloc(ctx, &d_out, 256);
    cudaStream_t st = ctx->stream;
    if (rc == ACE_OK) {
        k_fill_scalars<<<(unsigned)((nmax + 255) / 256), 256, 0, st>>>((uint32_t*)d_sc, nmax, 0x1234567u);
        ::ace::note_launch();
        rc = fixed_base_mul<fp_t>(ctx, (const uint32_t*)d_sc, nmax, (g1_aff*)d_b, true, st);
        k_fill_scalars<<<(unsigned)((nmax + 255) / 256), 256, 0, st>>>((uint32_t*)d_sc, nmax, 0xabcdefu);
        ::ace::note_launch();
    }
    int row = 0;
    for (uint32_t lg = log_min; lg <= log_max && rc == ACE_OK; lg++, row++) {
        size_t n = (size_t)1 << lg;
        MsmPlan model = msm_plan_glv(n);
        int best_c = model.c;
        float best = 1e30f, model_ms = 0;
        for (int c = model.c - 3; c <= model.c + 2 && rc == ACE_OK; c++) {
            if (c < 6 || c > 20) continue;
            MsmPlan p = msm_plan_glv(n, c);
            p.alone = true;  // as ace_msm_g1 runs it
            rc = arena_ensure(ctx, 0, msm_scratch_bytes<fp_t>(p, true));
            if (rc != ACE_OK) break;
            float t = 1e30f;
            for (int rep = 0; rep < 3 && rc == ACE_OK; rep++) {
                Timer tm;
                cudaEventRecord(tm.a, st);
                ctx->scratch[0].reset();
                rc = msm_run<fp_t>(p, (const g1_aff*)d_b, true, (const uint32_t*)d_sc, ctx->scratch[0], nullptr,
                                   (g1_aff*)d_out, st);
                cudaEventRecord(tm.b, st);
                float x = tm.ms();
                if (rep > 0 && x < t) t = x;  // first run warms up
            }
            if (c == model.c) model_ms = t;
            if (t < best) {
                best = t;
                best_c = c;
            }
        }
        ctx->tuned_msm_c[lg] = best_c;
        if (report) {
            double* r = report + 5 * row;
            r[0] = lg;
            r[1] = best_c;
            r[2] = best;
            r[3] = model.c;
            r[4] = model_ms;
        }
    }
    dev_free(ctx, d_sc, nmax * 32);
    dev_free(ctx, d_b, nmax * sizeof(g1_aff));
    dev_free(ctx, d_out, 256);
    return rc;
}

// Time NTT pass widths (2^10, 2^11, 2^12 elements per block) for
// N = 2^log_min .. 2^log_max on three arrays (the QAP batch shape); report:
// per size [log_n, best width, best ms, ms at 2^11].
int ace_autotune_ntt(ace_ctx* ctx, uint32_t log_min, uint32_t log_max, double* report) {
    clear_error();
    if (!ctx || log_min < 8 || log_max > 24 || log_min > log_max) {
        set_error("ace_autotune_ntt: sizes must satisfy 8 <= log_min <= log_max <= 24");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    size_t nmax = (size_t)3 << log_max;
    void* d = nullptr;
    ACE_TRY(dev_alloc(ctx, &d, nmax * 32));
    cudaStream_t st = ctx->stream;
    k_fill_scalars<<<(unsigned)((nmax + 255) / 256), 256, 0, st>>>((uint32_t*)d, nmax, 99u);
    ::ace::note_launch();
    int rc = ACE_OK, row = 0;
    for (uint32_t lg = log_min; lg <= log_max && rc == ACE_OK; lg++, row++) {
        NttPlan* plan = nullptr;
        rc = ntt_get_plan(ctx, (int)lg, &plan);
        if (rc != ACE_OK) break;
        int best_w = 11, best_r = ntt_default_radix((int)lg);
        float best = 1e30f, t11 = 0;
        for (int radix = 2; radix <= 4 && rc == ACE_OK; radix += 2) {
            for (int w = 10; w <= 12 && rc == ACE_OK; w++) {
                plan->smem_log = w;
                plan->radix = radix;
                NttScale none;
                float t = 1e30f;
                for (int rep = 0; rep < 3 && rc == ACE_OK; rep++) {
                    Timer tm;
                    cudaEventRecord(tm.a, st);
                    rc = ntt_run(*plan, (fr_t*)d, 3, true, false, none, none, st);
                    cudaEventRecord(tm.b, st);
                    float x = tm.ms();
                    if (rep > 0 && x < t) t = x;
                }
                if (w == 11 && radix == ntt_default_radix((int)lg)) t11 = t;
                if (t < best) {
                    best = t;
                    best_w = w;
                    best_r = radix;
                }
            }
        }
        plan->smem_log = best_w;
        plan->radix = best_r;
        ctx->tuned_ntt_smem[lg] = best_w;
        ctx->tuned_ntt_radix[lg] = best_r;
        if (report) {
            double* r = report + 5 * row;
            r[0] = lg;
            r[1] = best_w;
            r[2] = best;
            r[3] = t11;
            r[4] = best_r;
        }
    }
    dev_free(ctx, d, nmax * 32);
    return rc;
}

// Time batches of k proofs of (pk, d_z) spread over 1..max_slots proving
// slots and keep the fastest count; report: [ms per batch for 1..max_slots].
int ace_autotune_batch_slots(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, int k, int max_slots,
                             double* report) {
    clear_error();
    if (!ctx || !pk || !d_z || k < 1 || max_slots < 1 || max_slots > MAX_SLOTS) {
        set_error("ace_autotune_batch_slots: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    std::vector<ace_fr> rs(k), ss(k);
    for (int i = 0; i < k; i++) ACE_TRY(ace_rs_from_seed(777 + i, &rs[i], &ss[i]));
    std::vector<const ace_pk*> pks(k, pk);
    std::vector<const ace_fr*> zs(k, d_z);
    std::vector<uint8_t> proofs(256 * (size_t)k);
    std::vector<int32_t> status(k);
    // ms_of[layout][q]: layout 1 = every stage of a proof on one stream,
    // layout 0 = the MSMs spread over the slot's auxiliary streams
    std::vector<double> ms_of[2] = {std::vector<double>(max_slots + 1, 1e30),
                                    std::vector<double>(max_slots + 1, 1e30)};
    double best_ms = 1e30;
    for (int layout = 0; layout < 2; layout++) {
        ctx->batch_one_stream = layout == 1;
        for (int q = 1; q <= max_slots; q++) {
            ctx->batch_slots = q;
            ACE_TRY(prove_batch_on_slots(ctx, k, pks.data(), zs.data(), rs.data(), ss.data(), proofs.data(),
                                    status.data()));
            // the faster of two timed batches (one alone varied by about 1%)
            double ms = 1e30;
            for (int rep = 0; rep < 2; rep++) {
                auto t0 = std::chrono::steady_clock::now();
                ACE_TRY(prove_batch_on_slots(ctx, k, pks.data(), zs.data(), rs.data(), ss.data(), proofs.data(),
                                        status.data()));
                const double t =
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (t < ms) ms = t;
            }
            if (report) report[layout * max_slots + q - 1] = ms;
            ms_of[layout][q] = ms;
            if (ms < best_ms) best_ms = ms;
        }
    }
    // among the configurations within 1% of the fastest: one stream per proof
    // first (its kernels share the SMs with fewer others, at the same
    // throughput), then the fewest slots (each holds a proof's scratch).  A
    // 2% band let 2 slots win at 2^20 block proofs, 2% slower than 3 in the
    // timed batch.
    int best_layout = 0, best = max_slots;
    for (int layout = 1, found = 0; layout >= 0 && !found; layout--)
        for (int q = 1; q <= max_slots && !found; q++)
            if (ms_of[layout][q] <= 1.01 * best_ms) {
                best_layout = layout;
                best = q;
                found = 1;
            }
    ctx->batch_one_stream = best_layout == 1;
    ctx->batch_slots = best;
    return ACE_OK;
}

// The tuned choices as JSON: {"gpu": name, "batch_slots": q, "msm_c":
// {"log_n": c, ...}, "ntt_smem_log": {"log_n": w, ...}}
int ace_autotune_save(ace_ctx* ctx, const char* path) {
    clear_error();
    if (!ctx || !path) return ACE_E_ARG;
    std::string name;
    ACE_TRY(gpu_name(ctx, name));
    FILE* f = fopen(path, "w");
    if (!f) {
        set_error("ace_autotune_save: cannot open %s", path);
        return ACE_E_ARG;
    }
    fprintf(f, "{\"gpu\": \"%s\", \"batch_slots\": %d, \"batch_one_stream\": %d, \"msm_c\": {", name.c_str(),
            ctx->batch_slots, ctx->batch_one_stream ? 1 : 0);
    bool first = true;
    for (int i = 0; i < 32; i++)
        if (ctx->tuned_msm_c[i]) {
            fprintf(f, "%s\"%d\": %d", first ? "" : ", ", i, ctx->tuned_msm_c[i]);
            first = false;
        }
    fprintf(f, "}, \"ntt_smem_log\": {");
    first = true;
    for (int i = 0; i < 32; i++)
        if (ctx->tuned_ntt_smem[i]) {
            fprintf(f, "%s\"%d\": %d", first ? "" : ", ", i, ctx->tuned_ntt_smem[i]);
            first = false;
        }
    fprintf(f, "}, \"ntt_radix\": {");
    first = true;
    for (int i = 0; i < 32; i++)
        if (ctx->tuned_ntt_radix[i]) {
            fprintf(f, "%s\"%d\": %d", first ? "" : ", ", i, ctx->tuned_ntt_radix[i]);
            first = false;
        }
    fprintf(f, "}}\n");
    if (fclose(f) != 0) return ACE_E_ARG;
    return ACE_OK;
}

// Load choices saved by ace_autotune_save; ACE_E_ARG if the file is for a
// different GPU or malformed (the context is then unchanged).
int ace_autotune_load(ace_ctx* ctx, const char* path) {
    clear_error();
    if (!ctx || !path) return ACE_E_ARG;
    FILE* f = fopen(path, "r");
    if (!f) {
        set_error("ace_autotune_load: cannot open %s", path);
        return ACE_E_ARG;
    }
    std::string txt;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, k);
    fclose(f);
    std::string name;
    ACE_TRY(gpu_name(ctx, name));
    std::string want = "\"gpu\": \"" + name + "\"";
    if (txt.find(want) == std::string::npos) {
        set_error("ace_autotune_load: %s was tuned on another GPU", path);
        return ACE_E_ARG;
    }
    int msm[32] = {}, ntt[32] = {}, slots = 0;
    auto parse_map = [&](const char* key, int* out) -> bool {
        size_t p = txt.find(key);
        if (p == std::string::npos) return false;
        p = txt.find('{', p);
        size_t e = txt.find('}', p);
        if (p == std::string::npos || e == std::string::npos) return false;
        std::string body = txt.substr(p + 1, e - p - 1);
        size_t q = 0;
        while ((q = body.find('"', q)) != std::string::npos) {
            int a = 0, b = 0;
            if (sscanf(body.c_str() + q, "\"%d\": %d", &a, &b) != 2 || a < 0 || a >= 32) return false;
            out[a] = b;
            q = body.find(',', q);
            if (q == std::string::npos) break;
        }
        return true;
    };
    size_t ps = txt.find("\"batch_slots\":");
    if (ps == std::string::npos || sscanf(txt.c_str() + ps, "\"batch_slots\": %d", &slots) != 1 || slots < 1 ||
        slots > MAX_SLOTS || !parse_map("\"msm_c\"", msm) || !parse_map("\"ntt_smem_log\"", ntt)) {
        set_error("ace_autotune_load: %s is malformed", path);
        return ACE_E_ARG;
    }
    // the stage form per size (absent from files saved before it was tuned)
    int radix[32] = {};
    if (txt.find("\"ntt_radix\"") != std::string::npos && !parse_map("\"ntt_radix\"", radix)) {
        set_error("ace_autotune_load: %s is malformed", path);
        return ACE_E_ARG;
    }
    for (int i = 0; i < 32; i++)
        if ((msm[i] && (msm[i] < 6 || msm[i] > 20)) || (ntt[i] && (ntt[i] < 10 || ntt[i] > 12)) ||
            (radix[i] && radix[i] != 2 && radix[i] != 4)) {
            set_error("ace_autotune_load: %s holds out-of-range values", path);
            return ACE_E_ARG;
        }
    int one_stream = 0;  // absent from files saved before the layout was tuned
    size_t po = txt.find("\"batch_one_stream\":");
    if (po != std::string::npos &&
        (sscanf(txt.c_str() + po, "\"batch_one_stream\": %d", &one_stream) != 1 || one_stream < 0 || one_stream > 1)) {
        set_error("ace_autotune_load: %s is malformed", path);
        return ACE_E_ARG;
    }
    ctx->batch_slots = slots;
    ctx->batch_one_stream = one_stream == 1;
    memcpy(ctx->tuned_msm_c, msm, sizeof msm);
    memcpy(ctx->tuned_ntt_smem, ntt, sizeof ntt);
    memcpy(ctx->tuned_ntt_radix, radix, sizeof radix);
    for (auto& kv : ctx->ntt_plans) {
        if (ctx->tuned_ntt_smem[kv.first]) kv.second->smem_log = ctx->tuned_ntt_smem[kv.first];
        kv.second->radix = radix[kv.first] ? radix[kv.first] : ntt_default_radix(kv.first);
    }
    return ACE_OK;
}

}  // extern "C"
