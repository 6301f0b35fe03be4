// api.cu -- extern "C" entry points of libace.so: context, MSMs, fixed-base
// multiplication and device diagnostics.  Every entry point validates its
// arguments, records a message on failure and returns an ACE_E_* code.
#include <string.h>

#include "fixed_base.cuh"
#include "msm.cuh"
#include "ntt.cuh"

using namespace ace;

namespace {
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <class F>
static int msm_entry(ace_ctx* ctx, const void* d_bases, int base_form, const ace_fr* d_scalars, size_t n,
                     void* d_out, ace_stream stream) {
    clear_error();
    if (!ctx || !d_out || (n && (!d_bases || !d_scalars))) {
        set_error("ace_msm: NULL argument");
        return ACE_E_ARG;
    }
    if (base_form != ACE_FORM_CANONICAL && base_form != ACE_FORM_MONT) {
        set_error("ace_msm: base_form must be ACE_FORM_CANONICAL or ACE_FORM_MONT");
        return ACE_E_ARG;
    }
    if (!aligned16(d_bases) || !aligned16(d_scalars) || !aligned16(d_out)) {
        set_error("ace_msm: device buffers must be 16-byte aligned");
        return ACE_E_ARG;
    }
    if (n >= (1ull << 31)) {
        set_error("ace_msm: n = %zu exceeds 2^31 - 1", n);
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    int lg = 0;
    while (lg < 31 && ((size_t)1 << (lg + 1)) <= n) lg++;
    // G1: scalars split by the GLV endomorphism (half the windows; the 2 n
    // virtual points need n < 2^30), with the autotuned window if any; G2 up
    // to 2^16 points: scalars split four ways by psi, whose 4 n virtual points
    // (32 MB at 2^16) stay in L2 and whose 7 windows of 2^10 buckets cut the
    // reduction and the Horner chain (60 G2 doublings instead of 225);
    // larger G2 MSMs keep full-width scalars (at 2^18 the 128 MB of virtual
    // points made the split 8.0 ms against 6.0), window from the cost model
    MsmPlan plan;
    if (sizeof(F) == sizeof(fp_t) && n < (1ull << 30))
        plan = msm_plan_glv(n, ctx->tuned_msm_c[lg]);
    else if (sizeof(F) == sizeof(fp2_t) && n <= (1ull << 16))
        plan = msm_plan_gls(n);
    else
        plan = msm_plan(n);
    plan.alone = true;
    bool mont = base_form == ACE_FORM_MONT;
    ACE_TRY(arena_ensure(ctx, 0, msm_scratch_bytes<F>(plan, mont)));
    return msm_run<F>(plan, (const Affine<F>*)d_bases, mont, (const uint32_t*)d_scalars, ctx->scratch[0], nullptr,
                      (Affine<F>*)d_out, pick_stream(ctx, stream));
}

template <class F>
static int fixed_entry(ace_ctx* ctx, const ace_fr* d_scalars, size_t n, void* d_out, int out_form,
                       ace_stream stream) {
    clear_error();
    if (!ctx || (n && (!d_scalars || !d_out))) {
        set_error("ace_fixed_base: NULL argument");
        return ACE_E_ARG;
    }
    if (out_form != ACE_FORM_CANONICAL && out_form != ACE_FORM_MONT) {
        set_error("ace_fixed_base: bad out_form");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    return fixed_base_mul<F>(ctx, (const uint32_t*)d_scalars, n, (Affine<F>*)d_out, out_form == ACE_FORM_MONT,
                             pick_stream(ctx, stream));
}

}  // namespace

extern "C" {

const char* ace_last_error(void) { return ace::last_error(); }

int ace_ctx_create(ace_ctx** out, int device, size_t hbm_budget_bytes) {
    clear_error();
    if (!out) {
        set_error("ace_ctx_create: out is NULL");
        return ACE_E_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    ACE_TRY_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("ace_ctx_create: device %d not present (%d devices)", device, ndev);
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(device));
    ace_ctx* c = new ace_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    // a blocking stream: ordered with work the caller put on the legacy default
    // stream (e.g. PyTorch copies), so inputs written there are visible
    cudaError_t e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) {
        set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
        delete c;
        return ACE_E_CUDA;
    }
    *out = c;
    return ACE_OK;
}

}  // extern "C"

namespace {
void ctx_destroy_now(ace_ctx* c) {
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& a : c->scratch) dev_free(c, a.base, a.cap);
    for (auto& sl : c->slots) {
        for (auto& a : sl.ar) dev_free(c, a.base, a.cap);
        dev_free(c, sl.wit.base, sl.wit.cap);
        if (!sl.ready) continue;
        for (auto& lv : sl.lv) {
            cudaStreamDestroy(lv.main);
            for (auto s : lv.aux) cudaStreamDestroy(s);
        }
        cudaEventDestroy(sl.ev_in);
        cudaEventDestroy(sl.ev_start);
        cudaEventDestroy(sl.ev_done);
        for (auto e : sl.ev_aux) cudaEventDestroy(e);
        if (sl.ev_sort) cudaEventDestroy(sl.ev_sort);
    }
    ntt_release_plans(c);
    if (c->g1_fixed_tab) dev_free(c, c->g1_fixed_tab, 32 * 255 * sizeof(g1_aff));
    if (c->g2_fixed_tab) dev_free(c, c->g2_fixed_tab, 32 * 255 * sizeof(g2_aff));
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}
}  // namespace

namespace ace {
void ctx_ref(ace_ctx* ctx) {
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->users++;
}
void ctx_unref(ace_ctx* ctx) {
    bool last;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        last = --ctx->users == 0 && ctx->closing;
    }
    if (last) ctx_destroy_now(ctx);
}
}  // namespace ace

extern "C" {

int ace_ctx_destroy(ace_ctx* c) {
    if (!c) return ACE_OK;
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (c->users > 0) {  // freed by the last key or server released
            c->closing = true;
            return ACE_OK;
        }
    }
    ctx_destroy_now(c);
    return ACE_OK;
}

int ace_ctx_device_bytes(const ace_ctx* c, size_t* out) {
    if (!c || !out) {
        set_error("ace_ctx_device_bytes: NULL argument");
        return ACE_E_ARG;
    }
    *out = c->held;
    return ACE_OK;
}

int ace_msm_g1(ace_ctx* ctx, const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars, size_t n,
               ace_g1_affine* d_out, ace_stream stream) {
    return msm_entry<fp_t>(ctx, d_bases, base_form, d_scalars, n, d_out, stream);
}

int ace_msm_g2(ace_ctx* ctx, const ace_g2_affine* d_bases, int base_form, const ace_fr* d_scalars, size_t n,
               ace_g2_affine* d_out, ace_stream stream) {
    return msm_entry<fp2_t>(ctx, d_bases, base_form, d_scalars, n, d_out, stream);
}

// Diagnostic: same MSM with an explicit window size c (6..20).
int ace_msm_g1_window(ace_ctx* ctx, const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars,
                      size_t n, int c, ace_g1_affine* d_out, ace_stream stream) {
    clear_error();
    if (!ctx || !d_out || (n && (!d_bases || !d_scalars)) || c < 6 || c > 20) {
        set_error("ace_msm_g1_window: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    MsmPlan plan = msm_plan(n, c);
    plan.alone = true;
    bool mont = base_form == ACE_FORM_MONT;
    ACE_TRY(arena_ensure(ctx, 0, msm_scratch_bytes<fp_t>(plan, mont)));
    return msm_run<fp_t>(plan, (const g1_aff*)d_bases, mont, (const uint32_t*)d_scalars, ctx->scratch[0], nullptr,
                         (g1_aff*)d_out, pick_stream(ctx, stream));
}

// Diagnostic: the G1 MSM of ace_msm_g1 (GLV split) with an explicit window
// size c (6..20).
int ace_msm_g1_glv_window(ace_ctx* ctx, const ace_g1_affine* d_bases, int base_form, const ace_fr* d_scalars,
                          size_t n, int c, ace_g1_affine* d_out, ace_stream stream) {
    clear_error();
    if (!ctx || !d_out || (n && (!d_bases || !d_scalars)) || c < 6 || c > 20 || n >= (1ull << 30) ||
        (base_form != ACE_FORM_CANONICAL && base_form != ACE_FORM_MONT)) {
        set_error("ace_msm_g1_glv_window: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    MsmPlan plan = msm_plan_glv(n, c);
    plan.alone = true;
    bool mont = base_form == ACE_FORM_MONT;
    ACE_TRY(arena_ensure(ctx, 0, msm_scratch_bytes<fp_t>(plan, mont)));
    return msm_run<fp_t>(plan, (const g1_aff*)d_bases, mont, (const uint32_t*)d_scalars, ctx->scratch[0], nullptr,
                         (g1_aff*)d_out, pick_stream(ctx, stream));
}

// Diagnostic: the G2 MSM of ace_msm_g2 (psi split) with an explicit window
// size c (6..20).
int ace_msm_g2_gls_window(ace_ctx* ctx, const ace_g2_affine* d_bases, int base_form, const ace_fr* d_scalars,
                          size_t n, int c, ace_g2_affine* d_out, ace_stream stream) {
    clear_error();
    if (!ctx || !d_out || (n && (!d_bases || !d_scalars)) || c < 6 || c > 20 || n >= (1ull << 29) ||
        (base_form != ACE_FORM_CANONICAL && base_form != ACE_FORM_MONT)) {
        set_error("ace_msm_g2_gls_window: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    MsmPlan plan = msm_plan_gls(n, c);
    plan.alone = true;
    bool mont = base_form == ACE_FORM_MONT;
    ACE_TRY(arena_ensure(ctx, 0, msm_scratch_bytes<fp2_t>(plan, mont)));
    return msm_run<fp2_t>(plan, (const g2_aff*)d_bases, mont, (const uint32_t*)d_scalars, ctx->scratch[0], nullptr,
                          (g2_aff*)d_out, pick_stream(ctx, stream));
}

int ace_debug_msm_plan(size_t n, int kind, int force_c, uint32_t out[8]) {
    clear_error();
    if (!out || kind < 0 || kind > 3 || force_c < 0 || (force_c != 0 && (force_c < 6 || force_c > 20))) {
        set_error("ace_debug_msm_plan: bad argument");
        return ACE_E_ARG;
    }
    const MsmPlan p = kind == 0   ? msm_plan(n, force_c)
                      : kind == 1 ? msm_plan_tabled(n, force_c)
                      : kind == 2 ? msm_plan_glv(n, force_c)
                                  : msm_plan_gls(n, force_c);
    out[0] = (uint32_t)p.c;
    out[1] = (uint32_t)p.K;
    out[2] = p.B;
    out[3] = p.windows();
    out[4] = p.L;
    out[5] = p.M;
    out[6] = p.ones_mask() + 1u;
    out[7] = (uint32_t)p.n;
    return ACE_OK;
}

// NTT of N = 2^log_n canonical Fr values in natural order, in place.
// kind: 0 forward (coefficients -> values on H), 1 inverse, 2 coset forward
// (coefficients -> values on g H), 3 coset inverse.
int ace_ntt(ace_ctx* ctx, ace_fr* d_data, uint32_t log_n, int kind, ace_stream stream) {
    clear_error();
    if (!ctx || !d_data || kind < 0 || kind > 3 || log_n < 1 || log_n > 28) {
        set_error("ace_ntt: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    NttPlan* plan = nullptr;
    ACE_TRY(ntt_get_plan(ctx, (int)log_n, &plan));
    size_t n = (size_t)1 << log_n;
    ACE_TRY(arena_ensure(ctx, 0, n * sizeof(fr_t) + 256));
    fr_t* tmp = (fr_t*)ctx->scratch[0].take(n * sizeof(fr_t));
    cudaStream_t st = pick_stream(ctx, stream);
    fr_t* d = (fr_t*)d_data;
    // The transform runs on the canonical values themselves: a Montgomery
    // product of a canonical value by a Montgomery-form factor (a twiddle,
    // g^i, 1/N) is the canonical product, and the butterflies' additions do
    // not depend on the form.  So the passes convert nothing; the first
    // applies the coset factor as it loads (kind 2), the last the output
    // factor (kinds 1, 3) and writes each element to its bit-reversed
    // position, which turns the DIF order back into natural order.
    NttScale pre, post;
    if (kind == 2) {  // g^e
        pre.hi = plan->cg_hi;
        pre.lo = plan->cos_lo;
        pre.h = plan->h;
    }
    if (kind == 1) {  // 1 / N
        post.hi = plan->ninv;
        post.lo = plan->one;
        post.single = 1;
    }
    if (kind == 3) {  // g^-e / N at bit-reversed position
        post.hi = plan->icos_hi;
        post.lo = plan->icos_lo_m;
        post.h = plan->h;
        post.brev = 1;
    }
    const bool inverse = kind == 1 || kind == 3;
    ACE_TRY(ntt_run_io(*plan, d, tmp, d, true, 1, true, inverse, pre, post, st, true));
    return ACE_OK;
}

// Diagnostic: raw in-place passes over `count` arrays of Montgomery-form
// values (dif: natural -> bit-reversed; else bit-reversed -> natural), no
// scaling.  This is the transform the QAP step is built from.
int ace_ntt_mont(ace_ctx* ctx, ace_fr* d_data, uint32_t log_n, int count, int dif, int inverse,
                 ace_stream stream) {
    clear_error();
    if (!ctx || !d_data || count < 1 || log_n < 1 || log_n > 28) {
        set_error("ace_ntt_mont: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    NttPlan* plan = nullptr;
    ACE_TRY(ntt_get_plan(ctx, (int)log_n, &plan));
    NttScale none;
    return ntt_run(*plan, (fr_t*)d_data, count, dif != 0, inverse != 0, none, none, pick_stream(ctx, stream),
                   true);
}

int ace_g1_fixed_base(ace_ctx* ctx, const ace_fr* d_scalars, size_t n, ace_g1_affine* d_out, int out_form,
                      ace_stream stream) {
    return fixed_entry<fp_t>(ctx, d_scalars, n, d_out, out_form, stream);
}
int ace_g2_fixed_base(ace_ctx* ctx, const ace_fr* d_scalars, size_t n, ace_g2_affine* d_out, int out_form,
                      ace_stream stream) {
    return fixed_entry<fp2_t>(ctx, d_scalars, n, d_out, out_form, stream);
}

// ---------------------------------------------------------------------------
// Diagnostics: element-wise field and curve operations on the device, for
// unit-level parity tests of the arithmetic the hot path is built from.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace ace {
ACE_HD fp_t coord_to_mont_any(const fp_t& a) { return fe_to_mont(a); }
ACE_HD fr_t coord_to_mont_any(const fr_t& a) { return fe_to_mont(a); }
ACE_HD fp2_t coord_to_mont_any(const fp2_t& a) { return fe_to_mont(a); }
ACE_HD fp_t coord_from_mont_any(const fp_t& a) { return fe_from_mont(a); }
ACE_HD fr_t coord_from_mont_any(const fr_t& a) { return fe_from_mont(a); }
ACE_HD fp2_t coord_from_mont_any(const fp2_t& a) { return fe_from_mont(a); }
ACE_HD fp_t any_sqr(const fp_t& a) { return fe_sqr(a); }
ACE_HD fr_t any_sqr(const fr_t& a) { return fe_sqr(a); }
ACE_HD fp2_t any_sqr(const fp2_t& a) { return fe_sqr(a); }
ACE_HD fp_t any_inv(const fp_t& a) { return fe_inv(a); }
ACE_HD fr_t any_inv(const fr_t& a) { return fe_inv(a); }
ACE_HD fp2_t any_inv(const fp2_t& a) { return fe_inv(a); }

template <class F>
__global__ void k_field_op(int op, const F* a, const F* b, F* out, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    F x = coord_to_mont_any(a[i]);
    F y = coord_to_mont_any(b[i]);
    F r;
    switch (op) {
        case 0: r = x + y; break;
        case 1: r = x - y; break;
        case 2: r = x * y; break;
        case 3: r = any_sqr(x); break;
        default: r = any_inv(x); break;
    }
    out[i] = coord_from_mont_any(r);
}

// op: 0 P + Q (both as XYZZ), 1 P + Q (Q mixed), 2 2P, 3 k P (k from scal)
template <class F>
__global__ void k_curve_op(int op, const Affine<F>* a, const Affine<F>* b, const uint32_t* scal, Affine<F>* out,
                           size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Affine<F> p = aff_to_mont(a[i]);
    Affine<F> q = aff_to_mont(b[i]);
    Xyzz<F> r;
    switch (op) {
        case 0: r = xyzz_add(xyzz_from_aff(p), xyzz_from_aff(q)); break;
        case 1: r = xyzz_add_aff(xyzz_from_aff(p), q); break;
        case 2: r = xyzz_dbl(xyzz_from_aff(p)); break;
        default: r = xyzz_mul_aff(p, scal + 8 * i); break;
    }
    out[i] = aff_from_mont(xyzz_to_aff(r));
}
}  // namespace ace

extern "C" {

int ace_debug_field_op(int field, int op, const void* d_a, const void* d_b, void* d_out, size_t n,
                       ace_stream stream) {
    clear_error();
    if (field < 0 || field > 2 || op < 0 || op > 4 || (n && (!d_a || !d_b || !d_out))) {
        set_error("ace_debug_field_op: bad argument");
        return ACE_E_ARG;
    }
    if (n == 0) return ACE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned grid = (unsigned)((n + 127) / 128);
    if (field == 0)
        k_field_op<fp_t><<<grid, 128, 0, st>>>(op, (const fp_t*)d_a, (const fp_t*)d_b, (fp_t*)d_out, n);
    else if (field == 1)
        k_field_op<fr_t><<<grid, 128, 0, st>>>(op, (const fr_t*)d_a, (const fr_t*)d_b, (fr_t*)d_out, n);
    else
        k_field_op<fp2_t><<<grid, 128, 0, st>>>(op, (const fp2_t*)d_a, (const fp2_t*)d_b, (fp2_t*)d_out, n);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

int ace_debug_curve_op(int group, int op, const void* d_a, const void* d_b, const ace_fr* d_k, void* d_out,
                       size_t n, ace_stream stream) {
    clear_error();
    if (group < 1 || group > 2 || op < 0 || op > 3 || (n && (!d_a || !d_b || !d_out)) || (op == 3 && !d_k)) {
        set_error("ace_debug_curve_op: bad argument");
        return ACE_E_ARG;
    }
    if (n == 0) return ACE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned grid = (unsigned)((n + 63) / 64);
    if (group == 1)
        k_curve_op<fp_t><<<grid, 64, 0, st>>>(op, (const g1_aff*)d_a, (const g1_aff*)d_b, (const uint32_t*)d_k,
                                              (g1_aff*)d_out, n);
    else
        k_curve_op<fp2_t><<<grid, 64, 0, st>>>(op, (const g2_aff*)d_a, (const g2_aff*)d_b, (const uint32_t*)d_k,
                                               (g2_aff*)d_out, n);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}


// ---------------------------------------------------------------------------
// measurement hooks
// ---------------------------------------------------------------------------
int ace_launch_count(uint64_t* out) {
    if (!out) return ACE_E_ARG;
    *out = launch_count();
    return ACE_OK;
}

int ace_profile_enable(int on) {
    prof_enable(on != 0);
    return ACE_OK;
}

int ace_profile_read(int kind, double* ms, uint64_t* launches, uint64_t* units) {
    clear_error();
    if (kind < 0 || kind >= PROF_KINDS || !ms || !launches || !units) {
        set_error("ace_profile_read: bad argument");
        return ACE_E_ARG;
    }
    return prof_read(kind, ms, launches, units);
}

int ace_debug_serial_proofs(ace_ctx* ctx, int on) {
    clear_error();
    if (!ctx) {
        set_error("ace_debug_serial_proofs: NULL context");
        return ACE_E_ARG;
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->serial = on != 0;
    return ACE_OK;
}

int ace_profile_read_sum(int kind, double* sum_ms) {
    clear_error();
    if (kind < 0 || kind >= PROF_KINDS || !sum_ms) {
        set_error("ace_profile_read_sum: bad argument");
        return ACE_E_ARG;
    }
    double ms = 0;
    uint64_t n = 0, u = 0;
    return prof_read(kind, &ms, &n, &u, sum_ms);
}

}  // extern "C"

namespace ace {
// Independent multiply-add chains: 8 per thread, `iters` rounds, in one of
// four forms: 0 mad.lo.u32, 1 mad.hi.u32, 2 the carry-chained
// mad.lo.cc / madc.hi.cc pairs of the Montgomery product, 3 mad.wide.u32
// (32 x 32 + 64 -> 64 bits, the limb product of the wide form).
__global__ void k_imad_rate(int mode, int iters, uint32_t seed, uint32_t* out) {
    uint32_t a[8], b = seed ^ (threadIdx.x * 2654435761u), c = blockIdx.x + 12345u;
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = seed + k * 7919u + threadIdx.x;
    if (mode == 0) {
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < 8; k++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(b), "r"(c));
    } else if (mode == 1) {
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < 8; k++) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(b), "r"(c));
    } else if (mode == 3) {
        uint64_t w[8];
#pragma unroll
        for (int k = 0; k < 8; k++) w[k] = a[k];
        // the multiplier is the chain's own low word, so no product is loop-invariant
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < 8; k++)
                asm volatile("{\n\t.reg .u32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\tmad.wide.u32 %0, lo, %1, %0;\n\t}"
                             : "+l"(w[k])
                             : "r"(b | 1u));
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = (uint32_t)w[k] ^ (uint32_t)(w[k] >> 32);
    } else {
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < 8; k += 2)
                asm volatile("mad.lo.cc.u32 %0, %0, %2, %3;\n\tmadc.hi.u32 %1, %1, %2, %3;"
                             : "+r"(a[k]), "+r"(a[k + 1])
                             : "r"(b), "r"(c));
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) x ^= a[k];
    if (x == 0x9e3779b9u) out[0] = x;  // keeps the chains live
}
}  // namespace ace

extern "C" {

// Measured 32-bit multiply-add rate (operations per second) of the device:
// mode 0 mad.lo, 1 mad.hi, 2 carry-chained lo/hi pairs, 3 mad.wide.
int ace_debug_imad_rate(ace_ctx* ctx, int mode, double* ops_per_s) {
    clear_error();
    if (!ctx || !ops_per_s || mode < 0 || mode > 3) {
        set_error("ace_debug_imad_rate: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    int sms = 0;
    ACE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    ACE_TRY(arena_ensure(ctx, 0, 4096));
    uint32_t* d = (uint32_t*)ctx->scratch[0].take(16);
    const int threads = 256, iters = 4096;
    const int blocks = sms * 8;
    cudaEvent_t a, b;
    ACE_TRY_CUDA(cudaEventCreate(&a));
    ACE_TRY_CUDA(cudaEventCreate(&b));
    k_imad_rate<<<blocks, threads, 0, ctx->stream>>>(mode, 64, 1u, d);  // warm up
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaEventRecord(a, ctx->stream));
    k_imad_rate<<<blocks, threads, 0, ctx->stream>>>(mode, iters, 1u, d);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaEventRecord(b, ctx->stream));
    ACE_TRY_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    ACE_TRY_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ops_per_s = (double)blocks * threads * iters * 8.0 / (ms * 1e-3);
    return ACE_OK;
}


}  // extern "C"

namespace ace {
// one thread, `iters` dependent Montgomery products (Fp), or dependent G1
// XYZZ additions (what = 1): the latency a sequential chain pays per step
__global__ void k_chain_latency(int what, int iters, fp_t seed, g1_xyzz p0, uint32_t* out) {
    if (what == 0) {
        fp_t x = seed;
        for (int i = 0; i < iters; i++) x = x * x;
        if (x.v[0] == 0x12345678u) out[0] = x.v[1];
    } else {
        g1_xyzz a = p0;
        for (int i = 0; i < iters; i++) a = xyzz_add(a, p0 /* a + p0, a != p0 */);
        if (a.X.v[0] == 0x12345678u) out[0] = a.X.v[1];
    }
}
}  // namespace ace

extern "C" {

// Diagnostic: nanoseconds per step of a single-thread dependent chain of Fp
// Montgomery products (what = 0) or G1 XYZZ additions (what = 1).
int ace_debug_chain_latency(ace_ctx* ctx, int what, double* ns_per_step) {
    clear_error();
    if (!ctx || !ns_per_step || what < 0 || what > 1) {
        set_error("ace_debug_chain_latency: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    ACE_TRY(arena_ensure(ctx, 0, 4096));
    uint32_t* d = (uint32_t*)ctx->scratch[0].take(16);
    fp_t seed = fe_from_u32<FpCfg>(7);
    g1_aff g;
    g.x = fe_from_u32<FpCfg>(1);
    g.y = fe_from_u32<FpCfg>(2);
    g1_xyzz p0 = xyzz_dbl(xyzz_from_aff(g));
    const int iters = 2000;
    cudaEvent_t a, b;
    ACE_TRY_CUDA(cudaEventCreate(&a));
    ACE_TRY_CUDA(cudaEventCreate(&b));
    k_chain_latency<<<1, 1, 0, ctx->stream>>>(what, 10, seed, p0, d);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaEventRecord(a, ctx->stream));
    k_chain_latency<<<1, 1, 0, ctx->stream>>>(what, iters, seed, p0, d);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaEventRecord(b, ctx->stream));
    ACE_TRY_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    ACE_TRY_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ns_per_step = ms * 1e6 / iters;
    return ACE_OK;
}


}  // extern "C"

namespace ace {
// throughput of the two Montgomery product forms: 4 independent chains per
// thread; out[thread] receives a digest so both forms can be compared
template <int V>
__global__ void k_mul_rate(int iters, uint32_t* out) {
#if defined(__CUDA_ARCH__)
    fp_t x[4];
    for (int k = 0; k < 4; k++) {
        x[k] = fe_from_u32<FpCfg>(threadIdx.x + 7u * k + 3u + blockIdx.x);
    }
    fp_t y = fe_from_u32<FpCfg>(blockIdx.x + 11u);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            fp_t r;
            if (V == 0) d_mul<FpCfg>(r.v, x[k].v, y.v);
            else if (V == 1) d_mul_wide<FpCfg>(r.v, x[k].v, y.v);
            else d_mul_pw<FpCfg>(r.v, x[k].v, y.v);
            x[k] = r;
        }
    }
    uint32_t h = 0;
    for (int k = 0; k < 4; k++)
        for (int l = 0; l < 8; l++) h = h * 31u + x[k].v[l];
    out[blockIdx.x * blockDim.x + threadIdx.x] = h;
#endif
}
template <int V>
__global__ void k_mul_latency(int iters, fp_t x, uint32_t* out) {
#if defined(__CUDA_ARCH__)
    for (int i = 0; i < iters; i++) {
        fp_t r;
        if (V == 0) d_mul<FpCfg>(r.v, x.v, x.v);
        else if (V == 1) d_mul_wide<FpCfg>(r.v, x.v, x.v);
        else d_mul_pw<FpCfg>(r.v, x.v, x.v);
        x = r;
    }
    out[0] = x.v[0];
#endif
}
}  // namespace ace

extern "C" {

// Diagnostic: Montgomery products per second (all SMs) and single-thread
// latency (ns) of form 0 (lo/hi multiply-add chains), form 1 (64-bit wide
// multiply-adds) or form 2 (plain wide products, two carry chains per row);
// digest (optional, 4 words) lets callers compare the forms.
int ace_debug_mul_rate(ace_ctx* ctx, int form, double* per_s, double* latency_ns, uint32_t* digest) {
    clear_error();
    if (!ctx || !per_s || !latency_ns || form < 0 || form > 2) {
        set_error("ace_debug_mul_rate: bad argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    int sms = 0;
    ACE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int threads = 256, blocks = sms * 4, iters = 256;
    ACE_TRY(arena_ensure(ctx, 0, (size_t)blocks * threads * 4 + 4096));
    uint32_t* d = (uint32_t*)ctx->scratch[0].take((size_t)blocks * threads * 4);
    cudaEvent_t a, b;
    ACE_TRY_CUDA(cudaEventCreate(&a));
    ACE_TRY_CUDA(cudaEventCreate(&b));
    auto run = [&](int it) {
        if (form == 0) k_mul_rate<0><<<blocks, threads, 0, ctx->stream>>>(it, d);
        else if (form == 1) k_mul_rate<1><<<blocks, threads, 0, ctx->stream>>>(it, d);
        else k_mul_rate<2><<<blocks, threads, 0, ctx->stream>>>(it, d);
        ::ace::note_launch();
    };
    run(4);
    ACE_TRY_CUDA(cudaEventRecord(a, ctx->stream));
    run(iters);
    ACE_TRY_CUDA(cudaEventRecord(b, ctx->stream));
    ACE_TRY_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    ACE_TRY_CUDA(cudaEventElapsedTime(&ms, a, b));
    *per_s = (double)blocks * threads * iters * 4 / (ms * 1e-3);
    if (digest) ACE_TRY_CUDA(cudaMemcpy(digest, d, 16, cudaMemcpyDeviceToHost));
    fp_t x = fe_from_u32<FpCfg>(5);
    const int lit = 4000;
    ACE_TRY_CUDA(cudaEventRecord(a, ctx->stream));
    if (form == 0) k_mul_latency<0><<<1, 1, 0, ctx->stream>>>(lit, x, d);
    else if (form == 1) k_mul_latency<1><<<1, 1, 0, ctx->stream>>>(lit, x, d);
    else k_mul_latency<2><<<1, 1, 0, ctx->stream>>>(lit, x, d);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaEventRecord(b, ctx->stream));
    ACE_TRY_CUDA(cudaEventSynchronize(b));
    ACE_TRY_CUDA(cudaEventElapsedTime(&ms, a, b));
    *latency_ns = ms * 1e6 / lit;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ACE_OK;
}

}  // extern "C"
