// ntt.cu -- radix-2 NTT passes over Fr staged in shared memory (see ntt.cuh).
#include <cmath>
#include <vector>

#include "ntt.cuh"

namespace ace {

// ---------------------------------------------------------------------------
// host-side power tables
// ---------------------------------------------------------------------------
static fr_t h_pow_u64(const fr_t& a, uint64_t e) {
    uint32_t ex[8] = {(uint32_t)e, (uint32_t)(e >> 32), 0, 0, 0, 0, 0, 0};
    return fe_pow(a, ex);
}

// omega_N = 5^((r - 1) / N)
fr_t root_of_unity_host(int log_n) {
    uint32_t e[8];
    for (int i = 0; i < 8; i++) e[i] = mod_limb<FrCfg>(i);
    e[0] -= 1;  // r - 1 (r is odd: no borrow)
    for (int k = 0; k < log_n; k++) {
        for (int i = 0; i < 8; i++) e[i] = (e[i] >> 1) | (i < 7 ? (e[i + 1] << 31) : 0u);
    }
    return fe_pow(fe_from_u32<FrCfg>(5), e);
}

__global__ void k_expand_pow(const fr_t* hi, const fr_t* lo, int a, size_t n, fr_t* out) {
    size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    out[j] = hi[j >> a] * lo[j & ((1ull << a) - 1)];
}

static void h_powers(std::vector<fr_t>& out, const fr_t& base, const fr_t& first, size_t count) {
    out.resize(count);
    fr_t x = first;
    for (size_t i = 0; i < count; i++) {
        out[i] = x;
        x = x * base;
    }
}

int ntt_get_plan(ace_ctx* ctx, int log_n, NttPlan** out) {
    auto it = ctx->ntt_plans.find(log_n);
    if (it != ctx->ntt_plans.end()) {
        *out = it->second;
        return ACE_OK;
    }
    if (log_n < 1 || log_n > 28) {
        set_error("ntt: log_n = %d out of range [1, 28]", log_n);
        return ACE_E_ARG;
    }
    const size_t n = (size_t)1 << log_n;
    const size_t half = n / 2;
    const int h = (log_n + 1) / 2;
    const size_t nlo = (size_t)1 << h, nhi = (size_t)1 << (log_n - h);
    // twiddle seeds: tw[j] = T_hi[j >> a] * T_lo[j & (2^a - 1)], j < N/2
    const int a = log_n > 1 ? log_n / 2 : 0;
    const size_t tlo = (size_t)1 << a, thi = (half + tlo - 1) / tlo;

    fr_t omega = root_of_unity_host(log_n);
    fr_t omega_inv = fe_inv(omega);
    fr_t one = fe_one<FrCfg>();
    fr_t g = fe_from_u32<FrCfg>(5), ginv = fe_inv(g);
    fr_t ninv = fe_inv(fe_from_u32<FrCfg>(1) * h_pow_u64(fe_from_u32<FrCfg>(2), (uint64_t)log_n));
    fr_t gn = h_pow_u64(g, (uint64_t)n);
    fr_t zinv = fe_inv(gn - one);

    std::vector<fr_t> fw_lo, fw_hi, iw_lo, iw_hi;
    h_powers(fw_lo, omega, one, tlo);
    h_powers(fw_hi, h_pow_u64(omega, tlo), one, thi);
    h_powers(iw_lo, omega_inv, one, tlo);
    h_powers(iw_hi, h_pow_u64(omega_inv, tlo), one, thi);
    std::vector<fr_t> cos_lo, cg_hi, cos_hi, icos_lo_m, icos_lo, icos_hi;
    h_powers(cos_lo, g, one, nlo);
    h_powers(cg_hi, h_pow_u64(g, nlo), one, nhi);
    h_powers(cos_hi, h_pow_u64(g, nlo), ninv, nhi);
    h_powers(icos_lo_m, ginv, one, nlo);
    icos_lo.resize(nlo);
    for (size_t i = 0; i < nlo; i++) icos_lo[i] = fe_from_mont(icos_lo_m[i]);
    h_powers(icos_hi, h_pow_u64(ginv, nlo), ninv, nhi);
    fr_t plain1 = fe_zero<FrCfg>();
    plain1.v[0] = 1;
    fr_t rr = fe_rr<FrCfg>();

    // layout
    size_t off = 0;
    auto place = [&](size_t count) {
        size_t o = off;
        off += ((count * sizeof(fr_t)) + 255) & ~(size_t)255;
        return o;
    };
    size_t o_twf = place(half), o_twi = place(half), o_cos_hi = place(nhi), o_cos_lo = place(nlo),
           o_cg_hi = place(nhi), o_icos_lo_m = place(nlo), o_icos_hi = place(nhi), o_icos_lo = place(nlo), o_ninv = place(1),
           o_one = place(1), o_p1 = place(1), o_rr = place(1), o_seed = place(4 * (tlo + thi));
    void* mem = nullptr;
    ACE_TRY(dev_alloc(ctx, &mem, off));
    char* base = (char*)mem;
    NttPlan* p = new NttPlan();
    p->log_n = log_n;
    p->n = n;
    p->h = h;
    p->tw_fwd = (fr_t*)(base + o_twf);
    p->tw_inv = (fr_t*)(base + o_twi);
    p->cos_hi = (fr_t*)(base + o_cos_hi);
    p->cos_lo = (fr_t*)(base + o_cos_lo);
    p->cg_hi = (fr_t*)(base + o_cg_hi);
    p->icos_lo_m = (fr_t*)(base + o_icos_lo_m);
    p->icos_hi = (fr_t*)(base + o_icos_hi);
    p->icos_lo = (fr_t*)(base + o_icos_lo);
    p->ninv = (fr_t*)(base + o_ninv);
    p->one = (fr_t*)(base + o_one);
    p->plain_one = (fr_t*)(base + o_p1);
    p->rr = (fr_t*)(base + o_rr);
    p->zinv = zinv;
    p->mem = mem;
    p->bytes = off;
    fr_t* seed = (fr_t*)(base + o_seed);
    cudaStream_t st = ctx->stream;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    cudaError_t e = cudaSuccess;
    e = e ? e : up(seed, fw_lo.data(), tlo * sizeof(fr_t));
    e = e ? e : up(seed + tlo, fw_hi.data(), thi * sizeof(fr_t));
    e = e ? e : up(seed + tlo + thi, iw_lo.data(), tlo * sizeof(fr_t));
    e = e ? e : up(seed + 2 * tlo + thi, iw_hi.data(), thi * sizeof(fr_t));
    e = e ? e : up(p->cos_hi, cos_hi.data(), nhi * sizeof(fr_t));
    e = e ? e : up(p->cos_lo, cos_lo.data(), nlo * sizeof(fr_t));
    e = e ? e : up(p->cg_hi, cg_hi.data(), nhi * sizeof(fr_t));
    e = e ? e : up(p->icos_lo_m, icos_lo_m.data(), nlo * sizeof(fr_t));
    e = e ? e : up(p->icos_hi, icos_hi.data(), nhi * sizeof(fr_t));
    e = e ? e : up(p->icos_lo, icos_lo.data(), nlo * sizeof(fr_t));
    e = e ? e : up(p->ninv, &ninv, sizeof(fr_t));
    e = e ? e : up(p->one, &one, sizeof(fr_t));
    e = e ? e : up(p->plain_one, &plain1, sizeof(fr_t));
    e = e ? e : up(p->rr, &rr, sizeof(fr_t));
    if (e == cudaSuccess && half > 0) {
        unsigned grid = (unsigned)((half + 255) / 256);
        k_expand_pow<<<grid, 256, 0, st>>>(seed + tlo, seed, a, half, p->tw_fwd); ::ace::note_launch();
        k_expand_pow<<<grid, 256, 0, st>>>(seed + 2 * tlo + thi, seed + tlo + thi, a, half, p->tw_inv); ::ace::note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
    if (e != cudaSuccess) {
        set_error("ntt plan: %s", cudaGetErrorString(e));
        dev_free(ctx, mem, off);
        delete p;
        return ACE_E_CUDA;
    }
    if (ctx->tuned_ntt_smem[log_n]) p->smem_log = ctx->tuned_ntt_smem[log_n];
    p->radix = ctx->tuned_ntt_radix[log_n] ? ctx->tuned_ntt_radix[log_n] : ntt_default_radix(log_n);
    ctx->ntt_plans[log_n] = p;
    *out = p;
    return ACE_OK;
}

void ntt_release_plans(ace_ctx* ctx) {
    for (auto& kv : ctx->ntt_plans) {
        dev_free(ctx, kv.second->mem, kv.second->bytes);
        delete kv.second;
    }
    ctx->ntt_plans.clear();
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ fr_t ld_fr(const fr_t* p) {
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4 a = s[0], b = s[1];
    fr_t r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
    r.v[4] = b.x; r.v[5] = b.y; r.v[6] = b.z; r.v[7] = b.w;
    return r;
}
__device__ __forceinline__ void st_fr(fr_t* p, const fr_t& x) {
    uint4* d = reinterpret_cast<uint4*>(p);
    d[0] = make_uint4(x.v[0], x.v[1], x.v[2], x.v[3]);
    d[1] = make_uint4(x.v[4], x.v[5], x.v[6], x.v[7]);
}
__device__ __forceinline__ uint32_t brev_bits(uint32_t x, int bits) { return bits ? (__brev(x) >> (32 - bits)) : 0u; }

__device__ __forceinline__ fr_t scale_factor(const NttScale& s, uint32_t idx, int log_n) {
    if (s.single) return ld_fr(s.hi) * ld_fr(s.lo);
    uint32_t e = s.brev ? brev_bits(idx, log_n) : idx;
    return ld_fr(s.hi + (e >> s.h)) * ld_fr(s.lo + (e & ((1u << s.h) - 1u)));
}

// Shared-memory word of element e in one limb plane: e with its 5-bit column
// XORed by a function of its row (e >> 5).  A warp's lanes enumerate five
// index bits of the group; the stage's butterfly bits are skipped, so up to
// two of the column bits come from the row instead.  Row bit 0 is spread over
// every column bit and row bit 1 over columns 0, 2 and 4: for a radix-2
// stage (one missing column bit p < 5, row bit 0 supplying it) and for the
// radix-4 pairs (missing bits p, p + 1, supplied by row bits 0 and 1) the
// lanes then hit 32 distinct banks; contiguous runs stay a permutation of one
// row.
__device__ __forceinline__ uint32_t swz(uint32_t e) {
    const uint32_t r = e >> 5;
    return e ^ ((r & 1u) * 31u) ^ (((r >> 1) & 1u) * 21u);
}
__device__ __forceinline__ fr_t sm_ld(const uint32_t* sm, uint32_t S, uint32_t e) {
    const uint32_t w = swz(e);
    fr_t x;
#pragma unroll
    for (int l = 0; l < 8; l++) x.v[l] = sm[l * S + w];
    return x;
}
__device__ __forceinline__ void sm_st(uint32_t* sm, uint32_t S, uint32_t e, const fr_t& x) {
    const uint32_t w = swz(e);
#pragma unroll
    for (int l = 0; l < 8; l++) sm[l * S + w] = x.v[l];
}
// (x, y) -> (x + y, x - y)
__device__ __forceinline__ void bfly(fr_t& x, fr_t& y) {
    fr_t u = x + y;
    y = x - y;
    x = u;
}
// group index g with a zero bit inserted at position p
__device__ __forceinline__ uint32_t ins0(uint32_t g, int p) { return ((g >> p) << (p + 1)) | (g & ((1u << p) - 1u)); }

// One pass: t stages of radix-2 butterflies on 2^logG columns x 2^t rows
// staged in shared memory.  Stages are taken two at a time (a radix-4 unit:
// the four elements that two consecutive stages connect stay in registers
// between them, halving the shared-memory round trips and barriers); an odd
// t starts with one radix-2 stage.  Each butterfly is the radix-2 one of the
// stage it belongs to, with the same twiddle, so the output is the same as
// t radix-2 stages.  DIT: stage bits ascending, y *= w before (x + y, x - y);
// DIF: bits descending, (x + y, (x - y) w).  R4 = false: radix-2 stages only
// (fewer registers; the plan picks the form per size, see ntt_default_radix).
// ACE_NTT_MIN_BLOCKS: resident blocks of 256 threads per SM the register
// allocation must allow.
// ACE_NTT_THREADS: threads per block (fewer when a block holds fewer than
// twice as many elements).
#ifndef ACE_NTT_MIN_BLOCKS
#define ACE_NTT_MIN_BLOCKS 3
#endif
#ifndef ACE_NTT_THREADS
#define ACE_NTT_THREADS 256
#endif
// src / dst: the pass reads its groups from src and writes them to dst (the
// same array for an in-place pass; a block reads all of its elements before
// it writes any).  out_brev: element p is written to position bitrev(p) of
// dst, which must then be a different array unless one block holds a whole
// array (the pass is the transform's only one).
template <bool DIT, bool R4>
__global__ void __launch_bounds__(ACE_NTT_THREADS, ACE_NTT_MIN_BLOCKS) k_ntt_pass(const fr_t* src, fr_t* dst, int out_brev,
                                                  int log_n, int t, int b0, int logG,
                                                  const fr_t* __restrict__ tw, int first_stage, NttScale pre,
                                                  NttScale post) {
    extern __shared__ uint32_t sm[];
    const uint32_t G = 1u << logG;
    const uint32_t S = G << t;
    const fr_t* in = src + ((size_t)blockIdx.y << log_n);
    fr_t* out = dst + ((size_t)blockIdx.y << log_n);
    const uint32_t q0 = blockIdx.x * G;
    const uint32_t lomask = (1u << b0) - 1u;

    {
        fr_t c;
        if (pre.single) c = ld_fr(pre.hi) * ld_fr(pre.lo);
        for (uint32_t e = threadIdx.x; e < S; e += blockDim.x) {
            uint32_t g = e >> logG, ql = e & (G - 1u);
            uint32_t q = q0 + ql;
            uint32_t idx = ((q >> b0) << (b0 + t)) | (g << b0) | (q & lomask);
            fr_t x = ld_fr(in + idx);
            if (pre.hi) x = x * (pre.single ? c : scale_factor(pre, idx, log_n));
            sm_st(sm, S, e, x);
        }
    }
    __syncthreads();
    int ls = 0;
    // radix-2 stages until the rest pairs up (all of them without ACE_NTT_RADIX4)
    const int r2 = R4 ? (t & 1) : t;
    for (; ls < r2; ls++) {
        const int hb = DIT ? ls : t - 1 - ls;
        const int s_ = first_stage + ls;
        const int tshift = DIT ? (log_n - s_ - 1) : s_;
        for (uint32_t beta = threadIdx.x; beta < S / 2; beta += blockDim.x) {
            uint32_t ql = beta & (G - 1u), pi = beta >> logG;
            uint32_t lowbits = pi & ((1u << hb) - 1u);
            uint32_t et = (ins0(pi, hb) << logG) + ql, eb = et + ((1u << hb) << logG);
            fr_t x = sm_ld(sm, S, et), y = sm_ld(sm, S, eb);
            uint32_t j = (lowbits << b0) | ((q0 + ql) & lomask);
            if (DIT) {
                if (j) y = y * ld_fr(tw + ((size_t)j << tshift));
                bfly(x, y);
            } else {
                bfly(x, y);
                if (j) y = y * ld_fr(tw + ((size_t)j << tshift));
            }
            sm_st(sm, S, et, x);
            sm_st(sm, S, eb, y);
        }
        __syncthreads();
    }
    for (; R4 && ls < t; ls += 2) {
        // stages ls (first) and ls + 1 act on group bits lo and lo + 1
        const int lo = DIT ? ls : t - 2 - ls;
        const int sA = first_stage + ls, sB = sA + 1;
        const int tshA = DIT ? (log_n - sA - 1) : sA;
        const int tshB = DIT ? (log_n - sB - 1) : sB;
        const uint32_t dLo = (1u << lo) << logG, dHi = dLo << 1;
        for (uint32_t u = threadIdx.x; u < S / 4; u += blockDim.x) {
            const uint32_t ql = u & (G - 1u), p4 = u >> logG;
            const uint32_t g = ins0(ins0(p4, lo), lo + 1);
            const uint32_t e = (g << logG) + ql;
            const uint32_t col = (q0 + ql) & lomask;
            fr_t x00 = sm_ld(sm, S, e), x01 = sm_ld(sm, S, e + dLo);
            fr_t x10 = sm_ld(sm, S, e + dHi), x11 = sm_ld(sm, S, e + dLo + dHi);
            // twiddle positions: bits of g below the stage's bit
            const uint32_t jl = ((g & ((1u << lo) - 1u)) << b0) | col;          // stage on bit lo
            const uint32_t jh0 = ((g & ((2u << lo) - 1u)) << b0) | col;         // stage on bit lo + 1, x0.
            const uint32_t jh1 = (((g & ((2u << lo) - 1u)) | (1u << lo)) << b0) | col;  // ... x1. (never 0)
            if (DIT) {
                if (jl) {
                    const fr_t w = ld_fr(tw + ((size_t)jl << tshA));
                    x01 = x01 * w;
                    x11 = x11 * w;
                }
                bfly(x00, x01);
                bfly(x10, x11);
                if (jh0) x10 = x10 * ld_fr(tw + ((size_t)jh0 << tshB));
                x11 = x11 * ld_fr(tw + ((size_t)jh1 << tshB));
                bfly(x00, x10);
                bfly(x01, x11);
            } else {
                bfly(x00, x10);
                bfly(x01, x11);
                if (jh0) x10 = x10 * ld_fr(tw + ((size_t)jh0 << tshA));
                x11 = x11 * ld_fr(tw + ((size_t)jh1 << tshA));
                bfly(x00, x01);
                bfly(x10, x11);
                if (jl) {
                    const fr_t w = ld_fr(tw + ((size_t)jl << tshB));
                    x01 = x01 * w;
                    x11 = x11 * w;
                }
            }
            sm_st(sm, S, e, x00);
            sm_st(sm, S, e + dLo, x01);
            sm_st(sm, S, e + dHi, x10);
            sm_st(sm, S, e + dLo + dHi, x11);
        }
        __syncthreads();
    }
    fr_t c;
    if (post.single) c = ld_fr(post.hi) * ld_fr(post.lo);
    for (uint32_t e = threadIdx.x; e < S; e += blockDim.x) {
        uint32_t g = e >> logG, ql = e & (G - 1u);
        uint32_t q = q0 + ql;
        uint32_t idx = ((q >> b0) << (b0 + t)) | (g << b0) | (q & lomask);
        fr_t x = sm_ld(sm, S, e);
        if (post.hi) x = x * (post.single ? c : scale_factor(post, idx, log_n));
        st_fr(out + (out_brev ? brev_bits(idx, log_n) : idx), x);
    }
}

// a pass handles up to 2^smem_log elements per block (2^11 x 32 B = 64 KB of
// shared memory); the plan's smem_log is chosen by the autotuner (10..12)

// Columns per block (2^logG, at most the plan's width): the grid runs in
// waves of (resident blocks per SM x SMs), so a pass takes about
// ceil(blocks / slots) x (work of one block).  Narrower blocks can fill the
// last wave better (one 2^20 array: 512 blocks of 2^11 elements against 456
// slots take two waves, 1,024 of 2^10 take three half-size waves).
typedef void (*NttPassFn)(const fr_t*, fr_t*, int, int, int, int, int, const fr_t*, int, NttScale, NttScale);
static NttPassFn ntt_pass_fn(bool dif, bool r4) {
    if (dif) return r4 ? k_ntt_pass<false, true> : k_ntt_pass<false, false>;
    return r4 ? k_ntt_pass<true, true> : k_ntt_pass<true, false>;
}

static int ntt_pick_columns(bool dif, bool r4, int k, int t, int logG_max, int count) {
    static int sms_of[64] = {};  // SM count per device ordinal (written once, same value)
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = dev >= 0 && dev < 64 ? sms_of[dev] : 0;
    if (!sms) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (dev >= 0 && dev < 64) sms_of[dev] = sms;
    }
    int best = logG_max;
    double best_cost = 1e300;
    for (int lg = logG_max; lg >= 0 && lg >= logG_max - 2; lg--) {
        const uint32_t S = (1u << lg) << t;
        int threads = S / 2 < ACE_NTT_THREADS ? (int)(S / 2) : ACE_NTT_THREADS;
        if (threads < 32) threads = 32;
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ntt_pass_fn(dif, r4), threads, (size_t)S * 32);
        if (nb <= 0) continue;
        const double blocks = (double)count * (double)(1u << (k - t - lg));
        const double slots = (double)nb * sms;
        const double cost = std::ceil(blocks / slots) * (double)S;
        if (cost < best_cost) {  // ties keep the wider block
            best_cost = cost;
            best = lg;
        }
    }
    return best;
}

int ntt_run(const NttPlan& plan, fr_t* data, int count, bool dif, bool inverse, const NttScale& pre,
            const NttScale& post, cudaStream_t st, bool fill_waves) {
    return ntt_run_io(plan, data, data, data, false, count, dif, inverse, pre, post, st, fill_waves);
}

int ntt_run_io(const NttPlan& plan, const fr_t* in, fr_t* work, fr_t* out, bool out_brev, int count, bool dif,
               bool inverse, const NttScale& pre, const NttScale& post, cudaStream_t st, bool fill_waves) {
    const int k = plan.log_n;
    const int NTT_MAX_T = plan.smem_log, NTT_SMEM_LOG = plan.smem_log;
    int passes[4], np = 0;
    if (k <= NTT_MAX_T) {
        passes[np++] = k;
    } else if (k <= 2 * NTT_MAX_T) {
        passes[np++] = (k + 1) / 2;
        passes[np++] = k - (k + 1) / 2;
    } else {
        int t1 = (k + 2) / 3, t2 = (k - t1 + 1) / 2;
        passes[np++] = t1;
        passes[np++] = t2;
        passes[np++] = k - t1 - t2;
    }
    // dynamic shared memory above 48 KB, once per device
    static bool attr_done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        for (int v = 0; v < 4; v++)
            cudaFuncSetAttribute(ntt_pass_fn(v & 1, v >> 1), cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    if (out_brev && np > 1 && out == work) {  // the last pass would read and scatter one array
        set_error("ntt: a bit-reversed output of a multi-pass transform needs its own array");
        return ACE_E_INTERNAL;
    }
    const bool r4 = plan.radix == 4;
    const fr_t* tw = inverse ? plan.tw_inv : plan.tw_fwd;
    NttScale none;
    int done_bits = 0;
    for (int pi = 0; pi < np; pi++) {
        int t = passes[pi];
        int b0, first_stage;
        if (dif) {
            b0 = k - done_bits - t;
            first_stage = done_bits;
        } else {
            b0 = done_bits;
            first_stage = done_bits;
        }
        int logG = NTT_SMEM_LOG - t;
        if (logG < 0) logG = 0;
        if (logG > k - t) logG = k - t;
        if (fill_waves) logG = ntt_pick_columns(dif, r4, k, t, logG, count);
        uint32_t groups = 1u << (k - t);
        uint32_t blocks = groups >> logG;
        uint32_t S = (1u << logG) << t;
        int threads = S / 2 < ACE_NTT_THREADS ? (int)(S / 2) : ACE_NTT_THREADS;
        if (threads < 32) threads = 32;
        size_t smem = (size_t)S * 32;
        dim3 grid(blocks, (unsigned)count);
        const NttScale& a = pi == 0 ? pre : none;
        const NttScale& z = pi == np - 1 ? post : none;
        int prof = prof_begin(PROF_NTT, st);
        const fr_t* src = pi == 0 ? in : work;
        fr_t* dst = pi == np - 1 ? out : work;
        const int brev = pi == np - 1 && out_brev;
        ntt_pass_fn(dif, r4)<<<grid, threads, smem, st>>>(src, dst, brev, k, t, b0, logG, tw, first_stage, a, z);
        ::ace::note_launch();
        // work: butterflies of this pass
        prof_end(prof, st, nullptr, (uint64_t)count * ((uint64_t)1 << (k - 1)) * (uint64_t)t);
        done_bits += t;
    }
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

}  // namespace ace
