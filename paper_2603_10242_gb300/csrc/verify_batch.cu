// verify_batch.cu -- batch verification of Groth16 proofs of one verifying
// key (the validators' check of Section 3.4, Algorithm 4, and the batch-verify
// precompile of Section 5, for many proofs at once).
//
// k proofs (A_i, B_i, C_i) with public inputs x_i are all valid (except with
// probability about k 2^-128) iff, for random 128-bit rho_i,
//   prod_i e(rho_i A_i, B_i)
//     * e(-(sum rho_i) alpha, beta) * e(-IC, gamma) * e(-(sum rho_i C_i), delta) = 1,
//   IC = (sum rho_i) ic_0 + (sum rho_i x_i) ic_1,
// i.e. k + 3 Miller loops and one final exponentiation instead of 4k Miller
// loops and k final exponentiations.  The device runs, one thread per proof,
// the subgroup check r B_i = O, rho_i A_i, rho_i C_i and the Miller loop of
// (rho_i A_i, B_i) (homogeneous projective, pairing.cuh); pairwise kernels
// multiply the Miller values and add the sums; a last kernel adds the three
// fixed pairs; the host applies the final exponentiation.
#define ACE_FIELD_MUL_CALL 1
#include <string.h>

#include <vector>

#include "circuit.h"
#include "curve.cuh"
#include "pairing.cuh"
#include "runtime.cuh"

namespace ace {
void pairing_consts_raw(fp_t gamma[12], fp_t b2[2], uint64_t* ate_lo, uint64_t* ate_hi);
bool final_exp_is_one_raw(const fp_t in[12]);
bool parse_g1_raw(const uint8_t b[64], fp_t out[2]);
bool parse_g2_raw(const uint8_t b[128], fp_t out[4]);

namespace {

struct VbProof {
    g1_aff A, C;
    g2_aff B;
    fr_t rho;  // canonical, < 2^128
    fr_t x;    // public input, canonical
};

struct VbKey {
    g1_aff alpha, ic0, ic1;
    g2_aff beta, gamma, delta;
};

// running values of one pairwise reduction slot
struct VbAcc {
    F12 f;          // product of Miller values
    g1_xyzz sc;     // sum rho_i C_i
    fr_t srho, sx;  // sum rho_i, sum rho_i x_i (Montgomery)
};

__device__ bool miller_or_one(const g1_aff& P, const g2_aff& Q, const PairConsts& k, F12& f) {
    if (aff_is_inf(P) || aff_is_inf(Q)) {
        f = f12_one();
        return true;
    }
    return miller_proj(P.x, P.y, Q.x, Q.y, k, f);
}

// one thread per proof
__global__ void __launch_bounds__(64) k_vb_proof(const VbProof* pr, uint32_t k, PairConsts pc, VbAcc* acc,
                                                 int32_t* bad) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k) return;
    const VbProof p = pr[q];
    // r B = O: B in the order-r subgroup of the twist
    uint32_t rl[8];
    for (int i = 0; i < 8; i++) rl[i] = mod_limb<FrCfg>(i);
    if (!aff_is_inf(p.B) && !xyzz_is_inf(xyzz_mul_aff(p.B, rl))) atomicOr(bad, 1);
    g1_aff ra = xyzz_to_aff(xyzz_mul_aff(p.A, p.rho.v));
    VbAcc a;
    if (!miller_or_one(ra, p.B, pc, a.f)) atomicOr(bad, 2);
    a.sc = xyzz_mul_aff(p.C, p.rho.v);
    a.srho = fe_to_mont(p.rho);
    a.sx = a.srho * fe_to_mont(p.x);
    acc[q] = a;
}

// out[i] = in[2i] (+) in[2i+1] for i < n/2 rounded up (an odd last one is copied)
__global__ void __launch_bounds__(64) k_vb_pair(const VbAcc* in, uint32_t n, VbAcc* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * i >= n) return;
    VbAcc a = in[2 * i];
    if (2 * i + 1 < n) {
        const VbAcc& b = in[2 * i + 1];
        a.f = a.f * b.f;
        a.sc = xyzz_add(a.sc, b.sc);
        a.srho = a.srho + b.srho;
        a.sx = a.sx + b.sx;
    }
    out[i] = a;
}

// three threads: the fixed pairs (-(sum rho) alpha, beta), (-IC, gamma),
// (-(sum rho C), delta); thread 0 multiplies them into the product
__global__ void k_vb_fixed(const VbAcc* total, VbKey key, PairConsts pc, fp_t* f_out, int32_t* bad) {
    __shared__ F12 fs[3];
    const int t = threadIdx.x;
    if (t < 3) {
        const VbAcc& a = *total;
        fr_t srho = fe_from_mont(a.srho), sx = fe_from_mont(a.sx);
        g1_aff P;
        g2_aff Q;
        if (t == 0) {
            P = xyzz_to_aff(xyzz_mul_aff(key.alpha, srho.v));
            Q = key.beta;
        } else if (t == 1) {
            g1_xyzz ic = xyzz_add(xyzz_mul_aff(key.ic0, srho.v), xyzz_mul_aff(key.ic1, sx.v));
            P = xyzz_to_aff(ic);
            Q = key.gamma;
        } else {
            P = xyzz_to_aff(a.sc);
            Q = key.delta;
        }
        P = aff_neg(P);
        if (!miller_or_one(P, Q, pc, fs[t])) atomicOr(bad, 4);
    }
    __syncthreads();
    if (t == 0) {
        F12 f = total->f * fs[0] * fs[1] * fs[2];
        memcpy(f_out, &f, sizeof f);
    }
}

}  // namespace
}  // namespace ace

using namespace ace;

extern "C" {

int ace_verify_batch(ace_ctx* ctx, const ace_vk* vk, size_t k, const ace_fr* pubs, const uint8_t* proofs,
                     uint64_t seed) {
    clear_error();
    if (!ctx || !vk || (k && (!pubs || !proofs))) {
        set_error("ace_verify_batch: NULL argument");
        return ACE_E_ARG;
    }
    if (k == 0) return 1;
    if (k > (1u << 20)) {  // scratch: about 1.5 KB of device memory per proof
        set_error("ace_verify_batch: k = %zu proofs (at most 2^20 per call)", k);
        return ACE_E_ARG;
    }
    // host: parse and validate every point, draw rho
    std::vector<VbProof> hp(k);
    SplitMix64 g(seed, 12);
    for (size_t i = 0; i < k; i++) {
        const uint8_t* b = proofs + 256 * i;
        VbProof& p = hp[i];
        if (!parse_g1_raw(b, &p.A.x) || !parse_g2_raw(b + 64, &p.B.x.c0) || !parse_g1_raw(b + 192, &p.C.x)) {
            set_error("ace_verify_batch: proof %zu has a point that is not canonical or not on the curve", i);
            return ACE_E_NOT_ON_CURVE;
        }
        memcpy(p.x.v, pubs[i].l, 32);
        if (fe_geq_mod(p.x)) {
            set_error("ace_verify_batch: public input %zu is not canonical", i);
            return ACE_E_ARG;
        }
        uint64_t lo, hi;
        do {
            lo = g.next();
            hi = g.next();
        } while (lo == 0 && hi == 0);
        p.rho = fe_zero<FrCfg>();
        p.rho.v[0] = (uint32_t)lo;
        p.rho.v[1] = (uint32_t)(lo >> 32);
        p.rho.v[2] = (uint32_t)hi;
        p.rho.v[3] = (uint32_t)(hi >> 32);
    }
    static_assert(sizeof(g1_aff) == 2 * sizeof(fp_t) && sizeof(g2_aff) == 4 * sizeof(fp_t), "plain point layout");
    VbKey key;
    const uint8_t* v = (const uint8_t*)vk;
    if (!parse_g1_raw(v, &key.alpha.x) || !parse_g2_raw(v + 64, &key.beta.x.c0) ||
        !parse_g2_raw(v + 192, &key.gamma.x.c0) || !parse_g2_raw(v + 320, &key.delta.x.c0) ||
        !parse_g1_raw(v + 448, &key.ic0.x) || !parse_g1_raw(v + 512, &key.ic1.x)) {
        set_error("ace_verify_batch: verifying key point not on the curve");
        return ACE_E_NOT_ON_CURVE;
    }
    PairConsts pc;
    {
        fp_t gm[12], b2[2];
        pairing_consts_raw(gm, b2, &pc.ate_lo, &pc.ate_hi);
        for (int i = 0; i < 6; i++) pc.gamma[i] = {gm[2 * i], gm[2 * i + 1]};
        pc.b2 = {b2[0], b2[1]};
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t bytes = k * sizeof(VbProof) + 2 * k * sizeof(VbAcc) + 12 * sizeof(fp_t) + 4096;
    ACE_TRY(arena_ensure(ctx, 2, bytes));
    Arena& ar = ctx->scratch[2];
    VbProof* d_p = (VbProof*)ar.take(k * sizeof(VbProof));
    VbAcc* d_a = (VbAcc*)ar.take(k * sizeof(VbAcc));
    VbAcc* d_b = (VbAcc*)ar.take(k * sizeof(VbAcc));
    fp_t* d_f = (fp_t*)ar.take(12 * sizeof(fp_t));
    int32_t* d_bad = (int32_t*)ar.take(16);
    if (!d_p || !d_a || !d_b || !d_f || !d_bad) {
        set_error("ace_verify_batch: scratch too small");
        return ACE_E_OOM;
    }
    ACE_TRY_CUDA(cudaMemcpyAsync(d_p, hp.data(), k * sizeof(VbProof), cudaMemcpyHostToDevice, st));
    ACE_TRY_CUDA(cudaMemsetAsync(d_bad, 0, 4, st));
    k_vb_proof<<<(unsigned)((k + 63) / 64), 64, 0, st>>>(d_p, (uint32_t)k, pc, d_a, d_bad);
    ::ace::note_launch();
    uint32_t n = (uint32_t)k;
    VbAcc *in = d_a, *out = d_b;
    while (n > 1) {
        uint32_t half = (n + 1) / 2;
        k_vb_pair<<<(half + 63) / 64, 64, 0, st>>>(in, n, out);
        ::ace::note_launch();
        VbAcc* t = in;
        in = out;
        out = t;
        n = half;
    }
    k_vb_fixed<<<1, 32, 0, st>>>(in, key, pc, d_f, d_bad);
    ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    fp_t f[12];
    int32_t bad = 0;
    ACE_TRY_CUDA(cudaMemcpyAsync(f, d_f, sizeof f, cudaMemcpyDeviceToHost, st));
    ACE_TRY_CUDA(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, st));
    ACE_TRY_CUDA(cudaStreamSynchronize(st));
    if (bad) return 0;  // a B outside the subgroup (or a degenerate Miller loop)
    return final_exp_is_one_raw(f) ? 1 : 0;
}

}  // extern "C"
