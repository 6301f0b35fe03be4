// prove.cu -- the Groth16 prover on the device: Groth16.Prove of the paper's
// Phase 2 (Section 3.1, Algorithm 1 ProveAsync; Section 3.3, Algorithm 3
// Stage 1), producing the 256-byte proof of Section 3.3 / Appendix B.
//
//   1. a, b, c = Az, Bz, Cz (one thread per row, rows by decreasing length,
//      all three matrices in one loop), with the R1CS check a_i b_i = c_i
//      folded in (status word on failure);
//   2. QAP quotient: inverse NTT of a, b, c (decimation in frequency, scaled
//      by g^e / N on the way out: coset coefficients), forward NTT
//      (decimation in time: values on g H), q_i = (a b - c)/(g^N - 1) =
//      h(g omega^i), canonical, natural order;
//   3. five MSMs on their own streams: H (the q_i against the key's H query in
//      the Lagrange basis of g H) on the main stream, A, B1 (G1), B2 (G2) and
//      L on auxiliary streams, with the witness gathered per compacted query
//      (B2 reuses B1's sorted entries);
//   4. assembly: A = alpha + S_A + r delta, B = beta + S_B2 + s delta and
//      C = S_L + S_H + s A + r B1 - r s delta with B1 = beta + S_B1 + s delta,
//      i.e. C = S_L + S_H + s alpha + r beta + r s delta + s S_A + r S_B1:
//      the fixed-base terms come from the key's window tables at the start,
//      s S_A + r S_B1 (GLV chains) as soon as the A and B1 MSMs are done, and
//      the last kernel only adds and converts to affine.
// The field product, square and difference of products are called out of
// line: the single-thread chains of step 4 (hundreds of dependent curve
// operations) run about twice as fast from one shared body as from inlined
// copies that keep missing the instruction cache.
#define ACE_FIELD_MUL_CALL 1
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "curve_quad.cuh"
#include "fixed_base.cuh"
#include "glv.cuh"
#include "pk.h"

namespace ace {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ fr_t ldg_fr(const fr_t* p) {
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4 a = __ldg(s), b = __ldg(s + 1);
    fr_t r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
    r.v[4] = b.x; r.v[5] = b.y; r.v[6] = b.z; r.v[7] = b.w;
    return r;
}
__device__ __forceinline__ void st_fr2(fr_t* p, const fr_t& x) {
    uint4* d = reinterpret_cast<uint4*>(p);
    d[0] = make_uint4(x.v[0], x.v[1], x.v[2], x.v[3]);
    d[1] = make_uint4(x.v[4], x.v[5], x.v[6], x.v[7]);
}

struct CsrDev {
    const uint32_t* rp[3];
    const uint32_t* col[3];
    const fr_t* val[3];
};

// a, b, c (Montgomery) for every row; z canonical.  The product of a
// Montgomery coefficient and a canonical z_j is the canonical product, so the
// row sums are canonical and one multiplication by R^2 mod r returns them to
// Montgomery form.  Row lengths vary from 1 to a few hundred terms (S-box
// inputs are long linear combinations, packing rows carry one term per bit),
// so thread t takes row order[t] (rows by decreasing total length) and runs
// over the row's A, B and C terms in one loop: the lanes of a warp then do
// equal numbers of products whatever the split of their totals among A, B, C.
// The R1CS check a b = c is made on the way.
// inlined Montgomery product for the sparse products (one product per loop
// iteration: a short loop body that keeps 64 registers)
__device__ __forceinline__ fr_t mul_inl(const fr_t& x, const fr_t& y) {
#if defined(__CUDA_ARCH__)
    fr_t r;
    d_mul_form<FrCfg>(r.v, x.v, y.v);
    return r;
#else
    return x * y;
#endif
}

__device__ __forceinline__ void rows_abc(const CsrDev& m, const fr_t* __restrict__ z, uint32_t i, fr_t& a, fr_t& b,
                                         fr_t& c) {
    fr_t acc = fe_zero<FrCfg>(), sa = acc, sb = acc;
    int k = 0;
    const uint32_t* __restrict__ col = m.col[0];
    const fr_t* __restrict__ val = m.val[0];
    uint32_t t = __ldg(m.rp[0] + i), e = __ldg(m.rp[0] + i + 1);
    for (;;) {
        while (t == e) {  // matrix k done: keep its sum, go to the next
            if (k == 0) sa = acc;
            else if (k == 1) sb = acc;
            if (++k == 3) break;
            acc = fe_zero<FrCfg>();
            col = k == 1 ? m.col[1] : m.col[2];
            val = k == 1 ? m.val[1] : m.val[2];
            t = __ldg((k == 1 ? m.rp[1] : m.rp[2]) + i);
            e = __ldg((k == 1 ? m.rp[1] : m.rp[2]) + i + 1);
        }
        if (k == 3) break;
        acc = acc + mul_inl(ldg_fr(val + t), ldg_fr(z + __ldg(col + t)));
        t++;
    }
    a = mul_inl(sa, fe_rr<FrCfg>());
    b = mul_inl(sb, fe_rr<FrCfg>());
    c = mul_inl(acc, fe_rr<FrCfg>());
}

__global__ void __launch_bounds__(256) k_spmv3(CsrDev m, const uint32_t* __restrict__ order,
                                               const fr_t* __restrict__ z, uint32_t N, fr_t* abc, int32_t* status) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const uint32_t i = __ldg(order + t);
    fr_t a, b, c;
    rows_abc(m, z, i, a, b, c);
    st_fr2(abc + i, a);
    st_fr2(abc + (size_t)N + i, b);
    st_fr2(abc + 2 * (size_t)N + i, c);
    if (!fe_eq(a * b, c)) atomicOr(status, 1);
}

// q_i = (a_i b_i - c_i) * zinv, written over a (zinv in Montgomery form keeps
// q in Montgomery form; its plain value gives the canonical q)
__global__ void k_quotient(fr_t* abc, uint32_t N, fr_t zinv) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    fr_t a = ldg_fr(abc + i), b = ldg_fr(abc + N + i), c = ldg_fr(abc + 2 * (size_t)N + i);
    st_fr2(abc + i, (a * b - c) * zinv);
}

__global__ void k_gather(const fr_t* __restrict__ z, const uint32_t* __restrict__ idx, uint32_t n, fr_t* out) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    st_fr2(out + k, ldg_fr(z + __ldg(idx + k)));
}

// Fixed-base terms from the key's window tables, one warp each (lane 0):
// fx1 = {r delta1, s alpha1, r beta1, r s delta1}, fx2 = {s delta2}.
struct PkTabs {
    const g1_aff *alpha1, *beta1, *delta1;
    const g2_aff* delta2;
};
// k P from the 8-bit window table of P (tab[w 255 + d - 1] = d 2^(8w) P):
// the 32 byte-windows' table points summed on four lanes (the same sum as
// fixed_mul_tab, bit for bit); all four lanes of `mask` call with the same k
template <class F>
__device__ Xyzz<F> fixed_mul_tab_quad(const Affine<F>* tab, const uint32_t* k, int sub, unsigned mask) {
    Xyzz<F> acc = xyzz_inf<F>();
#pragma unroll 1
    for (int w = 0; w < 32; w++) {
        const uint32_t d = (k[w >> 2] >> ((w & 3) * 8)) & 255u;
        if (d) acc = quad_add(acc, xyzz_from_aff(tab[w * 255 + d - 1]), sub, mask);
    }
    return acc;
}
// fixed-base term w (0..4) on lanes 0..3 of the calling warp; lane 0 writes it
__device__ __forceinline__ void fixed_term(const PkTabs& t, const fr_t& r, const fr_t& s, const fr_t& rs, int w,
                                           g1_xyzz* fx1, g2_xyzz* fx2) {
    const int lane = threadIdx.x & 31;
    if (lane >= 4) return;
    const unsigned mask = 0xfu;
    if (w == 4) {
        g2_xyzz v = fixed_mul_tab_quad(t.delta2, s.v, lane, mask);
        if (lane == 0) fx2[0] = v;
        return;
    }
    const g1_aff* tab = w == 1 ? t.alpha1 : w == 2 ? t.beta1 : t.delta1;
    const uint32_t* k = w == 1 ? s.v : w == 3 ? rs.v : r.v;
    g1_xyzz v = fixed_mul_tab_quad(tab, k, lane, mask);
    if (lane == 0) fx1[w] = v;
}
// one term per warp (160 threads)
__global__ void __launch_bounds__(160) k_prove_fixed(PkTabs t, fr_t r, fr_t s, fr_t rs, g1_xyzz* fx1,
                                                     g2_xyzz* fx2) {
    fixed_term(t, r, s, rs, threadIdx.x >> 5, fx1, fx2);
}

// The variable-base part of C: V = s S_A + r S_B1, as soon as the A and B1
// MSMs are done.  With the GLV endomorphism phi(x, y) = (beta x, y) = lambda
// (x, y) on G1, s = s1 + s2 lambda and r = r1 + r2 lambda (mod r) with 128-bit
// halves (split on the host), so V = s1 S_A + s2 phi(S_A) + r1 S_B1 +
// r2 phi(S_B1): four 128-bit chains, one per warp, each on that warp's first
// four lanes with the four-lane point formulas (a doubling takes 3 levels of
// products instead of 9, an addition 4 instead of 16).  Each chain walks the
// width-5 NAF of its half (digits 0, +-1, +-3, ..., +-15, at most one non-zero
// digit in five): about 128 doublings and 22 additions of a table of the odd
// multiples P, 3P, ..., 15P, instead of 64 additions for the binary digits.
// Each chain has a warp to itself, so one chain's additions do not hold up
// another's doublings.
#define GLV_NAF_LEN 132
struct GlvScalars {
    uint32_t k[4][4];  // |s1|, |s2|, |r1|, |r2|
    uint32_t neg[4];
    int8_t naf[4][GLV_NAF_LEN];  // width-5 NAF of each |k_t|, least significant digit first
};
// block of 128 threads; sa, sb: S_A and S_B1; writes V to *v
__device__ __forceinline__ void var_term_quad(const g1_xyzz& sa, const g1_xyzz& sb, const GlvScalars& g,
                                              const fp_t& beta, g1_xyzz* v) {
    __shared__ g1_xyzz part[4];
    __shared__ g1_xyzz odd[4][8];  // (2 j + 1) P of chain t
    const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < 4) {
        const unsigned mask = 0xfu;
        g1_xyzz P = t < 2 ? sa : sb;
        if (t & 1) P.X = P.X * beta;
        if (g.neg[t]) P.Y = fe_neg(P.Y);
        const g1_xyzz P2 = quad_dbl(P, lane, mask);
        g1_xyzz m = P;
        if (lane == 0) odd[t][0] = m;
        for (int j = 1; j < 8; j++) {
            m = quad_add(m, P2, lane, mask);
            if (lane == 0) odd[t][j] = m;
        }
        __syncwarp(mask);
        const int8_t* naf = g.naf[t];
        int top = GLV_NAF_LEN - 1;
        while (top > 0 && naf[top] == 0) top--;
        g1_xyzz acc = xyzz_inf<fp_t>();
        for (int i = top; i >= 0; i--) {
            acc = quad_dbl(acc, lane, mask);
            const int d = naf[i];
            if (d) {
                g1_xyzz q = odd[t][(d > 0 ? d : -d) >> 1];
                if (d < 0) q.Y = fe_neg(q.Y);
                acc = quad_add(acc, q, lane, mask);
            }
        }
        if (lane == 0) part[t] = acc;
    }
    __syncthreads();
    if (t == 0 && lane < 4) {
        const unsigned mask = 0xfu;
        g1_xyzz x = quad_add(part[0], part[1], lane, mask);
        g1_xyzz y = quad_add(part[2], part[3], lane, mask);
        x = quad_add(x, y, lane, mask);
        if (lane == 0) *v = x;
    }
}
__global__ void __launch_bounds__(128) k_prove_var(const g1_xyzz* res1, const __grid_constant__ GlvScalars g,
                                                   fp_t beta, g1_xyzz* v) {
    var_term_quad(res1[1], res1[2], g, beta, v);
}

// The same term with one joint double-and-add over the 256 bits of s and r
// (one thread): the fallback if the split ever failed to give 128-bit
// halves, and the per-proof form of a block of proofs of one key.
__device__ g1_xyzz var_term_joint(const g1_xyzz& a, const g1_xyzz& b, const fr_t& r, const fr_t& s) {
    g1_xyzz ab = xyzz_add(a, b);
    g1_xyzz acc = xyzz_inf<fp_t>();
    for (int i = 255; i >= 0; i--) {
        acc = xyzz_dbl(acc);
        uint32_t bs = (s.v[i >> 5] >> (i & 31)) & 1u, br = (r.v[i >> 5] >> (i & 31)) & 1u;
        if (bs && br) acc = xyzz_add(acc, ab);
        else if (bs) acc = xyzz_add(acc, a);
        else if (br) acc = xyzz_add(acc, b);
    }
    return acc;
}
__global__ void k_prove_var_joint(const g1_xyzz* res1, fr_t r, fr_t s, g1_xyzz* v) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *v = var_term_joint(res1[1], res1[2], r, s);
}

// ---- GLV split on the host (glv.cuh) --------------------------------------
static const uint32_t GLV_BETA[8] = ACE_GLV_BETA;
static bool glv_split(const fr_t& k, uint32_t k1[4], uint32_t* n1, uint32_t k2[4], uint32_t* n2) {
    return glv_split_limbs(k.v, k1, n1, k2, n2);
}

// Width-5 NAF of a value below 2^128 (the window-w NAF of Solinas, in the
// form of Guide to Elliptic Curve Cryptography, Algorithm 3.35): while x > 0,
// an odd x gives the digit d = x mods 32 (in -15..15) and x -= d; then x /= 2.
// sum_i out[i] 2^i = k; false if the digits do not fit GLV_NAF_LEN.
static bool wnaf5(const uint32_t k[4], int8_t out[GLV_NAF_LEN]) {
    uint32_t x[5] = {k[0], k[1], k[2], k[3], 0};
    for (int i = 0; i < GLV_NAF_LEN; i++) {
        int d = 0;
        if (x[0] & 1u) {
            d = (int)(x[0] & 31u);
            if (d >= 16) d -= 32;
            // x -= d over five limbs (x + 15 < 2^129 stays in range)
            uint64_t c = d > 0 ? (uint64_t)(uint32_t)d : 0, a = d < 0 ? (uint64_t)(uint32_t)(-d) : 0;
            for (int l = 0; l < 5; l++) {
                uint64_t v = (uint64_t)x[l] + a - c;
                x[l] = (uint32_t)v;
                // carry (+1), borrow (-1) or neither into the next limb
                a = (v >> 32) == 1 ? 1 : 0;
                c = (v >> 32) > 1 ? 1 : 0;
            }
        }
        out[i] = (int8_t)d;
        for (int l = 0; l < 4; l++) x[l] = (x[l] >> 1) | (x[l + 1] << 31);
        x[4] >>= 1;
    }
    return (x[0] | x[1] | x[2] | x[3] | x[4]) == 0;
}

// The GLV halves of s and r and their NAFs (false if a split or a recoding failed)
static bool glv_scalars(const fr_t& r, const fr_t& s, GlvScalars& g) {
    if (!glv_split(s, g.k[0], &g.neg[0], g.k[1], &g.neg[1]) || !glv_split(r, g.k[2], &g.neg[2], g.k[3], &g.neg[3]))
        return false;
    for (int t = 0; t < 4; t++)
        if (!wnaf5(g.k[t], g.naf[t])) return false;
    return true;
}

__device__ void write_g1(uint32_t* dst, const g1_xyzz& p) {
    g1_aff a = aff_from_mont(xyzz_to_aff(p));
    for (int i = 0; i < 8; i++) {
        dst[i] = a.x.v[i];
        dst[8 + i] = a.y.v[i];
    }
}

// A = alpha + S_A + r delta;  B = beta2 + S_B2 + s delta2;
// C = S_L + S_H + (s alpha + r beta + r s delta) + V   (one warp each)
// res1: S_H, S_A, S_B1, S_L;  fx1 / fx2 from the fixed terms;  v = V
__device__ __forceinline__ void assemble_part(int w, const PkFixed* fx, const g1_xyzz* res1, const g2_xyzz* resB2,
                                              const g1_xyzz* fx1, const g2_xyzz* fx2, const g1_xyzz* v,
                                              uint32_t* proof) {
    if (w == 0) {
        g1_xyzz A = xyzz_add(xyzz_add(xyzz_from_aff(fx->alpha1), res1[1]), fx1[0]);
        write_g1(proof, A);
    } else if (w == 1) {
        g2_xyzz B = xyzz_add(xyzz_add(xyzz_from_aff(fx->beta2), resB2[0]), fx2[0]);
        g2_aff b = aff_from_mont(xyzz_to_aff(B));
        for (int i = 0; i < 8; i++) {
            proof[16 + i] = b.x.c0.v[i];
            proof[24 + i] = b.x.c1.v[i];
            proof[32 + i] = b.y.c0.v[i];
            proof[40 + i] = b.y.c1.v[i];
        }
    } else {
        g1_xyzz C = xyzz_add(xyzz_add(res1[3], res1[0]), xyzz_add(xyzz_add(fx1[1], fx1[2]), fx1[3]));
        C = xyzz_add(C, *v);
        write_g1(proof + 48, C);
    }
}
__global__ void k_assemble(const PkFixed* fx, const g1_xyzz* res1, const g2_xyzz* resB2, const g1_xyzz* fx1,
                           const g2_xyzz* fx2, const g1_xyzz* v, uint32_t* proof) {
    if ((threadIdx.x & 31) != 0) return;
    assemble_part(threadIdx.x >> 5, fx, res1, resB2, fx1, fx2, v, proof);
}

// ---------------------------------------------------------------------------
// tails of a batch of proofs (any keys): the fixed-base terms of every proof
// in one launch before the MSMs, V and the assembly of every proof in one
// launch each after them; block q serves proof q
// ---------------------------------------------------------------------------
struct TailDesc {
    PkTabs tabs;
    const PkFixed* fixed;
    fr_t r, s, rs;  // canonical
    GlvScalars glv;
    uint32_t glv_ok;
};
// per proof q: fx1[4 q .. 4 q + 3], fx2[q]; 160 threads per block
__global__ void __launch_bounds__(160) k_prove_fixed_batch(const TailDesc* d, g1_xyzz* fx1, g2_xyzz* fx2) {
    const TailDesc& q = d[blockIdx.x];
    fixed_term(q.tabs, q.r, q.s, q.rs, threadIdx.x >> 5, fx1 + 4 * (size_t)blockIdx.x, fx2 + blockIdx.x);
}
// res1: S_H, S_A, S_B1, S_L of proof q at res1[4 q ..]; 128 threads per block
__global__ void __launch_bounds__(128) k_prove_var_batch(const TailDesc* d, const g1_xyzz* res1, fp_t beta,
                                                         g1_xyzz* v) {
    const TailDesc& q = d[blockIdx.x];
    const g1_xyzz* r1 = res1 + 4 * (size_t)blockIdx.x;
    if (q.glv_ok) {
        var_term_quad(r1[1], r1[2], q.glv, beta, v + blockIdx.x);
    } else if (threadIdx.x == 0) {
        v[blockIdx.x] = var_term_joint(r1[1], r1[2], q.r, q.s);
    }
}
// 96 threads per block; proof q at proofs + 64 q (words)
__global__ void __launch_bounds__(96) k_assemble_batch(const TailDesc* d, const g1_xyzz* res1, const g2_xyzz* res2,
                                                       const g1_xyzz* fx1, const g2_xyzz* fx2, const g1_xyzz* v,
                                                       uint32_t* proofs) {
    if ((threadIdx.x & 31) != 0) return;
    const size_t q = blockIdx.x;
    assemble_part(threadIdx.x >> 5, d[q].fixed, res1 + 4 * q, res2 + q, fx1 + 4 * q, fx2 + q, v + q,
                  proofs + 64 * q);
}

// ---------------------------------------------------------------------------
// many proofs of one key in one pass (per-transaction proofs: every
// transaction of a block proves the same circuit, Section 3.3, Algorithm 3
// ParallelMap).  Proof q's witness is z + q m, its a, b, c are abc + 3 q N,
// its quotient h + q N; every kernel covers all proofs (blockIdx.y or one
// thread per proof).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_spmv3_many(CsrDev m, const uint32_t* __restrict__ order,
                                                    const fr_t* __restrict__ z, uint64_t wit, uint32_t N, fr_t* abc,
                                                    int32_t* status) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const uint32_t q = blockIdx.y, i = __ldg(order + t);
    z += (size_t)q * wit;
    abc += (size_t)q * 3 * N;
    fr_t a, b, c;
    rows_abc(m, z, i, a, b, c);
    st_fr2(abc + i, a);
    st_fr2(abc + (size_t)N + i, b);
    st_fr2(abc + 2 * (size_t)N + i, c);
    if (!fe_eq(a * b, c)) atomicOr(status + q, 1);
}

__global__ void k_quotient_many(const fr_t* abc, uint32_t N, fr_t zinv, fr_t* h) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t q = blockIdx.y;
    abc += (size_t)q * 3 * N;
    fr_t a = ldg_fr(abc + i), b = ldg_fr(abc + N + i), c = ldg_fr(abc + 2 * (size_t)N + i);
    st_fr2(h + (size_t)q * N + i, (a * b - c) * zinv);
}

__global__ void k_gather_many(const fr_t* __restrict__ z, uint64_t wit, const uint32_t* __restrict__ idx, uint32_t n,
                              fr_t* out) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t q = blockIdx.y;
    st_fr2(out + (size_t)q * n + k, ldg_fr(z + (size_t)q * wit + __ldg(idx + k)));
}

// per proof q: r_q, s_q, r_q s_q (canonical) at rsv[3 q .. 3 q + 2]
__global__ void k_prove_fixed_many(PkTabs t, const fr_t* rsv, uint32_t count, g1_xyzz* fx1, g2_xyzz* fx2) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 5 * count) return;
    const uint32_t q = g / 5, term = g % 5;
    const fr_t r = rsv[3 * q], s = rsv[3 * q + 1], rs = rsv[3 * q + 2];
    switch (term) {
        case 0: fx1[4 * q + 0] = fixed_mul_tab(t.delta1, r.v); break;
        case 1: fx1[4 * q + 1] = fixed_mul_tab(t.alpha1, s.v); break;
        case 2: fx1[4 * q + 2] = fixed_mul_tab(t.beta1, r.v); break;
        case 3: fx1[4 * q + 3] = fixed_mul_tab(t.delta1, rs.v); break;
        default: fx2[q] = fixed_mul_tab(t.delta2, s.v); break;
    }
}

__global__ void k_prove_var_many(const g1_xyzz* sa, const g1_xyzz* sb, const fr_t* rsv, uint32_t count,
                                 g1_xyzz* v) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    v[q] = var_term_joint(sa[q], sb[q], rsv[3 * q], rsv[3 * q + 1]);
}

// res1: S_H, S_A, S_B1, S_L, each `count` results; proof q at proof + 64 q
__global__ void k_assemble_many(const PkFixed* fx, const g1_xyzz* res1, const g2_xyzz* resB2, const g1_xyzz* fx1,
                                const g2_xyzz* fx2, const g1_xyzz* v, uint32_t count, uint32_t* proof) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * count) return;
    const uint32_t q = g / 3, w = g % 3;
    const g1_xyzz *SH = res1, *SA = res1 + count, *SL = res1 + 3 * (size_t)count;
    proof += 64 * (size_t)q;
    if (w == 0) {
        g1_xyzz A = xyzz_add(xyzz_add(xyzz_from_aff(fx->alpha1), SA[q]), fx1[4 * q + 0]);
        write_g1(proof, A);
    } else if (w == 1) {
        g2_xyzz B = xyzz_add(xyzz_add(xyzz_from_aff(fx->beta2), resB2[q]), fx2[q]);
        g2_aff b = aff_from_mont(xyzz_to_aff(B));
        for (int i = 0; i < 8; i++) {
            proof[16 + i] = b.x.c0.v[i];
            proof[24 + i] = b.x.c1.v[i];
            proof[32 + i] = b.y.c0.v[i];
            proof[40 + i] = b.y.c1.v[i];
        }
    } else {
        g1_xyzz C = xyzz_add(xyzz_add(SL[q], SH[q]),
                             xyzz_add(xyzz_add(fx1[4 * q + 1], fx1[4 * q + 2]), fx1[4 * q + 3]));
        C = xyzz_add(C, v[q]);
        write_g1(proof + 48, C);
    }
}

// ---------------------------------------------------------------------------
// drivers
// ---------------------------------------------------------------------------
static CsrDev csr_of(const ace_pk* pk) {
    CsrDev m;
    for (int k = 0; k < 3; k++) {
        m.rp[k] = pk->d_rp[k];
        m.col[k] = pk->d_col[k];
        m.val[k] = pk->d_val[k];
    }
    return m;
}

// steps 1-2.  coset = true (proving): leaves the canonical values h(g omega^i)
// in natural order in abc[0..N), the scalars of the H query in the coset
// Lagrange basis; coset = false: the canonical coefficients of h (one more
// inverse transform), in natural order in h_out (abc is scratch then)
static int qap_run(ace_ctx* ctx, const ace_pk* pk, const fr_t* d_z, fr_t* abc, int32_t* d_status,
                   cudaStream_t st, bool coset, fr_t* h_out = nullptr) {
    NttPlan* plan = nullptr;
    ACE_TRY(ntt_get_plan(ctx, pk->log_n, &plan));
    const uint32_t N = (uint32_t)pk->N;
    int prof = prof_begin(PROF_SPMV, st);
    k_spmv3<<<(N + 255) / 256, 256, 0, st>>>(csr_of(pk), pk->d_row_order, d_z, N, abc, d_status); ::ace::note_launch();
    prof_end(prof, st, nullptr, pk->nnz[0] + pk->nnz[1] + pk->nnz[2]);
    NttScale none, cos, icos;
    cos.hi = plan->cos_hi;
    cos.lo = plan->cos_lo;
    cos.h = plan->h;
    cos.brev = 1;
    icos.hi = plan->icos_hi;
    icos.lo = plan->icos_lo;
    icos.h = plan->h;
    icos.brev = 1;
    ACE_TRY(ntt_run(*plan, abc, 3, true, true, none, cos, st));
    ACE_TRY(ntt_run(*plan, abc, 3, false, false, none, none, st));
    if (coset) {
        // (a b - c) is in Montgomery form; a product with the plain value of
        // (g^N - 1)^-1 leaves Montgomery form: canonical h(g omega^i)
        k_quotient<<<(N + 255) / 256, 256, 0, st>>>(abc, N, fe_from_mont(plan->zinv)); ::ace::note_launch();
    } else {
        k_quotient<<<(N + 255) / 256, 256, 0, st>>>(abc, N, plan->zinv); ::ace::note_launch();
        ACE_TRY(ntt_run_io(*plan, abc, abc, h_out, true, 1, true, true, none, icos, st));
    }
    ACE_TRY_CUDA(cudaGetLastError());
    return ACE_OK;
}

struct ProvePlans {
    MsmPlan H, A, B, L;
    size_t slot_bytes[5];
};

static ProvePlans prove_plans(const ace_pk* pk) {
    ProvePlans p;
    p.H = pk->H_plan;
    p.A = pk->A.plan;
    p.B = pk->B1.plan;
    p.L = pk->L.plan;
    size_t N = pk->N;
    p.slot_bytes[0] = 3 * N * sizeof(fr_t) + msm_scratch_bytes<fp_t>(p.H, true) + (1 << 16);
    p.slot_bytes[1] = pk->A.count * sizeof(fr_t) + msm_scratch_bytes<fp_t>(p.A, true) + 4096;
    p.slot_bytes[2] = pk->B1.count * sizeof(fr_t) + msm_scratch_bytes<fp_t>(p.B, true) + 4096;
    p.slot_bytes[3] = pk->B2.count * sizeof(fr_t) + msm_scratch_bytes<fp2_t>(p.B, true) + 4096;
    p.slot_bytes[4] = pk->L.count * sizeof(fr_t) + msm_scratch_bytes<fp_t>(p.L, true) + 4096;
    return p;
}

size_t prove_slot_bytes(const ace_pk* pk, int arena) { return prove_plans(pk).slot_bytes[arena]; }

template <class F>
static int gathered_msm(const MsmPlan& plan, const Query<F>& q, const fr_t* d_z, Arena& ar, Xyzz<F>* res,
                        cudaStream_t s, MsmSorted* sorted = nullptr, cudaEvent_t sorted_ev = nullptr) {
    fr_t* zq = (fr_t*)ar.take((size_t)q.count * sizeof(fr_t) + 32);
    if (!zq) {
        set_error("prove: arena too small");
        return ACE_E_OOM;
    }
    if (q.count) {
        k_gather<<<(q.count + 255) / 256, 256, 0, s>>>(d_z, q.d_idx, q.count, zq);
        ::ace::note_launch();
    }
    return msm_run<F>(plan, q.d_pts, true, (const uint32_t*)zq, ar, res, nullptr, s, nullptr, sorted, sorted_ev);
}

// Full proof on proving slot `slot`, on the slot's streams of priority level
// `prio`: ordered after the work already on `st_in` and after the slot's
// previous proof; writes the 256 proof bytes to d_proof and the R1CS status
// to d_status (0 ok, 1 unsat), both device memory.  With join, st_in waits
// for the proof; without, the caller joins on the slot's ev_done.  The main
// stream runs the QAP and the H MSM, the auxiliary streams the A, B1, B2 and
// L MSMs and the fixed-base terms; proofs on other slots overlap.
// msm_out (a batch's proof): only the QAP and the five MSMs run; their sums go
// to msm_out->res1 (S_H, S_A, S_B1, S_L) and msm_out->res2 (S_B2), the slot's
// ev_done marks them complete, and the fixed-base terms, V and the assembly
// are left to the batch's tail kernels (d_proof is not written).
int prove_run(ace_ctx* ctx, int slot, int prio, const ace_pk* pk, const fr_t* d_z, const fr_t& r, const fr_t& s,
              uint32_t* d_proof, int32_t* d_status, cudaStream_t st_in, bool join, const MsmOut* msm_out,
              bool one_stream, bool alone) {
    if (prio < 0 || prio >= PRIO_LEVELS || slot < 0 || slot >= MAX_SLOTS) {
        set_error("prove: slot %d / priority level %d out of range", slot, prio);
        return ACE_E_ARG;
    }
    ACE_TRY(slot_ready(ctx, slot));
    ProveSlot& sl = ctx->slots[slot];
    // the slot's streams at this level; in serial mode (a measurement of the
    // per-stage split) every stage runs on the main stream, one after another
    SlotStreams ss = sl.lv[prio];
    if (ctx->serial || one_stream)
        for (int k = 0; k < 5; k++) ss.aux[k] = ss.main;
    ProvePlans pl = prove_plans(pk);
    pl.A.alone = pl.B.alone = pl.L.alone = pl.H.alone = alone;
    for (int k = 0; k < PROVE_ARENAS; k++) ACE_TRY(slot_arena_ensure(ctx, slot, k, pl.slot_bytes[k]));
    Arena& a0 = sl.ar[0];
    fr_t* abc = (fr_t*)a0.take(3 * pk->N * sizeof(fr_t));
    g1_xyzz* res1 = (g1_xyzz*)a0.take(10 * sizeof(g1_xyzz));
    g2_xyzz* res2 = (g2_xyzz*)a0.take(2 * sizeof(g2_xyzz));
    if (!abc || !res1 || !res2) {
        set_error("prove: arena too small");
        return ACE_E_OOM;
    }
    g1_xyzz* fx1 = res1 + 4;  // 4 fixed-base terms
    g1_xyzz* vterm = res1 + 8;
    g2_xyzz* fx2 = res2 + 1;
    if (msm_out) {
        res1 = msm_out->res1;
        res2 = msm_out->res2;
    }
    PkTabs tabs{pk->d_tab_alpha1, pk->d_tab_beta1, pk->d_tab_delta1, pk->d_tab_delta2};
    // r s mod r on the host
    fr_t rs = fe_from_mont(fe_to_mont(r) * fe_to_mont(s));

    // main waits for the caller's inputs and for the slot's previous proof
    // (its arenas are reused; it joined its own auxiliary streams); the
    // auxiliary streams start after main
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_in, st_in));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.main, sl.ev_in, 0));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.main, sl.ev_done, 0));
    ACE_TRY_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int32_t), ss.main));
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_start, ss.main));
    for (int k = 0; k < 5; k++) ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[k], sl.ev_start, 0));
    ACE_TRY(gathered_msm<fp_t>(pl.A, pk->A, d_z, sl.ar[1], res1 + 1, ss.aux[0]));
    // B1 and B2 multiply the same witness values under one plan: B2 takes B1's
    // sorted entries (B1's arena is not reused before this proof ends)
    MsmSorted sortB;
    ACE_TRY(gathered_msm<fp_t>(pl.B, pk->B1, d_z, sl.ar[2], res1 + 2, ss.aux[1], &sortB, sl.ev_sort));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[2], sl.ev_sort, 0));
    ACE_TRY(msm_run<fp2_t>(pl.B, pk->B2.d_pts, true, nullptr, sl.ar[3], res2, nullptr, ss.aux[2], &sortB));
    ACE_TRY(gathered_msm<fp_t>(pl.L, pk->L, d_z, sl.ar[4], res1 + 3, ss.aux[3]));
    if (msm_out) {
        ACE_TRY(qap_run(ctx, pk, d_z, abc, d_status, ss.main, true));
        ACE_TRY(msm_run<fp_t>(pl.H, pk->d_H, true, (const uint32_t*)abc, a0, res1, nullptr, ss.main));
        for (int k = 0; k < 4; k++) {
            ACE_TRY_CUDA(cudaEventRecord(sl.ev_aux[k], ss.aux[k]));
            ACE_TRY_CUDA(cudaStreamWaitEvent(ss.main, sl.ev_aux[k], 0));
        }
        ACE_TRY_CUDA(cudaGetLastError());
        ACE_TRY_CUDA(cudaEventRecord(sl.ev_done, ss.main));
        if (join) ACE_TRY_CUDA(cudaStreamWaitEvent(st_in, sl.ev_done, 0));
        return ACE_OK;
    }
    int pf = prof_begin(PROF_ASSEMBLY, ss.aux[4]);
    k_prove_fixed<<<1, 160, 0, ss.aux[4]>>>(tabs, r, s, rs, fx1, fx2); ::ace::note_launch();
    prof_end(pf, ss.aux[4], nullptr, 1);
    // V = s S_A + r S_B1 once the A and B1 MSMs are done, overlapping the rest
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_aux[0], ss.aux[0]));
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_aux[1], ss.aux[1]));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[4], sl.ev_aux[0], 0));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[4], sl.ev_aux[1], 0));
    int pv = prof_begin(PROF_ASSEMBLY, ss.aux[4]);
    GlvScalars glv;
    if (glv_scalars(r, s, glv)) {
        fp_t beta;
        memcpy(beta.v, GLV_BETA, 32);
        k_prove_var<<<1, 128, 0, ss.aux[4]>>>(res1, glv, fe_to_mont(beta), vterm);
    } else {  // not reached: the split always yields 128-bit halves
        k_prove_var_joint<<<1, 32, 0, ss.aux[4]>>>(res1, r, s, vterm);
    }
    ::ace::note_launch();
    prof_end(pv, ss.aux[4], nullptr, 1);
    ACE_TRY(qap_run(ctx, pk, d_z, abc, d_status, ss.main, true));
    ACE_TRY(msm_run<fp_t>(pl.H, pk->d_H, true, (const uint32_t*)abc, a0, res1, nullptr, ss.main));
    for (int k = 0; k < 5; k++) {
        ACE_TRY_CUDA(cudaEventRecord(sl.ev_aux[k], ss.aux[k]));
        ACE_TRY_CUDA(cudaStreamWaitEvent(ss.main, sl.ev_aux[k], 0));
    }
    int pa = prof_begin(PROF_ASSEMBLY, ss.main);
    k_assemble<<<1, 96, 0, ss.main>>>(pk->d_fixed, res1, res2, fx1, fx2, vterm, d_proof); ::ace::note_launch();
    prof_end(pa, ss.main, nullptr, 1);
    ACE_TRY_CUDA(cudaGetLastError());
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_done, ss.main));
    if (join) ACE_TRY_CUDA(cudaStreamWaitEvent(st_in, sl.ev_done, 0));
    return ACE_OK;
}

// ---- many proofs of one key ---------------------------------------------------
struct ManyPlans {
    MsmPlan H, A, B, L;
    size_t arena[PROVE_ARENAS];
};

static ManyPlans many_plans(const ace_pk* pk, uint32_t count) {
    ManyPlans p;
    p.H = pk->H_plan;
    p.A = pk->A.plan;
    p.B = pk->B1.plan;
    p.L = pk->L.plan;
    for (MsmPlan* q : {&p.H, &p.A, &p.B, &p.L}) msm_plan_set_batch(*q, count);
    const size_t N = pk->N, fr = sizeof(fr_t);
    // arena 0: a, b, c and h of every proof, the H MSM, all per-proof points
    p.arena[0] = 4 * N * count * fr + msm_scratch_bytes<fp_t>(p.H, true) +
                 (size_t)count * (10 * sizeof(g1_xyzz) + 2 * sizeof(g2_xyzz) + 3 * fr) + (1 << 16);
    p.arena[1] = pk->A.count * count * fr + msm_scratch_bytes<fp_t>(p.A, true) + 4096;
    p.arena[2] = pk->B1.count * count * fr + msm_scratch_bytes<fp_t>(p.B, true) + 4096;
    p.arena[3] = pk->B2.count * count * fr + msm_scratch_bytes<fp2_t>(p.B, true) + 4096;
    p.arena[4] = pk->L.count * count * fr + msm_scratch_bytes<fp_t>(p.L, true) + 4096;
    return p;
}

template <class F>
static int gathered_msm_many(const MsmPlan& plan, const Query<F>& q, const fr_t* d_z, uint64_t wit, Arena& ar,
                             Xyzz<F>* res, cudaStream_t s, MsmSorted* sorted = nullptr,
                             cudaEvent_t sorted_ev = nullptr) {
    fr_t* zq = (fr_t*)ar.take((size_t)q.count * plan.batch * sizeof(fr_t) + 32);
    if (!zq) {
        set_error("prove_many: arena too small");
        return ACE_E_OOM;
    }
    if (q.count) {
        dim3 grid((q.count + 255) / 256, plan.batch);
        k_gather_many<<<grid, 256, 0, s>>>(d_z, wit, q.d_idx, q.count, zq);
        ::ace::note_launch();
    }
    return msm_run<F>(plan, q.d_pts, true, (const uint32_t*)zq, ar, res, nullptr, s, nullptr, sorted, sorted_ev);
}

// `count` proofs of pk on proving slot 0 (level 0 streams), after the work on
// st_in; d_z: count witnesses of pk->m values; h_rsv: per proof r, s, r s
// (canonical); proofs and R1CS status to device memory; st_in waits for the end.
static int prove_many_run(ace_ctx* ctx, const ace_pk* pk, uint32_t count, const fr_t* d_z, const fr_t* h_rsv,
                          uint32_t* d_proofs, int32_t* d_status, cudaStream_t st_in) {
    NttPlan* plan = nullptr;
    ACE_TRY(ntt_get_plan(ctx, pk->log_n, &plan));
    ACE_TRY(slot_ready(ctx, 0));
    ProveSlot& sl = ctx->slots[0];
    SlotStreams& ss = sl.lv[0];
    ManyPlans pl = many_plans(pk, count);
    for (int k = 0; k < PROVE_ARENAS; k++) ACE_TRY(slot_arena_ensure(ctx, 0, k, pl.arena[k]));
    for (auto& a : sl.ar) a.reset();
    const uint32_t N = (uint32_t)pk->N;
    const uint64_t wit = pk->m;
    Arena& a0 = sl.ar[0];
    fr_t* abc = (fr_t*)a0.take(3 * (size_t)N * count * sizeof(fr_t));
    fr_t* h = (fr_t*)a0.take((size_t)N * count * sizeof(fr_t));
    g1_xyzz* res1 = (g1_xyzz*)a0.take(4 * (size_t)count * sizeof(g1_xyzz));  // S_H, S_A, S_B1, S_L
    g1_xyzz* fx1 = (g1_xyzz*)a0.take(4 * (size_t)count * sizeof(g1_xyzz));
    g1_xyzz* vterm = (g1_xyzz*)a0.take((size_t)count * sizeof(g1_xyzz));
    g2_xyzz* res2 = (g2_xyzz*)a0.take((size_t)count * sizeof(g2_xyzz));
    g2_xyzz* fx2 = (g2_xyzz*)a0.take((size_t)count * sizeof(g2_xyzz));
    fr_t* rsv = (fr_t*)a0.take(3 * (size_t)count * sizeof(fr_t));
    if (!abc || !h || !res1 || !fx1 || !vterm || !res2 || !fx2 || !rsv) {
        set_error("prove_many: arena too small");
        return ACE_E_OOM;
    }
    PkTabs tabs{pk->d_tab_alpha1, pk->d_tab_beta1, pk->d_tab_delta1, pk->d_tab_delta2};
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_in, st_in));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.main, sl.ev_in, 0));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.main, sl.ev_done, 0));
    ACE_TRY_CUDA(cudaMemcpyAsync(rsv, h_rsv, 3 * (size_t)count * sizeof(fr_t), cudaMemcpyHostToDevice, ss.main));
    ACE_TRY_CUDA(cudaMemsetAsync(d_status, 0, count * sizeof(int32_t), ss.main));
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_start, ss.main));
    for (int k = 0; k < 5; k++) ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[k], sl.ev_start, 0));
    // MSMs over the witness on the auxiliary streams
    ACE_TRY(gathered_msm_many<fp_t>(pl.A, pk->A, d_z, wit, sl.ar[1], res1 + count, ss.aux[0]));
    MsmSorted sortB;  // shared by B1 and B2, as in prove_run
    ACE_TRY(gathered_msm_many<fp_t>(pl.B, pk->B1, d_z, wit, sl.ar[2], res1 + 2 * (size_t)count, ss.aux[1], &sortB,
                                    sl.ev_sort));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[2], sl.ev_sort, 0));
    ACE_TRY(msm_run<fp2_t>(pl.B, pk->B2.d_pts, true, nullptr, sl.ar[3], res2, nullptr, ss.aux[2], &sortB));
    ACE_TRY(gathered_msm_many<fp_t>(pl.L, pk->L, d_z, wit, sl.ar[4], res1 + 3 * (size_t)count, ss.aux[3]));
    k_prove_fixed_many<<<(5 * count + 127) / 128, 128, 0, ss.aux[4]>>>(tabs, rsv, count, fx1, fx2); ::ace::note_launch();
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_aux[0], ss.aux[0]));
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_aux[1], ss.aux[1]));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[4], sl.ev_aux[0], 0));
    ACE_TRY_CUDA(cudaStreamWaitEvent(ss.aux[4], sl.ev_aux[1], 0));
    k_prove_var_many<<<(count + 63) / 64, 64, 0, ss.aux[4]>>>(res1 + count, res1 + 2 * (size_t)count, rsv, count,
                                                              vterm); ::ace::note_launch();
    // QAP of every proof, then the H MSM, on the main stream
    NttScale none, cos;
    cos.hi = plan->cos_hi;
    cos.lo = plan->cos_lo;
    cos.h = plan->h;
    cos.brev = 1;
    int prof = prof_begin(PROF_SPMV, ss.main);
    k_spmv3_many<<<dim3((N + 255) / 256, count), 256, 0, ss.main>>>(csr_of(pk), pk->d_row_order, d_z, wit, N, abc,
                                                                      d_status);
    ::ace::note_launch();
    prof_end(prof, ss.main, nullptr, (pk->nnz[0] + pk->nnz[1] + pk->nnz[2]) * count);
    ACE_TRY(ntt_run(*plan, abc, 3 * (int)count, true, true, none, cos, ss.main));
    ACE_TRY(ntt_run(*plan, abc, 3 * (int)count, false, false, none, none, ss.main));
    // canonical h(g omega^i) of every proof (see qap_run)
    k_quotient_many<<<dim3((N + 255) / 256, count), 256, 0, ss.main>>>(abc, N, fe_from_mont(plan->zinv), h);
    ::ace::note_launch();
    ACE_TRY(msm_run<fp_t>(pl.H, pk->d_H, true, (const uint32_t*)h, a0, res1, nullptr, ss.main));
    for (int k = 0; k < 5; k++) {
        ACE_TRY_CUDA(cudaEventRecord(sl.ev_aux[k], ss.aux[k]));
        ACE_TRY_CUDA(cudaStreamWaitEvent(ss.main, sl.ev_aux[k], 0));
    }
    k_assemble_many<<<(3 * count + 63) / 64, 64, 0, ss.main>>>(pk->d_fixed, res1, res2, fx1, fx2, vterm, count,
                                                               d_proofs); ::ace::note_launch();
    ACE_TRY_CUDA(cudaGetLastError());
    ACE_TRY_CUDA(cudaEventRecord(sl.ev_done, ss.main));
    ACE_TRY_CUDA(cudaStreamWaitEvent(st_in, sl.ev_done, 0));
    return ACE_OK;
}

static bool canonical_fr(const ace_fr* x) {
    fr_t t;
    memcpy(t.v, x->l, 32);
    return !fe_geq_mod(t);
}

}  // namespace ace

using namespace ace;

extern "C" {

int ace_qap_h(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, ace_fr* d_h_out, ace_stream stream) {
    clear_error();
    if (!ctx || !pk || !d_z || !d_h_out) {
        set_error("ace_qap_h: NULL argument");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = pick_stream(ctx, stream);
    ACE_TRY(arena_ensure(ctx, 0, 3 * pk->N * sizeof(fr_t) + 4096));
    fr_t* abc = (fr_t*)ctx->scratch[0].take(3 * pk->N * sizeof(fr_t));
    int32_t* status = (int32_t*)ctx->scratch[0].take(16);
    ACE_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    return qap_run(ctx, pk, (const fr_t*)d_z, abc, status, st, false, (fr_t*)d_h_out);
}

int ace_prove_async(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, const ace_fr* r, const ace_fr* s,
                    uint8_t* d_proof_out, int32_t* d_status, ace_stream stream) {
    clear_error();
    if (!ctx || !pk || !d_z || !r || !s || !d_proof_out || !d_status) {
        set_error("ace_prove_async: NULL argument");
        return ACE_E_ARG;
    }
    if (!canonical_fr(r) || !canonical_fr(s)) {
        set_error("ace_prove: r and s must be canonical Fr values");
        return ACE_E_ARG;
    }
    if (((uintptr_t)d_z & 15u) || ((uintptr_t)d_proof_out & 3u) || ((uintptr_t)d_status & 3u)) {
        set_error("ace_prove: d_z must be 16-byte aligned, outputs 4-byte aligned");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    fr_t rr, ss;
    memcpy(rr.v, r->l, 32);
    memcpy(ss.v, s->l, 32);
    return prove_run(ctx, 0, 0, pk, (const fr_t*)d_z, rr, ss, (uint32_t*)d_proof_out, d_status,
                     pick_stream(ctx, stream), true, nullptr, false, true);
}

int ace_prove(ace_ctx* ctx, const ace_pk* pk, const ace_fr* d_z, const ace_fr* r, const ace_fr* s,
              uint8_t proof_out[256], ace_stream stream) {
    clear_error();
    if (!proof_out) {
        set_error("ace_prove: proof_out is NULL");
        return ACE_E_ARG;
    }
    if (!ctx) {
        set_error("ace_prove: NULL context");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    // proof and status words in a scratch arena of their own
    ACE_TRY(arena_ensure(ctx, 3, 512));
    uint8_t* d_out = (uint8_t*)ctx->scratch[3].take(256);
    int32_t* d_status = (int32_t*)ctx->scratch[3].take(16);
    cudaStream_t st = pick_stream(ctx, stream);
    ACE_TRY(ace_prove_async(ctx, pk, d_z, r, s, d_out, d_status, stream));
    int32_t status = 0;
    ACE_TRY_CUDA(cudaMemcpyAsync(proof_out, d_out, 256, cudaMemcpyDeviceToHost, st));
    ACE_TRY_CUDA(cudaMemcpyAsync(&status, d_status, sizeof status, cudaMemcpyDeviceToHost, st));
    ACE_TRY_CUDA(cudaStreamSynchronize(st));
    if (status) {
        set_error("ace_prove: witness does not satisfy the R1CS");
        return ACE_E_UNSAT;
    }
    return ACE_OK;
}

}  // extern "C"

namespace ace {
static int prove_many_impl(ace_ctx* ctx, const ace_pk* pk, size_t k, const ace_fr* d_z, const ace_fr* rs,
                           const ace_fr* ss, uint8_t* proofs, int32_t* status) {
    if (!ctx || !pk || (k && (!d_z || !rs || !ss || !proofs || !status))) {
        set_error("ace_prove_many: NULL argument");
        return ACE_E_ARG;
    }
    if (k == 0) return ACE_OK;
    if ((uintptr_t)d_z & 15u) {
        set_error("ace_prove_many: d_z must be 16-byte aligned");
        return ACE_E_ARG;
    }
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    std::vector<fr_t> rsv(3 * k);
    for (size_t i = 0; i < k; i++) {
        if (!canonical_fr(rs + i) || !canonical_fr(ss + i)) {
            set_error("ace_prove_many: r and s of proof %zu must be canonical Fr values", i);
            return ACE_E_ARG;
        }
        memcpy(rsv[3 * i].v, rs[i].l, 32);
        memcpy(rsv[3 * i + 1].v, ss[i].l, 32);
        rsv[3 * i + 2] = fe_from_mont(fe_to_mont(rsv[3 * i]) * fe_to_mont(rsv[3 * i + 1]));
    }
    // chunks of proofs whose scratch stays within MANY_SCRATCH bytes (one
    // proof per chunk at least); 65535 bounds the grid's y dimension / 3
    const size_t MANY_SCRATCH = (size_t)24 << 30;
    ManyPlans one = many_plans(pk, 1);
    size_t per = 0;
    for (int a = 0; a < PROVE_ARENAS; a++) per += one.arena[a];
    size_t chunk = MANY_SCRATCH / (per ? per : 1);
    // entries (count n K) and keys (count windows 2^(c-1)) are 32-bit indices
    size_t ent = 1, keys = 1;
    for (const MsmPlan* q : {&one.H, &one.A, &one.B, &one.L}) {
        ent = ent > q->n * (size_t)q->K ? ent : q->n * (size_t)q->K;
        keys = keys > (size_t)q->keys_per() ? keys : (size_t)q->keys_per();
    }
    if (chunk > ((size_t)1 << 31) / ent) chunk = ((size_t)1 << 31) / ent;
    if (chunk > ((size_t)1 << 31) / keys) chunk = ((size_t)1 << 31) / keys;
    if (chunk < 1) chunk = 1;
    if (chunk > 21845) chunk = 21845;
    // ACE_MANY_MAX_CHUNK (environment): a smaller cap, e.g. to bound latency
    // per chunk or to exercise the chunk loop
    if (const char* env = getenv("ACE_MANY_MAX_CHUNK")) {
        long v = strtol(env, nullptr, 10);
        if (v >= 1 && (size_t)v < chunk) chunk = (size_t)v;
    }
    if (chunk > k) chunk = k;
    ACE_TRY(arena_ensure(ctx, 3, chunk * (256 + sizeof(int32_t)) + 1024));
    ctx->scratch[3].reset();
    uint32_t* d_proofs = (uint32_t*)ctx->scratch[3].take(chunk * 256);
    int32_t* d_status = (int32_t*)ctx->scratch[3].take(chunk * sizeof(int32_t));
    cudaStream_t st = ctx->stream;
    for (size_t b = 0; b < k; b += chunk) {
        uint32_t c = (uint32_t)(k - b < chunk ? k - b : chunk);
        ACE_TRY(prove_many_run(ctx, pk, c, (const fr_t*)d_z + b * pk->m, rsv.data() + 3 * b, d_proofs, d_status, st));
        ACE_TRY_CUDA(cudaMemcpyAsync(proofs + 256 * b, d_proofs, (size_t)c * 256, cudaMemcpyDeviceToHost, st));
        ACE_TRY_CUDA(cudaMemcpyAsync(status + b, d_status, (size_t)c * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        // the next chunk reuses the device outputs and the host r, s copy
        ACE_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return ACE_OK;
}

// A batch of at least MANY_MIN_PROOFS proofs of one key with N <= 2^MANY_MAX_LOG_N
// runs on the batch-dimension kernels of ace_prove_many (one launch per stage
// for all of its proofs): measured on 64 proofs of one key, 3.3x / 2.6x /
// 1.5x / 1.15x / 1.04x the slot pipelining at 2^10 / 12 / 14 / 16 / 18 rows,
// equal at 2^20 (where the slots are kept).  The witnesses are copied into
// one contiguous staging buffer first (host or device sources), in chunks of
// at most 2 GB.
static const size_t MANY_MIN_PROOFS = 8;
static const int MANY_MAX_LOG_N = 18;

static int prove_batch_as_many(ace_ctx* ctx, size_t k, const ace_pk* pk, const ace_fr* const* zs, bool host,
                               const ace_fr* rs, const ace_fr* ss, uint8_t* proofs, int32_t* status) {
    const size_t wb = pk->m * sizeof(fr_t);
    size_t chunk = ((size_t)2 << 30) / (wb ? wb : 1);
    if (chunk < 1) chunk = 1;
    if (chunk > k) chunk = k;
    ACE_TRY(slot_ready(ctx, 0));
    ACE_TRY(slot_witness_ensure(ctx, 0, chunk * wb));
    char* stage = ctx->slots[0].wit.base;
    cudaStream_t st = ctx->stream;
    for (size_t b = 0; b < k; b += chunk) {
        const size_t c = k - b < chunk ? k - b : chunk;
        for (size_t i = 0; i < c; i++)
            ACE_TRY_CUDA(cudaMemcpyAsync(stage + i * wb, zs[b + i], wb,
                                         host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
        // ordered after the copies on st; synchronises st before returning
        ACE_TRY(prove_many_impl(ctx, pk, c, (const ace_fr*)stage, rs + b, ss + b, proofs + 256 * b, status + b));
    }
    return ACE_OK;
}

// k proofs round-robin over the context's proving slots (consecutive proofs
// overlap); zs are device witnesses, or host witnesses (host = true) that are
// copied into the slot's staging buffer on the slot's main stream once the
// slot's previous proof is done.  The slots' scratch is sized for their
// largest proof up front, so no arena grows (and synchronises the device) in
// the middle of the batch.
static int prove_batch_impl(ace_ctx* ctx, const char* fn, size_t k, const ace_pk* const* pks,
                            const ace_fr* const* zs, bool host, const ace_fr* rs, const ace_fr* ss, uint8_t* proofs,
                            int32_t* status, bool allow_many = true) {
    if (!ctx || (k && (!pks || !zs || !rs || !ss || !proofs || !status))) {
        set_error("%s: NULL argument", fn);
        return ACE_E_ARG;
    }
    if (k == 0) return ACE_OK;
    ACE_TRY_CUDA(cudaSetDevice(ctx->device));
    for (size_t i = 0; i < k; i++) {
        if (!pks[i] || !zs[i] || !canonical_fr(rs + i) || !canonical_fr(ss + i)) {
            set_error("%s: proof %zu has a NULL key / witness or non-canonical r, s", fn, i);
            return ACE_E_ARG;
        }
    }
    bool one_key = allow_many && k >= MANY_MIN_PROOFS && pks[0]->log_n <= MANY_MAX_LOG_N;
    for (size_t i = 1; one_key && i < k; i++) one_key = pks[i] == pks[0];
    if (one_key) return prove_batch_as_many(ctx, k, pks[0], zs, host, rs, ss, proofs, status);
    // device outputs for all proofs (then one copy back), the proofs' MSM
    // sums and tail terms, and the tails' per-proof descriptors
    const size_t per = 256 + sizeof(int32_t) + 9 * sizeof(g1_xyzz) + 2 * sizeof(g2_xyzz) + sizeof(TailDesc);
    ACE_TRY(arena_ensure(ctx, 3, k * per + 8 * 1024));
    Arena& sc = ctx->scratch[3];
    uint32_t* d_proofs = (uint32_t*)sc.take(k * 256);
    int32_t* d_status = (int32_t*)sc.take(k * sizeof(int32_t));
    g1_xyzz* res1 = (g1_xyzz*)sc.take(4 * k * sizeof(g1_xyzz));
    g1_xyzz* fx1 = (g1_xyzz*)sc.take(4 * k * sizeof(g1_xyzz));
    g1_xyzz* vterm = (g1_xyzz*)sc.take(k * sizeof(g1_xyzz));
    g2_xyzz* res2 = (g2_xyzz*)sc.take(k * sizeof(g2_xyzz));
    g2_xyzz* fx2 = (g2_xyzz*)sc.take(k * sizeof(g2_xyzz));
    TailDesc* d_desc = (TailDesc*)sc.take(k * sizeof(TailDesc));
    if (!d_proofs || !d_status || !res1 || !fx1 || !vterm || !res2 || !fx2 || !d_desc) {
        set_error("%s: scratch arena too small", fn);
        return ACE_E_OOM;
    }
    std::vector<TailDesc> desc(k);
    for (size_t i = 0; i < k; i++) {
        TailDesc& d = desc[i];
        const ace_pk* pk = pks[i];
        d.tabs = PkTabs{pk->d_tab_alpha1, pk->d_tab_beta1, pk->d_tab_delta1, pk->d_tab_delta2};
        d.fixed = pk->d_fixed;
        memcpy(d.r.v, rs[i].l, 32);
        memcpy(d.s.v, ss[i].l, 32);
        d.rs = fe_from_mont(fe_to_mont(d.r) * fe_to_mont(d.s));
        d.glv_ok = glv_scalars(d.r, d.s, d.glv);
    }
    cudaStream_t st = ctx->stream;
    int nslots = (int)(k < (size_t)ctx->batch_slots ? k : (size_t)ctx->batch_slots);
    for (int q = 0; q < nslots; q++) {
        size_t need[PROVE_ARENAS] = {0, 0, 0, 0, 0};
        size_t wit = 0;
        for (size_t i = q; i < k; i += nslots) {
            ProvePlans pl = prove_plans(pks[i]);
            for (int a = 0; a < PROVE_ARENAS; a++) need[a] = need[a] > pl.slot_bytes[a] ? need[a] : pl.slot_bytes[a];
            wit = wit > pks[i]->m * sizeof(fr_t) ? wit : pks[i]->m * sizeof(fr_t);
        }
        ACE_TRY(slot_ready(ctx, q));
        for (int a = 0; a < PROVE_ARENAS; a++) ACE_TRY(slot_arena_ensure(ctx, q, a, need[a]));
        if (host) ACE_TRY(slot_witness_ensure(ctx, q, wit));
    }
    // With more proofs than slots the tails are batched: the fixed-base terms
    // of every proof in one launch, on slot 0's fifth auxiliary stream (unused
    // by proofs whose tails are batched), beside the proofs' MSMs, and V and
    // the assembly in one launch each at the end.  With at most one proof per
    // slot each proof keeps its own tail, which starts as soon as its own
    // MSMs allow (lower latency for a lone proof).
    const bool batched_tails = k > (size_t)nslots;
    ProveSlot& s0 = ctx->slots[0];
    cudaStream_t tail = s0.lv[0].aux[4];
    if (batched_tails) {
        ACE_TRY_CUDA(cudaMemcpyAsync(d_desc, desc.data(), k * sizeof(TailDesc), cudaMemcpyHostToDevice, st));
        ACE_TRY_CUDA(cudaEventRecord(s0.ev_aux[4], st));
        ACE_TRY_CUDA(cudaStreamWaitEvent(tail, s0.ev_aux[4], 0));
        int pf = prof_begin(PROF_ASSEMBLY, tail);
        k_prove_fixed_batch<<<(unsigned)k, 160, 0, tail>>>(d_desc, fx1, fx2); ::ace::note_launch();
        prof_end(pf, tail, nullptr, k);
        ACE_TRY_CUDA(cudaGetLastError());
    }
    for (size_t i = 0; i < k; i++) {
        const fr_t& rr = desc[i].r;
        const fr_t& sv = desc[i].s;
        const int q = (int)(i % nslots);
        const fr_t* z = (const fr_t*)zs[i];
        cudaStream_t st_in = st;
        if (host) {
            ProveSlot& sl = ctx->slots[q];
            st_in = sl.lv[0].main;
            fr_t* stage = (fr_t*)sl.wit.base;
            // the slot's previous proof may still read the staging buffer
            ACE_TRY_CUDA(cudaStreamWaitEvent(st_in, sl.ev_done, 0));
            ACE_TRY_CUDA(cudaMemcpyAsync(stage, z, pks[i]->m * sizeof(fr_t), cudaMemcpyHostToDevice, st_in));
            z = stage;
        }
        MsmOut mo{res1 + 4 * i, res2 + i};
        // a batch of one proof has the GPU to itself: it runs as ace_prove does
        const bool lone = k == 1;
        ACE_TRY(prove_run(ctx, q, 0, pks[i], z, rr, sv, d_proofs + 64 * i, d_status + i, st_in, false,
                          batched_tails ? &mo : nullptr, lone ? false : ctx->batch_one_stream, lone));
    }
    for (int q = 0; q < nslots; q++) ACE_TRY_CUDA(cudaStreamWaitEvent(st, ctx->slots[q].ev_done, 0));
    if (batched_tails) {
        // V and the assembly of every proof once all MSMs and fixed terms are done
        ACE_TRY_CUDA(cudaEventRecord(s0.ev_aux[4], tail));
        ACE_TRY_CUDA(cudaStreamWaitEvent(st, s0.ev_aux[4], 0));
        fp_t beta;
        memcpy(beta.v, GLV_BETA, 32);
        int pv = prof_begin(PROF_ASSEMBLY, st);
        k_prove_var_batch<<<(unsigned)k, 128, 0, st>>>(d_desc, res1, fe_to_mont(beta), vterm); ::ace::note_launch();
        k_assemble_batch<<<(unsigned)k, 96, 0, st>>>(d_desc, res1, res2, fx1, fx2, vterm, d_proofs);
        ::ace::note_launch();
        prof_end(pv, st, nullptr, k);
        ACE_TRY_CUDA(cudaGetLastError());
    }
    ACE_TRY_CUDA(cudaMemcpyAsync(proofs, d_proofs, k * 256, cudaMemcpyDeviceToHost, st));
    ACE_TRY_CUDA(cudaMemcpyAsync(status, d_status, k * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    ACE_TRY_CUDA(cudaStreamSynchronize(st));
    return ACE_OK;
}
// the slot path of ace_prove_batch whatever the keys (the batch autotuner
// times slot counts and layouts with it)
int prove_batch_on_slots(ace_ctx* ctx, size_t k, const ace_pk* const* pks, const ace_fr* const* d_zs,
                         const ace_fr* rs, const ace_fr* ss, uint8_t* proofs, int32_t* status) {
    return prove_batch_impl(ctx, "ace_autotune_batch_slots", k, pks, d_zs, false, rs, ss, proofs, status, false);
}
}  // namespace ace

extern "C" {

int ace_prove_batch(ace_ctx* ctx, size_t k, const ace_pk* const* pks, const ace_fr* const* d_zs, const ace_fr* rs,
                    const ace_fr* ss, uint8_t* proofs, int32_t* status) {
    clear_error();
    return prove_batch_impl(ctx, "ace_prove_batch", k, pks, d_zs, false, rs, ss, proofs, status);
}

int ace_prove_batch_host(ace_ctx* ctx, size_t k, const ace_pk* const* pks, const ace_fr* const* h_zs,
                         const ace_fr* rs, const ace_fr* ss, uint8_t* proofs, int32_t* status) {
    clear_error();
    return prove_batch_impl(ctx, "ace_prove_batch_host", k, pks, h_zs, true, rs, ss, proofs, status);
}

int ace_debug_glv_split(const ace_fr* k, uint32_t out[10]) {
    if (!k || !out) return ACE_E_ARG;
    fr_t x;
    memcpy(x.v, k->l, 32);
    if (fe_geq_mod(x)) return ACE_E_ARG;
    return glv_split(x, out, &out[4], out + 5, &out[9]) ? ACE_OK : ACE_E_ARG;
}

int ace_debug_gls_split(const ace_fr* k, uint32_t out[16]) {
    if (!k || !out) return ACE_E_ARG;
    fr_t x;
    memcpy(x.v, k->l, 32);
    if (fe_geq_mod(x)) return ACE_E_ARG;
    uint32_t mag[4][3], neg[4];
    if (!gls_split_limbs(x.v, mag, neg)) return ACE_E_INTERNAL;
    for (int i = 0; i < 4; i++) {
        for (int l = 0; l < 3; l++) out[4 * i + l] = mag[i][l];
        out[4 * i + 3] = neg[i];
    }
    return ACE_OK;
}

int ace_debug_wnaf5(const uint32_t k[4], int8_t out[132]) {
    static_assert(GLV_NAF_LEN == 132, "the declared digit count");
    if (!k || !out) return ACE_E_ARG;
    return wnaf5(k, out) ? ACE_OK : ACE_E_INTERNAL;
}

int ace_prove_many(ace_ctx* ctx, const ace_pk* pk, size_t k, const ace_fr* d_z, const ace_fr* rs, const ace_fr* ss,
                   uint8_t* proofs, int32_t* status) {
    clear_error();
    return prove_many_impl(ctx, pk, k, d_z, rs, ss, proofs, status);
}

}  // extern "C"
