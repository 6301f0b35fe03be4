// glv.cuh -- scalar decomposition for the GLV endomorphism of G1 (Gallant,
// Lambert and Vanstone, Crypto 2001), on the host and on the device.
//
// beta: a cube root of unity in Fp with (beta x, y) = lambda (x, y) on G1,
// lambda = 0xb3c4d79d41a917585bfc41088d8daaa78b17ea66b99c90dd (a cube root of
// unity mod r).  (a1, b1), (a2, b2): a reduced basis of the lattice
// {(a, b) : a + b lambda = 0 mod r} (b1 < 0, stored as |b1|); G1 = round(b2
// 2^256 / r), G2 = round(|b1| 2^256 / r).  c1 = (k G1) >> 256, c2 = (k G2) >>
// 256, k1 = k - c1 a1 - c2 a2, k2 = c1 |b1| - c2 b2, so k = k1 + k2 lambda
// (mod r).  For 0 <= k < r the roundings leave |c_i - exact| < 1.01, so
// |k1| < 1.01 (a1 + a2) < 2^127 and |k2| < 1.01 (|b1| + b2) < 2^127.
//
// The prover uses it for s S_A + r S_B1; the G1 MSM without window tables
// splits every scalar into two halves over the points P_i and phi(P_i), which
// halves the windows (and with them the bucket reduction and the Horner
// chain of doublings) for the same number of bucket additions.
#pragma once
#include "field.cuh"

namespace ace {

#define ACE_GLV_BETA {0x77fffffeu, 0x57634731u, 0xacdb5c4fu, 0xd4f263f1u, 0xa0d48bacu, 0x59e26bceu, 0u, 0u}
#define ACE_GLV_A1 {0x94d213e3u, 0x89d32568u}
#define ACE_GLV_B1 {0x7d4f1128u, 0x8211bbebu, 0xeeb859fcu, 0x6f4d8248u}
#define ACE_GLV_A2 {0x1221250bu, 0x0be4e154u, 0xeeb859fdu, 0x6f4d8248u}
#define ACE_GLV_B2 {0x94d213e3u, 0x89d32568u}
#define ACE_GLV_G1 {0xc7e0b3d7u, 0xd91d232eu, 0x00000002u}
#define ACE_GLV_G2 {0x391eb18eu, 0x7a7bd9d4u, 0xa773d2cfu, 0x4ccef014u, 0x00000002u}

// out (na + nb limbs) = a b
ACE_HD void glv_mp_mul(const uint32_t* a, int na, const uint32_t* b, int nb, uint32_t* out) {
    for (int i = 0; i < na + nb; i++) out[i] = 0;
    for (int i = 0; i < na; i++) {
        uint64_t c = 0;
        for (int j = 0; j < nb; j++) {
            c += (uint64_t)out[i + j] + (uint64_t)a[i] * b[j];
            out[i + j] = (uint32_t)c;
            c >>= 32;
        }
        out[i + nb] = (uint32_t)c;
    }
}
// x -= y (8 limbs, modulo 2^256); y has ny <= 8 limbs
ACE_HD void glv_mp_sub8(uint32_t* x, const uint32_t* y, int ny) {
    uint32_t br = 0;
    for (int i = 0; i < 8; i++) {
        const uint64_t d = (uint64_t)x[i] - (i < ny ? y[i] : 0u) - br;
        x[i] = (uint32_t)d;
        br = (uint32_t)(d >> 63);
    }
}
// a two's-complement 256-bit value of magnitude < 2^128 to (magnitude, sign)
ACE_HD bool glv_half(const uint32_t* x, uint32_t mag[4], uint32_t* neg) {
    uint32_t t[8];
    *neg = x[7] >> 31;
    for (int i = 0; i < 8; i++) t[i] = *neg ? ~x[i] : x[i];
    if (*neg) {
        for (int i = 0; i < 8; i++)
            if (++t[i] != 0) break;
    }
    for (int i = 4; i < 8; i++)
        if (t[i]) return false;
    for (int i = 0; i < 4; i++) mag[i] = t[i];
    return true;
}
// k (8 limbs, 0 <= k < r) -> |k1|, sign(k1), |k2|, sign(k2)
ACE_HD bool glv_split_limbs(const uint32_t k[8], uint32_t k1[4], uint32_t* n1, uint32_t k2[4], uint32_t* n2) {
    const uint32_t A1[2] = ACE_GLV_A1, B1[4] = ACE_GLV_B1, A2[4] = ACE_GLV_A2, B2[2] = ACE_GLV_B2;
    const uint32_t G1[3] = ACE_GLV_G1, G2[5] = ACE_GLV_G2;
    uint32_t p1[11], p2[13], t[9], x1[8], x2[8];
    glv_mp_mul(k, 8, G1, 3, p1);
    glv_mp_mul(k, 8, G2, 5, p2);
    const uint32_t* c1 = p1 + 8;  // 3 limbs
    const uint32_t* c2 = p2 + 8;  // 5 limbs
    for (int i = 0; i < 8; i++) x1[i] = k[i];
    glv_mp_mul(c1, 3, A1, 2, t);
    glv_mp_sub8(x1, t, 5);
    glv_mp_mul(c2, 5, A2, 4, t);
    glv_mp_sub8(x1, t, 8);
    glv_mp_mul(c1, 3, B1, 4, t);
    for (int i = 0; i < 8; i++) x2[i] = i < 7 ? t[i] : 0;
    glv_mp_mul(c2, 5, B2, 2, t);
    glv_mp_sub8(x2, t, 7);
    return glv_half(x1, k1, n1) && glv_half(x2, k2, n2);
}

// ---------------------------------------------------------------------------
// Four-dimensional split for the endomorphism psi of G2 (Galbraith, Lin and
// Scott, Eurocrypt 2009).  psi(x, y) = (conj(x) gx, conj(y) gy) with gx =
// xi^((p-1)/3), gy = xi^((p-1)/2), xi = 9 + u, is the Frobenius map carried to
// the twist; on G2 it is multiplication by lambda = p mod r = 6 x^2 (x the BN
// parameter 4965661367192848881).  k = k0 + k1 lambda + k2 lambda^2 + k3
// lambda^3 (mod r) with |k_i| < 2^66: the rows of a reduced basis of the
// lattice {v : v0 + v1 lambda + v2 lambda^2 + v3 lambda^3 = 0 mod r}
// (determinant -r, entries 0, 1, x, x + 1, 2x, 2x + 1) are
//   b0 = (2x + 1, 0, 2x, 1),          b1 = (2x, x + 1, -x, x),
//   b2 = (x + 1, x, x, -2x),          b3 = (2x + 1, -x, -(x + 1), -x),
// and (k, 0, 0, 0) = sum_j c_j b_j for rational c_j = k a_j / det, with a_j the
// first row of the adjugate.  With G_j = round(a_j 2^256 / det) (all
// positive), c_j = (k G_j) >> 256 is within 1.125 of the exact value (the
// rounding of G_j moves it by less than k 2^-257 < 1/8, the floor by less
// than 1), so v = (k, 0, 0, 0) - sum_j c_j b_j satisfies
// sum_i v_i lambda^i = k (mod r) and |v_i| < 1.125 sum_j |b_j[i]| <=
// 1.125 (7 x + 3) < 2^66.
#define ACE_GLS_GX0 {0x176f553du, 0x99e39557u, 0xc2c3330cu, 0xb78cc310u, 0xf559b143u, 0x4c0bec3cu, 0x4f7911f7u, 0x2fb34798u}
#define ACE_GLS_GX1 {0x640fcba2u, 0x1665d51cu, 0x0b7c9dceu, 0x32ae2a1du, 0xd75a0794u, 0x4ba4cc8bu, 0x61ebae20u, 0x16c9e550u}
#define ACE_GLS_GY0 {0x71a0135au, 0xdc540146u, 0xa9c95998u, 0xdbaae0edu, 0xb6e2f9b9u, 0xdc5ec698u, 0x489af5dcu, 0x063cf305u}
#define ACE_GLS_GY1 {0x2623b0e3u, 0x82d37f63u, 0x8fa25bd2u, 0x21807dc9u, 0xec796f2bu, 0x0704b5a7u, 0xac41049au, 0x07c03cbcu}
// G_0 .. G_3 (6 limbs each)
#define ACE_GLS_G                                                                                            \
    {{0x32e42728u, 0x2dff2915u, 0xa3e5577fu, 0x55b4ca7bu, 0xb0d92b95u, 0x9e80318au},                          \
     {0x95d51bb1u, 0x46f4bda9u, 0xfc7184aeu, 0x08e5da66u, 0xb0d92b93u, 0x9e80318au},                          \
     {0xc7e0b3d7u, 0xd91d232eu, 0x00000002u, 0x00000000u, 0x00000000u, 0x00000000u},                          \
     {0xcef3cd3fu, 0xc170977du, 0xa3e5577du, 0x55b4ca7bu, 0xb0d92b95u, 0x9e80318au}}
#define ACE_GLS_X 4965661367192848881ull

// x (8 limbs) += (neg ? -1 : 1) a b  (mod 2^256); a: 6 limbs, b < 2^64
ACE_HD void gls_mp_madd8(uint32_t* x, const uint32_t* a, uint64_t b, bool neg) {
    const uint32_t bl[2] = {(uint32_t)b, (uint32_t)(b >> 32)};
    uint32_t t[8];
    glv_mp_mul(a, 6, bl, 2, t);
    uint64_t c = 0;
    for (int i = 0; i < 8; i++) {
        const uint64_t v = neg ? (uint64_t)x[i] - t[i] - c : (uint64_t)x[i] + t[i] + c;
        x[i] = (uint32_t)v;
        c = neg ? (uint32_t)(v >> 63) : (uint32_t)(v >> 32);
    }
}
// a two's-complement 256-bit value of magnitude < 2^96 to (magnitude, sign)
ACE_HD bool gls_part(const uint32_t* x, uint32_t mag[3], uint32_t* neg) {
    uint32_t t[8];
    *neg = x[7] >> 31;
    for (int i = 0; i < 8; i++) t[i] = *neg ? ~x[i] : x[i];
    if (*neg) {
        for (int i = 0; i < 8; i++)
            if (++t[i] != 0) break;
    }
    for (int i = 3; i < 8; i++)
        if (t[i]) return false;
    for (int i = 0; i < 3; i++) mag[i] = t[i];
    return true;
}
// k (8 limbs, 0 <= k < r) -> |k_i| (3 limbs each, below 2^66) and sign(k_i)
ACE_HD bool gls_split_limbs(const uint32_t k[8], uint32_t mag[4][3], uint32_t neg[4]) {
    const uint32_t G[4][6] = ACE_GLS_G;
    const uint64_t X = ACE_GLS_X;
    // |b_j[i]| and whether b_j[i] < 0
    const uint64_t bm[4][4] = {{2 * X + 1, 0, 2 * X, 1},
                               {2 * X, X + 1, X, X},
                               {X + 1, X, X, 2 * X},
                               {2 * X + 1, X, X + 1, X}};
    const bool bn[4][4] = {{false, false, false, false},
                           {false, false, true, false},
                           {false, false, false, true},
                           {false, true, true, true}};
    uint32_t v[4][8];
    for (int i = 0; i < 4; i++)
        for (int l = 0; l < 8; l++) v[i][l] = i == 0 ? k[l] : 0u;
    for (int j = 0; j < 4; j++) {
        uint32_t p[14];
        glv_mp_mul(k, 8, G[j], 6, p);
        const uint32_t* c = p + 8;  // (k G_j) >> 256: 6 limbs
        for (int i = 0; i < 4; i++)
            if (bm[j][i]) gls_mp_madd8(v[i], c, bm[j][i], !bn[j][i]);  // v_i -= c_j b_j[i]
    }
    bool ok = true;
    for (int i = 0; i < 4; i++) ok = gls_part(v[i], mag[i], &neg[i]) && ok;
    return ok;
}

}  // namespace ace
