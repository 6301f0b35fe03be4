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

}  // namespace ace
