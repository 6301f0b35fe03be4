// field.cuh -- BN254 base field Fp, scalar field Fr and Fp2 = Fp[u]/(u^2+1).
//
// Elements are 8 little-endian 32-bit limbs held in registers, in Montgomery
// form (x * 2^256 mod m) unless a name says otherwise.  Multiplication is the
// coarsely integrated operand-scanning Montgomery product (Montgomery 1985;
// Koc, Acar and Kaliski 1996) written with PTX multiply-add carry chains on the
// device and with 64-bit products on the host.  Both moduli are below 2^254,
// so a + b of reduced inputs never overflows 256 bits and the running CIOS
// value stays below 2p; one conditional subtraction yields the reduced result.
//
// The curves and the fields are those of BN254, the curve the paper's circuit
// operates over (Section 3.3, "ZK-ACE circuit specification").
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define ACE_HD __host__ __device__ __forceinline__
#define ACE_DEV __device__ __forceinline__
#else
#define ACE_HD inline
#define ACE_DEV inline
#endif

namespace ace {

// p = 21888242871839275222246405745257275088696311157297823662689037894645226208583
struct FpCfg {
    static constexpr uint32_t M0 = 0xd87cfd47u, M1 = 0x3c208c16u, M2 = 0x6871ca8du, M3 = 0x97816a91u,
                              M4 = 0x8181585du, M5 = 0xb85045b6u, M6 = 0xe131a029u, M7 = 0x30644e72u;
    static constexpr uint32_t INV = 0xe4866389u;  // -p^{-1} mod 2^32
    static constexpr uint64_t INV64 = 0x87d20782e4866389ull;  // -p^{-1} mod 2^64
    static constexpr uint32_t ONE0 = 0xc58f0d9du, ONE1 = 0xd35d438du, ONE2 = 0xf5c70b3du, ONE3 = 0x0a78eb28u,
                              ONE4 = 0x7879462cu, ONE5 = 0x666ea36fu, ONE6 = 0x9a07df2fu, ONE7 = 0x0e0a77c1u;
    static constexpr uint32_t RR0 = 0x538afa89u, RR1 = 0xf32cfc5bu, RR2 = 0xd44501fbu, RR3 = 0xb5e71911u,
                              RR4 = 0x0a417ff6u, RR5 = 0x47ab1effu, RR6 = 0xcab8351fu, RR7 = 0x06d89f71u;
};
// r = 21888242871839275222246405745257275088548364400416034343698204186575808495617
struct FrCfg {
    static constexpr uint32_t M0 = 0xf0000001u, M1 = 0x43e1f593u, M2 = 0x79b97091u, M3 = 0x2833e848u,
                              M4 = 0x8181585du, M5 = 0xb85045b6u, M6 = 0xe131a029u, M7 = 0x30644e72u;
    static constexpr uint32_t INV = 0xefffffffu;  // -r^{-1} mod 2^32
    static constexpr uint64_t INV64 = 0xc2e1f593efffffffull;  // -r^{-1} mod 2^64
    static constexpr uint32_t ONE0 = 0x4ffffffbu, ONE1 = 0xac96341cu, ONE2 = 0x9f60cd29u, ONE3 = 0x36fc7695u,
                              ONE4 = 0x7879462eu, ONE5 = 0x666ea36fu, ONE6 = 0x9a07df2fu, ONE7 = 0x0e0a77c1u;
    static constexpr uint32_t RR0 = 0xae216da7u, RR1 = 0x1bb8e645u, RR2 = 0xe35c59e3u, RR3 = 0x53fe3ab1u,
                              RR4 = 0x53bb8085u, RR5 = 0x8c49833du, RR6 = 0x7f4e44a5u, RR7 = 0x0216d0b1u;
};

template <class C>
ACE_HD constexpr uint32_t mod_limb(int i) {
    return i == 0 ? C::M0 : i == 1 ? C::M1 : i == 2 ? C::M2 : i == 3 ? C::M3
         : i == 4 ? C::M4 : i == 5 ? C::M5 : i == 6 ? C::M6 : C::M7;
}
template <class C>
ACE_HD constexpr uint32_t one_limb(int i) {
    return i == 0 ? C::ONE0 : i == 1 ? C::ONE1 : i == 2 ? C::ONE2 : i == 3 ? C::ONE3
         : i == 4 ? C::ONE4 : i == 5 ? C::ONE5 : i == 6 ? C::ONE6 : C::ONE7;
}
template <class C>
ACE_HD constexpr uint32_t rr_limb(int i) {
    return i == 0 ? C::RR0 : i == 1 ? C::RR1 : i == 2 ? C::RR2 : i == 3 ? C::RR3
         : i == 4 ? C::RR4 : i == 5 ? C::RR5 : i == 6 ? C::RR6 : C::RR7;
}

template <class C>
struct Fe {
    uint32_t v[8];
};
typedef Fe<FpCfg> fp_t;
typedef Fe<FrCfg> fr_t;

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
template <class C>
ACE_HD Fe<C> fe_zero() {
    Fe<C> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = 0;
    return r;
}
template <class C>
ACE_HD Fe<C> fe_one() {  // Montgomery form of 1
    Fe<C> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = one_limb<C>(i);
    return r;
}
template <class C>
ACE_HD Fe<C> fe_rr() {  // R^2 mod m
    Fe<C> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = rr_limb<C>(i);
    return r;
}

template <class C>
ACE_HD bool fe_is_zero(const Fe<C>& a) {
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) t |= a.v[i];
    return t == 0;
}
template <class C>
ACE_HD bool fe_eq(const Fe<C>& a, const Fe<C>& b) {
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) t |= a.v[i] ^ b.v[i];
    return t == 0;
}
// a >= m for a canonical-candidate value (used to validate inputs)
template <class C>
ACE_HD bool fe_geq_mod(const Fe<C>& a) {
#pragma unroll
    for (int i = 7; i >= 0; i--) {
        if (a.v[i] > mod_limb<C>(i)) return true;
        if (a.v[i] < mod_limb<C>(i)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// host (portable) arithmetic
// ---------------------------------------------------------------------------
template <class C>
inline void h_add(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t t[8], d[8];
    uint64_t c = 0;
    for (int i = 0; i < 8; i++) { c += (uint64_t)a[i] + b[i]; t[i] = (uint32_t)c; c >>= 32; }
    int64_t br = 0;
    for (int i = 0; i < 8; i++) {
        int64_t x = (int64_t)t[i] - mod_limb<C>(i) + br;
        d[i] = (uint32_t)x;
        br = x < 0 ? -1 : 0;
    }
    bool keep = br != 0;  // t < m
    for (int i = 0; i < 8; i++) r[i] = keep ? t[i] : d[i];
}
template <class C>
inline void h_sub(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t d[8];
    int64_t br = 0;
    for (int i = 0; i < 8; i++) {
        int64_t x = (int64_t)a[i] - b[i] + br;
        d[i] = (uint32_t)x;
        br = x < 0 ? -1 : 0;
    }
    if (br) {
        uint64_t c = 0;
        for (int i = 0; i < 8; i++) { c += (uint64_t)d[i] + mod_limb<C>(i); d[i] = (uint32_t)c; c >>= 32; }
    }
    for (int i = 0; i < 8; i++) r[i] = d[i];
}
// CIOS over four 64-bit limbs with 128-bit products (host compilers on both
// x86-64 and AArch64 provide unsigned __int128)
template <class C>
inline void h_mul(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    typedef unsigned __int128 u128;
    uint64_t A[4], B[4], M[4], t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 4; i++) {
        A[i] = (uint64_t)a[2 * i] | ((uint64_t)a[2 * i + 1] << 32);
        B[i] = (uint64_t)b[2 * i] | ((uint64_t)b[2 * i + 1] << 32);
        M[i] = (uint64_t)mod_limb<C>(2 * i) | ((uint64_t)mod_limb<C>(2 * i + 1) << 32);
    }
    for (int i = 0; i < 4; i++) {
        u128 c = 0;
        for (int j = 0; j < 4; j++) {
            c += (u128)t[j] + (u128)A[j] * B[i];
            t[j] = (uint64_t)c;
            c >>= 64;
        }
        c += t[4];
        t[4] = (uint64_t)c;
        t[5] = (uint64_t)(c >> 64);
        uint64_t m = t[0] * C::INV64;
        c = (u128)t[0] + (u128)m * M[0];
        c >>= 64;
        for (int j = 1; j < 4; j++) {
            c += (u128)t[j] + (u128)m * M[j];
            t[j - 1] = (uint64_t)c;
            c >>= 64;
        }
        c += t[4];
        t[3] = (uint64_t)c;
        t[4] = t[5] + (uint64_t)(c >> 64);
    }
    // t < 2m: one conditional subtraction
    uint64_t d[4];
    u128 br = 0;
    for (int i = 0; i < 4; i++) {
        u128 x = (u128)t[i] - M[i] - br;
        d[i] = (uint64_t)x;
        br = (x >> 127) & 1;  // borrow
    }
    bool keep = (t[4] == 0) && br != 0;
    for (int i = 0; i < 4; i++) {
        uint64_t v = keep ? t[i] : d[i];
        r[2 * i] = (uint32_t)v;
        r[2 * i + 1] = (uint32_t)(v >> 32);
    }
}

// ---------------------------------------------------------------------------
// device arithmetic (PTX carry chains).  Products use d_mul_wide (64-bit
// limb products); d_mul (32-bit low/high chains) is kept for comparison.
// ---------------------------------------------------------------------------
#if defined(__CUDA_ARCH__)

template <class C>
ACE_DEV void d_add(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t t0, t1, t2, t3, t4, t5, t6, t7, d0, d1, d2, d3, d4, d5, d6, d7, mask;
    asm("add.cc.u32 %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32 %7, %15, %23;\n\t"
        : "=r"(t0), "=r"(t1), "=r"(t2), "=r"(t3), "=r"(t4), "=r"(t5), "=r"(t6), "=r"(t7)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
          "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;\n\t"
        : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3), "=r"(d4), "=r"(d5), "=r"(d6), "=r"(d7), "=r"(mask)
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7),
          "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5), "n"(C::M6), "n"(C::M7));
    // mask = 0xffffffff when t < m (keep t), else 0 (take t - m)
    r[0] = (t0 & mask) | (d0 & ~mask);
    r[1] = (t1 & mask) | (d1 & ~mask);
    r[2] = (t2 & mask) | (d2 & ~mask);
    r[3] = (t3 & mask) | (d3 & ~mask);
    r[4] = (t4 & mask) | (d4 & ~mask);
    r[5] = (t5 & mask) | (d5 & ~mask);
    r[6] = (t6 & mask) | (d6 & ~mask);
    r[7] = (t7 & mask) | (d7 & ~mask);
}

template <class C>
ACE_DEV void d_sub(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t d0, d1, d2, d3, d4, d5, d6, d7, mask;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;\n\t"
        : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3), "=r"(d4), "=r"(d5), "=r"(d6), "=r"(d7), "=r"(mask)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
          "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    // mask = 0xffffffff on borrow: add m back
    asm("add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\t"
        "addc.cc.u32 %4, %4, %13;\n\t"
        "addc.cc.u32 %5, %5, %14;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.u32 %7, %7, %16;\n\t"
        : "+r"(d0), "+r"(d1), "+r"(d2), "+r"(d3), "+r"(d4), "+r"(d5), "+r"(d6), "+r"(d7)
        : "r"(mask),
          "r"(C::M0 & mask), "r"(C::M1 & mask), "r"(C::M2 & mask), "r"(C::M3 & mask),
          "r"(C::M4 & mask), "r"(C::M5 & mask), "r"(C::M6 & mask), "r"(C::M7 & mask));
    r[0] = d0; r[1] = d1; r[2] = d2; r[3] = d3; r[4] = d4; r[5] = d5; r[6] = d6; r[7] = d7;
}

// t += a * b_i (9-limb accumulator t0..t8, t8 == 0 on entry)
#define ACE_MAC_ROW(bi)                                                                          \
    asm("mad.lo.cc.u32 %0, %9, %17, %0;\n\t"                                                     \
        "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"                                                   \
        "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"                                                   \
        "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"                                                   \
        "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"                                                   \
        "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"                                                   \
        "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"                                                   \
        "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"                                                   \
        "addc.u32 %8, 0, 0;\n\t"                                                                 \
        "mad.hi.cc.u32 %1, %9, %17, %1;\n\t"                                                     \
        "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"                                                   \
        "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"                                                   \
        "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"                                                   \
        "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"                                                   \
        "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"                                                   \
        "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"                                                   \
        "madc.hi.u32 %8, %16, %17, %8;\n\t"                                                      \
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8) \
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), \
          "r"(bi))

// t = (t + m p) / 2^32 with m = t0 * INV; result in t0..t7 (shifted), t8 := 0
#define ACE_REDUCE_ROW()                                                                         \
    asm("{\n\t.reg .u32 m;\n\t"                                                                  \
        "mul.lo.u32 m, %0, %9;\n\t"                                                              \
        "mad.lo.cc.u32 %0, m, %10, %0;\n\t"                                                      \
        "madc.lo.cc.u32 %1, m, %11, %1;\n\t"                                                     \
        "madc.lo.cc.u32 %2, m, %12, %2;\n\t"                                                     \
        "madc.lo.cc.u32 %3, m, %13, %3;\n\t"                                                     \
        "madc.lo.cc.u32 %4, m, %14, %4;\n\t"                                                     \
        "madc.lo.cc.u32 %5, m, %15, %5;\n\t"                                                     \
        "madc.lo.cc.u32 %6, m, %16, %6;\n\t"                                                     \
        "madc.lo.cc.u32 %7, m, %17, %7;\n\t"                                                     \
        "addc.u32 %8, %8, 0;\n\t"                                                                \
        "mad.hi.cc.u32 %0, m, %10, %1;\n\t"                                                      \
        "madc.hi.cc.u32 %1, m, %11, %2;\n\t"                                                     \
        "madc.hi.cc.u32 %2, m, %12, %3;\n\t"                                                     \
        "madc.hi.cc.u32 %3, m, %13, %4;\n\t"                                                     \
        "madc.hi.cc.u32 %4, m, %14, %5;\n\t"                                                     \
        "madc.hi.cc.u32 %5, m, %15, %6;\n\t"                                                     \
        "madc.hi.cc.u32 %6, m, %16, %7;\n\t"                                                     \
        "madc.hi.u32 %7, m, %17, %8;\n\t"                                                        \
        "mov.u32 %8, 0;\n\t}"                                                                    \
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8) \
        : "n"(C::INV), "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5),  \
          "n"(C::M6), "n"(C::M7))

template <class C>
ACE_DEV void d_mul(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8 = 0;
    ACE_MAC_ROW(b[0]);
    ACE_REDUCE_ROW();
    ACE_MAC_ROW(b[1]);
    ACE_REDUCE_ROW();
    ACE_MAC_ROW(b[2]);
    ACE_REDUCE_ROW();
    ACE_MAC_ROW(b[3]);
    ACE_REDUCE_ROW();
    ACE_MAC_ROW(b[4]);
    ACE_REDUCE_ROW();
    ACE_MAC_ROW(b[5]);
    ACE_REDUCE_ROW();
    ACE_MAC_ROW(b[6]);
    ACE_REDUCE_ROW();
    ACE_MAC_ROW(b[7]);
    ACE_REDUCE_ROW();
    // t < 2m: one conditional subtraction
    uint32_t d0, d1, d2, d3, d4, d5, d6, d7, mask;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;\n\t"
        : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3), "=r"(d4), "=r"(d5), "=r"(d6), "=r"(d7), "=r"(mask)
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7),
          "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5), "n"(C::M6), "n"(C::M7));
    r[0] = (t0 & mask) | (d0 & ~mask);
    r[1] = (t1 & mask) | (d1 & ~mask);
    r[2] = (t2 & mask) | (d2 & ~mask);
    r[3] = (t3 & mask) | (d3 & ~mask);
    r[4] = (t4 & mask) | (d4 & ~mask);
    r[5] = (t5 & mask) | (d5 & ~mask);
    r[6] = (t6 & mask) | (d6 & ~mask);
    r[7] = (t7 & mask) | (d7 & ~mask);
}
#undef ACE_MAC_ROW
#undef ACE_REDUCE_ROW

// Same product with 64-bit limb products: per row, eight independent
// mad.wide.u32 (a_j b_i + t_j, which cannot overflow 64 bits) followed by one
// carry chain that adds each high half into the next limb; the reduction row
// does the same with m p_j.  Per product this issues one wide multiply-add
// instead of a low and a high multiply-add.
#define ACE_WROW_MUL(bi)                                                                         \
    asm("{\n\t.reg .u64 p0,p1,p2,p3,p4,p5,p6,p7,c;\n\t"                                       \
        ".reg .u32 l0,l1,l2,l3,l4,l5,l6,l7,h0,h1,h2,h3,h4,h5,h6,h7;\n\t"                        \
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %9, %17, c;\n\t"                                \
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %10, %17, c;\n\t"                               \
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 p2, %11, %17, c;\n\t"                               \
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 p3, %12, %17, c;\n\t"                               \
        "mov.b64 c, {%4, 0};\n\tmad.wide.u32 p4, %13, %17, c;\n\t"                               \
        "mov.b64 c, {%5, 0};\n\tmad.wide.u32 p5, %14, %17, c;\n\t"                               \
        "mov.b64 c, {%6, 0};\n\tmad.wide.u32 p6, %15, %17, c;\n\t"                               \
        "mov.b64 c, {%7, 0};\n\tmad.wide.u32 p7, %16, %17, c;\n\t"                               \
        "mov.b64 {l0,h0}, p0;\n\tmov.b64 {l1,h1}, p1;\n\tmov.b64 {l2,h2}, p2;\n\t"             \
        "mov.b64 {l3,h3}, p3;\n\tmov.b64 {l4,h4}, p4;\n\tmov.b64 {l5,h5}, p5;\n\t"             \
        "mov.b64 {l6,h6}, p6;\n\tmov.b64 {l7,h7}, p7;\n\t"                                        \
        "mov.b32 %0, l0;\n\t"                                                                    \
        "add.cc.u32 %1, l1, h0;\n\t"                                                             \
        "addc.cc.u32 %2, l2, h1;\n\t"                                                            \
        "addc.cc.u32 %3, l3, h2;\n\t"                                                            \
        "addc.cc.u32 %4, l4, h3;\n\t"                                                            \
        "addc.cc.u32 %5, l5, h4;\n\t"                                                            \
        "addc.cc.u32 %6, l6, h5;\n\t"                                                            \
        "addc.cc.u32 %7, l7, h6;\n\t"                                                            \
        "addc.u32 %8, h7, 0;\n\t}"                                                               \
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8) \
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), \
          "r"(bi))

// t = (t + m p) / 2^32, m = t0 * INV; t8 holds the ninth limb on entry and is
// zero on exit (the shifted value is below 2p)
#define ACE_WROW_RED()                                                                           \
    asm("{\n\t.reg .u64 q0,q1,q2,q3,q4,q5,q6,q7,c;\n\t.reg .u32 m;\n\t"                       \
        ".reg .u32 l0,l1,l2,l3,l4,l5,l6,l7,h0,h1,h2,h3,h4,h5,h6,h7;\n\t"                        \
        "mul.lo.u32 m, %0, %9;\n\t"                                                              \
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 q0, m, %10, c;\n\t"                                 \
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 q1, m, %11, c;\n\t"                                 \
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 q2, m, %12, c;\n\t"                                 \
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 q3, m, %13, c;\n\t"                                 \
        "mov.b64 c, {%4, 0};\n\tmad.wide.u32 q4, m, %14, c;\n\t"                                 \
        "mov.b64 c, {%5, 0};\n\tmad.wide.u32 q5, m, %15, c;\n\t"                                 \
        "mov.b64 c, {%6, 0};\n\tmad.wide.u32 q6, m, %16, c;\n\t"                                 \
        "mov.b64 c, {%7, 0};\n\tmad.wide.u32 q7, m, %17, c;\n\t"                                 \
        "mov.b64 {l0,h0}, q0;\n\tmov.b64 {l1,h1}, q1;\n\tmov.b64 {l2,h2}, q2;\n\t"             \
        "mov.b64 {l3,h3}, q3;\n\tmov.b64 {l4,h4}, q4;\n\tmov.b64 {l5,h5}, q5;\n\t"             \
        "mov.b64 {l6,h6}, q6;\n\tmov.b64 {l7,h7}, q7;\n\t"                                        \
        "add.cc.u32 %0, h0, l1;\n\t"                                                             \
        "addc.cc.u32 %1, h1, l2;\n\t"                                                            \
        "addc.cc.u32 %2, h2, l3;\n\t"                                                            \
        "addc.cc.u32 %3, h3, l4;\n\t"                                                            \
        "addc.cc.u32 %4, h4, l5;\n\t"                                                            \
        "addc.cc.u32 %5, h5, l6;\n\t"                                                            \
        "addc.cc.u32 %6, h6, l7;\n\t"                                                            \
        "addc.u32 %7, h7, %8;\n\t"                                                               \
        "mov.u32 %8, 0;\n\t}"                                                                    \
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8) \
        : "n"(C::INV), "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5),  \
          "n"(C::M6), "n"(C::M7))

template <class C>
ACE_DEV void d_mul_wide(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8 = 0;
    ACE_WROW_MUL(b[0]);
    ACE_WROW_RED();
    ACE_WROW_MUL(b[1]);
    ACE_WROW_RED();
    ACE_WROW_MUL(b[2]);
    ACE_WROW_RED();
    ACE_WROW_MUL(b[3]);
    ACE_WROW_RED();
    ACE_WROW_MUL(b[4]);
    ACE_WROW_RED();
    ACE_WROW_MUL(b[5]);
    ACE_WROW_RED();
    ACE_WROW_MUL(b[6]);
    ACE_WROW_RED();
    ACE_WROW_MUL(b[7]);
    ACE_WROW_RED();
    uint32_t d0, d1, d2, d3, d4, d5, d6, d7, mask;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;\n\t"
        : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3), "=r"(d4), "=r"(d5), "=r"(d6), "=r"(d7), "=r"(mask)
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7),
          "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5), "n"(C::M6), "n"(C::M7));
    r[0] = (t0 & mask) | (d0 & ~mask);
    r[1] = (t1 & mask) | (d1 & ~mask);
    r[2] = (t2 & mask) | (d2 & ~mask);
    r[3] = (t3 & mask) | (d3 & ~mask);
    r[4] = (t4 & mask) | (d4 & ~mask);
    r[5] = (t5 & mask) | (d5 & ~mask);
    r[6] = (t6 & mask) | (d6 & ~mask);
    r[7] = (t7 & mask) | (d7 & ~mask);
}
#undef ACE_WROW_MUL
#undef ACE_WROW_RED

// Third form: plain 64-bit products (mul.wide, no addend) folded into the
// accumulator by two carry chains per row (low halves at limb j, high halves
// at limb j+1).  Same result as d_mul / d_mul_wide.
#define ACE_PROW_MUL(bi)                                                                         \
    asm("{\n\t.reg .u64 p0,p1,p2,p3,p4,p5,p6,p7;\n\t"                                       \
        ".reg .u32 l0,l1,l2,l3,l4,l5,l6,l7,h0,h1,h2,h3,h4,h5,h6,h7;\n\t"                        \
        "mul.wide.u32 p0, %9, %17;\n\tmul.wide.u32 p1, %10, %17;\n\t"                         \
        "mul.wide.u32 p2, %11, %17;\n\tmul.wide.u32 p3, %12, %17;\n\t"                        \
        "mul.wide.u32 p4, %13, %17;\n\tmul.wide.u32 p5, %14, %17;\n\t"                        \
        "mul.wide.u32 p6, %15, %17;\n\tmul.wide.u32 p7, %16, %17;\n\t"                        \
        "mov.b64 {l0,h0}, p0;\n\tmov.b64 {l1,h1}, p1;\n\tmov.b64 {l2,h2}, p2;\n\t"             \
        "mov.b64 {l3,h3}, p3;\n\tmov.b64 {l4,h4}, p4;\n\tmov.b64 {l5,h5}, p5;\n\t"             \
        "mov.b64 {l6,h6}, p6;\n\tmov.b64 {l7,h7}, p7;\n\t"                                        \
        "add.cc.u32 %0, %0, l0;\n\taddc.cc.u32 %1, %1, l1;\n\taddc.cc.u32 %2, %2, l2;\n\t"     \
        "addc.cc.u32 %3, %3, l3;\n\taddc.cc.u32 %4, %4, l4;\n\taddc.cc.u32 %5, %5, l5;\n\t"    \
        "addc.cc.u32 %6, %6, l6;\n\taddc.cc.u32 %7, %7, l7;\n\taddc.u32 %8, 0, 0;\n\t"          \
        "add.cc.u32 %1, %1, h0;\n\taddc.cc.u32 %2, %2, h1;\n\taddc.cc.u32 %3, %3, h2;\n\t"     \
        "addc.cc.u32 %4, %4, h3;\n\taddc.cc.u32 %5, %5, h4;\n\taddc.cc.u32 %6, %6, h5;\n\t"    \
        "addc.cc.u32 %7, %7, h6;\n\taddc.u32 %8, %8, h7;\n\t}"                                   \
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8) \
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), \
          "r"(bi))
#define ACE_PROW_RED()                                                                           \
    asm("{\n\t.reg .u64 q0,q1,q2,q3,q4,q5,q6,q7;\n\t.reg .u32 m;\n\t"                       \
        ".reg .u32 l0,l1,l2,l3,l4,l5,l6,l7,h0,h1,h2,h3,h4,h5,h6,h7;\n\t"                        \
        "mul.lo.u32 m, %0, %9;\n\t"                                                              \
        "mul.wide.u32 q0, m, %10;\n\tmul.wide.u32 q1, m, %11;\n\t"                             \
        "mul.wide.u32 q2, m, %12;\n\tmul.wide.u32 q3, m, %13;\n\t"                             \
        "mul.wide.u32 q4, m, %14;\n\tmul.wide.u32 q5, m, %15;\n\t"                             \
        "mul.wide.u32 q6, m, %16;\n\tmul.wide.u32 q7, m, %17;\n\t"                             \
        "mov.b64 {l0,h0}, q0;\n\tmov.b64 {l1,h1}, q1;\n\tmov.b64 {l2,h2}, q2;\n\t"             \
        "mov.b64 {l3,h3}, q3;\n\tmov.b64 {l4,h4}, q4;\n\tmov.b64 {l5,h5}, q5;\n\t"             \
        "mov.b64 {l6,h6}, q6;\n\tmov.b64 {l7,h7}, q7;\n\t"                                        \
        "add.cc.u32 %0, %0, l0;\n\taddc.cc.u32 %1, %1, l1;\n\taddc.cc.u32 %2, %2, l2;\n\t"     \
        "addc.cc.u32 %3, %3, l3;\n\taddc.cc.u32 %4, %4, l4;\n\taddc.cc.u32 %5, %5, l5;\n\t"    \
        "addc.cc.u32 %6, %6, l6;\n\taddc.cc.u32 %7, %7, l7;\n\taddc.u32 %8, %8, 0;\n\t"         \
        "add.cc.u32 %0, %1, h0;\n\taddc.cc.u32 %1, %2, h1;\n\taddc.cc.u32 %2, %3, h2;\n\t"     \
        "addc.cc.u32 %3, %4, h3;\n\taddc.cc.u32 %4, %5, h4;\n\taddc.cc.u32 %5, %6, h5;\n\t"    \
        "addc.cc.u32 %6, %7, h6;\n\taddc.u32 %7, %8, h7;\n\tmov.u32 %8, 0;\n\t}"               \
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8) \
        : "n"(C::INV), "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5),  \
          "n"(C::M6), "n"(C::M7))

template <class C>
ACE_DEV void d_mul_pw(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8 = 0;
    ACE_PROW_MUL(b[0]);
    ACE_PROW_RED();
    ACE_PROW_MUL(b[1]);
    ACE_PROW_RED();
    ACE_PROW_MUL(b[2]);
    ACE_PROW_RED();
    ACE_PROW_MUL(b[3]);
    ACE_PROW_RED();
    ACE_PROW_MUL(b[4]);
    ACE_PROW_RED();
    ACE_PROW_MUL(b[5]);
    ACE_PROW_RED();
    ACE_PROW_MUL(b[6]);
    ACE_PROW_RED();
    ACE_PROW_MUL(b[7]);
    ACE_PROW_RED();
    uint32_t d0, d1, d2, d3, d4, d5, d6, d7, mask;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;\n\t"
        : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3), "=r"(d4), "=r"(d5), "=r"(d6), "=r"(d7), "=r"(mask)
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7),
          "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5), "n"(C::M6), "n"(C::M7));
    r[0] = (t0 & mask) | (d0 & ~mask);
    r[1] = (t1 & mask) | (d1 & ~mask);
    r[2] = (t2 & mask) | (d2 & ~mask);
    r[3] = (t3 & mask) | (d3 & ~mask);
    r[4] = (t4 & mask) | (d4 & ~mask);
    r[5] = (t5 & mask) | (d5 & ~mask);
    r[6] = (t6 & mask) | (d6 & ~mask);
    r[7] = (t7 & mask) | (d7 & ~mask);
}
#undef ACE_PROW_MUL
#undef ACE_PROW_RED

// ---- separated product and reduction (lazy reduction) ----------------------
// t[I..I+8] = t[I..I+7] + a * bi for the 512-bit product t (t[I+8] is not
// read: no earlier row reached it)
template <int I>
ACE_DEV void d_w512_row(uint32_t (&t)[16], const uint32_t* a, uint32_t bi) {
    asm("{\n\t.reg .u64 p0,p1,p2,p3,p4,p5,p6,p7,c;\n\t"
        ".reg .u32 l0,l1,l2,l3,l4,l5,l6,l7,h0,h1,h2,h3,h4,h5,h6,h7;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %9, %17, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %10, %17, c;\n\t"
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 p2, %11, %17, c;\n\t"
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 p3, %12, %17, c;\n\t"
        "mov.b64 c, {%4, 0};\n\tmad.wide.u32 p4, %13, %17, c;\n\t"
        "mov.b64 c, {%5, 0};\n\tmad.wide.u32 p5, %14, %17, c;\n\t"
        "mov.b64 c, {%6, 0};\n\tmad.wide.u32 p6, %15, %17, c;\n\t"
        "mov.b64 c, {%7, 0};\n\tmad.wide.u32 p7, %16, %17, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\tmov.b64 {l1,h1}, p1;\n\tmov.b64 {l2,h2}, p2;\n\t"
        "mov.b64 {l3,h3}, p3;\n\tmov.b64 {l4,h4}, p4;\n\tmov.b64 {l5,h5}, p5;\n\t"
        "mov.b64 {l6,h6}, p6;\n\tmov.b64 {l7,h7}, p7;\n\t"
        "mov.b32 %0, l0;\n\t"
        "add.cc.u32 %1, l1, h0;\n\t"
        "addc.cc.u32 %2, l2, h1;\n\t"
        "addc.cc.u32 %3, l3, h2;\n\t"
        "addc.cc.u32 %4, l4, h3;\n\t"
        "addc.cc.u32 %5, l5, h4;\n\t"
        "addc.cc.u32 %6, l6, h5;\n\t"
        "addc.cc.u32 %7, l7, h6;\n\t"
        "addc.u32 %8, h7, 0;\n\t}"
        : "+r"(t[I]), "+r"(t[I + 1]), "+r"(t[I + 2]), "+r"(t[I + 3]), "+r"(t[I + 4]), "+r"(t[I + 5]),
          "+r"(t[I + 6]), "+r"(t[I + 7]), "=r"(t[I + 8])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(bi));
}
// the full 512-bit product of two 256-bit integers
ACE_DEV void d_mul512(uint32_t (&t)[16], const uint32_t* a, const uint32_t* b) {
#pragma unroll
    for (int i = 0; i < 8; i++) t[i] = 0;
    d_w512_row<0>(t, a, b[0]);
    d_w512_row<1>(t, a, b[1]);
    d_w512_row<2>(t, a, b[2]);
    d_w512_row<3>(t, a, b[3]);
    d_w512_row<4>(t, a, b[4]);
    d_w512_row<5>(t, a, b[5]);
    d_w512_row<6>(t, a, b[6]);
    d_w512_row<7>(t, a, b[7]);
}
// one Montgomery reduction row of a 512-bit value: m = t[I] * INV,
// t += m p 2^(32 I); e carries the bit that overflowed limb I+7 of the
// previous row into limb I+8 (e is 0/1 on entry and exit)
template <class C, int I>
ACE_DEV void d_redc_row(uint32_t (&t)[16], uint32_t& e) {
    asm("{\n\t.reg .u64 q0,q1,q2,q3,q4,q5,q6,q7,c;\n\t.reg .u32 m;\n\t"
        ".reg .u32 l0,l1,l2,l3,l4,l5,l6,l7,h0,h1,h2,h3,h4,h5,h6,h7;\n\t"
        "mul.lo.u32 m, %0, %10;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 q0, m, %11, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 q1, m, %12, c;\n\t"
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 q2, m, %13, c;\n\t"
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 q3, m, %14, c;\n\t"
        "mov.b64 c, {%4, 0};\n\tmad.wide.u32 q4, m, %15, c;\n\t"
        "mov.b64 c, {%5, 0};\n\tmad.wide.u32 q5, m, %16, c;\n\t"
        "mov.b64 c, {%6, 0};\n\tmad.wide.u32 q6, m, %17, c;\n\t"
        "mov.b64 c, {%7, 0};\n\tmad.wide.u32 q7, m, %18, c;\n\t"
        "mov.b64 {l0,h0}, q0;\n\tmov.b64 {l1,h1}, q1;\n\tmov.b64 {l2,h2}, q2;\n\t"
        "mov.b64 {l3,h3}, q3;\n\tmov.b64 {l4,h4}, q4;\n\tmov.b64 {l5,h5}, q5;\n\t"
        "mov.b64 {l6,h6}, q6;\n\tmov.b64 {l7,h7}, q7;\n\t"
        "add.u32 h7, h7, %9;\n\t"
        "add.cc.u32 %1, h0, l1;\n\t"
        "addc.cc.u32 %2, h1, l2;\n\t"
        "addc.cc.u32 %3, h2, l3;\n\t"
        "addc.cc.u32 %4, h3, l4;\n\t"
        "addc.cc.u32 %5, h4, l5;\n\t"
        "addc.cc.u32 %6, h5, l6;\n\t"
        "addc.cc.u32 %7, h6, l7;\n\t"
        "addc.cc.u32 %8, %8, h7;\n\t"
        "addc.u32 %9, 0, 0;\n\t}"
        : "+r"(t[I]), "+r"(t[I + 1]), "+r"(t[I + 2]), "+r"(t[I + 3]), "+r"(t[I + 4]), "+r"(t[I + 5]),
          "+r"(t[I + 6]), "+r"(t[I + 7]), "+r"(t[I + 8]), "+r"(e)
        : "n"(C::INV), "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5), "n"(C::M6),
          "n"(C::M7));
}
// r = t / 2^256 mod m for 0 <= t < m 2^256 (result fully reduced)
template <class C>
ACE_DEV void d_redc512(uint32_t* r, uint32_t (&t)[16]) {
    uint32_t e = 0;
    d_redc_row<C, 0>(t, e);
    d_redc_row<C, 1>(t, e);
    d_redc_row<C, 2>(t, e);
    d_redc_row<C, 3>(t, e);
    d_redc_row<C, 4>(t, e);
    d_redc_row<C, 5>(t, e);
    d_redc_row<C, 6>(t, e);
    d_redc_row<C, 7>(t, e);
    // t[8..15] < 2m (and e == 0): one conditional subtraction
    uint32_t d0, d1, d2, d3, d4, d5, d6, d7, mask;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;\n\t"
        : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3), "=r"(d4), "=r"(d5), "=r"(d6), "=r"(d7), "=r"(mask)
        : "r"(t[8]), "r"(t[9]), "r"(t[10]), "r"(t[11]), "r"(t[12]), "r"(t[13]), "r"(t[14]), "r"(t[15]),
          "n"(C::M0), "n"(C::M1), "n"(C::M2), "n"(C::M3), "n"(C::M4), "n"(C::M5), "n"(C::M6), "n"(C::M7));
    r[0] = (t[8] & mask) | (d0 & ~mask);
    r[1] = (t[9] & mask) | (d1 & ~mask);
    r[2] = (t[10] & mask) | (d2 & ~mask);
    r[3] = (t[11] & mask) | (d3 & ~mask);
    r[4] = (t[12] & mask) | (d4 & ~mask);
    r[5] = (t[13] & mask) | (d5 & ~mask);
    r[6] = (t[14] & mask) | (d6 & ~mask);
    r[7] = (t[15] & mask) | (d7 & ~mask);
}
// the 512-bit square of a 256-bit integer: the 28 products a_i a_j (i < j)
// row by row, doubled, plus the 8 squares a_i^2 on the diagonal (36 limb
// products instead of 64)
ACE_DEV void d_sqr512(uint32_t (&t)[16], const uint32_t* a) {
    t[0] = 0;
#pragma unroll
    for (int i = 1; i < 8; i++) t[i] = 0;
    t[15] = 0;
    asm("{\n\t.reg .u64 p0,p1,p2,p3,p4,p5,p6,c;\n\t.reg .u32 l0,l1,l2,l3,l4,l5,l6,h0,h1,h2,h3,h4,h5,h6;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %8, %15, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %9, %15, c;\n\t"
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 p2, %10, %15, c;\n\t"
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 p3, %11, %15, c;\n\t"
        "mov.b64 c, {%4, 0};\n\tmad.wide.u32 p4, %12, %15, c;\n\t"
        "mov.b64 c, {%5, 0};\n\tmad.wide.u32 p5, %13, %15, c;\n\t"
        "mov.b64 c, {%6, 0};\n\tmad.wide.u32 p6, %14, %15, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\t"
        "mov.b64 {l1,h1}, p1;\n\t"
        "mov.b64 {l2,h2}, p2;\n\t"
        "mov.b64 {l3,h3}, p3;\n\t"
        "mov.b64 {l4,h4}, p4;\n\t"
        "mov.b64 {l5,h5}, p5;\n\t"
        "mov.b64 {l6,h6}, p6;\n\t"
        "mov.b32 %0, l0;\n\t"
        "add.cc.u32 %1, l1, h0;\n\t"
        "addc.cc.u32 %2, l2, h1;\n\t"
        "addc.cc.u32 %3, l3, h2;\n\t"
        "addc.cc.u32 %4, l4, h3;\n\t"
        "addc.cc.u32 %5, l5, h4;\n\t"
        "addc.cc.u32 %6, l6, h5;\n\t"
        "addc.u32 %7, h6, 0;\n\t}"
        : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "=r"(t[8])
        : "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[0]));
    asm("{\n\t.reg .u64 p0,p1,p2,p3,p4,p5,c;\n\t.reg .u32 l0,l1,l2,l3,l4,l5,h0,h1,h2,h3,h4,h5;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %7, %13, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %8, %13, c;\n\t"
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 p2, %9, %13, c;\n\t"
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 p3, %10, %13, c;\n\t"
        "mov.b64 c, {%4, 0};\n\tmad.wide.u32 p4, %11, %13, c;\n\t"
        "mov.b64 c, {%5, 0};\n\tmad.wide.u32 p5, %12, %13, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\t"
        "mov.b64 {l1,h1}, p1;\n\t"
        "mov.b64 {l2,h2}, p2;\n\t"
        "mov.b64 {l3,h3}, p3;\n\t"
        "mov.b64 {l4,h4}, p4;\n\t"
        "mov.b64 {l5,h5}, p5;\n\t"
        "mov.b32 %0, l0;\n\t"
        "add.cc.u32 %1, l1, h0;\n\t"
        "addc.cc.u32 %2, l2, h1;\n\t"
        "addc.cc.u32 %3, l3, h2;\n\t"
        "addc.cc.u32 %4, l4, h3;\n\t"
        "addc.cc.u32 %5, l5, h4;\n\t"
        "addc.u32 %6, h5, 0;\n\t}"
        : "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "=r"(t[9])
        : "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[1]));
    asm("{\n\t.reg .u64 p0,p1,p2,p3,p4,c;\n\t.reg .u32 l0,l1,l2,l3,l4,h0,h1,h2,h3,h4;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %6, %11, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %7, %11, c;\n\t"
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 p2, %8, %11, c;\n\t"
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 p3, %9, %11, c;\n\t"
        "mov.b64 c, {%4, 0};\n\tmad.wide.u32 p4, %10, %11, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\t"
        "mov.b64 {l1,h1}, p1;\n\t"
        "mov.b64 {l2,h2}, p2;\n\t"
        "mov.b64 {l3,h3}, p3;\n\t"
        "mov.b64 {l4,h4}, p4;\n\t"
        "mov.b32 %0, l0;\n\t"
        "add.cc.u32 %1, l1, h0;\n\t"
        "addc.cc.u32 %2, l2, h1;\n\t"
        "addc.cc.u32 %3, l3, h2;\n\t"
        "addc.cc.u32 %4, l4, h3;\n\t"
        "addc.u32 %5, h4, 0;\n\t}"
        : "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "=r"(t[10])
        : "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[2]));
    asm("{\n\t.reg .u64 p0,p1,p2,p3,c;\n\t.reg .u32 l0,l1,l2,l3,h0,h1,h2,h3;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %5, %9, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %6, %9, c;\n\t"
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 p2, %7, %9, c;\n\t"
        "mov.b64 c, {%3, 0};\n\tmad.wide.u32 p3, %8, %9, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\t"
        "mov.b64 {l1,h1}, p1;\n\t"
        "mov.b64 {l2,h2}, p2;\n\t"
        "mov.b64 {l3,h3}, p3;\n\t"
        "mov.b32 %0, l0;\n\t"
        "add.cc.u32 %1, l1, h0;\n\t"
        "addc.cc.u32 %2, l2, h1;\n\t"
        "addc.cc.u32 %3, l3, h2;\n\t"
        "addc.u32 %4, h3, 0;\n\t}"
        : "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "=r"(t[11])
        : "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[3]));
    asm("{\n\t.reg .u64 p0,p1,p2,c;\n\t.reg .u32 l0,l1,l2,h0,h1,h2;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %4, %7, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %5, %7, c;\n\t"
        "mov.b64 c, {%2, 0};\n\tmad.wide.u32 p2, %6, %7, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\t"
        "mov.b64 {l1,h1}, p1;\n\t"
        "mov.b64 {l2,h2}, p2;\n\t"
        "mov.b32 %0, l0;\n\t"
        "add.cc.u32 %1, l1, h0;\n\t"
        "addc.cc.u32 %2, l2, h1;\n\t"
        "addc.u32 %3, h2, 0;\n\t}"
        : "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "=r"(t[12])
        : "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[4]));
    asm("{\n\t.reg .u64 p0,p1,c;\n\t.reg .u32 l0,l1,h0,h1;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %3, %5, c;\n\t"
        "mov.b64 c, {%1, 0};\n\tmad.wide.u32 p1, %4, %5, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\t"
        "mov.b64 {l1,h1}, p1;\n\t"
        "mov.b32 %0, l0;\n\t"
        "add.cc.u32 %1, l1, h0;\n\t"
        "addc.u32 %2, h1, 0;\n\t}"
        : "+r"(t[11]), "+r"(t[12]), "=r"(t[13])
        : "r"(a[6]), "r"(a[7]), "r"(a[5]));
    asm("{\n\t.reg .u64 p0,c;\n\t.reg .u32 l0,h0;\n\t"
        "mov.b64 c, {%0, 0};\n\tmad.wide.u32 p0, %2, %3, c;\n\t"
        "mov.b64 {l0,h0}, p0;\n\t"
        "mov.b32 %0, l0;\n\t"
        "mov.b32 %1, h0;\n\t}"
        : "+r"(t[13]), "=r"(t[14])
        : "r"(a[7]), "r"(a[6]));
    // t = 2 t + sum_i a_i^2 2^(64 i)
    asm("{\n\t.reg .u64 d0,d1,d2,d3,d4,d5,d6,d7;\n\t"
        ".reg .u32 l0,l1,l2,l3,l4,l5,l6,l7,h0,h1,h2,h3,h4,h5,h6,h7;\n\t"
        "add.cc.u32 %0, %0, %0;\n\taddc.cc.u32 %1, %1, %1;\n\taddc.cc.u32 %2, %2, %2;\n\t"
        "addc.cc.u32 %3, %3, %3;\n\taddc.cc.u32 %4, %4, %4;\n\taddc.cc.u32 %5, %5, %5;\n\t"
        "addc.cc.u32 %6, %6, %6;\n\taddc.cc.u32 %7, %7, %7;\n\taddc.cc.u32 %8, %8, %8;\n\t"
        "addc.cc.u32 %9, %9, %9;\n\taddc.cc.u32 %10, %10, %10;\n\taddc.cc.u32 %11, %11, %11;\n\t"
        "addc.cc.u32 %12, %12, %12;\n\taddc.cc.u32 %13, %13, %13;\n\taddc.cc.u32 %14, %14, %14;\n\t"
        "addc.u32 %15, %15, %15;\n\t"
        "mul.wide.u32 d0, %16, %16;\n\tmul.wide.u32 d1, %17, %17;\n\t"
        "mul.wide.u32 d2, %18, %18;\n\tmul.wide.u32 d3, %19, %19;\n\t"
        "mul.wide.u32 d4, %20, %20;\n\tmul.wide.u32 d5, %21, %21;\n\t"
        "mul.wide.u32 d6, %22, %22;\n\tmul.wide.u32 d7, %23, %23;\n\t"
        "mov.b64 {l0,h0}, d0;\n\tmov.b64 {l1,h1}, d1;\n\tmov.b64 {l2,h2}, d2;\n\tmov.b64 {l3,h3}, d3;\n\t"
        "mov.b64 {l4,h4}, d4;\n\tmov.b64 {l5,h5}, d5;\n\tmov.b64 {l6,h6}, d6;\n\tmov.b64 {l7,h7}, d7;\n\t"
        "add.cc.u32 %0, %0, l0;\n\taddc.cc.u32 %1, %1, h0;\n\taddc.cc.u32 %2, %2, l1;\n\t"
        "addc.cc.u32 %3, %3, h1;\n\taddc.cc.u32 %4, %4, l2;\n\taddc.cc.u32 %5, %5, h2;\n\t"
        "addc.cc.u32 %6, %6, l3;\n\taddc.cc.u32 %7, %7, h3;\n\taddc.cc.u32 %8, %8, l4;\n\t"
        "addc.cc.u32 %9, %9, h4;\n\taddc.cc.u32 %10, %10, l5;\n\taddc.cc.u32 %11, %11, h5;\n\t"
        "addc.cc.u32 %12, %12, l6;\n\taddc.cc.u32 %13, %13, h6;\n\taddc.cc.u32 %14, %14, l7;\n\t"
        "addc.u32 %15, %15, h7;\n\t}"
        : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
          "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]));
}
// a -= b over 16 limbs; returns the borrow mask (0xffffffff on borrow)
ACE_DEV uint32_t d_sub512(uint32_t (&a)[16], const uint32_t (&b)[16]) {
    uint32_t br;
    asm("sub.cc.u32 %0, %0, %17;\n\t"
        "subc.cc.u32 %1, %1, %18;\n\t"
        "subc.cc.u32 %2, %2, %19;\n\t"
        "subc.cc.u32 %3, %3, %20;\n\t"
        "subc.cc.u32 %4, %4, %21;\n\t"
        "subc.cc.u32 %5, %5, %22;\n\t"
        "subc.cc.u32 %6, %6, %23;\n\t"
        "subc.cc.u32 %7, %7, %24;\n\t"
        "subc.cc.u32 %8, %8, %25;\n\t"
        "subc.cc.u32 %9, %9, %26;\n\t"
        "subc.cc.u32 %10, %10, %27;\n\t"
        "subc.cc.u32 %11, %11, %28;\n\t"
        "subc.cc.u32 %12, %12, %29;\n\t"
        "subc.cc.u32 %13, %13, %30;\n\t"
        "subc.cc.u32 %14, %14, %31;\n\t"
        "subc.cc.u32 %15, %15, %32;\n\t"
        "subc.u32 %16, 0, 0;\n\t"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
          "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]),
          "=r"(br)
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]),
          "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(b[12]), "r"(b[13]), "r"(b[14]), "r"(b[15]));
    return br;
}
// a += b over 16 limbs (modulo 2^512)
ACE_DEV void d_add512(uint32_t (&a)[16], const uint32_t (&b)[16]) {
    asm("add.cc.u32 %0, %0, %16;\n\t"
        "addc.cc.u32 %1, %1, %17;\n\t"
        "addc.cc.u32 %2, %2, %18;\n\t"
        "addc.cc.u32 %3, %3, %19;\n\t"
        "addc.cc.u32 %4, %4, %20;\n\t"
        "addc.cc.u32 %5, %5, %21;\n\t"
        "addc.cc.u32 %6, %6, %22;\n\t"
        "addc.cc.u32 %7, %7, %23;\n\t"
        "addc.cc.u32 %8, %8, %24;\n\t"
        "addc.cc.u32 %9, %9, %25;\n\t"
        "addc.cc.u32 %10, %10, %26;\n\t"
        "addc.cc.u32 %11, %11, %27;\n\t"
        "addc.cc.u32 %12, %12, %28;\n\t"
        "addc.cc.u32 %13, %13, %29;\n\t"
        "addc.cc.u32 %14, %14, %30;\n\t"
        "addc.u32 %15, %15, %31;\n\t"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
          "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]),
          "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(b[12]), "r"(b[13]), "r"(b[14]), "r"(b[15]));
}
// a[8..15] += m & mask (adds m 2^256 when mask is all ones)
template <class C>
ACE_DEV void d_add_hi_mod(uint32_t (&a)[16], uint32_t mask) {
    asm("add.cc.u32 %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.cc.u32 %4, %4, %12;\n\t"
        "addc.cc.u32 %5, %5, %13;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.u32 %7, %7, %15;\n\t"
        : "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15])
        : "r"(C::M0 & mask), "r"(C::M1 & mask), "r"(C::M2 & mask), "r"(C::M3 & mask), "r"(C::M4 & mask),
          "r"(C::M5 & mask), "r"(C::M6 & mask), "r"(C::M7 & mask));
}
// a + b of two reduced elements as a plain 256-bit integer (< 2m < 2^255)
ACE_DEV void d_add_raw(uint32_t* r, const uint32_t* a, const uint32_t* b) {
    asm("add.cc.u32 %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32 %7, %15, %23;\n\t"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
          "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
}

#endif  // __CUDA_ARCH__

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <class C>
ACE_HD Fe<C> operator+(const Fe<C>& a, const Fe<C>& b) {
    Fe<C> r;
#if defined(__CUDA_ARCH__)
    d_add<C>(r.v, a.v, b.v);
#else
    h_add<C>(r.v, a.v, b.v);
#endif
    return r;
}
template <class C>
ACE_HD Fe<C> operator-(const Fe<C>& a, const Fe<C>& b) {
    Fe<C> r;
#if defined(__CUDA_ARCH__)
    d_sub<C>(r.v, a.v, b.v);
#else
    h_sub<C>(r.v, a.v, b.v);
#endif
    return r;
}
// Product form used by the field operators on the device: 0 lo/hi chains
// (d_mul), 1 wide multiply-adds (d_mul_wide), 2 plain wide products with two
// carry chains per row (d_mul_pw).  All three give identical results.
#ifndef ACE_MUL_FORM
#define ACE_MUL_FORM 2
#endif
#if defined(__CUDA_ARCH__)
template <class C>
ACE_DEV void d_mul_form(uint32_t* r, const uint32_t* a, const uint32_t* b) {
#if ACE_MUL_FORM == 0
    d_mul<C>(r, a, b);
#elif ACE_MUL_FORM == 2
    d_mul_pw<C>(r, a, b);
#else
    d_mul_wide<C>(r, a, b);
#endif
}
#endif
#if defined(__CUDA_ARCH__) && defined(ACE_FIELD_MUL_CALL)
// Out-of-line Montgomery product: translation units whose kernels chain many
// products (the MSM bucket loops) define ACE_FIELD_MUL_CALL so that all warps
// run one shared ~300-instruction body instead of an instruction stream of
// thousands of inlined copies that misses the instruction cache.
template <class C>
__device__ __noinline__ Fe<C> d_mul_call(const Fe<C> a, const Fe<C> b) {
    Fe<C> r;
    d_mul_form<C>(r.v, a.v, b.v);
    return r;
}
#endif

template <class C>
ACE_HD Fe<C> operator*(const Fe<C>& a, const Fe<C>& b) {
#if defined(__CUDA_ARCH__) && defined(ACE_FIELD_MUL_CALL)
    return d_mul_call<C>(a, b);
#else
    Fe<C> r;
#if defined(__CUDA_ARCH__)
    d_mul_form<C>(r.v, a.v, b.v);
#else
    h_mul<C>(r.v, a.v, b.v);
#endif
    return r;
#endif
}
// Squaring: on the device the 36-product square plus a separate Montgomery
// reduction (108 limb products instead of the 136 of a general product).
#if defined(__CUDA_ARCH__)
template <class C>
ACE_DEV void d_sqr_form(uint32_t* r, const uint32_t* a) {
    uint32_t t[16];
    d_sqr512(t, a);
    d_redc512<C>(r, t);
}
#if defined(ACE_FIELD_MUL_CALL)
template <class C>
__device__ __noinline__ Fe<C> d_sqr_call(const Fe<C> a) {
    Fe<C> r;
    d_sqr_form<C>(r.v, a.v);
    return r;
}
#endif
#endif
template <class C>
ACE_HD Fe<C> fe_sqr(const Fe<C>& a) {
#if defined(__CUDA_ARCH__) && defined(ACE_FIELD_MUL_CALL)
    return d_sqr_call<C>(a);
#elif defined(__CUDA_ARCH__)
    Fe<C> r;
    d_sqr_form<C>(r.v, a.v);
    return r;
#else
    return a * a;
#endif
}
// a b - c d with a single Montgomery reduction on the device: both products
// stay at 512 bits, their difference (in (-m^2, m^2)) is made non-negative by
// adding m 2^256 when it borrows, and one reduction gives the result.
#if defined(__CUDA_ARCH__)
template <class C>
ACE_DEV void d_mul_sub(uint32_t* r, const uint32_t* a, const uint32_t* b, const uint32_t* c, const uint32_t* d) {
    uint32_t t1[16], t2[16];
    d_mul512(t1, a, b);
    d_mul512(t2, c, d);
    uint32_t br = d_sub512(t1, t2);
    d_add_hi_mod<C>(t1, br);
    d_redc512<C>(r, t1);
}
#if defined(ACE_FIELD_MUL_CALL)
template <class C>
__device__ __noinline__ Fe<C> d_mul_sub_call(const Fe<C> a, const Fe<C> b, const Fe<C> c, const Fe<C> d) {
    Fe<C> r;
    d_mul_sub<C>(r.v, a.v, b.v, c.v, d.v);
    return r;
}
#endif
#endif
template <class C>
ACE_HD Fe<C> fe_mul_sub(const Fe<C>& a, const Fe<C>& b, const Fe<C>& c, const Fe<C>& d) {
#if defined(__CUDA_ARCH__) && defined(ACE_FIELD_MUL_CALL)
    return d_mul_sub_call<C>(a, b, c, d);
#elif defined(__CUDA_ARCH__)
    Fe<C> r;
    d_mul_sub<C>(r.v, a.v, b.v, c.v, d.v);
    return r;
#else
    return a * b - c * d;
#endif
}
template <class C>
ACE_HD Fe<C> fe_dbl(const Fe<C>& a) { return a + a; }
template <class C>
ACE_HD Fe<C> fe_neg(const Fe<C>& a) { return fe_zero<C>() - a; }
template <class C>
ACE_HD Fe<C> fe_to_mont(const Fe<C>& a) { return a * fe_rr<C>(); }
template <class C>
ACE_HD Fe<C> fe_from_mont(const Fe<C>& a) {
    Fe<C> one = fe_zero<C>();
    one.v[0] = 1;
    return a * one;
}
// small integer in Montgomery form
template <class C>
ACE_HD Fe<C> fe_from_u32(uint32_t x) {
    Fe<C> t = fe_zero<C>();
    t.v[0] = x;
    return fe_to_mont(t);
}

// a^e, e given as 8 little-endian limbs (plain integer): left-to-right binary
// square-and-multiply (rare: inversions and setup constants only)
template <class C>
ACE_HD Fe<C> fe_pow(const Fe<C>& a, const uint32_t* e) {
    Fe<C> acc = fe_one<C>();
#pragma unroll 1
    for (int i = 255; i >= 0; i--) {
        acc = fe_sqr(acc);
        if ((e[i >> 5] >> (i & 31)) & 1u) acc = acc * a;
    }
    return acc;
}
#if defined(__CUDA_ARCH__)
// Inverse on the device by the binary extended Euclidean algorithm (Hankerson,
// Menezes and Vanstone, Guide to Elliptic Curve Cryptography, Algorithm 2.22)
// applied to the stored residue x = a R: with u = x, v = m and invariants
// x1 x = u, x2 x = v (mod m), halve whichever of u, v is even (halving x1 or
// x2 mod m alongside) and subtract the smaller from the larger until one of
// them is 1; its x1 or x2 is then (a R)^-1 = a^-1 R^-1, and two Montgomery
// products with R^2 give a^-1 R.  About 2 x 254 halvings and 254
// subtractions of 8-limb values instead of Fermat's ~380 sequential
// products.  Variable time: the device inverts public values only (affine
// forms of results, proof elements and key points).
namespace detail {
ACE_DEV bool inv_is_one(const uint32_t* x) {
    uint32_t o = x[0] ^ 1u;
#pragma unroll
    for (int i = 1; i < 8; i++) o |= x[i];
    return o == 0;
}
ACE_DEV void inv_shr1(uint32_t* x) {
#pragma unroll
    for (int i = 0; i < 7; i++) x[i] = (x[i] >> 1) | (x[i + 1] << 31);
    x[7] >>= 1;
}
// x = x / 2 mod m (x < m, m odd and < 2^255: x + m does not overflow)
template <class C>
ACE_DEV void inv_half(uint32_t* x) {
    if (x[0] & 1u) {
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            c += (uint64_t)x[i] + mod_limb<C>(i);
            x[i] = (uint32_t)c;
            c >>= 32;
        }
    }
    inv_shr1(x);
}
// x = x - y (plain, x >= y)
ACE_DEV void inv_sub(uint32_t* x, const uint32_t* y) {
    int64_t b = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        b += (int64_t)x[i] - y[i];
        x[i] = (uint32_t)b;
        b >>= 32;
    }
}
// x = x - y mod m (x, y < m)
template <class C>
ACE_DEV void inv_sub_mod(uint32_t* x, const uint32_t* y) {
    int64_t b = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        b += (int64_t)x[i] - y[i];
        x[i] = (uint32_t)b;
        b >>= 32;
    }
    if (b) {
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            c += (uint64_t)x[i] + mod_limb<C>(i);
            x[i] = (uint32_t)c;
            c >>= 32;
        }
    }
}
ACE_DEV bool inv_geq(const uint32_t* x, const uint32_t* y) {
    bool gt = false, eq = true;
#pragma unroll
    for (int i = 7; i >= 0; i--) {
        gt = gt || (eq && x[i] > y[i]);
        eq = eq && x[i] == y[i];
    }
    return gt || eq;
}
ACE_DEV bool inv_is_zero(const uint32_t* x) {
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) o |= x[i];
    return o == 0;
}
}  // namespace detail

template <class C>
__device__ __noinline__ Fe<C> d_inv_binary(Fe<C> a) {
    if (fe_is_zero(a)) return a;
    uint32_t u[8], v[8], x1[8], x2[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        u[i] = a.v[i];
        v[i] = mod_limb<C>(i);
        x1[i] = i == 0 ? 1u : 0u;
        x2[i] = 0u;
    }
    // the loop ends within 2 x 256 halvings and 256 subtractions; the bound
    // and the zero tests only guard it against a non-canonical input (a
    // multiple of m would drive u to 0)
    for (int it = 0; it < 1024 && !detail::inv_is_one(u) && !detail::inv_is_one(v); it++) {
        if (detail::inv_is_zero(u) || detail::inv_is_zero(v)) break;
        while (!(u[0] & 1u)) {
            detail::inv_shr1(u);
            detail::inv_half<C>(x1);
        }
        while (!(v[0] & 1u)) {
            detail::inv_shr1(v);
            detail::inv_half<C>(x2);
        }
        if (detail::inv_geq(u, v)) {
            detail::inv_sub(u, v);
            detail::inv_sub_mod<C>(x1, x2);
        } else {
            detail::inv_sub(v, u);
            detail::inv_sub_mod<C>(x2, x1);
        }
    }
    Fe<C> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = detail::inv_is_one(u) ? x1[i] : x2[i];
    return r * fe_rr<C>() * fe_rr<C>();
}
#endif

// inverse of a (Montgomery form); inverse of 0 is 0.  Host: Fermat (a^{m-2});
// device: the binary algorithm above
template <class C>
ACE_HD Fe<C> fe_inv(const Fe<C>& a) {
#if defined(__CUDA_ARCH__)
    return d_inv_binary<C>(a);
#else
    uint32_t e[8];
    for (int i = 0; i < 8; i++) e[i] = mod_limb<C>(i);
    e[0] -= 2;  // m is odd and > 2: no borrow
    return fe_pow(a, e);
#endif
}

// ---------------------------------------------------------------------------
// Fp2 = Fp[u]/(u^2 + 1)
// ---------------------------------------------------------------------------
struct fp2_t {
    fp_t c0, c1;
};
ACE_HD fp2_t operator+(const fp2_t& a, const fp2_t& b) { return {a.c0 + b.c0, a.c1 + b.c1}; }
ACE_HD fp2_t operator-(const fp2_t& a, const fp2_t& b) { return {a.c0 - b.c0, a.c1 - b.c1}; }
// Karatsuba: (a0 b0 - a1 b1) + ((a0 + a1)(b0 + b1) - a0 b0 - a1 b1) u.
// On the device the three products stay unreduced (512 bits) and only the two
// coefficients are reduced (lazy reduction, Aranha, Karabina, Longa, Gebotys
// and Lopez, Eurocrypt 2011): with p < 2^254 both inputs to the reduction lie
// in [0, p 2^256) -- a0 b0 - a1 b1 after adding p 2^256 when it is negative,
// and a0 b1 + a1 b0 < 2 p^2 -- so each needs one conditional subtraction.
#if defined(__CUDA_ARCH__)
ACE_DEV void d_fp2_mul(fp2_t& r, const fp2_t& a, const fp2_t& b) {
    uint32_t t0[16], t1[16], t2[16], sa[8], sb[8];
    d_mul512(t0, a.c0.v, b.c0.v);
    d_mul512(t1, a.c1.v, b.c1.v);
    d_add_raw(sa, a.c0.v, a.c1.v);
    d_add_raw(sb, b.c0.v, b.c1.v);
    d_mul512(t2, sa, sb);
    d_sub512(t2, t0);
    d_sub512(t2, t1);
    uint32_t br = d_sub512(t0, t1);
    d_add_hi_mod<FpCfg>(t0, br);
    d_redc512<FpCfg>(r.c0.v, t0);
    d_redc512<FpCfg>(r.c1.v, t2);
}
#if defined(ACE_FIELD_MUL_CALL)
static __device__ __noinline__ fp2_t d_fp2_mul_call(const fp2_t a, const fp2_t b) {
    fp2_t r;
    d_fp2_mul(r, a, b);
    return r;
}
#endif
#endif
ACE_HD fp2_t operator*(const fp2_t& a, const fp2_t& b) {
#if defined(__CUDA_ARCH__) && defined(ACE_FIELD_MUL_CALL)
    return d_fp2_mul_call(a, b);
#elif defined(__CUDA_ARCH__)
    fp2_t r;
    d_fp2_mul(r, a, b);
    return r;
#else
    fp_t v0 = a.c0 * b.c0;
    fp_t v1 = a.c1 * b.c1;
    fp_t s = (a.c0 + a.c1) * (b.c0 + b.c1);
    return {v0 - v1, s - v0 - v1};
#endif
}
ACE_HD fp2_t fe_sqr(const fp2_t& a) {
    // (a0 + a1)(a0 - a1) + 2 a0 a1 u
    fp_t t = a.c0 * a.c1;
    return {(a.c0 + a.c1) * (a.c0 - a.c1), t + t};
}
// a b - c d in Fp2 with two reductions (instead of four): each coefficient's
// true value lies in (-2p^2, 2p^2), so the 512-bit two's-complement
// combination of the six unreduced products is exact; a negative one gets
// p 2^256 added (2 p^2 < p 2^256) before the reduction.
#if defined(__CUDA_ARCH__)
ACE_DEV void d_fp2_mul_sub(fp2_t& r, const fp2_t& a, const fp2_t& b, const fp2_t& c, const fp2_t& d) {
    // products P0 = a0 b0, P1 = a1 b1, P2 = (a0 + a1)(b0 + b1), Q0, Q1, Q2 the
    // same for c, d:  c0 = P0 - P1 - Q0 + Q1,  c1 = P2 - P0 - P1 - Q2 + Q0 + Q1
    uint32_t x[16], y[16], t[16], sa[8], sb[8];
    d_mul512(x, a.c0.v, b.c0.v);
#pragma unroll
    for (int i = 0; i < 16; i++) y[i] = 0;
    d_sub512(y, x);
    d_mul512(t, a.c1.v, b.c1.v);
    d_sub512(x, t);
    d_sub512(y, t);
    d_add_raw(sa, a.c0.v, a.c1.v);
    d_add_raw(sb, b.c0.v, b.c1.v);
    d_mul512(t, sa, sb);
    d_add512(y, t);
    d_mul512(t, c.c0.v, d.c0.v);
    d_sub512(x, t);
    d_add512(y, t);
    d_mul512(t, c.c1.v, d.c1.v);
    d_add512(x, t);
    d_add512(y, t);
    d_add_raw(sa, c.c0.v, c.c1.v);
    d_add_raw(sb, d.c0.v, d.c1.v);
    d_mul512(t, sa, sb);
    d_sub512(y, t);
    d_add_hi_mod<FpCfg>(x, 0u - (x[15] >> 31));
    d_add_hi_mod<FpCfg>(y, 0u - (y[15] >> 31));
    d_redc512<FpCfg>(r.c0.v, x);
    d_redc512<FpCfg>(r.c1.v, y);
}
#if defined(ACE_FIELD_MUL_CALL)
static __device__ __noinline__ fp2_t d_fp2_mul_sub_call(const fp2_t a, const fp2_t b, const fp2_t c, const fp2_t d) {
    fp2_t r;
    d_fp2_mul_sub(r, a, b, c, d);
    return r;
}
#endif
#endif
ACE_HD fp2_t fe_mul_sub(const fp2_t& a, const fp2_t& b, const fp2_t& c, const fp2_t& d) {
#if defined(__CUDA_ARCH__) && defined(ACE_FIELD_MUL_CALL)
    return d_fp2_mul_sub_call(a, b, c, d);
#elif defined(__CUDA_ARCH__)
    fp2_t r;
    d_fp2_mul_sub(r, a, b, c, d);
    return r;
#else
    return a * b - c * d;
#endif
}
ACE_HD fp2_t fe_dbl(const fp2_t& a) { return {a.c0 + a.c0, a.c1 + a.c1}; }
ACE_HD fp2_t fe_neg(const fp2_t& a) { return {fe_neg(a.c0), fe_neg(a.c1)}; }
ACE_HD bool fe_is_zero(const fp2_t& a) { return fe_is_zero(a.c0) && fe_is_zero(a.c1); }
ACE_HD bool fe_eq(const fp2_t& a, const fp2_t& b) { return fe_eq(a.c0, b.c0) && fe_eq(a.c1, b.c1); }
ACE_HD fp2_t fe_inv(const fp2_t& a) {
    fp_t n = a.c0 * a.c0 + a.c1 * a.c1;
    fp_t ni = fe_inv(n);
    return {a.c0 * ni, fe_neg(a.c1 * ni)};
}
ACE_HD fp2_t fe_to_mont(const fp2_t& a) { return {fe_to_mont(a.c0), fe_to_mont(a.c1)}; }
ACE_HD fp2_t fe_from_mont(const fp2_t& a) { return {fe_from_mont(a.c0), fe_from_mont(a.c1)}; }

template <class F>
ACE_HD F field_zero();
template <>
ACE_HD fp_t field_zero<fp_t>() { return fe_zero<FpCfg>(); }
template <>
ACE_HD fr_t field_zero<fr_t>() { return fe_zero<FrCfg>(); }
template <>
ACE_HD fp2_t field_zero<fp2_t>() { return {fe_zero<FpCfg>(), fe_zero<FpCfg>()}; }
template <class F>
ACE_HD F field_one();
template <>
ACE_HD fp_t field_one<fp_t>() { return fe_one<FpCfg>(); }
template <>
ACE_HD fr_t field_one<fr_t>() { return fe_one<FrCfg>(); }
template <>
ACE_HD fp2_t field_one<fp2_t>() { return {fe_one<FpCfg>(), fe_zero<FpCfg>()}; }

}  // namespace ace
