/*
 * groth16_oracle.c -- plain, slow, CPU reference for the Groth16/BN254 prover.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The product
 * path (paper_2603_10242_gb300) never imports, links or executes it, and the
 * two share no code: this file has its own 4x64-bit Montgomery field, its own
 * Jacobian curve formulas, its own NTT, its own SplitMix64 and its own circuit
 * builder.
 *
 * What it computes, and where that is defined:
 *   - The proof is Groth16.Prove(C, w, pub) of the paper's Phase 2
 *     (Section 3.1, Algorithm 1 ProveAsync; Section 3.3 Algorithm 3 Stage 1),
 *     over BN254 (Section 3.3, "ZK-ACE circuit specification"), serialised to
 *     the 256-byte proof of Section 3.3 / Appendix B.  The construction itself
 *     (QAP, setup, prover, verifier) is Groth 2016, which the paper cites and
 *     does not restate; this file writes it out in its textbook form.
 *   - Verification is the three-pairing check of Section 3.3 / Section 3.4
 *     (Algorithm 4 UpdateFinality), here with the reduced Tate pairing.
 *   - The synthetic circuit is a Poseidon-style permutation (the identity
 *     commitment of Section 2.1, Definition "ZK Identity Commitment") plus
 *     chained squaring gates and bit-packing rows.  Its exact recipe is a
 *     reading of the paper, fixed identically on both sides.
 *
 * Everything is deliberately plain: schoolbook operations, affine or textbook
 * Jacobian formulas, double-and-add scalar multiplication, an iterative
 * radix-2 NTT with an explicit bit-reversal, h by a 2N-point convolution and
 * long division by X^N - 1 (not the coset method the GPU uses), and the Tate
 * pairing with a plain square-and-multiply final exponentiation.
 *
 * All field elements are kept in Montgomery form internally; every exported
 * function takes and returns canonical little-endian 32-byte values.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------- */
/* 256-bit prime fields in Montgomery form (R = 2^256), 4 x 64-bit limbs.     */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t v[4]; } fe;

typedef struct {
    uint64_t p[4];   /* modulus, little-endian */
    uint64_t pinv;   /* -p^{-1} mod 2^64 */
    fe one;          /* R mod p  (Montgomery form of 1) */
    fe r2;           /* R^2 mod p */
} field;

static field FP, FR;
static int g_inited = 0;

/* BN254 base-field modulus p and scalar-field modulus r (BN parameter
 * x = 4965661367192848881, p = 36x^4+36x^3+24x^2+6x+1, r = 36x^4+36x^3+18x^2+6x+1). */
static const uint64_t P_LIMBS[4] = {0x3c208c16d87cfd47ULL, 0x97816a916871ca8dULL,
                                    0xb85045b68181585dULL, 0x30644e72e131a029ULL};
static const uint64_t R_LIMBS[4] = {0x43e1f593f0000001ULL, 0x2833e84879b97091ULL,
                                    0xb85045b68181585dULL, 0x30644e72e131a029ULL};

static int geq4(const uint64_t a[4], const uint64_t b[4]) {
    for (int i = 3; i >= 0; i--) {
        if (a[i] > b[i]) return 1;
        if (a[i] < b[i]) return 0;
    }
    return 1;
}

static uint64_t add4(uint64_t r[4], const uint64_t a[4], const uint64_t b[4]) {
    u128 c = 0;
    for (int i = 0; i < 4; i++) {
        c += (u128)a[i] + b[i];
        r[i] = (uint64_t)c;
        c >>= 64;
    }
    return (uint64_t)c;
}

static uint64_t sub4(uint64_t r[4], const uint64_t a[4], const uint64_t b[4]) {
    uint64_t borrow = 0;
    for (int i = 0; i < 4; i++) {
        uint64_t ai = a[i], bi = b[i];
        uint64_t d = ai - bi - borrow;
        borrow = (ai < bi) || (ai == bi && borrow) ? 1 : 0;
        r[i] = d;
    }
    return borrow;
}

static void f_add(const field* F, fe* r, const fe* a, const fe* b) {
    uint64_t t[4];
    uint64_t c = add4(t, a->v, b->v);
    if (c || geq4(t, F->p)) sub4(t, t, F->p);
    memcpy(r->v, t, sizeof t);
}

static void f_sub(const field* F, fe* r, const fe* a, const fe* b) {
    uint64_t t[4];
    uint64_t br = sub4(t, a->v, b->v);
    if (br) add4(t, t, F->p);
    memcpy(r->v, t, sizeof t);
}

static void f_neg(const field* F, fe* r, const fe* a) {
    fe z = {{0, 0, 0, 0}};
    f_sub(F, r, &z, a);
}

/* Montgomery product a*b*R^{-1} mod p, coarsely integrated operand scanning
 * (Montgomery 1985; Koc, Acar, Kaliski 1996). */
static void f_mul(const field* F, fe* r, const fe* a, const fe* b) {
    uint64_t t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 4; i++) {
        u128 c = 0;
        for (int j = 0; j < 4; j++) {
            c += (u128)t[j] + (u128)a->v[j] * b->v[i];
            t[j] = (uint64_t)c;
            c >>= 64;
        }
        c += t[4];
        t[4] = (uint64_t)c;
        t[5] = (uint64_t)(c >> 64);
        uint64_t m = t[0] * F->pinv;
        c = (u128)t[0] + (u128)m * F->p[0];
        c >>= 64;
        for (int j = 1; j < 4; j++) {
            c += (u128)t[j] + (u128)m * F->p[j];
            t[j - 1] = (uint64_t)c;
            c >>= 64;
        }
        c += t[4];
        t[3] = (uint64_t)c;
        t[4] = t[5] + (uint64_t)(c >> 64);
    }
    uint64_t res[4] = {t[0], t[1], t[2], t[3]};
    if (t[4] || geq4(res, F->p)) sub4(res, res, F->p);
    memcpy(r->v, res, sizeof res);
}

static int f_is_zero(const fe* a) { return (a->v[0] | a->v[1] | a->v[2] | a->v[3]) == 0; }
static int f_eq(const fe* a, const fe* b) { return memcmp(a->v, b->v, sizeof a->v) == 0; }

static void f_to_mont(const field* F, fe* r, const fe* a) { f_mul(F, r, a, &F->r2); }
static void f_from_mont(const field* F, fe* r, const fe* a) {
    fe one = {{1, 0, 0, 0}};
    f_mul(F, r, a, &one);
}

/* a^e for a 256-bit exponent e (plain integer, little-endian limbs). */
static void f_pow(const field* F, fe* r, const fe* a, const uint64_t e[4]) {
    fe acc = F->one, base = *a;
    for (int i = 0; i < 256; i++) {
        if ((e[i >> 6] >> (i & 63)) & 1) f_mul(F, &acc, &acc, &base);
        f_mul(F, &base, &base, &base);
    }
    *r = acc;
}

/* Inverse by Fermat: a^{p-2}.  The inverse of 0 is returned as 0. */
static void f_inv(const field* F, fe* r, const fe* a) {
    uint64_t e[4];
    uint64_t two[4] = {2, 0, 0, 0};
    sub4(e, F->p, two);
    f_pow(F, r, a, e);
}

static void f_from_u64(const field* F, fe* r, uint64_t x) {
    fe t = {{x, 0, 0, 0}};
    f_to_mont(F, r, &t);
}

static void field_init(field* F, const uint64_t p[4]) {
    memcpy(F->p, p, sizeof F->p);
    /* Newton iteration for p^{-1} mod 2^64, then negate. */
    uint64_t x = 1;
    for (int i = 0; i < 7; i++) x *= 2 - p[0] * x;
    F->pinv = (uint64_t)0 - x;
    /* R mod p and R^2 mod p by repeated doubling of 1 modulo p. */
    uint64_t t[4] = {1, 0, 0, 0};
    for (int i = 0; i < 512; i++) {
        uint64_t c = add4(t, t, t);
        if (c || geq4(t, p)) sub4(t, t, p);
        if (i == 255) memcpy(F->one.v, t, sizeof t);
    }
    memcpy(F->r2.v, t, sizeof t);
}

/* canonical little-endian bytes <-> Montgomery element.  Returns 0 if the
 * value is not < modulus. */
static int fe_from_bytes(const field* F, fe* r, const uint8_t b[32]) {
    fe t;
    for (int i = 0; i < 4; i++) {
        uint64_t w = 0;
        for (int k = 7; k >= 0; k--) w = (w << 8) | b[8 * i + k];
        t.v[i] = w;
    }
    if (geq4(t.v, F->p)) return 0;
    f_to_mont(F, r, &t);
    return 1;
}

static void fe_to_bytes(const field* F, uint8_t b[32], const fe* a) {
    fe t;
    f_from_mont(F, &t, a);
    for (int i = 0; i < 4; i++)
        for (int k = 0; k < 8; k++) b[8 * i + k] = (uint8_t)(t.v[i] >> (8 * k));
}

/* canonical (non-Montgomery) limbs of a Montgomery element */
static void fe_canon(const field* F, uint64_t out[4], const fe* a) {
    fe t;
    f_from_mont(F, &t, a);
    memcpy(out, t.v, 4 * sizeof(uint64_t));
}

/* ------------------------------------------------------------------------- */
/* Fp2 = Fp[u]/(u^2 + 1)                                                       */
/* ------------------------------------------------------------------------- */

typedef struct { fe c0, c1; } fe2;

static void f2_add(fe2* r, const fe2* a, const fe2* b) {
    f_add(&FP, &r->c0, &a->c0, &b->c0);
    f_add(&FP, &r->c1, &a->c1, &b->c1);
}
static void f2_sub(fe2* r, const fe2* a, const fe2* b) {
    f_sub(&FP, &r->c0, &a->c0, &b->c0);
    f_sub(&FP, &r->c1, &a->c1, &b->c1);
}
/* (a0 + a1 u)(b0 + b1 u) = (a0 b0 - a1 b1) + (a0 b1 + a1 b0) u, schoolbook. */
static void f2_mul(fe2* r, const fe2* a, const fe2* b) {
    fe t0, t1, t2, t3;
    f_mul(&FP, &t0, &a->c0, &b->c0);
    f_mul(&FP, &t1, &a->c1, &b->c1);
    f_mul(&FP, &t2, &a->c0, &b->c1);
    f_mul(&FP, &t3, &a->c1, &b->c0);
    f_sub(&FP, &r->c0, &t0, &t1);
    f_add(&FP, &r->c1, &t2, &t3);
}
/* 1/(a0 + a1 u) = (a0 - a1 u)/(a0^2 + a1^2) */
static void f2_inv(fe2* r, const fe2* a) {
    fe n, t, inv;
    f_mul(&FP, &n, &a->c0, &a->c0);
    f_mul(&FP, &t, &a->c1, &a->c1);
    f_add(&FP, &n, &n, &t);
    f_inv(&FP, &inv, &n);
    f_mul(&FP, &r->c0, &a->c0, &inv);
    f_mul(&FP, &t, &a->c1, &inv);
    f_neg(&FP, &r->c1, &t);
}
static int f2_is_zero(const fe2* a) { return f_is_zero(&a->c0) && f_is_zero(&a->c1); }
static int f2_eq(const fe2* a, const fe2* b) { return f_eq(&a->c0, &b->c0) && f_eq(&a->c1, &b->c1); }

/* ------------------------------------------------------------------------- */
/* Fp12 = Fp[w]/(w^12 - 18 w^6 + 82).  With u := w^6 - 9 one has u^2 = -1, so */
/* Fp2 embeds as a0 + a1 u = (a0 - 9 a1) + a1 w^6, and w^6 = 9 + u = xi, the  */
/* sextic non-residue of the BN254 twist.                                     */
/* ------------------------------------------------------------------------- */

typedef struct { fe c[12]; } fe12;

static void f12_zero(fe12* r) { memset(r, 0, sizeof *r); }
static void f12_one(fe12* r) { f12_zero(r); r->c[0] = FP.one; }
static void f12_sub(fe12* r, const fe12* a, const fe12* b) {
    for (int i = 0; i < 12; i++) f_sub(&FP, &r->c[i], &a->c[i], &b->c[i]);
}
static void f12_mul(fe12* r, const fe12* a, const fe12* b) {
    fe t[23];
    memset(t, 0, sizeof t);
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 12; j++) {
            fe pr;
            f_mul(&FP, &pr, &a->c[i], &b->c[j]);
            f_add(&FP, &t[i + j], &t[i + j], &pr);
        }
    fe c18, c82;
    f_from_u64(&FP, &c18, 18);
    f_from_u64(&FP, &c82, 82);
    /* w^k = w^{k-12} (18 w^6 - 82) for k >= 12 */
    for (int k = 22; k >= 12; k--) {
        fe x;
        f_mul(&FP, &x, &t[k], &c18);
        f_add(&FP, &t[k - 6], &t[k - 6], &x);
        f_mul(&FP, &x, &t[k], &c82);
        f_sub(&FP, &t[k - 12], &t[k - 12], &x);
    }
    for (int i = 0; i < 12; i++) r->c[i] = t[i];
}
static void f12_scale(fe12* r, const fe12* a, const fe* s) {
    for (int i = 0; i < 12; i++) f_mul(&FP, &r->c[i], &a->c[i], s);
}
static int f12_eq(const fe12* a, const fe12* b) {
    for (int i = 0; i < 12; i++)
        if (!f_eq(&a->c[i], &b->c[i])) return 0;
    return 1;
}
/* a^e, e a little-endian multi-limb integer of nlimbs 64-bit words */
static void f12_pow(fe12* r, const fe12* a, const uint64_t* e, int nlimbs) {
    fe12 acc, base = *a;
    f12_one(&acc);
    int top = nlimbs * 64 - 1;
    while (top >= 0 && !((e[top >> 6] >> (top & 63)) & 1)) top--;
    for (int i = top; i >= 0; i--) {
        f12_mul(&acc, &acc, &acc);
        if ((e[i >> 6] >> (i & 63)) & 1) f12_mul(&acc, &acc, &base);
    }
    *r = acc;
}

/* ------------------------------------------------------------------------- */
/* G1: y^2 = x^3 + 3 over Fp.  G2: y^2 = x^3 + 3/(9+u) over Fp2.              */
/* Jacobian coordinates (X, Y, Z) with x = X/Z^2, y = Y/Z^3; Z = 0 is O.       */
/* ------------------------------------------------------------------------- */

typedef struct { fe x, y; int inf; } g1a;
typedef struct { fe X, Y, Z; } g1j;
typedef struct { fe2 x, y; int inf; } g2a;
typedef struct { fe2 X, Y, Z; } g2j;

static fe B_G1;    /* 3 */
static fe2 B_G2;   /* 3/(9+u) */
static g1a G1_GEN; /* (1, 2) */
static g2a G2_GEN; /* EIP-197 generator */

static void g1j_set_inf(g1j* r) { memset(r, 0, sizeof *r); r->X = FP.one; r->Y = FP.one; }
static int g1j_is_inf(const g1j* a) { return f_is_zero(&a->Z); }
static void g1j_from_affine(g1j* r, const g1a* a) {
    if (a->inf) { g1j_set_inf(r); return; }
    r->X = a->x; r->Y = a->y; r->Z = FP.one;
}
static void g1j_to_affine(g1a* r, const g1j* a) {
    if (g1j_is_inf(a)) { memset(r, 0, sizeof *r); r->inf = 1; return; }
    fe zi, zi2, zi3;
    f_inv(&FP, &zi, &a->Z);
    f_mul(&FP, &zi2, &zi, &zi);
    f_mul(&FP, &zi3, &zi2, &zi);
    f_mul(&FP, &r->x, &a->X, &zi2);
    f_mul(&FP, &r->y, &a->Y, &zi3);
    r->inf = 0;
}
/* Doubling for a = 0 (textbook Jacobian: lambda = 3x^2/2y). */
static void g1j_dbl(g1j* r, const g1j* a) {
    if (g1j_is_inf(a) || f_is_zero(&a->Y)) { g1j_set_inf(r); return; }
    fe XX, YY, YYYY, S, M, T, X3, Y3, Z3;
    f_mul(&FP, &XX, &a->X, &a->X);
    f_mul(&FP, &YY, &a->Y, &a->Y);
    f_mul(&FP, &YYYY, &YY, &YY);
    f_mul(&FP, &S, &a->X, &YY);            /* S = 4 X Y^2 */
    f_add(&FP, &S, &S, &S);
    f_add(&FP, &S, &S, &S);
    f_add(&FP, &M, &XX, &XX);              /* M = 3 X^2 */
    f_add(&FP, &M, &M, &XX);
    f_mul(&FP, &X3, &M, &M);               /* X3 = M^2 - 2S */
    f_sub(&FP, &X3, &X3, &S);
    f_sub(&FP, &X3, &X3, &S);
    f_sub(&FP, &T, &S, &X3);               /* Y3 = M(S - X3) - 8 Y^4 */
    f_mul(&FP, &Y3, &M, &T);
    f_add(&FP, &T, &YYYY, &YYYY);
    f_add(&FP, &T, &T, &T);
    f_add(&FP, &T, &T, &T);
    f_sub(&FP, &Y3, &Y3, &T);
    f_mul(&FP, &Z3, &a->Y, &a->Z);         /* Z3 = 2 Y Z */
    f_add(&FP, &Z3, &Z3, &Z3);
    r->X = X3; r->Y = Y3; r->Z = Z3;
}
static void g1j_add(g1j* r, const g1j* a, const g1j* b) {
    if (g1j_is_inf(a)) { *r = *b; return; }
    if (g1j_is_inf(b)) { *r = *a; return; }
    fe Z1Z1, Z2Z2, U1, U2, S1, S2, H, Rr, HH, HHH, V, t;
    f_mul(&FP, &Z1Z1, &a->Z, &a->Z);
    f_mul(&FP, &Z2Z2, &b->Z, &b->Z);
    f_mul(&FP, &U1, &a->X, &Z2Z2);
    f_mul(&FP, &U2, &b->X, &Z1Z1);
    f_mul(&FP, &S1, &a->Y, &b->Z);
    f_mul(&FP, &S1, &S1, &Z2Z2);
    f_mul(&FP, &S2, &b->Y, &a->Z);
    f_mul(&FP, &S2, &S2, &Z1Z1);
    f_sub(&FP, &H, &U2, &U1);
    f_sub(&FP, &Rr, &S2, &S1);
    if (f_is_zero(&H)) {
        if (f_is_zero(&Rr)) { g1j_dbl(r, a); return; }
        g1j_set_inf(r);
        return;
    }
    f_mul(&FP, &HH, &H, &H);
    f_mul(&FP, &HHH, &H, &HH);
    f_mul(&FP, &V, &U1, &HH);
    g1j out;
    f_mul(&FP, &out.X, &Rr, &Rr);                 /* X3 = R^2 - H^3 - 2 U1 H^2 */
    f_sub(&FP, &out.X, &out.X, &HHH);
    f_sub(&FP, &out.X, &out.X, &V);
    f_sub(&FP, &out.X, &out.X, &V);
    f_sub(&FP, &t, &V, &out.X);                   /* Y3 = R (U1 H^2 - X3) - S1 H^3 */
    f_mul(&FP, &out.Y, &Rr, &t);
    f_mul(&FP, &t, &S1, &HHH);
    f_sub(&FP, &out.Y, &out.Y, &t);
    f_mul(&FP, &out.Z, &a->Z, &b->Z);             /* Z3 = Z1 Z2 H */
    f_mul(&FP, &out.Z, &out.Z, &H);
    *r = out;
}
static void g1j_neg(g1j* r, const g1j* a) { *r = *a; f_neg(&FP, &r->Y, &a->Y); }
/* double-and-add, most significant bit first; k is a canonical 256-bit integer */
static void g1j_mul(g1j* r, const g1j* a, const uint64_t k[4]) {
    g1j acc;
    g1j_set_inf(&acc);
    for (int i = 255; i >= 0; i--) {
        g1j_dbl(&acc, &acc);
        if ((k[i >> 6] >> (i & 63)) & 1) g1j_add(&acc, &acc, a);
    }
    *r = acc;
}
static int g1a_on_curve(const g1a* a) {
    if (a->inf) return 1;
    fe l, rr;
    f_mul(&FP, &l, &a->y, &a->y);
    f_mul(&FP, &rr, &a->x, &a->x);
    f_mul(&FP, &rr, &rr, &a->x);
    f_add(&FP, &rr, &rr, &B_G1);
    return f_eq(&l, &rr);
}

static void g2j_set_inf(g2j* r) {
    memset(r, 0, sizeof *r);
    r->X.c0 = FP.one; r->Y.c0 = FP.one;
}
static int g2j_is_inf(const g2j* a) { return f2_is_zero(&a->Z); }
static void g2j_from_affine(g2j* r, const g2a* a) {
    if (a->inf) { g2j_set_inf(r); return; }
    r->X = a->x; r->Y = a->y;
    memset(&r->Z, 0, sizeof r->Z);
    r->Z.c0 = FP.one;
}
static void g2j_to_affine(g2a* r, const g2j* a) {
    if (g2j_is_inf(a)) { memset(r, 0, sizeof *r); r->inf = 1; return; }
    fe2 zi, zi2, zi3;
    f2_inv(&zi, &a->Z);
    f2_mul(&zi2, &zi, &zi);
    f2_mul(&zi3, &zi2, &zi);
    f2_mul(&r->x, &a->X, &zi2);
    f2_mul(&r->y, &a->Y, &zi3);
    r->inf = 0;
}
static void g2j_dbl(g2j* r, const g2j* a) {
    if (g2j_is_inf(a) || f2_is_zero(&a->Y)) { g2j_set_inf(r); return; }
    fe2 XX, YY, YYYY, S, M, T, X3, Y3, Z3;
    f2_mul(&XX, &a->X, &a->X);
    f2_mul(&YY, &a->Y, &a->Y);
    f2_mul(&YYYY, &YY, &YY);
    f2_mul(&S, &a->X, &YY);
    f2_add(&S, &S, &S);
    f2_add(&S, &S, &S);
    f2_add(&M, &XX, &XX);
    f2_add(&M, &M, &XX);
    f2_mul(&X3, &M, &M);
    f2_sub(&X3, &X3, &S);
    f2_sub(&X3, &X3, &S);
    f2_sub(&T, &S, &X3);
    f2_mul(&Y3, &M, &T);
    f2_add(&T, &YYYY, &YYYY);
    f2_add(&T, &T, &T);
    f2_add(&T, &T, &T);
    f2_sub(&Y3, &Y3, &T);
    f2_mul(&Z3, &a->Y, &a->Z);
    f2_add(&Z3, &Z3, &Z3);
    r->X = X3; r->Y = Y3; r->Z = Z3;
}
static void g2j_add(g2j* r, const g2j* a, const g2j* b) {
    if (g2j_is_inf(a)) { *r = *b; return; }
    if (g2j_is_inf(b)) { *r = *a; return; }
    fe2 Z1Z1, Z2Z2, U1, U2, S1, S2, H, Rr, HH, HHH, V, t;
    f2_mul(&Z1Z1, &a->Z, &a->Z);
    f2_mul(&Z2Z2, &b->Z, &b->Z);
    f2_mul(&U1, &a->X, &Z2Z2);
    f2_mul(&U2, &b->X, &Z1Z1);
    f2_mul(&S1, &a->Y, &b->Z);
    f2_mul(&S1, &S1, &Z2Z2);
    f2_mul(&S2, &b->Y, &a->Z);
    f2_mul(&S2, &S2, &Z1Z1);
    f2_sub(&H, &U2, &U1);
    f2_sub(&Rr, &S2, &S1);
    if (f2_is_zero(&H)) {
        if (f2_is_zero(&Rr)) { g2j_dbl(r, a); return; }
        g2j_set_inf(r);
        return;
    }
    f2_mul(&HH, &H, &H);
    f2_mul(&HHH, &H, &HH);
    f2_mul(&V, &U1, &HH);
    g2j out;
    f2_mul(&out.X, &Rr, &Rr);
    f2_sub(&out.X, &out.X, &HHH);
    f2_sub(&out.X, &out.X, &V);
    f2_sub(&out.X, &out.X, &V);
    f2_sub(&t, &V, &out.X);
    f2_mul(&out.Y, &Rr, &t);
    f2_mul(&t, &S1, &HHH);
    f2_sub(&out.Y, &out.Y, &t);
    f2_mul(&out.Z, &a->Z, &b->Z);
    f2_mul(&out.Z, &out.Z, &H);
    *r = out;
}
static void g2j_mul(g2j* r, const g2j* a, const uint64_t k[4]) {
    g2j acc;
    g2j_set_inf(&acc);
    for (int i = 255; i >= 0; i--) {
        g2j_dbl(&acc, &acc);
        if ((k[i >> 6] >> (i & 63)) & 1) g2j_add(&acc, &acc, a);
    }
    *r = acc;
}
static int g2a_on_curve(const g2a* a) {
    if (a->inf) return 1;
    fe2 l, rr;
    f2_mul(&l, &a->y, &a->y);
    f2_mul(&rr, &a->x, &a->x);
    f2_mul(&rr, &rr, &a->x);
    f2_add(&rr, &rr, &B_G2);
    return f2_eq(&l, &rr);
}

/* Serialisation: G1 affine = x || y (64 B), G2 affine = x.c0 || x.c1 || y.c0 ||
 * y.c1 (128 B), each coordinate 32 B little-endian canonical; O = all zeros. */
static void g1a_to_bytes(uint8_t* b, const g1a* a) {
    if (a->inf) { memset(b, 0, 64); return; }
    fe_to_bytes(&FP, b, &a->x);
    fe_to_bytes(&FP, b + 32, &a->y);
}
static int g1a_from_bytes(g1a* a, const uint8_t* b) {
    int z = 1;
    for (int i = 0; i < 64; i++) z &= (b[i] == 0);
    if (z) { memset(a, 0, sizeof *a); a->inf = 1; return 1; }
    a->inf = 0;
    return fe_from_bytes(&FP, &a->x, b) && fe_from_bytes(&FP, &a->y, b + 32);
}
static void g2a_to_bytes(uint8_t* b, const g2a* a) {
    if (a->inf) { memset(b, 0, 128); return; }
    fe_to_bytes(&FP, b, &a->x.c0);
    fe_to_bytes(&FP, b + 32, &a->x.c1);
    fe_to_bytes(&FP, b + 64, &a->y.c0);
    fe_to_bytes(&FP, b + 96, &a->y.c1);
}
static int g2a_from_bytes(g2a* a, const uint8_t* b) {
    int z = 1;
    for (int i = 0; i < 128; i++) z &= (b[i] == 0);
    if (z) { memset(a, 0, sizeof *a); a->inf = 1; return 1; }
    a->inf = 0;
    return fe_from_bytes(&FP, &a->x.c0, b) && fe_from_bytes(&FP, &a->x.c1, b + 32) &&
           fe_from_bytes(&FP, &a->y.c0, b + 64) && fe_from_bytes(&FP, &a->y.c1, b + 96);
}

static void fe_from_dec(const field* F, fe* r, const char* s) {
    /* decimal string -> canonical limbs -> Montgomery */
    uint64_t t[4] = {0, 0, 0, 0};
    for (; *s; s++) {
        u128 c = (u128)(*s - '0');
        for (int i = 0; i < 4; i++) {
            c += (u128)t[i] * 10;
            t[i] = (uint64_t)c;
            c >>= 64;
        }
    }
    fe x;
    memcpy(x.v, t, sizeof t);
    f_to_mont(F, r, &x);
}

/* ------------------------------------------------------------------------- */
/* Multi-limb integer helper for the final exponent (p^12 - 1)/r.              */
/* ------------------------------------------------------------------------- */

#define BIG_LIMBS 52
static uint64_t FINAL_EXP[BIG_LIMBS];
static int FINAL_EXP_LIMBS;

static void big_mul_small4(uint64_t* acc, int n, const uint64_t m[4]) {
    uint64_t out[BIG_LIMBS + 4];
    memset(out, 0, sizeof out);
    for (int i = 0; i < n; i++) {
        u128 c = 0;
        for (int j = 0; j < 4; j++) {
            c += (u128)out[i + j] + (u128)acc[i] * m[j];
            out[i + j] = (uint64_t)c;
            c >>= 64;
        }
        int k = i + 4;
        while (c) {
            c += out[k];
            out[k] = (uint64_t)c;
            c >>= 64;
            k++;
        }
    }
    memcpy(acc, out, BIG_LIMBS * sizeof(uint64_t));
}

static void compute_final_exponent(void) {
    uint64_t acc[BIG_LIMBS];
    memset(acc, 0, sizeof acc);
    acc[0] = 1;
    for (int i = 0; i < 12; i++) big_mul_small4(acc, BIG_LIMBS - 4, P_LIMBS);
    /* acc -= 1 (acc = p^12 >= 1) */
    for (int i = 0; i < BIG_LIMBS; i++) {
        if (acc[i]--) break;
    }
    /* long division by r, bit by bit */
    uint64_t q[BIG_LIMBS];
    memset(q, 0, sizeof q);
    uint64_t rem[5] = {0, 0, 0, 0, 0};
    for (int bit = BIG_LIMBS * 64 - 1; bit >= 0; bit--) {
        /* rem = 2 rem + bit */
        uint64_t carry = (acc[bit >> 6] >> (bit & 63)) & 1;
        for (int i = 0; i < 5; i++) {
            uint64_t nc = rem[i] >> 63;
            rem[i] = (rem[i] << 1) | carry;
            carry = nc;
        }
        /* if rem >= r: rem -= r, set q bit */
        int ge = rem[4] != 0 || geq4(rem, R_LIMBS);
        if (ge) {
            uint64_t b = sub4(rem, rem, R_LIMBS);
            rem[4] -= b;
            q[bit >> 6] |= (uint64_t)1 << (bit & 63);
        }
    }
    if (rem[0] | rem[1] | rem[2] | rem[3] | rem[4]) {
        fprintf(stderr, "oracle: r does not divide p^12-1\n");
        abort();
    }
    memcpy(FINAL_EXP, q, sizeof q);
    FINAL_EXP_LIMBS = BIG_LIMBS;
    while (FINAL_EXP_LIMBS > 1 && FINAL_EXP[FINAL_EXP_LIMBS - 1] == 0) FINAL_EXP_LIMBS--;
}

static void oracle_init(void) {
    if (g_inited) return;
    field_init(&FP, P_LIMBS);
    field_init(&FR, R_LIMBS);
    f_from_u64(&FP, &B_G1, 3);
    fe2 xi, xi_inv, three;
    f_from_u64(&FP, &xi.c0, 9);
    f_from_u64(&FP, &xi.c1, 1);
    f2_inv(&xi_inv, &xi);
    memset(&three, 0, sizeof three);
    f_from_u64(&FP, &three.c0, 3);
    f2_mul(&B_G2, &three, &xi_inv);
    G1_GEN.inf = 0;
    f_from_u64(&FP, &G1_GEN.x, 1);
    f_from_u64(&FP, &G1_GEN.y, 2);
    /* EIP-197 generator of the order-r subgroup of the twist */
    G2_GEN.inf = 0;
    fe_from_dec(&FP, &G2_GEN.x.c0, "10857046999023057135944570762232829481370756359578518086990519993285655852781");
    fe_from_dec(&FP, &G2_GEN.x.c1, "11559732032986387107991004021392285783925812861821192530917403151452391805634");
    fe_from_dec(&FP, &G2_GEN.y.c0, "8495653923123431417604973247489272438418190587263600148770280649306958101930");
    fe_from_dec(&FP, &G2_GEN.y.c1, "4082367875863433681332203403145435568316851327593401208105741076214120093531");
    compute_final_exponent();
    g_inited = 1;
}

/* ------------------------------------------------------------------------- */
/* Reduced Tate pairing e(P, Q) = f_{r,P}(psi(Q))^{(p^12-1)/r}.                */
/* psi untwists Q = (x', y') in E'(Fp2) to (x' w^2, y' w^3) in E(Fp12).        */
/* Vertical-line denominators lie in the subfield Fp[w^2] (degree 6) and are   */
/* sent to 1 by the final exponentiation, so Miller's loop omits them.         */
/* ------------------------------------------------------------------------- */

static void fp2_embed(fe12* r, const fe2* a) {
    /* a0 + a1 u with u = w^6 - 9 */
    f12_zero(r);
    fe t, nine;
    f_from_u64(&FP, &nine, 9);
    f_mul(&FP, &t, &a->c1, &nine);
    f_sub(&FP, &r->c[0], &a->c0, &t);
    r->c[6] = a->c1;
}

static void untwist(fe12* xq, fe12* yq, const g2a* q) {
    fe12 x, y;
    fp2_embed(&x, &q->x);
    fp2_embed(&y, &q->y);
    /* multiply by w^2 and w^3: shift coefficients (degrees stay < 12 since the
     * embedded values only use degrees 0 and 6). */
    f12_zero(xq);
    f12_zero(yq);
    for (int i = 0; i < 12; i++) {
        if (!f_is_zero(&x.c[i])) xq->c[i + 2] = x.c[i];
        if (!f_is_zero(&y.c[i])) yq->c[i + 3] = y.c[i];
    }
}

/* line through T with slope lam, evaluated at (xq, yq): yq - yT - lam (xq - xT) */
static void line_eval(fe12* out, const fe* lam, const fe* xT, const fe* yT, const fe12* xq, const fe12* yq) {
    fe12 t, lx;
    t = *xq;
    f_sub(&FP, &t.c[0], &t.c[0], xT);
    f12_scale(&lx, &t, lam);
    *out = *yq;
    f_sub(&FP, &out->c[0], &out->c[0], yT);
    f12_sub(out, out, &lx);
}

static void tate_pairing(fe12* out, const g1a* P, const g2a* Q) {
    if (P->inf || Q->inf) { f12_one(out); return; }
    fe12 xq, yq, f, l;
    untwist(&xq, &yq, Q);
    f12_one(&f);
    fe xT = P->x, yT = P->y;
    int Tinf = 0;
    int top = 253; /* r < 2^254, bit 253 set */
    for (int i = top - 1; i >= 0; i--) {
        /* doubling step: f = f^2 * l_{T,T}(Q) */
        f12_mul(&f, &f, &f);
        if (!Tinf) {
            fe num, den, lam, t;
            f_mul(&FP, &num, &xT, &xT);
            f_add(&FP, &t, &num, &num);
            f_add(&FP, &num, &t, &num);     /* 3 xT^2 */
            f_add(&FP, &den, &yT, &yT);     /* 2 yT (nonzero: T has odd order r) */
            f_inv(&FP, &den, &den);
            f_mul(&FP, &lam, &num, &den);
            line_eval(&l, &lam, &xT, &yT, &xq, &yq);
            f12_mul(&f, &f, &l);
            fe x3, y3;
            f_mul(&FP, &x3, &lam, &lam);
            f_sub(&FP, &x3, &x3, &xT);
            f_sub(&FP, &x3, &x3, &xT);
            f_sub(&FP, &t, &xT, &x3);
            f_mul(&FP, &y3, &lam, &t);
            f_sub(&FP, &y3, &y3, &yT);
            xT = x3; yT = y3;
        }
        if ((R_LIMBS[i >> 6] >> (i & 63)) & 1) {
            /* addition step: f = f * l_{T,P}(Q) */
            if (f_eq(&xT, &P->x)) {
                /* T = -P: the line is vertical (absorbed by the final
                 * exponentiation) and T + P = O. */
                Tinf = 1;
            } else {
                fe num, den, lam, t;
                f_sub(&FP, &num, &P->y, &yT);
                f_sub(&FP, &den, &P->x, &xT);
                f_inv(&FP, &den, &den);
                f_mul(&FP, &lam, &num, &den);
                line_eval(&l, &lam, &xT, &yT, &xq, &yq);
                f12_mul(&f, &f, &l);
                fe x3, y3;
                f_mul(&FP, &x3, &lam, &lam);
                f_sub(&FP, &x3, &x3, &xT);
                f_sub(&FP, &x3, &x3, &P->x);
                f_sub(&FP, &t, &xT, &x3);
                f_mul(&FP, &y3, &lam, &t);
                f_sub(&FP, &y3, &y3, &yT);
                xT = x3; yT = y3;
            }
        }
    }
    f12_pow(out, &f, FINAL_EXP, FINAL_EXP_LIMBS);
}

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood 2014) and the Fr sampler.                     */
/* Stream for (seed, purpose): state0 = seed XOR purpose * 0x9E3779B97F4A7C15.  */
/* Fr: four outputs as little-endian limbs, top two bits cleared, rejected     */
/* while >= r.                                                                  */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t s; } smx;
static void smx_init(smx* g, uint64_t seed, uint64_t purpose) { g->s = seed ^ (purpose * 0x9E3779B97F4A7C15ULL); }
static uint64_t smx_next(smx* g) {
    g->s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = g->s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* returns the canonical limbs */
static void smx_fr_canon(smx* g, uint64_t out[4]) {
    for (;;) {
        for (int i = 0; i < 4; i++) out[i] = smx_next(g);
        out[3] &= 0x3FFFFFFFFFFFFFFFULL;
        if (!geq4(out, R_LIMBS)) return;
    }
}
static void smx_fr(smx* g, fe* out) {
    fe t;
    smx_fr_canon(g, t.v);
    f_to_mont(&FR, out, &t);
}

enum {
    PURPOSE_ROUND_CONST = 1, PURPOSE_MDS = 2, PURPOSE_INPUTS = 3, PURPOSE_TOXIC = 4,
    PURPOSE_RS = 5, PURPOSE_BASES = 6, PURPOSE_SCALARS = 7, PURPOSE_SIZES = 8,
    PURPOSE_ARRIVALS = 9, PURPOSE_CHAIN = 10
};

/* ------------------------------------------------------------------------- */
/* NTT over Fr: omega_N = 5^{(r-1)/N} (5 is a non-residue mod r, and 2^28      */
/* divides r-1).  Plain iterative radix-2 Cooley-Tukey with an explicit         */
/* bit-reversal permutation; natural order in and out.                          */
/* ------------------------------------------------------------------------- */

static void fr_root_of_unity(fe* w, uint32_t log_n) {
    uint64_t e[4];
    uint64_t one[4] = {1, 0, 0, 0};
    sub4(e, R_LIMBS, one);
    for (uint32_t k = 0; k < log_n; k++) {
        for (int i = 0; i < 4; i++) e[i] = (e[i] >> 1) | (i < 3 ? (e[i + 1] << 63) : 0);
    }
    fe five;
    f_from_u64(&FR, &five, 5);
    f_pow(&FR, w, &five, e);
}

static size_t bitrev(size_t x, uint32_t bits) {
    size_t r = 0;
    for (uint32_t i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

static void ntt_inplace(fe* a, uint32_t log_n, int inverse) {
    size_t n = (size_t)1 << log_n;
    for (size_t i = 0; i < n; i++) {
        size_t j = bitrev(i, log_n);
        if (i < j) { fe t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    fe w;
    fr_root_of_unity(&w, log_n);
    if (inverse) f_inv(&FR, &w, &w);
    for (uint32_t s = 1; s <= log_n; s++) {
        size_t len = (size_t)1 << s;
        /* wlen = w^(n/len) */
        fe wlen = w;
        for (uint32_t k = s; k < log_n; k++) f_mul(&FR, &wlen, &wlen, &wlen);
        for (size_t i = 0; i < n; i += len) {
            fe wj = FR.one;
            for (size_t j = 0; j < len / 2; j++) {
                fe u = a[i + j], v;
                f_mul(&FR, &v, &a[i + j + len / 2], &wj);
                f_add(&FR, &a[i + j], &u, &v);
                f_sub(&FR, &a[i + j + len / 2], &u, &v);
                f_mul(&FR, &wj, &wj, &wlen);
            }
        }
    }
    if (inverse) {
        fe ninv;
        f_from_u64(&FR, &ninv, (uint64_t)n);
        f_inv(&FR, &ninv, &ninv);
        for (size_t i = 0; i < n; i++) f_mul(&FR, &a[i], &a[i], &ninv);
    }
}

/* ------------------------------------------------------------------------- */
/* Multi-scalar multiplication  sum_i k_i P_i.                                  */
/*   method 0: one double-and-add per term, summed (the definition).            */
/*   method 1: plain Pippenger with unsigned c-bit windows, Jacobian buckets.   */
/* ------------------------------------------------------------------------- */

static int msm_window_bits(size_t n) {
    int c = 1;
    while (c < 16 && ((size_t)1 << (c + 2)) < n) c++;
    return c < 2 ? 2 : c;
}

static uint32_t scalar_window(const uint64_t k[4], int w, int c) {
    uint32_t out = 0;
    for (int b = 0; b < c; b++) {
        int bit = w * c + b;
        if (bit < 256 && ((k[bit >> 6] >> (bit & 63)) & 1)) out |= 1u << b;
    }
    return out;
}

static void msm_g1(g1j* out, const g1a* pts, const uint64_t (*k)[4], size_t n, int method) {
    g1j acc;
    g1j_set_inf(&acc);
    if (method == 0) {
#pragma omp parallel
        {
            g1j local;
            g1j_set_inf(&local);
#pragma omp for schedule(dynamic, 16)
            for (long i = 0; i < (long)n; i++) {
                g1j p, t;
                g1j_from_affine(&p, &pts[i]);
                g1j_mul(&t, &p, k[i]);
                g1j_add(&local, &local, &t);
            }
#pragma omp critical
            g1j_add(&acc, &acc, &local);
        }
        *out = acc;
        return;
    }
    int c = msm_window_bits(n);
    int K = (256 + c - 1) / c;
    size_t nb = ((size_t)1 << c) - 1;
    g1j* wsum = (g1j*)malloc(sizeof(g1j) * K);
#pragma omp parallel for schedule(dynamic, 1)
    for (int w = 0; w < K; w++) {
        g1j* bucket = (g1j*)malloc(sizeof(g1j) * nb);
        for (size_t b = 0; b < nb; b++) g1j_set_inf(&bucket[b]);
        for (size_t i = 0; i < n; i++) {
            uint32_t d = scalar_window(k[i], w, c);
            if (d && !pts[i].inf) {
                g1j p;
                g1j_from_affine(&p, &pts[i]);
                g1j_add(&bucket[d - 1], &bucket[d - 1], &p);
            }
        }
        g1j run, tot;
        g1j_set_inf(&run);
        g1j_set_inf(&tot);
        for (size_t b = nb; b-- > 0;) {
            g1j_add(&run, &run, &bucket[b]);
            g1j_add(&tot, &tot, &run);
        }
        wsum[w] = tot;
        free(bucket);
    }
    for (int w = K - 1; w >= 0; w--) {
        for (int s = 0; s < c; s++) g1j_dbl(&acc, &acc);
        g1j_add(&acc, &acc, &wsum[w]);
    }
    free(wsum);
    *out = acc;
}

static void msm_g2(g2j* out, const g2a* pts, const uint64_t (*k)[4], size_t n, int method) {
    g2j acc;
    g2j_set_inf(&acc);
    if (method == 0) {
#pragma omp parallel
        {
            g2j local;
            g2j_set_inf(&local);
#pragma omp for schedule(dynamic, 16)
            for (long i = 0; i < (long)n; i++) {
                g2j p, t;
                g2j_from_affine(&p, &pts[i]);
                g2j_mul(&t, &p, k[i]);
                g2j_add(&local, &local, &t);
            }
#pragma omp critical
            g2j_add(&acc, &acc, &local);
        }
        *out = acc;
        return;
    }
    int c = msm_window_bits(n);
    int K = (256 + c - 1) / c;
    size_t nb = ((size_t)1 << c) - 1;
    g2j* wsum = (g2j*)malloc(sizeof(g2j) * K);
#pragma omp parallel for schedule(dynamic, 1)
    for (int w = 0; w < K; w++) {
        g2j* bucket = (g2j*)malloc(sizeof(g2j) * nb);
        for (size_t b = 0; b < nb; b++) g2j_set_inf(&bucket[b]);
        for (size_t i = 0; i < n; i++) {
            uint32_t d = scalar_window(k[i], w, c);
            if (d && !pts[i].inf) {
                g2j p;
                g2j_from_affine(&p, &pts[i]);
                g2j_add(&bucket[d - 1], &bucket[d - 1], &p);
            }
        }
        g2j run, tot;
        g2j_set_inf(&run);
        g2j_set_inf(&tot);
        for (size_t b = nb; b-- > 0;) {
            g2j_add(&run, &run, &bucket[b]);
            g2j_add(&tot, &tot, &run);
        }
        wsum[w] = tot;
        free(bucket);
    }
    for (int w = K - 1; w >= 0; w--) {
        for (int s = 0; s < c; s++) g2j_dbl(&acc, &acc);
        g2j_add(&acc, &acc, &wsum[w]);
    }
    free(wsum);
    *out = acc;
}

/* ------------------------------------------------------------------------- */
/* Synthetic circuit: Poseidon-style permutations (width 3, x^5 S-box,         */
/* 4 + 57 + 4 rounds, seeded round constants, seeded Cauchy MDS matrix),       */
/* bit-packing rows, a chain of squaring gates, and one input-consistency row */
/* per public variable.  Linear layers fold into linear combinations (LCs).   */
/* ------------------------------------------------------------------------- */

#define PSN_RF_HALF 4
#define PSN_RP 57
#define PSN_ROUNDS (2 * PSN_RF_HALF + PSN_RP)
#define ROWS_PER_PERM ((2 * PSN_RF_HALF * 3 + PSN_RP) * 3)

typedef struct { uint32_t var; fe c; } term;
typedef struct { term* t; uint32_t n, cap; } lc_t;

static void lc_free(lc_t* a) { free(a->t); a->t = NULL; a->n = a->cap = 0; }
static void lc_push(lc_t* a, uint32_t var, const fe* c) {
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 8;
        a->t = (term*)realloc(a->t, sizeof(term) * a->cap);
    }
    a->t[a->n].var = var;
    a->t[a->n].c = *c;
    a->n++;
}
static int term_cmp(const void* x, const void* y) {
    uint32_t a = ((const term*)x)->var, b = ((const term*)y)->var;
    return a < b ? -1 : a > b;
}
/* sort by variable, merge equal variables, drop zero coefficients */
static void lc_normalise(lc_t* a) {
    if (a->n == 0) return;
    qsort(a->t, a->n, sizeof(term), term_cmp);
    uint32_t w = 0;
    for (uint32_t i = 0; i < a->n; i++) {
        if (w > 0 && a->t[w - 1].var == a->t[i].var) {
            f_add(&FR, &a->t[w - 1].c, &a->t[w - 1].c, &a->t[i].c);
        } else {
            a->t[w++] = a->t[i];
        }
    }
    uint32_t k = 0;
    for (uint32_t i = 0; i < w; i++)
        if (!f_is_zero(&a->t[i].c)) a->t[k++] = a->t[i];
    a->n = k;
}
static lc_t lc_single(uint32_t var) {
    lc_t a = {0};
    lc_push(&a, var, &FR.one);
    return a;
}
/* out = sum_i k_i * in_i */
static lc_t lc_combine(const lc_t* in, const fe* k, int count) {
    lc_t out = {0};
    for (int i = 0; i < count; i++)
        for (uint32_t j = 0; j < in[i].n; j++) {
            fe c;
            f_mul(&FR, &c, &in[i].t[j].c, &k[i]);
            lc_push(&out, in[i].t[j].var, &c);
        }
    lc_normalise(&out);
    return out;
}

typedef struct {
    uint32_t log_n, n_rows, n_perm, n_pack, pack_bits;
    uint64_t seed;
    size_t N, m, n_chain;
    /* CSR of A, B, C: rp[k][N+1], col[k][nnz], val[k][nnz] (Montgomery Fr) */
    size_t* rp[3];
    uint32_t* col[3];
    fe* val[3];
    size_t nnz[3], cap[3];
    size_t rows;
    fe rc[PSN_ROUNDS][3];
    fe mds[3][3];
    fe* chain_k;
    fe* z;           /* witness values (Montgomery), m entries */
    size_t next_var;
    int have_witness;
} circuit;

static void cs_push_row(circuit* cs, const lc_t* A, const lc_t* B, const lc_t* C) {
    const lc_t* M[3] = {A, B, C};
    for (int k = 0; k < 3; k++) {
        const lc_t* L = M[k];
        if (cs->nnz[k] + (L ? L->n : 0) > cs->cap[k]) {
            size_t nc = cs->cap[k] ? cs->cap[k] : 1024;
            while (nc < cs->nnz[k] + (L ? L->n : 0)) nc *= 2;
            cs->col[k] = (uint32_t*)realloc(cs->col[k], nc * sizeof(uint32_t));
            cs->val[k] = (fe*)realloc(cs->val[k], nc * sizeof(fe));
            cs->cap[k] = nc;
        }
        if (L)
            for (uint32_t i = 0; i < L->n; i++) {
                cs->col[k][cs->nnz[k]] = L->t[i].var;
                cs->val[k][cs->nnz[k]] = L->t[i].c;
                cs->nnz[k]++;
            }
        cs->rp[k][cs->rows + 1] = cs->nnz[k];
    }
    cs->rows++;
}

static fe lc_value(const circuit* cs, const lc_t* a) {
    fe acc = {{0, 0, 0, 0}};
    for (uint32_t i = 0; i < a->n; i++) {
        fe t;
        f_mul(&FR, &t, &a->t[i].c, &cs->z[a->t[i].var]);
        f_add(&FR, &acc, &acc, &t);
    }
    return acc;
}

static uint32_t cs_alloc(circuit* cs, const fe* value) {
    uint32_t v = (uint32_t)cs->next_var++;
    if (cs->have_witness) cs->z[v] = *value;
    return v;
}

/* S-box s^5 as three rows: s*s = x2, x2*x2 = x4, x4*s = x5.  Returns x5. */
static uint32_t cs_sbox(circuit* cs, const lc_t* s) {
    fe sv = {{0}}, x2v = {{0}}, x4v = {{0}}, x5v = {{0}};
    if (cs->have_witness) {
        sv = lc_value(cs, s);
        f_mul(&FR, &x2v, &sv, &sv);
        f_mul(&FR, &x4v, &x2v, &x2v);
        f_mul(&FR, &x5v, &x4v, &sv);
    }
    uint32_t x2 = cs_alloc(cs, &x2v);
    lc_t L2 = lc_single(x2);
    cs_push_row(cs, s, s, &L2);
    uint32_t x4 = cs_alloc(cs, &x4v);
    lc_t L4 = lc_single(x4);
    cs_push_row(cs, &L2, &L2, &L4);
    uint32_t x5 = cs_alloc(cs, &x5v);
    lc_t L5 = lc_single(x5);
    cs_push_row(cs, &L4, s, &L5);
    lc_free(&L2);
    lc_free(&L4);
    lc_free(&L5);
    return x5;
}

/* One permutation over three fresh private inputs; returns lane 0 of the
 * output as an LC. */
static lc_t cs_permutation(circuit* cs, smx* rin) {
    lc_t lane[3];
    for (int l = 0; l < 3; l++) {
        fe v = {{0}};
        if (cs->have_witness) smx_fr(rin, &v);
        lane[l] = lc_single(cs_alloc(cs, &v));
    }
    for (int r = 0; r < PSN_ROUNDS; r++) {
        int full = (r < PSN_RF_HALF) || (r >= PSN_RF_HALF + PSN_RP);
        for (int l = 0; l < 3; l++) {
            lc_push(&lane[l], 0, &cs->rc[r][l]);
            lc_normalise(&lane[l]);
        }
        for (int l = 0; l < (full ? 3 : 1); l++) {
            uint32_t x5 = cs_sbox(cs, &lane[l]);
            lc_free(&lane[l]);
            lane[l] = lc_single(x5);
        }
        lc_t nl[3];
        for (int i = 0; i < 3; i++) nl[i] = lc_combine(lane, cs->mds[i], 3);
        for (int i = 0; i < 3; i++) { lc_free(&lane[i]); lane[i] = nl[i]; }
    }
    lc_free(&lane[1]);
    lc_free(&lane[2]);
    return lane[0];
}

static void circuit_free(circuit* cs) {
    if (!cs) return;
    for (int k = 0; k < 3; k++) { free(cs->rp[k]); free(cs->col[k]); free(cs->val[k]); }
    free(cs->chain_k);
    free(cs->z);
    free(cs);
}

static circuit* circuit_build(uint32_t log_n, uint32_t n_rows, uint32_t n_perm, uint32_t n_pack,
                              uint32_t pack_bits, uint64_t seed, int with_witness, uint64_t input_seed) {
    oracle_init();
    size_t N = (size_t)1 << log_n;
    if (log_n < 2 || log_n > 28 || n_rows > N || pack_bits > 253) return NULL;
    size_t fixed = 2 + (size_t)ROWS_PER_PERM * n_perm + n_pack;
    if (n_rows < fixed + 1) return NULL;
    circuit* cs = (circuit*)calloc(1, sizeof(circuit));
    cs->log_n = log_n; cs->n_rows = n_rows; cs->n_perm = n_perm; cs->n_pack = n_pack;
    cs->pack_bits = pack_bits; cs->seed = seed; cs->N = N;
    cs->n_chain = n_rows - fixed;
    cs->m = 2 + (size_t)n_perm * (3 + ROWS_PER_PERM) + (size_t)n_pack * (pack_bits + 1) +
            (n_perm == 0 ? 1 : 0) + (cs->n_chain - 1);
    for (int k = 0; k < 3; k++) cs->rp[k] = (size_t*)calloc(N + 1, sizeof(size_t));
    cs->have_witness = with_witness;
    if (with_witness) cs->z = (fe*)calloc(cs->m, sizeof(fe));

    smx g;
    smx_init(&g, seed, PURPOSE_ROUND_CONST);
    for (int r = 0; r < PSN_ROUNDS; r++)
        for (int l = 0; l < 3; l++) smx_fr(&g, &cs->rc[r][l]);
    smx_init(&g, seed, PURPOSE_MDS);
    for (;;) {
        fe x[3], y[3];
        for (int i = 0; i < 3; i++) smx_fr(&g, &x[i]);
        for (int i = 0; i < 3; i++) smx_fr(&g, &y[i]);
        int ok = !f_eq(&x[0], &x[1]) && !f_eq(&x[0], &x[2]) && !f_eq(&x[1], &x[2]) &&
                 !f_eq(&y[0], &y[1]) && !f_eq(&y[0], &y[2]) && !f_eq(&y[1], &y[2]);
        for (int i = 0; i < 3 && ok; i++)
            for (int j = 0; j < 3 && ok; j++) {
                fe s;
                f_add(&FR, &s, &x[i], &y[j]);
                if (f_is_zero(&s)) ok = 0;
            }
        if (!ok) continue;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                fe s;
                f_add(&FR, &s, &x[i], &y[j]);
                f_inv(&FR, &cs->mds[i][j], &s);
            }
        break;
    }
    cs->chain_k = (fe*)malloc(sizeof(fe) * cs->n_chain);
    smx_init(&g, seed, PURPOSE_CHAIN);
    for (size_t i = 0; i < cs->n_chain; i++) smx_fr(&g, &cs->chain_k[i]);

    smx rin;
    smx_init(&rin, input_seed, PURPOSE_INPUTS);
    fe onev = FR.one, zero = {{0}};
    cs->next_var = 0;
    cs_alloc(cs, &onev);   /* z_0 = 1 */
    cs_alloc(cs, &zero);   /* z_1 = public output, set at the end of the chain */

    lc_t chain_start = {0};
    for (uint32_t p = 0; p < n_perm; p++) {
        lc_t out = cs_permutation(cs, &rin);
        if (p + 1 == n_perm) chain_start = out;
        else lc_free(&out);
    }
    /* bit-packing rows: (sum_k 2^k b_k) * 1 = y */
    for (uint32_t q = 0; q < n_pack; q++) {
        lc_t A = {0};
        fe yv = {{0}}, pw = FR.one;
        for (uint32_t k = 0; k < pack_bits; k++) {
            fe bv = {{0}};
            if (with_witness) {
                uint64_t bit = smx_next(&rin) & 1;
                bv = bit ? FR.one : zero;
                fe t;
                f_mul(&FR, &t, &bv, &pw);
                f_add(&FR, &yv, &yv, &t);
            }
            uint32_t b = cs_alloc(cs, &bv);
            lc_push(&A, b, &pw);
            f_add(&FR, &pw, &pw, &pw);
        }
        uint32_t y = cs_alloc(cs, &yv);
        lc_t B = lc_single(0), C = lc_single(y);
        cs_push_row(cs, &A, &B, &C);
        lc_free(&A); lc_free(&B); lc_free(&C);
    }
    if (n_perm == 0) {
        fe v = {{0}};
        if (with_witness) smx_fr(&rin, &v);
        chain_start = lc_single(cs_alloc(cs, &v));
    }
    /* chain: x_{i+1} = x_i^2 + k_i, as the row x_i * x_i = x_{i+1} - k_i */
    lc_t x = chain_start;
    for (size_t i = 0; i < cs->n_chain; i++) {
        fe nv = {{0}};
        if (with_witness) {
            fe xv = lc_value(cs, &x);
            f_mul(&FR, &nv, &xv, &xv);
            f_add(&FR, &nv, &nv, &cs->chain_k[i]);
        }
        uint32_t tgt;
        if (i + 1 == cs->n_chain) {
            tgt = 1;
            if (with_witness) cs->z[1] = nv;
        } else {
            tgt = cs_alloc(cs, &nv);
        }
        lc_t C = lc_single(tgt);
        fe negk;
        f_neg(&FR, &negk, &cs->chain_k[i]);
        lc_push(&C, 0, &negk);
        lc_normalise(&C);
        cs_push_row(cs, &x, &x, &C);
        lc_free(&C);
        lc_free(&x);
        x = lc_single(tgt);
    }
    lc_free(&x);
    /* input-consistency rows A = z_j, B = C = 0 for the public variables */
    for (uint32_t j = 0; j < 2; j++) {
        lc_t A = lc_single(j);
        cs_push_row(cs, &A, NULL, NULL);
        lc_free(&A);
    }
    while (cs->rows < N) cs_push_row(cs, NULL, NULL, NULL);
    if (cs->next_var != cs->m) {
        fprintf(stderr, "oracle: variable count mismatch %zu vs %zu\n", cs->next_var, cs->m);
        abort();
    }
    return cs;
}

static void spmv(const circuit* cs, int k, const fe* z, fe* out) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)cs->N; i++) {
        fe acc = {{0}};
        for (size_t e = cs->rp[k][i]; e < cs->rp[k][i + 1]; e++) {
            fe t;
            f_mul(&FR, &t, &cs->val[k][e], &z[cs->col[k][e]]);
            f_add(&FR, &acc, &acc, &t);
        }
        out[i] = acc;
    }
}

static int r1cs_check(const circuit* cs, const fe* z) {
    size_t N = cs->N;
    fe* a = (fe*)malloc(sizeof(fe) * N);
    fe* b = (fe*)malloc(sizeof(fe) * N);
    fe* c = (fe*)malloc(sizeof(fe) * N);
    spmv(cs, 0, z, a);
    spmv(cs, 1, z, b);
    spmv(cs, 2, z, c);
    int ok = 1;
    for (size_t i = 0; i < N && ok; i++) {
        fe t;
        f_mul(&FR, &t, &a[i], &b[i]);
        if (!f_eq(&t, &c[i])) ok = 0;
    }
    free(a); free(b); free(c);
    return ok;
}

/* h = (A(X) B(X) - C(X)) / (X^N - 1), where A, B, C interpolate Az, Bz, Cz on
 * H = {omega^i}.  The product is formed by a 2N-point convolution and the
 * division by X^N - 1 is long division: X^{N+i} = X^i (X^N - 1) + X^i.
 * Returns 1 if the remainder is zero (witness satisfies the R1CS). */
static int qap_h(const circuit* cs, const fe* z, fe* h) {
    size_t N = cs->N;
    uint32_t k = cs->log_n;
    fe* A = (fe*)calloc(2 * N, sizeof(fe));
    fe* B = (fe*)calloc(2 * N, sizeof(fe));
    fe* C = (fe*)calloc(N, sizeof(fe));
    spmv(cs, 0, z, A);
    spmv(cs, 1, z, B);
    spmv(cs, 2, z, C);
    ntt_inplace(A, k, 1);
    ntt_inplace(B, k, 1);
    ntt_inplace(C, k, 1);
    ntt_inplace(A, k + 1, 0);
    ntt_inplace(B, k + 1, 0);
    for (size_t i = 0; i < 2 * N; i++) f_mul(&FR, &A[i], &A[i], &B[i]);
    ntt_inplace(A, k + 1, 1);   /* A = coefficients of A(X) B(X), degree <= 2N-2 */
    for (size_t i = 0; i < N; i++) f_sub(&FR, &A[i], &A[i], &C[i]);
    int ok = f_is_zero(&A[2 * N - 1]);
    for (size_t i = 0; i < N; i++) {
        fe rem;
        f_add(&FR, &rem, &A[i], &A[N + i]);
        if (!f_is_zero(&rem)) ok = 0;
        h[i] = A[N + i];
    }
    free(A); free(B); free(C);
    return ok;
}

/* ------------------------------------------------------------------------- */
/* Groth16 setup (toy, seeded toxic waste), prover, in-the-exponent proof and  */
/* verifier.  pk = {[a]1, [b]1, [b]2, [d]1, [d]2, [u_j]1, [v_j]1, [v_j]2,      */
/* [(b u_j + a v_j + w_j)/d]1 (j > l), [tau^i Z(tau)/d]1 (i <= N-2)};          */
/* vk = {[a]1, [b]2, [g]2, [d]2, [(b u_j + a v_j + w_j)/g]1 (j <= l)}, l = 1.  */
/* ------------------------------------------------------------------------- */

#define N_PUBLIC 1

typedef struct {
    const circuit* cs;
    size_t N, m;
    fe tau, alpha, beta, gamma, delta;
    fe *u, *v, *w;   /* u_j(tau), v_j(tau), w_j(tau) */
    fe* lq;          /* j <= l: (b u + a v + w)/g ; j > l: (b u + a v + w)/d */
    fe* hq;          /* tau^i Z(tau)/d, i = 0..N-2 */
    int with_points;
    g1a alpha1, beta1, delta1;
    g2a beta2, gamma2, delta2;
    g1a *A, *B1, *L, *H, IC[N_PUBLIC + 1];
    g2a* B2;
} pk_t;

static g1a g1_mul_gen_fe(const fe* k_mont) {
    uint64_t k[4];
    fe_canon(&FR, k, k_mont);
    g1j g, r;
    g1j_from_affine(&g, &G1_GEN);
    g1j_mul(&r, &g, k);
    g1a out;
    g1j_to_affine(&out, &r);
    return out;
}
static g2a g2_mul_gen_fe(const fe* k_mont) {
    uint64_t k[4];
    fe_canon(&FR, k, k_mont);
    g2j g, r;
    g2j_from_affine(&g, &G2_GEN);
    g2j_mul(&r, &g, k);
    g2a out;
    g2j_to_affine(&out, &r);
    return out;
}

/* Fixed-base windowing for the many generator multiples of a key's query
 * points (Hankerson, Menezes and Vanstone, Guide to Elliptic Curve
 * Cryptography, fixed-base windowing): with the table T[w][d] = d 2^(8w) G,
 * k G = sum over the 32 byte-windows w of k of T[w][byte_w(k)].  The same
 * points as g1_mul_gen_fe / g2_mul_gen_fe (double-and-add), about eight times
 * fewer group operations; setup only (the in-the-exponent proof and the
 * exported generator multiples keep double-and-add). */
static g1j G1_TAB[32][256];
static g2j G2_TAB[32][256];
static int g_tab_ready = 0;

static void gen_tables_init(void) {
    if (g_tab_ready) return;
    g1j b1;
    g2j b2;
    g1j_from_affine(&b1, &G1_GEN);
    g2j_from_affine(&b2, &G2_GEN);
    for (int w = 0; w < 32; w++) {
        g1j_set_inf(&G1_TAB[w][0]);
        g2j_set_inf(&G2_TAB[w][0]);
        for (int d = 1; d < 256; d++) {
            g1j_add(&G1_TAB[w][d], &G1_TAB[w][d - 1], &b1);
            g2j_add(&G2_TAB[w][d], &G2_TAB[w][d - 1], &b2);
        }
        for (int s = 0; s < 8; s++) {
            g1j_dbl(&b1, &b1);
            g2j_dbl(&b2, &b2);
        }
    }
    g_tab_ready = 1;
}

static g1a g1_mul_gen_tab(const fe* k_mont) {
    uint64_t k[4];
    fe_canon(&FR, k, k_mont);
    g1j r;
    g1j_set_inf(&r);
    for (int w = 0; w < 32; w++) {
        unsigned d = (unsigned)((k[w >> 3] >> (8 * (w & 7))) & 0xff);
        if (d) g1j_add(&r, &r, &G1_TAB[w][d]);
    }
    g1a out;
    g1j_to_affine(&out, &r);
    return out;
}
static g2a g2_mul_gen_tab(const fe* k_mont) {
    uint64_t k[4];
    fe_canon(&FR, k, k_mont);
    g2j r;
    g2j_set_inf(&r);
    for (int w = 0; w < 32; w++) {
        unsigned d = (unsigned)((k[w >> 3] >> (8 * (w & 7))) & 0xff);
        if (d) g2j_add(&r, &r, &G2_TAB[w][d]);
    }
    g2a out;
    g2j_to_affine(&out, &r);
    return out;
}

static void sample_nonzero(smx* g, fe* out) {
    do { smx_fr(g, out); } while (f_is_zero(out));
}

static void pk_free(pk_t* pk) {
    if (!pk) return;
    free(pk->u); free(pk->v); free(pk->w); free(pk->lq); free(pk->hq);
    free(pk->A); free(pk->B1); free(pk->L); free(pk->H); free(pk->B2);
    free(pk);
}

static pk_t* setup(const circuit* cs, uint64_t toxic_seed, int with_points) {
    size_t N = cs->N, m = cs->m;
    pk_t* pk = (pk_t*)calloc(1, sizeof(pk_t));
    pk->cs = cs; pk->N = N; pk->m = m; pk->with_points = with_points;
    smx g;
    smx_init(&g, toxic_seed, PURPOSE_TOXIC);
    uint64_t nexp[4] = {(uint64_t)N, 0, 0, 0};
    for (;;) {
        sample_nonzero(&g, &pk->tau);
        fe tn;
        f_pow(&FR, &tn, &pk->tau, nexp);
        if (!f_eq(&tn, &FR.one)) break;
    }
    sample_nonzero(&g, &pk->alpha);
    sample_nonzero(&g, &pk->beta);
    sample_nonzero(&g, &pk->gamma);
    sample_nonzero(&g, &pk->delta);

    /* Lagrange basis on H at tau: L_i(tau) = (tau^N - 1) omega^i / (N (tau - omega^i)) */
    fe omega, zt, ninv;
    fr_root_of_unity(&omega, cs->log_n);
    f_pow(&FR, &zt, &pk->tau, nexp);
    f_sub(&FR, &zt, &zt, &FR.one);
    f_from_u64(&FR, &ninv, (uint64_t)N);
    f_inv(&FR, &ninv, &ninv);
    fe* Lt = (fe*)malloc(sizeof(fe) * N);
    fe* den = (fe*)malloc(sizeof(fe) * N);
    fe* pw = (fe*)malloc(sizeof(fe) * N);
    fe wi = FR.one;
    for (size_t i = 0; i < N; i++) {
        pw[i] = wi;
        f_sub(&FR, &den[i], &pk->tau, &wi);
        f_mul(&FR, &wi, &wi, &omega);
    }
    /* batch inversion (Montgomery's trick) of den[] */
    fe acc = FR.one;
    for (size_t i = 0; i < N; i++) { Lt[i] = acc; f_mul(&FR, &acc, &acc, &den[i]); }
    f_inv(&FR, &acc, &acc);
    for (size_t i = N; i-- > 0;) {
        fe inv_i;
        f_mul(&FR, &inv_i, &acc, &Lt[i]);
        f_mul(&FR, &acc, &acc, &den[i]);
        den[i] = inv_i;
    }
    fe zn;
    f_mul(&FR, &zn, &zt, &ninv);
    for (size_t i = 0; i < N; i++) {
        f_mul(&FR, &Lt[i], &zn, &pw[i]);
        f_mul(&FR, &Lt[i], &Lt[i], &den[i]);
    }
    free(den);
    free(pw);

    fe* q[3];
    for (int k = 0; k < 3; k++) {
        q[k] = (fe*)calloc(m, sizeof(fe));
        for (size_t i = 0; i < N; i++)
            for (size_t e = cs->rp[k][i]; e < cs->rp[k][i + 1]; e++) {
                fe t;
                f_mul(&FR, &t, &cs->val[k][e], &Lt[i]);
                f_add(&FR, &q[k][cs->col[k][e]], &q[k][cs->col[k][e]], &t);
            }
    }
    free(Lt);
    pk->u = q[0]; pk->v = q[1]; pk->w = q[2];
    fe dinv, ginv;
    f_inv(&FR, &dinv, &pk->delta);
    f_inv(&FR, &ginv, &pk->gamma);
    pk->lq = (fe*)malloc(sizeof(fe) * m);
    for (size_t j = 0; j < m; j++) {
        fe t, s;
        f_mul(&FR, &t, &pk->beta, &pk->u[j]);
        f_mul(&FR, &s, &pk->alpha, &pk->v[j]);
        f_add(&FR, &t, &t, &s);
        f_add(&FR, &t, &t, &pk->w[j]);
        f_mul(&FR, &pk->lq[j], &t, j <= N_PUBLIC ? &ginv : &dinv);
    }
    pk->hq = (fe*)malloc(sizeof(fe) * (N - 1));
    fe ti = FR.one, zd;
    f_mul(&FR, &zd, &zt, &dinv);
    for (size_t i = 0; i + 1 < N; i++) {
        f_mul(&FR, &pk->hq[i], &ti, &zd);
        f_mul(&FR, &ti, &ti, &pk->tau);
    }
    pk->alpha1 = g1_mul_gen_fe(&pk->alpha);
    pk->beta1 = g1_mul_gen_fe(&pk->beta);
    pk->delta1 = g1_mul_gen_fe(&pk->delta);
    pk->beta2 = g2_mul_gen_fe(&pk->beta);
    pk->gamma2 = g2_mul_gen_fe(&pk->gamma);
    pk->delta2 = g2_mul_gen_fe(&pk->delta);
    for (int j = 0; j <= N_PUBLIC; j++) pk->IC[j] = g1_mul_gen_fe(&pk->lq[j]);
    if (with_points) {
        pk->A = (g1a*)malloc(sizeof(g1a) * m);
        pk->B1 = (g1a*)malloc(sizeof(g1a) * m);
        pk->B2 = (g2a*)malloc(sizeof(g2a) * m);
        pk->L = (g1a*)malloc(sizeof(g1a) * m);
        pk->H = (g1a*)malloc(sizeof(g1a) * (N - 1));
        gen_tables_init();
#pragma omp parallel for schedule(dynamic, 8)
        for (long j = 0; j < (long)m; j++) {
            pk->A[j] = g1_mul_gen_tab(&pk->u[j]);
            pk->B1[j] = g1_mul_gen_tab(&pk->v[j]);
            pk->B2[j] = g2_mul_gen_tab(&pk->v[j]);
            if (j > N_PUBLIC) pk->L[j] = g1_mul_gen_tab(&pk->lq[j]);
            else { memset(&pk->L[j], 0, sizeof(g1a)); pk->L[j].inf = 1; }
        }
#pragma omp parallel for schedule(dynamic, 8)
        for (long i = 0; i < (long)(N - 1); i++) pk->H[i] = g1_mul_gen_tab(&pk->hq[i]);
    }
    return pk;
}

static void rs_from_seed(uint64_t seed, fe* r, fe* s) {
    smx g;
    smx_init(&g, seed, PURPOSE_RS);
    sample_nonzero(&g, r);
    sample_nonzero(&g, s);
}

static void proof_to_bytes(uint8_t out[256], const g1a* A, const g2a* B, const g1a* C) {
    g1a_to_bytes(out, A);
    g2a_to_bytes(out + 64, B);
    g1a_to_bytes(out + 192, C);
}

static void fe_array_canon(uint64_t (*out)[4], const fe* in, size_t n) {
    for (size_t i = 0; i < n; i++) fe_canon(&FR, out[i], &in[i]);
}

/* The Groth16 prover, step by step:  a = alpha + sum z_j u_j + r delta,
 * b = beta + sum z_j v_j + s delta, c = sum_{j>l} z_j L_j + sum h_i H_i + s A
 * + r B1 - r s delta, all in the exponent via MSMs over the pk points. */
static int prove(const pk_t* pk, const fe* z, const fe* r, const fe* s, int method, uint8_t out[256]) {
    const circuit* cs = pk->cs;
    size_t N = pk->N, m = pk->m;
    if (!pk->with_points) return -1;
    fe* h = (fe*)malloc(sizeof(fe) * N);
    if (!qap_h(cs, z, h)) { free(h); return 0; }
    uint64_t (*zk)[4] = malloc(sizeof(uint64_t[4]) * m);
    uint64_t (*hk)[4] = malloc(sizeof(uint64_t[4]) * N);
    fe_array_canon(zk, z, m);
    fe_array_canon(hk, h, N);
    free(h);
    uint64_t rk[4], sk[4], rsk[4];
    fe rs;
    f_mul(&FR, &rs, r, s);
    fe_canon(&FR, rk, r);
    fe_canon(&FR, sk, s);
    fe_canon(&FR, rsk, &rs);

    g1j Aj, B1j, Lj, Hj, t, d1;
    g2j B2j, t2, d2;
    msm_g1(&Aj, pk->A, (const uint64_t (*)[4])zk, m, method);
    msm_g1(&B1j, pk->B1, (const uint64_t (*)[4])zk, m, method);
    msm_g2(&B2j, pk->B2, (const uint64_t (*)[4])zk, m, method);
    msm_g1(&Lj, pk->L + (N_PUBLIC + 1), (const uint64_t (*)[4])(zk + (N_PUBLIC + 1)), m - (N_PUBLIC + 1), method);
    msm_g1(&Hj, pk->H, (const uint64_t (*)[4])hk, N - 1, method);
    free(zk);
    free(hk);

    g1j_from_affine(&d1, &pk->delta1);
    g2j_from_affine(&d2, &pk->delta2);
    /* A = alpha + S_A + r delta */
    g1j_from_affine(&t, &pk->alpha1);
    g1j_add(&Aj, &Aj, &t);
    g1j_mul(&t, &d1, rk);
    g1j_add(&Aj, &Aj, &t);
    /* B (G2) = beta + S_B + s delta */
    g2j_from_affine(&t2, &pk->beta2);
    g2j_add(&B2j, &B2j, &t2);
    g2j_mul(&t2, &d2, sk);
    g2j_add(&B2j, &B2j, &t2);
    /* B1 (G1) = beta + S_B1 + s delta */
    g1j_from_affine(&t, &pk->beta1);
    g1j_add(&B1j, &B1j, &t);
    g1j_mul(&t, &d1, sk);
    g1j_add(&B1j, &B1j, &t);
    /* C = S_L + S_H + s A + r B1 - r s delta */
    g1j C = Lj;
    g1j_add(&C, &C, &Hj);
    g1j_mul(&t, &Aj, sk);
    g1j_add(&C, &C, &t);
    g1j_mul(&t, &B1j, rk);
    g1j_add(&C, &C, &t);
    g1j_mul(&t, &d1, rsk);
    g1j_neg(&t, &t);
    g1j_add(&C, &C, &t);

    g1a Aa, Ca;
    g2a Ba;
    g1j_to_affine(&Aa, &Aj);
    g2j_to_affine(&Ba, &B2j);
    g1j_to_affine(&Ca, &C);
    proof_to_bytes(out, &Aa, &Ba, &Ca);
    return 1;
}

/* The proof computed "in the exponent": with the toxic waste known, the three
 * proof elements are [a]1, [b]2, [c]1 for Fr scalars a, b, c obtained by
 * O(nnz) field work, with no NTT and no MSM:
 *   a = alpha + A(tau) + r delta,  b = beta + B(tau) + s delta,
 *   c = (sum_{j>l} z_j (beta u_j + alpha v_j + w_j) + A(tau)B(tau) - C(tau))/delta
 *       + s a + r b - r s delta,
 * where A(tau) = sum_j z_j u_j(tau), and likewise B, C. */
static void expected_proof(const pk_t* pk, const fe* z, const fe* r, const fe* s, uint8_t out[256]) {
    size_t m = pk->m;
    fe At = {{0}}, Bt = {{0}}, Ct = {{0}}, Lsum = {{0}}, t;
    for (size_t j = 0; j < m; j++) {
        f_mul(&FR, &t, &z[j], &pk->u[j]); f_add(&FR, &At, &At, &t);
        f_mul(&FR, &t, &z[j], &pk->v[j]); f_add(&FR, &Bt, &Bt, &t);
        f_mul(&FR, &t, &z[j], &pk->w[j]); f_add(&FR, &Ct, &Ct, &t);
        if (j > N_PUBLIC) {
            fe x, y;
            f_mul(&FR, &x, &pk->beta, &pk->u[j]);
            f_mul(&FR, &y, &pk->alpha, &pk->v[j]);
            f_add(&FR, &x, &x, &y);
            f_add(&FR, &x, &x, &pk->w[j]);
            f_mul(&FR, &x, &x, &z[j]);
            f_add(&FR, &Lsum, &Lsum, &x);
        }
    }
    fe a, b, c, dinv;
    f_mul(&FR, &t, r, &pk->delta);
    f_add(&FR, &a, &pk->alpha, &At);
    f_add(&FR, &a, &a, &t);
    f_mul(&FR, &t, s, &pk->delta);
    f_add(&FR, &b, &pk->beta, &Bt);
    f_add(&FR, &b, &b, &t);
    f_mul(&FR, &t, &At, &Bt);
    f_sub(&FR, &t, &t, &Ct);
    f_add(&FR, &c, &Lsum, &t);
    f_inv(&FR, &dinv, &pk->delta);
    f_mul(&FR, &c, &c, &dinv);
    f_mul(&FR, &t, s, &a); f_add(&FR, &c, &c, &t);
    f_mul(&FR, &t, r, &b); f_add(&FR, &c, &c, &t);
    f_mul(&FR, &t, r, s);
    f_mul(&FR, &t, &t, &pk->delta);
    f_sub(&FR, &c, &c, &t);
    g1a Aa = g1_mul_gen_fe(&a);
    g2a Ba = g2_mul_gen_fe(&b);
    g1a Ca = g1_mul_gen_fe(&c);
    proof_to_bytes(out, &Aa, &Ba, &Ca);
}

/* e(A, B) == e(alpha, beta) e(IC_0 + x_1 IC_1, gamma) e(C, delta) */
static int verify(const pk_t* pk, const fe* pub, const uint8_t proof[256]) {
    g1a A, C;
    g2a B;
    if (!g1a_from_bytes(&A, proof) || !g2a_from_bytes(&B, proof + 64) || !g1a_from_bytes(&C, proof + 192))
        return -1;
    if (!g1a_on_curve(&A) || !g2a_on_curve(&B) || !g1a_on_curve(&C)) return -1;
    g1j acc, t;
    g1j_from_affine(&acc, &pk->IC[0]);
    uint64_t k[4];
    fe_canon(&FR, k, pub);
    g1j_from_affine(&t, &pk->IC[1]);
    g1j_mul(&t, &t, k);
    g1j_add(&acc, &acc, &t);
    g1a ICs;
    g1j_to_affine(&ICs, &acc);
    fe12 lhs, e1, e2, e3, rhs;
    tate_pairing(&lhs, &A, &B);
    tate_pairing(&e1, &pk->alpha1, &pk->beta2);
    tate_pairing(&e2, &ICs, &pk->gamma2);
    tate_pairing(&e3, &C, &pk->delta2);
    f12_mul(&rhs, &e1, &e2);
    f12_mul(&rhs, &rhs, &e3);
    return f12_eq(&lhs, &rhs) ? 1 : 0;
}

/* ========================================================================= */
/* Exported C interface (canonical little-endian bytes everywhere).            */
/* ========================================================================= */

#define EXPORT __attribute__((visibility("default")))

EXPORT int orc_init(void) { oracle_init(); return 0; }
EXPORT int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static const field* pick(int which) { return which ? &FR : &FP; }

/* which: 0 = Fp, 1 = Fr.  op: 0 add, 1 sub, 2 mul, 3 inv (b unused), 4 neg, 5 pow (b = exponent) */
EXPORT int orc_field_op(int which, int op, uint8_t* out, const uint8_t* a, const uint8_t* b) {
    oracle_init();
    const field* F = pick(which);
    fe x, y, r;
    if (!fe_from_bytes(F, &x, a)) return -1;
    switch (op) {
    case 0: if (!fe_from_bytes(F, &y, b)) return -1; f_add(F, &r, &x, &y); break;
    case 1: if (!fe_from_bytes(F, &y, b)) return -1; f_sub(F, &r, &x, &y); break;
    case 2: if (!fe_from_bytes(F, &y, b)) return -1; f_mul(F, &r, &x, &y); break;
    case 3: f_inv(F, &r, &x); break;
    case 4: f_neg(F, &r, &x); break;
    case 5: {
        uint64_t e[4];
        for (int i = 0; i < 4; i++) {
            uint64_t w = 0;
            for (int k = 7; k >= 0; k--) w = (w << 8) | b[8 * i + k];
            e[i] = w;
        }
        f_pow(F, &r, &x, e);
        break;
    }
    default: return -1;
    }
    fe_to_bytes(F, out, &r);
    return 0;
}

static void bytes_to_u256(uint64_t k[4], const uint8_t* b) {
    for (int i = 0; i < 4; i++) {
        uint64_t w = 0;
        for (int j = 7; j >= 0; j--) w = (w << 8) | b[8 * i + j];
        k[i] = w;
    }
}

EXPORT void orc_g1_generator(uint8_t* out) { oracle_init(); g1a_to_bytes(out, &G1_GEN); }
EXPORT void orc_g2_generator(uint8_t* out) { oracle_init(); g2a_to_bytes(out, &G2_GEN); }

EXPORT int orc_g1_on_curve(const uint8_t* a) {
    oracle_init();
    g1a p;
    if (!g1a_from_bytes(&p, a)) return -1;
    return g1a_on_curve(&p);
}
EXPORT int orc_g2_on_curve(const uint8_t* a) {
    oracle_init();
    g2a p;
    if (!g2a_from_bytes(&p, a)) return -1;
    return g2a_on_curve(&p);
}
/* out = a + b */
EXPORT int orc_g1_add(uint8_t* out, const uint8_t* a, const uint8_t* b) {
    oracle_init();
    g1a x, y, z;
    if (!g1a_from_bytes(&x, a) || !g1a_from_bytes(&y, b)) return -1;
    g1j X, Y;
    g1j_from_affine(&X, &x);
    g1j_from_affine(&Y, &y);
    g1j_add(&X, &X, &Y);
    g1j_to_affine(&z, &X);
    g1a_to_bytes(out, &z);
    return 0;
}
EXPORT int orc_g2_add(uint8_t* out, const uint8_t* a, const uint8_t* b) {
    oracle_init();
    g2a x, y, z;
    if (!g2a_from_bytes(&x, a) || !g2a_from_bytes(&y, b)) return -1;
    g2j X, Y;
    g2j_from_affine(&X, &x);
    g2j_from_affine(&Y, &y);
    g2j_add(&X, &X, &Y);
    g2j_to_affine(&z, &X);
    g2a_to_bytes(out, &z);
    return 0;
}
/* out = k a, k a 256-bit little-endian integer (not reduced) */
EXPORT int orc_g1_mul(uint8_t* out, const uint8_t* a, const uint8_t* k) {
    oracle_init();
    g1a x, z;
    if (!g1a_from_bytes(&x, a)) return -1;
    uint64_t kk[4];
    bytes_to_u256(kk, k);
    g1j X;
    g1j_from_affine(&X, &x);
    g1j_mul(&X, &X, kk);
    g1j_to_affine(&z, &X);
    g1a_to_bytes(out, &z);
    return 0;
}
EXPORT int orc_g2_mul(uint8_t* out, const uint8_t* a, const uint8_t* k) {
    oracle_init();
    g2a x, z;
    if (!g2a_from_bytes(&x, a)) return -1;
    uint64_t kk[4];
    bytes_to_u256(kk, k);
    g2j X;
    g2j_from_affine(&X, &x);
    g2j_mul(&X, &X, kk);
    g2j_to_affine(&z, &X);
    g2a_to_bytes(out, &z);
    return 0;
}

/* Batch k_i * G1 for canonical Fr scalars (used to build MSM inputs on the
 * oracle side from the shared seeded scalars). */
EXPORT int orc_g1_mul_gen_batch(uint8_t* out, const uint8_t* k, size_t n) {
    oracle_init();
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < (long)n; i++) {
        fe x;
        if (!fe_from_bytes(&FR, &x, k + 32 * i)) { bad = 1; continue; }
        g1a p = g1_mul_gen_fe(&x);
        g1a_to_bytes(out + 64 * i, &p);
    }
    return bad ? -1 : 0;
}
EXPORT int orc_g2_mul_gen_batch(uint8_t* out, const uint8_t* k, size_t n) {
    oracle_init();
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < (long)n; i++) {
        fe x;
        if (!fe_from_bytes(&FR, &x, k + 32 * i)) { bad = 1; continue; }
        g2a p = g2_mul_gen_fe(&x);
        g2a_to_bytes(out + 128 * i, &p);
    }
    return bad ? -1 : 0;
}

/* k G by the fixed-base windowing of the setup (group 1: G1, 64 B out;
 * group 2: G2, 128 B out), for pinning it against double-and-add. */
EXPORT int orc_gen_tab_mul(uint8_t* out, const uint8_t* k, int group) {
    oracle_init();
    fe x;
    if (!fe_from_bytes(&FR, &x, k)) return -1;
    gen_tables_init();
    if (group == 1) {
        g1a p = g1_mul_gen_tab(&x);
        g1a_to_bytes(out, &p);
    } else {
        g2a p = g2_mul_gen_tab(&x);
        g2a_to_bytes(out, &p);
    }
    return 0;
}

/* Pairing value as 12 canonical Fp coefficients of w^0..w^11 (384 bytes). */
EXPORT int orc_pairing(uint8_t* out, const uint8_t* g1, const uint8_t* g2) {
    oracle_init();
    g1a P;
    g2a Q;
    if (!g1a_from_bytes(&P, g1) || !g2a_from_bytes(&Q, g2)) return -1;
    fe12 e;
    tate_pairing(&e, &P, &Q);
    for (int i = 0; i < 12; i++) fe_to_bytes(&FP, out + 32 * i, &e.c[i]);
    return 0;
}
static int f12_from_bytes(fe12* r, const uint8_t* b) {
    for (int i = 0; i < 12; i++)
        if (!fe_from_bytes(&FP, &r->c[i], b + 32 * i)) return 0;
    return 1;
}
static void f12_to_bytes(uint8_t* b, const fe12* a) {
    for (int i = 0; i < 12; i++) fe_to_bytes(&FP, b + 32 * i, &a->c[i]);
}
EXPORT int orc_fp12_mul(uint8_t* out, const uint8_t* a, const uint8_t* b) {
    oracle_init();
    fe12 x, y;
    if (!f12_from_bytes(&x, a) || !f12_from_bytes(&y, b)) return -1;
    f12_mul(&x, &x, &y);
    f12_to_bytes(out, &x);
    return 0;
}
EXPORT int orc_fp12_pow(uint8_t* out, const uint8_t* a, const uint8_t* k) {
    oracle_init();
    fe12 x;
    if (!f12_from_bytes(&x, a)) return -1;
    uint64_t kk[4];
    bytes_to_u256(kk, k);
    f12_pow(&x, &x, kk, 4);
    f12_to_bytes(out, &x);
    return 0;
}
/* 1 if the untwisted image of Q satisfies y^2 = x^3 + 3 over Fp12 */
EXPORT int orc_untwist_on_curve(const uint8_t* g2) {
    oracle_init();
    g2a Q;
    if (!g2a_from_bytes(&Q, g2) || Q.inf) return -1;
    fe12 x, y, l, r;
    untwist(&x, &y, &Q);
    f12_mul(&l, &y, &y);
    f12_mul(&r, &x, &x);
    f12_mul(&r, &r, &x);
    f_add(&FP, &r.c[0], &r.c[0], &B_G1);
    return f12_eq(&l, &r);
}

EXPORT void orc_fr_root_of_unity(uint8_t* out, uint32_t log_n) {
    oracle_init();
    fe w;
    fr_root_of_unity(&w, log_n);
    fe_to_bytes(&FR, out, &w);
}

/* In-place NTT of n = 2^log_n canonical Fr values (natural order). */
EXPORT int orc_ntt(uint8_t* data, uint32_t log_n, int inverse) {
    oracle_init();
    size_t n = (size_t)1 << log_n;
    fe* a = (fe*)malloc(sizeof(fe) * n);
    for (size_t i = 0; i < n; i++)
        if (!fe_from_bytes(&FR, &a[i], data + 32 * i)) { free(a); return -1; }
    ntt_inplace(a, log_n, inverse);
    for (size_t i = 0; i < n; i++) fe_to_bytes(&FR, data + 32 * i, &a[i]);
    free(a);
    return 0;
}

/* Transforms on the coset g H of the domain H = {omega^j} (the quotient of
 * the Groth16 QAP is evaluated where Z(X) = X^N - 1 is the non-zero constant
 * g^N - 1).  Written from the definition, with the plain NTT above as a step:
 *   forward (inverse = 0): out_j = sum_i a_i (g omega^j)^i, i.e. the NTT of
 *     the scaled coefficients a_i g^i;
 *   inverse (inverse = 1): the coefficients c_i of the polynomial whose values
 *     at g omega^j are the inputs, i.e. c_i = (iNTT a)_i g^-i.
 * g is a small integer (the library uses g = 5), canonical values in and out. */
EXPORT int orc_coset_ntt(uint8_t* data, uint32_t log_n, uint32_t g, int inverse) {
    oracle_init();
    size_t n = (size_t)1 << log_n;
    fe* a = (fe*)malloc(sizeof(fe) * n);
    for (size_t i = 0; i < n; i++)
        if (!fe_from_bytes(&FR, &a[i], data + 32 * i)) { free(a); return -1; }
    fe gm;
    f_from_u64(&FR, &gm, g);
    if (f_is_zero(&gm)) { free(a); return -1; }
    if (inverse) {
        ntt_inplace(a, log_n, 1);
        f_inv(&FR, &gm, &gm);
    }
    fe gi = FR.one;
    for (size_t i = 0; i < n; i++) {
        f_mul(&FR, &a[i], &a[i], &gi);
        f_mul(&FR, &gi, &gi, &gm);
    }
    if (!inverse) ntt_inplace(a, log_n, 0);
    for (size_t i = 0; i < n; i++) fe_to_bytes(&FR, data + 32 * i, &a[i]);
    free(a);
    return 0;
}

/* MSM: pts are affine (64 B G1 / 128 B G2), scalars 32-byte canonical Fr. */
EXPORT int orc_msm_g1(uint8_t* out, const uint8_t* pts, const uint8_t* scalars, size_t n, int method) {
    oracle_init();
    g1a* P = (g1a*)malloc(sizeof(g1a) * (n ? n : 1));
    uint64_t (*k)[4] = malloc(sizeof(uint64_t[4]) * (n ? n : 1));
    for (size_t i = 0; i < n; i++) {
        if (!g1a_from_bytes(&P[i], pts + 64 * i)) { free(P); free(k); return -1; }
        bytes_to_u256(k[i], scalars + 32 * i);
    }
    g1j r;
    msm_g1(&r, P, (const uint64_t (*)[4])k, n, method);
    g1a ra;
    g1j_to_affine(&ra, &r);
    g1a_to_bytes(out, &ra);
    free(P);
    free(k);
    return 0;
}
EXPORT int orc_msm_g2(uint8_t* out, const uint8_t* pts, const uint8_t* scalars, size_t n, int method) {
    oracle_init();
    g2a* P = (g2a*)malloc(sizeof(g2a) * (n ? n : 1));
    uint64_t (*k)[4] = malloc(sizeof(uint64_t[4]) * (n ? n : 1));
    for (size_t i = 0; i < n; i++) {
        if (!g2a_from_bytes(&P[i], pts + 128 * i)) { free(P); free(k); return -1; }
        bytes_to_u256(k[i], scalars + 32 * i);
    }
    g2j r;
    msm_g2(&r, P, (const uint64_t (*)[4])k, n, method);
    g2a ra;
    g2j_to_affine(&ra, &r);
    g2a_to_bytes(out, &ra);
    free(P);
    free(k);
    return 0;
}

EXPORT void orc_splitmix64(uint64_t seed, uint64_t purpose, size_t n, uint64_t* out) {
    smx g;
    smx_init(&g, seed, purpose);
    for (size_t i = 0; i < n; i++) out[i] = smx_next(&g);
}
EXPORT void orc_sample_fr(uint64_t seed, uint64_t purpose, size_t n, uint8_t* out) {
    oracle_init();
    smx g;
    smx_init(&g, seed, purpose);
    for (size_t i = 0; i < n; i++) {
        fe x;
        smx_fr(&g, &x);
        fe_to_bytes(&FR, out + 32 * i, &x);
    }
}
EXPORT void orc_rs_from_seed(uint64_t seed, uint8_t* r, uint8_t* s) {
    oracle_init();
    fe rr, ss;
    rs_from_seed(seed, &rr, &ss);
    fe_to_bytes(&FR, r, &rr);
    fe_to_bytes(&FR, s, &ss);
}

/* ---- circuits ---- */
EXPORT void* orc_circuit_new(uint32_t log_n, uint32_t n_rows, uint32_t n_perm, uint32_t n_pack,
                             uint32_t pack_bits, uint64_t seed, int with_witness, uint64_t input_seed) {
    return circuit_build(log_n, n_rows, n_perm, n_pack, pack_bits, seed, with_witness, input_seed);
}
EXPORT void orc_circuit_free(void* h) { circuit_free((circuit*)h); }
/* info: N, m, n_rows, n_chain, nnz_A, nnz_B, nnz_C, rows_per_perm */
EXPORT void orc_circuit_info(const void* h, uint64_t* info) {
    const circuit* cs = (const circuit*)h;
    info[0] = cs->N; info[1] = cs->m; info[2] = cs->n_rows; info[3] = cs->n_chain;
    info[4] = cs->nnz[0]; info[5] = cs->nnz[1]; info[6] = cs->nnz[2]; info[7] = ROWS_PER_PERM;
}
EXPORT int orc_circuit_witness(const void* h, uint8_t* z_out) {
    const circuit* cs = (const circuit*)h;
    if (!cs->have_witness) return -1;
    for (size_t j = 0; j < cs->m; j++) fe_to_bytes(&FR, z_out + 32 * j, &cs->z[j]);
    return 0;
}
/* terms of row `row` of matrix k (0 A, 1 B, 2 C): returns count, fills up to max */
EXPORT long orc_circuit_row(const void* h, int k, size_t row, uint32_t* cols, uint8_t* vals, size_t max) {
    const circuit* cs = (const circuit*)h;
    if (k < 0 || k > 2 || row >= cs->N) return -1;
    size_t b = cs->rp[k][row], e = cs->rp[k][row + 1];
    for (size_t i = b; i < e && i - b < max; i++) {
        cols[i - b] = cs->col[k][i];
        fe_to_bytes(&FR, vals + 32 * (i - b), &cs->val[k][i]);
    }
    return (long)(e - b);
}
/* The Poseidon-style constants: rc (65x3), mds (3x3) as canonical bytes. */
EXPORT void orc_circuit_constants(const void* h, uint8_t* rc, uint8_t* mds) {
    const circuit* cs = (const circuit*)h;
    for (int r = 0; r < PSN_ROUNDS; r++)
        for (int l = 0; l < 3; l++) fe_to_bytes(&FR, rc + 32 * (3 * r + l), &cs->rc[r][l]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) fe_to_bytes(&FR, mds + 32 * (3 * i + j), &cs->mds[i][j]);
}

static fe* z_from_bytes(const circuit* cs, const uint8_t* zb) {
    fe* z = (fe*)malloc(sizeof(fe) * cs->m);
    for (size_t j = 0; j < cs->m; j++)
        if (!fe_from_bytes(&FR, &z[j], zb + 32 * j)) { free(z); return NULL; }
    return z;
}
EXPORT int orc_r1cs_check(const void* h, const uint8_t* zb) {
    const circuit* cs = (const circuit*)h;
    fe* z = z_from_bytes(cs, zb);
    if (!z) return -1;
    int ok = r1cs_check(cs, z);
    free(z);
    return ok;
}
/* a = Az, b = Bz, c = Cz (N entries each) */
EXPORT int orc_spmv(const void* h, const uint8_t* zb, uint8_t* a, uint8_t* b, uint8_t* c) {
    const circuit* cs = (const circuit*)h;
    fe* z = z_from_bytes(cs, zb);
    if (!z) return -1;
    uint8_t* outs[3] = {a, b, c};
    fe* tmp = (fe*)malloc(sizeof(fe) * cs->N);
    for (int k = 0; k < 3; k++) {
        spmv(cs, k, z, tmp);
        for (size_t i = 0; i < cs->N; i++) fe_to_bytes(&FR, outs[k] + 32 * i, &tmp[i]);
    }
    free(tmp);
    free(z);
    return 0;
}
EXPORT int orc_qap_h(const void* h, const uint8_t* zb, uint8_t* hout) {
    const circuit* cs = (const circuit*)h;
    fe* z = z_from_bytes(cs, zb);
    if (!z) return -1;
    fe* hh = (fe*)malloc(sizeof(fe) * cs->N);
    int ok = qap_h(cs, z, hh);
    for (size_t i = 0; i < cs->N; i++) fe_to_bytes(&FR, hout + 32 * i, &hh[i]);
    free(hh);
    free(z);
    return ok;
}

/* ---- setup / prove / verify ---- */
EXPORT void* orc_setup(const void* h, uint64_t toxic_seed, int with_points) {
    oracle_init();
    return setup((const circuit*)h, toxic_seed, with_points);
}
EXPORT void orc_pk_free(void* pk) { pk_free((pk_t*)pk); }
/* query: 0 u_j, 1 v_j, 2 w_j, 3 L/IC scalar, 4 H scalar, 5 toxic (0 tau,1 alpha,2 beta,3 gamma,4 delta) */
EXPORT int orc_pk_scalar(const void* pkv, int query, size_t idx, uint8_t* out) {
    const pk_t* pk = (const pk_t*)pkv;
    const fe* src = NULL;
    switch (query) {
    case 0: if (idx >= pk->m) return -1; src = &pk->u[idx]; break;
    case 1: if (idx >= pk->m) return -1; src = &pk->v[idx]; break;
    case 2: if (idx >= pk->m) return -1; src = &pk->w[idx]; break;
    case 3: if (idx >= pk->m) return -1; src = &pk->lq[idx]; break;
    case 4: if (idx + 1 >= pk->N) return -1; src = &pk->hq[idx]; break;
    case 5: {
        const fe* t[5] = {&pk->tau, &pk->alpha, &pk->beta, &pk->gamma, &pk->delta};
        if (idx >= 5) return -1;
        src = t[idx];
        break;
    }
    default: return -1;
    }
    fe_to_bytes(&FR, out, src);
    return 0;
}
/* point: 0 A_j, 1 B1_j, 2 B2_j (128 B), 3 L_j, 4 H_i, 5 vk/pk fixed points
 * (idx 0 alpha1, 1 beta1, 2 delta1, 3 beta2, 4 gamma2, 5 delta2, 6 IC0, 7 IC1) */
EXPORT int orc_pk_point(const void* pkv, int query, size_t idx, uint8_t* out) {
    const pk_t* pk = (const pk_t*)pkv;
    if (query == 5) {
        switch (idx) {
        case 0: g1a_to_bytes(out, &pk->alpha1); return 0;
        case 1: g1a_to_bytes(out, &pk->beta1); return 0;
        case 2: g1a_to_bytes(out, &pk->delta1); return 0;
        case 3: g2a_to_bytes(out, &pk->beta2); return 0;
        case 4: g2a_to_bytes(out, &pk->gamma2); return 0;
        case 5: g2a_to_bytes(out, &pk->delta2); return 0;
        case 6: g1a_to_bytes(out, &pk->IC[0]); return 0;
        case 7: g1a_to_bytes(out, &pk->IC[1]); return 0;
        default: return -1;
        }
    }
    if (!pk->with_points) return -1;
    switch (query) {
    case 0: if (idx >= pk->m) return -1; g1a_to_bytes(out, &pk->A[idx]); return 0;
    case 1: if (idx >= pk->m) return -1; g1a_to_bytes(out, &pk->B1[idx]); return 0;
    case 2: if (idx >= pk->m) return -1; g2a_to_bytes(out, &pk->B2[idx]); return 0;
    case 3: if (idx >= pk->m) return -1; g1a_to_bytes(out, &pk->L[idx]); return 0;
    case 4: if (idx + 1 >= pk->N) return -1; g1a_to_bytes(out, &pk->H[idx]); return 0;
    default: return -1;
    }
}
/* returns 1 on success, 0 if the witness does not satisfy the R1CS, <0 on error */
EXPORT int orc_prove(const void* pkv, const uint8_t* zb, const uint8_t* rb, const uint8_t* sb, int method,
                     uint8_t* proof) {
    const pk_t* pk = (const pk_t*)pkv;
    fe* z = z_from_bytes(pk->cs, zb);
    fe r, s;
    if (!z || !fe_from_bytes(&FR, &r, rb) || !fe_from_bytes(&FR, &s, sb)) { free(z); return -1; }
    int ok = prove(pk, z, &r, &s, method, proof);
    free(z);
    return ok;
}
EXPORT int orc_expected_proof(const void* pkv, const uint8_t* zb, const uint8_t* rb, const uint8_t* sb,
                              uint8_t* proof) {
    const pk_t* pk = (const pk_t*)pkv;
    fe* z = z_from_bytes(pk->cs, zb);
    fe r, s;
    if (!z || !fe_from_bytes(&FR, &r, rb) || !fe_from_bytes(&FR, &s, sb)) { free(z); return -1; }
    expected_proof(pk, z, &r, &s, proof);
    free(z);
    return 0;
}
EXPORT int orc_verify(const void* pkv, const uint8_t* pub, const uint8_t* proof) {
    oracle_init();
    fe x;
    if (!fe_from_bytes(&FR, &x, pub)) return -1;
    return verify((const pk_t*)pkv, &x, proof);
}
EXPORT size_t orc_rows_per_perm(void) { return ROWS_PER_PERM; }
