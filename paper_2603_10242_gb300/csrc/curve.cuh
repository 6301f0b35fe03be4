// curve.cuh -- BN254 G1 (y^2 = x^3 + 3 over Fp) and G2 (the twist
// y^2 = x^3 + 3/(9+u) over Fp2), in extended Jacobian "XYZZ" coordinates:
// (X, Y, ZZ, ZZZ) represents (X/ZZ, Y/ZZZ) with ZZ^3 = ZZZ^2; ZZ = 0 is the
// point at infinity.  Formulas: madd-2008-s (8M + 2S), add-2008-s
// (12M + 2S), dbl-2008-s-1 and mdbl-2008-s-1 of the Explicit-Formulas
// Database, specialised to a = 0.
//
// The MSMs of the Groth16 prover (the paper's Groth16.Prove, Section 3.1
// Algorithm 1) accumulate affine points into XYZZ buckets: one mixed addition
// per non-zero signed digit.
#pragma once
#include "field.cuh"

namespace ace {

template <class F>
struct Affine {
    F x, y;  // (0, 0) encodes infinity
};
template <class F>
struct Xyzz {
    F X, Y, ZZ, ZZZ;
};

typedef Affine<fp_t> g1_aff;
typedef Affine<fp2_t> g2_aff;
typedef Xyzz<fp_t> g1_xyzz;
typedef Xyzz<fp2_t> g2_xyzz;

template <class F>
ACE_HD Xyzz<F> xyzz_inf() {
    Xyzz<F> r;
    r.X = field_one<F>();
    r.Y = field_one<F>();
    r.ZZ = field_zero<F>();
    r.ZZZ = field_zero<F>();
    return r;
}
template <class F>
ACE_HD bool xyzz_is_inf(const Xyzz<F>& p) { return fe_is_zero(p.ZZ); }
template <class F>
ACE_HD bool aff_is_inf(const Affine<F>& p) { return fe_is_zero(p.x) && fe_is_zero(p.y); }
template <class F>
ACE_HD Xyzz<F> xyzz_from_aff(const Affine<F>& p) {
    if (aff_is_inf(p)) return xyzz_inf<F>();
    Xyzz<F> r;
    r.X = p.x;
    r.Y = p.y;
    r.ZZ = field_one<F>();
    r.ZZZ = field_one<F>();
    return r;
}
template <class F>
ACE_HD Affine<F> aff_neg(const Affine<F>& p) {
    Affine<F> r;
    r.x = p.x;
    r.y = fe_neg(p.y);
    return r;
}
template <class F>
ACE_HD Xyzz<F> xyzz_neg(const Xyzz<F>& p) {
    Xyzz<F> r = p;
    r.Y = fe_neg(p.Y);
    return r;
}

// 2P for an affine P (mdbl-2008-s-1)
template <class F>
ACE_HD Xyzz<F> xyzz_dbl_aff(const Affine<F>& p) {
    if (aff_is_inf(p)) return xyzz_inf<F>();
    F U = fe_dbl(p.y);
    F V = fe_sqr(U);
    F W = U * V;
    F S = p.x * V;
    F xx = fe_sqr(p.x);
    F M = fe_dbl(xx) + xx;
    Xyzz<F> r;
    r.X = fe_sqr(M) - fe_dbl(S);
    r.Y = fe_mul_sub(M, S - r.X, W, p.y);
    r.ZZ = V;
    r.ZZZ = W;
    return r;
}

// 2P (dbl-2008-s-1, a = 0)
template <class F>
ACE_HD Xyzz<F> xyzz_dbl(const Xyzz<F>& p) {
    if (xyzz_is_inf(p)) return p;
    F U = fe_dbl(p.Y);
    F V = fe_sqr(U);
    F W = U * V;
    F S = p.X * V;
    F xx = fe_sqr(p.X);
    F M = fe_dbl(xx) + xx;
    Xyzz<F> r;
    r.X = fe_sqr(M) - fe_dbl(S);
    r.Y = fe_mul_sub(M, S - r.X, W, p.Y);
    r.ZZ = V * p.ZZ;
    r.ZZZ = W * p.ZZZ;
    return r;
}

// P + Q with Q affine (madd-2008-s)
template <class F>
ACE_HD Xyzz<F> xyzz_add_aff(const Xyzz<F>& p, const Affine<F>& q) {
    if (aff_is_inf(q)) return p;
    if (xyzz_is_inf(p)) return xyzz_from_aff(q);
    F U2 = q.x * p.ZZ;
    F S2 = q.y * p.ZZZ;
    F P = U2 - p.X;
    F R = S2 - p.Y;
    if (fe_is_zero(P)) {
        if (fe_is_zero(R)) return xyzz_dbl_aff(q);
        return xyzz_inf<F>();
    }
    F PP = fe_sqr(P);
    F PPP = P * PP;
    F Q = p.X * PP;
    Xyzz<F> r;
    r.X = fe_sqr(R) - PPP - fe_dbl(Q);
    r.Y = fe_mul_sub(R, Q - r.X, p.Y, PPP);
    r.ZZ = p.ZZ * PP;
    r.ZZZ = p.ZZZ * PPP;
    return r;
}

// P + Q (add-2008-s)
template <class F>
ACE_HD Xyzz<F> xyzz_add(const Xyzz<F>& p, const Xyzz<F>& q) {
    if (xyzz_is_inf(q)) return p;
    if (xyzz_is_inf(p)) return q;
    F U1 = p.X * q.ZZ;
    F U2 = q.X * p.ZZ;
    F S1 = p.Y * q.ZZZ;
    F S2 = q.Y * p.ZZZ;
    F P = U2 - U1;
    F R = S2 - S1;
    if (fe_is_zero(P)) {
        if (fe_is_zero(R)) return xyzz_dbl(p);
        return xyzz_inf<F>();
    }
    F PP = fe_sqr(P);
    F PPP = P * PP;
    F Q = U1 * PP;
    Xyzz<F> r;
    r.X = fe_sqr(R) - PPP - fe_dbl(Q);
    r.Y = fe_mul_sub(R, Q - r.X, S1, PPP);
    r.ZZ = p.ZZ * q.ZZ * PP;
    r.ZZZ = p.ZZZ * q.ZZZ * PPP;
    return r;
}

// (X/ZZ, Y/ZZZ) with a single inversion: I = 1/(ZZ ZZZ), 1/ZZ = I ZZZ, 1/ZZZ = I ZZ
template <class F>
ACE_HD Affine<F> xyzz_to_aff(const Xyzz<F>& p) {
    Affine<F> r;
    if (xyzz_is_inf(p)) {
        r.x = field_zero<F>();
        r.y = field_zero<F>();
        return r;
    }
    F I = fe_inv(p.ZZ * p.ZZZ);
    r.x = p.X * (I * p.ZZZ);
    r.y = p.Y * (I * p.ZZ);
    return r;
}

// k P for a plain 256-bit integer k (8 little-endian limbs), double-and-add
// from the top bit.
template <class F>
ACE_HD Xyzz<F> xyzz_mul_aff(const Affine<F>& p, const uint32_t* k) {
    Xyzz<F> acc = xyzz_inf<F>();
    int top = 255;
    while (top >= 0 && !((k[top >> 5] >> (top & 31)) & 1u)) top--;
    for (int i = top; i >= 0; i--) {
        acc = xyzz_dbl(acc);
        if ((k[i >> 5] >> (i & 31)) & 1u) acc = xyzz_add_aff(acc, p);
    }
    return acc;
}

// Montgomery / canonical conversion of coordinates
ACE_HD fp_t coord_to_mont(const fp_t& a) { return fe_to_mont(a); }
ACE_HD fp2_t coord_to_mont(const fp2_t& a) { return fe_to_mont(a); }
ACE_HD fp_t coord_from_mont(const fp_t& a) { return fe_from_mont(a); }
ACE_HD fp2_t coord_from_mont(const fp2_t& a) { return fe_from_mont(a); }
template <class F>
ACE_HD Affine<F> aff_to_mont(const Affine<F>& p) {
    Affine<F> r;
    r.x = coord_to_mont(p.x);
    r.y = coord_to_mont(p.y);
    return r;
}
template <class F>
ACE_HD Affine<F> aff_from_mont(const Affine<F>& p) {
    Affine<F> r;
    r.x = coord_from_mont(p.x);
    r.y = coord_from_mont(p.y);
    return r;
}

// curve constants b (Montgomery form): G1 b = 3; G2 b' = 3/(9+u)
ACE_HD fp_t g1_b() { return fe_from_u32<FpCfg>(3); }
ACE_HD fp2_t g2_b() {
    fp2_t xi = {fe_from_u32<FpCfg>(9), fe_from_u32<FpCfg>(1)};
    fp2_t three = {fe_from_u32<FpCfg>(3), fe_zero<FpCfg>()};
    return three * fe_inv(xi);
}
template <class F>
ACE_HD F curve_b();
template <>
ACE_HD fp_t curve_b<fp_t>() { return g1_b(); }
template <>
ACE_HD fp2_t curve_b<fp2_t>() { return g2_b(); }

// y^2 == x^3 + b for a Montgomery-form affine point (infinity accepted)
template <class F>
ACE_HD bool aff_on_curve(const Affine<F>& p) {
    if (aff_is_inf(p)) return true;
    F l = fe_sqr(p.y);
    F r = fe_sqr(p.x) * p.x + curve_b<F>();
    return fe_eq(l, r);
}

}  // namespace ace
