// pairing.cuh -- the Fp12 tower of BN254 and a projective Miller loop of the
// optimal ate pairing, usable on the host and the device (internal).
//
// Tower: Fp2 = Fp[u]/(u^2 + 1), Fp6 = Fp2[v]/(v^3 - xi), Fp12 = Fp6[w]/(w^2 - v)
// with xi = 9 + u; Fp12 basis order c0 = (w^0, w^2, w^4), c1 = (w^1, w^3, w^5).
// G2 lives on the sextic twist E': y^2 = x^3 + b', b' = 3/xi; an untwisted
// point is (x w^2, y w^3).
//
// Miller loop in homogeneous projective coordinates (x = X/Z, y = Y/Z), no
// inversions.  Lines are scaled by factors in Fp2, which the final
// exponentiation removes.
//   doubling (the affine tangent line at T times 2 y Z^2 = 2 Y Z): with
//   B = Y^2, E = 3 b' Z^2
//     line = 2YZ yP  -  3X^2 xP w  +  (B - E) w^3
//     X3 = 2XY (B - 3E),  Y3 = (B + 3E)^2 - 12 E^2,  Z3 = 8 B YZ
//   mixed addition T + Q (Q affine): theta = y2 Z - Y, eta = x2 Z - X
//     line = eta yP  -  theta xP w  +  (theta x2 - eta y2) w^3
//     u = theta^2 Z - eta^2 (X + x2 Z),  X3 = eta u,
//     Y3 = theta (eta^2 X - u) - eta^3 Y,  Z3 = eta^3 Z
// (from the affine formulas lambda = 3x^2 / 2y and (y2 - y)/(x2 - x) with the
// curve equation Y^2 Z = X^3 + b' Z^3 used to remove X^3).  The loop runs over
// the bits of 6x + 2 (x = 4965661367192848881, Vercauteren 2010), then adds
// pi(Q) and -pi^2(Q).
#pragma once
#include "field.cuh"

namespace ace {
namespace {

typedef fp2_t F2;
struct F6 {
    F2 a0, a1, a2;
};
struct F12 {
    F6 c0, c1;
};

ACE_HD F2 f2_zero() { return field_zero<fp2_t>(); }
ACE_HD F2 f2_one() { return field_one<fp2_t>(); }
ACE_HD F2 f2_conj(const F2& a) { return {a.c0, fe_neg(a.c1)}; }
ACE_HD F2 f2_scale(const F2& a, const fp_t& s) { return {a.c0 * s, a.c1 * s}; }
// (a0 + a1 u)(9 + u) = (9 a0 - a1) + (a0 + 9 a1) u
ACE_HD F2 mul_xi(const F2& a) {
    fp_t a8 = fe_dbl(fe_dbl(fe_dbl(a.c0))), b8 = fe_dbl(fe_dbl(fe_dbl(a.c1)));
    return {a8 + a.c0 - a.c1, a.c0 + b8 + a.c1};
}

ACE_HD F6 f6_zero() { return {f2_zero(), f2_zero(), f2_zero()}; }
ACE_HD F6 f6_one() { return {f2_one(), f2_zero(), f2_zero()}; }
ACE_HD F6 operator+(const F6& a, const F6& b) { return {a.a0 + b.a0, a.a1 + b.a1, a.a2 + b.a2}; }
ACE_HD F6 operator-(const F6& a, const F6& b) { return {a.a0 - b.a0, a.a1 - b.a1, a.a2 - b.a2}; }
ACE_HD F6 f6_neg(const F6& a) { return {fe_neg(a.a0), fe_neg(a.a1), fe_neg(a.a2)}; }
// Karatsuba over Fp2 (6 products): with v_i = a_i b_i,
// c0 = v0 + xi ((a1 + a2)(b1 + b2) - v1 - v2), c1 = (a0 + a1)(b0 + b1) - v0 - v1 + xi v2,
// c2 = (a0 + a2)(b0 + b2) - v0 - v2 + v1
ACE_HD F6 operator*(const F6& a, const F6& b) {
    F2 v0 = a.a0 * b.a0, v1 = a.a1 * b.a1, v2 = a.a2 * b.a2;
    F2 c0 = v0 + mul_xi((a.a1 + a.a2) * (b.a1 + b.a2) - v1 - v2);
    F2 c1 = (a.a0 + a.a1) * (b.a0 + b.a1) - v0 - v1 + mul_xi(v2);
    F2 c2 = (a.a0 + a.a2) * (b.a0 + b.a2) - v0 - v2 + v1;
    return {c0, c1, c2};
}
// a (x0 + x1 v): the Fp6 product with a factor of zero v^2 coefficient
ACE_HD F6 f6_mul_01(const F6& a, const F2& x0, const F2& x1) {
    F2 v0 = a.a0 * x0, v1 = a.a1 * x1;
    F2 c0 = v0 + mul_xi((a.a1 + a.a2) * x1 - v1);
    F2 c1 = (a.a0 + a.a1) * (x0 + x1) - v0 - v1;
    F2 c2 = a.a2 * x0 + v1;
    return {c0, c1, c2};
}
ACE_HD F6 mul_v(const F6& a) { return {mul_xi(a.a2), a.a0, a.a1}; }
ACE_HD F6 f6_inv(const F6& a) {
    F2 t0 = fe_sqr(a.a0) - mul_xi(a.a1 * a.a2);
    F2 t1 = mul_xi(fe_sqr(a.a2)) - a.a0 * a.a1;
    F2 t2 = fe_sqr(a.a1) - a.a0 * a.a2;
    F2 d = a.a0 * t0 + mul_xi(a.a2 * t1 + a.a1 * t2);
    F2 di = fe_inv(d);
    return {t0 * di, t1 * di, t2 * di};
}
ACE_HD bool f6_eq(const F6& a, const F6& b) { return fe_eq(a.a0, b.a0) && fe_eq(a.a1, b.a1) && fe_eq(a.a2, b.a2); }

ACE_HD F12 f12_one() { return {f6_one(), f6_zero()}; }
// Karatsuba over Fp6: (a0 + a1 w)(b0 + b1 w) = a0 b0 + a1 b1 v + ((a0 + a1)(b0 + b1) - a0 b0 - a1 b1) w
ACE_HD F12 operator*(const F12& a, const F12& b) {
    F6 t0 = a.c0 * b.c0, t1 = a.c1 * b.c1;
    F6 t2 = (a.c0 + a.c1) * (b.c0 + b.c1);
    return {t0 + mul_v(t1), t2 - t0 - t1};
}
// (a0 + a1 w)^2 = (a0 + a1)(a0 + v a1) - a0 a1 - v a0 a1 + 2 a0 a1 w: two Fp6 products
ACE_HD F12 f12_sqr(const F12& a) {
    F6 t = a.c0 * a.c1;
    F6 u = (a.c0 + a.c1) * (a.c0 + mul_v(a.c1));
    return {u - t - mul_v(t), t + t};
}
ACE_HD F12 f12_conj(const F12& a) { return {a.c0, f6_neg(a.c1)}; }
ACE_HD F12 f12_inv(const F12& a) {
    F6 d = a.c0 * a.c0 - mul_v(a.c1 * a.c1);
    F6 di = f6_inv(d);
    return {a.c0 * di, f6_neg(a.c1 * di)};
}
ACE_HD bool f12_eq(const F12& a, const F12& b) { return f6_eq(a.c0, b.c0) && f6_eq(a.c1, b.c1); }

// f times a line value with only the w^0, w^1 and w^3 coefficients:
// l = l0 + l1 w + l3 w^3 = (l0 + 0 v + 0 v^2) + (l1 + l3 v + 0 v^2) w, so
// f0 l0 + v (f1 (l1 + l3 v)) + ((f0 + f1)(l0 + l1 + l3 v) - f0 l0 - f1 (l1 + l3 v)) w
ACE_HD F12 f12_mul_line(const F12& f, const F2& l0, const F2& l1, const F2& l3) {
    F6 t0 = {f.c0.a0 * l0, f.c0.a1 * l0, f.c0.a2 * l0};
    F6 t1 = f6_mul_01(f.c1, l1, l3);
    F6 t2 = f6_mul_01(f.c0 + f.c1, l0 + l1, l3);
    return {t0 + mul_v(t1), t2 - t0 - t1};
}

// constants of the Miller loop (built on the host)
struct PairConsts {
    F2 gamma[6];       // xi^(k (p-1)/6): Frobenius of w^k
    F2 b2;             // b' = 3 / xi
    uint64_t ate_lo;   // 6x + 2, a 65-bit value
    uint64_t ate_hi;
};

struct G2Proj {
    F2 X, Y, Z;
};

// f *= tangent line at T (evaluated at P), T = 2T
ACE_HD void miller_dbl(F12& f, G2Proj& T, const fp_t& xp, const fp_t& yp, const PairConsts& k) {
    F2 YZ = T.Y * T.Z;
    F2 B = fe_sqr(T.Y);
    F2 Z2 = fe_sqr(T.Z);
    F2 E = k.b2 * (Z2 + Z2 + Z2);
    F2 XX = fe_sqr(T.X);
    F2 l0 = f2_scale(YZ + YZ, yp);
    F2 l1 = fe_neg(f2_scale(XX + XX + XX, xp));
    F2 l3 = B - E;
    f = f12_mul_line(f, l0, l1, l3);
    F2 E3 = E + E + E;
    F2 XY = T.X * T.Y;
    F2 X3 = (XY + XY) * (B - E3);
    F2 BE = B + E3;
    F2 EE = fe_sqr(E);
    F2 EE4 = fe_dbl(fe_dbl(EE));
    F2 Y3 = fe_sqr(BE) - (EE4 + EE4 + EE4);
    F2 B8 = fe_dbl(fe_dbl(fe_dbl(B)));
    F2 Z3 = B8 * YZ;
    T.X = X3;
    T.Y = Y3;
    T.Z = Z3;
}

// f *= line through T and Q (Q affine), T = T + Q; false if the line is
// vertical (T = +-Q: not reached for inputs of order r)
ACE_HD bool miller_add(F12& f, G2Proj& T, const F2& x2, const F2& y2, const fp_t& xp, const fp_t& yp) {
    F2 theta = y2 * T.Z - T.Y;
    F2 eta = x2 * T.Z - T.X;
    if (fe_is_zero(eta)) return false;
    F2 l0 = f2_scale(eta, yp);
    F2 l1 = fe_neg(f2_scale(theta, xp));
    F2 l3 = theta * x2 - eta * y2;
    f = f12_mul_line(f, l0, l1, l3);
    F2 ee = fe_sqr(eta);
    F2 eee = ee * eta;
    F2 u = fe_sqr(theta) * T.Z - ee * (T.X + x2 * T.Z);
    F2 X3 = eta * u;
    F2 Y3 = theta * (ee * T.X - u) - eee * T.Y;
    F2 Z3 = eee * T.Z;
    T.X = X3;
    T.Y = Y3;
    T.Z = Z3;
    return true;
}

// Miller function of the optimal ate pairing for P = (xp, yp) in G1 and
// Q = (qx, qy) in G2 (Montgomery affine, neither at infinity)
ACE_HD bool miller_proj(const fp_t& xp, const fp_t& yp, const F2& qx, const F2& qy, const PairConsts& k, F12& out) {
    F12 f = f12_one();
    G2Proj T = {qx, qy, f2_one()};
    int top = 64;
    while (top > 0 && !(top >= 64 ? (k.ate_hi >> (top - 64)) & 1u : (k.ate_lo >> top) & 1u)) top--;
    for (int i = top - 1; i >= 0; i--) {
        f = f12_sqr(f);
        miller_dbl(f, T, xp, yp, k);
        const uint64_t bit = i >= 64 ? (k.ate_hi >> (i - 64)) & 1u : (k.ate_lo >> i) & 1u;
        if (bit && !miller_add(f, T, qx, qy, xp, yp)) return false;
    }
    // pi(Q) = (conj(x) gamma_2, conj(y) gamma_3); -pi^2(Q) = (x gamma_2 conj(gamma_2), -y gamma_3 conj(gamma_3))
    F2 q1x = f2_conj(qx) * k.gamma[2], q1y = f2_conj(qy) * k.gamma[3];
    F2 q2x = qx * k.gamma[2] * f2_conj(k.gamma[2]), q2y = fe_neg(qy * k.gamma[3] * f2_conj(k.gamma[3]));
    if (!miller_add(f, T, q1x, q1y, xp, yp)) return false;
    if (!miller_add(f, T, q2x, q2y, xp, yp)) return false;
    out = f;
    return true;
}

}  // namespace
}  // namespace ace
