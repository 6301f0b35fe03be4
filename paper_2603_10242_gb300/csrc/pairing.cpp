// pairing.cpp -- Groth16 verification on the host: the three-pairing check
// that finalises a block (Section 3.3: a single Groth16 verification, three
// bilinear pairing operations on BN254; Section 3.4, Algorithm 4).
//
// Optimal ate pairing on BN254 (Vercauteren 2010): Miller loop over
// 6x + 2 (x = 4965661367192848881) with Q on the sextic twist
// E': y^2 = x^3 + 3/xi (xi = 9 + u) in affine Fp2 coordinates, line values
// evaluated at P as sparse elements of the tower
//   Fp2 = Fp[u]/(u^2 + 1),  Fp6 = Fp2[v]/(v^3 - xi),  Fp12 = Fp6[w]/(w^2 - v),
// the two Frobenius correction lines (pi(Q), -pi^2(Q)), then one final
// exponentiation: f^(p^6 - 1) by conjugation and inversion, ^(p^2 + 1) by
// the Frobenius map, and ^((p^4 - p^2 + 1)/r) by square-and-multiply.
// For the untwisted T = (x' w^2, y' w^3) the slope is lambda' w, so the line
// through T at P is  y_P - lambda' x_P w + (lambda' x' - y') w^3.
#include <string.h>

#include <vector>

#include "../../include/ace.h"
#include "curve.cuh"
#include "field.cuh"
#include "pairing.cuh"

namespace ace {
void set_error(const char* fmt, ...);
void clear_error();
}  // namespace ace

namespace ace {
namespace {

// ---- constants -------------------------------------------------------------
struct Consts {
    F2 gamma[6];                 // xi^(k (p-1)/6): Frobenius of w^k
    F2 b2;                       // twist coefficient 3/xi
    std::vector<uint32_t> hard;  // (p^4 - p^2 + 1) / r
    uint32_t hard_p[4][8];       // its digits in base p: hard = sum_i hard_p[i] p^i
    unsigned __int128 ate = 0;   // 6x + 2 (a 65-bit value)
};

// small multi-precision helpers on little-endian 32-bit limbs
typedef std::vector<uint32_t> Big;
Big big_from(const uint32_t* l, int n) { return Big(l, l + n); }
Big big_mul(const Big& a, const Big& b) {
    Big r(a.size() + b.size(), 0);
    for (size_t i = 0; i < a.size(); i++) {
        uint64_t c = 0;
        for (size_t j = 0; j < b.size(); j++) {
            c += (uint64_t)r[i + j] + (uint64_t)a[i] * b[j];
            r[i + j] = (uint32_t)c;
            c >>= 32;
        }
        for (size_t k = i + b.size(); c; k++) {
            c += r[k];
            r[k] = (uint32_t)c;
            c >>= 32;
        }
    }
    return r;
}
void big_add_small(Big& a, uint32_t v, bool sub) {
    uint64_t c = v;
    for (size_t i = 0; i < a.size() && c; i++) {
        if (sub) {
            uint32_t old = a[i];
            a[i] = old - (uint32_t)c;
            c = old < c ? 1 : 0;
        } else {
            c += a[i];
            a[i] = (uint32_t)c;
            c >>= 32;
        }
    }
}
Big big_sub(const Big& a, const Big& b) {  // a >= b
    Big r(a);
    int64_t br = 0;
    for (size_t i = 0; i < r.size(); i++) {
        int64_t x = (int64_t)r[i] - (i < b.size() ? b[i] : 0) + br;
        r[i] = (uint32_t)x;
        br = x < 0 ? -1 : 0;
    }
    return r;
}
// quotient of a by the 254-bit modulus d (remainder must be 0)
bool big_div_exact(const Big& a, const uint32_t d[8], Big& q) {
    q.assign(a.size(), 0);
    Big rem(9, 0);
    for (int bit = (int)a.size() * 32 - 1; bit >= 0; bit--) {
        uint32_t carry = (a[bit >> 5] >> (bit & 31)) & 1u;
        for (int i = 0; i < 9; i++) {
            uint32_t nc = rem[i] >> 31;
            rem[i] = (rem[i] << 1) | carry;
            carry = nc;
        }
        bool ge = rem[8] != 0;
        if (!ge) {
            ge = true;
            for (int i = 7; i >= 0; i--) {
                if (rem[i] != d[i]) {
                    ge = rem[i] > d[i];
                    break;
                }
            }
        }
        if (ge) {
            int64_t br = 0;
            for (int i = 0; i < 9; i++) {
                int64_t x = (int64_t)rem[i] - (i < 8 ? d[i] : 0) + br;
                rem[i] = (uint32_t)x;
                br = x < 0 ? -1 : 0;
            }
            q[bit >> 5] |= 1u << (bit & 31);
        }
    }
    for (uint32_t v : rem)
        if (v) return false;
    return true;
}

// q = a / d, r = a mod d for the 254-bit modulus d (bit-serial long division)
void big_divmod(const Big& a, const uint32_t d[8], Big& q, Big& r) {
    q.assign(a.size(), 0);
    Big rem(9, 0);
    for (int bit = (int)a.size() * 32 - 1; bit >= 0; bit--) {
        uint32_t carry = (a[bit >> 5] >> (bit & 31)) & 1u;
        for (int i = 0; i < 9; i++) {
            uint32_t nc = rem[i] >> 31;
            rem[i] = (rem[i] << 1) | carry;
            carry = nc;
        }
        bool ge = rem[8] != 0;
        if (!ge) {
            ge = true;
            for (int i = 7; i >= 0; i--) {
                if (rem[i] != d[i]) {
                    ge = rem[i] > d[i];
                    break;
                }
            }
        }
        if (ge) {
            int64_t br = 0;
            for (int i = 0; i < 9; i++) {
                int64_t x = (int64_t)rem[i] - (i < 8 ? d[i] : 0) + br;
                rem[i] = (uint32_t)x;
                br = x < 0 ? -1 : 0;
            }
            q[bit >> 5] |= 1u << (bit & 31);
        }
    }
    r.assign(rem.begin(), rem.begin() + 8);
}

F2 f2_pow(const F2& a, const Big& e) {
    F2 acc = f2_one();
    for (int i = (int)e.size() * 32 - 1; i >= 0; i--) {
        acc = fe_sqr(acc);
        if ((e[i >> 5] >> (i & 31)) & 1u) acc = acc * a;
    }
    return acc;
}

Consts make_consts() {
    Consts c;
    uint32_t pl[8], rl[8];
    for (int i = 0; i < 8; i++) {
        pl[i] = mod_limb<FpCfg>(i);
        rl[i] = mod_limb<FrCfg>(i);
    }
    Big p = big_from(pl, 8);
    // (p - 1) / 6, then k (p - 1) / 6
    Big pm1 = p;
    big_add_small(pm1, 1, true);
    Big e6;
    {
        // divide by 6 (small divisor)
        e6.assign(pm1.size(), 0);
        uint64_t rem = 0;
        for (int i = (int)pm1.size() - 1; i >= 0; i--) {
            uint64_t cur = (rem << 32) | pm1[i];
            e6[i] = (uint32_t)(cur / 6);
            rem = cur % 6;
        }
    }
    F2 xi = {fe_from_u32<FpCfg>(9), fe_from_u32<FpCfg>(1)};
    for (int k = 0; k < 6; k++) {
        Big kk(1, (uint32_t)k);
        c.gamma[k] = f2_pow(xi, big_mul(e6, kk));
    }
    F2 three = {fe_from_u32<FpCfg>(3), fe_zero<FpCfg>()};
    c.b2 = three * fe_inv(xi);
    // (p^4 - p^2 + 1) / r
    Big p2 = big_mul(p, p);
    Big p4 = big_mul(p2, p2);
    Big num = big_sub(p4, p2);
    big_add_small(num, 1, false);
    Big q;
    big_div_exact(num, rl, q);
    while (q.size() > 1 && q.back() == 0) q.pop_back();
    c.hard = q;
    // base-p digits of the hard exponent (it has four: (p^4 - p^2 + 1)/r < p^4)
    Big rest = q;
    for (int i = 0; i < 4; i++) {
        Big quo, rem;
        big_divmod(rest, pl, quo, rem);
        for (int l = 0; l < 8; l++) c.hard_p[i][l] = l < (int)rem.size() ? rem[l] : 0;
        rest = quo;
    }
    c.ate = (unsigned __int128)6 * 4965661367192848881ull + 2u;
    return c;
}

// built once, thread-safely, on first use
const Consts& consts() {
    static const Consts c = make_consts();
    return c;
}

// a^p: coefficient of w^k is conjugated and multiplied by gamma_k.
// Basis order: c0 = (w^0, w^2, w^4), c1 = (w^1, w^3, w^5).
F12 frobenius(const F12& a) {
    const Consts& k = consts();
    F12 r;
    r.c0.a0 = f2_conj(a.c0.a0) * k.gamma[0];
    r.c0.a1 = f2_conj(a.c0.a1) * k.gamma[2];
    r.c0.a2 = f2_conj(a.c0.a2) * k.gamma[4];
    r.c1.a0 = f2_conj(a.c1.a0) * k.gamma[1];
    r.c1.a1 = f2_conj(a.c1.a1) * k.gamma[3];
    r.c1.a2 = f2_conj(a.c1.a2) * k.gamma[5];
    return r;
}

F12 f12_pow(const F12& a, const Big& e) {
    F12 acc = f12_one();
    for (int i = (int)e.size() * 32 - 1; i >= 0; i--) {
        acc = f12_sqr(acc);
        if ((e[i >> 5] >> (i & 31)) & 1u) acc = acc * a;
    }
    return acc;
}

// t^hard with hard = d0 + d1 p + d2 p^2 + d3 p^3: t^(d_i p^i) = frob^i(t)^d_i,
// so one joint square-and-multiply over the 254-bit digits with the 15
// products of the four Frobenius images (254 squarings instead of 761)
F12 hard_part(const F12& t) {
    const Consts& k = consts();
    F12 b[4];
    b[0] = t;
    for (int i = 1; i < 4; i++) b[i] = frobenius(b[i - 1]);
    F12 tab[16];
    tab[0] = f12_one();
    for (int m = 1; m < 16; m++) {
        int low = m & -m, i = 0;
        while ((1 << i) != low) i++;
        tab[m] = (m == low) ? b[i] : tab[m ^ low] * b[i];
    }
    F12 acc = f12_one();
    for (int bit = 253; bit >= 0; bit--) {
        acc = f12_sqr(acc);
        int m = 0;
        for (int i = 0; i < 4; i++) m |= (int)((k.hard_p[i][bit >> 5] >> (bit & 31)) & 1u) << i;
        if (m) acc = acc * tab[m];
    }
    return acc;
}

F12 final_exp(const F12& f) {
    F12 t = f12_conj(f) * f12_inv(f);          // f^(p^6 - 1)
    t = frobenius(frobenius(t)) * t;           // ^(p^2 + 1)
    return hard_part(t);                       // ^((p^4 - p^2 + 1)/r)
}

// the same power by plain square-and-multiply over the 761-bit exponent (for
// tests of hard_part)
F12 final_exp_plain(const F12& f) {
    F12 t = f12_conj(f) * f12_inv(f);
    t = frobenius(frobenius(t)) * t;
    return f12_pow(t, consts().hard);
}

struct G2a {
    F2 x, y;
    bool inf;
};

// line through T with twist slope lam, evaluated at P = (xp, yp)
F12 line(const F2& lam, const F2& xt, const F2& yt, const fp_t& xp, const fp_t& yp) {
    F12 l;
    l.c0 = f6_zero();
    l.c1 = f6_zero();
    l.c0.a0 = {yp, fe_zero<FpCfg>()};
    l.c1.a0 = fe_neg(f2_scale(lam, xp));
    l.c1.a1 = lam * xt - yt;
    return l;
}

// one Miller step: f *= l_{T,S}(P), T = T + S (S == T: tangent)
bool miller_step(F12& f, G2a& T, const G2a& S, const fp_t& xp, const fp_t& yp) {
    F2 lam;
    if (fe_eq(T.x, S.x)) {
        if (!fe_eq(T.y, S.y) || fe_is_zero(T.y)) return false;  // vertical: not reached for valid inputs
        F2 xx = fe_sqr(T.x);
        lam = (xx + xx + xx) * fe_inv(T.y + T.y);
    } else {
        lam = (S.y - T.y) * fe_inv(S.x - T.x);
    }
    f = f * line(lam, T.x, T.y, xp, yp);
    F2 x3 = fe_sqr(lam) - T.x - S.x;
    F2 y3 = lam * (T.x - x3) - T.y;
    T.x = x3;
    T.y = y3;
    return true;
}

// Miller function of the optimal ate pairing (before the final exponentiation)
bool miller(const fp_t& xp, const fp_t& yp, const G2a& Q, F12& out) {
    const Consts& k = consts();
    F12 f = f12_one();
    G2a T = Q;
    int top = 127;
    while (!((k.ate >> top) & 1u)) top--;
    for (int i = top - 1; i >= 0; i--) {
        f = f * f;
        if (!miller_step(f, T, T, xp, yp)) return false;
        if ((unsigned)(k.ate >> i) & 1u)
            if (!miller_step(f, T, Q, xp, yp)) return false;
    }
    // pi(Q) = (conj(x) gamma_2, conj(y) gamma_3); -pi^2(Q) = (x gamma_2 conj(gamma_2), -y gamma_3 conj(gamma_3))
    G2a Q1 = {f2_conj(Q.x) * k.gamma[2], f2_conj(Q.y) * k.gamma[3], false};
    G2a Q2 = {Q.x * k.gamma[2] * f2_conj(k.gamma[2]), fe_neg(Q.y * k.gamma[3] * f2_conj(k.gamma[3])), false};
    if (!miller_step(f, T, Q1, xp, yp)) return false;
    if (!miller_step(f, T, Q2, xp, yp)) return false;
    out = f;
    return true;
}

bool read_fp(const uint8_t* b, fp_t& out) {
    memcpy(out.v, b, 32);
    if (fe_geq_mod(out)) return false;
    out = fe_to_mont(out);
    return true;
}
bool read_g1(const uint8_t* b, fp_t& x, fp_t& y, bool& inf) {
    if (!read_fp(b, x) || !read_fp(b + 32, y)) return false;
    inf = fe_is_zero(x) && fe_is_zero(y);
    if (inf) return true;
    return fe_eq(fe_sqr(y), fe_sqr(x) * x + fe_from_u32<FpCfg>(3));
}
bool read_g2(const uint8_t* b, G2a& q) {
    if (!read_fp(b, q.x.c0) || !read_fp(b + 32, q.x.c1) || !read_fp(b + 64, q.y.c0) || !read_fp(b + 96, q.y.c1))
        return false;
    q.inf = fe_is_zero(q.x) && fe_is_zero(q.y);
    if (q.inf) return true;
    return fe_eq(fe_sqr(q.y), fe_sqr(q.x) * q.x + consts().b2);
}

// r Q == O on the twist (subgroup membership): XYZZ double-and-add
bool g2_in_subgroup(const G2a& q) {
    if (q.inf) return true;
    uint32_t rl[8];
    for (int i = 0; i < 8; i++) rl[i] = mod_limb<FrCfg>(i);
    g2_aff a = {q.x, q.y};
    return xyzz_is_inf(xyzz_mul_aff(a, rl));
}

// affine G1 helpers for the input term ic0 + x ic1
struct G1a {
    fp_t x, y;
    bool inf;
};
}  // namespace

// Constants and final exponentiation for the device Miller loops (batch
// verification): F12 values cross translation units as 12 Montgomery Fp
// limbs in the order of the tower (c0.a0.c0, c0.a0.c1, ..., c1.a2.c1).
void pairing_consts_raw(fp_t gamma[12], fp_t b2[2], uint64_t* ate_lo, uint64_t* ate_hi) {
    const Consts& k = consts();
    for (int i = 0; i < 6; i++) {
        gamma[2 * i] = k.gamma[i].c0;
        gamma[2 * i + 1] = k.gamma[i].c1;
    }
    b2[0] = k.b2.c0;
    b2[1] = k.b2.c1;
    *ate_lo = (uint64_t)k.ate;
    *ate_hi = (uint64_t)(k.ate >> 64);
}
void final_exp_raw(const fp_t in[12], fp_t out[12]) {
    F12 f;
    static_assert(sizeof(F12) == 12 * sizeof(fp_t), "F12 is 12 Fp values");
    memcpy(&f, in, sizeof f);
    F12 r = final_exp(f);
    memcpy(out, &r, sizeof r);
}
bool final_exp_is_one_raw(const fp_t in[12]) {
    F12 f;
    memcpy(&f, in, sizeof f);
    return f12_eq(final_exp(f), f12_one());
}
// Parse a proof / verifying-key point to Montgomery affine coordinates
// (infinity = zeros); false if not canonical or not on the curve.
bool parse_g1_raw(const uint8_t b[64], fp_t out[2]) {
    bool inf;
    if (!read_g1(b, out[0], out[1], inf)) return false;
    if (inf) out[0] = out[1] = fe_zero<FpCfg>();
    return true;
}
bool parse_g2_raw(const uint8_t b[128], fp_t out[4]) {
    G2a q;
    if (!read_g2(b, q)) return false;
    if (q.inf) q.x = q.y = f2_zero();
    out[0] = q.x.c0;
    out[1] = q.x.c1;
    out[2] = q.y.c0;
    out[3] = q.y.c1;
    return true;
}

// Miller function by the projective loop (the device's), for tests
bool miller_proj_raw(const fp_t& xp, const fp_t& yp, const fp_t q[4], fp_t out[12]) {
    PairConsts k;
    fp_t g[12], b[2];
    pairing_consts_raw(g, b, &k.ate_lo, &k.ate_hi);
    for (int i = 0; i < 6; i++) k.gamma[i] = {g[2 * i], g[2 * i + 1]};
    k.b2 = {b[0], b[1]};
    F12 f;
    if (!miller_proj(xp, yp, {q[0], q[1]}, {q[2], q[3]}, k, f)) return false;
    memcpy(out, &f, sizeof f);
    return true;
}

// product of pairings e(P_i, Q_i) == 1 ?  (P, Q given in Montgomery affine)
int pairing_product_is_one(int n, const fp_t* px, const fp_t* py, const bool* pinf, const G2a* q) {
    static const PairConsts pc = [] {
        PairConsts k;
        fp_t g[12], b[2];
        pairing_consts_raw(g, b, &k.ate_lo, &k.ate_hi);
        for (int i = 0; i < 6; i++) k.gamma[i] = {g[2 * i], g[2 * i + 1]};
        k.b2 = {b[0], b[1]};
        return k;
    }();
    F12 acc = f12_one();
    for (int i = 0; i < n; i++) {
        if (pinf[i] || q[i].inf) continue;
        F12 f;
        if (!miller_proj(px[i], py[i], q[i].x, q[i].y, pc, f)) return -1;
        acc = acc * f;
    }
    return f12_eq(final_exp(acc), f12_one()) ? 1 : 0;
}

}  // namespace ace

using namespace ace;

extern "C" {

int ace_verify(const ace_vk* vk, const ace_fr* pub, size_t n_pub, const uint8_t proof[256]) {
    clear_error();
    if (!vk || !pub || !proof) {
        set_error("ace_verify: NULL argument");
        return ACE_E_ARG;
    }
    if (n_pub != 1) {
        set_error("ace_verify: the circuit has exactly one public input (n_pub = %zu)", n_pub);
        return ACE_E_ARG;
    }
    fr_t x;
    memcpy(x.v, pub->l, 32);
    if (fe_geq_mod(x)) {
        set_error("ace_verify: public input not canonical");
        return ACE_E_ARG;
    }
    fp_t ax, ay, cx, cy;
    bool ainf, cinf;
    G2a B;
    if (!read_g1(proof, ax, ay, ainf) || !read_g1(proof + 192, cx, cy, cinf) || !read_g2(proof + 64, B)) {
        set_error("ace_verify: proof point not on the curve or not canonical");
        return ACE_E_NOT_ON_CURVE;
    }
    if (!g2_in_subgroup(B)) return 0;
    const uint8_t* v = (const uint8_t*)vk;
    fp_t alx, aly, i0x, i0y, i1x, i1y;
    bool alinf, i0inf, i1inf;
    G2a beta, gamma, delta;
    if (!read_g1(v, alx, aly, alinf) || !read_g2(v + 64, beta) || !read_g2(v + 192, gamma) ||
        !read_g2(v + 320, delta) || !read_g1(v + 448, i0x, i0y, i0inf) || !read_g1(v + 512, i1x, i1y, i1inf)) {
        set_error("ace_verify: verifying key point not on the curve");
        return ACE_E_NOT_ON_CURVE;
    }
    g1_xyzz icx = xyzz_mul_aff(g1_aff{i1x, i1y}, x.v);
    if (!i0inf) icx = xyzz_add_aff(icx, g1_aff{i0x, i0y});
    g1_aff ica = xyzz_to_aff(icx);
    G1a ic = {ica.x, ica.y, xyzz_is_inf(icx)};
    // e(-A, B) e(alpha, beta) e(IC, gamma) e(C, delta) == 1
    fp_t px[4] = {ax, alx, ic.x, cx};
    fp_t py[4] = {fe_neg(ay), aly, ic.y, cy};
    bool pinf[4] = {ainf, alinf, ic.inf, cinf};
    G2a q[4] = {B, beta, gamma, delta};
    int rc = pairing_product_is_one(4, px, py, pinf, q);
    if (rc < 0) {
        set_error("ace_verify: degenerate Miller loop");
        return 0;
    }
    return rc;
}

// Diagnostic: e(P, Q) as 12 canonical Fp limbs-triples, tower order
// (c0.a0, c0.a1, c0.a2, c1.a0, c1.a1, c1.a2; each Fp2 as c0, c1).
int ace_debug_pairing(const uint8_t g1[64], const uint8_t g2[128], uint8_t out[384]) {
    return ace_debug_pairing_form(0, g1, g2, out);
}

// form 0: affine Miller loop (the single verifier's); form 1: projective
// Miller loop (the batch verifier's device loop, run here on the host);
// form 2: affine Miller loop and the final exponentiation's hard part by
// plain square-and-multiply over its 761-bit exponent
int ace_debug_pairing_form(int form, const uint8_t g1[64], const uint8_t g2[128], uint8_t out[384]) {
    fp_t x, y;
    bool inf;
    G2a q;
    if (form < 0 || form > 2) return ACE_E_ARG;
    if (!read_g1(g1, x, y, inf) || !read_g2(g2, q)) return ACE_E_NOT_ON_CURVE;
    F12 f = f12_one();
    if (!inf && !q.inf) {
        if (form != 1 && !miller(x, y, q, f)) return ACE_E_ARG;
        if (form == 1) {
            fp_t qq[4] = {q.x.c0, q.x.c1, q.y.c0, q.y.c1}, raw[12];
            if (!miller_proj_raw(x, y, qq, raw)) return ACE_E_ARG;
            memcpy(&f, raw, sizeof f);
        }
    }
    f = form == 2 ? final_exp_plain(f) : final_exp(f);
    const F2* c[6] = {&f.c0.a0, &f.c0.a1, &f.c0.a2, &f.c1.a0, &f.c1.a1, &f.c1.a2};
    for (int i = 0; i < 6; i++) {
        fp_t a = fe_from_mont(c[i]->c0), b = fe_from_mont(c[i]->c1);
        memcpy(out + 64 * i, a.v, 32);
        memcpy(out + 64 * i + 32, b.v, 32);
    }
    return ACE_OK;
}

}  // extern "C"
