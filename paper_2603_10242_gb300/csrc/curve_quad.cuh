// curve_quad.cuh -- point doubling and addition on four lanes (internal).
#pragma once
#include "curve.cuh"

namespace ace {

// ---------------------------------------------------------------------------
// Four lanes on one point.  A sequential chain of doublings and additions
// (Horner over the windows) is bound by the latency of its field products,
// not by throughput.  The products of one step of dbl-2008-s-1 / add-2008-s
// form a few levels of independent products (3 levels for a doubling instead
// of 9 products, 4 for an addition instead of 16), so four lanes holding the
// same point each compute one product of a level and exchange the results by
// shuffles.  Every product is fully reduced, so a value does not depend on
// the lane that computed it, and squares are computed as plain products:
// the result equals xyzz_dbl / xyzz_add bit for bit.  `mask` names the four
// lanes, which must all call with the same arguments.
// ---------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ Fe<C> quad_get(unsigned mask, const Fe<C>& x, int src) {
    Fe<C> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = __shfl_sync(mask, x.v[i], src, 4);
    return r;
}
__device__ __forceinline__ fp2_t quad_get(unsigned mask, const fp2_t& x, int src) {
    return {quad_get(mask, x.c0, src), quad_get(mask, x.c1, src)};
}
template <class F>
__device__ __forceinline__ F quad_pick(int sub, const F& a, const F& b, const F& c, const F& d) {
    return sub == 0 ? a : sub == 1 ? b : sub == 2 ? c : d;
}

template <class F>
__device__ Xyzz<F> quad_dbl(const Xyzz<F>& p, int sub, unsigned mask) {
    if (xyzz_is_inf(p)) return p;
    const F U = fe_dbl(p.Y);
    // V = U^2, xx = X^2
    F a = quad_pick(sub, U, p.X, U, p.X);
    F m = a * a;
    const F V = quad_get(mask, m, 0), xx = quad_get(mask, m, 1);
    const F M = fe_dbl(xx) + xx;
    // W = U V, S = X V, ZZ3 = V ZZ, M^2
    m = quad_pick(sub, U, p.X, V, M) * quad_pick(sub, V, V, p.ZZ, M);
    const F W = quad_get(mask, m, 0), S = quad_get(mask, m, 1);
    Xyzz<F> r;
    r.ZZ = quad_get(mask, m, 2);
    r.X = quad_get(mask, m, 3) - fe_dbl(S);
    // M (S - X3), W Y, ZZZ3 = W ZZZ
    m = quad_pick(sub, M, W, W, W) * quad_pick(sub, S - r.X, p.Y, p.ZZZ, p.ZZZ);
    r.Y = quad_get(mask, m, 0) - quad_get(mask, m, 1);
    r.ZZZ = quad_get(mask, m, 2);
    return r;
}

template <class F>
__device__ Xyzz<F> quad_add(const Xyzz<F>& p, const Xyzz<F>& q, int sub, unsigned mask) {
    if (xyzz_is_inf(q)) return p;
    if (xyzz_is_inf(p)) return q;
    // U1 = X1 ZZ2, U2 = X2 ZZ1, S1 = Y1 ZZZ2, S2 = Y2 ZZZ1
    F m = quad_pick(sub, p.X, q.X, p.Y, q.Y) * quad_pick(sub, q.ZZ, p.ZZ, q.ZZZ, p.ZZZ);
    const F U1 = quad_get(mask, m, 0), U2 = quad_get(mask, m, 1);
    const F S1 = quad_get(mask, m, 2), S2 = quad_get(mask, m, 3);
    const F P = U2 - U1, R = S2 - S1;
    if (fe_is_zero(P)) {
        if (fe_is_zero(R)) return quad_dbl(p, sub, mask);
        return xyzz_inf<F>();
    }
    // PP = P^2, R^2, ZZ1 ZZ2, ZZZ1 ZZZ2
    m = quad_pick(sub, P, R, p.ZZ, p.ZZZ) * quad_pick(sub, P, R, q.ZZ, q.ZZZ);
    const F PP = quad_get(mask, m, 0), RR = quad_get(mask, m, 1);
    const F ZZ12 = quad_get(mask, m, 2), ZZZ12 = quad_get(mask, m, 3);
    // PPP = P PP, Q = U1 PP, ZZ3 = ZZ1 ZZ2 PP
    m = quad_pick(sub, P, U1, ZZ12, P) * PP;
    const F PPP = quad_get(mask, m, 0), Q = quad_get(mask, m, 1);
    Xyzz<F> r;
    r.ZZ = quad_get(mask, m, 2);
    r.X = RR - PPP - fe_dbl(Q);
    // R (Q - X3), S1 PPP, ZZZ3 = ZZZ1 ZZZ2 PPP
    m = quad_pick(sub, R, S1, ZZZ12, R) * quad_pick(sub, Q - r.X, PPP, PPP, PPP);
    r.Y = quad_get(mask, m, 0) - quad_get(mask, m, 1);
    r.ZZZ = quad_get(mask, m, 2);
    return r;
}

}  // namespace ace
