"""Pins for the CPU oracle against facts fixed outside it.

Each test compares the oracle with something other than itself: Python
integer arithmetic, textbook affine curve formulas, the O(N^2) DFT, Lagrange
interpolation, closed forms (r*G = O, Fermat, omega^N = 1), pairing
bilinearity / non-degeneracy, brute force on tiny inputs, the discrete-log
identity for MSMs, and the published BN254 constants (EIP-196/197).
"""
import json
import os
import random

import pytest

import oracle as O
import pyref as Y

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = random.Random(20260310)


def test_constants_match_bn_polynomials():
    c = json.load(open(os.path.join(GOLD, "bn254_constants.json")))
    x = int(c["bn_x"])
    assert int(c["p"]) == 36 * x**4 + 36 * x**3 + 24 * x**2 + 6 * x + 1 == O.P == Y.P
    assert int(c["r"]) == 36 * x**4 + 36 * x**3 + 18 * x**2 + 6 * x + 1 == O.R == Y.R
    assert (O.R - 1) % (1 << c["two_adicity_r_minus_1"]) == 0
    assert (O.R - 1) % (1 << (c["two_adicity_r_minus_1"] + 1)) != 0


@pytest.mark.parametrize("which,mod", [("fp", Y.P), ("fr", Y.R)])
def test_field_ops_vs_python_ints(which, mod):
    edge = [0, 1, 2, mod - 1, mod - 2, (1 << 253) % mod, (1 << 128) + 1, mod // 2]
    vals = edge + [rng.randrange(mod) for _ in range(60)]
    for a in vals:
        for b in (vals[rng.randrange(len(vals))], vals[rng.randrange(len(vals))]):
            assert O.field_op(which, "add", a, b) == (a + b) % mod
            assert O.field_op(which, "sub", a, b) == (a - b) % mod
            assert O.field_op(which, "mul", a, b) == (a * b) % mod
        assert O.field_op(which, "neg", a) == (-a) % mod
        if a:
            inv = O.field_op(which, "inv", a)
            assert inv * a % mod == 1
            # Fermat: a^(mod-1) = 1
            assert O.field_op(which, "pow", a, mod - 1) == 1


def test_field_rejects_non_canonical():
    with pytest.raises(ValueError):
        O.field_op("fp", "add", Y.P, 1)


def test_g1_generator_and_order():
    g = O.g1_generator()
    assert O.g1_from(g) == Y.G1
    assert O.g1_on_curve(g)
    assert O.g1_mul(g, O.R) == bytes(64)          # r G = O
    assert O.g1_mul(g, O.R + 1) == g              # (r+1) G = G
    assert O.g1_mul(g, O.R - 1) == O.g1_bytes((1, Y.P - 2))   # -G


def test_g1_add_mul_vs_affine_formulas():
    g = O.g1_generator()
    for _ in range(12):
        a, b = rng.randrange(1, O.R), rng.randrange(1, O.R)
        pa, pb = Y.g1_mul(Y.G1, a), Y.g1_mul(Y.G1, b)
        assert O.g1_from(O.g1_mul(g, a)) == pa
        assert O.g1_from(O.g1_add(O.g1_bytes(pa), O.g1_bytes(pb))) == Y.g1_add(pa, pb)
    # special cases: P + P, P + (-P), P + O
    p = Y.g1_mul(Y.G1, 12345)
    assert O.g1_from(O.g1_add(O.g1_bytes(p), O.g1_bytes(p))) == Y.g1_add(p, p)
    assert O.g1_add(O.g1_bytes(p), O.g1_bytes((p[0], Y.P - p[1]))) == bytes(64)
    assert O.g1_from(O.g1_add(O.g1_bytes(p), bytes(64))) == p


def test_g2_generator_and_order():
    c = json.load(open(os.path.join(GOLD, "bn254_constants.json")))
    g2 = O.g2_generator()
    want = ((int(c["g2_x"][0]), int(c["g2_x"][1])), (int(c["g2_y"][0]), int(c["g2_y"][1])))
    assert O.g2_from(g2) == want == Y.G2
    assert Y.g2_on_curve(Y.G2)
    assert O.g2_on_curve(g2)
    assert O.g2_mul(g2, O.R) == bytes(128)
    assert O.untwist_on_curve(g2)


def test_g2_add_mul_vs_affine_formulas():
    g2 = O.g2_generator()
    for _ in range(4):
        a, b = rng.randrange(1, O.R), rng.randrange(1, O.R)
        pa, pb = Y.g2_mul(Y.G2, a), Y.g2_mul(Y.G2, b)
        assert O.g2_from(O.g2_mul(g2, a)) == pa
        assert O.g2_from(O.g2_add(O.g2_bytes(pa), O.g2_bytes(pb))) == Y.g2_add(pa, pb)
        assert O.untwist_on_curve(O.g2_bytes(pa))
    p = Y.g2_mul(Y.G2, 777)
    assert O.g2_from(O.g2_add(O.g2_bytes(p), O.g2_bytes(p))) == Y.g2_add(p, p)


def test_pairing_bilinear_nondegenerate():
    g1, g2 = O.g1_generator(), O.g2_generator()
    e = O.pairing(g1, g2)
    assert e != O.FP12_ONE                          # non-degenerate
    assert O.fp12_pow(e, O.R) == O.FP12_ONE         # lands in mu_r
    a, b = rng.randrange(2, O.R), rng.randrange(2, O.R)
    eab = O.pairing(O.g1_mul(g1, a), O.g2_mul(g2, b))
    assert eab == O.fp12_pow(e, a * b % O.R)
    # linear in each argument separately
    q1, q2 = O.g2_mul(g2, 5), O.g2_mul(g2, 11)
    assert O.pairing(g1, O.g2_add(q1, q2)) == O.fp12_mul(O.pairing(g1, q1), O.pairing(g1, q2))
    assert O.pairing(bytes(64), g2) == O.FP12_ONE


def test_root_of_unity_orders():
    for k in (1, 5, 10, 20, 28):
        w = O.fr_root_of_unity(k)
        assert w == pow(5, (O.R - 1) >> k, O.R)
        assert pow(w, 1 << k, O.R) == 1
        assert pow(w, 1 << (k - 1), O.R) == O.R - 1   # primitive


@pytest.mark.parametrize("log_n", [1, 2, 3, 5, 6])
def test_ntt_vs_naive_dft(log_n):
    n = 1 << log_n
    vals = [rng.randrange(O.R) for _ in range(n)]
    w = pow(5, (O.R - 1) >> log_n, O.R)
    out = Y.ints_from_bytes(O.ntt(Y.ints_to_bytes(vals), log_n))
    assert out == Y.dft(vals, w)
    back = Y.ints_from_bytes(O.ntt(Y.ints_to_bytes(out), log_n, inverse=True))
    assert back == vals


@pytest.mark.parametrize("log_n", [1, 2, 3, 5])
@pytest.mark.parametrize("g", [5, 7])
def test_coset_ntt_vs_direct_evaluation(log_n, g):
    """Forward coset transform = the polynomial's values at g w^j by Horner;
    inverse = coefficients that Lagrange interpolation through the points
    (g w^j, a_j) reproduces at a random point; inverse after forward = id."""
    n = 1 << log_n
    coeffs = [rng.randrange(O.R) for _ in range(n)]
    w = pow(5, (O.R - 1) >> log_n, O.R)
    ev = Y.ints_from_bytes(O.coset_ntt(Y.ints_to_bytes(coeffs), log_n, g))
    assert ev == [Y.poly_eval(coeffs, g * pow(w, j, O.R) % O.R) for j in range(n)]
    vals = [rng.randrange(O.R) for _ in range(n)]
    cf = Y.ints_from_bytes(O.coset_ntt(Y.ints_to_bytes(vals), log_n, g, inverse=True))
    for j in range(n):
        assert Y.poly_eval(cf, g * pow(w, j, O.R) % O.R) == vals[j]
    # interpolation through the coset points, evaluated off the coset
    rho = rng.randrange(O.R)
    xs = [g * pow(w, j, O.R) % O.R for j in range(n)]
    lag = 0
    for j in range(n):
        num = den = 1
        for k in range(n):
            if k != j:
                num = num * (rho - xs[k]) % O.R
                den = den * (xs[j] - xs[k]) % O.R
        lag = (lag + vals[j] * num * pow(den, -1, O.R)) % O.R
    assert Y.poly_eval(cf, rho) == lag
    assert Y.ints_from_bytes(O.coset_ntt(Y.ints_to_bytes(cf), log_n, g)) == vals


def test_coset_ntt_large_horner_and_roundtrip():
    """At 2^12: random values checked by Horner at g w^j, and the round trip."""
    log_n = 12
    n = 1 << log_n
    coeffs = [rng.randrange(O.R) for _ in range(n)]
    ev = Y.ints_from_bytes(O.coset_ntt(Y.ints_to_bytes(coeffs), log_n))
    w = O.fr_root_of_unity(log_n)
    for j in (0, 1, 999, n - 1):
        assert ev[j] == Y.poly_eval(coeffs, 5 * pow(w, j, O.R) % O.R)
    back = O.coset_ntt(Y.ints_to_bytes(ev), log_n, inverse=True)
    assert Y.ints_from_bytes(back) == coeffs


def test_ntt_roundtrip_and_convolution_large():
    log_n = 12
    n = 1 << log_n
    a = [rng.randrange(O.R) for _ in range(n // 2)] + [0] * (n // 2)
    b = [rng.randrange(O.R) for _ in range(n // 2)] + [0] * (n // 2)
    fa = Y.ints_from_bytes(O.ntt(Y.ints_to_bytes(a), log_n))
    fb = Y.ints_from_bytes(O.ntt(Y.ints_to_bytes(b), log_n))
    prod = Y.ints_from_bytes(O.ntt(Y.ints_to_bytes([x * y % O.R for x, y in zip(fa, fb)]), log_n, True))
    # spot-check coefficients of a*b against schoolbook sums
    for k in (0, 1, 777, n // 2 - 1, n - 2):
        want = sum(a[i] * b[k - i] for i in range(max(0, k - n // 2 + 1), min(k, n // 2 - 1) + 1)) % O.R
        assert prod[k] == want
    # evaluation at random indices by Horner
    w = O.fr_root_of_unity(log_n)
    for i in (3, 1000, n - 1):
        assert fa[i] == Y.poly_eval(a, pow(w, i, O.R))


def test_msm_vs_double_and_add_tiny():
    n = 9
    ks = [rng.randrange(1, O.R) for _ in range(n)]
    pts = [Y.g1_mul(Y.G1, k) for k in ks]
    sc = [rng.randrange(O.R) for _ in range(n)]
    sc[0] = 0
    sc[1] = 1
    want = None
    for s, p in zip(sc, pts):
        want = Y.g1_add(want, Y.g1_mul(p, s))
    pb = b"".join(O.g1_bytes(p) for p in pts)
    sb = Y.ints_to_bytes(sc)
    assert O.g1_from(O.msm_g1(pb, sb, 0)) == want
    assert O.g1_from(O.msm_g1(pb, sb, 1)) == want


def test_msm_g2_vs_double_and_add_tiny():
    n = 4
    pts = [Y.g2_mul(Y.G2, rng.randrange(1, O.R)) for _ in range(n)]
    sc = [rng.randrange(O.R) for _ in range(n)]
    want = None
    for s, p in zip(sc, pts):
        want = Y.g2_add(want, Y.g2_mul(p, s))
    pb = b"".join(O.g2_bytes(p) for p in pts)
    assert O.g2_from(O.msm_g2(pb, Y.ints_to_bytes(sc), 1)) == want
    assert O.g2_from(O.msm_g2(pb, Y.ints_to_bytes(sc), 0)) == want


def test_msm_discrete_log_identity():
    """Bases k_i G give sum s_i (k_i G) = (sum s_i k_i mod r) G."""
    n = 3000
    ks = [rng.randrange(O.R) for _ in range(n)]
    ss = [rng.randrange(O.R) if rng.random() < 0.5 else rng.randrange(2) for _ in range(n)]
    pts = O.g1_mul_gen_batch(Y.ints_to_bytes(ks))
    got = O.msm_g1(pts, Y.ints_to_bytes(ss), 1)
    want = O.g1_mul(O.g1_generator(), sum(a * b for a, b in zip(ks, ss)) % O.R)
    assert got == want
    pts2 = O.g2_mul_gen_batch(Y.ints_to_bytes(ks[:300]))
    got2 = O.msm_g2(pts2, Y.ints_to_bytes(ss[:300]), 1)
    assert got2 == O.g2_mul(O.g2_generator(), sum(a * b for a, b in zip(ks[:300], ss[:300])) % O.R)


def test_splitmix64_published_definition():
    for seed, purpose in ((0, 0), (1234567, 0), (42, 3), (2**64 - 1, 10)):
        g = Y.SplitMix64(seed, purpose)
        assert O.splitmix64(seed, purpose, 1000) == [g.next() for _ in range(1000)]
    g = Y.SplitMix64(7, 4)
    assert Y.ints_from_bytes(O.sample_fr(7, 4, 50)) == [g.fr() for _ in range(50)]


def test_rs_from_seed_is_sampler_stream():
    g = Y.SplitMix64(99, O.PURPOSE["rs"])
    r, s = O.rs_from_seed(99)
    assert O.from32(r) == g.fr() and O.from32(s) == g.fr()
