"""GPU parity of the arithmetic layers against the CPU oracle.

Field and curve operations, fixed-base multiplication, G1/G2 MSMs (every
window size, ragged sizes, degenerate scalars and points) and the NTT family
are compared element by element, bit-exactly, with values computed by the
oracle (or, for large MSMs, by the discrete-log identity from the seeds
alone: bases k_i G give sum s_i k_i G = (sum s_i k_i mod r) G).
"""
import random

import numpy as np
import pytest

import oracle as O
from paper_2603_10242_gb300 import inputs

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace
P, R = gu.P, gu.R
rng = random.Random(1234)


def _field_vals(mod, n):
    edge = [0, 1, 2, mod - 1, mod - 2, (1 << 253) % mod, (1 << 224) - 1, mod >> 1, (1 << 32) - 1]
    return (edge + [rng.randrange(mod) for _ in range(n - len(edge))])[:n]


@pytest.mark.parametrize("field,mod", [(0, P), (1, R)])
def test_field_ops_vs_oracle(field, mod):
    n = 4096
    a = _field_vals(mod, n)
    b = list(reversed(_field_vals(mod, n)))
    da, db = gu.dev(gu.ints_bytes(a)), gu.dev(gu.ints_bytes(b))
    out = gu.empty(32 * n)
    which = "fr" if field else "fp"
    for op, name in ((0, "add"), (1, "sub"), (2, "mul"), (3, None), (4, "inv")):
        ace.debug_field_op(field, op, da, db, out, n)
        got = gu.bytes_ints(gu.host(out))
        # every inverse (the device inversion's path depends on the value)
        for i in range(0, n, 1 if name == "inv" else 7):
            if name == "inv":
                want = O.field_op(which, "inv", a[i]) if a[i] else 0
            elif name is None:
                want = O.field_op(which, "mul", a[i], a[i])
            else:
                want = O.field_op(which, name, a[i], b[i])
            assert got[i] == want, (op, i, a[i], b[i])


def test_fp2_ops_vs_python():
    n = 512
    a = [(rng.randrange(P), rng.randrange(P)) for _ in range(n)]
    b = [(rng.randrange(P), rng.randrange(P)) for _ in range(n)]
    a[0], b[0] = (0, 0), (P - 1, P - 1)
    da = gu.dev(gu.ints_bytes([v for x in a for v in x]))
    db = gu.dev(gu.ints_bytes([v for x in b for v in x]))
    out = gu.empty(64 * n)
    ace.debug_field_op(2, 2, da, db, out, n)
    got = gu.bytes_ints(gu.host(out))
    for i in range(n):
        (a0, a1), (b0, b1) = a[i], b[i]
        assert (got[2 * i], got[2 * i + 1]) == ((a0 * b0 - a1 * b1) % P, (a0 * b1 + a1 * b0) % P)
    ace.debug_field_op(2, 4, da, db, out, n)
    got = gu.bytes_ints(gu.host(out))
    for i in range(1, n):
        a0, a1 = a[i]
        x0, x1 = got[2 * i], got[2 * i + 1]
        assert ((a0 * x0 - a1 * x1) % P, (a0 * x1 + a1 * x0) % P) == (1, 0)


def _rand_g1(k):
    return O.g1_mul_gen_batch(gu.ints_bytes(k))


def test_g1_curve_ops_vs_oracle():
    n = 64
    ka = [rng.randrange(1, R) for _ in range(n)]
    kb = [rng.randrange(1, R) for _ in range(n)]
    kb[1] = ka[1]                    # P + P
    kb[2] = (R - ka[2]) % R          # P + (-P)
    pa, pb = _rand_g1(ka), _rand_g1(kb)
    pb = bytearray(pb)
    pb[64 * 3:64 * 4] = bytes(64)    # P + O
    pb = bytes(pb)
    da, db = gu.dev(pa), gu.dev(pb)
    ks = [rng.randrange(R) for _ in range(n)]
    dk = gu.dev(gu.ints_bytes(ks))
    out = gu.empty(64 * n)
    for op in (0, 1, 2, 3):
        ace.debug_curve_op(1, op, da, db, dk, out, n)
        got = gu.host(out)
        for i in range(n):
            A, B = pa[64 * i:64 * i + 64], pb[64 * i:64 * i + 64]
            if op in (0, 1):
                want = O.g1_add(A, B)
            elif op == 2:
                want = O.g1_add(A, A)
            else:
                want = O.g1_mul(A, ks[i])
            assert got[64 * i:64 * i + 64] == want, (op, i)


def test_g2_curve_ops_vs_oracle():
    n = 16
    ka = [rng.randrange(1, R) for _ in range(n)]
    kb = [rng.randrange(1, R) for _ in range(n)]
    kb[1] = ka[1]
    kb[2] = (R - ka[2]) % R
    pa = O.g2_mul_gen_batch(gu.ints_bytes(ka))
    pb = O.g2_mul_gen_batch(gu.ints_bytes(kb))
    ks = [rng.randrange(R) for _ in range(n)]
    da, db, dk = gu.dev(pa), gu.dev(pb), gu.dev(gu.ints_bytes(ks))
    out = gu.empty(128 * n)
    for op in (0, 1, 2, 3):
        ace.debug_curve_op(2, op, da, db, dk, out, n)
        got = gu.host(out)
        for i in range(n):
            A, B = pa[128 * i:128 * i + 128], pb[128 * i:128 * i + 128]
            want = (O.g2_add(A, B) if op in (0, 1) else O.g2_add(A, A) if op == 2 else O.g2_mul(A, ks[i]))
            assert got[128 * i:128 * i + 128] == want, (op, i)


def test_fixed_base_vs_oracle():
    c = gu.ctx()
    ks = [0, 1, 2, R - 1] + [rng.randrange(R) for _ in range(1000)]
    n = len(ks)
    dk = gu.dev(gu.ints_bytes(ks))
    out = gu.empty(64 * n)
    c.g1_fixed_base(dk, n, out)
    assert gu.host(out) == O.g1_mul_gen_batch(gu.ints_bytes(ks))
    ks2 = ks[:100]
    out2 = gu.empty(128 * 100)
    c.g2_fixed_base(gu.dev(gu.ints_bytes(ks2)), 100, out2)
    assert gu.host(out2) == O.g2_mul_gen_batch(gu.ints_bytes(ks2))


def _msm_expected_dlog(ks, ss):
    return O.g1_mul(O.g1_generator(), sum(a * b for a, b in zip(ks, ss)) % R)


@pytest.mark.parametrize("n", [0, 1, 2, 7, 100, 1000, 4097])
@pytest.mark.parametrize("dist", ["uniform", "sparse"])
def test_msm_g1_small_vs_oracle(n, dist):
    c = gu.ctx()
    ks = [rng.randrange(1, R) for _ in range(n)]
    pts = _rand_g1(ks) if n else b""
    ss = inputs.limbs_to_int(inputs.sample_scalars(1000 + n, n, dist)) if n else []
    out = gu.empty(64)
    c.msm_g1(gu.dev(pts), gu.dev(gu.ints_bytes(ss)), n, out, ace.FORM_CANONICAL)
    want = O.msm_g1(pts, gu.ints_bytes(ss), 1) if n else bytes(64)
    assert gu.host(out) == want


def test_msm_g1_montgomery_bases_and_degenerate():
    c = gu.ctx()
    n = 3000
    ks = [rng.randrange(1, R) for _ in range(n)]
    pts = _rand_g1(ks)
    ss = [rng.randrange(R) for _ in range(n)]
    ss[:10] = [0, 1, R - 1, 2, 2, 2, 1, 1, 0, R - 2]
    out = gu.empty(64)
    c.msm_g1(gu.dev(gu.to_mont_g1_bytes(pts)), gu.dev(gu.ints_bytes(ss)), n, out, ace.FORM_MONT)
    assert gu.host(out) == _msm_expected_dlog(ks, ss)
    # same base everywhere (buckets see P + P), and P next to -P with equal scalars
    g = O.g1_generator()
    same = g * n
    c.msm_g1(gu.dev(same), gu.dev(gu.ints_bytes(ss)), n, out, ace.FORM_CANONICAL)
    assert gu.host(out) == O.g1_mul(g, sum(ss) % R)
    neg = O.g1_mul(g, R - 1)
    pm = (g + neg) * (n // 2)
    s2 = [v for v in ss[: n // 2] for _ in (0, 1)]
    c.msm_g1(gu.dev(pm), gu.dev(gu.ints_bytes(s2)), len(s2), out, ace.FORM_CANONICAL)
    assert gu.host(out) == bytes(64)
    # all scalars zero / all one / points at infinity
    c.msm_g1(gu.dev(pts), gu.dev(bytes(32 * n)), n, out)
    assert gu.host(out) == bytes(64)
    c.msm_g1(gu.dev(pts), gu.dev(gu.ints_bytes([1] * n)), n, out)
    assert gu.host(out) == _msm_expected_dlog(ks, [1] * n)
    pinf = bytearray(pts)
    pinf[0:64 * 50] = bytes(64 * 50)
    c.msm_g1(gu.dev(bytes(pinf)), gu.dev(gu.ints_bytes(ss)), n, out)
    assert gu.host(out) == _msm_expected_dlog([0] * 50 + ks[50:], ss)


@pytest.mark.parametrize("c_bits", [6, 9, 13, 16, 20])
def test_msm_g1_every_window(c_bits):
    c = gu.ctx()
    n = 5000
    ks = [rng.randrange(1, R) for _ in range(n)]
    pts = _rand_g1(ks)
    ss = inputs.limbs_to_int(inputs.sample_scalars(77, n, "sparse"))
    out = gu.empty(64)
    c.msm_g1_window(gu.dev(pts), gu.dev(gu.ints_bytes(ss)), n, c_bits, out, ace.FORM_CANONICAL)
    assert gu.host(out) == _msm_expected_dlog(ks, ss)


LAMBDA = 0xb3c4d79d41a917585bfc41088d8daaa78b17ea66b99c90dd  # cube root of unity mod r


@pytest.mark.parametrize("c_bits", [6, 7, 9, 11, 13, 16, 17, 20])
def test_msm_g1_glv_every_window(c_bits):
    """The GLV form of the G1 MSM (k = k1 + k2 lambda, 128-bit halves over P
    and phi(P)) at every window size: ceil(128 / c) windows, the top one
    short."""
    c = gu.ctx()
    n = 3001
    ks = [rng.randrange(1, R) for _ in range(n)]
    pts = _rand_g1(ks)
    ss = inputs.limbs_to_int(inputs.sample_scalars(90 + c_bits, n, "sparse" if c_bits % 2 else "uniform"))
    out = gu.empty(64)
    c.msm_g1_glv_window(gu.dev(pts), gu.dev(gu.ints_bytes(ss)), n, c_bits, out, ace.FORM_CANONICAL)
    assert gu.host(out) == _msm_expected_dlog(ks, ss)


def test_msm_g1_glv_edge_scalars_and_points():
    """Scalars whose halves are negative or extreme (r - 1, lambda, lambda^2,
    (r - 1) / 2), scalars at or above r (taken modulo r, up to 2^256 - 1),
    zeros and ones, and points at infinity."""
    c = gu.ctx()
    edge = [0, 1, 2, R - 1, R - 2, LAMBDA, LAMBDA * LAMBDA % R, (R - 1) // 2, (R + 1) // 2, 1 << 127,
            (1 << 128) - 1, 1 << 253, R, R + 1, 2 * R + 5, (1 << 255) + 3, (1 << 256) - 1]
    n = 600
    ss = (edge * (n // len(edge) + 1))[:n]
    for i in range(len(edge), n, 3):
        ss[i] = rng.randrange(R)
    ks = [rng.randrange(1, R) for _ in range(n)]
    pts = bytearray(_rand_g1(ks))
    for i in range(0, n, 37):  # points at infinity
        pts[64 * i:64 * i + 64] = bytes(64)
        ks[i] = 0
    out = gu.empty(64)
    c.msm_g1(gu.dev(bytes(pts)), gu.dev(gu.ints_bytes(ss)), n, out, ace.FORM_CANONICAL)
    assert gu.host(out) == _msm_expected_dlog(ks, ss)
    for cb in (8, 16):
        c.msm_g1_glv_window(gu.dev(bytes(pts)), gu.dev(gu.ints_bytes(ss)), n, cb, out, ace.FORM_CANONICAL)
        assert gu.host(out) == _msm_expected_dlog(ks, ss)


@pytest.mark.parametrize("log_n,dist", [(16, "uniform"), (18, "sparse"), (20, "uniform"), (20, "sparse"),
                                        (22, "sparse"), (24, "uniform")])
def test_msm_g1_large_dlog(log_n, dist):
    """Bases from the fixed-base kernel; expected value from the seeds alone.
    The sizes span the G1 MSM sweep (2^16 to 2^24 points) in both scalar
    distributions, three points short of each power of two (a ragged tail)."""
    c = gu.ctx()
    n = (1 << log_n) - 3
    kb = inputs.sample_fr(log_n, inputs.PURPOSE["bases"], n)
    sc = inputs.sample_scalars(log_n, n, dist)
    bases = gu.empty(64 * n)
    c.g1_fixed_base(gu.dev(kb), n, bases, ace.FORM_MONT)
    out = gu.empty(64)
    c.msm_g1(bases, gu.dev(sc), n, out, ace.FORM_MONT)
    ks, ss = inputs.limbs_to_int(kb), inputs.limbs_to_int(sc)
    assert gu.host(out) == _msm_expected_dlog(ks, ss)
    # spot-check the fixed-base output itself
    got = gu.host(bases)
    for i in (0, 1, n // 2, n - 1):
        want = O.g1_mul(O.g1_generator(), ks[i])
        xy = gu.bytes_ints(got[64 * i:64 * i + 64])
        rinv = pow(gu.RMONT, -1, P)
        assert gu.ints_bytes([v * rinv % P for v in xy]) == want


@pytest.mark.parametrize("n", [1, 5, 300, 2049])
def test_msm_g2_vs_oracle(n):
    c = gu.ctx()
    ks = [rng.randrange(1, R) for _ in range(n)]
    pts = O.g2_mul_gen_batch(gu.ints_bytes(ks))
    ss = inputs.limbs_to_int(inputs.sample_scalars(500 + n, n, "sparse" if n % 2 else "uniform"))
    out = gu.empty(128)
    c.msm_g2(gu.dev(pts), gu.dev(gu.ints_bytes(ss)), n, out, ace.FORM_CANONICAL)
    want = O.g2_mul(O.g2_generator(), sum(a * b for a, b in zip(ks, ss)) % R)
    assert gu.host(out) == want
    if n <= 300:
        assert want == O.msm_g2(pts, gu.ints_bytes(ss), 1)


def test_msm_g2_large_dlog():
    c = gu.ctx()
    n = (1 << 16) + 5
    kb = inputs.sample_fr(3, inputs.PURPOSE["bases"], n)
    sc = inputs.sample_scalars(3, n, "uniform")
    bases = gu.empty(128 * n)
    c.g2_fixed_base(gu.dev(kb), n, bases, ace.FORM_MONT)
    out = gu.empty(128)
    c.msm_g2(bases, gu.dev(sc), n, out, ace.FORM_MONT)
    s = sum(a * b for a, b in zip(inputs.limbs_to_int(kb), inputs.limbs_to_int(sc))) % R
    assert gu.host(out) == O.g2_mul(O.g2_generator(), s)


def test_msm_g2_sparse_dlog():
    """G2 MSM with 70% {0,1} scalars (its {0,1} window and the four-lane
    Horner over Fp2), Montgomery bases, a ragged size."""
    c = gu.ctx()
    n = (1 << 15) + 11
    kb = inputs.sample_fr(4, inputs.PURPOSE["bases"], n)
    sc = inputs.sample_scalars(4, n, "sparse")
    bases = gu.empty(128 * n)
    c.g2_fixed_base(gu.dev(kb), n, bases, ace.FORM_MONT)
    out = gu.empty(128)
    c.msm_g2(bases, gu.dev(sc), n, out, ace.FORM_MONT)
    s = sum(a * b for a, b in zip(inputs.limbs_to_int(kb), inputs.limbs_to_int(sc))) % R
    assert gu.host(out) == O.g2_mul(O.g2_generator(), s)


@pytest.mark.parametrize("n,c,dist", [(1, 6, "uniform"), (7, 9, "sparse"), (333, 11, "uniform"),
                                      (1 << 12, 13, "sparse"), ((1 << 14) + 3, 17, "uniform"),
                                      ((1 << 15) - 1, 20, "uniform")])
def test_msm_g2_psi_split_windows(n, c, dist):
    """The G2 MSM over the four-way psi split (points psi^t(Q_i), parts below
    2^66) with forced windows, every digit kernel width from the smallest to
    the largest, ragged sizes and both scalar distributions, against the
    discrete-log sum computed on the host; canonical scalars >= r (reduced
    mod r first) included."""
    cx = gu.ctx()
    kb = inputs.sample_fr(40 + c, inputs.PURPOSE["bases"], n)
    sc = inputs.sample_scalars(60 + c, n, dist)
    ss = inputs.limbs_to_int(sc)
    if n >= 7:
        ss[3] = ss[3] + R if ss[3] + R < 1 << 256 else ss[3]  # a scalar above r
        ss[5] = 0
        ss[6] = R - 1
    bases = gu.empty(128 * n)
    cx.g2_fixed_base(gu.dev(kb), n, bases, ace.FORM_MONT)
    out = gu.empty(128)
    cx.msm_g2_gls_window(bases, gu.dev(gu.ints_bytes(ss)), n, c, out, ace.FORM_MONT)
    s = sum(a * b for a, b in zip(inputs.limbs_to_int(kb), ss)) % R
    assert gu.host(out) == O.g2_mul(O.g2_generator(), s)


NTT_KINDS = {0: "ntt", 1: "intt", 2: "coset_ntt", 3: "coset_intt"}


def _oracle_transform(raw, log_n, kind):
    if kind in (0, 1):
        return O.ntt(raw, log_n, inverse=(kind == 1))
    return O.coset_ntt(raw, log_n, 5, inverse=(kind == 3))


@pytest.mark.parametrize("kind", sorted(NTT_KINDS))
@pytest.mark.parametrize("log_n", [1, 2, 5, 10, 11, 12, 16, 20, 22, 23, 24])
def test_ntt_kinds_vs_oracle(log_n, kind):
    """Every transform kind (NTT, inverse NTT, coset NTT and coset inverse NTT
    on g H with g = 5) against the oracle, every element, from one pass up to
    the multi-pass plans of 2^20..2^24 (the top of the transform sweep)."""
    c = gu.ctx()
    n = 1 << log_n
    raw = inputs.sample_fr(log_n, 7, n).tobytes()
    d = gu.dev(raw)
    c.ntt(d, log_n, kind)
    got = gu.host(d)
    want = _oracle_transform(raw, log_n, kind)
    assert got == want, NTT_KINDS[kind]


def test_ntt_mont_roundtrip_batch():
    """DIF forward then DIT inverse over several arrays returns N x input."""
    c = gu.ctx()
    for log_n in (3, 11, 14, 22):
        n = 1 << log_n
        vals = inputs.sample_fr(100 + log_n, 7, 3 * n)
        d = gu.dev(vals)
        c.ntt_mont(d, log_n, 3, True, False)
        c.ntt_mont(d, log_n, 3, False, True)
        got = np.frombuffer(gu.host(d), dtype=np.uint32).reshape(-1, 8)
        # values are treated as Montgomery residues: result is N * x (mod r) in that form
        for i in (0, 1, n - 1, n, 2 * n + 5, 3 * n - 1):
            x = inputs.limbs_to_int(vals[i:i + 1])[0]
            assert inputs.limbs_to_int(got[i:i + 1])[0] == x * n % R
