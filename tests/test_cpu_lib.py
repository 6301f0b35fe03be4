"""CPU-side checks of the library: it builds, loads and exports every symbol
of include/ace.h; its host logic (circuit generator, witness, prover
randomness, Groth16 verifier) matches the oracle; the shared input
generators follow the published SplitMix64 definition.  No GPU calls.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import pyref as Y
import paper_2603_10242_gb300 as ace
from paper_2603_10242_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ace.build()
    return ace.lib()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|const char\*)\s+(ace_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_sampler_matches_published_definition():
    g = Y.SplitMix64(5, 7)
    assert inputs.limbs_to_int(inputs.sample_fr(5, 7, 500)) == [g.fr() for _ in range(500)]
    assert [int(x) for x in inputs.splitmix64(9, 3, 100)] == O.splitmix64(9, 3, 100)
    sp = inputs.limbs_to_int(inputs.sample_scalars(11, 20000, "sparse"))
    frac = sum(1 for v in sp if v in (0, 1)) / len(sp)
    assert 0.68 < frac < 0.72
    sel = Y.SplitMix64(11, inputs.PURPOSE["selector"])
    uni = Y.SplitMix64(11, inputs.PURPOSE["scalars"])
    for i in range(300):
        u = sel.next()
        want = (u >> 63) if u % 10 < 7 else uni.fr()
        assert sp[i] == want


@pytest.mark.parametrize("params", [(2, 4, 0, 0, 0), (3, 6, 0, 1, 3), (10, 1024, 4, 0, 0), (12, 4000, 8, 8, 172)])
def test_host_circuit_and_witness_match_oracle(lib, params):
    lc = ace.Circuit(*params, seed=4)
    oc = O.Circuit(*params, seed=4, input_seed=6)
    assert (lc.N, lc.m) == (oc.N, oc.m)
    assert lc.info[4:7] == [oc.nnz_a, oc.nnz_b, oc.nnz_c]
    assert lc.witness(6) == oc.witness()


def test_circuit_parameter_errors(lib):
    with pytest.raises(ace.AceError):
        ace.Circuit(10, 1024, 5, 0, 0)        # 5 permutations need more than 1024 rows
    with pytest.raises(ace.AceError):
        ace.Circuit(1, 2, 0, 0, 0)            # domain too small
    with pytest.raises(ace.AceError):
        ace.Circuit(10, 2000, 0, 0, 0)        # n_rows > N


def test_rs_from_seed_matches_oracle(lib):
    for seed in (0, 1, 12345):
        assert ace.rs_from_seed(seed) == O.rs_from_seed(seed)


def _vk_from_oracle(opk):
    vk = ace.VerifyingKey()
    raw = (opk.point("fixed", 0) + opk.point("fixed", 3) + opk.point("fixed", 4) + opk.point("fixed", 5)
           + opk.point("fixed", 6) + opk.point("fixed", 7))
    ctypes.memmove(ctypes.byref(vk), raw, len(raw))
    return vk


def test_host_verifier_accepts_oracle_proofs_and_rejects_forgeries(lib):
    oc = O.Circuit(10, 1024, 4, 0, 0, seed=1, input_seed=1)
    opk = O.ProvingKey(oc, 1, with_points=True)
    z = oc.witness()
    r, s = O.rs_from_seed(1)
    ok, proof = opk.prove(z, r, s)
    assert ok
    vk = _vk_from_oracle(opk)
    pub = z[32:64]
    assert ace.verify(vk, pub, proof) == 1
    wrong_pub = ((int.from_bytes(pub, "little") + 1) % Y.R).to_bytes(32, "little")
    assert ace.verify(vk, wrong_pub, proof) == 0
    swapped = proof[192:256] + proof[64:192] + proof[0:64]
    assert ace.verify(vk, pub, swapped) == 0
    bad = bytearray(proof)
    bad[3] ^= 1
    with pytest.raises(ace.AceError) as e:
        ace.verify(vk, pub, bytes(bad))
    assert e.value.code == -5
    # a proof for another witness of the same circuit also verifies (with its own public input)
    oc2 = O.Circuit(10, 1024, 4, 0, 0, seed=1, input_seed=2)
    z2 = oc2.witness()
    ok, proof2 = opk.prove(z2, r, s)
    assert ace.verify(vk, z2[32:64], proof2) == 1
    assert ace.verify(vk, pub, proof2) == 0


def test_host_pairing_bilinear(lib):
    f = lib.ace_debug_pairing
    f.restype = ctypes.c_int
    g1, g2 = O.g1_generator(), O.g2_generator()

    def e(p, q):
        out = ctypes.create_string_buffer(384)
        assert f(p, q, out) == 0
        return out.raw

    one = Y.ints_to_bytes([1] + [0] * 11)
    base = e(g1, g2)
    assert base != one
    a, b = 987654321987654321, 1234567
    lhs = e(O.g1_mul(g1, a), O.g2_mul(g2, b))
    assert lhs == e(O.g1_mul(g1, a * b % Y.R), g2) == e(g1, O.g2_mul(g2, a * b % Y.R))
    assert e(O.g1_mul(g1, Y.R - 1), g2) != base


def test_projective_miller_loop_matches_affine(lib):
    """The batch verifier's projective Miller loop (run here on the host) and
    the single verifier's affine one give the same pairing values."""
    import random
    f = lib.ace_debug_pairing_form
    f.restype = ctypes.c_int
    rng = random.Random(5)
    g1, g2 = O.g1_generator(), O.g2_generator()
    for _ in range(3):
        P = O.g1_mul(g1, rng.randrange(1, Y.R))
        Q = O.g2_mul(g2, rng.randrange(1, Y.R))
        a, b, c = (ctypes.create_string_buffer(384) for _ in range(3))
        assert f(0, P, Q, a) == 0 and f(1, P, Q, b) == 0 and f(2, P, Q, c) == 0
        assert a.raw == b.raw == c.raw
    # bilinearity through the projective loop: e(2P, Q) = e(P, 2Q)
    P, Q = O.g1_mul(g1, 77), O.g2_mul(g2, 99)
    a, b = ctypes.create_string_buffer(384), ctypes.create_string_buffer(384)
    assert f(1, O.g1_mul(P, 2), Q, a) == 0 and f(1, P, O.g2_mul(Q, 2), b) == 0
    assert a.raw == b.raw


def test_glv_split(lib):
    """k = k1 + k2 lambda (mod r) with |k1|, |k2| < 2^128, and (beta x, y) =
    lambda (x, y) on G1 for the constants the prover's split assumes."""
    import random
    lam = 0xb3c4d79d41a917585bfc41088d8daaa78b17ea66b99c90dd
    beta = 0x59e26bcea0d48bacd4f263f1acdb5c4f5763473177fffffe
    assert pow(lam, 3, Y.R) == 1 and lam != 1
    assert pow(beta, 3, Y.P) == 1 and beta != 1
    g = Y.g1_mul(Y.G1, 12345)
    assert Y.g1_mul(g, lam) == ((beta * g[0]) % Y.P, g[1])
    f = lib.ace_debug_glv_split
    f.restype = ctypes.c_int
    rng = random.Random(9)
    for k in [0, 1, 2, Y.R - 1, Y.R // 2, lam, (1 << 253) + 17] + [rng.randrange(Y.R) for _ in range(200)]:
        out = (ctypes.c_uint32 * 10)()
        assert f(k.to_bytes(32, "little"), out) == 0
        k1 = sum(out[i] << (32 * i) for i in range(4)) * (-1 if out[4] else 1)
        k2 = sum(out[5 + i] << (32 * i) for i in range(4)) * (-1 if out[9] else 1)
        assert abs(k1) < 1 << 128 and abs(k2) < 1 << 128
        assert (k1 + k2 * lam - k) % Y.R == 0


def _gls_constants():
    """gx, gy of the psi map as written in glv.cuh (two Fp coefficients each)."""
    text = open(os.path.join(os.path.dirname(__file__), "..", "paper_2603_10242_gb300", "csrc", "glv.cuh")).read()
    vals = {}
    for name in ("GX0", "GX1", "GY0", "GY1"):
        m = re.search(r"#define ACE_GLS_%s \{([^}]*)\}" % name, text)
        limbs = [int(w.strip().rstrip("u"), 16) for w in m.group(1).split(",")]
        vals[name] = sum(v << (32 * i) for i, v in enumerate(limbs))
    return (vals["GX0"], vals["GX1"]), (vals["GY0"], vals["GY1"])


def test_gls_psi_constants():
    """The constants the G2 MSM's psi uses satisfy their definitions and make
    psi(x, y) = (conj(x) gx, conj(y) gy) the multiplication by lambda = 6 x^2
    on G2 points, the identity the split relies on."""
    x = 4965661367192848881
    assert 36 * x**4 + 36 * x**3 + 18 * x**2 + 6 * x + 1 == Y.R
    assert 36 * x**4 + 36 * x**3 + 24 * x**2 + 6 * x + 1 == Y.P
    gx, gy = _gls_constants()

    def f2_pow(a, e):
        r = (1, 0)
        while e:
            if e & 1:
                r = Y.f2_mul(r, a)
            a = Y.f2_mul(a, a)
            e >>= 1
        return r

    assert gx == f2_pow((9, 1), (Y.P - 1) // 3) and gy == f2_pow((9, 1), (Y.P - 1) // 2)
    lam = 6 * x * x
    for k in (1, 7, 123456789, Y.R - 2):
        q = Y.g2_mul(Y.G2, k)
        conj = lambda a: (a[0], (-a[1]) % Y.P)
        psi = (Y.f2_mul(conj(q[0]), gx), Y.f2_mul(conj(q[1]), gy))
        assert Y.g2_on_curve(psi) and psi == Y.g2_mul(q, lam)


def test_gls_split(lib):
    """k = k0 + k1 lambda + k2 lambda^2 + k3 lambda^3 (mod r) with every
    |k_i| < 2^66, the bound the G2 plan's 67-bit digit windows assume."""
    import random
    x = 4965661367192848881
    lam = 6 * x * x
    f = lib.ace_debug_gls_split
    f.restype = ctypes.c_int
    rng = random.Random(13)
    worst = 0
    ks = [0, 1, 2, Y.R - 1, Y.R // 2, lam, lam * lam % Y.R, x, (1 << 253) + 5]
    for k in ks + [rng.randrange(Y.R) for _ in range(400)]:
        out = (ctypes.c_uint32 * 16)()
        assert f(k.to_bytes(32, "little"), out) == 0
        parts = []
        for i in range(4):
            mag = out[4 * i] | (out[4 * i + 1] << 32) | (out[4 * i + 2] << 64)
            parts.append(-mag if out[4 * i + 3] else mag)
        assert all(abs(v) < 1 << 66 for v in parts)
        assert sum(v * pow(lam, i, Y.R) for i, v in enumerate(parts)) % Y.R == k
        worst = max(worst, max(abs(v) for v in parts))
    assert worst.bit_length() <= 66
    assert f((Y.R).to_bytes(32, "little"), (ctypes.c_uint32 * 16)()) != 0


def test_wnaf5_digits(lib):
    """The width-5 NAF of the variable-base term's 128-bit GLV halves: the
    digits rebuild k, each is 0 or odd with |d| <= 15, and no five
    consecutive digits hold two non-zero ones (so the chain adds about
    once in six doublings)."""
    import random
    f = lib.ace_debug_wnaf5
    f.restype = ctypes.c_int
    rng = random.Random(11)
    ks = [0, 1, 15, 16, 17, 31, 32, (1 << 128) - 1, 1 << 127, (1 << 127) - 1, 0x5555 << 100]
    ks += [rng.getrandbits(128) for _ in range(300)]
    nonzero = 0
    for k in ks:
        words = (ctypes.c_uint32 * 4)(*[(k >> (32 * i)) & 0xFFFFFFFF for i in range(4)])
        out = (ctypes.c_int8 * 132)()
        assert f(words, out) == 0
        d = list(out)
        assert sum(x << i for i, x in enumerate(d)) == k
        assert all(x == 0 or (x % 2 == 1 and -15 <= x <= 15) for x in d)
        nz = [i for i, x in enumerate(d) if x]
        assert all(b - a >= 5 for a, b in zip(nz, nz[1:]))
        assert not nz or nz[-1] <= 128
        nonzero += len(nz)
    # random 128-bit values: about 128 / 6 non-zero digits each
    assert 18 < nonzero / len(ks) < 25


# window choices measured on the GB300 (G1 MSM sweep, block-proof keys)
MEASURED_PLANS = [
    (1 << 16, ace.MSM_GLV, 16), (1 << 20, ace.MSM_GLV, 16), (1 << 24, ace.MSM_GLV, 19),
    (1 << 16, ace.MSM_FULL, 15), (1 << 20, ace.MSM_FULL, 16),
    ((1 << 20) - 1, ace.MSM_TABLED, 17), (712705, ace.MSM_TABLED, 17), (1748994, ace.MSM_TABLED, 20),
]


@pytest.mark.parametrize("n,kind,c", MEASURED_PLANS)
def test_msm_plan_pinned_choices(lib, n, kind, c):
    assert ace.msm_plan(n, kind)["c"] == c


@pytest.mark.parametrize("kind", [ace.MSM_FULL, ace.MSM_TABLED, ace.MSM_GLV, ace.MSM_GLS])
def test_msm_plan_invariants(lib, kind):
    """Digit windows cover the scalar bits with no carry out of the top
    window (254-bit scalars: c K >= 255; GLV halves below 2^127: c K >= 128;
    the parts of the G2 split below 2^66: c K >= 67), the GLV plan runs 2n
    points with about half the windows and the G2 split 4n points, segments
    tile the buckets, and the {0,1} window's virtual buckets stay within B."""
    bits = {ace.MSM_GLV: 128, ace.MSM_GLS: 67}.get(kind, 255)
    mult = {ace.MSM_GLV: 2, ace.MSM_GLS: 4}.get(kind, 1)
    for lg in range(4, 26):
        for n in (1 << lg, (1 << lg) - 3, 3 * (1 << lg) // 2):
            for force in (0, 6, 11, 20):
                p = ace.msm_plan(n, kind, force)
                c, K = p["c"], p["K"]
                if force:
                    assert c == force
                else:
                    assert (8 if kind == ace.MSM_TABLED else 6) <= c <= 20
                assert K == -(-bits // c) and c * K >= bits and c * (K - 1) < bits
                # top window: bits - 1 - c (K - 1) value bits, at most c - 1
                assert bits - 1 - c * (K - 1) <= c - 1
                assert p["B"] == 1 << (c - 1) and p["L"] * p["M"] == p["B"]
                assert p["windows"] == (2 if kind == ace.MSM_TABLED else K + 1)
                ob = p["ones_buckets"]
                assert ob & (ob - 1) == 0 and 1 <= ob <= p["B"]
                assert p["points"] == (mult * n) & 0xFFFFFFFF
    with pytest.raises(ace.AceError):
        ace.msm_plan(1000, kind, 5)
    with pytest.raises(ace.AceError):
        ace.msm_plan(1000, 7)


def test_msm_plan_segment_length(lib):
    """Segments of 4 buckets for single MSMs whose windows hold at most 2^13
    buckets (c <= 14), 16 above."""
    for kind in (ace.MSM_FULL, ace.MSM_TABLED, ace.MSM_GLV):
        for c in range(8, 21):
            p = ace.msm_plan(1 << 16, kind, c)
            assert p["L"] == (4 if c <= 14 else 16), (kind, c)


def test_new_entry_points_reject_bad_arguments_without_a_gpu(lib):
    """Argument checks that return before any CUDA call: NULL context or
    arrays, empty batches."""
    L = lib
    vp = ctypes.c_void_p
    assert L.ace_debug_serial_proofs(None, 1) == -1
    assert L.ace_prove_batch_host(None, 1, None, None, None, None, None, None) == -1
    assert L.ace_prove_batch(None, 1, None, None, None, None, None, None) == -1
    assert L.ace_autotune_batch_slots(None, None, None, 1, 1, None) == -1
    assert "NULL" in L.ace_last_error().decode() or "bad argument" in L.ace_last_error().decode()
    assert ace.ERRORS[-8] == "ACE_E_INTERNAL"
    # the G2 split's window diagnostic: NULL context, window out of range,
    # too many points, unknown base form (all before any CUDA call)
    out = ctypes.create_string_buffer(128)
    f = L.ace_msm_g2_gls_window
    assert f(None, vp(1), 1, vp(1), 4, 11, out, None) == -1
    assert f(vp(1), vp(1), 1, vp(1), 4, 5, out, None) == -1
    assert f(vp(1), vp(1), 1, vp(1), 4, 21, out, None) == -1
    assert f(vp(1), vp(1), 1, vp(1), 1 << 29, 11, out, None) == -1
    assert f(vp(1), vp(1), 7, vp(1), 4, 11, out, None) == -1
    assert "ace_msm_g2_gls_window" in L.ace_last_error().decode()
    assert L.ace_debug_gls_split(None, None) == -1
    assert L.ace_debug_wnaf5(None, None) == -1
    assert L.ace_debug_msm_plan(16, 4, 0, (ctypes.c_uint32 * 8)()) == -1
