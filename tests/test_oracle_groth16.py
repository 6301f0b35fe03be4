"""Pins for the oracle's circuit, QAP and Groth16 paths.

The witness is re-derived here from the Poseidon-style permutation written
over Python integers; the QAP quotient is pinned by the polynomial identity
A(rho)B(rho) - C(rho) = h(rho)(rho^N - 1) at a random rho, with A, B, C
evaluated by Lagrange interpolation (no NTT); proofs are pinned by the pairing
equation and by the in-the-exponent proof, which needs no NTT and no MSM.
"""
import json
import os
import random

import pytest

import oracle as O
import pyref as Y

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SHAPES = json.load(open(os.path.join(GOLD, "circuit_shapes.json")))
rng = random.Random(7)


@pytest.fixture(scope="module")
def c10():
    s = SHAPES["single_proof_2p10"]
    return O.Circuit(s["log_n"], s["n_rows"], s["n_perm"], s["n_pack"], s["pack_bits"],
                     seed=1, input_seed=1)


def test_shapes_single_proof(c10):
    s = SHAPES["single_proof_2p10"]
    assert O.rows_per_perm() == SHAPES["rows_per_permutation"] == (8 * 3 + 57) * 3
    assert (c10.N, c10.m, c10.n_chain) == (1 << s["log_n"], s["m"], s["n_chain"])
    assert 4 * 243 + 2 + c10.n_chain == 1024


def _poseidon(inputs, rc, mds):
    lanes = list(inputs)
    sboxes = []
    for r in range(65):
        full = r < 4 or r >= 61
        lanes = [(lanes[l] + rc[r][l]) % Y.R for l in range(3)]
        for l in range(3 if full else 1):
            s = lanes[l]
            x2 = s * s % Y.R
            x4 = x2 * x2 % Y.R
            x5 = x4 * s % Y.R
            sboxes.append((x2, x4, x5))
            lanes[l] = x5
        lanes = [sum(mds[i][j] * lanes[j] for j in range(3)) % Y.R for i in range(3)]
    return lanes, sboxes


def test_witness_follows_permutation_and_chain(c10):
    z = Y.ints_from_bytes(c10.witness())
    rc, mds = c10.constants()
    # the MDS matrix is Cauchy: every square submatrix is non-singular
    for i in range(3):
        for j in range(3):
            assert mds[i][j] != 0
    for (i0, i1) in ((0, 1), (0, 2), (1, 2)):
        for (j0, j1) in ((0, 1), (0, 2), (1, 2)):
            assert (mds[i0][j0] * mds[i1][j1] - mds[i0][j1] * mds[i1][j0]) % Y.R
    det = (mds[0][0] * (mds[1][1] * mds[2][2] - mds[1][2] * mds[2][1])
           - mds[0][1] * (mds[1][0] * mds[2][2] - mds[1][2] * mds[2][0])
           + mds[0][2] * (mds[1][0] * mds[2][1] - mds[1][1] * mds[2][0])) % Y.R
    assert det
    # inputs drawn from the seeded sampler, in order
    g = Y.SplitMix64(1, O.PURPOSE["inputs"])
    pos = 2
    last = None
    for p in range(4):
        ins = [g.fr() for _ in range(3)]
        assert z[pos:pos + 3] == ins
        pos += 3
        out, sboxes = _poseidon(ins, rc, mds)
        for (x2, x4, x5) in sboxes:
            assert z[pos:pos + 3] == [x2, x4, x5]
            pos += 3
        last = out[0]
    # chain x_{i+1} = x_i^2 + k_i from the last permutation's lane 0
    gk = Y.SplitMix64(1, O.PURPOSE["chain"])
    x = last
    for i in range(c10.n_chain):
        x = (x * x + gk.fr()) % Y.R
        if i + 1 < c10.n_chain:
            assert z[pos] == x
            pos += 1
    assert z[1] == x and z[0] == 1 and pos == c10.m


def test_r1cs_rows(c10):
    z = c10.witness()
    assert c10.r1cs_check(z)
    # input-consistency rows for z_0 and z_1, then nothing
    assert c10.row(0, 1022) == [(0, 1)] and c10.row(0, 1023) == [(1, 1)]
    assert c10.row(1, 1023) == [] and c10.row(2, 1023) == []
    # first S-box row: s * s = x2 with s = input lane 0 + rc[0][0]
    rc, _ = c10.constants()
    assert c10.row(0, 0) == [(0, rc[0][0]), (2, 1)]
    assert c10.row(2, 0) == [(5, 1)]
    bad = bytearray(z)
    bad[32 * 7] ^= 1
    assert not c10.r1cs_check(bytes(bad))


def test_qap_identity_at_random_point(c10):
    z = c10.witness()
    ok, h = c10.qap_h(z)
    assert ok
    hv = Y.ints_from_bytes(h)
    assert hv[-1] == 0                               # deg h <= N - 2
    a, b, c = (Y.ints_from_bytes(v) for v in c10.spmv(z))
    w = pow(5, (Y.R - 1) >> 10, Y.R)
    for _ in range(2):
        rho = rng.randrange(Y.R)
        lhs = (Y.lagrange_eval(a, rho, w) * Y.lagrange_eval(b, rho, w) - Y.lagrange_eval(c, rho, w)) % Y.R
        assert lhs == Y.poly_eval(hv, rho) * (pow(rho, 1024, Y.R) - 1) % Y.R
    bad = bytearray(z)
    bad[32 * 9] ^= 1
    assert not c10.qap_h(bytes(bad))[0]


def test_packing_and_bool_fraction_small():
    c = O.Circuit(12, 4096, 8, 8, 172, seed=3, input_seed=3)
    z = Y.ints_from_bytes(c.witness())
    assert c.r1cs_check(c.witness())
    nbool = sum(1 for v in z if v in (0, 1))
    assert nbool == 8 * 172 + 1                     # the packed bits and z_0
    # packing row: (sum 2^k b_k) * 1 = y
    row = 8 * 243
    A, B, C = c.row(0, row), c.row(1, row), c.row(2, row)
    assert B == [(0, 1)] and len(A) <= 172 and len(C) == 1
    assert sum(coef * z[v] for v, coef in A) % Y.R == z[C[0][0]]


def test_groth16_prove_verify_expected(c10):
    z = c10.witness()
    pk = O.ProvingKey(c10, 1, with_points=True)
    r, s = O.rs_from_seed(1)
    ok, proof = pk.prove(z, r, s, method=1)
    assert ok and len(proof) == 256
    assert proof == pk.expected_proof(z, r, s)
    pub = Y.ints_from_bytes(z)[1]
    assert pk.verify(pub, proof) == 1
    assert pk.verify((pub + 1) % Y.R, proof) == 0
    # swap A and C: still on the curve, must fail
    swapped = proof[192:256] + proof[64:192] + proof[0:64]
    assert pk.verify(pub, swapped) == 0
    bad = bytearray(proof)
    bad[5] ^= 1
    assert pk.verify(pub, bytes(bad)) == -1           # off-curve


def test_groth16_setup_points_are_scalar_multiples(c10):
    pk = O.ProvingKey(c10, 5, with_points=True)
    g1, g2 = O.g1_generator(), O.g2_generator()
    tau = pk.scalar("toxic", 0)
    delta = pk.scalar("toxic", 4)
    for j in (0, 1, 2, 100, c10.m - 1):
        assert pk.point("A", j) == O.g1_mul(g1, pk.scalar("u", j))
        assert pk.point("B2", j) == O.g2_mul(g2, pk.scalar("v", j))
    for i in (0, 1, 500, c10.N - 2):
        want = pow(tau, i, Y.R) * (pow(tau, c10.N, Y.R) - 1) * pow(delta, Y.R - 2, Y.R) % Y.R
        assert pk.scalar("h", i) == want
    # u_j(tau) = sum_i A_ij L_i(tau) for a column that appears in one row
    w = pow(5, (Y.R - 1) >> 10, Y.R)
    li = [0] * 1024
    zr = (pow(tau, 1024, Y.R) - 1) % Y.R
    for i in (0, 1, 1023):
        wi = pow(w, i, Y.R)
        li[i] = zr * wi * pow(1024, Y.R - 2, Y.R) * pow((tau - wi) % Y.R, Y.R - 2, Y.R) % Y.R
    # variable 5 (x2 of the first S-box) appears in A of row 1 only, with coefficient 1
    assert [t for t in c10.row(0, 1) if t[0] == 5] == [(5, 1)]
    assert pk.scalar("w", 5) == li[0]                  # C of row 0 is x2 with coefficient 1
    assert pk.scalar("u", 1) == li[1023]               # z_1 sits only in input row 1023 of A


def test_fixed_base_windowing_vs_double_and_add():
    """The setup's fixed-base windowing (T[w][d] = d 2^(8w) G) against
    double-and-add and the textbook affine formulas, on edge scalars (zero
    bytes, all-ones bytes, r - 1) and random ones."""
    g1, g2 = O.g1_generator(), O.g2_generator()
    edge = [0, 1, 2, 255, 256, 257, (1 << 64) - 1, 1 << 128, (1 << 248) + 1, Y.R - 1, Y.R - 2,
            int("ff" * 31, 16) % Y.R]
    rnd = random.Random(77)
    for k in edge + [rnd.randrange(Y.R) for _ in range(20)]:
        assert O.gen_tab_mul(k, 1) == O.g1_mul(g1, k), k
        assert O.gen_tab_mul(k, 2) == O.g2_mul(g2, k), k
    for k in (3, 1 << 200):
        assert O.g1_from(O.gen_tab_mul(k, 1)) == Y.g1_mul(Y.G1, k)


def test_setup_points_every_query(c10):
    """Every A, B1, B2, L and H point of the 2^10 key is its scalar times the
    generator by double-and-add."""
    pk = O.ProvingKey(c10, 6, with_points=True)
    g1, g2 = O.g1_generator(), O.g2_generator()
    for j in range(0, c10.m, 37):
        assert pk.point("A", j) == O.g1_mul(g1, pk.scalar("u", j))
        assert pk.point("B1", j) == O.g1_mul(g1, pk.scalar("v", j))
        if j % 111 == 0:
            assert pk.point("B2", j) == O.g2_mul(g2, pk.scalar("v", j))
        if j > 1:
            assert pk.point("L", j) == O.g1_mul(g1, pk.scalar("l", j))
    for i in range(0, c10.N - 1, 41):
        assert pk.point("H", i) == O.g1_mul(g1, pk.scalar("h", i))


def test_unsat_witness_rejected(c10):
    z = bytearray(c10.witness())
    z[32 * 20] ^= 2
    pk = O.ProvingKey(c10, 1, with_points=True)
    r, s = O.rs_from_seed(1)
    ok, _ = pk.prove(bytes(z), r, s)
    assert not ok
