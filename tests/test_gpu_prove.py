"""GPU parity of the full Groth16 path against the CPU oracle.

Circuit and witness (host, byte-identical to the oracle's), setup points
(sampled, against scalar multiples of the oracle's setup scalars; the H query
in the coset Lagrange basis from its product definition), the QAP
quotient (bit-exact), and whole proofs: bit-exact against the oracle's own
prover at small sizes and against the in-the-exponent proof (no NTT, no MSM
on the oracle side) up to the 2^20 block-scale circuit, plus the oracle's
pairing verification.
"""
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace

# (log_n, n_rows, n_perm, n_pack, pack_bits)
SMALL = [
    (2, 4, 0, 0, 0),          # chain only, smallest domain
    (3, 6, 0, 1, 3),          # ragged: zero rows at the end, a packing row
    (10, 1024, 4, 0, 0),      # the 2^10 single-proof circuit
    (12, 4000, 8, 8, 172),    # packing rows, zero rows 4000..4095
]


def _coset_h_scalar(opk, log_n, i):
    """Scalar of H query point i: L'_i(tau) Z(tau)/delta, L'_i the Lagrange
    basis of the coset g H (g = 5) by its product definition
    prod_{j != i} (tau - x_j) / (x_i - x_j), x_j = g omega^j, at
    tau = h_1 / h_0 from the oracle's monomial scalars h_e = tau^e Z(tau)/delta."""
    R = gu.R
    h0, h1 = opk.scalar("h", 0), opk.scalar("h", 1)
    tau = h1 * pow(h0, -1, R) % R
    n = 1 << log_n
    w = O.fr_root_of_unity(log_n)
    xi = 5 * pow(w, i, R) % R
    num = den = 1
    x = 5
    for j in range(n):
        if j != i:
            num = num * (tau - x) % R
            den = den * (xi - x) % R
        x = x * w % R
    return num * pow(den, -1, R) * h0 % R


def _pair(params, seed=1):
    lc = ace.Circuit(*params, seed=seed)
    oc = O.Circuit(*params, seed=seed, input_seed=seed)
    return lc, oc


@pytest.mark.parametrize("params", SMALL)
def test_circuit_and_witness_match_oracle(params):
    lc, oc = _pair(params)
    assert (lc.N, lc.m) == (oc.N, oc.m)
    assert lc.info[4:7] == [oc.nnz_a, oc.nnz_b, oc.nnz_c]
    assert lc.witness(1) == oc.witness()


@pytest.mark.parametrize("params", SMALL)
def test_setup_points_match_oracle_scalars(params):
    lc, oc = _pair(params)
    ctx = gu.ctx()
    pk = ace.ProvingKey(ctx, lc, toxic_seed=3)
    opk = O.ProvingKey(oc, 3, with_points=False)
    g1, g2 = O.g1_generator(), O.g2_generator()
    js = sorted({0, 1, 2, lc.m // 2, lc.m - 1})
    for j in js:
        assert pk.point("A", j) == O.g1_mul(g1, opk.scalar("u", j))
        assert pk.point("B1", j) == O.g1_mul(g1, opk.scalar("v", j))
        assert pk.point("B2", j) == O.g2_mul(g2, opk.scalar("v", j))
        if j > 1:
            assert pk.point("L", j) == O.g1_mul(g1, opk.scalar("l", j))
    for i in sorted({0, 1, lc.N // 2, lc.N - 2, lc.N - 1}):
        assert pk.point("H", i) == O.g1_mul(g1, _coset_h_scalar(opk, params[0], i)), i
    # verifying key
    vk = bytes(pk.vk)
    assert vk[0:64] == opk.point("fixed", 0)
    assert vk[64:192] == opk.point("fixed", 3)
    assert vk[192:320] == opk.point("fixed", 4)
    assert vk[320:448] == opk.point("fixed", 5)
    assert vk[448:512] == opk.point("fixed", 6)
    assert vk[512:576] == opk.point("fixed", 7)


@pytest.mark.parametrize("params", SMALL)
def test_qap_h_matches_oracle(params):
    lc, oc = _pair(params)
    ctx = gu.ctx()
    pk = ace.ProvingKey(ctx, lc, toxic_seed=2)
    z = lc.witness(1)
    dz = gu.dev(z)
    dh = gu.empty(32 * lc.N)
    ctx.qap_h(pk, dz, dh)
    ok, want = oc.qap_h(z)
    assert ok
    assert gu.host(dh)[:32 * lc.N] == want


@pytest.mark.parametrize("params", SMALL)
def test_prove_matches_oracle_prover(params):
    lc, oc = _pair(params)
    ctx = gu.ctx()
    pk = ace.ProvingKey(ctx, lc, toxic_seed=5)
    z = lc.witness(1)
    r, s = ace.rs_from_seed(7)
    proof = ctx.prove(pk, gu.dev(z), r, s)
    opk = O.ProvingKey(oc, 5, with_points=True)
    ok, want = opk.prove(z, r, s, method=1)
    assert ok
    assert proof == want
    assert proof == opk.expected_proof(z, r, s)
    assert opk.verify(int.from_bytes(z[32:64], "little"), proof) == 1


def test_prove_repeatable_and_independent_of_stream():
    lc, oc = _pair((12, 4096, 10, 4, 100))
    ctx = gu.ctx()
    pk = ace.ProvingKey(ctx, lc, toxic_seed=9)
    z = lc.witness(1)
    r, s = ace.rs_from_seed(9)
    p1 = ctx.prove(pk, gu.dev(z), r, s)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        dz = gu.dev(z)
        p2 = ctx.prove(pk, dz, r, s, stream=st)
    p3 = ctx.prove(pk, gu.dev(z), r, s)
    opk = O.ProvingKey(oc, 9, with_points=False)
    assert p1 == p2 == p3 == opk.expected_proof(z, r, s)


def test_unsat_witness_rejected():
    lc, _ = _pair((10, 1024, 4, 0, 0))
    ctx = gu.ctx()
    pk = ace.ProvingKey(ctx, lc, toxic_seed=1)
    z = bytearray(lc.witness(1))
    z[32 * 40] ^= 1
    r, s = ace.rs_from_seed(1)
    with pytest.raises(ace.AceError) as e:
        ctx.prove(pk, gu.dev(bytes(z)), r, s)
    assert e.value.code == -4


@pytest.fixture(scope="module", params=[16, 20])
def block(request):
    """The 2^20 block circuit (2,048 tx x 2 permutations, 2 packing rows of
    172 bits per tx, chain to 2^20), and a 2^16 instance of the same family:
    library and oracle circuits, the witness and the library's key."""
    log_n = request.param
    if log_n == 20:
        params = (20, 1 << 20, 4096, 4096, 172)
    else:
        params = (16, 1 << 16, 256, 256, 172)
    lc, oc = _pair(params, seed=2)
    z = lc.witness(2)
    pk = ace.ProvingKey(gu.ctx(), lc, toxic_seed=2)
    yield log_n, lc, oc, z, pk
    pk.close()
    torch.cuda.synchronize()


def test_block_scale_proof_in_the_exponent(block):
    log_n, lc, oc, z, pk = block
    ctx = gu.ctx()
    assert z == oc.witness()
    r, s = ace.rs_from_seed(2)
    proof = ctx.prove(pk, gu.dev(z), r, s)
    opk = O.ProvingKey(oc, 2, with_points=False)
    assert proof == opk.expected_proof(z, r, s)
    assert opk.verify(int.from_bytes(z[32:64], "little"), proof) == 1
    # the bench's launch configuration: proofs pipelined over proving slots
    dz = gu.dev(z)
    rss = [ace.rs_from_seed(50 + i) for i in range(3)] + [(r, s)]
    proofs, status = ctx.prove_batch([pk] * 4, [dz] * 4, b"".join(a for a, _ in rss), b"".join(b for _, b in rss))
    assert status == [0] * 4 and proofs[3] == proof
    assert proofs[1] == opk.expected_proof(z, *rss[1])
    # sampled setup points at full size
    g1 = O.g1_generator()
    for j in (2, lc.m // 3, lc.m - 1):
        assert pk.point("A", j) == O.g1_mul(g1, opk.scalar("u", j))
    for i in (0, lc.N - 1):
        assert pk.point("H", i) == O.g1_mul(g1, _coset_h_scalar(opk, log_n, i))


def test_block_scale_qap_h_matches_oracle(block):
    """ace_qap_h (sparse products, 3 iNTT, 3 coset NTT, quotient, coset iNTT
    in the multi-pass plan of these sizes) against the oracle's h, computed by
    a 2N-point convolution and long division by X^N - 1: every coefficient,
    and h_{N-1} = 0."""
    log_n, lc, oc, z, pk = block
    ctx = gu.ctx()
    dh = gu.empty(32 * lc.N)
    ctx.qap_h(pk, gu.dev(z), dh)
    got = gu.host(dh)[:32 * lc.N]
    ok, want = oc.qap_h(z)
    assert ok
    assert got[-32:] == bytes(32)
    assert got == want


def test_pk_save_load_roundtrip(tmp_path):
    lc, oc = _pair((12, 4000, 8, 8, 172), seed=4)
    ctx = gu.ctx()
    pk = ace.ProvingKey(ctx, lc, toxic_seed=4)
    z = lc.witness(4)
    r, s = ace.rs_from_seed(4)
    want = ctx.prove(pk, gu.dev(z), r, s)
    path = str(tmp_path / "key.acepk")
    pk.save(path)
    pk2 = ace.ProvingKey.load(ctx, path)
    assert (pk2.N, pk2.m) == (pk.N, pk.m) and pk2.info[7:10] == pk.info[7:10]
    assert bytes(pk2.vk) == bytes(pk.vk)
    assert ctx.prove(pk2, gu.dev(z), r, s) == want
    assert pk2.verify(z[32:64], want) == 1
    # a truncated file is rejected
    data = open(path, "rb").read()
    bad = str(tmp_path / "bad.acepk")
    open(bad, "wb").write(data[: len(data) // 2])
    with pytest.raises(ace.AceError):
        ace.ProvingKey.load(ctx, bad)
