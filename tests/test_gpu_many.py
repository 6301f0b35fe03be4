"""Many proofs of one key in one pass (ace_prove_many): every proof is the
same bytes as the proof made alone; an unsatisfied witness flags only its own
proof; one proof is checked against the oracle's in-the-exponent proof."""
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace

CIRCUITS = [(10, 1024, 4, 0, 0), (11, 1400, 5, 0, 0), (12, 4000, 8, 8, 172)]
TINY = [(2, 4, 0, 0, 0), (3, 6, 0, 1, 3)]  # chain only; a packing row and a ragged tail


def _inputs(c, k, seed):
    zs = [c.witness(seed + i) for i in range(k)]
    rs = [ace.rs_from_seed(seed + 100 + i) for i in range(k)]
    return zs, rs


@pytest.mark.parametrize("params", CIRCUITS)
@pytest.mark.parametrize("k", [1, 3, 17])
def test_prove_many_equals_alone(params, k):
    ctx = gu.ctx()
    c = ace.Circuit(*params, seed=21)
    pk = ace.ProvingKey(ctx, c, toxic_seed=22)
    zs, rs = _inputs(c, k, 300)
    dz = gu.dev(b"".join(zs))
    proofs, status = ctx.prove_many(pk, dz, k, b"".join(r for r, _ in rs), b"".join(s for _, s in rs))
    assert status == [0] * k
    for i in (0, k // 2, k - 1):
        assert proofs[i] == ctx.prove(pk, gu.dev(zs[i]), *rs[i])
    assert pk.verify(zs[-1][32:64], proofs[-1]) == 1


def test_prove_many_against_oracle_and_unsat_flag():
    ctx = gu.ctx()
    params = CIRCUITS[1]
    c = ace.Circuit(*params, seed=23)
    oc = O.Circuit(*params, seed=23, input_seed=400)
    pk = ace.ProvingKey(ctx, c, toxic_seed=24)
    k = 5
    zs, rs = _inputs(c, k, 400)
    assert zs[0] == oc.witness()
    bad = bytearray(zs[3])
    bad[32 * 40] ^= 1
    zs[3] = bytes(bad)
    dz = gu.dev(b"".join(zs))
    proofs, status = ctx.prove_many(pk, dz, k, b"".join(r for r, _ in rs), b"".join(s for _, s in rs))
    assert status == [0, 0, 0, 1, 0]
    opk = O.ProvingKey(oc, 24, with_points=False)
    assert proofs[0] == opk.expected_proof(zs[0], *rs[0])
    for i in (1, 2, 4):
        assert proofs[i] == ctx.prove(pk, gu.dev(zs[i]), *rs[i])


def test_prove_many_rejects_bad_arguments():
    ctx = gu.ctx()
    c = ace.Circuit(*CIRCUITS[0], seed=25)
    pk = ace.ProvingKey(ctx, c, toxic_seed=26)
    z = c.witness(1)
    r, s = ace.rs_from_seed(1)
    bad_r = bytes([0xFF] * 32)
    with pytest.raises(ace.AceError):
        ctx.prove_many(pk, gu.dev(z), 1, bad_r, s)
    assert ctx.prove_many(pk, gu.dev(z), 0, b"", b"") == ([], [])


def test_prove_many_in_chunks(monkeypatch):
    """Proofs split into chunks of 3 (3 + 3 + 1) equal the proofs of one pass."""
    ctx = gu.ctx()
    c = ace.Circuit(*CIRCUITS[2], seed=27)
    pk = ace.ProvingKey(ctx, c, toxic_seed=28)
    k = 7
    zs, rs = _inputs(c, k, 500)
    dz = gu.dev(b"".join(zs))
    r_all, s_all = b"".join(r for r, _ in rs), b"".join(s for _, s in rs)
    whole, st1 = ctx.prove_many(pk, dz, k, r_all, s_all)
    monkeypatch.setenv("ACE_MANY_MAX_CHUNK", "3")
    chunked, st2 = ctx.prove_many(pk, dz, k, r_all, s_all)
    assert st1 == st2 == [0] * k and chunked == whole
    assert chunked[6] == ctx.prove(pk, gu.dev(zs[6]), *rs[6])


@pytest.mark.parametrize("params", TINY)
def test_prove_many_tiny_circuits(params):
    ctx = gu.ctx()
    c = ace.Circuit(*params, seed=29)
    pk = ace.ProvingKey(ctx, c, toxic_seed=30)
    k = 5
    zs, rs = _inputs(c, k, 600)
    proofs, status = ctx.prove_many(pk, gu.dev(b"".join(zs)), k, b"".join(r for r, _ in rs),
                                    b"".join(s for _, s in rs))
    assert status == [0] * k
    for i in range(k):
        assert proofs[i] == ctx.prove(pk, gu.dev(zs[i]), *rs[i])
