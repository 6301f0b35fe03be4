"""Batch verification (ace_verify_batch): a block of valid proofs passes; a
proof with another proof's C, swapped public inputs, or a single bad proof
among many fails; malformed points are rejected; one proof agrees with the
single verifier."""
import pytest

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace


@pytest.fixture(scope="module")
def block():
    ctx = gu.ctx()
    c = ace.Circuit(11, 1400, 5, 0, 0, seed=41)
    pk = ace.ProvingKey(ctx, c, toxic_seed=42)
    k = 37
    seeds = list(range(900, 900 + k))
    d = torch.empty(k * 32 * c.m, dtype=torch.uint8, device="cuda")
    ctx.witness_many(c, seeds, d)
    zs = gu.host(d)
    pubs = b"".join(zs[32 * c.m * i + 32:32 * c.m * i + 64] for i in range(k))
    rs = [ace.rs_from_seed(1000 + i) for i in range(k)]
    proofs, status = ctx.prove_many(pk, d, k, b"".join(r for r, _ in rs), b"".join(s for _, s in rs))
    assert status == [0] * k
    return ctx, pk, pubs, proofs


def test_valid_block_passes(block):
    ctx, pk, pubs, proofs = block
    allp = b"".join(proofs)
    assert ctx.verify_batch(pk.vk, pubs, allp, 7) == 1
    assert ctx.verify_batch(pk.vk, pubs, allp, 123456789) == 1
    assert ctx.verify_batch(pk.vk, pubs[:32], proofs[0], 1) == 1
    assert pk.verify(pubs[:32], proofs[0]) == 1


def test_tampered_blocks_fail(block):
    ctx, pk, pubs, proofs = block
    k = len(proofs)
    # one proof carries another proof's C
    bad = list(proofs)
    bad[5] = bad[5][:192] + bad[6][192:]
    assert ctx.verify_batch(pk.vk, pubs, b"".join(bad), 7) == 0
    # two public inputs swapped
    p = bytearray(pubs)
    p[32 * 3:32 * 4], p[32 * 4:32 * 5] = pubs[32 * 4:32 * 5], pubs[32 * 3:32 * 4]
    assert ctx.verify_batch(pk.vk, bytes(p), b"".join(proofs), 7) == 0
    # A and C swapped in the last proof
    bad = list(proofs)
    bad[k - 1] = bad[k - 1][192:] + bad[k - 1][64:192] + bad[k - 1][:64]
    assert ctx.verify_batch(pk.vk, pubs, b"".join(bad), 7) == 0


def test_malformed_point_rejected(block):
    ctx, pk, pubs, proofs = block
    bad = bytearray(proofs[2])
    bad[3] ^= 1
    allp = b"".join(proofs[:2]) + bytes(bad)
    with pytest.raises(ace.AceError) as e:
        ctx.verify_batch(pk.vk, pubs[:96], allp, 7)
    assert e.value.code == -5
