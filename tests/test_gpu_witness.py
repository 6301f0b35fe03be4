"""Witnesses made on the device (ace_witness_many) are byte-equal to the host
generator's (ace_witness, itself byte-equal to the oracle's), for circuits
with and without permutations and packing rows, several instances per call,
and the 2^20 block circuit; a block of them proves through ace_prove_many."""
import pytest

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace

PARAMS = [
    (2, 4, 0, 0, 0),        # chain only
    (3, 6, 0, 1, 3),        # a packing row, then the chain-start draw after its bits
    (10, 1024, 4, 0, 0),
    (11, 1400, 5, 0, 0),    # the per-transaction circuit
    (12, 4000, 8, 8, 172),  # permutations and packing rows
]
SEEDS = [5, 6, 1234567890123, 2**64 - 1]


@pytest.mark.parametrize("params", PARAMS)
def test_witness_many_equals_host(params):
    ctx = gu.ctx()
    c = ace.Circuit(*params, seed=31)
    d = torch.empty(len(SEEDS) * 32 * c.m, dtype=torch.uint8, device="cuda")
    ctx.witness_many(c, SEEDS, d)
    got = gu.host(d)
    for q, s in enumerate(SEEDS):
        assert got[32 * c.m * q:32 * c.m * (q + 1)] == c.witness(s)


def test_witness_many_block_circuit():
    ctx = gu.ctx()
    c = ace.Circuit(20, 1 << 20, 4096, 4096, 172, seed=2)
    d = torch.empty(32 * c.m, dtype=torch.uint8, device="cuda")
    ctx.witness_many(c, [2], d)
    assert gu.host(d) == c.witness(2)


def test_device_witnesses_prove():
    ctx = gu.ctx()
    c = ace.Circuit(*PARAMS[3], seed=32)
    pk = ace.ProvingKey(ctx, c, toxic_seed=33)
    seeds = list(range(700, 709))
    d = torch.empty(len(seeds) * 32 * c.m, dtype=torch.uint8, device="cuda")
    ctx.witness_many(c, seeds, d)
    rs = [ace.rs_from_seed(800 + i) for i in range(len(seeds))]
    proofs, status = ctx.prove_many(pk, d, len(seeds), b"".join(r for r, _ in rs), b"".join(s for _, s in rs))
    assert status == [0] * len(seeds)
    z = c.witness(seeds[4])
    assert proofs[4] == ctx.prove(pk, gu.dev(z), *rs[4])
    assert pk.verify(z[32:64], proofs[4]) == 1
