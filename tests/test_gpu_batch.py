"""Batched proving (several proofs pipelined over proving slots) must give,
for every proof, the same bytes as proving it alone, for uneven circuit
sizes, and must report an unsatisfied witness without disturbing the others.
"""
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace

PARAMS = [(10, 1024, 4, 0, 0), (12, 3000, 8, 4, 100), (14, 1 << 14, 40, 40, 172), (11, 2048, 6, 2, 50),
          (13, 5000, 12, 0, 0)]


def test_batch_matches_single_proofs_uneven_sizes():
    ctx = gu.ctx()
    circs = [ace.Circuit(*p, seed=10 + i) for i, p in enumerate(PARAMS)]
    pks = [ace.ProvingKey(ctx, c, toxic_seed=20 + i) for i, c in enumerate(circs)]
    zs = [c.witness(30 + i) for i, c in enumerate(circs)]
    dzs = [gu.dev(z) for z in zs]
    rss = [ace.rs_from_seed(40 + i) for i in range(len(PARAMS))]
    rs = b"".join(r for r, _ in rss)
    ss = b"".join(s for _, s in rss)
    proofs, status = ctx.prove_batch(pks, dzs, rs, ss)
    assert status == [0] * len(PARAMS)
    for i in range(len(PARAMS)):
        assert proofs[i] == ctx.prove(pks[i], dzs[i], *rss[i])
    # two of them against the oracle's in-the-exponent proof
    for i in (0, 2):
        oc = O.Circuit(*PARAMS[i], seed=10 + i, input_seed=30 + i)
        opk = O.ProvingKey(oc, 20 + i, with_points=False)
        assert proofs[i] == opk.expected_proof(zs[i], *rss[i])
    # a batch twice as long reuses the slots and still agrees
    proofs2, status2 = ctx.prove_batch(pks + pks, dzs + dzs, rs + rs, ss + ss)
    assert proofs2 == proofs + proofs and status2 == [0] * (2 * len(PARAMS))


def test_batch_reports_unsat_in_the_middle():
    ctx = gu.ctx()
    c = ace.Circuit(10, 1024, 4, 0, 0, seed=1)
    pk = ace.ProvingKey(ctx, c, toxic_seed=1)
    z = c.witness(1)
    bad = bytearray(z)
    bad[32 * 50] ^= 1
    dzs = [gu.dev(z), gu.dev(bytes(bad)), gu.dev(z)]
    r, s = ace.rs_from_seed(3)
    proofs, status = ctx.prove_batch([pk] * 3, dzs, r * 3, s * 3)
    assert status == [0, 1, 0]
    assert proofs[0] == proofs[2] == ctx.prove(pk, dzs[0], r, s)
