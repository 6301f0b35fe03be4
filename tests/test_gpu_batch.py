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


def test_batch_from_host_witnesses_matches_device_batch():
    """ace_prove_batch_host (witnesses in pinned and in pageable host memory,
    copied by the library into the slots' staging buffers) gives the same
    proofs and status as the device-resident batch, over mixed keys and a
    batch long enough to reuse every slot's staging buffer."""
    ctx = gu.ctx()
    circs = [ace.Circuit(*p, seed=50 + i) for i, p in enumerate(PARAMS)]
    pks = [ace.ProvingKey(ctx, c, toxic_seed=60 + i) for i, c in enumerate(circs)]
    zs = [c.witness(70 + i) for i, c in enumerate(circs)]
    rss = [ace.rs_from_seed(80 + i) for i in range(len(PARAMS))]
    rs = b"".join(r for r, _ in rss)
    ss = b"".join(s for _, s in rss)
    want, st = ctx.prove_batch(pks, [gu.dev(z) for z in zs], rs, ss)
    assert st == [0] * len(PARAMS)
    pinned = [torch.frombuffer(bytearray(z), dtype=torch.uint8).pin_memory() for z in zs]
    pageable = [torch.frombuffer(bytearray(z), dtype=torch.uint8) for z in zs]
    got, st2 = ctx.prove_batch_host(pks + pks, pinned + pageable, rs + rs, ss + ss)
    assert st2 == [0] * (2 * len(PARAMS))
    assert got == want + want
    with pytest.raises(ValueError):
        ctx.prove_batch_host(pks[:1], [gu.dev(zs[0])], rs[:32], ss[:32])


def test_batch_tails_same_bytes_for_every_slot_count(tmp_path):
    """The batch's tail kernels (fixed-base terms, V and assembly of every
    proof in one launch each) give the bytes of the one-proof path whatever
    the number of proving slots and the stage layout (MSMs on auxiliary
    streams, or every stage of a proof on one stream)."""
    import re
    ctx = ace.Context(0)
    circs = [ace.Circuit(*p, seed=90 + i) for i, p in enumerate(PARAMS[:3])]
    pks = [ace.ProvingKey(ctx, c, toxic_seed=95 + i) for i, c in enumerate(circs)]
    dzs = [gu.dev(c.witness(99 + i)) for i, c in enumerate(circs)]
    rss = [ace.rs_from_seed(101 + i) for i in range(3)]
    rs = b"".join(r for r, _ in rss)
    ss = b"".join(s for _, s in rss)
    want = [ctx.prove(pks[i], dzs[i], *rss[i]) for i in range(3)]
    path = str(tmp_path / "tune.json")
    ctx.autotune_save(path)
    txt = open(path).read()
    for q, one in ((1, 0), (2, 0), (3, 0), (5, 0), (1, 1), (3, 1), (12, 1)):
        t = re.sub(r'"batch_slots": \d+', f'"batch_slots": {q}', txt)
        t = re.sub(r'"batch_one_stream": \d+', f'"batch_one_stream": {one}', t)
        open(path, "w").write(t)
        ctx.autotune_load(path)
        proofs, status = ctx.prove_batch(pks * 2, dzs * 2, rs * 2, ss * 2)
        assert status == [0] * 6 and proofs == want + want, (q, one)
    ctx.close()


@pytest.mark.parametrize("host", [False, True])
def test_same_key_batch_on_batch_dimension_kernels(host):
    """A batch of 12 proofs of one small key runs on the batch-dimension
    kernels: every proof equals the one-proof path, the unsatisfied witness
    in the middle is reported without disturbing the others, from device and
    from host witnesses."""
    ctx = gu.ctx()
    c = ace.Circuit(11, 2000, 5, 2, 60, seed=61)
    pk = ace.ProvingKey(ctx, c, toxic_seed=62)
    zs = [c.witness(70 + i) for i in range(12)]
    bad = bytearray(zs[5])
    bad[32 * 40] ^= 1
    zs[5] = bytes(bad)
    rss = [ace.rs_from_seed(170 + i) for i in range(12)]
    rs = b"".join(r for r, _ in rss)
    ss = b"".join(s for _, s in rss)
    if host:
        hz = [torch.frombuffer(bytearray(z), dtype=torch.uint8).pin_memory() for z in zs]
        proofs, status = ctx.prove_batch_host([pk] * 12, hz, rs, ss)
    else:
        proofs, status = ctx.prove_batch([pk] * 12, [gu.dev(z) for z in zs], rs, ss)
    assert status == [0] * 5 + [1] + [0] * 6
    for i in (0, 4, 6, 11):
        assert proofs[i] == ctx.prove(pk, gu.dev(zs[i]), *rss[i]), i
    oc = O.Circuit(11, 2000, 5, 2, 60, seed=61, input_seed=77)
    opk = O.ProvingKey(oc, 62, with_points=False)
    assert proofs[7] == opk.expected_proof(zs[7], *rss[7])


def test_one_proof_batch_runs_as_a_lone_proof():
    """A batch of one proof takes the single-proof path (its MSMs on the
    slot's auxiliary streams, latency-first reductions): the same bytes as
    ace_prove and as the oracle's in-the-exponent proof, from device and from
    host witnesses, at a size whose tabled reductions run on four lanes."""
    ctx = gu.ctx()
    p = (14, 1 << 14, 40, 40, 172)
    c = ace.Circuit(*p, seed=71)
    pk = ace.ProvingKey(ctx, c, toxic_seed=72)
    z = c.witness(73)
    r, s = ace.rs_from_seed(74)
    dz = gu.dev(z)
    lone = ctx.prove(pk, dz, r, s)
    proofs, status = ctx.prove_batch([pk], [dz], r, s)
    assert status == [0] and proofs[0] == lone
    hz = torch.frombuffer(bytearray(z), dtype=torch.uint8).pin_memory()
    proofs_h, status_h = ctx.prove_batch_host([pk], [hz], r, s)
    assert status_h == [0] and proofs_h[0] == lone
    oc = O.Circuit(*p, seed=71, input_seed=73)
    opk = O.ProvingKey(oc, 72, with_points=False)
    assert lone == opk.expected_proof(z, r, s)
