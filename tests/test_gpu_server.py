"""The proof server with continuous batching on the GPU: every job's proof is
the same bytes as the proof made alone, whatever else is in flight; an
unsatisfied witness fails only its own job; queue deadlines expire."""
import pytest

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace

PARAMS = [(10, 1024, 4, 0, 0), (12, 4096, 10, 4, 100), (14, 1 << 14, 60, 20, 172)]


def _setup():
    ref = gu.ctx()
    circs = [ace.Circuit(*p, seed=70 + i) for i, p in enumerate(PARAMS)]
    pks = [ace.ProvingKey(ref, c, toxic_seed=80 + i) for i, c in enumerate(circs)]
    return ref, circs, pks


def test_server_results_equal_alone_in_a_mix():
    ref, circs, pks = _setup()
    jobs = []
    for k in range(9):
        i = k % 3
        z = circs[i].witness(100 + k)
        r, s = ace.rs_from_seed(200 + k)
        alone = ref.prove(pks[i], gu.dev(z), r, s)
        zh = torch.frombuffer(bytearray(z), dtype=torch.uint8).pin_memory()
        jobs.append((i, zh, r, s, alone, z))
    sctx = ace.Context(0)
    spks = [ace.ProvingKey(sctx, c, toxic_seed=80 + i) for i, c in enumerate(circs)]
    srv = ace.Server(sctx, spks[2], slots=3)
    ids = [srv.submit(spks[i], zh, r, s) for (i, zh, r, s, _, _) in jobs]
    for jid, (i, _, _, _, alone, z) in zip(ids, jobs):
        proof, lat = srv.wait(jid, timeout_s=120)
        assert proof == alone
        assert lat > 0
        assert spks[i].verify(z[32:64], proof) == 1
    st = srv.stats()
    assert st["submitted"] == 9 and st["collected"] == 9 and st["peak_running"] >= 2
    srv.close()


def test_server_unsat_and_deadline():
    ref, circs, pks = _setup()
    sctx = ace.Context(0)
    spk = ace.ProvingKey(sctx, circs[1], toxic_seed=81)
    z = circs[1].witness(5)
    bad = bytearray(z)
    bad[32 * 33] ^= 1
    r, s = ace.rs_from_seed(6)
    good_h = torch.frombuffer(bytearray(z), dtype=torch.uint8).pin_memory()
    bad_h = torch.frombuffer(bad, dtype=torch.uint8).pin_memory()
    srv = ace.Server(sctx, spk, slots=2)
    j1, j2, j3 = srv.submit(spk, good_h, r, s), srv.submit(spk, bad_h, r, s), srv.submit(spk, good_h, r, s)
    p1, _ = srv.wait(j1, 120)
    with pytest.raises(ace.AceError) as e:
        srv.wait(j2, 120)
    assert e.value.code == -4
    p3, _ = srv.wait(j3, 120)
    assert p1 == p3 == ref.prove(pks[1], gu.dev(z), r, s)
    srv.close()
    # one slot and a 2 ms queue deadline: the first job starts at once (the
    # server thread polls every 50 us), the jobs behind a proof of several
    # milliseconds cannot start in time
    big = ace.Circuit(15, 1 << 15, 100, 0, 0, seed=90)
    bpk = ace.ProvingKey(sctx, big, toxic_seed=91)
    big_h = torch.frombuffer(bytearray(big.witness(92)), dtype=torch.uint8).pin_memory()
    srv = ace.Server(sctx, bpk, slots=1, max_queue_wait_s=2e-3)
    ids = [srv.submit(bpk, big_h, r, s) for _ in range(4)]
    codes = []
    for jid in ids:
        try:
            srv.wait(jid, 120)
            codes.append(0)
        except ace.AceError as ex:
            codes.append(ex.code)
    assert codes[0] == 0 and -6 in codes[1:]
    srv.close()
