"""The autotuner picks among correct configurations only: results after
tuning are unchanged, and the tuned choices survive a save / load."""
import json
import random

import pytest

import oracle as O
from paper_2603_10242_gb300 import inputs

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace


def test_autotune_msm_ntt_and_persist(tmp_path):
    ctx = ace.Context(0)
    rep = ctx.autotune_msm(8, 12)
    assert [int(r[0]) for r in rep] == list(range(8, 13))
    assert all(6 <= r[1] <= 20 and r[2] > 0 for r in rep)
    nrep = ctx.autotune_ntt(10, 14)
    assert all(int(r[1]) in (10, 11, 12) and int(r[4]) in (2, 4) for r in nrep)
    # tuned MSM still exact
    rng = random.Random(3)
    n = 3000
    ks = [rng.randrange(1, gu.R) for _ in range(n)]
    ss = [rng.randrange(gu.R) for _ in range(n)]
    pts = O.g1_mul_gen_batch(gu.ints_bytes(ks))
    out = gu.empty(64)
    ctx.msm_g1(gu.dev(pts), gu.dev(gu.ints_bytes(ss)), n, out)
    assert gu.host(out) == O.g1_mul(O.g1_generator(), sum(a * b for a, b in zip(ks, ss)) % gu.R)
    # tuned NTT still exact
    vals = [rng.randrange(gu.R) for _ in range(1 << 12)]
    d = gu.dev(gu.ints_bytes(vals))
    ctx.ntt(d, 12, 0)
    assert gu.host(d) == O.ntt(gu.ints_bytes(vals), 12)
    path = str(tmp_path / "tune.json")
    ctx.autotune_save(path)
    data = json.load(open(path))
    assert data["msm_c"] and data["ntt_smem_log"]
    assert set(data["ntt_radix"].values()) <= {2, 4}
    ctx2 = ace.Context(0)
    ctx2.autotune_load(path)
    data["gpu"] = "another GPU"
    bad = str(tmp_path / "other.json")
    json.dump(data, open(bad, "w"))
    with pytest.raises(ace.AceError):
        ctx2.autotune_load(bad)


def test_autotune_batch_slots_keeps_results():
    ctx = ace.Context(0)
    c = ace.Circuit(12, 4096, 10, 0, 0, seed=3)
    pk = ace.ProvingKey(ctx, c, toxic_seed=3)
    z = c.witness(3)
    dz = gu.dev(z)
    r, s = ace.rs_from_seed(1)
    want = ctx.prove(pk, dz, r, s)
    times = ctx.autotune_batch_slots(pk, dz, 6, 3)
    assert len(times) == 6 and all(t > 0 for t in times)
    proofs, status = ctx.prove_batch([pk] * 4, [dz] * 4, r * 4, s * 4)
    assert status == [0] * 4 and all(p == want for p in proofs)


@pytest.mark.parametrize("log_n", [1, 2, 3, 5, 9, 12, 17, 20])
def test_both_ntt_stage_forms_match_oracle(tmp_path, log_n):
    """Radix-2 stages and radix-4 pairs (chosen per size by default, or by a
    tuning file) give the oracle's transform, every kind, every element, at
    one-pass sizes with odd and even stage counts and at multi-pass sizes."""
    ctx = ace.Context(0)
    path = str(tmp_path / "t.json")
    ctx.autotune_save(path)
    data = json.load(open(path))
    vals = inputs.sample_fr(300 + log_n, 7, 1 << log_n).tobytes()
    for radix in (2, 4):
        data["ntt_radix"] = {str(log_n): radix}
        json.dump(data, open(path, "w"))
        ctx.autotune_load(path)
        for kind in range(4):
            d = gu.dev(vals)
            ctx.ntt(d, log_n, kind)
            if kind < 2:
                want = O.ntt(vals, log_n, inverse=(kind == 1))
            else:
                want = O.coset_ntt(vals, log_n, 5, inverse=(kind == 3))
            assert gu.host(d) == want, (radix, kind)
