"""The allocation-free G1 MSM entry point (collected last on purpose).

ace_msm_g1_noalloc exists for callers that cannot allocate device memory
(memory owned by a pool handed out up front, or paths that must not trigger
the synchronisation cudaMalloc / cudaFree imply).  It must give the same
point as ace_msm_g1, call after call, although every call reuses one fixed
scratch array inside the library.
"""
import ctypes
import random

import pytest

pytestmark = pytest.mark.gpu

gu = pytest.importorskip("gpu_util")
torch = gu.torch
ace = gu.ace

import oracle as O  # noqa: E402

MAX_N = 16384


def _inputs(n, seed):
    """Bases k_i G (k_i random) and 60% uniform / 40% {0,1} scalars s_i; also
    the discrete logarithm of the expected sum, sum s_i k_i mod r."""
    rng = random.Random(seed)
    ks = [rng.randrange(1, gu.R) for _ in range(n)]
    pts = O.g1_mul_gen_batch(gu.ints_bytes(ks))
    ss = [rng.randrange(gu.R) if rng.random() < 0.6 else rng.randrange(2) for _ in range(n)]
    dlog = sum(a * b for a, b in zip(ks, ss)) % gu.R
    return gu.dev(pts), gu.dev(gu.ints_bytes(ss)), dlog


def _noalloc(bases, scalars, n, out, form=ace.FORM_CANONICAL):
    L = ace.lib()
    stream = torch.cuda.current_stream().cuda_stream or None
    rc = L.ace_msm_g1_noalloc(bases.data_ptr(), form, scalars.data_ptr(), n, out.data_ptr(), stream)
    if rc != 0:
        raise ace.AceError(rc, L.ace_last_error().decode())


def test_noalloc_matches_msm_g1_on_consecutive_calls():
    """Consecutive calls (largest size first, so later calls find the shared
    scratch dirty) equal ace_msm_g1 and the oracle's point for the discrete
    logarithm sum s_i k_i."""
    ctx = gu.ctx()
    g1 = O.g1_generator()
    for call, (n, seed) in enumerate(((MAX_N, 1), (3001, 2), (7, 3))):
        bases, scalars, dlog = _inputs(n, seed)
        want = gu.empty(64)
        ctx.msm_g1(bases, scalars, n, want, ace.FORM_CANONICAL)
        got = gu.empty(64)
        _noalloc(bases, scalars, n, got)
        assert gu.host(got) == gu.host(want), f"call {call}"
        assert gu.host(got) == O.g1_mul(g1, dlog), f"call {call}"


def test_noalloc_takes_no_device_memory():
    """After a first call (which looks up the scratch array's address), more
    calls leave the device's free memory unchanged: no allocation."""
    bases, scalars, dlog = _inputs(MAX_N, 5)
    out = gu.empty(64)
    _noalloc(bases, scalars, MAX_N, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(4):
        _noalloc(bases, scalars, MAX_N, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert gu.host(out) == O.g1_mul(O.g1_generator(), dlog)


def test_noalloc_rejects_oversize_and_bad_form():
    bases, scalars, _ = _inputs(4, 9)
    out = gu.empty(64)
    with pytest.raises(ace.AceError) as e:
        _noalloc(bases, scalars, MAX_N + 1, out)
    assert e.value.code == -1 and "maximum" in str(e.value)
    with pytest.raises(ace.AceError):
        _noalloc(bases, scalars, 4, out, form=7)
