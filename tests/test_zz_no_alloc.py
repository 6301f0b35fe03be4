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
    rng = random.Random(seed)
    ks = [rng.randrange(1, gu.R) for _ in range(n)]
    pts = O.g1_mul_gen_batch(gu.ints_bytes(ks))
    ss = [rng.randrange(gu.R) if rng.random() < 0.6 else rng.randrange(2) for _ in range(n)]
    return gu.dev(pts), gu.dev(gu.ints_bytes(ss))


def _noalloc(bases, scalars, n, out, form=ace.FORM_CANONICAL):
    L = ace.lib()
    stream = torch.cuda.current_stream().cuda_stream or None
    rc = L.ace_msm_g1_noalloc(bases.data_ptr(), form, scalars.data_ptr(), n, out.data_ptr(), stream)
    if rc != 0:
        raise ace.AceError(rc, L.ace_last_error().decode())


def test_noalloc_matches_msm_g1_on_consecutive_calls():
    ctx = gu.ctx()
    for call, (n, seed) in enumerate(((MAX_N, 1), (3001, 2), (7, 3))):
        bases, scalars = _inputs(n, seed)
        want = gu.empty(64)
        ctx.msm_g1(bases, scalars, n, want, ace.FORM_CANONICAL)
        got = gu.empty(64)
        _noalloc(bases, scalars, n, got)
        assert gu.host(got) == gu.host(want), f"call {call}"


def test_noalloc_rejects_oversize_and_bad_form():
    bases, scalars = _inputs(4, 9)
    out = gu.empty(64)
    with pytest.raises(ace.AceError) as e:
        _noalloc(bases, scalars, MAX_N + 1, out)
    assert e.value.code == -1 and "maximum" in str(e.value)
    with pytest.raises(ace.AceError):
        _noalloc(bases, scalars, 4, out, form=7)
