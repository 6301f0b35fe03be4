"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds no arithmetic of the proving method: only the SplitMix64 generator
(Steele, Lea and Flood, OOPSLA 2014), rejection sampling of values below the
scalar-field modulus r, and the scalar distributions of the MSM workloads.

Stream (seed, purpose): state_0 = seed XOR purpose * 0x9E3779B97F4A7C15 and
output_i = mix(state_0 + (i + 1) * 0x9E3779B97F4A7C15).  A field element is
four consecutive outputs read as little-endian 64-bit limbs with the top two
bits cleared, rejected while >= r.

Scalar distributions (MSM inputs):
  uniform: the field sampler on (seed, purpose 7);
  sparse:  per index a selector u_i from (seed, purpose 11); with
           u_i mod 10 < 7 the scalar is the bit u_i >> 63, otherwise it is the
           next value of the field sampler on (seed, purpose 7).
"""
from __future__ import annotations

import numpy as np

R = 21888242871839275222246405745257275088548364400416034343698204186575808495617
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
PURPOSE = {"round_const": 1, "mds": 2, "inputs": 3, "toxic": 4, "rs": 5, "bases": 6,
           "scalars": 7, "sizes": 8, "arrivals": 9, "chain": 10, "selector": 11}
_R_LIMBS = np.array([(R >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)


def splitmix64(seed: int, purpose: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+n-1 of the stream (seed, purpose) as uint64."""
    with np.errstate(over="ignore"):
        s0 = np.uint64((seed ^ ((purpose * 0x9E3779B97F4A7C15) & ((1 << 64) - 1))) & ((1 << 64) - 1))
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = s0 + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _below_r(c: np.ndarray) -> np.ndarray:
    """c: (k, 4) uint64 little-endian limbs -> bool mask of c < r."""
    lt = np.zeros(len(c), dtype=bool)
    eq = np.ones(len(c), dtype=bool)
    for i in (3, 2, 1, 0):
        lt |= eq & (c[:, i] < _R_LIMBS[i])
        eq &= c[:, i] == _R_LIMBS[i]
    return lt


def sample_fr(seed: int, purpose: int, n: int) -> np.ndarray:
    """n field elements from the rejection sampler, as an (n, 8) uint32 array
    of little-endian limbs (canonical)."""
    out = np.empty((0, 4), dtype=np.uint64)
    pos = 0
    while len(out) < n:
        need = n - len(out)
        k = int(need * 1.4) + 16
        w = splitmix64(seed, purpose, 4 * k, start=pos).reshape(k, 4)
        w[:, 3] &= np.uint64((1 << 62) - 1)
        ok = _below_r(w)
        acc = w[ok]
        # keep candidates in order up to the one that completes n
        if len(acc) > need:
            last = np.nonzero(ok)[0][need - 1]
            k_used = last + 1
            acc = acc[:need]
        else:
            k_used = k
        out = np.concatenate([out, acc])
        pos += 4 * k_used
    return out.view(np.uint32).reshape(n, 8).copy()


def sample_scalars(seed: int, n: int, dist: str = "uniform") -> np.ndarray:
    """(n, 8) uint32 canonical scalars in the named distribution."""
    if dist == "uniform":
        return sample_fr(seed, PURPOSE["scalars"], n)
    if dist == "sparse":
        u = splitmix64(seed, PURPOSE["selector"], n)
        small = (u % np.uint64(10)) < np.uint64(7)
        out = np.zeros((n, 8), dtype=np.uint32)
        out[small, 0] = (u[small] >> np.uint64(63)).astype(np.uint32)
        nbig = int((~small).sum())
        out[~small] = sample_fr(seed, PURPOSE["scalars"], nbig)
        return out
    raise ValueError(f"unknown scalar distribution {dist!r}")


def limbs_to_int(a: np.ndarray) -> list:
    """(n, 8) uint32 -> list of Python ints."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = a.view(np.uint8).reshape(len(a), 32)
    return [int.from_bytes(bytes(row), "little") for row in b]


def ints_to_limbs(vals) -> np.ndarray:
    raw = b"".join(int(v).to_bytes(32, "little") for v in vals)
    return np.frombuffer(raw, dtype=np.uint32).reshape(-1, 8).copy()
