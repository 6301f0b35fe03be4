"""Helpers for the GPU parity tests: device buffers from numpy / bytes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2603_10242_gb300 as ace  # noqa: E402

P = 21888242871839275222246405745257275088696311157297823662689037894645226208583
R = 21888242871839275222246405745257275088548364400416034343698204186575808495617
RMONT = 1 << 256


def dev(b) -> "torch.Tensor":
    """bytes / numpy array -> uint8 CUDA tensor (16-byte aligned allocation)."""
    if isinstance(b, np.ndarray):
        b = np.ascontiguousarray(b).view(np.uint8).reshape(-1)
        t = torch.from_numpy(b.copy())
    else:
        t = torch.frombuffer(bytearray(b), dtype=torch.uint8) if len(b) else torch.empty(0, dtype=torch.uint8)
    if t.numel() == 0:
        return torch.empty(16, dtype=torch.uint8, device="cuda")
    return t.cuda()


def host(t) -> bytes:
    torch.cuda.synchronize()
    return bytes(t.cpu().numpy().tobytes())


def empty(nbytes: int):
    return torch.zeros(max(nbytes, 16), dtype=torch.uint8, device="cuda")


def ints_bytes(vals, width=32) -> bytes:
    return b"".join(int(v).to_bytes(width, "little") for v in vals)


def bytes_ints(b, width=32):
    return [int.from_bytes(b[i:i + width], "little") for i in range(0, len(b), width)]


def to_mont_g1_bytes(pts: bytes) -> bytes:
    """affine canonical G1 bytes -> Montgomery-form coordinates (x R mod p)."""
    v = bytes_ints(pts)
    return ints_bytes([(x * RMONT) % P for x in v])


_ctx = None


def ctx():
    global _ctx
    if _ctx is None:
        _ctx = ace.Context(0)
    return _ctx
