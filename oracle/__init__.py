"""Plain CPU Groth16/BN254 oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product library never imports
it and shares no code with it.

The arithmetic lives in ``groth16_oracle.c`` (4x64-bit Montgomery fields,
Jacobian curve formulas, radix-2 NTT, double-and-add and plain Pippenger MSMs,
the synthetic Poseidon-style R1CS, Groth16 setup / prove / verify with the
reduced Tate pairing).  This module compiles it with gcc on first use and wraps
it with ctypes.  All values cross the boundary as canonical little-endian
32-byte field elements; G1 points are 64 bytes (x || y), G2 points 128 bytes
(x.c0 || x.c1 || y.c0 || y.c1); the point at infinity is all zeros.

What it follows: Groth16.Prove / Groth16.Verify of the paper's Phase 2
(Section 3.1 Algorithm 1, Section 3.3 Algorithm 3 and the ZK-ACE circuit
paragraph: BN254, 256-byte proof, three-pairing verification), with the
construction of Groth 2016 that the paper cites.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "groth16_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgroth16_oracle.so")
_lock = threading.Lock()
_lib = None

P = 21888242871839275222246405745257275088696311157297823662689037894645226208583
R = 21888242871839275222246405745257275088548364400416034343698204186575808495617

PURPOSE = {
    "round_const": 1, "mds": 2, "inputs": 3, "toxic": 4, "rs": 5,
    "bases": 6, "scalars": 7, "sizes": 8, "arrivals": 9, "chain": 10,
}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            vp, u8p, u64p = ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint64)
            sz, i32, u32, u64 = ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            sig = {
                "orc_init": (i32, []),
                "orc_num_threads": (i32, []),
                "orc_field_op": (i32, [i32, i32, u8p, u8p, u8p]),
                "orc_g1_generator": (None, [u8p]),
                "orc_g2_generator": (None, [u8p]),
                "orc_g1_on_curve": (i32, [u8p]),
                "orc_g2_on_curve": (i32, [u8p]),
                "orc_g1_add": (i32, [u8p, u8p, u8p]),
                "orc_g2_add": (i32, [u8p, u8p, u8p]),
                "orc_g1_mul": (i32, [u8p, u8p, u8p]),
                "orc_g2_mul": (i32, [u8p, u8p, u8p]),
                "orc_g1_mul_gen_batch": (i32, [u8p, u8p, sz]),
                "orc_g2_mul_gen_batch": (i32, [u8p, u8p, sz]),
                "orc_gen_tab_mul": (i32, [u8p, u8p, i32]),
                "orc_pairing": (i32, [u8p, u8p, u8p]),
                "orc_fp12_mul": (i32, [u8p, u8p, u8p]),
                "orc_fp12_pow": (i32, [u8p, u8p, u8p]),
                "orc_untwist_on_curve": (i32, [u8p]),
                "orc_fr_root_of_unity": (None, [u8p, u32]),
                "orc_ntt": (i32, [u8p, u32, i32]),
                "orc_coset_ntt": (i32, [u8p, u32, u32, i32]),
                "orc_msm_g1": (i32, [u8p, u8p, u8p, sz, i32]),
                "orc_msm_g2": (i32, [u8p, u8p, u8p, sz, i32]),
                "orc_splitmix64": (None, [u64, u64, sz, u64p]),
                "orc_sample_fr": (None, [u64, u64, sz, u8p]),
                "orc_rs_from_seed": (None, [u64, u8p, u8p]),
                "orc_circuit_new": (vp, [u32, u32, u32, u32, u32, u64, i32, u64]),
                "orc_circuit_free": (None, [vp]),
                "orc_circuit_info": (None, [vp, u64p]),
                "orc_circuit_witness": (i32, [vp, u8p]),
                "orc_circuit_row": (ctypes.c_long, [vp, i32, sz, ctypes.POINTER(ctypes.c_uint32), u8p, sz]),
                "orc_circuit_constants": (None, [vp, u8p, u8p]),
                "orc_r1cs_check": (i32, [vp, u8p]),
                "orc_spmv": (i32, [vp, u8p, u8p, u8p, u8p]),
                "orc_qap_h": (i32, [vp, u8p, u8p]),
                "orc_setup": (vp, [vp, u64, i32]),
                "orc_pk_free": (None, [vp]),
                "orc_pk_scalar": (i32, [vp, i32, sz, u8p]),
                "orc_pk_point": (i32, [vp, i32, sz, u8p]),
                "orc_prove": (i32, [vp, u8p, u8p, u8p, i32, u8p]),
                "orc_expected_proof": (i32, [vp, u8p, u8p, u8p, u8p]),
                "orc_verify": (i32, [vp, u8p, u8p]),
                "orc_rows_per_perm": (sz, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            L.orc_init()
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# encoding helpers
# --------------------------------------------------------------------------

def to32(x: int) -> bytes:
    return int(x).to_bytes(32, "little")


def from32(b: bytes) -> int:
    return int.from_bytes(bytes(b[:32]), "little")


def g1_bytes(pt) -> bytes:
    """(x, y) ints -> 64 bytes; None -> infinity."""
    if pt is None:
        return bytes(64)
    return to32(pt[0]) + to32(pt[1])


def g1_from(b: bytes):
    b = bytes(b)
    if b == bytes(64):
        return None
    return (from32(b[:32]), from32(b[32:64]))


def g2_bytes(pt) -> bytes:
    """((x0, x1), (y0, y1)) -> 128 bytes; None -> infinity."""
    if pt is None:
        return bytes(128)
    (x0, x1), (y0, y1) = pt
    return to32(x0) + to32(x1) + to32(y0) + to32(y1)


def g2_from(b: bytes):
    b = bytes(b)
    if b == bytes(128):
        return None
    v = [from32(b[32 * i:32 * i + 32]) for i in range(4)]
    return ((v[0], v[1]), (v[2], v[3]))


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------

def field_op(which: str, op: str, a: int, b: int = 0) -> int:
    ops = {"add": 0, "sub": 1, "mul": 2, "inv": 3, "neg": 4, "pow": 5}
    out = ctypes.create_string_buffer(32)
    rc = lib().orc_field_op(1 if which == "fr" else 0, ops[op], out, to32(a), to32(b))
    if rc != 0:
        raise ValueError("non-canonical field input")
    return from32(out.raw)


def g1_generator() -> bytes:
    out = ctypes.create_string_buffer(64)
    lib().orc_g1_generator(out)
    return out.raw


def g2_generator() -> bytes:
    out = ctypes.create_string_buffer(128)
    lib().orc_g2_generator(out)
    return out.raw


def g1_add(a: bytes, b: bytes) -> bytes:
    out = ctypes.create_string_buffer(64)
    assert lib().orc_g1_add(out, a, b) == 0
    return out.raw


def g2_add(a: bytes, b: bytes) -> bytes:
    out = ctypes.create_string_buffer(128)
    assert lib().orc_g2_add(out, a, b) == 0
    return out.raw


def g1_mul(a: bytes, k: int) -> bytes:
    out = ctypes.create_string_buffer(64)
    assert lib().orc_g1_mul(out, a, to32(k)) == 0
    return out.raw


def g2_mul(a: bytes, k: int) -> bytes:
    out = ctypes.create_string_buffer(128)
    assert lib().orc_g2_mul(out, a, to32(k)) == 0
    return out.raw


def g1_on_curve(a: bytes) -> bool:
    return lib().orc_g1_on_curve(a) == 1


def g2_on_curve(a: bytes) -> bool:
    return lib().orc_g2_on_curve(a) == 1


def g1_mul_gen_batch(scalars: bytes) -> bytes:
    n = len(scalars) // 32
    out = ctypes.create_string_buffer(64 * n)
    assert lib().orc_g1_mul_gen_batch(out, scalars, n) == 0
    return out.raw


def g2_mul_gen_batch(scalars: bytes) -> bytes:
    n = len(scalars) // 32
    out = ctypes.create_string_buffer(128 * n)
    assert lib().orc_g2_mul_gen_batch(out, scalars, n) == 0
    return out.raw


def gen_tab_mul(k: int, group: int = 1) -> bytes:
    """k G (G1 or G2 generator) by the setup's fixed-base windowing."""
    out = ctypes.create_string_buffer(64 if group == 1 else 128)
    assert lib().orc_gen_tab_mul(out, to32(k), group) == 0
    return out.raw


def pairing(g1: bytes, g2: bytes) -> bytes:
    out = ctypes.create_string_buffer(384)
    assert lib().orc_pairing(out, g1, g2) == 0
    return out.raw


def fp12_mul(a: bytes, b: bytes) -> bytes:
    out = ctypes.create_string_buffer(384)
    assert lib().orc_fp12_mul(out, a, b) == 0
    return out.raw


def fp12_pow(a: bytes, k: int) -> bytes:
    out = ctypes.create_string_buffer(384)
    assert lib().orc_fp12_pow(out, a, to32(k)) == 0
    return out.raw


FP12_ONE = to32(1) + bytes(32 * 11)


def untwist_on_curve(g2: bytes) -> bool:
    return lib().orc_untwist_on_curve(g2) == 1


def fr_root_of_unity(log_n: int) -> int:
    out = ctypes.create_string_buffer(32)
    lib().orc_fr_root_of_unity(out, log_n)
    return from32(out.raw)


def ntt(values: bytes, log_n: int, inverse: bool = False) -> bytes:
    buf = ctypes.create_string_buffer(bytes(values), len(values))
    assert lib().orc_ntt(buf, log_n, 1 if inverse else 0) == 0
    return buf.raw


def coset_ntt(values: bytes, log_n: int, g: int = 5, inverse: bool = False) -> bytes:
    """Transform on the coset g H: forward gives the values sum_i a_i (g w^j)^i
    at g w^j; inverse gives the coefficients whose values on g H are the
    input (iNTT then a_i g^-i).  Canonical 32-byte values in and out."""
    buf = ctypes.create_string_buffer(bytes(values), len(values))
    rc = lib().orc_coset_ntt(buf, log_n, g, 1 if inverse else 0)
    if rc != 0:
        raise ValueError("coset_ntt: non-canonical input or g = 0")
    return buf.raw


def msm_g1(points: bytes, scalars: bytes, method: int = 1) -> bytes:
    n = len(scalars) // 32
    assert len(points) == 64 * n
    out = ctypes.create_string_buffer(64)
    assert lib().orc_msm_g1(out, points, scalars, n, method) == 0
    return out.raw


def msm_g2(points: bytes, scalars: bytes, method: int = 1) -> bytes:
    n = len(scalars) // 32
    assert len(points) == 128 * n
    out = ctypes.create_string_buffer(128)
    assert lib().orc_msm_g2(out, points, scalars, n, method) == 0
    return out.raw


def splitmix64(seed: int, purpose: int, n: int):
    arr = (ctypes.c_uint64 * n)()
    lib().orc_splitmix64(seed, purpose, n, arr)
    return list(arr)


def sample_fr(seed: int, purpose: int, n: int) -> bytes:
    out = ctypes.create_string_buffer(32 * n)
    lib().orc_sample_fr(seed, purpose, n, out)
    return out.raw


def rs_from_seed(seed: int):
    r = ctypes.create_string_buffer(32)
    s = ctypes.create_string_buffer(32)
    lib().orc_rs_from_seed(seed, r, s)
    return r.raw, s.raw


def rows_per_perm() -> int:
    return int(lib().orc_rows_per_perm())


class Circuit:
    """Synthetic R1CS (Poseidon-style permutations, packing rows, chain)."""

    def __init__(self, log_n, n_rows, n_perm, n_pack=0, pack_bits=0, seed=1,
                 input_seed=None):
        L = lib()
        self.params = (log_n, n_rows, n_perm, n_pack, pack_bits, seed)
        self.input_seed = input_seed
        h = L.orc_circuit_new(log_n, n_rows, n_perm, n_pack, pack_bits, seed,
                              1 if input_seed is not None else 0,
                              input_seed if input_seed is not None else 0)
        if not h:
            raise ValueError("invalid circuit parameters")
        self.h = h
        info = (ctypes.c_uint64 * 8)()
        L.orc_circuit_info(h, info)
        (self.N, self.m, self.n_rows, self.n_chain, self.nnz_a, self.nnz_b,
         self.nnz_c, self.rows_per_perm) = [int(v) for v in info]

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_circuit_free(h)
            self.h = None

    def witness(self) -> bytes:
        out = ctypes.create_string_buffer(32 * self.m)
        assert lib().orc_circuit_witness(self.h, out) == 0
        return out.raw

    def row(self, k: int, i: int):
        L = lib()
        n = L.orc_circuit_row(self.h, k, i, None, None, 0)
        cols = (ctypes.c_uint32 * max(n, 1))()
        vals = ctypes.create_string_buffer(32 * max(n, 1))
        L.orc_circuit_row(self.h, k, i, cols, vals, n)
        return [(int(cols[t]), from32(vals.raw[32 * t:32 * t + 32])) for t in range(n)]

    def constants(self):
        rc = ctypes.create_string_buffer(32 * 65 * 3)
        mds = ctypes.create_string_buffer(32 * 9)
        lib().orc_circuit_constants(self.h, rc, mds)
        rcv = [[from32(rc.raw[32 * (3 * r + l):]) for l in range(3)] for r in range(65)]
        m = [[from32(mds.raw[32 * (3 * i + j):]) for j in range(3)] for i in range(3)]
        return rcv, m

    def r1cs_check(self, z: bytes) -> bool:
        rc = lib().orc_r1cs_check(self.h, z)
        if rc < 0:
            raise ValueError("bad witness encoding")
        return rc == 1

    def spmv(self, z: bytes):
        a = ctypes.create_string_buffer(32 * self.N)
        b = ctypes.create_string_buffer(32 * self.N)
        c = ctypes.create_string_buffer(32 * self.N)
        assert lib().orc_spmv(self.h, z, a, b, c) == 0
        return a.raw, b.raw, c.raw

    def qap_h(self, z: bytes):
        out = ctypes.create_string_buffer(32 * self.N)
        ok = lib().orc_qap_h(self.h, z, out)
        return ok == 1, out.raw


class ProvingKey:
    """Toy setup from seeded toxic waste; points only when with_points."""

    def __init__(self, circuit: Circuit, toxic_seed: int, with_points: bool = True):
        self.circuit = circuit
        self.h = lib().orc_setup(circuit.h, toxic_seed, 1 if with_points else 0)
        self.with_points = with_points

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_pk_free(h)
            self.h = None

    QUERY = {"u": 0, "v": 1, "w": 2, "l": 3, "h": 4, "toxic": 5}
    POINT = {"A": 0, "B1": 1, "B2": 2, "L": 3, "H": 4, "fixed": 5}

    def scalar(self, query: str, idx: int) -> int:
        out = ctypes.create_string_buffer(32)
        assert lib().orc_pk_scalar(self.h, self.QUERY[query], idx, out) == 0
        return from32(out.raw)

    def point(self, query: str, idx: int) -> bytes:
        g2 = query == "B2" or (query == "fixed" and idx in (3, 4, 5))
        out = ctypes.create_string_buffer(128 if g2 else 64)
        assert lib().orc_pk_point(self.h, self.POINT[query], idx, out) == 0
        return out.raw

    def prove(self, z: bytes, r: bytes, s: bytes, method: int = 1):
        out = ctypes.create_string_buffer(256)
        rc = lib().orc_prove(self.h, z, r, s, method, out)
        if rc < 0:
            raise ValueError("prove: bad input or pk without points")
        return (rc == 1), out.raw

    def expected_proof(self, z: bytes, r: bytes, s: bytes) -> bytes:
        out = ctypes.create_string_buffer(256)
        assert lib().orc_expected_proof(self.h, z, r, s, out) == 0
        return out.raw

    def verify(self, public: int, proof: bytes) -> int:
        return int(lib().orc_verify(self.h, to32(public), proof))
