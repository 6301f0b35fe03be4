"""GB300 (sm_103a) Groth16/BN254 prover: Python binding of libace.so.

This module only marshals arguments: every step of the proving path runs in
the CUDA kernels of ``libace.so`` (built in-tree by ``build.py``).  Device
memory and streams come from PyTorch; the library never falls back to the CPU
and importing a function here fails loudly if the extension is missing.

The C ABI is declared in ``include/ace.h``; the names below mirror it.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libace.so")

ACE_OK = 0
ERRORS = {-1: "ACE_E_ARG", -2: "ACE_E_OOM", -3: "ACE_E_CUDA", -4: "ACE_E_UNSAT",
          -5: "ACE_E_NOT_ON_CURVE", -6: "ACE_E_TIMEOUT", -7: "ACE_E_BUSY", -8: "ACE_E_INTERNAL"}
FORM_CANONICAL = 0
FORM_MONT = 1
INFO_LEN = 12

_lib = None


class AceError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """Load libace.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libace.so not built ({LIB_PATH}); run paper_2603_10242_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i32, u32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
        cp = ctypes.c_char_p
        sigs = {
            "ace_last_error": (ctypes.c_char_p, []),
            "ace_ctx_create": (i32, [ctypes.POINTER(vp), i32, sz]),
            "ace_ctx_destroy": (i32, [vp]),
            "ace_ctx_device_bytes": (i32, [vp, ctypes.POINTER(sz)]),
            "ace_msm_g1": (i32, [vp, vp, i32, vp, sz, vp, vp]),
            "ace_msm_g2": (i32, [vp, vp, i32, vp, sz, vp, vp]),
            "ace_msm_g1_window": (i32, [vp, vp, i32, vp, sz, i32, vp, vp]),
            "ace_msm_g1_glv_window": (i32, [vp, vp, i32, vp, sz, i32, vp, vp]),
            "ace_msm_g2_gls_window": (i32, [vp, vp, i32, vp, sz, i32, vp, vp]),
            "ace_msm_g1_noalloc": (i32, [vp, i32, vp, sz, vp, vp]),
            "ace_g1_fixed_base": (i32, [vp, vp, sz, vp, i32, vp]),
            "ace_g2_fixed_base": (i32, [vp, vp, sz, vp, i32, vp]),
            "ace_debug_field_op": (i32, [i32, i32, vp, vp, vp, sz, vp]),
            "ace_debug_curve_op": (i32, [i32, i32, vp, vp, vp, vp, sz, vp]),
            "ace_ntt": (i32, [vp, vp, u32, i32, vp]),
            "ace_ntt_mont": (i32, [vp, vp, u32, i32, i32, i32, vp]),
            "ace_circuit_gen": (i32, [vp, ctypes.POINTER(vp)]),
            "ace_circuit_free": (i32, [vp]),
            "ace_circuit_info": (i32, [vp, ctypes.POINTER(u64)]),
            "ace_witness": (i32, [vp, u64, vp, sz]),
            "ace_setup_toy": (i32, [vp, vp, u64, ctypes.POINTER(vp), vp]),
            "ace_pk_free": (i32, [vp]),
            "ace_pk_info": (i32, [vp, ctypes.POINTER(u64)]),
            "ace_pk_point": (i32, [vp, i32, sz, vp]),
            "ace_qap_h": (i32, [vp, vp, vp, vp, vp]),
            "ace_prove": (i32, [vp, vp, vp, vp, vp, vp, vp]),
            "ace_prove_async": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
            "ace_rs_from_seed": (i32, [u64, vp, vp]),
            "ace_verify": (i32, [vp, vp, sz, vp]),
            "ace_prove_batch": (i32, [vp, sz, vp, vp, vp, vp, vp, vp]),
            "ace_prove_batch_host": (i32, [vp, sz, vp, vp, vp, vp, vp, vp]),
            "ace_pk_save": (i32, [vp, cp]),
            "ace_pk_load": (i32, [vp, cp, ctypes.POINTER(vp), vp]),
            "ace_debug_pairing": (i32, [cp, cp, cp]),
            "ace_prove_many": (i32, [vp, vp, sz, vp, cp, cp, vp, vp]),
            "ace_witness_many": (i32, [vp, vp, sz, vp, vp, vp]),
            "ace_verify_batch": (i32, [vp, vp, sz, cp, cp, u64]),
            "ace_debug_pairing_form": (i32, [i32, cp, cp, cp]),
            "ace_debug_glv_split": (i32, [cp, vp]),
            "ace_debug_wnaf5": (i32, [vp, vp]),
            "ace_debug_gls_split": (i32, [cp, vp]),
            "ace_debug_msm_plan": (i32, [sz, i32, i32, vp]),
            "ace_autotune_msm": (i32, [vp, u32, u32, vp]),
            "ace_autotune_ntt": (i32, [vp, u32, u32, vp]),
            "ace_autotune_batch_slots": (i32, [vp, vp, vp, i32, i32, vp]),
            "ace_autotune_save": (i32, [vp, cp]),
            "ace_autotune_load": (i32, [vp, cp]),
            "ace_server_create": (i32, [vp, vp, i32, sz, ctypes.c_double, ctypes.POINTER(vp)]),
            "ace_server_submit": (i32, [vp, vp, vp, cp, cp, ctypes.POINTER(u64)]),
            "ace_server_poll": (i32, [vp, u64, vp, ctypes.POINTER(ctypes.c_double)]),
            "ace_server_wait": (i32, [vp, u64, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_double]),
            "ace_server_stats": (i32, [vp, ctypes.POINTER(u64)]),
            "ace_server_destroy": (i32, [vp]),
            "ace_debug_scheduler_sim": (i32, [i32, sz, sz, vp, vp, vp, ctypes.c_double, vp, vp, vp,
                                              ctypes.POINTER(u64), vp]),
            "ace_debug_imad_rate": (i32, [vp, i32, ctypes.POINTER(ctypes.c_double)]),
            "ace_debug_chain_latency": (i32, [vp, i32, ctypes.POINTER(ctypes.c_double)]),
            "ace_debug_mul_rate": (i32, [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_uint32)]),
            "ace_launch_count": (i32, [ctypes.POINTER(u64)]),
            "ace_profile_enable": (i32, [i32]),
            "ace_profile_read": (i32, [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64),
                                       ctypes.POINTER(u64)]),
            "ace_profile_read_sum": (i32, [i32, ctypes.POINTER(ctypes.c_double)]),
            "ace_debug_serial_proofs": (i32, [vp, i32]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> int:
    if rc < 0:
        raise AceError(rc, lib().ace_last_error().decode(errors="replace"))
    return rc


def _ptr(t) -> int:
    """Device (or host) address of a torch tensor, or an int address."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    """cudaStream_t handle: the given stream, else PyTorch's current stream
    (NULL selects the context's stream, which is ordered with the legacy
    default stream)."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                h = torch.cuda.current_stream().cuda_stream
                return h or None
        except Exception:
            return None
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


class Context:
    """ace_ctx: one CUDA device, its stream, scratch arenas and caches."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        check(lib().ace_ctx_create(ctypes.byref(h), device, hbm_budget_bytes))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().ace_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        check(lib().ace_ctx_device_bytes(self.h, ctypes.byref(v)))
        return v.value

    # ---- hot path ----
    def msm_g1(self, bases, scalars, n: int, out, base_form: int = FORM_CANONICAL, stream=None):
        check(lib().ace_msm_g1(self.h, _ptr(bases), base_form, _ptr(scalars), n, _ptr(out), _stream(stream)))

    def msm_g2(self, bases, scalars, n: int, out, base_form: int = FORM_CANONICAL, stream=None):
        check(lib().ace_msm_g2(self.h, _ptr(bases), base_form, _ptr(scalars), n, _ptr(out), _stream(stream)))

    def msm_g1_window(self, bases, scalars, n: int, c: int, out, base_form: int = FORM_CANONICAL, stream=None):
        check(lib().ace_msm_g1_window(self.h, _ptr(bases), base_form, _ptr(scalars), n, c, _ptr(out),
                                      _stream(stream)))

    def msm_g1_glv_window(self, bases, scalars, n: int, c: int, out, base_form: int = FORM_CANONICAL, stream=None):
        check(lib().ace_msm_g1_glv_window(self.h, _ptr(bases), base_form, _ptr(scalars), n, c, _ptr(out),
                                          _stream(stream)))

    def msm_g2_gls_window(self, bases, scalars, n: int, c: int, out, base_form: int = FORM_CANONICAL, stream=None):
        check(lib().ace_msm_g2_gls_window(self.h, _ptr(bases), base_form, _ptr(scalars), n, c, _ptr(out),
                                          _stream(stream)))

    def g1_fixed_base(self, scalars, n: int, out, out_form: int = FORM_CANONICAL, stream=None):
        check(lib().ace_g1_fixed_base(self.h, _ptr(scalars), n, _ptr(out), out_form, _stream(stream)))

    def g2_fixed_base(self, scalars, n: int, out, out_form: int = FORM_CANONICAL, stream=None):
        check(lib().ace_g2_fixed_base(self.h, _ptr(scalars), n, _ptr(out), out_form, _stream(stream)))

    def ntt(self, data, log_n: int, kind: int, stream=None):
        """kind: 0 forward, 1 inverse, 2 coset forward, 3 coset inverse (canonical, natural order)."""
        check(lib().ace_ntt(self.h, _ptr(data), log_n, kind, _stream(stream)))

    def ntt_mont(self, data, log_n: int, count: int, dif: bool, inverse: bool, stream=None):
        check(lib().ace_ntt_mont(self.h, _ptr(data), log_n, count, 1 if dif else 0, 1 if inverse else 0,
                                 _stream(stream)))

    def witness_many(self, circuit: "Circuit", seeds, d_z, stream=None):
        """Witnesses of len(seeds) instances into d_z (k x m canonical values) on the device."""
        k = len(seeds)
        arr = (ctypes.c_uint64 * max(1, k))(*seeds)
        check(lib().ace_witness_many(self.h, circuit.h, k, arr, _ptr(d_z), _stream(stream)))

    def verify_batch(self, vk: "VerifyingKey", pubs: bytes, proofs: bytes, seed: int) -> int:
        """1 if all len(proofs) / 256 proofs verify (random linear combination), else 0."""
        k = len(proofs) // 256
        return check(lib().ace_verify_batch(self.h, ctypes.byref(vk), k, pubs, proofs, seed))

    def prove_many(self, pk: "ProvingKey", d_z, k: int, rs: bytes, ss: bytes):
        """k proofs of one key in one pass; d_z holds the k witnesses back to back."""
        proofs = ctypes.create_string_buffer(256 * k)
        status = (ctypes.c_int32 * k)()
        check(lib().ace_prove_many(self.h, pk.h, k, _ptr(d_z), rs, ss, proofs, status))
        return [proofs.raw[256 * i:256 * i + 256] for i in range(k)], list(status)

    # ---- autotuning ----
    def autotune_msm(self, log_min: int, log_max: int):
        n = log_max - log_min + 1
        rep = (ctypes.c_double * (5 * n))()
        check(lib().ace_autotune_msm(self.h, log_min, log_max, rep))
        return [tuple(rep[5 * i:5 * i + 5]) for i in range(n)]

    def autotune_ntt(self, log_min: int, log_max: int):
        n = log_max - log_min + 1
        rep = (ctypes.c_double * (5 * n))()
        check(lib().ace_autotune_ntt(self.h, log_min, log_max, rep))
        return [tuple(rep[5 * i:5 * i + 5]) for i in range(n)]

    def autotune_batch_slots(self, pk: "ProvingKey", d_z, k: int, max_slots: int = 4):
        """ms per batch: [1..max_slots slots, MSMs on auxiliary streams] +
        [1..max_slots slots, one stream per proof]."""
        rep = (ctypes.c_double * (2 * max_slots))()
        check(lib().ace_autotune_batch_slots(self.h, pk.h, _ptr(d_z), k, max_slots, rep))
        return list(rep)

    def autotune_save(self, path: str):
        check(lib().ace_autotune_save(self.h, path.encode()))

    def autotune_load(self, path: str):
        check(lib().ace_autotune_load(self.h, path.encode()))

    def qap_h(self, pk: "ProvingKey", d_z, d_h, stream=None):
        check(lib().ace_qap_h(self.h, pk.h, _ptr(d_z), _ptr(d_h), _stream(stream)))

    def prove(self, pk: "ProvingKey", d_z, r: bytes, s: bytes, stream=None) -> bytes:
        out = ctypes.create_string_buffer(256)
        check(lib().ace_prove(self.h, pk.h, _ptr(d_z), r, s, out, _stream(stream)))
        return out.raw

    def prove_async(self, pk: "ProvingKey", d_z, r: bytes, s: bytes, d_proof, d_status, stream=None):
        check(lib().ace_prove_async(self.h, pk.h, _ptr(d_z), r, s, _ptr(d_proof), _ptr(d_status),
                                    _stream(stream)))

    def prove_batch(self, pks, d_zs, rs: bytes, ss: bytes):
        k = len(pks)
        pk_arr = (ctypes.c_void_p * k)(*[p.h.value for p in pks])
        z_arr = (ctypes.c_void_p * k)(*[_ptr(z) for z in d_zs])
        proofs = ctypes.create_string_buffer(256 * k)
        status = (ctypes.c_int32 * k)()
        check(lib().ace_prove_batch(self.h, k, pk_arr, z_arr, rs, ss, proofs, status))
        return [proofs.raw[256 * i:256 * i + 256] for i in range(k)], list(status)

    def prove_batch_host(self, pks, h_zs, rs: bytes, ss: bytes):
        """ace_prove_batch with witnesses in host memory (CPU tensors, pinned
        for overlapped copies); the library copies them to the device."""
        k = len(pks)
        for z in h_zs:
            if getattr(z, "is_cuda", False):
                raise ValueError("prove_batch_host takes host witnesses")
        pk_arr = (ctypes.c_void_p * k)(*[p.h.value for p in pks])
        z_arr = (ctypes.c_void_p * k)(*[_ptr(z) for z in h_zs])
        proofs = ctypes.create_string_buffer(256 * k)
        status = (ctypes.c_int32 * k)()
        check(lib().ace_prove_batch_host(self.h, k, pk_arr, z_arr, rs, ss, proofs, status))
        return [proofs.raw[256 * i:256 * i + 256] for i in range(k)], list(status)


def msm_g1_noalloc(bases, scalars, n: int, out, base_form: int = FORM_CANONICAL, stream=None):
    """G1 MSM without any device allocation (n <= 16384); see include/ace.h."""
    check(lib().ace_msm_g1_noalloc(_ptr(bases), base_form, _ptr(scalars), n, _ptr(out), _stream(stream)))


# ---- diagnostics (device element-wise arithmetic) ----
def debug_field_op(field: int, op: int, d_a, d_b, d_out, n: int, stream=None):
    check(lib().ace_debug_field_op(field, op, _ptr(d_a), _ptr(d_b), _ptr(d_out), n, _stream(stream)))


def debug_curve_op(group: int, op: int, d_a, d_b, d_k, d_out, n: int, stream=None):
    check(lib().ace_debug_curve_op(group, op, _ptr(d_a), _ptr(d_b), _ptr(d_k), _ptr(d_out), n, _stream(stream)))


MSM_FULL, MSM_TABLED, MSM_GLV, MSM_GLS = 0, 1, 2, 3


def msm_plan(n: int, kind: int, force_c: int = 0) -> dict:
    """The MSM plan the library picks for n points (host only)."""
    out = (ctypes.c_uint32 * 8)()
    check(lib().ace_debug_msm_plan(n, kind, force_c, out))
    keys = ("c", "K", "B", "windows", "L", "M", "ones_buckets", "points")
    return dict(zip(keys, list(out)))


class CircuitParams(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_rows", ctypes.c_uint32), ("n_perm", ctypes.c_uint32),
                ("n_pack", ctypes.c_uint32), ("pack_bits", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class Circuit:
    """ace_circuit: the seeded synthetic R1CS (host)."""

    def __init__(self, log_n, n_rows, n_perm, n_pack=0, pack_bits=0, seed=1):
        self.params = CircuitParams(log_n, n_rows, n_perm, n_pack, pack_bits, seed)
        h = ctypes.c_void_p()
        check(lib().ace_circuit_gen(ctypes.byref(self.params), ctypes.byref(h)))
        self.h = h
        info = (ctypes.c_uint64 * INFO_LEN)()
        check(lib().ace_circuit_info(h, info))
        self.info = list(info)
        self.N, self.m = int(info[0]), int(info[1])

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None and self.h.value:
                lib().ace_circuit_free(self.h)
                self.h = None
        except Exception:
            pass

    def witness(self, input_seed: int) -> bytes:
        out = ctypes.create_string_buffer(32 * self.m)
        check(lib().ace_witness(self.h, input_seed, out, self.m))
        return out.raw


class VerifyingKey(ctypes.Structure):
    _fields_ = [("alpha1", ctypes.c_uint8 * 64), ("beta2", ctypes.c_uint8 * 128), ("gamma2", ctypes.c_uint8 * 128),
                ("delta2", ctypes.c_uint8 * 128), ("ic", ctypes.c_uint8 * 128)]


class ProvingKey:
    """ace_pk: device-resident proving key from the toy setup."""

    def __init__(self, ctx: Context, circuit: Circuit | None, toxic_seed: int = 0, _handle=None, vk=None):
        self.ctx = ctx
        self.circuit = circuit
        if _handle is not None:
            self.h, self.vk = _handle, vk
        else:
            h = ctypes.c_void_p()
            self.vk = VerifyingKey()
            check(lib().ace_setup_toy(ctx.h, circuit.h, toxic_seed, ctypes.byref(h), ctypes.byref(self.vk)))
            self.h = h
        info = (ctypes.c_uint64 * INFO_LEN)()
        check(lib().ace_pk_info(self.h, info))
        self.info = list(info)
        self.N, self.m = int(info[0]), int(info[1])

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().ace_pk_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    QUERY = {"A": 0, "B1": 1, "B2": 2, "L": 3, "H": 4}

    def point(self, query: str, idx: int) -> bytes:
        out = ctypes.create_string_buffer(128 if query == "B2" else 64)
        check(lib().ace_pk_point(self.h, self.QUERY[query], idx, out))
        return out.raw

    def save(self, path: str):
        check(lib().ace_pk_save(self.h, path.encode()))

    @classmethod
    def load(cls, ctx: Context, path: str) -> "ProvingKey":
        h = ctypes.c_void_p()
        vk = VerifyingKey()
        check(lib().ace_pk_load(ctx.h, path.encode(), ctypes.byref(h), ctypes.byref(vk)))
        return cls(ctx, None, _handle=h, vk=vk)

    def verify(self, public: bytes, proof: bytes) -> int:
        return check(lib().ace_verify(ctypes.byref(self.vk), public, 1, proof))


def rs_from_seed(seed: int):
    r = ctypes.create_string_buffer(32)
    s = ctypes.create_string_buffer(32)
    check(lib().ace_rs_from_seed(seed, r, s))
    return r.raw, s.raw


def verify(vk: VerifyingKey, public: bytes, proof: bytes) -> int:
    return check(lib().ace_verify(ctypes.byref(vk), public, 1, proof))


# ---- measurement hooks ----
PROF_G1_BUCKET, PROF_G2_BUCKET, PROF_NTT, PROF_SPMV = 0, 1, 2, 3
PROF_SORT, PROF_REDUCE, PROF_ASSEMBLY = 4, 5, 6


def launch_count() -> int:
    v = ctypes.c_uint64()
    check(lib().ace_launch_count(ctypes.byref(v)))
    return v.value


def profile_enable(on: bool = True):
    check(lib().ace_profile_enable(1 if on else 0))


def profile_read_sum(kind: int) -> float:
    """Total length (ms) of one kind's launch intervals since enabling."""
    v = ctypes.c_double()
    check(lib().ace_profile_read_sum(kind, ctypes.byref(v)))
    return v.value


def serial_proofs(ctx: "Context", on: bool):
    """Measurement mode: later proofs on ctx run every stage on one stream."""
    check(lib().ace_debug_serial_proofs(ctx.h, 1 if on else 0))


def profile_read(kind: int):
    """(ms, launches, units) for one profiled kernel kind since enabling."""
    ms, n, u = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().ace_profile_read(kind, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(u)))
    return ms.value, n.value, u.value


def imad_rate(ctx: Context, mode: int) -> float:
    v = ctypes.c_double()
    check(lib().ace_debug_imad_rate(ctx.h, mode, ctypes.byref(v)))
    return v.value


def chain_latency_ns(ctx: Context, what: int) -> float:
    v = ctypes.c_double()
    check(lib().ace_debug_chain_latency(ctx.h, what, ctypes.byref(v)))
    return v.value


def mul_rate(ctx: Context, form: int):
    """(products/s, single-thread latency ns, digest) of Montgomery product form 0, 1 or 2."""
    a, b = ctypes.c_double(), ctypes.c_double()
    d = (ctypes.c_uint32 * 4)()
    check(lib().ace_debug_mul_rate(ctx.h, form, ctypes.byref(a), ctypes.byref(b), d))
    return a.value, b.value, list(d)


class Server:
    """ace_server: continuous-batching proof server on its own context."""

    def __init__(self, ctx: Context, max_pk: "ProvingKey", slots: int = 2, hbm_budget_bytes: int = 0,
                 max_queue_wait_s: float = 0.0):
        h = ctypes.c_void_p()
        check(lib().ace_server_create(ctx.h, max_pk.h, slots, hbm_budget_bytes, max_queue_wait_s, ctypes.byref(h)))
        self.h = h
        # the server thread uses the context until destroyed, and each job its
        # key and host witness until collected: keep them alive that long
        self._ctx, self._max_pk = ctx, max_pk
        self._keep = {}

    def submit(self, pk: "ProvingKey", z_host, r: bytes, s: bytes) -> int:
        """z_host: a host buffer (ctypes buffer or pinned torch tensor) kept alive until collected."""
        jid = ctypes.c_uint64()
        addr = z_host.data_ptr() if hasattr(z_host, "data_ptr") else ctypes.addressof(z_host)
        check(lib().ace_server_submit(self.h, pk.h, addr, r, s, ctypes.byref(jid)))
        self._keep[jid.value] = (z_host, pk)
        return jid.value

    def _result(self, rc, jid, out, lat):
        self._keep.pop(jid, None)
        if rc < 0:
            raise AceError(rc, lib().ace_last_error().decode(errors="replace"))
        return out.raw, lat.value

    def poll(self, jid: int):
        """None while running, else (proof bytes, latency ms); raises on job errors."""
        out = ctypes.create_string_buffer(256)
        lat = ctypes.c_double()
        rc = lib().ace_server_poll(self.h, jid, out, ctypes.byref(lat))
        if rc == -7:
            return None
        return self._result(rc, jid, out, lat)

    def wait(self, jid: int, timeout_s: float = 0.0):
        out = ctypes.create_string_buffer(256)
        lat = ctypes.c_double()
        rc = lib().ace_server_wait(self.h, jid, out, ctypes.byref(lat), timeout_s)
        if rc == -7:
            return None
        return self._result(rc, jid, out, lat)

    def stats(self) -> dict:
        v = (ctypes.c_uint64 * 8)()
        check(lib().ace_server_stats(self.h, v))
        keys = ["submitted", "collected", "timeouts", "waiting", "peak_running", "peak_bytes", "budget", "slots"]
        return dict(zip(keys, [int(x) for x in v]))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().ace_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scheduler_sim(slots: int, budget: int, arrival, duration, mem, max_wait: float = 0.0):
    """Run the server's admission logic on a virtual clock (host only)."""
    n = len(arrival)
    A = (ctypes.c_double * n)(*arrival)
    D = (ctypes.c_double * n)(*duration)
    M = (ctypes.c_size_t * n)(*mem)
    st, fi = (ctypes.c_double * n)(), (ctypes.c_double * n)()
    status = (ctypes.c_int32 * n)()
    peaks = (ctypes.c_uint64 * 2)()
    prio = (ctypes.c_int32 * n)()
    check(lib().ace_debug_scheduler_sim(slots, budget, n, A, D, M, max_wait, st, fi, status, peaks, prio))
    return list(st), list(fi), list(status), (int(peaks[0]), int(peaks[1])), list(prio)
