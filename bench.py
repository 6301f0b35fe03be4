"""Benchmark: Groth16/BN254 proofs/s of the 2^20 block-scale proof on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one whole proof (sparse products + R1CS check, QAP quotient with 7
NTTs, four G1 MSMs and one G2 MSM, assembly) of the block-scale circuit:
N = 2^20 constraints, 2,048 transactions x 2 Poseidon-style permutations,
2 bit-packing rows of 172 bits per transaction (~40% of the witness in {0,1}),
squaring chain up to 2^20.  Inputs (witness, proving key) are resident in HBM
for `value`; `e2e` copies the witness from pinned host memory and reads the
proof back inside every step through the public C ABI.  One JSON line is
printed by rank 0.  Under torchrun each rank proves its own proofs on its own
GPU (independent replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Groth16 proofs/s and G1 MSM points/s at 2^20 (BN254), bit-exact; p99 prove latency"
UNIT = "proofs/s"
WORKLOAD = {
    "workload": "groth16_block_2p20",
    "constraints": 1 << 20,
    "transactions": 2048,
    "permutations": 4096,
    "pack_rows": 4096,
    "pack_bits": 172,
    "curve": "BN254",
}
CIRCUIT = dict(log_n=20, n_rows=1 << 20, n_perm=4096, n_pack=4096, pack_bits=172)
SEED = 2
# Algorithmic cost of one mixed XYZZ addition (madd-2008-s): 8M + 2S field
# multiplications on G1, 8 Fp2 mul (3 Fp mul) + 2 Fp2 sqr (2 Fp mul) on G2;
# one 8-limb Montgomery product = 2 * 8^2 + 8 = 136 limb products = 272
# 32-bit multiply-adds (lo and hi halves).
IMAD_PER_FP_MUL = 272
IMAD_PER_G1_MADD = 10 * IMAD_PER_FP_MUL
IMAD_PER_G2_MADD = 28 * IMAD_PER_FP_MUL
# ALU roofline: SMs x 64 32-bit IMAD per clock per SM x maximum SM clock; the
# SM count is read from the device and the maximum clock from the GPU
# (nvidia-smi), both at run time.
IMAD_PER_CLK_PER_SM = 64
SM_MAX_MHZ_DEFAULT = 2070.0
# DRAM traffic of the dominant kernel from the latest ncu capture of it inside
# the 2^20 block proofs (dram__bytes_read.sum + dram__bytes_write.sum per
# launch, divided by the launch's mixed additions).  It describes one version
# of the kernel: `kernel_version` must match G1_BUCKET_KERNEL_VERSION below,
# otherwise the bench reports traffic as null (the counters predate the code).
G1_BUCKET_KERNEL_VERSION = "xyzz-madd-v2-gather-l2-64b"
G1_BUCKET_TRAFFIC = {
    "kernel_version": "xyzz-madd-v2-gather-l2-64b",
    "bytes_per_unit": 1.0754e9 / 13.619e6,
    "source": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
              "--clock-control none -k regex:k_bucket_acc -c 20 python bench.py --case prove20 --steps 4 "
              "(GB300, the 16 G1 launches of four 2^20 proofs: 1.075 GB per launch for 13.62 M additions, "
              "79 B per addition)",
}


def _device_sms(device) -> int:
    import torch

    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def _sm_max_mhz(clocks) -> float:
    """Maximum SM clock: sampled from nvidia-smi during the run, else the
    driver's measured-peaks record, else the GB300's 2070 MHz."""
    if clocks and clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"])
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return SM_MAX_MHZ_DEFAULT


def _tuned_batch(ctx) -> dict:
    """The batch configuration the library's autotuner kept (proving slots
    and stage layout), read back from its saved choices."""
    import tempfile

    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.json")
        ctx.autotune_save(path)
        t = json.load(open(path))
    return {"slots": t["batch_slots"], "one_stream_per_proof": bool(t.get("batch_one_stream", 0))}


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (x itself without a process
    group): every rank's timed region is bracketed by barriers, and the job
    takes as long as its slowest rank."""
    if not dist:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world_size: int, seconds: float) -> float:
    """Throughput of the whole job: the units all ranks processed (each rank
    proves its own, no data is exchanged) over the slowest rank's time."""
    return world_size * units_per_rank / seconds


# compacted query sizes of the block circuit (m_A, m_B, m_L: witness values
# whose A / B / L setup scalar is non-zero); run_ours checks them against the key
BLOCK_SHAPE = {"N": 1 << 20, "m": 1765375, "m_A": 1748994, "m_B": 712705, "m_L": 1765373}


def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def _clock_summary(path, device):
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
    except OSError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
class OracleBlockProof:
    """The oracle's whole Groth16 proof of the 2^20 block circuit on the host
    cores.  Its circuit, witness and proving key (with points) are made first
    and not timed: the toy setup is not part of a proof.  Each step then times
    one call of the oracle prover: sparse products, the QAP quotient by a
    2N-point convolution and long division by X^N - 1, the A, B1, L and H G1
    MSMs and the B G2 MSM by plain Pippenger, and the assembly.  Same circuit,
    witness, toxic waste and (r, s) as the GPU arm, so its proof bytes equal
    the GPU's."""

    def __init__(self):
        import oracle as O

        self.O = O
        t0 = time.perf_counter()
        self.c = O.Circuit(CIRCUIT["log_n"], CIRCUIT["n_rows"], CIRCUIT["n_perm"], CIRCUIT["n_pack"],
                           CIRCUIT["pack_bits"], seed=SEED, input_seed=SEED)
        self.z = self.c.witness()
        self.pk = O.ProvingKey(self.c, SEED, with_points=True)
        self.setup_s = time.perf_counter() - t0
        self.cores = O.lib().orc_num_threads()
        self.verified = None

    def step(self, i):
        r, s_ = self.O.rs_from_seed(1000 + i)
        t0 = time.perf_counter()
        ok, proof = self.pk.prove(self.z, r, s_, 1)
        dt = time.perf_counter() - t0
        assert ok, "the oracle found the witness unsatisfied"
        if self.verified is None:
            self.verified = self.pk.verify(int.from_bytes(self.z[32:64], "little"), proof) == 1
        return proof, dt

    def record(self, times):
        per = statistics.median(times)
        return {
            "value": 1.0 / per, "unit": UNIT, "cores": self.cores, "kind": "oracle",
            "sample": (f"{len(times)} whole oracle proof(s) of the 2^20 block circuit, timed one by one "
                       f"({', '.join(f'{t:.1f}' for t in times)} s; median {per:.1f} s per proof) after an "
                       f"untimed setup of {self.setup_s:.0f} s; proof verified by the oracle's pairing check: "
                       f"{bool(self.verified)}"),
            "seconds_per_proof": per,
        }


def run_reference(args):
    """The oracle prover on the host cores (rank 0 only).  A proof takes tens
    of seconds, so the arm runs whole proofs until --ref-seconds of proving
    have passed (at least one) and reports the number it ran as `steps`
    (the requested K and W are recorded beside it); no warm-up proof is run,
    the oracle has nothing to warm up."""
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    o = OracleBlockProof()
    times = []
    while not times or (sum(times) < args.ref_seconds and len(times) < args.steps):
        times.append(o.step(len(times))[1])
    rec = o.record(times)
    v = rec["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": 0, "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(WORKLOAD), "cpu_baseline": rec,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import paper_2603_10242_gb300 as ace
    from paper_2603_10242_gb300 import inputs

    ws, rank, local = _dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    device = local if ws > 1 else 0
    torch.cuda.set_device(device)
    ace.build()
    ctx = ace.Context(device)
    circ = ace.Circuit(seed=SEED, **CIRCUIT)
    z = circ.witness(SEED)
    pk = ace.ProvingKey(ctx, circ, toxic_seed=SEED)
    m, N = circ.m, circ.N
    shape = {"N": N, "m": m, "m_A": pk.info[7], "m_B": pk.info[8], "m_L": pk.info[9]}
    assert shape == BLOCK_SHAPE, f"block circuit shape changed: {shape}"
    zb = np.frombuffer(z, dtype=np.uint8)
    bool_frac = float(np.mean((zb.reshape(-1, 32)[:, 1:] == 0).all(axis=1) & (zb.reshape(-1, 32)[:, 0] <= 1)))
    stream = torch.cuda.current_stream(device)
    dz = torch.from_numpy(zb.copy()).to(device)
    proofs = torch.zeros((args.steps + args.warmup) * 256, dtype=torch.uint8, device=device)
    status = torch.zeros(args.steps + args.warmup, dtype=torch.int32, device=device)
    rs = [ace.rs_from_seed(1000 + i) for i in range(args.warmup + args.steps)]

    # correctness of the bench's own proof: verify on the host
    proof0 = ctx.prove(pk, dz, *rs[0])
    verified = pk.verify(z[32:64], proof0) == 1

    rs_all = b"".join(r for r, _ in rs)
    ss_all = b"".join(s_ for _, s_ in rs)

    def batch(k, start):
        return ctx.prove_batch([pk] * k, [dz] * k, rs_all[32 * start:32 * (start + k)],
                               ss_all[32 * start:32 * (start + k)])

    for i in range(args.warmup):
        ctx.prove_async(pk, dz, rs[i][0], rs[i][1], proofs[256 * i:], status[i:])
    # proving slots for the batch: the autotuner times 1..4 slots (untimed)
    slot_ms = ctx.autotune_batch_slots(pk, dz, 6, 4)
    batch_cfg = _tuned_batch(ctx)
    batch(min(4, args.steps), 0)
    torch.cuda.synchronize()

    # ---- timed region: K proofs pipelined over proving slots (one batch call), inputs in HBM ----
    sampler, sf = _clock_sampler(f"/tmp/bench_clocks_{rank}.csv")
    ace.profile_enable(True)
    launches0 = ace.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    bproofs, bstatus = batch(args.steps, args.warmup)
    eb1.record(stream)
    torch.cuda.synchronize()
    launches = ace.launch_count() - launches0
    total_ms = eb0.elapsed_time(eb1)
    prof = {k: ace.profile_read(k) for k in range(7)}
    g1_sum_ms = ace.profile_read_sum(ace.PROF_G1_BUCKET)
    ace.profile_enable(False)
    if sampler:
        sampler.terminate()
        sampler.wait()
        sf.close()
    clocks = _clock_summary(f"/tmp/bench_clocks_{rank}.csv", device)
    assert not any(bstatus), "a batched proof reported an unsatisfied witness"
    for j in (0, args.steps - 1):
        verified = verified and pk.verify(z[32:64], bproofs[j]) == 1
    if dist:
        dist.barrier()

    # ---- plain path: one proof per call, back to back (per-proof latency) ----
    # args.latency_proofs proofs (at least K), each bracketed by CUDA events
    n_lat = max(args.steps, args.latency_proofs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_lat + 1)]
    lat_proofs = torch.zeros(n_lat * 256, dtype=torch.uint8, device=device)
    lat_status = torch.zeros(n_lat, dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(n_lat):
        j = args.warmup + (i % args.steps)
        ctx.prove_async(pk, dz, rs[j][0], rs[j][1], lat_proofs[256 * i:], lat_status[i:])
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(n_lat)]
    plain_ms = ev[0].elapsed_time(ev[args.steps])
    assert int(lat_status.sum().item()) == 0, "a proof reported an unsatisfied witness"
    allp = lat_proofs.cpu().numpy().reshape(-1, 256)
    # the plain path gives the same bytes as the batch for the same (r, s)
    for i in (0, args.steps - 1):
        assert bytes(allp[i]) == bproofs[i], "batched and plain proofs differ"

    total_ms = max_over_ranks(total_ms, dist, device)
    value = whole_job_rate(args.steps, ws, total_ms / 1000.0)
    plain_value = args.steps / (plain_ms / 1000.0)

    # ---- e2e through the public C ABI with host buffers ----
    # ace_prove_batch_host takes the witnesses in pinned host memory, copies
    # each to the device inside the call and returns the proofs and status
    # words in host memory; groups of at most 64 proofs per call
    zpins = [torch.from_numpy(zb.copy()).pin_memory() for _ in range(min(args.steps, 64))]

    def e2e_run(k, start):
        out = []
        for g0 in range(0, k, len(zpins)):
            g = min(len(zpins), k - g0)
            p, st_ = ctx.prove_batch_host([pk] * g, zpins[:g], rs_all[32 * (start + g0):32 * (start + g0 + g)],
                                          ss_all[32 * (start + g0):32 * (start + g0 + g)])
            assert st_ == [0] * g
            out += p
        return out

    e2e_run(min(len(zpins), 4), 0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_proofs = e2e_run(args.steps, args.warmup)
    e2e_s = time.perf_counter() - t0
    assert e2e_proofs == bproofs, "proofs from host witnesses differ from the device-resident batch"
    e2e_s = max_over_ranks(e2e_s, dist, device)
    e2e = {"value": whole_job_rate(args.steps, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 32 * m,
           "d2h_bytes_per_step": 256 + 4, "path": "ace_prove_batch_host (witness in pinned host memory, "
                                                 "proof and status returned to host memory)"}

    # ---- per-stage split: one proof with every stage on one stream ----
    # (untimed for `value`): the profiled intervals then do not overlap, so
    # each stage's time is exclusive and the stages plus `other` (gathers,
    # quotient, bucket combine, memsets, gaps between launches) add up to the
    # proof's serial time
    ace.serial_proofs(ctx, True)
    r0, s_0 = rs[args.warmup]  # the (r, s) of bproofs[0]
    ctx.prove_async(pk, dz, r0, s_0, proofs, status)
    torch.cuda.synchronize()
    ace.profile_enable(True)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    ctx.prove_async(pk, dz, r0, s_0, proofs, status)
    s1.record(stream)
    torch.cuda.synchronize()
    serial_ms = s0.elapsed_time(s1)
    names = {ace.PROF_SPMV: "spmv_r1cs_check", ace.PROF_NTT: "ntt_passes", ace.PROF_SORT: "msm_digit_sort",
             ace.PROF_G1_BUCKET: "g1_bucket_acc", ace.PROF_G2_BUCKET: "g2_bucket_acc",
             ace.PROF_REDUCE: "msm_bucket_reduce_and_final", ace.PROF_ASSEMBLY: "assembly_fixed_var_terms"}
    stages = {v: ace.profile_read(k)[0] for k, v in names.items()}
    stages["other"] = serial_ms - sum(stages.values())
    stages = {"serial_proof_ms": serial_ms, "exclusive_ms": stages,
              "how": "one 2^20 proof with every stage on the slot's main stream (ace_debug_serial_proofs), "
                     "CUDA events around each stage; the batched step overlaps these stages across streams "
                     "and proofs"}
    ace.profile_enable(False)
    ace.serial_proofs(ctx, False)
    assert bytes(proofs[:256].cpu().numpy().tobytes()) == bproofs[0], "serial proof differs"

    # ---- G1 MSM points/s at 2^20 (second half of the metric) ----
    n = 1 << 20
    kb = inputs.sample_fr(20, inputs.PURPOSE["bases"], n)
    bases = torch.empty(64 * n, dtype=torch.uint8, device=device)
    ctx.g1_fixed_base(torch.from_numpy(kb.view(np.uint8).reshape(-1)).to(device), n, bases, ace.FORM_MONT)
    msm = {}
    iso = None
    for dist_name in ("uniform", "sparse"):
        sc = torch.from_numpy(inputs.sample_scalars(20, n, dist_name).view(np.uint8).reshape(-1)).to(device)
        out = torch.empty(64, dtype=torch.uint8, device=device)
        for _ in range(3):
            ctx.msm_g1(bases, sc, n, out, ace.FORM_MONT)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        torch.cuda.synchronize()
        if dist_name == "uniform":
            ace.profile_enable(True)
        a.record(stream)
        for _ in range(reps):
            ctx.msm_g1(bases, sc, n, out, ace.FORM_MONT)
        b.record(stream)
        torch.cuda.synchronize()
        msm[dist_name] = n * reps / (a.elapsed_time(b) / 1000.0)
        if dist_name == "uniform":
            iso = ace.profile_read(ace.PROF_G1_BUCKET)
            ace.profile_enable(False)

    # ---- roofline of the dominant kernel (G1 bucket accumulation) ----
    ms, nl, units = prof[ace.PROF_G1_BUCKET]
    sms = _device_sms(device)
    sm_max = _sm_max_mhz(clocks)
    peak = sms * IMAD_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
    # algorithmic multiply-adds per launch / average launch duration (the
    # launches of the batched proofs overlap other kernels and one another)
    achieved = units * IMAD_PER_G1_MADD / (g1_sum_ms / 1000.0) / 1e12 if g1_sum_ms > 0 else None
    union = {"achieved": units * IMAD_PER_G1_MADD / (ms / 1000.0) / 1e12 if ms > 0 else None, "ms": ms,
             "how": "the same work over the union of the launch intervals (time during which at least one "
                    "launch of the kernel was running)"}
    union["frac"] = union["achieved"] / peak if union["achieved"] else None
    measured_peak = {k: ace.imad_rate(ctx, mode) / 1e12 for k, mode in (("mad_lo", 0), ("mad_hi", 1),
                                                                       ("mad_lo_hi_chain", 2))}
    # one mad.wide is one limb product = two 32-bit multiply-adds (lo and hi)
    measured_peak["mad_wide_as_lo_hi"] = 2.0 * ace.imad_rate(ctx, 3) / 1e12
    traffic = None
    if G1_BUCKET_TRAFFIC["kernel_version"] == G1_BUCKET_KERNEL_VERSION and nl:
        traffic = G1_BUCKET_TRAFFIC["bytes_per_unit"] * units / nl
    # the same kernel with the GPU to itself (the 2^20 G1 MSM loop above)
    iso_ms, iso_nl, iso_units = iso
    isolated = {"achieved": iso_units * IMAD_PER_G1_MADD / (iso_ms / 1000.0) / 1e12 if iso_ms > 0 else None,
                "units_per_launch": iso_units / iso_nl if iso_nl else None, "launches": iso_nl,
                "where": "G1 MSM of 2^20 points, uniform scalars, alone on the GPU"}
    isolated["frac"] = isolated["achieved"] / peak if isolated["achieved"] else None
    # every kernel of the proof: algorithmic multiply-adds per proof / step time
    per_proof = {
        "g1_bucket": prof[ace.PROF_G1_BUCKET][2] / args.steps * IMAD_PER_G1_MADD,
        "g2_bucket": prof[ace.PROF_G2_BUCKET][2] / args.steps * IMAD_PER_G2_MADD,
        "ntt": prof[ace.PROF_NTT][2] / args.steps * IMAD_PER_FP_MUL,
        "spmv": prof[ace.PROF_SPMV][2] / args.steps * IMAD_PER_FP_MUL,
    }
    step_imad = sum(per_proof.values())
    step_alu = {"achieved": step_imad / (total_ms / args.steps / 1000.0) / 1e12, "imad_per_proof": step_imad,
                "counted": "bucket additions (G1, G2), NTT butterflies, sparse-product non-zeros"}
    step_alu["frac"] = step_alu["achieved"] / peak
    roofline = {"bound": "alu", "kernel": "k_bucket_acc<G1>", "achieved": achieved, "peak": peak,
                "unit": "T IMAD/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "algorithmic_per_unit": f"{IMAD_PER_G1_MADD} IMAD per mixed addition (10 Fp mul x 272)",
                "units_per_launch": units / nl if nl else None, "launches": nl,
                "avg_launch_ms": g1_sum_ms / nl if nl else None,
                "peak_source": f"{sms} SMs (device attribute) x 64 IMAD/clk/SM x {sm_max:.0f} MHz (maximum SM "
                               "clock): nominal unit counts",
                "traffic_source": G1_BUCKET_TRAFFIC["source"] if traffic is not None else
                "no ncu capture of this kernel version yet",
                "kernel_version": G1_BUCKET_KERNEL_VERSION,
                "peak_measured_T_per_s": measured_peak,
                "measured": "CUDA events around every launch inside the timed proofs; proofs overlap across "
                            "proving slots (configuration in `batch`), so a launch can share the SMs with "
                            "other proofs' kernels",
                "union": union, "isolated": isolated, "whole_step": step_alu}
    step_sorted = sorted(step_ms)
    p50 = statistics.median(step_sorted)
    p99 = step_sorted[min(len(step_sorted) - 1, int(round(0.99 * (len(step_sorted) - 1))))]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(WORKLOAD, l2="inputs larger than L2 (proving key %.2f GB resident)" % (pk.info[10] / 1e9),
                           m=m, m_A=shape["m_A"], m_B=shape["m_B"], m_L=shape["m_L"],
                           witness_bool_fraction=round(bool_frac, 4), parallelism="replicas" if ws > 1 else "1gpu"),
            "e2e": e2e,
            "gpu_launches": launches,
            "launches_before_timed": launches0,
            "roofline": roofline,
            "latency_ms": {"p50": p50, "p99": p99, "max": max(step_ms), "proofs": len(step_ms),
                           "budget_ms": 600.0,
                           "path": "one proof per call, back to back on one stream, CUDA events between calls"},
            "plain_proofs_per_s": plain_value,
            "batch": batch_cfg,
            "batch_tuning_ms": {"aux_streams": slot_ms[:4], "one_stream_per_proof": slot_ms[4:]},
            "msm_g1_2p20_points_per_s": msm,
            "stages": stages,
            "verified": bool(verified),
            "clocks": clocks,
        }
        if ws == 1 and not args.no_cpu_baseline:
            # the oracle on the host cores, after the GPU work: one whole proof
            # with the (r, s) of the first timed proof, whose bytes it must equal
            o = OracleBlockProof()
            oproof, dt = o.step(args.warmup)
            line["cpu_baseline"] = o.record([dt])
            line["cpu_baseline"]["proof_equals_gpu"] = oproof == bproofs[0]
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def batch_sizes(base_seed: int, k: int):
    """Row counts of the batched workload: T_i = round(2^(12 + 6 u_i)), u_i
    uniform in [0, 1) from SplitMix64 (seed, purpose 8); the QAP domain is the
    next power of two; the circuit is floor((T_i - 3)/243) permutations plus the
    chain up to T_i rows."""
    from paper_2603_10242_gb300 import inputs

    out = []
    u64 = inputs.splitmix64(base_seed, inputs.PURPOSE["sizes"], k)
    for x in u64:
        u = float(int(x) >> 11) * (2.0 ** -53)
        t = int(round(2.0 ** (12 + 6 * u)))
        log_n = max(12, (t - 1).bit_length())
        n_perm = (t - 3) // 243
        out.append((log_n, t, n_perm, 0, 0))
    return out


def run_batch_workload(args):
    """The batched workload: 64 independent proofs of uneven sizes (2^12..2^18
    rows), each with its own circuit, key and seed; one batch call (proofs
    pipelined over proving slots) against one proof per call."""
    import torch

    import paper_2603_10242_gb300 as ace

    ace.build()
    ctx = ace.Context(0)
    k = 64
    base = 4000
    sizes = batch_sizes(base, k)
    t0 = time.perf_counter()
    circs = [ace.Circuit(*p, seed=base + i) for i, p in enumerate(sizes)]
    pks = [ace.ProvingKey(ctx, c, toxic_seed=base + i) for i, c in enumerate(circs)]
    zs = [c.witness(base + i) for i, c in enumerate(circs)]
    setup_s = time.perf_counter() - t0
    dzs = [torch.frombuffer(bytearray(z), dtype=torch.uint8).cuda() for z in zs]
    rss = [ace.rs_from_seed(base + i) for i in range(k)]
    rs = b"".join(r for r, _ in rss)
    ss = b"".join(s_ for _, s_ in rss)
    # proving slots from the autotuner, timed on the median-size proof
    mid = sorted(range(k), key=lambda i: sizes[i][1])[k // 2]
    slot_ms = ctx.autotune_batch_slots(pks[mid], dzs[mid], 16, 12)
    slots = _tuned_batch(ctx)
    ctx.prove_batch(pks, dzs, rs, ss)            # warm-up (sizes the slots)
    for i in range(k):
        ctx.prove(pks[i], dzs[i], *rss[i])
    torch.cuda.synchronize()
    best_b, best_p = 1e30, 1e30
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        proofs, status = ctx.prove_batch(pks, dzs, rs, ss)
        best_b = min(best_b, time.perf_counter() - t0)
        t0 = time.perf_counter()
        plain = [ctx.prove(pks[i], dzs[i], *rss[i]) for i in range(k)]
        torch.cuda.synchronize()
        best_p = min(best_p, time.perf_counter() - t0)
    assert status == [0] * k and proofs == plain
    ok = all(pks[i].verify(zs[i][32:64], proofs[i]) == 1 for i in (0, k // 2, k - 1))
    rows = sum(p[1] for p in sizes)
    print(json.dumps({"workload": "groth16_batch64_2p12_2p18", "proofs": k, "rows_total": rows,
                      "log_n_hist": {str(l): sum(1 for p in sizes if p[0] == l) for l in range(12, 19)},
                      "batched_proofs_per_s": k / best_b, "plain_proofs_per_s": k / best_p,
                      "batched_constraints_per_s": rows / best_b, "setup_s": setup_s, "verified": ok,
                      "batch_slots": slots}))


# per-transaction circuit: 5 permutations (the commitment and key-derivation
# stand-in) and the chain to 1,400 rows, the paper's ~1,400-constraint
# ZK-ACE circuit size (Appendix B); N = 2^11
PERTX_CIRCUIT = (11, 1400, 5, 0, 0)
PERTX_BLOCK = 2000


def run_pertx(args):
    """Per-transaction proofs of a block (the paper's own design, Algorithm 3
    ParallelMap): 2,000 proofs of the same ~1,400-constraint circuit per block,
    all through one key.  ace_prove_many (every stage once for the whole
    block) against the proof-per-call batch path (ace_prove_batch over
    proving slots) on a slice of the block."""
    import numpy as np
    import torch

    import paper_2603_10242_gb300 as ace

    ace.build()
    ctx = ace.Context(0)
    k = PERTX_BLOCK
    c = ace.Circuit(*PERTX_CIRCUIT, seed=6100)
    pk = ace.ProvingKey(ctx, c, toxic_seed=6100)
    seeds = [6200 + i for i in range(k)]
    # the block's witnesses on the device (checked against the host generator
    # on a sample), then a pinned host copy for the end-to-end runs
    dz = torch.empty(k * 32 * c.m, dtype=torch.uint8, device="cuda")
    ctx.witness_many(c, seeds, dz)
    torch.cuda.synchronize()
    wit_ms = []
    for _ in range(3):
        t0 = time.perf_counter()
        ctx.witness_many(c, seeds, dz)
        wit_ms.append((time.perf_counter() - t0) * 1e3)
    zall = bytes(dz.cpu().numpy().tobytes())
    zs = [zall[32 * c.m * i:32 * c.m * (i + 1)] for i in range(k)]
    t0 = time.perf_counter()
    for i in (0, k // 2, k - 1):
        assert zs[i] == c.witness(seeds[i]), "device witness differs from the host generator"
    wit_s = (time.perf_counter() - t0) / 3 * k
    zpin = torch.frombuffer(bytearray(zall), dtype=torch.uint8).pin_memory()
    rss = [ace.rs_from_seed(6300 + i) for i in range(k)]
    rs = b"".join(r for r, _ in rss)
    ss = b"".join(s_ for _, s_ in rss)
    proofs, status = ctx.prove_many(pk, dz, k, rs, ss)  # warm-up (sizes the scratch)
    torch.cuda.synchronize()
    ms = []
    for _ in range(max(3, args.steps)):
        t0 = time.perf_counter()
        proofs, status = ctx.prove_many(pk, dz, k, rs, ss)
        ms.append((time.perf_counter() - t0) * 1e3)
    # end to end: the block's witnesses copied from pinned host memory each time
    e2e = []
    for _ in range(3):
        t0 = time.perf_counter()
        dz.copy_(zpin, non_blocking=True)
        proofs2, _ = ctx.prove_many(pk, dz, k, rs, ss)
        e2e.append((time.perf_counter() - t0) * 1e3)
    assert status == [0] * k and proofs2 == proofs
    # from seeds: the block's witnesses made on the device, then its proofs
    seeds_ms = []
    for _ in range(3):
        t0 = time.perf_counter()
        ctx.witness_many(c, seeds, dz)
        proofs3, _ = ctx.prove_many(pk, dz, k, rs, ss)
        seeds_ms.append((time.perf_counter() - t0) * 1e3)
    assert proofs3 == proofs
    # a slice through ace_prove_batch (same key: routed to the same
    # batch-dimension kernels) must give the same bytes; the slot-pipelined
    # rate of such a slice comes from the batch autotuner's timings (it runs
    # the slot path for 1..8 slots in both stage layouts)
    sl = 128
    dzs = [dz[i * 32 * c.m:(i + 1) * 32 * c.m] for i in range(sl)]
    bp, bst = ctx.prove_batch([pk] * sl, dzs, rs[:32 * sl], ss[:32 * sl])
    assert bst == [0] * sl and bp == proofs[:sl]
    slot_ms = ctx.autotune_batch_slots(pk, dzs[0], sl, 8)
    slot_s = min(slot_ms) / 1e3
    ok = all(pk.verify(zs[i][32:64], proofs[i]) == 1 for i in (0, k // 2, k - 1))
    # the validators' side: the whole block checked by one batch verification
    pubs = b"".join(z[32:64] for z in zs)
    allp = b"".join(proofs)
    vb_ms = []
    for rep in range(3):
        t0 = time.perf_counter()
        vb = ctx.verify_batch(pk.vk, pubs, allp, 0xACE0 + rep)
        vb_ms.append((time.perf_counter() - t0) * 1e3)
        ok = ok and vb == 1
    t0 = time.perf_counter()
    pk.verify(zs[0][32:64], proofs[0])
    single_verify_ms = (time.perf_counter() - t0) * 1e3
    best = min(ms)
    print(json.dumps({
        "workload": "groth16_pertx_block", "proofs_per_block": k, "constraints": PERTX_CIRCUIT[1],
        "N": 1 << PERTX_CIRCUIT[0], "m": c.m, "block_ms": {"best": best, "median": float(np.median(ms))},
        "proofs_per_s": k / (best / 1e3), "e2e_block_ms": min(e2e), "e2e_proofs_per_s": k / (min(e2e) / 1e3),
        "h2d_bytes_per_block": len(zall), "slot_pipelined_proofs_per_s": sl / slot_s,
        "witness_ms_device": min(wit_ms), "witness_s_host_estimate": wit_s,
        "seeds_to_proofs_block_ms": min(seeds_ms), "seeds_to_proofs_per_s": k / (min(seeds_ms) / 1e3),
        "verify_batch_block_ms": min(vb_ms), "verify_batch_proofs_per_s": k / (min(vb_ms) / 1e3),
        "single_verify_ms_host": single_verify_ms,
        "verified": ok,
        "paper_model": "2,000 tx x 15 ms per proof, 128 in parallel: ~240 ms per block (Section 3.1, Table "
                       "'Critical path analysis'; RTX 4090 estimate)"}))


SINGLE_CIRCUIT = (10, 1 << 10, 4, 0, 0)  # 4 permutations + chain to 2^10 rows


def run_single(args):
    """The single-proof workload: the plain proof of the 2^10 circuit (4
    Poseidon-style permutations and the chain), seed 1 for the circuit,
    witness, toxic waste and (r, s).  One proof per call: per-call latency
    from the host (witness already on the device, proof bytes back on the
    host), device time per proof back to back, end to end from pinned host
    memory through ace_prove_batch_host with one proof per call; and the
    same proofs in one batch call.  The oracle's proof of the same inputs is
    timed on the host cores and must equal the GPU's bytes."""
    import numpy as np
    import torch

    import oracle as O
    import paper_2603_10242_gb300 as ace

    ace.build()
    ctx = ace.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    c = ace.Circuit(*SINGLE_CIRCUIT, seed=1)
    z = c.witness(1)
    pk = ace.ProvingKey(ctx, c, toxic_seed=1)
    dz = torch.frombuffer(bytearray(z), dtype=torch.uint8).to(dev)
    zpin = torch.frombuffer(bytearray(z), dtype=torch.uint8).pin_memory()
    r, s_ = ace.rs_from_seed(1)
    want = ctx.prove(pk, dz, r, s_)
    n = max(200, args.steps)
    for _ in range(max(3, args.warmup)):
        ctx.prove(pk, dz, r, s_)
    # host-measured latency of one synchronous call (proof bytes on the host)
    lat = []
    for _ in range(n):
        t0 = time.perf_counter()
        p = ctx.prove(pk, dz, r, s_)
        lat.append((time.perf_counter() - t0) * 1e3)
    assert p == want
    # device time per proof, back to back on one stream
    d_proof = torch.zeros(256 * n, dtype=torch.uint8, device=dev)
    d_status = torch.zeros(n, dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(n):
        ctx.prove_async(pk, dz, r, s_, d_proof[256 * i:], d_status[i:])
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    dev_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]
    # end to end, one proof per call from pinned host memory
    e2e = []
    for _ in range(n):
        t0 = time.perf_counter()
        p2, st2 = ctx.prove_batch_host([pk], [zpin], r, s_)
        e2e.append((time.perf_counter() - t0) * 1e3)
    assert p2[0] == want and st2 == [0]
    # n proofs in one batch call: all of one small key, so ace_prove_batch
    # runs them on the batch-dimension kernels; beside it the best slot-
    # pipelined configuration the autotuner measured (64 proofs per batch)
    tune_ms = ctx.autotune_batch_slots(pk, dz, 64, 16)
    batch_cfg = _tuned_batch(ctx)
    slots_rate = 64 / (min(tune_ms) / 1e3)
    pb, sb = ctx.prove_batch([pk] * n, [dz] * n, r * n, s_ * n)
    t0 = time.perf_counter()
    pb, sb = ctx.prove_batch([pk] * n, [dz] * n, r * n, s_ * n)
    batch_s = time.perf_counter() - t0
    assert sb == [0] * n and pb[0] == want
    # the same batch end to end: witnesses in pinned host memory
    t0 = time.perf_counter()
    ph, sh = ctx.prove_batch_host([pk] * n, [zpin] * n, r * n, s_ * n)
    batch_host_s = time.perf_counter() - t0
    assert sh == [0] * n and ph == pb
    # the oracle on the host cores: same inputs, same bytes
    oc = O.Circuit(*SINGLE_CIRCUIT, seed=1, input_seed=1)
    opk = O.ProvingKey(oc, 1, with_points=True)
    ot = []
    for _ in range(5):
        t0 = time.perf_counter()
        ok, op = opk.prove(z, r, s_, 1)
        ot.append(time.perf_counter() - t0)
    assert ok

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]

    print(json.dumps({
        "workload": "groth16_single_2p10", "constraints": 1 << 10, "m": c.m, "proofs": n,
        "one_per_call": {"proofs_per_s": n / (sum(lat) / 1e3), "latency_ms": {"p50": pct(lat, 0.5),
                         "p99": pct(lat, 0.99), "max": max(lat)},
                         "path": "ace_prove, witness on the device, proof bytes on the host, host clock"},
        "device_ms_per_proof": {"p50": pct(dev_ms, 0.5), "p99": pct(dev_ms, 0.99)},
        "e2e_one_per_call": {"proofs_per_s": n / (sum(e2e) / 1e3), "latency_ms": {"p50": pct(e2e, 0.5),
                             "p99": pct(e2e, 0.99)}, "h2d_bytes_per_proof": len(z), "d2h_bytes_per_proof": 260,
                             "path": "ace_prove_batch_host with one proof per call"},
        "batched_proofs_per_s": n / batch_s,
        "batched_path": "ace_prove_batch, all proofs of one key: batch-dimension kernels (one launch per stage "
                        "for all proofs)",
        "e2e_batched_proofs_per_s": n / batch_host_s,
        "slot_pipelined_proofs_per_s": slots_rate, "slot_config": batch_cfg,
        "batch_tuning_ms": {"aux_streams": tune_ms[:16], "one_stream_per_proof": tune_ms[16:]},
        "verified": pk.verify(z[32:64], want) == 1, "oracle_equal": op == want,
        "cpu_baseline": {"kind": "oracle", "cores": O.lib().orc_num_threads(),
                         "value": 1.0 / statistics.median(ot), "unit": "proofs/s",
                         "sample": "5 oracle proofs of the same 2^10 inputs (setup untimed)"},
    }))


SERVE_CLASSES = (19, 20, 21, 22, 23)


def serve_class_params(log_n):
    """Size class of the served workload: 2 permutations per transaction, the
    chain fills the domain; capacity floor((N - 3) / 486) transactions."""
    n = 1 << log_n
    cap = (n - 3) // 486
    return (log_n, n, 2 * cap, 0, 0), cap


def run_serve(args):
    """The served workload: Poisson arrivals (mean 400 ms) of block-proof jobs
    with 1,000..16,000 transactions, each proved under the smallest size class
    (2^19..2^23) that holds it, by the continuous-batching server; keys of all
    classes resident.  Reports p50/p99 latency (submission -> proof bytes on
    the host) against the 600 ms budget, and proofs/s."""
    import math
    import threading

    import numpy as np
    import torch

    import paper_2603_10242_gb300 as ace
    from paper_2603_10242_gb300 import inputs

    ace.build()
    ctx = ace.Context(0)
    t0 = time.perf_counter()
    classes = {}
    for ln in SERVE_CLASSES:
        params, cap = serve_class_params(ln)
        c = ace.Circuit(*params, seed=5000 + ln)
        pk = ace.ProvingKey(ctx, c, toxic_seed=5000 + ln)
        pool = []
        for w in range(2):
            z = c.witness(6000 + 10 * ln + w)
            pool.append((torch.frombuffer(bytearray(z), dtype=torch.uint8).pin_memory(), z[32:64]))
        classes[ln] = (cap, c, pk, pool)
    setup_s = time.perf_counter() - t0
    # latency of one proof per class with the GPU otherwise idle (same path:
    # pinned host witness -> device, prove, proof bytes -> host)
    alone_ms = {}
    for ln in SERVE_CLASSES:
        _, _, pk, pool = classes[ln]
        zh = pool[0][0]
        r, s_ = ace.rs_from_seed(8000 + ln)
        ts = []
        for _ in range(3):
            dz = torch.empty(zh.numel(), dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            a = time.perf_counter()
            dz.copy_(zh, non_blocking=True)
            ctx.prove(pk, dz, r, s_)
            ts.append((time.perf_counter() - a) * 1e3)
            del dz
        alone_ms[str(ln)] = min(ts)
    n_jobs = args.jobs
    gaps = inputs.splitmix64(7, inputs.PURPOSE["arrivals"], n_jobs)
    txs = inputs.splitmix64(7, inputs.PURPOSE["sizes"], n_jobs)
    arrivals, t = [], 0.0
    for g in gaps:
        u = float(int(g) >> 11) * (2.0 ** -53)
        t += -0.4 * math.log(1.0 - u)
        arrivals.append(t)
    tx_counts = [1000 + int(x) % 15001 for x in txs]
    job_class = [min(ln for ln in SERVE_CLASSES if classes[ln][0] >= tx) for tx in tx_counts]
    srv = ace.Server(ctx, classes[SERVE_CLASSES[-1]][2], slots=args.serve_slots)
    ids = [None] * n_jobs
    start = time.perf_counter()

    def submitter():
        for i in range(n_jobs):
            now = time.perf_counter() - start
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
            ln = job_class[i]
            zh, _ = classes[ln][3][i % 2]
            r, s_ = ace.rs_from_seed(9000 + i)
            ids[i] = srv.submit(classes[ln][2], zh, r, s_)

    th = threading.Thread(target=submitter)
    th.start()
    lat, codes, proofs = [0.0] * n_jobs, [0] * n_jobs, {}
    for i in range(n_jobs):
        while ids[i] is None:
            time.sleep(0.0005)
        try:
            proof, l = srv.wait(ids[i], 600)
            lat[i] = l
            if i % 97 == 0:
                proofs[i] = proof
        except ace.AceError as e:
            codes[i] = e.code
    th.join()
    elapsed = time.perf_counter() - start
    stats = srv.stats()
    srv.close()
    ok = [l for l, c in zip(lat, codes) if c == 0]
    ok_sorted = sorted(ok)
    verified = all(classes[job_class[i]][2].verify(classes[job_class[i]][3][i % 2][1], p) == 1
                   for i, p in proofs.items())

    def pct(q, xs=None):
        xs = ok_sorted if xs is None else xs
        return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))] if xs else None

    per_class = {}
    for ln in SERVE_CLASSES:
        xs = sorted(l for l, c, jc in zip(lat, codes, job_class) if c == 0 and jc == ln)
        if xs:
            per_class[str(ln)] = {"jobs": len(xs), "p50": pct(0.5, xs), "p99": pct(0.99, xs), "max": xs[-1],
                                  "alone_ms": alone_ms[str(ln)]}

    print(json.dumps({
        "workload": "groth16_served_poisson_400ms", "jobs": n_jobs, "completed": len(ok),
        "errors": sum(1 for c in codes if c), "proofs_per_s": len(ok) / elapsed,
        "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": ok_sorted[-1] if ok_sorted else None,
                       "mean": float(np.mean(ok)) if ok else None, "budget_ms": 600.0,
                       "over_budget_fraction": sum(1 for l in ok if l > 600.0) / max(1, len(ok))},
        "class_counts": {str(ln): job_class.count(ln) for ln in SERVE_CLASSES},
        "per_class_ms": per_class,
        "mean_tx": float(np.mean(tx_counts)), "slots": args.serve_slots, "server": stats,
        "elapsed_s": elapsed, "setup_s": setup_s, "verified_sampled": verified,
        "key_device_bytes": {str(ln): classes[ln][2].info[10] for ln in SERVE_CLASSES}}))


def run_case(args):
    """Small fixed launches for profiler captures (not a bench line):
    msm_g1 -- one G1 MSM of 2^log_n points (uniform scalars; --log-n, default 20);
    msm_g2 -- one G2 MSM of 2^18 points (uniform scalars);
    ntt -- one 2^20 forward transform of three arrays (QAP batch shape);
    prove16 -- one proof of the 2^16 instance of the block circuit family;
    prove10 -- `steps` proofs of the 2^10 single-proof circuit, one per call
    (prints the launches issued before them, for a profiler's skip count);
    prove20 -- `steps` proofs of the 2^20 block circuit in one batch (prints
    the launches issued before the batch, for a profiler's skip count)."""
    import numpy as np
    import torch

    import paper_2603_10242_gb300 as ace
    from paper_2603_10242_gb300 import inputs

    ace.build()
    ctx = ace.Context(0)
    if args.case == "msm_g2":
        n = 1 << 18
        kb = inputs.sample_fr(20, inputs.PURPOSE["bases"], n)
        bases = torch.empty(128 * n, dtype=torch.uint8, device="cuda")
        ctx.g2_fixed_base(torch.from_numpy(kb.view(np.uint8).reshape(-1)).cuda(), n, bases, ace.FORM_MONT)
        sc = torch.from_numpy(inputs.sample_scalars(20, n, "uniform").view(np.uint8).reshape(-1)).cuda()
        out = torch.empty(128, dtype=torch.uint8, device="cuda")
        for _ in range(args.steps):
            ctx.msm_g2(bases, sc, n, out, ace.FORM_MONT)
    elif args.case == "msm_g1":
        n = 1 << args.log_n
        kb = inputs.sample_fr(20, inputs.PURPOSE["bases"], n)
        bases = torch.empty(64 * n, dtype=torch.uint8, device="cuda")
        ctx.g1_fixed_base(torch.from_numpy(kb.view(np.uint8).reshape(-1)).cuda(), n, bases, ace.FORM_MONT)
        sc = torch.from_numpy(inputs.sample_scalars(args.log_n, n, "uniform").view(np.uint8).reshape(-1)).cuda()
        out = torch.empty(64, dtype=torch.uint8, device="cuda")
        for _ in range(args.steps):
            ctx.msm_g1(bases, sc, n, out, ace.FORM_MONT)
    elif args.case == "ntt":
        n = 1 << 20
        d = torch.from_numpy(inputs.sample_fr(1, 7, 3 * n).view(np.uint8).reshape(-1)).cuda()
        for _ in range(args.steps):
            ctx.ntt_mont(d, 20, 3, True, False)
    elif args.case == "prove10":
        c = ace.Circuit(*SINGLE_CIRCUIT, seed=1)
        z = c.witness(1)
        pk = ace.ProvingKey(ctx, c, toxic_seed=1)
        dz = torch.frombuffer(bytearray(z), dtype=torch.uint8).cuda()
        r, s_ = ace.rs_from_seed(1)
        ctx.prove(pk, dz, r, s_)
        torch.cuda.synchronize()
        before = ace.launch_count()
        for _ in range(args.steps):
            assert pk.verify(z[32:64], ctx.prove(pk, dz, r, s_)) == 1
        print(json.dumps({"case": args.case, "steps": args.steps, "launches_before": before,
                          "launches": ace.launch_count()}))
        return
    elif args.case == "prove20":
        c = ace.Circuit(seed=SEED, **CIRCUIT)
        z = c.witness(SEED)
        pk = ace.ProvingKey(ctx, c, toxic_seed=SEED)
        dz = torch.frombuffer(bytearray(z), dtype=torch.uint8).cuda()
        r, s_ = ace.rs_from_seed(1)
        torch.cuda.synchronize()
        before = ace.launch_count()
        proofs, st = ctx.prove_batch([pk] * args.steps, [dz] * args.steps, r * args.steps, s_ * args.steps)
        assert st == [0] * args.steps and pk.verify(z[32:64], proofs[0]) == 1
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "steps": args.steps, "launches_before_batch": before,
                          "launches": ace.launch_count()}))
        return
    else:
        c = ace.Circuit(16, 1 << 16, 256, 256, 172, seed=SEED)
        z = c.witness(SEED)
        pk = ace.ProvingKey(ctx, c, toxic_seed=SEED)
        dz = torch.frombuffer(bytearray(z), dtype=torch.uint8).cuda()
        r, s_ = ace.rs_from_seed(1)
        for _ in range(args.steps):
            ctx.prove(pk, dz, r, s_)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "steps": args.steps, "launches": ace.launch_count()}))


def run_sweep(args):
    """The kernel sweep: G1 MSM at 2^16..2^24 points (bases k_i G stored
    affine in Montgomery form, k_i seeded) in the uniform and the 70%-{0,1}
    scalar distributions, the G2 MSM at 2^12..2^18 points (uniform), and the
    Fr NTT, inverse NTT and coset NTT at 2^16..2^24 elements (uniform inputs),
    alone and in the prover's three-array shape.  Every timed call is bracketed by
    CUDA events on the launching stream; a 256 MiB buffer (larger than the
    129 MB L2) is written between timed calls, so no call starts with its
    inputs in L2.  Sizes are prefixes of one seeded stream per distribution."""
    import numpy as np
    import torch

    import paper_2603_10242_gb300 as ace
    from paper_2603_10242_gb300 import inputs

    ace.build()
    ctx = ace.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peak_imad = _device_sms(dev) * IMAD_PER_CLK_PER_SM * _sm_max_mhz(None) * 1e6
    hbm_peak = _measured_hbm_gbs()
    reps = max(3, args.steps)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b) / 1000.0)
        return statistics.median(ts)

    logs = (16, 18, 20, 22, 24)
    nmax = 1 << logs[-1]
    kb = inputs.sample_fr(20, inputs.PURPOSE["bases"], nmax)
    bases = torch.empty(64 * nmax, dtype=torch.uint8, device=dev)
    ctx.g1_fixed_base(torch.from_numpy(kb.view(np.uint8).reshape(-1)).to(dev), nmax, bases, ace.FORM_MONT)
    out = torch.empty(64, dtype=torch.uint8, device=dev)
    msm_rows = []
    for dist_name in ("uniform", "sparse"):
        sc = torch.from_numpy(inputs.sample_scalars(24, nmax, dist_name).view(np.uint8).reshape(-1)).to(dev)
        for lg in logs:
            n = 1 << lg
            t = timed(lambda: ctx.msm_g1(bases, sc, n, out, ace.FORM_MONT))
            # one more call under the launch profiler for the bucket kernel's work and time
            ace.profile_enable(True)
            ctx.msm_g1(bases, sc, n, out, ace.FORM_MONT)
            torch.cuda.synchronize()
            ms, nl, adds = ace.profile_read(ace.PROF_G1_BUCKET)
            sort_ms = ace.profile_read(ace.PROF_SORT)[0]
            red_ms = ace.profile_read(ace.PROF_REDUCE)[0]
            ace.profile_enable(False)
            bucket_rate = adds * IMAD_PER_G1_MADD / (ms / 1000.0) if ms > 0 else None
            msm_rows.append({
                "log_n": lg, "scalars": dist_name, "ms": t * 1000.0, "points_per_s": n / t,
                "bucket_additions": adds,
                "stage_ms": {"sort": sort_ms, "bucket_acc": ms, "reduce_and_final": red_ms},
                "bucket_kernel_frac": bucket_rate / peak_imad if bucket_rate else None,
                "msm_frac": adds * IMAD_PER_G1_MADD / t / peak_imad,
            })
        del sc
    del bases
    torch.cuda.empty_cache()

    # G2 MSM (the generic entry point: the psi split up to 2^16 points,
    # full-width scalars above), uniform scalars
    g2_rows = []
    n2 = 1 << 18
    kb2 = inputs.sample_fr(21, inputs.PURPOSE["bases"], n2)
    bases2 = torch.empty(128 * n2, dtype=torch.uint8, device=dev)
    ctx.g2_fixed_base(torch.from_numpy(kb2.view(np.uint8).reshape(-1)).to(dev), n2, bases2, ace.FORM_MONT)
    sc2 = torch.from_numpy(inputs.sample_scalars(21, n2, "uniform").view(np.uint8).reshape(-1)).to(dev)
    out2 = torch.empty(128, dtype=torch.uint8, device=dev)
    for lg in (12, 14, 16, 18):
        n = 1 << lg
        t = timed(lambda: ctx.msm_g2(bases2, sc2, n, out2, ace.FORM_MONT))
        split = n <= 1 << 16
        g2_rows.append({"log_n": lg, "scalars": "uniform", "ms": t * 1000.0, "points_per_s": n / t,
                        "plan": "psi split, 4n points" if split else "full-width scalars",
                        "c": ace.msm_plan(n, ace.MSM_GLS if split else ace.MSM_FULL)["c"]})
    del bases2, sc2
    torch.cuda.empty_cache()

    ntt_rows = []
    kinds = {0: "ntt", 1: "intt", 2: "coset_ntt", 3: "coset_intt"}
    vals = torch.from_numpy(inputs.sample_fr(24, 7, 1 << 24).view(np.uint8).reshape(-1)).to(dev)
    for lg in range(16, 25):
        n = 1 << lg
        d = vals[:32 * n].clone()
        for kind, name in kinds.items():
            t = timed(lambda: ctx.ntt(d, lg, kind))
            # radix-2 count: (N/2) log2 N butterflies (one product each) plus the
            # N scalings of the inverse and coset forms
            muls = (n // 2) * lg + (n if kind else 0)
            ntt_rows.append({
                "log_n": lg, "kind": name, "ms": t * 1000.0, "elements_per_s": n / t,
                "hbm_gbs_algorithmic": 64.0 * n / t / 1e9,
                "hbm_frac": 64.0 * n / t / 1e9 / hbm_peak,
                "imad_frac": muls * IMAD_PER_FP_MUL / t / peak_imad,
            })
        del d
    # the prover's own shape: one launch sequence over three arrays (the QAP's
    # a, b, c), Montgomery form in and out, natural order in, bit-reversed out
    ntt_batch_rows = []
    for lg in range(16, 25):
        n = 1 << lg
        d3 = torch.empty(3 * 32 * n, dtype=torch.uint8, device=dev)
        for j in range(3):
            d3[j * 32 * n:(j + 1) * 32 * n].copy_(vals[:32 * n])
        t = timed(lambda: ctx.ntt_mont(d3, lg, 3, True, False))
        muls = 3 * (n // 2) * lg
        ntt_batch_rows.append({
            "log_n": lg, "arrays": 3, "ms": t * 1000.0, "elements_per_s": 3 * n / t,
            "hbm_frac": 3 * 64.0 * n / t / 1e9 / hbm_peak,
            "imad_frac": muls * IMAD_PER_FP_MUL / t / peak_imad,
        })
        del d3
    cpu = None if args.no_cpu_baseline else sweep_cpu_sample()
    print(json.dumps({
        "workload": "kernel_sweep_msm_g1_ntt_2p16_2p24", "curve": "BN254", "reps": reps,
        "cpu_baseline": cpu,
        "timing": "median of reps, CUDA events per call, L2 flushed (256 MiB write) before each call",
        "msm_g1": msm_rows, "msm_g2": g2_rows, "ntt": ntt_rows, "ntt_qap_batch": ntt_batch_rows,
        "roofline": {"imad_peak_T_per_s": peak_imad / 1e12, "hbm_peak_gbs": hbm_peak,
                     "msm": f"{IMAD_PER_G1_MADD} IMAD per bucket addition (algorithmic, bucket additions only)",
                     "ntt": "64 B per element (read + write once) against HBM; "
                            f"{IMAD_PER_FP_MUL} IMAD per butterfly product against the ALU"},
    }))


def sweep_cpu_sample():
    """The oracle on a bounded sample of the sweep: its plain Pippenger G1 MSM
    over 2^16 points (uniform and 70%-{0,1} scalars) and its radix-2 NTT at
    2^16, 2^18 and 2^20 elements, on the host's cores (a few seconds)."""
    import numpy as np

    import oracle as O
    from paper_2603_10242_gb300 import inputs

    n = 1 << 16
    pts = O.g1_mul_gen_batch(inputs.sample_fr(20, inputs.PURPOSE["bases"], n).tobytes())
    msm = {}
    for dist_name in ("uniform", "sparse"):
        sc = inputs.sample_scalars(24, n, dist_name).tobytes()
        t0 = time.perf_counter()
        O.msm_g1(pts, sc, 1)
        msm[dist_name] = n / (time.perf_counter() - t0)
    ntt = {}
    vals = inputs.sample_fr(24, 7, 1 << 20)
    for lg in (16, 18, 20):
        raw = np.ascontiguousarray(vals[:1 << lg]).tobytes()
        t0 = time.perf_counter()
        O.ntt(raw, lg)
        ntt[str(lg)] = (1 << lg) / (time.perf_counter() - t0)
    return {"kind": "oracle", "cores": O.lib().orc_num_threads(),
            "msm_g1_2p16_points_per_s": msm, "ntt_elements_per_s": ntt,
            "sample": "plain Pippenger over 2^16 G1 points per scalar distribution; forward NTT at 2^16, 2^18, 2^20"}


def _measured_hbm_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=2000, help="served workload: number of jobs")
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--workload", choices=["block2p20", "single2p10", "batch64", "serve", "pertx", "sweep"],
                    default="block2p20",
                    help="batch64: 64 proofs of log-uniform sizes 2^12..2^18 (batched vs one per call)")
    ap.add_argument("--case", choices=["msm_g1", "msm_g2", "ntt", "prove10", "prove16", "prove20"], default=None,
                    help="run a small fixed case for profiler captures instead of the bench")
    ap.add_argument("--log-n", type=int, default=20, help="--case msm_g1: log2 of the number of points")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="reference arm: seconds of oracle proving after the first proof")
    ap.add_argument("--latency-proofs", type=int, default=200,
                    help="one-proof-per-call latency: proofs timed back to back (at least --steps)")
    args = ap.parse_args()
    if args.case:
        run_case(args)
    elif args.workload == "single2p10":
        run_single(args)
    elif args.workload == "batch64":
        run_batch_workload(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "pertx":
        run_pertx(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        if args.warmup < 3:
            args.warmup = 3
        run_ours(args)


if __name__ == "__main__":
    main()
