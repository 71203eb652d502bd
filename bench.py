#!/usr/bin/env python3
"""Pauli-rotation throughput on GB300: rotations/s at n = 24, HBM fraction, and
the speedup over the gate-decomposed path on the same GPU.

Workload (one step): a seeded Jordan-Wigner-shaped Hamiltonian on n = 24 qubits
with 2000 terms, 10 first-order Trotter steps at dt = 0.05 (20,000 rotations),
applied to the Hartree-Fock state with 12 electrons, followed by the FP64
energy <H> and norm.  Synthetic data: the chemistry Hamiltonians the paper
measures are not available.

Arms:
  default            the library (plan compiled once; per step: basis state,
                     all fused passes, FP64 <H>); e2e repeats the step through
                     the C ABI with host buffers (state upload from pinned
                     memory, rotation list planned and uploaded per call,
                     final state and energy read back).
  --impl reference   the FP64 CPU oracle (gate-decomposed), on a bounded
                     sample of the same rotation list per step.

Multi-GPU (torchrun): every rank runs an independent replica of the workload
(weak scaling); value = all ranks' rotations / max time.  The global-qubit
sharded path is timed on one GPU, all its slices on that GPU, as the
``sharded_one_gpu`` extra.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_09020_gb300 import synth  # noqa: E402

METRIC = "Pauli rotations/s at n=24 & HBM fraction; speedup vs gate-decomposed, same GPU"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--n", type=int, default=24)
    ap.add_argument("--terms", type=int, default=2000)
    ap.add_argument("--trotter-steps", type=int, default=10)
    ap.add_argument("--dt", type=float, default=0.05)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--fusion-depth", type=int, default=-1)
    ap.add_argument("--tour", action="store_true",
                    help="launch every kernel family once on states larger than L2 and print their "
                         "event-timed algorithmic bandwidth (for profiler captures), instead of the bench")
    ap.add_argument("--skip-extras", action="store_true",
                    help="only the timed steps (for profiler launch lists)")
    return ap.parse_args()


def workload_name(a) -> str:
    return (f"JW-shaped H, n={a.n}, {a.terms} terms, {a.trotter_steps} first-order Trotter steps "
            f"at dt={a.dt} ({a.terms * a.trotter_steps} rotations), HF state, then FP64 <H>")


def config_dict(a, dtype) -> dict:
    return {"workload": workload_name(a), "n_qubits": a.n, "terms": a.terms, "trotter_steps": a.trotter_steps,
            "order": 1, "dt": a.dt, "seed": a.seed, "state": dtype,
            "rotations_per_step": a.terms * a.trotter_steps,
            "l2": "inputs > L2 for c128; L2 flushed (512 MB write) between timed steps",
            "parallelism": "replicas"}


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# source files that define each traced kernel family, per precision: a stored
# ncu traffic figure counts only while these are unchanged since the capture
KERNEL_SOURCES = {("k_coset", "c64"): ("kernels.cuh", "rotate.cu"),
                  ("k_chain2", "c64"): ("chain.cu", "kernels.cuh", "internal.h"),
                  ("k_coset", "c128"): ("coset_fx.cuh", "fixed64.cuh", "kernels.cuh", "rotate.cu"),
                  ("k_diag_sum", "c64"): ("kernels.cuh", "rotate.cu"),
                  ("k_diag_sum", "c128"): ("kernels.cuh", "rotate.cu"),
                  ("k_expval", "c64"): ("reduce.cu",), ("k_expval", "c128"): ("reduce.cu", "fixed64.cuh")}


def kernel_source_digest(name: str, dtype: str):
    for (prefix, dt), files in KERNEL_SOURCES.items():
        if name.startswith(prefix) and dt == dtype:
            h = hashlib.sha256()
            for f in files:
                with open(os.path.join(ROOT, "paper_2602_09020_gb300", "csrc", f), "rb") as fh:
                    h.update(fh.read())
            return h.hexdigest()
    return None


def ncu_traffic(name: str, dtype: str, n: int):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of one
    ncu capture of this kernel at this size, or None when there is none or the
    kernel's sources changed after it was taken."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        entry = json.load(fh).get(f"{name}/{dtype}/n{n}")
    if not entry or entry.get("sources_sha256") != kernel_source_digest(name, dtype):
        return None
    return entry["dram_bytes_per_launch"]


# ------------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def mhz(s):
            try:
                return float(s.split()[0])
            except (ValueError, IndexError):
                return None
        sm = [mhz(r[1]) for r in rows if mhz(r[1]) is not None]
        mx = [mhz(r[2]) for r in rows if mhz(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [nm for i, nm in enumerate(names) if any(r[5 + i].lower().startswith("active") for r in rows)]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle

def strided_sample(rx, rz, rt, count: int, period: int):
    """Every k-th rotation of the first `period` rotations (one Trotter step: the
    list repeats it), k chosen so that about `count` are taken.  The oracle's
    cost per rotation depends only on the string's support, so a stride across
    a whole step gives the list's mix of localities, which a prefix does not
    (the step starts with all its Z and ZZ terms)."""
    period = min(period, len(rt))
    k = max(1, period // max(1, count))
    sel = np.arange(0, period, k)
    return rx[sel], rz[sel], rt[sel], k


def oracle_rate(n, rx, rz, rt, seconds: float, basis: int, period: int):
    """Time the oracle on a strided sample of one Trotter step sized to take
    about `seconds`: a short pilot (every 50th rotation of the step) gives the
    rate, then the sample is drawn at the stride that fills the time.
    Returns (rot/s, count, threads, elapsed s, stride, mean locality of the sample)."""
    import oracle
    px, pz, pt, _ = strided_sample(rx, rz, rt, max(2, period // 50), period)
    psi = oracle.basis_state(n, basis)
    t0 = time.perf_counter()
    oracle.apply_rotations(psi, n, px[:8], pz[:8], pt[:8])
    pilot = 8 / (time.perf_counter() - t0)
    sx, sz, st, stride = strided_sample(rx, rz, rt, max(2, int(pilot * seconds)), period)
    psi = oracle.basis_state(n, basis)
    t0 = time.perf_counter()
    oracle.apply_rotations(psi, n, sx, sz, st)
    el = time.perf_counter() - t0
    loc = float(synth.locality(sx, sz).mean())
    return len(st) / el, len(st), oracle.num_threads(), el, stride, loc


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    ham = synth.jw_hamiltonian(a.n, a.terms, a.seed)
    rx, rz, rt = oracle.trotter_rotations(ham.x, ham.z, ham.c, a.dt, a.trotter_steps, 1)
    basis = synth.hartree_fock_index(a.n // 2)
    # a strided sample of one Trotter step, sized so that warmup + steps take
    # about two minutes (the oracle's cost per rotation depends only on the
    # string's support, so the stride keeps the list's mix of localities)
    r1, _, threads, _, _, _ = oracle_rate(a.n, rx, rz, rt, 2.0, basis, a.terms)
    sx, sz, st, stride = strided_sample(rx, rz, rt, max(2, int(r1 * 120.0 / max(1, a.steps + a.warmup))),
                                        a.terms)
    times = []
    for s in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        psi = oracle.basis_state(a.n, basis)
        oracle.apply_rotations(psi, a.n, sx, sz, st)
        el = time.perf_counter() - t0
        if s >= a.warmup:
            times.append(el)
    ms = 1000.0 * statistics.mean(times)
    value = len(st) / (ms / 1000.0)
    sample = (f"every {stride}th rotation of the first Trotter step ({len(st)} of {len(rt)} rotations per step, "
              f"mean locality {float(synth.locality(sx, sz).mean()):.2f} vs "
              f"{float(synth.locality(rx, rz).mean()):.2f} for the list; n={a.n}, complex128, gate-decomposed)")
    line = {"metric": METRIC, "value": value, "unit": "rotations/s", "impl": "reference", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": config_dict(a, "c128"),
            "cpu_baseline": {"value": value, "unit": "rotations/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "rotations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_ours(a):
    import torch
    from paper_2602_09020_gb300 import capi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2602_09020_gb300 import replicas

    def max_over_ranks(v: float) -> float:
        return replicas.max_over_ranks(v, dist, "cuda")

    ham = synth.jw_hamiltonian(a.n, a.terms, a.seed)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, a.dt, a.trotter_steps, 1, False)
    R = len(rt)
    basis = synth.hartree_fock_index(a.n // 2)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    pk = peaks()

    def measure(dtype: str, steps: int, warmup: int, trace: str = "", clocks: Clocks = None):
        """trace: "" (untimed per kernel), "blocks" (an event per change of kernel)
        or "launches" (an event pair around every launch)."""
        t0 = time.perf_counter()
        plan = capi.plan_create(a.n, dtype, rx, rz, rt, a.fusion_depth, sh)
        plan_ms = 1000.0 * (time.perf_counter() - t0)
        nrot, nruns, ndiag = capi.plan_stats(plan)
        nsweeps = capi.plan_sweeps(plan)
        dmax = a.fusion_depth if a.fusion_depth >= 0 else capi.plan_tuned_depth(a.n, dtype)[0]
        sv = capi.sv_alloc(a.n, dtype, sh)
        out = {}

        def step():
            capi.sv_set_basis_state(sv, basis)
            capi.plan_apply(sv, plan)
            out["energy"], out["norm2"] = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)

        for _ in range(warmup):
            step()
        barrier()
        if clocks:
            clocks.start()
        if trace:
            capi.sv_trace_start(sv, blocks=(trace == "blocks"))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        barrier()
        rows = capi.sv_trace_stop(sv) if trace else {}
        ck = clocks.stop() if clocks else None
        ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        capi.sv_free(sv)
        capi.plan_free(plan)
        return {"ms": ms, "plan_ms": plan_ms, "runs": nruns, "sweeps": nsweeps, "dmax": dmax, "diag_runs": ndiag, "nrot": nrot,
                "trace": rows, "clocks": ck, "energy": out["energy"], "norm2": out["norm2"]}

    def roofline(rows: dict, steps: int, dtype: str):
        if not rows:
            return None, 0
        name = max(rows, key=lambda k: rows[k][1])
        launches, tot_ms, by, fl = rows[name]
        traffic = ncu_traffic(name, dtype, a.n)
        common = {"kernel": name, "traffic": traffic, "launches_per_step": launches / steps,
                  "timing": "CUDA events at every change of kernel in a repeat of the timed step: "
                            "consecutive launches of one kernel run chained between two events, as "
                            "they do untraced; per launch = block time / launches",
                  "ms_per_launch": tot_ms / launches, "algorithmic_bytes_per_launch": by / launches,
                  "algorithmic_flops_per_launch": fl / launches,
                  "hbm_gbs": by / (tot_ms / 1000.0) / 1e9}
        achieved = by / (tot_ms / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "peak_source": pk["source"]}
        if name.startswith("k_chain"):
            # a chained pass applies two runs per sweep of the state and is bound
            # by the FP32 FMA pipe (the pair updates: 4 flops per amplitude and
            # rotation), not by HBM; its HBM figures stay beside the roofline
            tflops = fl / (tot_ms / 1000.0) / 1e12
            if fp32_peak.get("tflops"):
                peak, src = fp32_peak["tflops"], fp32_peak["source"]
            else:
                sms = torch.cuda.get_device_properties(0).multi_processor_count
                peak = sms * 128 * 2 * 2.070e9 / 1e12
                src = f"nominal: {sms} SMs x 128 FP32 FMA per clock x 2 flops x 2070 MHz"
            roof = {"bound": "alu", "pipe": "fp32_fma", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                    "frac": tflops / peak, "peak_source": src,
                    "hbm": {"achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": achieved / pk["hbm_gbs"], "peak_source": pk["source"]},
                    "runs_per_sweep": 2,
                    # the bytes the two runs would move as one-run passes, over
                    # the chained pass's time: the HBM rate one-run passes would
                    # need to match it
                    "run_equivalent_hbm_frac": 2.0 * achieved / pk["hbm_gbs"]}
        if dtype == "c128" and name.startswith("k_coset"):
            # the complex128 pass runs its products on the integer pipes: per
            # amplitude and rotation two 62-bit fixed-point products of three
            # 32x32->64 multiply-adds each (the trace counts 4 FP64-equivalent
            # flops there); the wide-multiply rate is set against the measured
            # peak of the probe kernel when the bench has measured it, and is
            # then the roofline (the pass is bound by the integer pipes), with
            # its HBM fraction beside it
            imads = 1.5 * fl / (tot_ms / 1000.0) / 1e12
            roof["alu"] = {"pipe": "int_mul_wide", "achieved": imads, "unit": "Tops/s",
                           "ops_per_amplitude_rotation": 6,
                           "peak": int_peak.get("tops"), "peak_source": int_peak.get("source"),
                           "frac": (imads / int_peak["tops"]) if int_peak.get("tops") else None}
            if int_peak.get("tops"):
                hbm = {k: roof[k] for k in ("achieved", "peak", "unit", "frac", "peak_source")}
                roof = {"bound": "alu", "pipe": "int_mul_wide", "achieved": imads, "peak": int_peak["tops"],
                        "unit": "Tops/s", "frac": imads / int_peak["tops"], "peak_source": int_peak["source"],
                        "ops_per_amplitude_rotation": 6, "hbm": hbm}
        roof.update(common)
        return roof, sum(r[0] for r in rows.values())

    # measured arithmetic peaks (FP64 FMA, wide integer multiply-add), taken
    # before the timed steps so the complex128 roofline can use them
    int_peak, fp32_peak = {}, {}
    arith = None
    if not a.skip_extras:
        arith = probe_peaks(capi, torch)
        int_peak = {"tops": arith["int_mul_wide_tops"], "source": "measured (probe kernel, this run)"}
        fp32_peak = {"tflops": arith["fp32_tflops"], "source": "measured (packed FP32x2 FMA probe kernel, this run)"}

    # the fusion depth plan_create(-1) takes comes from the library's autotuner,
    # run on the first Trotter step of the list for each precision (untimed
    # setup), unless the tune table already holds a depth for (n, dtype) (read
    # from PAULIROT_TUNE_CACHE, which a tuning run also writes back)
    tuning = {}
    if a.fusion_depth < 0:
        for dt_name in ([a.dtype] if a.skip_extras else [a.dtype, "c128" if a.dtype == "c64" else "c64"]):
            cached, is_tuned = capi.plan_tuned_depth(a.n, dt_name)
            if is_tuned:
                tuning[dt_name] = {"depth": cached, "source": "tune cache"}
                continue
            svt = capi.sv_alloc(a.n, dt_name, sh)
            t0 = time.perf_counter()
            depth, tms = capi.plan_autotune(svt, rx[:a.terms], rz[:a.terms], rt[:a.terms], reps=2)
            tuning[dt_name] = {"depth": depth, "source": "autotuned", "tune_s": time.perf_counter() - t0,
                               "sample": f"first {a.terms} rotations",
                               "ms_per_sample_by_depth": {str(d + 1): v for d, v in enumerate(tms) if v > 0}}
            capi.sv_free(svt)
        barrier()

    clocks = Clocks(dev)
    # the headline steps run untraced: per-launch event records between the
    # kernels would keep consecutive passes from overlapping (programmatic
    # dependent launch); a short traced run gives the per-kernel figures
    main = measure(a.dtype, a.steps, a.warmup, "", clocks)
    tsteps = max(1, min(a.steps, 2))
    traced = measure(a.dtype, tsteps, 1, "blocks")
    per_launch = measure(a.dtype, tsteps, 1, "launches")
    ms_step = statistics.mean(main["ms"])
    ms_max = max_over_ranks(ms_step)
    value = replicas.whole_job_rate(R, ms_max / 1000.0, world)
    roof, t_launches = roofline(traced["trace"], tsteps, a.dtype)
    launches = int(round(t_launches * a.steps / tsteps))
    s_bytes = 16 if a.dtype == "c128" else 8
    sweep_bytes = 2.0 * s_bytes * (1 << a.n)

    extras = {}
    if not a.skip_extras:
        # the other precision, device-timed
        other = "c128" if a.dtype == "c64" else "c64"
        o = measure(other, max(1, min(a.steps, 2)), 1, "blocks")
        o_roof, _ = roofline(o["trace"], max(1, min(a.steps, 2)), other)
        extras[other] = {"value": R / (statistics.mean(o["ms"]) / 1000.0), "ms_per_step": statistics.mean(o["ms"]),
                         "passes_per_step": o["sweeps"], "runs_per_step": o["runs"], "fusion_depth": o["dmax"], "energy": o["energy"], "roofline": o_roof}
        # gate-decomposed path on the same GPU, same dtype: a strided sample of one Trotter step
        sample = slice(0, a.terms, 4)
        gx, gz, gt = rx[sample], rz[sample], rt[sample]
        svg = capi.sv_alloc(a.n, a.dtype, sh)
        capi.sv_set_basis_state(svg, basis)
        capi.apply_pauli_rotations_gates(svg, gx[:20], gz[:20], gt[:20])  # warm
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ngates = capi.apply_pauli_rotations_gates(svg, gx, gz, gt)
        e1.record(stream)
        barrier()
        g_ms = e0.elapsed_time(e1)
        capi.sv_free(svg)
        g_rate = len(gt) / (g_ms / 1000.0)
        extras["gate_decomposed"] = {"rotations": len(gt), "gates": ngates, "ms": g_ms,
                                     "rotations_per_s": g_rate, "speedup": (R / (ms_step / 1000.0)) / g_rate,
                                     "sample": "every 4th rotation of the first Trotter step"}

    # batched independent states: one persistent launch vs one launch per pass per state
    if not a.skip_extras:
        extras["batched"] = batch_measure(capi, torch, stream, sh, barrier)
        extras["locality_sweep"] = locality_measure(capi, torch, a.n, a.dtype, barrier)
        extras["cfhs_gate_stream"] = cfhs_measure(capi, torch, a.n, a.dtype, rx[:a.terms], rz[:a.terms],
                                                  rt[:a.terms], ham, basis, barrier)
        extras["large_state"] = large_measure(capi, torch, barrier)
        extras["large_state"]["n29_c64_vs_c128"] = large_compare(capi, torch, barrier)
        extras["adjoint"] = adjoint_measure(capi, torch, barrier)
        extras["arith_peaks"] = arith
        extras["sharded_one_gpu"] = shard_measure(capi, torch, barrier)
        extras["precision"] = precision_report(capi, a, ham, rx, rz, rt, basis, sh)

    # end to end through the C ABI with host buffers
    e2e = None
    if not a.skip_extras:
        amp_dt = torch.complex128 if a.dtype == "c128" else torch.complex64
        h_in = torch.zeros(1 << a.n, dtype=amp_dt, pin_memory=True)
        h_in[basis] = 1.0
        h_out = torch.empty(1 << a.n, dtype=amp_dt, pin_memory=True)
        sv = capi.sv_alloc(a.n, a.dtype, sh)
        lib = capi.lib()
        xs, zs, ts = np.ascontiguousarray(rx), np.ascontiguousarray(rz), np.ascontiguousarray(rt)
        e_out, n_out = ctypes.c_double(), ctypes.c_double()

        def e2e_step():
            capi._check(lib.sv_from_host(sv, h_in.data_ptr()))
            capi._check(lib.apply_pauli_rotations(sv, xs.ctypes.data, zs.ctypes.data, ts.ctypes.data, R))
            capi._check(lib.expval_pauli_sum(sv, ham.x.ctypes.data, ham.z.ctypes.data, ham.c.ctypes.data,
                                             len(ham.c), ctypes.byref(e_out), ctypes.byref(n_out)))
            capi._check(lib.sv_to_host(sv, h_out.data_ptr(), 1))

        e2e_step()
        barrier()
        n_e2e = max(1, min(a.steps, 2))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        barrier()
        el = (time.perf_counter() - t0) / n_e2e
        el = max_over_ranks(el)
        capi.sv_free(sv)
        state_bytes = s_bytes << a.n
        e2e = {"value": world * R / el, "unit": "rotations/s",
               "h2d_bytes_per_step": state_bytes + R * 24 + len(ham.c) * 24,
               "d2h_bytes_per_step": state_bytes + 16, "ms_per_step": 1000.0 * el}

    cpu = None
    if world == 1 and not a.skip_extras:
        rate, k, threads, el, stride, loc = oracle_rate(a.n, rx, rz, rt, 12.0, basis, a.terms)
        cpu = {"value": rate, "unit": "rotations/s", "cores": threads, "kind": "oracle",
               "sample": (f"every {stride}th rotation of the first Trotter step ({k} rotations, mean locality "
                          f"{loc:.2f} vs {float(synth.locality(rx, rz).mean()):.2f} for the whole list) at "
                          f"n={a.n}, complex128 gate-decomposed ({el:.1f} s)")}
        import oracle
        oracle.set_num_threads(1)
        try:
            rate1, k1, _, el1, stride1, _ = oracle_rate(a.n, rx, rz, rt, 4.0, basis, a.terms)
        finally:
            oracle.set_num_threads(0)
        cpu["single_thread"] = {"value": rate1, "unit": "rotations/s", "cores": 1,
                                "sample": f"every {stride1}th rotation of the first step ({k1}), one thread "
                                          f"({el1:.1f} s)"}

    if rank != 0:
        return 0
    passes = main["sweeps"]
    line = {
        "metric": METRIC, "value": value, "unit": "rotations/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": a.dtype, "data": "synthetic (seeded JW-shaped Hamiltonian)",
        "config": dict(config_dict(a, a.dtype), fusion_depth=main["dmax"],
                       fusion_depth_source=(tuning[a.dtype]["source"] if a.fusion_depth < 0
                                            else "--fusion-depth")),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": main["clocks"],
        "passes_per_step": passes, "runs_per_step": main["runs"], "diag_passes_per_step": main["diag_runs"],
        "rotations_per_pass": main["nrot"] / max(1, passes),
        "effective_gbs": R * sweep_bytes / (ms_step / 1000.0) / 1e9,
        "rescaled_runtime_s": (ms_step / 1000.0) / (R * (1 << a.n)),
        "plan_ms": main["plan_ms"], "energy": main["energy"], "norm2": main["norm2"],
        "fusion_depth_tuning": tuning or None,
        "kernels_timing": "event pair around every launch (no chaining between passes)",
        "kernels": {k: {"launches": v[0], "ms": v[1], "gbs": (v[2] / (v[1] / 1000.0) / 1e9) if v[1] else None,
                        "tflops": (v[3] / (v[1] / 1000.0) / 1e12) if v[1] else None}
                    for k, v in per_launch["trace"].items()},
    }
    line.update(extras)
    prec = extras.get("precision")
    if prec:
        # the per-result errors against the FP64 oracle, for the headline precision
        # and for complex128
        line["infidelity_vs_oracle"] = prec[a.dtype]["infidelity_vs_oracle_sampled"]
        line["energy_error_vs_oracle"] = prec[a.dtype]["energy_error_vs_oracle"]
        line["max_abs_vs_oracle"] = prec[a.dtype]["max_abs_vs_oracle"]
        line["c128_max_abs_vs_oracle"] = prec["c128"]["max_abs_vs_oracle"]
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


GOLDEN = os.path.join(ROOT, "tests", "golden", "full_n24_trotter.npz")


def precision_report(capi, a, ham, rx, rz, rt, basis, sh):
    """Both precisions against the oracle's values for this workload (stored by
    tests/golden/make_full_size.py: the FP64 gate-level oracle's amplitudes at
    8192 seeded non-zero indices plus the largest ones, its norm and <H>).
    Complex64: infidelity of the stored sub-vector, largest amplitude error,
    energy error; complex128: largest amplitude error and energy error.  The
    oracle's <H> is divided by its norm (its Hadamard passes drift the norm by a
    uniform factor of ~1 + 2.6e-11)."""
    if not os.path.exists(GOLDEN):
        return None
    g = np.load(GOLDEN)
    if (int(g["n"]), int(g["terms"]), int(g["seed"]), float(g["dt"]), int(g["steps"])) != \
            (a.n, a.terms, a.seed, a.dt, a.trotter_steps):
        return None
    idx, want = g["indices"], g["amps"]
    e_orc = float(g["energy"]) / float(g["norm2"])
    out = {"reference": f"FP64 gate-level oracle, {len(idx)} stored amplitudes of the final state "
                        f"(8192 seeded draws among its {int(g['nonzero_count'])} non-zero ones, the 16 largest "
                        f"and the initial basis state), its <H> / norm",
           "oracle_energy": e_orc}
    for dtype in ("c64", "c128"):
        plan = capi.plan_create(a.n, dtype, rx, rz, rt, a.fusion_depth, sh)
        sv = capi.sv_alloc(a.n, dtype, sh)
        try:
            capi.sv_set_basis_state(sv, basis)
            capi.plan_apply(sv, plan)
            e, nrm = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
            got = capi.sv_to_host(sv, True)[idx].astype(np.complex128)
        finally:
            capi.sv_free(sv)
            capi.plan_free(plan)
        ov = np.vdot(want, got)
        inf = float(1.0 - abs(ov) ** 2 / (np.vdot(want, want).real * np.vdot(got, got).real))
        out[dtype] = {"max_abs_vs_oracle": float(np.max(np.abs(got - want))),
                      "infidelity_vs_oracle_sampled": inf, "energy": e,
                      "energy_error_vs_oracle": abs(e - e_orc), "norm2_minus_1": nrm - 1.0}
    return out


def probe_peaks(capi, torch, reps: int = 3) -> dict:
    """Measured arithmetic peaks on this GPU: FP64 FMA, 32x32->64 integer
    multiply-add and packed FP32x2 FMA rates from the library's probe kernels (grids of 8 CTAs per SM,
    CUDA events on the launching stream, best of `reps` launches), with the SM
    clock sampled during the launches; ops x 2 for FLOP/s (x 4 for the packed
    FP32x2 FMA)."""
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = 8 * sms
    buf = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    out = {"blocks": blocks, "threads_per_block": 256, "chains_per_thread": 8}
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    for kind, name, iters in ((0, "fp64_fma", 4000), (1, "int_mul_wide", 40000), (2, "fp32x2_fma", 40000)):
        capi.sv_probe_rate(kind, blocks, 16, buf.data_ptr(), sh)  # warm
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(own)
            ops = capi.sv_probe_rate(kind, blocks, iters, buf.data_ptr(), sh)
            e1.record(own)
            own.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name] = {"ops_per_s": ops / (best / 1000.0), "ms": best, "ops": ops}
    out["fp64_tflops"] = 2.0 * out["fp64_fma"]["ops_per_s"] / 1e12
    out["int_mul_wide_tops"] = out["int_mul_wide"]["ops_per_s"] / 1e12
    out["fp32_tflops"] = 4.0 * out["fp32x2_fma"]["ops_per_s"] / 1e12
    out["clocks"] = clocks.stop()
    return out


def large_compare(capi, torch, barrier, n: int = 29, terms: int = 5000, seed: int = 1):
    """n = 29 in both precisions (8 GiB and 4 GiB): one symmetric second-order
    Trotter step of the 5000-term JW-shaped Hamiltonian (9,999 merged rotations)
    from the Hartree-Fock state, <H> after it; complex64 against the complex128
    GPU run: infidelity of the whole state and |dE|.  Device time per step."""
    ham = synth.jw_hamiltonian(n, terms, seed)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 1, 2, True)
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    basis = synth.hartree_fock_index(n // 2)
    res = {}
    for dtype in ("c128", "c64"):
        t = torch.zeros(1 << n, dtype=torch.complex128 if dtype == "c128" else torch.complex64, device="cuda")
        sv = capi.sv_wrap(t.data_ptr(), n, dtype, sh)
        plan = capi.plan_create(n, dtype, rx, rz, rt, -1, sh)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        try:
            capi.sv_set_basis_state(sv, basis)
            barrier()
            e0.record(own)
            capi.plan_apply(sv, plan)
            e1.record(own)
            e, nrm = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
            capi.sv_materialize(sv)
            barrier()
            passes = capi.plan_sweeps(plan)
        finally:
            capi.plan_free(plan)
            capi.sv_free(sv)
        ms = e0.elapsed_time(e1)
        res[dtype] = (t, e, nrm, ms, passes)
    t128, e128, n128, ms128, p128 = res["c128"]
    t64, e64, n64, ms64, p64 = res["c64"]
    g = t64.to(torch.complex128)
    ov = torch.vdot(t128, g)
    inf = float(1.0 - (ov.abs() ** 2) / (torch.vdot(t128, t128).real * torch.vdot(g, g).real))
    del g, t64, t128
    torch.cuda.empty_cache()
    return {"n": n, "terms": terms, "rotations": len(rt),
            "c128": {"rotations_ms": ms128, "passes": p128, "rotations_per_s": len(rt) / (ms128 / 1000.0),
                     "energy": e128, "norm_drift": abs(n128 - 1.0)},
            "c64": {"rotations_ms": ms64, "passes": p64, "rotations_per_s": len(rt) / (ms64 / 1000.0),
                    "energy": e64, "norm_drift": abs(n64 - 1.0)},
            "c64_infidelity_vs_c128": inf, "c64_energy_error_vs_c128": abs(e64 - e128),
            "reference": "the complex128 GPU run of the same step (FP64-class reference)"}


def shard_measure(capi, torch, barrier, n: int = 24, terms: int = 2000, seed: int = 1, gs=(1, 2, 3)):
    """The global-qubit sharded path on one GPU: the first Trotter step of the
    n = 24 workload (2000 rotations, complex64) with the state split into 2^g
    slices that all live on this GPU (InProcessComm: an exchange is a device
    copy standing in for the transfer between GPUs), then <H>.  Wall time with
    the stream synchronised, against the same step on one unsharded state;
    counts the exchanges and the rotations run on pair states."""
    from paper_2602_09020_gb300.shard import InProcessComm, ShardedState
    ham = synth.jw_hamiltonian(n, terms, seed)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 1, 1, False)
    basis = synth.hartree_fock_index(n // 2)
    out = {"n": n, "dtype": "c64", "rotations": len(rt), "rows": []}
    sv = capi.sv_alloc(n, "c64", int(torch.cuda.current_stream().cuda_stream))
    try:
        for rep in range(2):
            capi.sv_set_basis_state(sv, basis)
            barrier()
            t0 = time.perf_counter()
            capi.apply_pauli_rotations(sv, rx, rz, rt)
            e1, _ = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
            barrier()
            single = time.perf_counter() - t0
    finally:
        capi.sv_free(sv)
    out["unsharded_ms"] = 1000.0 * single
    for g in gs:
        comm = InProcessComm(1 << g)
        st = ShardedState(n, "c64", g, comm)
        try:
            steps = capi.shard_rotations(n, g, 0, rx, rz, rt)[0]
            for rep in range(2):
                st.set_basis_state(basis)
                barrier()
                t0 = time.perf_counter()
                st.apply_pauli_rotations(rx, rz, rt)
                e, _ = st.expval_pauli_sum(ham.x, ham.z, ham.c)
                barrier()
                el = time.perf_counter() - t0
        finally:
            st.close()
        pair_rot = sum(c for k, _, _, c in steps if k == 1)
        out["rows"].append({"global_qubits": g, "slices": 1 << g, "ms": 1000.0 * el,
                            "rotations_per_s": len(rt) / el, "rotation_steps": len(steps),
                            "exchanges_for_rotations": sum(1 for k, *_ in steps if k == 1),
                            "rotations_on_pair_states": pair_rot, "energy": e,
                            "energy_minus_unsharded": e - e1})
    return out


def locality_measure(capi, torch, n: int, dtype: str, barrier, terms: int = 100,
                     localities=(4, 8, 12, 16, 20, 24)):
    """The paper's locality study (Sec. "Evaluation on Random Hamiltonians"): one
    first-order Trotter step of a random k-local Hamiltonian with 100 terms at
    each locality L, run as fused rotations and gate-decomposed on the same GPU.
    Device time (CUDA events on the states' stream); the fused path should be
    flat in L, the gate path linear in L."""
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    rows = []
    for L in localities:
        if L > n:
            continue
        ham = synth.random_klocal_hamiltonian(n, terms, L, seed=1000 + L)
        rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 1.0, 1, 1, False)
        sv = capi.sv_alloc(n, dtype, sh)
        capi.sv_set_basis_state(sv, 0)
        plan = capi.plan_create(n, dtype, rx, rz, rt, -1, sh)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        capi.plan_apply(sv, plan)  # warm both paths
        capi.apply_pauli_rotations_gates(sv, rx[:2], rz[:2], rt[:2])
        barrier()
        e[0].record(own)
        capi.plan_apply(sv, plan)
        e[1].record(own)
        e[2].record(own)
        ngates = capi.apply_pauli_rotations_gates(sv, rx, rz, rt)
        e[3].record(own)
        barrier()
        fused_ms, gate_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
        passes = capi.plan_sweeps(plan)
        capi.plan_free(plan)
        capi.sv_free(sv)
        rows.append({"L": L, "rotations": len(rt), "fused_ms": fused_ms, "fused_passes": passes,
                     "gates": ngates, "gate_ms": gate_ms, "speedup": gate_ms / fused_ms})
    return {"n": n, "terms": terms, "dtype": dtype, "rows": rows}


def staircase_stream(x: int, z: int, theta: float, out: list) -> None:
    """Append the textbook gate decomposition of exp(-i theta/2 P) (basis
    change, CNOT ladder over the support, Rz on its top qubit, undo) as
    (code, q0, q1, theta) tuples in the SV_CG numbering."""
    H, S, SDG, CNOT, RZ = 0, 1, 2, 6, 11
    sup = [q for q in range(64) if ((x | z) >> q) & 1]
    basis = []
    for q in sup:
        if (x >> q) & 1 and (z >> q) & 1:
            basis += [(SDG, q, -1, 0.0), (H, q, -1, 0.0)]
        elif (x >> q) & 1:
            basis.append((H, q, -1, 0.0))
    ladder = [(CNOT, a, b, 0.0) for a, b in zip(sup, sup[1:])]
    undo = [((S if g == SDG else g), q, -1, 0.0) for (g, q, _, _) in reversed(basis)]
    out += basis + ladder + [(RZ, sup[-1], -1, theta)] + ladder[::-1] + undo


def cfhs_measure(capi, torch, n: int, dtype: str, rx, rz, rt, ham, basis: int, barrier):
    """The hybrid simulator's use case (Sec. "Description of the Clifford-fullstate
    hybrid simulation"): the first Trotter step written out as a gate-level
    circuit -- every rotation as basis changes, a CNOT ladder, one Rz and the
    undo -- fed to cfhs_apply_gates.  The Clifford gates only update the host
    frame; the Rz gates reach the GPU as fused rotations about the frame's Z_q.
    Wall time around the call (host frame updates, planning and the GPU work);
    the energy through the frame is compared with the direct rotation path."""
    stream = []
    for x, z, t in zip(rx, rz, rt):
        if int(x) | int(z):
            staircase_stream(int(x), int(z), float(t), stream)
    arr = np.array(stream, dtype=np.float64)
    code = np.ascontiguousarray(arr[:, 0].astype(np.int32))
    q0 = np.ascontiguousarray(arr[:, 1].astype(np.int32))
    q1 = np.ascontiguousarray(arr[:, 2].astype(np.int32))
    th = np.ascontiguousarray(arr[:, 3])
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    lib = capi.lib()
    sv = capi.sv_alloc(n, dtype, sh)
    f = capi.cliff_create(n)
    ref = capi.sv_alloc(n, dtype, sh)
    try:
        capi.sv_set_basis_state(sv, basis)
        capi._check(lib.cfhs_apply_gates(sv, f, code.ctypes.data, q0.ctypes.data, q1.ctypes.data, th.ctypes.data,
                                         len(code)))  # warm (first launches)
        capi.cliff_reset(f)
        capi.sv_set_basis_state(sv, basis)
        barrier()
        t0 = time.perf_counter()
        capi._check(lib.cfhs_apply_gates(sv, f, code.ctypes.data, q0.ctypes.data, q1.ctypes.data, th.ctypes.data,
                                         len(code)))
        barrier()
        wall = time.perf_counter() - t0
        e_cfhs, _ = capi.cfhs_expval(sv, f, ham.x, ham.z, ham.c)
        capi.sv_set_basis_state(ref, basis)
        capi.apply_pauli_rotations(ref, rx, rz, rt)
        e_ref, _ = capi.expval_pauli_sum(ref, ham.x, ham.z, ham.c)
    finally:
        capi.cliff_free(f)
        capi.sv_free(sv)
        capi.sv_free(ref)
    n_rz = int(np.count_nonzero(code == 11))
    return {"rotations": n_rz, "gates": len(code), "clifford_gates": len(code) - n_rz, "wall_ms": 1000.0 * wall,
            "rotations_per_s": n_rz / wall, "gates_per_s": len(code) / wall,
            "energy_through_frame": e_cfhs, "energy_direct": e_ref,
            "sample": "the first Trotter step as a gate-level circuit"}


def large_measure(capi, torch, barrier, n: int = 30, terms: int = 5000, seed: int = 1):
    """The large-state workload: complex64 at n = 30 (8 GiB), a 5000-term JW-shaped
    Hamiltonian, one symmetric second-order Trotter step (neighbours merged:
    9,999 rotations) from the Hartree-Fock state, then <H> and the norm.  Device
    time of one step after one warm-up step; the norm drift is |<psi|psi> - 1|."""
    ham = synth.jw_hamiltonian(n, terms, seed)
    rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, 0.05, 1, 2, True)
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    plan = capi.plan_create(n, "c64", rx, rz, rt, -1, sh)
    sv = capi.sv_alloc(n, "c64", sh)
    basis = synth.hartree_fock_index(n // 2)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    try:
        capi.sv_set_basis_state(sv, basis)
        capi.plan_apply(sv, plan)  # warm
        capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
        capi.sv_set_basis_state(sv, basis)
        barrier()
        e0.record(own)
        capi.plan_apply(sv, plan)
        e1.record(own)
        e, nrm = capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
        e2.record(own)
        barrier()
        passes = capi.plan_sweeps(plan)
        runs = capi.plan_stats(plan)[1]
    finally:
        capi.sv_free(sv)
        capi.plan_free(plan)
    rot_ms, h_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    return {"n": n, "dtype": "c64", "terms": terms, "rotations": len(rt), "passes": passes, "runs": runs,
            "rotations_ms": rot_ms, "expval_ms": h_ms, "rotations_per_s": len(rt) / (rot_ms / 1000.0),
            "hbm_fraction_algorithmic": passes * 2.0 * 8 * (1 << n) / (rot_ms / 1000.0) / 1e9 / peaks()["hbm_gbs"],
            # the same with every run as its own sweep (the HBM rate one-run
            # passes would need to keep pace)
            "run_equivalent_hbm_frac": runs * 2.0 * 8 * (1 << n) / (rot_ms / 1000.0) / 1e9 / peaks()["hbm_gbs"],
            "energy": e, "norm_drift": abs(nrm - 1.0)}


def adjoint_measure(capi, torch, barrier, n: int = 20, n_rot: int = 500, n_obs: int = 300):
    """The gradient workload: E(theta) = <psi(theta)|H|psi(theta)> and all 500
    dE/dtheta_j at n = 20 by the adjoint sweep (rotation_grads), in both
    precisions; wall time of one call after a warm-up call."""
    x, z, th, obs = synth.adjoint_workload(n, n_rot, n_obs, seed=20)
    basis = synth.hartree_fock_index(n // 2)
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    out = {"n": n, "rotations": n_rot, "observable_terms": n_obs}
    for dtype in ("c128", "c64"):
        sv = capi.sv_alloc(n, dtype, sh)
        try:
            capi.sv_set_basis_state(sv, basis)
            capi.rotation_grads(sv, x, z, th, obs.x, obs.z, obs.c)  # warm
            barrier()
            t0 = time.perf_counter()
            e, g = capi.rotation_grads(sv, x, z, th, obs.x, obs.z, obs.c)
            barrier()
            el = time.perf_counter() - t0
        finally:
            capi.sv_free(sv)
        out[dtype] = {"ms": 1000.0 * el, "gradients_per_s": n_rot / el, "energy": e,
                      "max_abs_grad": float(np.abs(g).max())}
        if dtype == "c128":
            e128, g128 = e, g
        else:
            out[dtype]["energy_error_vs_c128"] = abs(e - e128)
            out[dtype]["max_grad_error_vs_c128"] = float(np.abs(g - g128).max())
    return out


def batch_measure(capi, torch, stream, sh, barrier, reps: int = 3):
    """64 independent JW-shaped problems, n ~ U{12..22}, complex64, T ~ U{100..800},
    dt ~ U[0.01, 0.2], 1..8 first-order steps each.  The states live on a stream
    of their own: the legacy default stream cannot be captured into a graph."""
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    wl = synth.batch_workload(64, seed=4)
    lists = [capi.trotter_expand(c.ham.x, c.ham.z, c.ham.c, c.dt, c.steps, 1, False) for c in wl]
    states, plans, total = [], [], 0
    out = {"states": len(wl), "n_range": [min(c.n for c in wl), max(c.n for c in wl)]}
    try:
        for circ in wl:
            states.append(capi.sv_alloc(circ.n, "c64", sh))
        # fusion depth from the library's batched autotuner: the persistent
        # launch itself timed at depths 1..4; the states are its scratch
        t0 = time.perf_counter()
        depth, bms = capi.batch_autotune(states, lists, max_depth=4, reps=2)
        out.update({"fusion_depth": depth, "tune_s": time.perf_counter() - t0,
                    "ms_per_launch_by_depth": {str(d + 1): v for d, v in enumerate(bms) if v > 0}})
        for sv, circ, (rx, rz, rt) in zip(states, wl, lists):
            total += len(rt)
            capi.sv_set_basis_state(sv, circ.basis_state)
            plans.append(capi.plan_create(circ.n, "c64", rx, rz, rt, -1, sh))
        out["rotations"] = total
        capi.batch_run(states, plans, use_graph=True)  # builds, captures, warms
        barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            capi.batch_run(states, plans, use_graph=True)
        barrier()
        el = (time.perf_counter() - t0) / reps
        grid, multi, used_graph = capi.batch_info()
        out.update({"persistent_ms": 1000 * el, "persistent_rotations_per_s": total / el, "grid_ctas": grid,
                    "multi_cta_states": multi, "graph_mode": used_graph})
        for sv, p in zip(states, plans):  # warm the one-launch-per-pass path
            capi.plan_apply(sv, p)
        barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            for sv, p in zip(states, plans):
                capi.plan_apply(sv, p)
        barrier()
        el2 = (time.perf_counter() - t0) / reps
        launches = sum(capi.plan_stats(p)[1] for p in plans)
        # algorithmic bytes of the persistent launch: every pass of every state
        # reads and writes that state once (2 x 8 x 2^n bytes)
        nbytes = sum(capi.plan_stats(p)[1] * 2.0 * 8.0 * (1 << c.n) for p, c in zip(plans, wl))
        pk = peaks()
        out.update({"per_state_ms": 1000 * el2, "per_state_rotations_per_s": total / el2,
                    "per_state_launches": launches, "speedup": el2 / el,
                    "algorithmic_bytes": nbytes, "persistent_gbs": nbytes / el / 1e9,
                    "persistent_hbm_frac": nbytes / el / 1e9 / pk["hbm_gbs"],
                    "per_state_hbm_frac": nbytes / el2 / 1e9 / pk["hbm_gbs"],
                    "hbm_peak": pk["hbm_gbs"], "peak_source": pk["source"]})
    finally:
        for p in plans:
            capi.plan_free(p)
        for sv in states:
            capi.sv_free(sv)
    return out


def run_tour(a) -> int:
    """Every kernel family once, in one process, on states larger than L2: the
    complex64 state at n = 25 (256 MB) and the complex128 state at n = 24
    (256 MB), a 100-term JW Hamiltonian, one first-order step, <H>, frame
    materialisation, a few gate-decomposed rotations, one Pauli measurement, a
    50-rotation adjoint gradient, then a 16-state batched launch.  Kernels are
    timed with the library's per-launch trace (the adjoint's work states record
    into their owner's trace); the JSON line gives, per kernel, launches, device
    time per launch and algorithmic bytes per second against the measured HBM
    copy peak.  A profiler run over the same command adds the DRAM counters."""
    import torch
    from paper_2602_09020_gb300 import capi
    torch.cuda.set_device(0)
    own = torch.cuda.Stream()
    sh = int(own.cuda_stream)
    pk = peaks()
    out = {"tour": True, "hbm_peak_gbs": pk["hbm_gbs"], "peak_source": pk["source"], "kernels": {}}
    for dtype, n in (("c64", 25), ("c128", 24)):
        ham = synth.jw_hamiltonian(n, 100, a.seed)
        rx, rz, rt = capi.trotter_expand(ham.x, ham.z, ham.c, a.dt, 1, 1, False)
        ax, az, ath, obs = synth.adjoint_workload(n, 50, 100, seed=a.seed)
        # one rotation with X and Y parts on three qubits for the gate path
        gx, gz = np.array([0b10011], dtype=np.uint64), np.array([0b00110], dtype=np.uint64)
        sv = capi.sv_alloc(n, dtype, sh)
        plan = capi.plan_create(n, dtype, rx, rz, rt, -1, sh)
        try:
            capi.sv_trace_start(sv)
            capi.sv_set_basis_state(sv, synth.hartree_fock_index(n // 2))
            capi.plan_apply(sv, plan)
            capi.expval_pauli_sum(sv, ham.x, ham.z, ham.c)
            capi.frame_apply_pauli(sv, "Y", 3)
            capi.sv_materialize(sv)
            capi.apply_pauli_rotations_gates(sv, gx, gz, [0.3])
            capi.cfhs_measure_pauli(sv, None, 0b1010, 0b0110, 0.5)
            capi.rotation_grads(sv, ax, az, ath, obs.x, obs.z, obs.c)
            rows = capi.sv_trace_stop(sv)
        finally:
            capi.plan_free(plan)
            capi.sv_free(sv)
        out["kernels"][f"{dtype}_n{n}"] = {
            k: {"launches": v[0], "us_per_launch": 1000.0 * v[1] / v[0],
                "algorithmic_gbs": (v[2] / (v[1] / 1000.0) / 1e9) if v[1] else None,
                "frac_of_hbm": (v[2] / (v[1] / 1000.0) / 1e9 / pk["hbm_gbs"]) if v[1] else None}
            for k, v in rows.items()}
    # the batched launch: 16 states, n ~ U{12..22}
    wl = synth.batch_workload(16, seed=a.seed)
    states, plans, nbytes = [], [], 0.0
    try:
        for c in wl:
            rx, rz, rt = capi.trotter_expand(c.ham.x, c.ham.z, c.ham.c, c.dt, c.steps, 1, False)
            sv = capi.sv_alloc(c.n, "c64", sh)
            capi.sv_set_basis_state(sv, c.basis_state)
            states.append(sv)
            plans.append(capi.plan_create(c.n, "c64", rx, rz, rt, 4, sh))
            nbytes += capi.plan_stats(plans[-1])[1] * 2.0 * 8.0 * (1 << c.n)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(own)
        capi.batch_run(states, plans, use_graph=False)
        e1.record(own)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["kernels"]["batched_16_states"] = {"k_batch": {
            "launches": 1, "us_per_launch": 1000.0 * ms, "algorithmic_gbs": nbytes / (ms / 1000.0) / 1e9,
            "frac_of_hbm": nbytes / (ms / 1000.0) / 1e9 / pk["hbm_gbs"],
            "note": "one launch timed with CUDA events around batch_run (the call also uploads the "
                    "states' frames); bytes = passes x 2 x 8 x 2^n over the states"}}
    finally:
        for p in plans:
            capi.plan_free(p)
        for sv in states:
            capi.sv_free(sv)
    print(json.dumps(out), flush=True)
    return 0


def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)
    if a.tour:
        return run_tour(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
