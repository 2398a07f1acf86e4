#!/usr/bin/env python
"""Benchmark: gate bootstraps per second of CGGI gate bootstrapping on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl arx|reference]
                    [--workload netlists|gates|dag|matmul|simon|serve|alu] [--mode graph|plain]

A step is one evaluation of the workload's netlist through the C-ABI
(arx_plan_run): every wave's blind rotations (mod switch, n CMux external
products, sample extraction) and key switches, all on the GPU.  The default
workload is the plain-netlist configuration: a 32-bit ripple-carry adder and an
8x8-bit array multiplier (CGGI n=630, N=1024, Bg=2^7, l=3, key switch 2^2 x 8),
evaluated one wave per launch.  Inputs are synthetic (seeded keys, bits, netlists).

value   = bootstraps per step (MUX counts two) / mean device time per step,
          inputs resident in HBM, L2 flushed (256 MiB write) between steps;
e2e     = the same through the C-ABI with pinned HOST buffers (H2D of the inputs,
          D2H of the outputs inside the timed region);
latency = p50 / p99 of the per-step device time (netlist latency);
roofline= the blind-rotation kernels' modular multiplications per second against
          the IMAD-pipe peak (an integer-ALU roofline);
batched / served = the default line also carries the batched-persistent figure
          (random levelized DAG of 65,536 gates, one CUDA graph) and the served
          figure (4 clients with their own keys, Poisson arrivals), each with its
          own roofline fraction and clocks (--no-extra leaves them out);
cpu_baseline = the plain C oracle on this host's cores evaluating the WHOLE
          netlist once with the same keys and inputs; every wire of the GPU run
          (inputs, all gate outputs) is compared with the oracle's bit for bit,
          and that comparison is part of `verified`.
With --impl reference the oracle itself is the timed arm: its K timed steps are
K consecutive slices of the netlist's waves, so that together they evaluate the
whole netlist once (about 20 s on 16 cores), each slice on the previous slices'
outputs.  Under torchrun (N > 1) every rank evaluates its own replica on its own
GPU (no collective on the data path); value sums all ranks, time is the max over
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2306_11006_gb300 import inputs as I  # noqa: E402

METRIC = "gate bootstraps/sec on 1 GB300 (bit-exact vs oracle); netlist p50/p99 latency ms"
LWE_N = 630
# blind rotation work per bootstrap in 32-bit modular multiply-accumulates (two CRT
# primes): per CMux, (2l + 2) length-1024 transforms x 5120 butterflies + 2 x 2l x 1024
# MACs, each once per prime (l = 3: 8 transforms, 12 MAC rows).


def modmul_per_cmux(l: int = 3) -> int:
    return 2 * ((2 * l + 2) * 5120 + 2 * 2 * l * 1024)


MODMUL_PER_CMUX = modmul_per_cmux(3)
# integer-ALU peak: 152 SMs x 2070 MHz x 64 IMAD-capable lanes per clock, a
# Shoup or Montgomery modular multiply taking 3 of those lane slots
ALU_PEAK_TMODMUL = 152 * 2.070e9 * 64 / 3 / 1e12
# DRAM bytes (read + write) per launch from one ncu capture of the current kernel
# build (profiles/): the key once per launch.  Only kernels listed here report it.
TRAFFIC_PER_LAUNCH = {
    "br_cluster16_kernel": 62.06e6 + 2.46e6,  # 7 gates
    "br_cluster16_kernel<L=2>": 33.66e6 + 0.0e6,  # 7 gates, n = 512, l = 2
    "br_cluster8_kernel": 62.06e6 + 2.08e6,   # 8 gates
    "br_kernel<1,6>": 66.82e6 + 3.14e6,       # 912 gates
    "br_kernel<1,6,L=2>": 37.97e6 + 0.06e6,   # 912 gates, n = 512, l = 2
    "br_cluster8_kernel<L=2>": 33.68e6 + 6.40e6,  # 8 gates, n = 512, l = 2
    "br_kernel<4,1,L=2>": 34.26e6 + 0.001e6,      # 128 gates, n = 512, l = 2
}
KERNEL_OF_H = {12: "br_cluster_kernel", 24: "br_cluster4_kernel", 48: "br_cluster8_kernel",
               40: "br_cluster8_kernel<L=2>", 80: "br_cluster16_kernel<L=2>", 96: "br_cluster16_kernel"}


def kernel_name(H: int, GT: int) -> str:
    return KERNEL_OF_H.get(H, f"br_kernel<{H - 100},{GT},L=2>" if H > 100 else f"br_kernel<{H},{GT}>")


def replica_max_ms(ms: float, world: int, device="cpu") -> float:
    """The job's time under replicas: the max over ranks of each rank's time."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_step: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_step * steps * world / (max_ms / 1e3)


def replica_seed(base: int, rank: int) -> int:
    """Each replica evaluates its own inputs (no rank shares an input seed)."""
    return base + rank


def workload(name: str, gates: int = 64, blocks: int = 8, copies: int = 1):
    if name == "netlists":
        if copies > 1:  # independent copies whose ready gates share every launch
            return I.union([I.ripple_carry_adder(32), I.array_multiplier(8)] * copies,
                           name=f"{copies}x(adder32+mult8)"), \
                f"{copies} copies of the 32-bit ripple-carry adder + 8x8 array multiplier, batched per wave"
        return I.union([I.ripple_carry_adder(32), I.array_multiplier(8)], name="adder32+mult8"), \
            "32-bit ripple-carry adder + 8x8 array multiplier (plain netlists, one wave per launch)"
    if name in ("gates", "gates64"):
        g = gates
        t = I.random_gate_types(1, g)
        nl = I.Netlist(2 * g, t, np.arange(g, dtype=np.uint32), np.arange(g, 2 * g, dtype=np.uint32),
                       np.zeros(g, np.uint32), np.arange(2 * g, 3 * g, dtype=np.uint32), f"gates{g}")
        return nl, f"{g} independent 2-input gates (one wave)"
    if name == "dag":
        return I.random_dag(seed=3), "random levelized DAG, 65,536 gates over 40 waves, 5% MUX"
    if name == "simon":
        from paper_2306_11006_gb300 import simon as S
        nl = S.simon_netlist(blocks=blocks)
        return nl, f"Simon-128/128, {blocks} blocks x 68 rounds (transciphering), one launch per wave"
    if name == "matmul":
        return I.union([I.matmul4x4() for _ in range(8)], name="8x matmul4x4"), \
            "8 simultaneous 4x4 8-bit matrix products (16-bit accumulators), one launch per wave"
    raise SystemExit(f"unknown workload {name}")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region
    (the samples go to a temporary file that is removed once read)."""

    def __init__(self, gpu: int):
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="arx_clocks_", suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            if getattr(self, "f", None):
                self.f.close()
            os.unlink(self.path)
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


# ---------------------------------------------------------------------------
# the oracle leg (CPU): the timed baseline and the bit-exact check of the GPU run
# ---------------------------------------------------------------------------
def all_wires(nl):
    """The same netlist with every wire (inputs and gate outputs) as an output."""
    W = nl.num_inputs + nl.num_gates
    return I.Netlist(nl.num_inputs, nl.type, nl.in0, nl.in1, nl.in2, np.arange(W, dtype=np.uint32), nl.name)


def wave_slices(waves: np.ndarray, k: int):
    """Gate ids of k consecutive groups of waves (wave order, gate order inside a wave)."""
    depth = int(waves.max()) + 1 if len(waves) else 0
    order = np.argsort(waves, kind="stable")
    bounds = [round(j * depth / k) for j in range(k + 1)]
    w = waves[order]
    return [order[(w >= bounds[j]) & (w < bounds[j + 1])] for j in range(k)]


def slice_netlist(nl, gates: np.ndarray):
    """One slice of gates as a netlist of its own: every wire of the full netlist is
    an input of the slice, except the slice's own gate outputs, which become its
    gates (wire W + j for the slice's j-th gate, W = all wires); outputs = the
    slice's gates.  Pure re-indexing, no arithmetic."""
    W = nl.num_inputs + nl.num_gates
    pos = np.full(W, -1, np.int64)
    pos[nl.num_inputs + gates] = np.arange(len(gates))

    def remap(ids):
        ids = np.asarray(ids, np.int64)[gates]
        p = pos[ids]
        return np.where(p >= 0, W + p, ids).astype(np.uint32)

    return I.Netlist(W, np.asarray(nl.type)[gates], remap(nl.in0), remap(nl.in1), remap(nl.in2),
                     np.arange(W, W + len(gates), dtype=np.uint32), f"{nl.name}[slice]")


def oracle_inputs(nl, n: int, l: int, rank: int = 0):
    """Oracle key context and input ciphertexts from the same seeded randomness as
    the GPU arm (keys seed 0; bits and encryption seeds 1000 / 2000 + rank)."""
    from oracle import oracle as O
    kr = I.key_randomness(0, n, l=l)
    bsk, ksk = O.keygen(kr)
    ctx = O.Context(n, bsk, ksk)
    bits = I.random_bits(replica_seed(1000, rank), nl.num_inputs)
    m, e = I.encryption_randomness(replica_seed(2000, rank), nl.num_inputs, n)
    return O, kr, ctx, bits, O.encrypt(n, kr.s, m, e, bits)


def single_core_rate(O, ctx, nl, wires, n: int, gates: int = 8):
    """Oracle on one thread: the first `gates` bootstrapped gates of the netlist on
    their (oracle-computed) input wires."""
    g = np.array([k for k in range(nl.num_gates) if I.BOOTSTRAPS[int(nl.type[k])]][:gates], np.int64)
    if len(g) == 0:
        return None
    a, b, c = (wires[np.asarray(x, np.int64)[g]] for x in (nl.in0, nl.in1, nl.in2))
    t0 = time.perf_counter()
    ctx.gates(np.asarray(nl.type)[g].astype(np.uint8), a, b, c, nthreads=1)
    dt = time.perf_counter() - t0
    boots = int(sum(I.BOOTSTRAPS[int(t)] for t in np.asarray(nl.type)[g]))
    return {"value": boots / dt, "unit": "bootstraps/s", "cores": 1,
            "sample": f"the netlist's first {len(g)} bootstrapped gates on one thread, {dt:.1f} s"}


def oracle_leg(nl, n: int, l: int, gpu_wires=None, sample_gates: int = 48, gates=None):
    """The plain C oracle on this host's cores.  Small netlists (config 2) are
    evaluated in full with every wire kept, timed, and -- given gpu_wires(ids), a
    reader of the GPU run's wires -- compared bit for bit, every wire.  Large
    netlists are sampled: the given `gates` (else `sample_gates` gates drawn from
    the netlist), each evaluated by the oracle on the GPU run's input wires and
    compared with the GPU's output wire (and timed)."""
    cores = os.cpu_count() or 1
    O, kr, ctx, bits, ct_in = oracle_inputs(nl, n, l)
    boots_total = nl.num_bootstraps
    rec = {"unit": "bootstraps/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model()}
    if boots_total <= 2048:
        full = all_wires(nl)
        t0 = time.perf_counter()
        wires = ctx.eval_netlist(full, ct_in, nthreads=cores)
        dt = time.perf_counter() - t0
        rec.update({"value": boots_total / dt, "seconds": dt,
                    "sample": f"the whole netlist ({nl.num_gates} gates, {boots_total} bootstraps) evaluated "
                              f"once wave by wave, {dt:.1f} s on {cores} threads"})
        sc = single_core_rate(O, ctx, nl, wires, n)
        if sc:
            rec["single_core"] = sc
        ok_dec = bool(np.array_equal(O.decrypt(n, kr.s, wires[nl.outputs])[0], nl.plain_eval(bits)))
        check = {"wires_compared": None, "mismatched": None, "oracle_outputs_decrypt_ok": ok_dec}
        if gpu_wires is not None:
            got = gpu_wires(np.arange(len(wires), dtype=np.uint32))
            bad = int(np.count_nonzero(np.any(got != wires, axis=1)))
            check.update({"wires_compared": int(len(wires)), "mismatched": bad})
        return rec, check
    # sampled form (large netlists): gates drawn from the netlist, GPU input wires
    rng = np.random.default_rng(11)
    boot_gates = np.array([k for k in range(nl.num_gates) if I.BOOTSTRAPS[int(nl.type[k])]], np.int64)
    g = np.sort(rng.choice(boot_gates, size=min(sample_gates, len(boot_gates)), replace=False))
    if gates is not None:
        g = np.sort(np.asarray(gates, np.int64))
    rec_check = {"wires_compared": 0, "mismatched": None}
    if gpu_wires is None:
        return None, rec_check
    a, b, c = (gpu_wires(np.asarray(x, np.uint32)[g]) for x in (nl.in0, nl.in1, nl.in2))
    t0 = time.perf_counter()
    got = ctx.gates(np.asarray(nl.type)[g].astype(np.uint8), a, b, c, nthreads=cores)
    dt = time.perf_counter() - t0
    boots = int(sum(I.BOOTSTRAPS[int(t)] for t in np.asarray(nl.type)[g]))
    what = "gates given" if gates is not None else "gates drawn from the netlist"
    rec.update({"value": boots / dt, "seconds": dt,
                "sample": f"{len(g)} {what}, each on the GPU run's input wires, {dt:.1f} s on {cores} threads"})
    bad = int(np.count_nonzero(np.any(got != gpu_wires((nl.num_inputs + g).astype(np.uint32)), axis=1)))
    return rec, {"wires_compared": int(len(g)), "mismatched": bad}


def run_reference(args, nl, desc):
    """The oracle as the timed arm: the K timed steps are K consecutive slices of the
    netlist's waves (wave order), each evaluated on the previous slices' outputs, so
    the K steps together evaluate the whole netlist once; W warm-up steps evaluate
    the first W slices beforehand (untimed)."""
    n, l = (512, 2) if args.paper_params else (LWE_N, 3)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    O, kr, ctx, bits, ct_in = oracle_inputs(nl, n, l)
    _, waves = O.levelize(nl)
    K = max(args.steps, 1)
    slices = [slice_netlist(nl, g) for g in wave_slices(waves, K)]
    gates_of = wave_slices(waves, K)
    W = nl.num_inputs + nl.num_gates

    def fresh():
        w = np.zeros((W, n + 1), np.uint32)
        w[: nl.num_inputs] = ct_in
        return w

    wires = fresh()
    for j in range(min(args.warmup, K)):  # warm-up: the first slices, untimed
        if len(gates_of[j]):
            wires[nl.num_inputs + gates_of[j]] = ctx.eval_netlist(slices[j], wires, nthreads=cores)
    wires = fresh()
    step_s = []
    for j in range(K):
        t0 = time.perf_counter()
        if len(gates_of[j]):
            wires[nl.num_inputs + gates_of[j]] = ctx.eval_netlist(slices[j], wires, nthreads=cores)
        step_s.append(time.perf_counter() - t0)
    total = sum(step_s)
    boots = nl.num_bootstraps
    ok = bool(np.array_equal(O.decrypt(n, kr.s, wires[nl.outputs])[0], nl.plain_eval(bits)))
    v = boots / total
    sc = single_core_rate(O, ctx, nl, wires, n)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "bootstraps/s", "n_gpus": args.gpus,
            "steps": K, "warmup": args.warmup, "ms_per_step": 1000.0 * total / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": desc, "lwe_n": n, "N": 1024, "gadget": f"l={l}, Bg=2^{7 if l == 3 else 10}",
                       "gates": nl.num_gates, "bootstraps_per_step": boots,
                       "waves": int(waves.max()) + 1 if len(waves) else 0,
                       "step": f"1/{K} of the netlist's waves in order; the {K} timed steps together are one "
                               f"full evaluation ({total:.1f} s)"},
            "latency_ms": {"full_netlist": 1000.0 * total},
            "verified": ok,
            "cpu_baseline": {"kind": "oracle", "cores": cores, "cpu_model": cpu_model(), "value": v,
                             "sample": f"the whole netlist ({boots} bootstraps) evaluated once, split over the "
                                       f"{K} timed steps, {total:.1f} s on {cores} threads",
                             "single_core": sc},
            "e2e": {"value": v, "unit": "bootstraps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def measure_plan(arx, torch, nl, desc, args, n, l, keyset, kr, dev, stream, steps, warmup, mode, world=1,
                 rank=0, e2e=True):
    """Times `steps` evaluations of one plan (after `warmup`), L2 flushed between
    steps; returns the record and the plan (still open) with its inputs."""
    bits = I.random_bits(replica_seed(1000, rank), nl.num_inputs)
    m, e = I.encryption_randomness(replica_seed(2000, rank), nl.num_inputs, n)
    ct_host = arx.client_encrypt(n, kr.s, m, e, bits)
    ct_in = torch.from_numpy(ct_host.view(np.int32)).to(dev)
    out = torch.zeros((len(nl.outputs), n + 1), dtype=torch.int32, device=dev)
    plan = arx.Plan(nl, keyset=keyset, mode=mode)
    boots = plan.bootstraps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(max(warmup, 1)):
        plan.run(ct_in, out, stream)
    torch.cuda.synchronize(dev)
    truth = nl.plain_eval(bits)
    verified = bool(np.array_equal(arx.client_decrypt(n, kr.s, out.cpu().numpy().view(np.uint32)), truth))

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(dev.index or 0)
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        plan.run(ct_in, out, stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = replica_max_ms(sum(step_ms), world, dev)
    ok = verified and np.array_equal(arx.client_decrypt(n, kr.s, out.cpu().numpy().view(np.uint32)), truth)

    rec_e2e = None
    if e2e:  # end to end through the C-ABI with pinned host buffers
        host_in = torch.from_numpy(ct_host.view(np.int32).copy()).pin_memory()
        host_out = torch.zeros((len(nl.outputs), n + 1), dtype=torch.int32).pin_memory()
        e2e_s = []
        for k in range(steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            plan.run(host_in, host_out)
            e2e_s.append(time.perf_counter() - t0)
        ok = ok and np.array_equal(arx.client_decrypt(n, kr.s, host_out.numpy().view(np.uint32)), truth)
        rec_e2e = {"value": boots / statistics.mean(e2e_s), "unit": "bootstraps/s",
                   "h2d_bytes_per_step": int(nl.num_inputs * (n + 1) * 4),
                   "d2h_bytes_per_step": int(len(nl.outputs) * (n + 1) * 4),
                   "p50_ms": 1e3 * float(np.percentile(e2e_s, 50))}

    # roofline of the dominant kernels (blind rotation), timed launch by launch
    br_ms, ks_ms, br_l, ks_l = plan.profile(ct_in)
    waves_of = {}
    for _, H, GT, jobs in plan.launches():
        if jobs:
            k = kernel_name(H, GT)
            waves_of[k] = waves_of.get(k, 0) + 1
    br_kernels = sorted(waves_of, key=lambda k: -waves_of[k])  # dominant (most waves) first
    achieved = boots * n * modmul_per_cmux(l) / (br_ms / 1e3) / 1e12
    launches_per_step = br_l + ks_l + (1 if len(nl.outputs) else 0)
    rec = {
        "value": replica_value(boots, steps, world, total_ms), "unit": "bootstraps/s", "steps": steps,
        "warmup": warmup, "ms_per_step": total_ms / steps,
        "config": {"workload": desc, "lwe_n": n, "N": 1024, "gadget": f"l={l}, Bg=2^{arx.GADGET_BITS[l]}",
                   "mode": "graph" if mode == arx.MODE_GRAPH else "plain", "shape": args.shape,
                   "gates": nl.num_gates, "bootstraps_per_step": boots, "waves": plan.waves,
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "gates_per_s": nl.num_gates * steps * world / (total_ms / 1e3),
        "verified": bool(ok),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TMODMUL, "unit": "Tmodmul/s",
                     "frac": achieved / ALU_PEAK_TMODMUL,
                     "traffic": TRAFFIC_PER_LAUNCH.get(br_kernels[0]) if br_kernels else None,
                     "kernel": br_kernels[0] if br_kernels else None,
                     "waves_per_kernel": waves_of,
                     "scope": "achieved over all blind-rotation launches of a step",
                     "kernel_ms_per_step": br_ms, "ks_ms_per_step": ks_ms},
        "gpu_launches": launches_per_step * steps,
        "clocks": clk,
    }
    if rec_e2e:
        rec["e2e"] = rec_e2e
    return rec, plan


def run_serve(args, record_only=False):
    """Served throughput: `clients` key sets, Poisson arrivals of a seeded request
    mix, continuous batching in the library's server."""
    import torch

    from paper_2306_11006_gb300 import arx

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    n = LWE_N
    keys = []
    for c in range(args.clients):
        kr = I.key_randomness(100 + c, n)
        bsk, ksk = arx.client_keygen(kr)
        keys.append((kr, arx.load_keys(bsk, ksk, n)))
    pool = serve_request_pool(args.requests, args.clients)
    inputs = []
    for r, (c, nl) in enumerate(pool):
        bits = I.random_bits(7000 + r, nl.num_inputs)
        m, e = I.encryption_randomness(8000 + r, nl.num_inputs, n)
        inputs.append((bits, arx.client_encrypt(n, keys[c][0].s, m, e, bits)))
    srv = arx.Server(hbm_budget=0, arena_bytes=4 << 30)
    # warm-up: one small request per client (also triggers shape calibration)
    warm = [srv.submit(I.comparator(4), arx.client_encrypt(n, keys[c][0].s, *I.encryption_randomness(1, 8, n),
                                                           I.random_bits(1, 8)), keyset=keys[c][1])
            for c in range(args.clients)]
    for w in warm:
        srv.wait(w)
    base = srv.stats()
    rng = np.random.default_rng(9)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, len(pool)))
    clocks = Clocks(local)
    ids = []
    t0 = time.perf_counter()
    for (c, nl), (bits, ct), at in zip(pool, inputs, arrivals):
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        ids.append(srv.submit(nl, ct, keyset=keys[c][1]))
    outs = [srv.wait(i) for i in ids]
    elapsed = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    srv.stop()
    ok = all(np.array_equal(arx.client_decrypt(n, keys[c][0].s, o), nl.plain_eval(b))
             for (c, nl), (b, _), o in zip(pool, inputs, outs))
    boots = st["bootstraps"] - base["bootstraps"]
    gates = st["gates"] - base["gates"]
    busy = st["busy_s"] - base["busy_s"]
    achieved = boots * n * MODMUL_PER_CMUX / max(busy, 1e-9) / 1e12
    for _, ks in keys:
        arx.unload_keys(ks)
    rec = {
        "value": boots / elapsed, "unit": "bootstraps/s", "steps": len(pool), "warmup": len(warm),
        "ms_per_step": 1e3 * elapsed / len(pool),
        "config": {"workload": f"serving: {args.clients} clients, Poisson {args.rate}/s, {len(pool)} requests "
                               "(adder32 | mult8 | cmp16 | random DAG 1k-50k gates)", "lwe_n": n,
                   "arrival_rate": args.rate, "clients": args.clients},
        "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"]},
        "gates_per_s": gates / elapsed, "verified": bool(ok),
        "serve": {"requests": len(pool), "bootstraps": int(boots), "gates": int(gates), "elapsed_s": elapsed,
                  "busy_s": busy, "ticks": int(st["ticks"] - base["ticks"]),
                  "launches": int(st["launches"] - base["launches"]), "peak_active": int(st["peak_active"])},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TMODMUL, "unit": "Tmodmul/s",
                     "frac": achieved / ALU_PEAK_TMODMUL, "traffic": None,
                     "kernel": "all blind rotations of the run over the server's busy time"},
        "gpu_launches": int(st["launches"] - base["launches"]),
        "clocks": clk,
    }
    if record_only:
        return rec
    line = {"metric": METRIC, "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic", **rec,
            "e2e": {"value": boots / elapsed, "unit": "bootstraps/s",
                    "h2d_bytes_per_step": int(np.mean([nl.num_inputs for _, nl in pool]) * (n + 1) * 4),
                    "d2h_bytes_per_step": int(np.mean([len(nl.outputs) for _, nl in pool]) * (n + 1) * 4)}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_request_pool(count: int, clients: int, seed: int = 5):
    """Seeded request mix: 32-bit adder, 8x8 multiplier, 16-bit comparator, random
    DAG with a log-uniform gate count in [1k, 50k]; client c = request % clients."""
    rng = np.random.default_rng(seed)
    pool = []
    for r in range(count):
        kind = int(rng.integers(0, 4))
        if kind == 0:
            nl = I.ripple_carry_adder(32)
        elif kind == 1:
            nl = I.array_multiplier(8)
        elif kind == 2:
            nl = I.comparator(16)
        else:
            g = int(np.exp(rng.uniform(np.log(1000), np.log(50000))))
            levels = 20
            wmin = max(8, g // 80)
            wmax = max(2 * wmin, g // 8)
            g = min(max(g, wmin * levels), wmax * levels)
            nl = I.random_dag(seed=1000 + r, total=g, levels=levels, num_inputs=max(64, g // 20), wmin=wmin,
                              wmax=wmax)
        pool.append((r % clients, nl))
    return pool


def run_alu(args):
    """Integer-pipe throughput of this GPU (arx_probe_alu): the measured side of the
    blind rotation's ALU roofline, next to the derived peak."""
    from paper_2306_11006_gb300 import arx
    if int(os.environ.get("RANK", "0")) != 0:
        return
    local = int(os.environ.get("LOCAL_RANK", "0"))
    clk = Clocks(local)
    rates = arx.probe_alu()
    clocks = clk.stop()
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    shoup_t = rates["shoup_bfly_q27"] * sms * mhz * 1e6 / 1e12
    print(json.dumps({
        "metric": "integer pipe throughput (lane operations per clock per SM, 32 warps per SM)",
        "value": rates["shoup_bfly_q27"], "unit": "Shoup butterflies/clk/SM", "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic", "rates_per_sm_clk": rates,
        "shoup_bfly_tmodmul_per_s": shoup_t, "derived_peak_tmodmul_per_s": ALU_PEAK_TMODMUL,
        "goldilocks_vs_crt27_butterflies": rates["goldilocks_bfly"] / (2 * rates["shoup_bfly_q27"]),
        "sms": sms, "clocks": clocks}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="arx", choices=["arx", "reference"])
    ap.add_argument("--workload", default="netlists",
                    choices=["netlists", "gates", "gates64", "dag", "matmul", "serve", "alu", "simon"])
    ap.add_argument("--clients", type=int, default=4, help="serve: clients (key sets)")
    ap.add_argument("--rate", type=float, default=16.0, help="serve: Poisson arrival rate, requests/s")
    ap.add_argument("--requests", type=int, default=32, help="serve: requests per run")
    ap.add_argument("--gates", type=int, default=64, help="gate count of the independent-gates workload")
    ap.add_argument("--blocks", type=int, default=8, help="cipher blocks of the simon workload")
    ap.add_argument("--copies", type=int, default=1, help="netlists: independent copies batched per wave")
    ap.add_argument("--shape", default=None, help="force the blind-rotation launch shape H,GT")
    ap.add_argument("--mode", default="graph", choices=["graph", "plain"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="leave out the batched and served sub-records")
    ap.add_argument("--paper-params", action="store_true",
                    help="the paper's own set: n = 512, gadget l = 2 (Bg = 2^10), instead of n = 630, l = 3")
    args = ap.parse_args()
    if args.workload == "alu":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the integer-pipe probe has no CPU counterpart"}))
            return
        return run_alu(args)
    if args.workload == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle has no server; its netlist "
                                                                  "throughput is the default workload's line"}))
            return
        return run_serve(args)
    nl, desc = workload(args.workload, args.gates, args.blocks, args.copies)
    if args.impl == "reference":
        return run_reference(args, nl, desc)

    import torch
    import torch.distributed as dist

    from paper_2306_11006_gb300 import arx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    # keys and inputs: client-side key generation and encryption from seeded randomness
    n, l = (512, 2) if args.paper_params else (LWE_N, 3)
    kr = I.key_randomness(0, n, l=l)
    bsk, ksk = arx.client_keygen(kr)
    keyset = arx.load_keys(bsk, ksk, n, l=l)
    mode = arx.MODE_GRAPH if args.mode == "graph" else arx.MODE_PLAIN
    if args.shape:
        H, GT = (int(v) for v in args.shape.split(","))
        arx.set_launch_shape(H, GT)
    rec, plan = measure_plan(arx, torch, nl, desc, args, n, l, keyset, kr, dev, stream, args.steps, args.warmup,
                             mode, world, rank)
    line = {"metric": METRIC, "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic", **rec}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle leg: timed on this host's cores, and the GPU run's wires checked bit for bit
        cb, check = oracle_leg(nl, n, l, lambda ids: plan.wires(ids, n))
        if cb:
            line["cpu_baseline"] = cb
        line["oracle_check"] = check
        line["verified"] = bool(line["verified"] and check["mismatched"] == 0)
    plan.close()
    # batched-persistent and served figures beside the plain per-level line
    extra = (rank == 0 and world == 1 and not args.no_extra and args.workload == "netlists"
             and args.copies == 1 and not args.paper_params and not args.shape)
    if extra:
        dag, ddesc = workload("dag")
        brec, bplan = measure_plan(arx, torch, dag, ddesc + " (batched: one CUDA graph, autotuned shapes)", args,
                                   n, l, keyset, kr, dev, stream, 3, 1, arx.MODE_GRAPH, e2e=False)
        # every gate of three levels of the netlist's levelization (the narrowest of
        # each third of its depth), each on the GPU run's own input wires
        wave, depth = arx.levelize(dag)
        widths = np.bincount(wave, minlength=depth)
        thirds = [range(k * depth // 3, max((k + 1) * depth // 3, k * depth // 3 + 1)) for k in range(3)]
        picked = sorted({min(t, key=lambda L: widths[L]) for t in thirds})
        gates = np.nonzero(np.isin(wave, picked))[0]
        _, bcheck = oracle_leg(dag, n, l, lambda ids: bplan.wires(ids, n), gates=gates)
        bcheck["levels"] = [int(L) for L in picked]
        brec["oracle_check"] = bcheck
        brec["verified"] = bool(brec["verified"] and bcheck["mismatched"] == 0)
        bplan.close()
        line["batched"] = brec
    arx.unload_keys(keyset)
    if extra:
        line["served"] = run_serve(args, record_only=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
