#!/usr/bin/env python
"""Benchmark of the DQAOA hot path on GB300: one step = one DQAOA cycle of the batch workload.

Workload (the DQAOA batch configuration): a dense N = 1000 QUBO with Q_ij i.i.d. uniform[-1, 1]
(symmetric, seed 2) is decomposed into m = 256 random sub-QUBOs of k = 16 variables conditioned on
the current global solution; every sub-QUBO runs depth p = 3 QAOA with the fixed parameters
gamma = (0.2, 0.4, 0.6), beta = (0.6, 0.4, 0.2) in complex64; <C> and the top-8 bitstrings of each
are reduced on the device and merged into the global solution on the host.

One step (one cycle, all steps of the hot path): index draw (host) -> sub-QUBO matrices,
energies, p layers, <C>, top-k (device) -> merge (host). `value` is sub-QUBO solves/s with Q
already resident in HBM; `e2e` is the same through dqaoa_session_cycle with Q copied from pinned
host memory every step. Between timed steps L2 is flushed by writing a 256 MiB buffer.

--impl reference times the FP64 oracle (the CPU baseline) on a bounded sample of the same cycle.
Multi-GPU (torchrun): every rank runs an independent cycle on its own GPU (sub-QUBOs are
independent units; no collective on the data path), weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CFG = dict(synth.DQAOA_BATCH)
WORKLOAD = ("DQAOA batch cycle: dense N=1000 QUBO U[-1,1], 256 random conditioned sub-QUBOs "
            "of n=16, p=3 fixed parameters, complex64, top-8 merged")
METRIC = "sub-QUBO solves/s (DQAOA cycle: decompose + energies + p layers + <C> + top-k + merge)"
UNIT = "solves/s"
# the same cycle at N = 10^4 (ten times the sub-QUBOs): where the aggregation grows with N
CFG_10K = dict(synth.DQAOA_BATCH, N=10000, m=2560)
WORKLOAD_10K = ("DQAOA batch cycle at large N: dense N=10000 QUBO U[-1,1], 2560 random conditioned "
                "sub-QUBOs of n=16, p=3 fixed parameters, complex64, top-8 merged")


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, device=None):
    """Largest value over the ranks of the default process group (the value itself with one
    rank). Timing uses it: the job takes as long as its slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base, rank):
    """Seed of a replica's workload: independent problems per rank (weak scaling)."""
    return base + 1000 * rank


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.2)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Source files that define each kernel family (the kernel itself and the headers it includes).
KERNEL_SOURCES = {
    "stream": ["k_stream.cu", "qaoa_engine.cuh", "qaoa_common.cuh", "qaoa_stream.h", "qaoa_kernels.h"],
    "tstream_pass": ["k_tstream.cu", "qaoa_tma.cuh", "qaoa_engine.cuh", "qaoa_common.cuh", "qaoa_tstream.h",
                     "qaoa_stream.h", "qaoa_kernels.h"],
    "cstream": ["k_cstream.cu", "qaoa_tma.cuh", "qaoa_engine.cuh", "qaoa_common.cuh", "qaoa_cstream.h",
                "qaoa_kernels.h"],
    "resident": ["k_resident.cu", "qaoa_engine.cuh", "qaoa_common.cuh", "qaoa_kernels.h"],
    "cluster": ["k_cluster.cu", "qaoa_engine.cuh", "qaoa_common.cuh", "qaoa_kernels.h"],
}


def kernel_source_hash(family):
    """Hash of the sources of a kernel family (stream_* and energy: the streaming files)."""
    group = "stream" if family.startswith("stream") or family == "energy" else family
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2506_10531_gb300", "csrc")
    for f in KERNEL_SOURCES.get(group, sorted(os.listdir(d))):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel_family):
    """DRAM bytes per launch of a kernel family in a workload (profiles/traffic.json, written from
    ncu captures), if it was taken on the current sources of that kernel."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except OSError:
        return None
    e = t.get("workloads", {}).get(workload, {}).get(kernel_family)
    if e is None or e.get("source_hash") != kernel_source_hash(kernel_family):
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------------------------

def oracle_cycle_sample(Q, x, n_sub, cycle):
    """The oracle on the first n_sub sub-QUBOs of one cycle: decompose, energies, state, <C>,
    top-k, merge. Returns the number of sub-QUBOs solved."""
    import oracle
    idx, qs = oracle.decompose(Q, x, CFG["m"], CFG["k"], CFG["seed"], cycle)
    idx, qs = idx[:n_sub], qs[:n_sub]
    cand = np.zeros((n_sub, CFG["topk"]), dtype=np.uint64)
    for j in range(n_sub):
        Qs = qs[j].astype(np.float32).astype(np.float64)
        E = oracle.energies(Qs)
        psi = oracle.state(CFG["k"], CFG["gamma"], CFG["beta"], E)
        oracle.expect(psi, E)
        cand[j], _ = oracle.topk(psi, CFG["topk"])
    oracle.merge(Q, x, idx, cand)
    return n_sub


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    Q = synth.symmetric_q(CFG["N"], seed=CFG["seed"])
    x = synth.bits(CFG["seed"] + 1, CFG["N"])
    n_sub = 16
    for w in range(args.warmup):
        oracle_cycle_sample(Q, x, n_sub, w)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        oracle_cycle_sample(Q, x, n_sub, 100 + s)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n_sub * args.steps / tot
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_per_step": n_sub},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_sub} of the 256 sub-QUBOs of a cycle per step "
                                       "(decompose, energies, state, <C>, top-8, merge), FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample():
    import oracle
    oracle.build()
    Q = synth.symmetric_q(CFG["N"], seed=CFG["seed"])
    x = synth.bits(CFG["seed"] + 1, CFG["N"])
    # whole cycles of 256 sub-QUBOs until at least 10 s of CPU work (at most 64 cycles)
    solved, cycles = 0, 0
    t0 = time.perf_counter()
    while cycles < 64 and (time.perf_counter() - t0) < 10.0:
        solved += oracle_cycle_sample(Q, x, CFG["m"], cycles)
        cycles += 1
    dt = time.perf_counter() - t0
    return {"value": solved / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{cycles} full cycle(s) of 256 sub-QUBOs (decompose, energies, state, <C>, "
                      f"top-8, merge) in FP64 with OpenMP, {dt:.1f} s"}


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2506_10531_gb300 as q
    from paper_2506_10531_gb300 import build as qbuild

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        qbuild.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    N, m, k, p, K = CFG["N"], CFG["m"], CFG["k"], CFG["p"], CFG["topk"]
    seed = replica_seed(CFG["seed"], rank)
    Q = synth.symmetric_q(N, seed=seed)
    Q_pin = torch.from_numpy(Q).pin_memory()
    Qh = Q_pin.numpy()
    x0 = synth.bits(seed + 1, N)
    ctx = q.qaoa_create(local)
    sess = q.dqaoa_session_create(ctx, N, m, k, p, K, q.DQAOA_RANDOM, True, CFG["gamma"], CFG["beta"])
    plans = q.dqaoa_session_plans(sess)      # the sub-QUBO chunks, solved one after the other
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def l2_flush():
        flush.fill_(1)

    # ---- value: Q resident in HBM ----
    x = x0.copy()
    q.dqaoa_session_cycle(sess, Qh, 1, x, seed, 0, stream)         # uploads Q once
    for w in range(args.warmup):
        q.dqaoa_session_cycle(sess, Qh, 0, x, seed, 1 + w, stream)
    for pl in plans:
        q.qaoa_plan_set_timing(pl, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern = {}
    energies = []
    phases = []
    spans = []
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with Clocks(local) as clk:
        for s in range(args.steps):
            l2_flush()
            ev[s][0].record(stream)
            e, acc = q.dqaoa_session_cycle(sess, Qh, 0, x, seed, 100 + s, stream)
            ev[s][1].record(stream)
            energies.append(e)
            phases.append(q.dqaoa_session_timing(sess))
            spans.append(q.dqaoa_session_solve_ms(sess))
            for pl in plans:
                for name, ms in q.qaoa_plan_kernel_times(pl):
                    kern.setdefault(name, []).append(ms)
        torch.cuda.synchronize()
    for pl in plans:
        q.qaoa_plan_set_timing(pl, False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_s = max_over_ranks(sum(step_ms) / 1e3, dev)
    value = m * args.steps * world / tot_s
    plan_kernels = sum(q.qaoa_plan_kernel_count(pl) for pl in plans)
    gpu_launches = args.steps * (plan_kernels + 1)

    # ---- dominant kernel and its roofline ----
    def relaunch():
        q.dqaoa_session_cycle(sess, Qh, 0, x, seed, 999, stream)
    roof = plan_roofline(q, plans, kern, relaunch, clk, dev, method_flops_per_step=method_flops_per_step(m, k, p),
                         steps=args.steps, workload="dqaoa", span_ms=spans if len(plans) > 1 else None)

    # ---- kernel-only batch throughput and the plain one-instance-per-launch path ----
    kb = time_plan_only(q, plans, stream, args.steps, l2_flush)
    plain = time_plain(q, ctx, sess, stream, n_inst=16)

    # ---- e2e: the public one-call cycle with Q from pinned host memory every step ----
    xe = x0.copy()
    for w in range(2):
        q.dqaoa_session_cycle(sess, Qh, 1, xe, seed, 500 + w, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(args.steps):
        q.dqaoa_session_cycle(sess, Qh, 1, xe, seed, 600 + s, stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e = {"value": m * args.steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": N * N * 8 + N + m * k * 4, "d2h_bytes_per_step": m * K * 8 + m * 8}

    q.dqaoa_session_destroy(sess)
    q.qaoa_destroy(ctx)
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    amps = m * (1 << k) * p
    ms_step = 1e3 * tot_s / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64/f32 state, f64 reductions and merge", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "sub_qubos": m, "n": k, "p": p, "topk": K,
                   "decomposition": "random, conditioned", "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": f"replicas x{world}"},
        "amp_layer_updates_per_s": amps * args.steps * world / tot_s,
        "amp_gate_updates_per_s": amps * (k + 1) * args.steps * world / tot_s,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "kernel_only": kb, "plain_gpu_path": plain,
        "batched_over_plain": kb["solves_per_s"] / plain["solves_per_s"],
        "kernel_ms_per_step": {nm: sum(v) / args.steps for nm, v in kern.items()},
        "solve_span_ms_per_step": statistics.mean(spans),
        # host clock: index draw + uploads + launches, device span, merge, whole call
        "cycle_phases_ms": {key: float(np.mean([ph[key] for ph in phases])) for key in phases[0]},
        "roofline": roof,
        "final_energy": energies[-1],
        "e2e": e2e, "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


HBM_FAMILIES = ("stream_pass", "tstream_pass", "stream_adjoint", "energy", "stream_finalize", "stream_grad_reduce")


def plan_roofline(q, plans, kern, relaunch, clk, dev, method_flops_per_step=None, steps=None, workload=None,
                  span_ms=None):
    """Roofline entry of the kernel family with the largest time in `kern` ({family: [ms per
    launch]}, measured with CUDA events on the launch stream inside the timed region).

    HBM-bound workloads (a state in HBM; method_flops_per_step None): algorithmic bytes per launch
    come from the plan(s) (states, energies and matrices read or written once per pass); `relaunch`
    runs them once more with timing on to map launch order to families.
    On-chip workloads (method_flops_per_step given: the method's arithmetic on states that fit on
    chip, SMEM / FP32 bound): achieved = the method's FP32 operations per step / the dominant
    family's event time per step, against SMs x 128 FP32 lanes x 2 x median SM clock. The same
    family's HBM view (the bytes the implementation chose to move) is reported beside it as
    `implementation_traffic`, not as the bound. span_ms (per step): the dominant family's device
    span when its launches overlap (two chunk solves on two streams); it replaces the sum of its
    launch times."""
    import torch
    if not isinstance(plans, (list, tuple)):
        plans = [plans]
    kbytes, order = [], []
    fam_ms = {nm: sum(v) for nm, v in kern.items()}
    dom = max(fam_ms, key=fam_ms.get)
    for pl in plans:
        q.qaoa_plan_set_timing(pl, True)
    relaunch()
    for pl in plans:
        kb = q.qaoa_plan_kernel_bytes(pl, 8192)
        kbytes += kb
        order += [nm for nm, _ in q.qaoa_plan_kernel_times(pl, 8192)][:len(kb)]
        q.qaoa_plan_set_timing(pl, False)
    fam_bytes = [b for nm, b in zip(order, kbytes) if nm == dom]
    per_launch_ms = statistics.mean(kern[dom])
    per_launch_bytes = statistics.mean(fam_bytes) if fam_bytes else 0.0
    if span_ms:
        # one "launch" = the overlapped launches of one step
        per_launch_ms = statistics.mean(span_ms)
        per_launch_bytes = float(sum(fam_bytes))
        fam_ms[dom] = sum(span_ms) * steps / len(span_ms)
    peaks, peak_kind = measured_peaks()
    hbm_achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    hbm = {"bound": "hbm", "kernel": dom, "achieved": hbm_achieved, "peak": peaks["hbm_gbs"],
           "unit": "GB/s", "frac": hbm_achieved / peaks["hbm_gbs"],
           "traffic": ncu_traffic(workload, dom), "peak_source": peak_kind + " (hbm_gbs, copy burst)",
           "algorithmic_bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms,
           "launches_per_step": 1 if span_ms else len(fam_bytes)}
    if method_flops_per_step is None:
        return hbm
    props = torch.cuda.get_device_properties(dev)
    mhz = clk.summary().get("sm_mhz") or 1900.0
    peak_tf = props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12
    fam_ms_step = fam_ms[dom] / steps
    achieved = method_flops_per_step / (fam_ms_step * 1e-3) / 1e12
    hbm_impl = {key: hbm[key] for key in ("achieved", "peak", "unit", "frac", "algorithmic_bytes_per_launch",
                                          "ms_per_launch", "launches_per_step", "peak_source")}
    hbm_impl["what"] = "bytes this kernel family moves through HBM per launch (the implementation's choice)"
    return {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tf,
            "unit": "TFLOP/s", "frac": achieved / peak_tf, "traffic": ncu_traffic(workload, dom),
            "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz "
                           "(median SM clock under load)",
            "method_flops_per_step": method_flops_per_step, "kernel_ms_per_step": fam_ms_step,
            "ms_per_launch": per_launch_ms, "implementation_traffic": hbm_impl}


def method_flops_per_step(m, k, p):
    """FP32 operations of the method per step: (4n + 20) per amplitude and layer (cost phase with
    its sine and cosine, n mixer rotations at 4 per amplitude, and the fused reductions), times
    m sub-QUBOs x 2^n amplitudes x p layers."""
    return m * (1 << k) * p * (4 * k + 20)


def time_plan_only(q, plans, stream, steps, l2_flush):
    """The chunk plans alone, launched as the session launches them: the first on `stream`, the
    others on a second stream that starts with it (their solves overlap on the device)."""
    import torch
    side = torch.cuda.Stream()

    def launch_all():
        start = torch.cuda.Event()
        start.record(stream)
        side.wait_event(start)
        for i, pl in enumerate(plans):
            q.qaoa_plan_launch(pl, stream if i == 0 else side)
        done = torch.cuda.Event()
        done.record(side)
        stream.wait_event(done)

    for _ in range(3):
        launch_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for s in range(steps):
        l2_flush()
        ev[s][0].record(stream)
        launch_all()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    return {"ms_per_batch": ms, "solves_per_s": CFG["m"] / (ms * 1e-3)}


def time_plain(q, ctx, sess, stream, n_inst):
    """The plain path (one instance per call, one kernel per gate) on n_inst sub-QUBOs of the
    same cycle."""
    import torch
    k, p, K = CFG["k"], CFG["p"], CFG["topk"]
    Qs = torch.as_tensor(np.stack([synth.symmetric_q(k, seed=70 + i) for i in range(n_inst)]),
                         dtype=torch.float32, device="cuda")
    g = torch.tensor(CFG["gamma"], dtype=torch.float32, device="cuda")
    b = torch.tensor(CFG["beta"], dtype=torch.float32, device="cuda")
    E = torch.empty(1 << k, dtype=torch.float32, device="cuda")
    psi = torch.empty(2 << k, dtype=torch.float32, device="cuda")
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    ti = torch.zeros(K, dtype=torch.int64, device="cuda")
    tp = torch.zeros(K, dtype=torch.float64, device="cuda")
    q.qaoa_reserve(ctx, q.qaoa_workspace_bytes(k))
    for i in range(2):
        q.qaoa_plain_solve(ctx, k, p, Qs[i], g, b, E, psi, K, ex, ti, tp, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n_inst):
        q.qaoa_plain_solve(ctx, k, p, Qs[i], g, b, E, psi, K, ex, ti, tp, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n_inst
    return {"ms_per_solve": ms, "solves_per_s": 1e3 / ms, "kernels_per_solve": 2 + p * (k + 1) + 2}


# ---------------------------------------------------------------------------------------------
# Other measured configurations (one JSON line each, same keys)
# ---------------------------------------------------------------------------------------------

LARGE = dict(seed=5, n=30, p=2, gamma=(0.4, 0.7), beta=(0.6, 0.3), k=8)
PLAIN10 = dict(seed=1, n=10, k=8)


def _timed_steps(stream, steps, body, flush=None):
    """Run body() `steps` times between CUDA events on `stream`; returns ms per step list."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s in range(steps):
        if flush is not None:
            flush()
        ev[s][0].record(stream)
        body(s)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _line(metric, value, unit, args, world, ms_step, dtype, config, **extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}
    d.update(extra)
    return d


def _plan_kern_times(q, plan, kern):
    for name, ms in q.qaoa_plan_kernel_times(plan, 8192):
        kern.setdefault(name, []).append(ms)


def run_large(args):
    """The n = 30, p = 2 streaming solve: energies, two layers, <C> and top-8 (one plan)."""
    import torch
    import paper_2506_10531_gb300 as q
    from paper_2506_10531_gb300 import build as qbuild
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n, p, k = args.large_n, LARGE["p"], LARGE["k"]
    Q = synth.symmetric_q(n, seed=LARGE["seed"] + 1000 * rank).astype(np.float32)
    par = np.array(LARGE["gamma"] + LARGE["beta"], dtype=np.float32)
    ctx = q.qaoa_create(local)
    qd = torch.as_tensor(Q.reshape(-1)).to(dev)
    pd = torch.as_tensor(par).to(dev)
    ex = torch.zeros(1, dtype=torch.float64, device=dev)
    ti = torch.zeros(k, dtype=torch.int64, device=dev)
    tp = torch.zeros(k, dtype=torch.float64, device=dev)
    grad = torch.zeros(2 * p, dtype=torch.float64, device=dev) if args.large_grad else None
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=k, grad=grad)
    insts = q.make_insts([(n, p, k, q.QAOA_INST_GRAD if args.large_grad else 0, 0, 0, -1, -1)])
    plan = q.qaoa_plan_create(ctx, insts, io)
    for _ in range(args.warmup):
        q.qaoa_plan_launch(plan, stream)
    torch.cuda.synchronize()
    kern = {}
    q.qaoa_plan_set_timing(plan, True)

    def body(s):
        q.qaoa_plan_launch(plan, stream)
        _plan_kern_times(q, plan, kern)
    with Clocks(local) as clk:
        step_ms = _timed_steps(stream, args.steps, body)
    q.qaoa_plan_set_timing(plan, False)
    tot_s = max_over_ranks(sum(step_ms) / 1e3, dev)
    amps = (1 << n) * p * world
    roof = plan_roofline(q, plan, kern, lambda: q.qaoa_plan_launch(plan, stream), clk, dev,
                         workload=f"large_n{n}")
    per_pass = {"ms": [round(v, 3) for v in (kern.get("tstream_pass") or kern.get("stream_pass") or [])[:8]]}
    # e2e: Q and parameters from pinned host memory, <C> and top-k back, every step
    Qp = torch.from_numpy(Q.reshape(-1)).pin_memory()
    Pp = torch.from_numpy(par).pin_memory()
    out = torch.empty(1 + 2 * k, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(args.steps):
        qd.copy_(Qp, non_blocking=True)
        pd.copy_(Pp, non_blocking=True)
        q.qaoa_plan_launch(plan, stream)
        out[0:1].copy_(ex, non_blocking=True)
        out[1:1 + k].copy_(tp, non_blocking=True)
        out[1 + k:].copy_(ti.view(torch.float64), non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    kernels = q.qaoa_plan_kernel_count(plan)
    q.qaoa_plan_destroy(plan)
    q.qaoa_destroy(ctx)
    line = _line(f"amp-layer-updates/s (n={n} streaming solve: energies + 2 layers + <C> + top-8)",
                 amps * args.steps / tot_s, "amp-layer-updates/s", args, world, 1e3 * tot_s / args.steps,
                 "c64 state, f32 energies, f64 reductions",
                 {"workload": f"large instance: dense n={n} QUBO U[-1,1] (seed 5), p=2, gamma=(0.4,0.7), "
                              f"beta=(0.6,0.3), complex64 ({(8 << n) / 2**30:g} GiB) + FP32 energies, top-8"
                              + (", with adjoint gradients (profiling case)" if args.large_grad else ""),
                  "l2": "inputs larger than L2 (state + energies)", "parallelism": f"replicas x{world}"},
                 solves_per_s=args.steps * world / tot_s,
                 amp_gate_updates_per_s=amps * (n + 1) * args.steps / tot_s,
                 latency_ms={"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
                 kernel_ms_per_step={nm: sum(v) / args.steps for nm, v in kern.items()},
                 pass_ms_first_step=per_pass, roofline=roof,
                 e2e={"value": amps * args.steps / e2e_s, "unit": "amp-layer-updates/s",
                      "h2d_bytes_per_step": Q.nbytes + par.nbytes, "d2h_bytes_per_step": 8 * (1 + 2 * k)},
                 gpu_launches=kernels * args.steps, clocks=clk.summary())
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = large_cpu_baseline()
    return line


def large_cpu_baseline():
    """The oracle on the n = 24 twin of the large instance (same generator and parameters)."""
    import oracle
    oracle.build()
    n, p = 24, LARGE["p"]
    Q = synth.symmetric_q(n, seed=LARGE["seed"]).astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    E = oracle.energies(Q)
    psi = oracle.state(n, LARGE["gamma"], LARGE["beta"], E)
    oracle.expect(psi, E)
    oracle.topk(psi, LARGE["k"])
    dt = time.perf_counter() - t0
    return {"value": (1 << n) * p / dt, "unit": "amp-layer-updates/s", "cores": os.cpu_count(),
            "kind": "oracle", "sample": f"one n=24 twin solve (energies, 2 layers, <C>, top-8) in FP64, {dt:.1f} s"}


def run_plain10(args):
    """The plain n = 10 grid: 256 (gamma, beta) points at p = 1 in complex128, one batch."""
    import torch
    import paper_2506_10531_gb300 as q
    from paper_2506_10531_gb300 import build as qbuild
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n, k = PLAIN10["n"], PLAIN10["k"]
    Q = synth.symmetric_q(n, seed=PLAIN10["seed"] + 1000 * rank)
    gg, bb = synth.grid_params(16)
    count = gg.size
    par = np.stack([gg, bb], axis=1).reshape(-1)
    ctx = q.qaoa_create(local)
    qd = torch.as_tensor(Q.reshape(-1)).to(dev)
    pd = torch.as_tensor(par).to(dev)
    ex = torch.zeros(count, dtype=torch.float64, device=dev)
    ti = torch.zeros(count * k, dtype=torch.int64, device=dev)
    tp = torch.zeros(count * k, dtype=torch.float64, device=dev)
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=k)
    insts = q.make_insts([(n, 1, k, 0, 0, 2 * i, -1, -1) for i in range(count)])
    plan = q.qaoa_plan_create(ctx, insts, io, dbl=True)
    for _ in range(args.warmup):
        q.qaoa_plan_launch(plan, stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    kern = {}
    q.qaoa_plan_set_timing(plan, True)

    def body(s):
        q.qaoa_plan_launch(plan, stream)
        _plan_kern_times(q, plan, kern)
    with Clocks(local) as clk:
        step_ms = _timed_steps(stream, args.steps, body, flush=lambda: flush.fill_(1))
    q.qaoa_plan_set_timing(plan, False)
    tot_s = max_over_ranks(sum(step_ms) / 1e3, dev)
    # on-chip FP64 work: phase (sincos ~ 20 flops) + 4 flops + 4 flops per qubit per amplitude
    flops = count * (1 << n) * (24 + 4 * n)
    props = torch.cuda.get_device_properties(dev)
    ms_launch = statistics.mean(kern["resident"])
    mhz = clk.summary().get("sm_mhz") or 1900.0
    fp64_peak = props.multi_processor_count * 2 * 2 * mhz * 1e6 / 1e12   # 2 FP64 FMA lanes per SM
    roof = {"bound": "alu", "kernel": "resident", "achieved": flops / (ms_launch * 1e-3) / 1e12,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": flops / (ms_launch * 1e-3) / 1e12 / fp64_peak,
            "traffic": ncu_traffic("plain10", "resident"), "ms_per_launch": ms_launch,
            "peak_source": "derived: SMs x 2 FP64 FMA lanes x 2 x median SM clock (FP64 at 1/64 of FP32)"}
    Pp = torch.from_numpy(par).pin_memory()
    Qp = torch.from_numpy(Q.reshape(-1)).pin_memory()
    oex = torch.empty(count, dtype=torch.float64).pin_memory()
    oti = torch.empty(count * k, dtype=torch.int64).pin_memory()
    otp = torch.empty(count * k, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(args.steps):
        qd.copy_(Qp, non_blocking=True)
        pd.copy_(Pp, non_blocking=True)
        q.qaoa_plan_launch(plan, stream)
        oex.copy_(ex, non_blocking=True)
        oti.copy_(ti, non_blocking=True)
        otp.copy_(tp, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    kernels = q.qaoa_plan_kernel_count(plan)
    q.qaoa_plan_destroy(plan)
    q.qaoa_destroy(ctx)
    line = _line("grid points solved/s (n=10, p=1, complex128: energies + layer + <C> + top-8)",
                 count * args.steps * world / tot_s, "solves/s", args, world, 1e3 * tot_s / args.steps,
                 "c128 state, f64 energies and reductions",
                 {"workload": "plain n=10 QUBO U[-1,1] (seed 1), p=1, 16x16 (gamma, beta) grid over "
                              "[0,pi]x[0,pi/2] as 256 resident instances sharing Q, complex128, top-8",
                  "l2": "flushed (256 MiB write) between timed steps", "parallelism": f"replicas x{world}"},
                 amp_layer_updates_per_s=count * (1 << n) * args.steps * world / tot_s,
                 latency_ms={"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
                 kernel_ms_per_step={nm: sum(v) / args.steps for nm, v in kern.items()},
                 roofline=roof,
                 e2e={"value": count * args.steps * world / e2e_s, "unit": "solves/s",
                      "h2d_bytes_per_step": Q.nbytes + par.nbytes, "d2h_bytes_per_step": count * (8 + 16 * k)},
                 gpu_launches=kernels * args.steps, clocks=clk.summary())
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        E = oracle.energies(Q)
        for i in range(count):
            psi = oracle.state(n, [gg[i]], [bb[i]], E)
            oracle.expect(psi, E)
            oracle.topk(psi, k)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": count / dt, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"all 256 grid points in FP64, {dt:.2f} s"}
    return line


def run_uneven(args):
    """The uneven training batch: 4096 instances (n 8..24, p 1..6, normal Q); one step = <C> and
    adjoint gradients of every instance plus one Adam update, all on the device."""
    import torch
    import paper_2506_10531_gb300 as q
    from paper_2506_10531_gb300 import build as qbuild
    from paper_2506_10531_gb300.train import QAOABatch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    U = dict(synth.UNEVEN_BATCH)
    U["count"] = args.uneven_count or U["count"]
    inst = synth.uneven_batch(U["count"], U["seed"] + 1000 * rank, *U["n"], *U["p"], dist=U["dist"])
    ns = np.array([x[0].shape[0] for x in inst])
    ps = np.array([len(x[1]) for x in inst])
    ctx = q.qaoa_create(local)
    B = QAOABatch(ctx, [x[0] for x in inst], [(x[1], x[2]) for x in inst], device=dev)
    # a side stream: the plan is captured into a CUDA graph there (capture needs a non-legacy stream)
    gs = torch.cuda.Stream(dev)
    stream = gs
    for _ in range(args.warmup):
        B.run(stream)
        B.adam_step(U["lr"], stream)
    torch.cuda.synchronize()
    # (1) per-kernel event timing of uncaptured steps: the roofline's kernel durations
    kern = {}
    q.qaoa_plan_set_timing(B.plan, True)

    def body_timed(s):
        B.run(stream)
        _plan_kern_times(q, B.plan, kern)
        B.adam_step(U["lr"], stream)
    with Clocks(local) as clk_k:
        kstep_ms = _timed_steps(stream, args.steps, body_timed)
    roof = plan_roofline(q, B.plan, kern, lambda: B.run(stream), clk_k, dev, workload=f"uneven_{U['count']}")
    q.qaoa_plan_set_timing(B.plan, False)
    # (2) the timed steps: one graph replay of the whole batch plus the Adam kernel per step
    B.capture(stream)
    B.run(stream)
    B.adam_step(U["lr"], stream)
    torch.cuda.synchronize()

    def body(s):
        B.run(stream)
        B.adam_step(U["lr"], stream)
    with Clocks(local) as clk:
        step_ms = _timed_steps(stream, args.steps, body)
    tot_s = max_over_ranks(sum(step_ms) / 1e3, dev)
    amps = float(np.sum((2.0 ** ns) * ps))
    # e2e: Q pool and parameters from pinned host memory, <C> of every instance back, per step
    qh = B.q.cpu().pin_memory()
    ph = B.params.cpu().pin_memory()
    eh = torch.empty(B.count, dtype=torch.float64).pin_memory()
    e2e_steps = max(2, args.steps // 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):      # the copies are ordered with the graph on the same stream
        for s in range(e2e_steps):
            B.q.copy_(qh, non_blocking=True)
            B.params.copy_(ph, non_blocking=True)
            B.run(stream)
            B.adam_step(U["lr"], stream)
            eh.copy_(B.expect, non_blocking=True)
            torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    kernels = B.kernels_per_launch + 1
    B.close()
    q.qaoa_destroy(ctx)
    line = _line("instance optimisation steps/s (uneven batch: <C> + adjoint gradient + Adam, all instances)",
                 B.count * args.steps * world / tot_s, "instance-steps/s", args, world, 1e3 * tot_s / args.steps,
                 "c64 state, f32 energies, f64 reductions and gradients",
                 {"workload": f"uneven batch: {U['count']} sub-QUBOs, n uniform 8..24, p uniform 1..6, Q N(0,1) "
                              "symmetric (seed 3), complex64, adjoint gradients, Adam lr 0.05",
                  "l2": "inputs larger than L2 (about 160 GB of states and energies)",
                  "parallelism": f"replicas x{world}"},
                 amp_layer_updates_per_s=amps * args.steps * world / tot_s,
                 latency_ms={"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
                 kernel_ms_per_step={nm: sum(v) / args.steps for nm, v in kern.items()},
                 roofline=roof,
                 e2e={"value": B.count * e2e_steps * world / e2e_s, "unit": "instance-steps/s",
                      "h2d_bytes_per_step": int(qh.numel() * 4 + ph.numel() * 4),
                      "d2h_bytes_per_step": B.count * 8},
                 gpu_launches=kernels * args.steps,
                 launch_calls_per_step={"graph": 1, "kernel": 1, "kernels_in_graph": kernels - 1},
                 uncaptured_ms_per_step=float(np.mean(kstep_ms)), clocks=clk.summary())
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        done, sampled = 0, 0.0
        for Qi, g, b in inst:
            if time.perf_counter() - t0 > 10.0:
                break
            if Qi.shape[0] > 20:
                continue
            E = oracle.energies(Qi.astype(np.float32).astype(np.float64))
            oracle.grad(Qi.shape[0], g, b, E)
            done += 1
            sampled += (2.0 ** Qi.shape[0]) * len(g)
        dt = time.perf_counter() - t0
        # the oracle's amp-layer rate on the sample, converted to whole-batch instance steps
        rate = sampled / dt
        line["cpu_baseline"] = {"value": B.count * rate / amps, "unit": "instance-steps/s",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{done} instances of the batch with n <= 20 (energies + adjoint "
                                          f"gradient, FP64) in {dt:.1f} s: {rate:.3g} amp-layers/s, scaled "
                                          f"to the batch's {amps:.3g} amp-layers per step"}
    return line


SERVING = dict(seed=4, n=(12, 26), p=(1, 8), steps=50, k=16, lr=0.05,
               rates=(10.0, 20.0, 100.0, 1000.0, 5000.0))


def serving_requests(rate, count, seed):
    """The same job mix (seed) at every rate; only the arrival times depend on the rate."""
    from paper_2506_10531_gb300.serve import Request
    ns, ps = synth.uneven_mix(count, seed, *SERVING["n"], *SERVING["p"])
    arr = synth.poisson_arrivals(rate, count, seed + 7 + int(rate))
    arr = arr - arr[0]
    seeds = synth.splitmix64(seed ^ 0x3C3C3C3C, count)
    out = []
    for i in range(count):
        n, p = int(ns[i]), int(ps[i])
        g, b = synth.random_params(p, int(seeds[i]) ^ 0x77)
        out.append(Request(n=n, p=p, Q=synth.symmetric_q(n, int(seeds[i])).astype(np.float32),
                           params=np.concatenate([g, b]).astype(np.float32), steps=SERVING["steps"],
                           lr=SERVING["lr"], arrival=float(arr[i])))
    return out


def run_serving(args):
    """Poisson streams of optimise-and-sample jobs (n 12..26, p 1..8, 50 adjoint-Adam steps, then
    top-16) through the continuous-batching server; latency percentiles and throughput per rate."""
    import torch
    import paper_2506_10531_gb300 as q
    from paper_2506_10531_gb300 import build as qbuild
    from paper_2506_10531_gb300.serve import serve_stream
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = q.qaoa_create(local)
    free, _ = torch.cuda.mem_get_info(dev)
    scratch = int(free * 0.8)
    count = args.requests
    # warm-up: a short stream at a low rate
    serve_stream(ctx, serving_requests(50.0, 8, 999), scratch, 4096, SERVING["k"], stream)
    rows = []
    with Clocks(local) as clk:
        for rate in SERVING["rates"]:
            reqs = serving_requests(rate, count, SERVING["seed"] + 1000 * rank)
            rep = serve_stream(ctx, reqs, scratch, 4096, SERVING["k"], stream)
            rows.append({"rate_req_s": rate, "requests": count, "solves_per_s": rep.solves_per_s,
                         "p50_s": float(np.percentile(rep.latency_s, 50)),
                         "p99_s": float(np.percentile(rep.latency_s, 99)),
                         "max_active": rep.max_active, "ticks": rep.ticks,
                         "elapsed_s": rep.elapsed_s, "bytes": rep.bytes_total, "gpu_ms": rep.gpu_ms,
                         "launches": rep.launches,
                         "h2d_bytes_per_job": float(np.mean([(r.n * r.n + 2 * r.p) * 4 for r in reqs])),
                         "d2h_bytes_per_job": 8 + 16 * 16 + 128 * 4})
    q.qaoa_destroy(ctx)
    sat = max(rows, key=lambda r: r["solves_per_s"])
    peaks, peak_kind = measured_peaks()
    achieved = sat["bytes"] / (sat["gpu_ms"] * 1e-3) / 1e9 if sat["gpu_ms"] > 0 else 0.0
    roof = {"bound": "hbm", "kernel": "all kernels of a tick (whole serving step)", "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
            "peak_source": peak_kind + " (hbm_gbs, copy burst)",
            "note": "algorithmic bytes of every tick at the saturating rate over the ticks' device time"}
    # replicas: the whole job serves world streams, at the pace of the slowest replica
    job_rate = -max_over_ranks(-sat["solves_per_s"], dev) * world
    line = _line("optimise-and-sample jobs/s at saturation (serving: Poisson arrivals, continuous batching)",
                 job_rate, "jobs/s", args, world, 1e3 / sat["solves_per_s"] if sat["solves_per_s"] else None,
                 "c64 state, f32 energies, f64 reductions and gradients",
                 {"workload": f"serving: Poisson arrivals at {list(SERVING['rates'])} req/s, {count} requests per "
                              "rate, n uniform 12..26, p uniform 1..8, Q U[-1,1], 50 adjoint-Adam steps then "
                              "top-16, admitted by HBM footprint",
                  "scratch_bytes": scratch, "max_jobs": 4096, "l2": "inputs larger than L2",
                  "parallelism": f"replicas x{world}"},
                 latency_s={"p50": sat["p50_s"], "p99": sat["p99_s"]}, rates=rows, roofline=roof,
                 e2e={"value": job_rate, "unit": "jobs/s",
                      "h2d_bytes_per_step": sat["h2d_bytes_per_job"], "d2h_bytes_per_step": sat["d2h_bytes_per_job"],
                      "note": "the serving loop is end to end (host Q and parameters in, results out); "
                              "bytes per job"},
                 gpu_launches=sat["launches"], clocks=clk.summary())
    line["steps"] = count
    return line


MAXCUT = dict(seed=6, N=1000, m=500, k=12, p=3, topk=8, gamma=(0.2, 0.4, 0.6), beta=(0.6, 0.4, 0.2),
              max_cycles=60, patience=5)
MAXCUT_METHODS = ("random", "ifd", "bfs", "pfs")


def maxcut_cpu_baseline():
    """The oracle on whole PFS cycles of the Max-Cut workload until at least 10 s of CPU work."""
    import oracle
    oracle.build()
    c = MAXCUT
    Q = synth.maxcut_graph_q(c["N"], seed=c["seed"])
    x = synth.bits(c["seed"] + 1, c["N"])
    solved, cycles = 0, 0
    t0 = time.perf_counter()
    while cycles < 16 and (time.perf_counter() - t0) < 10.0:
        idx, qs = oracle.decompose(Q, x, c["m"], c["k"], c["seed"], cycles, method=oracle.PFS)
        cand = np.zeros((c["m"], c["topk"]), dtype=np.uint64)
        for j in range(c["m"]):
            Qs = qs[j].astype(np.float32).astype(np.float64)
            E = oracle.energies(Qs)
            psi = oracle.state(c["k"], c["gamma"], c["beta"], E)
            oracle.expect(psi, E)
            cand[j], _ = oracle.topk(psi, c["topk"])
        x, _, _ = oracle.merge(Q, x, idx, cand)
        solved += c["m"]
        cycles += 1
    dt = time.perf_counter() - t0
    return {"value": solved / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{cycles} full PFS cycle(s) of {c['m']} sub-QUBOs of n={c['k']} (decompose, "
                      f"energies, state, <C>, top-8, merge) in FP64, {dt:.1f} s"}


def run_maxcut(args):
    """DQAOA cycles on the synthetic Max-Cut workload with each decomposition method (random,
    IFD, BFS, PFS; Section V-A and the Max-Cut study of Section VI): throughput per cycle with
    CUDA events, and per method the cut reached and the cycles until the stopping rule holds."""
    import torch
    import paper_2506_10531_gb300 as q
    from paper_2506_10531_gb300 import build as qbuild
    from paper_2506_10531_gb300 import dqaoa
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    qbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    c = MAXCUT
    N, m, k, p, K = c["N"], c["m"], c["k"], c["p"], c["topk"]
    seed = replica_seed(c["seed"], rank)
    Q = synth.maxcut_graph_q(N, seed=seed)
    Qh = torch.from_numpy(Q).pin_memory().numpy()
    x0 = synth.bits(seed + 1, N)
    ctx = q.qaoa_create(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    codes = {"random": q.DQAOA_RANDOM, "ifd": q.DQAOA_IFD, "bfs": q.DQAOA_BFS, "pfs": q.DQAOA_PFS}
    per, kern, all_ms, launches = {}, {}, [], 0
    e2e_s, e2e_cycles = 0.0, 0
    roof_args = None
    with Clocks(local) as clk:
        for name in MAXCUT_METHODS:
            sess = q.dqaoa_session_create(ctx, N, m, k, p, K, codes[name], True, c["gamma"], c["beta"])
            plans = q.dqaoa_session_plans(sess)
            x = x0.copy()
            q.dqaoa_session_cycle(sess, Qh, 1, x, seed, 0, stream)
            for w in range(args.warmup):
                q.dqaoa_session_cycle(sess, Qh, 0, x, seed, 1 + w, stream)
            for pl in plans:
                q.qaoa_plan_set_timing(pl, True)
            mk = {}

            def body(s):
                q.dqaoa_session_cycle(sess, Qh, 0, x, seed, 100 + s, stream)
                for pl in plans:
                    _plan_kern_times(q, pl, mk)
            step_ms = _timed_steps(stream, args.steps, body, flush=lambda: flush.fill_(1))
            for pl in plans:
                q.qaoa_plan_set_timing(pl, False)
            for nm, v in mk.items():
                kern.setdefault(nm, []).extend(v)
            launches += args.steps * (sum(q.qaoa_plan_kernel_count(pl) for pl in plans) + 1)
            # e2e: Q from pinned host memory every cycle (the session rebuilds what depends on Q)
            xe = x0.copy()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in range(args.steps):
                q.dqaoa_session_cycle(sess, Qh, 1, xe, seed, 600 + s, stream)
            torch.cuda.synchronize()
            e2e_s += time.perf_counter() - t0
            e2e_cycles += args.steps
            if name == "pfs":
                roof_args = (sess, plans, mk, x)      # roofline after the clock sampler stops
            else:
                q.dqaoa_session_destroy(sess)
            # solution quality: cycles from x0 until the energy stops decreasing (patience cycles)
            r = dqaoa.solve(ctx, Q, m, k, p, K, c["gamma"], c["beta"], x0, seed=seed, method=codes[name],
                            max_cycles=c["max_cycles"], patience=c["patience"], stream=stream)
            per[name] = {"ms_per_cycle": float(np.mean(step_ms)),
                         "solves_per_s": m * args.steps / (sum(step_ms) / 1e3),
                         "cut_x0": synth.cut_value(Q, x0), "cut": synth.cut_value(Q, r.x),
                         "cycles": r.cycles, "converged": r.converged, "tts_s": r.tts_s, "wall_s": r.wall_s,
                         "host_phases_ms": {key: float(np.mean([t[key] for t in r.timing])) for key in r.timing[0]}}
            all_ms += step_ms
    sess, plans, mk, x = roof_args
    roof = plan_roofline(q, plans, mk, lambda: q.dqaoa_session_cycle(sess, Qh, 0, x, seed, 999, stream),
                         clk, dev, method_flops_per_step=method_flops_per_step(m, k, p), steps=args.steps,
                         workload="maxcut")
    q.dqaoa_session_destroy(sess)
    q.qaoa_destroy(ctx)
    tot_s = max_over_ranks(sum(all_ms) / 1e3, dev)
    cycles = len(MAXCUT_METHODS) * args.steps
    line = _line(f"sub-QUBO solves/s (DQAOA cycles on synthetic Max-Cut, random / IFD / BFS / PFS decompositions)",
                 m * cycles * world / tot_s, UNIT, args, world, 1e3 * tot_s / cycles, "c64/f32 state, f64 reductions and merge",
                 {"workload": f"DQAOA on synthetic Max-Cut: unweighted graph of N={N} vertices with N(N-1)/8 edges "
                              f"(seed {c['seed']}), m={m} conditioned sub-QUBOs of n={k}, p={p} fixed parameters, "
                              f"complex64, top-{K} merged; {args.steps} timed cycles per decomposition method",
                  "N": N, "sub_qubos": m, "n": k, "p": p, "topk": K, "methods": list(MAXCUT_METHODS),
                  "l2": "flushed (256 MiB write) between timed steps", "parallelism": f"replicas x{world}"},
                 latency_ms={"p50": float(np.percentile(all_ms, 50)), "p99": float(np.percentile(all_ms, 99))},
                 per_method=per,
                 kernel_ms_per_step={nm: sum(v) / cycles for nm, v in kern.items()},
                 roofline=roof,
                 e2e={"value": m * e2e_cycles * world / max_over_ranks(e2e_s, dev), "unit": UNIT,
                      "h2d_bytes_per_step": N * N * 8 + N + m * k * 4, "d2h_bytes_per_step": m * K * 8 + m * 8},
                 gpu_launches=launches, clocks=clk.summary())
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = maxcut_cpu_baseline()
    return line


CONFIGS = {"large": run_large, "maxcut": run_maxcut, "plain10": run_plain10, "uneven": run_uneven, "serving": run_serving}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 500 DQAOA cycles, about 0.25 s, for the dqaoa "
                         "configuration; 20 for the others)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=100, help="requests per rate (serving config)")
    ap.add_argument("--large-n", type=int, default=LARGE["n"],
                    help="qubits of the large configuration (smaller values: profiling cases)")
    ap.add_argument("--large-grad", action="store_true",
                    help="large configuration with adjoint gradients (a profiling case of the adjoint passes)")
    ap.add_argument("--uneven-count", type=int, default=0,
                    help="instances of the uneven batch (0: the full 4096; smaller: profiling cases)")
    ap.add_argument("--config", default="dqaoa", choices=["dqaoa", "dqaoa10k"] + sorted(CONFIGS),
                    help="dqaoa: the DQAOA batch cycle (headline); the others are the further "
                         "measured configurations")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 500 if args.config == "dqaoa" and args.impl == "ours" else 20
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "dqaoa":
        run_ours(args)
    elif args.config == "dqaoa10k":
        global CFG, WORKLOAD
        CFG, WORKLOAD = dict(CFG_10K), WORKLOAD_10K
        args.no_cpu_baseline = True   # the oracle baseline is quoted on the N = 1000 cycle
        run_ours(args)
    else:
        import torch
        import torch.distributed as dist
        rank, world, local = dist_env()
        if world > 1:
            torch.cuda.set_device(local)
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
            dist.barrier()
        line = CONFIGS[args.config](args)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
