#!/usr/bin/env python
"""Benchmark: energy + full gradient evaluations per second on GB300.

Workload (default): the transverse-field Ising chain n=20, J=1, h_i ~ U[0.5,1.5], with the
L=6 RY/RZ + CZ brick-wall ansatz and a batch of B=64 parameter sets; one step = one
call of the whole hot path (gate tables, the batched causal-cone kernel with its adjoint,
and the FP64 term/gradient reductions) for all 64 sets. Synthetic, seeded inputs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tlq|reference]

``--impl reference`` times the CPU oracle (complex128 statevector with its own adjoint)
on the host cores over a bounded sample of the same workload. Under torchrun each rank
runs an independent replica (no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "expectation+gradient evals/sec"
UNIT = "grad-evals/s"
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant kernel,
# taken from one ncu capture of that kernel on that workload (summaries in profiles/). Workloads
# without an entry report null; an entry is removed when its kernel changes after the capture.
NCU_TRAFFIC = {
    ("tfim_n20_L6_B64", "cone_kernel"): 856576.0 + 0.0,
    ("tfim_n500_L4_B256", "cone_kernel"): 10280960.0 + 18432.0,
    ("tfim_n400_L8_B1", "cone_kernel"): 12117756928.0 + 14537556224.0,
    ("partial_trace_n20_m13", "herk_ws_kernel"): 8826624.0 + 475120128.0,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tlq", choices=["tlq", "reference"])
    ap.add_argument("--workload", default="tfim_n20_L6_B64",
                    help="tfim_n20_L6_B64 (default), tfim_n500_L4_B256, tfim_n8_L2_B1, tfim_n<N>_L<L>_B<B> (any "
                         "Ising chain, h ~ U[0.5, 1.5], seed 5) or qaoa_n<N>_p<P> (3-regular graph, dense "
                         "statevector path, one parameter set)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "mixed_tc"],
                    help="precision of the timed workload (mixed_tc: tensor-core gate blocks on the dense path)")
    ap.add_argument("--energy-only", action="store_true",
                    help="time energy-only calls (expectation evals/s) instead of energy + gradient; no CPU baseline "
                         "or plain path")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the chosen workload only: no other workloads, serving replay or CPU baseline "
                         "(short runs for a profiler)")
    return ap.parse_args()


def workload(name):
    from paper_2112_10239_gb300 import workloads as W
    if name == "tfim_n20_L6_B64":
        return W.tfim_n20_L6_B64()
    if name == "tfim_n500_L4_B256":
        return W.tfim_n500_L4_B256()
    if name == "tfim_n8_L2_B1":
        return W.tfim_n8_L2()
    m = re.fullmatch(r"tfim_n(\d+)_L(\d+)_B(\d+)", name)
    if m:   # any chain: h_i ~ U[0.5, 1.5], brick-wall ansatz, seed 5
        n, L, Bs = int(m.group(1)), int(m.group(2)), int(m.group(3))
        if not (2 <= n and 1 <= L and 1 <= Bs):
            raise SystemExit("tfim workloads take n >= 2, L >= 1, B >= 1")
        return W.tfim_problem(n, L, Bs, seed=5, h_range=(0.5, 1.5), name=name)
    m = re.fullmatch(r"qaoa_n(\d+)_p(\d+)", name)
    if m:
        n, p = int(m.group(1)), int(m.group(2))
        if not 13 <= n <= 31 or p < 1:
            raise SystemExit("qaoa workloads take 13 <= n <= 31 and p >= 1")
        return W.qaoa_problem(n, p, 1, seed=2, name=name)
    raise SystemExit(f"unknown workload {name}")


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_throughput(local_s, units, world, device=None):
    """Whole-job throughput of `world` replicas that each processed `units` in `local_s` seconds:
    all units over the slowest rank's time (a MAX all-reduce of the times when world > 1).
    Returns (value, max_seconds)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(local_s)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_s = float(t.item())
    return world * units / local_s, local_s


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def algorithmic_flops(B_mod, ctx, c, h, prob, grad=True):
    """Algorithmic FP32 flops of one batched cone launch (forward, measurement, adjoint).

    Per work cone of true width w (A = 2^w amplitudes), with R rotations, D diagonal layers,
    Pd parametrised diagonal gates and m terms measured on its window:
      forward   A * (6 R + 6 D)       real 2x2 rotation on (re, im): 6 flop/amp; one complex
                                      multiply per amplitude per diagonal layer
      measure   A * 8 m               <psi|P_t|psi> and lambda += c_t P_t psi per term
      adjoint   A * (4 R + 12 R + 12 D + 3 D + Pd)
                                      Im<lam|G|psi> (4/amp), un-apply on psi and lam (2 x 6),
                                      diagonal un-apply (2 x 6), Im(conj(lam) psi) (3) and one
                                      signed add per parametrised diagonal gate
    Padding to the kernel's minimum width is not counted.
    """
    n_terms = len(prob.terms)
    nrot, ndiag, npdiag, _, w, nterms, _ = B_mod.tlq_plan_cone_stats(ctx.h, c.h, h.h, n_terms)
    A = np.power(2.0, w.astype(np.float64))
    f = A * (6 * nrot + 6 * ndiag + 8 * nterms)
    if grad:
        f += A * (16 * nrot + 15 * ndiag + npdiag)
    return float(np.sum(f)) * prob.B


def unfused_flops(prob, grad=True):
    """The scope table's algorithmic count for a layered brick-wall Ising workload: every term
    contracted over its own exact causal cone (no window sharing). For a term with support
    [a, b] the live rotations of layer l (1..L) span [a - (L - l), b + (L - l)] clipped to the
    chain (ZZ: width 2 + 2(L - l); X: 3 + 2(L - l), counting the two CZ neighbours of the last
    layer); the window is the layer-1 span. Forward flops 2^W (6 sum_l live_l + 6 D + 8), with
    D = L diagonal layers for X terms and L - 1 for Z-only terms (the last layer's diagonal
    commutes with them); the adjoint is counted as three times the forward. Per batch."""
    n, L = prob.n, prob.meta.get("L")
    if L is None or prob.meta.get("layout") != "brickwall":
        return None, None
    fwd = 0.0
    for _, sites, letters in prob.terms:
        a, b = min(sites), max(sites)
        zonly = set(letters) <= {"Z"}
        if not zonly:           # X/Y: the CZs of the last layer reach one site further
            a, b = a - 1, b + 1
        live = [min(n - 1, b + (L - l)) - max(0, a - (L - l)) + 1 for l in range(1, L + 1)]
        W = live[0]
        D = L - 1 if zonly else L
        fwd += 2.0 ** W * (6 * sum(live) + 6 * D + 8)
    fwd *= prob.B
    return fwd, (4 * fwd if grad else fwd)


def fp64_errors(E, G, E_ref, G_ref):
    """Max relative energy error |E - E_ref| / max(|E_ref|, 1) and gradient error
    ||G - G_ref||_inf / max(1, ||G_ref||_inf) of a timed result against its FP64 reference."""
    E, E_ref = np.asarray(E, dtype=np.float64), np.asarray(E_ref, dtype=np.float64)
    out = {"energy_max_rel": float(np.max(np.abs(E - E_ref) / np.maximum(np.abs(E_ref), 1.0)))}
    if G is not None and G_ref is not None:
        G, G_ref = np.asarray(G, dtype=np.float64), np.asarray(G_ref, dtype=np.float64)
        out["grad_inf_rel"] = float(np.max(np.abs(G - G_ref)) / max(1.0, float(np.max(np.abs(G_ref)))))
    return out


def fp64_reference(B, ctx, c, h, theta, grad=True):
    """The same inputs through the complex128 mode of the same kernels (TLQ_FP64_REF), untimed."""
    if grad:
        return B.tlq_expectation_grad(ctx.h, c.h, h.h, theta, B.TLQ_FP64_REF)
    return B.tlq_expectation(ctx.h, c.h, h.h, theta, B.TLQ_FP64_REF), None


def plain_one_set_per_call(B, ctx, c, h, prob, dev, flush, grad=True, reps=3):
    """The plain per-circuit path: the same kernels called once per parameter set (B = 1),
    device pointers, all sets of the batch in sequence; device time with CUDA events (median
    of `reps` sweeps, L2 flushed before each sweep). Returns (ms per batch, launches per batch)."""
    import torch
    Bsz, P = prob.theta.shape
    stream = torch.cuda.current_stream(dev)
    theta_d = torch.tensor(prob.theta, dtype=torch.float64, device=dev)
    E_d = torch.empty(Bsz, dtype=torch.float64, device=dev)
    G_d = torch.empty(Bsz, P, dtype=torch.float64, device=dev)

    def sweep():
        for b in range(Bsz):
            B.tlq_expectation_grad_dev(ctx.h, c.h, h.h, theta_d[b].data_ptr(), 1, B.TLQ_FP32, E_d[b:].data_ptr(),
                                       G_d[b].data_ptr() if grad else None, stream.cuda_stream)

    B.tlq_profile_enable(ctx.h, False)
    sweep()
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sweep()
        b.record(stream)
        b.synchronize()
        t.append(a.elapsed_time(b))
    return float(np.median(t))


def run_reference(args, rank):
    """CPU oracle arm: each step evaluates energy + gradient of a sample of the workload's
    parameter sets with the complex128 statevector and its adjoint."""
    if rank != 0:
        return
    from oracle import dense
    from oracle.dense import omp_threads
    prob = workload(args.workload)
    sample = 2 if prob.n >= 16 else prob.B
    sets = [prob.theta[i % prob.B] for i in range(sample)]

    def step():
        for th in sets:
            dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    cores = omp_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": prob.n, "L": prob.meta.get("L"), "B": prob.B,
                   "sample_sets_per_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} of the {prob.B} parameter sets per step, dense 2^{prob.n} "
                                   f"complex128 statevector + adjoint"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(prob, budget_s=12.0):
    """The oracle as it stands on this host's cores over a bounded sample of the workload."""
    from oracle import dense
    from oracle.dense import omp_threads
    done = 0
    t0 = time.perf_counter()
    while True:
        th = prob.theta[done % prob.B]
        dense.grad_adjoint(prob.n, prob.gates, prob.terms, th, prob.n_params)
        done += 1
        if time.perf_counter() - t0 > budget_s or done >= prob.B:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
            "sample": f"{done} parameter sets of the workload (dense 2^{prob.n} complex128 statevector "
                      f"+ adjoint), {dt:.1f} s wall"}


def serving_replay(B, device, count, rate, seed=4, plain_path=True):
    """Replay a Poisson request stream (n ~ U[16,400], L ~ U[2,8], h ~ U[0.5,1.5], 30% with
    gradient) open-loop through tlq_submit/tlq_poll, and the same arrivals served one at a
    time through the synchronous calls (the plain path). Circuits are created once per
    (n, L) shape and kept resident; each request has its own Hamiltonian and angles."""
    import threading
    from paper_2112_10239_gb300 import workloads as W
    reqs = W.serving_stream(count, rate, seed)

    def prepare(ctx):
        circ, hams = {}, []
        for r in reqs:
            p = r.problem
            key = (p.n, p.meta["L"])
            if key not in circ:
                circ[key] = ctx.circuit(p.n, p.gates, p.n_params)
            hams.append(ctx.hamiltonian(p.n, p.terms))
        return circ, hams

    # warm-up in a throwaway context (module loading, kernel attributes)
    with B.Context(device=device) as wctx:
        c0, h0 = wctx.problem(reqs[0].problem)
        B.tlq_expectation(wctx.h, c0.h, h0.h, reqs[0].problem.theta)

    # batched serving
    ctx = B.Context(device=device)
    circ, hams = prepare(ctx)
    outs = [(np.zeros(1), np.zeros((1, r.problem.n_params)) if r.want_grad else None) for r in reqs]
    tickets = [None] * count
    ready = threading.Semaphore(0)
    t0 = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            due = t0 + r.t_arrival
            while True:
                d = due - time.perf_counter()
                if d <= 0:
                    break
                time.sleep(d if d > 2e-3 else 0)
            p = r.problem
            tickets[i] = B.tlq_submit(ctx.h, circ[(p.n, p.meta["L"])].h, hams[i].h, p.theta, outs[i][0], outs[i][1])
            ready.release()

    th = threading.Thread(target=submitter)
    th.start()
    for i in range(count):
        ready.acquire()
        B.tlq_poll(ctx.h, tickets[i], -1)
    t_end = time.perf_counter()
    th.join()
    n_done, p50, p99, mean_batch = B.tlq_serving_stats(ctx.h)
    batched = {"throughput_rps": count / (t_end - t0), "p50_ms": 1e3 * p50, "p99_ms": 1e3 * p99,
               "mean_batch": mean_batch, "completed": n_done}
    ctx.close()

    if not plain_path:
        return {"requests": count, "rate_per_s": rate, "batched": batched}
    # plain path: one request at a time through the synchronous calls, same arrivals
    ctx = B.Context(device=device)
    circ, hams = prepare(ctx)
    lat = []
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        due = t0 + r.t_arrival
        while time.perf_counter() < due:
            pass
        p = r.problem
        c = circ[(p.n, p.meta["L"])]
        if r.want_grad:
            B.tlq_expectation_grad(ctx.h, c.h, hams[i].h, p.theta)
        else:
            B.tlq_expectation(ctx.h, c.h, hams[i].h, p.theta)
        lat.append(time.perf_counter() - due)
    t_end = time.perf_counter()
    ctx.close()
    lat.sort()
    plain = {"throughput_rps": count / (t_end - t0), "p50_ms": 1e3 * lat[len(lat) // 2],
             "p99_ms": 1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]}
    return {"requests": count, "rate_per_s": rate, "grad_fraction": 0.3, "n": [16, 400], "L": [2, 8],
            "batched": batched, "one_at_a_time": plain}


def dense_bytes(B, ctx, c, h, grad, prec=None):
    """HBM bytes one evaluation of the dense pass sequence moves by its schedule (the library's
    own count, tlq_plan_dense_bytes: start state, forward passes, X/Y sweeps, and with the
    gradient lambda and the reverse passes). Returns (bytes, forward passes)."""
    _, _, n_fwd, _, _, _ = B.tlq_plan_dense_info(ctx.h, c.h, h.h)
    prec = B.TLQ_FP32 if prec is None else prec
    return B.tlq_plan_dense_bytes(ctx.h, c.h, h.h, grad, prec), n_fwd


def device_steps(B, ctx, c, h, prob, grad, steps, dev, flush, warmup=3, mps=False, prec=None):
    """Time `steps` device-pointer calls (inputs resident, L2 flushed between steps); mps=True
    times the exact MPS route (tlq_mps_expectation_grad_dev) instead of the default path."""
    prec = B.TLQ_FP32 if prec is None else prec
    import torch
    Bsz, P = prob.theta.shape
    stream = torch.cuda.current_stream(dev)
    theta_d = torch.tensor(prob.theta, dtype=torch.float64, device=dev)
    E_d = torch.empty(Bsz, dtype=torch.float64, device=dev)
    G_d = torch.empty(Bsz, P, dtype=torch.float64, device=dev) if grad else None

    call = B.tlq_mps_expectation_grad_dev if mps else B.tlq_expectation_grad_dev

    def step():
        call(ctx.h, c.h, h.h, theta_d.data_ptr(), Bsz, prec, E_d.data_ptr(),
             G_d.data_ptr() if grad else None, stream.cuda_stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    step_ms, kern_ms, launches = [], [], 0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        ms, nl = B.tlq_profile_last(ctx.h)
        kern_ms.append(ms)
        launches = nl
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    return float(np.median(step_ms)), float(np.median(kern_ms)), launches


def mps_workload(B, dev, local, flush, peaks, name, steps=5, warmup=3):
    """The exact MPS route (energy + gradient) on an Ising workload: device time of its five
    kernels, FP32 roofline from the plan's contraction flops, and the cone path beside it."""
    prob = workload(name)
    with B.Context(device=local) as ctx:
        c, h = ctx.problem(prob)
        B.tlq_profile_enable(ctx.h, True)
        bits, elems, _, fl = B.tlq_plan_mps_info(ctx.h, c.h, h.h)
        ms, kms, nl = device_steps(B, ctx, c, h, prob, True, steps, dev, flush, warmup=warmup, mps=True)
        cone_ms, _, _ = device_steps(B, ctx, c, h, prob, True, steps, dev, flush, warmup=warmup)
        c.close()
        h.close()
    peak = 152 * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    flops = fl * prob.B
    return {"value": prob.B / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "launches": nl,
            "bond_dimension": 2 ** bits, "elems_per_set": elems, "cone_path_ms_per_step": cone_ms,
            "roofline": {"bound": "alu", "achieved": flops / (kms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (kms * 1e-3) / 1e12 / peak, "kernel_ms": kms, "algorithmic_flops": flops,
                         "kernel": "mps_table/build/sweep/site/reduce kernels (complex64 contractions)",
                         "traffic": None}}


def golden_qaoa28():
    """The complex128 oracle's energy and gradient of the n=28, p=4 QAOA workload (seed 2),
    written by tests/golden/make_golden.py --large; None when absent."""
    path = os.path.join(ROOT, "tests", "golden", "qaoa_n28_p4.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def fp32_peak_tflops(peaks):
    return SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def n500_workload(B, dev, local, flush, peaks):
    """The n=500, L=4 Ising chain, 256 sets, energy + gradient (the paper's n=500 shape): one
    batched launch, the plain per-circuit path (one set per call) beside it, FP64 error."""
    from paper_2112_10239_gb300 import workloads as W
    prob = W.tfim_n500_L4_B256()
    with B.Context(device=local) as ctx:
        c, h = ctx.problem(prob)
        B.tlq_profile_enable(ctx.h, True)
        ms, kms, nl = device_steps(B, ctx, c, h, prob, True, 5, dev, flush)
        flops = algorithmic_flops(B, ctx, c, h, prob, grad=True)
        _, flops_unf = unfused_flops(prob)
        E, G = B.tlq_expectation_grad(ctx.h, c.h, h.h, prob.theta)
        E64, G64 = fp64_reference(B, ctx, c, h, prob.theta)
        plain_ms = plain_one_set_per_call(B, ctx, c, h, prob, dev, flush)
        c.close()
        h.close()
    peak = fp32_peak_tflops(peaks)
    ach = flops / (kms * 1e-3) / 1e12
    return {"value": prob.B / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "launches": nl,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "kernel_ms": kms, "algorithmic_flops": flops, "algorithmic_flops_unfused": flops_unf,
                         "frac_unfused": flops_unf / (kms * 1e-3) / 1e12 / peak,
                         "traffic": NCU_TRAFFIC.get(("tfim_n500_L4_B256", "cone_kernel"))},
            "err_vs_fp64": fp64_errors(E, G, E64, G64),
            "plain_path": {"kind": "one parameter set per call (B = 1), same kernels", "ms_per_batch": plain_ms,
                           "value": prob.B / (plain_ms * 1e-3), "unit": UNIT},
            "speedup_vs_plain": plain_ms / ms}


def qaoa28_workload(B, dev, local, flush, peaks):
    """n=28 QAOA on a 3-regular graph (dense statevector): energy and energy + gradient with the
    FP32 register passes, with the tensor-core blocks (TLQ_MIXED_TC), and with the plain
    per-gate FP32 sweeps; errors against the complex128 oracle's stored values."""
    import ctypes
    from paper_2112_10239_gb300 import workloads as W
    prob = W.qaoa_n28_p4()
    gold = golden_qaoa28()
    if gold is not None and not np.array_equal(np.asarray(gold["theta"]), prob.theta[0]):
        gold = None
    res = {}
    for name, fk, prec, grad, steps in (("fused", 0, B.TLQ_FP32, False, 5), ("fused_grad", 0, B.TLQ_FP32, True, 5),
                                        ("tc", 0, B.TLQ_MIXED_TC, False, 5), ("tc_grad", 0, B.TLQ_MIXED_TC, True, 5),
                                        ("per_gate", 1, B.TLQ_FP32, False, 2),
                                        ("per_gate_grad", 1, B.TLQ_FP32, True, 1)):
        cfg = B.tlq_config(local, 0, 0, B.TLQ_FP32, fk)
        hnd = ctypes.c_void_p()
        B._check(B.lib().tlq_init(ctypes.byref(cfg), ctypes.byref(hnd)))
        ctx = B.Context.__new__(B.Context)
        ctx.h = hnd
        c, h = ctx.problem(prob)
        B.tlq_profile_enable(ctx.h, True)
        ms, kms, nl = device_steps(B, ctx, c, h, prob, grad, steps, dev, flush, warmup=3 if fk == 0 else 1,
                                   prec=prec)
        nbytes, passes = dense_bytes(B, ctx, c, h, grad, prec)
        err = None
        if gold is not None and fk == 0:
            B.tlq_profile_enable(ctx.h, False)
            if grad:
                E, G = B.tlq_expectation_grad(ctx.h, c.h, h.h, prob.theta, prec)
                err = fp64_errors(E, G, [gold["energy"]], [gold["grad"]])
            else:
                err = fp64_errors(B.tlq_expectation(ctx.h, c.h, h.h, prob.theta, prec), None, [gold["energy"]], None)
        res[name] = (ms, kms, nl, nbytes, passes, err)
        c.close()
        h.close()
        ctx.close()

    def hbm(key, kernel):
        ms, kms, nl, nbytes, passes, _ = res[key]
        achieved = nbytes / (kms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "frac": achieved / float(peaks["hbm_gbs"]), "traffic": None, "kernel": kernel,
                "kernel_ms": kms, "bytes_per_eval": nbytes}

    ref = "complex128 CPU oracle (tests/golden/qaoa_n28_p4.json)" if gold is not None else None
    out = {}
    out["qaoa_n28_p4"] = {
        "value": 1.0 / (res["fused"][0] * 1e-3), "unit": "evals/s", "ms_per_eval": res["fused"][0],
        "passes": res["fused"][4], "launches": res["fused"][2],
        "roofline": hbm("fused", "dense_pass_kernel x passes (read + write of the 2 GiB state each)"),
        "err_vs_fp64": res["fused"][5], "fp64_reference": ref,
        "plain_path": {"kind": "per-gate FP32 statevector sweeps", "ms_per_eval": res["per_gate"][0]},
        "speedup_vs_plain": res["per_gate"][0] / res["fused"][0],
        "mixed_tc": {"ms_per_eval": res["tc"][0], "value": 1.0 / (res["tc"][0] * 1e-3), "launches": res["tc"][2],
                     "roofline": hbm("tc", "dense_tc_pass_kernel x passes (tcgen05 kind::tf32 split blocks)"),
                     "err_vs_fp64": res["tc"][5], "speedup_vs_plain": res["per_gate"][0] / res["tc"][0],
                     "vs_fp32_fused": res["fused"][0] / res["tc"][0]}}
    out["qaoa_n28_p4_grad"] = {
        "value": 1.0 / (res["fused_grad"][0] * 1e-3), "unit": "grad-evals/s", "ms_per_eval": res["fused_grad"][0],
        "launches": res["fused_grad"][2],
        "roofline": hbm("fused_grad", "forward dense_pass_kernel x passes, then dense_adjoint_kernel x passes "
                                      "(psi and lam read + written)"),
        "err_vs_fp64": res["fused_grad"][5], "fp64_reference": ref,
        "plain_path": {"kind": "per-gate FP32 statevector sweeps", "ms_per_eval": res["per_gate_grad"][0]},
        "speedup_vs_plain": res["per_gate_grad"][0] / res["fused_grad"][0],
        "mixed_tc": {"ms_per_eval": res["tc_grad"][0], "err_vs_fp64": res["tc_grad"][5],
                     "speedup_vs_plain": res["per_gate_grad"][0] / res["tc_grad"][0],
                     "vs_fp32_fused": res["fused_grad"][0] / res["tc_grad"][0]}}
    return out


SERVING_RATES = (100.0, 300.0, 1000.0, 2000.0, 5000.0)
SERVING_REQUESTS = 10000


def extra_workloads(B, dev, local, flush, peaks):
    """The other workloads, each with its own throughput and roofline (not the headline)."""
    out = {}
    out["tfim_n500_L4_B256"] = n500_workload(B, dev, local, flush, peaks)
    # the exact MPS route on the two Ising batches (bond dimension 16 and 64), beside the cone path
    for name in ("tfim_n500_L4_B256", "tfim_n20_L6_B64"):
        out["mps_" + name] = mps_workload(B, dev, local, flush, peaks, name, steps=3)
    # n=8, L=2, one set: latency of the synchronous call (launch-bound; no roofline)
    out["tfim_n8_L2_B1_latency"] = latency_n8(B, local)
    out.update(qaoa28_workload(B, dev, local, flush, peaks))
    # partial traces of an n=20 state down to m=14 and m=10 qubits (the paper's density-operator
    # sizes): rho_A = Psi Psi^dagger
    out.update(partial_trace_workloads(B, dev, local, flush, peaks))
    # serving: Poisson arrivals of 10,000 requests at each offered rate, continuous batching; the
    # plain path (one request at a time through the synchronous calls) at 2000 requests/s
    sweep = []
    for rate in SERVING_RATES:
        r = serving_replay(B, local, SERVING_REQUESTS, rate, seed=4, plain_path=(rate == 2000.0))
        entry = {"rate_per_s": rate, "requests": SERVING_REQUESTS, **r["batched"]}
        if "one_at_a_time" in r:
            entry["one_at_a_time"] = r["one_at_a_time"]
        sweep.append(entry)
    out["serving_sweep"] = sweep
    return out


def summary_of(line, extras):
    """A compact digest of every workload's headline figures (kept short: it closes the line)."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def r3(x):
        return None if x is None else float(f"{x:.4g}")

    out = {line["config"]["workload"]: {"evals_s": r3(line["value"]), "e2e_evals_s": r3(line["e2e"]["value"]),
                               "frac": r3(line["roofline"]["frac"]),
                               "frac_unfused": r3(line["roofline"].get("frac_unfused")),
                               "err_vs_fp64": {k: r3(v) for k, v in (line.get("err_vs_fp64") or {}).items()},
                               "speedup_vs_one_set_per_call": r3(g(line, "plain_path", "speedup_one_set_per_call")),
                               "speedup_vs_per_gate": r3(g(line, "plain_path", "speedup_per_gate_statevector"))}}
    if not extras:
        return out
    c4 = extras.get("tfim_n500_L4_B256", {})
    out["tfim_n500_L4_B256"] = {"evals_s": r3(c4.get("value")), "ms": r3(c4.get("ms_per_step")),
                                "frac": r3(g(c4, "roofline", "frac")), "frac_unfused": r3(g(c4, "roofline", "frac_unfused")),
                                "err_vs_fp64": {k: r3(v) for k, v in (c4.get("err_vs_fp64") or {}).items()},
                                "speedup_vs_one_set_per_call": r3(c4.get("speedup_vs_plain"))}
    c1 = extras.get("tfim_n8_L2_B1_latency", {})
    out["tfim_n8_L2_B1"] = {"p50_us": r3(g(c1, "gpu", "p50_us")), "p99_us": r3(g(c1, "gpu", "p99_us")),
                            "cpu_p50_us": r3(g(c1, "cpu_oracle", "p50_us")),
                            "err_vs_fp64": {k: r3(v) for k, v in (c1.get("err_vs_fp64") or {}).items()}}
    c3, c3g = extras.get("qaoa_n28_p4", {}), extras.get("qaoa_n28_p4_grad", {})
    out["qaoa_n28_p4"] = {"ms": r3(c3.get("ms_per_eval")), "frac_hbm": r3(g(c3, "roofline", "frac")),
                          "grad_ms": r3(c3g.get("ms_per_eval")), "grad_frac_hbm": r3(g(c3g, "roofline", "frac")),
                          "err": {k: r3(v) for k, v in (c3g.get("err_vs_fp64") or {}).items()},
                          "tc_ms": r3(g(c3, "mixed_tc", "ms_per_eval")), "tc_grad_ms": r3(g(c3g, "mixed_tc", "ms_per_eval")),
                          "tc_err": {k: r3(v) for k, v in (g(c3g, "mixed_tc", "err_vs_fp64") or {}).items()},
                          "speedup_vs_per_gate": r3(c3.get("speedup_vs_plain"))}
    for key in ("partial_trace_n20_m14", "partial_trace_n20_m10"):
        pt = extras.get(key, {})
        out[key] = {"ms": r3(pt.get("ms")), "bound": g(pt, "roofline", "bound"), "frac": r3(g(pt, "roofline", "frac")),
                    "max_abs_err": r3(pt.get("max_abs_err_vs_oracle"))}
    out["serving"] = [{"rate": s["rate_per_s"], "rps": r3(s.get("throughput_rps")), "p50_ms": r3(s.get("p50_ms")),
                       "p99_ms": r3(s.get("p99_ms")),
                       **({"plain_rps": r3(s["one_at_a_time"]["throughput_rps"]),
                           "plain_p50_ms": r3(s["one_at_a_time"]["p50_ms"])} if "one_at_a_time" in s else {})}
                      for s in extras.get("serving_sweep", [])]
    return out


def latency_n8(B, local, calls=10000):
    """n=8, L=2, one parameter set, energy only: a launch-bound call, reported as latency.
    GPU: the synchronous host-pointer call (H2D of the angles, kernels, D2H of the energy) timed
    with the host clock per call. CPU: the oracle's plain statevector energy per call."""
    from oracle import dense
    from paper_2112_10239_gb300 import workloads as W
    prob = W.tfim_n8_L2()
    th = np.ascontiguousarray(prob.theta)

    def pct(v):
        v = sorted(v)
        return {"p50_us": 1e6 * v[len(v) // 2], "p99_us": 1e6 * v[min(len(v) - 1, int(math.ceil(0.99 * len(v))) - 1)]}

    with B.Context(device=local) as ctx:
        c, h = ctx.problem(prob)
        for _ in range(100):
            B.tlq_expectation(ctx.h, c.h, h.h, th)
        err = fp64_errors(B.tlq_expectation(ctx.h, c.h, h.h, th), None,
                          B.tlq_expectation(ctx.h, c.h, h.h, th, B.TLQ_FP64_REF), None)
        t = []
        for _ in range(calls):
            t0 = time.perf_counter()
            B.tlq_expectation(ctx.h, c.h, h.h, th)
            t.append(time.perf_counter() - t0)
        c.close()
        h.close()
    cpu = []
    for _ in range(calls // 10):
        t0 = time.perf_counter()
        dense.energy(prob.n, prob.gates, prob.terms, prob.theta[0])
        cpu.append(time.perf_counter() - t0)
    return {"workload": "tfim_n8_L2_B1 (energy)", "calls": calls, "gpu": pct(t),
            "cpu_oracle": {**pct(cpu), "calls": len(cpu)}, "err_vs_fp64": err,
            "fp64_reference": "TLQ_FP64_REF (complex128 mode of the same kernels)"}


def partial_trace_workloads(B, dev, local, flush, peaks, n=20, ms=(14, 10), steps=10, warmup=3, with_cpu=True):
    """Device time of tlq_partial_trace_dev on a seeded random n-qubit state, and the oracle
    (numpy: one reshape/transpose and one complex128 matrix product) on the host."""
    import torch
    from oracle import density
    rng = np.random.default_rng(11)
    psi = rng.normal(size=2 ** n) + 1j * rng.normal(size=2 ** n)
    psi /= np.linalg.norm(psi)
    psi_d = torch.tensor(psi.astype(np.complex64).view(np.float32), device=dev)
    peak = 152 * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    out = {}
    with B.Context(device=local) as ctx:
        B.tlq_profile_enable(ctx.h, True)
        stream = torch.cuda.Stream(dev)   # a real handle: the events and the library share it
        torch.cuda.set_stream(stream)
        for m in ms:
            keep = list(range(n - m, n)) if m == ms[0] else list(range(m))
            rho_d = torch.empty(2 * 4 ** m, dtype=torch.float32, device=dev)
            for _ in range(max(1, warmup)):
                B.tlq_partial_trace_dev(ctx.h, psi_d.data_ptr(), n, keep, rho_d.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            t, kt = [], []
            for _ in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                B.tlq_partial_trace_dev(ctx.h, psi_d.data_ptr(), n, keep, rho_d.data_ptr(), stream.cuda_stream)
                b.record(stream)
                kms, nl = B.tlq_profile_last(ctx.h)
                b.synchronize()
                t.append(a.elapsed_time(b))
                kt.append(kms)
            D, K = 2 ** m, 2 ** (n - m)
            flops = 8.0 * D * (D + 1) / 2 * K      # Hermitian half of rho = Psi Psi^dagger (complex MACs x 8)
            kms = float(np.median(kt))
            rho_h = rho_d.cpu().numpy().view(np.complex64).reshape(D, D)
            cpu_s = None
            t0 = time.perf_counter()
            rho_ref = density.reduced_density(psi, n, keep)
            cpu_s = time.perf_counter() - t0
            max_err = 0.0
            for r0 in range(0, D, 1024):   # in row blocks: the m=14 output is 2 GiB
                blk = rho_h[r0:r0 + 1024].astype(np.complex128) - rho_ref[r0:r0 + 1024]
                max_err = max(max_err, float(np.max(np.abs(blk))))
            del rho_ref, rho_h
            del rho_d
            hbm_bytes = 8 * D * D + 3 * 8 * 2 ** n     # rho written; psi read, Psi written and read
            hbm_peak = float(peaks["hbm_gbs"])
            hbm_floor = hbm_bytes / (hbm_peak * 1e9)
            if m >= 7:
                # tensor cores (tcgen05 kind::tf32): the bound is set by the algorithmic flops against
                # the TF32 peak; executed flops (six split-TF32 MMAs of 128 x 256 x 8 per 128 x 128
                # upper tile and 8 complex k) are reported beside it
                T = (D + 127) // 128
                tc_flops = T * (T + 1) // 2 * (K / 8) * 6 * 2 * 128 * 256 * 8
                ws = T * (T + 1) // 2 >= torch.cuda.get_device_properties(0).multi_processor_count and n - m >= 3
                tf32_peak = float(peaks["bf16_tflops"]) * 1.1 / 2.25   # nominal TF32 / BF16 dense ratio
                tc_floor = flops / (tf32_peak * 1e12)
                if hbm_floor >= tc_floor:
                    roof = {"bound": "hbm", "achieved": hbm_bytes / (kms * 1e-3) / 1e9, "peak": hbm_peak,
                            "unit": "GB/s", "frac": hbm_bytes / (kms * 1e-3) / 1e9 / hbm_peak}
                else:
                    roof = {"bound": "tensor", "achieved": flops / (kms * 1e-3) / 1e12, "peak": tf32_peak,
                            "unit": "TFLOP/s", "frac": flops / (kms * 1e-3) / 1e12 / tf32_peak,
                            "peak_basis": "measured bf16 dense x 1.1/2.25 (nominal TF32/BF16)"}
                roof.update({"kernel": ("herk_ws_kernel (persistent, warp-specialised" if ws else
                                        "herk_tc_kernel (split k") + "; tcgen05 kind::tf32, TMEM accumulators)",
                             "tensor_tflops_algorithmic": flops / (kms * 1e-3) / 1e12,
                             "tensor_frac_algorithmic": flops / (kms * 1e-3) / 1e12 / tf32_peak,
                             "tensor_tflops_executed": tc_flops / (kms * 1e-3) / 1e12,
                             "hbm_gbs": hbm_bytes / (kms * 1e-3) / 1e9, "hbm_frac": hbm_bytes / (kms * 1e-3) / 1e9 / hbm_peak})
            else:
                roof = {"bound": "alu", "achieved": flops / (kms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": flops / (kms * 1e-3) / 1e12 / peak, "kernel": "herk_tile_kernel (FP32)"}
            kname = roof["kernel"].split(" ")[0]
            roof.update({"kernel_ms": kms, "traffic": NCU_TRAFFIC.get((f"partial_trace_n{n}_m{m}", kname)),
                         "hbm_bytes": hbm_bytes, "algorithmic_flops": flops})
            out[f"partial_trace_n{n}_m{m}"] = {
                "value": 1e3 / float(np.median(t)), "unit": "traces/s", "ms": float(np.median(t)), "launches": nl,
                "keep": f"qubits {keep[0]}..{keep[-1]}", "roofline": roof, "max_abs_err_vs_oracle": max_err,
                "cpu_baseline": None if not with_cpu else {
                    "value": 1.0 / cpu_s, "unit": "traces/s", "kind": "oracle", "cores": len(os.sched_getaffinity(0)),
                    "sample": "one full trace (numpy complex128)"}}
    return out


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from __graft_entry__ import build
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    from paper_2112_10239_gb300 import binding as B

    if args.workload.startswith("mps_"):   # the exact MPS route alone, one replica per rank
        dev = torch.device("cuda", local)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        torch.cuda.set_stream(torch.cuda.Stream(dev))   # a real stream handle (the legacy default is 0)
        peaks, peak_kind = measured_peaks()
        r = mps_workload(B, dev, local, flush, peaks, args.workload[4:], steps=args.steps,
                         warmup=max(3, args.warmup))
        if rank == 0:
            prob = workload(args.workload[4:])
            print(json.dumps({"metric": METRIC, "value": world * r["value"], "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic", "config": {"workload": args.workload, "n": prob.n,
                                                              "L": prob.meta.get("L"), "B": prob.B,
                                                              "route": "exact MPS", "l2": "flushed between steps"},
                              "gpu_launches": r["launches"] * args.steps, "roofline": r["roofline"],
                              "bond_dimension": r["bond_dimension"],
                              "cone_path_ms_per_step": r["cone_path_ms_per_step"], "peak_source": peak_kind}),
                  flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    pt = re.fullmatch(r"partial_trace_n(\d+)_m(\d+)", args.workload)
    if pt:   # the partial trace alone (device time of tlq_partial_trace_dev), one replica per rank
        n, m = int(pt.group(1)), int(pt.group(2))
        if not 1 <= m <= min(n, 15) or n > 31:
            raise SystemExit("partial_trace workloads take 1 <= m <= min(n, 15), n <= 31")
        dev = torch.device("cuda", local)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        peaks, peak_kind = measured_peaks()
        res = partial_trace_workloads(B, dev, local, flush, peaks, n=n, ms=(m,), steps=args.steps,
                                      warmup=args.warmup, with_cpu=not args.no_extras)
        r = res[f"partial_trace_n{n}_m{m}"]
        if rank == 0:
            print(json.dumps({"metric": "partial traces/sec", "value": world * r["value"], "unit": "traces/s",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                              "data": "synthetic", "config": {"workload": args.workload, "n": n, "m": m,
                                                              "keep": r["keep"], "l2": "flushed between steps"},
                              "gpu_launches": r["launches"] * args.steps, "roofline": r["roofline"],
                              "peak_source": peak_kind, "cpu_baseline": r.get("cpu_baseline")}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    prob = workload(args.workload)
    ctx = B.Context(device=local)
    c, h = ctx.problem(prob)
    Bsz, P = prob.theta.shape
    dev = torch.device("cuda", local)
    theta_d = torch.tensor(prob.theta, dtype=torch.float64, device=dev)
    E_d = torch.empty(Bsz, dtype=torch.float64, device=dev)
    G_d = torch.empty(Bsz, P, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)       # a real stream handle (the legacy default is 0)
    torch.cuda.set_stream(stream)
    B.tlq_profile_enable(ctx.h, True)

    prec = B.TLQ_MIXED_TC if args.prec == "mixed_tc" else B.TLQ_FP32
    grad = not args.energy_only
    metric, unit = (METRIC, UNIT) if grad else ("expectation evals/sec", "evals/s")

    def step():
        B.tlq_expectation_grad_dev(ctx.h, c.h, h.h, theta_d.data_ptr(), Bsz, prec, E_d.data_ptr(),
                                   G_d.data_ptr() if grad else 0, stream.cuda_stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    step_ms, kern_ms, launches = [], [], 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()                      # evict L2 between timed steps (untimed)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        ms, nl = B.tlq_profile_last(ctx.h)
        kern_ms.append(ms)
        launches += nl
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_s = job_throughput(sum(step_ms) / 1e3, Bsz * args.steps, world, dev)

    # end to end through the host-pointer API (H2D of theta and D2H of energy + gradient inside);
    # kernel profiling off, as for any caller (it records events around single kernels)
    B.tlq_profile_enable(ctx.h, False)
    theta_h = np.ascontiguousarray(prob.theta)

    def host_call():
        if grad:
            return B.tlq_expectation_grad(ctx.h, c.h, h.h, theta_h, prec)
        return B.tlq_expectation(ctx.h, c.h, h.h, theta_h, prec), None

    for _ in range(3):
        host_call()
    e2e_t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        E_h, G_h = host_call()
        e2e_t.append(time.perf_counter() - t0)
    e2e_value, _ = job_throughput(sum(e2e_t), Bsz * len(e2e_t), world, dev)

    # error of the timed result (FP32) against the complex128 mode of the same kernels
    path, *_ = B.tlq_plan_info(ctx.h, c.h, h.h, len(prob.terms))
    err64 = None
    if path == B.TLQ_PATH_CONE:
        E64, G64 = fp64_reference(B, ctx, c, h, theta_h, grad)
        err64 = fp64_errors(E_h, G_h, E64, G64)

    # the plain per-circuit FP32 path on the same GPU: one parameter set per call, and (up to 24
    # qubits) the per-gate statevector sweeps
    plain = None
    if rank == 0 and not args.no_extras and grad and path == B.TLQ_PATH_CONE:
        import ctypes
        one_ms = plain_one_set_per_call(B, ctx, c, h, prob, dev, flush)
        plain = {"one_set_per_call": {"kind": "one parameter set per call (B = 1), same kernels",
                                      "ms_per_batch": one_ms, "value": Bsz / (one_ms * 1e-3), "unit": UNIT}}
        if prob.n <= 24:
            cfg = B.tlq_config(local, 0, 0, B.TLQ_FP32, 1)
            hnd = ctypes.c_void_p()
            B._check(B.lib().tlq_init(ctypes.byref(cfg), ctypes.byref(hnd)))
            pctx = B.Context.__new__(B.Context)
            pctx.h = hnd
            pc, ph = pctx.problem(prob)
            B.tlq_profile_enable(pctx.h, True)
            pg_ms, _, _ = device_steps(B, pctx, pc, ph, prob, True, 1, dev, flush, warmup=1)
            pc.close()
            ph.close()
            pctx.close()
            plain["per_gate_statevector"] = {"kind": "per-gate FP32 sweeps of the 2^n statevector, "
                                                     "per-gate adjoint", "ms_per_batch": pg_ms,
                                             "value": Bsz / (pg_ms * 1e-3), "unit": UNIT}
        torch.cuda.set_stream(stream)

    # roofline of the dominant kernel (the batched cone kernel), ALU-bound FP32
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    kern_mean_ms = float(np.mean(kern_ms))
    if path == B.TLQ_PATH_DENSE:
        nbytes, passes = dense_bytes(B, ctx, c, h, grad, prec)
        achieved = nbytes / (kern_mean_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                    "frac": achieved / float(peaks["hbm_gbs"]), "traffic": None,
                    "kernel": ("dense_tc_pass_kernel" if args.prec == "mixed_tc" else "dense_pass_kernel") +
                              (" + dense_adjoint_kernel (forward and reverse passes)" if grad else
                               " (forward passes)"),
                    "kernel_ms": kern_mean_ms, "bytes_per_eval": nbytes, "passes": passes}
    else:
        flops = algorithmic_flops(B, ctx, c, h, prob, grad=grad)
        _, flops_unf = unfused_flops(prob, grad=grad)
        achieved = flops / (kern_mean_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                    "frac": achieved / peak_tflops, "traffic": NCU_TRAFFIC.get((args.workload, "cone_kernel")),
                    "kernel": ("cone_kernel<float,grad> (batched causal cones + adjoint)" if grad else
                               "cone_kernel<float,energy> (batched causal cones)"),
                    "kernel_ms": kern_mean_ms, "algorithmic_flops": flops,
                    "algorithmic_flops_basis": "work the shared windows require (terms nested in a window are "
                                               "measured on it)",
                    "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop/FMA x {sm_max:.0f} MHz"}
        if flops_unf is not None:
            roofline.update({"algorithmic_flops_unfused": flops_unf,
                             "frac_unfused": flops_unf / (kern_mean_ms * 1e-3) / 1e12 / peak_tflops,
                             "unfused_basis": "every term on its own exact causal cone" +
                                              (", adjoint = 3 x forward" if grad else ", forward and measurement")})

    extras = extra_workloads(B, dev, local, flush, peaks) if rank == 0 and not args.no_extras else {}
    if rank == 0:
        cpu = None if (args.no_extras or not grad) else cpu_baseline(prob)
        sm = sorted(step_ms)
        line = {
            "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n": prob.n, "L": prob.meta.get("L"), "B": Bsz, "prec": args.prec,
                       "n_params": P, "terms": len(prob.terms), "l2": "flushed: 256 MiB write between timed steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "latency_ms": {"p50": sm[len(sm) // 2], "p99": sm[min(len(sm) - 1, int(math.ceil(0.99 * len(sm))) - 1)],
                           "per": f"batch of {Bsz} parameter sets"},
            "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": int(theta_h.nbytes),
                    "d2h_bytes_per_step": int(E_h.nbytes + (G_h.nbytes if G_h is not None else 0))},
            "gpu_launches": launches,
            "roofline": roofline,
            "err_vs_fp64": err64,
            "fp64_reference": "TLQ_FP64_REF (complex128 mode of the same kernels), same inputs" if err64 else None,
            "peak_source": peak_kind,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        if plain is not None:
            for k, v in list(plain.items()):
                plain[f"speedup_{k}"] = v["ms_per_batch"] / (1e3 * total_s / args.steps)
            line["plain_path"] = plain
        line["other_workloads"] = extras
        line["summary"] = summary_of(line, extras)   # last: the compact digest closes the line
        print(json.dumps(line), flush=True)
    c.close()
    h.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
