#!/usr/bin/env python
"""Throughput benchmark of the GB300 DGSEM path: DOF-stage updates per second.

Workload (default): the Taylor-Green vortex (Re 1600, Mach 0.1, Pr 0.71) on
32^3 elements at P = 3, 16^3 at P = 6 and 16^3 at P = 8, FP32 operator with FP64
state and FP64 RK3 accumulation.  One step = one RK3 time step (three stages, each a
BR1-gradient launch and a flux/lift/RK-update launch) on each of the three meshes.
A DOF is a node carrying five variables (dof = N_el (P+1)^3); one DOF-stage update is
one node advanced through one RK stage.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs the same workload on
its own GPU (independent replicas: the method needs no data exchange for this
workload); timing is the max over ranks.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = [(32, 3), (16, 6), (16, 8)]
WORKLOAD_NAME = "tgv-re1600-m0.1: 32^3/P3 + 16^3/P6 + 16^3/P8, FP32 operator, FP64 state, RK3"
RE, MACH, PR, CFL = 1600.0, 0.1, 0.71, 0.7
METRIC = "DOF-stage updates/s (TGV 32^3/P3, 16^3/P6, 16^3/P8 per RK3 step)"
UNIT = "DOF-stage updates/s"
CPU_SAMPLE = [(8, 3), (8, 6), (8, 8)]
KERNEL_SOURCES = ["dg_kernels.cuh", "dg_device.cuh", "dg_launch.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["tgv3", "batched"], default="tgv3",
                    help="tgv3: the three TGV meshes (default); batched: 12 independent TGV instances "
                         "(Re from {30, 200, 1600}, meshes 8^3-16^3, P in {3, 6}) in one batch")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_11571_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernels."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    rec = data.get(kernel, {}).get(workload)
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


def nn_measure(stream, steps=100):
    """Forcing network of the corrected P=3 run (5 x 64 = 320 inputs and outputs, 4 hidden
    layers of 512, batch 4096): one training step (forward, MSE, backward, Adam) and one
    forcing evaluation on a 16^3 P=3 state, timed with CUDA events."""
    import torch

    from paper_2207_11571_gb300 import dg, inputs, nn
    feat, width, hidden, batch = 320, 512, 4, 4096
    dims = [feat] + [width] * hidden + [feat]
    flop_fwd = 2 * batch * sum(dims[i] * dims[i + 1] for i in range(len(dims) - 1))
    net = nn.nn_create(feat, feat, width, hidden, 0, 5, batch, inputs.uniform_draws(dims, 7))
    rows = 4 * batch
    X = torch.from_numpy(inputs.normal((rows, feat), 8).astype("float32")).cuda()
    Y = torch.from_numpy(inputs.normal((rows, feat), 9).astype("float32")).cuda()
    nn.nn_compute_scalers(net, X, Y)
    perm = torch.from_numpy(inputs.epoch_permutation(rows, 7, 0)).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(5):
        nn.nn_train_step(net, X, Y, perm[:batch], want_loss=False, stream=stream)
    e0.record(stream)
    for i in range(steps):
        j = (i % 4) * batch
        nn.nn_train_step(net, X, Y, perm[j:j + batch], want_loss=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    train_us = e0.elapsed_time(e1) / steps * 1e3
    c = dg.dg_create(16, 3, RE, MACH, PR, 0, precision=dg.DG_PREC_FP32)
    N = dg.dg_sizes(c)[0]
    q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(c, q)
    s = torch.empty(5 * N, dtype=torch.float32, device="cuda")
    for i in range(5):
        nn.nn_forcing_infer(net, c, q, s, stream)
    e0.record(stream)
    for i in range(steps):
        nn.nn_forcing_infer(net, c, q, s, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    infer_us = e0.elapsed_time(e1) / steps * 1e3
    dg.dg_destroy(c)
    nn.nn_destroy(net)
    peak, kind = bf16_peak()
    tr = 3 * flop_fwd / (train_us * 1e-6) / 1e12
    inf = flop_fwd / (infer_us * 1e-6) / 1e12
    return {"network": "320-512x4-320, batch 4096 (16^3 elements at P=3)",
            "train_step_us": round(train_us, 1), "train_tflops": round(tr, 1),
            "forcing_infer_us": round(infer_us, 1), "forcing_infer_tflops": round(inf, 1),
            "note": "forcing_infer includes the phase-A stage-state launch; tensor work is the 5 GEMMs",
            "roofline": {"bound": "tensor", "peak": peak, "unit": "TFLOP/s", "peak_source": kind,
                         "train_frac": round(tr / peak, 4), "infer_frac": round(inf / peak, 4)}}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.tmp.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample_rate(repeats=1):
    """FP64 oracle (numpy, single thread) on one RK3 stage of an 8^3 mesh at each order."""
    import numpy as np

    from oracle import dgsem, physics
    flow = physics.Flow(Re=RE, Mach=MACH, Pr=PR)
    total_nodes, total_s = 0, 0.0
    for K, P in CPU_SAMPLE:
        mesh = dgsem.Mesh(K, P)
        q = dgsem.tgv_state(mesh, flow)
        dt = dgsem.stable_dt(q, mesh, flow, CFL)
        for _ in range(repeats):
            t0 = time.perf_counter()
            g = dt * dgsem.rhs(q, mesh, flow)       # one RK3 stage (first stage: A = 0)
            q = q + dgsem.RK3_B[0] * g
            total_s += time.perf_counter() - t0
            total_nodes += q[0].size
        del q, g
    return total_nodes / total_s, total_s, "one RK3 stage of the FP64 oracle on 8^3 elements at P=3, 6, 8 " \
                                           "(same per-DOF work as the benchmark meshes)"


def run_reference(args, rank, ws):
    if rank != 0:
        return 0
    times, nodes = [], 0
    for i in range(args.warmup + args.steps):
        rate, secs, sample = oracle_sample_rate()
        if i >= args.warmup:
            times.append(secs)
    total_nodes = sum(K ** 3 * (P + 1) ** 3 for K, P in CPU_SAMPLE) * args.steps
    value = total_nodes / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (closed-form TGV field)",
            "config": {"workload": WORKLOAD_NAME, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU path

def run_ours(args, rank, ws):
    import torch

    from paper_2207_11571_gb300 import build as _build
    from paper_2207_11571_gb300 import dg, inputs
    if not os.path.exists(_build.LIB):
        _build.build()
    dg.lib()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    ctxs, states, dts, nodes, tuned = [], [], [], [], []
    for K, P in WORKLOAD:
        c = dg.dg_create(K, P, RE, MACH, PR, 0, precision=dg.DG_PREC_FP32)
        N = dg.dg_sizes(c)[0]
        q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        pert = torch.from_numpy(inputs.perturbation((5, N), seed=inputs.TGV_SEED + rank).ravel()).cuda()
        dg.dg_init_tgv(c, q, pert)
        del pert
        dts.append(dg.dg_stable_dt(c, q, CFL))
        tuned.append(dg.dg_autotune(c, q, dts[-1])[0])
        ctxs.append(c)
        states.append(q)
        nodes.append(N)
    updates_per_step = 3 * sum(nodes)

    def step():
        for c, q, dt in zip(ctxs, states, dts):
            dg.dg_rk3_step(c, q, dt, 1, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    value = updates_per_step * args.steps * ws / (ms / 1e3)

    # per-kernel device times (CUDA events around each launch, on the launching stream)
    prof = []
    for (K, P), c, q, dt in zip(WORKLOAD, ctxs, states, dts):
        p = dg.dg_profile_rk3(c, q, dt, 3, stream)
        p["workload"] = f"{K}^3/P{P}"
        prof.append(p)
    total_ms = sum(p["ms_gradient"] + p["ms_flux"] for p in prof)
    kernels = []
    for p in prof:
        for kind in ("flux", "gradient"):
            kernels.append({"kernel": "k_flux" if kind == "flux" else "k_gradient", "workload": p["workload"],
                            "ms": p[f"ms_{kind}"], "launches": p[f"launches_{kind}"],
                            "bytes_per_launch": p[f"{kind}_bytes_per_launch"],
                            "share": p[f"ms_{kind}"] / total_ms})
    dom = max(kernels, key=lambda k: k["ms"])
    peak, peak_kind = peaks()
    achieved = dom["bytes_per_launch"] / (dom["ms"] / dom["launches"] / 1e3) / 1e9
    traffic = measured_traffic(dom["kernel"], dom["workload"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "kernel": f'{dom["kernel"]} {dom["workload"]}',
                "traffic": traffic}
    # the whole timed step on the same bytes: every launch of one RK3 step of every mesh
    # (3 stages x both phases, stage-averaged bytes per launch) over the timed ms per step
    step_bytes = sum(3 * (p["flux_bytes_per_launch"] + p["gradient_bytes_per_launch"]) for p in prof)
    step_gbs = step_bytes / (ms / args.steps / 1e3) / 1e9
    roofline["step"] = {"achieved": step_gbs, "frac": step_gbs / peak,
                        "bytes_per_dof_stage": step_bytes / updates_per_step,
                        "note": "all launches of the timed steps, including the gaps between them"}
    per_kernel =[{k: (round(v, 5) if isinstance(v, float) else v) for k, v in kk.items()} for kk in kernels]

    # end to end through the C ABI with HOST buffers (pinned), copies inside the timed region
    host = [torch.empty(5 * n, dtype=torch.float64, pin_memory=True) for n in nodes]
    for h, q in zip(host, states):
        h.copy_(q)
    torch.cuda.synchronize()
    barrier(ws)
    # one stream per mesh: each mesh's copies overlap the other meshes' kernels.  Every
    # step of a mesh copies its state in, advances it, copies it out and reads its
    # diagnostics; a mesh waits for its own previous step only, so the meshes' steps
    # interleave on the host link.
    streams = [torch.cuda.Stream() for _ in ctxs]
    for c, h, dt, s in zip(ctxs, host, dts, streams):   # untimed: allocates each context's device copy
        dg.dg_advance_host_async(c, h, dt, 0, None, s, want_diag=False)
        dg.dg_advance_host_wait(c, s, want_diag=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(args.e2e_steps):
        for c, h, dt, s in zip(ctxs, host, dts, streams):
            if step:
                dg.dg_advance_host_wait(c, s, want_diag=True)
            dg.dg_advance_host_async(c, h, dt, 1, None, s, want_diag=True)
    for c, s in zip(ctxs, streams):
        dg.dg_advance_host_wait(c, s, want_diag=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": updates_per_step * args.e2e_steps * ws / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": sum(5 * 8 * n for n in nodes), "d2h_bytes_per_step": sum(5 * 8 * n for n in nodes),
           "call": "dg_advance_host_async + dg_advance_host_wait per mesh, one stream per mesh (pinned host "
                   "state copied in and out, 1 RK3 step + diagnostics per mesh every step)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, secs, sample = oracle_sample_rate(repeats=4)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               "seconds": round(secs, 2)}

    nn_line = nn_measure(stream)

    per_workload = {}
    for (K, P), n, p in zip(WORKLOAD, nodes, prof):
        per_workload[f"{K}^3/P{P}"] = {"nodes": n, "dof_stage_per_s_kernels":
                                       3 * 3 * n / ((p["ms_gradient"] + p["ms_flux"]) / 1e3)}
    shapes = ["cube 2x2x2" if dg.dg_blocking(c)[1] else "row" for c in ctxs]
    for c in ctxs:
        dg.dg_destroy(c)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 operator / f64 state",
                "data": "synthetic (closed-form TGV field + seeded 1e-6 perturbation)",
                "config": {"workload": WORKLOAD_NAME, "meshes": [f"{K}^3/P{P}" for K, P in WORKLOAD],
                           "nodes": nodes, "l2": "working set per mesh 190-400 MB > 129 MB L2 (no flush)",
                           "elems_per_block": tuned,
                           "block_shape": shapes,
                           "parallelism": f"replicas x{ws}", "per_workload": per_workload},
                "roofline": roofline, "kernels": per_kernel, "network": nn_line, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 6 * len(WORKLOAD) * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- batched instances

# FP32-operator algorithmic bytes per node of one RK3 step (both launches of all stages)
STEP_BYTES_PER_NODE = 676.0


def run_batched(args, rank, ws):
    import torch

    from paper_2207_11571_gb300 import build as _build
    from paper_2207_11571_gb300 import dg, inputs
    if not os.path.exists(_build.LIB):
        _build.build()
    dg.lib()
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    members = inputs.batch_members()
    b = dg.dg_create_batch([(K, P, Re, MACH, PR, 0) for K, P, Re in members], precision=dg.DG_PREC_FP32)
    qs, dts, nodes = [], [], []
    for i, (K, P, Re) in enumerate(members):
        c = dg.dg_batch_member(b, i)
        N = dg.dg_sizes(c)[0]
        q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        pert = torch.from_numpy(inputs.perturbation((5, N), seed=inputs.TGV_SEED + 100 * rank + i).ravel()).cuda()
        dg.dg_init_tgv(c, q, pert)
        qs.append(q)
        dts.append(dg.dg_stable_dt(c, q, CFL))
        nodes.append(N)
    dg.dg_batch_autotune(b, qs, dts)
    updates_per_step = 3 * sum(nodes)

    dg.dg_batch_rk3_step(b, qs, dts, args.warmup, 0, stream)
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dg.dg_batch_rk3_step(b, qs, dts, args.steps, 0, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    value = updates_per_step * args.steps * ws / (ms / 1e3)

    # the same members advanced one at a time (dg_rk3_step per member), for comparison
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_cmp = max(1, args.steps // 4)
    u0.record(stream)
    for _ in range(n_cmp):
        for i, q in enumerate(qs):
            dg.dg_rk3_step(dg.dg_batch_member(b, i), q, dts[i], 1, None, stream)
    u1.record(stream)
    torch.cuda.synchronize()
    one_at_a_time = updates_per_step * n_cmp / (u0.elapsed_time(u1) / 1e3)

    # end to end: pinned host states copied in and out around every batched step
    host = [torch.empty(5 * n, dtype=torch.float64, pin_memory=True) for n in nodes]
    for h, q in zip(host, qs):
        h.copy_(q)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        for h, q in zip(host, qs):
            q.copy_(h, non_blocking=True)
        dg.dg_batch_rk3_step(b, qs, dts, 1, 0, stream)
        for h, q in zip(host, qs):
            h.copy_(q, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    bytes_state = sum(5 * 8 * n for n in nodes)
    e2e = {"value": updates_per_step * args.e2e_steps * ws / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state,
           "call": "dg_batch_rk3_step (pinned host states copied in and out every step)"}
    peak, peak_kind = peaks()
    achieved = STEP_BYTES_PER_NODE * sum(nodes) * args.steps / (ms / 1e3) / 1e9
    groups = len({P for _, P, _ in members})
    dg.dg_batch_destroy(b)
    if rank == 0:
        line = {"metric": "DOF-stage updates/s (12 batched TGV instances per RK3 step)", "value": value,
                "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 operator / f64 state",
                "data": "synthetic (closed-form TGV fields + seeded 1e-6 perturbations)",
                "config": {"workload": "12 independent TGV instances, (K, P, Re) drawn with seed 12 from "
                                       "{8,12,16} x {3,6} x {30,200,1600}, Mach 0.1, one batch, graph replay",
                           "members": [f"{K}^3/P{P}/Re{int(Re)}" for K, P, Re in members], "nodes": sum(nodes),
                           "l2": "working set ~260 B/node x 2.9M nodes > 129 MB L2 (no flush)",
                           "parallelism": f"replicas x{ws}"},
                "one_at_a_time": {"value": one_at_a_time, "unit": UNIT, "call": "dg_rk3_step per member"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_kind,
                             "kernel": "whole batched step (all launches)", "traffic": None},
                "e2e": e2e, "gpu_launches": 6 * groups * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, ws = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, rank, ws)
    elif args.workload == "batched":
        rc = run_batched(args, rank, ws)
    else:
        rc = run_ours(args, rank, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
