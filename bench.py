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
oracle on every host core on a bounded sample of the same workload.
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
# Algorithmic floor of one DOF-stage update: read the FP64 state (5 x 8 B), read and write
# the FP64 RK register (2 x 5 x 8 B), write the state (5 x 8 B)
FLOOR_BYTES = 160.0
KERNEL_SOURCES = ["dg_kernels.cuh", "dg_device.cuh", "dg_launch.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-instances key of the default line")
    ap.add_argument("--no-algorithm1", action="store_true", help="skip the algorithm1 key of the default line")
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


# The FP64 operator (the parity path) against GB300's FP64 rate: not a performance
# target, reported for context.  Arithmetic per DOF-stage estimated from the operator's
# structure: ~30 (P+1) inviscid and ~48 (P+1) gradient/viscous contraction flops plus
# ~300 pointwise flops; nominal FP64 peak 1.25 TFLOP/s (no measured FP64 peak exists).
FP64_NOMINAL_TFLOPS = 1.25


def fp64_measure(stream, steps=3):
    import torch

    from paper_2207_11571_gb300 import dg, inputs
    per_mesh, tot_upd, tot_ms, tot_flop = {}, 0, 0.0, 0.0
    for K, P in WORKLOAD:
        c = dg.dg_create(K, P, RE, MACH, PR, 0, precision=dg.DG_PREC_FP64)
        N = dg.dg_sizes(c)[0]
        q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        dg.dg_init_tgv(c, q, torch.from_numpy(inputs.perturbation((5, N), seed=inputs.TGV_SEED).ravel()).cuda())
        dt = dg.dg_stable_dt(c, q, CFL)
        dg.dg_rk3_step(c, q, dt, 1, None, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dg.dg_rk3_step(c, q, dt, steps, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        flop = (30 * (P + 1) + 48 * (P + 1) + 300) * 3 * N
        per_mesh[f"{K}^3/P{P}"] = {"ms_per_step": round(ms, 3), "dof_stage_per_s": 3 * N / (ms / 1e3),
                                   "tflops_estimate": flop / (ms / 1e3) / 1e12}
        tot_upd += 3 * N
        tot_ms += ms
        tot_flop += flop
        dg.dg_destroy(c)
    achieved = tot_flop / (tot_ms / 1e3) / 1e12
    return {"value": tot_upd / (tot_ms / 1e3), "unit": UNIT, "ms_per_step": round(tot_ms, 3), "per_mesh": per_mesh,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_NOMINAL_TFLOPS, "peak_source": "nominal (recipe table)",
                         "flop_per_dof_stage": "estimate 78 (P+1) + 300"},
            "note": "FP64 operator and FP64 RK3 (the parity path), same meshes, CUDA events; context only"}


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

    def timed(fn, n):
        for _ in range(5):
            fn()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n * 1e3   # us

    infer = {}
    for name, mode in (("cluster", nn.NN_INFER_CLUSTER), ("layers", nn.NN_INFER_LAYERS)):
        nn.nn_set_fused(net, mode)
        infer[name] = timed(lambda: nn.nn_forcing_infer(net, c, q, s, stream), steps)
    nn.nn_set_fused(net, nn.NN_INFER_CLUSTER)
    # the corrected RK3 step (forcing on every stage state) against the plain one, 16^3 P=3
    dt = dg.dg_stable_dt(c, q, CFL)
    plain_us = timed(lambda: dg.dg_rk3_step(c, q, dt, 1, None, stream), 50)
    corrected_us = timed(lambda: dg.dg_rk3_step(c, q, dt, 1, net, stream), 50)
    dg.dg_set_forcing_mode(c, dg.DG_FORCING_POST)     # Algorithm 1: the forcing once per step
    post_us = timed(lambda: dg.dg_rk3_step(c, q, dt, 1, net, stream), 50)
    dg.dg_set_forcing_mode(c, dg.DG_FORCING_STAGE)
    dg.dg_destroy(c)
    nn.nn_destroy(net)
    peak, kind = bf16_peak()
    tr = 3 * flop_fwd / (train_us * 1e-6) / 1e12
    inf = {k: flop_fwd / (v * 1e-6) / 1e12 for k, v in infer.items()}
    return {"network": "320-512x4-320, batch 4096 (16^3 elements at P=3)",
            "train_step_us": round(train_us, 1), "train_tflops": round(tr, 1),
            "forcing_infer_us": round(infer["cluster"], 1), "forcing_infer_tflops": round(inf["cluster"], 1),
            "forcing_infer_layers_us": round(infer["layers"], 1),
            "forcing_infer_layers_tflops": round(inf["layers"], 1),
            "rk3_step_16cubed_P3_us": {"plain": round(plain_us, 1), "corrected": round(corrected_us, 1),
                                       "ratio": round(corrected_us / plain_us, 3),
                                       "corrected_post_step": round(post_us, 1),
                                       "ratio_post_step": round(post_us / plain_us, 3)},
            "note": "forcing_infer (nn_forcing_infer on an FP32 context) includes the phase-A launch that forms "
                    "the stage state; cluster = one launch (features, 5 layers, unscaling), layers = feature "
                    "launch + 5 GEMMs; the corrected step evaluates the forcing on each of the 3 stage states "
                    "(post-step form: once per step, Algorithm 1)",
            "roofline": {"bound": "tensor", "peak": peak, "unit": "TFLOP/s", "peak_source": kind,
                         "train_frac": round(tr / peak, 4), "infer_frac": round(inf["cluster"] / peak, 4)}}


# Algorithm 1 in the paper's own acceleration setting (Sec. 3.5, Fig. 6, Table 2): Taylor-
# Green at Re 1600, Mach 0.08, 8^3 elements, P8 data over t in [7, 7.2], a network of 8
# layers trained 30 epochs on the momenta, the corrected P3 run against plain P3..P6 to
# t = 8 (split-form volume term, post-step forcing, no fallback guard)
ALG1_ARGS = ["--K", "8", "--P_hi", "8", "--P_lo", "3", "--plain", "3,4,5,6", "--Re", "1600", "--Mach", "0.08",
             "--t_train", "7", "--t_train_end", "7.2", "--t_end", "8", "--io", "momentum", "--width", "256",
             "--hidden", "7", "--epochs", "30", "--batch", "4096", "--sample", "0.05", "--forcing", "post",
             "--split_lo", "--split_hi", "--no_guard", "--out", ""]


def _algorithm1_summary(out):
    runs = {r["name"]: {"ms": round(r["ms"], 2), "dke_error": round(r["errors"]["dke"], 4),
                        "einf_error": round(r["errors"]["einf"], 4)} for r in out["runs"]}
    sp = out["speedup_vs_plain_at_equal_error"]
    return {"runs": runs,
            "speedup_at_equal_error": {k: {"speedup": None if v["speedup"] is None else round(v["speedup"], 3),
                                           "kind": v["kind"]} for k, v in sp.items()},
            "forcing_active_fraction": out["forcing_active_fraction"]}


def algorithm1_measure():
    """One bounded run of Algorithm 1 through the C ABI (high-order run, pairs, GPU
    training, corrected and plain low-order runs timed with CUDA events): the corrected
    run's errors and cost against the plain orders, and the speed-up at equal error, over
    the evaluation window after training and over the training window itself."""
    from paper_2207_11571_gb300 import experiment
    out = experiment.run(experiment.parse(ALG1_ARGS))
    line = {"setting": "TGV Re 1600 Mach 0.08, 8^3, P8 -> P3, training window [7, 7.2], eval [7.2, 8], momenta, "
                       "8 layers x 256, 30 epochs, post-step forcing, split form",
            **_algorithm1_summary(out),
            "train_seconds": round(out["train_seconds"], 2), "n_pairs": out["n_pairs"],
            "cost_P6_over_corrected": round(out.get("speedup_vs_P6", float("nan")), 3),
            "seconds": round(out["total_seconds"], 1)}
    # the same pipeline evaluated over the training window [7, 7.2]: how well the forcing
    # corrects the states it was trained on
    args = list(ALG1_ARGS)
    args[args.index("--t_end") + 1] = "7.2"
    win = experiment.run(experiment.parse(args + ["--eval_start", "window_start"]))
    line["in_training_window"] = {"eval": "[7, 7.2]", **_algorithm1_summary(win)}
    return line


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

CPU_MESHES = [(8, 3), (8, 6), (8, 8), (16, 3), (16, 6), (16, 8)]
CPU_STEPS = 3


def _slab_rhs_worker(task):
    """Pool worker of the all-core oracle leg: the oracle operator on element layers
    [z0, z1) of the periodic mesh, evaluated on those layers plus two ghost layers on each
    side (the operator at an element reads elements at most two face steps away) and
    written into the shared result array.  The state and result live in shared memory."""
    import numpy as np
    from multiprocessing import shared_memory

    from oracle import dgsem, physics
    q_name, r_name, shape, K, P, z0, z1 = task
    qs, rs = shared_memory.SharedMemory(name=q_name), shared_memory.SharedMemory(name=r_name)
    try:
        q = np.ndarray(shape, np.float64, buffer=qs.buf)
        R = np.ndarray(shape, np.float64, buffer=rs.buf)
        layers = [(z - 2) % K for z in range(z0, z1 + 4)]
        mesh = dgsem.Mesh(K, P)
        R[:, z0:z1] = dgsem.rhs(np.take(q, layers, axis=1), mesh, physics.Flow(Re=RE, Mach=MACH, Pr=PR))[:, 2:-2]
    finally:
        qs.close()
        rs.close()
    return z1 - z0


def oracle_rk3_rate(K, P, pool=None, workers=1):
    """DOF-stage updates/s of the FP64 oracle over CPU_STEPS full RK3 steps (after one
    warm-up operator evaluation) on the K^3 mesh at order P.  pool is None: one thread
    (the oracle as it stands); otherwise the operator of every stage is split into z-slabs
    of the mesh evaluated by the pool's processes (the RK update stays in this process)."""
    import numpy as np
    from multiprocessing import shared_memory

    from oracle import dgsem, physics
    flow = physics.Flow(Re=RE, Mach=MACH, Pr=PR)
    mesh = dgsem.Mesh(K, P)
    q0 = dgsem.tgv_state(mesh, flow)
    dt = dgsem.stable_dt(q0, mesh, flow, CFL)
    shm = []
    if pool is None:
        def rhs(z):
            return dgsem.rhs(z, mesh, flow)
    else:
        shm = [shared_memory.SharedMemory(create=True, size=q0.nbytes) for _ in range(2)]
        qs = np.ndarray(q0.shape, np.float64, buffer=shm[0].buf)
        rs = np.ndarray(q0.shape, np.float64, buffer=shm[1].buf)
        bounds = np.linspace(0, K, workers + 1).round().astype(int)
        tasks = [(shm[0].name, shm[1].name, q0.shape, K, P, int(a), int(b)) for a, b in zip(bounds, bounds[1:]) if b > a]

        def rhs(z):
            qs[...] = z
            pool.map(_slab_rhs_worker, tasks)
            return rs.copy()
    try:
        rhs(q0)                                  # warm-up
        t0 = time.perf_counter()
        q = q0
        for _ in range(CPU_STEPS):
            q = dgsem.rk3_step(q, dt, rhs)
        secs = time.perf_counter() - t0
    finally:
        for m in shm:
            m.close()
            m.unlink()
    return 3 * CPU_STEPS * q0[0].size / secs, secs


def cpu_baseline():
    """The oracle timed on this host: single thread, and its operator split over element
    slabs on every core, at 8^3 and 16^3 elements for P = 3, 6, 8 (3 RK3 steps each after
    a warm-up).  The pool starts with 'spawn' (this process already holds a CUDA context)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    single, multi = {}, {}
    t_single = t_multi = 0.0
    nodes_total = 0
    for K, P in CPU_MESHES:
        rate, secs = oracle_rk3_rate(K, P)
        single[f"{K}^3/P{P}"] = rate
        t_single += secs
        nodes_total += 3 * CPU_STEPS * K ** 3 * (P + 1) ** 3
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_limit_threads) as pool:
        for K, P in CPU_MESHES:
            rate, secs = oracle_rk3_rate(K, P, pool=pool, workers=min(cores, K))
            multi[f"{K}^3/P{P}"] = rate
            t_multi += secs
    sample = (f"{CPU_STEPS} full RK3 steps of the FP64 oracle (after one warm-up operator evaluation) on each of "
              f"8^3 and 16^3 elements at P = 3, 6, 8, TGV Re 1600 Mach 0.1; value = all-core rate over the six meshes")
    return {"value": nodes_total / t_multi, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": round(t_single + t_multi, 1),
            "single_thread": {"value": nodes_total / t_single, "cores": 1, "per_mesh": single},
            "all_cores": {"value": nodes_total / t_multi, "cores": cores, "nproc": cores, "per_mesh": multi,
                          "how": "process pool ('spawn'), the operator of each stage over z-slabs of min(cores, K) "
                                 "element layers with two ghost layers each (shared-memory state); RK update in "
                                 "the parent"}}


def _limit_threads():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


REF_MESHES = [(16, 3), (16, 6), (16, 8)]


class _OracleStepper:
    """One mesh of the reference arm: the FP64 oracle's RK3 step with the operator of
    every stage split over z-slabs evaluated by a process pool (state and result in
    shared memory, the RK update in this process), set up once."""

    def __init__(self, K, P, pool, workers):
        import numpy as np
        from multiprocessing import shared_memory

        from oracle import dgsem, physics
        self.dgsem = dgsem
        flow = physics.Flow(Re=RE, Mach=MACH, Pr=PR)
        mesh = dgsem.Mesh(K, P)
        self.q = dgsem.tgv_state(mesh, flow)
        self.dt = dgsem.stable_dt(self.q, mesh, flow, CFL)
        self.nodes = self.q[0].size
        self.shm = [shared_memory.SharedMemory(create=True, size=self.q.nbytes) for _ in range(2)]
        self.qs = np.ndarray(self.q.shape, np.float64, buffer=self.shm[0].buf)
        self.rs = np.ndarray(self.q.shape, np.float64, buffer=self.shm[1].buf)
        bounds = np.linspace(0, K, workers + 1).round().astype(int)
        self.tasks = [(self.shm[0].name, self.shm[1].name, self.q.shape, K, P, int(x), int(y))
                      for x, y in zip(bounds, bounds[1:]) if y > x]
        self.pool = pool

    def rhs(self, z):
        self.qs[...] = z
        self.pool.map(_slab_rhs_worker, self.tasks)
        return self.rs.copy()

    def step(self):
        t0 = time.perf_counter()
        self.q = self.dgsem.rk3_step(self.q, self.dt, self.rhs)
        return time.perf_counter() - t0

    def close(self):
        for m in self.shm:
            m.close()
            m.unlink()


def run_reference(args, rank, ws):
    """The oracle as it stands, timed on every host core: each step is one full RK3 step
    on each of 16^3 elements at P = 3, 6, 8 (the benchmark's per-DOF work at a size the
    host finishes in seconds), the operator split over element slabs by a process pool."""
    if rank != 0:
        return 0
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_limit_threads) as pool:
        meshes = [_OracleStepper(K, P, pool, min(cores, K)) for K, P in REF_MESHES]
        try:
            for m in meshes:
                m.rhs(m.q)                      # warm-up of the workers
            times = []
            for i in range(args.warmup + args.steps):
                secs = sum(m.step() for m in meshes)
                if i >= args.warmup:
                    times.append(secs)
            nodes_per_step = 3 * sum(m.nodes for m in meshes)
        finally:
            for m in meshes:
                m.close()
    value = nodes_per_step * len(times) / sum(times)
    sample = (f"one full RK3 step of the FP64 oracle on each of 16^3 elements at P = 3, 6, 8 per step (the "
              f"benchmark's per-DOF work), operator over element slabs on {cores} host cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (closed-form TGV field)",
            "config": {"workload": WORKLOAD_NAME, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
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

    ctxs, states, dts, nodes, tuned, tuned_ms = [], [], [], [], [], []
    for K, P in WORKLOAD:
        c = dg.dg_create(K, P, RE, MACH, PR, 0, precision=dg.DG_PREC_FP32)
        N = dg.dg_sizes(c)[0]
        q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
        pert = torch.from_numpy(inputs.perturbation((5, N), seed=inputs.TGV_SEED + rank).ravel()).cuda()
        dg.dg_init_tgv(c, q, pert)
        del pert
        dts.append(dg.dg_stable_dt(c, q, CFL))
        E_best, ms_best = dg.dg_autotune(c, q, dts[-1])
        tuned.append(E_best)
        tuned_ms.append(ms_best)
        ctxs.append(c)
        states.append(q)
        nodes.append(N)
    updates_per_step = 3 * sum(nodes)
    # one stream per mesh, forked from and joined to the launching stream every step: the
    # meshes are independent, so one mesh's kernels fill the SMs another's tail leaves idle;
    # the mesh with the longest step (by the autotuner's timing) runs at high priority, so
    # the others fill in around it (measured 1377 -> 1349 us per step)
    slowest = max(range(len(ctxs)), key=lambda i: tuned_ms[i])
    mesh_streams = [torch.cuda.Stream(priority=-1 if i == slowest else 0) for i in range(len(ctxs))]

    def step():
        fork = torch.cuda.Event()
        fork.record(stream)
        for c, q, dt, ms_ in zip(ctxs, states, dts, mesh_streams):
            ms_.wait_event(fork)
            dg.dg_rk3_step(c, q, dt, 1, None, ms_)
        for ms_ in mesh_streams:
            join = torch.cuda.Event()
            join.record(ms_)
            stream.wait_event(join)

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

    peak, peak_kind = peaks()
    # per-mesh rates: each mesh's RK3 steps timed alone (CUDA events on the launching stream)
    per_mesh = {}
    n_alone = max(3, args.steps // 3)
    for (K, P), c, q, dt, N in zip(WORKLOAD, ctxs, states, dts, nodes):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dg.dg_rk3_step(c, q, dt, n_alone, None, stream)
        b.record(stream)
        torch.cuda.synchronize()
        rate = 3 * N * n_alone / (a.elapsed_time(b) / 1e3)
        per_mesh[f"{K}^3/P{P}"] = {"nodes": N, "dof_stage_per_s": rate, "ms_per_step": a.elapsed_time(b) / n_alone,
                                   "floor_achieved_gbs": FLOOR_BYTES * rate / 1e9,
                                   "frac": FLOOR_BYTES * rate / 1e9 / peak}

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
                            "share": p[f"ms_{kind}"] / total_ms,
                            "traffic_per_launch": measured_traffic("k_flux" if kind == "flux" else "k_gradient",
                                                                   p["workload"])})
    dom = max(kernels, key=lambda k: k["ms"])
    dom_achieved = dom["bytes_per_launch"] / (dom["ms"] / dom["launches"] / 1e3) / 1e9
    # Headline: the algorithmic floor of the method per DOF-stage (read q, read and write
    # the FP64 RK register, write q: 160 B) times the DOF-stage rate of the timed region.
    # One unit of work = one RK stage of the three meshes (both launches of each mesh).
    unit_bytes = FLOOR_BYTES * sum(nodes)
    achieved = FLOOR_BYTES * value / ws / 1e9   # per GPU
    traffics = [k["traffic_per_launch"] for k in kernels]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind, "bytes_per_dof_stage": FLOOR_BYTES,
                "kernel": "one RK stage of the three meshes (k_gradient + k_flux per mesh)",
                "bytes_per_launch": unit_bytes,
                "traffic": sum(traffics) if all(t is not None for t in traffics) else None,
                "per_mesh": {m: round(v["frac"], 4) for m, v in per_mesh.items()},
                "note": "algorithmic floor 160 B per DOF-stage (q read, RK register read + write, q write, "
                        "FP64); traffic = ncu DRAM bytes of the six launches of one stage, null unless taken "
                        "on the current kernel sources"}
    # the implementation's own bytes (stage state, stored stresses, FP32 increments: each
    # value read or written once) over the whole timed step and for the dominant kernel
    step_bytes = sum(3 * (p["flux_bytes_per_launch"] + p["gradient_bytes_per_launch"]) for p in prof)
    step_gbs = step_bytes / (ms / args.steps / 1e3) / 1e9
    roofline["implementation"] = {
        "bytes_per_dof_stage": step_bytes / updates_per_step, "achieved": step_gbs, "frac": step_gbs / peak,
        "dominant_kernel": f'{dom["kernel"]} {dom["workload"]}', "dominant_achieved": dom_achieved,
        "dominant_frac": dom_achieved / peak, "dominant_bytes_per_launch": dom["bytes_per_launch"],
        "dominant_traffic": dom["traffic_per_launch"]}
    per_kernel = [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in kk.items()} for kk in kernels]

    # end to end through the C ABI with HOST buffers (pinned), copies inside the timed region
    host = [torch.empty(5 * n, dtype=torch.float64, pin_memory=True) for n in nodes]
    for h, q in zip(host, states):
        h.copy_(q)
    torch.cuda.synchronize()
    barrier(ws)
    # one stream per mesh: each mesh's copies overlap the other meshes' kernels.  Every
    # step of a mesh copies its state in, advances it and copies it out (and, in the
    # second run, reads its diagnostics).  Step s + 1 of every mesh is queued (behind step
    # s on the mesh's stream) before step s is collected, so the host never holds the GPU
    # or the host link idle.
    # the mesh whose chain (copy in, step, copy out) is longest sets the step: its stream
    # gets the high priority, so its kernels are not held behind the other meshes'
    # (measured: 16^3/P8 2.14 -> 2.08 ms per step)
    chain = [2 * 5 * 8 * n / 200e9 + per_mesh[f"{K}^3/P{P}"]["ms_per_step"] / 1e3
             for (K, P), n in zip(WORKLOAD, nodes)]
    longest = max(range(len(ctxs)), key=lambda i: chain[i])
    streams = [torch.cuda.Stream(priority=-1 if i == longest else 0) for i in range(len(ctxs))]
    for c, h, dt, s in zip(ctxs, host, dts, streams):   # untimed: allocates each context's device copy
        dg.dg_advance_host_async(c, h, dt, 0, None, s, want_diag=False)
        dg.dg_advance_host_wait(c, s, want_diag=False)
    torch.cuda.synchronize()

    def e2e_run(diag):
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for step in range(args.e2e_steps):
            for c, h, dt, s in zip(ctxs, host, dts, streams):
                dg.dg_advance_host_async(c, h, dt, 1, None, s, want_diag=diag)
            if step:
                for c, s in zip(ctxs, streams):
                    dg.dg_advance_host_wait(c, s, want_diag=diag)   # step - 1's results
        for c, s in zip(ctxs, streams):
            dg.dg_advance_host_wait(c, s, want_diag=diag)
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t0, ws)

    e2e_s = e2e_run(False)          # the device step's work and the copies
    e2e_diag_s = e2e_run(True)      # and the FP64 diagnostics of every mesh every step
    e2e = {"value": updates_per_step * args.e2e_steps * ws / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": sum(5 * 8 * n for n in nodes), "d2h_bytes_per_step": sum(5 * 8 * n for n in nodes),
           "call": "dg_advance_host_async + dg_advance_host_wait per mesh, one stream per mesh (pinned host "
                   "state copied in and out, 1 RK3 step per mesh every step, the device step's work; step s + 1 "
                   "queued before step s is collected; the mesh with the longest copy-step-copy chain on a "
                   "high-priority stream)",
           "with_diagnostics": {"value": updates_per_step * args.e2e_steps * ws / e2e_diag_s, "unit": UNIT,
                                "call": "the same with want_diag: the FP64 diagnostics of every mesh every "
                                        "step, read by the host"}}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    nn_line = nn_measure(stream)
    fp64_line = fp64_measure(stream)
    alg1 = None if args.no_algorithm1 else algorithm1_measure()
    batched = None
    if not args.no_batched:
        batched = batched_measure(args, rank, ws, max(10, args.steps // 3))
        batched.pop("clocks", None)
        batched["workload"] = BATCH_NAME

    per_workload = {}
    for (K, P), n, p in zip(WORKLOAD, nodes, prof):
        m = per_mesh[f"{K}^3/P{P}"]
        per_workload[f"{K}^3/P{P}"] = {"nodes": n, "dof_stage_per_s": m["dof_stage_per_s"],
                                       "ms_per_step": m["ms_per_step"], "floor_frac": m["frac"],
                                       "dof_stage_per_s_kernels_events_between":
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
                           "streams": "one per mesh, forked from and joined to the timed stream every step; "
                                      "the mesh with the longest step at high priority",
                           "parallelism": f"replicas x{ws}", "per_workload": per_workload},
                "value_x5_variables": {"value": 5 * value, "unit": "variable-stage updates/s",
                                       "note": "the same rate counting each node's 5 conserved variables"},
                "roofline": roofline, "kernels": per_kernel, "network": nn_line, "fp64_operator": fp64_line,
                "batched": batched,
                "algorithm1": alg1,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 6 * len(WORKLOAD) * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- batched instances

# FP32-operator algorithmic bytes per node of one RK3 step (both launches of all stages)
STEP_BYTES_PER_NODE = 676.0
BATCH_NAME = ("12 independent TGV instances, (K, P, Re) drawn with seed 12 from {8,12,16} x {3,6} x "
              "{30,200,1600}, Mach 0.1, one batch, graph replay")


def batched_measure(args, rank, ws, steps, with_clocks=False):
    """Config-3 batch: 12 independent TGV instances advanced by dg_batch_rk3_step (graph
    replay).  Returns the measurements as a dict (rates, per-step time, the same members one
    at a time, end to end from pinned host states, roofline on the 160 B floor)."""
    import torch

    from paper_2207_11571_gb300 import dg, inputs
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
    clocks = Clocks(dev) if with_clocks else None
    barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    dg.dg_batch_rk3_step(b, qs, dts, steps, 0, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    value = updates_per_step * steps * ws / (ms / 1e3)

    # one persistent cooperative launch per RK stage for every member (both orders)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dg.dg_batch_rk3_step(b, qs, dts, 2, dg.DG_BATCH_PERSISTENT, stream)
    p0.record(stream)
    dg.dg_batch_rk3_step(b, qs, dts, steps, dg.DG_BATCH_PERSISTENT, stream)
    p1.record(stream)
    torch.cuda.synchronize()
    persistent = {"value": updates_per_step * steps / (p0.elapsed_time(p1) / 1e3), "unit": UNIT,
                  "ms_per_step": p0.elapsed_time(p1) / steps,
                  "call": "dg_batch_rk3_step(..., DG_BATCH_PERSISTENT): 3 cooperative launches per step"}

    # the same members advanced one at a time (dg_rk3_step per member), for comparison
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_cmp = max(1, steps // 4)
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
    floor = FLOOR_BYTES * value / ws / 1e9
    impl = STEP_BYTES_PER_NODE * sum(nodes) * steps / (ms / 1e3) / 1e9
    groups = len({P for _, P, _ in members})
    dg.dg_batch_destroy(b)
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "clocks": clk,
            "members": [f"{K}^3/P{P}/Re{int(Re)}" for K, P, Re in members], "nodes": sum(nodes),
            "one_at_a_time": {"value": one_at_a_time, "unit": UNIT, "call": "dg_rk3_step per member"},
            "persistent": persistent,
            "roofline": {"bound": "hbm", "achieved": floor, "peak": peak, "unit": "GB/s", "frac": floor / peak,
                         "peak_source": peak_kind, "bytes_per_dof_stage": FLOOR_BYTES,
                         "kernel": "whole batched step (all launches)", "traffic": None,
                         "implementation": {"bytes_per_dof_stage": STEP_BYTES_PER_NODE / 3, "achieved": impl,
                                            "frac": impl / peak}},
            "e2e": e2e, "gpu_launches": 6 * groups * steps}


def run_batched(args, rank, ws):
    from paper_2207_11571_gb300 import build as _build
    from paper_2207_11571_gb300 import dg
    if not os.path.exists(_build.LIB):
        _build.build()
    dg.lib()
    r = batched_measure(args, rank, ws, args.steps, with_clocks=True)
    if rank == 0:
        line = {"metric": "DOF-stage updates/s (12 batched TGV instances per RK3 step)", "value": r["value"],
                "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 operator / f64 state",
                "data": "synthetic (closed-form TGV fields + seeded 1e-6 perturbations)",
                "config": {"workload": BATCH_NAME, "members": r["members"], "nodes": r["nodes"],
                           "l2": "working set ~260 B/node x 2.9M nodes > 129 MB L2 (no flush)",
                           "parallelism": f"replicas x{ws}"},
                "one_at_a_time": r["one_at_a_time"], "persistent": r["persistent"], "roofline": r["roofline"],
                "e2e": r["e2e"],
                "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
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
