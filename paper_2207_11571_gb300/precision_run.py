"""FP32 operator against FP64 operator over a long Taylor-Green run (Sec. 3.1), on one GPU.

Both operators advance the same seeded initial state (Eq. 11 field plus the 1e-6
perturbation) with the same CFL-limited RK3 steps; at every sample time both record KE
and -dKE/dt (dg_diagnostics: FP64 reductions, -dKE/dt from each context's own operator).
The FP64 GPU operator matches the FP64 oracle to 1e-12 per operator call and 1e-10
after 100 steps, so over runs the oracle cannot finish it stands in for the oracle.

Reported: the largest relative KE difference over the samples, the relative L2 and
largest relative difference of the dissipation history (the benchmark's error measure),
the peak dissipation and its time for both, the relative L2 difference of the momentum
fields at the end (pointwise divergence of the two runs once the flow turns turbulent),
and the device time per RK3 step of each operator.

    python -m paper_2207_11571_gb300.precision_run --K 32 --P 3 --t_end 10 --out r.json

--split runs both operators with the kinetic-energy-preserving split-form volume term
(the standard form without a closure is not stable on the under-resolved Re 1600 meshes
past the dissipation peak).  --max_seconds bounds the wall time of the time loop; the run then stops at the last
completed sample time (reported as t_reached).  A run whose state turns non-finite
(the standard-form operator on an under-resolved mesh without a closure) stops there:
diverged_at gives the first sample time at which each diverged run was non-finite, and
the comparison covers the samples before it.
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import dg, inputs


def run(K, P, Re=1600.0, Mach=0.1, Pr=0.71, les=False, cfl=0.7, t_end=10.0, sample=0.1, max_seconds=0.0,
        split=False):
    precs = {"fp32": dg.DG_PREC_FP32, "fp64": dg.DG_PREC_FP64}
    ctx = {k: dg.dg_create(K, P, Re, Mach, Pr, int(les), precision=p, volume_flux=int(split))
           for k, p in precs.items()}
    try:
        N = dg.dg_sizes(ctx["fp64"])[0]
        pert = torch.from_numpy(inputs.perturbation((5, N)).ravel()).cuda()
        q = {}
        for k, c in ctx.items():
            q[k] = torch.empty(5 * N, dtype=torch.float64, device="cuda")
            dg.dg_init_tgv(c, q[k], pert)
        del pert
        dt0 = dg.dg_stable_dt(ctx["fp64"], q["fp64"], cfl)
        tuned = {k: dg.dg_autotune(c, q[k], dt0)[0] for k, c in ctx.items()}
        stream = torch.cuda.current_stream()
        ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in ctx}
        ms = {k: 0.0 for k in ctx}
        steps = 0
        hist = {"t": [], "fp32": {"ke": [], "eps": []}, "fp64": {"ke": [], "eps": []}}

        diverged = {}

        def record(t):
            hist["t"].append(t)
            for k, c in ctx.items():
                d = dg.dg_diagnostics(c, q[k], raise_nonfinite=False)
                if d["nonfinite"]:
                    diverged.setdefault(k, t)
                hist[k]["ke"].append(d["ke"])
                hist[k]["eps"].append(-d["dke_dt"])

        t = 0.0
        record(t)
        wall0 = time.time()
        while t < t_end - 1e-12 and not diverged:
            if max_seconds > 0 and time.time() - wall0 > max_seconds:
                break
            dt = dg.dg_stable_dt(ctx["fp64"], q["fp64"], cfl)
            t_next = min(t + sample, t_end)
            n = max(1, math.ceil((t_next - t) / dt - 1e-9))
            h = (t_next - t) / n
            for k, c in ctx.items():
                a, b = ev[k]
                a.record(stream)
                dg.dg_rk3_step(c, q[k], h, n, None, stream)
                b.record(stream)
            torch.cuda.synchronize()
            for k in ctx:
                ms[k] += ev[k][0].elapsed_time(ev[k][1])
            steps += n
            t = t_next
            record(t)

        N3 = q["fp64"].view(5, N)[1:4]
        mom_diff = float(torch.linalg.vector_norm(q["fp32"].view(5, N)[1:4] - N3) / torch.linalg.vector_norm(N3))
    finally:
        for c in ctx.values():
            dg.dg_destroy(c)

    # compare the samples where both runs are finite
    m = len(hist["t"]) - (1 if diverged else 0)
    ke32, ke64 = np.array(hist["fp32"]["ke"][:m]), np.array(hist["fp64"]["ke"][:m])
    e32, e64 = np.array(hist["fp32"]["eps"][:m]), np.array(hist["fp64"]["eps"][:m])
    i32, i64 = int(np.argmax(e32)), int(np.argmax(e64))
    return {
        "mesh": f"{K}^3/P{P}", "nodes": N, "Re": Re, "Mach": Mach, "les": les, "split_form": split, "cfl": cfl,
        "t_end": t_end, "t_reached": hist["t"][m - 1], "diverged_at": diverged or None, "steps": steps,
        "elems_per_block": tuned,
        "ke_rel_max": float(np.max(np.abs(ke32 - ke64) / ke64)),
        "dissipation_rel_l2": float(np.linalg.norm(e32 - e64) / np.linalg.norm(e64)),
        "dissipation_rel_max": float(np.max(np.abs(e32 - e64)) / np.max(np.abs(e64))),
        "peak_dissipation": {"fp32": [float(e32[i32]), hist["t"][i32]], "fp64": [float(e64[i64]), hist["t"][i64]]},
        "momentum_rel_l2_at_end": None if diverged else mom_diff,
        "ms_per_step": {k: (ms[k] / steps if steps else None) for k in ms},
        "history": hist,
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--K", type=int, default=32)
    ap.add_argument("--P", type=int, default=3)
    ap.add_argument("--Re", type=float, default=1600.0)
    ap.add_argument("--Mach", type=float, default=0.1)
    ap.add_argument("--Pr", type=float, default=0.71)
    ap.add_argument("--les", action="store_true")
    ap.add_argument("--split", action="store_true",
                    help="kinetic-energy-preserving split-form volume term (dg_opts.volume_flux = 1)")
    ap.add_argument("--cfl", type=float, default=0.7)
    ap.add_argument("--t_end", type=float, default=10.0)
    ap.add_argument("--sample", type=float, default=0.1)
    ap.add_argument("--max_seconds", type=float, default=0.0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    dg.lib()
    r = run(a.K, a.P, a.Re, a.Mach, a.Pr, a.les, a.cfl, a.t_end, a.sample, a.max_seconds, a.split)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)
    print(json.dumps({k: v for k, v in r.items() if k != "history"}), flush=True)
    return r


if __name__ == "__main__":
    main()
