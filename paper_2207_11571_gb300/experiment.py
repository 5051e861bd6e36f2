"""Algorithm 1 of arXiv 2207.11571 end to end on one GPU, through the C ABI.

1. High-order evolution (P_HO) of the Taylor-Green vortex to the start of the training
   window, then Algorithm 1's first loop over the window: filter (G q_HO^n), one
   uncorrected low-order step, the matching high-order steps, filter again, and the pair
   (G q_HO^n, (G q_HO^{n+1} - q_NN^{n+1}) / dt) of every element (dg_project,
   dg_rk3_step, dg_make_pairs).
2. Training of the forcing network on the pairs (nn_compute_scalers, nn_train_step),
   shuffled mini-batches.
3. Evaluation window (from the end of the training window, or replayed from its start):
   the high-order run continues as the reference; from its filtered state, the corrected
   low-order run (forcing in every RK stage, or after each step with --forcing post) and
   plain runs at P = P_LO .. 6 advance in
   lockstep.  Every sample interval
   records -dKE/dt and KE (dg_diagnostics) and the L-inf momentum error against the
   filtered reference (Eq. 9).  Each run's advance is timed with CUDA events.

Outputs a JSON summary: per run the relative L2 error of the dissipation history
against the reference, the mean e_n, and the wall time; plus the corrected-vs-plain
speed-up at equal dissipation error (log-log interpolation over the plain orders).

    python -m paper_2207_11571_gb300.experiment --out result.json [--K 16 --Re 1600 ...]
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import dg, inputs, nn


def make_ctx(K, P, args, les=False, precision=None, split=False):
    prec = dg.DG_PREC_FP32 if precision is None else precision
    return dg.dg_create(K, P, args.Re, args.Mach, args.Pr, int(les), precision=prec, volume_flux=int(split))


def new_state(ctx):
    return torch.empty(5 * dg.dg_sizes(ctx)[0], dtype=torch.float64, device="cuda")


class Run:
    """One solver run advancing in lockstep with the others, with its own timer.  A run
    whose state turns non-finite is marked diverged and stops advancing.

    With `guard`, a corrected run falls back to the uncorrected solver (forcing off for
    the rest of the run) at the first sample where its kinetic energy grows: the decaying
    Taylor-Green flow has dKE/dt < 0, so growth means the network injects energy."""

    def __init__(self, name, P, ctx, q, dt_max, net=None, guard=False):
        self.name, self.P, self.ctx, self.q, self.net = name, P, ctx, q, net
        self.dt_max = dt_max
        self.guard = guard
        self.ms = 0.0
        self.steps = 0
        self.t = []
        self.dke = []
        self.ke = []
        self.einf = []
        self.diverged_at = None
        self.fallback_at = None
        self.active_time = 0.0   # time units advanced with the network forcing on

    def advance(self, interval):
        if self.diverged_at is not None:
            return
        n = max(1, math.ceil(interval / self.dt_max - 1e-9))
        dt = interval / n
        if self.net is not None:
            self.active_time += interval
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dg.dg_rk3_step(self.ctx, self.q, dt, n, forcing=self.net)
        b.record()
        b.synchronize()
        self.ms += a.elapsed_time(b)
        self.steps += n

    def sample(self, t, qref=None):
        if self.diverged_at is not None:
            return None
        try:
            d = dg.dg_diagnostics(self.ctx, self.q, q_ref=qref, forcing=self.net)
        except dg.DGError as e:
            if e.status != dg.DG_ERR_NONFINITE:
                raise
            self.diverged_at = t
            return None
        self.t.append(t)
        self.dke.append(d["dke_dt"])
        self.ke.append(d["ke"])
        self.einf.append(max(d["e_inf"]) if qref is not None else None)
        if self.guard and self.net is not None and d["dke_dt"] > 0:
            self.net = None
            self.fallback_at = t
        return d


def stable_dt(ctx, q, cfl):
    return dg.dg_stable_dt(ctx, q, cfl)


def generate_pairs(args, ctx_hi, q_hi, ctx_lo, dt_lo, ratio, n_steps, first_var, n_vars):
    """Training pairs of Algorithm 1 (Sec. 2.1): per low-order step of the window, the
    input is the filtered high-order state at the step start and the target the forcing
    that carries the uncorrected low-order step from there onto the filtered high-order
    state at the step end, divided by the step.  Returns device tensors X, Y (n_steps K^3
    rows)."""
    nodes_lo, elems = dg.dg_sizes(ctx_lo)
    feat = n_vars * (args.P_lo + 1) ** 3
    X = torch.empty((n_steps * elems, feat), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    qbar = new_state(ctx_lo)
    qnn = new_state(ctx_lo)
    qbar1 = new_state(ctx_lo)
    dt_hi = dt_lo / ratio
    for n in range(n_steps):
        dg.dg_project(ctx_hi, ctx_lo, q_hi, qbar)                 # filtered state, step start
        qnn.copy_(qbar)
        dg.dg_rk3_step(ctx_lo, qnn, dt_lo, 1)                     # low order, no forcing
        dg.dg_rk3_step(ctx_hi, q_hi, dt_hi, ratio)               # high order over the same dt
        dg.dg_project(ctx_hi, ctx_lo, q_hi, qbar1)                # filtered state, step end
        dg.dg_make_pairs(ctx_lo, qbar, qnn, qbar1, dt_lo, first_var, n_vars,
                         X[n * elems:(n + 1) * elems], Y[n * elems:(n + 1) * elems])
    return X, Y


def train(args, X, Y, first_var, n_vars):
    """Trains on the pairs.  With --init_net the network (weights and scalers) starts from a
    saved one trained at another time window or Re, the paper's transfer learning
    (retraining from earlier weights needs far fewer epochs); otherwise from seeded
    He-uniform weights and the pairs' scalers."""
    feat = X.shape[1]
    dims = [feat] + [args.width] * args.hidden + [feat]
    if args.init_net:
        net = nn.nn_load(args.init_net, args.batch)
        d = nn.nn_get_desc(net)
        if (d.n_in, d.n_out, d.first_var, d.n_vars) != (feat, feat, first_var, n_vars):
            raise ValueError("--init_net does not match the features of this run")
    else:
        net = nn.nn_create(feat, feat, args.width, args.hidden, first_var, n_vars, args.batch,
                           inputs.uniform_draws(dims, args.seed))
        nn.nn_compute_scalers(net, X, Y)
    t0 = time.perf_counter()
    losses = run_epochs(args, net, X, Y, args.epochs, args.seed)
    return net, losses, time.perf_counter() - t0


def run_epochs(args, net, X, Y, epochs, seed):
    """Shuffled mini-batch epochs of nn_train_step; returns the last batch's loss per epoch."""
    rows = X.shape[0]
    losses = []
    for epoch in range(epochs):
        perm = torch.from_numpy(inputs.epoch_permutation(rows, seed, epoch)).cuda()
        ep = []
        for b0 in range(0, rows - args.batch + 1, args.batch):
            ep.append(nn.nn_train_step(net, X, Y, perm[b0:b0 + args.batch], lr=args.lr,
                                       want_loss=(b0 + args.batch > rows - args.batch)))
        losses.append(ep[-1])
    torch.cuda.synchronize()
    return losses


def retrain(args, run, net, ctx_hi, ctx_lo, dt_lo, ratio, first_var, n_vars, seed):
    """Train-advance-retrain (the extension the paper proposes as future work): a short
    high-order burst restarted from the corrected low-order state (prolonged to P_HO, the
    exact embedding), Algorithm 1's pairs over it, and more epochs of the same network from
    its current weights and scalers.  Returns (seconds, losses)."""
    t0 = time.perf_counter()
    q_burst = new_state(ctx_hi)
    dg.dg_prolong(ctx_lo, ctx_hi, run.q, q_burst)
    n = max(1, math.ceil(args.retrain_window / dt_lo - 1e-9))
    X, Y = generate_pairs(args, ctx_hi, q_burst, ctx_lo, dt_lo, ratio, n, first_var, n_vars)
    losses = run_epochs(args, net, X, Y, args.retrain_epochs, seed)
    del X, Y, q_burst
    return time.perf_counter() - t0, losses


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_errors(run, ref_t, ref_dke, ref_ke, bar_ke):
    """Error histories of one run over the sampled times (infinite if it diverged):
    dke: -dKE/dt from the operator against the high-order run's (the benchmark metric);
    ke: KE(t) against the high-order run's; dke_filtered: centred differences of KE(t)
    against those of the filtered high-order field (what the forcing is trained on)."""
    if run.diverged_at is not None:
        return {"dke": float("inf"), "ke": float("inf"), "dke_filtered": float("inf"), "einf": float("inf")}
    t = np.asarray(ref_t)
    en = [e for e in run.einf if e is not None]
    return {"dke": rel_l2(-np.asarray(run.dke), -np.asarray(ref_dke)),
            "ke": rel_l2(run.ke, ref_ke),
            "dke_filtered": rel_l2(-np.gradient(np.asarray(run.ke), t), -np.gradient(np.asarray(bar_ke), t)),
            # e_n of Eq. 9: largest momentum difference from the high-order run filtered to
            # the run's own order, averaged over the samples
            "einf": float(np.mean(en)) if en else float("nan")}


def speedup_at_equal_error(corr, plain, key):
    """Cost of the plain orders at the corrected run's error, over the corrected run's cost,
    and how that cost was found:
      "interpolated": the plain runs' error falls as their cost grows; their error/cost
          curve is interpolated log-log at the corrected error;
      "lower_bound": the corrected error is below every plain error (no extrapolation:
          the cost of the most accurate plain run);
      "cheapest_plain_is_more_accurate": the corrected error is above every plain error;
          the cost of the cheapest plain run, which is already more accurate (the speed-up
          at equal error is at most this);
      "pareto": the plain errors do not fall with cost (e.g. saturated errors); the cost of
          the cheapest plain run at least as accurate as the corrected one."""
    pts = sorted([(r["ms"], r["errors"][key]) for r in plain if math.isfinite(r["errors"][key])])
    e = corr["errors"][key]
    if not pts or not math.isfinite(e):
        return None, None
    costs = [p[0] for p in pts]
    errs = [p[1] for p in pts]
    if e > max(errs):
        return min(costs) / corr["ms"], "cheapest_plain_is_more_accurate"
    if all(b < a for a, b in zip(errs, errs[1:])):
        if e < errs[-1]:
            return costs[-1] / corr["ms"], "lower_bound"
        le = np.log(errs[::-1])
        lc = np.log(costs[::-1])
        return float(math.exp(np.interp(math.log(e), le, lc))) / corr["ms"], "interpolated"
    ok = [c for c, er in pts if er <= e]
    if not ok:
        return max(costs) / corr["ms"], "lower_bound"
    return min(ok) / corr["ms"], "pareto"


def parse(argv=None):
    ap = argparse.ArgumentParser(description="Algorithm 1: pairs, training, corrected vs plain runs")
    ap.add_argument("--K", type=int, default=16)
    ap.add_argument("--P_hi", type=int, default=8)
    ap.add_argument("--P_lo", type=int, default=3)
    ap.add_argument("--plain", type=str, default="3,4,5,6")
    ap.add_argument("--Re", type=float, default=1600.0)
    ap.add_argument("--Mach", type=float, default=0.1)
    ap.add_argument("--Pr", type=float, default=0.71)
    ap.add_argument("--les_hi", action="store_true")
    ap.add_argument("--les_lo", action="store_true")
    ap.add_argument("--split_lo", action="store_true",
                    help="low-order runs with the kinetic-energy-preserving split-form volume term")
    ap.add_argument("--split_hi", action="store_true", help="the same for the high-order run")
    ap.add_argument("--cfl", type=float, default=0.7)
    ap.add_argument("--t_train", type=float, default=4.0)
    ap.add_argument("--t_train_end", type=float, default=5.0)
    ap.add_argument("--window_precision", choices=["fp32", "fp64"], default="fp64")
    ap.add_argument("--t_end", type=float, default=14.0)
    ap.add_argument("--sample", type=float, default=0.1)
    ap.add_argument("--no_guard", action="store_true",
                    help="keep the forcing on even when the corrected flow gains kinetic energy")
    ap.add_argument("--eval_start", choices=["window_end", "window_start"], default="window_end",
                    help="start of the corrected and plain runs: after the training window "
                         "(extrapolation) or at its start (as in the paper's Table 1 cases)")
    ap.add_argument("--io", choices=["all", "momentum"], default="all")
    ap.add_argument("--forcing", choices=["stage", "post"], default="stage",
                    help="corrected run: s in every RK stage (Eq. 4) or added after the "
                         "uncorrected step (Algorithm 1, q += dt s(q^n))")
    ap.add_argument("--width", type=int, default=512)
    ap.add_argument("--hidden", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=2207)
    ap.add_argument("--retrain_every", type=float, default=0.0,
                    help="corrected run: every this many time units, retrain on a high-order burst "
                         "restarted from its own state (0: off)")
    ap.add_argument("--retrain_window", type=float, default=0.15, help="length of each high-order burst")
    ap.add_argument("--retrain_epochs", type=int, default=10, help="epochs of each retraining")
    ap.add_argument("--init_net", type=str, default="", help="start training from this saved network")
    ap.add_argument("--save_net", type=str, default="", help="save the trained network here")
    ap.add_argument("--out", type=str, default="experiment.json")
    return ap.parse_args(argv)


def run(args):
    """Runs the three phases; returns the summary dict (also written to args.out if set)."""
    first_var, n_vars = (1, 3) if args.io == "momentum" else (0, 5)
    dg.lib()
    K = args.K
    wall0 = time.perf_counter()

    # 1. high-order evolution to the training window
    ctx_hi = make_ctx(K, args.P_hi, args, args.les_hi, split=args.split_hi)
    q_hi = new_state(ctx_hi)
    nodes_hi = dg.dg_sizes(ctx_hi)[0]
    dg.dg_init_tgv(ctx_hi, q_hi, torch.from_numpy(inputs.perturbation((5, nodes_hi)).ravel()).cuda())
    dt_hi = stable_dt(ctx_hi, q_hi, args.cfl)
    t = 0.0
    while t < args.t_train - 1e-12:
        interval = min(1.0, args.t_train - t)
        n = max(1, math.ceil(interval / dt_hi))
        dg.dg_rk3_step(ctx_hi, q_hi, interval / n, n)
        t += interval
        try:
            dt_hi = stable_dt(ctx_hi, q_hi, args.cfl)
        except dg.DGError as e:
            raise RuntimeError(f"the P={args.P_hi} run failed before t={t:g}: {e}") from e
    torch.cuda.synchronize()
    t_ho_initial = time.perf_counter() - wall0

    # 2. pairs over the training window (Algorithm 1, first loop)
    ctx_lo = make_ctx(K, args.P_lo, args, args.les_lo, split=args.split_lo)
    qtmp = new_state(ctx_lo)
    dg.dg_project(ctx_hi, ctx_lo, q_hi, qtmp)
    dt_lo_cfl = stable_dt(ctx_lo, qtmp, args.cfl)
    window = args.t_train_end - args.t_train
    n_pairs = max(1, math.ceil(window / dt_lo_cfl))
    dt_lo = window / n_pairs
    ratio = max(1, math.ceil(dt_lo / dt_hi - 1e-9))
    q_hi_start = q_hi.clone() if args.eval_start == "window_start" else None
    t1 = time.perf_counter()
    if args.window_precision == "fp64":   # the training window in an FP64 operator
        w_hi = make_ctx(K, args.P_hi, args, args.les_hi, dg.DG_PREC_FP64, split=args.split_hi)
        w_lo = make_ctx(K, args.P_lo, args, args.les_lo, dg.DG_PREC_FP64, split=args.split_lo)
    else:
        w_hi, w_lo = ctx_hi, ctx_lo
    X, Y = generate_pairs(args, w_hi, q_hi, w_lo, dt_lo, ratio, n_pairs, first_var, n_vars)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t1
    if args.window_precision == "fp64":
        dg.dg_destroy(w_hi)
        dg.dg_destroy(w_lo)

    # 3. training
    net, losses, t_train = train(args, X, Y, first_var, n_vars)
    del X, Y
    torch.cuda.empty_cache()

    # 4. evaluation window: reference HO, corrected LO, plain LO at several orders
    t0 = args.t_train_end
    if q_hi_start is not None:            # replay the window: the runs start where training did
        q_hi.copy_(q_hi_start)
        del q_hi_start
        t0 = args.t_train
    ref = Run(f"P{args.P_hi} reference", args.P_hi, ctx_hi, q_hi, stable_dt(ctx_hi, q_hi, args.cfl))
    runs = []
    q_c = new_state(ctx_lo)
    dg.dg_project(ctx_hi, ctx_lo, q_hi, q_c)
    dg.dg_set_forcing_mode(ctx_lo, dg.DG_FORCING_POST if args.forcing == "post" else dg.DG_FORCING_STAGE)
    runs.append(Run(f"P{args.P_lo}+NN", args.P_lo, ctx_lo, q_c, stable_dt(ctx_lo, q_c, args.cfl), net=net,
                    guard=not args.no_guard))
    plain_ctx = {}
    for P in [int(p) for p in args.plain.split(",")]:
        c = make_ctx(K, P, args, args.les_lo, split=args.split_lo)
        plain_ctx[P] = c
        qp = new_state(c)
        dg.dg_project(ctx_hi, c, q_hi, qp)
        runs.append(Run(f"P{P}", P, c, qp, stable_dt(c, qp, args.cfl)))
    # the high-order run filtered to every order present, for e_n (Eq. 9): each low-order
    # run is compared with the high-order solution filtered to its own order
    qbar = new_state(ctx_lo)
    qbars = {args.P_lo: (ctx_lo, qbar)}
    for P, c in plain_ctx.items():
        if P != args.P_lo:
            qbars[P] = (c, new_state(c))

    def filtered_refs():
        for c, qb in qbars.values():
            dg.dg_project(ctx_hi, c, q_hi, qb)

    bar_ke = []
    ref.sample(t0)
    filtered_refs()
    bar_ke.append(dg.dg_diagnostics(ctx_lo, qbar)["ke"])
    for r in runs:
        r.sample(t0, qbars[r.P][1])
    n_samples = round((args.t_end - t0) / args.sample)
    retrains = []
    every = round(args.retrain_every / args.sample) if args.retrain_every > 0 else 0
    for j in range(1, n_samples + 1):
        tj = t0 + j * args.sample
        ref.advance(args.sample)
        ref.sample(tj)
        filtered_refs()
        bar_ke.append(dg.dg_diagnostics(ctx_lo, qbar)["ke"])
        for r in runs:
            r.advance(args.sample)
            r.sample(tj, qbars[r.P][1])
        corr_run = runs[0]
        if every and j % every == 0 and j < n_samples and corr_run.diverged_at is None:
            secs, rl = retrain(args, corr_run, net, ctx_hi, ctx_lo, dt_lo, ratio, first_var, n_vars,
                               args.seed + 1000 + j)
            corr_run.ms += 1e3 * secs          # the burst and the training are part of its cost
            corr_run.net = net                 # forcing back on after a fallback
            retrains.append({"t": tj, "seconds": secs, "loss_first": rl[0], "loss_last": rl[-1]})

    out = {"config": vars(args), "dt_lo": dt_lo, "ratio_hi_per_lo": ratio, "n_pairs": n_pairs,
           "pairs_rows": n_pairs * K ** 3, "train_loss": losses, "train_seconds": t_train,
           "pairs_seconds": t_pairs, "ho_to_window_seconds": t_ho_initial,
           "reference": {"name": ref.name, "ms": ref.ms, "steps": ref.steps}, "runs": [],
           "retrains": retrains}
    for r in runs:
        rec = {"name": r.name, "P": r.P, "ms": r.ms, "steps": r.steps,
               "errors": run_errors(r, ref.t, ref.dke, ref.ke, bar_ke),
               "diverged_at": r.diverged_at, "fallback_at": r.fallback_at}
        rec["dke_error"] = rec["errors"]["dke"]
        if r is runs[0]:
            # the share of the evaluation horizon over which the network forcing was on (the
            # rest ran as the uncorrected solver after the guard's fallback)
            rec["forcing_active_fraction"] = r.active_time / (args.t_end - t0)
        rec["einf_mean"] = rec["errors"]["einf"]
        out["runs"].append(rec)
    corr, plain = out["runs"][0], out["runs"][1:]
    out["speedup_vs_plain_at_equal_error"] = {}
    for key in ("dke", "ke", "dke_filtered", "einf"):
        sp, kind = speedup_at_equal_error(corr, plain, key)
        out["speedup_vs_plain_at_equal_error"][key] = {"speedup": sp, "kind": kind,
                                                       "forcing_active_fraction": corr["forcing_active_fraction"]}
    out["forcing_active_fraction"] = corr["forcing_active_fraction"]
    p6 = [r for r in plain if r["P"] == 6]
    if p6:
        out["speedup_vs_P6"] = p6[0]["ms"] / corr["ms"]
        out["corrected_error_over_P6_error"] = {k: corr["errors"][k] / p6[0]["errors"][k]
                                                for k in corr["errors"]}
    out["history"] = {"t": ref.t, "ref_dke": ref.dke, "ref_ke": ref.ke, "filtered_ke": bar_ke,
                      **{r.name + "_ke": r.ke for r in runs},
                      **{r.name + "_dke": r.dke for r in runs},
                      **{r.name + "_einf": r.einf for r in runs if r.P == args.P_lo}}
    out["total_seconds"] = time.perf_counter() - wall0
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    if args.save_net:
        nn.nn_save(net, args.save_net)
    nn.nn_destroy(net)
    for c in list(plain_ctx.values()) + [ctx_lo, ctx_hi]:
        dg.dg_destroy(c)
    return out


def main(argv=None):
    out = run(parse(argv))
    summary = {k: out[k] for k in ("speedup_vs_plain_at_equal_error", "n_pairs", "train_seconds")}
    summary["runs"] = [(r["name"], {k: round(v, 4) for k, v in r["errors"].items()}, round(r["ms"], 1),
                        r["diverged_at"], r["fallback_at"]) for r in out["runs"]]
    summary["speedup_vs_P6"] = out.get("speedup_vs_P6")
    summary["forcing_active_fraction"] = out["forcing_active_fraction"]
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
