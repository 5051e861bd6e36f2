"""Runs a few RK3 steps of one Taylor-Green mesh through the C ABI: the command that
ncu captures for the kernel profiles.  With --nn it instead runs a few training steps
and forcing evaluations of the corrected-P3 network (320-512x4-320, batch 4096, on a
16^3 P=3 state).

    python -m paper_2207_11571_gb300.profile_case --K 32 --P 3 --steps 2 [--fp64] [--E 8]
    python -m paper_2207_11571_gb300.profile_case --nn --steps 4
"""
import argparse

import torch

from . import dg, inputs, nn


def network_case(steps):
    feat, width, hidden, batch = 320, 512, 4, 4096
    dims = [feat] + [width] * hidden + [feat]
    net = nn.nn_create(feat, feat, width, hidden, 0, 5, batch, inputs.uniform_draws(dims, 7))
    rows = 4 * batch
    X = torch.from_numpy(inputs.normal((rows, feat), 8).astype("float32")).cuda()
    Y = torch.from_numpy(inputs.normal((rows, feat), 9).astype("float32")).cuda()
    nn.nn_compute_scalers(net, X, Y)
    perm = torch.from_numpy(inputs.epoch_permutation(rows, 7, 0)).cuda()
    loss = None
    for i in range(steps):
        j = (i % 4) * batch
        loss = nn.nn_train_step(net, X, Y, perm[j:j + batch], want_loss=(i == steps - 1))
    c = dg.dg_create(16, 3, 1600.0, 0.1, 0.71, 0, precision=dg.DG_PREC_FP32)
    N = dg.dg_sizes(c)[0]
    q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(c, q)
    s = torch.empty(5 * N, dtype=torch.float32, device="cuda")
    for i in range(steps):
        nn.nn_forcing_infer(net, c, q, s)
    torch.cuda.synchronize()
    print(f"network steps={steps} loss={loss:.6f} forcing_norm={float(s.norm()):.6e}")
    dg.dg_destroy(c)
    nn.nn_destroy(net)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=32)
    ap.add_argument("--P", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--les", action="store_true")
    ap.add_argument("--E", type=int, default=0, help="elements per block (0: the default for P)")
    ap.add_argument("--nn", action="store_true", help="profile the network instead of the operator")
    a = ap.parse_args()
    if a.nn:
        network_case(a.steps)
        return
    c = dg.dg_create(a.K, a.P, 1600.0, 0.1, 0.71, int(a.les),
                     precision=dg.DG_PREC_FP64 if a.fp64 else dg.DG_PREC_FP32, elems_per_block=a.E)
    N = dg.dg_sizes(c)[0]
    q = torch.empty(5 * N, dtype=torch.float64, device="cuda")
    dg.dg_init_tgv(c, q, torch.from_numpy(inputs.perturbation((5, N)).ravel()).cuda())
    dt = dg.dg_stable_dt(c, q, 0.7)
    dg.dg_rk3_step(c, q, dt, a.steps)
    d = dg.dg_diagnostics(c, q)
    torch.cuda.synchronize()
    print(f"K={a.K} P={a.P} nodes={N} steps={a.steps} ke={d['ke']:.12f} mass={d['mass']:.12f}")
    dg.dg_destroy(c)


if __name__ == "__main__":
    main()
