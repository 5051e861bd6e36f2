"""Runs a few RK3 steps of one Taylor-Green mesh through the C ABI: the command that
ncu captures for the kernel profiles.

    python -m paper_2207_11571_gb300.profile_case --K 32 --P 3 --steps 2 [--fp64] [--E 8]
"""
import argparse

import torch

from . import dg, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=32)
    ap.add_argument("--P", type=int, default=3)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--les", action="store_true")
    ap.add_argument("--E", type=int, default=0, help="elements per block (0: the default for P)")
    a = ap.parse_args()
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
