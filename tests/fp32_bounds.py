"""Bounds of the FP32 operator's error against the FP64 oracle, per parity case.

The FP32 operator rounds the fluxes (~6e-8 relative), the derivative matrix amplifies
that by |D| ~ P^2, and in the energy equation div(v (rho e + p)) cancels
rho e + p ~ 250 at Mach 0.1 down to an O(1) divergence.  Each case's bound is about
three times the error measured on GB300 for that case (relative L2 per variable group:
momenta, energy; the density equation of the Taylor-Green flow is near zero and is
bounded against the momentum scale), so that a lost or mis-rounded FP32 term of
relative size well above the rounding level fails the case.

check() appends the measured errors to the JSON-lines file named by DGNN_ERROR_LOG
(nothing is written when it is unset), the record the bounds come from.
"""
import json
import os

import numpy as np

# label -> (momenta, energy, density against the momentum norm): about 3x the error
# measured on GB300 for the case (measured values beside each entry).  Labels: rows /
# cube / split: K^3 meshes, rows of elements, 2 x 2 x 2 cubes or the split-form volume
# term, LES on or off (tests/test_gpu_dg.py); fullsize: the benchmark meshes on sampled
# elements (tests/test_gpu_fullsize.py); noalloc: dg_rhs_noalloc (tests/test_zz_no_alloc.py).
# The full-size errors are larger: with h = 2 pi / K smaller, the 2/h of the derivatives
# scales the same FP32 rounding against a smaller operator.
FP32_BOUND = {
    "cube K4 P2 les1": (6.6e-06, 3.1e-06, 7.9e-07),   # measured 2.18e-06, 1.02e-06, 2.63e-07
    "cube K4 P3 les0": (3.1e-05, 3.7e-05, 3.4e-06),   # measured 1.03e-05, 1.20e-05, 1.10e-06
    "fullsize K16 P6": (0.0004, 0.0071, 5.4e-05),   # measured 1.31e-04, 2.35e-03, 1.79e-05
    "fullsize K16 P8": (0.00059, 0.011, 7.1e-05),   # measured 1.94e-04, 3.39e-03, 2.37e-05
    "fullsize K32 P3": (0.00032, 0.0068, 3e-05),   # measured 1.05e-04, 2.26e-03, 9.79e-06
    "noalloc K2 P6": (6.3e-06, 0.00051, 4.6e-06),   # measured 2.09e-06, 1.70e-04, 1.52e-06
    "noalloc K3 P6": (6.7e-05, 0.0013, 9.2e-06),   # measured 2.23e-05, 4.09e-04, 3.05e-06
    "rows K2 P5 les1": (3.8e-06, 0.00011, 2.7e-06),   # measured 1.26e-06, 3.54e-05, 8.71e-07
    "rows K2 P6 les1": (6.2e-06, 0.00053, 4.7e-06),   # measured 2.05e-06, 1.74e-04, 1.54e-06
    "rows K2 P8 les0": (8.8e-06, 0.00058, 5.8e-06),   # measured 2.92e-06, 1.92e-04, 1.91e-06
    "rows K3 P3 les1": (1.6e-05, 1.3e-05, 1.6e-06),   # measured 5.27e-06, 4.29e-06, 5.32e-07
    "rows K3 P4 les0": (3.4e-05, 0.00013, 4e-06),   # measured 1.13e-05, 4.23e-05, 1.32e-06
    "rows K3 P6 les1": (6.4e-05, 0.0013, 9.3e-06),   # measured 2.12e-05, 4.04e-04, 3.08e-06
    "rows K3 P8 les0": (9.8e-05, 0.0019, 1.3e-05),   # measured 3.26e-05, 6.19e-04, 4.10e-06
    "rows K4 P3 les0": (3.1e-05, 3.7e-05, 3.4e-06),   # measured 1.03e-05, 1.21e-05, 1.10e-06
    "rows K8 P3 les0": (6.6e-05, 0.00053, 7.1e-06),   # measured 2.19e-05, 1.73e-04, 2.37e-06
    "split K2 P6 les1": (9.3e-06, 0.00083, 1.1e-05),   # measured 3.08e-06, 2.74e-04, 3.35e-06
    "split K2 P8 les0": (1.4e-05, 0.0011, 1.4e-05),   # measured 4.42e-06, 3.37e-04, 4.41e-06
    "split K4 P3 les0": (3.5e-05, 7.6e-05, 1.2e-05),   # measured 1.15e-05, 2.52e-05, 3.73e-06
}


def bound(label):
    """Every FP32 parity case has a bound of its own: an unlisted case is an error."""
    return FP32_BOUND[label]


def errors(R, Ro, axis_vars=0):
    """Relative L2 error per variable (variables along axis_vars) and the density error
    against the momentum norm."""
    R = np.moveaxis(np.asarray(R, np.float64), axis_vars, 0)
    Ro = np.moveaxis(np.asarray(Ro, np.float64), axis_vars, 0)
    per_var = [float(np.linalg.norm(R[v] - Ro[v]) / np.linalg.norm(Ro[v])) for v in range(5)]
    dens = float(np.linalg.norm(R[0] - Ro[0]) / np.linalg.norm(Ro[1]))
    return per_var, dens


def record(label, per_var, dens):
    path = os.environ.get("DGNN_ERROR_LOG")
    if not path:
        return
    if os.path.dirname(path):
        os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "a") as f:
        f.write(json.dumps({"case": label, "per_var": per_var, "density_vs_momentum": dens}) + "\n")


def check(label, R, Ro, axis_vars=0):
    per_var, dens = errors(R, Ro, axis_vars)
    record(label, per_var, dens)
    mom, energy, rho = bound(label)
    assert max(per_var[1:4]) < mom, (label, per_var, mom)
    assert per_var[4] < energy, (label, per_var, energy)
    assert dens < rho, (label, dens, rho)
    return per_var
