"""Algorithm 1 of Sec. 2.1 (high-order evolution and pair generation, training,
corrected low-order evolution) and the corrected system of Eq. 4.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from . import dgsem, mlp


def generate_pairs(q_ho, mesh_ho, mesh_lo, flow_ho, flow_lo, dt_lo, ratio, n_steps, io_vars=(0, 1, 2, 3, 4)):
    """High-order evolution with pair generation (first loop of Algorithm 1).

    For n = 0 .. n_steps-1:
      q_NN^n   = G q_HO^n                      (match low order with filtered high order)
      q_NN^n+1 = RK3_LO(q_NN^n, dt_lo)          (advance without correction)
      q_HO     advanced ``ratio`` steps of dt_lo/ratio
      s_n      = (G q_HO^{n+1} - q_NN^{n+1}) / dt_lo
    Returns (X, T, q_ho_final): per-element inputs G q_HO^n and targets s_n,
    shapes (n_steps * K^3, len(io_vars) * n_lo^3).
    """
    P_hi, P_lo = mesh_ho.P, mesh_lo.P
    dt_ho = dt_lo / ratio
    X, T = [], []
    q = q_ho
    for _ in range(n_steps):
        q_nn = dgsem.project(q, P_hi, P_lo)
        q_nn1 = dgsem.rk3_step(q_nn, dt_lo, lambda z: dgsem.rhs(z, mesh_lo, flow_lo))
        for _m in range(ratio):
            q = dgsem.rk3_step(q, dt_ho, lambda z: dgsem.rhs(z, mesh_ho, flow_ho))
        s = (dgsem.project(q, P_hi, P_lo) - q_nn1) / dt_lo
        X.append(dgsem.element_features(q_nn, io_vars))
        T.append(dgsem.element_features(s, io_vars))
    return np.concatenate(X), np.concatenate(T), q


def scalers_from_data(X, T):
    """Per-feature mean and (population) standard deviation; a feature with zero
    spread keeps std 1 so that scaling is the identity shift."""
    def ms(A):
        m = A.mean(axis=0)
        s = np.sqrt(((A - m) ** 2).mean(axis=0))
        return m, np.where(s > 0.0, s, 1.0)
    mi, si = ms(X)
    mo, so = ms(T)
    return mi, si, mo, so


def forcing_field(params, scalers, q, n, io_vars=(0, 1, 2, 3, 4), bf16=False):
    """s(q) on the whole mesh: the network applied to every element (Sec. 2.2)."""
    K = q.shape[1]
    F = mlp.infer(params, scalers, dgsem.element_features(q, io_vars), bf16)
    return dgsem.field_from_features(F, K, n, io_vars)


def corrected_step(q, dt, mesh, flow, params, scalers, mode='stage', io_vars=(0, 1, 2, 3, 4), bf16=False):
    """One step of the corrected low-order system (Eq. 4).

    mode 'stage': s evaluated on every RK stage state and added to p_LO (Eq. 4
    integrated by RK3).  mode 'post': Algorithm 1's third loop taken literally,
    q^{n+1} = RK3(q^n) + dt * s(q^n).
    """
    n = mesh.n
    if mode == 'stage':
        return dgsem.rk3_step(q, dt, lambda z: dgsem.rhs(z, mesh, flow)
                              + forcing_field(params, scalers, z, n, io_vars, bf16))
    if mode == 'post':
        s = forcing_field(params, scalers, q, n, io_vars, bf16)
        return dgsem.rk3_step(q, dt, lambda z: dgsem.rhs(z, mesh, flow)) + dt * s
    raise ValueError(mode)
