"""Algorithm 1 of Sec. 2.1 (high-order evolution and pair generation, training,
corrected low-order evolution) and the corrected system of Eq. 4.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from . import dgsem, mlp


def forcing_target(q_ho_start, q_ho_end, mesh_lo, flow_lo, dt_lo, P_hi):
    """The corrective forcing the network is trained to produce (Sec. 2.1, Algorithm 1;
    Eq. 4): the source that, added over one low-order step of length dt_lo, carries the
    uncorrected low-order solution started from the filtered high-order state onto the
    filtered high-order state at the end of the step,

        s = (G q_HO(t + dt_lo) - RK3_LO(G q_HO(t), dt_lo)) / dt_lo,

    G the filter of Eq. 2.  Returns (G q_HO(t), s): the network's input and target."""
    q_in = dgsem.project(q_ho_start, P_hi, mesh_lo.P)
    q_lo_end = dgsem.rk3_step(q_in, dt_lo, lambda z: dgsem.rhs(z, mesh_lo, flow_lo))
    return q_in, (dgsem.project(q_ho_end, P_hi, mesh_lo.P) - q_lo_end) / dt_lo


def generate_pairs(q_ho, mesh_ho, mesh_lo, flow_ho, flow_lo, dt_lo, ratio, n_steps, io_vars=(0, 1, 2, 3, 4)):
    """Training pairs over a window of the high-order run (Sec. 2.1, Algorithm 1): the
    high-order solution advances in ``ratio`` RK3 steps of dt_lo / ratio per low-order
    step, and every low-order step of the window gives one pair per element, the
    forcing_target of that step.  Returns (X, T, q_ho_final): per-element inputs and
    targets, shapes (n_steps * K^3, len(io_vars) * n_lo^3)."""
    dt_ho = dt_lo / ratio
    X, T = [], []
    q = q_ho
    for _ in range(n_steps):
        q_next = q
        for _m in range(ratio):
            q_next = dgsem.rk3_step(q_next, dt_ho, lambda z: dgsem.rhs(z, mesh_ho, flow_ho))
        q_in, s = forcing_target(q, q_next, mesh_lo, flow_lo, dt_lo, mesh_ho.P)
        X.append(dgsem.element_features(q_in, io_vars))
        T.append(dgsem.element_features(s, io_vars))
        q = q_next
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
