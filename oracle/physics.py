"""Compressible Navier-Stokes physics for the oracle (Appendix A; Sec. 3.1).

State q = (rho, rho v1, rho v2, rho v3, rho e) on axis 0 of every array.
Nondimensionalisation (the paper gives only rho0; this is the reading used
throughout): rho0 = V0 = L = 1, mu = 1/Re constant, p0 = 1/(gamma M^2),
heat flux kappa grad T = mu gamma / ((gamma-1) Pr) grad(p/rho), so the gas
constant cancels.  Gradient variables for BR1: (v1, v2, v3, theta = p/rho).

Test infrastructure only (see the package docstring).
"""
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Flow:
    Re: float = 1600.0
    Mach: float = 0.1
    Pr: float = 0.71
    gamma: float = 1.4
    les: bool = False      # Smagorinsky closure (Sec. 3.1, Table 1 "LES")
    Cs: float = 0.1
    Prt: float = 0.9
    les_delta: float = 0.0  # filter width; 0 -> h/(P+1) (reading: not stated in the paper)
    inviscid: bool = False  # mu = 0 (used by the Euler convergence pin)
    split: bool = False     # kinetic-energy-preserving split-form volume term (see dgsem.rhs)

    @property
    def mu(self):
        return 0.0 if self.inviscid else 1.0 / self.Re

    @property
    def p0(self):
        return 1.0 / (self.gamma * self.Mach ** 2)


def pressure(q, gamma):
    """p = (gamma - 1) (rho e - |rho v|^2 / (2 rho))."""
    return (gamma - 1.0) * (q[4] - 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2) / q[0])


def gradient_variables(q, gamma):
    """U = (v1, v2, v3, theta) with theta = p / rho (BR1 gradient variables)."""
    rho = q[0]
    return np.stack([q[1] / rho, q[2] / rho, q[3] / rho, pressure(q, gamma) / rho])


def inviscid_flux(q, d, gamma):
    """Column d of the Euler flux f^a (Appendix A, Eq. A.2)."""
    rho = q[0]
    v = q[1:4] / rho
    p = pressure(q, gamma)
    vd = v[d]
    f = np.empty_like(q)
    f[0] = q[1 + d]
    for i in range(3):
        f[1 + i] = q[1 + i] * vd + (p if i == d else 0.0)
    f[4] = vd * (q[4] + p)  # rho v_d H
    return f


def kep_flux(qa, qb, d, gamma):
    """Two-point flux of the kinetic-energy-preserving split form (Pirozzoli's averages,
    as used in split-form DGSEM; not part of the paper, a robustness variant of its
    volume term): with {a} = (a_a + a_b)/2, mass flux m = {rho}{v_d},
        (m, m {v_1} + {p} delta_1d, m {v_2} + {p} delta_2d, m {v_3} + {p} delta_3d, m {H}),
    H = (rho e + p) / rho.  Symmetric in (qa, qb); equal to the Euler flux column d when
    qa = qb."""
    def prim(q):
        rho = q[0]
        v = q[1:4] / rho
        p = pressure(q, gamma)
        return rho, v, p, (q[4] + p) / rho
    ra, va, pa, Ha = prim(qa)
    rb, vb, pb, Hb = prim(qb)
    m = 0.25 * (ra + rb) * (va[d] + vb[d])
    pm = 0.5 * (pa + pb)
    F = np.empty(np.broadcast_shapes(qa.shape, qb.shape))
    F[0] = m
    for j in range(3):
        F[1 + j] = m * 0.5 * (va[j] + vb[j]) + (pm if j == d else 0.0)
    F[4] = m * 0.5 * (Ha + Hb)
    return F


def transport_coefficients(q, G, flow, delta):
    """Dynamic viscosity and heat coefficient (mu, lam), lam = kappa in grad(p/rho) form.

    Without closure: mu = 1/Re, lam = mu gamma / ((gamma-1) Pr).
    With the Smagorinsky closure: mu_t = rho (Cs delta)^2 |S|, |S| = sqrt(2 S_ij S_ij),
    S_ij = (dv_i/dx_j + dv_j/dx_i)/2 from the BR1 gradients, added to mu, and
    mu_t gamma / ((gamma-1) Pr_t) added to lam.  Parity of the closure constants
    (delta, Pr_t) is unpinned: the paper does not state them.
    G[d, a] = d U_a / d x_d.
    """
    g = flow.gamma
    mu = np.full(q.shape[1:], flow.mu)
    lam = mu * g / ((g - 1.0) * flow.Pr)
    if flow.les:
        SS = np.zeros(q.shape[1:])
        for i in range(3):
            for j in range(3):
                Sij = 0.5 * (G[j, i] + G[i, j])
                SS = SS + Sij * Sij
        mu_t = q[0] * (flow.Cs * delta) ** 2 * np.sqrt(2.0 * SS)
        mu = mu + mu_t
        lam = lam + mu_t * g / ((g - 1.0) * flow.Prt)
    return mu, lam


def viscous_flux(q, G, mu, lam, d):
    """Column d of the viscous flux f^nu (Appendix A, Eq. A.3).

    tau = mu (grad v + grad v^T) - 2/3 mu (div v) I;
    f^nu_d = (0, tau_1d, tau_2d, tau_3d, sum_j v_j tau_jd + kappa dT/dx_d).
    """
    rho = q[0]
    v = q[1:4] / rho
    div = G[0, 0] + G[1, 1] + G[2, 2]
    f = np.zeros_like(q)
    energy = lam * G[d, 3]
    for i in range(3):
        tau_id = mu * (G[d, i] + G[i, d])
        if i == d:
            tau_id = tau_id - (2.0 / 3.0) * mu * div
        f[1 + i] = tau_id
        energy = energy + v[i] * tau_id
    f[4] = energy
    return f


def roe_flux(qL, qR, d, gamma):
    """Roe approximate Riemann flux in direction +e_d (Sec. 3.1: Roe for the
    advective fluxes), F* = (f(qL) + f(qR))/2 - |A~| (qR - qL) / 2, with Roe
    averages and the standard eigen-decomposition of |A~| dq.  No entropy fix.
    """
    rL, rR = qL[0], qR[0]
    vL, vR = qL[1:4] / rL, qR[1:4] / rR
    pL, pR = pressure(qL, gamma), pressure(qR, gamma)
    HL, HR = (qL[4] + pL) / rL, (qR[4] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    vt = (sL * vL + sR * vR) / (sL + sR)
    Ht = (sL * HL + sR * HR) / (sL + sR)
    ke = 0.5 * (vt[0] ** 2 + vt[1] ** 2 + vt[2] ** 2)
    c2 = (gamma - 1.0) * (Ht - ke)
    c = np.sqrt(c2)
    rt = sL * sR
    Vn = vt[d]

    drho = rR - rL
    dp = pR - pL
    dv = vR - vL
    dVn = dv[d]
    a1 = (dp - rt * c * dVn) / (2.0 * c2)   # wave Vn - c
    a2 = drho - dp / c2                     # entropy wave Vn
    a5 = (dp + rt * c * dVn) / (2.0 * c2)   # wave Vn + c
    l1, l2, l5 = np.abs(Vn - c), np.abs(Vn), np.abs(Vn + c)

    diss = np.empty_like(qL)
    diss[0] = l1 * a1 + l2 * a2 + l5 * a5
    for i in range(3):
        n_i = 1.0 if i == d else 0.0
        shear_i = rt * (dv[i] - dVn * n_i)   # shear waves, speed Vn
        diss[1 + i] = (l1 * a1 * (vt[i] - c * n_i) + l2 * (a2 * vt[i] + shear_i)
                       + l5 * a5 * (vt[i] + c * n_i))
    vt_dot_shear = rt * (vt[0] * dv[0] + vt[1] * dv[1] + vt[2] * dv[2] - Vn * dVn)
    diss[4] = (l1 * a1 * (Ht - c * Vn) + l2 * (a2 * ke + vt_dot_shear)
               + l5 * a5 * (Ht + c * Vn))
    return 0.5 * (inviscid_flux(qL, d, gamma) + inviscid_flux(qR, d, gamma)) - 0.5 * diss
