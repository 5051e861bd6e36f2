"""Strong-form nodal DGSEM operator p(q) for the 3D compressible Navier-Stokes
equations on a periodic Cartesian hex mesh (Eq. 1 / Eq. 3 of Sec. 2; fluxes of
Appendix A; Roe advective and BR1 viscous interface fluxes of Sec. 3.1), the
Taylor-Green initial field (Sec. 3.1, Eq. 11), low-storage RK3 (Sec. 2, "third
order Runge-Kutta"), the filter G (Eq. 2, Sec. 2.6) and the diagnostics (Eq. 9).

Array layout: every field has the six trailing axes (ez, ey, ex, k, j, i):
element indices then node indices, x fastest.  Flattening (var, ez, ey, ex,
k, j, i) gives the library's [var][elem][node] layout with
elem = ex + K (ey + K ez) and node = i + n (j + n k), n = P + 1.

Test infrastructure only (see the package docstring).
"""
import math

import numpy as np

from . import basis, physics

# trailing-axis positions: direction d = 0 (x), 1 (y), 2 (z)
NODE_AXIS = (-1, -2, -3)
ELEM_AXIS = (-4, -5, -6)

# Williamson (1980) 2N-storage third-order RK: the paper's "third-order three-stage
# Runge-Kutta scheme" (Sec. 3.1) is unnamed; this member of the family is the reading.
RK3_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK3_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)


class Mesh:
    """K^3 periodic elements on [-pi, pi]^3 (Sec. 3.1), polynomial order P on GL nodes."""

    def __init__(self, K, P):
        self.K, self.P, self.n = K, P, P + 1
        self.h = 2.0 * math.pi / K
        self.xi, self.w = basis.gl_nodes_weights(P)
        self.D = basis.derivative_matrix(P)

    def coordinates(self):
        """x, y, z arrays of shape (K, K, K, n, n, n): x = -pi + (e + (xi+1)/2) h."""
        K, n, h = self.K, self.n, self.h
        e = np.arange(K)
        c1d = -math.pi + (e[:, None] + 0.5 * (self.xi[None, :] + 1.0)) * h   # (K, n)
        X = c1d[None, None, :, None, None, :]
        Y = c1d[None, :, None, None, :, None]
        Z = c1d[:, None, None, :, None, None]
        shape = (K, K, K, n, n, n)
        return (np.broadcast_to(X, shape), np.broadcast_to(Y, shape), np.broadcast_to(Z, shape))

    def quadrature_weights(self):
        """w_i w_j w_k (h/2)^3 on shape (n, n, n) (GL quadrature, Cartesian Jacobian)."""
        w = self.w
        return w[None, None, :] * w[None, :, None] * w[:, None, None] * (self.h / 2.0) ** 3


# ----------------------------------------------------------------------------- helpers

def d_contract(F, D, d):
    """sum_m D[a, m] F[..., m along node axis of direction d]."""
    if d == 0:
        return np.einsum('im,...m->...i', D, F)
    if d == 1:
        return np.einsum('jm,...mi->...ji', D, F)
    return np.einsum('km,...mji->...kji', D, F)


def face(a, d, side):
    """Node layer on the left (side=0, node index 0) or right (side=1, index P)
    face of every element in direction d, keeping the axis (size 1)."""
    ax = NODE_AXIS[d]
    idx = 0 if side == 0 else a.shape[ax] - 1
    return np.take(a, [idx], axis=ax)


def neighbour(a, d, shift):
    """Value held by element e + shift (periodic) along direction d, for every e."""
    return np.roll(a, -shift, axis=ELEM_AXIS[d])


def add_on_face(R, d, side, val):
    ax = NODE_AXIS[d]
    idx = 0 if side == 0 else R.shape[ax] - 1
    sl = [slice(None)] * R.ndim
    sl[ax] = slice(idx, idx + 1)
    R[tuple(sl)] += val


# ----------------------------------------------------------------------------- initial field

def tgv_state(mesh, flow, perturbation=None):
    """Taylor-Green vortex, Sec. 3.1 Eq. 11, with rho0 = V0 = 1:
        rho = 1, v1 = sin x cos y cos z, v2 = -cos x sin y cos z, v3 = 0,
        p = 1/(gamma M^2) + (cos 2x + cos 2y)(cos 2z + 2)/16,
    rho e = p/(gamma-1) + rho |v|^2 / 2.  ``perturbation`` (shape of q, drawn by
    the caller) is added to the conserved variables.
    """
    x, y, z = mesh.coordinates()
    g = flow.gamma
    rho = np.ones(x.shape)
    v1 = np.sin(x) * np.cos(y) * np.cos(z)
    v2 = -np.cos(x) * np.sin(y) * np.cos(z)
    v3 = np.zeros(x.shape)
    p = flow.p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    q = np.stack([rho, rho * v1, rho * v2, rho * v3,
                  p / (g - 1.0) + 0.5 * rho * (v1 ** 2 + v2 ** 2 + v3 ** 2)])
    if perturbation is not None:
        q = q + perturbation.reshape(q.shape)
    return q


# ----------------------------------------------------------------------------- operator

def br1_gradient(U, mesh):
    """BR1 lifted gradient G[d, a] = dU_a/dx_d in strong form:
        G_d = (2/h) [ D_d U + (U^ - U)|_right / w_P  -  (U^ - U)|_left / w_0 ],
    U^ = (U^- + U^+)/2 on every face (Bassi-Rebay 1, cited in Sec. 3.1).
    """
    h, w, P = mesh.h, mesh.w, mesh.P
    G = np.empty((3,) + U.shape)
    for d in range(3):
        Gd = (2.0 / h) * d_contract(U, mesh.D, d)
        U_right = face(U, d, 1)
        U_left = face(U, d, 0)
        Uhat = 0.5 * (U_right + neighbour(U_left, d, +1))     # on each element's right face
        Uhat_left = neighbour(Uhat, d, -1)                    # the left face is the left neighbour's right face
        add_on_face(Gd, d, 1, (2.0 / h) * (Uhat - U_right) / w[P])
        add_on_face(Gd, d, 0, -(2.0 / h) * (Uhat_left - U_left) / w[0])
        G[d] = Gd
    return G


def rhs(q, mesh, flow, forcing=None):
    """Semi-discrete operator dq/dt = p(q) (+ s if ``forcing`` is given, Eq. 4):

        p(q) = -(2/h) sum_d [ D_d F_d + (F*_d - F_d)|_right / w_P - (F*_d - F_d)|_left / w_0 ]

    F_d = f^a_d - f^nu_d at the nodes; F*_d = Roe(q^-, q^+) - (f^nu(q^-, G^-) + f^nu(q^+, G^+))/2.
    """
    g = flow.gamma
    h, w, P = mesh.h, mesh.w, mesh.P
    U = physics.gradient_variables(q, g)
    G = br1_gradient(U, mesh)
    delta = flow.les_delta if flow.les_delta > 0.0 else h / (P + 1)
    mu, lam = physics.transport_coefficients(q, G, flow, delta)
    R = np.zeros_like(q)
    for d in range(3):
        F = physics.inviscid_flux(q, d, g) - physics.viscous_flux(q, G, mu, lam, d)
        if flow.split:
            # split form: the Euler part of the volume term is 2 sum_m D_im F#(q_i, q_m)
            # along each line (kep_flux); the viscous part keeps the standard form.  The
            # surface term below uses the nodal flux F as in the standard form.
            Fv = physics.viscous_flux(q, G, mu, lam, d)
            R -= (2.0 / h) * (split_volume(q, mesh.D, d, g) - d_contract(Fv, mesh.D, d))
        else:
            R -= (2.0 / h) * d_contract(F, mesh.D, d)

        qm = face(q, d, 1)
        qp = neighbour(face(q, d, 0), d, +1)
        Gm = face(G, d, 1)
        Gp = neighbour(face(G, d, 0), d, +1)
        mum, lamm = face(mu, d, 1), face(lam, d, 1)
        mup, lamp = neighbour(face(mu, d, 0), d, +1), neighbour(face(lam, d, 0), d, +1)
        Fstar = (physics.roe_flux(qm, qp, d, g)
                 - 0.5 * (physics.viscous_flux(qm, Gm, mum, lamm, d)
                          + physics.viscous_flux(qp, Gp, mup, lamp, d)))
        Fstar_left = neighbour(Fstar, d, -1)
        add_on_face(R, d, 1, -(2.0 / h) * (Fstar - face(F, d, 1)) / w[P])
        add_on_face(R, d, 0, (2.0 / h) * (Fstar_left - face(F, d, 0)) / w[0])
    if forcing is not None:
        R += forcing
    return R


def split_volume(q, D, d, gamma):
    """2 sum_m D[i, m] F#(q_i, q_m) along the node lines of direction d (F# = kep_flux)."""
    ax = NODE_AXIS[d]
    qd = np.moveaxis(q, ax, -1)                          # (..., n): the line along d last
    Fs = physics.kep_flux(qd[..., :, None], qd[..., None, :], d, gamma)   # (..., i, m)
    V = 2.0 * np.einsum('im,...im->...i', D, Fs)
    return np.moveaxis(V, -1, ax)


def rk3_step(q, dt, rhs_fn):
    """One low-storage RK3 step (2N form): for k = 1..3,
        g <- A_k g + dt * rhs(q);  q <- q + B_k g.
    ``rhs_fn(q)`` includes the corrective forcing when it is evaluated inside
    every stage (Eq. 4 integrated by RK3)."""
    q = q.copy()
    g = np.zeros_like(q)
    for k in range(3):
        g = RK3_A[k] * g + dt * rhs_fn(q)
        q = q + RK3_B[k] * g
    return q


# ----------------------------------------------------------------------------- filter G

def project(q_hi, P_hi, P_lo):
    """q_bar = G q_hi (Eq. 2): tensor-product Legendre truncation of each element,
    nodal P_hi -> nodal P_lo (Sec. 2.6)."""
    G1 = basis.modal_filter_matrix(P_hi, P_lo)
    out = np.einsum('im,...m->...i', G1, q_hi)
    out = np.einsum('jm,...mi->...ji', G1, out)
    out = np.einsum('km,...mji->...kji', G1, out)
    return out


def prolong(q_lo, P_lo, P_hi):
    """Each element's order-P_lo nodal polynomial evaluated at the order-P_hi GL nodes
    (Lagrange interpolation in each direction): the exact embedding of Q_{P_lo} into
    Q_{P_hi}, the inverse of the filter on Q_{P_lo}."""
    xi_lo, _ = basis.gl_nodes_weights(P_lo)
    xi_hi, _ = basis.gl_nodes_weights(P_hi)
    I1 = basis.lagrange_interpolation_matrix(xi_lo, xi_hi)
    out = np.einsum('im,...m->...i', I1, q_lo)
    out = np.einsum('jm,...mi->...ji', I1, out)
    out = np.einsum('km,...mji->...kji', I1, out)
    return out


# ----------------------------------------------------------------------------- diagnostics

def diagnostics(q, mesh, flow, R=None, q_ref=None):
    """Integral diagnostics under GL quadrature.

    mass, momentum (3), energy: sum w_i w_j w_k (h/2)^3 q.
    ke = (1/|Omega|) int rho |v|^2 / 2, |Omega| = (2 pi)^3.
    dke_dt (if R given) = (1/|Omega|) int (v . R_m - |v|^2 R_rho / 2), the exact
    time derivative of ke under dq/dt = R; the dissipation is -dke_dt.
    e_inf (if q_ref given): ||q - q_ref||_inf for rho u, rho v, rho w (Eq. 9).
    max_wave: max over nodes of |v| + c.
    """
    W = mesh.quadrature_weights()
    vol = (2.0 * math.pi) ** 3
    rho = q[0]
    v = q[1:4] / rho
    vsq = (v ** 2).sum(axis=0)
    p = physics.pressure(q, flow.gamma)
    c = np.sqrt(flow.gamma * p / rho)
    out = {
        'mass': float((W * q[0]).sum()),
        'momentum': [float((W * q[1 + i]).sum()) for i in range(3)],
        'energy': float((W * q[4]).sum()),
        'ke': float((W * 0.5 * rho * vsq).sum() / vol),
        'max_wave': float((np.sqrt(vsq) + c).max()),
    }
    if R is not None:
        dk = (v * R[1:4]).sum(axis=0) - 0.5 * vsq * R[0]
        out['dke_dt'] = float((W * dk).sum() / vol)
    if q_ref is not None:
        out['e_inf'] = [float(np.abs(q[1 + i] - q_ref[1 + i]).max()) for i in range(3)]
    return out


def stable_dt(q, mesh, flow, cfl):
    """dt = cfl * h / ((P+1)^2 * max(|v| + c)).  Sec. 2.3 gives CFL only as a
    proportionality; this form and its constant are a reading (parity unpinned
    for the constant; the formula is checked by definition)."""
    lam = diagnostics(q, mesh, flow)['max_wave']
    return cfl * mesh.h / ((mesh.P + 1) ** 2 * lam)


# ----------------------------------------------------------------------------- element features

def element_features(q, vars_=(0, 1, 2, 3, 4)):
    """Per-element feature vectors: (K^3, len(vars) * n^3), feature = var_slot * n^3 + node."""
    sel = q[list(vars_)]
    nv = sel.shape[0]
    K = sel.shape[1]
    n = sel.shape[-1]
    return np.ascontiguousarray(sel.reshape(nv, K ** 3, n ** 3).transpose(1, 0, 2).reshape(K ** 3, nv * n ** 3))


def field_from_features(F, K, n, vars_=(0, 1, 2, 3, 4)):
    """Inverse of element_features; variables not in ``vars_`` are zero."""
    nv = len(vars_)
    out = np.zeros((5, K ** 3, n ** 3))
    out[list(vars_)] = F.reshape(K ** 3, nv, n ** 3).transpose(1, 0, 2)
    return out.reshape(5, K, K, K, n, n, n)
