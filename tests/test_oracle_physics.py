"""Pins of the oracle's flux functions (Appendix A; Roe flux of Sec. 3.1)."""
import numpy as np
import pytest

from oracle import physics

GAMMA = 1.4


def conserved(rho, v, p):
    rho = np.asarray(rho, float)
    v = np.asarray(v, float)
    return np.concatenate([[rho], rho * v, [p / (GAMMA - 1) + 0.5 * rho * (v ** 2).sum()]])


def states(seed, n, vd_range, d):
    """n random primitive states with the d-velocity in vd_range."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        rho = rng.uniform(0.8, 1.3)
        v = rng.uniform(-0.5, 0.5, 3)
        v[d] = rng.uniform(*vd_range)
        p = rng.uniform(0.6, 1.2)
        out.append(conserved(rho, v, p))
    return np.array(out).T   # (5, n)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_roe_consistency(d):
    q = states(1, 16, (-2, 2), d)
    np.testing.assert_allclose(physics.roe_flux(q, q, d, GAMMA), physics.inviscid_flux(q, d, GAMMA),
                               rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_roe_property_supersonic_upwinding(d):
    """Roe's linearisation satisfies f(qR) - f(qL) = A~ (qR - qL) exactly, so when every
    wave moves right F* = f(qL), and when every wave moves left F* = f(qR).  This checks
    every term of the wave decomposition at once."""
    # sound speed ~ sqrt(1.4 * 1 / 1) ~ 1.2; |v_d| in [3, 4] is supersonic on both sides
    qL = states(2, 32, (3.0, 4.0), d)
    qR = states(3, 32, (3.0, 4.0), d)
    np.testing.assert_allclose(physics.roe_flux(qL, qR, d, GAMMA), physics.inviscid_flux(qL, d, GAMMA),
                               rtol=1e-12, atol=1e-12)
    qL = states(4, 32, (-4.0, -3.0), d)
    qR = states(5, 32, (-4.0, -3.0), d)
    np.testing.assert_allclose(physics.roe_flux(qL, qR, d, GAMMA), physics.inviscid_flux(qR, d, GAMMA),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_roe_mirror_symmetry(d):
    """Reflecting the d axis: F*(M qR, M qL) = -M F*(qL, qR), M flips rho v_d."""
    qL = states(6, 32, (-1, 1), d)
    qR = states(7, 32, (-1, 1), d)
    M = np.ones((5, 1))
    M[1 + d] = -1.0
    np.testing.assert_allclose(physics.roe_flux(M * qR, M * qL, d, GAMMA),
                               -M * physics.roe_flux(qL, qR, d, GAMMA), rtol=1e-13, atol=1e-13)


def test_roe_subsonic_contact_is_upwinded():
    """A contact (jump in rho only, same v and p) moving right is carried with f(qL)."""
    qL = conserved(1.0, [0.3, 0.1, -0.2], 1.0)[:, None]
    qR = conserved(1.7, [0.3, 0.1, -0.2], 1.0)[:, None]
    np.testing.assert_allclose(physics.roe_flux(qL, qR, 0, GAMMA), physics.inviscid_flux(qL, 0, GAMMA),
                               rtol=1e-14, atol=1e-14)


def test_inviscid_flux_rotation_equivariance():
    """Permuting the axes (x,y,z) -> (y,z,x) permutes the flux columns accordingly."""
    q = states(8, 8, (-1, 1), 0)
    perm = [1, 2, 0]  # new velocity component i is old component perm[i]
    qp = q.copy()
    qp[1:4] = q[1:4][perm]
    for d in range(3):
        f_old = physics.inviscid_flux(q, perm[d], GAMMA)
        f_new = physics.inviscid_flux(qp, d, GAMMA)
        expect = f_old.copy()
        expect[1:4] = f_old[1:4][perm]
        np.testing.assert_allclose(f_new, expect, rtol=1e-15)


def test_viscous_flux_couette_values():
    """Plain shear u = a y (only du/dy = a): tau_xy = mu a, energy flux v . tau + kappa grad T."""
    mu, lam, a = 0.3, 0.7, 2.0
    q = conserved(1.0, [0.5, 0.0, 0.0], 1.0)[:, None]
    G = np.zeros((3, 4, 1))
    G[1, 0] = a            # d u / d y
    G[0, 3] = 0.25         # d theta / d x
    fx = physics.viscous_flux(q, G, mu, lam, 0)[:, 0]
    fy = physics.viscous_flux(q, G, mu, lam, 1)[:, 0]
    np.testing.assert_allclose(fx, [0, 0, mu * a, 0, lam * 0.25], atol=1e-15)
    np.testing.assert_allclose(fy, [0, mu * a, 0, 0, 0.5 * mu * a], atol=1e-15)
    # dilatation only: du/dx = b -> tau_xx = 2 mu b - 2/3 mu b = 4/3 mu b, tau_yy = -2/3 mu b
    G = np.zeros((3, 4, 1))
    G[0, 0] = 1.5
    fx = physics.viscous_flux(q, G, mu, lam, 0)[:, 0]
    fy = physics.viscous_flux(q, G, mu, lam, 1)[:, 0]
    np.testing.assert_allclose(fx[1], 4.0 / 3.0 * mu * 1.5, rtol=1e-15)
    np.testing.assert_allclose(fy[2], -2.0 / 3.0 * mu * 1.5, rtol=1e-15)


def test_smagorinsky_viscosity_closed_forms():
    """Sec. 3.1's eddy viscosity mu_t = rho (Cs delta)^2 |S|, |S| = sqrt(2 S_ij S_ij):
    plain shear du/dy = a gives |S| = |a|; pure rotation (antisymmetric gradient) gives
    |S| = 0; uniform dilatation du/dx = dv/dy = dw/dz = b gives |S| = sqrt(6) |b|.  The
    heat coefficient gains mu_t gamma / ((gamma - 1) Pr_t)."""
    flow = physics.Flow(Re=100.0, les=True, Cs=0.2, Prt=0.9)
    rho, delta = 1.3, 0.25
    q = conserved(rho, [0.1, -0.2, 0.3], 1.0)[:, None]
    c = rho * (flow.Cs * delta) ** 2
    base_mu = 1.0 / flow.Re
    base_lam = base_mu * GAMMA / ((GAMMA - 1) * flow.Pr)
    cases = []
    G = np.zeros((3, 4, 1))
    G[1, 0] = -2.5                       # du/dy
    cases.append((G, 2.5))
    G = np.zeros((3, 4, 1))
    G[1, 0], G[0, 1] = 1.7, -1.7         # du/dy = -dv/dx: rigid rotation
    cases.append((G, 0.0))
    G = np.zeros((3, 4, 1))
    G[0, 0] = G[1, 1] = G[2, 2] = 0.4    # uniform dilatation
    cases.append((G, np.sqrt(6.0) * 0.4))
    for G, s_norm in cases:
        mu, lam = physics.transport_coefficients(q, G, flow, delta)
        mu_t = c * s_norm
        np.testing.assert_allclose(mu[0], base_mu + mu_t, rtol=1e-14)
        np.testing.assert_allclose(lam[0], base_lam + mu_t * GAMMA / ((GAMMA - 1) * flow.Prt), rtol=1e-14)
