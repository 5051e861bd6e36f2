"""Pins of the oracle's 1D basis and filter G against closed forms, exactness
properties and an independent quadrature (no GPU)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import basis, dgsem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_gl_golden():
    rows = []
    with open(os.path.join(GOLDEN, "gauss_lobatto_closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            P, node, weight = line.split()
            env = {"sqrt": math.sqrt}
            rows.append((int(P), eval(node, env), eval(weight.replace("/", "/"), env)))
    return rows


def test_gl_nodes_weights_closed_forms():
    rows = _read_gl_golden()
    for P in range(1, 5):
        xi, w = basis.gl_nodes_weights(P)
        ref = [(n, wt) for (p, n, wt) in rows if p == P]
        assert len(ref) == P + 1
        np.testing.assert_allclose(xi, [r[0] for r in ref], atol=1e-15)
        np.testing.assert_allclose(w, [r[1] for r in ref], rtol=1e-14)


@pytest.mark.parametrize("P", range(1, 9))
def test_gl_quadrature_exactness(P):
    """GL with P+1 points integrates degree <= 2P-1 exactly and nodes are roots of (1-x^2) L_P'."""
    xi, w = basis.gl_nodes_weights(P)
    for k in range(2 * P):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs((w * xi ** k).sum() - exact) < 1e-14
    dLP = npleg.legder(basis.legendre_unit(P))
    assert np.all(np.abs(npleg.legval(xi[1:-1], dLP)) < 1e-12 * P * P)
    assert np.all(np.diff(xi) > 0)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 8])
def test_derivative_matrix_exact_on_polynomials(P):
    """D differentiates x^k exactly for k <= P (Kopriva, nodal collocation)."""
    xi, _ = basis.gl_nodes_weights(P)
    D = basis.lagrange_derivative_matrix(xi)
    for k in range(P + 1):
        exact = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** k, exact, atol=1e-12 * (k + 1))
    # summation-by-parts: W D + D^T W = diag(-1, 0, ..., 0, 1)
    W = np.diag(basis.gl_nodes_weights(P)[1])
    B = np.zeros((P + 1, P + 1))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(W @ D + D.T @ W, B, atol=1e-13)


@pytest.mark.parametrize("P_hi,P_lo", [(8, 3), (8, 2), (6, 3), (4, 2)])
def test_filter_idempotent_exact_and_mean_preserving(P_hi, P_lo):
    G = basis.modal_filter_matrix(P_hi, P_lo)
    xi_hi, w_hi = basis.gl_nodes_weights(P_hi)
    xi_lo, w_lo = basis.gl_nodes_weights(P_lo)
    # exact on polynomials of degree <= P_lo
    for k in range(P_lo + 1):
        np.testing.assert_allclose(G @ xi_hi ** k, xi_lo ** k, atol=1e-13)
    # idempotent: lift the LO result back to HO nodes and filter again
    rng = np.random.default_rng(5)
    u = rng.standard_normal(P_hi + 1)
    lo = G @ u
    lift = basis.lagrange_interpolation_matrix(xi_lo, xi_hi) @ lo
    np.testing.assert_allclose(G @ lift, lo, atol=1e-13)
    # element mean preserved
    assert abs(w_lo @ lo - w_hi @ u) < 1e-13


@pytest.mark.parametrize("P_hi,P_lo", [(8, 3), (6, 2)])
def test_filter_equals_l2_projection_by_gauss_quadrature(P_hi, P_lo):
    """G u = L2 projection of the HO polynomial onto P_lo, computed independently
    with 12-point Gauss-Legendre quadrature of the Lagrange interpolant."""
    xi_hi, _ = basis.gl_nodes_weights(P_hi)
    xi_lo, _ = basis.gl_nodes_weights(P_lo)
    xg, wg = npleg.leggauss(12)
    u = np.random.default_rng(7).standard_normal(P_hi + 1)
    ug = basis.lagrange_interpolation_matrix(xi_hi, xg) @ u
    coeffs = [(2 * m + 1) / 2.0 * np.sum(wg * ug * npleg.legval(xg, basis.legendre_unit(m)))
              for m in range(P_lo + 1)]
    ref = npleg.legval(xi_lo, np.array(coeffs))
    np.testing.assert_allclose(basis.modal_filter_matrix(P_hi, P_lo) @ u, ref, atol=1e-13)


def test_project_3d_tensor_product_reproduces_q3_field():
    """3D projection P8 -> P3 reproduces a polynomial of degree <= 3 per direction."""
    m8, m3 = dgsem.Mesh(2, 8), dgsem.Mesh(2, 3)
    def poly(X, Y, Z):
        return 1 + X - 2 * Y ** 2 + X * Y * Z + Z ** 3 - 0.5 * X ** 3 * Y ** 2
    f8 = poly(*m8.coordinates())[None]
    f3 = poly(*m3.coordinates())[None]
    np.testing.assert_allclose(dgsem.project(f8, 8, 3), f3, atol=1e-12)


@pytest.mark.parametrize("P_lo,P_hi", [(3, 8), (2, 8), (3, 6), (5, 5)])
def test_prolong_is_exact_on_low_order_polynomials(P_lo, P_hi):
    """Prolongation evaluates the order-P_lo interpolant at the P_hi nodes: a polynomial of
    degree <= P_lo per direction sampled on the P_lo nodes comes out as its values on the
    P_hi nodes."""
    ml, mh = dgsem.Mesh(2, P_lo), dgsem.Mesh(2, P_hi)
    def poly(X, Y, Z):
        return 2 - X + 0.5 * Y * Z + X ** min(P_lo, 2) * Y - (Z ** P_lo) / 3
    fl = poly(*ml.coordinates())[None]
    fh = poly(*mh.coordinates())[None]
    np.testing.assert_allclose(dgsem.prolong(fl, P_lo, P_hi), fh, atol=1e-11, rtol=1e-12)


@pytest.mark.parametrize("P_lo,P_hi", [(3, 8), (2, 7), (4, 6)])
def test_filter_inverts_prolongation(P_lo, P_hi):
    """Any nodal P_lo field is a polynomial in Q_{P_lo}; the filter G (the L2 projection
    onto Q_{P_lo}) returns it unchanged after prolongation."""
    rng = np.random.default_rng(P_lo + 10 * P_hi)
    q = rng.standard_normal((5, 2, 2, 2) + (P_lo + 1,) * 3)
    back = dgsem.project(dgsem.prolong(q, P_lo, P_hi), P_hi, P_lo)
    np.testing.assert_allclose(back, q, atol=1e-12)
