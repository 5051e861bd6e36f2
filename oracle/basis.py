"""One-dimensional nodal basis for the DGSEM (Sec. 2.6: nodal Lagrange bases on
Gauss-Lobatto points, as in Kopriva's DGSEM book cited there) and the modal
filter G of Sec. 2 (Eq. 2) / Sec. 2.6 (nodal -> modal -> truncate -> nodal).

Test infrastructure only (see the package docstring).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def legendre_unit(m):
    """Legendre-series coefficient vector of L_m (library representation)."""
    c = np.zeros(m + 1)
    c[m] = 1.0
    return c


def gl_nodes_weights(P):
    """Gauss-Lobatto nodes xi_0 = -1 < ... < xi_P = 1 and weights.

    Nodes: the endpoints and the roots of L_P'(xi) (numpy's Legendre root finder,
    polished by two Newton steps on L_P').
    Weights: w_i = 2 / (P (P+1) L_P(xi_i)^2).
    """
    if P < 1:
        raise ValueError("P >= 1 required")
    dLP = npleg.legder(legendre_unit(P))
    interior = np.sort(np.real(npleg.legroots(dLP))) if P > 1 else np.zeros(0)
    d2LP = npleg.legder(dLP)
    for _ in range(2):
        interior = interior - npleg.legval(interior, dLP) / npleg.legval(interior, d2LP)
    xi = np.concatenate(([-1.0], interior, [1.0]))
    w = 2.0 / (P * (P + 1) * npleg.legval(xi, legendre_unit(P)) ** 2)
    return xi, w


def lagrange_derivative_matrix(xi):
    """D[i, j] = l_j'(xi_i), l_j the Lagrange polynomial through the nodes xi.

    Written from the definition
        l_j'(x) = sum_{m != j} 1/(xi_j - xi_m) * prod_{k != j, m} (x - xi_k)/(xi_j - xi_k).
    """
    n = len(xi)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            total = 0.0
            for m in range(n):
                if m == j:
                    continue
                prod = 1.0 / (xi[j] - xi[m])
                for k in range(n):
                    if k == j or k == m:
                        continue
                    prod *= (xi[i] - xi[k]) / (xi[j] - xi[k])
                total += prod
            D[i, j] = total
    return D


def lagrange_interpolation_matrix(xi_from, x_to):
    """I[a, j] = l_j(x_to[a]) for the Lagrange basis on xi_from."""
    n = len(xi_from)
    I = np.ones((len(x_to), n))
    for a, x in enumerate(x_to):
        for j in range(n):
            for k in range(n):
                if k != j:
                    I[a, j] *= (x - xi_from[k]) / (xi_from[j] - xi_from[k])
    return I


def legendre_vandermonde(xi, nmodes):
    """V[i, m] = L_m(xi_i) for m < nmodes (modal <-> nodal map)."""
    return np.stack([npleg.legval(xi, legendre_unit(m)) for m in range(nmodes)], axis=1)


def modal_filter_matrix(P_hi, P_lo):
    """1D filter G_1d: nodal values at the P_hi GL nodes -> nodal values at the
    P_lo GL nodes of the Legendre expansion truncated to modes m <= P_lo.

    Steps as stated in Sec. 2.6: nodal -> modal (invert the P_hi Vandermonde),
    keep modes 0..P_lo, evaluate them at the P_lo nodes.
    """
    xi_hi, _ = gl_nodes_weights(P_hi)
    xi_lo, _ = gl_nodes_weights(P_lo)
    V_hi = legendre_vandermonde(xi_hi, P_hi + 1)
    modal = np.linalg.inv(V_hi)                       # (modes, nodes_hi)
    V_lo = legendre_vandermonde(xi_lo, P_lo + 1)      # (nodes_lo, modes_lo)
    return V_lo @ modal[: P_lo + 1, :]
