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


def _legendre_ext(P, x):
    """L_P(x) and L_P'(x) by the three-term recurrence, in the dtype of x."""
    one = np.ones_like(x)
    l0, l1, d0, d1 = one, x, 0 * x, one
    if P == 0:
        return one, 0 * x
    for k in range(1, P):
        l0, l1 = l1, ((2 * k + 1) * x * l1 - k * l0) / (k + 1)
        d0, d1 = d1, d0 + (2 * k + 1) * l0
    return l1, d1


def gl_nodes_weights_ext(P):
    """Gauss-Lobatto nodes and weights in extended precision (np.longdouble).

    Nodes: the endpoints and the roots of L_P'(xi) (numpy's Legendre root finder in
    FP64, then Newton on L_P' in extended precision).
    Weights: w_i = 2 / (P (P+1) L_P(xi_i)^2).
    """
    if P < 1:
        raise ValueError("P >= 1 required")
    ext = np.longdouble
    dLP = npleg.legder(legendre_unit(P))
    interior = np.sort(np.real(npleg.legroots(dLP))).astype(ext) if P > 1 else np.zeros(0, ext)
    for _ in range(6):
        # Newton on f = (1 - x^2) L_P'(x), f' = -P (P+1) L_P(x) (Legendre's equation)
        L, dL = _legendre_ext(P, interior)
        interior = interior - (1 - interior * interior) * dL / (-P * (P + 1) * L)
    xi = np.concatenate((np.array([-1.0], ext), interior, np.array([1.0], ext)))
    L, _ = _legendre_ext(P, xi)
    w = ext(2) / (P * (P + 1) * L * L)
    return xi, w


def gl_nodes_weights(P):
    """Gauss-Lobatto nodes xi_0 = -1 < ... < xi_P = 1 and weights, rounded once to FP64."""
    xi, w = gl_nodes_weights_ext(P)
    return xi.astype(np.float64), w.astype(np.float64)


def lagrange_derivative_matrix(xi):
    """D[i, j] = l_j'(xi_i), l_j the Lagrange polynomial through the nodes xi,
    computed in the dtype of ``xi`` (pass extended-precision nodes and round the
    result once to obtain the correctly rounded FP64 matrix).

    Written from the definition
        l_j'(x) = sum_{m != j} 1/(xi_j - xi_m) * prod_{k != j, m} (x - xi_k)/(xi_j - xi_k).
    """
    n = len(xi)
    D = np.zeros((n, n), dtype=np.asarray(xi).dtype)
    for i in range(n):
        for j in range(n):
            total = 0 * xi[0]
            for m in range(n):
                if m == j:
                    continue
                prod = 1 / (xi[j] - xi[m])
                for k in range(n):
                    if k == j or k == m:
                        continue
                    prod *= (xi[i] - xi[k]) / (xi[j] - xi[k])
                total += prod
            D[i, j] = total
    return D


def derivative_matrix(P):
    """The FP64 derivative matrix of order P: D of the extended nodes, rounded once."""
    xi, _ = gl_nodes_weights_ext(P)
    return lagrange_derivative_matrix(xi).astype(np.float64)


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
