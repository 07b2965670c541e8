"""1-D nodal tables (oracle; test infrastructure only).

Sec. II.A.3 (basis functions): Legendre-Gauss-Lobatto (LGL) collocation
points xi_alpha and the Lagrange polynomials l_alpha built on them
(eq. Lagrange_Basis).  Sec. II.A.5 (quadrature): Gauss-Legendre (GL)
abscissas/weights and the interpolation matrix I_{sigma alpha} =
psi_alpha(xi_GL^sigma).

Pins: closed-form LGL nodes/weights for p = 1, 2, 4, the LGL node positions
drawn in the mortar figure (Sec. II.A.5), quadrature exactness, Lagrange
interpolation/derivative exactness on polynomials (tests/test_oracle_tables.py).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def lgl_nodes_weights(n):
    """LGL points and weights for n = p + 1 points on [-1, 1].

    Nodes: -1, +1 and the roots of P_p'(x); weights 2 / (p (p+1) P_p(x_i)^2).
    Roots come from numpy's Legendre-series root finder and are polished
    with Newton steps on P_p'.
    """
    if n < 2:
        raise ValueError("LGL needs at least 2 points")
    N = n - 1
    c = np.zeros(N + 1)
    c[N] = 1.0
    dc = npleg.legder(c)
    if N == 1:
        inner = np.zeros(0)
    else:
        inner = np.sort(npleg.legroots(dc).real)
        ddc = npleg.legder(dc)
        for _ in range(4):
            inner = inner - npleg.legval(inner, dc) / npleg.legval(inner, ddc)
    x = np.concatenate([[-1.0], inner, [1.0]])
    PN = npleg.legval(x, c)
    w = 2.0 / (N * (N + 1) * PN ** 2)
    return x, w


def gl_nodes_weights(q):
    """Gauss-Legendre rule with q points (numpy's leggauss)."""
    x, w = npleg.leggauss(q)
    return x, w


def lagrange_values(nodes, x):
    """V[i, a] = l_a(x_i), product formula of Sec. II.A.3."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    for a in range(n):
        for m in range(n):
            if m != a:
                V[:, a] *= (x - nodes[m]) / (nodes[a] - nodes[m])
    return V


def lagrange_derivs(nodes, x):
    """V[i, a] = l_a'(x_i), product rule applied to the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.zeros((len(x), n))
    for a in range(n):
        for m in range(n):
            if m == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[m]))
            for k in range(n):
                if k != a and k != m:
                    term *= (x - nodes[k]) / (nodes[a] - nodes[k])
            V[:, a] += term
    return V


def basis3d(nodes, xi):
    """Tensor-product nodal basis psi_alpha (eq. Lagrange_Basis) and its
    reference gradient at arbitrary reference points.

    xi: (P, 3) reference coordinates.  Node index alpha = a + n b + n^2 c
    (first coordinate fastest).  Returns (Psi (P, n^3), dPsi (3, P, n^3)).
    """
    xi = np.asarray(xi, dtype=np.float64).reshape(-1, 3)
    n = len(nodes)
    L = [lagrange_values(nodes, xi[:, d]) for d in range(3)]
    dL = [lagrange_derivs(nodes, xi[:, d]) for d in range(3)]
    P = xi.shape[0]

    def kron3(A, B, C):
        return np.einsum('pa,pb,pc->pcba', A, B, C).reshape(P, n ** 3)

    Psi = kron3(L[0], L[1], L[2])
    dPsi = np.stack([kron3(dL[0], L[1], L[2]),
                     kron3(L[0], dL[1], L[2]),
                     kron3(L[0], L[1], dL[2])])
    return Psi, dPsi


def tensor_points(x1):
    """All (x1[i], x1[j], x1[k]) with the first coordinate fastest."""
    n = len(x1)
    c, b, a = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing='ij')
    return np.stack([x1[a.ravel()], x1[b.ravel()], x1[c.ravel()]], axis=1)


def tensor_weights(w1):
    return np.einsum('c,b,a->cba', w1, w1, w1).ravel()
