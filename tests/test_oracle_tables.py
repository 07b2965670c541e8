"""Pins for the oracle's 1-D tables (Sec. II.A.3, II.A.5)."""
import os

import numpy as np
import pytest

from oracle import tables

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lgl_mortar_figure.txt")


def test_lgl_closed_forms():
    x, w = tables.lgl_nodes_weights(2)
    assert np.allclose(x, [-1, 1]) and np.allclose(w, [1, 1])
    x, w = tables.lgl_nodes_weights(3)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-14)
    x, w = tables.lgl_nodes_weights(5)
    s = np.sqrt(3 / 7)
    assert np.allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-14)


def test_lgl_nodes_drawn_in_mortar_figure():
    """Node positions of the mortar figure (degrees 3, 4, 6), 6-digit drawing."""
    for line in open(GOLD):
        if line.startswith('#') or not line.strip():
            continue
        v = [float(t) for t in line.split()]
        p, lo, hi, pts = int(v[0]), v[1], v[2], np.array(v[3:])
        a, b = lo + 0.041667, hi - 0.041667
        ref = 2 * (pts - a) / (b - a) - 1
        x, _ = tables.lgl_nodes_weights(p + 1)
        assert np.allclose(x, ref, atol=2e-5), (p, x, ref)


@pytest.mark.parametrize("n", range(2, 11))
def test_quadrature_exactness(n):
    xl, wl = tables.lgl_nodes_weights(n)
    xg, wg = tables.gl_nodes_weights(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        if k <= 2 * n - 3:
            assert abs(wl @ xl ** k - exact) < 1e-13
        assert abs(wg @ xg ** k - exact) < 1e-13
    # LGL is not exact at degree 2n - 2 (pins that the rule really is Lobatto)
    k = 2 * n - 2
    assert abs(wl @ xl ** k - 2.0 / (k + 1)) > 1e-6


def test_gl_two_points():
    x, w = tables.gl_nodes_weights(2)
    assert np.allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)]) and np.allclose(w, [1, 1])


@pytest.mark.parametrize("n", range(2, 10))
def test_lagrange_interpolation_and_derivative(n):
    xl, _ = tables.lgl_nodes_weights(n)
    t = np.linspace(-1, 1, 17)
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n)            # polynomial of degree n - 1
    f = np.polynomial.polynomial.polyval
    df = np.polynomial.polynomial.polyder(c)
    V = tables.lagrange_values(xl, t)
    D = tables.lagrange_derivs(xl, t)
    assert np.allclose(V @ f(xl, c), f(t, c), atol=1e-12)
    assert np.allclose(D @ f(xl, c), f(t, df), atol=1e-10)
    assert np.allclose(tables.lagrange_values(xl, xl), np.eye(n), atol=1e-14)
    # derivative of a constant is zero (rows sum to 0)
    assert np.allclose(D.sum(axis=1), 0, atol=1e-11)


def test_basis3d_partition_of_unity_and_gradient():
    xl, _ = tables.lgl_nodes_weights(4)
    rng = np.random.default_rng(0)
    xi = rng.uniform(-1, 1, size=(11, 3))
    Psi, dPsi = tables.basis3d(xl, xi)
    assert np.allclose(Psi.sum(axis=1), 1.0)
    nodes = tables.tensor_points(xl)
    f = lambda x: x[:, 0] ** 2 * x[:, 1] - 3 * x[:, 2] ** 3 + x[:, 0] * x[:, 1] * x[:, 2]
    grad = lambda x: np.stack([2 * x[:, 0] * x[:, 1] + x[:, 1] * x[:, 2],
                               x[:, 0] ** 2 + x[:, 0] * x[:, 2],
                               -9 * x[:, 2] ** 2 + x[:, 0] * x[:, 1]], axis=1)
    assert np.allclose(Psi @ f(nodes), f(xi), atol=1e-12)
    for l in range(3):
        assert np.allclose(dPsi[l] @ f(nodes), grad(xi)[:, l], atol=1e-11)
