"""Pins for the puncture source terms and Newton (Sec. III.D, Alg. 1)."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import puncture, sipg
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def test_single_puncture_closed_form():
    rng = np.random.default_rng(0)
    x = rng.uniform(-5, 5, size=(50, 3))
    c = np.array([0.3, -0.2, 0.1])
    P = np.array([0.1, 0.2, -0.05])
    al, be, AA = puncture.alpha_beta(x, [(0.7, c, P)])
    r = np.linalg.norm(x - c, axis=1)
    n = (x - c) / r[:, None]
    expect = 9.0 / (2 * r ** 4) * (P @ P + 2 * (n @ P) ** 2)
    assert np.allclose(AA, expect, rtol=1e-12)
    assert np.allclose(al, 2 * r / 0.7, rtol=1e-14)
    assert np.allclose(be, al ** 7 * expect / 8, rtol=1e-12)


def _problem():
    lv = inputs.uniform_leaves(1)
    m = Mesh((-6, -6, -6), (6, 6, 6), lv, [3] * 8)
    punc = [(0.5, (3.0, 0.1, 0.05), (0, 0.2, 0)), (0.5, (-3.0, 0.1, 0.05), (0, -0.2, 0))]
    return m, puncture.PunctureProblem(m, punc)


def test_jacobian_matches_finite_difference():
    m, pr = _problem()
    rng = np.random.default_rng(1)
    u = 0.05 * rng.standard_normal(m.n_dofs)
    v = rng.standard_normal(m.n_dofs)
    J = pr.jacobian(u)
    h = 1e-5
    fd = (pr.residual(u + h * v) - pr.residual(u - h * v)) / (2 * h)
    assert np.linalg.norm(J @ v - fd) < 1e-7 * np.linalg.norm(fd)


def test_newton_quadratic_convergence():
    m, pr = _problem()

    def ls(coef, rhs):
        return spla.spsolve(sipg.assemble(m, 10.0, coef=coef).tocsc(), rhs)

    u, k, hist = puncture.newton(pr, np.zeros(m.n_dofs), ls, tol=1e-13)
    assert hist[-1] < 1e-13 and k <= 5
    # quadratic: each error roughly the square of the previous (relative to the first)
    assert hist[2] / hist[0] < (hist[1] / hist[0]) ** 1.5
