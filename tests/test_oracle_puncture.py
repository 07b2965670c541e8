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


def test_spinning_puncture_closed_form():
    """A spin alone: A_ij = 3 / r^3 (n_i (S x n)_j + n_j (S x n)_i), so
    A_ij A^ij = 18 |S x n|^2 / r^6 = 18 (|S|^2 - (S.n)^2) / r^6."""
    rng = np.random.default_rng(3)
    x = rng.uniform(-5, 5, size=(50, 3))
    c = np.array([0.3, -0.2, 0.1])
    S = np.array([0.05, -0.02, 0.07])
    _, _, AA = puncture.alpha_beta(x, [(0.7, c, (0.0, 0.0, 0.0), S)])
    r = np.linalg.norm(x - c, axis=1)
    n = (x - c) / r[:, None]
    assert np.allclose(AA, 18.0 * (S @ S - (n @ S) ** 2) / r ** 6, rtol=1e-12)
    # a spin along the line of sight contributes nothing there
    _, _, AA0 = puncture.alpha_beta(c[None] + np.array([[0.0, 0.0, 2.0]]), [(0.7, c, (0, 0, 0), (0, 0, 0.3))])
    assert AA0[0] < 1e-30


def test_extrinsic_curvature_symmetric_traceless_divergence_free():
    """Momenta and spins of the paper's three-puncture table together:
    A_ij is symmetric and traceless, and d_j A_ij = 0 (flat momentum
    constraint) by fourth-order central differences."""
    punc = inputs.table_punctures()
    rng = np.random.default_rng(4)
    x = rng.uniform(-4, 4, size=(40, 3)) + np.array([0.0, 0.0, 0.5])
    A, _ = puncture.extrinsic_curvature(x, punc)
    assert np.abs(A - A.transpose(0, 2, 1)).max() < 1e-15 * np.abs(A).max()
    assert np.abs(np.einsum('pii->p', A)).max() < 1e-14 * np.abs(A).max()
    h = 1e-3
    div = np.zeros((len(x), 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        Ap2, _ = puncture.extrinsic_curvature(x + 2 * e, punc)
        Ap1, _ = puncture.extrinsic_curvature(x + e, punc)
        Am1, _ = puncture.extrinsic_curvature(x - e, punc)
        Am2, _ = puncture.extrinsic_curvature(x - 2 * e, punc)
        div += (-Ap2[:, :, j] + 8 * Ap1[:, :, j] - 8 * Am1[:, :, j] + Am2[:, :, j]) / (12 * h)
    scale = np.abs(A).max(axis=(1, 2)) / np.min([np.linalg.norm(x - np.asarray(pu[1]), axis=1) for pu in punc], axis=0)
    assert np.all(np.abs(div).max(axis=1) < 1e-7 * scale)
    # a wrongly scaled spin term breaks the constraint only when it is not divergence-free on
    # its own; the momentum and spin terms must each be divergence-free:
    for pu in punc:
        for part in ((pu[0], pu[1], pu[2]), (pu[0], pu[1], (0.0, 0.0, 0.0), pu[3])):
            d = np.zeros((len(x), 3))
            for j in range(3):
                e = np.zeros(3)
                e[j] = h
                d += (puncture.extrinsic_curvature(x + e, [part])[0][:, :, j]
                      - puncture.extrinsic_curvature(x - e, [part])[0][:, :, j]) / (2 * h)
            a = np.abs(puncture.extrinsic_curvature(x, [part])[0]).max()
            assert np.abs(d).max() < 1e-4 * a


def test_momentum_and_spin_cross_term_closed_form():
    """One puncture with both: the cross term 2 A^P : A^S = 18 P.(S x n) / r^5
    fixes the orientation of the spin term relative to the momentum term."""
    rng = np.random.default_rng(6)
    x = rng.uniform(-5, 5, size=(50, 3))
    c = np.array([0.1, 0.2, -0.3])
    P = np.array([0.1, -0.2, 0.05])
    S = np.array([-0.03, 0.04, 0.08])
    _, _, AA = puncture.alpha_beta(x, [(0.5, c, P, S)])
    r = np.linalg.norm(x - c, axis=1)
    n = (x - c) / r[:, None]
    expect = (9.0 / (2 * r ** 4) * (P @ P + 2 * (n @ P) ** 2) + 18.0 * (S @ S - (n @ S) ** 2) / r ** 6
              + 18.0 * (np.cross(S[None], n) @ P) / r ** 5)
    assert np.allclose(AA, expect, rtol=1e-12)
