"""Pins of the constant-density star (Sec. III.C): the closed form against the
PDE and its matching conditions, and the oracle's power-law-source Newton
(oracle/puncture.py PowerSourceProblem) against the closed form."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import puncture, sipg
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def radial(psi, r):
    return psi(np.column_stack([r, 0.3 * 0 * r, 0 * r]))


def test_closed_form_solves_the_pde_and_matches_at_the_surface():
    st = inputs.constant_density_star(rho0=1e-3, r0=1.0)
    # a from psi' continuous at r0: rho0 r0^2 = 3 a^10 / (2 pi (1 + a^2)^6)
    a = st["a"]
    assert abs(3 * a ** 10 / (2 * np.pi * (1 + a * a) ** 6) - 1e-3) < 1e-15
    h = 1e-4
    for r in (0.2, 0.5, 0.9, 1.3, 3.0, 7.0):
        f = lambda rr: radial(st["psi"], np.array([rr]))[0]
        lap = (f(r + h) - 2 * f(r) + f(r - h)) / h ** 2 + (2 / r) * (f(r + h) - f(r - h)) / (2 * h)
        rho = 1e-3 if r < 1.0 else 0.0
        assert abs(lap + 2 * np.pi * rho * f(r) ** 5) < 1e-6 * max(1.0, abs(lap))
    # psi and psi' continuous at r0; psi -> 1 far away
    f = lambda rr: radial(st["psi"], np.array([rr]))[0]
    assert abs(f(1 - 1e-9) - f(1 + 1e-9)) < 1e-8
    h = 1e-4   # second-order one-sided differences on each side of r0
    x0 = 1.0 - 1e-12
    dl = (3 * f(x0) - 4 * f(x0 - h) + f(x0 - 2 * h)) / (2 * h)
    x1 = 1.0 + 1e-12
    dr = (-3 * f(x1) + 4 * f(x1 + h) - f(x1 + 2 * h)) / (2 * h)
    assert abs(dl - dr) < 1e-6 * abs(dl)
    assert abs(f(1e8) - 1.0) < 1e-6
    assert 1.0 < f(0.0) < 1.1 and st["a"] > np.sqrt(5.0)     # weak-field branch


def _solve(desc, st):
    m = Mesh(desc["lo"], desc["hi"], desc["leaves"], desc["p"])
    F = sipg.rhs(m, lambda x: np.zeros(len(x)), st["psi"], 10.0)
    prob = puncture.PowerSourceProblem(m, st["coef"], 5, F)

    def ls(coef, rhs):
        # J = L + blockdiag(int coef psi_a psi_b): L is assembled once by the problem
        M = sp.block_diag([sp.csr_matrix(sipg.element_mass(m, e, coef[e])) for e in range(m.n_elems)], format="csr")
        x, info = spla.cg(prob.L + M, rhs, rtol=1e-14, maxiter=20000)
        assert info == 0
        return x

    u, k, hist = puncture.newton(prob, np.ones(m.n_dofs), ls, tol=1e-11 * np.linalg.norm(F))
    return m, prob, u, k, hist


def test_newton_converges_quadratically_and_to_the_closed_form():
    """Newton from psi = 1 reaches the weak-field solution in two quadratic
    steps; the L2 error against the closed form falls under h-refinement of
    the cells cut by the star surface (the density jump inside elements makes
    the p-direction non-monotone, so it is not used)."""
    st = inputs.constant_density_star()
    errs = {}
    for refine, p in ((0, 4), (1, 4)):
        desc = inputs.const_star_mesh(level=2, refine=refine, p=p)
        m, prob, u, k, hist = _solve(desc, st)
        assert k <= 4 and hist[-1] < 1e-10 * hist[0]
        assert hist[1] < 1e-4 * hist[0]                 # quadratic: 1e-1 -> 1e-6 -> round-off
        errs[(refine, p)] = sipg.l2_error(m, u, st["psi"], extra=3)
    assert errs[(1, 4)] < 0.8 * errs[(0, 4)] and errs[(1, 4)] < 4e-3


def test_jacobian_matches_finite_differences():
    st = inputs.constant_density_star(rho0=0.02)
    desc = inputs.const_star_mesh(level=1, refine=1, p=3)
    m = Mesh(desc["lo"], desc["hi"], desc["leaves"], desc["p"])
    F = sipg.rhs(m, lambda x: np.zeros(len(x)), st["psi"], 10.0)
    prob = puncture.PowerSourceProblem(m, st["coef"], 5, F)
    rng = np.random.default_rng(0)
    u = 1.0 + 0.1 * rng.standard_normal(m.n_dofs)
    v = rng.standard_normal(m.n_dofs)
    Jv = sipg.assemble(m, 10.0, coef=prob.jacobian_coef(u)) @ v
    eps = 1e-6
    fd = (prob.residual(u + eps * v) - prob.residual(u - eps * v)) / (2 * eps)
    assert np.linalg.norm(Jv - fd) < 1e-6 * np.linalg.norm(fd)


def test_lorentzian_closed_form_and_sign():
    """Problem C's Lorentzian u = (1 + r^2)^(-1/2): -Lap u equals the source
    3 (1 + r^2)^(-5/2) (central differences in all three directions at random
    points), so the printed +3 on the Laplacian side is a sign slip (reading
    A2: the coercive form -Lap u = g is solved)."""
    rng = np.random.default_rng(3)
    X = rng.uniform(-3, 3, (20, 3))
    h = 1e-3
    u = inputs.lorentzian_solution
    lap = -6 * u(X)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        lap = lap + u(X + e) + u(X - e)
    lap /= h * h
    g = inputs.lorentzian_source(X)
    assert np.abs(-lap - g).max() < 1e-5 * np.abs(g).max()
    assert np.abs(lap - g).max() > 0.5 * np.abs(g).max()      # the printed sign does not hold
