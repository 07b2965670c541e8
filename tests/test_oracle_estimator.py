"""Pins for the oracle a-posteriori estimator (eqs. Eta2_Ingredients,
Eta2_Integrals, Eta2_Local): closed forms for each term's weight, zero for
solutions the discrete space holds exactly, and the 1-D second derivative
against numpy's polynomial calculus."""
import numpy as np
import pytest

from oracle import estimator, sipg, tables
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs

BOX = ((-1, -1, -1), (1, 1, 1))


def _uniform(p, warp=None):
    lv = inputs.uniform_leaves(1)
    return Mesh(*BOX, lv, [p] * len(lv) if np.isscalar(p) else p, warp=warp)


def _two_to_one(p=2, seed=None, warp=None):
    lv = inputs.refine(inputs.uniform_leaves(1), lambda lf: lf[1:] == (0, 0, 0))
    pp = [p] * len(lv) if seed is None else list(np.random.default_rng(seed).integers(2, 5, size=len(lv)))
    return Mesh(*BOX, lv, pp, warp=warp)


def _elem(m, leaf):
    return m.key[tuple(leaf)]


@pytest.mark.parametrize("n", [2, 3, 5, 9])
def test_second_derivative_matches_polynomial_calculus(n):
    xl, _ = tables.lgl_nodes_weights(n)
    x = np.linspace(-1, 1, 7)
    V = estimator.lagrange_second_derivs(xl, x)
    for a in range(n):
        y = np.zeros(n)
        y[a] = 1.0
        c = np.polynomial.polynomial.polyfit(xl, y, n - 1)
        ref = np.polynomial.polynomial.polyval(x, np.polynomial.polynomial.polyder(c, 2))
        assert np.allclose(V[:, a], ref, atol=1e-9 * max(1.0, np.abs(ref).max()))


def test_constant_source_closed_form():
    """u = 0, g = 1: R = -1, eta^2 = h_e^2 p^2 |e| = (sqrt 3)^2 * 4 * 1 = 12."""
    m = _uniform(2)
    eta = estimator.estimate(m, np.zeros(m.n_dofs), g_fn=lambda x: np.ones(len(x)))
    assert np.allclose(eta, 12.0, rtol=1e-12)


def test_indicator_conforming_closed_form():
    """u = 1 on one unit cube, 0 elsewhere (p = 2, C = 10): every face of it
    carries sigma h^-1 p^2 |m| = 40 * 4 = 160 (interior jump or Dirichlet),
    so eta^2 = 960 there and 160 on its three face neighbours."""
    m = _uniform(2)
    e0 = _elem(m, (1, 0, 0, 0))
    u = np.zeros(m.n_dofs)
    u[m.dof_off[e0]:m.dof_off[e0 + 1]] = 1.0
    eta = estimator.estimate(m, u, C=10.0)
    exp = np.zeros(m.n_elems)
    exp[e0] = 960.0
    for nb in [(1, 1, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1)]:
        exp[_elem(m, nb)] = 160.0
    assert np.allclose(eta, exp, rtol=1e-12, atol=1e-10)


def test_indicator_degree_jump_uses_mortar_degree():
    """Same with p = 3 around a p = 2 cube: its interior faces have p_m = 3,
    sigma = 10 * 9, eta_m2 = 90 * 9 = 810; its boundary faces keep p = 2."""
    m = _uniform(3)
    e0 = _elem(m, (1, 0, 0, 0))
    m = Mesh(*BOX, m.leaves, [2 if e == e0 else 3 for e in range(m.n_elems)])
    u = np.zeros(m.n_dofs)
    u[m.dof_off[e0]:m.dof_off[e0 + 1]] = 1.0
    eta = estimator.estimate(m, u, C=10.0)
    assert eta[e0] == pytest.approx(3 * 810.0 + 3 * 160.0, rel=1e-12)
    assert eta[_elem(m, (1, 1, 0, 0))] == pytest.approx(810.0, rel=1e-12)


def test_indicator_two_to_one_closed_form():
    """u = 1 on the unit cube next to a refined one: each of the 4 sub-mortars
    has h_m = 1/2 (the fine side), sigma = 10 * 4 / 0.5 = 80 and area 1/4:
    80 / 0.5 * 4 / 4 = 160 each; the cube's 5 other faces give 160 each."""
    m = _two_to_one()
    e0 = _elem(m, (1, 1, 0, 0))
    u = np.zeros(m.n_dofs)
    u[m.dof_off[e0]:m.dof_off[e0 + 1]] = 1.0
    eta = estimator.estimate(m, u, C=10.0)
    assert eta[e0] == pytest.approx(4 * 160.0 + 5 * 160.0, rel=1e-12)
    fine = [_elem(m, (2, 1, b, c)) for b in range(2) for c in range(2)]
    assert np.allclose(eta[fine], 160.0, rtol=1e-12)


def test_kink_flux_jump_closed_form():
    """u = max(x, 0): the normal derivative jumps by 1 across x = 0 and
    nothing else is nonzero: eta_m1 = h_m / p_m |m| = 1/2 for every cube."""
    m = _uniform(2)
    f = lambda x: np.maximum(x[:, 0], 0.0)
    u = sipg.interpolate(m, f)
    eta = estimator.estimate(m, u, gD_fn=f, C=10.0)
    assert np.allclose(eta, 0.5, rtol=1e-12)


def test_quadratic_solution_affine_hp_two_to_one_is_zero():
    """A quadratic solution of -Lap u + f u = g (f varying) interpolated on an
    affine mesh with 2:1 faces and degree jumps (p >= 2): every term is 0."""
    m = _two_to_one(seed=4)
    P = lambda x: 0.3 + x[:, 0] - 0.5 * x[:, 1] + 2 * x[:, 1] ** 2 - x[:, 0] * x[:, 2] + 0.7 * x[:, 2] ** 2
    f = lambda x: 1.5 + x[:, 0] ** 2
    g = lambda x: -5.4 + f(x) * P(x)
    eta = estimator.estimate(m, sipg.interpolate(m, P), g_fn=g, f_fn=f, gD_fn=P)
    ref = estimator.estimate(m, sipg.interpolate(m, lambda x: x[:, 0] ** 3), g_fn=g, f_fn=f, gD_fn=P)
    assert eta.max() < 1e-20 * ref.max()
    assert ref.min() > 0


def test_linear_solution_on_curved_elements_is_zero():
    """u linear in x lies in the isoparametric space, so Lap u_h = 0 exactly;
    this needs the second-derivative-of-the-map term of the chain rule, which
    alone is far from zero on these curved elements.  With one degree and
    conforming faces the two sides' faces coincide and the jumps vanish too;
    with 2:1 faces and degree jumps the two sides interpolate the face
    differently, so only the volume part is zero there."""
    lin = lambda x: 0.4 + 1.3 * x[:, 0] - 0.7 * x[:, 1] + 0.9 * x[:, 2]
    warp = (0.05, (1, 2, 1))
    mu = _uniform(3, warp=warp)
    assert estimator.estimate(mu, sipg.interpolate(mu, lin), gD_fn=lin).max() < 1e-20
    m = _two_to_one(seed=5, warp=warp)
    u = sipg.interpolate(m, lin)
    _, vol, mort = estimator.estimate(m, u, gD_fn=lin, parts=True)
    assert vol.max() < 1e-20
    assert mort.max() > 1.0
    # the reference-Hessian part alone (no map curvature term) on one element
    e = 3
    n = int(m.n[e])
    xl, _ = tables.lgl_nodes_weights(n)
    xi, w, J, detJ, Jinv = sipg.volume_geometry(m, e)
    d2 = np.einsum('lmpa,a->plm', estimator.basis3d_second(xl, xi), u[m.dof_off[e]:m.dof_off[e + 1]])
    naive = np.einsum('pli,plm,pmi->p', Jinv, d2, Jinv)
    assert np.abs(naive).max() > 1e-2


def test_estimator_is_local_and_additive():
    """eta^2 of a field supported on one element touches only that element
    and its face neighbours; the volume part of a sum of two such fields
    supported on distant elements is the sum of their volume parts."""
    m = _two_to_one(seed=6)
    rng = np.random.default_rng(0)
    a, b = _elem(m, (2, 0, 0, 0)), _elem(m, (1, 1, 1, 1))
    ua = np.zeros(m.n_dofs)
    ua[m.dof_off[a]:m.dof_off[a + 1]] = rng.standard_normal(m.dof_off[a + 1] - m.dof_off[a])
    ub = np.zeros(m.n_dofs)
    ub[m.dof_off[b]:m.dof_off[b + 1]] = rng.standard_normal(m.dof_off[b + 1] - m.dof_off[b])
    ea, va, _ = estimator.estimate(m, ua, parts=True)
    eb, vb, _ = estimator.estimate(m, ub, parts=True)
    _, vab, _ = estimator.estimate(m, ua + ub, parts=True)
    assert np.allclose(vab, va + vb, rtol=1e-12, atol=0)
    touched = {a} | {mm.eB if mm.eA == a else mm.eA for mm in m.mortars
                     if a in (mm.eA, mm.eB) and mm.eB is not None}
    assert set(np.nonzero(ea)[0]) == touched
