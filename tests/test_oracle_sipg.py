"""Pins for the oracle SIPG operator (eqs. lh2, equationFh2, penaltyparameter)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import sipg
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def _mixed_mesh(warp=None, seed=3, pmin=2, pmax=5):
    lv = inputs.refine(inputs.uniform_leaves(1), lambda lf: lf[1] == 0 and lf[2] == 0 and lf[3] == 0)
    p = np.random.default_rng(seed).integers(pmin, pmax + 1, size=len(lv))
    return Mesh((-1, -1, -1), (1, 1, 1), lv, p, warp=warp)


@pytest.mark.parametrize("warp", [None, (0.00625, (1, 2, 3))])
def test_symmetric_positive_definite(warp):
    m = _mixed_mesh(warp=warp, pmax=4)
    A = sipg.assemble(m, 10.0).toarray()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_spd_small_meshes_all_degrees(p):
    for leaves in ([(0, 0, 0, 0)], inputs.uniform_leaves(1)):
        m = Mesh((0, 0, 0), (1, 1, 1), leaves, [p] * len(leaves))
        A = sipg.assemble(m, 10.0).toarray()
        assert np.linalg.eigvalsh(A).min() > 0


def test_patch_test_affine_2to1_pjumps():
    """SIPG consistency: the interpolant of a quadratic u solves L u = F exactly
    on an affine mesh with 2:1 faces and degree jumps (all p >= 2)."""
    m = _mixed_mesh()
    A = sipg.assemble(m, 10.0)
    u = lambda x: x[:, 0] ** 2 + 0.5 * x[:, 1] * x[:, 2] - 0.3 * x[:, 2] + 1.0
    g = lambda x: -2.0 * np.ones(len(x))
    F = sipg.rhs(m, g, u, 10.0)
    uI = sipg.interpolate(m, u)
    assert np.abs(A @ uI - F).max() < 1e-12 * np.abs(F).max()


def test_patch_test_catches_planted_normal_sign(monkeypatch):
    """Plant a flipped normal in the oracle's face terms: the patch test fails."""
    m = _mixed_mesh()
    orig = sipg.MortarData.__init__

    def bad_init(self, *a, **k):
        orig(self, *a, **k)
        self.dn = [-d for d in self.dn]

    monkeypatch.setattr(sipg.MortarData, "__init__", bad_init)
    A = sipg.assemble(m, 10.0)
    u = lambda x: x[:, 0] ** 2 + 0.5 * x[:, 1] * x[:, 2] - 0.3 * x[:, 2] + 1.0
    F = sipg.rhs(m, lambda x: -2.0 * np.ones(len(x)), u, 10.0)
    assert np.abs(A @ sipg.interpolate(m, u) - F).max() > 1e-3 * np.abs(F).max()


def test_penalty_closed_form():
    """sigma = C p_m^2 / h_m with h_m the smaller element width at the face."""
    m = _mixed_mesh()
    for mi, mm in enumerate(m.mortars):
        md = sipg.MortarData(m, mi, 7.0)
        widths = [2.0 / 2 ** m.leaves[mm.eA][0]]
        if mm.eB is not None:
            widths.append(2.0 / 2 ** m.leaves[mm.eB][0])
        assert abs(md.sigma - 7.0 * mm.pm ** 2 / min(widths)) < 1e-12 * md.sigma


def test_apply_local_matches_assembly():
    m = _mixed_mesh(warp=(0.00625, (2, 1, 3)))
    A = sipg.assemble(m, 10.0)
    x = np.random.default_rng(1).standard_normal(m.n_dofs)
    y = sipg.apply_local(m, x, 10.0)
    assert np.abs(y - A @ x).max() < 1e-12 * np.abs(y).max()
    part = sipg.apply_local(m, x, 10.0, elems=[0, 5, 14])
    for e, ye in part.items():
        assert np.abs(ye - y[m.dof_off[e]:m.dof_off[e + 1]]).max() < 1e-12 * np.abs(y).max()


def test_convergence_rate_poisson():
    """L2 error of the Poisson problem with u = sin(pi x) sin(pi y) sin(pi z),
    p = 3: rate h^(p+1) = 4 between 2^3 and 4^3 elements (Sec. II.F.1)."""
    u = lambda x: np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])
    g = lambda x: 3 * np.pi ** 2 * u(x)
    errs = []
    for L in (1, 2):
        lv = inputs.uniform_leaves(L)
        m = Mesh((-1, -1, -1), (1, 1, 1), lv, [3] * len(lv))
        A = sipg.assemble(m, 10.0)
        uh = spla.spsolve(A.tocsc(), sipg.rhs(m, g, u, 10.0))
        errs.append(sipg.l2_error(m, uh, u))
    rate = np.log2(errs[0] / errs[1])
    assert 3.6 < rate < 4.6, rate
    assert errs[1] < 4e-3
