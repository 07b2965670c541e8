"""Pins of the oracle's V-cycle (Alg. 3), flexible CG (Alg. 2) and CG
eigenvalue bound (Alg. 5, eq. tridiag) against definitions that do not come
from the oracle itself: the V-cycle's closed form built from explicit
matrices, textbook CG / preconditioned CG iterates, and an independent
Lanczos run.  Each pin is shown to fail on a planted mistake in the oracle."""
import types

import numpy as np
import pytest

from oracle import krylov, multigrid, sipg
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def _mesh(levels):
    """levels = 2: a curved 2x2x2 mesh with p in 2..4 (one coarsening step);
    3: the curved sweep mesh with one refined octant (15 elements), p in 2..4."""
    if levels == 3:
        a, k = inputs.oracle_mesh_args(inputs.sweep_mesh(level=1, seed=0, pmin=2, pmax=4))
        return Mesh(*a, **k)
    d = inputs.sweep_mesh(level=1, seed=0, pmin=2, pmax=4, refine_octant=False)
    a, k = inputs.oracle_mesh_args(d)
    return Mesh(*a, **k)


_H = {}


def hier(level):
    if level not in _H:
        _H[level] = multigrid.Hierarchy(_mesh(level))
    return _H[level]


def cheb_error_matrix(A, lam, Lam, k):
    """R = T_k(Z) / T_k(d / c), Z = (d I - A) / c: the error propagation of k
    Chebyshev steps on [lam / Lam, lam] (textbook three-term recurrence of
    the Chebyshev polynomials, evaluated on the matrix)."""
    lmin = lam / Lam
    c, d = (lam - lmin) / 2, (lam + lmin) / 2
    n = A.shape[0]
    Z = (d * np.eye(n) - A) / c
    T0, T1 = np.eye(n), Z
    t0, t1 = 1.0, d / c
    for _ in range(k - 1):
        T0, T1 = T1, 2 * Z @ T1 - T0
        t0, t1 = t1, 2 * (d / c) * t1 - t0
    return (T1 if k >= 1 else T0) / (t1 if k >= 1 else t0)


def closed_form_vcycle(H, f, lams, Lam, k, coarse):
    """Alg. 3 written as matrices: S_l(x, b) = R_l x + (I - R_l) J_l^-1 b;
    down: v_l = S_l(0, f_l), f_{l-1} = P^T (f_l - J_l v_l); level 0: J_0^-1 f_0
    (cholesky) or S_0(0, f_0); up: v_l = S_l(v_l + P v_{l-1}, f_l)."""
    J = [H.J[l].toarray() for l in range(H.n_levels)]
    P = [H.P[l].toarray() for l in range(H.n_levels - 1)]
    R = [cheb_error_matrix(J[l], lams[l], Lam, k) for l in range(H.n_levels)]
    Jinv = [np.linalg.inv(Jl) for Jl in J]

    def S(l, x, b):
        return R[l] @ x + (np.eye(len(b)) - R[l]) @ (Jinv[l] @ b)

    def V(l, fl):
        if l == 0:
            return Jinv[0] @ fl if coarse == 'cholesky' else S(0, np.zeros_like(fl), fl)
        v = S(l, np.zeros_like(fl), fl)
        vc = V(l - 1, P[l - 1].T @ (fl - J[l] @ v))
        return S(l, v + P[l - 1] @ vc, fl)

    return V(H.n_levels - 1, f)


def level_lams(H):
    return [1.05 * np.linalg.eigvalsh(H.J[l].toarray()).max() for l in range(H.n_levels)]


@pytest.mark.parametrize("levels", [2, 3])
@pytest.mark.parametrize("coarse", ["cholesky", "smoother"])
def test_vcycle_equals_closed_form(levels, coarse):
    """Fixed-lambda Chebyshev smoothing (linear) on 2 and 3 levels, both
    coarse solves: the oracle's V-cycle equals the matrix closed form."""
    H = hier(levels)
    assert H.n_levels == levels
    f = inputs.random_vector(H.meshes[-1].n_dofs, seed=31)
    lams = level_lams(H)
    for k in (3, 8):
        v = H.vcycle(f, n_cheb=k, Lam=20.0, coarse=coarse, lam_fixed=lams)
        ve = closed_form_vcycle(H, f, lams, 20.0, k, coarse)
        assert np.linalg.norm(v - ve) <= 1e-10 * np.linalg.norm(ve), k


def _planted(monkeypatch, H, kind):
    if kind == "no_post_smooth":
        orig = multigrid.chebyshev

        def cheb(A, x, b, lam, Lam, n):
            return x.copy() if np.any(x) else orig(A, x, b, lam, Lam, n)   # skips smoothing from v != 0

        monkeypatch.setattr(multigrid, "chebyshev", cheb)
    elif kind == "restrict_f":
        monkeypatch.setattr(multigrid.Hierarchy, "residual", lambda self, l, f, v: f)
    elif kind == "no_plus_v":
        monkeypatch.setattr(multigrid.Hierarchy, "coarse_correction", lambda self, l, v, vc: self.prolong(l, vc))


@pytest.mark.parametrize("kind", ["no_post_smooth", "restrict_f", "no_plus_v"])
def test_vcycle_closed_form_catches_planted_mistakes(monkeypatch, kind):
    H = hier(3)
    f = inputs.random_vector(H.meshes[-1].n_dofs, seed=31)
    lams = level_lams(H)
    ve = closed_form_vcycle(H, f, lams, 20.0, 5, "cholesky")
    _planted(monkeypatch, H, kind)
    v = H.vcycle(f, n_cheb=5, Lam=20.0, coarse="cholesky", lam_fixed=lams)
    assert np.linalg.norm(v - ve) > 1e-3 * np.linalg.norm(ve), kind


def _system():
    m = _mesh(3)
    A = sipg.assemble(m, 10.0)
    b = inputs.random_vector(m.n_dofs, seed=5)
    return m, A, b


def test_fcg_iterates_equal_textbook_cg_and_pcg():
    """Alg. 2 without a preconditioner produces CG's iterates; with a fixed
    SPD preconditioner (the inverse element diagonal blocks) PCG's."""
    m, A, b = _system()
    for precond in (None, "blockjacobi"):
        if precond is None:
            Minv = lambda r: r.copy()
            pc = None
        else:
            inv = multigrid.schwarz_blocks(A, m.dof_off)

            def Minv(r):
                z = np.empty_like(r)
                for e, Ai in enumerate(inv):
                    sl = slice(m.dof_off[e], m.dof_off[e + 1])
                    z[sl] = Ai @ r[sl]
                return z
            pc = Minv
        xs = {}
        krylov.fcg(A, b, precond=pc, tol=1e-12, max_iter=25, callback=lambda k, x: xs.__setitem__(k, x.copy()))
        # textbook preconditioned CG (M = I gives plain CG)
        x = np.zeros_like(b)
        r = b.copy()
        z = Minv(r)
        p = z.copy()
        rz = r @ z
        for k in range(1, 26):
            if k not in xs:
                break
            Ap = A @ p
            a = rz / (p @ Ap)
            x = x + a * p
            r = r - a * Ap
            z = Minv(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
            assert np.linalg.norm(xs[k] - x) <= 1e-8 * np.linalg.norm(x), (precond, k)
        assert len(xs) > 10


def lanczos(A, q1, k):
    """k steps of Lanczos (full reorthogonalisation): diagonal alpha_j and
    off-diagonal beta_j (> 0) of the tridiagonal T."""
    Q = [q1 / np.linalg.norm(q1)]
    al, be = [], []
    for j in range(k):
        w = A @ Q[j]
        al.append(Q[j] @ w)
        for q in Q:
            w = w - (q @ w) * q
        for q in Q:
            w = w - (q @ w) * q
        be.append(np.linalg.norm(w))
        Q.append(w / be[-1])
    return np.array(al), np.array(be)


def test_cgeigs_tridiagonal_equals_lanczos():
    """Alg. 5 / eq. tridiag: the tridiagonal built from the CG coefficients is
    Lanczos's T for the starting vector r_0; lambda_max is the largest
    Gershgorin row bound of it, which bounds every Ritz value from above."""
    m, A, b = _system()
    K = 12
    tr = []
    lam, _ = multigrid.cgeigs(A, np.zeros_like(b), b, K, trace=tr)
    al, be = lanczos(A, b, K)
    diag = np.array([t[0] for t in tr])
    off = np.array([t[1] for t in tr])
    assert np.allclose(diag, al, rtol=1e-8)
    assert np.allclose(off, be, rtol=1e-7)
    rows = al + be + np.concatenate([[0.0], be[:-1]])
    assert abs(lam - rows.max()) <= 1e-8 * lam
    T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    ritz = np.linalg.eigvalsh(T)
    assert ritz.max() <= lam and ritz.max() <= np.linalg.eigvalsh(A.toarray()).max() * (1 + 1e-10)


def test_cgeigs_catches_planted_offdiagonal(monkeypatch):
    """A planted beta_k in place of sqrt(beta_k) / alpha_k for the off-diagonal
    fails the Lanczos comparison."""
    m, A, b = _system()
    al, be = lanczos(A, b, 8)
    fake = types.SimpleNamespace(**{k: getattr(np, k) for k in dir(np) if not k.startswith("__")})
    fake.sqrt = lambda v: v * 1.0
    monkeypatch.setattr(multigrid, "np", fake)
    tr = []
    multigrid.cgeigs(A, np.zeros_like(b), b, 8, trace=tr)
    off = np.array([t[1] for t in tr])
    assert not np.allclose(off, be, rtol=1e-3)
