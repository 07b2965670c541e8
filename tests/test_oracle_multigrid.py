"""Pins for the oracle's multigrid pieces (Algs. 2-5, eqs. psi-interpolation,
temp-G, operator_oh)."""
import numpy as np
import pytest

from oracle import krylov, multigrid, sipg, tables
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def test_chebyshev_error_polynomial():
    """Alg. 4 (with p <- alpha r + beta p): after k steps from x = 0 each
    eigencomponent of the error is T_k((d - lam)/c) / T_k(d/c) times the initial one."""
    rng = np.random.default_rng(0)
    lmax, Lam = 4.0, 20.0
    lam = np.sort(rng.uniform(0.05, lmax, 40))
    A = np.diag(lam)
    xs = rng.standard_normal(40)
    b = A @ xs
    lmin = lmax / Lam
    c, d = (lmax - lmin) / 2, (lmax + lmin) / 2
    for k in (1, 2, 3, 7, 15):
        x = multigrid.chebyshev(A, np.zeros(40), b, lmax, Lam, k)
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        expect = Tk((d - lam) / c) / Tk(d / c) * xs
        assert np.allclose(xs - x, expect, atol=1e-10), k


def test_chebyshev_printed_sign_is_not_chebyshev():
    """The printed update p <- alpha r - beta p does not give the Chebyshev
    error polynomial (pins the reading)."""
    rng = np.random.default_rng(1)
    lam = np.sort(rng.uniform(0.2, 4.0, 30))
    A = np.diag(lam)
    xs = rng.standard_normal(30)
    b = A @ xs
    lmax, Lam = 4.0, 20.0
    lmin = lmax / Lam
    c, d = (lmax - lmin) / 2, (lmax + lmin) / 2
    x, p, alpha = np.zeros(30), np.zeros(30), 0.0
    for k in range(1, 4):
        r = b - A @ x
        alpha = 1 / d if k == 1 else (2 * d / (2 * d * d - c * c) if k == 2 else 1 / (d - alpha * c * c / 4))
        beta = alpha * d - 1
        p = alpha * r - beta * p
        x = x + p
    T3 = np.polynomial.chebyshev.Chebyshev.basis(3)
    assert not np.allclose(xs - x, T3((d - lam) / c) / T3(d / c) * xs, atol=1e-6)


def test_cgeigs_cg_iterates_and_bound():
    m = Mesh((-1, -1, -1), (1, 1, 1), inputs.uniform_leaves(1), [3] * 8)
    A = sipg.assemble(m, 10.0)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(m.n_dofs)
    lam, x = multigrid.cgeigs(A, np.zeros(m.n_dofs), b, 10)
    # textbook CG (written independently)
    xx, r = np.zeros(m.n_dofs), b.copy()
    p = r.copy()
    for _ in range(10):
        Ap = A @ p
        a = (r @ r) / (p @ Ap)
        xx = xx + a * p
        rn = r - a * Ap
        p = rn + (rn @ rn) / (r @ r) * p
        r = rn
    assert np.allclose(x, xx, rtol=1e-10, atol=1e-12)
    lmax = np.linalg.eigvalsh(A.toarray()).max()
    assert lam >= 0.8 * lmax
    lam50, _ = multigrid.cgeigs(A, np.zeros(m.n_dofs), b, 50)
    assert lam50 >= lmax * (1 - 1e-8)


def test_prolongation_exact_and_restriction_transpose():
    d = inputs.sweep_mesh(level=2, seed=0)
    a, k = inputs.oracle_mesh_args(d)
    fine = Mesh(*a, **k)
    coarse, groups = multigrid.coarsen(fine)
    P = multigrid.prolongation(fine, coarse, groups)
    # prolonging the interpolant of a polynomial of degree <= min p (= 2) reproduces it
    f = lambda x: 1 + x[:, 0] - 2 * x[:, 1] * x[:, 2] + 0.5 * x[:, 0] ** 2
    # on the unwarped mesh, nodal interpolation is exact for this quadratic
    fine0 = Mesh(fine.lo, fine.hi, fine.leaves, fine.p)
    coarse0 = Mesh(coarse.lo, coarse.hi, coarse.leaves, coarse.p)
    P0 = multigrid.prolongation(fine0, coarse0, groups)
    assert np.abs(P0 @ sipg.interpolate(coarse0, f) - sipg.interpolate(fine0, f)).max() < 1e-13
    # coarse p is the minimum of the children and all families are 2:1 balanced
    for H, grp in enumerate(groups):
        assert coarse.p[H] == min(fine.p[c] for c, _ in grp)
    assert P.shape == (fine.n_dofs, coarse.n_dofs)


def test_hierarchy_levels_and_balance():
    d = inputs.sweep_mesh(level=2, seed=0)
    a, k = inputs.oracle_mesh_args(d)
    meshes, groups = multigrid.hierarchy(Mesh(*a, **k))
    assert [m.n_elems for m in meshes] == [1, 8, 15, 120]
    # every level is a valid 2:1 mesh (Mesh construction raises otherwise)
    for m in meshes:
        assert m.n_dofs > 0


def test_galerkin_zeroth_order_identity():
    """O^H = I^T O^h I equals the coarse mass matrix assembled with the fine
    level's quadrature (eq. temp-H) -- checked through bilinear forms."""
    lv = inputs.uniform_leaves(1)
    fine = Mesh((-1, -1, -1), (1, 1, 1), lv, [2] * 8)
    coarse, groups = multigrid.coarsen(fine)
    P = multigrid.prolongation(fine, coarse, groups)
    coef = [np.full((fine.n[e]) ** 3, 1.5) for e in range(8)]
    Oh = sipg.assemble(fine, 10.0, coef=coef) - sipg.assemble(fine, 10.0)
    OH = (P.T @ Oh @ P).toarray()
    # coarse mass with constant coefficient 1.5 on the p=2 coarse element is exact
    Mc = sipg.element_mass(coarse, 0, np.full(125, 1.5), extra=2)
    assert np.abs(OH - Mc).max() < 1e-12 * np.abs(Mc).max()


def test_fcg_identity_is_cg_and_mg_solve():
    m = Mesh((-1, -1, -1), (1, 1, 1), inputs.uniform_leaves(2), [3] * 64)
    H = multigrid.Hierarchy(m)
    u = lambda x: np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])
    F = sipg.rhs(m, lambda x: 3 * np.pi ** 2 * u(x), u)
    x, it, hist = krylov.fcg(H.J[-1], F, precond=lambda r: H.vcycle(r), tol=1e-10)
    assert hist[-1] < 1e-10 and it <= 12
    r = F - H.J[-1] @ x
    assert np.linalg.norm(r) / np.linalg.norm(F) < 1e-9
    x2, it2, _ = krylov.fcg(H.J[-1], F, precond=lambda r: H.vcycle(r, coarse='cholesky'), tol=1e-10)
    assert it2 <= it + 1
    # no preconditioner: FCG(1) iterates are CG's, far more iterations
    _, it3, _ = krylov.fcg(H.J[-1], F, tol=1e-10, max_iter=1000)
    assert it3 > 5 * it


def test_element_schwarz_smoother():
    """Element-subdomain Schwarz (overlap 0): exact in one undamped cycle when
    the matrix is block diagonal; on SIPG the spectrum of the block-Jacobi
    operator lies inside (0, 2) (a convergent, damped smoother); MG-FCG with it
    reaches 1e-10."""
    import numpy as np
    import scipy.sparse as sp
    from oracle import krylov, multigrid, sipg
    from oracle.mesh import Mesh
    from paper_1907_01572_gb300 import inputs
    rng = np.random.default_rng(0)
    blocks = []
    for n in (3, 5, 4):
        B = rng.standard_normal((n, n))
        blocks.append(B @ B.T + n * np.eye(n))
    A = sp.block_diag([sp.csr_matrix(B) for B in blocks], format="csr")
    off = np.array([0, 3, 8, 12])
    b = rng.standard_normal(12)
    x = multigrid.schwarz_smoother(A, multigrid.schwarz_blocks(A, off), off, np.zeros(12), b, 1, 1.0)
    assert np.abs(A @ x - b).max() < 1e-12
    desc = inputs.sweep_mesh(level=1, seed=0)
    a, k = inputs.oracle_mesh_args(desc)
    m = Mesh(*a, **k)
    L = sipg.assemble(m, 10.0)
    inv = multigrid.schwarz_blocks(L, m.dof_off)
    Dinv = sp.block_diag([sp.csr_matrix(Ai) for Ai in inv], format="csr")
    ev = np.linalg.eigvals((Dinv @ L).toarray()).real
    assert ev.min() > 0 and ev.max() < 2
    H = multigrid.Hierarchy(m)
    f = inputs.random_vector(m.n_dofs, seed=3)
    u, its, hist = krylov.fcg(L, f, precond=lambda r: H.vcycle(r, smoother_kind="schwarz"), tol=1e-10, max_iter=100)
    assert np.linalg.norm(f - L @ u) <= 1e-10 * np.linalg.norm(f) and its < 80


def test_galerkin_coarse_operators_on_the_compactified_sphere():
    """13-block cubed sphere with the inverse-radius shell to r = 1e9 (level
    1, p = 3, two levels, exact coarse solve): with element-Schwarz
    smoothing, Galerkin coarse operators P^T J P make MG-FCG reach 1e-10,
    the re-discretised coarse level does not within the same 150 iterations.
    The Galerkin operators satisfy their definition exactly."""
    from oracle import krylov, multigrid
    from paper_1907_01572_gb300 import inputs
    levels = multigrid.uniform_block_levels(inputs.cubed_sphere_blocks(a=2.0, r=10.0, r_out=1e9), 1, 3)
    b = np.random.default_rng(0).standard_normal(levels[0][-1].n_dofs)
    its = {}
    for ops in ("galerkin", "rediscretised"):
        H = multigrid.Hierarchy(None, levels=levels, coarse_ops=ops)
        x, it, hist = krylov.fcg(H.J[-1], b, precond=lambda r: H.vcycle(r, coarse='cholesky', smoother_kind='schwarz'),
                                 tol=1e-10, max_iter=150)
        its[ops] = (it, hist[-1])
        if ops == "galerkin":
            G = (H.P[0].T @ H.J[1] @ H.P[0]).toarray()
            assert np.abs(H.J[0].toarray() - G).max() <= 1e-12 * np.abs(G).max()
    assert its["galerkin"][1] < 1e-10 and its["galerkin"][0] < 150, its
    assert its["rediscretised"][1] > 1e-9, its


def test_schwarz_weight_function():
    """eq. schwarz_weight: phi is C^2 at +-1 and odd; w_h is 1 in the core, 0
    beyond the overlap, 1/2 on the element boundary, and neighbouring
    subdomains' weights add to one across the overlap."""
    from oracle.multigrid import schwarz_phi, schwarz_weight
    t = np.linspace(-1, 1, 41)
    assert np.allclose(schwarz_phi(-t), -schwarz_phi(t))
    h = 1e-6
    for s in (-1.0, 1.0):
        assert abs(schwarz_phi(s) - s) < 1e-15
        d1 = (schwarz_phi(s + h) - schwarz_phi(s - h)) / (2 * h)
        assert abs(d1) < 1e-5
    for delta in (0.25, 0.553, 1.0):
        assert np.allclose(schwarz_weight(np.linspace(-1 + delta, 1 - delta, 9), delta), 1.0)
        assert np.allclose(schwarz_weight(np.array([1 + delta, 1.7 + delta, -1 - delta]), delta), 0.0)
        assert np.allclose(schwarz_weight(np.array([-1.0, 1.0]), delta), 0.5)
        xi = np.linspace(1 - delta, 1 + delta, 17)
        assert np.allclose(schwarz_weight(xi, delta) + schwarz_weight(xi - 2.0, delta), 1.0)


def test_overlap_subdomains_on_a_uniform_box():
    """Affine 4^3 box, p = 3, two overlap layers: an interior element's
    subdomain holds 4^3 + 6*2*16 + 12*4*4 + 8*8 = 512 nodes; its face
    neighbour's second node layer sits at xi_ext = 2 + x_1 (x_1 the second
    LGL node); the weights of every node off the domain boundary add to one
    over the subdomains that hold it."""
    from oracle import multigrid, tables
    from oracle.mesh import Mesh
    from paper_1907_01572_gb300 import inputs
    m = Mesh((0, 0, 0), (1, 1, 1), inputs.uniform_leaves(2), [3] * 64)
    subs = multigrid.overlap_subdomains(m, 2)
    e = m.key[(2, 1, 1, 1)]
    d, W = subs[e]
    assert len(d) == 512
    tot = np.zeros(m.n_dofs)
    for dd, WW in subs:
        np.add.at(tot, dd, WW)
    X = np.vstack([m.node_coords(k) for k in range(m.n_elems)])
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    assert np.allclose(tot[inner], 1.0, atol=1e-13)
    xl, _ = tables.lgl_nodes_weights(4)
    delta = 1.0 + xl[1]
    # the +x face neighbour's node (a = 1, b = c = 1) in e's subdomain
    nb = m.key[(2, 2, 1, 1)]
    j = int(m.dof_off[nb]) + 1 + 4 * 1 + 16 * 1
    k = int(np.nonzero(d == j)[0][0])
    w_expect = multigrid.schwarz_weight(2.0 + xl[1], delta) * multigrid.schwarz_weight(xl[1], delta) ** 2
    assert abs(W[k] - w_expect) < 1e-14


def test_overlapping_schwarz_on_the_compactified_sphere():
    """The paper's smoother for stretched cubed spheres: with overlapping
    subdomains (two layers, or one: the touching elements' nodes that
    coincide with e_c's boundary; weights w_h) and the re-discretised coarse
    level, MG-FCG reaches 1e-10 on the sphere with the shell to r = 1e9
    (level 1, p = 3), where the non-overlapping element smoother stalls
    (test_galerkin_coarse_operators_on_the_compactified_sphere)."""
    from oracle import krylov, multigrid
    from paper_1907_01572_gb300 import inputs
    levels = multigrid.uniform_block_levels(inputs.cubed_sphere_blocks(a=2.0, r=10.0, r_out=1e9), 1, 3)
    H = multigrid.Hierarchy(None, levels=levels)
    b = np.random.default_rng(0).standard_normal(levels[0][-1].n_dofs)
    for n_overlap, cap in ((2, 40), (1, 25)):
        if hasattr(H, "_ovl"):
            del H._ovl
        x, it, hist = krylov.fcg(H.J[-1], b, tol=1e-10, max_iter=60,
                                 precond=lambda r: H.vcycle(r, coarse='cholesky', smoother_kind='schwarz_overlap',
                                                            n_overlap=n_overlap))
        assert hist[-1] < 1e-10 and it <= cap, (n_overlap, it, hist[-1])


def test_overlap_one_layer_step_weights_and_conforming_only():
    """One overlap layer: the contact nodes lie on e_c's boundary, so the
    weights are the step values 1 / 1/2 / 1/4 / 1/8 (interior, face, edge,
    corner); a mesh with 2:1 faces is rejected with a ValueError."""
    from oracle import multigrid, tables
    from oracle.mesh import Mesh
    from paper_1907_01572_gb300 import inputs
    m = Mesh((0, 0, 0), (1, 1, 1), inputs.uniform_leaves(1), [2] * 8)
    subs = multigrid.overlap_subdomains(m, 1)
    n = 3
    xl, _ = tables.lgl_nodes_weights(n)
    for d, W in subs:
        assert set(np.round(W, 12)) <= {1.0, 0.5, 0.25, 0.125}
        own = W[:n ** 3]
        for k in range(n ** 3):
            a, b, c = k % n, (k // n) % n, k // (n * n)
            on = sum(int(i in (0, n - 1)) for i in (a, b, c))
            assert abs(own[k] - 0.5 ** on) < 1e-12
    lv = inputs.refine(inputs.uniform_leaves(1), lambda lf: lf == (1, 0, 0, 0))
    with pytest.raises(ValueError):
        multigrid.overlap_subdomains(Mesh((0, 0, 0), (1, 1, 1), lv, [2] * len(lv)), 1)


def test_overlap_one_layer_partition_of_unity_and_single_element():
    """One overlap layer on a conforming box: the weights of all subdomains
    holding a DOF add up to 1 wherever the DOF's position is not on the domain
    boundary (a node on a face, edge or corner is shared by 2, 4 or 8 elements,
    each weighting it 1/2, 1/4 or 1/8), and on a single element one cycle from
    x = 0 is W A^-1 b (its subdomain is the element itself)."""
    m = Mesh((0, 0, 0), (1, 1, 1), inputs.uniform_leaves(1), [2] * 8)
    subs = multigrid.overlap_subdomains(m, 1)
    tot = np.zeros(m.n_dofs)
    for d, W in subs:
        np.add.at(tot, d, W)
    X = np.vstack([m.node_coords(e) for e in range(m.n_elems)])
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    assert inner.sum() > 0 and np.allclose(tot[inner], 1.0, atol=1e-14)
    assert np.all(tot[~inner] < 1.0)
    one = Mesh((0, 0, 0), (1, 1, 1), [(0, 0, 0, 0)], [3])
    A = sipg.assemble(one, 10.0)
    (d, W), = multigrid.overlap_subdomains(one, 1)
    b = np.random.default_rng(4).standard_normal(one.n_dofs)
    x = multigrid.overlap_schwarz_smoother(A, [(d, W)], np.zeros_like(b), b, n_cycles=1)
    assert np.allclose(x, W * np.linalg.solve(A.toarray(), b), rtol=1e-10, atol=1e-12)
