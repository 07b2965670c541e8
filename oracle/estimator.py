"""A-posteriori error estimator eta^2(e) (oracle; test infrastructure only).

Sec. II.D (a posteriori error estimator), eqs. (Eta2_Ingredients),
(Eta2_Integrals) and (Eta2_Local), for the linear model problem
-Lap u + f u = g with Dirichlet data g_D, i.e. the flux a = grad u and the
lower-order part f u - g of the estimator's problem class (eq.
classofproblems).  Per element e and mortar m:

  R_e     = f u_h - g - Lap u_h                    (element residual)
  J_{m,1} = [[grad u_h]] . n = (grad u_A - grad u_B) . n_A   (interior m)
  J_{m,2} = [[u_h]] = u_A - u_B                                (interior m)
  J_{m,3} = u_A - g_D                                         (Dirichlet m)

  eta^2_e     = h_e^2 p_e^2 ||R_e||^2_{0,e}
  eta^2_{m,1} = h_m p_m^-1 ||J_{m,1}||^2_{0,m}
  eta^2_{m,2} = sigma h_m^-1 p_m^2 ||J_{m,2}||^2_{0,m}
  eta^2_{m,3} = sigma h_m^-1 p_m^2 ||J_{m,3}||^2_{0,m}

  eta^2(e) = eta^2_e + sum over the mortars touching e of their terms.

Lap u_h is the exact Laplacian of the mapped polynomial u_h(x(xi)): with
J = dx/dxi, H_xi the reference Hessian of u_h and X^k_{lm} = d^2 x_k / dxi_l dxi_m,
  Hess_x u = J^-T (H_xi - sum_k (du/dx_k) X^k) J^-1,   Lap u = trace,
where x(xi) is the element's geometry: the isoparametric interpolant on
single-box meshes, the exact block map on multi-block meshes (whose J the
operator uses too; X^k its second derivatives).

Fiducial grid (Sec. II.D, the fiducial-grid paragraph; Problem C's
compactified grid): with `fiducial`, a mesh of identical structure and
connectivity on other block maps, the integrands R_e, J_{m,.} stay those of
the physical grid while the integration weights (w det J, w S^m) and h_e, h_m
and sigma come from the fiducial grid.
Every quantity is evaluated at the element's GL points (p + 1 per direction)
and the mortar's GL points (p_m + 1 per direction), the quadrature of the
operator itself.

Readings (where the paper leaves the choice open or prints something odd):
 * The weights are taken exactly as printed in eq. (Eta2_Integrals)
   (h_e^2 p_e^2 on the residual, sigma h_m^-1 p_m^2 on the jumps), although
   residual estimators in the cited literature scale the residual by
   h^2 / p^2.
 * h_e, "the diameter of the element": the largest distance between two of
   the element's eight vertices.
 * h_m, p_m and sigma: those of the operator's own penalty (eq.
   penaltyparameter): p_m = max(p_A, p_B), h_m = min over both sides and the
   mortar's points of 2 J / S, sigma = C p_m^2 / h_m.
 * J_{m,1} is defined on interior mortars only; Dirichlet mortars carry
   eta^2_{m,3} alone.  Each interior mortar's terms are added in full to both
   elements it touches.
 * The volume residual uses the isoparametric geometry of the element (the
   single-box meshes of this module).  On curved meshes the two sides of a
   2:1 or degree-jump mortar interpolate the face differently, so the jump
   terms also see that geometry error.

Pins: closed forms for a constant source, an element indicator function
(conforming and 2:1 mortars) and a kink across a plane; zero for a quadratic
solution on affine elements and for a linear solution on curved ones
(tests/test_oracle_estimator.py); on block meshes the map's second
derivatives against differences of its Jacobian, Lap u_h of the interpolant
of a smooth field against that field's Laplacian on curved wedge and shell
elements, and the exact scaling of the three estimator terms (s^5, s^3, s^0)
under a uniformly scaled fiducial grid (tests/test_oracle_estimator_blocks.py).
"""
import numpy as np

from . import tables
from .sipg import MortarData, volume_geometry


def lagrange_second_derivs(nodes, x):
    """V[i, a] = l_a''(x_i): the product rule applied twice to the product
    formula of the Lagrange polynomial (Sec. II.A.3)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.zeros((len(x), n))
    for a in range(n):
        den = 1.0
        for j in range(n):
            if j != a:
                den *= nodes[a] - nodes[j]
        for m in range(n):
            if m == a:
                continue
            for k in range(n):
                if k == a or k == m:
                    continue
                term = np.ones(len(x))
                for j in range(n):
                    if j not in (a, m, k):
                        term *= x - nodes[j]
                V[:, a] += term / den
    return V


def basis3d_second(nodes, xi):
    """d2Psi[l, m, P, n^3] = d^2 psi_alpha / dxi_l dxi_m at reference points xi
    (node index alpha = a + n b + n^2 c, as in tables.basis3d)."""
    xi = np.asarray(xi, dtype=np.float64).reshape(-1, 3)
    n = len(nodes)
    P = xi.shape[0]
    D = [[tables.lagrange_values(nodes, xi[:, d]),
          tables.lagrange_derivs(nodes, xi[:, d]),
          lagrange_second_derivs(nodes, xi[:, d])] for d in range(3)]
    out = np.zeros((3, 3, P, n ** 3))
    for l in range(3):
        for m in range(3):
            order = [0, 0, 0]
            order[l] += 1
            order[m] += 1
            A, B, C = D[0][order[0]], D[1][order[1]], D[2][order[2]]
            out[l, m] = np.einsum('pa,pb,pc->pcba', A, B, C).reshape(P, n ** 3)
    return out


def element_diameter(mesh, e):
    """Largest distance between two of element e's vertices (its corner LGL nodes)."""
    n = int(mesh.n[e])
    X = mesh.node_coords(e)
    corners = [X[a + n * b + n * n * c] for c in (0, n - 1) for b in (0, n - 1) for a in (0, n - 1)]
    return max(np.linalg.norm(P - Q) for P in corners for Q in corners)


def laplacian_at_gl(mesh, e, ue):
    """Lap u_h, u_h and the weights w det J at element e's GL points (exact
    chain rule on the isoparametric map, see the module docstring)."""
    n = int(mesh.n[e])
    xl, _ = tables.lgl_nodes_weights(n)
    xi, w, J, detJ, Jinv = volume_geometry(mesh, e)
    Psi, dPsi = tables.basis3d(xl, xi)
    d2Psi = basis3d_second(xl, xi)
    if hasattr(mesh, "hessian_at"):                     # exact block map
        Xss = mesh.hessian_at(e, xi)
    else:                                               # isoparametric interpolant
        X = mesh.node_coords(e)
        Xss = np.einsum('lmpa,ai->pilm', d2Psi, X)      # d^2 x_i / dxi_l dxi_m
    u = Psi @ ue
    du = np.einsum('lpa,a->pl', dPsi, ue)               # du / dxi_l
    d2u = np.einsum('lmpa,a->plm', d2Psi, ue)           # d^2 u / dxi_l dxi_m
    gx = np.einsum('pli,pl->pi', Jinv, du)              # du / dx_i
    M = d2u - np.einsum('pi,pilm->plm', gx, Xss)
    H = np.einsum('pli,plm,pmj->pij', Jinv, M, Jinv)    # physical Hessian
    lap = np.einsum('pii->p', H)
    return lap, u, w * detJ


def _volume_term(mesh, e, u, g_fn, f_fn, fid=None):
    from .sipg import volume_points
    ue = u[mesh.dof_off[e]:mesh.dof_off[e + 1]]
    lap, uq, wd = laplacian_at_gl(mesh, e, ue)
    xq = volume_points(mesh, e)
    g = g_fn(xq) if g_fn is not None else 0.0
    f = f_fn(xq) if f_fn is not None else 0.0
    R = f * uq - g - lap
    if fid is not None:                                 # weights and h_e of the fiducial grid
        xi, w, J, detJ, Jinv = volume_geometry(fid, e)
        wd = w * detJ
    he = element_diameter(mesh if fid is None else fid, e)
    pe = float(mesh.p[e])
    return he * he * pe * pe * float(np.sum(wd * R * R))


def _mortar_term(mesh, mi, u, gD_fn, C, fid=None):
    """eta^2_{m,1} + eta^2_{m,2} (interior) or eta^2_{m,3} (Dirichlet) of mortar mi."""
    return sum(_mortar_terms(mesh, mi, u, gD_fn, C, fid))


def _mortar_terms(mesh, mi, u, gD_fn, C, fid=None):
    """(eta^2_{m,1}, eta^2_{m,2} or eta^2_{m,3}) of mortar mi."""
    m = mesh.mortars[mi]
    md = MortarData(mesh, mi, C)
    mw = md if fid is None else MortarData(fid, mi, C)   # weights, h_m and sigma
    hm = min(h.min() for h in mw.h)
    pm = float(m.pm)
    uA = u[mesh.dof_off[m.eA]:mesh.dof_off[m.eA + 1]]
    vA = md.psi[0] @ uA
    if m.eB is None:
        gD = gD_fn(md.x) if gD_fn is not None else 0.0
        J3 = vA - gD
        return 0.0, mw.sigma / hm * pm * pm * float(np.sum(mw.W * J3 * J3))
    uB = u[mesh.dof_off[m.eB]:mesh.dof_off[m.eB + 1]]
    J1 = md.dn[0] @ uA - md.dn[1] @ uB
    J2 = vA - md.psi[1] @ uB
    return hm / pm * float(np.sum(mw.W * J1 * J1)), mw.sigma / hm * pm * pm * float(np.sum(mw.W * J2 * J2))


def estimate(mesh, u, g_fn=None, f_fn=None, gD_fn=None, C=10.0, parts=False, elems=None, fiducial=None):
    """eta^2(e) for every element of `mesh` (oracle Mesh or BlockMesh), or for
    the elements listed in `elems` only (in that order).

    u: nodal coefficients (n_dofs,); g_fn, f_fn, gD_fn: callables of physical
    points (P, 3) -> (P,) or None for zero.  fiducial: a BlockMesh of identical
    structure (mesh.with_blocks(...)) whose geometry supplies the weights,
    h_e, h_m and sigma, or None.  With parts=True also returns the volume part
    and the mortar part separately.
    """
    u = np.asarray(u, dtype=np.float64)
    fid = fiducial
    if fid is not None:
        same = all((a.eA, a.fA, a.eB, a.fB) == (b.eA, b.fA, b.eB, b.fB) for a, b in zip(mesh.mortars, fid.mortars))
        if fid.n_elems != mesh.n_elems or len(fid.mortars) != len(mesh.mortars) or not same:
            raise ValueError("estimate: the fiducial grid must have the mesh's structure and connectivity")
    sel = list(range(mesh.n_elems)) if elems is None else [int(e) for e in elems]
    pos = {e: i for i, e in enumerate(sel)}
    vol = np.zeros(len(sel))
    mort = np.zeros(len(sel))
    for i, e in enumerate(sel):
        vol[i] = _volume_term(mesh, e, u, g_fn, f_fn, fid)
    if elems is None:
        mortars = range(len(mesh.mortars))
    else:
        mortars = sorted({mi for e in sel for f in range(6) for mi in mesh.elem_mortars[e][f]})
    for mi in mortars:
        m = mesh.mortars[mi]
        t = _mortar_term(mesh, mi, u, gD_fn, C, fid)
        for e in (m.eA, m.eB):
            if e is not None and e in pos:
                mort[pos[e]] += t
    if parts:
        return vol + mort, vol, mort
    return vol + mort
