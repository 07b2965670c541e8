"""SIPG operator and right-hand side by dense brute-force quadrature
(oracle; test infrastructure only).

Implements, element by element and mortar by mortar, the bilinear form of
eq. (lh2) (stiffness, consistency, symmetry, penalty and zeroth-order terms;
Dirichlet boundaries only) and the right-hand side of eq. (equationFh2),
with jumps and averages from eq. (20), metric terms from eqs. (Jacobian),
(Surface-Jacobian) and the normal formula that follows them, GL quadrature
with interpolated polynomial quantities (Sec. II.A.5, eq. harald-stiff) and
the penalty sigma = C p_m^2 / h_m of eq. (penaltyparameter).

Readings:
 * Model problem is taken in its coercive form -Lap u + f u = g (the printed
   eq. Laplacian has the opposite sign of its own weak form, eq. lh).
 * h_m = min over both sides and over the mortar's GL points of
   2 J / S, with J and S of each side's own [-1, 1] map (= the element width
   normal to the face for affine hexahedra; eq. penaltyparameter states the
   [0, 1] maps).
 * N_GL = p + 1 (+ extra) volume points; mortars use p_m + 1 points.
Basis functions and their physical gradients are evaluated directly at the
quadrature points with dense (P x n^3) matrices -- no sum factorisation.

Pins: symmetry, positive definiteness, polynomial patch test on 2:1 / p-jump
meshes, penalty closed form, volume identities on curved elements and
h^(p+1) convergence (tests/test_oracle_sipg.py, tests/test_oracle_geometry.py).
"""
import numpy as np
import scipy.sparse as sp

from . import tables
from .mesh import tangential_dims


def volume_geometry(mesh, e, extra=0):
    n = int(mesh.n[e])
    q = n + extra
    xg, wg = tables.gl_nodes_weights(q)
    xi = tables.tensor_points(xg)
    w = tables.tensor_weights(wg)
    J = mesh.jacobian_at(e, xi)
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)          # Jinv[p, l, i] = d xi_l / d x_i
    return xi, w, J, detJ, Jinv


def element_stiffness(mesh, e, extra=0):
    """L^stiff,e_{alpha beta} of eq. (harald-stiff) by dense quadrature."""
    n = int(mesh.n[e])
    xl, _ = tables.lgl_nodes_weights(n)
    xi, w, J, detJ, Jinv = volume_geometry(mesh, e, extra)
    _, dPsi = tables.basis3d(xl, xi)
    B = np.einsum('pli,lpa->ipa', Jinv, dPsi)       # physical gradient of psi_a
    wd = w * detJ
    return np.einsum('ipa,p,ipb->ab', B, wd, B)


def element_mass(mesh, e, coef, extra=0):
    """int_e c psi_a psi_b dx at GL points; coef: array of c at the points."""
    n = int(mesh.n[e])
    xl, _ = tables.lgl_nodes_weights(n)
    xi, w, J, detJ, Jinv = volume_geometry(mesh, e, extra)
    Psi, _ = tables.basis3d(xl, xi)
    return Psi.T @ (Psi * (w * detJ * coef)[:, None])


def volume_points(mesh, e, extra=0):
    """Physical coordinates of element e's volume GL points."""
    xi, _, _, _, _ = volume_geometry(mesh, e, extra)
    return mesh.position_at(e, xi)


class MortarData:
    """Both sides' traces and physical gradients at a mortar's GL points."""

    def __init__(self, mesh, mi, C):
        m = mesh.mortars[mi]
        self.m = m
        q = m.pm + 1
        s, ws = tables.gl_nodes_weights(q)
        s1 = np.tile(s, q)
        s2 = np.repeat(s, q)
        wts = np.tile(ws, q) * np.repeat(ws, q)
        sides = [(m.eA, m.fA, m.posA)]
        if m.eB is not None:
            sides.append((m.eB, m.fB, m.posB))
        self.psi, self.grad, self.h = [], [], []
        for k, (e, f, pos) in enumerate(sides):
            n = int(mesh.n[e])
            xl, _ = tables.lgl_nodes_weights(n)
            xi = mesh.side_ref_points(m, k, s1, s2)
            J = mesh.jacobian_at(e, xi)
            detJ = np.linalg.det(J)
            Jinv = np.linalg.inv(J)
            d, sgn = divmod(f, 2)
            gnu = Jinv[:, d, :]                     # grad of xi_nu in physical space
            nrm = np.linalg.norm(gnu, axis=1)
            if k == 0:
                S = detJ * nrm                      # eq. (Surface-Jacobian)
                normal = (1.0 if sgn == 1 else -1.0) * gnu / nrm[:, None]
                self.x = mesh.position_at(e, xi)
            self.h.append(2.0 / nrm)
            Psi, dPsi = tables.basis3d(xl, xi)
            G = np.einsum('pli,lpa->pai', Jinv, dPsi)
            self.psi.append(Psi)
            self.grad.append(G)
        self.W = wts * S
        self.normal = normal
        hm = min(h.min() for h in self.h)
        self.sigma = C * m.pm ** 2 / hm
        self.dn = [np.einsum('pai,pi->pa', G, normal) for G in self.grad]

    def blocks(self):
        """{(test side, trial side): block} of the face integrals of eq. (lh2)."""
        W, sig = self.W, self.sigma
        if self.m.eB is None:
            P, dn = self.psi[0], self.dn[0]
            blk = (sig * P.T @ (P * W[:, None])
                   - dn.T @ (P * W[:, None])
                   - P.T @ (dn * W[:, None]))
            return {(0, 0): blk}
        eps = (1.0, -1.0)
        out = {}
        for s in range(2):
            for t in range(2):
                Ps, Pt = self.psi[s], self.psi[t]
                ds, dt = self.dn[s], self.dn[t]
                blk = (sig * eps[s] * eps[t] * Ps.T @ (Pt * W[:, None])
                       - 0.5 * eps[t] * ds.T @ (Pt * W[:, None])
                       - 0.5 * eps[s] * Ps.T @ (dt * W[:, None]))
                out[(s, t)] = blk
        return out


def _mortar_elems(m):
    return [m.eA] if m.eB is None else [m.eA, m.eB]


def assemble(mesh, C=10.0, extra=0, coef=None):
    """Global SIPG matrix (CSR) of eq. (semidiscrete) for Dirichlet boundaries.

    coef: optional list (per element) of zeroth-order coefficients f at the
    volume GL points (the int f u v term of eq. lh2)."""
    rows, cols, vals = [], [], []
    off = mesh.dof_off

    def add(ea, eb, blk):
        ia = np.arange(off[ea], off[ea + 1])
        ib = np.arange(off[eb], off[eb + 1])
        rr, cc = np.meshgrid(ia, ib, indexing='ij')
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(blk.ravel())

    for e in range(mesh.n_elems):
        blk = element_stiffness(mesh, e, extra)
        if coef is not None:
            blk = blk + element_mass(mesh, e, coef[e], extra)
        add(e, e, blk)
    for mi in range(len(mesh.mortars)):
        md = MortarData(mesh, mi, C)
        es = _mortar_elems(md.m)
        for (s, t), blk in md.blocks().items():
            add(es[s], es[t], blk)
    N = mesh.n_dofs
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return A.tocsr()


def apply_local(mesh, x, C=10.0, extra=0, elems=None):
    """Matrix-free dense-local apply y = L x (no assembly).

    elems: optional iterable of element indices; then only those elements'
    rows are computed and returned as {e: y_e}."""
    off = mesh.dof_off
    if elems is None:
        y = np.zeros(mesh.n_dofs)
        for e in range(mesh.n_elems):
            y[off[e]:off[e + 1]] += element_stiffness(mesh, e, extra) @ x[off[e]:off[e + 1]]
        for mi in range(len(mesh.mortars)):
            md = MortarData(mesh, mi, C)
            es = _mortar_elems(md.m)
            for (s, t), blk in md.blocks().items():
                y[off[es[s]]:off[es[s] + 1]] += blk @ x[off[es[t]]:off[es[t] + 1]]
        return y
    out = {}
    for e in elems:
        ye = element_stiffness(mesh, e, extra) @ x[off[e]:off[e + 1]]
        mis = sorted({mi for f in range(6) for mi in mesh.elem_mortars[e][f]})
        for mi in mis:
            md = MortarData(mesh, mi, C)
            es = _mortar_elems(md.m)
            s = es.index(e)
            for (ss, t), blk in md.blocks().items():
                if ss == s:
                    ye = ye + blk @ x[off[es[t]]:off[es[t] + 1]]
        out[e] = ye
    return out


def rhs(mesh, g, gD, C=10.0, extra=0):
    """F_h of eq. (equationFh2) with Dirichlet data: int g v
    - int_{Gamma_D} g_D n . grad v + int_{Gamma_D} sigma g_D v.

    g, gD: callables on physical points (P, 3)."""
    F = np.zeros(mesh.n_dofs)
    off = mesh.dof_off
    for e in range(mesh.n_elems):
        n = int(mesh.n[e])
        xl, _ = tables.lgl_nodes_weights(n)
        xi, w, J, detJ, Jinv = volume_geometry(mesh, e, extra)
        Psi, _ = tables.basis3d(xl, xi)
        x = mesh.position_at(e, xi)
        F[off[e]:off[e + 1]] += Psi.T @ (w * detJ * g(x))
    for mi, m in enumerate(mesh.mortars):
        if m.eB is not None:
            continue
        md = MortarData(mesh, mi, C)
        gd = gD(md.x)
        e = m.eA
        F[off[e]:off[e + 1]] += md.psi[0].T @ (md.W * md.sigma * gd) - md.dn[0].T @ (md.W * gd)
    return F


def interpolate(mesh, u):
    """Nodal interpolant: values of callable u at every element's LGL nodes."""
    out = np.zeros(mesh.n_dofs)
    for e in range(mesh.n_elems):
        out[mesh.dof_off[e]:mesh.dof_off[e + 1]] = u(mesh.node_coords(e))
    return out


def l2_error(mesh, uh, u, extra=4):
    """||u - u_h||_2 of eq. (l2norm) with (p + 1 + extra)-point GL quadrature."""
    tot = 0.0
    for e in range(mesh.n_elems):
        n = int(mesh.n[e])
        xl, _ = tables.lgl_nodes_weights(n)
        xi, w, J, detJ, Jinv = volume_geometry(mesh, e, extra)
        Psi, _ = tables.basis3d(xl, xi)
        x = mesh.position_at(e, xi)
        d = Psi @ uh[mesh.dof_off[e]:mesh.dof_off[e + 1]] - u(x)
        tot += np.sum(w * detJ * d * d)
    return np.sqrt(tot)
