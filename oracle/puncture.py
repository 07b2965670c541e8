"""Puncture initial data (Sec. III.D, eqs. Two_Punctures_PDE, Two_Punctures_Aij)
and Newton-Raphson (Alg. 1) (oracle; test infrastructure only).

With 1/alpha = sum_I m_I / (2 r_I) and psi = 1 + 1/alpha + u the equation
-Lap u = (1/8) A_ij A^ij psi^-7 becomes
    R(u) = -Lap u - beta (1 + alpha (1 + u))^-7 = 0,  beta = alpha^7 A_ij A^ij / 8,
and its linearisation J_R du = -Lap du + 7 alpha beta (1 + alpha (1 + u))^-8 du
(eq. temp-F form: the zeroth-order coefficient f(u_0)).  Nonlinear terms are
evaluated at the volume GL points after interpolating u there (Sec. III.B).

Readings:
 * A_ij = sum_I { 3 / (2 r_I^2) [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n]
                 + 3 / r_I^3 [n_i (S x n)_j + n_j (S x n)_i] }.
   The printed spin term, (4 / r) n_(i eps_j)kl S^k n^l inside the bracket
   that 3 / (2 r^2) multiplies, is read with the symmetrisation
   t_(ij) = (t_ij + t_ji) / 2 and eps_jkl S^k n^l = (S x n)_j, which gives
   the 3 / r^3 term above; punctures without a spin vector have S = 0.
 * Outer boundary: u = 0 Dirichlet on the box (u -> 0 at infinity).
 * Newton loop: while k < N_NK and ||R(u_k)|| >= tol_NK (Alg. 1 joins the two
   tests with "or").

Pins: single-puncture closed forms A_ij A^ij = 9 / (2 r^4) (|P|^2 + 2 (P.n)^2)
and, for a spin alone, 18 (|S|^2 - (S.n)^2) / r^6; A_ij symmetric, traceless
and divergence-free (the flat momentum constraint, by finite differences)
with momenta and spins together,
J_R v against a central finite difference of R, quadratic Newton
convergence (tests/test_oracle_puncture.py).

PowerSourceProblem (the constant-density star of Sec. III.C) is pinned by its
closed-form solution (tests/test_oracle_star.py): the discrete Newton solution
converges to it under refinement, the Jacobian matches finite differences of
the residual and Newton converges quadratically.
"""
import numpy as np

from . import tables, sipg


def extrinsic_curvature(x, punctures):
    """A_ij (P, 3, 3) and 1/alpha at points x (P, 3); punctures: list of
    (m, c(3), P(3)) or (m, c(3), P(3), S(3))."""
    x = np.asarray(x, dtype=np.float64)
    inv_alpha = np.zeros(len(x))
    A = np.zeros((len(x), 3, 3))
    I3 = np.eye(3)
    for pu in punctures:
        m, c, P = pu[0], pu[1], pu[2]
        S = np.asarray(pu[3] if len(pu) > 3 else (0.0, 0.0, 0.0), dtype=np.float64)
        dx = x - np.asarray(c, dtype=np.float64)
        r = np.linalg.norm(dx, axis=1)
        nvec = dx / r[:, None]
        P = np.asarray(P, dtype=np.float64)
        Pn = nvec @ P
        term = (np.einsum('i,pj->pij', P, nvec) + np.einsum('pi,j->pij', nvec, P)
                - (I3[None] - np.einsum('pi,pj->pij', nvec, nvec)) * Pn[:, None, None])
        A += (1.5 / r ** 2)[:, None, None] * term
        Sxn = np.cross(S[None, :], nvec)
        spin = np.einsum('pi,pj->pij', nvec, Sxn) + np.einsum('pi,pj->pij', Sxn, nvec)
        A += (3.0 / r ** 3)[:, None, None] * spin
        inv_alpha += m / (2.0 * r)
    return A, inv_alpha


def alpha_beta(x, punctures):
    """alpha and beta at points x (P, 3); punctures: list of (m, c(3), P(3))
    or (m, c(3), P(3), S(3))."""
    A, inv_alpha = extrinsic_curvature(x, punctures)
    AA = np.einsum('pij,pij->p', A, A)
    alpha = 1.0 / inv_alpha
    beta = alpha ** 7 * AA / 8.0
    return alpha, beta, AA


class PunctureProblem:
    def __init__(self, mesh, punctures, C=10.0):
        self.mesh = mesh
        self.C = C
        self.L = sipg.assemble(mesh, C)
        self.data = []
        for e in range(mesh.n_elems):
            n = int(mesh.n[e])
            xl, _ = tables.lgl_nodes_weights(n)
            xi, w, J, detJ, Jinv = sipg.volume_geometry(mesh, e)
            Psi, _ = tables.basis3d(xl, xi)
            x = mesh.position_at(e, xi)
            al, be, _ = alpha_beta(x, punctures)
            self.data.append((Psi, w * detJ, al, be))

    def _gl(self, u):
        off = self.mesh.dof_off
        for e, (Psi, wd, al, be) in enumerate(self.data):
            yield e, Psi, wd, al, be, Psi @ u[off[e]:off[e + 1]]

    def residual(self, u):
        """R_alpha = (L u)_alpha - int beta (1 + alpha (1 + u))^-7 psi_alpha."""
        R = self.L @ u
        off = self.mesh.dof_off
        for e, Psi, wd, al, be, ug in self._gl(u):
            R[off[e]:off[e + 1]] -= Psi.T @ (wd * be * (1.0 + al * (1.0 + ug)) ** -7)
        return R

    def jacobian_coef(self, u):
        """Per element: f(u) = 7 alpha beta (1 + alpha (1 + u))^-8 at GL points."""
        return [7.0 * al * be * (1.0 + al * (1.0 + ug)) ** -8 for e, Psi, wd, al, be, ug in self._gl(u)]

    def jacobian(self, u):
        return sipg.assemble(self.mesh, self.C, coef=self.jacobian_coef(u))


def newton(prob, u0, lsolve, tol=1e-10, max_iter=20):
    """Alg. 1 with linear solver lsolve(J_coef, rhs) -> du."""
    u = u0.copy()
    hist = []
    k = 0
    while k < max_iter:
        R = prob.residual(u)
        hist.append(np.linalg.norm(R))
        if hist[-1] < tol:
            break
        du = lsolve(prob.jacobian_coef(u), -R)
        u = u + du
        k += 1
    return u, k, hist


class PowerSourceProblem:
    """Power-law source (Sec. III.C, constant-density star Lap psi + 2 pi rho
    psi^5 = 0 in the coercive form): R(u) = L u - F - int c u^k v with the
    nonlinearity evaluated at the volume GL points after interpolating u
    there; the Jacobian's zeroth-order coefficient is -k c u^(k-1) (J = L -
    k c u^(k-1) mass, the source growing with u).  c: callable on points (P, 3);
    F: forcing vector (Dirichlet lift), e.g. sipg.rhs with g = 0."""

    def __init__(self, mesh, coef, power, F, C=10.0):
        self.mesh = mesh
        self.C = C
        self.k = int(power)
        self.F = np.asarray(F, dtype=np.float64)
        self.L = sipg.assemble(mesh, C)
        self.data = []
        for e in range(mesh.n_elems):
            n = int(mesh.n[e])
            xl, _ = tables.lgl_nodes_weights(n)
            xi, w, J, detJ, Jinv = sipg.volume_geometry(mesh, e)
            Psi, _ = tables.basis3d(xl, xi)
            self.data.append((Psi, w * detJ, coef(mesh.position_at(e, xi))))

    def residual(self, u):
        R = self.L @ u - self.F
        off = self.mesh.dof_off
        for e, (Psi, wd, c) in enumerate(self.data):
            ug = Psi @ u[off[e]:off[e + 1]]
            R[off[e]:off[e + 1]] -= Psi.T @ (wd * c * ug ** self.k)
        return R

    def jacobian_coef(self, u):
        off = self.mesh.dof_off
        return [-self.k * c * (Psi @ u[off[e]:off[e + 1]]) ** (self.k - 1)
                for e, (Psi, wd, c) in enumerate(self.data)]
