"""Multigrid hierarchy, transfer operators, smoothers and V-cycle
(oracle; test infrastructure only).

Sec. II.E.3 (multigrid meshes): coarse meshes by h-coarsening complete
sibling families into their parent (surrogate mesh), then restoring 2:1
balance; a coarse element takes the minimum degree of its children and no
level is purely p-coarsened.  Sec. II.E.6 (inter-mesh operators): the
prolongation I_h^H of eq. (psi-interpolation) is nodal interpolation of the
parent basis at the children's LGL nodes; restriction is its transpose
(eq. temp-G); the zeroth-order term is restricted as O^H = I^T O^h I
(eq. operator_oh) while the Laplacian part is re-discretised per level.
Alg. 3 (V-cycle), Alg. 4 (Chebyshev smoother), Alg. 5 (CG spectral bound).

Readings:
 * Balancing: a coarsened parent that would touch an element two or more
   levels finer is un-coarsened (its children kept with their own degrees);
   repeated to a fixpoint.  The hierarchy ends when no family can be merged.
 * Alg. 4 update is p <- alpha r + beta p (standard Chebyshev three-term
   recurrence; the printed minus sign does not give a Chebyshev polynomial).
 * Alg. 5 eigenvalue estimate: Lanczos tridiagonal from the CG coefficients,
   T_kk = 1/a_k + b_{k-1}/a_{k-1}, |T_{k,k+1}| = sqrt(b_k)/a_k, and
   lambda_k = T_kk + |T_{k,k-1}| + |T_{k,k+1}| (Gershgorin row k);
   lambda_max = max_k lambda_k.  CG stops early when p.Jp <= 0 or r.r = 0;
   a smoother whose estimate stayed 0 skips its Chebyshev steps.
 * Level 0 "solve": the smoother (paper) or an exact dense Cholesky solve.
 * Overlapping Schwarz subdomains (Alg. 6, eq. schwarz_weight), for meshes of
   one degree with conforming faces: the node layers of the touching
   elements; xi_ext beyond e_c's boundary = the coinciding e_c coordinate
   moved outward by the neighbour node's LGL distance from the contact;
   delta = the overlap width in xi_ext; local problems solved exactly (the
   paper uses CG to 1e-3).  At the domain boundary and where three or five
   blocks meet along an edge the weights do not sum to one, as the
   construction implies.
 * Coarse operators: re-discretised per level (paper); as an option the
   Galerkin products P^T J P (not in the paper), which keep the V-cycle
   contracting on the compactified cubed sphere where re-discretised levels
   do not (tests/test_oracle_multigrid.py).

Pins: Chebyshev error polynomial on a diagonal matrix, Gershgorin bound >=
lambda_max, CG iterates vs textbook CG, prolongation exactness on coarse
polynomials, restriction/Galerkin identities (tests/test_oracle_multigrid.py);
the V-cycle with a fixed-lambda (linear) Chebyshev smoother equals its
closed form built from explicit matrices -- smoother S(x, b) = R x + (I - R)
J^-1 b with the Chebyshev error matrix R = T_k(Z) / T_k(d / c), Z = (d - J) / c
-- on two and three levels, and planted mistakes (no post-smoothing, f
restricted instead of f - J v, no "+ v_l") fail that comparison; the CG
tridiagonal of Alg. 5 equals the one of an independent Lanczos run, and a
planted beta in place of sqrt(beta) / alpha fails (tests/test_oracle_pins.py);
element Schwarz: exact in one undamped cycle on a block-diagonal matrix, the
spectrum of A_ee^-1 A inside (0, 2), MG-FCG with it reaching 1e-10.
"""
import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla

from . import tables
from .mesh import Mesh


def coarsen(mesh):
    """One coarsening step.  Returns (coarse Mesh, groups) or None.

    groups[H] = list of (fine element, (bx, by, bz)) for a merged family,
    or [(fine element, None)] for an element carried over unchanged."""
    leaves = [tuple(int(v) for v in lf) for lf in mesh.leaves]
    idx = {lf: e for e, lf in enumerate(leaves)}
    fams = {}
    for e, (L, i, j, k) in enumerate(leaves):
        if L == 0:
            continue
        fams.setdefault((L - 1, i >> 1, j >> 1, k >> 1), []).append(e)
    complete = {P for P, ch in fams.items() if len(ch) == 8}
    if not complete:
        return None
    merged = set(complete)
    while True:
        cur = {}
        for lf, e in idx.items():
            P = (lf[0] - 1, lf[1] >> 1, lf[2] >> 1, lf[3] >> 1) if lf[0] > 0 else None
            if P in merged:
                cur[P] = True
            else:
                cur[lf] = True
        cells = set(cur)
        maxL = max(c[0] for c in cells)
        undo = set()
        for P in merged:
            L, i, j, k = P
            for d in range(3):
                for sgn in (-1, 1):
                    c = [i, j, k]
                    c[d] += sgn
                    if c[d] < 0 or c[d] >= (1 << L):
                        continue
                    for L2 in range(L + 2, maxL + 1):
                        sh = L2 - L
                        span = 1 << sh
                        lo = [v << sh for v in c]
                        rng = [range(lo[t], lo[t] + span) for t in range(3)]
                        rng[d] = [lo[d] + (span - 1 if sgn < 0 else 0)]
                        if any((L2, a, b, cc) in cells for a in rng[0] for b in rng[1] for cc in rng[2]):
                            undo.add(P)
                            break
                    if P in undo:
                        break
                if P in undo:
                    break
        if not undo:
            break
        merged -= undo
        if not merged:
            return None
    new_leaves, new_p, groups, seen = [], [], [], set()
    for e, lf in enumerate(leaves):
        P = (lf[0] - 1, lf[1] >> 1, lf[2] >> 1, lf[3] >> 1) if lf[0] > 0 else None
        if P in merged:
            if P in seen:
                continue
            seen.add(P)
            ch = sorted(fams[P])
            grp = []
            for c in ch:
                L, i, j, k = leaves[c]
                grp.append((c, (i - 2 * P[1], j - 2 * P[2], k - 2 * P[3])))
            new_leaves.append(P)
            new_p.append(min(int(mesh.p[c]) for c in ch))
            groups.append(grp)
        else:
            new_leaves.append(lf)
            new_p.append(int(mesh.p[e]))
            groups.append([(e, None)])
    coarse = Mesh(mesh.lo, mesh.hi, new_leaves, new_p, warp=mesh.warp)
    return coarse, groups


def hierarchy(mesh):
    """Meshes [level 0 (coarsest), ..., level L (= mesh)] and groups per level."""
    meshes, groups = [mesh], []
    while True:
        r = coarsen(meshes[0])
        if r is None:
            break
        meshes.insert(0, r[0])
        groups.insert(0, r[1])
    return meshes, groups


def child_interp_1d(nH, nh, b):
    """E[i, a] = l^H_a evaluated at child node i (child half b of the parent)."""
    xH, _ = tables.lgl_nodes_weights(nH)
    xh, _ = tables.lgl_nodes_weights(nh)
    if b is None:
        return tables.lagrange_values(xH, xh)
    return tables.lagrange_values(xH, (xh + (2 * b - 1)) / 2.0)


def prolongation(fine, coarse, groups):
    """Sparse I_h^H (fine dofs x coarse dofs) of eq. (psi-interpolation)."""
    rows, cols, vals = [], [], []
    for H, grp in enumerate(groups):
        nH = int(coarse.n[H])
        for (c, bits) in grp:
            nh = int(fine.n[c])
            if bits is None:
                E = [child_interp_1d(nH, nh, None)] * 3
            else:
                E = [child_interp_1d(nH, nh, b) for b in bits]
            blk = np.kron(E[2], np.kron(E[1], E[0]))
            r = np.arange(fine.dof_off[c], fine.dof_off[c + 1])
            q = np.arange(coarse.dof_off[H], coarse.dof_off[H + 1])
            rr, qq = np.meshgrid(r, q, indexing='ij')
            rows.append(rr.ravel()); cols.append(qq.ravel()); vals.append(blk.ravel())
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.n_dofs, coarse.n_dofs)).tocsr()
    P.eliminate_zeros()
    return P


def cgeigs(A, x, b, n_iter, trace=None):
    """Alg. 5: n_iter CG steps from x with the Gershgorin bound of the
    Lanczos tridiagonal.  Returns (lambda_max, x).  trace, if a list, receives
    (T_kk, |T_k,k+1|, lambda_k) of every step k."""
    x = x.copy()
    r = b - A @ x
    p = r.copy()
    rr = r @ r
    lam = 0.0
    a_prev = b_prev = None
    for k in range(n_iter):
        Ap = A @ p
        pAp = p @ Ap
        if not (pAp > 0.0) or rr == 0.0:
            break
        a = rr / pAp
        x += a * p
        r -= a * Ap
        rr_new = r @ r
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p
        diag = 1.0 / a
        left = 0.0
        if a_prev is not None:
            diag += b_prev / a_prev
            left = np.sqrt(b_prev) / a_prev
        right = np.sqrt(beta) / a
        lam = max(lam, diag + left + right)
        if trace is not None:
            trace.append((diag, right, diag + left + right))
        a_prev, b_prev = a, beta
    return lam, x


def chebyshev(A, x, b, lam_max, Lam, n_iter):
    """Chebyshev steps of Alg. 4 on [lam_max / Lam, lam_max]."""
    x = x.copy()
    if not (lam_max > 0.0):
        return x
    lmin = lam_max / Lam
    c = 0.5 * (lam_max - lmin)
    d = 0.5 * (lam_max + lmin)
    p = np.zeros_like(x)
    alpha = 0.0
    for k in range(1, n_iter + 1):
        r = b - A @ x
        if k == 1:
            alpha = 1.0 / d
        elif k == 2:
            alpha = 2.0 * d / (2.0 * d * d - c * c)
        else:
            alpha = 1.0 / (d - alpha * c * c / 4.0)
        beta = alpha * d - 1.0
        p = alpha * r + beta * p
        x = x + p
    return x


def smoother(A, x, b, n_eigs=15, n_cheb=15, Lam=20.0):
    """Alg. 4: CGEIGS then Chebyshev from the CG-updated x."""
    lam, x = cgeigs(A, x, b, n_eigs)
    return chebyshev(A, x, b, lam, Lam, n_cheb), lam


def schwarz_blocks(A, dof_off):
    """Dense inverses of the element diagonal blocks of A (element-centred
    Schwarz subdomains without overlap)."""
    Ad = A.tocsr()
    return [np.linalg.inv(Ad[dof_off[e]:dof_off[e + 1], dof_off[e]:dof_off[e + 1]].toarray())
            for e in range(len(dof_off) - 1)]


def schwarz_smoother(A, inv_blocks, dof_off, x, b, n_cycles=3, omega=0.7):
    """Alg. 6 (Schwarz smoother) with subdomains = single elements (overlap 0):
    n_cycles times r = b - A x, then x += omega R_e^T A_ee^-1 R_e r for every
    element e, the local problems solved exactly.  Without overlap the
    paper's weights are 1; omega < 1 damps the top of the spectrum of
    A_ee^-1 A (which reaches nearly 2 for SIPG)."""
    x = x.copy()
    for _ in range(n_cycles):
        r = b - A @ x
        dx = np.zeros_like(x)
        for e, Ai in enumerate(inv_blocks):
            sl = slice(dof_off[e], dof_off[e + 1])
            dx[sl] = Ai @ r[sl]
        x += omega * dx
    return x


def schwarz_phi(t):
    """phi of the Schwarz weight (eq. schwarz_weight): sgn(t) for |t| > 1,
    (15 t - 10 t^3 + 3 t^5) / 8 inside."""
    t = np.asarray(t, dtype=np.float64)
    return np.where(np.abs(t) > 1.0, np.sign(t), (15.0 * t - 10.0 * t ** 3 + 3.0 * t ** 5) / 8.0)


def schwarz_weight(xi_ext, delta):
    """w_h(xi_ext) = (phi((xi_ext + 1) / delta) - phi((xi_ext - 1) / delta)) / 2
    (eq. schwarz_weight)."""
    return 0.5 * (schwarz_phi((np.asarray(xi_ext) + 1.0) / delta) - schwarz_phi((np.asarray(xi_ext) - 1.0) / delta))


def overlap_subdomains(mesh, n_overlap=2):
    """Element-centred Schwarz subdomains with overlap (Sec. II.E.5) for a
    mesh whose elements all have the same degree and meet conformingly
    (any block layout).  Subdomain of e_c: its own nodes, the nodes of every
    element touching it that coincide with e_c's boundary nodes (faces,
    edges, corners), and the nodes of those elements within n_overlap - 1
    further index layers of them.  Each node gets its extended LGL
    coordinate xi_ext in e_c's frame -- its own LGL coordinate on e_c, and
    beyond e_c's boundary the coinciding e_c coordinate moved outward by the
    node's LGL distance from the contact (the direction found from the
    neighbour's node positions and e_c's Jacobian) -- and the weight
    W = prod_i w_h(xi_ext^i) with delta the overlap width in xi_ext.  With
    n_overlap = 1 every xi_ext lies in [-1, 1] (the contact nodes sit on e_c's
    boundary), the overlap width is zero and delta falls to its 1e-12 floor:
    the weights become the step function 1 inside, 1/2 on faces, 1/4 on edges
    and 1/8 on corners (pinned by test_overlap_one_layer_step_weights).
    Returns [(global dofs, weights)] per element."""
    from scipy.spatial import cKDTree
    n = int(mesh.n[0])
    if np.any(mesh.n != n):
        raise ValueError("overlap_subdomains: one degree for every element")
    if any(not m.boundary and (mesh.leaves[m.eA][0] != mesh.leaves[m.eB][0]) for m in mesh.mortars):
        raise ValueError("overlap_subdomains: conforming faces only (no 2:1 faces)")
    n3 = n ** 3
    xl, _ = tables.lgl_nodes_weights(n)
    X = np.vstack([mesh.node_coords(e) for e in range(mesh.n_elems)])
    tree = cKDTree(X)
    idx3 = np.array([(a, b, c) for c in range(n) for b in range(n) for a in range(n)])
    lin = lambda q: int(q[0] + n * q[1] + n * n * q[2])
    bnd = [k for k in range(n3) if (idx3[k] == 0).any() or (idx3[k] == n - 1).any()]
    subs = []
    for e in range(mesh.n_elems):
        o = int(mesh.dof_off[e])
        contact = {}
        for k in bnd:
            for j in tree.query_ball_point(X[o + k], 1e-9 * max(1.0, np.linalg.norm(X[o + k]))):
                if not (o <= j < o + n3):
                    contact[j] = k
        by_elem = {}
        for j, k in contact.items():
            e2 = int(np.searchsorted(mesh.dof_off, j, side='right') - 1)
            by_elem.setdefault(e2, {})[j - int(mesh.dof_off[e2])] = k
        dofs = list(range(o, o + n3))
        xis = list(tables.tensor_points(xl))
        for e2 in sorted(by_elem):
            cmap = by_elem[e2]
            o2 = int(mesh.dof_off[e2])
            C = idx3[np.array(sorted(cmap))]
            pinned = [a for a in range(3) if len(set(C[:, a])) == 1]
            for q in range(n3):
                qi = idx3[q]
                if np.abs(C - qi[None]).max(axis=1).min() > n_overlap - 1:
                    continue
                c = qi.copy()
                for a in pinned:
                    c[a] = C[0, a]
                xi = xl[idx3[cmap[lin(c)]]].astype(np.float64)
                for a in pinned:
                    if qi[a] == c[a]:
                        continue
                    nxt = c.copy()
                    nxt[a] += 1 if qi[a] > c[a] else -1
                    dxi = np.linalg.solve(mesh.jacobian_at(e, xi[None])[0], X[o2 + lin(nxt)] - X[o2 + lin(c)])
                    ax = int(np.argmax(np.abs(dxi)))
                    xi[ax] += np.sign(dxi[ax]) * abs(xl[qi[a]] - xl[c[a]])
                dofs.append(o2 + q)
                xis.append(xi)
        xis = np.array(xis)
        delta = max(float(np.abs(xis).max()) - 1.0, 1e-12)
        subs.append((np.array(dofs, dtype=np.int64), np.prod(schwarz_weight(xis, delta), axis=1)))
    return subs


def overlap_schwarz_smoother(A, subs, x, b, n_cycles=3, factors=None):
    """Alg. 6 with overlapping subdomains: n_cycles times r = b - A x, then
    x += sum_s R_s^T W_s dx_s with R_s A R_s^T dx_s = R_s r solved exactly
    (Cholesky; factors from overlap_factors may be passed in)."""
    Ad = A.tocsr()
    if factors is None:
        factors = overlap_factors(Ad, subs)
    x = x.copy()
    for _ in range(n_cycles):
        r = b - Ad @ x
        dx = np.zeros_like(x)
        for (d, W), f in zip(subs, factors):
            np.add.at(dx, d, W * sla.cho_solve(f, r[d]))
        x = x + dx
    return x


def overlap_factors(A, subs):
    Ad = A.tocsr()
    return [sla.cho_factor(Ad[d][:, d].toarray()) for d, _ in subs]


def uniform_block_levels(blocks, level, p):
    """Level meshes 0..level of a multi-block mesh refined uniformly (every
    block at the same level, degree p everywhere) and their family groups,
    for Hierarchy(levels=...)."""
    from .blockmesh import BlockMesh
    meshes, groups = [], []
    for L in range(level + 1):
        m = 1 << L
        lv = [(L, i, j, k) for k in range(m) for j in range(m) for i in range(m)]
        eb = [b for b in range(len(blocks)) for _ in lv]
        leaves = [tuple(lf) for _ in blocks for lf in lv]
        meshes.append(BlockMesh(blocks, eb, leaves, [p] * len(leaves)))
    for L in range(level):
        fine, coarse = meshes[L + 1], meshes[L]
        fkey = {(int(b),) + tuple(int(v) for v in lf): e for e, (b, lf) in enumerate(zip(fine.elem_block, fine.leaves))}
        grp = []
        for b, lf in zip(coarse.elem_block, coarse.leaves):
            l, i, j, k = (int(v) for v in lf)
            grp.append([(fkey[(int(b), l + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1))],
                         (c & 1, (c >> 1) & 1, (c >> 2) & 1)) for c in range(8)])
        groups.append(grp)
    return meshes, groups


class Hierarchy:
    """Level operators J_l and prolongations for the V-cycle of Alg. 3.

    coarse_ops='rediscretised' (the paper: the SIPG operator assembled on
    every level mesh) or 'galerkin' (every coarse operator P^T J P from the
    next finer one); levels=(meshes, groups) gives the level meshes directly
    (e.g. uniform_block_levels) instead of coarsening a single-box mesh."""

    def __init__(self, mesh, C=10.0, coef=None, extra=0, coarse_ops='rediscretised', levels=None):
        from . import sipg
        if levels is None:
            self.meshes, self.groups = hierarchy(mesh)
        else:
            self.meshes, self.groups = list(levels[0]), list(levels[1])
        self.P = [prolongation(self.meshes[l + 1], self.meshes[l], self.groups[l])
                  for l in range(len(self.meshes) - 1)]
        if coarse_ops == 'galerkin':
            self.L = [None] * len(self.meshes)
            self.L[-1] = sipg.assemble(self.meshes[-1], C, extra)
            for l in range(len(self.meshes) - 2, -1, -1):
                self.L[l] = (self.P[l].T @ self.L[l + 1] @ self.P[l]).tocsr()
        elif coarse_ops == 'rediscretised':
            self.L = [sipg.assemble(m, C, extra) for m in self.meshes]
        else:
            raise ValueError("coarse_ops is 'rediscretised' or 'galerkin'")
        self.J = list(self.L)
        if coef is not None:
            O = sipg.assemble(self.meshes[-1], C, extra, coef) - self.L[-1]
            self.O = [None] * len(self.meshes)
            self.O[-1] = O
            for l in range(len(self.meshes) - 2, -1, -1):
                self.O[l] = (self.P[l].T @ self.O[l + 1] @ self.P[l]).tocsr()
            self.J = [self.L[l] + self.O[l] for l in range(len(self.meshes))]
        self._chol = None

    @property
    def n_levels(self):
        return len(self.meshes)

    def coarse_cholesky(self, f):
        if self._chol is None:
            self._chol = sla.cho_factor(self.J[0].toarray())
        return sla.cho_solve(self._chol, f)

    def residual(self, l, f, v):
        """f - J_l v on level l."""
        return f - self.J[l] @ v

    def restrict(self, l, r):
        """(I_h^H)^T r from level l to level l - 1 (eq. temp-G)."""
        return self.P[l - 1].T @ r

    def prolong(self, l, v):
        """I_h^H v from level l - 1 to level l (eq. psi-interpolation)."""
        return self.P[l - 1] @ v

    def coarse_correction(self, l, v, v_coarse):
        """The smoothed v_l plus the prolonged coarse solution (Alg. 3, on the
        way up)."""
        return self.prolong(l, v_coarse) + v

    def vcycle(self, f, n_eigs=15, n_cheb=15, Lam=20.0, coarse='smoother', smoother_kind='chebyshev',
               n_schwarz=3, omega=0.7, n_overlap=2, lam_fixed=None):
        """Alg. 3 with the level meshes fixed in advance; smoother_kind
        'chebyshev' (Alg. 4 with Alg. 5), 'schwarz' (element subdomains,
        exact local solves) or 'schwarz_overlap' (Alg. 6 with overlapping
        subdomains and the weights w_h, exact local solves).  lam_fixed (a
        number, or one per level, coarsest first): Chebyshev steps on
        [lam / Lam, lam] with that lam and no CG steps -- a linear smoother."""
        Lt = self.n_levels - 1
        if smoother_kind == 'schwarz' and not hasattr(self, '_sinv'):
            self._sinv = [schwarz_blocks(self.J[l], self.meshes[l].dof_off) for l in range(Lt + 1)]
        if smoother_kind == 'schwarz_overlap' and not hasattr(self, '_ovl'):
            self._ovl = []
            for l in range(Lt + 1):
                subs = overlap_subdomains(self.meshes[l], n_overlap)
                self._ovl.append((subs, overlap_factors(self.J[l], subs)))

        def smooth(l, v, b):
            if smoother_kind == 'schwarz':
                return schwarz_smoother(self.J[l], self._sinv[l], self.meshes[l].dof_off, v, b, n_schwarz, omega)
            if smoother_kind == 'schwarz_overlap':
                subs, fac = self._ovl[l]
                return overlap_schwarz_smoother(self.J[l], subs, v, b, n_schwarz, fac)
            if lam_fixed is not None:
                lam = lam_fixed[l] if np.ndim(lam_fixed) else lam_fixed
                return chebyshev(self.J[l], v, b, lam, Lam, n_cheb)
            return smoother(self.J[l], v, b, n_eigs, n_cheb, Lam)[0]

        fs = [None] * (Lt + 1)
        vs = [None] * (Lt + 1)
        fs[Lt] = f
        for l in range(Lt, 0, -1):
            v = smooth(l, np.zeros_like(fs[l]), fs[l])
            vs[l] = v
            fs[l - 1] = self.restrict(l, self.residual(l, fs[l], v))
        if coarse == 'cholesky':
            vs[0] = self.coarse_cholesky(fs[0])
        else:
            vs[0] = smooth(0, np.zeros_like(fs[0]), fs[0])
        for l in range(1, Lt + 1):
            v = self.coarse_correction(l, vs[l], vs[l - 1])
            vs[l] = smooth(l, v, fs[l])
        return vs[Lt]
