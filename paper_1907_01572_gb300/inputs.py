"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds mesh *descriptions* (octree leaves, per-element degrees,
block-map parameters), seeded random vectors and source parameters only.
It contains none of the DG method's arithmetic: both the CUDA library and the
oracle turn these descriptions into geometry, operators and right-hand sides
with their own code.

Leaf format: (level, ix, iy, iz) of a single box block; level-L cells have
width (hi - lo) / 2^L.  Leaves are emitted in Morton (z-curve) order.
"""
import numpy as np


def _morton_key(L, ix, iy, iz, maxL):
    s = maxL - L
    x, y, z = ix << s, iy << s, iz << s
    key = 0
    for b in range(maxL):
        key |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
    return key


def morton_sort(leaves):
    leaves = [tuple(int(v) for v in lf) for lf in leaves]
    maxL = max(lf[0] for lf in leaves)
    return sorted(leaves, key=lambda lf: (_morton_key(lf[0], lf[1], lf[2], lf[3], maxL), lf[0]))


def uniform_leaves(level):
    m = 1 << level
    return morton_sort([(level, i, j, k) for k in range(m) for j in range(m) for i in range(m)])


def refine(leaves, predicate):
    """Replace every leaf for which predicate(leaf) holds by its 8 children."""
    out = []
    for lf in leaves:
        L, i, j, k = lf
        if predicate(lf):
            for c in range(8):
                out.append((L + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1)))
        else:
            out.append(tuple(lf))
    return out


def balance_2to1(leaves):
    """Refine leaves until every face neighbour differs by at most one level."""
    leaves = [tuple(lf) for lf in leaves]
    while True:
        S = set(leaves)
        maxL = max(lf[0] for lf in leaves)
        bad = set()
        for (L, i, j, k) in leaves:
            for d in range(3):
                for sgn in (-1, 1):
                    c = [i, j, k]
                    c[d] += sgn
                    if c[d] < 0 or c[d] >= (1 << L):
                        continue
                    # a neighbour two levels finer exists iff some level L+2 leaf lies in the
                    # adjacent level-L cell: check all deeper levels.
                    for L2 in range(L + 2, maxL + 1):
                        sh = L2 - L
                        lo = [v << sh for v in c]
                        found = False
                        span = 1 << sh
                        # only cells touching our face matter
                        rng = [range(lo[t], lo[t] + span) for t in range(3)]
                        rng[d] = [lo[d] + (span - 1 if sgn < 0 else 0)]
                        for a in rng[0]:
                            for b in rng[1]:
                                for cc in rng[2]:
                                    if (L2, a, b, cc) in S:
                                        found = True
                                        break
                                if found:
                                    break
                            if found:
                                break
                        if found:
                            bad.add((L, i, j, k))
                            break
        if not bad:
            return morton_sort(leaves)
        leaves = refine(leaves, lambda lf: lf in bad)


def config1_mesh():
    """Poisson on [-1,1]^3, 4x4x4 affine elements, uniform p = 3."""
    leaves = uniform_leaves(2)
    return dict(lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), leaves=np.array(leaves, dtype=np.int32),
                p=np.full(len(leaves), 3, dtype=np.int32), warp=None)


def sweep_mesh(level=5, seed=0, pmin=2, pmax=7, curved=True, refine_octant=True, h=1.0 / 16.0):
    """Operator-apply sweep mesh: 2^level per axis on [-1,1]^3, the octant
    x, y, z < 0 h-refined once (2:1 non-conforming faces), per-element p drawn
    uniformly from {pmin..pmax}, node positions curved by the seeded sine warp
    with amplitude 0.1 h and k_i drawn from {1,2,3}.  h is the coarse element
    width of the full 32^3 workload (1/16) at every level, so smaller test
    meshes carry the same physical block map.  level = 5 gives the full
    workload (61,440 elements)."""
    rng = np.random.default_rng(seed)
    half = 1 << (level - 1)
    leaves = uniform_leaves(level)
    if refine_octant:
        leaves = refine(leaves, lambda lf: lf[1] < half and lf[2] < half and lf[3] < half)
    leaves = morton_sort(leaves)
    p = rng.integers(pmin, pmax + 1, size=len(leaves)).astype(np.int32)
    warp = None
    if curved:
        k = tuple(int(v) for v in rng.integers(1, 4, size=3))
        warp = (0.1 * h, k)
    return dict(lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), leaves=np.array(leaves, dtype=np.int32),
                p=p, warp=warp)


def random_vector(n, seed=1):
    """i.i.d. N(0, 1) input vector in FP64."""
    return np.random.default_rng(seed).standard_normal(n)


def oracle_mesh_args(desc):
    """Positional/keyword arguments for the oracle's Mesh constructor."""
    return (desc['lo'], desc['hi'], desc['leaves'], desc['p']), dict(warp=desc['warp'])


# ---- radially symmetric star with a density jump (-Lap u = 4 pi rho) -------------
def star_density(r):
    """rho(r) = (1 - r^2) for 0.5 <= r < 1, 0.6 (1 - r^2) for r < 0.5, 0 outside."""
    r = np.asarray(r, dtype=np.float64)
    rho = np.where(r < 1.0, 1.0 - r * r, 0.0)
    return np.where(r < 0.5, 0.6 * rho, rho)


def star_solution(x):
    """Exact u of -Lap u = 4 pi rho with u -> 0 at infinity:
    u(r) = M(r)/r + int_r^inf 4 pi rho(s) s ds,  M(r) = int_0^r 4 pi rho(s) s^2 ds."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(x, axis=1)
    P = lambda s: s ** 3 / 3.0 - s ** 5 / 5.0          # int s^2 (1 - s^2)
    Q = lambda s: s ** 2 / 2.0 - s ** 4 / 4.0          # int s (1 - s^2)
    h = 0.5
    M_in = 4 * np.pi * 0.6 * P(np.minimum(r, h))
    M_mid = 4 * np.pi * (P(np.clip(r, h, 1.0)) - P(h))
    M = M_in + np.where(r > h, M_mid, 0.0)
    K_mid = 4 * np.pi * (Q(1.0) - Q(np.clip(r, h, 1.0)))
    K_in = 4 * np.pi * 0.6 * (Q(h) - Q(np.minimum(r, h)))
    K = np.where(r < 1.0, K_mid, 0.0) + np.where(r < h, K_in, 0.0)
    rs = np.maximum(r, 1e-300)
    return np.where(r > 0, M / rs, 0.0) + K


def star_source(x):
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    return 4 * np.pi * star_density(np.linalg.norm(x, axis=1))


# ---- Lorentzian (Problem C): u = (1 + r^2)^(-1/2), solving -Lap u = 3 (1 + r^2)^(-5/2) ----
def lorentzian_solution(x):
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    return 1.0 / np.sqrt(1.0 + np.sum(x * x, axis=1))


def lorentzian_source(x):
    """g of -Lap u = g for the Lorentzian (the coercive sign; the printed
    equation carries the opposite sign, which the closed form does not satisfy)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    return 3.0 * (1.0 + np.sum(x * x, axis=1)) ** -2.5


def _cell_bounds(lf, lo, hi):
    L, i, j, k = lf
    w = (np.asarray(hi) - np.asarray(lo)) / (1 << L)
    a = np.asarray(lo) + w * np.array([i, j, k])
    return a, a + w


def _dist_range(a, b, c=(0.0, 0.0, 0.0)):
    c = np.asarray(c, dtype=np.float64)
    near = np.clip(c, a, b)
    dmin = np.linalg.norm(near - c)
    far = np.where(np.abs(a - c) > np.abs(b - c), a, b)
    return dmin, np.linalg.norm(far - c)


def star_mesh(R=4.0, level=3, refine=2, seed=3, p_cut=4, p_lo=5, p_hi=8):
    """Box [-R, R]^3, uniform level `level`, cells cut by the spheres r = 0.5 and
    r = 1 refined `refine` times (2:1 balanced); p = p_cut on the finest cut
    cells, p ~ U{p_lo..p_hi} (seed) elsewhere."""
    lo, hi = (-R, -R, -R), (R, R, R)
    leaves = uniform_leaves(level)

    def cut(lf):
        a, b = _cell_bounds(lf, lo, hi)
        dmin, dmax = _dist_range(a, b)
        return any(dmin <= s <= dmax for s in (0.5, 1.0))

    for _ in range(refine):
        leaves = refine_(leaves, cut)
        leaves = balance_2to1(leaves)
    leaves = morton_sort(leaves)
    rng = np.random.default_rng(seed)
    maxL = max(lf[0] for lf in leaves)
    p = rng.integers(p_lo, p_hi + 1, size=len(leaves))
    p = np.array([p_cut if (lf[0] == maxL and cut(lf)) else pv for lf, pv in zip(leaves, p)], dtype=np.int32)
    return dict(lo=lo, hi=hi, leaves=np.array(leaves, dtype=np.int32), p=p, warp=None)


refine_ = refine


# ---- puncture initial data -----------------------------------------------------------
def two_punctures():
    """m = 0.5 at (+-3, 0, 0) with momenta +-0.2 along y (zero spin); the
    positions are shifted off the element faces of the meshes below."""
    return [(0.5, (3.0 + 1e-3, 2e-3, 3e-3), (0.0, 0.2, 0.0)), (0.5, (-3.0 - 1e-3, 2e-3, 3e-3), (0.0, -0.2, 0.0))]


def three_punctures(seed=2):
    """m in {0.4, 0.3, 0.3} on an equilateral triangle of side 6 in z = 0,
    in-plane momenta |P| <= 0.2 drawn by seed, zero spin."""
    rng = np.random.default_rng(seed)
    out = []
    for i, m in enumerate((0.4, 0.3, 0.3)):
        ang = np.pi / 2 + 2 * np.pi * i / 3
        c = (6 / np.sqrt(3)) * np.array([np.cos(ang), np.sin(ang), 0.0]) + np.array([1e-3, 2e-3, 3e-3])
        th = rng.uniform(0, 2 * np.pi)
        mag = rng.uniform(0, 0.2)
        out.append((m, tuple(c), (mag * np.cos(th), mag * np.sin(th), 0.0)))
    return out


def table_punctures():
    """The three spinning punctures of Sec. III.D (table Multi_Punctures):
    mass m, position (x, y, 0), momentum (P_x, P_y, 0) and spin (0, 0, S_z)
    as printed there."""
    rows = [(0.2691, 0.0152, -0.6933, 0.0585, 0.0082, -0.0134),
            (0.4063, -2.316, 1.8274, -0.0284, -0.1497, -0.0332),
            (0.3245, -1.0279, -2.2711, 0.1640, 0.0515, -0.0708)]
    return [(m, (x, y, 0.0), (px, py, 0.0), (0.0, 0.0, sz)) for (m, x, y, px, py, sz) in rows]


def puncture_mesh(punctures, R=24.0, level=3, refine=2, p_base=4, p_fine=6):
    """Box [-R, R]^3, cells within one cell width of a puncture refined `refine`
    times (2:1 balanced); p_fine on the finest cells, p_base elsewhere."""
    lo, hi = (-R, -R, -R), (R, R, R)
    leaves = uniform_leaves(level)
    cs = [np.asarray(c) for (_, c, _) in punctures]

    def near(lf):
        a, b = _cell_bounds(lf, lo, hi)
        w = b[0] - a[0]
        return any(_dist_range(a, b, c)[0] <= w for c in cs)

    for _ in range(refine):
        leaves = refine_(leaves, near)
        leaves = balance_2to1(leaves)
    leaves = morton_sort(leaves)
    maxL = max(lf[0] for lf in leaves)
    p = np.array([p_fine if lf[0] == maxL else p_base for lf in leaves], dtype=np.int32)
    return dict(lo=lo, hi=hi, leaves=np.array(leaves, dtype=np.int32), p=p, warp=None)


# ---- multi-block meshes ------------------------------------------------------------
# Block descriptions: dict(kind="hex8", corners=8 x 3) | dict(kind="wedge", face,
# a, r) | dict(kind="shell", face, r1, r2); a mesh dict with blocks carries
# "blocks", "elem_block" (per leaf), "leaves" (level, ix, iy, iz in the leaf's
# block frame) and "p".
def cube_rotations():
    """The 24 proper rotations of the reference cube (signed permutation matrices)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((-1, 1), repeat=3):
            R = np.zeros((3, 3))
            for i in range(3):
                R[i, perm[i]] = signs[i]
            if np.linalg.det(R) > 0:
                out.append(R)
    return out


def hex8_box(lo, hi, R=None):
    """hex8 block of the box [lo, hi] whose reference frame is turned by the rotation R."""
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
    corners = []
    for c in range(8):
        xi = np.array([2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1], dtype=np.float64)
        corners.append(lo + 0.5 * (R @ xi + 1.0) * (hi - lo))
    return dict(kind="hex8", corners=np.array(corners))


def _block_mesh(blocks, per_block_leaves, p):
    eb, lv = [], []
    for b, leaves in enumerate(per_block_leaves):
        eb += [b] * len(leaves)
        lv += list(leaves)
    return dict(blocks=blocks, elem_block=np.array(eb, dtype=np.int32), leaves=np.array(lv, dtype=np.int32),
                p=np.asarray(p, dtype=np.int32))


def block_pair_mesh(rot=5, level=1, refine_block=0, seed=0, pmin=2, pmax=5, refine_count=1):
    """Two unit boxes side by side along x, the second with its reference frame
    turned by cube_rotations()[rot]; in block refine_block the `refine_count`
    elements nearest the point (1, 0, 0) of the interface x = 1 are refined
    once (2:1 faces across the block interface); p ~ U{pmin..pmax} (seed)."""
    R = cube_rotations()[rot]
    blocks = [hex8_box((0, 0, 0), (1, 1, 1)), hex8_box((1, 0, 0), (2, 1, 1), R)]
    per = [uniform_leaves(level), uniform_leaves(level)]
    C = blocks[refine_block]["corners"]

    def centre(lf):
        L, i, j, k = lf
        xi = -1.0 + (2.0 * np.array([i, j, k], dtype=np.float64) + 1.0) / (1 << L)
        w = [0.5 * (1 - xi[0]), 0.5 * (1 + xi[0])], [0.5 * (1 - xi[1]), 0.5 * (1 + xi[1])], \
            [0.5 * (1 - xi[2]), 0.5 * (1 + xi[2])]
        return sum(w[0][c & 1] * w[1][(c >> 1) & 1] * w[2][(c >> 2) & 1] * C[c] for c in range(8))

    dist = [np.linalg.norm(centre(lf) - np.array([1.0, 0.0, 0.0])) for lf in per[refine_block]]
    chosen = set(tuple(per[refine_block][i]) for i in np.argsort(dist)[:refine_count])
    per[refine_block] = morton_sort(refine(per[refine_block], lambda lf: tuple(lf) in chosen))
    rng = np.random.default_rng(seed)
    n = sum(len(v) for v in per)
    return _block_mesh(blocks, per, rng.integers(pmin, pmax + 1, size=n))


def cubed_sphere_blocks(a=2.0, r=10.0, r_out=None):
    """Centre cube [-a, a]^3, six wedges out to the sphere of radius r and, if
    r_out is given, six inverse-radius shell blocks from r to r_out (13 blocks)."""
    blocks = [hex8_box((-a, -a, -a), (a, a, a))]
    blocks += [dict(kind="wedge", face=f, a=a, r=r) for f in range(6)]
    if r_out is not None:
        blocks += [dict(kind="shell", face=f, r1=r, r2=r_out) for f in range(6)]
    return blocks


def cubed_sphere_mesh(level=1, a=2.0, r=10.0, r_out=None, seed=0, pmin=3, pmax=5, refine_wedge=None):
    """Every block at `level`, p ~ U{pmin..pmax} (seed).  refine_wedge = (block,
    count): the `count` first leaves (Morton order) of that wedge refined once,
    giving 2:1 faces on wedge-wedge, wedge-cube and wedge-shell interfaces."""
    blocks = cubed_sphere_blocks(a, r, r_out)
    per = [uniform_leaves(level) for _ in blocks]
    if refine_wedge is not None:
        b, count = refine_wedge
        chosen = set(per[b][:count])
        per[b] = morton_sort(refine(per[b], lambda lf: tuple(lf) in chosen))
    rng = np.random.default_rng(seed)
    n = sum(len(v) for v in per)
    return _block_mesh(blocks, per, rng.integers(pmin, pmax + 1, size=n))


def star_sphere_mesh(level=3, refine=2, seed=3, p_cut=4, p_lo=5, p_hi=8, a=2.0, r=10.0, r_out=1e9):
    """The density-jump star on the 13-block cubed sphere: centre cube of
    half-width a, wedges out to r, inverse-radius shell to r_out; every block
    at `level`; centre-cube cells cut by the spheres r = 0.5 and r = 1 refined
    `refine` times (2:1 balanced inside the cube, at most one level finer than
    the wedges on the cube faces); p = p_cut on the finest cut cells, p ~
    U{p_lo..p_hi} (seed) elsewhere."""
    blocks = cubed_sphere_blocks(a, r, r_out)
    lo, hi = (-a, -a, -a), (a, a, a)
    centre = uniform_leaves(level)

    def cut(lf):
        x0, x1 = _cell_bounds(lf, lo, hi)
        dmin, dmax = _dist_range(x0, x1)
        return any(dmin <= s <= dmax for s in (0.5, 1.0))

    for _ in range(refine):
        centre = balance_2to1(refine_(centre, cut))
    for L, i, j, k in centre:
        m = 1 << L
        if (min(i, j, k) == 0 or max(i, j, k) == m - 1) and L > level + 1:
            raise ValueError("refinement reaches the cube faces: raise `level` or lower `refine`")
    centre = morton_sort(centre)
    per = [centre] + [uniform_leaves(level) for _ in blocks[1:]]
    rng = np.random.default_rng(seed)
    maxL = max(lf[0] for lf in centre)
    p = []
    for b, leaves in enumerate(per):
        for lf in leaves:
            pv = int(rng.integers(p_lo, p_hi + 1))
            p.append(p_cut if (b == 0 and lf[0] == maxL and cut(lf)) else pv)
    return _block_mesh(blocks, per, p)


def oracle_block_mesh_args(desc):
    """Positional arguments for the oracle's BlockMesh constructor."""
    return desc["blocks"], desc["elem_block"], desc["leaves"], desc["p"]


def _cell_points(block, lf):
    """Physical corners and centre of a leaf of a block (cell selection only)."""
    L, i, j, k = lf
    pts = []
    for c in range(9):
        off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], dtype=np.float64) if c < 8 else np.full(3, 0.5)
        xi = -1.0 + 2.0 * (np.array([i, j, k], dtype=np.float64) + off) / (1 << L)
        if block["kind"] == "hex8":
            C = np.asarray(block["corners"], dtype=np.float64)
            w = [(0.5 * (1 - xi[0]), 0.5 * (1 + xi[0])), (0.5 * (1 - xi[1]), 0.5 * (1 + xi[1])),
                 (0.5 * (1 - xi[2]), 0.5 * (1 + xi[2]))]
            pts.append(sum(w[0][q & 1] * w[1][(q >> 1) & 1] * w[2][(q >> 2) & 1] * C[q] for q in range(8)))
            continue
        d, s = divmod(int(block["face"]), 2)
        t1, t2 = ((d + 1) % 3, (d + 2) % 3) if s else ((d + 2) % 3, (d + 1) % 3)
        v = np.zeros(3)
        v[d] = 1.0 if s else -1.0
        v[t1], v[t2] = xi[0], xi[1]
        t = 0.5 * (xi[2] + 1.0)
        u = v / np.linalg.norm(v)
        if block["kind"] == "wedge":
            pts.append((1 - t) * block["a"] * v + t * block["r"] * u)
        else:
            pts.append(u / ((1 - t) / block["r1"] + t / block["r2"]))
    return np.array(pts)


def puncture_sphere_mesh(punctures, level=2, a=2.0, r=10.0, r_out=20.0, p_base=4, p_fine=6):
    """Puncture initial data on the 13-block cubed sphere (centre cube a, wedges
    to r, inverse-radius shell to r_out, u = 0 there): every block at `level`,
    the cells whose bounding box (grown by a quarter of its size) holds a
    puncture refined once (2:1 across block interfaces at most), p_fine on the
    refined cells, p_base elsewhere."""
    blocks = cubed_sphere_blocks(a, r, r_out)
    cs = [np.asarray(c, dtype=np.float64) for (_, c, _) in punctures]
    per, p = [], []
    for blk in blocks:
        leaves = uniform_leaves(level)

        def near(lf):
            P = _cell_points(blk, lf)
            lo, hi = P.min(axis=0), P.max(axis=0)
            grow = 0.25 * (hi - lo)
            return any(np.all(c >= lo - grow) and np.all(c <= hi + grow) for c in cs)

        leaves = morton_sort(refine(leaves, near))
        per.append(leaves)
        p += [p_fine if lf[0] > level else p_base for lf in leaves]
    return _block_mesh(blocks, per, p)


# ---- constant-density star: Lap psi + 2 pi rho psi^5 = 0, psi -> 1 at infinity ----
def constant_density_star(rho0=1e-3, r0=1.0):
    """Closed-form solution of the constant-density star (density rho0 inside
    r0): psi = C u_a(r) inside with u_a = (a r0)^(1/2) / (r^2 + (a r0)^2)^(1/2),
    C = (2 pi rho0 / 3)^(-1/4), and psi = b / r + 1 outside, b = r0 (C u_a(r0)
    - 1).  a follows from continuity of psi' at r0, which works out to
    rho0 r0^2 = 3 a^10 / (2 pi (1 + a^2)^6) (the paper prints the power 3 of
    (1 + a^2), with which psi' jumps at r0).  The right side rises up to
    a = sqrt(5) and falls after it; the weak-field root a > sqrt(5) (psi -> 1
    as rho0 -> 0, the solution Newton reaches from psi = 1) is taken.
    Returns dict(a, b, C, psi, rho, coef) with psi, rho and coef = 2 pi rho
    callables on points (P, 3)."""
    target = rho0 * r0 * r0 * 2.0 * np.pi / 3.0
    lo, hi = np.sqrt(5.0), 1e8
    for _ in range(300):
        mid = np.sqrt(lo * hi)
        if mid ** 10 / (1.0 + mid * mid) ** 6 > target:
            lo = mid
        else:
            hi = mid
    a = np.sqrt(lo * hi)
    C = (2.0 * np.pi * rho0 / 3.0) ** -0.25
    ua = lambda r: np.sqrt(a * r0) / np.sqrt(r * r + (a * r0) ** 2)
    b = r0 * (C * ua(r0) - 1.0)

    def psi(x):
        r = np.linalg.norm(np.asarray(x, dtype=np.float64).reshape(-1, 3), axis=1)
        return np.where(r <= r0, C * ua(r), b / np.maximum(r, 1e-300) + 1.0)

    def rho(x):
        r = np.linalg.norm(np.asarray(x, dtype=np.float64).reshape(-1, 3), axis=1)
        return np.where(r <= r0, rho0, 0.0)

    return dict(a=a, b=b, C=C, psi=psi, rho=rho, coef=lambda x: 2.0 * np.pi * rho(x))


def const_star_mesh(R=8.0, level=2, refine=2, p=4, r0=1.0):
    """Box [-R, R]^3 (the paper's boundary at 8 r0), uniform level `level`,
    cells cut by the star surface r = r0 refined `refine` times (2:1
    balanced); degree p everywhere."""
    lo, hi = (-R, -R, -R), (R, R, R)
    leaves = uniform_leaves(level)

    def cut(lf):
        a, b = _cell_bounds(lf, lo, hi)
        dmin, dmax = _dist_range(a, b)
        return dmin <= r0 <= dmax

    for _ in range(refine):
        leaves = balance_2to1(refine_(leaves, cut))
    leaves = morton_sort(leaves)
    return dict(lo=lo, hi=hi, leaves=np.array(leaves, dtype=np.int32), p=np.full(len(leaves), p, dtype=np.int32),
                warp=None)
