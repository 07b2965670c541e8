"""dg_estimate (eqs. Eta2_Ingredients, Eta2_Integrals, Eta2_Local) against the
oracle estimator on the same seeded meshes and fields (FP64, per element),
its closed forms and zero cases on the GPU, the sampled full-size sweep mesh,
and the hp-adaptive loop (Algorithm 4) through the C ABI."""
import math

import numpy as np
import pytest

from gpu_util import CASES, oracle_mesh, rel_l2
from oracle import estimator, hpamr, sipg
from paper_1907_01572_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    import __graft_entry__
    __graft_entry__.build()
    return t


def g_np(x):
    return np.sin(2 * x[:, 0]) * np.cos(x[:, 1]) + 0.5 * x[:, 2] ** 2


def f_np(x):
    return 1.0 + 0.5 * x[:, 0] ** 2 + 0.25 * x[:, 1] * x[:, 2]


def gD_np(x):
    return np.exp(0.3 * x[:, 0]) - x[:, 1] * x[:, 2]


def _fields(ctx, torch):
    vxyz, bxyz = ctx.quadrature_points()
    v = vxyz.T.cpu().numpy()
    b = bxyz.T.cpu().numpy()
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    return dev(g_np(v)), dev(f_np(v)), dev(gD_np(b))


def _estimate(ctx, u, torch, g=None, f=None, gD=None):
    eta = torch.empty(ctx.level_info()["n_elems"], dtype=torch.float64, device="cuda")
    ctx.estimate(u, eta, g_qp=g, f_qp=f, gD_qp=gD)
    torch.cuda.synchronize()
    return eta.cpu().numpy()


@pytest.mark.parametrize("name", ["config1_affine_p3", "mixed_curved_2to1_l1", "affine_2to1_p2to8",
                                  "single_element_p8_curved", "uniform_p8_2x2x2"])
def test_estimator_matches_oracle(name, torch):
    from paper_1907_01572_gb300 import dgell
    desc = CASES[name]()
    m = oracle_mesh(desc)
    ctx = dgell.Context(desc)
    u = inputs.random_vector(m.n_dofs, seed=21)
    g, f, gD = _fields(ctx, torch)
    eta = _estimate(ctx, torch.tensor(u, device="cuda"), torch, g, f, gD)
    ref = estimator.estimate(m, u, g_fn=g_np, f_fn=f_np, gD_fn=gD_np, C=10.0)
    assert rel_l2(eta, ref) < 1e-12
    assert np.max(np.abs(eta - ref) / ref) < 1e-10
    # without the optional fields (g = f = g_D = 0)
    eta0 = _estimate(ctx, torch.tensor(u, device="cuda"), torch)
    assert rel_l2(eta0, estimator.estimate(m, u, C=10.0)) < 1e-12
    ctx.close()


def test_closed_forms_and_exact_solutions(torch):
    """Indicator of one unit cube (p = 2, C = 10): 960 there and 160 on its
    face neighbours; u = 0, g = 1: 12 per cube; a quadratic solution on an
    affine 2:1 / degree-jump mesh: zero up to rounding."""
    from paper_1907_01572_gb300 import dgell
    lv = inputs.uniform_leaves(1)
    desc = dict(lo=(-1, -1, -1), hi=(1, 1, 1), leaves=np.array(lv, dtype=np.int32),
                p=np.full(8, 2, dtype=np.int32), warp=None)
    ctx = dgell.Context(desc)
    n = ctx.level_info()["n_dofs"]
    e0 = lv.index((1, 0, 0, 0))
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    u[27 * e0:27 * (e0 + 1)] = 1.0
    eta = _estimate(ctx, u, torch)
    exp = np.zeros(8)
    exp[e0] = 960.0
    for nb in [(1, 1, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1)]:
        exp[lv.index(nb)] = 160.0
    assert np.allclose(eta, exp, rtol=1e-12, atol=1e-10)
    nv = ctx.level_info()["n_vol_qp"]
    eta = _estimate(ctx, torch.zeros(n, dtype=torch.float64, device="cuda"), torch,
                    g=torch.ones(nv, dtype=torch.float64, device="cuda"))
    assert np.allclose(eta, 12.0, rtol=1e-12)
    ctx.close()

    desc = CASES["affine_2to1_p2to8"]()
    m = oracle_mesh(desc)
    ctx = dgell.Context(desc)
    P = lambda x: 0.3 + x[:, 0] - 0.5 * x[:, 1] + 2 * x[:, 1] ** 2 - x[:, 0] * x[:, 2] + 0.7 * x[:, 2] ** 2
    vxyz, bxyz = ctx.quadrature_points()
    v, b = vxyz.T.cpu().numpy(), bxyz.T.cpu().numpy()
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    g = dev(-5.4 + f_np(v) * P(v))
    eta = _estimate(ctx, dev(sipg.interpolate(m, P)), torch, g=g, f=dev(f_np(v)), gD=dev(P(b)))
    ref = _estimate(ctx, dev(sipg.interpolate(m, lambda x: x[:, 0] ** 3)), torch, g=g, f=dev(f_np(v)), gD=dev(P(b)))
    assert eta.max() < 1e-18 * ref.max()
    ctx.close()


@pytest.mark.parametrize("name", ["blocks_turned_fine_side", "cubed_sphere_shell_2to1"])
def test_estimator_on_block_meshes_matches_oracle(name, torch):
    """Multi-block meshes (exact block maps and their second derivatives in
    Lap u; turned interfaces, wedges and an inverse-radius shell with 2:1
    faces): eta^2(e) within 1e-12 relative L2 (1e-10 per element) of the
    oracle's, with and without the problem data."""
    from paper_1907_01572_gb300 import dgell
    desc = CASES[name]()
    m = oracle_mesh(desc)
    ctx = dgell.Context(desc)
    u = inputs.random_vector(m.n_dofs, seed=22)
    g, f, gD = _fields(ctx, torch)
    eta = _estimate(ctx, torch.tensor(u, device="cuda"), torch, g, f, gD)
    ref = estimator.estimate(m, u, g_fn=g_np, f_fn=f_np, gD_fn=gD_np, C=10.0)
    assert rel_l2(eta, ref) < 1e-12
    assert np.max(np.abs(eta - ref) / ref) < 1e-10
    eta0 = _estimate(ctx, torch.tensor(u, device="cuda"), torch)
    assert rel_l2(eta0, estimator.estimate(m, u, C=10.0)) < 1e-12
    ctx.close()


def test_fiducial_grid_estimator_matches_oracle(torch):
    """The compactified cubed sphere (cube half-width 2, wedges to r = 10,
    inverse-radius shell to r = 1e4) estimated on Problem C's fiducial grid
    (cube of side 2/sqrt(3), wedges to r = 2, shell from 2 to 3): eta^2(e)
    against the oracle's fiducial estimator; the fiducial weights change the
    shell elements' eta^2 by orders of magnitude; mismatched fiducial blocks
    are rejected."""
    from paper_1907_01572_gb300 import dgell
    desc = inputs.cubed_sphere_mesh(level=1, a=2.0, r=10.0, r_out=1e4, seed=4, pmin=2, pmax=4)
    fid = inputs.cubed_sphere_blocks(a=1.0 / math.sqrt(3.0), r=2.0, r_out=3.0)
    m = oracle_mesh(desc)
    mf = m.with_blocks(fid)
    ctx = dgell.Context(desc)
    u = inputs.random_vector(m.n_dofs, seed=23)
    # fields bounded out to r = 1e4: the Lorentzian's source and solution, f = 1 + 1 / (1 + r^2)
    f_l = lambda x: 1.0 + 1.0 / (1.0 + np.sum(x * x, axis=1))
    vxyz, bxyz = ctx.quadrature_points()
    v, b = vxyz.T.cpu().numpy(), bxyz.T.cpu().numpy()
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    g, f, gD = dev(inputs.lorentzian_source(v)), dev(f_l(v)), dev(inputs.lorentzian_solution(b))
    ud = torch.tensor(u, device="cuda")
    eta = torch.empty(m.n_elems, dtype=torch.float64, device="cuda")
    ctx.estimate(ud, eta, g_qp=g, f_qp=f, gD_qp=gD, fiducial=fid)
    eta = eta.cpu().numpy()
    ref = estimator.estimate(m, u, g_fn=inputs.lorentzian_source, f_fn=f_l, gD_fn=inputs.lorentzian_solution,
                             C=10.0, fiducial=mf)
    assert rel_l2(eta, ref) < 1e-12
    assert np.max(np.abs(eta - ref) / ref) < 1e-10
    phys = _estimate(ctx, ud, torch, g, f, gD)
    shell = np.asarray(desc["elem_block"]) >= 7
    assert np.median(phys[shell] / eta[shell]) > 1e3
    bad = [dict(b) for b in fid]
    bad[3] = dict(bad[3], kind="shell", face=bad[3]["face"], r1=2.0, r2=3.0)
    with pytest.raises(dgell.DgError) as ei:
        ctx.estimate(ud, torch.empty_like(torch.tensor(eta, device="cuda")), fiducial=bad)
    assert ei.value.code == dgell.DG_ERR_INVALID
    ctx.close()


def test_sweep32_sampled_elements(torch):
    """The full operator-apply sweep mesh (61,440 elements, 1.3e7 DOFs): the
    oracle computes a seeded sample of elements one by one."""
    from paper_1907_01572_gb300 import dgell
    desc = inputs.sweep_mesh(level=5, seed=0)
    m = oracle_mesh(desc)
    ctx = dgell.Context(desc)
    u = inputs.random_vector(m.n_dofs, seed=1)
    g, f, gD = _fields(ctx, torch)
    eta = _estimate(ctx, torch.tensor(u, device="cuda"), torch, g, f, gD)
    rng = np.random.default_rng(5)
    sample = sorted(set(rng.choice(m.n_elems, size=16, replace=False).tolist()) | {0, m.n_elems - 1})
    ref = estimator.estimate(m, u, g_fn=g_np, f_fn=f_np, gD_fn=gD_np, C=10.0, elems=sample)
    assert np.max(np.abs(eta[sample] - ref) / ref) < 1e-10
    assert np.all(np.isfinite(eta)) and eta.min() > 0
    ctx.close()


def _front(x, xp):
    """u = atan(a (r - r0)), r = |x - c| with c outside the box: a steep
    spherical front; returns (u, -Lap u)."""
    a, r0 = 10.0, 1.5
    c = (-1.25, -1.25, -1.25)
    r = xp.sqrt((x[0] - c[0]) ** 2 + (x[1] - c[1]) ** 2 + (x[2] - c[2]) ** 2)
    s = a * (r - r0)
    d1 = a / (1 + s * s)
    d2 = -2 * a ** 3 * (r - r0) / (1 + s * s) ** 2
    return xp.arctan(s), -(d2 + 2 * d1 / r)


def test_hp_adaptive_loop(torch):
    """Three smooth-pred steps from a level-1, p = 2 mesh on a steep front:
    the marking on the GPU's eta^2 equals the oracle's, both h- and
    p-refinement occur, and the summed estimator and the true L2 error fall."""
    from paper_1907_01572_gb300 import amr, dgell
    lv = inputs.uniform_leaves(1)
    desc = dict(lo=(-1, -1, -1), hi=(1, 1, 1), leaves=np.array(lv, dtype=np.int32),
                p=np.full(8, 2, dtype=np.int32), warp=None)
    hist = amr.adapt(desc, g_fn=lambda x: _front(x, torch)[1], gD_fn=lambda x: _front(x, torch)[0],
                     steps=3, theta=0.3, keep_solution=True)
    assert len(hist) == 4
    errs, sums = [], []
    pred = np.full(8, math.inf)
    for k, h in enumerate(hist):
        assert h["rel_residual"] < 1e-10
        m = oracle_mesh(h["desc"])
        errs.append(sipg.l2_error(m, h["u"], lambda x: _front(x.T, np)[0]))
        sums.append(h["eta2"].sum())
        if h["action"] is not None:
            lvl = np.asarray(h["desc"]["leaves"])[:, 0]
            marked = hpamr.mark(list(h["eta2"]), 'fraction', 0.3)
            act, nxt = hpamr.smooth_pred(list(h["eta2"]), list(pred), list(h["desc"]["p"]), list(lvl), marked,
                                         0.25, 0.1)
            assert h["action"].tolist() == act
            out = hpamr.refine(np.asarray(h["desc"]["leaves"]).tolist(), list(h["desc"]["p"]), act, nxt, math.inf)
            nd = hist[k + 1]["desc"]
            pred = np.array([out[tuple(int(v) for v in lf)][1] for lf in np.asarray(nd["leaves"])])
    acts = np.concatenate([h["action"] for h in hist[:-1]])
    assert (acts == dgell.DG_AMR_H_REFINE).any() and (acts == dgell.DG_AMR_P_REFINE).any()
    assert sums[-1] < 0.25 * sums[0], sums
    assert errs[-1] < 0.25 * errs[0], errs
    assert hist[-1]["n_dofs"] > hist[0]["n_dofs"]


def test_hp_adaptive_loop_on_a_block_mesh(torch):
    """The adaptive loop on the 13-block cubed sphere (shell to r = 20, every
    block at level 1, p = 2) with the steep front inside it: every mesh is
    solved to 1e-10, the marking on the GPU's eta^2 equals the oracle's, the
    leaf set is refined across block interfaces (dg_hp_refine_mesh), and the
    summed estimator and the L2 error against the closed form fall."""
    from paper_1907_01572_gb300 import amr
    desc = inputs.cubed_sphere_mesh(level=1, a=2.0, r=10.0, r_out=20.0, seed=0, pmin=2, pmax=2)
    hist = amr.adapt(desc, g_fn=lambda x: _front(x, torch)[1], gD_fn=lambda x: _front(x, torch)[0],
                     steps=2, theta=0.3, keep_solution=True)
    assert len(hist) == 3
    errs, sums = [], []
    for h in hist:
        assert h["rel_residual"] < 1e-10
        m = oracle_mesh(h["desc"])
        errs.append(sipg.l2_error(m, h["u"], lambda x: _front(x.T, np)[0]))
        sums.append(h["eta2"].sum())
    # the first marking (predictions all infinite) against the oracle's
    h = hist[0]
    lvl = np.asarray(h["desc"]["leaves"])[:, 0]
    marked = hpamr.mark(list(h["eta2"]), 'fraction', 0.3)
    act, _ = hpamr.smooth_pred(list(h["eta2"]), [math.inf] * len(lvl), list(h["desc"]["p"]), list(lvl), marked,
                               0.25, 0.1)
    assert h["action"].tolist() == act
    assert hist[-1]["n_dofs"] > hist[0]["n_dofs"]
    assert len(np.asarray(hist[-1]["desc"]["elem_block"])) == hist[-1]["n_elems"]
    assert sums[-1] < sums[0], sums
    assert errs[-1] < errs[0], errs
