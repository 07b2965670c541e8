"""GPU parity of the operator apply (eq. lh2) against the oracle's assembled
SIPG matrix: FP64 within 1e-12 relative L2, FP32 within 1e-5 (the FP32 path
gets x rounded to float; the oracle applies the same rounded x in FP64)."""
import numpy as np
import pytest

from gpu_util import CASES, oracle_mesh, rel_l2
from oracle import multigrid, sipg
from paper_1907_01572_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


_MATS = {}


def oracle_matrix(name):
    if name not in _MATS:
        desc = CASES[name]()
        m = oracle_mesh(desc)
        _MATS[name] = (desc, m, sipg.assemble(m, 10.0))
    return _MATS[name]


@pytest.mark.parametrize("name", sorted(CASES))
def test_apply_fp64_and_fp32(name, torch):
    from paper_1907_01572_gb300 import dgell
    desc, m, A = oracle_matrix(name)
    ctx = dgell.Context(desc)
    assert ctx.level_info()["n_dofs"] == m.n_dofs
    x = inputs.random_vector(m.n_dofs, seed=1)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    ctx.apply(xd, yd)
    assert rel_l2(yd.cpu().numpy(), A @ x) < 1e-12
    x32 = xd.float()
    y32 = torch.empty_like(x32)
    ctx.apply(x32, y32)
    ref = A @ x32.double().cpu().numpy()
    assert rel_l2(y32.double().cpu().numpy(), ref) < 1e-5
    # BF16 operands, FP32 arithmetic: exact-input parity 1e-5, and within 2e-3
    # of the FP64 operator applied to the unrounded input
    x16 = xd.bfloat16()
    y16 = torch.empty(m.n_dofs, dtype=torch.float32, device="cuda")
    ctx.apply(x16, y16)
    assert rel_l2(y16.double().cpu().numpy(), A @ x16.double().cpu().numpy()) < 1e-5
    assert rel_l2(y16.double().cpu().numpy(), A @ x) < 2e-3
    # repeat: deterministic, bit-identical
    y2 = torch.empty_like(xd)
    ctx.apply(xd, y2)
    assert torch.equal(yd, y2)
    ctx.close()


def test_apply_rejects_aliasing_and_bad_level(torch):
    from paper_1907_01572_gb300 import dgell
    ctx = dgell.Context(CASES["config1_affine_p3"]())
    x = torch.zeros(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(dgell.DgError):
        ctx.apply(x, x)
    with pytest.raises(dgell.DgError):
        ctx.apply(x, torch.empty_like(x), level=7)
    ctx.close()


@pytest.mark.parametrize("name", ["config1_affine_p3", "mixed_curved_2to1_l1"])
def test_hierarchy_matches_oracle_and_coarse_apply(name, torch):
    """Level meshes (Sec. II.E.3) equal the oracle's, element for element, and
    the re-discretised operator on every level matches."""
    from paper_1907_01572_gb300 import dgell
    desc = CASES[name]()
    ctx = dgell.Context(desc)
    meshes, groups = multigrid.hierarchy(oracle_mesh(desc))
    assert ctx.n_levels == len(meshes)
    for l, m in enumerate(meshes):
        leaves, p, off = ctx.level_leaves(l)
        assert np.array_equal(leaves, m.leaves) and np.array_equal(p, m.p)
        A = sipg.assemble(m, 10.0)
        x = inputs.random_vector(m.n_dofs, seed=5 + l)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        ctx.apply(xd, yd, level=l)
        assert rel_l2(yd.cpu().numpy(), A @ x) < 1e-12
    # transfers: prolongation and restriction against the oracle's I_h^H
    for l in range(len(meshes) - 1):
        P = multigrid.prolongation(meshes[l + 1], meshes[l], groups[l])
        xc = inputs.random_vector(meshes[l].n_dofs, seed=11)
        xf = inputs.random_vector(meshes[l + 1].n_dofs, seed=12)
        out = torch.tensor(xf, device="cuda")
        ctx.transfer(l, 0, torch.tensor(xc, device="cuda"), out)
        assert rel_l2(out.cpu().numpy(), xf + P @ xc) < 1e-13
        outc = torch.empty(meshes[l].n_dofs, dtype=torch.float64, device="cuda")
        ctx.transfer(l, 1, torch.tensor(xf, device="cuda"), outc)
        assert rel_l2(outc.cpu().numpy(), P.T @ xf) < 1e-13
    ctx.close()
