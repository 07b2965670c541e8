"""Parity at the full operator-apply sweep size (32^3 + refined octant, 61,440
elements, 1.3e7 DOFs) in the launch configuration bench.py times: the oracle
computes a seeded sample of element outputs one by one (dense local blocks of
each element and its mortars)."""
import numpy as np
import pytest

from gpu_util import oracle_mesh
from oracle import sipg
from paper_1907_01572_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_sweep32_sampled_elements_fp64_fp32():
    import torch
    from paper_1907_01572_gb300 import dgell
    desc = inputs.sweep_mesh(level=5, seed=0)
    m = oracle_mesh(desc)
    ctx = dgell.Context(desc)
    assert ctx.level_info()["n_dofs"] == m.n_dofs == 13151246
    x = inputs.random_vector(m.n_dofs, seed=1)
    xd = torch.tensor(x, device="cuda")
    y64 = torch.empty_like(xd)
    ctx.apply(xd, y64)
    x32 = xd.float()
    y32 = torch.empty_like(x32)
    ctx.apply(x32, y32)
    x32h = x32.double().cpu().numpy()
    rng = np.random.default_rng(123)
    # random elements plus the ones that own 2:1 faces (coarse side) and the last (ragged tail)
    coarse_21 = [e for e in range(m.n_elems) if any(len(m.elem_mortars[e][f]) == 4 for f in range(6))]
    sample = sorted(set(rng.choice(m.n_elems, 20, replace=False).tolist() + coarse_21[:4] + [m.n_elems - 1]))
    ref64 = sipg.apply_local(m, x, 10.0, elems=sample)
    ref32 = sipg.apply_local(m, x32h, 10.0, elems=sample)
    y64h = y64.cpu().numpy()
    y32h = y32.double().cpu().numpy()
    num64 = den64 = num32 = den32 = 0.0
    for e in sample:
        a, b = m.dof_off[e], m.dof_off[e + 1]
        num64 += np.sum((y64h[a:b] - ref64[e]) ** 2)
        den64 += np.sum(ref64[e] ** 2)
        num32 += np.sum((y32h[a:b] - ref32[e]) ** 2)
        den32 += np.sum(ref32[e] ** 2)
        assert np.linalg.norm(y64h[a:b] - ref64[e]) <= 1e-12 * np.linalg.norm(ref64[e]) * 10
    assert np.sqrt(num64 / den64) < 1e-12
    assert np.sqrt(num32 / den32) < 1e-5
    # property at full size: the operator is symmetric -> x^T L z = z^T L x
    z = torch.tensor(inputs.random_vector(m.n_dofs, seed=2), device="cuda")
    Lz = torch.empty_like(z)
    ctx.apply(z, Lz)
    a1 = float(torch.dot(xd, Lz))
    a2 = float(torch.dot(z, y64))
    assert abs(a1 - a2) < 1e-10 * abs(a1)
    ctx.close()


@pytest.mark.parametrize("level", [3, 4])
def test_mid_size_levels_sampled(level):
    """Meshes of 960 and 7,680 elements run the single-launch warp-per-element
    path (the smallest test meshes run the CTA-per-element path and the full
    sweep the per-bucket path): sampled elements against the oracle."""
    import torch
    from paper_1907_01572_gb300 import dgell
    desc = inputs.sweep_mesh(level=level, seed=0)
    m = oracle_mesh(desc)
    ctx = dgell.Context(desc)
    x = inputs.random_vector(m.n_dofs, seed=3)
    xd = torch.tensor(x, device="cuda")
    y = torch.empty_like(xd)
    ctx.apply(xd, y)
    y32 = torch.empty_like(xd.float())
    ctx.apply(xd.float(), y32)
    rng = np.random.default_rng(level)
    sample = sorted(set(rng.choice(m.n_elems, 12, replace=False).tolist() + [0, m.n_elems - 1]))
    ref = sipg.apply_local(m, x, 10.0, elems=sample)
    ref32 = sipg.apply_local(m, xd.float().double().cpu().numpy(), 10.0, elems=sample)
    yh, y32h = y.cpu().numpy(), y32.double().cpu().numpy()
    num = den = num32 = den32 = 0.0
    for e in sample:
        a, b = m.dof_off[e], m.dof_off[e + 1]
        num += np.sum((yh[a:b] - ref[e]) ** 2)
        num32 += np.sum((y32h[a:b] - ref32[e]) ** 2)
        den += np.sum(ref[e] ** 2)
        den32 += np.sum(ref32[e] ** 2)
    assert np.sqrt(num / den) < 1e-12 and np.sqrt(num32 / den32) < 1e-5
    ctx.close()
