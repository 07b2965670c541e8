"""dg_smooth_static -- the smoother for callers that cannot allocate device
memory when they smooth (memory fully handed to a caching allocator, or loops
that cannot accept cudaMalloc's device synchronisation) -- gives the same
result as dg_smooth, on two calls in a row through the C ABI, and rejects
levels larger than its fixed scratch array.  Collected last on purpose."""
import numpy as np
import pytest

from gpu_util import CASES, rel_l2
from paper_1907_01572_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name", ["config1_affine_p3", "mixed_curved_2to1_l1"])
def test_static_smoother_matches_allocating_one(name):
    import torch
    from paper_1907_01572_gb300 import dgell
    ctx = dgell.Context(CASES[name]())
    n = ctx.level_info()["n_dofs"]
    b = torch.tensor(inputs.random_vector(n, seed=31), device="cuda")
    x0 = torch.tensor(0.1 * inputs.random_vector(n, seed=32), device="cuda")
    for call in range(2):
        for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            bb = b.to(dtype)
            x_ref = x0.to(dtype).clone()
            lam_ref = ctx.smooth(bb, x_ref)
            x_st = x0.to(dtype).clone()
            lam_st = ctx.smooth_static(bb, x_st)
            torch.cuda.synchronize()
            assert abs(lam_st - lam_ref) <= tol * abs(lam_ref), (call, dtype)
            assert rel_l2(x_st.double().cpu().numpy(), x_ref.double().cpu().numpy()) <= tol, (call, dtype)
    # coarse levels too.  On levels of at most 1024 DOFs dg_smooth applies the assembled operator
    # and dg_smooth_static applies it matrix-free, so in FP32 the two differ by rounding; with a
    # fixed Chebyshev bound (no CG steps, a linear smoother) that rounding stays at the FP32 level.
    for l in range(ctx.n_levels - 1):
        nl = ctx.level_info(l)["n_dofs"]
        bl = torch.tensor(inputs.random_vector(nl, seed=40 + l), device="cuda")
        xa = torch.zeros_like(bl)
        xb = torch.zeros_like(bl)
        lam = ctx.smooth(bl, xa, level=l)
        ctx.smooth_static(bl, xb, level=l)
        assert rel_l2(xb.cpu().numpy(), xa.cpu().numpy()) <= 1e-12
        b32 = bl.float()
        xa32 = torch.zeros_like(b32)
        xb32 = torch.zeros_like(b32)
        ctx.smooth(b32, xa32, level=l, lam_fixed=1.05 * lam)
        ctx.smooth_static(b32, xb32, level=l, lam_fixed=1.05 * lam)
        torch.cuda.synchronize()
        assert rel_l2(xb32.double().cpu().numpy(), xa32.double().cpu().numpy()) <= 1e-5, l
    ctx.close()


def test_static_smoother_rejects_oversized_level():
    import torch
    from paper_1907_01572_gb300 import dgell
    ctx = dgell.Context(inputs.sweep_mesh(level=4, seed=0))
    n = ctx.level_info()["n_dofs"]
    assert n > 262144
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(dgell.DgError) as e:
        ctx.smooth_static(b, torch.zeros_like(b))
    assert e.value.code == dgell.DG_ERR_INVALID
    # coarser levels of the same context fit
    l = ctx.n_levels - 2
    nl = ctx.level_info(l)["n_dofs"]
    assert nl <= 262144
    bl = torch.tensor(np.ones(nl), device="cuda")
    xl = torch.zeros_like(bl)
    ctx.smooth_static(bl, xl, level=l)
    assert torch.isfinite(xl).all()
    ctx.close()
