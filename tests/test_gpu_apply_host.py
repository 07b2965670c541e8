"""dg_apply_host: the operator applied to vectors held in host memory, with the
copies in and out overlapping the applies.  Its outputs must equal dg_apply's
on the same inputs bit for bit (the same kernels run on device copies of the
inputs), for pinned and pageable host memory, FP64 and FP32, odd and even
vector counts (staging slots reused), and one of them must match the oracle's
assembled operator."""
import numpy as np
import pytest

from gpu_util import CASES, oracle_mesh, rel_l2
from oracle import sipg
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


@pytest.mark.parametrize("name", ["mixed_curved_2to1_l2", "cubed_sphere_shell_2to1"])
def test_apply_host_equals_device_apply(name, torch):
    from paper_1907_01572_gb300 import dgell
    desc = CASES[name]()
    ctx = dgell.Context(desc)
    n = ctx.level_info()["n_dofs"]
    for dtype in (torch.float64, torch.float32):
        for nvec, pinned in ((1, True), (4, True), (5, False)):
            X = torch.stack([torch.tensor(inputs.random_vector(n, seed=40 + r)) for r in range(nvec)]).to(dtype)
            hx = X.pin_memory() if pinned else X.clone()
            hy = torch.full_like(hx, float("nan"))
            if pinned:
                hy = hy.pin_memory()
            ctx.apply_host(hx, hy)
            torch.cuda.current_stream().synchronize()
            for r in range(nvec):
                y = torch.empty(n, dtype=dtype, device="cuda")
                ctx.apply(X[r].cuda(), y)
                assert torch.equal(hy[r], y.cpu()), (name, dtype, nvec, pinned, r)
    ctx.close()


def test_apply_host_against_oracle_and_guards(torch):
    from paper_1907_01572_gb300 import dgell
    desc = CASES["affine_2to1_p2to8"]()
    m = oracle_mesh(desc)
    A = sipg.assemble(m, 10.0)
    ctx = dgell.Context(desc)
    n = ctx.level_info()["n_dofs"]
    X = np.stack([inputs.random_vector(n, seed=60 + r) for r in range(3)])
    hx = torch.tensor(X).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    ctx.apply_host(hx, hy)
    torch.cuda.current_stream().synchronize()
    for r in range(3):
        assert rel_l2(hy[r].numpy(), A @ X[r]) < 1e-12
    # nvec = 0 does nothing; BF16 and device tensors are refused
    assert dgell.lib().dg_apply_host(ctx.h, -1, dgell.DG_FP32, 0, None, None) == dgell.DG_OK
    assert dgell.lib().dg_apply_host(ctx.h, -1, dgell.DG_BF16, 1, dgell._ptr(hx), dgell._ptr(hy)) == \
        dgell.DG_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        ctx.apply_host(hx.cuda(), hy)
    ctx.close()
