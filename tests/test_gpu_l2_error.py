"""The benchmark's L2 error against a closed form, computed from library calls
only (two applies for M u_h, dg_rhs for the projections), equals the oracle's
||u_h - u||_2 (eq. l2norm) with the same GL quadrature, on config 1 and on a
star on the 13-block cubed sphere."""
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


def _sine(X):
    return np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])


@pytest.mark.parametrize("case", ["config1", "star_sphere"])
def test_l2_error_from_library_calls_matches_oracle(case):
    import torch
    import bench
    from paper_1907_01572_gb300 import dgell
    if case == "config1":
        desc, gfun, ufun = inputs.config1_mesh(), lambda X: 3 * np.pi ** 2 * _sine(X), _sine
    else:
        desc = inputs.star_sphere_mesh(level=1, refine=0, p_cut=3, p_lo=3, p_hi=4, r_out=20.0)
        gfun, ufun = inputs.star_source, inputs.star_solution
    ctx = dgell.Context(desc)
    xyz, bxyz = ctx.quadrature_points()
    gq = torch.tensor(gfun(xyz.T.cpu().numpy()), device="cuda")
    gd = torch.tensor(ufun(bxyz.T.cpu().numpy()), device="cuda") if bxyz.shape[1] else None
    F = torch.empty(ctx.level_info()["n_dofs"], dtype=torch.float64, device="cuda")
    ctx.rhs(gq, gd, F)
    u = torch.zeros_like(F)
    ctx.solve(F, u, tol=1e-10, max_iter=200)
    e_gpu = bench.l2_error_closed_form(dgell, torch, desc, u, ufun)
    e_or = sipg.l2_error(oracle_mesh(desc), u.cpu().numpy(), ufun, extra=0)
    assert e_gpu is not None and abs(e_gpu - e_or) < 1e-9 * e_or, (e_gpu, e_or)
    ctx.close()
