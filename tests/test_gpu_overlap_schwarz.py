"""GPU Schwarz smoother with overlapping subdomains (Alg. 6, eq. schwarz_weight;
one overlap layer, exact local solves) against the oracle's
overlap_schwarz_smoother inside the V-cycle (Alg. 3), and the solve it makes
possible: MG-FCG on the cubed sphere with the inverse-radius shell out to
r = 1e9, where the Chebyshev V-cycle stops converging."""
import numpy as np
import pytest

from gpu_util import oracle_level_mesh, oracle_mesh, rel_l2, CASES
from oracle import multigrid
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


def gpu_levels(ctx, desc):
    """The context's level meshes as oracle meshes, with the family groups of
    uniform refinement (every coarse leaf split into its 8 children, or
    carried over unchanged)."""
    nl = ctx.level_info()["n_levels"]
    meshes = [oracle_level_mesh(ctx, desc, l) for l in range(nl)]
    groups = []
    for l in range(nl - 1):
        fine, coarse = meshes[l + 1], meshes[l]
        fkey = {(int(b),) + tuple(int(v) for v in lf): e for e, (b, lf) in enumerate(zip(fine.elem_block, fine.leaves))}
        grp = []
        for b, lf in zip(coarse.elem_block, coarse.leaves):
            key = (int(b),) + tuple(int(v) for v in lf)
            if key in fkey:
                grp.append([(fkey[key], None)])
                continue
            L, i, j, k = (int(v) for v in lf)
            grp.append([(fkey[(int(b), L + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1))],
                         (c & 1, (c >> 1) & 1, (c >> 2) & 1)) for c in range(8)])
        groups.append(grp)
    return meshes, groups


def sphere(r_out):
    return inputs.cubed_sphere_mesh(level=1, a=2.0, r=10.0, r_out=r_out, seed=0, pmin=3, pmax=3)


@pytest.mark.parametrize("coarse", [1, 0])
def test_overlap_vcycle_matches_oracle_on_the_compactified_sphere(coarse, torch):
    from paper_1907_01572_gb300 import dgell
    desc = sphere(1e9)
    ctx = dgell.Context(desc)
    H = multigrid.Hierarchy(None, levels=gpu_levels(ctx, desc))
    f = inputs.random_vector(H.meshes[-1].n_dofs, seed=5)
    vo = H.vcycle(f, coarse='cholesky' if coarse else 'smoother', smoother_kind='schwarz_overlap', n_overlap=1)
    v = torch.empty(len(f), dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(f, device="cuda"), v, coarse=coarse, smoother=2, n_schwarz=3)
    assert rel_l2(v.cpu().numpy(), vo) < 1e-9
    ctx.close()


def test_overlap_vcycle_matches_oracle_on_a_box(torch):
    from paper_1907_01572_gb300 import dgell
    desc = CASES["config1_affine_p3"]()
    m = oracle_mesh(desc)
    H = multigrid.Hierarchy(m)
    ctx = dgell.Context(desc)
    f = inputs.random_vector(m.n_dofs, seed=6)
    vo = H.vcycle(f, coarse='cholesky', smoother_kind='schwarz_overlap', n_overlap=1)
    v = torch.empty(m.n_dofs, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(f, device="cuda"), v, coarse=1, smoother=2, n_schwarz=3)
    assert rel_l2(v.cpu().numpy(), vo) < 1e-9
    # FP32 (local inverses rounded to float): within 1e-5 of the oracle on the rounded input
    f32 = f.astype(np.float32)
    v32 = torch.empty(m.n_dofs, dtype=torch.float32, device="cuda")
    ctx.vcycle(torch.tensor(f32, device="cuda"), v32, coarse=1, smoother=2, n_schwarz=3)
    vo32 = H.vcycle(f32.astype(np.float64), coarse='cholesky', smoother_kind='schwarz_overlap', n_overlap=1)
    assert rel_l2(v32.cpu().double().numpy(), vo32) < 1e-5
    ctx.close()


@pytest.mark.parametrize("mg_prec", ["fp64", "fp32"])
def test_overlap_mg_fcg_converges_with_the_shell_to_1e9(mg_prec, torch):
    """FCG preconditioned by the overlap-smoothed V-cycle reaches 1e-10 on the
    sphere with the shell to r = 1e9 in at most 25 iterations (the oracle's
    count with this smoother is at most 25, pinned on the CPU), and the
    oracle's operator gives the solution the same small residual."""
    from paper_1907_01572_gb300 import dgell
    desc = sphere(1e9)
    ctx = dgell.Context(desc)
    H = multigrid.Hierarchy(None, levels=gpu_levels(ctx, desc))
    A = H.J[-1].tocsc()
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    prec = dgell.DG_FP64 if mg_prec == "fp64" else dgell.DG_FP32
    st = ctx.solve(torch.tensor(b, device="cuda"), x, tol=1e-10, max_iter=60, mg_prec=prec, smoother=2, coarse=1)
    assert st["rel_residual"] < 1e-10 and st["iterations"] <= 25, st
    # the oracle's operator agrees (its own residual of the GPU solution)
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xh) / np.linalg.norm(b) < 1e-8
    ctx.close()


def test_overlap_needs_one_degree_and_conforming_faces(torch):
    from paper_1907_01572_gb300 import dgell
    for desc in (inputs.cubed_sphere_mesh(level=1, a=2.0, r=10.0, r_out=20.0, seed=1, pmin=2, pmax=4),
                 CASES["mixed_curved_2to1_l1"]()):
        ctx = dgell.Context(desc)
        n = ctx.level_info()["n_dofs"]
        f = torch.ones(n, dtype=torch.float64, device="cuda")
        v = torch.empty_like(f)
        with pytest.raises(dgell.DgError) as ei:
            ctx.vcycle(f, v, coarse=0, smoother=2)
        assert ei.value.code == dgell.DG_ERR_UNSUPPORTED
        ctx.close()
