"""Shared helpers of the GPU parity tests (oracle side built from the same
seeded mesh descriptions)."""
import numpy as np

from oracle.blockmesh import BlockMesh
from oracle.mesh import Mesh
from paper_1907_01572_gb300 import inputs


def oracle_mesh(desc):
    if desc.get("blocks"):
        return BlockMesh(*inputs.oracle_block_mesh_args(desc))
    a, k = inputs.oracle_mesh_args(desc)
    return Mesh(*a, **k)


def oracle_level_mesh(ctx, desc, level):
    """Oracle mesh of a context level (leaves, degrees and blocks as the library built them)."""
    leaves, p, _ = ctx.level_leaves(level)
    if desc.get("blocks"):
        return BlockMesh(desc["blocks"], ctx.level_blocks(level), leaves, p)
    return Mesh(desc["lo"], desc["hi"], leaves, p, warp=desc["warp"])


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def single(p, level=0, warp=None, lo=(-1, -1, -1), hi=(1, 1, 1)):
    lv = inputs.uniform_leaves(level)
    return dict(lo=lo, hi=hi, leaves=np.array(lv, dtype=np.int32), p=np.full(len(lv), p, dtype=np.int32), warp=warp)


CASES = {
    "config1_affine_p3": lambda: inputs.config1_mesh(),
    "mixed_curved_2to1_l1": lambda: inputs.sweep_mesh(level=1, seed=0),
    "mixed_curved_2to1_l2": lambda: inputs.sweep_mesh(level=2, seed=4),
    "single_element_p1": lambda: single(1),
    "single_element_p8_curved": lambda: single(8, warp=(0.05, (1, 1, 1))),
    "uniform_p8_2x2x2": lambda: single(8, level=1),
    "affine_2to1_p2to8": lambda: inputs.sweep_mesh(level=1, seed=7, pmin=2, pmax=8, curved=False),
    "blocks_turned_fine_side": lambda: inputs.block_pair_mesh(rot=5, level=1, refine_block=0, seed=1),
    "blocks_turned_coarse_side": lambda: inputs.block_pair_mesh(rot=17, level=1, refine_block=1, seed=2,
                                                                 refine_count=2),
    "cubed_sphere_shell_2to1": lambda: inputs.cubed_sphere_mesh(level=1, a=1.0, r=3.0, r_out=30.0,
                                                               refine_wedge=(2, 3), pmin=2, pmax=4),
}
