"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/dgell.h (no device calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dgell.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_01572_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1907_01572_gb300 import dgell
    assert set(declared_functions()) <= set(dgell._SIGS)


def test_version_and_error_text(lib):
    from paper_1907_01572_gb300 import dgell
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dgell.h")).read()
    assert dgell.lib().dg_version() == int(re.search(r"#define DGELL_VERSION (\d+)", hdr).group(1))
    assert isinstance(dgell.lib().dg_last_error(), bytes)


def test_footprint_host_only_and_invalid_meshes(lib):
    """Host-side validation (no GPU): footprint of a valid mesh, DG_ERR_INVALID
    for a 4:1 face, a hole, a bad degree and an empty mesh."""
    import numpy as np
    from paper_1907_01572_gb300 import dgell, inputs
    ok = inputs.config1_mesh()
    assert dgell.dg_ctx_footprint(ok) > 4096 * 8
    sw = inputs.sweep_mesh(level=2, seed=0)
    assert dgell.dg_ctx_footprint(sw) > 0
    # 4:1: refine one level-1 cell twice next to an unrefined level-1 cell
    lv = inputs.refine(inputs.uniform_leaves(1), lambda lf: lf == (1, 0, 0, 0))
    lv = inputs.refine(lv, lambda lf: lf == (2, 1, 1, 1))
    bad = dict(lo=(0, 0, 0), hi=(1, 1, 1), leaves=np.array(lv), p=np.full(len(lv), 2), warp=None)
    with pytest.raises(dgell.DgError) as e:
        dgell.dg_ctx_footprint(bad)
    assert e.value.code == dgell.DG_ERR_INVALID
    hole = dict(ok)
    hole["leaves"] = ok["leaves"][1:]
    hole["p"] = ok["p"][1:]
    with pytest.raises(dgell.DgError):
        dgell.dg_ctx_footprint(hole)
    badp = dict(ok)
    badp["p"] = np.full(64, 9)
    with pytest.raises(dgell.DgError):
        dgell.dg_ctx_footprint(badp)
    empty = dict(ok)
    empty["leaves"] = np.zeros((0, 4), dtype=np.int32)
    empty["p"] = np.zeros(0, dtype=np.int32)
    with pytest.raises(dgell.DgError):
        dgell.dg_ctx_footprint(empty)


def test_block_meshes_host_validation(lib):
    """Multi-block meshes (no GPU): every relative orientation of two glued
    boxes and the 13-block cubed sphere are accepted; a 4:1 face across a
    block interface, a bad block index and an unknown block kind are not."""
    import numpy as np
    from paper_1907_01572_gb300 import dgell, inputs
    for rot in range(24):
        for side in (0, 1):
            d = inputs.block_pair_mesh(rot=rot, level=1, refine_block=side, seed=rot)
            assert dgell.dg_ctx_footprint(d) > 0
    assert dgell.dg_ctx_footprint(inputs.cubed_sphere_mesh(level=1, r_out=1e3, refine_wedge=(3, 2))) > 0
    assert dgell.dg_ctx_footprint(inputs.star_sphere_mesh(level=2, refine=1)) > 0
    # refine the interface element of block 0 twice: its grandchildren face a level-1 cell of block 1
    d = inputs.block_pair_mesh(rot=7, level=1, refine_block=0)
    lv = [tuple(x) for x in d["leaves"]]
    eb = list(d["elem_block"])
    tgt = [i for i, (b, lf) in enumerate(zip(eb, lv)) if b == 0 and lf[0] == 2 and lf[1] == 3][0]
    L, i, j, k = lv[tgt]
    kids = [(L + 1, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1)) for c in range(8)]
    bad = dict(blocks=d["blocks"], leaves=np.array(lv[:tgt] + kids + lv[tgt + 1:], dtype=np.int32),
               elem_block=np.array(eb[:tgt] + [0] * 8 + eb[tgt + 1:], dtype=np.int32),
               p=np.full(len(lv) + 7, 2, dtype=np.int32))
    with pytest.raises(dgell.DgError) as e:
        dgell.dg_ctx_footprint(bad)
    assert e.value.code == dgell.DG_ERR_INVALID
    wrong = dict(d)
    wrong["elem_block"] = np.full(len(d["p"]), 2, dtype=np.int32)
    with pytest.raises(dgell.DgError):
        dgell.dg_ctx_footprint(wrong)
    kind = dict(d)
    kind["blocks"] = [dict(b) for b in d["blocks"]]
    kind["blocks"][1]["kind"] = "shell"
    kind["blocks"][1]["face"] = 0
    kind["blocks"][1]["r1"], kind["blocks"][1]["r2"] = 2.0, 1.0
    with pytest.raises(dgell.DgError):
        dgell.dg_ctx_footprint(kind)


def test_mesh_object_and_boundary_tags(lib):
    """dg_mesh_create / dg_mesh_destroy (no GPU): a mesh object gives the same
    footprint as the description it was built from; boundary tags are checked
    -- all Dirichlet accepted, a Neumann or Robin tag on a boundary face
    rejected as unsupported (this version implements Dirichlet data only), a
    non-Dirichlet tag on a face glued to another block ignored, a tag out of
    range rejected as invalid."""
    import ctypes
    import numpy as np
    from paper_1907_01572_gb300 import dgell, inputs
    d = inputs.config1_mesh()
    m = dgell.Mesh(d)
    assert m.footprint() == dgell.dg_ctx_footprint(d)
    m.close()
    m.close()    # idempotent on the Python side; dg_mesh_destroy(NULL) is a no-op
    dgell.lib().dg_mesh_destroy(None)
    ok = dict(d, bc=np.zeros(6, dtype=np.int32))
    assert dgell.Mesh(ok).footprint() > 0
    for kind in (dgell.DG_BC_NEUMANN, dgell.DG_BC_ROBIN):
        bc = np.zeros(6, dtype=np.int32)
        bc[3] = kind
        with pytest.raises(dgell.DgError) as e:
            dgell.Mesh(dict(d, bc=bc))
        assert e.value.code == dgell.DG_ERR_UNSUPPORTED
    with pytest.raises(dgell.DgError) as e:
        dgell.Mesh(dict(d, bc=np.full(6, 7, dtype=np.int32)))
    assert e.value.code == dgell.DG_ERR_INVALID
    # two glued boxes: block 0's face towards block 1 may carry any tag
    pair = inputs.block_pair_mesh(rot=0, level=1, refine_block=0)
    probe = dgell.Mesh(pair)
    probe.close()
    glued = None
    for f in range(6):
        bc = np.zeros(12, dtype=np.int32)
        bc[f] = dgell.DG_BC_NEUMANN
        try:
            dgell.Mesh(dict(pair, bc=bc)).close()
            glued = f
        except dgell.DgError as e:
            assert e.code == dgell.DG_ERR_UNSUPPORTED
    assert glued is not None
    # a NULL out pointer and a NULL mesh are invalid arguments
    desc = dgell.make_mesh_desc(d)
    assert dgell.lib().dg_mesh_create(ctypes.byref(desc), None) == dgell.DG_ERR_INVALID
    sz = ctypes.c_size_t(0)
    assert dgell.lib().dg_ctx_footprint(None, None, ctypes.byref(sz)) == dgell.DG_ERR_INVALID
