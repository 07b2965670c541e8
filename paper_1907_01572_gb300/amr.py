"""hp-adaptive solve loop (Sec. II.D): solve, estimate, mark, refine.

Each step builds a context on the current mesh (a single box or a
multi-block mesh), solves -Lap u + f u = g (u = g_D on the boundary) with
dg_solve, computes eta^2(e) with dg_estimate (or dg_estimate_fiducial),
applies Algorithm 4 with dg_hp_mark and refines the leaf set with
dg_hp_refine or dg_hp_refine_mesh (2:1 balanced, across block interfaces
too).  The compute is entirely in libdgell
(CUDA kernels for the solve and the estimator, host C++ for marking and
refinement); this module sequences the calls and evaluates the caller's
problem functions at the quadrature points the library reports.

Problem functions take a (3, P) torch tensor of physical points on the
device and return P values (torch), so they run where the points are.
"""
import math

import numpy as np

from . import dgell


def _values(fn, pts):
    import torch
    if fn is None:
        return None
    v = fn(pts)
    return torch.as_tensor(v, dtype=torch.float64, device=pts.device).contiguous()


def adapt(desc, g_fn, gD_fn=None, f_fn=None, steps=3, theta=0.2, criterion=dgell.DG_MARK_FRACTION,
          gamma_h=0.25, gamma_p=0.1, p_max=8, pred_init=math.inf, tol=1e-10, max_iter=200, mg_prec=dgell.DG_FP64,
          penalty_c=10.0, keep_solution=False, fiducial=None):
    """Runs `steps` solve-estimate-refine cycles (plus the final solve and
    estimate) from the mesh description `desc` (inputs-style dict: a single
    box, refined with dg_hp_refine, or a multi-block mesh, refined with
    dg_hp_refine_mesh; fiducial: the blocks of a fiducial grid for the
    estimator, multi-block meshes only).  Returns one record per mesh:
    n_elems, n_dofs, iterations, rel_residual, eta2 (host array), action
    (host array, None on the last mesh) and desc; with keep_solution=True
    also u (host array)."""
    import torch
    desc = dict(desc)
    leaves = np.asarray(desc["leaves"], dtype=np.int32).reshape(-1, 4)
    p = np.asarray(desc["p"], dtype=np.int32).ravel()
    pred = np.full(len(p), pred_init, dtype=np.float64)
    history = []
    for step in range(steps + 1):
        desc["leaves"], desc["p"] = leaves, p
        ctx = dgell.Context(desc, penalty_c=penalty_c)
        try:
            info = ctx.level_info()
            vxyz, bxyz = ctx.quadrature_points()
            g = _values(g_fn, vxyz)
            gD = _values(gD_fn, bxyz) if info["n_bnd_qp"] > 0 else None
            f = _values(f_fn, vxyz)
            if f is not None:
                ctx.set_zeroth_order(f)
            F = torch.empty(info["n_dofs"], dtype=torch.float64, device="cuda")
            ctx.rhs(g, gD, F)
            u = torch.zeros_like(F)
            st = ctx.solve(F, u, tol=tol, max_iter=max_iter, mg_prec=mg_prec)
            eta = torch.empty(info["n_elems"], dtype=torch.float64, device="cuda")
            ctx.estimate(u, eta, g_qp=g, f_qp=f, gD_qp=gD, fiducial=fiducial)
            eta2 = eta.cpu().numpy()
            rec = dict(n_elems=info["n_elems"], n_dofs=info["n_dofs"], iterations=st["iterations"],
                       rel_residual=st["rel_residual"], eta2=eta2, action=None,
                       desc=dict(desc, leaves=leaves.copy(), p=p.copy()))
            if keep_solution:
                rec["u"] = u.cpu().numpy()
        finally:
            ctx.close()
        history.append(rec)
        if step == steps:
            break
        act, nxt = dgell.hp_mark(eta2, pred, p, leaves[:, 0], criterion, theta, gamma_h, gamma_p, p_max)
        rec["action"] = act
        if desc.get("blocks"):
            desc, pred, _ = dgell.hp_refine_mesh(desc, act, nxt, pred_init=pred_init)
            leaves = np.asarray(desc["leaves"], dtype=np.int32).reshape(-1, 4)
            p = np.asarray(desc["p"], dtype=np.int32).ravel()
        else:
            leaves, p, pred, _ = dgell.hp_refine(leaves, p, act, nxt, pred_init=pred_init)
    return history
