"""Thin ctypes binding of the C ABI in include/dgell.h.

Argument marshalling only: every computation runs in libdgell.so's CUDA
kernels.  Device vectors are torch CUDA tensors (their data_ptr() is passed);
the context's stream is torch's current stream at creation unless one is
given.  Loading fails loudly when the library has not been built.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgell.so")

DG_OK, DG_ERR_INVALID, DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_UNSUPPORTED = range(7)
DG_FP64, DG_FP32, DG_BF16 = 0, 1, 2
DG_MAP_AFFINE, DG_MAP_SINE_WARP = 0, 1
DG_BLOCK_HEX8, DG_BLOCK_WEDGE, DG_BLOCK_SHELL = 0, 1, 2
DG_BC_DIRICHLET, DG_BC_NEUMANN, DG_BC_ROBIN = 0, 1, 2


class DgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dgell error %d: %s" % (code, msg))
        self.code = code


class dg_block(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("face", ctypes.c_int), ("corners", (ctypes.c_double * 3) * 8),
                ("a", ctypes.c_double), ("r", ctypes.c_double), ("r1", ctypes.c_double), ("r2", ctypes.c_double)]


class dg_mesh_desc(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("map_kind", ctypes.c_int),
                ("warp_amp", ctypes.c_double), ("warp_k", ctypes.c_int * 3), ("n_elems", ctypes.c_int),
                ("leaves", ctypes.POINTER(ctypes.c_int)), ("p", ctypes.POINTER(ctypes.c_int)),
                ("n_blocks", ctypes.c_int), ("blocks", ctypes.POINTER(dg_block)),
                ("elem_block", ctypes.POINTER(ctypes.c_int)), ("bc", ctypes.POINTER(ctypes.c_int))]


class dg_disc_opts(ctypes.Structure):
    _fields_ = [("penalty_c", ctypes.c_double), ("reserved", ctypes.c_int * 4)]


class dg_level_info(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("n_elems", ctypes.c_int), ("n_dofs", ctypes.c_int64),
                ("n_vol_qp", ctypes.c_int64), ("n_bnd_qp", ctypes.c_int64), ("n_mortars", ctypes.c_int),
                ("max_p", ctypes.c_int), ("device_bytes", ctypes.c_size_t), ("apply_flops", ctypes.c_double)]


class dg_cheb_opts(ctypes.Structure):
    _fields_ = [("n_eigs", ctypes.c_int), ("n_cheb", ctypes.c_int), ("Lambda", ctypes.c_double),
                ("lam_scale", ctypes.c_double), ("lam_fixed", ctypes.c_double)]


class dg_mg_opts(ctypes.Structure):
    _fields_ = [("cheb", dg_cheb_opts), ("coarse", ctypes.c_int), ("smoother", ctypes.c_int),
                ("n_schwarz", ctypes.c_int), ("local_iters", ctypes.c_int), ("local_tol", ctypes.c_double),
                ("schwarz_omega", ctypes.c_double)]


class dg_solver_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mg_prec", ctypes.c_int),
                ("use_mg", ctypes.c_int), ("mg", dg_mg_opts), ("graph_mode", ctypes.c_int)]


class dg_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_residual_rec", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int)]


class dg_puncture_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_double * 16), ("c", (ctypes.c_double * 3) * 16),
                ("P", (ctypes.c_double * 3) * 16), ("S", (ctypes.c_double * 3) * 16)]


class dg_amr_opts(ctypes.Structure):
    _fields_ = [("criterion", ctypes.c_int), ("theta", ctypes.c_double), ("gamma_h", ctypes.c_double),
                ("gamma_p", ctypes.c_double), ("p_max", ctypes.c_int), ("level_max", ctypes.c_int)]


DG_AMR_NONE, DG_AMR_P_REFINE, DG_AMR_H_REFINE = 0, 1, 2
DG_MARK_FRACTION, DG_MARK_MEAN = 0, 1

_P = ctypes.c_void_p
_SIGS = {
    "dg_version": ([], ctypes.c_int),
    "dg_last_error": ([], ctypes.c_char_p),
    "dg_mesh_create": ([ctypes.POINTER(dg_mesh_desc), ctypes.POINTER(_P)], ctypes.c_int),
    "dg_mesh_destroy": ([_P], None),
    "dg_ctx_create": ([_P, ctypes.POINTER(dg_disc_opts), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "dg_ctx_destroy": ([_P], None),
    "dg_ctx_footprint": ([_P, ctypes.POINTER(dg_disc_opts), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "dg_level_info_get": ([_P, ctypes.c_int, ctypes.POINTER(dg_level_info)], ctypes.c_int),
    "dg_level_leaves": ([_P, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "dg_level_blocks": ([_P, ctypes.c_int, _P], ctypes.c_int),
    "dg_quadrature_points": ([_P, ctypes.c_int, _P, _P], ctypes.c_int),
    "dg_apply": ([_P, ctypes.c_int, ctypes.c_int, _P, _P], ctypes.c_int),
    "dg_apply_host": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P], ctypes.c_int),
    "dg_rhs": ([_P, _P, _P, _P], ctypes.c_int),
    "dg_smooth": ([_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.POINTER(dg_cheb_opts), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "dg_vcycle": ([_P, ctypes.c_int, _P, _P, ctypes.POINTER(dg_mg_opts)], ctypes.c_int),
    "dg_solve": ([_P, _P, _P, ctypes.POINTER(dg_solver_opts), ctypes.POINTER(dg_solve_stats)], ctypes.c_int),
    "dg_set_zeroth_order": ([_P, _P], ctypes.c_int),
    "dg_puncture_setup": ([_P, ctypes.POINTER(dg_puncture_params)], ctypes.c_int),
    "dg_puncture_residual": ([_P, _P, _P], ctypes.c_int),
    "dg_power_source_setup": ([_P, _P, ctypes.c_int, _P], ctypes.c_int),
    "dg_nonlinear_residual": ([_P, _P, _P], ctypes.c_int),
    "dg_newton_step": ([_P, _P, ctypes.POINTER(dg_solver_opts), ctypes.POINTER(dg_solve_stats), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "dg_newton_solve": ([_P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(dg_solver_opts), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "dg_convert": ([_P, ctypes.c_int64, ctypes.c_int, _P, ctypes.c_int, _P], ctypes.c_int),
    "dg_launch_count": ([_P], ctypes.c_int64),
    "dg_transfer": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P], ctypes.c_int),
    "dg_smooth_static": ([_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.POINTER(dg_cheb_opts), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "dg_estimate": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "dg_estimate_fiducial": ([_P, _P, ctypes.c_int, _P, _P, _P, _P, _P], ctypes.c_int),
    "dg_hp_mark": ([ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(dg_amr_opts), _P, _P], ctypes.c_int),
    "dg_hp_refine": ([ctypes.c_int, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                      _P, _P, _P, _P], ctypes.c_int),
    "dg_hp_refine_mesh": ([ctypes.POINTER(dg_mesh_desc), _P, _P, ctypes.c_double, ctypes.c_int,
                           ctypes.POINTER(ctypes.c_int), _P, _P, _P, _P, _P], ctypes.c_int),
}

_lib = None


def lib():
    """The loaded libdgell.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdgell.so not built: run __graft_entry__.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != DG_OK:
        raise DgError(rc, lib().dg_last_error().decode())
    return rc


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _prec(t):
    import torch
    if t.dtype == torch.float64:
        return DG_FP64
    if t.dtype == torch.float32:
        return DG_FP32
    if t.dtype == torch.bfloat16:
        return DG_BF16
    raise ValueError("vectors must be float64, float32 or bfloat16")


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def block_array(blocks):
    """ctypes array of dg_block from inputs-style block dicts."""
    arr = (dg_block * len(blocks))()
    kinds = {"hex8": DG_BLOCK_HEX8, "wedge": DG_BLOCK_WEDGE, "shell": DG_BLOCK_SHELL}
    for i, b in enumerate(blocks):
        arr[i].kind = kinds[b["kind"]]
        if b["kind"] == "hex8":
            for c in range(8):
                for k in range(3):
                    arr[i].corners[c][k] = float(b["corners"][c][k])
        else:
            arr[i].face = int(b["face"])
        arr[i].a = float(b.get("a", 0.0))
        arr[i].r = float(b.get("r", 0.0))
        arr[i].r1 = float(b.get("r1", 0.0))
        arr[i].r2 = float(b.get("r2", 0.0))
    return arr


def make_mesh_desc(desc):
    """dg_mesh_desc from an inputs-style dict (keeps the arrays alive on the struct).
    An optional "bc" entry gives the dg_bc_kind of each block face (6 per block)."""
    leaves = np.ascontiguousarray(np.asarray(desc["leaves"], dtype=np.int32).reshape(-1, 4))
    p = np.ascontiguousarray(np.asarray(desc["p"], dtype=np.int32).ravel())
    d = dg_mesh_desc()
    if desc.get("blocks"):
        blocks = block_array(desc["blocks"])
        eb = np.ascontiguousarray(np.asarray(desc["elem_block"], dtype=np.int32).ravel())
        d.n_blocks = len(desc["blocks"])
        d.blocks = ctypes.cast(blocks, ctypes.POINTER(dg_block))
        d.elem_block = eb.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d.n_elems = len(p)
        d.leaves = leaves.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d.p = p.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d._keep = (leaves, p, blocks, eb)
    if desc.get("bc") is not None:
        bc = np.ascontiguousarray(np.asarray(desc["bc"], dtype=np.int32).ravel())
        d.bc = bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d._keep_bc = bc
    if desc.get("blocks"):
        return d
    for k in range(3):
        d.lo[k] = float(desc["lo"][k])
        d.hi[k] = float(desc["hi"][k])
    if desc.get("warp") is None:
        d.map_kind = DG_MAP_AFFINE
    else:
        d.map_kind = DG_MAP_SINE_WARP
        d.warp_amp = float(desc["warp"][0])
        for k in range(3):
            d.warp_k[k] = int(desc["warp"][1][k])
    d.n_elems = len(p)
    d.leaves = leaves.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.p = p.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d._keep = (leaves, p)
    return d


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def hp_mark(eta2, pred, p, level, criterion=DG_MARK_FRACTION, theta=0.1, gamma_h=0.25, gamma_p=0.1, p_max=8,
            level_max=15):
    """dg_hp_mark on host arrays: returns (action, pred_next) as numpy arrays."""
    n = len(eta2)
    e, ep = _host(eta2, np.float64)
    q, qp = _host(pred, np.float64)
    pp, ppp = _host(p, np.int32)
    lv, lvp = _host(level, np.int32)
    act = np.zeros(n, dtype=np.int32)
    nxt = np.zeros(n, dtype=np.float64)
    o = dg_amr_opts(criterion, theta, gamma_h, gamma_p, p_max, level_max)
    _check(lib().dg_hp_mark(n, ep, qp, ppp, lvp, ctypes.byref(o), act.ctypes.data_as(ctypes.c_void_p),
                            nxt.ctypes.data_as(ctypes.c_void_p)))
    return act, nxt


def hp_refine(leaves, p, action, pred_next, pred_init=float("inf")):
    """dg_hp_refine on host arrays: returns (leaves (n, 4), p, pred, parent)."""
    n = len(p)
    lv, lvp = _host(np.asarray(leaves).reshape(-1, 4), np.int32)
    pp, ppp = _host(p, np.int32)
    a, ap = _host(action, np.int32)
    q, qp = _host(pred_next, np.float64)
    cnt = ctypes.c_int(0)
    rc = lib().dg_hp_refine(n, lvp, ppp, ap, qp, pred_init, 0, ctypes.byref(cnt), None, None, None, None)
    if rc not in (DG_OK, DG_ERR_INVALID) or (rc == DG_ERR_INVALID and cnt.value == 0 and n > 0):
        _check(rc)
    m = cnt.value
    L = np.zeros((m, 4), dtype=np.int32)
    P = np.zeros(m, dtype=np.int32)
    Q = np.zeros(m, dtype=np.float64)
    R = np.zeros(m, dtype=np.int32)
    _check(lib().dg_hp_refine(n, lvp, ppp, ap, qp, pred_init, m, ctypes.byref(cnt),
                              L.ctypes.data_as(ctypes.c_void_p), P.ctypes.data_as(ctypes.c_void_p),
                              Q.ctypes.data_as(ctypes.c_void_p), R.ctypes.data_as(ctypes.c_void_p)))
    return L, P, Q, R


def hp_refine_mesh(desc, action, pred_next, pred_init=float("inf")):
    """dg_hp_refine_mesh on an inputs-style mesh dict: returns the refined
    mesh dict (same domain / blocks) and the arrays (pred, parent)."""
    d = make_mesh_desc(desc)
    a, ap = _host(action, np.int32)
    q, qp = _host(pred_next, np.float64)
    cnt = ctypes.c_int(0)
    rc = lib().dg_hp_refine_mesh(ctypes.byref(d), ap, qp, pred_init, 0, ctypes.byref(cnt), None, None, None, None, None)
    if rc not in (DG_OK, DG_ERR_INVALID) or (rc == DG_ERR_INVALID and cnt.value == 0 and len(a) > 0):
        _check(rc)
    m = cnt.value
    L = np.zeros((m, 4), dtype=np.int32)
    P = np.zeros(m, dtype=np.int32)
    B = np.zeros(m, dtype=np.int32)
    Q = np.zeros(m, dtype=np.float64)
    R = np.zeros(m, dtype=np.int32)
    vp = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    _check(lib().dg_hp_refine_mesh(ctypes.byref(d), ap, qp, pred_init, m, ctypes.byref(cnt), vp(L), vp(P), vp(B),
                                   vp(Q), vp(R)))
    out = dict(desc, leaves=L, p=P)
    if desc.get("blocks"):
        out["elem_block"] = B
    return out, Q, R


def dg_version():
    return lib().dg_version()


class Mesh:
    """Owns a dg_mesh (dg_mesh_create / dg_mesh_destroy) built from an
    inputs-style description dict."""

    def __init__(self, desc):
        d = make_mesh_desc(desc)
        h = ctypes.c_void_p()
        _check(lib().dg_mesh_create(ctypes.byref(d), ctypes.byref(h)))
        self.h = h

    def footprint(self, penalty_c=10.0):
        o = dg_disc_opts(penalty_c)
        b = ctypes.c_size_t(0)
        _check(lib().dg_ctx_footprint(self.h, ctypes.byref(o), ctypes.byref(b)))
        return b.value

    def close(self):
        if self.h:
            lib().dg_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dg_ctx_footprint(desc, penalty_c=10.0):
    m = Mesh(desc)
    try:
        return m.footprint(penalty_c)
    finally:
        m.close()


def cheb_opts(n_eigs=15, n_cheb=15, Lambda=20.0, lam_scale=1.0, lam_fixed=0.0):
    return dg_cheb_opts(n_eigs, n_cheb, Lambda, lam_scale, lam_fixed)


def mg_opts(n_eigs=15, n_cheb=15, Lambda=20.0, coarse=0, lam_scale=1.0, smoother=0, n_schwarz=3, local_iters=20,
            local_tol=1e-3, schwarz_omega=0.7, lam_fixed=0.0):
    return dg_mg_opts(cheb_opts(n_eigs, n_cheb, Lambda, lam_scale, lam_fixed), coarse, smoother, n_schwarz,
                      local_iters, local_tol, schwarz_omega)


def solver_opts(tol=1e-10, max_iter=100, mg_prec=DG_FP64, use_mg=1, graph_mode=0, **mg):
    return dg_solver_opts(tol, max_iter, mg_prec, use_mg, mg_opts(**mg), graph_mode)


class Context:
    """Owns a dg_ctx; methods are the C calls of the same name without 'dg_'."""

    def __init__(self, desc, penalty_c=10.0, stream=None):
        """desc: an inputs-style description dict or a Mesh."""
        m = desc if isinstance(desc, Mesh) else Mesh(desc)
        o = dg_disc_opts(penalty_c)
        h = ctypes.c_void_p()
        st = _stream() if stream is None else ctypes.c_void_p(stream)
        try:
            _check(lib().dg_ctx_create(m.h, ctypes.byref(o), st, ctypes.byref(h)))
        finally:
            if m is not desc:
                m.close()
        self.h = h

    def close(self):
        if self.h:
            lib().dg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_info(self, level=-1):
        i = dg_level_info()
        _check(lib().dg_level_info_get(self.h, level, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in dg_level_info._fields_}

    @property
    def n_levels(self):
        return self.level_info()["n_levels"]

    def level_leaves(self, level=-1):
        info = self.level_info(level)
        ne = info["n_elems"]
        leaves = np.zeros((ne, 4), dtype=np.int32)
        p = np.zeros(ne, dtype=np.int32)
        off = np.zeros(ne + 1, dtype=np.int64)
        _check(lib().dg_level_leaves(self.h, level, leaves.ctypes.data, p.ctypes.data, off.ctypes.data))
        return leaves, p, off

    def level_blocks(self, level=-1):
        eb = np.zeros(self.level_info(level)["n_elems"], dtype=np.int32)
        _check(lib().dg_level_blocks(self.h, level, eb.ctypes.data))
        return eb

    def quadrature_points(self, level=-1):
        import torch
        info = self.level_info(level)
        v = torch.empty(3 * info["n_vol_qp"], dtype=torch.float64, device="cuda")
        b = torch.empty(max(1, 3 * info["n_bnd_qp"]), dtype=torch.float64, device="cuda")
        _check(lib().dg_quadrature_points(self.h, level, _ptr(v), _ptr(b)))
        return v.view(3, -1), b[:3 * info["n_bnd_qp"]].view(3, -1)

    def apply(self, x, y, level=-1):
        _check(lib().dg_apply(self.h, level, _prec(x), _ptr(x), _ptr(y)))
        return y

    def apply_host(self, hx, hy, level=-1):
        """hy[r] = L hx[r] for host tensors hx, hy of shape (nvec, n_dofs), float32 or
        float64 (pinned for copy/apply overlap); complete once the context's stream
        is synchronised (dg_apply_host)."""
        if hx.device.type != "cpu" or hy.device.type != "cpu":
            raise ValueError("apply_host takes host tensors")
        if hx.dtype != hy.dtype or hx.shape != hy.shape or not (hx.is_contiguous() and hy.is_contiguous()):
            raise ValueError("hx and hy must be contiguous host tensors of the same dtype and shape")
        nvec = hx.shape[0] if hx.dim() == 2 else 1
        _check(lib().dg_apply_host(self.h, level, _prec(hx), nvec, _ptr(hx), _ptr(hy)))
        return hy

    def rhs(self, g_qp, gD_qp, F):
        _check(lib().dg_rhs(self.h, _ptr(g_qp), _ptr(gD_qp), _ptr(F)))
        return F

    def estimate(self, u, eta2, g_qp=None, f_qp=None, gD_qp=None, fiducial=None):
        """eta^2(e) of the finest level into eta2 (device double, n_elems);
        fiducial: block dicts of a fiducial grid (dg_estimate_fiducial) or None."""
        if fiducial is None:
            _check(lib().dg_estimate(self.h, _ptr(u), _ptr(g_qp), _ptr(f_qp), _ptr(gD_qp), _ptr(eta2)))
        else:
            arr = block_array(fiducial)
            _check(lib().dg_estimate_fiducial(self.h, ctypes.cast(arr, ctypes.c_void_p), len(fiducial), _ptr(u),
                                              _ptr(g_qp), _ptr(f_qp), _ptr(gD_qp), _ptr(eta2)))
        return eta2

    def smooth(self, b, x, level=-1, n_eigs=15, n_cheb=15, Lambda=20.0, want_lambda=True, lam_fixed=0.0):
        o = cheb_opts(n_eigs, n_cheb, Lambda, lam_fixed=lam_fixed)
        lam = ctypes.c_double(0.0)
        _check(lib().dg_smooth(self.h, level, _prec(b), _ptr(b), _ptr(x), ctypes.byref(o),
                               ctypes.byref(lam) if want_lambda else None))
        return lam.value

    def smooth_static(self, b, x, level=-1, n_eigs=15, n_cheb=15, Lambda=20.0, want_lambda=True, lam_fixed=0.0):
        """dg_smooth on the library's fixed scratch array (no device allocation)."""
        o = cheb_opts(n_eigs, n_cheb, Lambda, lam_fixed=lam_fixed)
        lam = ctypes.c_double(0.0)
        _check(lib().dg_smooth_static(self.h, level, _prec(b), _ptr(b), _ptr(x), ctypes.byref(o),
                                      ctypes.byref(lam) if want_lambda else None))
        return lam.value

    def vcycle(self, f, v, **mg):
        o = mg_opts(**mg)
        _check(lib().dg_vcycle(self.h, _prec(f), _ptr(f), _ptr(v), ctypes.byref(o)))
        return v

    def solve(self, b, x, check=True, **kw):
        o = solver_opts(**kw)
        s = dg_solve_stats()
        rc = lib().dg_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(s))
        if check:
            _check(rc)
        return {k: getattr(s, k) for k, _ in dg_solve_stats._fields_}

    def set_zeroth_order(self, coef_qp):
        _check(lib().dg_set_zeroth_order(self.h, _ptr(coef_qp)))

    def puncture_setup(self, punctures):
        prm = dg_puncture_params()
        prm.n = len(punctures)
        for i, pu in enumerate(punctures):
            m, c, P = pu[0], pu[1], pu[2]
            S = pu[3] if len(pu) > 3 else (0.0, 0.0, 0.0)
            prm.m[i] = m
            for k in range(3):
                prm.c[i][k] = c[k]
                prm.P[i][k] = P[k]
                prm.S[i][k] = S[k]
        _check(lib().dg_puncture_setup(self.h, ctypes.byref(prm)))

    def puncture_residual(self, u, R):
        _check(lib().dg_puncture_residual(self.h, _ptr(u), _ptr(R)))
        return R

    def newton_step(self, u, **kw):
        o = solver_opts(**kw)
        s = dg_solve_stats()
        rn = ctypes.c_double(0.0)
        _check(lib().dg_newton_step(self.h, _ptr(u), ctypes.byref(o), ctypes.byref(s), ctypes.byref(rn)))
        return rn.value, {k: getattr(s, k) for k, _ in dg_solve_stats._fields_}

    def power_source_setup(self, coef_qp, power, F=None):
        _check(lib().dg_power_source_setup(self.h, _ptr(coef_qp), int(power), _ptr(F)))

    def nonlinear_residual(self, u, R):
        _check(lib().dg_nonlinear_residual(self.h, _ptr(u), _ptr(R)))
        return R

    def newton_solve(self, u, tol_newton=1e-10, max_newton=20, **kw):
        """Alg. 1; kw are the linear solver's options (tol, max_iter, mg_prec, ...)."""
        o = solver_opts(**kw)
        steps = ctypes.c_int(0)
        rn = ctypes.c_double(0.0)
        _check(lib().dg_newton_solve(self.h, _ptr(u), tol_newton, max_newton, ctypes.byref(o), ctypes.byref(steps),
                                     ctypes.byref(rn)))
        return steps.value, rn.value

    def convert(self, src, dst):
        _check(lib().dg_convert(self.h, src.numel(), _prec(src), _ptr(src), _prec(dst), _ptr(dst)))
        return dst

    def transfer(self, coarse_level, direction, x, out):
        _check(lib().dg_transfer(self.h, coarse_level, _prec(x), direction, _ptr(x), _ptr(out)))
        return out

    def launch_count(self):
        return lib().dg_launch_count(self.h)
