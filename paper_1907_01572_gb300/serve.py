"""Serving loop: elliptic solves of different meshes, degrees and sources that
arrive over time, continuously admitted while others run on the GPU.

* Each admitted request runs on a worker with its own CUDA stream, so the work
  of concurrent solves overlaps on the device; the V-cycle of each solve is
  replayed as a CUDA graph (dg_solve, graph_mode 0).
* Admission is by device footprint (dg_ctx_footprint) against an HBM budget
  and by the number of worker slots; a request waits until both free up.
* Mesh, geometry and multigrid hierarchy stay resident: every worker keeps a
  context per mesh it has served and reuses it for later requests on that mesh.
* All kernels and reductions are deterministic, so a request's result does not
  depend on what else runs at the same time (checked by the tests).

The compute is entirely in libdgell; this module only schedules host threads,
streams and device buffers.
"""
import threading
import time

import numpy as np

from . import dgell, inputs


# (octree level, degree) of the served Poisson boxes: every uniform box with
# 1e4 to 5e6 DOFs (13,824 at level 2, p = 5 up to 4,194,304 at level 5, p = 4)
SERVED_POISSON = [(L, p) for L in range(2, 6) for p in range(3, 9) if 1e4 <= 8 ** L * (p + 1) ** 3 <= 5e6]


def make_requests(n=32, rate_hz=20.0, seed=2, full=False, served=False):
    """Seeded mix of Poisson (manufactured sine), star and puncture requests
    with Poisson-process arrival times.  full=False: small meshes (Poisson
    4^3-8^3 elements, p 3..5; star and punctures on box meshes).  full=True:
    Poisson 4^3-16^3 elements with p 3..8 (4e3 to 3e6 DOFs), the density-jump
    star and the two punctures on the 13-block cubed sphere (shell to r = 20;
    1.5e5 to 4.4e5 DOFs).  served=True: the served workload -- Poisson boxes
    drawn uniformly from SERVED_POISSON (1.4e4 to 4.2e6 DOFs), the star and the
    two punctures on cubed spheres with every block at level 1 or 2 (shell to
    r = 20; 1.6e4 to 4.4e5 DOFs)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    meshes = {}   # one description per mesh key, shared by the requests on that mesh
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        kind = rng.choice(["poisson", "star", "puncture"], p=[0.5, 0.3, 0.2])
        if kind == "poisson" and served:
            level, p = SERVED_POISSON[int(rng.integers(len(SERVED_POISSON)))]
            lv = inputs.uniform_leaves(level)
            desc = dict(lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), leaves=np.array(lv, dtype=np.int32),
                        p=np.full(len(lv), p, dtype=np.int32), warp=None)
            key = ("poisson", level, p)
            params = dict(amp=float(rng.uniform(0.5, 2.0)))
        elif kind == "star" and served:
            level = int(rng.integers(1, 3))
            refine = int(rng.integers(0, 2))
            key = ("star_sphere", level, refine)
            if key not in meshes:
                meshes[key] = inputs.star_sphere_mesh(level=level, refine=refine, r_out=20.0)
            desc = meshes[key]
            params = dict(amp=float(rng.uniform(0.5, 2.0)))
        elif kind == "puncture" and served:
            punc = inputs.two_punctures()
            level = int(rng.integers(1, 3))
            key = ("puncture_sphere", level)
            if key not in meshes:
                meshes[key] = inputs.puncture_sphere_mesh(punc, level=level)
            desc = meshes[key]
            s = float(rng.uniform(0.5, 1.5))
            params = dict(punctures=[(m, c, tuple(s * np.asarray(P))) for (m, c, P) in punc])
        elif kind == "poisson":
            level = int(rng.integers(2, 5 if full else 4))
            p = int(rng.integers(3, 9 if full else 6))
            lv = inputs.uniform_leaves(level)
            desc = dict(lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), leaves=np.array(lv, dtype=np.int32),
                        p=np.full(len(lv), p, dtype=np.int32), warp=None)
            key = ("poisson", level, p)
            params = dict(amp=float(rng.uniform(0.5, 2.0)))
        elif kind == "star":
            if full:
                refine = int(rng.integers(0, 2))
                desc = inputs.star_sphere_mesh(level=2, refine=refine, r_out=20.0)
                key = ("star_sphere", 2, refine)
            else:
                desc = inputs.star_mesh(level=3, refine=1, seed=3, p_lo=4, p_hi=6)
                key = ("star", 3, 1)
            params = dict(amp=float(rng.uniform(0.5, 2.0)))
        else:
            punc = inputs.two_punctures()
            if full:
                desc = inputs.puncture_sphere_mesh(punc, level=2)
                key = ("puncture_sphere", 2)
            else:
                desc = inputs.puncture_mesh(punc, refine=1, p_fine=5)
                key = ("puncture", 1)
            s = float(rng.uniform(0.5, 1.5))
            params = dict(punctures=[(m, c, tuple(s * np.asarray(P))) for (m, c, P) in punc])
        reqs.append(dict(id=i, kind=str(kind), key=key, desc=desc, params=params, arrival=t))
    return reqs


class Server:
    """Continuous admission of solve requests onto worker streams."""

    def __init__(self, hbm_budget_bytes=64 << 30, slots=4, mg_prec=dgell.DG_FP32, tol=1e-10, mg=None):
        """mg: V-cycle options (dgell.mg_opts keywords) of the solves whose request
        carries none of its own (req["mg"]); default the paper's."""
        import torch
        self.torch = torch
        self.mg = dict(mg or {})
        self.budget = hbm_budget_bytes
        self.slots = slots
        self.mg_prec = mg_prec
        self.tol = tol
        self.lock = threading.Condition()
        self.in_use = 0
        self.busy = 0
        self.results = {}
        self.footprints = {}

    def _footprint(self, req):
        if req["key"] not in self.footprints:
            self.footprints[req["key"]] = dgell.dg_ctx_footprint(req["desc"])
        return self.footprints[req["key"]]

    def _solve(self, ctx, req, stream):
        torch = self.torch
        info = ctx.level_info()
        n = info["n_dofs"]
        if req["kind"] == "puncture":
            ctx.puncture_setup(req["params"]["punctures"])
            u = torch.zeros(n, dtype=torch.float64, device="cuda")
            steps, rn = ctx.newton_solve(u, tol_newton=1e-9, max_newton=12, mg_prec=self.mg_prec, tol=self.tol,
                                         max_iter=300, **req.get("mg", self.mg))
            stream.synchronize()
            return u, {"newton_steps": steps, "residual_norm": rn}
        if not hasattr(ctx, "_qp_host"):   # the mesh's quadrature points, fetched once per context
            xyz, bxyz = ctx.quadrature_points()
            ctx._qp_host = (xyz.T.cpu().numpy(), bxyz.T.cpu().numpy())
        X, XB = ctx._qp_host
        amp = req["params"]["amp"]
        if req["kind"] == "poisson":
            g = amp * 3 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
            gd = None
        else:
            g = amp * inputs.star_source(X)
            gd = torch.tensor(amp * inputs.star_solution(XB), device="cuda")
        F = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.rhs(torch.tensor(g, device="cuda"), gd, F)
        x = torch.zeros_like(F)
        st = ctx.solve(F, x, tol=self.tol, max_iter=300, mg_prec=self.mg_prec, **req.get("mg", self.mg))
        stream.synchronize()
        return x, st

    def _worker(self, wid, queue, t0):
        torch = self.torch
        stream = torch.cuda.Stream()
        contexts = {}
        while True:
            with self.lock:
                while True:
                    if not queue:
                        for c in contexts.values():
                            c.close()
                        return
                    req = queue[0]
                    fp = self._footprint(req)
                    now = time.perf_counter() - t0
                    if req["arrival"] > now:
                        self.lock.wait(timeout=req["arrival"] - now)
                        continue
                    extra = 0 if req["key"] in contexts else fp
                    if self.busy < self.slots and self.in_use + extra > self.budget:
                        # evict this worker's other resident contexts to make room
                        for k in [k for k in contexts if k != req["key"]]:
                            contexts.pop(k).close()
                            self.in_use -= self.footprints[k]
                    if self.busy < self.slots and (self.in_use + extra <= self.budget or self.busy == 0):
                        queue.pop(0)
                        self.busy += 1
                        self.in_use += extra
                        break
                    self.lock.wait(timeout=0.01)
            with torch.cuda.stream(stream):
                if req["key"] not in contexts:
                    contexts[req["key"]] = dgell.Context(req["desc"])
                start = time.perf_counter() - t0
                x, st = self._solve(contexts[req["key"]], req, stream)
                done = time.perf_counter() - t0
            with self.lock:
                self.busy -= 1
                self.results[req["id"]] = dict(x=x.cpu().numpy(), stats=st, arrival=req["arrival"], start=start,
                                               done=done, latency=done - req["arrival"], kind=req["kind"])
                self.lock.notify_all()

    def run(self, requests, workers=None):
        """Serves the requests (arrival times in seconds from now); returns
        {id: result} and the summary (solves/s, p50/p99 latency)."""
        queue = sorted(requests, key=lambda r: r["arrival"])
        for r in queue:
            self._footprint(r)
        t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(w, queue, t0), daemon=True)
                   for w in range(workers or self.slots)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        lat = sorted(r["latency"] for r in self.results.values())
        summary = {"requests": len(lat), "wall_s": wall, "solves_per_s": len(lat) / wall,
                   "p50_ms": 1e3 * lat[len(lat) // 2], "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                   "slots": self.slots, "hbm_budget_gb": self.budget / 2 ** 30}
        return self.results, summary


def solve_alone(req, mg_prec=dgell.DG_FP32, tol=1e-10):
    """The same request on an otherwise idle device (fresh context and stream)."""
    srv = Server(slots=1, mg_prec=mg_prec, tol=tol)
    r = dict(req)
    r["arrival"] = 0.0
    res, _ = srv.run([r])
    return res[req["id"]]
