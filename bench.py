"""Benchmark: matrix-free SIPG operator apply on the curved, 2:1 h-refined,
mixed-degree 32^3 sweep mesh (61,440 elements, p drawn from {2..7}, ~1.32e7
DOFs), plus the Poisson solve of the 4x4x4, p = 3 problem at 1e-10 relative
residual (solves/s, p50/p99).

One step = one operator apply y = L x over the whole mesh (all degree
buckets) in FP32; the FP64 apply and the solve are reported beside it.
Prints ONE JSON line.  Multi-GPU: independent replicas (no collective on the
data path), value = DOFs applied by all ranks / max time.

--impl reference times the oracle (plain FP64 numpy, dense per-element
blocks) on the host cores on a bounded element sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK = 6800.0
# ncu DRAM bytes (read + write) of one FP32 apply of the sweep mesh, measured for the
# kernels of that library version (profiles/apply_sweep32_traffic_v4.md,
# profiles/apply_sweep32_traffic_v105.md, _v106.md, _v108.md, _v110.md, _v112.md); null for other
# versions.  Version 109 changed only the nonlinear-source kernels; its apply kernels are those of 108.
# Versions 113 (estimator, hp-AMR calls), 114 (puncture spins) and 115 (block-mesh refinement, host
# code) keep the apply kernels of 112.
TRAFFIC_BYTES_PER_APPLY = {104: 1.3634e9, 105: 1.3709e9, 106: 1.3770e9, 108: 1.3775e9, 109: 1.3775e9,
                           110: 1.3774e9, 112: 1.3770e9, 113: 1.3770e9, 114: 1.3770e9, 115: 1.3770e9}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling (every 50 ms) of SM clocks and throttle reasons; summary() keeps the
    samples taken between mark(True) and mark(False), i.e. during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.samples = []        # (host time, line)
        self.window = [None, None]

    def _reader(self):
        for line in self.proc.stdout:
            if line.strip():
                self.samples.append((time.perf_counter(), line))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._reader, daemon=True).start()
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 10:   # sampler running before timing
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def mark(self, start):
        self.window[0 if start else 1] = time.perf_counter()

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.06)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        t0, t1 = self.window
        inside = [l for t, l in self.samples if t0 is not None and t1 is not None and t0 <= t <= t1 + 0.05]
        self.lines = inside or [l for t, l in self.samples][-1:]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_sample(n_elems_sample, seed=0):
    """Times the oracle's dense-local apply on a sample of the sweep mesh's
    elements in a single-threaded subprocess; returns (GDOF/s, dofs, seconds)."""
    code = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
from paper_1907_01572_gb300 import inputs
from oracle.mesh import Mesh
from oracle import sipg
desc = inputs.sweep_mesh(level=5, seed=0)
a, k = inputs.oracle_mesh_args(desc)
m = Mesh(*a, **k)
rng = np.random.default_rng(%d)
els = rng.choice(m.n_elems, size=%d, replace=False)
x = inputs.random_vector(m.n_dofs, seed=1)
t = time.perf_counter()
out = sipg.apply_local(m, x, 10.0, elems=[int(e) for e in els])
dt = time.perf_counter() - t
dofs = int(sum((m.p[e] + 1) ** 3 for e in els))
print(json.dumps({"dofs": dofs, "seconds": dt}))
""" % (ROOT, seed, n_elems_sample)
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["dofs"] / d["seconds"] / 1e9, d["dofs"], d["seconds"]


def max_over_ranks(values, dist, device):
    """Per-step times reduced with MAX over the ranks of the replica job (no
    data-path collective: each rank applies its own copy of the operator)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_throughput(dofs_per_rank, world, ms_max):
    """Whole-job GDOF/s: DOFs applied by all ranks / the slowest rank's time."""
    return dofs_per_rank * world / (ms_max * 1e-3) / 1e9


WORKLOAD = "operator-apply sweep: 32^3 hex on [-1,1]^3, octant x,y,z<0 h-refined 2:1 (61440 elems), " \
           "p~U{2..7} seed 0, sine-warped isoparametric geometry, x~N(0,1) seed 1"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals, secs = [], []
    for s in range(args.warmup + args.steps):
        g, dofs, dt = cpu_baseline_sample(16, seed=100 + s)
        if s >= args.warmup:
            vals.append(g)
            secs.append(dt)
    v = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": "DG apply GDOF/s", "value": v, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
                             "sample": "16 random elements per step, dense-local FP64 apply incl. their mortars"},
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--level", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # CPU baseline first (own process, before any heavy GPU work)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        g, dofs, dt = cpu_baseline_sample(48, seed=0)
        cpu = {"value": g, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
               "sample": "48 random elements (%d DOFs, %.1f s) of the same mesh, dense-local FP64 apply "
                         "incl. their mortars, single thread" % (dofs, dt)}

    import __graft_entry__
    __graft_entry__.build()
    from paper_1907_01572_gb300 import dgell, inputs

    stream = torch.cuda.current_stream()
    desc = inputs.sweep_mesh(level=args.level, seed=0)
    ctx = dgell.Context(desc)
    info = ctx.level_info()
    N = info["n_dofs"]
    x64 = torch.tensor(inputs.random_vector(N, seed=1), device="cuda")
    x32 = x64.float()
    y32 = torch.empty_like(x32)
    y64 = torch.empty_like(x64)

    def timed(fn, steps, warmup, clk=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if clk:
            clk.mark(True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.mark(False)
        if dist:
            dist.barrier()
        return e0.elapsed_time(e1) / steps  # ms per step

    hbm, peak_kind = peaks()
    launches0 = ctx.launch_count()
    with Clocks(local) as clk:
        ms32 = timed(lambda: ctx.apply(x32, y32), args.steps, args.warmup, clk)
    launches = (ctx.launch_count() - launches0) * args.steps // (args.steps + args.warmup)
    ms64 = timed(lambda: ctx.apply(x64, y64), max(3, args.steps // 4), args.warmup)
    x16 = x64.bfloat16()
    ms16 = timed(lambda: ctx.apply(x16, y32), args.steps, args.warmup)

    # end to end through the C ABI with host buffers (pinned), copies inside the region
    hx = x32.cpu().pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    dx = torch.empty_like(x32)
    dy = torch.empty_like(x32)

    def e2e_step():
        dx.copy_(hx, non_blocking=True)
        ctx.apply(dx, dy)
        hy.copy_(dy, non_blocking=True)

    ms_e2e = timed(e2e_step, max(3, args.steps // 2), 2)

    ms32, ms64, ms_e2e, ms16 = max_over_ranks([ms32, ms64, ms_e2e, ms16], dist, "cuda")
    total_dofs = N * world
    g32 = job_throughput(N, world, ms32)
    g64 = job_throughput(N, world, ms64)
    ge2e = job_throughput(N, world, ms_e2e)

    # algorithmic bytes per DOF: x + y + 3 coordinates per LGL node (curved isoparametric geometry)
    b32 = 4 + 4 + 12
    b64 = 8 + 8 + 24
    ach32 = N * b32 / (ms32 * 1e-3) / 1e9
    ach64 = N * b64 / (ms64 * 1e-3) / 1e9

    solve = None
    peaks_alu = alu_peaks(torch) if rank == 0 else {}
    if not args.no_solve and rank == 0:
        solve = solve_bench(dgell, inputs, torch)
    flops = info["apply_flops"]

    if rank == 0:
        line = {
            "metric": "DG apply GDOF/s", "value": g32, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_dofs": N, "n_elems": info["n_elems"], "levels": info["n_levels"],
                       "l2": "inputs larger than L2 (x, y, metric terms ~0.6 GB)", "parallelism": "replicas"},
            "roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm, "unit": "GB/s", "frac": ach32 / hbm,
                         "traffic": TRAFFIC_BYTES_PER_APPLY.get(dgell.dg_version()) if args.level == 5 else None,
                         "peak_kind": peak_kind, "bytes_per_dof": b32,
                         "kernel": "dg_apply FP32: trace + element kernels of all degree buckets (one apply)"},
            "cpu_baseline": cpu,
            "e2e": {"value": ge2e, "unit": "GDOF/s", "h2d_bytes_per_step": N * 4, "d2h_bytes_per_step": N * 4},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "fp64": {"value": g64, "unit": "GDOF/s", "ms_per_step": ms64, "achieved_gbs": ach64,
                     "bytes_per_dof": b64,
                     "roofline": {"bound": "alu", "achieved": flops / (ms64 * 1e-3) / 1e12,
                                  "peak": peaks_alu.get("fp64"), "unit": "TFLOP/s",
                                  "frac": (flops / (ms64 * 1e-3) / 1e12) / peaks_alu["fp64"] if peaks_alu else None,
                                  "peak_kind": "measured this run: cuBLAS DGEMM 4096^3"}},
            "bf16_operands": {"value": total_dofs / (ms16 * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": ms16,
                              "bytes_per_dof": 18, "achieved_gbs": N * 18 / (ms16 * 1e-3) / 1e9,
                              "frac_hbm": N * 18 / (ms16 * 1e-3) / 1e9 / hbm,
                              "note": "x bf16, FP32 arithmetic, y fp32"},
            "fp32_alu": {"achieved": flops / (ms32 * 1e-3) / 1e12, "peak": peaks_alu.get("fp32"), "unit": "TFLOP/s",
                         "frac": (flops / (ms32 * 1e-3) / 1e12) / peaks_alu["fp32"] if peaks_alu else None,
                         "peak_kind": "measured this run: cuBLAS SGEMM 8192^3, TF32 off",
                         "flops_per_apply": flops},
            "solve": solve,
        }
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _latency(lat):
    lat = sorted(lat)
    return {"solves_per_s": len(lat) / sum(lat), "p50_ms": 1e3 * lat[len(lat) // 2],
            "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]}


def solve_bench(dgell, inputs, torch, n_solves=8):
    """Linear solves to 1e-10 relative residual (FP64 outer FCG) with the plain
    FP64 V-cycle and with the FP32 V-cycle, each V-cycle replayed as a CUDA graph
    on a dedicated stream: the 4^3 p=3 Poisson problem and the star with a
    density jump on the 13-block cubed sphere (centre cube a = 2, wedges to
    r = 10, inverse-radius shell to r = 20, closed-form Dirichlet data); then
    the two-puncture Newton solve on the same kind of cubed sphere."""
    import numpy as np
    out = {}
    stream = torch.cuda.Stream()
    cases = [
        ("poisson_4x4x4_p3", inputs.config1_mesh(),
         lambda X: 3 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2]),
         None, n_solves),
        ("star_cubed_sphere", inputs.star_sphere_mesh(level=2, refine=1, r_out=20.0), inputs.star_source,
         inputs.star_solution, 3),
    ]
    with torch.cuda.stream(stream):
        for name, desc, g, gD, n_case in cases:
            ctx = dgell.Context(desc)
            info = ctx.level_info()
            xyz, bxyz = ctx.quadrature_points()
            gq = torch.tensor(g(xyz.T.cpu().numpy()), device="cuda")
            gd = torch.tensor(gD(bxyz.T.cpu().numpy()), device="cuda") if gD is not None else None
            F = torch.empty(info["n_dofs"], dtype=torch.float64, device="cuda")
            ctx.rhs(gq, gd, F)
            res = {"n_dofs": info["n_dofs"], "n_elems": info["n_elems"], "levels": info["n_levels"]}
            if desc.get("blocks"):
                res["blocks"] = len(desc["blocks"])
            for pname, prec in (("fp64", dgell.DG_FP64), ("mixed_fp32_vcycle", dgell.DG_FP32)):
                lat, its, rr = [], [], []
                for s in range(n_case + 2):
                    x = torch.zeros_like(F)
                    stream.synchronize()
                    t = time.perf_counter()
                    st = ctx.solve(F, x, tol=1e-10, max_iter=300, mg_prec=prec)
                    stream.synchronize()
                    dt = time.perf_counter() - t
                    if s >= 2:
                        lat.append(dt)
                        its.append(st["iterations"])
                        rr.append(st["rel_residual"])
                r = _latency(lat)
                r.update({"iterations": its[-1], "max_rel_residual": max(rr)})
                res[pname] = r
            out[name] = res
            ctx.close()
        # puncture Newton on the 13-block cubed sphere (shell to r = 20, u = 0 there)
        punc = inputs.two_punctures()
        desc = inputs.puncture_sphere_mesh(punc, level=2)
        ctx = dgell.Context(desc)
        info = ctx.level_info()
        ctx.puncture_setup(punc)
        res = {"n_dofs": info["n_dofs"], "n_elems": info["n_elems"], "levels": info["n_levels"],
               "blocks": len(desc["blocks"])}
        for pname, prec in (("fp64", dgell.DG_FP64), ("mixed_fp32_vcycle", dgell.DG_FP32)):
            lat = []
            for s in range(3):
                u = torch.zeros(info["n_dofs"], dtype=torch.float64, device="cuda")
                stream.synchronize()
                t = time.perf_counter()
                steps, rn = ctx.newton_solve(u, tol_newton=1e-9, max_newton=12, mg_prec=prec, tol=1e-10,
                                             max_iter=300)
                stream.synchronize()
                lat.append(time.perf_counter() - t)
            r = _latency(lat[1:])
            r.update({"newton_steps": steps, "final_residual_norm": rn})
            res[pname] = r
        out["two_puncture_newton_cubed_sphere"] = res
        ctx.close()
    stream.synchronize()
    # served workload: requests of mixed type and size arriving as a Poisson process,
    # admitted by footprint onto 4 worker streams (FP32 V-cycle, FP64 outer, 1e-10)
    from paper_1907_01572_gb300 import serve
    # arrival rate ~70 % of the capacity measured for this mix with 4 slots (2.9 solves/s)
    reqs = serve.make_requests(n=64, rate_hz=2.0, seed=2, full=True)
    _, summary = serve.Server(slots=4).run(reqs)
    sizes = [int(((np.asarray(r["desc"]["p"]) + 1) ** 3).sum()) for r in reqs]
    summary["workload"] = ("64 requests, Poisson arrivals 2/s (seed 2); mix 50/30/20 % of Poisson (4^3-16^3 "
                           "elements, p 3..8), the density-jump star and two-puncture Newton solves on the 13-block "
                           "cubed sphere (shell to r = 20); FP32 V-cycle, FP64 outer FCG, 1e-10")
    summary["dofs_min_max"] = [min(sizes), max(sizes)]
    out["served"] = summary
    return out


def alu_peaks(torch):
    """Measured dense FP64 and FP32 (CUDA-core, TF32 off) GEMM rates in TFLOP/s."""
    res = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    for name, dt, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        best = 1e9
        for _ in range(3):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        res[name] = 2.0 * n ** 3 / best / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = prev
    return res


if __name__ == "__main__":
    sys.exit(main())
