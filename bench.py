"""Benchmark: matrix-free SIPG operator apply on the curved, 2:1 h-refined,
mixed-degree 32^3 sweep mesh (61,440 elements, p drawn from {2..7}, ~1.32e7
DOFs), plus the Poisson solve of the 4x4x4, p = 3 problem at 1e-10 relative
residual (solves/s, p50/p99).

One step = the FP32 operator apply y = L x over the whole mesh (all degree
buckets) for a batch of distinct resident input vectors (--batch, 64 by
default, so that 20 steps keep the GPU busy for about a second); the FP64 apply
and the solves are reported beside it.
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
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, ncu, every kernel of one FP32 apply of the
# sweep mesh with per-bucket launches), keyed by a hash of the sources that define the apply kernels and
# the data they read (kernels, launcher, packed records, geometry and mesh tables): any change to one of
# them makes the entry miss and the bench report null until the counters are taken again.
APPLY_SOURCES = ["apply_impl.cuh", "apply.h", "apply_f32.cu", "internal.h", "geom.cu", "geom.h", "host_mesh.cpp"]
TRAFFIC_BYTES_PER_APPLY = {"3db6ad468e9b020c": 1.3154e9,    # library versions 118-120
                           "0c7f8ffb426d0fae": 1.3316e9}    # versions 121-122: one capture per kernel


def apply_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in APPLY_SOURCES:
        with open(os.path.join(ROOT, "paper_1907_01572_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


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


CPU_LEGS = r"""
import os, sys, time, json
sys.path.insert(0, %(root)r)
import numpy as np
from paper_1907_01572_gb300 import inputs
from oracle.mesh import Mesh
from oracle import sipg, multigrid, krylov
cores = len(os.sched_getaffinity(0))
out = {"cores": cores}
desc = inputs.sweep_mesh(level=5, seed=0)
a, k = inputs.oracle_mesh_args(desc)
m = Mesh(*a, **k)
x = inputs.random_vector(m.n_dofs, seed=1)
rng = np.random.default_rng(%(seed)d)
els = [int(e) for e in rng.choice(m.n_elems, size=%(n1)d, replace=False)]
t = time.perf_counter()
sipg.apply_local(m, x, 10.0, elems=els)
dt = time.perf_counter() - t
dofs = int(sum((m.p[e] + 1) ** 3 for e in els))
out["dense_local_1"] = {"dofs": dofs, "seconds": dt, "gdofs": dofs / dt / 1e9, "elements": len(els)}
if %(legs)d:
    # dense-local apply on every core: forked workers (this process never touches a GPU)
    import multiprocessing as mp
    els_all = [int(e) for e in rng.choice(m.n_elems, size=%(nall)d, replace=False)]
    chunks = [els_all[i::cores] for i in range(cores)]
    def work(ch):
        sipg.apply_local(m, x, 10.0, elems=ch)
        return 0
    ctx = mp.get_context("fork")
    with ctx.Pool(cores) as pool:
        pool.map(work, [els_all[:1]] * cores)          # workers up
        t = time.perf_counter()
        pool.map(work, chunks)
        dt = time.perf_counter() - t
    dofs = int(sum((m.p[e] + 1) ** 3 for e in els_all))
    out["dense_local_all"] = {"dofs": dofs, "seconds": dt, "gdofs": dofs / dt / 1e9, "elements": len(els_all)}
    # CSR SpMV of the assembled FP64 operator of a scaled sweep mesh (same recipe, 15 x 8 fewer elements)
    d2 = inputs.sweep_mesh(level=2, seed=0)
    a2, k2 = inputs.oracle_mesh_args(d2)
    m2 = Mesh(*a2, **k2)
    A = sipg.assemble(m2, 10.0).tocsr()
    v = inputs.random_vector(m2.n_dofs, seed=1)
    reps = 20
    t = time.perf_counter()
    for _ in range(reps):
        A @ v
    dt = (time.perf_counter() - t) / reps
    spmv = {"n_dofs": m2.n_dofs, "nnz": int(A.nnz), "seconds_1": dt, "gdofs_1": m2.n_dofs / dt / 1e9}
    rows = np.array_split(np.arange(m2.n_dofs), cores)
    blocks = [A[r[0]:r[-1] + 1] for r in rows]
    def mv(i):
        for _ in range(reps):
            blocks[i] @ v
        return 0
    with ctx.Pool(cores) as pool:
        pool.map(mv, range(cores))
        t = time.perf_counter()
        pool.map(mv, range(cores))
        dt = (time.perf_counter() - t) / reps
    spmv.update({"seconds_all": dt, "gdofs_all": m2.n_dofs / dt / 1e9})
    out["csr_spmv"] = spmv
    # config-1 Poisson solve: MG-preconditioned FCG to 1e-10 (Alg. 2, 3)
    m1 = Mesh(*inputs.oracle_mesh_args(inputs.config1_mesh())[0], **inputs.oracle_mesh_args(inputs.config1_mesh())[1])
    u = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
    t = time.perf_counter()
    H = multigrid.Hierarchy(m1)
    F = sipg.rhs(m1, lambda X: 3 * np.pi ** 2 * u(X), u)
    t1 = time.perf_counter()
    xs, it, hist = krylov.fcg(H.J[-1], F, precond=lambda r: H.vcycle(r), tol=1e-10)
    t2 = time.perf_counter()
    out["config1_solve"] = {"setup_s": t1 - t, "solve_s": t2 - t1, "iterations": it, "rel_residual": hist[-1]}
print(json.dumps(out))
"""


def cpu_legs(n1, seed=0, legs=True, nall=None):
    """The oracle timed on the host cores in a subprocess that never touches a
    GPU: its dense-local apply on a sample of the sweep mesh's elements (one
    thread; with legs also on all cores), CSR SpMV of the assembled operator
    of a scaled sweep mesh (one thread and all cores), and the config-1
    MG-FCG solve.  Returns the parsed dict."""
    cores = len(os.sched_getaffinity(0))
    code = CPU_LEGS % dict(root=ROOT, seed=seed, n1=n1, legs=1 if legs else 0, nall=nall or 16 * cores)
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1200)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_sample(n_elems_sample, seed=0):
    """Single-thread dense-local oracle apply on a sample: (GDOF/s, dofs, seconds)."""
    d = cpu_legs(n_elems_sample, seed=seed, legs=False)["dense_local_1"]
    return d["gdofs"], d["dofs"], d["seconds"]


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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--batch", type=int, default=64,
                    help="input vectors per step (each step applies the operator to all of them)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--level", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--served", type=int, default=96, help="requests of the served stream to serve (512 in all)")
    ap.add_argument("--compactified", action="store_true",
                    help="also solve the star on the cubed sphere with the shell to r = 1e9 (level 3, p = 3, overlapping Schwarz)")
    ap.add_argument("--full-configs", action="store_true",
                    help="also solve configs 3 and 4 at their stated sizes (several minutes)")
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
        legs = cpu_legs(48, seed=0)
        d1 = legs["dense_local_1"]
        cpu = {"value": d1["gdofs"], "unit": "GDOF/s", "cores": 1, "kind": "oracle",
               "sample": "48 random elements (%d DOFs, %.1f s) of the same mesh, dense-local FP64 apply "
                         "incl. their mortars, single thread" % (d1["dofs"], d1["seconds"]),
               "dense_local_all_cores": dict(legs["dense_local_all"], cores=legs["cores"]),
               "csr_spmv": dict(legs["csr_spmv"], cores=legs["cores"],
                                mesh="sweep mesh at level 2 (120 elements, same recipe), assembled FP64 CSR, scipy"),
               "config1_oracle_solve": legs["config1_solve"]}

    import __graft_entry__
    __graft_entry__.build()
    from paper_1907_01572_gb300 import dgell, inputs

    stream = torch.cuda.current_stream()
    desc = inputs.sweep_mesh(level=args.level, seed=0)
    ctx = dgell.Context(desc)
    info = ctx.level_info()
    N = info["n_dofs"]
    R = max(1, args.batch)
    x64 = torch.tensor(inputs.random_vector(N, seed=1), device="cuda")
    # a batch of R distinct input vectors (x ~ N(0,1), seeds 1..R), all resident in HBM
    X32 = torch.empty(R, N, dtype=torch.float32, device="cuda")
    X32[0] = x64.float()
    for r in range(1, R):
        X32[r] = torch.tensor(inputs.random_vector(N, seed=1 + r), device="cuda").float()
    Y32 = torch.empty_like(X32)
    R64 = max(1, R // 8)
    X64 = torch.empty(R64, N, dtype=torch.float64, device="cuda")
    for r in range(R64):
        X64[r] = X32[r].double() if r else x64
    Y64 = torch.empty_like(X64)
    X16 = X32.bfloat16()

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

    def batch_apply(X, Y):
        for r in range(X.shape[0]):
            ctx.apply(X[r], Y[r])

    launches0 = ctx.launch_count()
    with Clocks(local) as clk:
        ms32 = timed(lambda: batch_apply(X32, Y32), args.steps, args.warmup, clk)
    launches = (ctx.launch_count() - launches0) * args.steps // (args.steps + args.warmup)
    ms64 = timed(lambda: batch_apply(X64, Y64), max(3, args.steps // 4), args.warmup)
    ms16 = timed(lambda: batch_apply(X16, Y32), args.steps, args.warmup)

    # end to end through the C ABI with host buffers (pinned): every step is one
    # dg_apply_host call that copies its batch of inputs host -> device and its
    # outputs device -> host inside the region, overlapping them with the applies
    Re = max(1, R // 8)
    hx = X32[:Re].cpu().pin_memory()
    hy = torch.empty_like(hx).pin_memory()

    def e2e_step():
        ctx.apply_host(hx, hy)

    ms_e2e = timed(e2e_step, max(3, args.steps), 3)

    ms32, ms64, ms_e2e, ms16 = max_over_ranks([ms32, ms64, ms_e2e, ms16], dist, "cuda")
    total_dofs = N * world
    g32 = job_throughput(N * R, world, ms32)
    g64 = job_throughput(N * R64, world, ms64)
    ge2e = job_throughput(N * Re, world, ms_e2e)
    ms32_apply = ms32 / R

    # algorithmic bytes per DOF: x + y + 3 coordinates per LGL node (curved isoparametric geometry)
    b32 = 4 + 4 + 12
    b64 = 8 + 8 + 24
    ach32 = N * R * b32 / (ms32 * 1e-3) / 1e9
    ach64 = N * R64 * b64 / (ms64 * 1e-3) / 1e9

    solve = None
    peaks_alu = alu_peaks(torch) if rank == 0 else {}
    if not args.no_solve and rank == 0:
        solve = solve_bench(dgell, inputs, torch, n_served=args.served)
    if args.full_configs and rank == 0:
        solve = dict(solve or {}, full_size=full_configs(dgell, inputs, torch))
    if args.compactified and rank == 0:
        solve = dict(solve or {}, compactified_shell=compactified_config(dgell, inputs, torch))
    flops = info["apply_flops"]

    if rank == 0:
        line = {
            "metric": "DG apply GDOF/s", "value": g32, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_dofs": N, "n_elems": info["n_elems"], "levels": info["n_levels"],
                       "batch": R, "step": "%d applies of the FP32 operator to %d distinct resident inputs" % (R, R),
                       "ms_per_apply": ms32_apply,
                       "l2": "inputs larger than L2 (%.1f GB of inputs and outputs, metric terms ~0.4 GB)"
                             % (2 * 4 * N * R / 1e9), "parallelism": "replicas"},
            "roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm, "unit": "GB/s", "frac": ach32 / hbm,
                         "traffic": TRAFFIC_BYTES_PER_APPLY.get(apply_source_hash()) if args.level == 5 else None,
                         "peak_kind": peak_kind, "bytes_per_dof": b32, "apply_source_hash": apply_source_hash(),
                         # the stricter vector-only figure: read x and write y once (8 B/DOF in FP32)
                         "frac_vec": N * R * 8 / (ms32 * 1e-3) / 1e9 / hbm,
                         "kernel": "dg_apply FP32: trace + element kernels of all degree buckets (one apply)"},
            "cpu_baseline": cpu,
            "e2e": {"value": ge2e, "unit": "GDOF/s", "h2d_bytes_per_step": N * 4 * Re, "d2h_bytes_per_step": N * 4 * Re,
                    "batch": Re, "call": "dg_apply_host: pinned host vectors, copies in and out overlapped with the applies"},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "fp64": {"value": g64, "unit": "GDOF/s", "ms_per_step": ms64, "batch": R64, "achieved_gbs": ach64,
                     "bytes_per_dof": b64,
                     "roofline": {"bound": "alu", "achieved": R64 * flops / (ms64 * 1e-3) / 1e12,
                                  "peak": peaks_alu.get("fp64"), "unit": "TFLOP/s",
                                  "frac": (R64 * flops / (ms64 * 1e-3) / 1e12) / peaks_alu["fp64"] if peaks_alu
                                  else None,
                                  "peak_kind": "measured this run: cuBLAS DGEMM 4096^3"}},
            "bf16_operands": {"value": total_dofs * R / (ms16 * 1e-3) / 1e9, "unit": "GDOF/s", "ms_per_step": ms16,
                              "bytes_per_dof": 18, "achieved_gbs": N * R * 18 / (ms16 * 1e-3) / 1e9,
                              "frac_hbm": N * R * 18 / (ms16 * 1e-3) / 1e9 / hbm,
                              "note": "x bf16, FP32 arithmetic (n = 8 volume passes on TF32 tensor cores), y fp32"},
            "fp32_alu": {"achieved": R * flops / (ms32 * 1e-3) / 1e12, "peak": peaks_alu.get("fp32"),
                         "unit": "TFLOP/s",
                         "frac": (R * flops / (ms32 * 1e-3) / 1e12) / peaks_alu["fp32"] if peaks_alu else None,
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


SERVED_RATE_HZ = 2.2   # 70 % of the 3.1 solves/s this mix sustains on 4 slots (GB300, 128 saturated requests)
# V-cycle options of the star solves on the cubed sphere (measured at 4.4e5 and 4.1e6 DOFs: 40 / 63 FCG
# iterations against 87 / 115 with the paper's N_eigs = N_cheb = 15, about 20-30 % less time).  The
# Newton problems and the served mix keep the paper's options: the exact coarse solve's setup (the
# level-0 operator assembled by applies and inverted on the host, per context and, for Newton, per
# Jacobian) cost the served mix far more than it saved (capacity 0.46 against 3.0 solves/s).  The
# library's defaults stay the paper's.
SPHERE_MG = dict(n_eigs=35, n_cheb=10, coarse=1)
# V-cycle of the star with the inverse-radius shell out to r = 1e9 (one degree, conforming faces): the
# Schwarz smoother with overlapping subdomains, exact local and coarse solves
OVERLAP_MG = dict(smoother=2, coarse=1, n_schwarz=3)


def l2_error_closed_form(dgell, torch, desc, u, u_fn):
    """||u_h - u||_2 (eq. l2norm) by the operator's own GL quadrature, from
    library calls only: u_h^T M u_h - 2 u_h^T F(u) + sum F(u^2), with M u_h the
    difference of two applies (with and without the zeroth-order term f = 1)
    and F(g) = dg_rhs of g (sum_i phi_i = 1).  None if any call fails."""
    try:
        ctx = dgell.Context(desc)
        try:
            xyz, _ = ctx.quadrature_points()
            ue = torch.tensor(u_fn(xyz.T.cpu().numpy()), dtype=torch.float64, device="cuda")
            Lu = torch.empty_like(u)
            ctx.apply(u, Lu)
            ctx.set_zeroth_order(torch.ones_like(ue))
            LMu = torch.empty_like(u)
            ctx.apply(u, LMu)
            F1 = torch.empty_like(u)
            ctx.rhs(ue, None, F1)
            F2 = torch.empty_like(u)
            ctx.rhs(ue * ue, None, F2)
            torch.cuda.current_stream().synchronize()
            e2 = float(u @ (LMu - Lu)) - 2.0 * float(u @ F1) + float(F2.sum())
            return max(e2, 0.0) ** 0.5
        finally:
            ctx.close()
    except Exception:
        return None


def solve_bench(dgell, inputs, torch, n_solves=8, n_served=96, n_cap=32):
    """Linear solves to 1e-10 relative residual (FP64 outer FCG) with the plain
    FP64 V-cycle and with the FP32 V-cycle, each V-cycle replayed as a CUDA graph
    on a dedicated stream: the 4^3 p=3 Poisson problem and the star with a
    density jump on the 13-block cubed sphere (centre cube a = 2, wedges to
    r = 10, inverse-radius shell to r = 20, closed-form Dirichlet data), and
    the same star on a uniform p = 4 sphere with the shell out to r = 1e9
    (overlapping Schwarz smoother); then the two-puncture Newton solve on the
    same kind of cubed sphere."""
    import numpy as np
    out = {}
    stream = torch.cuda.Stream()
    cases = [
        ("poisson_4x4x4_p3", inputs.config1_mesh(),
         lambda X: 3 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2]),
         None, n_solves, {}),
        ("star_cubed_sphere", inputs.star_sphere_mesh(level=2, refine=1, r_out=20.0), inputs.star_source,
         inputs.star_solution, 3, SPHERE_MG),
        ("star_compactified_sphere_overlap",
         inputs.star_sphere_mesh(level=2, refine=0, p_cut=4, p_lo=4, p_hi=4, r_out=1e9), inputs.star_source,
         inputs.star_solution, 3, OVERLAP_MG),
    ]
    with torch.cuda.stream(stream):
        for name, desc, g, gD, n_case, mg in cases:
            ctx = dgell.Context(desc)
            info = ctx.level_info()
            xyz, bxyz = ctx.quadrature_points()
            gq = torch.tensor(g(xyz.T.cpu().numpy()), device="cuda")
            gd = torch.tensor(gD(bxyz.T.cpu().numpy()), device="cuda") if gD is not None else None
            F = torch.empty(info["n_dofs"], dtype=torch.float64, device="cuda")
            ctx.rhs(gq, gd, F)
            res = {"n_dofs": info["n_dofs"], "n_elems": info["n_elems"], "levels": info["n_levels"], "mg_opts": mg}
            if desc.get("blocks"):
                res["blocks"] = len(desc["blocks"])
            exact = gD if gD is not None else (
                lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2]))
            for pname, prec in (("fp64", dgell.DG_FP64), ("mixed_fp32_vcycle", dgell.DG_FP32)):
                lat, its, rr = [], [], []
                for s in range(n_case + 2):
                    x = torch.zeros_like(F)
                    stream.synchronize()
                    t = time.perf_counter()
                    st = ctx.solve(F, x, tol=1e-10, max_iter=300, mg_prec=prec, **mg)
                    stream.synchronize()
                    dt = time.perf_counter() - t
                    if s >= 2:
                        lat.append(dt)
                        its.append(st["iterations"])
                        rr.append(st["rel_residual"])
                r = _latency(lat)
                r.update({"iterations": its[-1], "max_rel_residual": max(rr),
                          "l2_error_vs_closed_form": l2_error_closed_form(dgell, torch, desc, x, exact)})
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
    # served workload: requests of mixed type and size (1.4e4 to 4.2e6 DOFs) arriving as a Poisson
    # process, admitted by footprint onto 4 worker streams (FP64 outer FCG, 1e-10)
    from paper_1907_01572_gb300 import serve
    reqs = serve.make_requests(n=n_served, rate_hz=SERVED_RATE_HZ, seed=2, served=True)
    _, summary = serve.Server(slots=4).run([dict(r) for r in reqs])
    sizes = [int(((np.asarray(r["desc"]["p"]) + 1) ** 3).sum()) for r in reqs]
    summary["workload"] = ("first %d requests of the 512-request stream, Poisson arrivals %.1f/s (seed 2, about 70 %% "
                           "of the mix's measured capacity); mix 50/30/20 %% of Poisson boxes (1.4e4-4.2e6 DOFs, p 3..8), "
                           "the density-jump star and two-puncture Newton solves on level-1/2 13-block cubed spheres "
                           "(shell to r = 20); FP32 V-cycle, FP64 outer FCG, 1e-10" % (n_served, SERVED_RATE_HZ))
    summary["dofs_min_max"] = [min(sizes), max(sizes)]
    out["served"] = summary
    # capacity of the same mix, mixed precision vs the plain FP64 V-cycle: its first n_cap
    # requests all queued at once (solves/s at saturation)
    cap = {}
    for pname, prec in (("mixed_fp32_vcycle", dgell.DG_FP32), ("fp64", dgell.DG_FP64)):
        burst = [dict(r, arrival=0.0) for r in reqs[:n_cap]]
        _, s = serve.Server(slots=4, mg_prec=prec).run(burst)
        cap[pname] = {k: s[k] for k in ("requests", "wall_s", "solves_per_s", "p50_ms", "p99_ms")}
    out["served_capacity"] = cap
    return out


def compactified_config(dgell, inputs, torch, level=3, p=3):
    """The density-jump star on config 3's domain as stated: the 13-block cubed
    sphere with the inverse-radius shell out to r = 1e9, every block at `level`
    with one degree p (the overlapping Schwarz smoother needs one degree and
    conforming faces), closed-form Dirichlet data at r = 1e9.  One warm-up
    solve (subdomain setup, plan tuning, graph capture), then a timed one, with
    the FP32 and the FP64 V-cycle, to 1e-10."""
    out = {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        desc = inputs.star_sphere_mesh(level=level, refine=0, p_cut=p, p_lo=p, p_hi=p, r_out=1e9)
        ctx = dgell.Context(desc)
        info = ctx.level_info()
        xyz, bxyz = ctx.quadrature_points()
        gq = torch.tensor(inputs.star_source(xyz.T.cpu().numpy()), device="cuda")
        gd = torch.tensor(inputs.star_solution(bxyz.T.cpu().numpy()), device="cuda")
        F = torch.empty(info["n_dofs"], dtype=torch.float64, device="cuda")
        ctx.rhs(gq, gd, F)
        out = {"n_dofs": info["n_dofs"], "n_elems": info["n_elems"], "levels": info["n_levels"], "p": p,
               "blocks": len(desc["blocks"]), "r_out": 1e9, "mg_opts": OVERLAP_MG}
        sols = {}
        for pname, prec in (("mixed_fp32_vcycle", dgell.DG_FP32), ("fp64", dgell.DG_FP64)):
            for s in range(2):
                x = torch.zeros_like(F)
                stream.synchronize()
                t = time.perf_counter()
                st = ctx.solve(F, x, tol=1e-10, max_iter=300, mg_prec=prec, **OVERLAP_MG)
                stream.synchronize()
                dt = time.perf_counter() - t
                if s == 0:
                    out[pname + "_first_solve_s"] = dt   # includes the subdomain setup
            sols[pname] = x
            out[pname] = {"seconds": dt, "solves_per_s": 1.0 / dt, "iterations": st["iterations"],
                          "rel_residual": st["rel_residual"]}
        out["device_gb"] = ctx.level_info()["device_bytes"] / 1e9
        out["mixed_vs_fp64_rel_l2"] = float((sols["mixed_fp32_vcycle"] - sols["fp64"]).norm() / sols["fp64"].norm())
        ctx.close()
    stream.synchronize()
    return out


def full_configs(dgell, inputs, torch):
    """Configs 3 and 4 at the stated sizes (shell ended at r = 20: the
    Chebyshev-smoothed V-cycle stops contracting on longer compactified
    shells): the density-jump star on the 13-block cubed sphere at level 4
    with the cells cut by r = 0.5 and r = 1 refined three times (115,968
    elements, p 4..8, 4.4e7 DOFs), and the two then three punctures with
    every block at level 4, p = 5, p = 8 on the cells holding a puncture
    (53,360 elements, 1.2e7 DOFs), Newton from u = 0.  Each problem is solved
    once to warm up (plan tuning, graph capture) and then timed, with the FP32
    V-cycle (mixed) and with the plain FP64 V-cycle, to 1e-10."""
    import numpy as np
    out = {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        desc = inputs.star_sphere_mesh(level=4, refine=3, r_out=20.0)
        ctx = dgell.Context(desc)
        info = ctx.level_info()
        xyz, bxyz = ctx.quadrature_points()
        gq = torch.tensor(inputs.star_source(xyz.T.cpu().numpy()), device="cuda")
        gd = torch.tensor(inputs.star_solution(bxyz.T.cpu().numpy()), device="cuda")
        F = torch.empty(info["n_dofs"], dtype=torch.float64, device="cuda")
        ctx.rhs(gq, gd, F)
        res = {"n_dofs": info["n_dofs"], "n_elems": info["n_elems"], "levels": info["n_levels"],
               "blocks": len(desc["blocks"]), "device_gb": info["device_bytes"] / 1e9}
        sols = {}
        for pname, prec in (("mixed_fp32_vcycle", dgell.DG_FP32), ("fp64", dgell.DG_FP64)):
            for s in range(2):
                x = torch.zeros_like(F)
                stream.synchronize()
                t = time.perf_counter()
                st = ctx.solve(F, x, tol=1e-10, max_iter=600, mg_prec=prec, **SPHERE_MG)
                stream.synchronize()
                dt = time.perf_counter() - t
            sols[pname] = x
            res[pname] = {"seconds": dt, "solves_per_s": 1.0 / dt, "iterations": st["iterations"],
                          "rel_residual": st["rel_residual"]}
        res["mixed_vs_fp64_rel_l2"] = float((sols["mixed_fp32_vcycle"] - sols["fp64"]).norm() / sols["fp64"].norm())
        out["config3_star_cubed_sphere"] = res
        ctx.close()
        del sols, F, gq, gd
        for name, punc in (("two_punctures", inputs.two_punctures()), ("three_punctures", inputs.three_punctures())):
            desc = inputs.puncture_sphere_mesh(punc, level=4, p_base=5, p_fine=8)
            ctx = dgell.Context(desc)
            info = ctx.level_info()
            ctx.puncture_setup(punc)
            res = {"n_dofs": info["n_dofs"], "n_elems": info["n_elems"], "levels": info["n_levels"],
                   "blocks": len(desc["blocks"])}
            us = {}
            for pname, prec in (("mixed_fp32_vcycle", dgell.DG_FP32), ("fp64", dgell.DG_FP64)):
                for s in range(2):
                    u = torch.zeros(info["n_dofs"], dtype=torch.float64, device="cuda")
                    stream.synchronize()
                    t = time.perf_counter()
                    steps, rn = ctx.newton_solve(u, tol_newton=1e-9, max_newton=12, mg_prec=prec, tol=1e-10,
                                                 max_iter=600)
                    stream.synchronize()
                    dt = time.perf_counter() - t
                us[pname] = u
                res[pname] = {"seconds": dt, "solves_per_s": 1.0 / dt, "newton_steps": steps,
                              "final_residual_norm": rn}
            res["mixed_vs_fp64_rel_l2"] = float((us["mixed_fp32_vcycle"] - us["fp64"]).norm() / us["fp64"].norm())
            out["config4_" + name + "_cubed_sphere"] = res
            ctx.close()
    stream.synchronize()
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
