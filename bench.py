"""Benchmark of the GPU multigrid Poisson solver (one JSON line on rank 0).

Workload: Q1 FEM Poisson on the unit square at level L=10 (1025^2 = 1,050,625 nodes), a = 1, zero
Dirichlet boundary, b ~ U[-1,1] on interior nodes (seeded), V(2,2) damped Jacobi (omega 0.7),
coarsest level 2 solved exactly, relative residual 1e-8.  The headline is FP32-inner multigrid
under FP64 defect correction (inner reduction 1e-2); plain FP64 multigrid is measured on the same
GPU beside it.  A step is one complete solve to 1e-8 from x = 0 (setup excluded, reported apart).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: per-step CUDA events on the solve stream after W warm-up solves; a 512 MiB buffer is
written between timed steps (outside the events) to flush the 129 MB L2.  `e2e` repeats the
measurement through the same C call with host buffers (host->device copy of b and device->host
copy of x inside the timed region).  `roofline` times the dominant kernel of the headline solve
with events around each of its launches (a separate profiled pass over K solves), against the
measured HBM copy bandwidth.  Beside the headline the line carries the band kernels alone at
L = 12, the L = 12 lognormal configuration (`l12_lognormal`: FP64 MG, FP32-inner and FP16-band
DC), the 256-problem batch (`batch256`), a sample of the serving workload (`serve`), and at the
end the L = 10 solves per precision (`mixed`, `fp64`, `fp16band`, `pcg_fp32`), each with its
relative L2 difference from the oracle solved to 1e-13.  `cpu_baseline` times the FP64 CPU oracle
on one full solve of the same problem on one host core (and, under `all_cores`, one independent
solve per host core); that leg also evaluates this run's results with the oracle.  With N > 1
(torchrun) every rank solves its own independent problem (weak scaling, no collective on the data
path); value = all ranks' DOF / slowest rank.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_BENCH = 10
TOL = 1e-8
WORKLOAD = "poisson-q1-L10-const-coef-uniform-rhs"


def bench_config(L=L_BENCH):
    """The workload of the default line (both arms print the same dict)."""
    N = ((1 << L) + 1) ** 2
    return {"workload": WORKLOAD if L == L_BENCH else "poisson-q1-L%d-const-coef-uniform-rhs" % L,
            "L": L, "dof": N, "coef": "a=1", "rhs": "U[-1,1] interior, seed=rank",
            "cycle": "V(2,2) jacobi omega=0.7", "coarse_L": 2, "tol": TOL,
            "prec": "fp32-inner defect correction, inner 1e-2",
            "l2_between_steps": "flushed (512 MiB write)"}


def sig(v, d=4):
    """Round floats (recursively) to d significant digits: keeps the line short."""
    if isinstance(v, float):
        return float("%.*g" % (d, v)) if v == v and abs(v) != float("inf") else v
    if isinstance(v, dict):
        return {k: sig(x, d) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [sig(x, d) for x in v]
    return v


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=None,
                    help="refinement level (default 10, the benchmark workload, and 12 for the "
                         "kernels workload; others for profiling)")
    ap.add_argument("--quick", action="store_true",
                    help="timed solves only (no e2e, profiled pass or CPU baseline): for ncu captures")
    ap.add_argument("--host-loop", action="store_true",
                    help="run solves as one graph launch per iteration (ncu cannot profile kernels "
                         "inside the device-side loop)")
    ap.add_argument("--workload", default="solve", choices=["solve", "batch", "serve", "kernels", "blas1", "swe", "solvers"],
                    help="solve: the L=10 benchmark (default); batch: 256 uneven problems in one "
                         "batched solve; serve: Poisson-arrival requests through the solve server; "
                         "kernels: band-SpMV / defect / Jacobi alone at L=12 in FP64, FP32, FP16-band; "
                         "blas1: axpy / dot rate vs length; swe: fused shallow-water prediction step "
                         "vs the same step composed from library calls; solvers: solve time of "
                         "multigrid / defect correction vs PCG, exact vs CG coarse solve")
    ap.add_argument("--requests", type=int, default=10000, help="serve: number of requests")
    ap.add_argument("--load", type=float, default=0.7, help="serve: offered load / capacity")
    ap.add_argument("--serve-requests", type=int, default=1500,
                    help="requests of the serving sample in the default line (0: none)")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="serve: device memory budget")
    ap.add_argument("--slots", type=int, default=64, help="serve: concurrently active requests")
    ap.add_argument("--swe-grid", type=int, default=0, help="swe: one W x W grid only (default: 256, 1024, 4096)")
    ap.add_argument("--swe-type", default="all", choices=["all", "f32", "f64"], help="swe: element types")
    return ap.parse_args()


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("HN_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def max_over_ranks(v, pg, device=None):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg, device=None):
    if pg is not None:
        import torch
        t = torch.zeros(1, device=device)
        pg.all_reduce(t)


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def ncu_traffic_per_node(kernel):
    """DRAM bytes per node of `kernel` from the committed ncu summary (profiles/), or None."""
    path = os.path.join(ROOT, "profiles", "jacobi_f32_L12_ncu.md")
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_node") and kernel in line:
                return float(line.split("=")[1].split()[0])
    except OSError:
        pass
    return None


def solve_roofline(n_dof, ms, peak_gbs, inner_cycles=0, outer_iters=0, fp64_cycles=0):
    """A whole solve against its bandwidth roofline: the algorithmic (compulsory, unfused) bytes
    per DOF of the cycles and outer steps it ran, moved at the measured copy bandwidth, as a
    fraction of the measured time.  A V(2,2) cycle moves, on the finest level, four smoothing
    sweeps and one defect (x, b in, x' or r out, with the bands: 48 B/DOF in FP32, 96 in FP64), the
    restriction (5 / 10 B) and the prolongation with its correction (9 / 18 B), and 4/3 of that
    over the hierarchy; the residual check rides in the next cycle's first sweep.  A defect
    correction adds one FP64 defect per outer step and a last one that stops it (96 B each), and
    one FP64 update per step (x += s c: 24 B)."""
    fp32_cycle = (4 * 48 + 48 + 5 + 9) * 4.0 / 3.0
    fp64_cycle = (4 * 96 + 96 + 10 + 18) * 4.0 / 3.0
    outer = (outer_iters + 1) * 96.0 + outer_iters * 24.0 if outer_iters > 0 else 0.0
    per_dof = inner_cycles * fp32_cycle + fp64_cycles * fp64_cycle + outer
    roof_ms = per_dof * n_dof / (peak_gbs * 1e9) * 1e3
    return {"bytes_per_dof": per_dof, "roofline_ms": roof_ms, "ms": ms, "frac": roof_ms / ms}


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(L, seed, prec):
    """The oracle, as it stands, on one host core: one full solve of the bench problem."""
    import numpy as np
    import oracle as O
    from paper_0904_4152_gb300 import inputs as I
    b = I.rhs_uniform(L, seed)
    O.lib()
    t0 = time.perf_counter()
    x, st = O.mg_solve(L, b, prec=prec, tol=TOL)
    dt = time.perf_counter() - t0
    N = ((1 << L) + 1) ** 2
    return {"value": N / dt, "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": "one full %s solve to 1e-8 at L=%d (%d DOF), %.2f s, %d cycles"
                      % ("FP32-inner DC" if prec == 1 else "FP64 MG", L, N, dt, st["cycles"]),
            "seconds": dt}


def _oracle_warm(_):
    import oracle as O
    from paper_0904_4152_gb300 import inputs as I   # noqa: F401
    O.lib()
    return os.getpid()


def _oracle_solve(task):
    L, seed, prec = task
    import oracle as O
    from paper_0904_4152_gb300 import inputs as I
    b = I.rhs_uniform(L, seed)
    t0 = time.perf_counter()
    O.mg_solve(L, b, prec=prec, tol=TOL)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(L, seed, prec):
    """The same oracle, unchanged, on every host core: one independent solve per core in spawned
    processes (spawned, not forked: this process has a CUDA context)."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(_oracle_warm, range(n))           # imports and library loads outside the timing
        t0 = time.perf_counter()
        pool.map(_oracle_solve, [(L, seed + k, prec) for k in range(n)], chunksize=1)
        wall = time.perf_counter() - t0
    N = ((1 << L) + 1) ** 2
    return {"value": n * N / wall, "unit": "DOF/s", "cores": n, "kind": "oracle",
            "sample": "%d independent %s solves to 1e-8 at L=%d, one per core, %.2f s wall"
                      % (n, "FP32-inner DC" if prec == 1 else "FP64 MG", L, wall)}


def run_reference(args, rank, world, pg):
    if rank != 0:
        return
    import oracle as O
    O.lib()
    times = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(L_BENCH, 0, 1)
        if i >= args.warmup:
            times.append(r["seconds"])
    N = ((1 << L_BENCH) + 1) ** 2
    total = sum(times)
    value = N * len(times) / total
    line = {"impl": "reference", "metric": "MG Poisson DOF/s to 1e-8 (mixed vs FP64)",
            "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic", "config": bench_config(),
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                             "sample": "%d full FP32-inner DC solves to 1e-8 at L=%d on one core "
                                       "(CPU oracle, plain C++)" % (len(times), L_BENCH)},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# FP64 operations per node of the FP64 band and transfer kernels (the defect is one FMA chain
# from b; Jacobi adds one FMA; the restriction does 9 per coarse node, 2.25 per fine node; the
# prolongation 1, 2 or 4 per fine node by its position, 2.25 on average)
FP64_OPS_PER_NODE = {"spmv": 9.0, "defect": 9.0, "jacobi": 10.0, "restrict": 2.25, "prolong": 2.25}


def band_kernels(hn, stream, peak, L=12, reps=20, rates=None):
    """Band-SpMV, defect and Jacobi launched alone on level L (FP64, FP32, FP16-band storage):
    mean launch time by CUDA events and algorithmic bytes -> GB/s and fraction of `peak`.  For
    FP64 also the fraction of min(HBM, FP64 rate) (`rates`: hn_measure_fp_rates)."""
    band = {}
    A = hn.hn_band_create(L)
    N = ((1 << L) + 1) ** 2
    for pname, prec in (("fp64", hn.HN_PREC_FP64), ("fp32", hn.HN_PREC_FP32_DC),
                        ("fp16band", hn.HN_PREC_FP16BAND_DC)):
        mg = hn.hn_mg_setup(A, prec=prec, stream=stream.cuda_stream)
        row = {}
        for oname, op in (("spmv", hn.HN_OP_SPMV), ("defect", hn.HN_OP_DEFECT),
                          ("jacobi", hn.HN_OP_JACOBI), ("restrict", hn.HN_OP_RESTRICT),
                          ("prolong", hn.HN_OP_PROLONG_ADD)):
            ms, by = hn.hn_mg_time_kernel(mg, op, L, reps=reps)
            r = {"gb_per_s": by / (ms * 1e-3) / 1e9, "frac": by / (ms * 1e-3) / 1e9 / peak,
                 "us": ms * 1e3, "bytes": by}
            if pname == "fp64" and rates:
                t_hbm = by / (peak * 1e9)
                t_fp64 = FP64_OPS_PER_NODE[oname] * N / rates["fp64_fma_per_s"]
                r["bound"] = "fp64" if t_fp64 > t_hbm else "hbm"
                r["frac_of_bound"] = max(t_hbm, t_fp64) / (ms * 1e-3)
            row[oname] = r
        band[pname] = row
        hn.hn_mg_destroy(mg)
    hn.hn_band_destroy(A)
    return band


def run_kernels(args, rank, local):
    import torch
    import __graft_entry__ as g
    from paper_0904_4152_gb300 import hn
    torch.cuda.set_device(local)
    g.build()
    peak, kind = measured_peak_gbs()
    rates = hn.hn_measure_fp_rates()
    band = band_kernels(hn, torch.cuda.current_stream(), peak, L=args.level if args.level is not None else 12,
                        rates=rates)
    if rank == 0:
        print(json.dumps({"metric": "band kernels alone, HBM GB/s", "peak": peak, "peak_kind": kind,
                          "fp_rates": rates, "fp64_ops_per_node": FP64_OPS_PER_NODE,
                          "kernels": band}), flush=True)


def run_blas1(args, rank, local):
    """BLAS level-1 kernels (Sec. 6.1, Fig. 2): axpy / dot rate against vector length."""
    import torch
    import __graft_entry__ as g
    from paper_0904_4152_gb300 import hn
    torch.cuda.set_device(local)
    g.build()
    peak, kind = measured_peak_gbs()
    stream = torch.cuda.current_stream()
    rows = []
    for dtype, name in ((torch.float32, "f32"), (torch.float64, "f64")):
        esize = 4 if dtype == torch.float32 else 8
        for lg in range(10, 29, 2):
            n = 1 << lg
            x = torch.rand(n, dtype=dtype, device="cuda")
            y = torch.rand(n, dtype=dtype, device="cuda")
            r = torch.zeros(1, dtype=torch.float64, device="cuda")
            for op in ("axpy", "dot"):
                def call(st):
                    if op == "axpy":
                        hn.hn_axpy(1e-9, x, y, st)
                    else:
                        hn.hn_dot(x, y, r, st)
                for _ in range(3):
                    call(stream)
                torch.cuda.synchronize()
                # back-to-back calls captured into a CUDA graph: device time, not host call overhead
                reps = max(5, min(200, int(2e8 / (n * esize))))
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.stream(side):
                    with torch.cuda.graph(graph, stream=side):
                        cs = torch.cuda.current_stream()
                        for _ in range(reps):
                            call(cs)
                torch.cuda.current_stream().wait_stream(side)
                graph.replay()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                graph.replay()
                e1.record(stream)
                torch.cuda.synchronize()
                us = e0.elapsed_time(e1) * 1e3 / reps
                del graph
                nbytes = (3 if op == "axpy" else 2) * n * esize
                rows.append({"op": op, "type": name, "n": n, "us": us, "gb_per_s": nbytes / us / 1e3,
                             "mflop_per_s": 2 * n / us, "in_l2": nbytes < 120e6,
                             "frac_hbm": nbytes / us / 1e3 / peak})
            del x, y
    if rank == 0:
        print(json.dumps({"metric": "BLAS-1 axpy / dot rate vs length (HBM GB/s, MFLOP/s)", "peak": peak,
                          "peak_kind": kind, "rows": rows}), flush=True)


def run_swe(args, rank, local):
    """Shallow-water prediction step u + M1 v + M2 w + M3 u + M4 u + s with four-band matrices
    (Sec. 2.2): the fused kernel against the same step composed from library calls (four band
    products into temporaries, then axpy), on W x W grids, FP32 and FP64."""
    import torch
    import __graft_entry__ as g
    from paper_0904_4152_gb300 import hn
    torch.cuda.set_device(local)
    g.build()
    peak, kind = measured_peak_gbs()
    stream = torch.cuda.current_stream()
    rows = []
    for dtype, name in ((torch.float32, "f32"), (torch.float64, "f64")):
        if args.swe_type not in ("all", name):
            continue
        esize = 4 if dtype == torch.float32 else 8
        for W in ((args.swe_grid,) if args.swe_grid else (256, 1024, 4096)):
            n = W * W
            offs = [[-2, -1, 1, 2], [-2 * W, -W, W, 2 * W], [-1, 0, 1, 2], [-W - 1, -W + 1, W - 1, W + 1]]
            bands = [[torch.rand(n, dtype=dtype, device="cuda") - 0.5 for _ in range(4)] for _ in range(4)]
            u, v, w, src = (torch.rand(n, dtype=dtype, device="cuda") for _ in range(4))
            out = torch.empty_like(u)
            tmp = [torch.empty_like(u) for _ in range(4)]
            xs = (v, w, u, u)

            def call_on(label, st):
                if label == "fused":
                    hn.hn_swe_predict(offs, bands, u, v, w, src, out, st)
                    return
                for m in range(4):
                    hn.hn_band4_spmv(offs[m], bands[m], xs[m], tmp[m], st)
                out.copy_(u)
                for m in range(4):
                    hn.hn_axpy(1.0, tmp[m], out, st)
                hn.hn_axpy(1.0, src, out, st)

            def fused():
                call_on("fused", stream)

            def composed():
                call_on("composed", stream)

            res = {}
            for label, call in (("fused", fused), ("composed", composed)):
                for _ in range(3):
                    call()
                torch.cuda.synchronize()
                # the calls are captured into a CUDA graph and replayed, so that the device time
                # is measured rather than the host's call overhead
                reps = max(5, min(200, int(4e9 / (21 * n * esize))))
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.stream(side):
                    with torch.cuda.graph(graph, stream=side):
                        cs = torch.cuda.current_stream()
                        for _ in range(reps):
                            call_on(label, cs)
                torch.cuda.current_stream().wait_stream(side)
                graph.replay()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                graph.replay()
                e1.record(stream)
                torch.cuda.synchronize()
                res[label] = e0.elapsed_time(e1) * 1e3 / reps
                del graph
            nbytes = 21 * n * esize           # 16 bands + u, v, w, s read, u_new written
            rows.append({"type": name, "grid": "%dx%d" % (W, W), "n": n, "fused_us": res["fused"],
                         "composed_us": res["composed"], "speedup": res["composed"] / res["fused"],
                         "fused_gb_per_s": nbytes / res["fused"] / 1e3,
                         "fused_frac_hbm": nbytes / res["fused"] / 1e3 / peak,
                         "in_l2": nbytes < 120e6})
            del bands, u, v, w, src, out, tmp
    if rank == 0:
        print(json.dumps({"metric": "SWE prediction step, fused vs composed (HBM GB/s)", "peak": peak,
                          "peak_kind": kind, "bytes_per_row": "21 x element size (algorithmic)",
                          "rows": rows}), flush=True)


def run_solvers(args, rank, local):
    """Solve time to 1e-8 of each outer solver (multigrid / defect correction, CG preconditioned by
    one V cycle), coarse solver (exact, CG) and precision, at L = 10 (a = 1 and a lognormal field)
    and L = 12 (a = 1, and the lognormal field seed 0 with right-hand side seed 1); graph solves,
    L2 flushed between solves, CUDA events."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_0904_4152_gb300 import hn, inputs as I
    torch.cuda.set_device(local)
    g.build()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    for L, lognormal, rhs_seed in ((10, False, 0), (10, True, 0), (12, False, 0), (12, True, 1)):
        coef = I.lognormal_coef(L, 0) if lognormal else None
        b = torch.from_numpy(I.rhs_uniform(L, rhs_seed)).cuda()
        x = torch.zeros_like(b)
        A = hn.hn_band_create(L, coef)
        for prec in (hn.HN_PREC_FP64, hn.HN_PREC_FP32_DC, hn.HN_PREC_FP16BAND_DC):
            for solver in (hn.HN_SOLVER_MG, hn.HN_SOLVER_PCG):
                for coarse in (hn.HN_COARSE_EXACT, hn.HN_COARSE_CG):
                    mg = hn.hn_mg_setup(A, prec=prec, solver=solver, coarse_solver=coarse,
                                        stream=stream.cuda_stream)
                    for _ in range(3):
                        hn.hn_mg_solve(mg, L, b, x)
                    ms = []
                    for _ in range(args.steps):
                        flush.fill_(1)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        _, st, status = hn.hn_mg_solve(mg, L, b, x)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        assert status == hn.HN_OK
                        ms.append(e0.elapsed_time(e1))
                    rows.append({"L": L, "coef": "lognormal" if lognormal else "a=1", "rhs_seed": rhs_seed,
                                 "prec": ["fp64", "fp32", "fp16band"][prec],
                                 "solver": "pcg" if solver == hn.HN_SOLVER_PCG else "mg",
                                 "coarse": "cg" if coarse == hn.HN_COARSE_CG else "exact",
                                 "ms_median": float(np.median(ms)), "ms_min": float(np.min(ms)),
                                 "cycles": st["cycles"], "outer_iters": st["outer_iters"],
                                 "relres": st["relres"], "launches": hn.hn_mg_last_launches(mg)})
                    hn.hn_mg_destroy(mg)
        hn.hn_band_destroy(A)
    if rank == 0:
        print(json.dumps({"metric": "solve time to 1e-8 per solver, coarse solver and precision",
                          "l2_between_steps": "flushed (512 MiB write)", "rows": rows}), flush=True)


def l12_solves(hn, I, stream, flush, dev, steps, warmup):
    """The L = 12 configuration: lognormal a (sigma 1, correlation length 0.1, field seed 0),
    b ~ U[-1,1] seed 1; FP64 multigrid, FP32-inner and FP16-band-inner defect correction; CUDA
    events per solve, L2 flushed between solves.  Returns the rows and the solutions (host)."""
    import torch
    L = 12
    N = ((1 << L) + 1) ** 2
    coef = I.lognormal_coef(L, 0)
    b = torch.from_numpy(I.rhs_uniform(L, 1)).to(dev)
    x = torch.zeros_like(b)
    A = hn.hn_band_create(L, coef)
    rows, sols = {}, {}
    try:
        for name, prec in (("fp64", hn.HN_PREC_FP64), ("fp32dc", hn.HN_PREC_FP32_DC),
                           ("fp16dc", hn.HN_PREC_FP16BAND_DC)):
            mg = hn.hn_mg_setup(A, prec=prec, stream=stream.cuda_stream)
            try:
                for _ in range(warmup):
                    hn.hn_mg_solve(mg, L, b, x)
                ms = []
                for _ in range(steps):
                    flush.fill_(1)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    _, st, status = hn.hn_mg_solve(mg, L, b, x)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    assert status == hn.HN_OK, st
                    ms.append(e0.elapsed_time(e1))
            finally:
                hn.hn_mg_destroy(mg)
            t = statistics.median(ms)
            rows[name] = {"dof_per_s": N / (t * 1e-3), "ms": t, "cycles": st["cycles"],
                          "outer": st["outer_iters"], "relres": st["relres"]}
            sols[name] = x.cpu().numpy().copy()
    finally:
        hn.hn_band_destroy(A)
    return rows, sols, (L, coef, b.cpu().numpy())


def batch256_solves(hn, I, stream, flush, dev, steps, warmup):
    """The batched configuration: 256 problems, L ~ U{5..9} (seed 0), lognormal a (seeds 1000 + j),
    b ~ U[-1,1] (seeds 2000 + j), FP32-inner defect correction, one batched solve per step against
    the same problems solved one after the other.  Returns the row and a sample of solutions."""
    import torch
    count = 256
    levels = [int(v) for v in I.batch_levels(count, seed=0)]
    mgs, bs, xs, probs = [], [], [], []
    try:
        for j, L in enumerate(levels):
            coef, b = I.batch_problem(j, L)
            A = hn.hn_band_create(L, coef)
            try:
                mgs.append(hn.hn_mg_setup(A, prec=hn.HN_PREC_FP32_DC, stream=stream.cuda_stream))
            finally:
                hn.hn_band_destroy(A)
            probs.append((L, coef, b))
            bs.append(torch.from_numpy(b).to(dev))
            xs.append(torch.zeros_like(bs[-1]))
        dofs = sum(((1 << L) + 1) ** 2 for L in levels)
        stats = {}

        def batched():
            _, st, status = hn.hn_mg_solve_batch(mgs, levels, bs, xs)
            assert status == hn.HN_OK
            stats["b"] = st

        def looped():
            for mg, L, b, x in zip(mgs, levels, bs, xs):
                _, st, status = hn.hn_mg_solve(mg, L, b, x)
                assert status == hn.HN_OK

        def timed(fn, n, w):
            for _ in range(w):
                fn()
            ms = []
            for _ in range(n):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms.append(e0.elapsed_time(e1))
            return statistics.median(ms)

        t_loop = timed(looped, 1, 1)
        t_b = timed(batched, steps, warmup)            # last: xs hold the batched results
        cyc = [s["cycles"] for s in stats["b"]]
        sample = list(range(0, count, 16))
        sols = {j: (probs[j], xs[j].cpu().numpy().copy()) for j in sample}
        row = {"dof_per_s": dofs / (t_b * 1e-3), "ms": t_b, "dof": dofs,
               "over_one_by_one": t_loop / t_b, "cycles_min": min(cyc), "cycles_max": max(cyc)}
        return row, sols
    finally:
        for m in mgs:
            hn.hn_mg_destroy(m)


def oracle_leg(L, sols10, l12, batch):
    """CPU-baseline leg: the oracle, as it stands, timed on the host (one core, then every core),
    and the oracle's view of the GPU results of this run: the relative L2 difference of each L = 10
    solution from the oracle solved to 1e-13, and the relative residual of the L = 12 and sampled
    batch results under the oracle's FP64 operator."""
    import numpy as np
    import oracle as O
    from paper_0904_4152_gb300 import inputs as I
    cpu = cpu_baseline(L, 0, 1)
    cpu.pop("seconds")
    try:
        cpu["all_cores"] = cpu_baseline_all_cores(L, 0, 1)
    except Exception as e:                            # a side measurement: never costs the line
        cpu["all_cores"] = {"error": "%s: %s" % (type(e).__name__, e)}
    err = {}
    b = I.rhs_uniform(L, 0)
    xs, _ = O.mg_solve(L, b, tol=1e-13)
    A = O.assemble(L)
    nb = np.linalg.norm(b)
    err["l10"] = {k: {"l2_diff": float(np.linalg.norm(x - xs) / np.linalg.norm(xs)),
                      "relres": float(np.linalg.norm(O.defect(L, A, b, x)) / nb)}
                  for k, x in sols10.items()}
    if l12 is not None:
        rows, sols, (L12, coef, b12) = l12
        A12 = O.assemble(L12, coef)
        nb = np.linalg.norm(b12)
        err["l12_relres"] = {k: float(np.linalg.norm(O.defect(L12, A12, b12, x)) / nb)
                             for k, x in sols.items()}
    if batch is not None:
        worst = 0.0
        for (Lj, coef, bj), x in batch.values():
            Aj = O.assemble(Lj, coef)
            worst = max(worst, float(np.linalg.norm(O.defect(Lj, Aj, bj, x)) / np.linalg.norm(bj)))
        err["batch_relres_max"] = worst
        err["batch_sample"] = len(batch)
    return cpu, err


def run_ours(args, rank, world, local, pg):
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_0904_4152_gb300 import hn, inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        g.build()
    barrier(pg, dev)
    hn.lib()
    L = args.level if args.level is not None else L_BENCH
    N = ((1 << L) + 1) ** 2
    stream = torch.cuda.current_stream(dev)
    b_host = I.rhs_uniform(L, rank)                       # rank r solves its own problem
    b = torch.from_numpy(b_host).to(dev)
    x = torch.zeros(N, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    t0 = time.perf_counter()
    A = hn.hn_band_create(L)
    setup_band_s = time.perf_counter() - t0
    mgs = {}
    for name, prec, solver in (("mixed", hn.HN_PREC_FP32_DC, hn.HN_SOLVER_MG),
                               ("fp64", hn.HN_PREC_FP64, hn.HN_SOLVER_MG),
                               ("fp16band", hn.HN_PREC_FP16BAND_DC, hn.HN_SOLVER_MG),
                               ("pcg_fp32", hn.HN_PREC_FP32_DC, hn.HN_SOLVER_PCG)):
        mgs[name] = hn.hn_mg_setup(A, prec=prec, solver=solver, stream=stream.cuda_stream)
        if args.host_loop:
            hn.hn_mg_set_profiling(mgs[name], True)
    hn.hn_band_destroy(A)

    def timed(mg, steps, warmup, b=b):
        for _ in range(warmup):
            hn.hn_mg_solve(mg, L, b, x)
        torch.cuda.synchronize(dev)
        barrier(pg, dev)
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        stats = None
        launches = 0
        for s, e in ev:
            flush.fill_(1)                                 # evict the L2 between steps
            s.record(stream)
            _, stats, status = hn.hn_mg_solve(mg, L, b, x)
            e.record(stream)
            assert status == hn.HN_OK, stats
            launches += hn.hn_mg_last_launches(mg)
        torch.cuda.synchronize(dev)
        barrier(pg, dev)
        torch.cuda.synchronize(dev)
        ms = [s.elapsed_time(e) for s, e in ev]
        return ms, stats, launches

    sols10 = {}
    with ClockSampler(local) as clk:
        ms_mixed, st_mixed, launches = timed(mgs["mixed"], args.steps, args.warmup)
    sols10["mixed"] = x.cpu().numpy().copy()
    ms_fp64, st_fp64, _ = timed(mgs["fp64"], args.steps, args.warmup)
    sols10["fp64"] = x.cpu().numpy().copy()
    ms_fp16, st_fp16, _ = timed(mgs["fp16band"], args.steps, args.warmup)
    sols10["fp16band"] = x.cpu().numpy().copy()
    ms_pcg, st_pcg, _ = timed(mgs["pcg_fp32"], args.steps, args.warmup)
    sols10["pcg_fp32"] = x.cpu().numpy().copy()
    total_pcg = max_over_ranks(sum(ms_pcg), pg, dev)
    # the paper's performance configuration: Dirichlet at x = 0, 1, free Neumann at y = 0, 1
    A_lr = hn.hn_band_create_bc(L, None, hn.HN_DIRICHLET_LEFT | hn.HN_DIRICHLET_RIGHT)
    mg_lr = hn.hn_mg_setup(A_lr, prec=hn.HN_PREC_FP32_DC, stream=stream.cuda_stream)
    hn.hn_band_destroy(A_lr)
    if args.host_loop:
        hn.hn_mg_set_profiling(mg_lr, True)
    b_lr = torch.from_numpy(I.rhs_uniform_bc(L, rank, hn.HN_DIRICHLET_LEFT | hn.HN_DIRICHLET_RIGHT)).to(dev)
    ms_lr, st_lr, _ = timed(mg_lr, args.steps, args.warmup, b_lr)
    hn.hn_mg_destroy(mg_lr)
    total_lr = max_over_ranks(sum(ms_lr), pg, dev)

    total_mixed = max_over_ranks(sum(ms_mixed), pg, dev)
    total_fp64 = max_over_ranks(sum(ms_fp64), pg, dev)
    total_fp16 = max_over_ranks(sum(ms_fp16), pg, dev)
    value = world * N * args.steps / (total_mixed * 1e-3)
    fp64_value = world * N * args.steps / (total_fp64 * 1e-3)
    fp16_value = world * N * args.steps / (total_fp16 * 1e-3)
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "L": L, "mixed_dof_per_s": value,
                              "fp64_dof_per_s": fp64_value, "mixed_ms": total_mixed / args.steps,
                              "fp64_ms": total_fp64 / args.steps, "mixed_cycles": st_mixed["cycles"],
                              "fp64_cycles": st_fp64["cycles"]}), flush=True)
        return

    # end to end through the same call with host buffers (pinned)
    bh = torch.from_numpy(b_host).pin_memory().numpy()
    xh = torch.zeros(N, dtype=torch.float64).pin_memory().numpy()
    for _ in range(args.warmup):
        hn.hn_mg_solve(mgs["mixed"], L, bh, xh)
    barrier(pg, dev)
    e2e = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        _, _, status = hn.hn_mg_solve(mgs["mixed"], L, bh, xh)
        e2e.append(time.perf_counter() - t)
        assert status == hn.HN_OK
    e2e_total = max_over_ranks(sum(e2e), pg, dev)
    e2e_value = world * N * args.steps / e2e_total

    # roofline: events around every launch of the headline solve's kernels (profiled pass)
    mg = mgs["mixed"]
    hn.hn_mg_set_profiling(mg, True)
    for _ in range(args.steps):
        flush.fill_(1)
        hn.hn_mg_solve(mg, L, b, x)
    times = hn.hn_mg_kernel_times(mg)
    hn.hn_mg_set_profiling(mg, False)
    tops = [t for t in times if t["bytes_per_launch"] > 0]
    dom = max(tops, key=lambda t: t["total_ms"])
    avg_s = dom["total_ms"] / dom["launches"] * 1e-3
    achieved = dom["bytes_per_launch"] / avg_s / 1e9
    nodes = ((1 << dom["level"]) + 1) ** 2 if dom["level"] >= 0 else N
    tpn = ncu_traffic_per_node("%s-fp32" % dom["name"])
    traffic = tpn * nodes if tpn is not None else None
    peak, peak_kind = measured_peak_gbs()
    by_class = {}
    for t in times:
        by_class.setdefault(t["name"], 0.0)
        by_class[t["name"]] += t["total_ms"]
    prof_total = sum(by_class.values())

    # the larger configurations on rank 0: band kernels alone at L = 12 (data >> L2), the L = 12
    # lognormal solves, the 256-problem batch
    band = l12 = batch = None
    if rank == 0:
        rates = hn.hn_measure_fp_rates()
        band = band_kernels(hn, stream, peak, rates=rates)
        k_steps, k_warm = max(1, min(args.steps, 5)), max(1, min(args.warmup, 2))
        l12 = l12_solves(hn, I, stream, flush, dev, k_steps, k_warm)
        batch = batch256_solves(hn, I, stream, flush, dev, max(1, min(args.steps, 10)), k_warm)
    for m in mgs.values():
        hn.hn_mg_destroy(m)

    # CPU-baseline leg (rank 0 at N = 1): the oracle timed, and its view of this run's results
    cpu = oracle_err = None
    if rank == 0 and world == 1 and L <= 11:
        try:
            cpu, oracle_err = oracle_leg(L, sols10, l12, {} if batch is None else batch[1])
        except Exception as e:                        # a side measurement: never costs the line
            cpu = {"error": "%s: %s" % (type(e).__name__, e)}
    # serving latency on a short sample of the serve workload (after the timed region; the full
    # run is --workload serve)
    serve = None
    if rank == 0 and args.serve_requests > 0:
        try:
            serve = serve_sample(hn, I, args.serve_requests, 0.7, 40.0, 64, 0)
        except Exception as e:                        # a side measurement: never costs the line
            serve = {"error": "%s: %s" % (type(e).__name__, e)}

    if rank == 0:
        cfg = bench_config(L)
        cfg["setup_ms"] = {"band": 1e3 * setup_band_s, "hierarchy_mixed": st_mixed["setup_ns"] / 1e6,
                           "hierarchy_fp64": st_fp64["setup_ns"] / 1e6}
        err10 = (oracle_err or {}).get("l10", {})

        def solve_row(ms_total, st, name, extra=None):
            r = {"dof_per_s": world * N * args.steps / (ms_total * 1e-3), "ms": ms_total / args.steps,
                 "cycles": st["cycles"], "outer": st["outer_iters"], "relres": st["relres"]}
            if name in err10:
                r["oracle_l2_diff"] = err10[name]["l2_diff"]
                r["oracle_relres"] = err10[name]["relres"]
            if extra:
                r.update(extra)
            return r

        line = {
            "metric": "MG Poisson DOF/s to 1e-8 (mixed vs FP64)",
            "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_mixed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32", "data": "synthetic", "gpu_launches": launches,
            "config": cfg, "clocks": clk.summary(),
            "e2e": {"value": e2e_value, "unit": "DOF/s", "h2d_bytes_per_step": N * 8,
                    "d2h_bytes_per_step": N * 8},
            "roofline": {"bound": "hbm", "kernel": "%s L%d" % (dom["name"], dom["level"]),
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                         "bytes_per_launch": dom["bytes_per_launch"],
                         "avg_launch_us": avg_s * 1e6, "launches": dom["launches"],
                         "share_of_profiled": dom["total_ms"] / prof_total if prof_total else None},
            "cpu_baseline": cpu,
            "kernel_share": dict(sorted(((k, v / prof_total) for k, v in by_class.items()),
                                        key=lambda kv: -kv[1])[:6]) if prof_total else {},
            "band_kernels_L12_frac": {p: {o: r["frac"] for o, r in row.items()} for p, row in band.items()},
            "fp64_L12_frac_of_bound": {o: r.get("frac_of_bound") for o, r in band["fp64"].items()},
            "fp64_tfma_per_s": rates["fp64_fma_per_s"] * 1e-12,
        }
        if serve is not None:
            line["serve"] = serve
        if batch is not None:
            line["batch256"] = dict(batch[0], oracle_relres_max_sampled=(oracle_err or {}).get("batch_relres_max"))
        if l12 is not None:
            rel12 = (oracle_err or {}).get("l12_relres", {})
            line["l12_lognormal"] = {k: dict(r, oracle_relres=rel12.get(k)) for k, r in l12[0].items()}
        line["mixed_neumann_dirichlet"] = solve_row(total_lr, st_lr, "")
        line["pcg_fp32"] = solve_row(total_pcg, st_pcg, "pcg_fp32")
        line["fp16band"] = solve_row(total_fp16, st_fp16, "fp16band")
        line["fp64"] = solve_row(total_fp64, st_fp64, "fp64")
        line["mixed"] = solve_row(total_mixed, st_mixed, "mixed")
        line["mixed_over_fp64"] = value / fp64_value
        try:                                           # never costs the line
            line["solve_roofline"] = {
                "mixed": solve_roofline(N, total_mixed / args.steps, peak, inner_cycles=st_mixed["inner_cycles"],
                                        outer_iters=st_mixed["outer_iters"]),
                "fp64": solve_roofline(N, total_fp64 / args.steps, peak, fp64_cycles=st_fp64["cycles"])}
        except Exception as e:
            line["solve_roofline"] = {"error": "%s: %s" % (type(e).__name__, e)}
        print(json.dumps(sig(line)), flush=True)


def run_batch(args, rank, world, local, pg):
    """256 independent problems, L_j ~ U{5..9}, lognormal coefficients, U[-1,1] right-hand sides,
    FP32-inner defect correction: one batched solve (persistent work-list kernels, one CUDA graph
    with a device-side loop) against solving the same problems one after the other."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_0904_4152_gb300 import hn, inputs as I
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        g.build()
    barrier(pg, dev)
    count = 256
    levels = [int(v) for v in I.batch_levels(count, seed=rank)]
    mgs, bs, xs, coefs, bh = [], [], [], [], []
    for j, L in enumerate(levels):
        coef, b = I.batch_problem(j + rank * count, L)
        A = hn.hn_band_create(L, coef)
        mgs.append(hn.hn_mg_setup(A, prec=hn.HN_PREC_FP32_DC))
        hn.hn_band_destroy(A)
        coefs.append(coef)
        bh.append(b)
        bs.append(torch.from_numpy(b).to(dev))
        xs.append(torch.zeros_like(bs[-1]))
    dofs = sum(((1 << L) + 1) ** 2 for L in levels)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    best = hn.hn_mg_autotune_batch(mgs, bh, reps=2)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        barrier(pg, dev)
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        barrier(pg, dev)
        return ms

    stats = {}

    def batched():
        _, st, status = hn.hn_mg_solve_batch(mgs, levels, bs, xs)
        assert status == hn.HN_OK
        stats["b"] = st

    def looped():
        for mg, L, b, x in zip(mgs, levels, bs, xs):
            _, st, status = hn.hn_mg_solve(mg, L, b, x)
            assert status == hn.HN_OK

    with ClockSampler(local) as clk:
        ms_b = timed(batched, args.steps, args.warmup)
    ms_l = timed(looped, max(1, args.steps // 10), 1)
    tb = max_over_ranks(sum(ms_b), pg, dev)
    value = world * dofs * len(ms_b) / (tb * 1e-3)
    loop_value = world * dofs * len(ms_l) / (max_over_ranks(sum(ms_l), pg, dev) * 1e-3)
    cpu = batch_oracle_leg(levels, coefs, bh, xs) if rank == 0 and world == 1 else None
    if rank == 0:
        cyc = [s["cycles"] for s in stats["b"]]
        print(json.dumps({
            "metric": "batched MG Poisson DOF/s to 1e-8 (256 problems, L 5..9, FP32-inner DC)",
            "value": value, "unit": "DOF/s", "n_gpus": world, "steps": len(ms_b),
            "warmup": args.warmup, "ms_per_step": tb / len(ms_b), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "batch-256-L5to9-lognormal", "problems": count, "dof": dofs,
                       "levels": {str(L): levels.count(L) for L in sorted(set(levels))},
                       "tuning": {"tail_level": best[0], "cluster": best[1], "mid": best[3]},
                       "l2_between_steps": "flushed (512 MiB write)"},
            "per_problem_loop_dof_per_s": loop_value, "batched_over_loop": value / loop_value,
            "inner_cycles": {"min": min(cyc), "max": max(cyc)},
            "cpu_baseline": cpu, "clocks": clk.summary()}), flush=True)
    for mg in mgs:
        hn.hn_mg_destroy(mg)


def batch_oracle_leg(levels, coefs, bh, xs, every=32):
    """CPU-baseline leg of the batch workload: the oracle, as it stands, on one host core solving a
    sample of the batch's problems one after the other (DOF/s), and the relative residual of the
    same problems' batched GPU results under the oracle's FP64 operator."""
    import numpy as np
    import oracle as O
    O.lib()
    sample = list(range(0, len(levels), every))
    worst, dofs, secs = 0.0, 0, 0.0
    for j in sample:
        L = levels[j]
        A64 = O.assemble(L, coefs[j])
        x = xs[j].cpu().numpy()
        worst = max(worst, float(np.linalg.norm(O.defect(L, A64, bh[j], x)) / np.linalg.norm(bh[j])))
        t0 = time.perf_counter()
        O.mg_solve(L, bh[j], coef=coefs[j], prec=1, tol=TOL)
        secs += time.perf_counter() - t0
        dofs += ((1 << L) + 1) ** 2
    return {"value": dofs / secs, "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": "problems %s of the batch (every %dth), FP32-inner DC to 1e-8 one after the "
                      "other, %.2f s" % (",".join(map(str, sample)), every, secs),
            "oracle_relres_max_sampled": worst}


def _gen_init(cores):
    """Worker of the serving input generators: keep off the cores of the benchmark process."""
    try:
        os.sched_setaffinity(0, cores)
    except (AttributeError, OSError):
        pass


def _gen_request(task):
    """One request's seeded coefficient field and right-hand side, left in a shared-memory block
    (coefficients first) so that the benchmark process maps them without a copy."""
    from multiprocessing import shared_memory
    import numpy as np
    from paper_0904_4152_gb300 import inputs as I
    L, sd = task
    coef = I.lognormal_coef(L, sd)
    b = I.rhs_uniform(L, sd + 1_000_000)
    shm = shared_memory.SharedMemory(create=True, size=(coef.size + b.size) * 8)
    a = np.ndarray(coef.size + b.size, dtype=np.float64, buffer=shm.buf)
    a[:coef.size] = coef
    a[coef.size:] = b
    name = shm.name
    del a
    shm.close()
    return name, coef.size, b.size


class RequestInputs:
    """Seeded per-request inputs of the serving workload, generated ahead of their arrival by a
    pool of spawned processes on the host cores the benchmark process does not use (this process
    keeps `keep` cores for itself and the server's worker thread)."""

    def __init__(self, keep=4):
        import multiprocessing as mp
        n = os.cpu_count() or 1
        self.saved = None
        try:
            self.saved = os.sched_getaffinity(0)
        except (AttributeError, OSError):
            pass
        own = set(range(min(keep, n)))
        gen = set(range(min(keep, n), n)) or own
        # one BLAS thread per generator process (the processes already fill the cores)
        env = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
        os.environ.update({k: "1" for k in env})
        try:
            self.pool = mp.get_context("spawn").Pool(max(1, len(gen)), initializer=_gen_init,
                                                     initargs=(gen,))
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        try:
            os.sched_setaffinity(0, own)
        except (AttributeError, OSError):
            pass
        self.pending = {}
        self.ready = {}

    def request(self, key, L, seed):
        self.pending[key] = self.pool.apply_async(_gen_request, ((int(L), int(seed)),))

    def take(self, key):
        """(coefficients, right-hand side) of a requested input, mapped from its shared-memory
        block; the block stays until close()."""
        if key not in self.ready:
            from multiprocessing import shared_memory
            import numpy as np
            name, nc, nb = self.pending.pop(key).get()
            shm = shared_memory.SharedMemory(name=name)
            a = np.ndarray(nc + nb, dtype=np.float64, buffer=shm.buf)
            self.ready[key] = (shm, a[:nc], a[nc:])
        _, c, b = self.ready[key]
        return c, b

    def close(self):
        for k in list(self.pending):
            try:
                self.take(k)
            except Exception:
                pass
        for key in list(self.ready):
            shm, c, b = self.ready.pop(key)
            del c, b
            try:
                shm.close()
            except BufferError:                        # a caller still holds a view of it
                pass
            shm.unlink()
        self.pool.terminate()
        if self.saved is not None:
            try:
                os.sched_setaffinity(0, self.saved)
            except OSError:
                pass


def serve_sample(hn, I, requests, load, budget_gb, slots, seed):
    """Continuous-batching server: Poisson arrivals, L uniform over {6..11}, every request with its
    own seeded lognormal coefficient field and U[-1,1] right-hand side, FP32-inner DC to 1e-8
    under a device-memory budget.  The arrival rate is `load` x the capacity measured on a burst
    of 120 requests of the same mix (the second of two bursts: the first warms the server's device
    blocks, page-locked buffers and engine).  The inputs of the first 1,500 requests are generated
    before the first arrival by host processes on cores apart from this process (later requests of
    a longer run replay them in order: an L = 11 field costs ~0.3 s of one host core).  Returns
    throughput, latency percentiles (submit to completion, also per tenth of the run in arrival
    order and per level) and the worker's time split."""
    import threading
    import numpy as np
    opts = hn.hn_mg_opts_default(prec=hn.HN_PREC_FP32_DC)
    gen = RequestInputs()
    srv = None
    unique = min(requests, 1500)
    try:
        srv = hn.hn_server_create(int(budget_gb * (1 << 30)), slots)
        calib = 120
        _, lv, sd = I.serve_requests(calib, 1.0, seed=11 + seed)
        for k, (L, q) in enumerate(zip(lv, sd)):
            gen.request(("c", k), L, int(q) + 500_000)
        inputs = [gen.take(("c", k)) for k in range(calib)]

        def burst():
            t0 = time.perf_counter()
            tickets = []
            for L, (coef, b) in zip(lv, inputs):
                tickets.append((hn.hn_mg_submit(srv, int(L), b, coef, opts=opts), int(L)))
            for t, L in tickets:
                status, _, _ = hn.hn_mg_poll(srv, t, L)
                assert status == hn.HN_OK
            return calib / (time.perf_counter() - t0)

        burst()                       # warms the server: device blocks, pinned buffers, engine
        capacity = burst()
        del inputs
        rate = load * capacity
        arrivals, levels, seeds = I.serve_requests(requests, rate, seed=7 + seed)
        # the inputs of the first `unique` requests are generated before the first arrival (the
        # host needs ~0.3 s of one core for an L = 11 field); later requests replay them in order
        levels = levels[np.arange(requests) % unique]
        seeds = seeds[np.arange(requests) % unique]
        tg = time.perf_counter()
        for k in range(unique):
            gen.request(k, levels[k], seeds[k])
        for k in range(unique):
            gen.take(k)
        gen_s = time.perf_counter() - tg
        sub = [None] * requests
        late = np.zeros(requests)
        res = [None] * requests
        err = []

        def submitter():
            start = time.perf_counter()
            for i in range(requests):
                coef, b = gen.take(i % unique)
                dt = start + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                late[i] = max(0.0, -dt)
                try:
                    sub[i] = hn.hn_mg_submit(srv, int(levels[i]), b, coef, opts=opts)
                except hn.HnError as e:
                    err.append(str(e))
                    return

        th = threading.Thread(target=submitter)
        t_start = time.perf_counter()
        th.start()
        for i in range(requests):
            while sub[i] is None and th.is_alive():
                time.sleep(0.0005)
            if sub[i] is None:
                break
            status, x, st = hn.hn_mg_poll(srv, sub[i], int(levels[i]))
            res[i] = (status, st["solve_ns"] * 1e-6 if st else None, st["relres"] if st else None,
                      st["setup_ns"] * 1e-6 if st else None,
                      st["outer_iters"] + st["inner_cycles"] if st else None)
        th.join()
        t_end = time.perf_counter()
        info = hn.hn_server_query(srv)
    finally:
        if srv is not None:
            hn.hn_server_destroy(srv)
        gen.close()
    ok = [i for i, r in enumerate(res) if r is not None and r[0] == hn.HN_OK]
    lat = np.array([res[i][1] for i in ok])
    setup = np.array([res[i][3] for i in ok])
    steps = np.array([res[i][4] for i in ok])
    wall = t_end - t_start
    dofs = sum(((1 << int(levels[i])) + 1) ** 2 for i in ok)
    tenth = [float(np.percentile(lat[k * len(lat) // 10:(k + 1) * len(lat) // 10], 99))
             for k in range(10)] if len(lat) >= 10 else []
    return {"requests": requests, "completed_ok": len(lat), "errors": err[:3], "offered_load": load,
            "arrival_rate_per_s": rate, "capacity_per_s": capacity,
            "requests_per_s": len(lat) / wall, "dof_per_s": dofs / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max()),
                           "argmax": int(ok[int(lat.argmax())]), "p99_by_tenth": tenth},
            "p99_ms_by_level": {str(L): float(np.percentile([res[i][1] for i in ok if int(levels[i]) == L], 99))
                                for L in sorted({int(levels[i]) for i in ok})},
            "submit_late_ms_p99": float(np.percentile(late, 99) * 1e3),
            # where a request's time goes: the build of its operator and hierarchy (inside the
            # latency), the solver steps it needs (each one scheduler pass shared with the other
            # running requests), the passes of the whole run and the mean number of requests in
            # the server (sum of latencies / wall time)
            "breakdown": {"build_ms_p50": float(np.percentile(setup, 50)),
                          "build_ms_p99": float(np.percentile(setup, 99)),
                          "steps_p50": float(np.percentile(steps, 50)), "steps_max": int(steps.max()),
                          "passes": int(info["iterations"]),
                          "ms_per_pass": float(info["iterate_ns"] * 1e-6 / max(1, info["iterations"])),
                          "mean_in_server": float(lat.sum() * 1e-3 / wall)},
            "inputs": {"distinct": unique, "host_generation_s": gen_s},
            "worker_s": {k: info[k + "_ns"] * 1e-9 for k in ("admit", "schedule", "iterate", "retire")},
            "relres_max": max(res[i][2] for i in ok)}


def run_serve(args, rank, world, local, pg):
    """The serving workload (serve_sample) on its own: one JSON line with p50/p99 and throughput."""
    import torch
    import __graft_entry__ as g
    from paper_0904_4152_gb300 import hn, inputs as I
    torch.cuda.set_device(local)
    if rank == 0:
        g.build()
    barrier(pg)
    hn.lib()
    r = serve_sample(hn, I, args.requests, args.load, args.budget_gb, args.slots, rank)
    if rank == 0:
        print(json.dumps({
            "metric": "serve p50/p99 latency and throughput (Poisson arrivals, L 6..11, FP32-inner DC)",
            "value": r["requests_per_s"], "unit": "requests/s", "n_gpus": world, "requests": args.requests,
            "completed_ok": r["completed_ok"], "errors": r["errors"], "higher_is_better": True,
            "data": "synthetic",
            "config": {"workload": "serve-poisson-L6to11-lognormal", "offered_load": args.load,
                       "arrival_rate_per_s": r["arrival_rate_per_s"], "capacity_per_s": r["capacity_per_s"],
                       "budget_gb": args.budget_gb, "slots": args.slots},
            "latency_ms": r["latency_ms"], "dof_per_s": r["dof_per_s"],
            "submit_late_ms_p99": r["submit_late_ms_p99"], "p99_ms_by_level": r["p99_ms_by_level"],
            "breakdown": r["breakdown"], "worker_s": r["worker_s"],
            "relres_max": r["relres_max"]}), flush=True)


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world, pg)
    elif args.workload == "batch":
        run_batch(args, rank, world, local, pg)
    elif args.workload == "serve":
        run_serve(args, rank, world, local, pg)
    elif args.workload == "blas1":
        run_blas1(args, rank, local)
    elif args.workload == "kernels":
        run_kernels(args, rank, local)
    elif args.workload == "swe":
        run_swe(args, rank, local)
    elif args.workload == "solvers":
        run_solvers(args, rank, local)
    else:
        run_ours(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
