"""Benchmark: SA-AMG hierarchy setup + PCG solve to 1e-8 relative residual on one GB300.

Workload (default): Q1 finite-element diffusion on the unit cube with 128^3 interior nodes
(2,097,152 unknowns, 55,742,968 stored entries), per-element coefficient 10^U(-3,3) (SplitMix64
seed 2), strength threshold 0.02 with 1Norm + OffLmp, right-hand side uniform in [-1, 1)
(seed 2); one step = amg_setup + amg_solve (+ amg_free) in FP64, with the mixed form (FP32
hierarchy values and V-cycle inside FP64 PCG) timed the same way beside it.  Synthetic inputs
stand in for the paper's coefficient-jump problems (SPE10 is not available).  Other workloads:
stretched64 (64^3 box, z spacing x1.1 per layer, five methods per step), laplace20.

Prints one JSON line (rank 0): solves/s over the timed steps (inputs resident in HBM) with the
setup and solve milliseconds per solve, the end-to-end number through the C ABI with host
buffers, the roofline of the dominant kernel class (taken from a separate profiled pass),
the oracle timed on the host cores (one whole solve at full size, in a process of its own)
and each result's error against the oracle's solution, the SM clocks sampled during the
timed region, and the side lines (batched, served, several right-hand sides, GMRES,
systems, the 16-combination study).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload randcoef128|stretched64|laplace20] [--precision fp64|mixed]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SA-AMG setup+PCG solve s to 1e-8 rel-res, FP64 vs mixed; solves/s; p99 latency"
TOL = 1e-8
VARIANT_SETS = {
    "stretched64": [("traditional", 0), ("1norm", 1), ("offlmp", 2), ("sprsfy", 4), ("cnstrnt", 8)],
    "randcoef128": [("1norm+offlmp", 3)],
    "laplace20": [("traditional", 0)],
    "elasticity40": [("traditional", 0)],     # --once only (the systems line times it otherwise)
    "convdiff64": [("1norm+offlmp", 3)],      # --once only (the GMRES line times it otherwise)
}
L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def make_workload(name: str):
    from paper_2103_10476_gb300 import problems as P
    if name == "stretched64":
        A, b, cfg = P.workload_stretched64()
        theta = 0.02
    elif name == "randcoef128":
        A, b, cfg = P.workload_randcoef128()
        theta = 0.02
    elif name == "laplace20":
        A, b, cfg = P.workload_laplace20()
        theta = 0.0
    elif name == "elasticity40":
        A, b, cfg = P.workload_elasticity()
        theta = cfg["theta"]
    elif name == "convdiff64":
        A, b, cfg = P.workload_convdiff64()
        theta = cfg["theta"]
        A.meta["krylov"] = (cfg["krylov"], cfg["restart"])
    else:
        raise SystemExit(f"unknown workload {name}")
    return A, b, theta


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1000.0)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], parts[3]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for nm, flag in zip(names, r[2]):
                if flag.lower() in ("active", "1", "yes"):
                    seen.add(nm)
        sm = sorted(r[0] for r in rows)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows), "reasons": sorted(seen),
                "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# the sources each timed kernel class is compiled from (its kernels, launch code and headers)
KERNEL_SOURCES = {
    # api.cu chooses the fine level's layout (CSR tiles or the sliced-ELL copy), hence which
    # kernel the class runs
    "vcycle_fine_spmv": ("solve.cu", "tma.cuh", "api.cu"),
    "pcg_spmv_fp64": ("solve.cu", "tma.cuh", "api.cu"),
    "galerkin_spgemm": ("spgemm.cu",),
}


def kernel_source_hash(kclass_name: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_10476_gb300", "csrc")
    for f in KERNEL_SOURCES[kclass_name]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kclass_name: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(workload, {}).get(kclass_name)
        if e and e.get("source_hash") == kernel_source_hash(kclass_name):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# ------------------------------------------------------------------------------ CPU baseline / reference arm

# workloads whose CPU baseline is one whole oracle solve at full size (minutes of CPU time),
# run in a spawned process beside the GPU work; its solution also gives each result's error
ORACLE_FULL = ("randcoef128",)


def _oracle_full_child(workload: str, out_prefix: str):
    """Spawned process: the oracle's setup + solve of the full workload (first method)."""
    import numpy as np
    import oracle
    oracle.build()
    A, b, theta = make_workload(workload)
    name, v = VARIANT_SETS[workload][0]
    t0 = time.perf_counter()
    h, st = oracle.setup(A, theta=theta, variants=v)
    t1 = time.perf_counter()
    res = {"status": int(st), "method": name, "setup_s": t1 - t0}
    if h is not None:
        x, info, st2 = h.solve(b, TOL)
        res.update(solve_s=time.perf_counter() - t1, iters=int(info.iters), status=int(st2),
                   relres=float(info.relres_true), levels=int(info.levels))
        np.save(out_prefix + ".npy", x)
    with open(out_prefix + ".json", "w") as f:
        json.dump(res, f)


class OracleFullRun:
    """The oracle's whole solve of a workload in a spawned process (a fresh interpreter, so
    it is safe to start after the GPU is in use)."""

    def __init__(self, workload: str):
        import multiprocessing as mp
        self.dir = tempfile.mkdtemp(prefix="oracle_full_")
        self.prefix = os.path.join(self.dir, "run")
        self.proc = mp.get_context("spawn").Process(target=_oracle_full_child, args=(workload, self.prefix),
                                                    daemon=True)
        self.proc.start()

    def result(self, timeout_s: float = 1800.0):
        import numpy as np
        self.proc.join(timeout_s)
        if self.proc.is_alive():
            self.proc.terminate()
            return {"status": -1, "error": "oracle run exceeded its time limit"}
        try:
            res = json.load(open(self.prefix + ".json"))
        except Exception as e:      # the child failed before writing its result
            return {"status": -1, "error": f"no result ({e}); exit code {self.proc.exitcode}"}
        if os.path.exists(self.prefix + ".npy"):
            res["x"] = np.load(self.prefix + ".npy")
        return res


# the reference arm's bounded sample of the 128^3 workload: whole oracle solves of a smaller
# cube of the same family (iid coefficients 10^U(-3,3), theta 0.02, 1Norm+OffLmp), each timed
# and scaled to the full cube by the ratio of stored entries
SAMPLE_EDGE = {"randcoef128": 48}

def oracle_sample(A, b, theta, variants, budget_s: float):
    """Times the oracle (as it stands) on whole setup+solve runs of the workload's methods,
    cycling through them until about budget_s seconds have passed.  Returns (solves, seconds,
    description)."""
    import oracle
    oracle.build()
    done = 0
    t0 = time.perf_counter()
    names = []
    k = 0
    while True:
        name, v = variants[k % len(variants)]
        h, st = oracle.setup(A, theta=theta, variants=v)
        if h is not None:
            h.solve(b, TOL)
            del h
        done += 1
        names.append(name)
        k += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (el / done) * (done + 1) > 2.5 * budget_s:
            break
    return done, time.perf_counter() - t0, names


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    if args.workload in SAMPLE_EDGE:
        return run_reference_scaled(args)
    A, b, theta = make_workload(args.workload)
    variants = VARIANT_SETS[args.workload]
    # the oracle keeps no state between runs, so warm-up steps are not run (bounds the wall time)
    budget = float(os.environ.get("REF_STEP_BUDGET_S", "4"))
    solves = 0
    secs = 0.0
    per = []
    for k in range(args.steps):
        n, s, names = oracle_sample(A, b, theta, variants[k % len(variants):] + variants[:k % len(variants)], budget)
        solves += n
        secs += s
        per.append(s / n)
    value = solves / secs
    cores = 1
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{solves} oracle setup+solve runs of the workload's methods, "
                                   f"each step about {budget:.0f} s, single thread, host has {os.cpu_count()} cores"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "p50_ms": 1000 * statistics.median(per), "p99_ms": 1000 * max(per),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_scaled(args):
    """Reference arm for a workload whose single solve takes the oracle minutes: every step is
    one whole oracle setup + solve of a smaller cube of the same family, and its time is
    scaled to the full workload by the ratio of stored entries (AMG setup and each PCG
    iteration are linear in them; the iteration count of the sample is reported beside)."""
    import oracle
    from paper_2103_10476_gb300 import problems as P
    oracle.build()
    edge = int(os.environ.get("REF_SAMPLE_EDGE", SAMPLE_EDGE[args.workload]))
    As = P.random_coefficient_cube(edge, 2, 3.0)
    bs = P.rhs_uniform(As.n, 2)
    full_nnz = (3 * 128 - 2) ** 3
    scale = full_nnz / As.nnz
    name, v = VARIANT_SETS[args.workload][0]
    per, iters = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        h, st = oracle.setup(As, theta=0.02, variants=v)
        if h is not None:
            _, info, _ = h.solve(bs, TOL)
            iters = info.iters
            del h
        per.append((time.perf_counter() - t0) * scale)
    secs = sum(per)
    value = args.steps / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step one whole oracle setup + solve ({name}) of a {edge}^3 cube of the same "
                                   f"family ({As.n} unknowns, {As.nnz} entries, {iters} PCG iterations), its time "
                                   f"scaled by {scale:.2f} (the full cube's entries over the sample's); single "
                                   f"thread, host has {os.cpu_count()} cores; warm-up steps not run (no state)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "p50_ms": 1000 * statistics.median(per), "p99_ms": 1000 * max(per),
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args):
    desc = {
        "stretched64": "Q1 FE Laplacian, 64^3 interior nodes, z spacing x1.1 per layer, theta=0.02; "
                       "5 methods (traditional, 1Norm, OffLmp, Sprsfy, Cnstrnt) per step",
        "randcoef128": "Q1 FE diffusion, 128^3 interior nodes, coefficient 10^U(-3,3), theta=0.02, 1Norm+OffLmp",
        "laplace20": "Q1 FE Laplacian, 20^3 interior nodes, theta=0",
        "elasticity40": "3D elasticity, 40^3 hexahedra, 3 unknowns per node, 6 rigid-body modes, theta=0.02",
        "convdiff64": "convection-diffusion 64^3, theta=0.02, 1Norm+OffLmp, GMRES(30)",
    }[args.workload]
    return {"workload": args.workload, "description": desc, "precision": args.precision, "tol": TOL,
            "rhs": "uniform[-1,1) SplitMix64", "inputs": "matrix and right-hand side resident in HBM",
            "l2": "flushed (256 MiB write) before every timed step",
            "parallelism": f"replicas x{args.gpus}"}


# ------------------------------------------------------------------------------ our arm

def run_once(args):
    """One setup + solve (or V-cycles) of one method: a bounded number of kernel launches for
    profiler captures (ncu) of the same code path the benchmark times."""
    import numpy as np
    import torch
    from paper_2103_10476_gb300 import amg
    A, b, theta = make_workload(args.workload)
    variants = dict(VARIANT_SETS[args.workload])
    name = args.method or VARIANT_SETS[args.workload][0][0]
    prec = amg.AMG_MIXED if args.precision == "mixed" else amg.AMG_FP64
    lay = {"auto": amg.AMG_LAYOUT_AUTO, "csr": amg.AMG_LAYOUT_CSR, "sell": amg.AMG_LAYOUT_SELL}[args.layout]
    rp = torch.from_numpy(A.row_ptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    v = torch.from_numpy(A.val).cuda()
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    arg = amg.csr_arg(A.n, rp, ci, v)
    phases = None
    if args.trace:
        # a warm-up setup, then one with every phase boundary synchronised and timed
        for trace in (0, 1):
            ht = amg.amg_setup(arg, None, amg.amg_params_default(theta=theta, variants=variants[name],
                                                                 precision=prec, trace=trace, spmv_layout=lay))
            if trace:
                levels = amg.amg_num_levels(ht)
                phases = [{k: round(t, 3) for k, t in amg.amg_setup_trace(ht, l).items() if t > 0}
                          for l in range(levels)]
            amg.amg_free(ht)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ns, block = None, {}
    if "rbm" in A.meta:       # a system: three unknowns per node, the six rigid-body modes
        ns = torch.from_numpy(np.ascontiguousarray(A.meta["rbm"]).reshape(-1)).cuda()
        block = dict(block_size=3, nullspace_dim=6)
    if "krylov" in A.meta:    # a nonsymmetric operator: flexible GMRES
        block = dict(krylov=A.meta["krylov"][0], restart=A.meta["krylov"][1])
    h = amg.amg_setup(arg, ns, amg.amg_params_default(theta=theta, variants=variants[name], precision=prec,
                                                     spmv_layout=lay, **block))
    torch.cuda.synchronize()
    out = {"workload": args.workload, "method": name, "layout": args.layout,
           "setup_ms": 1000 * (time.perf_counter() - t0)}
    if phases is not None:
        out["phases_ms"] = phases
    t0 = time.perf_counter()
    if args.vcycles:
        for _ in range(args.vcycles):
            amg.amg_vcycle(h, bd, xd)
        torch.cuda.synchronize()
        out["vcycles"] = args.vcycles
    else:
        info = amg.amg_solve(h, bd, xd, TOL)
        out.update(iters=info.iters, relres=info.relres_true, levels=info.levels)
    out["run_ms"] = 1000 * (time.perf_counter() - t0)
    out["launches"] = amg.amg_launch_count()
    amg.amg_free(h)
    print(json.dumps(out), flush=True)
    return 0


def pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, int(q * len(v)))] if v else None


def run_batched(args, amg, torch):
    """512 independent systems (edge 8..40 nodes, half stretched, half 10^U(-2,2) coefficients,
    seed 3), one hierarchy each, theta 0.02 with 1Norm + OffLmp; one step = amg_setup_batch of
    all 512 (matrices resident on the device) + the batched PCG solve of all 512 to 1e-8.
    Host wall time between device synchronisations (setup runs on one stream per host
    thread).  Mixed precision (FP32 levels, FP64 PCG) and FP64."""
    from paper_2103_10476_gb300 import problems as P
    t0 = time.perf_counter()
    count = args.batch_count
    systems = P.batched_systems(count, engine="c")
    gen_s = time.perf_counter() - t0
    dev = []
    for A, b in systems:
        dev.append((torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(),
                    torch.from_numpy(A.val).cuda(), torch.from_numpy(b).cuda(),
                    torch.zeros(A.n, dtype=torch.float64, device="cuda")))
    args_d = [amg.csr_arg(A.n, rp, ci, v) for (A, _), (rp, ci, v, _, _) in zip(systems, dev)]
    bs = [d[3] for d in dev]
    xs = [d[4] for d in dev]
    out = {"workload": f"{count} Q1 systems, edge U{{8..40}} nodes, half stretched z ratio U[1.05,1.2], half "
                       "10^U(-2,2) coefficients, seed 3; theta 0.02, 1Norm+OffLmp",
           "rows": sum(A.n for A, _ in systems), "nnz": sum(A.nnz for A, _ in systems), "generate_s": gen_s}
    precs = (("mixed", amg.AMG_MIXED), ("fp64", amg.AMG_FP64))
    if args.batch_precision != "both":
        precs = tuple(q for q in precs if q[0] == args.batch_precision)
    for prec_name, prec in precs:
        p = amg.amg_params_default(theta=0.02, variants=3, precision=prec)
        steps = []
        for k in range(1 + args.batch_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hs = amg.amg_setup_batch(args_d, None, p)
            t1 = time.perf_counter()
            bt = amg.amg_batch_create(hs, tune=True)
            st, infos = amg.amg_batch_solve(bt, bs, xs, TOL)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            gk = amg.amg_batch_info(bt)[3]
            amg.amg_batch_free(bt)
            for h in hs:
                amg.amg_free(h)
            if k > 0:   # the first step is the warm-up (graph capture, lane tuning, pool growth)
                its = [i.iters for i in infos]
                steps.append({"setup_ms": 1e3 * (t1 - t0), "solve_ms": 1e3 * (t2 - t1), "status": st,
                              "iters_mean": sum(its) / len(its), "iters_max": max(its),
                              "relres_max": max(i.relres_true for i in infos), "kernels_per_iteration": gk})
        tot = sum(s_["setup_ms"] + s_["solve_ms"] for s_ in steps)
        out[prec_name] = {"value": count * len(steps) / (tot / 1000.0), "unit": "solves/s",
                          "ms_per_step": tot / len(steps), "steps": len(steps), "per_step": steps}
    if not args.no_plain:
        # the plain FP64 GPU path on the same systems: amg_setup + amg_solve + amg_free one
        # system after another (device-resident matrices), no batching
        p = amg.amg_params_default(theta=0.02, variants=3, precision=amg.AMG_FP64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its = []
        for arg, b_, x_ in zip(args_d, bs, xs):
            h = amg.amg_setup(arg, None, p)
            its.append(amg.amg_solve(h, b_, x_, TOL).iters)
            amg.amg_free(h)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        out["plain_fp64"] = {"value": count / tp, "unit": "solves/s", "ms": 1e3 * tp,
                             "iters_mean": sum(its) / len(its),
                             "how": "amg_setup + amg_solve + amg_free one system at a time, FP64"}
    return out


def run_multi(args, amg, torch):
    """Several right-hand sides of one system: eight right-hand sides of the benchmark's stretched64 system (1Norm) solved
    at once by amg_solve_multi against the same eight solved one after another by amg_solve on
    the same hierarchy; matrix, right-hand sides and solutions resident on the device; solve
    phase only (one setup shared), FP64 and mixed.  Host wall time between device
    synchronisations; L2 flushed before each timed repetition."""
    import numpy as np
    from paper_2103_10476_gb300 import problems as P
    A, b, _ = P.workload_stretched64()
    k = 8
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    B = torch.from_numpy(np.stack([P.rhs_uniform(A.n, 200 + j) for j in range(k)])).cuda()
    X = torch.zeros_like(B)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"workload": f"stretched64, 1Norm, {k} right-hand sides (SplitMix64 seeds 200..207), one hierarchy; "
                       "solve phase only, device-resident", "rhs": k}
    for prec_name, prec in (("fp64", amg.AMG_FP64), ("mixed", amg.AMG_MIXED)):
        p = amg.amg_params_default(theta=0.02, variants=1, precision=prec, cuda_stream=stream.cuda_stream)
        h = amg.amg_setup(amg.csr_arg(A.n, rp, ci, v), None, p)
        amg.amg_solve_multi(h, B, X, TOL)          # warm-up: work vectors, graphs
        for j in range(k):
            amg.amg_solve(h, B[j], X[j], TOL)
        reps = 3
        t_multi = t_single = 0.0
        iters_multi = iters_single = None
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, infos = amg.amg_solve_multi(h, B, X, TOL)
            torch.cuda.synchronize()
            t_multi += time.perf_counter() - t0
            iters_multi = [i.iters for i in infos]
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its = []
            for j in range(k):
                its.append(amg.amg_solve(h, B[j], X[j], TOL).iters)
            torch.cuda.synchronize()
            t_single += time.perf_counter() - t0
            iters_single = its
        amg.amg_free(h)
        out[prec_name] = {"multi_solves_per_s": k * reps / t_multi, "single_solves_per_s": k * reps / t_single,
                          "speedup": t_single / t_multi, "iters_multi": iters_multi, "iters_single": iters_single}
    return out


def run_gmres(args, amg, torch):
    """Nonsymmetric operators: the stand-in for §3's pressure system (convection-diffusion,
    64^3 interior nodes, 6.86M entries) with the symmetrised strength mask, the general
    coarsest inverse and flexible GMRES(30) to 1e-8, one V-cycle per step; matrix, right-hand
    side and solution resident on the device; one step = amg_setup + amg_solve + amg_free, host
    wall time between device synchronisations, L2 flushed before each; FP64 and mixed."""
    import numpy as np
    from paper_2103_10476_gb300 import problems as P
    A, b, kw = P.workload_convdiff64()
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    arg = amg.csr_arg(A.n, rp, ci, v)
    out = {"workload": "convection-diffusion 64^3 interior nodes (velocity (0.16,0.08,0.04), unit x/y spacing, "
                       "z ratio 1.05), theta 0.02, 1Norm+OffLmp, symmetrised strength, GMRES(30) to 1e-8, "
                       "RHS seed 1; setup+solve per step, device-resident",
           "rows": A.n, "nnz": A.nnz}
    for prec_name, prec in (("fp64", amg.AMG_FP64), ("mixed", amg.AMG_MIXED)):
        p = amg.amg_params_default(precision=prec, cuda_stream=stream.cuda_stream, **kw)
        steps = []
        for k in range(1 + 3):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = amg.amg_setup(arg, None, p)
            t1 = time.perf_counter()
            info = amg.amg_solve(h, bd, xd, TOL)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            amg.amg_free(h)
            if k > 0:
                steps.append({"setup_ms": 1e3 * (t1 - t0), "solve_ms": 1e3 * (t2 - t1), "iters": info.iters,
                              "status": info.status, "relres": info.relres_true, "levels": info.levels})
        tot = sum(s_["setup_ms"] + s_["solve_ms"] for s_ in steps)
        its = steps[-1]["iters"]
        out[prec_name] = {"solves_per_s": len(steps) / (tot / 1000.0), "ms_per_step": tot / len(steps),
                          "solve_ms_per_iteration": steps[-1]["solve_ms"] / max(its, 1), "per_step": steps}
    return out


def run_systems(args, amg, torch):
    """A system of PDEs: 3D linear elasticity on 40^3 unit hexahedra (face x = 0
    clamped; 201,720 unknowns, three per node; 15.5M entries) with its six rigid-body modes as
    the near-null space: block strength, node aggregation, QR tentative prolongator; theta
    0.02, PCG to 1e-8; matrix, near-null space and RHS resident on the device; one step =
    amg_setup + amg_solve + amg_free, host wall time between device synchronisations, L2
    flushed before each; FP64 and mixed, 3 steps after a warm-up."""
    import numpy as np
    from paper_2103_10476_gb300 import problems as P
    t0 = time.perf_counter()
    A, b, kw = P.workload_elasticity()
    gen_s = time.perf_counter() - t0
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    Bd = torch.from_numpy(np.ascontiguousarray(A.meta["rbm"]).reshape(-1)).cuda()
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    arg = amg.csr_arg(A.n, rp, ci, v)
    out = {"workload": "3D elasticity 40^3 hexahedra, E 1, nu 0.3, face x=0 clamped, 3 unknowns per node, "
                       "6 rigid-body modes, theta 0.02, PCG to 1e-8, RHS seed 6; setup+solve per step, "
                       "device-resident", "rows": A.n, "nnz": A.nnz, "generate_s": gen_s}
    for prec_name, prec in (("fp64", amg.AMG_FP64), ("mixed", amg.AMG_MIXED)):
        p = amg.amg_params_default(precision=prec, cuda_stream=stream.cuda_stream, **kw)
        steps = []
        for k in range(1 + 3):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = amg.amg_setup(arg, Bd, p)
            t1 = time.perf_counter()
            info = amg.amg_solve(h, bd, xd, TOL)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            amg.amg_free(h)
            if k > 0:
                steps.append({"setup_ms": 1e3 * (t1 - t0), "solve_ms": 1e3 * (t2 - t1), "iters": info.iters,
                              "status": info.status, "relres": info.relres_true, "levels": info.levels,
                              "op_complexity": info.op_complexity})
        tot = sum(s_["setup_ms"] + s_["solve_ms"] for s_ in steps)
        out[prec_name] = {"solves_per_s": len(steps) / (tot / 1000.0), "ms_per_step": tot / len(steps),
                          "per_step": steps}
    return out


COMBOS = [(m, "+".join(n for b, n in ((1, "1Norm"), (2, "OffLmp"), (8, "Cnstrnt"), (4, "Sprsfy")) if m & b)
           or "traditional") for m in range(16)]


def run_study(args, amg, torch):
    """§3.1's study on its stand-in: the randomly perturbed cube (ne^3 elements, z spacing 100x,
    nodes moved by up to 20% of the spacing, seeds 5, 6, ...), strength from the distance
    Laplacian (theta 0.025), coarsest level <= 1000 rows, PCG to 1e-10, all 16 combinations of
    1Norm, OffLmp, Cnstrnt and Sprsfy.  Matrix, coordinates and right-hand side resident on
    the device; each run is amg_setup_coords + amg_solve + amg_free, timed on the host
    between device synchronisations."""
    import numpy as np
    from paper_2103_10476_gb300 import problems as P
    seeds = list(range(5, 5 + args.study_seeds))
    t0 = time.perf_counter()
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=len(seeds)) as ex:
        meshes = list(ex.map(lambda s: P.perturbed_cube(args.study_ne, seed=s), seeds))
    gen_s = time.perf_counter() - t0
    rows = {name: {"iters": [], "fail": 0, "opc": []} for _, name in COMBOS}
    ms = []
    for A in meshes:
        rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
        X = torch.from_numpy(np.ascontiguousarray(A.meta["coords"])).cuda()
        b = torch.from_numpy(P.rhs_uniform(A.n, 1)).cuda()
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        arg = amg.csr_arg(A.n, rp, ci, v)
        for k, (mask, name) in enumerate([(0, "warm-up")] + COMBOS):
            p = amg.amg_params_default(theta=0.025, variants=mask, max_coarse=1000,
                                       strength=amg.AMG_STRENGTH_DISTANCE)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            h = amg.C.c_void_p()
            st = amg.lib.amg_setup_coords(amg.C.byref(arg), None, X.data_ptr(), 3, amg.C.byref(p), amg.C.byref(h))
            info = None
            if st == amg.AMG_OK:
                info = amg.amg_solve(h, b, x, 1e-10)
                amg.amg_free(h)
            torch.cuda.synchronize()
            if k == 0:
                continue
            ms.append(1e3 * (time.perf_counter() - t1))
            r = rows[name]
            if st != amg.AMG_OK or info.status != amg.AMG_OK:
                r["fail"] += 1
            else:
                r["iters"].append(info.iters)
                r["opc"].append(info.op_complexity)
    table = {name: {"iters_mean": (sum(r["iters"]) / len(r["iters"])) if r["iters"] else None,
                    "failures": r["fail"], "runs": len(seeds),
                    "op_complexity": (sum(r["opc"]) / len(r["opc"])) if r["opc"] else None}
             for name, r in rows.items()}
    return {"workload": f"perturbed cube {args.study_ne}^3 elements ({meshes[0].n} unknowns), z spacing x100, "
                        f"nodes moved up to 20% of the spacing, seeds {seeds[0]}..{seeds[-1]}; distance-Laplacian "
                        "strength theta 0.025, coarsest <= 1000, PCG to 1e-10, 16 combinations",
            "generate_s": gen_s, "runs": len(ms), "ms_per_run": sum(ms) / len(ms),
            "solves_per_s": len(ms) / (sum(ms) / 1000.0), "combinations": table}


def run_serving(args, amg, seconds: float, precisions):
    """The request stream of problems.serving_stream (Poisson 200 req/s, operators with edge
    log-uniform 16..96 nodes, stretched or 10^U(-2,2) coefficients, 30% repeats, 1..8
    right-hand sides, seed 4) over the first `seconds` of arrivals, served with a 120 GB HBM
    budget.  Operators and right-hand sides are host arrays generated before the clock
    starts; each request is submitted at its arrival time and its latency runs from submit
    until its solutions are in host memory."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np
    from paper_2103_10476_gb300 import problems as P
    reqs, ops = P.serving_stream(seconds, rate=args.serve_rate)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        mats = list(ex.map(lambda o: P.make_operator(o, engine="c"), ops))

        def rhs(r):
            n = mats[r[1]].n
            return np.concatenate([P.rhs_uniform(n, r[3] ^ (k << 20)) for k in range(r[2])])
        bs = list(ex.map(rhs, reqs))
    gen_s = time.perf_counter() - t0
    csr = [amg.csr_arg(A.n, A.row_ptr, A.col, A.val) for A in mats]
    out = {"workload": f"Poisson {args.serve_rate:g} req/s for {seconds:g} s of arrivals ({len(reqs)} requests, "
                       f"{len(ops)} distinct operators, {sum(r[2] for r in reqs)} right-hand sides), edge "
                       "log-uniform 16..96 nodes, stretched or 10^U(-2,2) coefficients, 30% repeats, 1..8 RHS, "
                       "seed 4; theta 0.02 1Norm+OffLmp; 120 GB HBM budget",
           "generate_s": gen_s, "rows_mean": float(np.mean([A.n for A in mats]))}
    for prec_name in precisions:
        prec = amg.AMG_MIXED if prec_name == "mixed" else amg.AMG_FP64
        p = amg.amg_params_default(theta=0.02, variants=3, precision=prec)
        cfg = amg.amg_server_config_default(p, hbm_budget_bytes=120 << 30, setup_threads=8, max_systems=8192,
                                            max_rows=1 << 27, tol=TOL, tune=1)
        srv = amg.amg_server_create(cfg)
        xs = [np.empty_like(b) for b in bs]
        for x in xs:
            x.fill(0.0)     # written once by the CPU, so every page is populated
        tickets = [None] * len(reqs)
        infos = [None] * len(reqs)
        submitted = threading.Event()

        def collect():
            for i in range(len(reqs)):
                while tickets[i] is None:
                    time.sleep(0.0005)
                infos[i] = amg.amg_server_wait(srv, tickets[i])
        th = threading.Thread(target=collect)
        th.start()
        start = time.perf_counter()
        for i, r in enumerate(reqs):
            dt = r[0] - (time.perf_counter() - start)
            if dt > 0:
                time.sleep(dt)
            tickets[i] = amg.amg_server_submit(srv, csr[r[1]], r[2], bs[i], xs[i])
        submitted.set()
        th.join()
        wall = time.perf_counter() - start
        stats = amg.amg_server_stats(srv)
        amg.amg_server_destroy(srv)
        lat = [i.latency_ms for i in infos]
        ok = sum(1 for i in infos if i.status == 0)
        out[prec_name] = {
            "solves_per_s": stats.solves / wall, "requests_per_s": len(reqs) / wall, "wall_s": wall,
            "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "mean_ms": sum(lat) / len(lat),
            "queue_p50_ms": pct([i.queue_ms for i in infos], 0.5),
            "setup_p50_ms": pct([i.setup_ms for i in infos if not i.cache_hit], 0.5),
            "ok": ok, "failed": len(infos) - ok, "relres_max": max(i.relres_max for i in infos),
            "cache_hits": stats.cache_hits, "cache_misses": stats.cache_misses, "evictions": stats.evictions,
            "engine_iterations": stats.iterations, "engine_busy_s": stats.engine_busy_ms / 1000.0,
            "commits": stats.commits, "first_error": stats.first_error.decode(errors="replace") or None,
            "statuses": sorted({amg.amg_status_string(i.status) for i in infos}),
            "hbm_hierarchies_gb": stats.bytes_hierarchies / 2**30,
            "hbm_engine_gb": stats.bytes_engine / 2**30}
    if not args.no_plain:
        # the plain FP64 GPU path on the first requests of the same stream, one after another:
        # amg_setup of the request's operator from its host arrays, amg_solve of each of its
        # right-hand sides, amg_free (no server, no cache, no batching)
        k = min(len(reqs), args.plain_requests)
        p = amg.amg_params_default(theta=0.02, variants=3, precision=amg.AMG_FP64)
        xs = [np.zeros_like(bs[i]) for i in range(k)]
        lat = []
        t0 = time.perf_counter()
        solves = 0
        for i in range(k):
            r = reqs[i]
            n = mats[r[1]].n
            ts = time.perf_counter()
            h = amg.amg_setup(csr[r[1]], None, p)
            for j in range(r[2]):
                amg.amg_solve(h, bs[i][j * n:(j + 1) * n], xs[i][j * n:(j + 1) * n], TOL)
            amg.amg_free(h)
            solves += r[2]
            lat.append(1e3 * (time.perf_counter() - ts))
        tp = time.perf_counter() - t0
        out["plain_fp64"] = {"solves_per_s": solves / tp, "requests_per_s": k / tp, "requests": k, "solves": solves,
                             "wall_s": tp, "mean_ms_per_request": sum(lat) / len(lat),
                             "how": "the first requests of the same stream, one after another: amg_setup from host "
                                    "arrays + amg_solve per right-hand side + amg_free, FP64, no server or cache"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="randcoef128", choices=sorted(VARIANT_SETS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision line beside the FP64 one")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--once", action="store_true",
                    help="one setup + solve (or --vcycles V-cycles) of one method, for profiler captures")
    ap.add_argument("--method", default=None, help="with --once: which method of the workload (default: first)")
    ap.add_argument("--vcycles", type=int, default=0)
    ap.add_argument("--layout", default="auto", choices=["auto", "csr", "sell"],
                    help="with --once: storage of the solve's operator products (spmv_layout)")
    ap.add_argument("--trace", action="store_true", help="with --once: also report the setup's phase times")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-system batched line")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-count", type=int, default=512, help="systems of the batched line")
    ap.add_argument("--batch-precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched line, printed alone (for profiler captures)")
    ap.add_argument("--no-study", action="store_true", help="skip the 16-combination perturbed-cube study line")
    ap.add_argument("--study-ne", type=int, default=60, help="elements per direction of the study's cube")
    ap.add_argument("--study-seeds", type=int, default=3, help="meshes (seeds) of the study")
    ap.add_argument("--study-only", action="store_true", help="only the study line, printed alone")
    ap.add_argument("--no-multi", action="store_true", help="skip the eight-right-hand-side line")
    ap.add_argument("--multi-only", action="store_true", help="only the eight-right-hand-side line, printed alone")
    ap.add_argument("--no-systems", action="store_true", help="skip the elasticity (systems of PDEs) line")
    ap.add_argument("--systems-only", action="store_true", help="only the elasticity line, printed alone")
    ap.add_argument("--no-gmres", action="store_true", help="skip the nonsymmetric (GMRES) line")
    ap.add_argument("--gmres-only", action="store_true", help="only the nonsymmetric (GMRES) line, printed alone")
    ap.add_argument("--no-serving", action="store_true", help="skip the served request stream")
    ap.add_argument("--serving-only", action="store_true", help="only the served stream, printed alone")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="seconds of arrivals of the served stream")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-mixed-only", action="store_true", help="serve the stream in mixed precision only")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain FP64 one-at-a-time baselines of the batched and served lines")
    ap.add_argument("--plain-requests", type=int, default=300,
                    help="requests of the served stream timed through the plain FP64 path")
    args = ap.parse_args()
    world, rank, local = dist_init()

    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.once:
        return run_once(args)
    if args.multi_only:
        import torch
        torch.cuda.set_device(local)
        from paper_2103_10476_gb300 import amg
        print(json.dumps(run_multi(args, amg, torch)), flush=True)
        return 0
    if args.serving_only:
        import torch
        torch.cuda.set_device(local)
        from paper_2103_10476_gb300 import amg
        print(json.dumps(run_serving(args, amg, args.serve_seconds,
                                     ["mixed"] if args.serve_mixed_only else ["mixed", "fp64"])), flush=True)
        return 0
    if args.systems_only:
        import torch
        torch.cuda.set_device(local)
        from paper_2103_10476_gb300 import amg
        print(json.dumps(run_systems(args, amg, torch)), flush=True)
        return 0
    if args.gmres_only:
        import torch
        torch.cuda.set_device(local)
        from paper_2103_10476_gb300 import amg
        print(json.dumps(run_gmres(args, amg, torch)), flush=True)
        return 0
    if args.study_only:
        import torch
        torch.cuda.set_device(local)
        from paper_2103_10476_gb300 import amg
        print(json.dumps(run_study(args, amg, torch)), flush=True)
        return 0
    if args.batched_only:
        import torch
        torch.cuda.set_device(local)
        from paper_2103_10476_gb300 import amg
        print(json.dumps(run_batched(args, amg, torch)), flush=True)
        return 0

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_2103_10476_gb300 import amg

    if args.workload in ("elasticity40", "convdiff64"):
        raise SystemExit(f"{args.workload} is timed by its own line (--systems-only, --gmres-only); use it with --once")
    A, b, theta = make_workload(args.workload)
    variants = VARIANT_SETS[args.workload]
    prec = amg.AMG_MIXED if args.precision == "mixed" else amg.AMG_FP64
    stream = torch.cuda.current_stream()
    params = [amg.amg_params_default(theta=theta, variants=v, precision=prec, cuda_stream=stream.cuda_stream)
              for _, v in variants]
    # device-resident inputs
    rp_d = torch.from_numpy(A.row_ptr).cuda()
    ci_d = torch.from_numpy(A.col).cuda()
    v_d = torch.from_numpy(A.val).cuda()
    b_d = torch.from_numpy(b).cuda()
    x_d = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    arg_d = amg.csr_arg(A.n, rp_d, ci_d, v_d)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step(params_list, record, evs=None):
        """Setup + solve (+ free) of every method of the workload; with `evs`, CUDA events on
        the launching stream before each setup, after it and after the solve."""
        for k, ((name, _), p) in enumerate(zip(variants, params_list)):
            if evs is not None:
                evs[k][0].record(stream)
            h, st = amg.amg_setup_status(arg_d, None, p)
            if evs is not None:
                evs[k][1].record(stream)
            if h is None:
                if record is not None:
                    record["status"][name] = amg.amg_status_string(st)
                if evs is not None:
                    evs[k][2].record(stream)
                continue
            info = amg.amg_solve(h, b_d, x_d, TOL)
            amg.amg_free(h)
            if evs is not None:
                evs[k][2].record(stream)
            if record is not None:
                record["iters"][name] = info.iters
                record["status"][name] = amg.amg_status_string(info.status)
                record["relres"][name] = info.relres_true
                record["levels"][name] = info.levels

    def timed(params_list, steps, warmup):
        """Warm-up, then `steps` timed steps: CUDA events on the launching stream around each
        step and around each method's setup and solve, L2 flushed before each step (outside
        the events).  Nothing else is recorded inside the timed region."""
        rec = {"iters": {}, "status": {}, "relres": {}, "levels": {}}
        for _ in range(warmup):
            one_step(params_list, None)
        torch.cuda.synchronize()
        mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        ev0 = [mk() for _ in range(steps)]
        ev1 = [mk() for _ in range(steps)]
        per = [[[mk(), mk(), mk()] for _ in variants] for _ in range(steps)]
        launches0 = amg.amg_launch_count()
        barrier(world)
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            ev0[k].record(stream)
            one_step(params_list, rec if k == steps - 1 else None, per[k])
            ev1[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        launches = amg.amg_launch_count() - launches0
        step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(steps)]
        setup_ms = [e[0].elapsed_time(e[1]) for st in per for e in st]
        solve_ms = [e[1].elapsed_time(e[2]) for st in per for e in st]
        return step_ms, setup_ms, solve_ms, rec, launches

    def profiled(params_list, steps):
        """Kernel-class timing (library CUDA events around the first method's fine-level
        launches) over `steps` extra steps, outside the timed region."""
        amg.amg_profile_enable(1)      # reset the totals
        amg.amg_profile_enable(0)
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            for k, ((name, _), p) in enumerate(zip(variants, params_list)):
                if k == 0:
                    amg.amg_profile_enable(2)
                h, st = amg.amg_setup_status(arg_d, None, p)
                if h is not None:
                    amg.amg_solve(h, b_d, x_d, TOL)
                    amg.amg_free(h)
                if k == 0:
                    amg.amg_profile_enable(0)
        torch.cuda.synchronize()
        return {kc: amg.amg_profile_read(kc) for kc in (amg.KC_PCG_SPMV, amg.KC_VCYCLE_SPMV, amg.KC_SPGEMM)}

    def solution(params_list):
        """The first method's solution, solved once more after the timed regions (host copy)."""
        h, st = amg.amg_setup_status(arg_d, None, params_list[0])
        if h is None:
            return None
        x_d.zero_()
        amg.amg_solve(h, b_d, x_d, TOL)
        amg.amg_free(h)
        torch.cuda.synchronize()
        return x_d.cpu().numpy().copy()

    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        step_ms, setup_ms, solve_ms, rec, launches = timed(params, args.steps, args.warmup)
    t_wall = time.perf_counter() - t_wall
    total_ms = max_over_ranks(world, sum(step_ms))
    solves_per_step = len(variants)
    value = whole_job_rate(solves_per_step * args.steps, world, total_ms)

    # the oracle's whole solve of the full workload (the CPU baseline) runs in a process of its
    # own while the rest of the benchmark uses the GPU; its solution gives each result's error
    oracle_job = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in ORACLE_FULL:
        oracle_job = OracleFullRun(args.workload)

    # the other precision, same workload and timing rules (reported beside the headline)
    other = None
    mparams = None
    if args.precision == "fp64" and not args.no_mixed:
        mparams = [amg.amg_params_default(theta=theta, variants=v, precision=amg.AMG_MIXED,
                                          cuda_stream=stream.cuda_stream) for _, v in variants]
        msteps = max(3, args.steps // 2)
        m_ms, m_setup, m_solve, m_rec, _ = timed(mparams, msteps, 2)
        m_total = max_over_ranks(world, sum(m_ms))
        other = {"precision": "mixed (FP32 hierarchy values and V-cycle, FP64 flexible PCG)",
                 "value": whole_job_rate(solves_per_step * msteps, world, m_total), "unit": "solves/s",
                 "ms_per_step": m_total / msteps, "steps": msteps,
                 "setup_ms_per_solve": statistics.median(m_setup), "solve_ms_per_solve": statistics.median(m_solve),
                 "iters": m_rec["iters"], "status": m_rec["status"], "relres": m_rec["relres"]}

    # end to end through the C ABI with host buffers (host -> device copy of the matrix and the
    # right-hand side inside every step, device -> host copy of the solution)
    b_h = torch.from_numpy(b).pin_memory()
    x_h = torch.zeros(A.n, dtype=torch.float64).pin_memory()
    rp_h = torch.from_numpy(A.row_ptr).pin_memory()
    ci_h = torch.from_numpy(A.col).pin_memory()
    val_h = torch.from_numpy(A.val).pin_memory()
    arg_h = amg.csr_arg(A.n, rp_h, ci_h, val_h)
    e2e_steps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        for p in params:
            h, st = amg.amg_setup_status(arg_h, None, p)
            if h is None:
                continue
            amg.amg_solve(h, b_h, x_h, TOL)
            amg.amg_free(h)
    torch.cuda.synchronize()
    te = time.perf_counter() - te
    e2e_value = whole_job_rate(solves_per_step * e2e_steps, world, 1000.0 * max_over_ranks(world, te))
    h2d = solves_per_step * (8 * (A.n + 1) + 12 * A.nnz + 8 * A.n)
    d2h = solves_per_step * 8 * A.n

    # roofline classes from a separate, profiled pass
    prof = profiled(params, 2)
    x_fp64 = solution(params) if oracle_job is not None else None
    x_mixed = solution(mparams) if (oracle_job is not None and mparams is not None) else None

    batched = None if args.no_batched else run_batched(args, amg, torch)
    study = None if args.no_study else run_study(args, amg, torch)
    multi = None if args.no_multi else run_multi(args, amg, torch)
    gmres = None if args.no_gmres else run_gmres(args, amg, torch)
    systems = None if args.no_systems else run_systems(args, amg, torch)
    serving = None if args.no_serving else run_serving(args, amg, args.serve_seconds,
                                                        ["mixed"] if args.serve_mixed_only else ["mixed", "fp64"])

    if rank != 0:
        return 0

    # Roofline of the dominant kernel: the fine level's V-cycle products (the largest kernel by
    # device time in the ncu launch list of a setup + solve: profiles/launches_randcoef128.md),
    # timed by the library's CUDA events around each of its launches in the profiled pass.  The
    # other classes are listed beside it; the Galerkin class brackets whole products, host
    # synchronisations between their phases included, so its rate is not a kernel's.
    peak, peak_src = measured_peaks()
    names = {amg.KC_PCG_SPMV: "pcg_spmv_fp64", amg.KC_VCYCLE_SPMV: "vcycle_fine_spmv", amg.KC_SPGEMM: "galerkin_spgemm"}
    dom = amg.KC_VCYCLE_SPMV if prof[amg.KC_VCYCLE_SPMV][0] > 0 else max(prof, key=lambda k: prof[k][1])
    n_l, ms_l, by_l = prof[dom]
    achieved = (by_l / (ms_l / 1000.0)) / 1e9 if ms_l > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "launches": n_l,
                "avg_launch_us": 1000.0 * ms_l / max(n_l, 1), "bytes_per_launch": by_l / max(n_l, 1),
                "traffic": ncu_traffic(names[dom], args.workload),
                "classes": {names[k]: {"launches": prof[k][0], "ms": prof[k][1],
                                       "GBps": (prof[k][2] / (prof[k][1] / 1000.0) / 1e9) if prof[k][1] > 0 else None}
                            for k in prof}}

    cpu = None
    errors = None
    if oracle_job is not None:
        full = oracle_job.result()
        if full is not None and full.get("status") == 0:
            secs = full["setup_s"] + full["solve_s"]
            cpu = {"value": 1.0 / secs, "unit": "solves/s", "cores": 1, "kind": "oracle",
                   "sample": f"one whole setup + solve of the same workload at full size ({A.n} unknowns, "
                             f"{variants[0][0]}, FP64): setup {full['setup_s']:.1f} s + solve {full['solve_s']:.1f} s "
                             f"({full['iters']} PCG iterations), single-threaded C oracle in a process of its own "
                             f"while the GPU side lines ran; host has {os.cpu_count()} cores",
                   "setup_s": full["setup_s"], "solve_s": full["solve_s"], "iters": full["iters"],
                   "levels": full["levels"]}
            xo = full["x"]
            nxo = float(np.linalg.norm(xo))
            errors = {"reference": "FP64 oracle solution of the same system (1e-8 relative residual)",
                      "fp64": float(np.linalg.norm(x_fp64 - xo) / nxo) if x_fp64 is not None else None,
                      "mixed": float(np.linalg.norm(x_mixed - xo) / nxo) if x_mixed is not None else None,
                      "oracle_iters": full["iters"]}
        else:
            cpu = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                   "sample": f"oracle full run failed: {full}"}
    elif not args.no_cpu_baseline:
        n_s, secs, done = oracle_sample(A, b, theta, variants, args.cpu_budget)
        cpu = {"value": n_s / secs, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"{n_s} whole setup+solve runs ({', '.join(done)}) of the same workload, single-threaded C "
                         f"oracle, {secs:.1f} s; host has {os.cpu_count()} cores"}

    per_solve_ms = [a_ + b_ for a_, b_ in zip(setup_ms, solve_ms)]
    lat = sorted(per_solve_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == amg.AMG_FP64 else "f64+f32", "data": "synthetic",
        "config": workload_config(args),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "p50_ms": lat[len(lat) // 2] if lat else None,
        "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
        "setup_ms_per_solve": statistics.median(setup_ms), "solve_ms_per_solve": statistics.median(solve_ms),
        "iters": rec["iters"], "status": rec["status"], "relres": rec["relres"], "levels": rec["levels"],
        "wall_s": t_wall,
        "error_vs_oracle": errors,
        "mixed": other,
        "batched": batched,
        "study": study,
        "multi": multi,
        "gmres": gmres,
        "systems": systems,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
