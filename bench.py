"""Benchmark: DOF-solves/s of the stand-alone Helmholtz multigrid solver to a
relative residual of 1e-6 on one GB300 (or N replicas under torchrun).

Workload (default): the batched constant-k configuration -- 64 unit point
sources evenly spaced along the first interior row below the top boundary
of a 1025 x 1025 grid (n = 1024) at k = 300, solved together; GMRES(3)
V(2,2) smoothing with complex shift beta2 = 1/k, complex64 cycles inside
FP64 iterative refinement (the plain FP64 path is timed beside it).  One
step = one complete solve of all 64 right-hand sides from x0 = 0 (setup of
the hierarchy excluded and reported separately).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line on rank 0.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-solves/s to rel. residual 1e-6 (FP64 vs mixed, batched); % HBM roofline"
UNIT = "DOF-solves/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--k", type=float, default=300.0)
    p.add_argument("--n", type=int, default=1024, help="intervals per side (0: k/0.625)")
    p.add_argument("--smoother", default="gmres3", choices=["jacobi", "gmres3"])
    p.add_argument("--cycle", default="V", choices=["V", "W"])
    p.add_argument("--nu", type=int, default=2, help="pre = post smoothing steps")
    p.add_argument("--beta2", type=float, default=-1.0, help="complex shift (default 1/k for GMRES, 0.7 Jacobi)")
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "mixed-ff"])
    p.add_argument("--batch", type=int, default=64)
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--no-fp64-line", action="store_true", help="skip the FP64 comparison solve")
    p.add_argument("--no-ff-line", action="store_true", help="skip the float-float outer-loop variant")
    p.add_argument("--cpu-sample-cycles", type=int, default=10,
                   help="oracle cycles of the one-core CPU baseline (0: no CPU baseline)")
    p.add_argument("--cpu-allcore-cycles", type=int, default=4,
                   help="oracle cycles per host core of the all-core CPU baseline (batched workloads)")
    p.add_argument("--no-error-vs-oracle", action="store_true",
                   help="skip the oracle's solve of the first right-hand side (error against the FP64 oracle)")
    p.add_argument("--error-max-cycles", type=int, default=100,
                   help="run the oracle's solve for error_vs_oracle only when it needs at most this many cycles")
    p.add_argument("--workload", default="batched",
                   choices=["batched", "layered", "ragged", "gradient", "two-grid", "sweep", "absorbing"],
                   help="batched: the bench line (default); the others print one JSON line for the other "
                        "workloads: layered velocity model at --freq Hz, a ragged batch of 32 problems, the "
                        "adjoint gradient of a receiver misfit")
    p.add_argument("--freq", type=float, default=10.0, help="layered workload: frequency in Hz (10, 20, 40)")
    p.add_argument("--abc", type=int, default=1, choices=[1, 2],
                   help="absorbing boundary rows: 1 the first-order condition of Sec. 2, 2 the second-order "
                        "Engquist-Majda condition (a variant; batched, layered and absorbing workloads)")
    p.add_argument("--transfer", default="bezier", choices=["bezier", "linear"],
                   help="inter-grid transfers: Eq. (xex) or linear interpolation (ablation)")
    p.add_argument("--krylov", type=int, default=0,
                   help="m > 0: restarted FGMRES(m) with one cycle as the right preconditioner")
    p.add_argument("--march", type=int, default=-1, choices=[-1, 0, 1],
                   help="GMRES(3) as row/column marches: 1 always, 0 never, -1 by level size (library default)")
    p.add_argument("--probe", action="store_true",
                   help="profiling probe: set up the workload and run two solves capped at --max-cycles; no timing")
    p.add_argument("--max-cycles", type=int, default=2)
    p.add_argument("--flat", type=int, default=0, choices=[0, 1],
                   help="ragged workload: 0 = problems of one shape batched, a graph per group (library default); "
                        "1 = one flattened launch per kernel over all problems")
    p.add_argument("--coarse-nodes", type=int, default=-1,
                   help=">= 0: levels with at most this many nodes run in the coarse-cycle launch (overrides the "
                        "autotuner's choice)")
    p.add_argument("--coarse-mode", type=int, default=-1, help=">= 0: coarse-cycle launch organisation (override)")
    p.add_argument("--no-autotune", action="store_true", help="library default launch shapes instead of the autotuner's")
    a = p.parse_args()
    if a.warmup < 3:
        p.error("--warmup must be >= 3")
    if a.n == 0:
        a.n = int(round(a.k / 0.625))
    if a.beta2 < 0:
        a.beta2 = 1.0 / a.k if a.smoother == "gmres3" else 0.7
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_throughput(my_seconds, my_units):
    """Whole-job throughput over all ranks: the units every rank processed
    divided by the slowest rank's time (torch.distributed when initialised,
    any backend; a single process otherwise).  Returns (value, seconds)."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
        t = torch.tensor([float(my_seconds)], dtype=torch.float64, device=dev)
        u = torch.tensor([float(my_units)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        return float(u.item()) / float(t.item()), float(t.item())
    return my_units / my_seconds, my_seconds


def workload_config(a):
    src = (f"{a.batch} point sources along the first interior row below the top boundary" if a.batch > 1
           else "centre point source")
    return {
        "workload": f"MP 2-A constant k={a.k:g}, kh={a.k / a.n:.3f}, {a.n + 1}x{a.n + 1} unknowns per RHS, {src}",
        "unknowns": (a.n + 1) ** 2,
        "rhs_per_gpu": a.batch,
        "smoother": a.smoother,
        "cycle": f"{a.cycle}({a.nu},{a.nu})",
        "transfer": "Eq. (xex) higher-order" if a.transfer == "bezier" else "linear interpolation (ablation)",
        "outer": (f"FGMRES({a.krylov}), one cycle from zero as the right preconditioner; cycles = "
                  f"preconditioner applications" if a.krylov else "stand-alone cycle iteration"),
        "beta2": a.beta2,
        "precision": a.precision,
        "tol": a.tol,
        "l2": "L2 flushed between timed solves (256 MiB write)",
        "parallelism": "replicas",
    }


# ------------------------------------------------------------------ clocks


class ClockSampler:
    def __init__(self, gpu):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle


def oracle_cycle_seconds(a, ncycles):  # noqa: D401
    """Time ``ncycles`` oracle cycles on the full workload (setup excluded);
    with --krylov, ``ncycles`` FGMRES steps (each one preconditioning cycle
    plus its Arnoldi work) of one restart cycle."""
    from oracle import cycle as oc
    b = _oracle_rhs0(a)
    H, opt = _oracle_setup(a)
    x = np.zeros_like(b)
    if a.krylov:
        from oracle import krylov as okr
        t0 = time.perf_counter()
        okr.fgmres_cycle(H.A[0], lambda v: oc.mg_cycle(H, 0, np.zeros_like(v), v, opt), x, b, ncycles, 0.0,
                         np.linalg.norm(b))
        return (time.perf_counter() - t0) / ncycles
    t0 = time.perf_counter()
    for _ in range(ncycles):
        x = oc.mg_cycle(H, 0, x, b, opt)
        _ = np.linalg.norm(b - H.A[0] @ x)     # the per-cycle stopping test
    return (time.perf_counter() - t0) / ncycles


def run_reference(a):
    """The oracle as the reference arm: W untimed and K timed oracle cycles on
    the full workload (one cycle per step), scaled to a whole solve with the
    cycle count of the method on this workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    from oracle import cycle as oc
    from oracle import hierarchy as oh
    h = 1.0 / a.n
    b = (synth.source_row(a.n, a.n, h, a.batch)[0] if a.batch > 1 else synth.point_source(a.n, a.n, h)).ravel()
    H = oh.build_hierarchy(a.n, a.n, h, a.k, a.beta2, kind=a.transfer, abc=a.abc)
    opt = oc.CycleOptions(1 if a.cycle == "V" else 2, a.smoother, a.nu, a.nu, 4.5)
    x = np.zeros_like(b)
    if a.krylov:   # one FGMRES step (a preconditioning cycle and its Arnoldi work) per step
        from oracle import krylov as okr
        M = lambda v: oc.mg_cycle(H, 0, np.zeros_like(v), v, opt)  # noqa: E731
        okr.fgmres_cycle(H.A[0], M, x, b, a.warmup, 0.0, np.linalg.norm(b))
        t0 = time.perf_counter()
        okr.fgmres_cycle(H.A[0], M, x, b, a.steps, 0.0, np.linalg.norm(b))
        tc = (time.perf_counter() - t0) / a.steps
    else:
        for _ in range(a.warmup):
            x = oc.mg_cycle(H, 0, x, b, opt)
            _ = np.linalg.norm(b - H.A[0] @ x)
        t0 = time.perf_counter()
        for _ in range(a.steps):
            x = oc.mg_cycle(H, 0, x, b, opt)
            _ = np.linalg.norm(b - H.A[0] @ x)
        tc = (time.perf_counter() - t0) / a.steps
    cycles_needed = _cycles_from_cache(a)
    N = (a.n + 1) ** 2 * a.batch
    value = N / (tc * a.batch * cycles_needed) if cycles_needed else None
    sample = (f"{a.steps} timed oracle cycles (after {a.warmup} untimed) of one right-hand side of the workload, "
              f"one core, scaled to {a.batch} right-hand sides x the oracle's {cycles_needed} cycles per solve "
              f"(oracle/bench_cycles.json)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": tc * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic", "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _cycles_from_cache(a):
    """Cycles of one solve of the workload by the oracle (written by
    oracle/bench_cycles.py), or None."""
    p = os.path.join(ROOT, "oracle", "bench_cycles.json")
    try:
        d = json.load(open(p))
        return int(d.get(f"{a.k:g}/{a.n}/{a.smoother}/{a.cycle}{a.nu}/{a.beta2:g}" +
                         (f"/fgmres{a.krylov}" if a.krylov else "") + ("/linear" if a.transfer == "linear" else "") +
                         ("/abc2" if getattr(a, "abc", 1) == 2 else "")))
    except Exception:
        return None


# ------------------------------------------------------------------ GPU arm


# FP64 flops per node of one GMRES(3) smoothing step as the method states it
# (Sec. 5.3; counted on an interior node with complex arithmetic: add 2, real
# scale 2, conjugated multiply-accumulate 8, |z|^2 accumulate 4): initial
# residual 14, its norm and scaling 6; Arnoldi step j = 0, 1, 2: apply 12,
# j + 1 inner products and updates 16 each, norm 4, scaling 2 (none after the
# last): 34, 50, 64; update of x by three basis vectors 24.  Total 192.
GMRES_STEP_FLOPS_PER_NODE = 192.0


def _oracle_rhs0(a):
    import synth
    h = 1.0 / a.n
    return (synth.source_row(a.n, a.n, h, a.batch)[0] if a.batch > 1 else synth.point_source(a.n, a.n, h)).ravel()


def _oracle_setup(a):
    from oracle import cycle as oc
    from oracle import hierarchy as oh
    H = oh.build_hierarchy(a.n, a.n, 1.0 / a.n, a.k, a.beta2, kind=a.transfer, abc=a.abc)
    opt = oc.CycleOptions(1 if a.cycle == "V" else 2, a.smoother, a.nu, a.nu, 4.5)
    return H, opt


def _oracle_solution_job(a):
    """The oracle's solve of the workload's first right-hand side to the
    bench tolerance (run in a spawned process beside the GPU work)."""
    from oracle import cycle as oc
    b = _oracle_rhs0(a)
    H, opt = _oracle_setup(a)
    t0 = time.perf_counter()
    if a.krylov:
        from oracle import krylov as okr
        r = okr.fgmres_solve(H, b, a.tol, opt, a.krylov)
    else:
        r = oc.mg_solve(H, b, a.tol, opt)
    return r.x, r.cycles, float(r.relres), bool(r.converged), time.perf_counter() - t0


def _oracle_cycles_job(args):
    """Per-cycle seconds of the oracle on right-hand side ``q`` of the
    workload (one process per host core for the all-core figure)."""
    a, q, ncycles = args
    import synth
    from oracle import cycle as oc
    h = 1.0 / a.n
    src = synth.source_row(a.n, a.n, h, a.batch) if a.batch > 1 else synth.point_source(a.n, a.n, h)[None]
    b = src[q % len(src)].ravel()
    H, opt = _oracle_setup(a)
    x = np.zeros_like(b)
    t0 = time.perf_counter()
    for _ in range(ncycles):
        x = oc.mg_cycle(H, 0, x, b, opt)
        _ = np.linalg.norm(b - H.A[0] @ x)     # the per-cycle stopping test
    return (time.perf_counter() - t0) / ncycles


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_ours(a):
    import multiprocessing as mp
    rank, world, local = dist_env()
    # the oracle's solution of the first right-hand side, for the error
    # against the FP64 oracle, runs in a process spawned before any GPU call
    cyc_oracle = _cycles_from_cache(a)
    pool, sol_job = None, None
    want_error = rank == 0 and world == 1 and not a.no_error_vs_oracle and cyc_oracle is not None and \
        cyc_oracle <= a.error_max_cycles
    if want_error:
        pool = mp.get_context("spawn").Pool(1)
        sol_job = pool.apply_async(_oracle_solution_job, (a,))

    import torch
    import paper_2308_13476_gb300 as hm
    import synth

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    hm.load_library()
    dev = torch.device("cuda", torch.cuda.current_device())
    n, k = a.n, a.k
    h = 1.0 / n
    N = (n + 1) ** 2
    if a.batch > 1:
        rhs_np = synth.source_row(n, n, h, a.batch)
    else:
        rhs_np = synth.point_source(n, n, h)[None].copy()
    rhs = torch.from_numpy(rhs_np).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # the library runs on its own stream; every CUDA event of the timings is
    # recorded on that stream (the launching stream)
    S = torch.cuda.Stream(device=dev)

    tuned = {}
    if not a.no_autotune:   # launch shapes from the autotuner (cached per GPU and problem shape)
        from paper_2308_13476_gb300 import autotune
        tuned, _ = autotune.tune(n, n, h, k, a.beta2, rhs, smoother=a.smoother, cycle=a.cycle, nu=a.nu,
                                 precision=a.precision, cache_path=os.path.join(ROOT, "paper_2308_13476_gb300",
                                                                                "autotune_cache.json"))
    tuned = dict(tuned or {})
    for name in ("coarse_nodes", "coarse_mode"):   # explicit overrides of the tuned shapes
        if getattr(a, name) >= 0:
            tuned[name] = getattr(a, name)
    if a.march != -1 or "march" not in tuned:   # an explicit --march overrides the tuned one
        tuned["march"] = a.march

    def make(precision, shapes=None):
        t0 = time.perf_counter()
        shapes = dict(shapes or {"march": a.march})
        s = hm.Solver(n, n, h, k, a.beta2, cycle=a.cycle, smoother=a.smoother, nu_pre=a.nu, nu_post=a.nu,
                      precision=precision, batch=a.batch, max_cycles=20000, krylov=a.krylov,
                      transfer=a.transfer, abc=a.abc, stream=S, **shapes)
        torch.cuda.synchronize()
        return s, time.perf_counter() - t0

    def timed_solves(s, steps):
        st_ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        en_ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        cyc = None
        launches = 0
        x = None
        for q in range(steps):
            flush.zero_()
            x = torch.zeros_like(rhs)
            torch.cuda.synchronize()
            st_ev[q].record(S)
            x, status, cyc, rr = s.solve(rhs, x=x, tol=a.tol)
            en_ev[q].record(S)
            torch.cuda.synchronize()
            if status != hm.MG_OK:
                raise RuntimeError(f"solve failed: {hm.STATUS_NAMES[status]} cycles={cyc} relres={rr}")
            launches += s.counters()[0]
        ms = [st_ev[q].elapsed_time(en_ev[q]) for q in range(steps)]
        return ms, cyc, launches, rr, x

    def e2e_pipelined(s, steps):
        """End to end through the public API with host buffers: every step
        copies its right-hand sides from pinned host memory and reads its
        solution back, on a copy stream, double-buffered so that the copies
        of neighbouring steps overlap the solve (as a serving loop does).
        Timed from the first copy's start to the last copy's end."""
        C = torch.cuda.Stream(device=dev)
        host_in = torch.from_numpy(rhs_np).pin_memory()
        host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
        r_dev = [torch.empty_like(rhs) for _ in range(2)]
        x_dev = [torch.empty_like(rhs) for _ in range(2)]
        ev_in = [torch.cuda.Event() for _ in range(steps)]
        ev_done = [torch.cuda.Event() for _ in range(steps)]
        ev_out = [torch.cuda.Event() for _ in range(steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(C):
            e0.record(C)
            r_dev[0].copy_(host_in, non_blocking=True)
            ev_in[0].record(C)
        for q in range(steps):
            if q + 1 < steps:   # next step's input, into the buffer step q-1 read
                with torch.cuda.stream(C):
                    if q >= 1:
                        C.wait_event(ev_done[q - 1])
                    r_dev[(q + 1) % 2].copy_(host_in, non_blocking=True)
                    ev_in[q + 1].record(C)
            S.wait_event(ev_in[q])
            if q >= 2:          # x buffer of step q-2 read back
                S.wait_event(ev_out[q - 2])
            with torch.cuda.stream(S):
                x_dev[q % 2].zero_()
            x, status, cyc, rr = s.solve(r_dev[q % 2], x=x_dev[q % 2], tol=a.tol)
            ev_done[q].record(S)
            if status != hm.MG_OK:
                raise RuntimeError(f"solve failed: {hm.STATUS_NAMES[status]}")
            with torch.cuda.stream(C):
                C.wait_event(ev_done[q])
                host_out[q % 2].copy_(x_dev[q % 2], non_blocking=True)
                ev_out[q].record(C)
        with torch.cuda.stream(C):
            e1.record(C)
        torch.cuda.synchronize()
        # the copy bandwidths on their own (not overlapped), one copy each way
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        with torch.cuda.stream(C):
            c0.record(C)
            r_dev[0].copy_(host_in, non_blocking=True)
            c1.record(C)
            host_out[0].copy_(x_dev[0], non_blocking=True)
            c2.record(C)
        torch.cuda.synchronize()
        nbytes = rhs.numel() * 16
        return e0.elapsed_time(e1), nbytes / (c0.elapsed_time(c1) * 1e-3) / 1e9, \
            nbytes / (c1.elapsed_time(c2) * 1e-3) / 1e9

    s, setup_s = make(a.precision, tuned)
    timed_solves(s, a.warmup)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    ms, cyc, launches, rr, x_last = timed_solves(s, a.steps)
    clk = clocks.stop()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    value, tmax = job_throughput(sum(ms) / 1e3, N * a.batch * a.steps)
    x0_gpu = x_last[0].cpu().numpy().ravel()
    # end to end through the public API with host buffers (one untimed run first)
    e2e_pipelined(s, 2)
    ms_e2e, h2d_gbs, d2h_gbs = e2e_pipelined(s, a.steps)
    e2e_value, _ = job_throughput(ms_e2e / 1e3, N * a.batch * a.steps)
    # roofline of the dominant kernel, timed live with CUDA events on the library's stream
    what = 5 if a.krylov else (0 if a.smoother == "jacobi" else 4)
    kms, kbytes = s.profile(what, 0, reps=20)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s (no measured peaks file)"
    achieved = kbytes / (kms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": step_traffic(a, what),
            "kernel": ({0: "level-0 weighted-Jacobi sweep",
                        4: ("level-0 GMRES(3) smoothing step: 4 row-march passes + update, 16 vector passes"
                            if a.precision == "fp64" else
                            "level-0 GMRES(3) smoothing step: 3 row-march passes + update, 13 vector passes "
                            "(the last Arnoldi vector's norm from the Gram form)"),
                        5: f"last FGMRES({a.krylov}) Arnoldi step (MGS-coefficient pass + new-vector pass, "
                           f"{2 * a.krylov + 1} FP64 and 3 cycle-precision vector passes)"}[what]) +
                      f" ({'complex128' if a.precision == 'fp64' else 'complex64'}), "
                      f"{kbytes / 1e6:.1f} MB algorithmic per step, {kms * 1e3:.0f} us per step, "
                      f"peak = {peak_src}"}
    extra = {"setup_s": setup_s, "cycles": cyc, "relres": rr}
    if not a.no_ff_line and a.precision == "mixed" and not a.krylov:   # float-float outer loop, same shapes
        s.close()
        sff, _ = make("mixed-ff", tuned)
        timed_solves(sff, 1)
        msff, cycff, _, rrff, _ = timed_solves(sff, a.steps)
        extra["mixed_ff_path"] = {"value": N * a.batch * a.steps / (sum(msff) / 1e3), "unit": UNIT,
                                  "cycles": cycff, "max_relres": max(rrff), "ms_per_solve": sum(msff) / a.steps}
        s = sff
    if not a.no_fp64_line and a.precision in ("mixed", "mixed-ff"):
        s.close()
        s64, setup64 = make("fp64")
        timed_solves(s64, 1)                      # warm-up: graph capture
        nfp = max(3, min(a.steps, 5))
        ms64, cyc64, _, rr64, _ = timed_solves(s64, nfp)
        fp = {"value": N * a.batch * nfp / (sum(ms64) / 1e3), "unit": UNIT, "cycles": cyc64,
              "max_relres": max(rr64), "ms_per_solve": sum(ms64) / nfp, "solves_timed": nfp}
        if a.smoother == "gmres3" and not a.krylov:
            # FP64 roofline: the fine-level GMRES(3) step against the FP64 FMA
            # rate measured in this run by the library's probe (mg_profile 6)
            pms, pflops = s64.profile(6, 0, reps=3)
            fp64_peak = pflops / (pms * 1e-3) / 1e12
            sms, sbytes = s64.profile(4, 0, reps=5)
            flops = GMRES_STEP_FLOPS_PER_NODE * N * a.batch
            ach = flops / (sms * 1e-3) / 1e12
            fp["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                              "frac": ach / fp64_peak, "hbm_frac": sbytes / (sms * 1e-3) / 1e9 / peak,
                              "kernel": f"level-0 GMRES(3) smoothing step (complex128), "
                                        f"{GMRES_STEP_FLOPS_PER_NODE:g} algorithmic FP64 flops and "
                                        f"{sbytes / (N * a.batch):g} B per node, {sms * 1e3:.0f} us per step",
                              "peak_source": "FP64 FMA throughput probe of the library (mg_profile kind 6: 8 "
                                             "independent FMA chains per thread, 2048 threads per SM, every SM), "
                                             "measured in this run"}
        extra["fp64_path"] = fp
        s64.close()
    else:
        s.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": tmax * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "c64+f64", "mixed-ff": "c64+ff"}.get(a.precision, "c128"), "data": "synthetic",
        "config": dict(workload_config(a), launch_shapes=tuned or "library defaults"), "clocks": clk,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(rhs.numel() * 16),
                "d2h_bytes_per_step": int(rhs.numel() * 16), "h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs,
                "how": "double-buffered: the host-to-device copy of the next step's right-hand sides and the "
                       "device-to-host copy of the last step's solutions run on a copy stream beside the solve; "
                       "h2d_gbs / d2h_gbs: one 1-way copy timed on its own"},
        "roofline": roof, "extra": extra,
    }
    if want_error:
        xo, co, ro, ok, ts = sol_job.get()
        pool.close()
        pool.join()
        line["error_vs_oracle"] = {
            "rhs": 0, "rel_l2": float(np.linalg.norm(x0_gpu - xo) / np.linalg.norm(xo)),
            "rel_max": float(np.abs(x0_gpu - xo).max() / np.abs(xo).max()),
            "gpu_cycles": int(cyc[0]), "oracle_cycles": int(co), "oracle_relres": ro, "oracle_converged": ok,
            "oracle_seconds": ts,
            "reference": "the FP64 oracle's solve of the same right-hand side to the same tolerance"}
    elif pool is not None:
        pool.terminate()
    if rank == 0 and world == 1 and a.cpu_sample_cycles > 0:
        cyc_needed = cyc_oracle or max(cyc)
        src = "the oracle's" if cyc_oracle else "the GPU path's (no oracle count stored)"
        tc = oracle_cycle_seconds(a, a.cpu_sample_cycles)
        one = N / (tc * cyc_needed)
        cb = {"value": one, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"{a.cpu_sample_cycles} oracle cycles (FP64, one core) of one right-hand side of the "
                        f"workload, scaled to a whole solve by {src} {cyc_needed} cycles"}
        if a.batch > 1 and not a.krylov and a.cpu_allcore_cycles > 0:
            cores = min(_host_cores(), a.batch)
            with mp.get_context("spawn").Pool(cores) as p2:
                secs = p2.map(_oracle_cycles_job, [(a, q, a.cpu_allcore_cycles) for q in range(cores)])
            allc = sum(N / (t * cyc_needed) for t in secs)
            cb = {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
                  "sample": f"{cores} processes, one per host core, each timing {a.cpu_allcore_cycles} oracle "
                            f"cycles (FP64) of its own right-hand side of the workload side by side; the sum of "
                            f"their rates, each scaled to a whole solve by {src} {cyc_needed} cycles",
                  "single_core": cb}
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def step_traffic(a, what):
    """DRAM bytes of the roofline unit (the fine-level GMRES(3) step, or the
    last FGMRES Arnoldi step) from the committed ncu capture, scaled to this
    run's right-hand sides; None unless the workload is the captured one and
    the hashed kernel sources are unchanged."""
    import hashlib
    name = {4: "traffic_gmres_step_level0.json", 5: "traffic_fgmres_step_level0.json"}.get(what)
    if name is None or a.n != 1024 or a.precision == "fp64":
        return None
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if what == 5 and rec.get("m") != a.krylov:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return rec["dram_bytes_per_rhs"] * a.batch


def run_probe(a):
    """Two solves of the workload capped at a.max_cycles cycles (for ncu captures)."""
    import torch
    import paper_2308_13476_gb300 as hm
    import synth
    torch.cuda.set_device(0)
    h = 1.0 / a.n
    src = synth.source_row(a.n, a.n, h, a.batch) if a.batch > 1 else synth.point_source(a.n, a.n, h)[None]
    rhs = torch.from_numpy(src).cuda()
    kw = {}
    if a.coarse_nodes >= 0:
        kw["coarse_nodes"] = a.coarse_nodes
    if a.coarse_mode >= 0:
        kw["coarse_mode"] = a.coarse_mode
    s = hm.Solver(a.n, a.n, h, a.k, a.beta2, cycle=a.cycle, smoother=a.smoother, nu_pre=a.nu, nu_post=a.nu,
                  precision=a.precision, batch=a.batch, max_cycles=a.max_cycles, **kw)
    for _ in range(2):
        s.solve(rhs, tol=a.tol)
        torch.cuda.synchronize()
    print(json.dumps({"probe": "ok", "kernel_launches": s.counters()[0]}))
    s.close()


def _event_ms(fn, steps):
    """Mean CUDA-event time of fn() over `steps` calls (device synchronised around each)."""
    import torch
    tot = 0.0
    out = None
    for _ in range(steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps, out


def run_absorbing(a):
    """What the second-order absorbing rows buy: a centre point source in a
    homogeneous medium (k = 0.625 n on the unit square, n = --n), solved with
    the first- and the second-order rows, each compared with a reference on
    a domain five times as wide (the same h; first-order rows two domain
    widths away, where the outgoing wave has spread and been absorbed)
    restricted to the unit square: the relative difference is the boundary's
    reflection in the solution.  FP64 path, GMRES(3) V(2,2), tol 1e-10; the
    cycle counts and DOF-solves/s of both rows on the unit square."""
    import torch
    import paper_2308_13476_gb300 as hm
    import synth
    torch.cuda.set_device(0)
    n = a.n if a.n != 1024 else 256
    k = 0.625 * n
    h = 1.0 / n
    N = 5 * n
    big = hm.Solver(N, N, h, k, 1.0 / k, smoother="gmres3", nu_pre=2, nu_post=2, precision="fp64", max_cycles=20000)
    bb = torch.from_numpy(synth.point_source(N, N, h, N // 2, N // 2)).cuda()
    xr, st, cyc_r, _ = big.solve(bb, tol=1e-10)
    if st != hm.MG_OK:
        raise RuntimeError(f"reference solve failed: {hm.STATUS_NAMES[st]}")
    lo = 2 * n   # the unit square's nodes inside the wide domain
    ref = xr[0, lo:lo + n + 1, lo:lo + n + 1].cpu().numpy()
    big.close()
    b = torch.from_numpy(synth.point_source(n, n, h, n // 2, n // 2)).cuda()
    out = {"workload": f"point source, homogeneous medium, {n} x {n} cells, k = {k:g} (kh = 0.625)",
           "unit": "relative difference from the wide-domain reference", "data": "synthetic",
           "reference": f"{N} x {N} cells, same h, source at the centre, first-order rows "
                        f"({int(cyc_r[0])} cycles to 1e-10)", "smoother": "gmres3", "cycle": "V(2,2)", "tol": 1e-10}
    for abc in (1, 2):
        s = hm.Solver(n, n, h, k, 1.0 / k, smoother="gmres3", nu_pre=2, nu_post=2, precision="fp64",
                      max_cycles=20000, abc=abc)
        s.solve(b, tol=1e-10)
        ms, (x, st, cyc, rr) = _event_ms(lambda: s.solve(b, tol=1e-10), a.steps)
        if st != hm.MG_OK:
            raise RuntimeError(f"abc {abc} solve failed: {hm.STATUS_NAMES[st]}")
        u = x[0].cpu().numpy()
        inner = slice(n // 8, n - n // 8 + 1)   # away from the boundary rows themselves
        out[f"abc{abc}"] = {"rel_diff": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
                            "rel_diff_inner": float(np.linalg.norm((u - ref)[inner, inner]) /
                                                    np.linalg.norm(ref[inner, inner])),
                            "cycles": int(cyc[0]), "ms_per_solve": ms,
                            "dof_solves_per_s": (n + 1) ** 2 / (ms / 1e3)}
        s.close()
    out["value"] = out["abc2"]["rel_diff"]
    print(json.dumps(out))


def run_layered(a):
    """Variable-k workload: the seeded layered model (stand-in for the 9.2 x
    3.0 km benchmark model), h = 1500 / (10 f) m, grid 640 x 224 cells at
    10 Hz scaled with f, source at (centre, 2h), GMRES(3) V(2,2),
    beta2 = 1/(k_max L), one right-hand side, mixed and FP64 paths."""
    import torch
    import paper_2308_13476_gb300 as hm
    import synth
    torch.cuda.set_device(0)
    f = a.freq
    h = 1500.0 / (10.0 * f)
    nx, nz = int(round(640 * f / 10)), int(round(224 * f / 10))
    v = synth.layered_velocity(nx, nz, h, seed=11)
    k = 2 * np.pi * f / v
    b = torch.from_numpy(synth.point_source(nx, nz, h, nx // 2, 2)).cuda()
    kd = torch.from_numpy(k).cuda()
    beta2 = 1.0 / (k.max() * nx * h)
    N = (nx + 1) * (nz + 1)
    out = {"workload": f"layered velocity model, {f:g} Hz, {nx} x {nz} cells, h = {h:g} m", "unit": "DOF-solves/s",
           "data": "synthetic", "smoother": "gmres3", "cycle": "V(2,2)", "beta2": beta2, "tol": a.tol, "abc": a.abc}
    for prec in ([a.precision, "fp64"] if not a.no_fp64_line and a.precision != "fp64" else [a.precision]):
        s = hm.Solver(nx, nz, h, kd, beta2, smoother="gmres3", nu_pre=2, nu_post=2, precision=prec,
                      max_cycles=20000, march=a.march, abc=a.abc)
        s.solve(b, tol=a.tol)   # warm-up (graph capture)
        ms, (x, st, cyc, rr) = _event_ms(lambda: s.solve(b, tol=a.tol), a.steps)
        if st != hm.MG_OK:
            raise RuntimeError(f"layered solve failed: {hm.STATUS_NAMES[st]}")
        out[prec] = {"value": N / (ms / 1e3), "cycles": int(cyc[0]), "relres": float(rr[0]), "ms_per_solve": ms}
        s.close()
    out["value"] = out[a.precision]["value"]
    print(json.dumps(out))


def run_two_grid(a):
    """Dense two-grid analysis (mg_two_grid): the four columns of Table conv1
    (Linear / Bezier transfers, A_c on A or on the CSL with beta2 = 0.7) at
    k = 30, kh = 0.625 (49 x 49 grid, N = 2401), one post-smoothing Jacobi
    step, omega = 4.5.  FP64 on CUDA cores; the roofline is the FP64 FMA rate
    (FLOPs of the dense products, the two Gauss-Jordan inverses, the Cholesky
    and the power method)."""
    import torch
    import paper_2308_13476_gb300 as hm
    torch.cuda.set_device(0)
    k = 30.0
    n = int(round(k / 0.625))
    N, Nc = (n + 1) ** 2, (n // 2 + 1) ** 2
    variants = [("linear", 0.0), ("linear", 0.7), ("bezier", 0.0), ("bezier", 0.7)]
    results, ms_all, flops_all = {}, [], 0.0
    for kind, beta2 in variants:
        s = hm.Solver(n, n, 1.0 / n, k, beta2, transfer=kind)
        r = s.two_grid()   # warm-up
        for _ in range(max(0, a.warmup - 1)):
            s.two_grid()
        ms, r = _event_ms(lambda: s.two_grid(), a.steps)
        s.close()
        # complex MACs: Y = A1^-1 R (Nc^2 N), P Y (N^2 Nc), CG (N^3), T0 (N^3), T0^H T0 (N^3), E^H E (N^3),
        # two Gauss-Jordan inverses (2 Nc^3, 2 N^3), Cholesky (N^3 / 6), power method (N^2 per iteration)
        cmac = Nc * Nc * N + N * N * Nc + 4.0 * N ** 3 + 2.0 * Nc ** 3 + 2.0 * N ** 3 + N ** 3 / 6.0 + \
            r["iterations"] * N * N
        flops_all += 8.0 * cmac * a.steps
        ms_all.append(ms)
        results[f"{kind}/{'C' if beta2 else 'A'}"] = {"norm_t0": r["norm_t0"], "hpd": r["hpd"],
                                                       "gamma_ratio": r["gamma_ratio"],
                                                       "power_iterations": r["iterations"], "ms": ms}
    t = sum(ms_all) * a.steps / 1e3
    peak = 1194.0   # measured FP64 FMA rate of this machine's GB300 (GFLOP/s)
    line = {"metric": "two-grid analyses/s (dense T0, ||T0||_2, Gamma~ HPD test and kappa_1; Table conv1, k = 30)",
            "value": len(variants) * a.steps / t, "unit": "analyses/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": sum(ms_all), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": f"MP 2-A, k = {k:g}, {n + 1} x {n + 1} grid (N = {N}), two finest levels",
                       "variants": [f"{kk}/{'C' if b else 'A'}" for kk, b in variants], "nu": 1, "omega": 4.5},
            "roofline": {"bound": "alu", "achieved": flops_all / t / 1e9, "peak": peak, "unit": "GFLOP/s",
                         "frac": flops_all / t / 1e9 / peak, "traffic": None,
                         "kernel": "all kernels of one analysis (FP64 complex GEMM, Gauss-Jordan, Cholesky, power "
                                   "method); peak = FP64 FMA rate measured on this pool"},
            "results": results}
    if a.cpu_sample_cycles > 0:   # the oracle's dense analysis of one variant (Bezier / CSL)
        from oracle import analysis as oan
        t0 = time.perf_counter()
        A, P, R, Ac = oan.two_grid_parts(n, n, 1.0 / n, k, 0.7, coarsen_on="C")
        np.linalg.norm(oan.two_grid_matrix(A, P, R, Ac, 4.5, 1), 2)
        G = oan.gamma_tilde(A, P, R, Ac, 4.5)
        oan.is_hpd(G)
        np.linalg.norm(G, 1) / np.linalg.cond(G, 1)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / tc, "unit": "analyses/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "one oracle analysis (numpy dense SVD, inverse, Cholesky) of the Bezier/CSL "
                                          "variant; numpy's BLAS threads over the host cores"}
    print(json.dumps(line))


def run_ragged(a):
    """Ragged batch: 32 square constant-k problems with interval counts drawn
    in [127, 1023] and rounded to c * 2^m (synth.ragged_sizes, seed 3),
    h = 1/n, k = 0.625 n (kh = 0.625), beta2 = 1/k each, centre source,
    GMRES(3) V(2,2) in one handle; value = all problems' unknowns / time."""
    import torch
    import paper_2308_13476_gb300 as hm
    import synth
    torch.cuda.set_device(0)
    ns = synth.ragged_sizes(32, 3)
    probs = [(n, n, 1.0 / n, 0.625 * n) for n in ns]
    rhs = [torch.from_numpy(synth.point_source(n, n, 1.0 / n)).cuda() for n in ns]
    rs = hm.RaggedSolver(probs, [1.0 / p[3] for p in probs], smoother="gmres3", nu_pre=2, nu_post=2,
                         precision=a.precision, max_cycles=20000, march=a.march, flat=a.flat)
    rs.solve(rhs, tol=a.tol)
    ms, (xs, st, cyc, rr) = _event_ms(lambda: rs.solve(rhs, tol=a.tol), a.steps)
    if st != hm.MG_OK:
        raise RuntimeError(f"ragged solve failed: {hm.STATUS_NAMES[st]}")
    rs.close()
    N = sum((n + 1) ** 2 for n in ns)
    print(json.dumps({"workload": "ragged batch of 32 constant-k problems, kh = 0.625", "unit": "DOF-solves/s",
                      "value": N / (ms / 1e3), "ms_per_solve": ms, "unknowns_total": N, "sizes": ns,
                      "cycles": [int(c) for c in cyc], "max_relres": float(max(rr)), "precision": a.precision,
                      "flat": a.flat,
                      "data": "synthetic", "smoother": "gmres3", "cycle": "V(2,2)", "tol": a.tol}))


def run_gradient(a):
    """Adjoint gradient: L = 1/2 sum_s ||P u_s - d_s||^2, 16 sources and 256
    receivers on the first interior row of a 1025^2 grid, 15 Hz, squared
    slowness m = m0 (1 + 0.1 rho) with m0 = 1/2000^2 and rho a smooth seeded
    field, h = 0.625 * 1800 / (2 pi 15) m; data from the unperturbed model;
    one evaluation = batched forward solve + batched adjoint solve + gradient
    kernel through torch.autograd."""
    import torch
    import synth
    from paper_2308_13476_gb300 import autograd as hag
    torch.cuda.set_device(0)
    n, nsrc, nrec = 1024, 16, 256
    omega = 2 * np.pi * 15.0
    h = 0.625 * 1800.0 / omega
    m0 = np.full((n + 1, n + 1), 1.0 / 2000.0**2)
    m = m0 * (1 + 0.1 * synth.smooth_perturbation(n, n, 7, sigma_nodes=20.0))
    src = torch.from_numpy(synth.source_row(n, n, h, nsrc)).cuda()
    cols = np.linspace(1, n - 1, nrec).round().astype(np.int64)
    rec = torch.from_numpy((n - 1) * (n + 1) + cols).cuda()
    grid = (n, n, h, omega)
    kw = dict(tol=a.tol, smoother="gmres3", nu_pre=2, nu_post=2, precision=a.precision, march=a.march)
    # data: the unperturbed model's receiver traces (the misfit with zero data returns them)
    m0t = torch.from_numpy(m0).cuda()
    from paper_2308_13476_gb300 import Solver
    k0 = (omega * torch.sqrt(m0t)).contiguous()
    s0 = Solver(n, n, h, k0, 1.0 / (float(k0.max()) * n * h), batch=nsrc, smoother="gmres3", nu_pre=2, nu_post=2,
                precision=a.precision)
    u0, st, _, _ = s0.solve(src, tol=1e-8)
    s0.close()
    data = u0.reshape(nsrc, -1)[:, rec].contiguous()
    mt = torch.from_numpy(m).cuda()

    def evaluate():
        mm = mt.clone().requires_grad_(True)
        L = hag.misfit(mm, src, rec, data, grid, **kw)
        L.backward()
        return float(L.detach()), mm.grad

    evaluate()
    ms, (L, g) = _event_ms(evaluate, a.steps)
    N = (n + 1) ** 2
    print(json.dumps({"workload": "adjoint gradient, 16 sources, 256 receivers, 1025^2, 15 Hz",
                      "unit": "gradient evaluations/s", "value": 1e3 / ms, "ms_per_evaluation": ms,
                      "dof_solves_per_s": 2 * nsrc * N / (ms / 1e3), "misfit": L,
                      "grad_norm": float(g.norm()), "precision": a.precision, "data": "synthetic",
                      "smoother": "gmres3", "cycle": "V(2,2)", "tol": a.tol}))


def run_sweep(a):
    """Constant-k sweep (synth.sweep_points): wavenumber at kh = 0.625,
    h-refinement at k = 100, smoothing steps, V and W, shifts; one centre
    source per point, relative residual 1e-6 (cap 400 cycles), the mixed and
    the FP64 path.  Each point: one untimed solve (graph capture), one timed
    solve (CUDA events on the library's stream).  The oracle's count for
    each point is read from oracle/sweep_cycles.json (written by
    python -m oracle.sweep_cycles)."""
    import torch
    import paper_2308_13476_gb300 as hm
    import synth
    torch.cuda.set_device(0)
    S = torch.cuda.Stream()
    try:
        with open(os.path.join(ROOT, "oracle", "sweep_cycles.json")) as f:
            oracle_counts = json.load(f)
    except OSError:
        oracle_counts = {}
    rows = []
    for p in synth.sweep_points():
        n, k = p["n"], p["k"]
        h = 1.0 / n
        b = torch.from_numpy(synth.point_source(n, n, h)).cuda()
        row = dict(p, oracle_cycles=oracle_counts.get(synth.sweep_key(p)))
        for prec in ("mixed", "fp64"):
            s = hm.Solver(n, n, h, k, p["beta2"], cycle=p["cycle"], smoother=p["smoother"], nu_pre=p["nu"],
                          nu_post=p["nu"], precision=prec, max_cycles=400, stream=S)
            s.solve(b, tol=a.tol)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(S)
            x, st, cyc, rr = s.solve(b, tol=a.tol)
            e1.record(S)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            status = {hm.MG_OK: "ok", hm.MG_EMAXIT: "none", hm.MG_EDIVERGED: "div"}.get(st, str(st))
            row[prec] = {"cycles": int(cyc[0]), "status": status, "relres": float(rr[0]), "ms": ms,
                         "dof_solves_per_s": (n + 1) ** 2 / (ms / 1e3) if status == "ok" else None}
            s.close()
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"workload": "constant-k sweep (MP 2-A, centre source, one right-hand side): k at kh = 0.625, "
                                  "h-refinement at k = 100, nu, V/W, shifts; mixed and FP64 paths",
                      "unit": "DOF-solves/s", "tol": a.tol, "max_cycles": 400, "data": "synthetic",
                      "points": rows}))


def main():
    a = parse()
    if a.probe:
        run_probe(a)
        return
    if a.workload != "batched":
        if a.impl == "reference":   # the oracle arm times the headline workload only
            if dist_env()[0] == 0:
                print(json.dumps({"impl": "reference", "unavailable": f"the oracle reference arm covers the batched "
                                  f"workload (the bench headline), not the {a.workload} line"}))
            return
        {"layered": run_layered, "ragged": run_ragged, "gradient": run_gradient, "absorbing": run_absorbing,
         "two-grid": run_two_grid, "sweep": run_sweep}[a.workload](a)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
