"""A small autotuner for the launch shapes of a solve.

It times a few cycles of the actual workload for each candidate setting of
the library's shape options, with CUDA events, keeps the fastest per cycle,
and caches the choice in a JSON file keyed by GPU name and problem shape
(grid, batch, precision, smoother, cycle).  The search runs in stages, each
over the product of a few options with the earlier stages' choice fixed:
first the node kernels' rows per thread (tile_rows), the size below which
levels run inside one launch (coarse_nodes) and how that launch is organised
(coarse_mode: one CTA per RHS or one cooperative grid); then the GMRES(3)
kernels (march: row and column marches by level size, or everywhere) and the
chunk height of the Kronecker-level column marches (kron_chunk: 0 = chosen
from the kernels' occupancy, else rows per chunk).
"""
import itertools
import json
import os
import time

DEFAULT_CANDIDATES = {
    "tile_rows": [0, 1, 2, 4],
    "coarse_nodes": [300, 1100, 5000],
    "coarse_mode": [0, 1],
}
DEFAULT_STAGES = [
    DEFAULT_CANDIDATES,
    {"march": [-1, 1], "kron_chunk": [0, 16, 32, 48, 64]},
]


def cache_key(gpu, nx, ny, batch, precision, smoother, cycle, nu):
    return f"{gpu}|{nx}x{ny}|B{batch}|{precision}|{smoother}|{cycle}({nu},{nu})"


def load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(path, cache):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def best_of(results):
    """The candidate with the lowest time per cycle (ties: first)."""
    return min(results, key=lambda r: r["ms_per_cycle"])


def candidates(space=None):
    space = space or DEFAULT_CANDIDATES
    keys = sorted(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        yield dict(zip(keys, vals))


def tune(nx, ny, h, k, beta2, rhs, smoother="gmres3", cycle="V", nu=2, precision="mixed", cycles=4,
         space=None, cache_path=None, reps=2, stages=None):
    """Time `cycles` cycles for every candidate (best of `reps`) and return
    (best settings, all results).  rhs: complex128 CUDA tensor (B, ny+1, nx+1).
    `space` (one dict of option -> values) searches that product alone;
    otherwise `stages` (default DEFAULT_STAGES) are searched one after the
    other, each with the earlier stages' best settings fixed."""
    import torch

    from . import Solver

    batch = rhs.shape[0]
    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, nx, ny, batch, precision, smoother, cycle, nu)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache:
        return cache[key]["best"], cache[key]["results"]
    results = []
    fixed = {}
    for stage in ([space] if space else (stages or DEFAULT_STAGES)):
        stage_results = []
        for cand in candidates(stage):
            cfg = dict(fixed, **cand)
            s = Solver(nx, ny, h, k, beta2, cycle=cycle, smoother=smoother, nu_pre=nu, nu_post=nu,
                       precision=precision, batch=batch, max_cycles=cycles, **cfg)
            s.solve(rhs, tol=1e-300)            # graph capture and warm-up
            best = float("inf")
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                s.solve(rhs, tol=1e-300)
                b.record()
                torch.cuda.synchronize()
                best = min(best, a.elapsed_time(b))
            s.close()
            stage_results.append(dict(cfg, ms_per_cycle=best / cycles))
        results += stage_results
        fixed = {k: v for k, v in best_of(stage_results).items() if k != "ms_per_cycle"}
    if cache_path:
        cache[key] = {"best": fixed, "results": results, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
        store_cache(cache_path, cache)
    return fixed, results
