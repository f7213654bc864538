"""Oracle cycle counts of the constant-k sweep (``synth.sweep_points``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Writes
``oracle/sweep_cycles.json``: for every sweep point, the number of cycles
the oracle's solve of the centre point source takes to relative residual
1e-6 from x = 0 ("div" when it diverges, "none" when it has not converged
within MAXC cycles), keyed by ``synth.sweep_key``.  The GPU sweep
(``bench.py --workload sweep``) prints its own counts beside these.

    python -m oracle.sweep_cycles            (about 30 minutes on 8 cores)

This module only calls ``oracle/`` and the seeded generators in ``synth/``.
"""
import json
import multiprocessing as mp
import os
import time

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_cycles.json")
MAXC = 400
TOL = 1e-6


def count(p):
    import synth
    from . import cycle as oc
    from . import hierarchy as oh
    t0 = time.perf_counter()
    n = p["n"]
    h = 1.0 / n
    H = oh.build_hierarchy(n, n, h, p["k"], p["beta2"])
    b = synth.point_source(n, n, h).ravel()
    opt = oc.CycleOptions(1 if p["cycle"] == "V" else 2, p["smoother"], p["nu"], p["nu"], 4.5)
    r = oc.mg_solve(H, b, TOL, opt, max_cycles=MAXC)
    c = r.cycles if r.converged else ("div" if r.diverged else "none")
    return synth.sweep_key(p), c, time.perf_counter() - t0


def main():
    import synth
    pts = sorted(synth.sweep_points(), key=lambda p: -p["n"] * (2 if p["cycle"] == "W" else 1))
    table = {}
    if os.path.exists(PATH):
        with open(PATH) as f:
            table = json.load(f)
    todo = [p for p in pts if synth.sweep_key(p) not in table]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        for key, c, t in pool.imap_unordered(count, todo):
            table[key] = c
            print(f"{key}: {c} ({t:.0f} s)", flush=True)
            with open(PATH, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
