"""Writes ``jacobi_readings.json``: the oracle's omega-Jacobi cycle counts
under each candidate reading of the points the paper leaves open, beside the
counts the paper prints (Sec. 5.1.1 Table tabhind, Sec. 5.1.2 Table cons1).

    python tests/golden/jacobi_readings.py          (about 3 minutes on 8 cores)

Only ``oracle/`` and ``synth/`` are called.  Each reading changes one point
of the default reading (the hierarchy and cycle of ``oracle/``) and keeps
the rest:

* the edge rule of Eq. (xex): linear extrapolation instead of zero extension;
* the boundary rows: unscaled ghost-eliminated rows, or first-order one-sided
  absorbing-condition rows as their own equations;
* the unknowns: interior nodes only, boundary nodes eliminated by the
  first-order one-sided absorbing condition;
* the smoother's diagonal on the fine level: that of the shifted operator;
* the stopping test: the residual of the unscaled rows;
* the meaning of nu: post-smoothing only (V(0, nu)), or nu steps in total
  split over pre- and post-smoothing;
* omega: 3 and 2 (Sec. 4 puts the best omega in [2, 4.5]).

A count is the number of V-cycles to relative residual 1e-5 from x = 0 with
the centre point source, or "div" (relative residual above 1e6) or "none"
(no convergence within MAXC cycles).
"""
import json
import multiprocessing as mp
import os
import sys

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")     # one core per worker process

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

MAXC = 1200
TOL = 1e-5

# name -> (hierarchy kwargs, cycle-option overrides, split rule, stopping-norm rule)
READINGS = {
    "default": ({}, {}, "pre+post", "scaled"),
    "edge_inject": ({"edge": "inject"}, {}, "pre+post", "scaled"),
    "rows_unscaled": ({"rows": "unscaled"}, {}, "pre+post", "scaled"),
    "rows_bc1": ({"rows": "bc1"}, {}, "pre+post", "scaled"),
    "grid_interior": ({"grid": "interior"}, {}, "pre+post", "scaled"),
    "fine_diag_C": ({}, {"fine_diag": "C"}, "pre+post", "scaled"),
    "norm_unscaled": ({}, {}, "pre+post", "unscaled"),
    "post_only": ({}, {}, "post", "scaled"),
    "nu_total": ({}, {}, "total", "scaled"),
    "omega_3": ({}, {"omega": 3.0}, "pre+post", "scaled"),
    "omega_2": ({}, {"omega": 2.0}, "pre+post", "scaled"),
}

# (table, k, n, nu, paper's V-cycle count)
def paper_cases():
    cases = []
    for line in open(os.path.join(HERE, "table_tabhind.txt")):
        f = line.split("#")[0].split()
        if not f:
            continue
        p = int(f[0])
        if p not in (6, 7):
            continue
        for kk, vals in ((15.0, f[1:4]), (30.0, f[4:7])):
            for nu, v in zip((1, 2, 4), vals):
                cases.append(("tabhind", kk, 2**p, nu, int(v)))
    for line in open(os.path.join(HERE, "table_cons1.txt")):
        f = line.split("#")[0].split()
        if not f:
            continue
        nu = int(f[0])
        if nu in (4, 8):
            cases.append(("cons1", 50.0, 80, nu, int(f[1])))
        if nu == 4:
            cases.append(("cons1", 100.0, 160, nu, int(f[3])))
    return cases


def count(reading, k, n, nu):
    from oracle import cycle as oc
    from oracle import hierarchy as oh
    from oracle import problem as op
    hk, ok, split, norm = READINGS[reading]
    h = 1.0 / n
    H = oh.build_hierarchy(n, n, h, k, 0.7, **hk)
    if hk.get("grid") == "interior":
        b = np.zeros((n - 1) ** 2, dtype=np.complex128)
        b[(n // 2 - 1) * (n - 1) + (n // 2 - 1)] = 1.0 / h**2
    else:
        b = op.point_source_rhs(n, n, h, n // 2, n // 2)
    pre, post = {"pre+post": (nu, nu), "post": (0, nu), "total": ((nu + 1) // 2, nu // 2)}[split]
    opt = oc.CycleOptions(1, "jacobi", pre, post, ok.get("omega", 4.5), ok.get("fine_diag", "A"))
    w = op.boundary_weights(n, n).ravel() if norm == "unscaled" else None
    r = oc.mg_solve(H, b, TOL, opt, max_cycles=MAXC, norm_w=w)
    return r.cycles if r.converged else ("div" if r.diverged else "none")


def _job(args):
    reading, case = args
    return reading, case, count(reading, case[1], case[2], case[3])


def main():
    cases = paper_cases()
    jobs = [(r, c) for r in READINGS for c in cases]
    jobs.sort(key=lambda j: -j[1][2])            # largest grids first
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        results = pool.map(_job, jobs, chunksize=1)
    table = {"tol": TOL, "max_cycles": MAXC, "beta2": 0.7, "smoother": "jacobi", "cycle": "V",
             "cases": [{"table": c[0], "k": c[1], "n": c[2], "nu": c[3], "paper": c[4]} for c in cases],
             "counts": {r: [None] * len(cases) for r in READINGS}}
    for reading, case, cnt in results:
        table["counts"][reading][cases.index(case)] = cnt
    with open(os.path.join(HERE, "jacobi_readings.json"), "w") as f:
        json.dump(table, f, indent=1)
    for r in READINGS:
        print(f"{r:14s}", table["counts"][r])
    print(f"{'paper':14s}", [c[4] for c in cases])


if __name__ == "__main__":
    main()
