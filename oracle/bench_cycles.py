"""Oracle cycle counts of the bench workloads.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  The reference arm and
the CPU baseline of ``bench.py`` time a few oracle cycles and scale them to a
whole solve; the number of cycles a solve takes comes from here: the oracle's
own solve of the workload's first right-hand side to the bench tolerance,
written to ``oracle/bench_cycles.json`` under the key
``"{k:g}/{n}/{smoother}/{cycle}{nu}/{beta2:g}"``, with ``"/fgmres{m}"``
appended for the FGMRES(m) outer loop (``oracle.krylov``; the count is then
preconditioner applications) and ``"/linear"`` for linear-interpolation
transfers.

    python -m oracle.bench_cycles --k 300 --n 1024 --batch 64
    python -m oracle.bench_cycles --k 300 --n 1024 --smoother jacobi --nu 1 --krylov 20

This module only calls ``oracle/`` and the seeded generators in ``synth/``.
"""
import argparse
import json
import os
import time

from . import cycle as oc
from . import hierarchy as oh
from . import krylov as okr

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_cycles.json")


def key(k, n, smoother, cycle, nu, beta2, krylov=0, transfer="bezier"):
    return (f"{k:g}/{n}/{smoother}/{cycle}{nu}/{beta2:g}" + (f"/fgmres{krylov}" if krylov else "") +
            ("/linear" if transfer == "linear" else ""))


def count(k, n, smoother="gmres3", cycle="V", nu=2, beta2=None, batch=64, tol=1e-6, krylov=0, transfer="bezier"):
    """Cycles the oracle needs for the first right-hand side of the workload."""
    import synth
    if beta2 is None:
        beta2 = 1.0 / k if smoother == "gmres3" else 0.7
    h = 1.0 / n
    b = (synth.source_row(n, n, h, batch)[0] if batch > 1 else synth.point_source(n, n, h)).ravel()
    H = oh.build_hierarchy(n, n, h, k, beta2, kind=transfer)
    opt = oc.CycleOptions(1 if cycle == "V" else 2, smoother, nu, nu, 4.5)
    res = okr.fgmres_solve(H, b, tol, opt, krylov) if krylov else oc.mg_solve(H, b, tol, opt)
    return key(k, n, smoother, cycle, nu, beta2, krylov, transfer), res.cycles, res.converged


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--k", type=float, default=300.0)
    p.add_argument("--n", type=int, default=1024)
    p.add_argument("--smoother", default="gmres3")
    p.add_argument("--cycle", default="V")
    p.add_argument("--nu", type=int, default=2)
    p.add_argument("--beta2", type=float, default=None)
    p.add_argument("--batch", type=int, default=64)
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--krylov", type=int, default=0, help="m > 0: FGMRES(m) around the cycle")
    p.add_argument("--transfer", default="bezier", choices=["bezier", "linear"])
    a = p.parse_args()
    t0 = time.perf_counter()
    kk, cyc, ok = count(a.k, a.n, a.smoother, a.cycle, a.nu, a.beta2, a.batch, a.tol, a.krylov, a.transfer)
    if not ok:
        raise SystemExit(f"oracle did not converge for {kk}")
    table = {}
    if os.path.exists(PATH):
        with open(PATH) as f:
            table = json.load(f)
    table[kk] = cyc
    with open(PATH, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(f"{kk}: {cyc} cycles ({time.perf_counter() - t0:.0f} s)")


if __name__ == "__main__":
    main()
