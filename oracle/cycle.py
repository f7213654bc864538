"""Multigrid cycle and outer iteration.

Test infrastructure only (see ``oracle/__init__``).

Sec. 3 defines the coarse-grid correction I - P A_c^{-1} R A and the
smoother; the cycle applies them recursively with gamma = 1 (V-cycle) or
gamma = 2 (W-cycle) recursive calls per level (Table cons1 caption).
Sec. 5: stop when the relative residual reaches the tolerance (1e-5 in the
paper), coarsening until N_c < 10 with a direct solve there.

Readings: nu_pre sweeps before and nu_post after the coarse correction on
every level, the same smoother on every level; x_0 = 0; the stopping test is
the 2-norm of the fine residual divided by ||b||, checked after each cycle;
on the level just above the coarsest one the coarse problem is solved once
(repeating an exact solve gamma times gives the same correction).
"""
from dataclasses import dataclass

import numpy as np

from . import hierarchy, smoothers


@dataclass
class CycleOptions:
    gamma: int = 1            # 1 = V-cycle, 2 = W-cycle
    smoother: str = "jacobi"  # "jacobi" | "gmres3"
    nu_pre: int = 1
    nu_post: int = 1
    omega: float = 4.5        # X = omega * diag(A), Sec. 3 / Sec. 5
    fine_diag: str = "A"      # "C": fine-level Jacobi with X = omega diag(C) (an alternative reading)


def mg_cycle(H, l, x, b, opt):
    """One cycle on level ``l`` for A_l x = b; returns the new x."""
    A = H.A[l]
    if l == H.nlevels - 1:
        return hierarchy.coarsest_solve(H, b)
    d = H.C0.diagonal() if (l == 0 and opt.fine_diag == "C") else None
    x = smoothers.smooth(A, x, b, opt.smoother, opt.nu_pre, opt.omega, d)
    r = b - A @ x
    rc = H.R[l] @ r
    if l + 1 == H.nlevels - 1:
        ec = hierarchy.coarsest_solve(H, rc)
    else:
        ec = np.zeros_like(rc)
        for _ in range(opt.gamma):
            ec = mg_cycle(H, l + 1, ec, rc, opt)
    x = x + H.P[l] @ ec
    x = smoothers.smooth(A, x, b, opt.smoother, opt.nu_post, opt.omega, d)
    return x


@dataclass
class SolveResult:
    x: np.ndarray
    cycles: int
    relres: float
    history: list
    iterates: list
    converged: bool
    diverged: bool


def mg_solve(H, b, tol, opt, max_cycles=10000, x0=None, keep_iterates=False,
             diverge_at=1e6, norm_w=None):
    """Repeat cycles from x0 (default 0) until ||b - A x|| / ||b|| <= tol.
    ``norm_w`` (an alternative reading of the stopping test): the norms are
    taken of the residual and of b divided node by node by these weights,
    e.g. the boundary row weights, to test the unscaled rows' residual."""
    A = H.A[0]
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    wn = (lambda v: np.linalg.norm(v)) if norm_w is None else (lambda v: np.linalg.norm(v / norm_w))
    nb = wn(b)
    if nb == 0.0:
        return SolveResult(np.zeros_like(b), 0, 0.0, [], [], True, False)
    hist, its = [], []
    relres = wn(b - A @ x) / nb
    if relres <= tol:
        return SolveResult(x, 0, relres, hist, its, True, False)
    for c in range(1, max_cycles + 1):
        x = mg_cycle(H, 0, x, b, opt)
        relres = wn(b - A @ x) / nb
        hist.append(relres)
        if keep_iterates:
            its.append(x.copy())
        if not np.isfinite(relres) or relres > diverge_at:
            return SolveResult(x, c, relres, hist, its, False, True)
        if relres <= tol:
            return SolveResult(x, c, relres, hist, its, True, False)
    return SolveResult(x, max_cycles, relres, hist, its, False, False)
