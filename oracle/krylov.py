"""The multigrid cycle as a preconditioner of an outer Krylov iteration.

Test infrastructure only (see ``oracle/__init__``).

Sec. 1 of the paper recalls the common use of multigrid: one cycle as an
approximate inverse inside a Krylov method such as GMRES, and the closing
section calls that combination the industry standard.  Here the cycle of this
package (the paper's stand-alone method, ``cycle.mg_cycle`` from a zero
initial guess) is the right preconditioner of a restarted flexible GMRES,
FGMRES(m) (Saad, SIAM J. Sci. Comput. 14 (1993)); "flexible" because a cycle
with GMRES(3) smoothing is not a fixed linear operator, so the preconditioned
vectors z_j are kept.

One restart cycle from x:
    r = b - A x, beta = ||r||, v_0 = r / beta
    for j = 0 .. m-1:
        z_j = M(v_j)                      (one multigrid cycle on A e = v_j)
        w = A z_j
        h_ij = <v_i, w>, w -= h_ij v_i     (modified Gram-Schmidt, i <= j)
        h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
        Givens rotations on column j of Hbar and on g = beta e_1;
        |g_{j+1}| is the residual norm of the best x + Z_{j+1} y
        stop the cycle when |g_{j+1}| / ||b|| <= tol or h_{j+1,j} <= 1e-14 beta
    x += Z_k y, y the solution of the k x k triangular system
Readings (the paper gives no Krylov details): x_0 = 0; "cycles" counts the
preconditioner applications, so that it compares with the stand-alone count;
the solve stops when the true relative residual at a restart is at or below
tol (the estimate only ends a restart cycle early).
"""
from dataclasses import dataclass

import numpy as np

from . import cycle as mgc


@dataclass
class FgmresResult:
    x: np.ndarray
    cycles: int          # preconditioner applications (= Arnoldi steps)
    restarts: int
    relres: float        # true relative residual of x
    history: list        # |g_{j+1}| / ||b|| after every Arnoldi step
    converged: bool


def _givens(a, b):
    """(c, s) with c real >= 0 and [[c, s], [-conj(s), c]] [a, b]^T = [r, 0]^T."""
    na, nb = abs(a), abs(b)
    nr = np.hypot(na, nb)
    if nr == 0.0:
        return 1.0, 0.0
    if na == 0.0:
        return 0.0, np.conj(b) / nb
    return na / nr, (a / na) * np.conj(b) / nr


def fgmres_cycle(A, precond, x, b, m, tol, nb, breakdown=1e-14):
    """One FGMRES(m) restart cycle from x.  Returns (x, steps, history, Z)."""
    r0 = b - A @ x
    beta = np.linalg.norm(r0)
    n = b.shape[0]
    V = np.zeros((n, m + 1), dtype=np.complex128)
    Z = np.zeros((n, m), dtype=np.complex128)
    Hbar = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    V[:, 0] = r0 / beta
    hist = []
    k = 0
    for j in range(m):
        Z[:, j] = precond(V[:, j])
        w = A @ Z[:, j]
        for i in range(j + 1):
            Hbar[i, j] = np.vdot(V[:, i], w)
            w = w - Hbar[i, j] * V[:, i]
        Hbar[j + 1, j] = np.linalg.norm(w)
        brk = Hbar[j + 1, j].real <= breakdown * beta
        if not brk:
            V[:, j + 1] = w / Hbar[j + 1, j]
        for i in range(j):       # earlier rotations on the new column
            a, bb = Hbar[i, j], Hbar[i + 1, j]
            Hbar[i, j] = cs[i] * a + sn[i] * bb
            Hbar[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * bb
        cs[j], sn[j] = _givens(Hbar[j, j], Hbar[j + 1, j])
        Hbar[j, j] = cs[j] * Hbar[j, j] + sn[j] * Hbar[j + 1, j]
        Hbar[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        hist.append(abs(g[j + 1]) / nb)
        if brk or abs(g[j + 1]) / nb <= tol:
            break
    y = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - Hbar[i, i + 1:k] @ y[i + 1:k]) / Hbar[i, i]
    return x + Z[:, :k] @ y, k, hist, Z[:, :k]


def fgmres_solve(H, b, tol, opt, m, max_cycles=10000, x0=None):
    """FGMRES(m) on A_0 x = b with one multigrid cycle (options ``opt``,
    zero initial guess) as the right preconditioner."""
    A = H.A[0]
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    if nb == 0.0:
        return FgmresResult(np.zeros_like(b), 0, 0, 0.0, [], True)

    def precond(v):
        return mgc.mg_cycle(H, 0, np.zeros_like(v), v, opt)

    cycles, restarts, hist = 0, 0, []
    while True:
        relres = np.linalg.norm(b - A @ x) / nb
        if relres <= tol:
            return FgmresResult(x, cycles, restarts, relres, hist, True)
        if cycles >= max_cycles or not np.isfinite(relres):
            return FgmresResult(x, cycles, restarts, relres, hist, False)
        x, k, h, _ = fgmres_cycle(A, precond, x, b, min(m, max_cycles - cycles), tol, nb)
        cycles += k
        restarts += 1
        hist += h
