"""Smoothers: weighted Jacobi and GMRES(3).

Test infrastructure only (see ``oracle/__init__``).

Weighted Jacobi, Sec. 3: S_JAC = I - X^{-1} A with X = omega * Lambda_A,
Lambda_A the diagonal of A.  One sweep is x <- x + X^{-1} (b - A x).  In
this convention omega = 4.5 (Sec. 5) means a step of (1/4.5) D^{-1} r.

GMRES(3), Sec. 5.3: each smoothing step runs three GMRES iterations from
the current iterate (a polynomial smoother).  Readings: no preconditioner,
Hermitian inner products, Arnoldi with modified Gram-Schmidt, the small
least-squares problem min ||beta e_1 - Hbar y|| solved exactly, and a step
ends early when the new Arnoldi vector vanishes (h_{j+1,j} <= 1e-14 beta).
"""
import numpy as np


def jacobi(A, x, b, omega, nu, diag=None):
    """``nu`` weighted-Jacobi sweeps x <- x + (omega diag A)^{-1} (b - A x).
    ``diag`` replaces diag A in X (an alternative reading kept for the
    comparison of readings: the diagonal of the shifted operator)."""
    X = omega * (A.diagonal() if diag is None else diag)
    for _ in range(nu):
        x = x + (b - A @ x) / X
    return x


def gmres_step(A, x, b, m=3, breakdown=1e-14):
    """One GMRES(m) cycle from x (m = 3 in the paper).  Returns the new x."""
    r0 = b - A @ x
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return x
    n = r0.shape[0]
    V = np.zeros((n, m + 1), dtype=np.complex128)
    Hbar = np.zeros((m + 1, m), dtype=np.complex128)
    V[:, 0] = r0 / beta
    steps = m
    for j in range(m):
        w = A @ V[:, j]
        for i in range(j + 1):            # modified Gram-Schmidt
            Hbar[i, j] = np.vdot(V[:, i], w)
            w = w - Hbar[i, j] * V[:, i]
        Hbar[j + 1, j] = np.linalg.norm(w)
        if Hbar[j + 1, j].real <= breakdown * beta:
            steps = j + 1
            break
        V[:, j + 1] = w / Hbar[j + 1, j]
    rhs = np.zeros(steps + 1, dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(Hbar[: steps + 1, :steps], rhs, rcond=None)[0]
    return x + V[:, :steps] @ y


def gmres(A, x, b, nu, m=3):
    """``nu`` GMRES(m) smoothing steps."""
    for _ in range(nu):
        x = gmres_step(A, x, b, m)
    return x


def smooth(A, x, b, kind, nu, omega, diag=None):
    if nu <= 0:
        return x
    if kind == "jacobi":
        return jacobi(A, x, b, omega, nu, diag)
    if kind == "gmres3":
        return gmres(A, x, b, nu, 3)
    raise ValueError(kind)
