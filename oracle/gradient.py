"""Adjoint-state gradient of a receiver misfit with respect to squared slowness.

Test infrastructure only (see ``oracle/__init__``).

The operator is the MP 2-B operator of Sec. 2 with k(x)^2 = w_f^2 m(x)
(angular frequency w_f, squared slowness m), so only the diagonal of A
depends on m:  A_pp = w_p (4/h^2 - w_f^2 m_p) - i b_p w_f sqrt(m_p) / h, with
w_p the boundary row weight (1, 1/2, 1/4) and b_p = 1 on boundary nodes,
0 inside (the ghost-eliminated, row-scaled Sommerfeld rows of
``oracle.problem``).  For the misfit

    L(m) = 1/2 sum_s || S u_s - d_s ||^2,   A(m) u_s = f_s,

(S samples the receiver nodes) the adjoint-state method gives

    dL/dm_p = - Re sum_s conj(lam_s[p]) (dA_pp/dm_p) u_s[p],
    A^H lam_s = S^T (S u_s - d_s),
    dA_pp/dm_p = - w_p w_f^2 - i b_p w_f / (2 h sqrt(m_p)).

All solves here are direct (scipy sparse LU).
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import problem


def operator(nx, ny, h, m, omega_f):
    return problem.helmholtz_matrix(nx, ny, h, omega_f * np.sqrt(m), 0.0)


def diag_derivative(nx, ny, h, m, omega_f):
    """dA_pp / dm_p on the grid, shape (ny+1, nx+1)."""
    w = problem.boundary_weights(nx, ny)
    b = np.zeros((ny + 1, nx + 1))
    b[0, :] = b[-1, :] = 1.0
    b[:, 0] = b[:, -1] = 1.0
    return -w * omega_f**2 - 1j * b * omega_f / (2.0 * h * np.sqrt(m))


def forward(nx, ny, h, m, omega_f, F):
    """Solve A(m) U = F for the columns of F (one source per column)."""
    lu = spla.splu(operator(nx, ny, h, m, omega_f).tocsc())
    return lu.solve(np.asarray(F, dtype=np.complex128)), lu


def misfit(nx, ny, h, m, omega_f, F, rec, D):
    U, _ = forward(nx, ny, h, m, omega_f, F)
    res = U[rec, :] - D
    return 0.5 * float(np.sum(np.abs(res) ** 2))


def gradient(nx, ny, h, m, omega_f, F, rec, D):
    """dL/dm as an (ny+1, nx+1) array, by the adjoint-state formula above."""
    U, lu = forward(nx, ny, h, m, omega_f, F)
    res = U[rec, :] - D
    G = np.zeros_like(U)
    G[rec, :] = res
    lam = lu.solve(G, trans="H")                 # A^H lam = S^T res
    dA = diag_derivative(nx, ny, h, m, omega_f).ravel()
    g = -np.real(np.sum(np.conj(lam) * dA[:, None] * U, axis=1))
    return g.reshape(ny + 1, nx + 1)
