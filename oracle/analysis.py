"""Dense two-grid analysis (small grids only).

Test infrastructure only (see ``oracle/__init__``).

Sec. 3, Eq. (tgi1): with post-smoothing only, the two-grid iteration matrix
is T0 = (I - P A_c^{-1} R A)(I - X^{-1} A), X = omega * diag(A).  Table conv1
reports ||T0||_2 with A_c built on A or on the CSL C.  Definition def2s:
D~ = X^{-1} + P A_c^{-1} R and Gamma~ = A^H D~^H + D~ A - A^H D~^H D~ A;
Table conv1 marks whether Gamma~ is Hermitian positive definite and Table
opt1 reports ||Gamma~||_1 / kappa_1(Gamma~).
"""
import numpy as np

from . import problem, transfer


def two_grid_parts(nx, ny, h, k, beta2, kind="bezier", edge="zero", coarsen_on="C"):
    A = problem.helmholtz_matrix(nx, ny, h, k, 0.0).toarray()
    M = A if coarsen_on == "A" else problem.helmholtz_matrix(nx, ny, h, k, beta2).toarray()
    P = transfer.prolongation(nx, ny, kind, edge).toarray()
    R = transfer.restriction(nx, ny, kind, edge).toarray()
    Ac = R @ M @ P
    return A, P, R, Ac


def two_grid_matrix(A, P, R, Ac, omega, nu=1):
    """T0 = (I - P Ac^{-1} R A)(I - X^{-1} A)^nu, Eq. (tgi1) with nu sweeps.

    As an error propagator this applies the sweeps first and the coarse-grid
    correction second (the paper calls the sweep a post-smoothing step)."""
    n = A.shape[0]
    I = np.eye(n)
    X = omega * np.diag(A)
    S = I - A / X[:, None]
    CGC = I - P @ np.linalg.solve(Ac, R @ A)
    return CGC @ np.linalg.matrix_power(S, nu)


def two_grid_norm(nx, ny, h, k, beta2, omega=4.5, kind="bezier", edge="zero",
                  coarsen_on="C", nu=1):
    A, P, R, Ac = two_grid_parts(nx, ny, h, k, beta2, kind, edge, coarsen_on)
    return np.linalg.norm(two_grid_matrix(A, P, R, Ac, omega, nu), 2)


def gamma_tilde(A, P, R, Ac, omega):
    """Gamma~ of Definition def2s."""
    X = omega * np.diag(A)
    Dt = np.diag(1.0 / X) + P @ np.linalg.solve(Ac, R)
    AH = A.conj().T
    DtH = Dt.conj().T
    return AH @ DtH + Dt @ A - AH @ DtH @ Dt @ A


def is_hpd(B):
    """Hermitian positive definite test by Cholesky (Sec. 3, after Cor. mgc1)."""
    if not np.allclose(B, B.conj().T, rtol=0, atol=1e-10 * np.abs(B).max()):
        return False
    try:
        np.linalg.cholesky(0.5 * (B + B.conj().T))
        return True
    except np.linalg.LinAlgError:
        return False
