"""Multigrid hierarchy: level sizes, Galerkin coarse operators, coarsest LU.

Test infrastructure only (see ``oracle/__init__``).

Paper passages followed:

* Sec. 3: A_c is the Galerkin product of restriction, operator and
  prolongation.  Sec. 4 / Table conv1: the product is taken on the CSL C
  (complex shift beta2) rather than on A.  Sec. 4 states the shift is a
  constant, not level dependent, and Sec. 6 that it is added only for the
  coarsening.  Reading: the shift enters once, on the fine level,
  A_1 = R_0 C_0 P_0; deeper levels are A_{l+1} = R_l A_l P_l.  The fine level
  keeps the unshifted A for smoothing and residuals.
* Sec. 5: coarsen "until the dimension N_c is smaller than 10".  Reading:
  halve while both interval counts are even and the current grid still has
  at least 10 nodes; the last grid is solved directly (dense LU).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import problem, transfer


def level_sizes(nx, ny, levels=0, min_coarse=10, grid="vertex"):
    """Interval counts [(nx_0, ny_0), (nx_1, ny_1), ...] of the hierarchy.

    ``levels = 0`` coarsens as far as the rule allows (Sec. 5); a positive
    value caps the number of levels (1 = direct solve only).  ``grid``
    ("vertex" or "interior") says whether the boundary nodes are unknowns,
    which changes the unknown count the rule tests."""
    sizes = [(nx, ny)]
    nodes = (lambda a, b: (a + 1) * (b + 1)) if grid == "vertex" else (lambda a, b: (a - 1) * (b - 1))
    while True:
        cx, cy = sizes[-1]
        if levels and len(sizes) >= levels:
            break
        if cx % 2 or cy % 2 or nodes(cx, cy) < min_coarse:
            break
        sizes.append((cx // 2, cy // 2))
    return sizes


@dataclass
class Hierarchy:
    sizes: list
    h: float
    A: list = field(default_factory=list)   # A[0] = fine Helmholtz, A[l>0] Galerkin
    P: list = field(default_factory=list)   # P[l]: level l+1 -> level l
    R: list = field(default_factory=list)   # R[l]: level l -> level l+1
    C0: object = None                       # fine-level CSL used for A[1]
    lu: object = None                       # LU factors of the coarsest A

    @property
    def nlevels(self):
        return len(self.sizes)


def build_hierarchy(nx, ny, h, k, beta2, levels=0, kind="bezier", edge="zero",
                    min_coarse=10, rows="scaled", grid="vertex", abc=1):
    """All operators of the cycle.  ``k`` scalar (MP 2-A) or field (MP 2-B).

    ``rows`` and ``grid`` select alternative readings of the discretisation,
    kept to compare their cycle counts with the paper's tables: ``rows`` is
    passed to ``problem.helmholtz_matrix``; ``grid="interior"`` takes only the
    interior nodes as unknowns (``problem.helmholtz_matrix_interior``) with
    the transfers of Eq. (xex) restricted to them (a boundary value of a
    coarse correction is zero).  ``abc=2`` takes the second-order absorbing
    rows (a variant the paper does not use, ``problem.tangential_abc2``); the
    coarse operators are the Galerkin products of the same transfers."""
    sizes = level_sizes(nx, ny, levels, min_coarse, grid)
    H = Hierarchy(sizes=sizes, h=h)
    if grid == "interior":
        op = lambda b2: problem.helmholtz_matrix_interior(nx, ny, h, k, b2)
    elif grid == "vertex":
        op = lambda b2: problem.helmholtz_matrix(nx, ny, h, k, b2, rows, abc)
    else:
        raise ValueError(grid)
    H.A.append(op(0.0))
    if len(sizes) > 1:
        H.C0 = op(beta2)
    for l in range(len(sizes) - 1):
        fx, fy = sizes[l]
        P = transfer.prolongation(fx, fy, kind, edge)
        R = transfer.restriction(fx, fy, kind, edge)
        if grid == "interior":
            P = interior_block(P, fx, fy)
            R = interior_block(R.T.tocsr(), fx, fy).T.tocsr()
        Af = H.C0 if l == 0 else H.A[l]
        Ac = (R @ Af @ P).tocsr()
        Ac.sum_duplicates()
        H.P.append(P)
        H.R.append(R)
        H.A.append(Ac)
    H.lu = sla.lu_factor(H.A[-1].toarray())
    return H


def interior_block(P, fx, fy):
    """Rows and columns of a vertex-grid prolongation (fine (fx+1)(fy+1) x
    coarse (fx/2+1)(fy/2+1)) that belong to interior nodes of both grids."""
    def inner(nx, ny):
        j, i = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        return ((i > 0) & (i < nx) & (j > 0) & (j < ny)).ravel()
    return P.tocsr()[inner(fx, fy)][:, inner(fx // 2, fy // 2)].tocsr()


def coarsest_solve(H, r):
    """Direct solve with the coarsest Galerkin operator (Sec. 5: N_c < 10)."""
    return sla.lu_solve(H.lu, r)


def stencil_of(A, nx, ny, radius):
    """Per-node stencil of a grid operator: array [ny+1, nx+1, 2r+1, 2r+1]
    with entry [j, i, dy+r, dx+r] = A[(i,j), (i+dx, j+dy)] (0 off the grid).
    Raises if A couples nodes further apart than ``radius``."""
    A = A.tocoo()
    N = (nx + 1) * (ny + 1)
    assert A.shape == (N, N)
    ri, rj = A.row % (nx + 1), A.row // (nx + 1)
    ci, cj = A.col % (nx + 1), A.col // (nx + 1)
    dx, dy = ci - ri, cj - rj
    if len(dx) and (np.abs(dx).max() > radius or np.abs(dy).max() > radius):
        raise ValueError("operator wider than the given stencil radius")
    S = np.zeros((ny + 1, nx + 1, 2 * radius + 1, 2 * radius + 1), dtype=np.complex128)
    np.add.at(S, (rj, ri, dy + radius, dx + radius), A.data)
    return S


def stencil_radius(A, nx):
    """Largest |dx| or |dy| coupling of a grid operator."""
    A = A.tocoo()
    if A.nnz == 0:
        return 0
    dx = np.abs(A.col % (nx + 1) - A.row % (nx + 1))
    dy = np.abs(A.col // (nx + 1) - A.row // (nx + 1))
    return int(max(dx.max(), dy.max()))
