"""Inter-grid transfer operators.

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 4, Eq. (xex): the prolongation built on the quadratic rational
Bezier curve maps a coarse grid function u_2h to the fine grid by

    even fine node i:  (u_{(i-2)/2} + 6 u_{i/2} + u_{(i+2)/2}) / 8
    odd  fine node i:  (u_{(i-1)/2} + u_{(i+1)/2}) / 2

(the odd rule alone is linear interpolation).  Restriction is the transpose
of the prolongation (Sec. 1; Sec. 3 writes A_c = P' A P with P' the
transpose), scaled so that interior rows sum to one.

Readings:

* Vertex-centred coarsening: fine node 2J coincides with coarse node J; a
  fine grid of n intervals (n even) has a coarse grid of n/2 intervals.
* The edge rule is the formula as printed: a coarse value with an index
  outside 0..n/2 is dropped (zero extension).  Table conv1's CSL column is
  reproduced to 0.014 with this rule and only to 0.046 with linear
  extrapolation (injection at the edge).  ``edge="inject"`` keeps the
  alternative for the tests.
* 2D operators are tensor products of the 1D ones (x fastest, so the 2D
  prolongation is kron(P_y, P_x)).
* Restriction R = P^T / 4 in 2D (P_1^T / 2 per direction).  The factor
  cancels in P (R A P)^{-1} R and therefore in the whole cycle.
"""
import numpy as np
import scipy.sparse as sp


def prolongation_1d(n, kind="bezier", edge="zero"):
    """(n+1) x (n/2+1) sparse prolongation for one direction, Eq. (xex).

    kind="bezier": Eq. (xex); kind="linear": even nodes copy the coincident
    coarse value, odd nodes average the two neighbours (Table conv1 "Linear").
    """
    if n % 2:
        raise ValueError("prolongation needs an even interval count")
    nc = n // 2
    rows, cols, vals = [], [], []

    def add(i, J, v):
        rows.append(i)
        cols.append(J)
        vals.append(v)

    for i in range(n + 1):
        if i % 2 == 1:
            add(i, (i - 1) // 2, 0.5)
            add(i, (i + 1) // 2, 0.5)
        elif kind == "linear":
            add(i, i // 2, 1.0)
        else:
            J = i // 2
            add(i, J, 6.0 / 8.0)
            for Jn in (J - 1, J + 1):
                if 0 <= Jn <= nc:
                    add(i, Jn, 1.0 / 8.0)
                elif edge == "inject":
                    # linear extrapolation u_{J+-1} = 2 u_J - u_{J-+1}
                    add(i, J, 2.0 / 8.0)
                    add(i, 2 * J - Jn, -1.0 / 8.0)
                elif edge != "zero":
                    raise ValueError(edge)
    P = sp.coo_matrix((vals, (rows, cols)), shape=(n + 1, nc + 1)).tocsr()
    P.sum_duplicates()
    return P


def prolongation(nx, ny, kind="bezier", edge="zero"):
    """2D prolongation kron(P_y, P_x): coarse (nx/2+1)(ny/2+1) -> fine (nx+1)(ny+1)."""
    return sp.kron(prolongation_1d(ny, kind, edge), prolongation_1d(nx, kind, edge)).tocsr()


def restriction(nx, ny, kind="bezier", edge="zero"):
    """2D restriction P^T / 4 (transpose of the prolongation, Sec. 1 / Sec. 3)."""
    return (prolongation(nx, ny, kind, edge).T * 0.25).tocsr()
