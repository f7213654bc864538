"""Model problems MP 2-A / MP 2-B and the complex-shifted Laplacian (CSL).

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 2: -Lap u - k^2 u = delta(x-1/2, y-1/2) on [0,1]^2 with the
first-order absorbing (Sommerfeld) condition (d/dn - i k) u = 0 on the whole
boundary, discretised with second-order finite differences, h = 1/n,
kh = 0.625.  (The printed "k^2 u u" is read as k^2 u.)

Readings (the paper does not spell these out):

* Unknowns are all (nx+1)*(ny+1) grid nodes, boundary nodes included; node
  (i, j) has flat index j*(nx+1) + i (x fastest).  Cells are square with side
  h, so a rectangle of nx*h by ny*h is allowed as well as the unit square.
* Boundary rows: the 5-point stencil is applied at a boundary node with a
  ghost node outside the domain; the central difference of the boundary
  condition, (u_out - u_in) / (2h) = i k u_P along the outward normal,
  eliminates the ghost value: u_out = u_in + 2 i k h u_P.  The row is then
  multiplied by 1/2 on an edge and by 1/4 at a corner.  That scaling makes A
  complex symmetric (A^T = A) without changing the solution.  It is the
  reading that reproduces the qualitative pattern and the magnitudes of the
  two-grid norms in Table conv1; the unscaled rows do not.
* CSL (Sec. 4, "CSL with complex shift beta_2"): the mass term k^2 becomes
  (1 + i*beta2) k^2, boundary rows keep the unshifted k.  The sign +i makes
  the shift push Im(x^H C x) the same way as the absorbing boundary term; the
  opposite sign gives two-grid norms of 5-16 against the paper's 0.91-0.98.

A variant the paper does not use (``abc=2``): the second-order absorbing
condition of Engquist and Majda (1977), d u/dn - i k u - (i / 2k) d^2 u / dtau^2
= 0 along every side (tau tangential; the paraxial expansion
sqrt(k^2 + d^2/dtau^2) ~ k + d^2/dtau^2 / (2k) of the outgoing normal
derivative).  In the weak form the tangential term is the boundary stiffness
(i / 2k) int dtau u dtau v over each side, with no term at the corners (the
natural corner condition).  On the grid every boundary segment P-Q of a side
adds c (u_P - u_Q) to row P and c (u_Q - u_P) to row Q, c = i (1/k_P + 1/k_Q)
/ (4 h^3) in the scaled-row units above (1/h^2 times the finite-volume row):
an edge node gains (i / 2k h^3) (2 u_P - u_tau+ - u_tau-), a corner one
segment on each of its two sides.  A stays complex symmetric.
"""
import numpy as np
import scipy.sparse as sp


def node_index(nx, i, j):
    """Flat index of grid node (i, j) on an (nx+1)-wide row-major grid."""
    return j * (nx + 1) + i


def _k_field(nx, ny, k):
    k = np.asarray(k, dtype=np.float64)
    if k.ndim == 0:
        return np.full((ny + 1, nx + 1), float(k))
    if k.shape != (ny + 1, nx + 1):
        raise ValueError("k field must have shape (ny+1, nx+1)")
    return k


def helmholtz_matrix(nx, ny, h, k, beta2=0.0, rows="scaled", abc=1):
    """Sparse (CSR, complex128) matrix of -Lap_h - (1 + i beta2) k^2 with
    ghost-eliminated Sommerfeld rows scaled by 1/2 (edge) and 1/4 (corner).

    ``beta2 = 0`` gives the Helmholtz operator A of MP 2-A / MP 2-B (Sec. 2);
    ``beta2 > 0`` gives the CSL operator C used for coarsening (Sec. 4, Sec. 5).
    ``k`` is a scalar (MP 2-A) or an (ny+1, nx+1) array (MP 2-B).

    ``rows`` selects the reading of the boundary rows (the paper names only
    "second-order finite differences"): "scaled" (the default above),
    "unscaled" (the same ghost-eliminated rows without the 1/2, 1/4 factors;
    not symmetric), or "bc1" (``helmholtz_matrix_bc1``: the boundary rows are
    the first-order one-sided absorbing condition itself).  ``abc=2`` adds the
    second-order absorbing condition's tangential terms to the scaled rows
    (``tangential_abc2``; see the module notes).
    """
    if abc not in (1, 2):
        raise ValueError(abc)
    if abc == 2:
        if rows != "scaled":
            raise ValueError("the second-order absorbing rows are defined on the scaled rows")
        return (helmholtz_matrix(nx, ny, h, k, beta2) + tangential_abc2(nx, ny, h, k)).tocsr()
    if rows == "bc1":
        return helmholtz_matrix_bc1(nx, ny, h, k, beta2)
    if rows not in ("scaled", "unscaled"):
        raise ValueError(rows)
    scaled = rows == "scaled"
    kf = _k_field(nx, ny, k)
    N = (nx + 1) * (ny + 1)
    inv_h2 = 1.0 / (h * h)
    jj, ii = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    p = node_index(nx, ii, jj)
    kp = kf.ravel()

    rows = [p]
    cols = [p]
    # centre of the 5-point stencil: 4/h^2 - (1 + i beta2) k^2
    diag = 4.0 * inv_h2 - (1.0 + 1j * beta2) * kp * kp
    vals = [None]  # filled after the ghost terms are added to diag
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        qi = ii + di
        qj = jj + dj
        inside = (qi >= 0) & (qi <= nx) & (qj >= 0) & (qj <= ny)
        # neighbour inside: the usual -1/h^2 coupling
        rows.append(p[inside])
        cols.append(node_index(nx, qi[inside], qj[inside]))
        vals.append(np.full(int(inside.sum()), -inv_h2, dtype=np.complex128))
        # neighbour outside: ghost value u_in + 2 i k h u_P, where u_in is the
        # node mirrored through P (the opposite neighbour)
        out = ~inside
        mi = ii[out] - di
        mj = jj[out] - dj
        rows.append(p[out])
        cols.append(node_index(nx, mi, mj))
        vals.append(np.full(int(out.sum()), -inv_h2, dtype=np.complex128))
        diag = diag - np.where(out, 2j * kp / h, 0.0)
    vals[0] = diag.astype(np.complex128)
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(N, N),
    ).tocsr()
    A.sum_duplicates()
    if not scaled:
        return A
    # row scaling 1/2 per boundary direction
    w = boundary_weights(nx, ny).ravel()
    return (sp.diags(w) @ A).tocsr()


def tangential_abc2(nx, ny, h, k):
    """The second-order absorbing condition's boundary stiffness (module
    notes): for every pair P, Q of neighbouring nodes on one side of the
    boundary, c (u_P - u_Q) in row P and c (u_Q - u_P) in row Q with
    c = i (1/k_P + 1/k_Q) / (4 h^3).  A sparse (N, N) complex matrix."""
    kf = _k_field(nx, ny, k)
    N = (nx + 1) * (ny + 1)
    segs = []   # (P, Q) flat indices of the boundary segments
    for j in (0, ny):                     # bottom and top: neighbours along x
        for i in range(nx):
            segs.append((node_index(nx, i, j), node_index(nx, i + 1, j)))
    for i in (0, nx):                     # left and right: neighbours along y
        for j in range(ny):
            segs.append((node_index(nx, i, j), node_index(nx, i, j + 1)))
    kr = kf.ravel()
    P = np.array([a for a, _ in segs])
    Q = np.array([b for _, b in segs])
    c = 1j * (1.0 / kr[P] + 1.0 / kr[Q]) / (4.0 * h ** 3)
    rows = np.concatenate([P, Q, P, Q])
    cols = np.concatenate([P, Q, Q, P])
    vals = np.concatenate([c, c, -c, -c])
    T = sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()
    T.sum_duplicates()
    return T


def helmholtz_matrix_bc1(nx, ny, h, k, beta2=0.0):
    """Alternative reading of the boundary rows (kept for the comparison of
    readings): interior nodes carry the 5-point rows of -Lap_h - (1 + i
    beta2) k^2, and each boundary node carries the first-order one-sided
    difference of the absorbing condition along its outward normal,
    ((u_P - u_in)/h - i k u_P) / h = 0 (a corner sums its two normals).  The
    matrix is not symmetric."""
    kf = _k_field(nx, ny, k)
    N = (nx + 1) * (ny + 1)
    rows, cols, vals = [], [], []
    for j in range(ny + 1):
        for i in range(nx + 1):
            p = node_index(nx, i, j)
            kk = kf[j, i]
            if 0 < i < nx and 0 < j < ny:
                rows.append(p)
                cols.append(p)
                vals.append(4.0 / h**2 - (1 + 1j * beta2) * kk**2)
                for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    rows.append(p)
                    cols.append(node_index(nx, i + di, j + dj))
                    vals.append(-1.0 / h**2)
                continue
            for on, (qi, qj) in ((i == 0, (1, j)), (i == nx, (nx - 1, j)), (j == 0, (i, 1)), (j == ny, (i, ny - 1))):
                if on:
                    rows += [p, p]
                    cols += [p, node_index(nx, qi, qj)]
                    vals += [(1.0 / h - 1j * kk) / h, -1.0 / h**2]
    A = sp.coo_matrix((vals, (rows, cols)), shape=(N, N), dtype=np.complex128).tocsr()
    A.sum_duplicates()
    return A


def helmholtz_matrix_interior(nx, ny, h, k, beta2=0.0):
    """Alternative reading of the unknowns (kept for the comparison of
    readings): only the interior nodes are unknowns, (nx-1)*(ny-1) of them,
    row-major over i = 1..nx-1, j = 1..ny-1.  A boundary node is eliminated
    with the first-order one-sided absorbing condition
    (u_in - u_B)/h = i k u_B, i.e. u_B = u_in / (1 - i k h), which adds
    -1/(h^2 (1 - i k h)) to the diagonal of each interior row next to the
    boundary (once per boundary neighbour).  ``k`` is a scalar or an
    (ny+1, nx+1) field (the boundary node's k is used)."""
    kf = _k_field(nx, ny, k)
    mx, my = nx - 1, ny - 1
    N = mx * my
    rows, cols, vals = [], [], []
    for j in range(1, ny):
        for i in range(1, nx):
            p = (j - 1) * mx + (i - 1)
            d = 4.0 / h**2 - (1 + 1j * beta2) * kf[j, i] ** 2
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                qi, qj = i + di, j + dj
                if 0 < qi < nx and 0 < qj < ny:
                    rows.append(p)
                    cols.append((qj - 1) * mx + (qi - 1))
                    vals.append(-1.0 / h**2)
                else:
                    d -= 1.0 / (h**2 * (1.0 - 1j * kf[qj, qi] * h))
            rows.append(p)
            cols.append(p)
            vals.append(d)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(N, N), dtype=np.complex128).tocsr()
    A.sum_duplicates()
    return A


def boundary_weights(nx, ny):
    """Row scaling: 1 inside, 1/2 on an edge, 1/4 at a corner; shape (ny+1, nx+1)."""
    wx = np.ones(nx + 1)
    wx[0] = wx[-1] = 0.5
    wy = np.ones(ny + 1)
    wy[0] = wy[-1] = 0.5
    return np.outer(wy, wx)


def helmholtz_dense_rowwise(nx, ny, h, k, beta2=0.0):
    """Same operator as ``helmholtz_matrix`` written node by node with Python
    loops (for tiny grids): used as an independent restatement in the tests."""
    kf = _k_field(nx, ny, k)
    N = (nx + 1) * (ny + 1)
    A = np.zeros((N, N), dtype=np.complex128)
    for j in range(ny + 1):
        for i in range(nx + 1):
            p = node_index(nx, i, j)
            kk = kf[j, i]
            row = np.zeros(N, dtype=np.complex128)
            row[p] += 4.0 / h**2 - (1 + 1j * beta2) * kk**2
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                qi, qj = i + di, j + dj
                if 0 <= qi <= nx and 0 <= qj <= ny:
                    row[node_index(nx, qi, qj)] -= 1.0 / h**2
                else:
                    row[node_index(nx, i - di, j - dj)] -= 1.0 / h**2
                    row[p] -= 2j * kk / h
            s = (0.5 if i in (0, nx) else 1.0) * (0.5 if j in (0, ny) else 1.0)
            A[p] = s * row
    return A


def point_source_rhs(nx, ny, h, i, j):
    """Discrete delta at node (i, j): 1/h^2 there, 0 elsewhere (Sec. 2 source).
    Rows are scaled like the operator, so a source on the boundary carries the
    boundary weight."""
    b = np.zeros((ny + 1) * (nx + 1), dtype=np.complex128)
    b[node_index(nx, i, j)] = boundary_weights(nx, ny)[j, i] / (h * h)
    return b


def sommerfeld_rhs(nx, ny, h, f, g):
    """Right-hand side for -Lap u - k^2 u = f with (d/dn - i k) u = g on the
    boundary, consistent with the ghost elimination above: the ghost value
    picks up 2 h g, which enters the row as +2 g / h before the row scaling.
    ``f`` is an (ny+1, nx+1) array, ``g`` a function g(i, j, nx_out, ny_out)
    returning the boundary datum for the outward normal (nx_out, ny_out)."""
    b = np.array(f, dtype=np.complex128).copy()
    for j in range(ny + 1):
        for i in range(nx + 1):
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                qi, qj = i + di, j + dj
                if not (0 <= qi <= nx and 0 <= qj <= ny):
                    b[j, i] += 2.0 * g(i, j, di, dj) / h
    return (boundary_weights(nx, ny) * b).ravel()
