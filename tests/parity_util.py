"""Helpers shared by the parity tests (test code only, not part of the oracle).

* ``rel2`` / ``relmax`` / ``relbnd``: relative differences in the 2-norm, node
  by node (max |a - b| / max |b|), and node by node on the boundary ring of
  the grid only, where the ghost-eliminated Sommerfeld rows and the edge rule
  of Eq. (xex) act and where a 2-norm over the whole grid would dilute an
  error confined to O(n) nodes.
* ``assert_close``: all three at one bar.
* ``gram_gmres_step`` and ``gram_spread``: a second FP64 implementation of the
  GMRES(3) smoothing step of Sec. 5.3, written in the Gram-matrix form of
  modified Gram-Schmidt that the CUDA path uses (all inner products of an
  Arnoldi step from one pass; h_lj = <v_l, w> - sum_{q<l} h_qj <v_l, v_q>).
  In exact arithmetic it equals the oracle's MGS.  Run in the oracle's cycle
  in place of the oracle's step, it measures how far two correct FP64
  implementations of the same GMRES(3)-smoothed solve drift apart through
  rounding alone; the parity bars of whole GMRES(3) solves are derived from
  that spread.
"""
import numpy as np

from oracle import cycle as ocycle
from oracle import smoothers as osm


def rel2(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def relmax(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def boundary_mask(ny1, nx1):
    m = np.zeros((ny1, nx1), dtype=bool)
    m[0, :] = m[-1, :] = True
    m[:, 0] = m[:, -1] = True
    return m


def relbnd(a, b, shape):
    """max over boundary nodes of |a - b|, relative to max |b| over the grid."""
    a = np.reshape(a, shape)
    b = np.reshape(b, shape)
    m = boundary_mask(*shape)
    return np.abs(a - b)[m].max() / max(np.abs(b).max(), 1e-300)


def assert_close(a, b, bar, shape=None, what=""):
    """2-norm, node-wise and (given the grid shape) boundary-node-wise
    relative differences all at most ``bar``."""
    d2, dm = rel2(a, b), relmax(a, b)
    assert d2 <= bar, f"{what}: 2-norm rel diff {d2:.3e} > {bar:.1e}"
    assert dm <= bar, f"{what}: node-wise rel diff {dm:.3e} > {bar:.1e}"
    if shape is not None:
        db = relbnd(a, b, shape)
        assert db <= bar, f"{what}: boundary node-wise rel diff {db:.3e} > {bar:.1e}"


def gram_gmres_step(A, x, b, m=3, breakdown=1e-14):
    """One GMRES(m) step from x with MGS written through the Gram matrix of
    the basis (the CUDA path's form); same breakdown rule and exact small
    least-squares solve as the oracle's step."""
    r0 = b - A @ x
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return x
    V = [r0 / beta]
    Hb = np.zeros((m + 1, m), dtype=np.complex128)
    G = np.eye(m + 1, dtype=np.complex128)        # G[l, q] = <v_l, v_q>
    steps = m
    for j in range(m):
        w = A @ V[j]
        d = [np.vdot(V[l], w) for l in range(j + 1)]
        for l in range(j + 1):
            Hb[l, j] = d[l] - sum(Hb[q, j] * G[l, q] for q in range(l))
        u = w - sum(Hb[l, j] * V[l] for l in range(j + 1))
        Hb[j + 1, j] = np.linalg.norm(u)
        if Hb[j + 1, j].real <= breakdown * beta:
            steps = j + 1
            break
        V.append(u / Hb[j + 1, j])
        for l in range(j + 1):
            G[j + 1, l] = np.vdot(V[j + 1], V[l])
    rhs = np.zeros(steps + 1, dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(Hb[: steps + 1, :steps], rhs, rcond=None)[0]
    return x + sum(y[q] * V[q] for q in range(steps))


def solve_with_gram_form(H, b, tol, opt, **kw):
    """The oracle's cycle and outer loop with the Gram-form GMRES step."""
    saved = osm.gmres_step
    osm.gmres_step = gram_gmres_step
    try:
        return ocycle.mg_solve(H, b, tol, opt, **kw)
    finally:
        osm.gmres_step = saved


# Variants of the oracle's solve used to measure the rounding spread: the
# Gram form on b, and both forms on b scaled by 1 + eps (a relative change of
# a few ulp, which changes nothing but the rounding of the whole solve).
SPREAD_VARIANTS = [("gram", 0.0), ("gram", 1e-15), ("mgs", 1e-15), ("gram", -1e-15), ("mgs", -1e-15),
                   ("gram", 3e-15), ("mgs", 3e-15)]


def gram_spread(H, b, tol, opt, ref):
    """(iterate spread, history spread) of the oracle's solve ``ref`` (run
    with keep_iterates): the largest node-wise relative difference of the
    final iterate and the largest relative difference of the residual
    histories between ``ref`` and each of SPREAD_VARIANTS, maximised over
    the variants (one sample of the drift varies by 20x from variant to
    variant and from machine to machine).  Every variant must take the same
    number of cycles (b scaled by 1 + eps keeps the relative residuals)."""
    dx, dh = 0.0, 0.0
    for form, eps in SPREAD_VARIANTS:
        bb = b * (1.0 + eps)
        if form == "gram":
            alt = solve_with_gram_form(H, bb, tol, opt, keep_iterates=True)
        else:
            alt = ocycle.mg_solve(H, bb, tol, opt, keep_iterates=True)
        assert alt.cycles == ref.cycles
        xs = alt.x / (1.0 + eps)
        dx = max(dx, relmax(xs, ref.x), rel2(xs, ref.x))
        hr = np.abs(np.array(alt.history) - np.array(ref.history)) / np.array(ref.history)
        dh = max(dh, float(hr.max()))
    return dx, dh


# Whole-solve cases of the FP64 parity tests:
# (name, nx, ny, k, beta2, smoother, gamma, nu_pre, nu_post, tol)
CASES = [
    ("cfg1_jacobi_V11", 32, 32, 20.0, 0.7, "jacobi", 1, 1, 1, 1e-6),
    ("jacobi_W22", 32, 32, 20.0, 0.7, "jacobi", 2, 2, 2, 1e-6),
    ("jacobi_V21_odd", 40, 40, 25.0, 0.7, "jacobi", 1, 2, 1, 1e-6),
    ("gmres_V11_shift1k", 64, 64, 40.0, 1 / 40.0, "gmres3", 1, 1, 1, 1e-6),
    ("gmres_W22", 48, 48, 30.0, 1 / 30.0, "gmres3", 2, 2, 2, 1e-8),
    ("gmres_V11_shift0", 32, 32, 20.0, 0.0, "gmres3", 1, 1, 1, 1e-6),
    ("rect_jacobi", 56, 24, 20.0, 0.7, "jacobi", 1, 2, 2, 1e-6),
]

# A GMRES(3) whole solve on the GPU is held to SPREAD_FACTOR times the largest
# spread between the oracle's FP64 solve and its variants (``gram_spread``),
# floored at the FP64 bars of the affine (Jacobi) solves and capped at the
# loosest bars any case is allowed (the CPU test of the spread checks that no
# case reaches the caps).
SPREAD_FACTOR = 10.0
X_FLOOR, X_CAP = 1e-10, 1e-6
HIST_FLOOR, HIST_CAP = 1e-9, 1e-2


def whole_solve_bars(spread_x, spread_hist):
    bx = min(max(SPREAD_FACTOR * spread_x, X_FLOOR), X_CAP)
    bh = min(max(SPREAD_FACTOR * spread_hist, HIST_FLOOR), HIST_CAP)
    return bx, bh
