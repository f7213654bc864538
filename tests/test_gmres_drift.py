"""The spread between two correct FP64 implementations of a GMRES(3)-smoothed
solve (CPU only).

The CUDA path forms the modified Gram-Schmidt coefficients of each Arnoldi
step of the GMRES(3) smoother (Sec. 5.3) from the Gram matrix of the basis,
so that one pass over the grid yields every inner product of the step; the
oracle runs MGS vector by vector.  The two are equal in exact arithmetic.
A GMRES(3)-smoothed cycle is a nonlinear map of the iterate, so rounding
differences grow through a solve.  This test runs the oracle's cycle with
each form (``tests/parity_util.gram_gmres_step`` for the Gram form) on the
GMRES(3) cases of the FP64 parity tests and pins what the GPU bars rest on:

* the drift is real: on gmres_V11_shift1k (V(1,1), k = 40, 65^2) the two
  forms end 1e-9 .. 1e-7 apart node by node, far above the 1e-10 bar of an
  affine solve, with identical cycle counts;
* on the W(2,2) case the spread stays at rounding level (<= 1e-13);
* the spread over the variants of ``parity_util.SPREAD_VARIANTS`` (b
  scaled by 1 + a few ulp, either form) stays inside the caps after the
  factor 10 of the GPU bars, so those bars never rest on the caps: about
  1e-8 (iterates) and 5e-4 (residual histories) on gmres_V11_shift1k,
  1e-10 and 1e-6 on gmres_V11_shift0, rounding level on gmres_W22.
"""
import numpy as np

import parity_util as pu
import synth
from oracle import cycle as ocycle
from oracle import hierarchy as ohier


def _spread(name):
    case = next(c for c in pu.CASES if c[0] == name)
    _, nx, ny, k, beta2, sm, gamma, n1, n2, tol = case
    h = 1.0 / max(nx, ny)
    b = synth.point_source(nx, ny, h).ravel()
    H = ohier.build_hierarchy(nx, ny, h, k, beta2)
    opt = ocycle.CycleOptions(gamma, sm, n1, n2, 4.5)
    ref = ocycle.mg_solve(H, b, tol, opt, keep_iterates=True)
    alt = pu.solve_with_gram_form(H, b, tol, opt, keep_iterates=True)
    per_cycle = [pu.relmax(a, r) for a, r in zip(alt.iterates, ref.iterates)]
    return ref, alt, per_cycle, pu.gram_spread(H, b, tol, opt, ref)


def test_gram_form_equals_mgs_in_one_step():
    # one step from the same iterate: the two forms agree to rounding
    n, k = 32, 20.0
    h = 1.0 / n
    H = ohier.build_hierarchy(n, n, h, k, 1 / k)
    b = synth.point_source(n, n, h).ravel()
    x = 1e-3 * synth.random_complex((n + 1, n + 1), 4).ravel()
    from oracle import smoothers
    x1 = smoothers.gmres_step(H.A[0], x, b)
    x2 = pu.gram_gmres_step(H.A[0], x, b)
    assert pu.relmax(x2, x1) <= 1e-13


def test_gmres_v11_forms_drift_apart_through_the_solve():
    ref, alt, per_cycle, (dx, dh) = _spread("gmres_V11_shift1k")
    assert alt.cycles == ref.cycles
    assert per_cycle[0] <= 1e-13                    # first cycle: rounding level
    assert max(per_cycle) >= 1e-8                   # mid-solve peak of the Gram form
    assert 1e-9 <= dx <= 1e-7                       # final iterate, over the variants
    assert 1e-5 <= dh                               # residual histories, over the variants
    assert pu.SPREAD_FACTOR * dx < pu.X_CAP and pu.SPREAD_FACTOR * dh < pu.HIST_CAP


def test_gmres_w22_spread_stays_at_rounding_level():
    ref, alt, per_cycle, (dx, dh) = _spread("gmres_W22")
    assert alt.cycles == ref.cycles
    assert dx <= 1e-13 and max(per_cycle) <= 1e-13


def test_gmres_shift0_spread_inside_the_caps():
    ref, alt, per_cycle, (dx, dh) = _spread("gmres_V11_shift0")
    assert alt.cycles == ref.cycles
    bx, bh = pu.whole_solve_bars(dx, dh)
    assert pu.SPREAD_FACTOR * dx < pu.X_CAP and pu.SPREAD_FACTOR * dh < pu.HIST_CAP
    assert bx < 1e-7 and bh < 1e-4


def test_last_arnoldi_norm_from_the_gram_form():
    """The complex64 GMRES(3) steps take h_32 = |u3| without a pass over u3:
    with unit basis vectors the modified Gram-Schmidt steps of the Arnoldi
    process remove |h_l2|^2 from the squared norm one by one, so |u3|^2 =
    |A v2|^2 - sum_l |h_l2|^2 exactly.  On the fine operator of a bench-like
    problem, with the coefficients in the Gram-matrix form the kernels use
    (and in plain MGS), the identity holds to FP64 rounding, and in float32
    arithmetic to float rounding relative to |A v2|^2."""
    n, k = 48, 30.0
    h = 1.0 / n
    A = ohier.build_hierarchy(n, n, h, k, 1 / k).A[0]
    b = synth.point_source(n, n, h).ravel() + 1e-2 * synth.random_complex((n + 1) ** 2, 23) / h**2
    for dt, tol in ((np.complex128, 1e-12), (np.complex64, 3e-6)):
        Ad = A.astype(dt)
        v = [(b / np.linalg.norm(b)).astype(dt)]
        G = np.eye(3, dtype=dt)           # <v_i, v_l>
        for j in range(3):
            w = Ad @ v[j]
            d = np.array([np.vdot(v[l], w) for l in range(j + 1)])
            hcol = np.zeros(j + 1, dtype=dt)
            for l in range(j + 1):        # Gram form of MGS: h_l = <v_l, w> - sum_{q<l} h_q <v_l, v_q>
                hcol[l] = d[l] - sum(hcol[q] * G[l, q] for q in range(l))
            u = w - sum(hcol[l] * v[l] for l in range(j + 1))
            gram = np.vdot(w, w).real - np.sum(np.abs(hcol) ** 2)
            exact = np.vdot(u, u).real
            assert abs(gram - exact) <= tol * np.vdot(w, w).real, (dt, j, gram, exact)
            if j < 2:
                vn = u / np.linalg.norm(u)
                for l in range(j + 1):
                    G[j + 1, l] = np.vdot(vn, v[l])
                    G[l, j + 1] = np.conj(G[j + 1, l])
                v.append(vn)
