"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Bars: FP64 operators and Galerkin stencils to 1e-13 relative (max norm),
FP64 iterates to 1e-10 relative at every checked cycle with identical cycle
counts, the mixed path to 1e-6 relative of the FP64 oracle solution.
"""
import functools

import numpy as np
import pytest

import synth
import parity_util as pu
from oracle import cycle as ocycle
from oracle import gradient as ograd
from oracle import hierarchy as ohier
from oracle import problem as oprob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runner deselects -m gpu anyway
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    """Larger of the 2-norm and the node-wise relative difference."""
    return max(pu.rel2(a, b), pu.relmax(a, b))


def opts(smoother):
    return hm.SMOOTHERS[smoother]


# ------------------------------------------------------------------ operators


@pytest.mark.parametrize("nx,ny,kvar", [(32, 32, False), (40, 24, True), (10, 6, False)])
def test_operators_and_galerkin_stencils(nx, ny, kvar):
    h = 1.0 / 32
    k = synth.k_field(synth.chi_sharp(nx, ny, 7), 10.0, 20.0) if kvar else 20.0
    H = ohier.build_hierarchy(nx, ny, h, k, 0.7)
    s = hm.Solver(nx, ny, h, dev(k, torch.float64) if kvar else k, 0.7)
    assert s.nlevels == H.nlevels
    for l, (cx_, cy_) in enumerate(H.sizes):
        gnx, gny, r, _ = s.level_info(l)
        assert (gnx, gny) == (cx_, cy_)
        x = synth.random_complex((cy_ + 1, cx_ + 1), 100 + l)
        y = host(s.apply(l, dev(x)[None]))[0]
        ref = (H.A[l] @ x.ravel()).reshape(x.shape)
        assert rel(y, ref) <= 1e-13, l
        S = host(s.stencil(l))
        So = ohier.stencil_of(H.A[l], cx_, cy_, r)
        assert np.abs(S - So).max() <= 1e-13 * np.abs(So).max(), l
    s.close()


# ------------------------------------------------------------------ iterates


def _oracle_run(nx, ny, h, k, beta2, opt, b, tol, keep=True, levels=0, max_cycles=10000):
    H = ohier.build_hierarchy(nx, ny, h, k, beta2, levels=levels)
    return ocycle.mg_solve(H, b.ravel(), tol, opt, keep_iterates=keep, max_cycles=max_cycles)


CASES = pu.CASES


# execution modes: every level as grid-wide kernels; the library default
# (small levels in one CTA per RHS); level 0 as grid-wide kernels and the rest
# in one cooperative launch; the whole cycle in one CTA per RHS; the whole
# cycle in one cooperative launch; grid-wide kernels without fusion; grid-wide
# kernels with the GMRES(3) marches forced on (small grids run them on the
# boundary path only)
COARSE = [dict(coarse_nodes=0), dict(), dict(coarse_nodes=1200, coarse_mode=1),
          dict(coarse_nodes=10**6, coarse_mode=0), dict(coarse_nodes=10**6, coarse_mode=1),
          dict(coarse_nodes=0, fuse=0), dict(coarse_nodes=0, march=1)]
COARSE_IDS = ["grid", "default", "hybrid", "cta", "coop", "grid_unfused", "grid_march"]


@functools.lru_cache(maxsize=None)
def _reference(case):
    """The oracle's solve of a case, and for GMRES(3) the whole-solve bars
    derived from the spread between the oracle's MGS and Gram-form steps."""
    name, nx, ny, k, beta2, sm, gamma, n1, n2, tol = case
    h = 1.0 / max(nx, ny)
    b = synth.point_source(nx, ny, h)
    opt = ocycle.CycleOptions(gamma, sm, n1, n2, 4.5)
    H = ohier.build_hierarchy(nx, ny, h, k, beta2)
    ref = ocycle.mg_solve(H, b.ravel(), tol, opt, keep_iterates=True)
    assert ref.converged
    if sm == "jacobi":
        bars = (1e-10, 1e-9)
    else:
        bars = pu.whole_solve_bars(*pu.gram_spread(H, b.ravel(), tol, opt, ref))
    return b, ref, bars


@pytest.mark.parametrize("cn", COARSE, ids=COARSE_IDS)
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_iterates_and_cycle_counts(case, cn):
    """Jacobi cycles are a fixed affine map, so whole-solve iterates must agree
    to 1e-10 node by node (boundary ring included) and the residual
    histories to 1e-9.  GMRES(3)-smoothed cycles are a nonlinear map that
    amplifies rounding differences: the oracle's own MGS and its Gram-matrix
    form (the CUDA path's), or either on b scaled by 1 + a few ulp, drift
    apart by up to ~2e-7 mid-solve on gmres_V11_shift1k
    (tests/test_gmres_drift.py).  For GMRES the 1e-10 bar therefore applies
    to one cycle started from the oracle's previous iterate, and the whole
    solve is held to 10x the largest spread between the oracle and those
    variants on the same case (floored at 1e-10 / 1e-9, capped at 1e-6 /
    1e-2).  Cycle counts are identical in every case."""
    name, nx, ny, k, beta2, sm, gamma, n1, n2, tol = case
    h = 1.0 / max(nx, ny)
    b, ref, (whole, hist_rtol) = _reference(case)
    shape = (ny + 1, nx + 1)
    s = hm.Solver(nx, ny, h, k, beta2, cycle=gamma, smoother=sm, nu_pre=n1, nu_post=n2, **cn)
    x, st, cyc, rr = s.solve(dev(b), tol=tol)
    assert st == hm.MG_OK
    assert cyc[0] == ref.cycles
    pu.assert_close(host(x)[0], ref.x.reshape(shape), whole, shape, "whole solve")
    hist = np.array(s.history(ref.cycles)[0])
    assert np.allclose(hist, ref.history, rtol=hist_rtol, atol=0)
    s.close()
    # one cycle from the same input iterate, at several points of the solve
    s1 = hm.Solver(nx, ny, h, k, beta2, cycle=gamma, smoother=sm, nu_pre=n1, nu_post=n2, max_cycles=1, **cn)
    for m in sorted({1, 2, ref.cycles // 2, ref.cycles}):
        x0 = np.zeros_like(b) if m == 1 else ref.iterates[m - 2].reshape(b.shape)
        xm, st1, cm, _ = s1.solve(dev(b), x=dev(x0)[None].contiguous(), tol=1e-300)
        assert st1 == hm.MG_EMAXIT and cm[0] == 1
        pu.assert_close(host(xm)[0], ref.iterates[m - 1].reshape(shape), 1e-10, shape, f"one cycle {m}")
    s1.close()


def test_variable_k_iterates():
    nx = ny = 40
    h = 1.0 / 40
    k = synth.k_field(synth.chi_smooth(nx, ny, 3), 10.0, 25.0)
    b = synth.point_source(nx, ny, h)
    opt = ocycle.CycleOptions(1, "gmres3", 1, 1, 4.5)
    ref = _oracle_run(nx, ny, h, k, 1 / 25.0, opt, b, 1e-7)
    s = hm.Solver(nx, ny, h, dev(k, torch.float64), 1 / 25.0, smoother="gmres3")
    x, st, cyc, _ = s.solve(dev(b), tol=1e-7)
    assert st == hm.MG_OK and cyc[0] == ref.cycles
    assert rel(host(x)[0], ref.x) <= 1e-6
    s1 = hm.Solver(nx, ny, h, dev(k, torch.float64), 1 / 25.0, smoother="gmres3", max_cycles=1)
    x0 = ref.iterates[ref.cycles // 2 - 1].reshape(b.shape)
    xm, _, _, _ = s1.solve(dev(b), x=dev(x0)[None].contiguous(), tol=1e-300)
    pu.assert_close(host(xm)[0], ref.iterates[ref.cycles // 2], 1e-10, (ny + 1, nx + 1), "variable k, one cycle")
    # Jacobi on the same variable-k problem: whole-solve iterates at 1e-10
    optj = ocycle.CycleOptions(1, "jacobi", 2, 2, 4.5)
    refj = _oracle_run(nx, ny, h, k, 0.7, optj, b, 1e-6)
    sj = hm.Solver(nx, ny, h, dev(k, torch.float64), 0.7, nu_pre=2, nu_post=2)
    x, st, cyc, _ = sj.solve(dev(b), tol=1e-6)
    assert st == hm.MG_OK and cyc[0] == refj.cycles
    pu.assert_close(host(x)[0], refj.x, 1e-10, (ny + 1, nx + 1), "variable k, Jacobi whole solve")


@pytest.mark.parametrize("cn", COARSE, ids=COARSE_IDS)
def test_batch_each_rhs_matches_oracle(cn):
    nx = ny = 32
    h = 1.0 / 32
    srcs = synth.source_row(nx, ny, h, 3)
    srcs[2] = synth.random_complex((ny + 1, nx + 1), 5)
    H = ohier.build_hierarchy(nx, ny, h, 20.0, 0.7)
    opt = ocycle.CycleOptions(1, "jacobi", 1, 1, 4.5)
    refs = [ocycle.mg_solve(H, srcs[q].ravel(), 1e-6, opt) for q in range(3)]
    s = hm.Solver(nx, ny, h, 20.0, 0.7, batch=3, **cn)
    x, st, cyc, rr = s.solve(dev(srcs), tol=1e-6)
    assert st == hm.MG_OK
    for q in range(3):
        assert cyc[q] == refs[q].cycles
        pu.assert_close(host(x)[q], refs[q].x, 1e-10, (ny + 1, nx + 1), f"rhs {q}")


@pytest.mark.parametrize("precision", ["mixed", "mixed-ff"])
def test_mixed_precision_against_fp64_oracle(precision):
    # complex64 cycles inside the refinement loop (outer values in FP64, or
    # float-float for mixed-ff): the FP64 residual of the returned x meets
    # tol and equals the reported one, and driven to 1e-10 the solution
    # agrees with the FP64 oracle's to 1e-6 relative.
    nx = ny = 64
    h = 1.0 / 64
    k = 40.0
    b = synth.point_source(nx, ny, h)
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    H = ohier.build_hierarchy(nx, ny, h, k, 1 / k)
    ref = ocycle.mg_solve(H, b.ravel(), 1e-12, opt)
    for sm, beta2, cn in (("gmres3", 1 / k, COARSE[1]), ("jacobi", 0.7, COARSE[1]), ("gmres3", 1 / k, COARSE[0]),
                          ("gmres3", 1 / k, COARSE[2]), ("gmres3", 1 / k, COARSE[4])):
        s = hm.Solver(nx, ny, h, k, beta2, smoother=sm, nu_pre=2, nu_post=2, precision=precision, **cn)
        x, st, cyc, rr = s.solve(dev(b), tol=1e-6)
        assert st == hm.MG_OK and rr[0] <= 1e-6
        r = b.ravel() - H.A[0] @ host(x)[0].ravel()
        assert abs(np.linalg.norm(r) / np.linalg.norm(b) - rr[0]) <= 1e-3 * rr[0]
        x, st, cyc, rr = s.solve(dev(b), tol=1e-10)
        assert st == hm.MG_OK
        assert rel(host(x)[0], ref.x) <= 1e-6
        s.close()


def test_adjoint_solves_hermitian_system():
    nx = ny = 32
    h = 1.0 / 32
    g = synth.random_complex((ny + 1, nx + 1), 11)
    A = oprob.helmholtz_matrix(nx, ny, h, 20.0)
    s = hm.Solver(nx, ny, h, 20.0, 1 / 20.0, smoother="gmres3", nu_pre=2, nu_post=2)
    lam, st, cyc, rr = s.adjoint(dev(g), tol=1e-10)
    assert st == hm.MG_OK
    lam = host(lam)[0].ravel()
    r = g.ravel() - A.conj().T @ lam
    assert np.linalg.norm(r) / np.linalg.norm(g) <= 1e-10


def test_gradient_kernel_matches_oracle_formula():
    nx = ny = 24
    h = 20.0
    omega_f = 2 * np.pi * 4.0
    m = (1.0 / 2000.0**2) * (1 + 0.1 * synth.smooth_perturbation(nx, ny, 2, 4.0))
    u = synth.random_complex((3, ny + 1, nx + 1), 1)
    lam = synth.random_complex((3, ny + 1, nx + 1), 2)
    dA = ograd.diag_derivative(nx, ny, h, m, omega_f)
    ref = -np.real(np.sum(np.conj(lam) * dA[None] * u, axis=0))
    s = hm.Solver(nx, ny, h, dev(omega_f * np.sqrt(m), torch.float64), 0.0)
    g = host(s.gradient(dev(u), dev(lam), dev(m, torch.float64), omega_f))
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


# ------------------------------------------------------------------ edge cases


def test_zero_rhs_and_direct_levels():
    nx = ny = 8
    h = 1.0 / 8
    s = hm.Solver(nx, ny, h, 5.0, 0.7)
    x0 = dev(synth.random_complex((1, ny + 1, nx + 1), 3))
    x, st, cyc, rr = s.solve(dev(np.zeros((1, ny + 1, nx + 1))), x=x0, tol=1e-6)
    assert st == hm.MG_OK and cyc[0] == 0 and np.abs(host(x)).max() == 0.0
    # one level: the cycle is the direct solve, one cycle reaches any tol
    b = synth.point_source(nx, ny, h)
    s1 = hm.Solver(nx, ny, h, 5.0, 0.7, levels=1)
    x, st, cyc, rr = s1.solve(dev(b), tol=1e-12)
    A = oprob.helmholtz_matrix(nx, ny, h, 5.0).toarray()
    assert st == hm.MG_OK and cyc[0] == 1
    assert rel(host(x)[0].ravel(), np.linalg.solve(A, b.ravel())) <= 1e-12


def test_divergence_reported_not_hung():
    # kh > 0.625 with Jacobi (excluded in Table tabhind): the oracle diverges,
    # the library must return MG_EDIVERGED after the same number of cycles.
    nx = ny = 16
    h = 1.0 / 16
    k = 30.0
    b = synth.point_source(nx, ny, h)
    opt = ocycle.CycleOptions(1, "jacobi", 1, 1, 4.5)
    ref = _oracle_run(nx, ny, h, k, 0.7, opt, b, 1e-6, keep=False, max_cycles=5000)
    s = hm.Solver(nx, ny, h, k, 0.7, max_cycles=5000)
    x, st, cyc, rr = s.solve(dev(b), tol=1e-6)
    if ref.diverged:
        assert st == hm.MG_EDIVERGED and cyc[0] == ref.cycles
    else:
        assert st in (hm.MG_OK, hm.MG_EMAXIT) and cyc[0] == ref.cycles


def test_invalid_arguments_rejected():
    with pytest.raises(hm.HelmmgError):
        hm.Solver(7, 8, 0.1, 5.0, 0.7, levels=0, cycle=1, nu_pre=-1)
    with pytest.raises(hm.HelmmgError):
        hm.Solver(1, 8, 0.1, 5.0, 0.7)
    with pytest.raises(hm.HelmmgError):
        hm.Solver(8, 8, -0.1, 5.0, 0.7)
    # coarsest grid too large for the direct solver
    with pytest.raises(hm.HelmmgError):
        hm.Solver(63, 63, 0.1, 5.0, 0.7)


def test_interior_row_march_path_on_a_larger_grid():
    """On 257^2 the fine level's row marches (forced on) run most warps on
    the interior path (no boundary tests); the small cases above only reach
    the boundary path.  The node-parallel kernels are checked on the same
    grid.  FP64: one cycle from the oracle's iterate equals the oracle's next
    iterate to 1e-10 at cycles 1, 2 and 3; mixed and mixed-ff: the oracle's
    FP64 residual of the returned x meets tol."""
    n, k = 256, 100.0
    h = 1.0 / n
    b = synth.point_source(n, n, h) + 1e-2 * synth.random_complex((n + 1, n + 1), 5) / h**2
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    ref = _oracle_run(n, n, h, k, 1 / k, opt, b, 1e-300, max_cycles=3)
    for march in (1, 0):
        s1 = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, max_cycles=1, march=march)
        for m in (1, 2, 3):
            x0 = np.zeros_like(b) if m == 1 else ref.iterates[m - 2].reshape(b.shape)
            xm, st1, cm, _ = s1.solve(dev(b), x=dev(x0)[None].contiguous(), tol=1e-300)
            assert cm[0] == 1
            pu.assert_close(host(xm)[0], ref.iterates[m - 1], 1e-10, (n + 1, n + 1), f"march {march}, cycle {m}")
        s1.close()
    A = oprob.helmholtz_matrix(n, n, h, k)
    for precision in ("mixed", "mixed-ff"):
        s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, precision=precision, march=1)
        x, st, cyc, rr = s.solve(dev(b), tol=1e-6)
        assert st == hm.MG_OK and rr[0] <= 1e-6
        r = b.ravel() - A @ host(x)[0].ravel()
        assert abs(np.linalg.norm(r) / np.linalg.norm(b) - rr[0]) <= 1e-3 * rr[0], precision
        s.close()


def test_batched_solves_are_bitwise_reproducible():
    """Every reduction sums its block partials in a fixed order and no result
    depends on which block or stream finishes first, so a batched mixed solve
    (fine-level row marches with their boundary launches on a side stream,
    Kronecker-level column marches, the coarse interpreter) repeats bit for
    bit: twice on one handle (graph replays) and once on a fresh handle."""
    n, k, B = 256, 75.0, 8
    h = 1.0 / n
    b = dev(synth.source_row(n, n, h, B))
    runs = []
    s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, precision="mixed", batch=B, march=1)
    for _ in range(2):
        x, st, cyc, rr = s.solve(b, tol=1e-8)
        assert st == hm.MG_OK
        runs.append((host(x), cyc, rr))
    s.close()
    s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, precision="mixed", batch=B, march=1)
    x, st, cyc, rr = s.solve(b, tol=1e-8)
    runs.append((host(x), cyc, rr))
    s.close()
    for x_, cyc_, rr_ in runs[1:]:
        assert np.array_equal(x_, runs[0][0])
        assert cyc_ == runs[0][1] and rr_ == runs[0][2]
