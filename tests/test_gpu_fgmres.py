"""GPU parity of the FGMRES(m) outer loop (the cycle as right preconditioner)
against the oracle's restarted FGMRES (oracle/krylov.py), through the C-ABI.

Bars: with Jacobi-smoothed FP64 cycles (a fixed affine preconditioner) the
same preconditioner-application counts, whole-solve iterates to 1e-10 and
residual estimates to 1e-6; with GMRES(3) smoothing (a nonlinear cycle) the
same counts, iterates to 1e-6 and estimates to 5e-2.  The GMRES(3)-smoothed
cycle amplifies input differences in some directions by ~1e5 (with a centred
source, whose symmetry rounding breaks), and FGMRES feeds each z_j into the
next basis vector: the oracle's own MGS smoother and its Gram-matrix form
(equal in exact arithmetic) give estimate histories 2e-2 apart and
solutions 1e-9 apart on the n = 64 case.  The
mixed path (complex64 cycles, FP64 Arnoldi) reaches the FP64 tol on the true
residual and, driven to 1e-10, the FP64 oracle's solution to 1e-6.
"""
import numpy as np
import pytest

import synth
from oracle import cycle as ocycle
from oracle import hierarchy as ohier
from oracle import krylov as okry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def two_sources(n, h):
    return np.stack([synth.point_source(n, n, h), synth.point_source(n, n, h, n // 4, n // 3)])


# (n, k, beta2, smoother, nu, m, tol): the Jacobi V(1,1) cycles with beta2 = 0.7
# diverge stand-alone at these wavenumbers (kh = 0.625) and converge inside FGMRES
CASES = [
    (64, 40.0, 0.7, "jacobi", 1, 10, 1e-8),
    (64, 40.0, 0.7, "jacobi", 1, 5, 1e-8),
    (96, 60.0, 0.7, "jacobi", 1, 10, 1e-8),
    (64, 40.0, 1 / 40.0, "gmres3", 2, 5, 1e-8),
]


@pytest.mark.parametrize("coarse_nodes", [1100, 0])
@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}-{c[3]}-m{c[5]}" for c in CASES])
def test_fgmres_fp64_matches_oracle(case, coarse_nodes):
    n, k, beta2, sm, nu, m, tol = case
    h = 1.0 / n
    H = ohier.build_hierarchy(n, n, h, k, beta2)
    opt = ocycle.CycleOptions(1, sm, nu, nu, 4.5)
    srcs = two_sources(n, h)
    refs = [okry.fgmres_solve(H, srcs[q].ravel(), tol, opt, m) for q in range(2)]
    assert all(r.converged for r in refs)
    s = hm.Solver(n, n, h, k, beta2, smoother=sm, nu_pre=nu, nu_post=nu, batch=2, krylov=m,
                  coarse_nodes=coarse_nodes)
    x, st, cyc, rr = s.solve(dev(srcs), tol=tol)
    assert st == hm.MG_OK
    whole = 1e-10 if sm == "jacobi" else 1e-6
    hist = s.history(max(r.cycles for r in refs))
    for q in range(2):
        assert cyc[q] == refs[q].cycles, q
        assert rel(host(x)[q], refs[q].x) <= whole, q
        assert rr[q] <= tol
        assert abs(rr[q] - refs[q].relres) <= (1e-6 if sm == "jacobi" else 0.1) * refs[q].relres
        assert np.allclose(hist[q][:refs[q].cycles], refs[q].history, rtol=1e-6 if sm == "jacobi" else 5e-2, atol=0)
    s.close()


def test_fgmres_converges_where_the_cycle_alone_diverges():
    n, k = 64, 40.0
    h = 1.0 / n
    b = synth.point_source(n, n, h)
    alone = hm.Solver(n, n, h, k, 0.7, max_cycles=200)
    _, st, cyc, _ = alone.solve(dev(b), tol=1e-8)
    assert st in (hm.MG_EDIVERGED, hm.MG_EMAXIT)
    alone.close()
    s = hm.Solver(n, n, h, k, 0.7, krylov=10)
    x, st, cyc, rr = s.solve(dev(b), tol=1e-8)
    assert st == hm.MG_OK and rr[0] <= 1e-8
    H = ohier.build_hierarchy(n, n, h, k, 0.7)
    r = b.ravel() - H.A[0] @ host(x)[0].ravel()
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - rr[0]) <= 1e-6 * rr[0]
    s.close()


@pytest.mark.parametrize("sm", ["jacobi", "gmres3"])
def test_fgmres_mixed_against_fp64_oracle(sm):
    n, k = 64, 40.0
    h = 1.0 / n
    beta2 = 0.7 if sm == "jacobi" else 1 / k
    nu = 1 if sm == "jacobi" else 2
    H = ohier.build_hierarchy(n, n, h, k, beta2)
    opt = ocycle.CycleOptions(1, sm, nu, nu, 4.5)
    srcs = two_sources(n, h)
    s = hm.Solver(n, n, h, k, beta2, smoother=sm, nu_pre=nu, nu_post=nu, batch=2, krylov=10, precision="mixed")
    x, st, cyc, rr = s.solve(dev(srcs), tol=1e-6)
    assert st == hm.MG_OK
    for q in range(2):
        r = srcs[q].ravel() - H.A[0] @ host(x)[q].ravel()
        true = np.linalg.norm(r) / np.linalg.norm(srcs[q])
        assert true <= 1e-6 and abs(true - rr[q]) <= 1e-6 * rr[q]
    x, st, cyc, rr = s.solve(dev(srcs), tol=1e-10)
    assert st == hm.MG_OK
    for q in range(2):
        ref = okry.fgmres_solve(H, srcs[q].ravel(), 1e-10, opt, 10)
        assert rel(host(x)[q], ref.x) <= 1e-6
        assert abs(cyc[q] - ref.cycles) <= max(3, ref.cycles // 10)
    s.close()


def test_fgmres_variable_k():
    n = 48
    h = 1.0 / n
    k = synth.k_field(synth.chi_smooth(n, n, 3), 15.0, 30.0)
    b = synth.point_source(n, n, h)
    H = ohier.build_hierarchy(n, n, h, k, 0.7)
    opt = ocycle.CycleOptions(1, "jacobi", 1, 1, 4.5)
    ref = okry.fgmres_solve(H, b.ravel(), 1e-8, opt, 8)
    assert ref.converged
    s = hm.Solver(n, n, h, dev(k, torch.float64), 0.7, krylov=8)
    x, st, cyc, rr = s.solve(dev(b), tol=1e-8)
    assert st == hm.MG_OK and cyc[0] == ref.cycles
    assert rel(host(x)[0], ref.x) <= 1e-10
    s.close()


def test_fgmres_edge_cases():
    """A zero right-hand side, an initial guess that already meets tol, and a
    cap on preconditioner applications below the count needed."""
    n, k = 32, 20.0
    h = 1.0 / n
    H = ohier.build_hierarchy(n, n, h, k, 0.7)
    opt = ocycle.CycleOptions(1, "jacobi", 1, 1, 4.5)
    b = synth.point_source(n, n, h)
    ref = okry.fgmres_solve(H, b.ravel(), 1e-9, opt, 6)
    tight = okry.fgmres_solve(H, b.ravel(), 1e-12, opt, 6)   # well inside tol on either side's rounding
    srcs = np.stack([b, np.zeros_like(b), b])
    x0 = np.stack([np.zeros_like(b), np.zeros_like(b), tight.x.reshape(b.shape)])
    s = hm.Solver(n, n, h, k, 0.7, batch=3, krylov=6)
    x, st, cyc, rr = s.solve(dev(srcs), x=dev(x0), tol=1e-9)
    assert st == hm.MG_OK
    assert cyc == [ref.cycles, 0, 0]
    assert rel(host(x)[0], ref.x) <= 1e-10
    assert not np.any(host(x)[1])
    assert np.array_equal(host(x)[2], x0[2])
    s.close()
    cap = ref.cycles - 3
    refc = okry.fgmres_solve(H, b.ravel(), 1e-9, opt, 6, max_cycles=cap)
    assert not refc.converged and refc.cycles == cap
    s = hm.Solver(n, n, h, k, 0.7, krylov=6, max_cycles=cap)
    x, st, cyc, rr = s.solve(dev(b), tol=1e-9)
    assert st == hm.MG_EMAXIT and cyc[0] == cap
    assert rel(host(x)[0], refc.x) <= 1e-10
    s.close()


def test_fgmres_adjoint_and_ragged():
    n, k = 32, 20.0
    h = 1.0 / n
    g = synth.random_complex((n + 1, n + 1), 11)
    H = ohier.build_hierarchy(n, n, h, k, 0.7)
    s = hm.Solver(n, n, h, k, 0.7, krylov=8)
    lam, st, cyc, rr = s.adjoint(dev(g), tol=1e-10)
    assert st == hm.MG_OK
    r = g.ravel() - H.A[0].conj().T @ host(lam)[0].ravel()
    assert np.linalg.norm(r) / np.linalg.norm(g) <= 1e-10
    s.close()
    sizes = [(32, 32, 1 / 32, 20.0), (48, 48, 1 / 48, 30.0)]
    rs = hm.RaggedSolver(sizes, 0.7, krylov=8)
    rhs = [dev(synth.point_source(a, b_, hh)) for a, b_, hh, _ in sizes]
    xs, st, cyc, rr = rs.solve(rhs, tol=1e-8)
    assert st == hm.MG_OK
    opt = ocycle.CycleOptions(1, "jacobi", 1, 1, 4.5)
    for p, (a, b_, hh, kk) in enumerate(sizes):
        Hp = ohier.build_hierarchy(a, b_, hh, kk, 0.7)
        ref = okry.fgmres_solve(Hp, host(rhs[p]).ravel(), 1e-8, opt, 8)
        assert cyc[p] == ref.cycles
        assert rel(host(xs[p]), ref.x) <= 1e-10
    rs.close()


def test_fgmres_options_rejected():
    with pytest.raises(hm.HelmmgError, match="krylov"):
        hm.Solver(32, 32, 1 / 32, 20.0, 0.7, krylov=33)
    with pytest.raises(hm.HelmmgError, match="precision"):
        hm.Solver(32, 32, 1 / 32, 20.0, 0.7, krylov=4, precision="mixed-ff")
