"""The second-order absorbing rows (option abc=2: the Engquist-Majda
condition, a variant the paper does not use) on the GPU against the oracle's
abc=2 hierarchy: every level operator to 1e-13, FP64 iterates to 1e-10 node
by node (boundary nodes included) with identical cycle counts, for constant
and variable k, Jacobi and GMRES(3) cycles, node-parallel and row-march
fine-level kernels, batched right-hand sides and the FGMRES outer loop; the
mixed path's solution meets the tolerance in the oracle's FP64 residual."""
import numpy as np
import pytest

import parity_util as pu
import synth
from oracle import cycle as ocycle
from oracle import hierarchy as ohier
from oracle import krylov as okry
from oracle import problem as oprob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _k(nx, ny, variable):
    return synth.k_field(synth.chi_sharp(nx, ny, 7), 15.0, 30.0) if variable else 25.0


@pytest.mark.parametrize("nx,ny,variable", [(32, 32, False), (48, 24, True)])
def test_level_operators_match_the_oracle(nx, ny, variable):
    h = 1.0 / 32
    k = _k(nx, ny, variable)
    H = ohier.build_hierarchy(nx, ny, h, k, 0.7, abc=2)
    s = hm.Solver(nx, ny, h, dev(k, torch.float64) if variable else k, 0.7, abc=2)
    assert s.nlevels == H.nlevels
    for l, (cx_, cy_) in enumerate(H.sizes):
        x = synth.random_complex((cy_ + 1, cx_ + 1), 300 + l)
        y = s.apply(l, dev(x)[None]).cpu().numpy()[0]
        ref = (H.A[l] @ x.ravel()).reshape(x.shape)
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max(), l
    s.close()


CASES = [
    dict(smoother="jacobi", beta2=0.7, nu=1, variable=False, march=None),
    dict(smoother="gmres3", beta2=1 / 25.0, nu=2, variable=False, march=None),
    dict(smoother="gmres3", beta2=1 / 25.0, nu=2, variable=False, march=1),
    dict(smoother="jacobi", beta2=0.7, nu=1, variable=True, march=None),
    dict(smoother="gmres3", beta2=0.05, nu=2, variable=True, march=None),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['smoother']}-var{int(c['variable'])}-march{c['march']}")
def test_fp64_iterates_and_cycle_counts_match_the_oracle(case):
    n, B = 64, 2
    h = 1.0 / n
    k = _k(n, n, case["variable"])
    opt = ocycle.CycleOptions(1, case["smoother"], case["nu"], case["nu"], 4.5)
    H = ohier.build_hierarchy(n, n, h, k, case["beta2"], abc=2)
    rhs = synth.source_row(n, n, h, B) + 1e-2 * synth.random_complex((B, n + 1, n + 1), 9) / h**2
    refs = [ocycle.mg_solve(H, rhs[b].ravel(), 1e-8, opt, keep_iterates=True) for b in range(B)]
    kk = dev(k, torch.float64) if case["variable"] else k
    kw = dict(smoother=case["smoother"], nu_pre=case["nu"], nu_post=case["nu"], batch=B, abc=2)
    if case["march"] is not None:
        kw["march"] = case["march"]
    s1 = hm.Solver(n, n, h, kk, case["beta2"], max_cycles=1, **kw)
    x0 = np.zeros_like(rhs)
    for m in (1, 2, 3):
        if m > 1:
            x0 = np.stack([refs[b].iterates[m - 2].reshape(n + 1, n + 1) for b in range(B)])
        x, st, cyc, _ = s1.solve(dev(rhs), x=dev(x0), tol=1e-300)
        for b in range(B):
            pu.assert_close(x[b].cpu().numpy(), refs[b].iterates[m - 1].reshape(n + 1, n + 1), 1e-10, (n + 1, n + 1),
                            f"rhs {b}, cycle {m}")
    s1.close()
    # the whole solve: each right-hand side's cycle count, converged or (the
    # variable-k Jacobi case) diverged, equals the oracle's
    s = hm.Solver(n, n, h, kk, case["beta2"], **kw)
    x, st, cyc, rr = s.solve(dev(rhs), tol=1e-8)
    assert st == (hm.MG_EDIVERGED if any(r.diverged for r in refs) else hm.MG_OK)
    assert cyc == [r.cycles for r in refs]
    s.close()


def test_fgmres_matches_the_oracle():
    n, k, m = 64, 25.0, 5
    h = 1.0 / n
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    H = ohier.build_hierarchy(n, n, h, k, 1 / k, abc=2)
    b = synth.point_source(n, n, h) + 1e-2 * synth.random_complex((n + 1, n + 1), 11) / h**2
    ref = okry.fgmres_solve(H, b.ravel(), 1e-9, opt, m)
    s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, krylov=m, abc=2)
    x, st, cyc, rr = s.solve(dev(b)[None], tol=1e-9)
    assert st == hm.MG_OK and cyc[0] == ref.cycles
    pu.assert_close(x[0].cpu().numpy().ravel(), ref.x, 1e-8, None, "fgmres")
    s.close()


@pytest.mark.parametrize("variable", [False, True])
def test_mixed_path_meets_the_tolerance_in_the_oracle_residual(variable):
    n = 96
    h = 1.0 / n
    k = _k(n, n, variable) if variable else 30.0
    kk = dev(k, torch.float64) if variable else k
    b = synth.point_source(n, n, h) + 1e-2 * synth.random_complex((n + 1, n + 1), 13) / h**2
    A = oprob.helmholtz_matrix(n, n, h, k, abc=2)
    s = hm.Solver(n, n, h, kk, 0.05, smoother="gmres3", nu_pre=2, nu_post=2, precision="mixed", abc=2)
    x, st, cyc, rr = s.solve(dev(b)[None], tol=1e-7)
    assert st == hm.MG_OK
    r = b.ravel() - A @ x[0].cpu().numpy().ravel()
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1e-7 and abs(rel - rr[0]) <= 1e-3 * rr[0]
    s.close()


def test_option_validation():
    with pytest.raises(hm.HelmmgError):
        hm.Solver(32, 32, 1 / 32, 20.0, 0.7, precision="mixed-ff", abc=2)
    with pytest.raises(hm.HelmmgError):
        hm.Solver(32, 32, 1 / 32, 20.0, 0.7, abc=3)
    s = hm.Solver(32, 32, 1 / 32, 20.0, 0.7, abc=2)
    u = torch.zeros((1, 33, 33), dtype=torch.complex128, device="cuda")
    with pytest.raises(hm.HelmmgError):
        s.gradient(u, u, torch.ones((33, 33), dtype=torch.float64, device="cuda"), 10.0)
    s.close()


@pytest.mark.parametrize("cycle,coarse", [("W", {}), ("V", dict(coarse_nodes=10**6, coarse_mode=1)),
                                          ("V", dict(coarse_nodes=0))])
def test_w_cycles_and_coarse_launch_organisations(cycle, coarse):
    """W-cycles, the cooperative coarse-cycle launch over the whole hierarchy
    and no coarse-cycle launch at all: FP64 iterates of cycles 1-2 to 1e-10
    and the cycle count of the whole solve equal the oracle's."""
    n, k = 48, 20.0
    h = 1.0 / n
    opt = ocycle.CycleOptions(2 if cycle == "W" else 1, "gmres3", 2, 2, 4.5)
    H = ohier.build_hierarchy(n, n, h, k, 1 / k, abc=2)
    b = synth.point_source(n, n, h) + 1e-2 * synth.random_complex((n + 1, n + 1), 21) / h**2
    ref = ocycle.mg_solve(H, b.ravel(), 1e-8, opt, keep_iterates=True)
    kw = dict(cycle=cycle, smoother="gmres3", nu_pre=2, nu_post=2, abc=2, **coarse)
    s1 = hm.Solver(n, n, h, k, 1 / k, max_cycles=1, **kw)
    x0 = np.zeros_like(b)
    for m in (1, 2):
        x, st, cyc, _ = s1.solve(dev(b)[None], x=dev(x0)[None], tol=1e-300)
        pu.assert_close(x[0].cpu().numpy(), ref.iterates[m - 1].reshape(n + 1, n + 1), 1e-10, (n + 1, n + 1),
                        f"cycle {m}")
        x0 = ref.iterates[m - 1].reshape(n + 1, n + 1)
    s1.close()
    s = hm.Solver(n, n, h, k, 1 / k, **kw)
    x, st, cyc, rr = s.solve(dev(b)[None], tol=1e-8)
    assert st == hm.MG_OK and cyc[0] == ref.cycles
    s.close()


def test_ragged_batch_with_second_order_rows():
    """A ragged batch with abc=2 (grouped handles; the flattened launches are
    not used with these rows): every problem's one-cycle FP64 iterate equals
    its oracle's to 1e-10 and its whole solve takes the oracle's cycles."""
    sizes = [(48, 48, 30.0), (32, 64, 30.0), (48, 48, 30.0)]
    probs, rhs = [], []
    for q, (nx, ny, k) in enumerate(sizes):
        h = 1.0 / max(nx, ny)
        probs.append((nx, ny, h, k))
        b = synth.point_source(nx, ny, h, i=nx // 2 - q, j=ny // 3 + q)
        rhs.append(torch.from_numpy(b).cuda())
    beta2 = [1.0 / k for _, _, k in sizes]
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    refs = []
    for p, (nx, ny, h, k) in enumerate(probs):
        H = ohier.build_hierarchy(nx, ny, h, k, beta2[p], abc=2)
        refs.append(ocycle.mg_solve(H, rhs[p].cpu().numpy().ravel(), 1e-8, opt, keep_iterates=True))
    for flat in (0, 1):
        rs1 = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, abc=2, flat=flat, max_cycles=1)
        xs, st, cyc, rr = rs1.solve(rhs, tol=1e-300)
        for p, (nx, ny, h, k) in enumerate(probs):
            pu.assert_close(xs[p].cpu().numpy(), refs[p].iterates[0].reshape(ny + 1, nx + 1), 1e-10, (ny + 1, nx + 1),
                            f"flat {flat}, problem {p}")
        rs1.close()
        rs = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, abc=2, flat=flat)
        xs, st, cyc, rr = rs.solve(rhs, tol=1e-8)
        assert st == hm.MG_OK and cyc == [r.cycles for r in refs], flat
        rs.close()
