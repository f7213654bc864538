"""Ragged batch: problems of different sizes in one handle; each problem's
result and cycle count must equal the oracle's solve of that problem alone,
whether the batch runs one flattened launch per kernel over all problems or
one cycle graph per problem (the two agree bit for bit)."""
import numpy as np
import pytest

import parity_util as pu
import synth
from oracle import cycle as ocycle
from oracle import hierarchy as ohier
from oracle import problem as oprob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402


@pytest.mark.parametrize("smoother,beta2", [("jacobi", 0.7), ("gmres3", 0.05)])
def test_ragged_batch_matches_oracle_per_problem(smoother, beta2):
    sizes = [(32, 32, 20.0), (48, 24, 25.0), (40, 40, 25.0), (28, 56, 30.0)]
    probs, rhs = [], []
    for nx, ny, k in sizes:
        h = 1.0 / max(nx, ny)
        probs.append((nx, ny, h, k))
        rhs.append(torch.from_numpy(synth.point_source(nx, ny, h)).cuda())
    rs = hm.RaggedSolver(probs, beta2, smoother=smoother, nu_pre=2, nu_post=2)
    xs, st, cyc, rr = rs.solve(rhs, tol=1e-7)
    assert st == hm.MG_OK
    opt = ocycle.CycleOptions(1, smoother, 2, 2, 4.5)
    for p, (nx, ny, h, k) in enumerate(probs):
        H = ohier.build_hierarchy(nx, ny, h, k, beta2)
        ref = ocycle.mg_solve(H, rhs[p].cpu().numpy().ravel(), 1e-7, opt)
        assert cyc[p] == ref.cycles, p
        x = xs[p].cpu().numpy().ravel()
        bound = 1e-10 if smoother == "jacobi" else 1e-6
        assert np.linalg.norm(x - ref.x) <= bound * np.linalg.norm(ref.x), p
    rs.close()


# Problems large enough that the flattened launches cover the fine level's
# row marches, Kronecker levels of both radii and the coarse-cycle launch.
FLAT_SIZES = [(160, 160, 100.0), (128, 64, 80.0), (96, 96, 60.0), (32, 32, 20.0), (64, 128, 70.0)]


def _ragged(sizes, **kw):
    probs, rhs = [], []
    for q, (nx, ny, k) in enumerate(sizes):
        h = 1.0 / max(nx, ny)
        probs.append((nx, ny, h, k))
        b = synth.point_source(nx, ny, h) + 1e-2 * synth.random_complex((ny + 1, nx + 1), 40 + q) / h**2
        rhs.append(torch.from_numpy(b).cuda())
    beta2 = [1.0 / k for _, _, k in sizes]
    return probs, rhs, beta2


@pytest.mark.parametrize("precision,cycle", [("fp64", "V"), ("mixed", "V"), ("fp64", "W")])
def test_flattened_launches_equal_per_problem_graphs(precision, cycle):
    """One launch per kernel over all problems (flat=1) computes, problem by
    problem, bit for bit what each problem's own cycle graph computes
    (flat=0): the same kernel bodies on the same geometries, with every
    reduction in a fixed order."""
    probs, rhs, beta2 = _ragged(FLAT_SIZES)
    out = []
    for flat in (1, 0):
        rs = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, precision=precision,
                             cycle=cycle, march=1, flat=flat)
        xs, st, cyc, rr = rs.solve(rhs, tol=1e-8)
        assert st == hm.MG_OK
        out.append(([x.cpu().numpy() for x in xs], cyc, rr))
        rs.close()
    (x1, c1, r1), (x0, c0, r0) = out
    assert c1 == c0 and r1 == r0
    for p in range(len(probs)):
        assert np.array_equal(x1[p], x0[p]), p


def test_flattened_ragged_matches_oracle():
    """FP64, flattened: one cycle from x = 0 equals each problem's oracle
    iterate to 1e-10 node by node, and the whole solve takes each problem's
    oracle cycle count."""
    probs, rhs, beta2 = _ragged(FLAT_SIZES)
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    refs = []
    for p, (nx, ny, h, k) in enumerate(probs):
        H = ohier.build_hierarchy(nx, ny, h, k, beta2[p])
        refs.append(ocycle.mg_solve(H, rhs[p].cpu().numpy().ravel(), 1e-7, opt, keep_iterates=True))
    rs1 = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, max_cycles=1)
    xs, st, cyc, rr = rs1.solve(rhs, tol=1e-300)
    assert st == hm.MG_EMAXIT and all(c == 1 for c in cyc)
    for p, (nx, ny, h, k) in enumerate(probs):
        pu.assert_close(xs[p].cpu().numpy(), refs[p].iterates[0].reshape(ny + 1, nx + 1), 1e-10, (ny + 1, nx + 1),
                        f"problem {p}")
    rs1.close()
    rs = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2)
    xs, st, cyc, rr = rs.solve(rhs, tol=1e-7)
    assert st == hm.MG_OK
    for p in range(len(probs)):
        assert cyc[p] == refs[p].cycles, p
        pu.assert_close(xs[p].cpu().numpy().ravel(), refs[p].x, 1e-6, None, f"problem {p}")
    rs.close()


# Repeated shapes: with flat = 0 the problems of one shape share a batched
# handle (their right-hand sides side by side); each must still get its own
# oracle solve.
GROUPED_SIZES = [(64, 64, 40.0), (48, 96, 45.0), (64, 64, 40.0), (32, 32, 20.0), (48, 96, 45.0), (64, 64, 40.0)]


def _ragged_distinct_rhs(sizes):
    probs, rhs = [], []
    for q, (nx, ny, k) in enumerate(sizes):
        h = 1.0 / max(nx, ny)
        probs.append((nx, ny, h, k))
        b = synth.point_source(nx, ny, h, i=(q * 7) % (nx - 1) + 1, j=(q * 5) % (ny - 1) + 1)
        b = b + 1e-2 * synth.random_complex((ny + 1, nx + 1), 70 + q) / h**2
        rhs.append(torch.from_numpy(b).cuda())
    return probs, rhs, [1.0 / k for _, _, k in sizes]


def test_grouped_problems_match_oracle():
    """flat = 0 with repeated shapes, FP64: one cycle from x = 0 equals each
    problem's oracle iterate to 1e-10 node by node, and the whole solve takes
    each problem's oracle cycle count, results scattered back in the
    caller's order."""
    probs, rhs, beta2 = _ragged_distinct_rhs(GROUPED_SIZES)
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    refs = []
    for p, (nx, ny, h, k) in enumerate(probs):
        H = ohier.build_hierarchy(nx, ny, h, k, beta2[p])
        refs.append(ocycle.mg_solve(H, rhs[p].cpu().numpy().ravel(), 1e-7, opt, keep_iterates=True))
    rs1 = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, flat=0, max_cycles=1)
    xs, st, cyc, rr = rs1.solve(rhs, tol=1e-300)
    assert st == hm.MG_EMAXIT and all(c == 1 for c in cyc)
    for p, (nx, ny, h, k) in enumerate(probs):
        pu.assert_close(xs[p].cpu().numpy(), refs[p].iterates[0].reshape(ny + 1, nx + 1), 1e-10, (ny + 1, nx + 1),
                        f"problem {p}")
    rs1.close()
    rs = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, flat=0)
    xs, st, cyc, rr = rs.solve(rhs, tol=1e-7)
    assert st == hm.MG_OK
    for p in range(len(probs)):
        assert cyc[p] == refs[p].cycles, p
        pu.assert_close(xs[p].cpu().numpy().ravel(), refs[p].x, 1e-6, None, f"problem {p}")
    rs.close()


def test_grouped_problems_mixed_precision():
    """flat = 0 with repeated shapes, mixed path: every problem's FP64
    residual, recomputed with the oracle's matrix, meets the tolerance and
    equals the reported one; the cycle counts are within one of the
    oracle's."""
    probs, rhs, beta2 = _ragged_distinct_rhs(GROUPED_SIZES)
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    rs = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, precision="mixed", flat=0)
    xs, st, cyc, rr = rs.solve(rhs, tol=1e-7)
    assert st == hm.MG_OK
    for p, (nx, ny, h, k) in enumerate(probs):
        b = rhs[p].cpu().numpy().ravel()
        A = oprob.helmholtz_matrix(nx, ny, h, k)
        r = b - A @ xs[p].cpu().numpy().ravel()
        rel = np.linalg.norm(r) / np.linalg.norm(b)
        assert rel <= 1e-7 and abs(rel - rr[p]) <= 1e-3 * rr[p], p
        H = ohier.build_hierarchy(nx, ny, h, k, beta2[p])
        ref = ocycle.mg_solve(H, b, 1e-7, opt)
        assert abs(cyc[p] - ref.cycles) <= 1, p
    rs.close()


def test_grouped_problems_with_fgmres():
    """The grouped handles also serve the FGMRES outer loop: each problem
    equals the same solve through its own single-problem handle to the solve
    tolerance."""
    probs, rhs, beta2 = _ragged_distinct_rhs(GROUPED_SIZES)
    for kw in (dict(krylov=5), dict()):
        rs = hm.RaggedSolver(probs, beta2, smoother="gmres3", nu_pre=2, nu_post=2, precision="fp64", flat=0, **kw)
        xs, st, cyc, rr = rs.solve(rhs, tol=1e-10)
        assert st == hm.MG_OK
        for p, (nx, ny, h, k) in enumerate(probs):
            s = hm.Solver(nx, ny, h, k, beta2[p], smoother="gmres3", nu_pre=2, nu_post=2, precision="fp64", **kw)
            x1, st1, cyc1, rr1 = s.solve(rhs[p], tol=1e-10)
            assert st1 == hm.MG_OK and abs(cyc1[0] - cyc[p]) <= 1, p
            pu.assert_close(xs[p].cpu().numpy().ravel(), x1.cpu().numpy().ravel(), 1e-8, None, f"problem {p}")
            s.close()
        rs.close()
