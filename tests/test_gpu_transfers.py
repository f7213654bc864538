"""GPU parity of the linear-interpolation transfers (mg_options.transfer = 1,
the "Linear" column of Table conv1) against the oracle's hierarchy built
with kind="linear", through the C-ABI.  Same bars as the Eq. (xex) path:
operators and Galerkin stencils to 1e-13, Jacobi iterates to 1e-10 with
identical cycle counts, GMRES(3) one-cycle iterates to 1e-10 and whole
solves to 1e-6, the mixed path to 1e-6 of the FP64 oracle solution."""
import numpy as np
import pytest

import synth
from oracle import cycle as ocycle
from oracle import hierarchy as ohier

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


# every implementation of the transfers: grid kernels (fused residual +
# restriction), unfused grid kernels, the single-CTA and the cooperative
# coarse-cycle interpreters
MODES = [dict(coarse_nodes=0), dict(coarse_nodes=0, fuse=0), dict(coarse_nodes=10**6, coarse_mode=0),
         dict(coarse_nodes=1200, coarse_mode=1)]
MODE_IDS = ["grid", "grid_unfused", "cta", "hybrid_coop"]


@pytest.mark.parametrize("nx,ny,kvar", [(32, 32, False), (40, 24, True)])
def test_linear_operators_and_galerkin_stencils(nx, ny, kvar):
    h = 1.0 / 32
    k = synth.k_field(synth.chi_sharp(nx, ny, 7), 10.0, 20.0) if kvar else 20.0
    H = ohier.build_hierarchy(nx, ny, h, k, 0.7, kind="linear")
    Hb = ohier.build_hierarchy(nx, ny, h, k, 0.7)
    s = hm.Solver(nx, ny, h, dev(k, torch.float64) if kvar else k, 0.7, transfer="linear")
    for l, (cx_, cy_) in enumerate(H.sizes):
        gnx, gny, r, _ = s.level_info(l)
        assert (gnx, gny) == (cx_, cy_)
        x = synth.random_complex((cy_ + 1, cx_ + 1), 200 + l)
        y = host(s.apply(l, dev(x)[None]))[0]
        ref = (H.A[l] @ x.ravel()).reshape(x.shape)
        assert rel(y, ref) <= 1e-13, l
        if l > 0:   # the option changes the coarse operators
            assert rel(ref, (Hb.A[l] @ x.ravel()).reshape(x.shape)) > 1e-3
        S = host(s.stencil(l))
        So = ohier.stencil_of(H.A[l], cx_, cy_, r)
        assert np.abs(S - So).max() <= 1e-13 * np.abs(So).max(), l
    s.close()


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_linear_jacobi_iterates(mode):
    n, k = 32, 20.0
    h = 1.0 / n
    b = synth.point_source(n, n, h)
    H = ohier.build_hierarchy(n, n, h, k, 0.7, kind="linear")
    ref = ocycle.mg_solve(H, b.ravel(), 1e-6, ocycle.CycleOptions(1, "jacobi", 1, 1, 4.5))
    assert ref.converged
    s = hm.Solver(n, n, h, k, 0.7, transfer="linear", **mode)
    x, st, cyc, rr = s.solve(dev(b), tol=1e-6)
    assert st == hm.MG_OK and cyc[0] == ref.cycles
    assert rel(host(x)[0], ref.x) <= 1e-10
    hist = np.array(s.history(ref.cycles)[0])
    assert np.allclose(hist, ref.history, rtol=1e-9, atol=0)
    s.close()


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_linear_gmres_iterates(mode):
    n, k = 64, 40.0
    h = 1.0 / n
    b = synth.point_source(n, n, h)
    H = ohier.build_hierarchy(n, n, h, k, 1 / k, kind="linear")
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    ref = ocycle.mg_solve(H, b.ravel(), 1e-6, opt, keep_iterates=True)
    assert ref.converged
    s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, transfer="linear", **mode)
    x, st, cyc, rr = s.solve(dev(b), tol=1e-6)
    assert st == hm.MG_OK and cyc[0] == ref.cycles
    assert rel(host(x)[0], ref.x) <= 1e-6
    s.close()
    s1 = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, transfer="linear", max_cycles=1,
                   **mode)
    for m in sorted({1, ref.cycles // 2, ref.cycles}):
        x0 = np.zeros_like(b) if m == 1 else ref.iterates[m - 2].reshape(b.shape)
        xm, st1, cm, _ = s1.solve(dev(b), x=dev(x0)[None].contiguous(), tol=1e-300)
        assert st1 == hm.MG_EMAXIT and cm[0] == 1
        assert rel(host(xm)[0], ref.iterates[m - 1]) <= 1e-10, m
    s1.close()


def test_linear_mixed_and_the_ablation_counts():
    """Mixed precision with linear transfers meets the FP64 oracle, and the
    GPU reproduces the oracle's cycle counts for both transfers on a case
    where the choice matters (GMRES(3) V(2,2), k = 40)."""
    n, k = 64, 40.0
    h = 1.0 / n
    b = synth.point_source(n, n, h)
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    counts = {}
    for kind in ("bezier", "linear"):
        H = ohier.build_hierarchy(n, n, h, k, 1 / k, kind=kind)
        ref = ocycle.mg_solve(H, b.ravel(), 1e-6, opt)
        s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, transfer=kind)
        _, st, cyc, _ = s.solve(dev(b), tol=1e-6)
        assert st == hm.MG_OK and cyc[0] == ref.cycles
        counts[kind] = cyc[0]
        s.close()
    assert counts["linear"] > counts["bezier"]
    H = ohier.build_hierarchy(n, n, h, k, 1 / k, kind="linear")
    ref = ocycle.mg_solve(H, b.ravel(), 1e-12, opt)
    s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, transfer="linear", precision="mixed")
    x, st, cyc, rr = s.solve(dev(b), tol=1e-10)
    assert st == hm.MG_OK
    assert rel(host(x)[0], ref.x) <= 1e-6
    s.close()


def test_linear_transfers_fail_at_scale_where_bezier_converges():
    """The ablation at scale (8 sources on 513^2, k = 150, GMRES(3) V(2,2),
    mixed): Eq. (xex) converges in about 20 cycles; with linear
    interpolation the cycle does not reach 1e-6 (it diverges or stalls)."""
    n, k = 512, 150.0
    h = 1.0 / n
    b = dev(synth.source_row(n, n, h, 8))
    cyc = {}
    for kind in ("bezier", "linear"):
        s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", nu_pre=2, nu_post=2, precision="mixed", batch=8,
                      transfer=kind, max_cycles=400)
        _, st, c, _ = s.solve(b, tol=1e-6)
        cyc[kind] = (st, c)
        s.close()
    st, c = cyc["bezier"]
    assert st == hm.MG_OK and max(c) <= 30
    st, c = cyc["linear"]
    assert st in (hm.MG_EDIVERGED, hm.MG_EMAXIT)
