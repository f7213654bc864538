"""mg_profile: every `what` runs through the C-ABI, reports a positive time and
the documented algorithmic byte count, and leaves the handle usable (a solve
afterwards still equals the oracle's)."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed-ff"])
def test_profile_all_kinds_then_solve(precision):
    n, B, k = 64, 2, 20.0
    h = 1.0 / n
    s = hm.Solver(n, n, h, k, 0.05, smoother="gmres3", nu_pre=2, nu_post=2, precision=precision, batch=B,
                  march=1)
    e = 16 if precision == "fp64" else 8
    nodes = (n + 1) ** 2 * B
    # what 4, a fine-level GMRES(3) step: 16 vector passes in complex128, 13
    # in complex64 (no fourth march pass: the last Arnoldi vector's norm comes
    # from the Gram form)
    expect = {0: 3 * e, 1: 3 * e, 2: 1.25 * e, 3: 2.25 * e, 4: (16 if precision == "fp64" else 13) * e}
    for what, per_node in expect.items():
        ms, nbytes = s.profile(what, 0, reps=3)
        assert ms > 0
        assert abs(nbytes - per_node * nodes) <= 1e-9 * nbytes, what
    # level 1 (Kronecker form): column marches, two of them fused and no
    # closing norm pass in complex64 (19 vector passes), the eight unfused
    # passes in complex128 (28)
    ms, nbytes = s.profile(4, 1, reps=2)
    vec1 = 28 if precision == "fp64" else 19
    assert ms > 0 and abs(nbytes - vec1 * e * (n // 2 + 1) ** 2 * B) <= 1e-9 * nbytes
    rhs = torch.from_numpy(np.stack([synth.point_source(n, n, h)] * B)).cuda()
    x, st, cyc, rr = s.solve(rhs, tol=1e-8)
    assert st == hm.MG_OK
    H = ohier.build_hierarchy(n, n, h, k, 0.05)
    ref = ocycle.mg_solve(H, rhs[0].cpu().numpy().ravel(), 1e-8, ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5))
    assert list(cyc) == [ref.cycles] * B
    # whole-solve bar of GMRES(3) (its rounding is amplified through a
    # nonlinear map; see test_gpu_parity)
    bound = 1e-6
    for b in range(B):
        assert np.linalg.norm(x[b].cpu().numpy().ravel() - ref.x) <= bound * np.linalg.norm(ref.x)
    s.close()


def test_profile_gmres_step_needs_gmres_smoother():
    s = hm.Solver(32, 32, 1.0 / 32, 10.0, 0.7, smoother="jacobi")
    with pytest.raises(hm.HelmmgError, match="GMRES"):
        s.profile(4, 0, reps=1)
    s.close()
