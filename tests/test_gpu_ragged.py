"""Ragged batch: problems of different sizes in one handle; each problem's
result and cycle count must equal the oracle's solve of that problem alone."""
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
