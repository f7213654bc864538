"""The autotuner on the GPU: it returns one of its candidates, caches it, and
a solver built with the tuned launch shapes reproduces the default solver's
iterate and cycle count (launch shapes do not change the arithmetic)."""
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402
from paper_2308_13476_gb300 import autotune  # noqa: E402


def test_tuned_shapes_reproduce_default(tmp_path):
    n, k = 96, 60.0
    h = 1.0 / n
    rhs = torch.from_numpy(synth.source_row(n, n, h, 3)).cuda()
    space = {"tile_rows": [0, 1, 4], "coarse_nodes": [0, 1100], "coarse_mode": [0, 1]}
    path = os.path.join(tmp_path, "tune.json")
    best, results = autotune.tune(n, n, h, k, 1 / k, rhs, nu=1, space=space, cache_path=path, cycles=2, reps=1)
    assert len(results) == 12 and best in [{kk: r[kk] for kk in space} for r in results]
    assert autotune.tune(n, n, h, k, 1 / k, rhs, nu=1, space=space, cache_path=path)[0] == best   # cached
    ref = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", precision="fp64", batch=3, nu_pre=1, nu_post=1)
    tun = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", precision="fp64", batch=3, nu_pre=1, nu_post=1, **best)
    x1, s1, c1, _ = ref.solve(rhs, tol=1e-8)
    x2, s2, c2, _ = tun.solve(rhs, tol=1e-8)
    assert s1 == s2 == hm.MG_OK and c1 == c2
    a, b = x1.cpu().numpy(), x2.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)


def test_staged_search_over_march_and_chunk_height(tmp_path):
    """The staged search: the second stage (march, chunk height of the
    Kronecker-level marches) runs with the first stage's choice fixed, and
    every chunk height computes the same solve (FP64: the same cycle count,
    iterates equal to 1e-10)."""
    n, k = 128, 60.0
    h = 1.0 / n
    rhs = torch.from_numpy(synth.source_row(n, n, h, 3)).cuda()
    stages = [{"tile_rows": [0, 4]}, {"march": [-1, 1], "kron_chunk": [0, 8, 16]}]
    path = os.path.join(tmp_path, "tune.json")
    best, results = autotune.tune(n, n, h, k, 1 / k, rhs, nu=1, stages=stages, cache_path=path, cycles=2, reps=1)
    assert len(results) == 2 + 6 and set(best) == {"tile_rows", "march", "kron_chunk"}
    assert all(r["tile_rows"] == best["tile_rows"] for r in results[2:])
    ref = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", precision="fp64", batch=3, nu_pre=2, nu_post=2, march=1)
    x0, s0, c0, _ = ref.solve(rhs, tol=1e-9)
    ref.close()
    for ch in (8, 16, 40, 64):
        s = hm.Solver(n, n, h, k, 1 / k, smoother="gmres3", precision="fp64", batch=3, nu_pre=2, nu_post=2, march=1,
                      kron_chunk=ch)
        x, st, c, _ = s.solve(rhs, tol=1e-9)
        assert st == hm.MG_OK and c == c0, ch
        a, b = x0.cpu().numpy(), x.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a), ch
        s.close()
