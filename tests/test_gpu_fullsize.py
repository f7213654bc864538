"""Full-size FP64 parity at the batched workload's launch geometry.

The batched workload solves 64 point sources on a 1025 x 1025 grid at
k = 300 with GMRES(3) V(2,2) cycles, beta2 = 1/k.  Here the FP64 path runs
that batch with the library's default options (the automatic choice of row
and column marches, the occupancy-based chunk heights of the column marches
and the coarse interpreter), i.e. the launch geometry of the bench apart
from the precision, and sampled right-hand sides are compared with the
oracle, which computes them one at a time:

* one cycle from x = 0, and one cycle from the oracle's first iterate,
  each equal to the oracle's next iterate to 1e-10 node by node, with the
  boundary ring checked on its own;
* the whole FP64 solve takes, for the first right-hand side, the cycle count
  the oracle needs for it (``oracle/bench_cycles.json``, written by
  ``python -m oracle.bench_cycles --k 300 --n 1024 --batch 64``);
* the mixed-precision solve of the same batch (the bench's arithmetic): the
  FP64 residual of the returned x, formed with the oracle's matrix, meets
  the tolerance and equals the reported one for the sampled right-hand sides.
"""
import json
import os

import numpy as np
import pytest

import parity_util as pu
import synth
from oracle import cycle as ocycle
from oracle import hierarchy as ohier

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402

N, K, B = 1024, 300.0, 64
SAMPLED = (0, 37, 63)
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def workload():
    h = 1.0 / N
    src = synth.source_row(N, N, h, B)
    H = ohier.build_hierarchy(N, N, h, K, 1.0 / K)
    opt = ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5)
    refs = {q: ocycle.mg_solve(H, src[q].ravel(), 1e-300, opt, max_cycles=2, keep_iterates=True)
            for q in SAMPLED}
    return h, src, H, refs


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda")


def test_fullsize_fp64_one_cycle_matches_oracle(workload):
    h, src, H, refs = workload
    shape = (N + 1, N + 1)
    s1 = hm.Solver(N, N, h, K, 1.0 / K, smoother="gmres3", nu_pre=2, nu_post=2, batch=B, max_cycles=1)
    b = _dev(src)
    for m in (1, 2):
        x0 = np.zeros_like(src)
        if m == 2:
            for q in SAMPLED:
                x0[q] = refs[q].iterates[0].reshape(shape)
        x, st, cyc, _ = s1.solve(b, x=_dev(x0), tol=1e-300)
        assert st == hm.MG_EMAXIT and all(c == 1 for c in cyc)
        xh = x.cpu().numpy()
        for q in SAMPLED:
            pu.assert_close(xh[q], refs[q].iterates[m - 1].reshape(shape), 1e-10, shape, f"rhs {q}, cycle {m}")
    s1.close()


def test_fullsize_cycle_counts_and_mixed_residuals(workload):
    h, src, H, refs = workload
    with open(os.path.join(ROOT, "oracle", "bench_cycles.json")) as f:
        oracle_cycles = json.load(f)["300/1024/gmres3/V2/0.00333333"]
    b = _dev(src)
    s = hm.Solver(N, N, h, K, 1.0 / K, smoother="gmres3", nu_pre=2, nu_post=2, batch=B)
    x, st, cyc, rr = s.solve(b, tol=1e-6)
    assert st == hm.MG_OK and cyc[0] == oracle_cycles
    s.close()
    sm = hm.Solver(N, N, h, K, 1.0 / K, smoother="gmres3", nu_pre=2, nu_post=2, batch=B, precision="mixed")
    x, st, cyc, rr = sm.solve(b, tol=1e-6)
    assert st == hm.MG_OK and max(rr) <= 1e-6
    xh = x.cpu().numpy()
    for q in SAMPLED:
        bq = src[q].ravel()
        r = np.linalg.norm(bq - H.A[0] @ xh[q].ravel()) / np.linalg.norm(bq)
        assert r <= 1e-6 and abs(r - rr[q]) <= 1e-3 * rr[q], (q, r, rr[q])
    sm.close()
