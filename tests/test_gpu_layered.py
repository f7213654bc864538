"""Variable-k workload: the seeded layered velocity model that stands in
for the 9.2 km x 3.0 km benchmark model, at 10 Hz (h = v_min / (10 f),
grid rounded up to 640 x 224 cells), source near the top centre.  The mixed
paths meet the tolerance in the oracle's FP64 residual; the FP64 path takes
one cycle from the oracle's iterate to the oracle's next iterate to 1e-10."""
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


def _layered(f=10.0):
    h = 1500.0 / (10.0 * f)
    nx, nz = 640, 224
    v = synth.layered_velocity(nx, nz, h, seed=11)
    k = 2 * np.pi * f / v
    b = synth.point_source(nx, nz, h, nx // 2, 2)
    beta2 = 1.0 / (k.max() * nx * h)          # the paper's 1/k_max on the unit square
    return nx, nz, h, k, b, beta2


def test_layered_model_mixed_and_fp64():
    nx, nz, h, k, b, beta2 = _layered()
    kd = torch.from_numpy(k).cuda()
    bd = torch.from_numpy(b).cuda()
    A = oprob.helmholtz_matrix(nx, nz, h, k)
    for precision, march in (("mixed", -1), ("mixed-ff", 1)):
        s = hm.Solver(nx, nz, h, kd, beta2, smoother="gmres3", nu_pre=2, nu_post=2, precision=precision,
                      march=march)
        x, st, cyc, rr = s.solve(bd, tol=1e-6)
        assert st == hm.MG_OK and rr[0] <= 1e-6
        r = b.ravel() - A @ x.cpu().numpy().ravel()
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-6
        s.close()
    # FP64: one cycle from the oracle's iterate equals the oracle's next
    # iterate to 1e-10 node by node (boundary ring included), cycles 1..3
    H = ohier.build_hierarchy(nx, nz, h, k, beta2)
    ref = ocycle.mg_solve(H, b.ravel(), 1e-300, ocycle.CycleOptions(1, "gmres3", 2, 2, 4.5), max_cycles=3,
                          keep_iterates=True)
    s64 = hm.Solver(nx, nz, h, kd, beta2, smoother="gmres3", nu_pre=2, nu_post=2, max_cycles=1)
    shape = (nz + 1, nx + 1)
    for m in (1, 2, 3):
        x0 = np.zeros_like(b) if m == 1 else ref.iterates[m - 2].reshape(shape)
        xm, st1, cm, _ = s64.solve(bd, x=torch.from_numpy(x0).cuda()[None].contiguous(), tol=1e-300)
        assert cm[0] == 1
        pu.assert_close(xm.cpu().numpy()[0], ref.iterates[m - 1].reshape(shape), 1e-10, shape, f"cycle {m}")
    s64.close()
