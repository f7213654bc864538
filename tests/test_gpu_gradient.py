"""Adjoint gradient through torch.autograd against the oracle's adjoint-state
gradient (direct sparse solves) and against central finite differences of
the misfit computed by the GPU solver itself."""
import numpy as np
import pytest

import synth
from oracle import gradient as ograd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2308_13476_gb300 import autograd as hag  # noqa: E402


def _setup(n=32, nsrc=3, seed=5):
    # a small version of the 15 Hz gradient workload: 2000 m/s background,
    # +-10 % smooth perturbation of the squared slowness, kh <= 0.6 everywhere
    omega_f = 2 * np.pi * 15.0
    m0 = np.full((n + 1, n + 1), 1.0 / 2000.0**2)
    m = m0 * (1 + 0.1 * synth.smooth_perturbation(n, n, seed, sigma_nodes=n / 8))
    h = 0.6 / (omega_f * np.sqrt(m.max()))
    src = synth.source_row(n, n, h, nsrc)
    rec = np.array([(n - 1) * (n + 1) + i for i in range(1, n, 2)])
    F = src.reshape(nsrc, -1).T
    D, _ = ograd.forward(n, n, h, m0, omega_f, F)
    data = D[rec, :].T.copy()
    return n, h, omega_f, m, src, rec, data


def _t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def test_autograd_gradient_matches_oracle_adjoint_state():
    n, h, omega_f, m, src, rec, data = _setup()
    mt = _t(m, torch.float64).requires_grad_(True)
    L = hag.misfit(mt, _t(src, torch.complex128), _t(rec, torch.int64), _t(data, torch.complex128),
                   (n, n, h, omega_f), tol=1e-12, smoother="gmres3", nu_pre=2, nu_post=2)
    L.backward()
    g = mt.grad.cpu().numpy()
    F = src.reshape(src.shape[0], -1).T
    g_ref = ograd.gradient(n, n, h, m, omega_f, F, rec, data.T)
    L_ref = ograd.misfit(n, n, h, m, omega_f, F, rec, data.T)
    assert abs(float(L.detach()) - L_ref) <= 1e-9 * L_ref
    assert np.linalg.norm(g - g_ref) <= 1e-7 * np.linalg.norm(g_ref)


def test_autograd_gradient_matches_central_differences():
    n, h, omega_f, m, src, rec, data = _setup(seed=6)
    kw = dict(tol=1e-12, smoother="gmres3", nu_pre=2, nu_post=2)
    args = (_t(src, torch.complex128), _t(rec, torch.int64), _t(data, torch.complex128), (n, n, h, omega_f))
    mt = _t(m, torch.float64).requires_grad_(True)
    hag.misfit(mt, *args, **kw).backward()
    g = mt.grad.cpu().numpy()
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.standard_normal(m.shape) * m
        eps = 1e-5
        Lp = float(hag.misfit(_t(m + eps * d, torch.float64), *args, **kw))
        Lm = float(hag.misfit(_t(m - eps * d, torch.float64), *args, **kw))
        fd = (Lp - Lm) / (2 * eps)
        ad = float(np.sum(g * d))
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
