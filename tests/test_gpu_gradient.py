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


# ---- the gradient workload's stated arithmetic, at a larger size ----------
#
# 65^2 nodes, 4 sources, receivers every other node of the first interior
# row, and 20 seeded smooth finite-difference directions, for the FP64 path (solves
# to 1e-10) and for the mixed path (complex64 cycles inside FP64 refinement,
# the arithmetic the gradient workload runs in).  The mixed gradient is
# compared with the oracle's adjoint-state gradient at the solve tolerance
# of the workload (1e-6) and must agree to 1e-2 relative; its difference
# quotients are taken from solves to 1e-9, so that solve noise stays far
# below the 1e-2 bar.  The FP64 difference quotients come from solves to
# 1e-12 (see below).

def _fd_check(n, nsrc, precision, tol_grad, tol_fd, eps, bar, seed):
    n, h, omega_f, m, src, rec, data = _setup(n=n, nsrc=nsrc, seed=seed)
    base = dict(smoother="gmres3", nu_pre=2, nu_post=2, precision=precision)
    args = (_t(src, torch.complex128), _t(rec, torch.int64), _t(data, torch.complex128), (n, n, h, omega_f))
    mt = _t(m, torch.float64).requires_grad_(True)
    hag.misfit(mt, *args, tol=tol_grad, **base).backward()
    g = mt.grad.cpu().numpy()
    worst = 0.0
    for q in range(20):
        # smooth seeded directions: the misfit responds to them well above
        # the solve noise (white-noise directions project weakly onto it)
        d = synth.smooth_perturbation(n, n, 1000 * seed + q, sigma_nodes=n / 16) * m
        Lp = float(hag.misfit(_t(m + eps * d, torch.float64), *args, tol=tol_fd, **base))
        Lm = float(hag.misfit(_t(m - eps * d, torch.float64), *args, tol=tol_fd, **base))
        fd = (Lp - Lm) / (2 * eps)
        ad = float(np.sum(g * d))
        worst = max(worst, abs(fd - ad) / abs(ad))
    assert worst <= bar, worst
    return n, h, omega_f, m, src, rec, data, g


def test_fp64_gradient_20_directions_65():
    # solves to 1e-12: at 65^2 the solution error of a 1e-10 solve already
    # moves the difference quotients by ~1e-4 of the derivative
    _fd_check(64, 4, "fp64", 1e-12, 1e-12, 1e-5, 1e-5, seed=7)


def test_mixed_gradient_against_oracle_and_20_directions():
    n, h, omega_f, m, src, rec, data, g_fd = _fd_check(64, 4, "mixed", 1e-9, 1e-9, 1e-4, 1e-2, seed=8)
    F = src.reshape(src.shape[0], -1).T
    g_ref = ograd.gradient(n, n, h, m, omega_f, F, rec, data.T)
    # at the workload's tolerance
    mt = _t(m, torch.float64).requires_grad_(True)
    L = hag.misfit(mt, _t(src, torch.complex128), _t(rec, torch.int64), _t(data, torch.complex128),
                   (n, n, h, omega_f), tol=1e-6, smoother="gmres3", nu_pre=2, nu_post=2, precision="mixed")
    L.backward()
    g6 = mt.grad.cpu().numpy()
    assert np.linalg.norm(g6 - g_ref) <= 1e-2 * np.linalg.norm(g_ref)
    assert np.linalg.norm(g_fd - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
