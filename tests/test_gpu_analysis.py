"""GPU two-grid analysis (mg_two_grid) against the oracle's dense two-grid
matrices (oracle/analysis.py) and the printed Table conv1.

Bars: ||T0||_2 within 1e-9 of the oracle's SVD (the power method stops when
its Rayleigh quotient settles to 1e-14), the HPD verdict on Gamma~ equal to
the oracle's Cholesky test, ||Gamma~||_1 / kappa_1(Gamma~) within 1e-8 of
numpy's, and the Bezier + CSL column of Table conv1 within 0.02.
"""
import numpy as np
import pytest

import synth
from oracle import analysis as oan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402

# Table conv1 (tests/golden/table_conv1.txt): k, Linear/A, Linear/C, Bezier/A, Bezier/C
CONV1 = {5: (2.284, 1.304, 0.991, 0.911), 10: (5.888, 1.351, 1.105, 0.913), 20: (8.786, 1.328, 1.306, 0.951)}


def oracle_parts(n, k, beta2, kind, coarsen_on, omega=4.5, nu=1):
    A, P, R, Ac = oan.two_grid_parts(n, n, 1.0 / n, k, beta2, kind=kind, coarsen_on=coarsen_on)
    T0 = oan.two_grid_matrix(A, P, R, Ac, omega, nu)
    G = oan.gamma_tilde(A, P, R, Ac, omega)
    return np.linalg.norm(T0, 2), oan.is_hpd(G), np.linalg.norm(G, 1) / np.linalg.cond(G, 1)


@pytest.mark.parametrize("k", [5, 10, 20])
@pytest.mark.parametrize("kind,coarsen_on", [("bezier", "C"), ("bezier", "A"), ("linear", "A"), ("linear", "C")])
def test_two_grid_matches_oracle_and_table_conv1(k, kind, coarsen_on):
    n = int(round(k / 0.625))
    beta2 = 0.7 if coarsen_on == "C" else 0.0
    s = hm.Solver(n, n, 1.0 / n, float(k), beta2, transfer=kind)
    r = s.two_grid(nu=1)
    s.close()
    norm, hpd, ratio = oracle_parts(n, float(k), 0.7, kind, coarsen_on)
    assert r["converged"] and not r["coarse_singular"]
    assert abs(r["norm_t0"] - norm) <= 1e-9 * norm, (r, norm)
    assert r["hpd"] == hpd
    assert abs(r["gamma_ratio"] - ratio) <= 1e-8 * ratio, (r, ratio)
    col = {("linear", "A"): 0, ("linear", "C"): 1, ("bezier", "A"): 2, ("bezier", "C"): 3}[(kind, coarsen_on)]
    if (kind, coarsen_on) == ("bezier", "C"):
        assert abs(r["norm_t0"] - CONV1[k][col]) < 0.02
        assert r["norm_t0"] < 1.0 and r["hpd"]
    if kind == "linear":
        assert r["norm_t0"] > 1.0


@pytest.mark.parametrize("nu,omega", [(2, 4.5), (3, 4.5), (1, 2.5)])
def test_two_grid_smoothing_steps_and_omega(nu, omega):
    n, k = 16, 10.0
    s = hm.Solver(n, n, 1.0 / n, k, 0.7, omega=omega)
    r = s.two_grid(nu=nu)
    s.close()
    norm, hpd, ratio = oracle_parts(n, k, 0.7, "bezier", "C", omega=omega, nu=nu)
    assert abs(r["norm_t0"] - norm) <= 1e-9 * norm
    assert r["hpd"] == hpd and abs(r["gamma_ratio"] - ratio) <= 1e-8 * ratio


def test_two_grid_variable_k_and_rectangle():
    nx, ny = 24, 16
    h = 1.0 / 24
    kf = synth.k_field(synth.chi_sharp(nx, ny, 5), 8.0, 15.0)
    s = hm.Solver(nx, ny, h, torch.from_numpy(kf).cuda(), 0.7)
    r = s.two_grid(nu=1)
    s.close()
    A, P, R, Ac = oan.two_grid_parts(nx, ny, h, kf, 0.7, coarsen_on="C")
    T0 = oan.two_grid_matrix(A, P, R, Ac, 4.5, 1)
    G = oan.gamma_tilde(A, P, R, Ac, 4.5)
    norm = np.linalg.norm(T0, 2)
    assert abs(r["norm_t0"] - norm) <= 1e-9 * norm
    assert r["hpd"] == oan.is_hpd(G)
    ratio = np.linalg.norm(G, 1) / np.linalg.cond(G, 1)
    assert abs(r["gamma_ratio"] - ratio) <= 1e-8 * ratio


def test_two_grid_rejects_large_or_one_level_grids():
    s = hm.Solver(64, 64, 1.0 / 64, 40.0, 0.7)
    with pytest.raises(hm.HelmmgError, match="4096"):
        s.two_grid()
    s.close()
    s = hm.Solver(16, 16, 1.0 / 16, 10.0, 0.7, levels=1)
    with pytest.raises(hm.HelmmgError, match="two levels"):
        s.two_grid()
    s.close()
