"""Pins of the oracle's second-order absorbing rows (abc=2, the Engquist-Majda
condition d u/dn - i k u - (i/2k) d^2 u/dtau^2 = 0; a variant the paper does
not use) against what the mathematics fixes: the symmetry of the weak form,
the tangential stiffness annihilating functions constant along the boundary,
and the boundary residual of exact outgoing plane waves, which must follow
the paraxial theory: k |cos t - 1| for the first-order rows, k |cos t - 1 +
sin^2 t / 2| for the second-order ones (a wrong sign, factor or power of k in
the tangential term fails it)."""
import numpy as np
import pytest

from oracle import cycle as ocycle
from oracle import hierarchy as ohier
from oracle import problem as oprob


@pytest.mark.parametrize("variable", [False, True])
def test_abc2_rows_are_complex_symmetric(variable):
    nx, ny, h = 12, 8, 1.0 / 12
    k = 20.0 if not variable else 15.0 + 10.0 * np.random.default_rng(3).random((ny + 1, nx + 1))
    for b2 in (0.0, 0.5):
        A = oprob.helmholtz_matrix(nx, ny, h, k, b2, abc=2)
        assert abs(A - A.T).max() == 0.0


def test_tangential_stiffness_annihilates_constants_and_lives_on_the_boundary():
    nx, ny, h = 10, 7, 0.1
    k = 5.0 + np.random.default_rng(4).random((ny + 1, nx + 1))
    T = oprob.tangential_abc2(nx, ny, h, k)
    assert np.abs(T @ np.ones(T.shape[0])).max() < 1e-9 * abs(T).max()
    D = (oprob.helmholtz_matrix(nx, ny, h, k, abc=2) - oprob.helmholtz_matrix(nx, ny, h, k)).tocoo()
    ii, jj = D.row % (nx + 1), D.row // (nx + 1)
    assert np.all((ii == 0) | (ii == nx) | (jj == 0) | (jj == ny))
    # an edge node couples to its two neighbours along the side (equally for
    # constant k), a corner to one on each side
    Td = oprob.tangential_abc2(nx, ny, h, 6.0).toarray()
    edge = oprob.node_index(nx, 0, 3)
    assert np.count_nonzero(Td[edge]) == 3
    assert Td[edge, oprob.node_index(nx, 0, 2)] == Td[edge, oprob.node_index(nx, 0, 4)]
    corner = oprob.node_index(nx, 0, 0)
    assert set(np.nonzero(Td[corner])[0]) == {corner, oprob.node_index(nx, 1, 0), oprob.node_index(nx, 0, 1)}


@pytest.mark.parametrize("theta_deg", [0.0, 20.0, 35.0, 50.0])
def test_plane_wave_boundary_residual_follows_the_paraxial_theory(theta_deg):
    """An outgoing plane wave through the left side x = 0 (travelling in -x,
    angle t to the normal) leaves, in row P of a left-edge node, h (A u)_P =
    i k (cos t - 1 + s sin^2 t / 2) u_P + O(h k^2) (s = 0 first-order rows,
    s = 1 second-order rows)."""
    k, n = 10.0, 800
    h = 1.0 / n
    t = np.deg2rad(theta_deg)
    x = np.arange(n + 1) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.exp(-1j * k * X * np.cos(t) + 1j * k * Y * np.sin(t)).ravel()
    rows = [oprob.node_index(n, 0, j) for j in range(n // 4, 3 * n // 4, n // 16)]
    for abc, s in ((1, 0.0), (2, 1.0)):
        A = oprob.helmholtz_matrix(n, n, h, k, abc=abc)
        r = h * (A @ u)[rows] / u[rows]
        want = 1j * k * (np.cos(t) - 1.0 + s * np.sin(t) ** 2 / 2.0)
        assert np.abs(r - want).max() <= 0.03 * k * (1.0 + abs(want) / k) * max(np.sin(t), 0.05), (abc, r[:2], want)
    if theta_deg > 0:
        # the second-order rows absorb oblique waves better
        r1 = abs(np.cos(t) - 1.0)
        r2 = abs(np.cos(t) - 1.0 + np.sin(t) ** 2 / 2.0)
        assert r2 < r1


def test_abc2_hierarchy_converges_and_galerkin_keeps_symmetry():
    n, k = 32, 20.0
    h = 1.0 / n
    H = ohier.build_hierarchy(n, n, h, k, 0.7, abc=2)
    for A in H.A:
        assert abs(A - A.T).max() <= 1e-9 * abs(A).max()
    b = oprob.helmholtz_matrix(n, n, h, k, abc=2) @ np.ones((n + 1) ** 2)
    res = ocycle.mg_solve(H, b, 1e-8, ocycle.CycleOptions(1, "jacobi", 1, 1, 4.5), max_cycles=400)
    assert res.converged
    assert np.abs(res.x - 1.0).max() < 1e-6
