"""mg_residual_norm_static: the residual norm without any device allocation.

Some callers cannot allocate device memory when they need a residual: code
that runs while another framework's memory pool owns the device, loops that
cannot absorb the device-wide synchronisation an allocation brings, or
contexts where allocation is not allowed.  This call serves them from a
file-scope device array.  Here it is checked, through the C-ABI, on two calls
in a row: against ||b - A x|| and ||b|| formed with the oracle's explicitly
assembled sparse matrix (its ghost-eliminated, row-scaled Sommerfeld rows at
edges and corners included), and against the relative residual that the
handle-based mg_solve reports for the same initial guess when it is given an
unreachable tolerance (0 cycles).  The file is named so that pytest collects
it last.
"""
import numpy as np
import pytest

import synth
from oracle import problem as oprob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runner deselects -m gpu anyway
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2308_13476_gb300 as hm  # noqa: E402


def _dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


@pytest.mark.parametrize("nx,ny,kvar", [(64, 64, False), (40, 24, True)])
def test_static_residual_norm_matches_oracle_and_solver(nx, ny, kvar):
    h = 1.0 / 64
    k = synth.k_field(synth.chi_smooth(nx, ny, 3), 8.0, 20.0) if kvar else 20.0
    kk = _dev(k, torch.float64) if kvar else k
    A = oprob.helmholtz_matrix(nx, ny, h, k)
    s = hm.Solver(nx, ny, h, kk, 0.7)
    for call in range(2):                       # two calls in a row share the scratch
        b = synth.point_source(nx, ny, h) + 1e-3 * synth.random_complex((ny + 1, nx + 1), 10 + call)
        x0 = 1e-2 * synth.random_complex((ny + 1, nx + 1), 20 + call)
        bd, xd = _dev(b), _dev(x0)
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        hm.mg_residual_norm_static(nx, ny, h, kk, xd, bd, out)
        torch.cuda.synchronize()
        rnorm, bnorm = out.cpu().numpy()
        # the oracle's assembled operator on the same x and b
        r_ref = np.linalg.norm(b.ravel() - A @ x0.ravel())
        b_ref = np.linalg.norm(b)
        assert abs(bnorm - b_ref) <= 1e-13 * b_ref
        assert abs(rnorm - r_ref) <= 1e-12 * r_ref
        # the existing entry point: 0 cycles, relres of the initial guess
        xs = xd.clone()[None].contiguous()
        _, st, cyc, rr = s.solve(bd, x=xs, tol=1e300)
        assert st == hm.MG_OK and cyc[0] == 0
        assert abs(rnorm / bnorm - rr[0]) <= 1e-12 * rr[0]
    s.close()


def test_static_residual_norm_boundary_rows_against_oracle():
    """x supported on the boundary ring only, so the whole residual comes
    from the ghost-eliminated edge and corner rows."""
    nx, ny, h, k = 24, 16, 1.0 / 24, 11.0
    x0 = synth.random_complex((ny + 1, nx + 1), 31)
    x0[1:-1, 1:-1] = 0.0
    b = np.zeros_like(x0)
    A = oprob.helmholtz_matrix(nx, ny, h, k)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        hm.mg_residual_norm_static(nx, ny, h, k, _dev(x0), _dev(b), out)
        torch.cuda.synchronize()
        rnorm, bnorm = out.cpu().numpy()
        r_ref = np.linalg.norm(A @ x0.ravel())
        assert bnorm == 0.0
        assert abs(rnorm - r_ref) <= 1e-12 * r_ref


def test_static_residual_norm_rejects_oversized_grid():
    # 8193^2 nodes (1.07 GB per grid) is beyond the scratch's 16384 blocks
    x = torch.zeros(8193 * 8193, dtype=torch.complex128, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(hm.HelmmgError, match="too large for the static scratch"):
        hm.mg_residual_norm_static(8192, 8192, 1.0, 1.0, x, x, out)
    # an undersized grid is refused by the binding before any device access
    with pytest.raises(ValueError, match="needs"):
        hm.mg_residual_norm_static(8, 8, 1.0, 1.0, x[:4], x[:4], out)
