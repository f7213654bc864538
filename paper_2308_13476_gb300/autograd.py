"""Receiver-misfit gradient with respect to squared slowness as a
torch.autograd.Function over the helmmg C-ABI.

Forward: k(x)^2 = omega_f^2 m(x) defines the MP 2-B operator A(m) of the
paper (Sec. 2); the library solves A(m) u_s = f_s for all sources in one
batched multigrid solve and the misfit is L = 1/2 sum_s ||S u_s - d_s||^2
(S samples the receiver nodes).  Backward: one batched adjoint solve
A^H lam_s = S^T (S u_s - d_s) (mg_adjoint) and the gradient kernel
(mg_gradient) give dL/dm = -Re sum_s conj(lam_s) dA_pp/dm_p u_s.

Only argument marshalling happens here (k = omega_f sqrt(m) for mg_setup,
sampling and scattering the receiver values); every solve and the gradient
run in the library's kernels.
"""
import torch

from . import Solver, MG_OK, HelmmgError


class HelmholtzMisfit(torch.autograd.Function):
    """L = HelmholtzMisfit.apply(m, sources, receivers, data, grid, solver_kw)

    m          float64 CUDA tensor (ny+1, nx+1): squared slowness (> 0)
    sources    complex128 CUDA tensor (nsrc, ny+1, nx+1): right-hand sides f_s
    receivers  int64 CUDA tensor (nrec,): flat node indices j*(nx+1)+i
    data       complex128 CUDA tensor (nsrc, nrec): observed d_s
    grid       (nx, ny, h, omega_f)
    solver_kw  dict of Solver options (tol, beta2, smoother, ...); beta2
               defaults to 1/(k_max L), L = max(nx, ny) h, the paper's
               beta2 = 1/k on the unit square
    Returns the misfit as a 0-d float64 tensor; its gradient flows to m.
    """

    @staticmethod
    def forward(ctx, m, sources, receivers, data, grid, solver_kw):
        nx, ny, h, omega_f = grid
        kw = dict(solver_kw)
        tol = kw.pop("tol", 1e-8)
        nsrc = sources.shape[0]
        k = (omega_f * torch.sqrt(m)).contiguous()
        # the paper's shift beta2 = 1/k refers to the unit square; on a domain
        # of length L the same dimensionless shift is 1/(k_max L)
        beta2 = kw.pop("beta2", 1.0 / (float(k.max()) * max(nx, ny) * h))
        s = Solver(nx, ny, h, k, beta2, batch=nsrc, **kw)
        u, st, cyc, rr = s.solve(sources, tol=tol)
        if st != MG_OK:
            s.close()
            raise HelmmgError(st, f"forward solve did not converge (cycles {cyc}, relres {rr})")
        res = u.reshape(nsrc, -1)[:, receivers] - data
        ctx.solver = s
        ctx.tol = tol
        ctx.omega_f = omega_f
        ctx.save_for_backward(m, u, res, receivers)
        return 0.5 * (res.real.square().sum() + res.imag.square().sum())

    @staticmethod
    def backward(ctx, gL):
        m, u, res, receivers = ctx.saved_tensors
        s = ctx.solver
        nsrc = u.shape[0]
        rhs = torch.zeros_like(u).reshape(nsrc, -1)
        rhs[:, receivers] = res
        lam, st, cyc, rr = s.adjoint(rhs.reshape(u.shape), tol=ctx.tol)
        if st != MG_OK:
            raise HelmmgError(st, f"adjoint solve did not converge (cycles {cyc}, relres {rr})")
        g = s.gradient(u, lam, m, ctx.omega_f)
        s.close()
        ctx.solver = None
        return gL * g, None, None, None, None, None


def misfit(m, sources, receivers, data, grid, **solver_kw):
    """Convenience wrapper: HelmholtzMisfit.apply with keyword solver options."""
    return HelmholtzMisfit.apply(m, sources, receivers, data, grid, solver_kw)
