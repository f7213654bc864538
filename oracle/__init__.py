"""Plain CPU oracle for the stand-alone multigrid Helmholtz solver of
Dwarka & Vuik, "Stand-alone multigrid for Helmholtz revisited" (arXiv 2308.13476).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

Everything here is FP64 complex (complex128), assembles explicit sparse
matrices with scipy, and follows the paper's definitions step by step:

* ``problem``   -- MP 2-A / MP 2-B operator (Sec. 2), CSL operator (Sec. 4).
* ``transfer``  -- higher-order (rational Bezier) prolongation, Eq. (xex),
                   and its transpose as restriction (Sec. 1, Sec. 3).
* ``hierarchy`` -- Galerkin coarse operators built on the CSL, coarsening
                   until the system has fewer than 10 unknowns (Sec. 5).
* ``smoothers`` -- weighted Jacobi S = I - X^{-1} A, X = omega*diag(A)
                   (Sec. 3) and the GMRES(3) polynomial smoother (Sec. 5.3).
* ``cycle``     -- V (gamma=1) / W (gamma=2) recursion and the outer loop to a
                   relative residual tolerance (Sec. 3, Sec. 5).
* ``analysis``  -- dense two-grid operator T0 (Eq. tgi1), Gamma-tilde
                   (Definition def2s) for the Table conv1 / opt1 checks.
* ``gradient``  -- adjoint-state gradient of a receiver misfit with respect
                   to squared slowness, by direct sparse solves.
* ``krylov``    -- the cycle as the right preconditioner of a restarted
                   flexible GMRES (the Krylov use recalled in Sec. 1).

Readings of passages the paper leaves open are documented at each function
(shift sign, boundary rows, edge rule of Eq. (xex), pre/post smoothing split).
"""
from . import problem, transfer, hierarchy, smoothers, cycle, analysis, gradient, krylov  # noqa: F401
