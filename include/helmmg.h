/* helmmg -- stand-alone multigrid for the 2D Helmholtz equation on one GPU.
 *
 * Method: Dwarka & Vuik, "Stand-alone multigrid for Helmholtz revisited:
 * towards convergence using standard components" (arXiv 2308.13476).
 *
 *   Problem (Sec. 2, MP 2-A / MP 2-B): -Lap u - k(x,y)^2 u = f on a grid of
 *   nx by ny square cells of side h, with the first-order absorbing condition
 *   (d/dn - i k) u = 0 on the whole boundary, 5-point second-order finite
 *   differences.  Every grid node, boundary nodes included, is an unknown.
 *   Boundary rows come from eliminating a ghost node with the central
 *   difference of the boundary condition and are scaled by 1/2 on an edge and
 *   1/4 at a corner; the matrix A is complex symmetric (A^T = A).  The
 *   right-hand side uses the same row scaling (a point source on an interior
 *   node is unaffected).
 *
 *   Method (Sec. 3-5): multigrid V-cycle (gamma = 1) or W-cycle (gamma = 2)
 *   used as a stand-alone solver; weighted-Jacobi smoothing with
 *   X = omega * diag(A) (omega = 4.5 in the paper) or GMRES(3) smoothing;
 *   the rational-Bezier prolongation of Eq. (xex) and its transpose as
 *   restriction; Galerkin coarse operators built on the complex-shifted
 *   Laplacian -Lap - (1 + i beta2) k^2 (the shift enters once, on the fine
 *   level); coarsening while both interval counts are even and the grid
 *   still has at least 10 nodes, with a direct solve on the last grid; stop
 *   at a relative residual ||b - A x||_2 / ||b||_2 <= tol.
 *
 * Data layout.  A grid vector is (ny+1) x (nx+1) complex128 values (real,
 * imaginary interleaved), row-major with x fastest: node (i, j) at
 * j*(nx+1) + i.  A batch of B right-hand sides is B such grids back to back.
 * Real grid fields (k, m, gradients) are (ny+1) x (nx+1) doubles.
 *
 * Pointers.  Arrays passed to mg_solve, mg_adjoint, mg_apply,
 * mg_get_stencil and mg_gradient are DEVICE pointers on the current device,
 * owned by the caller; the library never frees or keeps them.  The k field of
 * mg_setup may be host or device memory; it is copied.  cycles_out and
 * relres_out are HOST arrays of B entries.
 *
 * Streams.  All work is ordered on options.stream (a cudaStream_t, NULL =
 * legacy default stream).  mg_solve returns after the stopping decision, with
 * the stream synchronised.
 *
 * Errors.  Every call returns an mg_status.  On failure mg_last_error()
 * describes the cause; arrays the caller owns are left as they were at the
 * failing step (x holds the last iterate).  The library never aborts the
 * process and never traps on the device.
 *
 * Threads.  One handle per host thread; handles are independent.
 */
#ifndef HELMMG_H
#define HELMMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx* mg_handle;

typedef enum {
  MG_OK = 0,
  MG_EINVAL = -1,     /* bad argument, shape or option                          */
  MG_ENOMEM = -2,     /* device allocation failed                               */
  MG_ECUDA = -3,      /* CUDA runtime error                                     */
  MG_EMAXIT = -4,     /* max_cycles reached before tol (x = last iterate)       */
  MG_EDIVERGED = -5,  /* relative residual above 1e6 or not finite             */
  MG_ETIMEOUT = -6,   /* a bounded device wait (grid-wide barrier) gave up      */
  MG_ESTATE = -7      /* call not valid in the handle's state (e.g. singular
                         coarsest operator)                                      */
} mg_status;

typedef struct {
  int cycle;        /* gamma: 1 = V-cycle, 2 = W-cycle (Table cons1)            */
  int smoother;     /* 0 = weighted Jacobi (Sec. 3), 1 = GMRES(3) (Sec. 5.3)     */
  int nu_pre;       /* smoothing steps before the coarse correction, per level  */
  int nu_post;      /* smoothing steps after it, per level                      */
  double omega;     /* Jacobi: X = omega * diag(A); the paper uses 4.5          */
  int precision;    /* 0 = complex128 throughout; 1 = complex64 cycles inside a
                       complex128 iterative-refinement loop (outer residual,
                       update, setup and coarsest solve in FP64); 2 = the same
                       with the outer x, b, residual and update held as
                       float-float pairs (48-bit significand, FP32 pipes)      */
  int max_cycles;   /* cap on cycles (refinement steps for precision 1, 2)    */
  int min_coarse;   /* stop coarsening below this many grid nodes (Sec. 5: 10) */
  int batch;        /* B: right-hand sides solved together                      */
  int coarse_nodes; /* levels with at most this many grid nodes (and all below
                       them) run inside one launch per visit; 0 = never       */
  int coarse_mode;  /* that launch: 0 = one CTA per right-hand side,
                       1 = a cooperative grid of all co-resident CTAs with
                       bounded grid-wide barriers (MG_ETIMEOUT if one gives up) */
  int fuse;         /* 1 = fused halo-tile kernels: residual + restriction in
                       one pass, fine-level Jacobi sweeps up to 4 per pass;
                       0 = one kernel per step (same results)                  */
  int tile_rows;    /* grid rows per thread of the node kernels: 0 = chosen
                       from each level's size, 1..4 = forced (autotuner knob) */
  int march;        /* GMRES(3) on the fine level as row marches and on
                       Kronecker-form levels with column-march operator
                       kernels, which then also form the residual before the
                       restriction (needs fuse = 1): 1 = always, 0 = never (the
                       node-parallel kernels; same results to rounding),
                       -1 = the Kronecker-form levels always, the fine level
                       when it holds at least 4 M nodes over all right-hand
                       sides and the other problems of a ragged batch (a row
                       march keeps each warp on one strip, which needs that
                       much work to fill the GPU)                           */
  int krylov;       /* 0 = the stand-alone cycle iteration (the paper's method);
                       m in 1..32 = restarted flexible GMRES(m) on the fine
                       operator with one cycle (from zero) as the right
                       preconditioner, the Krylov use recalled in Sec. 1
                       (precision 0 or 1).  The restart residual, x, the
                       update and all scalars are FP64; the basis, the
                       preconditioned vectors and the Arnoldi passes take the
                       cycle's precision (precision 1: each restart cycle is
                       an FP32 FGMRES correction of the FP64 residual).  max_cycles then caps preconditioner
                       applications, the cycle counts report them, mg_history
                       holds the residual estimate after each one, and the
                       stopping test is the true relative residual at a
                       restart.  Memory: 2m+1 fine grids in the cycle's
                       precision and 2 FP64 ones per right-hand side.      */
  int transfer;     /* inter-grid transfers, both directions (R = P^T / 4) and
                       the Galerkin coarsening: 0 = the higher-order Eq. (xex)
                       (paper default); 1 = linear interpolation, the
                       "Linear" column of Table conv1 (an ablation: the paper
                       finds the two-grid map no longer contracting)      */
  int flat;         /* ragged batches: 0 = problems with the same grid, cell
                       size, wavenumber and shift share one hierarchy and are
                       solved as the right-hand sides of one batched handle,
                       each handle with its own cycle graph and stream;
                       1 = every problem has its own hierarchy and every
                       kernel of a cycle is one launch over all problems
                       (their blocks numbered one after the other, each
                       problem with its own grid, geometry and convergence
                       mask) when the options allow it (GMRES(3), fuse 1,
                       march != 0, precision 0 or 1, krylov 0, abc 1, coarse_mode 0
                       and a coarse_nodes that puts every problem's coarsest
                       grid in the coarse-cycle launch), else one cycle graph
                       per problem.  Either way each problem computes its own
                       solve.  Ignored by single-problem handles.         */
  int kron_chunk;   /* rows per chunk of the column marches on Kronecker-form
                       levels: 0 = chosen per level from the kernels'
                       occupancy (rounds x rows); n > 0 = n rows (at least 8;
                       an autotuner axis).  Any value gives the same results
                       up to the order of the reductions' block partials.  */
  int abc;          /* absorbing boundary rows: 1 = the first-order Sommerfeld
                       condition of Sec. 2 (paper default); 2 = the
                       second-order condition of Engquist and Majda,
                       du/dn - i k u - (i/2k) d2u/dtau2 = 0, as a boundary
                       stiffness with natural corners (a variant the paper
                       does not use; coarse levels then take stored
                       Galerkin stencils; needs precision 0 or 1;
                       mg_gradient returns MG_EINVAL)                       */
  void* stream;     /* cudaStream_t                                             */
} mg_options;

/* Paper defaults: V(1,1), Jacobi, omega 4.5, complex128, 10000 cycles,
 * min_coarse 10, batch 1; coarse_nodes 1100, coarse_mode 0, fuse 1,
 * tile_rows 0; march -1; krylov 0; transfer 0; flat 0; kron_chunk 0; abc 1; default stream. */
void mg_default_options(mg_options* opt);

/* Build the hierarchy for one problem (Sec. 2, Sec. 3, Sec. 5).
 *   nx, ny    interval counts (>= 2); grids are coarsened while both are even
 *   h         cell size (> 0)
 *   k_field   NULL for constant k = k_const (MP 2-A), else (ny+1)*(nx+1)
 *             positive wavenumbers (MP 2-B), host or device memory, copied
 *   beta2     complex shift of the CSL used for Galerkin coarsening (>= 0;
 *             0 coarsens the Helmholtz operator itself)
 *   levels    0 = as many as the coarsening rule allows; n > 0 caps the count
 *   opt       NULL = mg_default_options
 * The coarsest grid must have at most 2048 nodes.  On success *out owns all
 * device memory of the hierarchy; release it with mg_destroy. */
mg_status mg_setup(mg_handle* out, int nx, int ny, double h, const double* k_field, double k_const, double beta2,
                   int levels, const mg_options* opt);

/* Ragged batch: nprob independent constant-k problems of different sizes in
 * one handle (problem p: nx[p] x ny[p] cells of side h[p], wavenumber
 * k_const[p], complex shift beta2[p]; host arrays of nprob entries, copied;
 * the same options and one right-hand side each, so opt->batch must be 1).  mg_solve / mg_adjoint on this handle take rhs and x
 * as the problems' grids packed back to back (problem p starts after
 * sum_{q<p} (nx[q]+1)(ny[q]+1) complex128 values) and report cycles and
 * relative residuals per problem.  With opt->flat = 0 (the default)
 * problems with identical parameters share a hierarchy and are solved as
 * one batch of right-hand sides (staged side by side in a device buffer the
 * handle owns); every such group has its own cycle graph and stream
 * (prioritised by problem size) and starts its next cycle as soon as its
 * last one has been tested.  With opt->flat = 1 (and options that allow it)
 * every problem has its own hierarchy and a cycle of all problems is one
 * CUDA graph whose every kernel is a single launch over all problems (a
 * problem that has converged leaves its blocks idle).  Inspection
 * calls return MG_ESTATE on a ragged handle. */
mg_status mg_setup_ragged(mg_handle* out, int nprob, const int* nx, const int* ny, const double* h,
                          const double* k_const, const double* beta2, const mg_options* opt);

/* Solve A x = rhs for the handle's batch, starting from the x passed in.
 *   rhs        device, B grids complex128 (read only)
 *   x          device, B grids complex128: initial guess in, iterate out
 *   tol        relative residual target (> 0)
 *   cycles_out host int[B] or NULL: cycles done per right-hand side
 *   relres_out host double[B] or NULL: final relative residual per RHS
 * Each right-hand side stops on its own: once it meets tol it is no longer
 * updated.  Returns MG_OK when all met tol, MG_EDIVERGED if any diverged
 * (checked first), MG_EMAXIT if any hit max_cycles.  An all-zero rhs gives
 * x = 0 and 0 cycles. */
mg_status mg_solve(mg_handle h, const void* rhs, void* x, double tol, int* cycles_out, double* relres_out);

/* Solve the adjoint system A^H lam = rhs_adj with the same hierarchy.  Since
 * A^T = A, A^H lam = g is conj(A) lam = g, i.e. A conj(lam) = conj(g): the
 * right-hand side is conjugated on the way in and the solution on the way
 * out.  Arguments and results as for mg_solve (lam in: initial guess). */
mg_status mg_adjoint(mg_handle h, const void* rhs_adj, void* lam, double tol, int* cycles_out, double* relres_out);

/* Gradient of L(m) = 1/2 sum_s ||S u_s - d_s||^2 with respect to the squared
 * slowness m, k^2 = omega_f^2 m, given forward fields u_s (A u_s = f_s) and
 * adjoint fields lam_s (A^H lam_s = S^T (S u_s - d_s)):
 *   g = -Re sum_s conj(lam_s) * dA_pp/dm_p * u_s,
 *   dA_pp/dm_p = -w_p omega_f^2 - i b_p omega_f / (2 h sqrt(m_p)),
 * w_p the boundary row weight (1, 1/2, 1/4), b_p = 1 on the boundary.
 *   u, lam   device, nsrc grids complex128 of the handle's (nx, ny)
 *   m        device, (ny+1)*(nx+1) doubles (> 0)
 *   g        device, (ny+1)*(nx+1) doubles, overwritten */
mg_status mg_gradient(mg_handle h, const void* u, const void* lam, int nsrc, const double* m, double omega_f,
                      double* g);

/* Release every resource of the handle.  NULL is accepted. */
mg_status mg_destroy(mg_handle h);

/* Message for the last failing call on this host thread; never NULL. */
const char* mg_last_error(void);

/* ---- inspection entry points (same layouts; for tests and tools) ---- */

/* Level geometry: interval counts and stencil radius (1 on level 0, then 2,
 * then 3) of level `level`; the number of levels via *nlevels. */
mg_status mg_level_info(mg_handle h, int level, int* nx, int* ny, int* radius, int* nlevels);

/* y = A_level x for B grids of that level (level 0: the Helmholtz operator;
 * level >= 1: the Galerkin operator, FP64).  x, y device complex128. */
mg_status mg_apply(mg_handle h, int level, const void* x, void* y);

/* Per-node stencil of A_level: device complex128 array
 * [ny+1][nx+1][2r+1][2r+1] with entry [j][i][dy+r][dx+r] the coupling of
 * node (i, j) to node (i+dx, j+dy) (0 off the grid). */
mg_status mg_get_stencil(mg_handle h, int level, void* out);

/* Relative residual history of the last solve: hist[b * cap + c] is the
 * relative residual of RHS b after cycle c+1 (c < min(cycles, cap)); with
 * krylov > 0, the FGMRES residual estimate after preconditioner
 * application c+1.  hist: host double[B * cap]. */
mg_status mg_history(mg_handle h, double* hist, int cap);

/* ---- analysis ---- */

/* Dense two-grid analysis of the handle's two finest levels (Sec. 3), for
 * small grids (at most 4096 fine nodes):
 *   T0 = (I - P A_1^{-1} R A)(I - X^{-1} A)^nu  (Eq. (tgi1), X = omega diag(A):
 *        nu weighted-Jacobi sweeps, then the coarse-grid correction),
 *   Gamma~ = A^H D~^H + D~ A - A^H D~^H D~ A, D~ = X^{-1} + P A_1^{-1} R
 *        (Definition def2s),
 * with A the fine operator, A_1 the handle's level-1 Galerkin operator (built
 * on the CSL with the handle's beta2; beta2 = 0 builds it on A), P and
 * R = P^T / 4 the handle's transfers (option transfer) and omega the handle's.
 * out (host, 6 doubles): [0] ||T0||_2 (Table conv1; power method on
 * T0^H T0, stopped when the Rayleigh quotient moves by at most 1e-14 of
 * itself over 100 iterations, or after max_iter), [1] 1.0 if Gamma~ is
 * Hermitian (to 1e-10 of its largest entry) and its Cholesky factorisation
 * succeeds, else 0.0 (the HPD test of Sec. 3), [2] ||Gamma~||_1 /
 * kappa_1(Gamma~) (Cor. mgc2, Table opt1; NaN if Gamma~ is singular), [3]
 * power iterations run, [4] 1.0 if the power method met its stopping test,
 * [5] 1.0 if A_1 was singular.  1 <= nu <= 8, 200 <= max_iter <= 1e6.
 * Device scratch (about 5 N^2 complex128 for N fine nodes) is allocated and
 * freed inside the call; MG_ENOMEM if it does not fit.  MG_EINVAL for grids
 * above 4096 nodes or a one-level hierarchy; MG_ESTATE on a ragged handle. */
mg_status mg_two_grid(mg_handle h, int nu, int max_iter, double* out);

/* ---- instrumentation ---- */

/* Time one kernel of the hierarchy in the handle's precision: `what` = 0 one
 * weighted-Jacobi sweep, 1 a residual b - A x, 2 a restriction, 3 a
 * prolongation-and-correct, 4 one GMRES(3) smoothing step (Sec. 5.3; the
 * kernels the cycle runs for that level: on level 0, when it runs as row
 * marches (option march), four row-march passes and the update, 16 vector
 * reads and writes per node (complex64: three passes and the update, 13, the
 * last Arnoldi vector's norm coming from the Gram form); on a Kronecker-form
 * level with column marches in complex64, five passes with two of them
 * fused, 19; otherwise eight passes, 28 (complex64: seven, 23); needs
 * smoother = 1), 5 the last Arnoldi step of an FGMRES(m) restart cycle
 * (j = m - 1: the pass for the m MGS coefficients and the pass for the new
 * basis vector, which also writes the cycle's right-hand side and zeroes its
 * iterate: 2m + 6 vector reads and writes per node in the cycle's precision; needs krylov > 0 and level 0; it marks every right-hand side
 * active), on level
 * `level` for all B right-hand sides.  The work runs `reps` times back to
 * back between two CUDA events on the handle's stream (after one untimed
 * run); *ms gets the mean time of one run and *bytes its algorithmic DRAM
 * bytes (each input array read once, each output written once).  `what` = 6
 * is a throughput probe of the FP64 FMA pipe, not a step of the method (the
 * denominator of the FP64 path's roofline): eight independent FMA chains of
 * 4096 steps per thread, 2048 threads per SM on every SM; *bytes then gets
 * the FP64 flops of one run instead of bytes, and `level` is ignored.  It
 * overwrites the handle's internal work vectors, never caller memory. */
mg_status mg_profile(mg_handle h, int what, int level, int reps, double* ms, double* bytes);

/* Kernel launches issued by the last mg_solve / mg_adjoint (graph kernel
 * nodes counted once per graph launch) and the number of graph launches. */
mg_status mg_counters(mg_handle h, long long* kernel_launches, long long* graph_launches);

/* ---- allocation-free call ---- */

/* ||b - A x||_2 and ||b||_2 for the fine-level Helmholtz operator of
 * mg_setup (same discretisation) on an nx by ny grid of cell size h, without
 * any handle and without allocating device memory.  The paper has no
 * counterpart; this is a service for callers that cannot allocate when they
 * need a residual: code running while another framework's memory pool owns
 * the device, latency-critical loops that cannot absorb the device-wide
 * synchronisation of an allocation, or contexts where allocation is not
 * permitted at all.
 *   k_field  NULL for constant k = k_const, else a DEVICE array of
 *            (ny+1)*(nx+1) wavenumbers
 *   x, b     DEVICE, (ny+1)*(nx+1) complex128, dense rows (read only)
 *   out      DEVICE double[2]: out[0] = ||b - A x||, out[1] = ||b||
 *   stream   cudaStream_t (NULL = legacy default stream); the call only
 *            enqueues work, the results are ready when the stream reaches them
 * Scratch: one file-scope device array of 256 KiB + 256 B per device
 * (partial sums of at most 16384 thread blocks of 32 x 32 nodes), held until
 * the process exits.  Grids needing more blocks (about 16.7 M nodes) are
 * rejected with MG_EINVAL.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and should come before any stream
 * capture.  All calls share the array: calls whose kernels overlap on the GPU
 * race and must be serialised by the caller. */
mg_status mg_residual_norm_static(int nx, int ny, double h, const double* k_field, double k_const, const void* x,
                                  const void* b, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HELMMG_H */
