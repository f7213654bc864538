"""Python binding of the helmmg C-ABI (include/helmmg.h): stand-alone
multigrid for the 2D Helmholtz equation (Dwarka & Vuik, arXiv 2308.13476)
on one GB300 GPU.

This module only marshals arguments: every step of a solve runs in the
library's CUDA kernels.  Device arrays are torch CUDA tensors (complex128
grids of shape (B, ny+1, nx+1) or (ny+1, nx+1), float64 fields); the library
never keeps references to them.  If the compiled library is missing the
import of this package still succeeds, but every call raises
``HelmmgUnavailable``: there is no CPU fallback.

Low-level functions carry the C names (``mg_setup``, ``mg_solve``,
``mg_adjoint``, ``mg_gradient``, ``mg_destroy`` ...); ``Solver`` wraps them.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhelmmg.so")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_EMAXIT, MG_EDIVERGED, MG_ETIMEOUT, MG_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "MG_OK", -1: "MG_EINVAL", -2: "MG_ENOMEM", -3: "MG_ECUDA", -4: "MG_EMAXIT",
                -5: "MG_EDIVERGED", -6: "MG_ETIMEOUT", -7: "MG_ESTATE"}
EXPORTED = ["mg_default_options", "mg_setup", "mg_solve", "mg_adjoint", "mg_gradient", "mg_destroy",
            "mg_last_error", "mg_level_info", "mg_apply", "mg_get_stencil", "mg_history", "mg_profile",
            "mg_counters", "mg_residual_norm_static", "mg_setup_ragged", "mg_two_grid"]


class HelmmgUnavailable(RuntimeError):
    """The compiled CUDA library could not be loaded."""


class HelmmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class MgOptions(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int), ("smoother", ctypes.c_int), ("nu_pre", ctypes.c_int),
                ("nu_post", ctypes.c_int), ("omega", ctypes.c_double), ("precision", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("min_coarse", ctypes.c_int), ("batch", ctypes.c_int),
                ("coarse_nodes", ctypes.c_int), ("coarse_mode", ctypes.c_int), ("fuse", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("march", ctypes.c_int), ("krylov", ctypes.c_int),
                ("transfer", ctypes.c_int), ("flat", ctypes.c_int), ("kron_chunk", ctypes.c_int),
                ("abc", ctypes.c_int), ("stream", ctypes.c_void_p)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libhelmmg.so (built by ``paper_2308_13476_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HelmmgUnavailable(f"{path} is missing: run paper_2308_13476_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
    lib.mg_default_options.argtypes = [ctypes.POINTER(MgOptions)]
    lib.mg_default_options.restype = None
    lib.mg_setup.argtypes = [ctypes.POINTER(vp), i, i, d, vp, d, d, i, ctypes.POINTER(MgOptions)]
    lib.mg_solve.argtypes = [vp, vp, vp, d, ip, dp]
    lib.mg_adjoint.argtypes = [vp, vp, vp, d, ip, dp]
    lib.mg_gradient.argtypes = [vp, vp, vp, i, vp, d, vp]
    lib.mg_destroy.argtypes = [vp]
    lib.mg_last_error.argtypes = []
    lib.mg_last_error.restype = ctypes.c_char_p
    lib.mg_level_info.argtypes = [vp, i, ip, ip, ip, ip]
    lib.mg_apply.argtypes = [vp, i, vp, vp]
    lib.mg_get_stencil.argtypes = [vp, i, vp]
    lib.mg_history.argtypes = [vp, dp, i]
    lib.mg_profile.argtypes = [vp, i, i, i, dp, dp]
    lib.mg_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.mg_residual_norm_static.argtypes = [i, i, d, vp, d, vp, vp, vp, vp]
    lib.mg_setup_ragged.argtypes = [ctypes.POINTER(vp), i, ip, ip, dp, dp, dp, ctypes.POINTER(MgOptions)]
    lib.mg_two_grid.argtypes = [vp, i, i, dp]
    for name in EXPORTED:
        if name not in ("mg_default_options", "mg_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, allow=()):
    if status != MG_OK and status not in allow:
        raise HelmmgError(status, load_library().mg_last_error().decode())
    return status


def _ptr(t, dtype=None, name="array"):
    """Device pointer of a contiguous CUDA tensor (checked)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------- C-named calls


def mg_default_options():
    o = MgOptions()
    load_library().mg_default_options(ctypes.byref(o))
    return o


def mg_setup(nx, ny, h, k_field=None, k_const=0.0, beta2=0.0, levels=0, opt=None):
    """Returns an opaque handle (int).  ``k_field``: float64 tensor
    (ny+1, nx+1) on the host or the device, or None for constant k."""
    lib = load_library()
    opt = opt or mg_default_options()
    hdl = ctypes.c_void_p()
    kp = None
    if k_field is not None:
        import torch
        if k_field.dtype != torch.float64 or not k_field.is_contiguous():
            raise TypeError("k_field must be a contiguous float64 tensor")
        if tuple(k_field.shape) != (ny + 1, nx + 1):
            raise ValueError("k_field must have shape (ny+1, nx+1)")
        kp = ctypes.c_void_p(k_field.data_ptr())
    _check(lib.mg_setup(ctypes.byref(hdl), int(nx), int(ny), float(h), kp, float(k_const), float(beta2),
                        int(levels), ctypes.byref(opt)))
    return hdl.value


def _solve_call(fn, hdl, rhs, x, tol, batch):
    import torch
    cyc = (ctypes.c_int * batch)()
    rr = (ctypes.c_double * batch)()
    st = fn(ctypes.c_void_p(hdl), _ptr(rhs, torch.complex128, "rhs"), _ptr(x, torch.complex128, "x"), float(tol),
            cyc, rr)
    _check(st, allow=(MG_EMAXIT, MG_EDIVERGED))
    return st, list(cyc), list(rr)


def mg_solve(hdl, rhs, x, tol, batch=1):
    """In-place solve; returns (status, cycles per RHS, relres per RHS)."""
    return _solve_call(load_library().mg_solve, hdl, rhs, x, tol, batch)


def mg_adjoint(hdl, rhs_adj, lam, tol, batch=1):
    """In-place solve of A^H lam = rhs_adj; returns (status, cycles, relres)."""
    return _solve_call(load_library().mg_adjoint, hdl, rhs_adj, lam, tol, batch)


def mg_gradient(hdl, u, lam, m, omega_f, g):
    import torch
    nsrc = u.shape[0] if u.dim() == 3 else 1
    _check(load_library().mg_gradient(ctypes.c_void_p(hdl), _ptr(u, torch.complex128, "u"),
                                      _ptr(lam, torch.complex128, "lam"), int(nsrc), _ptr(m, torch.float64, "m"),
                                      float(omega_f), _ptr(g, torch.float64, "g")))


def mg_destroy(hdl):
    if hdl:
        load_library().mg_destroy(ctypes.c_void_p(hdl))


def mg_level_info(hdl, level):
    a, b, r, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().mg_level_info(ctypes.c_void_p(hdl), int(level), ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(r), ctypes.byref(n)))
    return a.value, b.value, r.value, n.value


def mg_apply(hdl, level, x, y):
    import torch
    _check(load_library().mg_apply(ctypes.c_void_p(hdl), int(level), _ptr(x, torch.complex128, "x"),
                                   _ptr(y, torch.complex128, "y")))


def mg_get_stencil(hdl, level, out):
    import torch
    _check(load_library().mg_get_stencil(ctypes.c_void_p(hdl), int(level), _ptr(out, torch.complex128, "out")))


def mg_history(hdl, batch, cap):
    buf = (ctypes.c_double * (batch * cap))()
    _check(load_library().mg_history(ctypes.c_void_p(hdl), buf, int(cap)))
    return [list(buf[b * cap:(b + 1) * cap]) for b in range(batch)]


def mg_two_grid(hdl, nu=1, max_iter=20000):
    """Dense two-grid analysis of the two finest levels: a dict with the
    spectral norm of T0, whether Gamma~ is HPD, ||Gamma~||_1 / kappa_1 and
    the power-method bookkeeping (see include/helmmg.h)."""
    out = (ctypes.c_double * 6)()
    _check(load_library().mg_two_grid(ctypes.c_void_p(hdl), int(nu), int(max_iter), out))
    return {"norm_t0": out[0], "hpd": out[1] == 1.0, "gamma_ratio": out[2], "iterations": int(out[3]),
            "converged": out[4] == 1.0, "coarse_singular": out[5] == 1.0}


def mg_profile(hdl, what, level, reps):
    """(ms per launch, algorithmic bytes per launch) of one kernel kind."""
    ms, nb = ctypes.c_double(), ctypes.c_double()
    _check(load_library().mg_profile(ctypes.c_void_p(hdl), int(what), int(level), int(reps), ctypes.byref(ms),
                                     ctypes.byref(nb)))
    return ms.value, nb.value


def mg_counters(hdl):
    k, g = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load_library().mg_counters(ctypes.c_void_p(hdl), ctypes.byref(k), ctypes.byref(g)))
    return k.value, g.value


def mg_residual_norm_static(nx, ny, h, k, x, b, out, stream=None):
    """out[0] = ||b - A x||, out[1] = ||b|| on the device, without any device
    allocation by the library (see include/helmmg.h).  ``k``: float or a
    float64 CUDA tensor (ny+1, nx+1); x, b: complex128 CUDA grids; out: a
    float64 CUDA tensor of 2 entries.  Every tensor must sit on the current
    CUDA device; the call is enqueued on ``stream`` (default: torch's current
    stream).  The C side cannot see tensor sizes, so they are checked here:
    an undersized tensor would otherwise become an out-of-bounds access."""
    import torch
    nodes = (int(nx) + 1) * (int(ny) + 1)
    dev = torch.cuda.current_device()
    named = [("x", x, nodes), ("b", b, nodes), ("out", out, 2)]
    if not isinstance(k, (int, float)):
        named.append(("k", k, nodes))
    for name, t, need in named:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA torch tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if (t.numel() != need) if name != "out" else (t.numel() < need):
            raise ValueError(f"{name} has {t.numel()} elements, needs {need}")
    kp, kc = (None, float(k)) if isinstance(k, (int, float)) else (_ptr(k, torch.float64, "k"), 0.0)
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    _check(load_library().mg_residual_norm_static(int(nx), int(ny), float(h), kp, kc, _ptr(x, torch.complex128, "x"),
                                                  _ptr(b, torch.complex128, "b"), _ptr(out, torch.float64, "out"),
                                                  ctypes.c_void_p(st)))


def mg_setup_ragged(nx, ny, h, k_const, beta2=0.0, opt=None):
    """Handle of a ragged batch (lists of per-problem sizes, cell sizes,
    wavenumbers and shifts; a scalar beta2 applies to every problem)."""
    lib = load_library()
    opt = opt or mg_default_options()
    n = len(nx)
    hdl = ctypes.c_void_p()
    ia = lambda v: (ctypes.c_int * n)(*[int(q) for q in v])
    da = lambda v: (ctypes.c_double * n)(*[float(q) for q in v])
    b2 = [float(beta2)] * n if isinstance(beta2, (int, float)) else list(beta2)
    _check(lib.mg_setup_ragged(ctypes.byref(hdl), n, ia(nx), ia(ny), da(h), da(k_const), da(b2),
                               ctypes.byref(opt)))
    return hdl.value


# ------------------------------------------------------------- convenience


SMOOTHERS = {"jacobi": 0, "gmres3": 1}
TRANSFERS = {"bezier": 0, "linear": 1}


def _options(cycle="V", smoother="jacobi", nu_pre=1, nu_post=1, omega=4.5, precision="fp64", batch=1,
             max_cycles=10000, min_coarse=10, coarse_nodes=None, coarse_mode=None, fuse=None, tile_rows=None,
             march=None, krylov=None, transfer="bezier", flat=None, kron_chunk=None, abc=None, stream=None):
    o = mg_default_options()
    o.cycle = {"V": 1, "W": 2, 1: 1, 2: 2}[cycle]
    o.smoother = SMOOTHERS[smoother]
    o.nu_pre, o.nu_post, o.omega = int(nu_pre), int(nu_post), float(omega)
    o.precision = PRECISIONS[precision]
    o.batch, o.max_cycles, o.min_coarse = int(batch), int(max_cycles), int(min_coarse)
    for name, val in (("coarse_nodes", coarse_nodes), ("coarse_mode", coarse_mode), ("fuse", fuse),
                      ("tile_rows", tile_rows), ("march", march), ("krylov", krylov), ("flat", flat),
                      ("kron_chunk", kron_chunk), ("abc", abc)):
        if val is not None:
            setattr(o, name, int(val))
    o.transfer = TRANSFERS[transfer]
    o.stream = ctypes.c_void_p(stream.cuda_stream if stream is not None else None)
    return o
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed-ff": 2}


class RaggedSolver:
    """Independent constant-k problems of different sizes solved together.

    RaggedSolver(sizes=[(nx, ny, h, k), ...], beta2, **options), beta2 a
    scalar or one shift per problem.  solve() takes and returns a list of
    complex128 CUDA grids (ny+1, nx+1).  ``flat=0`` (the default) solves
    problems with identical parameters as one batch of right-hand sides,
    each group with its own cycle graph; ``flat=1`` runs a cycle of all
    problems as one launch per kernel when the options allow it."""

    def __init__(self, sizes, beta2, **options):
        self.sizes = [(int(a), int(b), float(c), float(d)) for a, b, c, d in sizes]
        o = _options(**options)
        self.handle = mg_setup_ragged([s[0] for s in self.sizes], [s[1] for s in self.sizes],
                                      [s[2] for s in self.sizes], [s[3] for s in self.sizes], beta2, o)

    def solve(self, rhs_list, tol=1e-6):
        import torch
        flat = torch.cat([r.reshape(-1).to(torch.complex128) for r in rhs_list]).contiguous()
        x = torch.zeros_like(flat)
        n = len(self.sizes)
        st, cyc, rr = mg_solve(self.handle, flat, x, tol, n)
        out, o = [], 0
        for nx, ny, _, _ in self.sizes:
            m = (nx + 1) * (ny + 1)
            out.append(x[o:o + m].reshape(ny + 1, nx + 1))
            o += m
        return out, st, cyc, rr

    def close(self):
        if getattr(self, "handle", None):
            mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One multigrid hierarchy on the current CUDA device.

    Solver(nx, ny, h, k, beta2, cycle="V"|"W", smoother="jacobi"|"gmres3",
           nu_pre, nu_post, omega, precision="fp64"|"mixed"|"mixed-ff", batch, levels,
           max_cycles, min_coarse, coarse_nodes, coarse_mode, fuse, tile_rows, march, krylov,
           transfer="bezier"|"linear", kron_chunk, abc=1|2, stream)
    ``abc=2`` replaces the first-order absorbing rows of Sec. 2 by the
    second-order Engquist-Majda condition (a variant the paper does not use).
    ``k`` is a float (constant wavenumber) or a float64 tensor (ny+1, nx+1).
    ``krylov`` = m > 0 wraps the cycle in restarted FGMRES(m) as its right
    preconditioner (cycles then count preconditioner applications).
    ``transfer="linear"`` replaces the higher-order transfers of Eq. (xex) by
    linear interpolation (an ablation).
    """

    def __init__(self, nx, ny, h, k, beta2, cycle="V", smoother="jacobi", nu_pre=1, nu_post=1, omega=4.5,
                 precision="fp64", batch=1, levels=0, max_cycles=10000, min_coarse=10, coarse_nodes=None,
                 coarse_mode=None, fuse=None, tile_rows=None, march=None, krylov=0, transfer="bezier",
                 kron_chunk=None, abc=1, stream=None):
        o = mg_default_options()
        o.cycle = {"V": 1, "W": 2, 1: 1, 2: 2}[cycle]
        o.smoother = SMOOTHERS[smoother]
        o.nu_pre, o.nu_post, o.omega = int(nu_pre), int(nu_post), float(omega)
        o.precision = PRECISIONS[precision]
        o.batch, o.max_cycles, o.min_coarse = int(batch), int(max_cycles), int(min_coarse)
        if coarse_nodes is not None:
            o.coarse_nodes = int(coarse_nodes)
        if coarse_mode is not None:
            o.coarse_mode = int(coarse_mode)
        if fuse is not None:
            o.fuse = int(fuse)
        if tile_rows is not None:
            o.tile_rows = int(tile_rows)
        if march is not None:
            o.march = int(march)
        o.krylov = int(krylov)
        if kron_chunk is not None:
            o.kron_chunk = int(kron_chunk)
        o.abc = int(abc)
        o.transfer = TRANSFERS[transfer]
        o.stream = ctypes.c_void_p(stream.cuda_stream if stream is not None else None)
        self.nx, self.ny, self.h, self.batch = nx, ny, h, batch
        if isinstance(k, (int, float)):
            self.handle = mg_setup(nx, ny, h, None, float(k), beta2, levels, o)
        else:
            self.handle = mg_setup(nx, ny, h, k, 0.0, beta2, levels, o)
        self.nlevels = mg_level_info(self.handle, 0)[3]

    def _grid(self, t):
        import torch
        t = t.reshape(self.batch, self.ny + 1, self.nx + 1)
        return t.to(torch.complex128).contiguous()

    def solve(self, rhs, x=None, tol=1e-6):
        """Returns (x, status, cycles, relres); x is a new tensor unless given."""
        import torch
        rhs = self._grid(rhs)
        if x is None:
            x = torch.zeros_like(rhs)
        st, cyc, rr = mg_solve(self.handle, rhs, x, tol, self.batch)
        return x, st, cyc, rr

    def adjoint(self, rhs_adj, lam=None, tol=1e-6):
        import torch
        rhs_adj = self._grid(rhs_adj)
        if lam is None:
            lam = torch.zeros_like(rhs_adj)
        st, cyc, rr = mg_adjoint(self.handle, rhs_adj, lam, tol, self.batch)
        return lam, st, cyc, rr

    def gradient(self, u, lam, m, omega_f):
        import torch
        g = torch.empty((self.ny + 1, self.nx + 1), dtype=torch.float64, device=u.device)
        mg_gradient(self.handle, u.contiguous(), lam.contiguous(), m.contiguous(), omega_f, g)
        return g

    def level_info(self, level):
        return mg_level_info(self.handle, level)

    def apply(self, level, x):
        import torch
        y = torch.empty_like(x)
        mg_apply(self.handle, level, x.contiguous(), y)
        return y

    def stencil(self, level):
        import torch
        nx, ny, r, _ = mg_level_info(self.handle, level)
        out = torch.empty((ny + 1, nx + 1, 2 * r + 1, 2 * r + 1), dtype=torch.complex128, device="cuda")
        mg_get_stencil(self.handle, level, out)
        return out

    def history(self, cap):
        return mg_history(self.handle, self.batch, cap)

    def two_grid(self, nu=1, max_iter=20000):
        return mg_two_grid(self.handle, nu, max_iter)

    def profile(self, what, level=0, reps=20):
        return mg_profile(self.handle, what, level, reps)

    def counters(self):
        return mg_counters(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
