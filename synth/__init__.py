"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds no arithmetic of the multigrid method: it only draws and
lays out input data (sources, wavenumber fields, velocity models, random
vectors).  Every generator takes an explicit seed.

Layout of every grid array: (ny+1, nx+1), row-major, x fastest, node (i, j)
at [j, i].
"""
import numpy as np


def point_source(nx, ny, h, i=None, j=None, dtype=np.complex128):
    """Discrete unit point source: 1/h^2 at the interior node (i, j)
    (default: the centre node), zero elsewhere; shape (ny+1, nx+1)."""
    i = nx // 2 if i is None else i
    j = ny // 2 if j is None else j
    if not (0 < i < nx and 0 < j < ny):
        raise ValueError("point sources are placed on interior nodes")
    b = np.zeros((ny + 1, nx + 1), dtype=dtype)
    b[j, i] = 1.0 / (h * h)
    return b


def source_row(nx, ny, h, nsrc, j=None, dtype=np.complex128):
    """``nsrc`` point sources evenly spaced along row j (default: the first
    interior row below the top boundary), x_s = (s + 1/2) / nsrc of the width,
    nearest node.  Returns an array (nsrc, ny+1, nx+1)."""
    j = ny - 1 if j is None else j
    out = np.zeros((nsrc, ny + 1, nx + 1), dtype=dtype)
    for s in range(nsrc):
        i = int(round((s + 0.5) / nsrc * nx))
        out[s, j, i] = 1.0 / (h * h)
    return out


def random_complex(shape, seed, dtype=np.complex128):
    """Standard complex normal entries."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return z.astype(dtype)


def chi_smooth(nx, ny, seed, nbumps=6, sigma=0.15):
    """Smooth random profile in [0, 1]: a sum of ``nbumps`` Gaussian bumps of
    width ``sigma`` at random centres with random signs, min-max normalised."""
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.linspace(0, 1, ny + 1), np.linspace(0, 1, nx + 1), indexing="ij")
    f = np.zeros_like(x)
    for _ in range(nbumps):
        cx, cy = rng.uniform(0, 1, 2)
        f += rng.choice([-1.0, 1.0]) * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * sigma**2))
    return (f - f.min()) / (f.max() - f.min())


def chi_sharp(nx, ny, seed, blocks=16):
    """Sharp random profile in [0, 1]: i.i.d. uniform values, constant on a
    ``blocks`` x ``blocks`` partition of the domain."""
    rng = np.random.default_rng(seed)
    vals = rng.uniform(0, 1, (blocks, blocks))
    bi = np.minimum((np.arange(nx + 1) * blocks) // (nx + 1), blocks - 1)
    bj = np.minimum((np.arange(ny + 1) * blocks) // (ny + 1), blocks - 1)
    return vals[np.ix_(bj, bi)]


def k_field(chi, k1, k2):
    """Wavenumber between k1 and k2: k = k1 + (k2 - k1) chi."""
    return k1 + (k2 - k1) * np.asarray(chi)


def layered_velocity(nx, nz, h, seed, nlayers=10, vmin=1500.0, vmax=5500.0,
                     nanom=3, fault_throw=150.0):
    """Seeded layered velocity model v(x, z) in m/s on an (nz+1, nx+1) grid of
    spacing h metres (z downwards from row 0): ``nlayers`` dipping interfaces
    (dip angles uniform in +-8 degrees), layer velocities increasing with
    depth in [vmin, vmax], ``nanom`` Gaussian anomalies (+-15 %, width
    200-500 m) and one normal fault dipping 60 degrees that shifts the
    interfaces by ``fault_throw`` metres on its hanging-wall side."""
    rng = np.random.default_rng(seed)
    X = nx * h
    Z = nz * h
    z, x = np.meshgrid(np.arange(nz + 1) * h, np.arange(nx + 1) * h, indexing="ij")
    z0 = np.sort(rng.uniform(0.05 * Z, 0.95 * Z, nlayers))
    dips = np.tan(np.deg2rad(rng.uniform(-8, 8, nlayers)))
    vel = np.sort(rng.uniform(vmin, vmax, nlayers + 1))
    vel[0], vel[-1] = vmin, vmax
    xf = rng.uniform(0.3 * X, 0.7 * X)
    hanging = x > xf + z / np.tan(np.deg2rad(60.0))
    zz = z - np.where(hanging, fault_throw, 0.0)
    layer = np.zeros_like(x, dtype=np.int64)
    for t in range(nlayers):
        layer += (zz > z0[t] + (x - 0.5 * X) * dips[t]).astype(np.int64)
    v = vel[layer]
    for _ in range(nanom):
        cx, cz = rng.uniform(0.1 * X, 0.9 * X), rng.uniform(0.1 * Z, 0.9 * Z)
        s = rng.uniform(200.0, 500.0)
        amp = rng.uniform(-0.15, 0.15)
        v = v * (1.0 + amp * np.exp(-((x - cx) ** 2 + (z - cz) ** 2) / (2 * s * s)))
    return v


def smooth_perturbation(nx, ny, seed, sigma_nodes=20.0):
    """Seeded random field smoothed by a Gaussian of ``sigma_nodes`` nodes
    (FFT convolution, periodic), normalised to [-1, 1]."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((ny + 1, nx + 1))
    ky = np.fft.fftfreq(ny + 1)[:, None]
    kx = np.fft.fftfreq(nx + 1)[None, :]
    g = np.exp(-2.0 * (np.pi * sigma_nodes) ** 2 * (kx**2 + ky**2))
    s = np.real(np.fft.ifft2(np.fft.fft2(f) * g))
    s -= s.min()
    return 2.0 * s / s.max() - 1.0


def ragged_sizes(nprob, seed, lo=127, hi=1023):
    """``nprob`` interval counts drawn uniformly in [lo, hi], each rounded to
    the nearest c * 2^m with c in 4..7 so that every grid coarsens to a small
    coarsest grid."""
    rng = np.random.default_rng(seed)
    cands = sorted({c * 2**m for c in range(4, 8) for m in range(0, 12)})
    cands = np.array(cands)
    out = []
    for n in rng.integers(lo, hi + 1, nprob):
        out.append(int(cands[np.argmin(np.abs(cands - (n + 1)))]))
    return out


def sweep_points():
    """The constant-k sweep workloads (MP 2-A, centre point source, one
    right-hand side, relative residual 1e-6), as dicts with keys k, n,
    smoother ("gmres3" | "jacobi"), cycle ("V" | "W"), nu (pre = post
    smoothing steps), beta2 and group:

    * "k": k = 50, 100, 200, 400, 800 at kh = 0.625 (n = k / 0.625), GMRES(3)
      V(2,2) and W(2,2) with beta2 = 1/k, GMRES(3) V(1,1) without shift, and
      omega-Jacobi V(4,4) with beta2 = 0.7 up to k = 400;
    * "h": k = 100 at h = 1/128 .. 1/2048, GMRES(3) V(2,2), beta2 = 1/k;
    * "nu": k = 50 and 100 at kh = 0.625, GMRES(3) nu = 1..5, V and W, beta2 in
      {1/k, 0.7} (the settings of Sec. 5.3 Tables cons2g and cons1g), and
      omega-Jacobi V(nu, nu), nu = 1, 2, 4, beta2 = 0.7.
    """
    pts = []
    for k in (50.0, 100.0, 200.0, 400.0, 800.0):
        n = int(round(k / 0.625))
        for cyc in ("V", "W"):
            pts.append(dict(group="k", k=k, n=n, smoother="gmres3", cycle=cyc, nu=2, beta2=1.0 / k))
        pts.append(dict(group="k", k=k, n=n, smoother="gmres3", cycle="V", nu=1, beta2=0.0))
        if k <= 400.0:
            pts.append(dict(group="k", k=k, n=n, smoother="jacobi", cycle="V", nu=4, beta2=0.7))
    for n in (128, 256, 512, 1024, 2048):
        pts.append(dict(group="h", k=100.0, n=n, smoother="gmres3", cycle="V", nu=2, beta2=1.0 / 100.0))
    for k in (50.0, 100.0):
        n = int(round(k / 0.625))
        for nu in (1, 2, 3, 4, 5):
            for cyc in ("V", "W"):
                for b2 in (1.0 / k, 0.7):
                    pts.append(dict(group="nu", k=k, n=n, smoother="gmres3", cycle=cyc, nu=nu, beta2=b2))
        for nu in (1, 2, 4):
            pts.append(dict(group="nu", k=k, n=n, smoother="jacobi", cycle="V", nu=nu, beta2=0.7))
    return pts


def sweep_key(p):
    """Key of a sweep point in the stored tables."""
    return f"{p['k']:g}/{p['n']}/{p['smoother']}/{p['cycle']}{p['nu']}/{p['beta2']:g}"
