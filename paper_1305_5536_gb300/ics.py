"""Seeded synthetic initial conditions in the DG interchange layout.

This module holds no arithmetic of the DG step.  It evaluates analytic fields
(shaped like the paper's tests, Sec. 3: smooth advected waves, the Orszag-Tang
vortex, a Kelvin-Helmholtz shear layer, Gaussian random fields, stream-function
magnetic fields) and L2-projects them onto the cell bases of Sec. 2.2 with a
4-point Gauss rule per dimension:

* Taylor variables (rho, rho v, rho e): coefficients of 1, x, y[, z] about the
  cell centroid; the basis is orthogonal on a Cartesian cell, so
  c_k = int f W_k / int W_k^2.
* Magnetic field (2D MHD): coefficients (b1, b2, a1, a2, a3) of the locally
  divergence-free basis V1=(1,0), V2=(0,1), V3=(y,0), V4=(0,x), V5=(x,-y), also
  orthogonal on a Cartesian cell.

Interchange layout: float64 ``[plane, ny, nx]`` (2D) or ``[plane, nz, ny, nx]``
(3D); planes are variable-major, (average, d/dx, d/dy[, d/dz]) per Taylor
variable, then the magnetic block.  All randomness comes from
``numpy.random.default_rng(seed)``.
"""
import math

import numpy as np

EULER, MHD = 0, 1

# 4-point Gauss-Legendre rule on [-1/2, 1/2]
_g, _w = np.polynomial.legendre.leggauss(4)
GX = 0.5 * _g
GW = 0.5 * _w


def nplanes(eq, dim):
    return (4 if dim == 2 else 5) * (dim + 1) + (5 if eq == MHD else 0)


def _cell_points_2d(n, box):
    nx, ny = n[0], n[1]
    dx, dy = box[0] / nx, box[1] / ny
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    # global coordinates of the 4x4 Gauss points of every cell: [ny, nx, 4(y), 4(x)]
    X = xc[None, :, None, None] + dx * GX[None, None, None, :]
    Y = yc[:, None, None, None] + dy * GX[None, None, :, None]
    X = np.broadcast_to(X, (ny, nx, 4, 4))
    Y = np.broadcast_to(Y, (ny, nx, 4, 4))
    lx = np.broadcast_to(dx * GX[None, None, None, :], (ny, nx, 4, 4))
    ly = np.broadcast_to(dy * GX[None, None, :, None], (ny, nx, 4, 4))
    W = (GW[:, None] * GW[None, :])  # [4(y), 4(x)], sums to 1
    return X, Y, lx, ly, W, dx, dy


def _proj_taylor_2d(f, lx, ly, W, dx, dy):
    """(average, d/dx, d/dy) of samples f[ny, nx, 4, 4]."""
    c0 = np.einsum("ijab,ab->ij", f, W)
    cx = np.einsum("ijab,ab->ij", f * lx, W) / (dx * dx / 12.0)
    cy = np.einsum("ijab,ab->ij", f * ly, W) / (dy * dy / 12.0)
    return c0, cx, cy


def _proj_divfree_2d(bx, by, lx, ly, W, dx, dy):
    b1 = np.einsum("ijab,ab->ij", bx, W)
    b2 = np.einsum("ijab,ab->ij", by, W)
    a1 = np.einsum("ijab,ab->ij", bx * ly, W) / (dy * dy / 12.0)
    a2 = np.einsum("ijab,ab->ij", by * lx, W) / (dx * dx / 12.0)
    a3 = np.einsum("ijab,ab->ij", bx * lx - by * ly, W) / ((dx * dx + dy * dy) / 12.0)
    return b1, b2, a1, a2, a3


def project_2d(prim_fn, n, box=(1.0, 1.0), gamma=5.0 / 3.0, eq=EULER):
    """Project primitive fields onto the 2D bases.

    ``prim_fn(X, Y)`` returns (rho, vx, vy, p) for Euler, plus (Bx, By) for MHD,
    evaluated at arrays of global coordinates.
    """
    X, Y, lx, ly, W, dx, dy = _cell_points_2d(n, box)
    fields = prim_fn(X, Y)
    rho, vx, vy, p = [np.broadcast_to(np.asarray(a, dtype=np.float64), X.shape) for a in fields[:4]]
    if eq == MHD:
        Bx, By = [np.broadcast_to(np.asarray(a, dtype=np.float64), X.shape) for a in fields[4:6]]
        b2 = Bx * Bx + By * By
    else:
        b2 = 0.0
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy) + 0.5 * b2
    out = []
    for f in (rho, rho * vx, rho * vy, E):
        out.extend(_proj_taylor_2d(f, lx, ly, W, dx, dy))
    if eq == MHD:
        out.extend(_proj_divfree_2d(Bx, By, lx, ly, W, dx, dy))
    return np.ascontiguousarray(np.stack(out, axis=0))


def add_slope_noise(u, eq, dim, amp, rng):
    """Add U(-amp, amp) to every derivative coefficient of every Taylor variable."""
    u = u.copy()
    nT = 4 if dim == 2 else 5
    for v in range(nT):
        for k in range(1, dim + 1):
            u[v * (dim + 1) + k] += rng.uniform(-amp, amp, size=u.shape[1:])
    return u


# ----------------------------------------------------------------------------
# The workloads.  Each returns (u0, meta) with u0 float64 in interchange layout.
# ----------------------------------------------------------------------------

def euler2d_wave(n=(64, 64), amp=0.2, v=(1.0, 1.0), p=1.0, gamma=5.0 / 3.0, noise=1e-3,
                 seed=1305, direction=(1, 1)):
    """Smooth density wave rho = 1 + amp sin(2 pi (kx x + ky y)), uniform v and p,
    plus seeded U(-noise, noise) on every slope coefficient (2D Euler)."""
    kx, ky = direction

    def f(X, Y):
        return (1.0 + amp * np.sin(2 * np.pi * (kx * X + ky * Y)), v[0], v[1], p)

    u = project_2d(f, n, gamma=gamma)
    if noise > 0:
        u = add_slope_noise(u, EULER, 2, noise, np.random.default_rng(seed))
    return u


def orszag_tang(n=(512, 512), gamma=5.0 / 3.0):
    """Orszag-Tang vortex (Sec. 3.9): rho = gamma^2/(4 pi), p = gamma/(4 pi),
    v = (-sin 2 pi y, sin 2 pi x), B = (-sin 2 pi y, sin 4 pi x)/sqrt(4 pi)."""
    s4p = math.sqrt(4.0 * math.pi)

    def f(X, Y):
        return (gamma * gamma / (4 * np.pi), -np.sin(2 * np.pi * Y), np.sin(2 * np.pi * X),
                gamma / (4 * np.pi), -np.sin(2 * np.pi * Y) / s4p, np.sin(4 * np.pi * X) / s4p)

    return project_2d(f, n, gamma=gamma, eq=MHD)


def kh3d(n=(256, 256, 256), gamma=5.0 / 3.0, w0=0.01, sigma=0.05 / math.sqrt(2.0),
         vz_noise=1e-4, seed=1305):
    """3D Kelvin-Helmholtz shear layer (the 2D test of Sec. 3.6 extruded in z):
    rho = 2, vx = +0.5 for |y - 0.5| < 0.25, else rho = 1, vx = -0.5; p = 2.5;
    vy = w0 sin(4 pi x) (exp(-(y-.25)^2/2s^2) + exp(-(y-.75)^2/2s^2));
    seeded cell-constant U(-vz_noise, vz_noise) vz.  The bands are cell aligned
    when ny is a multiple of 4, so every field is smooth inside each cell."""
    nx, ny, nz = n
    inner = lambda Y: np.abs(Y - 0.5) < 0.25

    def f(X, Y):
        rho = np.where(inner(Y), 2.0, 1.0)
        vx = np.where(inner(Y), 0.5, -0.5)
        vy = w0 * np.sin(4 * np.pi * X) * (np.exp(-(Y - 0.25) ** 2 / (2 * sigma ** 2)) +
                                           np.exp(-(Y - 0.75) ** 2 / (2 * sigma ** 2)))
        return rho, vx, vy, 2.5

    # (x, y) projection of the z-independent part ...
    X, Y, lx, ly, W, dx, dy = _cell_points_2d((nx, ny), (1.0, 1.0))
    # sample at the cell-interior points, nudging exact-boundary points inside
    rho, vx, vy, p = [np.broadcast_to(np.asarray(a, dtype=np.float64), X.shape) for a in f(X, Y)]
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
    planes2d = []
    for fld in (rho, rho * vx, rho * vy, E):
        planes2d.append(_proj_taylor_2d(fld, lx, ly, W, dx, dy))
    # rho and vx are constant inside a cell (cell-aligned bands)
    rho_c = planes2d[0][0]
    rng = np.random.default_rng(seed)
    vz = rng.uniform(-vz_noise, vz_noise, size=(nz, ny, nx))
    u = np.zeros((20, nz, ny, nx))
    # ... extruded along z; variables (rho, mx, my, mz, E) x (avg, dx, dy, dz)
    order = [0, 1, 2, None, 3]
    for v, src in enumerate(order):
        if src is None:
            continue
        c0, cx, cy = planes2d[src]
        u[v * 4 + 0] = c0[None]
        u[v * 4 + 1] = cx[None]
        u[v * 4 + 2] = cy[None]
    u[3 * 4 + 0] = rho_c[None] * vz
    u[4 * 4 + 0] += 0.5 * rho_c[None] * vz * vz
    return u


def gaussian_random_field_2d(n_modes_max, ell, rms, rng):
    """Random smooth periodic field as an explicit Fourier sum: modes
    |k| <= n_modes_max * 2 pi, amplitudes ~ exp(-|k|^2 ell^2 / 4), random phases,
    normalised to the requested RMS.  Returns a callable f(X, Y)."""
    ks = []
    for a in range(-n_modes_max, n_modes_max + 1):
        for b in range(0, n_modes_max + 1):
            if b == 0 and a <= 0:
                continue
            if a * a + b * b > n_modes_max * n_modes_max:
                continue
            ks.append((a, b))
    ks = np.array(ks, dtype=np.float64)
    kk = 2 * np.pi * np.sqrt((ks ** 2).sum(1))
    amp = np.exp(-kk ** 2 * ell ** 2 / 4.0) * rng.standard_normal(len(ks))
    ph = rng.uniform(0, 2 * np.pi, len(ks))
    norm = rms / math.sqrt(0.5 * float((amp ** 2).sum()))

    def f(X, Y):
        s = np.zeros(np.broadcast(X, Y).shape)
        for (a, b), A, P in zip(ks, amp, ph):
            s += A * np.cos(2 * np.pi * (a * X + b * Y) + P)
        return norm * s

    return f


def euler2d_random_density(n=(256, 256), rms=0.05, ell=0.1, kmax=16, v=(1.0, 1.0), p=1.0,
                           gamma=5.0 / 3.0, seed=1305):
    """Background of the smooth-wave workload with rho = 1 + delta, delta a seeded
    Gaussian random field.  Returns (u0, delta) with delta callable."""
    rng = np.random.default_rng(seed)
    delta = gaussian_random_field_2d(kmax, ell, rms, rng)

    def f(X, Y):
        return (1.0 + delta(X, Y), v[0], v[1], p)

    return project_2d(f, n, gamma=gamma), delta


def _stream_modes(kmax, rng):
    ks = [(a, b) for a in range(-kmax, kmax + 1) for b in range(0, kmax + 1)
          if (b > 0 or a > 0) and a * a + b * b <= kmax * kmax]
    ks = np.array(ks, dtype=np.float64)
    amp = rng.standard_normal(len(ks)) / (1.0 + (ks ** 2).sum(1))
    ph = rng.uniform(0, 2 * np.pi, len(ks))
    return ks, amp, ph


def _curl_on_grid(modes, x1, y1):
    """(d psi/dy, -d psi/dx) of psi = sum A cos(2 pi (a x + b y) + P) on the tensor
    grid of 1D coordinate arrays x1 [nx, 4] and y1 [ny, 4] -> [ny, nx, 4, 4]."""
    ks, amp, ph = modes
    gx = np.zeros((y1.shape[0], x1.shape[0], y1.shape[1], x1.shape[1]))
    gy = np.zeros_like(gx)
    for (a, b), A, P in zip(ks, amp, ph):
        cx, sx = np.cos(2 * np.pi * a * x1), np.sin(2 * np.pi * a * x1)
        cy, sy = np.cos(2 * np.pi * b * y1 + P), np.sin(2 * np.pi * b * y1 + P)
        # sin(2 pi (a x + b y) + P) = sin(ax) cos(by + P) + cos(ax) sin(by + P)
        s = sx[None, :, None, :] * cy[:, None, :, None] + cx[None, :, None, :] * sy[:, None, :, None]
        s *= -2 * np.pi * A
        gx += s * a
        gy += s * b
    return gy, -gx


def mhd_random_smooth(N, kmax=4, vmax=0.3, bmax=0.3, gamma=5.0 / 3.0, rng=None):
    """One problem of the batched workload: rho = 1, p = 1, v and B the curls of
    seeded random-phase stream functions (modes |k| <= kmax * 2 pi), scaled so that
    max|v| = vmax and max|B| = bmax on the Gauss points; the curl of a stream
    function is divergence free, and so is its projection on the magnetic basis."""
    rng = np.random.default_rng(1305) if rng is None else rng
    mv = _stream_modes(kmax, rng)
    mb = _stream_modes(kmax, rng)
    h = 1.0 / N
    x1 = (np.arange(N) + 0.5)[:, None] * h + h * GX[None, :]
    vx, vy = _curl_on_grid(mv, x1, x1)
    bx, by = _curl_on_grid(mb, x1, x1)
    sv = vmax / max(np.sqrt(vx * vx + vy * vy).max(), 1e-300)
    sb = bmax / max(np.sqrt(bx * bx + by * by).max(), 1e-300)
    vals = (1.0, sv * vx, sv * vy, 1.0, sb * bx, sb * by)
    return project_2d(lambda X, Y: vals, (N, N), gamma=gamma, eq=MHD)


def batch_sizes(nprob=64, nmin=32, nmax=512, seed=1305):
    """Grid sizes N = round(nmin (nmax/nmin)^u), u ~ U(0, 1) (log-uniform)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, nprob)
    return [int(round(nmin * (nmax / nmin) ** x)) for x in u]


def mhd_batch(nprob=64, nmin=32, nmax=512, seed=1305):
    sizes = batch_sizes(nprob, nmin, nmax, seed)
    rng = np.random.default_rng(seed + 1)
    return sizes, [mhd_random_smooth(N, rng=rng) for N in sizes]


# ----------------------------------------------------------------------------
# The paper's test problems (Sec. 3), analytic fields projected as above.
# ----------------------------------------------------------------------------

def gresho_fields(r):
    """Sec. 3.3 triangle vortex: azimuthal velocity and pressure at radius r."""
    vphi = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    rs = np.maximum(r, 1e-300)
    p = np.where(r < 0.2, 5.0 + 12.5 * r * r,
                 np.where(r < 0.4, 9.0 + 12.5 * r * r - 20.0 * r + 4.0 * np.log(rs / 0.2),
                          3.0 + 4.0 * math.log(2.0)))
    return vphi, p


def gresho(n=(64, 64), gamma=5.0 / 3.0):
    """Sec. 3.3 Gresho vortex: rho = 1, the steady triangle vortex centred in the
    unit periodic box."""
    def f(X, Y):
        dx, dy = X - 0.5, Y - 0.5
        r = np.sqrt(dx * dx + dy * dy)
        vphi, p = gresho_fields(r)
        rs = np.maximum(r, 1e-300)
        return 1.0, -vphi * dy / rs, vphi * dx / rs, p
    return project_2d(f, n, gamma=gamma)


def implosion(n=(256, 256), gamma=1.4):
    """Sec. 3.4 implosion: periodic box of side 0.3, gas at rest, (rho, p) = (1, 1)
    for x + y > 0.15, else (0.125, 0.14)."""
    def f(X, Y):
        hi = X + Y > 0.15
        return np.where(hi, 1.0, 0.125), 0.0, 0.0, np.where(hi, 1.0, 0.14)
    return project_2d(f, n, box=(0.3, 0.3), gamma=gamma)


def rotor(n=(512, 512), gamma=5.0 / 3.0, r0=0.1, r1=0.115):
    """Sec. 3.7 magnetic rotor: p = 0.5, B = (2.5/sqrt(4 pi), 0), a dense disc
    (rho = 10) spinning with angular velocity 1/r0 inside r0, tapered off to the
    ambient gas at rest between r0 and r1 with f = (r1 - r)/(r1 - r0):
    rho = 1 + 9 f, v = f v(r0) r0/r (continuous across both radii)."""
    def f(X, Y):
        dx, dy = X - 0.5, Y - 0.5
        r = np.sqrt(dx * dx + dy * dy)
        rs = np.maximum(r, 1e-300)
        fr = (r1 - r) / (r1 - r0)
        inner, taper = r <= r0, (r > r0) & (r <= r1)
        rho = np.where(inner, 10.0, np.where(taper, 1.0 + 9.0 * fr, 1.0))
        vx = np.where(inner, -dy / r0, np.where(taper, -fr * dy / rs, 0.0))
        vy = np.where(inner, dx / r0, np.where(taper, fr * dx / rs, 0.0))
        return rho, vx, vy, 0.5, 2.5 / math.sqrt(4.0 * math.pi), 0.0
    return project_2d(f, n, gamma=gamma, eq=MHD)


def sod_tube(N=64, L=20.0, gamma=1.4, left=(1.0, 1.0), right=(0.25, 0.1795)):
    """Sec. 3.2 shock tube as a periodic 1D problem in 2D storage (one cell in y):
    box [-L, L) with the left state (rho, p) on [-L, 0) and the right state on
    [0, L), gas at rest; N cells per half.  Returns (u0, box)."""
    nx = 2 * N
    box = (2.0 * L, L / N)

    def f(X, Y):
        lft = X - L < 0
        return (np.where(lft, left[0], right[0]), 0.0, 0.0, np.where(lft, left[1], right[1]))
    return project_2d(f, (nx, 1), box=box, gamma=gamma), box


# ----------------------------------------------------------------------------
# 3D projection (Taylor variables and the 11-function divergence-free field
# basis of Sec. 2.2), one z-layer of cells at a time.
# ----------------------------------------------------------------------------

def _proj_divfree_3d(B, l, W, h):
    """Coefficients (b1, b2, b3, a4, ..., a11) of the 3D basis V1..V11 from the
    field samples B[3][...,4,4,4] at local offsets l[3] with weights W (sum 1):
    the basis is orthogonal on a Cartesian cell except V10 = (x,-y,0) and
    V11 = (x,0,-z), whose 2x2 block [[hx^2+hy^2, hx^2], [hx^2, hx^2+hz^2]] / 12 is
    solved explicitly."""
    m = lambda f: np.einsum("...abc,abc->...", f, W)
    hx2, hy2, hz2 = h[0] ** 2 / 12.0, h[1] ** 2 / 12.0, h[2] ** 2 / 12.0
    b1, b2, b3 = m(B[0]), m(B[1]), m(B[2])
    a4, a5 = m(B[0] * l[1]) / hy2, m(B[0] * l[2]) / hz2
    a6, a7 = m(B[1] * l[0]) / hx2, m(B[1] * l[2]) / hz2
    a8, a9 = m(B[2] * l[0]) / hx2, m(B[2] * l[1]) / hy2
    r10 = m(B[0] * l[0] - B[1] * l[1])
    r11 = m(B[0] * l[0] - B[2] * l[2])
    det = (hx2 + hy2) * (hx2 + hz2) - hx2 * hx2
    a10 = ((hx2 + hz2) * r10 - hx2 * r11) / det
    a11 = ((hx2 + hy2) * r11 - hx2 * r10) / det
    return b1, b2, b3, a4, a5, a6, a7, a8, a9, a10, a11


def project_3d(prim_fn, n, box=(1.0, 1.0, 1.0), gamma=5.0 / 3.0, eq=EULER):
    """Project primitive fields onto the 3D bases.  ``prim_fn(X, Y, Z)`` returns
    (rho, vx, vy, vz, p) for Euler, plus (Bx, By, Bz) for MHD."""
    nx, ny, nz = n
    h = (box[0] / nx, box[1] / ny, box[2] / nz)
    npl = 20 + (11 if eq == MHD else 0)
    u = np.zeros((npl, nz, ny, nx))
    xc = (np.arange(nx) + 0.5) * h[0]
    yc = (np.arange(ny) + 0.5) * h[1]
    W = GW[:, None, None] * GW[None, :, None] * GW[None, None, :]  # [z, y, x]
    lz = np.broadcast_to(h[2] * GX[:, None, None], (4, 4, 4))
    ly = np.broadcast_to(h[1] * GX[None, :, None], (4, 4, 4))
    lx = np.broadcast_to(h[0] * GX[None, None, :], (4, 4, 4))
    X = xc[None, :, None, None, None] + lx[None, None]
    Y = yc[:, None, None, None, None] + ly[None, None]
    shp = (ny, nx, 4, 4, 4)
    X, Y = np.broadcast_to(X, shp), np.broadcast_to(Y, shp)
    for k in range(nz):
        Z = np.broadcast_to((k + 0.5) * h[2] + lz, shp)
        f = [np.broadcast_to(np.asarray(a, dtype=np.float64), shp) for a in prim_fn(X, Y, Z)]
        rho, vx, vy, vz, p = f[:5]
        b2 = 0.0
        if eq == MHD:
            b2 = f[5] ** 2 + f[6] ** 2 + f[7] ** 2
        E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * b2
        for v, fld in enumerate((rho, rho * vx, rho * vy, rho * vz, E)):
            u[4 * v, k] = np.einsum("ijabc,abc->ij", fld, W)
            for d, (ll, hh) in enumerate(((lx, h[0]), (ly, h[1]), (lz, h[2]))):
                u[4 * v + 1 + d, k] = np.einsum("ijabc,abc->ij", fld * ll, W) / (hh * hh / 12.0)
        if eq == MHD:
            co = _proj_divfree_3d(f[5:8], (lx, ly, lz), W, h)
            for j, c in enumerate(co):
                u[20 + j, k] = c
    return u


def alfven_cp_3d(n=(16, 16, 16), t=0.0, eps=0.1, rho=1.0, p=0.1, B0=1.0, gamma=5.0 / 3.0):
    """Circularly polarised Alfven wave travelling along k = 2 pi (1, 1, 1) in the
    unit periodic cube: B = B0 k^ + eps (e1 sin phi + e2 cos phi), v = -(B - B0 k^)
    / sqrt(rho), rho and p uniform, phi = k.x - |k| B0/sqrt(rho) t: an exact
    solution of ideal MHD of any amplitude."""
    kh = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    e1 = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    e2 = np.cross(kh, e1)
    vA = B0 / math.sqrt(rho)

    def f(X, Y, Z):
        ph = 2 * math.pi * ((X + Y + Z) - math.sqrt(3.0) * vA * t)
        s, c = np.sin(ph), np.cos(ph)
        dB = [eps * (e1[i] * s + e2[i] * c) for i in range(3)]
        v = [-dB[i] / math.sqrt(rho) for i in range(3)]
        B = [B0 * kh[i] + dB[i] for i in range(3)]
        return (rho, v[0], v[1], v[2], p, B[0], B[1], B[2])
    return project_3d(f, n, gamma=gamma, eq=MHD)


def orszag_tang_3d(n=(128, 128, 128), gamma=5.0 / 3.0, eps=0.2):
    """A 3D extension of the Orszag-Tang vortex: the 2D fields of Sec. 3.8 (B
    scaled by 1/sqrt(4 pi)) with a z-modulated velocity, v = ((1 + eps sin 2 pi z)
    (-sin 2 pi y), (1 + eps sin 2 pi z) sin 2 pi x, eps sin 2 pi z); B has no z
    dependence and stays divergence free."""
    s4 = 1.0 / math.sqrt(4 * math.pi)

    def f(X, Y, Z):
        m = 1 + eps * np.sin(2 * np.pi * Z)
        return (gamma ** 2 / (4 * math.pi), -m * np.sin(2 * np.pi * Y), m * np.sin(2 * np.pi * X),
                eps * np.sin(2 * np.pi * Z), gamma / (4 * math.pi), -s4 * np.sin(2 * np.pi * Y),
                s4 * np.sin(4 * np.pi * X), 0.0)
    return project_3d(f, n, gamma=gamma, eq=MHD)
