"""Seeded synthetic inputs: grids, snapshot fields and camera views.

This module only builds inputs.  It holds none of the rendering arithmetic
(no ray traversal, no Doppler factor, no temporal weights), so that the FP64
oracle and the GPU library can both take their inputs from here without
sharing any code of the method itself.

Conventions
-----------
* Fields are C-ordered ``j[M][nz][ny][nx]`` and ``beta[M][nz][ny][nx][3]``
  (x fastest), sampled at cell centres ``origin + (i + 1/2) dx``.
* ``c`` is in cells per unit time, epochs sit at ``t_m = t0 + m dt``.
* A view looks along ``dir`` (into the scene).  The direction *to* the
  observer is ``n = (sin th cos ph, sin th sin ph, cos th)`` with theta
  measured from +z (the jet / velocity axis), so ``dir = -n``.  Image "up" is
  +z projected onto the image plane, or +y when the view is along z.
* Random numbers are counter based: splitmix64 of (seed, stream, cell index)
  followed by Box-Muller, so any subset of cells can be regenerated alone.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

__all__ = [
    "Grid", "View", "view_from_angles", "fibonacci_directions", "splitmix64",
    "uniform01", "normal", "conical_jet", "gaussian_blob", "uniform_fields",
    "config_tiny", "config_time_delay", "twin_ejecta", "kolmogorov",
    "config_precision", "config_batched", "view_from_direction", "kolmogorov_torch",
    "turbulent_jet_torch", "config_precision_device", "config_batched_device",
]


@dataclass(frozen=True)
class Grid:
    """Uniform Cartesian mesh with ``n_epochs`` snapshots at cadence ``dt``."""
    n: tuple[int, int, int]
    origin: tuple[float, float, float] = (0.0, 0.0, 0.0)
    dx: tuple[float, float, float] = (1.0, 1.0, 1.0)
    n_epochs: int = 1
    t0: float = 0.0
    dt: float = 1.0

    @property
    def extent(self) -> np.ndarray:
        return np.asarray(self.n, dtype=np.float64) * np.asarray(self.dx, dtype=np.float64)

    @property
    def center(self) -> np.ndarray:
        return np.asarray(self.origin, dtype=np.float64) + 0.5 * self.extent

    @property
    def n_cells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def cell_centres(self, axis: int) -> np.ndarray:
        return self.origin[axis] + (np.arange(self.n[axis], dtype=np.float64) + 0.5) * self.dx[axis]


@dataclass(frozen=True)
class View:
    """One orthographic camera plus its image size and physics switches."""
    dir: tuple[float, float, float]
    up: tuple[float, float, float]
    center: tuple[float, float, float]
    t_obs: float = 0.0
    c: float = 1.0
    alpha: float = -0.6
    nu_ratio: float = 1.0
    beaming: bool = True
    lookback: bool = True
    width: int = 64
    height: int = 64
    fov_u: float = 1.0
    fov_v: float = 1.0

    def with_(self, **kw) -> "View":
        return replace(self, **kw)


def view_from_angles(grid: Grid, theta_deg: float, phi_deg: float = 0.0, *, size: int = 64,
                     fov: float | None = None, **kw) -> View:
    """View whose observer direction is at polar angle theta from +z."""
    th, ph = math.radians(theta_deg), math.radians(phi_deg)
    n_hat = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    return view_from_direction(grid, -n_hat, size=size, fov=fov, **kw)


def view_from_direction(grid: Grid, direction, *, size: int = 64, fov: float | None = None,
                        height: int | None = None, **kw) -> View:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    up = (0.0, 0.0, 1.0)
    if abs(abs(d[2]) - 1.0) < 1e-12:
        up = (0.0, 1.0, 0.0)
    if fov is None:
        fov = math.sqrt(3.0) * float(np.max(grid.extent))
    h = size if height is None else height
    return View(dir=tuple(float(x) for x in d), up=up, center=tuple(float(x) for x in grid.center),
                width=size, height=h, fov_u=fov, fov_v=fov * h / size, **kw)


def fibonacci_directions(n: int) -> np.ndarray:
    """``n`` unit vectors spread uniformly over the sphere (Fibonacci lattice)."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    phi = golden * k
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


# --------------------------------------------------------------------------
# Counter-based random numbers
# --------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea & Flood 2014) on uint64 counters."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Uniform numbers in (0, 1) from (seed, stream, counter)."""
    key = splitmix64(np.array([(seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        bits = splitmix64(counters.astype(np.uint64) ^ key)
    return ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Standard normal numbers by Box-Muller on two counter streams."""
    u1 = uniform01(seed, 2 * stream, counters)
    u2 = uniform01(seed, 2 * stream + 1, counters)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# Field builders (all return float64 arrays)
# --------------------------------------------------------------------------
def conical_jet(grid: Grid, seed: int, *, j0: float = 1.0, half_angle_deg: float = 5.0,
                apex=None, noise: float = 0.01, epoch: int = 0, floor: float = 0.0) -> np.ndarray:
    """Conical jet along +z: Gaussian cross-section of width r tan(half-angle),
    emissivity falling as max(r, 1)^-2 with distance r from the apex, times a
    lognormal factor exp(noise * N(0, 1)).  Returns j[nz][ny][nx]."""
    nx, ny, nz = grid.n
    if apex is None:
        apex = (grid.center[0], grid.center[1], grid.origin[2] + grid.extent[2] / 16.0)
    x = grid.cell_centres(0)[None, None, :]
    y = grid.cell_centres(1)[None, :, None]
    z = grid.cell_centres(2)[:, None, None]
    r = z - apex[2]
    rr = np.maximum(r, 1.0)
    sig = rr * math.tan(math.radians(half_angle_deg))
    rho2 = (x - apex[0]) ** 2 + (y - apex[1]) ** 2
    j = j0 * rr ** -2.0 * np.exp(-rho2 / (2.0 * sig * sig))
    j = np.where(r >= 0.0, j, 0.0)
    if noise > 0.0:
        cnt = np.arange(grid.n_cells, dtype=np.uint64).reshape(nz, ny, nx)
        j = j * np.exp(noise * normal(seed, 1000 + epoch, cnt))
    if floor > 0.0:
        j = j + floor
    return j


def gaussian_blob(grid: Grid, centre, sigma: float, j0: float = 1.0) -> np.ndarray:
    x = grid.cell_centres(0)[None, None, :]
    y = grid.cell_centres(1)[None, :, None]
    z = grid.cell_centres(2)[:, None, None]
    d2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return j0 * np.exp(-d2 / (2.0 * sigma * sigma))


def uniform_fields(grid: Grid, j: float = 1.0, beta=(0.0, 0.0, 0.0)):
    nx, ny, nz = grid.n
    M = grid.n_epochs
    jj = np.full((M, nz, ny, nx), j, dtype=np.float64)
    bb = np.empty((M, nz, ny, nx, 3), dtype=np.float64)
    bb[...] = np.asarray(beta, dtype=np.float64)
    return jj, bb


def config_tiny(seed: int = 1):
    """32^3 single epoch, seeded conical jet, beta = 0.9 z, one 64x64 view at
    theta = 30 deg without light-travel delay (alpha = -0.6, i.e. D^2.6)."""
    grid = Grid(n=(32, 32, 32), n_epochs=1, t0=0.0, dt=1.0)
    j = conical_jet(grid, seed)[None]
    _, beta = uniform_fields(grid, 0.0, (0.0, 0.0, 0.9))
    view = view_from_angles(grid, 30.0, 0.0, size=64, lookback=False, beaming=True, alpha=-0.6)
    return grid, j, beta, [view]


def config_time_delay(seed: int = 2, n: int = 256, n_epochs: int = 16, size: int = 512,
                      thetas=(10.0, 45.0), n_tobs: int = 9, dtype=np.float64):
    """Moving Gaussian blob (sigma = n/32) over a steady conical jet, both at
    beta = 0.95 z; c dt = 4 cells so the blob moves 3.8 cells per epoch.
    Views: every theta x ``n_tobs`` observer times whose blob-centre retarded
    time sweeps epochs 3 .. 12 (scaled to ``n_epochs``)."""
    c, dt, beta_z = 1.0, 4.0, 0.95
    grid = Grid(n=(n, n, n), n_epochs=n_epochs, t0=0.0, dt=dt)
    s = n / 256.0
    sigma = 8.0 * s
    start = np.array([grid.center[0], grid.center[1], 64.0 * s])
    jet = 0.1 * conical_jet(grid, seed)
    j = np.empty((n_epochs, n, n, n), dtype=dtype)
    for m in range(n_epochs):
        pos = start + np.array([0.0, 0.0, beta_z * c * dt * m])
        j[m] = jet + gaussian_blob(grid, pos, sigma, 1.0)
    beta = np.zeros((n_epochs, n, n, n, 3), dtype=dtype)
    beta[..., 2] = beta_z
    views = []
    lo, hi = 3.0 * (n_epochs - 1) / 15.0, 12.0 * (n_epochs - 1) / 15.0
    for th in thetas:
        base = view_from_angles(grid, th, 0.0, size=size, c=c, lookback=True, beaming=True)
        shat = np.asarray(base.dir)
        for k in range(n_tobs):
            m_ret = lo + (hi - lo) * k / max(n_tobs - 1, 1)
            # Observer time at which the blob centre is seen at epoch m_ret:
            # the blob is at `pos` when t = m_ret dt, and its depth along the
            # line of sight from the image plane is (pos - centre) . s_hat.
            pos = start + np.array([0.0, 0.0, beta_z * c * dt * m_ret])
            depth = float(np.dot(pos - grid.center, shat))
            views.append(base.with_(t_obs=m_ret * dt + depth / c))
    return grid, j, beta, views


def twin_ejecta(*, n: int = 96, radius: float = 12.0, gamma: float = 2.0, theta_deg: float = 45.0,
                n_epochs: int = 64, c_dt: float = 1.0, size: int = 128, separation: float = 0.0):
    """Two homogeneous ejecta (j' = 1), spheres of rest-frame radius ``radius``,
    moving along +z and -z with Lorentz factor ``gamma``: in the lab frame each
    is an oblate spheroid with axial ratio 1/gamma along z.  Both start at the
    grid centre offset by +-``separation`` along z.  Returns
    (grid, j, beta, views, meta) with one view per observer time whose
    retarded time of the grid centre covers the middle of the epoch range."""
    beta_mag = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    c = 1.0
    dt = c_dt / c
    grid = Grid(n=(n, n, n), n_epochs=n_epochs, t0=0.0, dt=dt)
    nx = ny = nz = n
    x = grid.cell_centres(0)[None, None, :]
    y = grid.cell_centres(1)[None, :, None]
    z = grid.cell_centres(2)[:, None, None]
    ctr = grid.center
    j = np.zeros((n_epochs, nz, ny, nx), dtype=np.float64)
    beta = np.zeros((n_epochs, nz, ny, nx, 3), dtype=np.float64)
    t_start = 0.0
    for m in range(n_epochs):
        t = t_start + m * dt
        for sign in (+1.0, -1.0):
            zc = ctr[2] + sign * (separation + beta_mag * c * t)
            inside = ((x - ctr[0]) ** 2 + (y - ctr[1]) ** 2) / radius ** 2 \
                + ((z - zc) * gamma) ** 2 / radius ** 2 <= 1.0
            j[m] = np.where(inside, 1.0, j[m])
            beta[m, ..., 2] = np.where(inside, sign * beta_mag, beta[m, ..., 2])
    meta = dict(beta=beta_mag, gamma=gamma, radius=radius, c=c, dt=dt, theta=theta_deg)
    view = view_from_angles(grid, theta_deg, 0.0, size=size, c=c, fov=float(n))
    return grid, j, beta, [view], meta


def ejectum(sign: int, *, radius: float = 8.0, gamma: float = 2.0, theta_deg: float = 45.0, c_dt: float = 1.0,
            size: int = 64, lookback: bool = True, view_shift: float = 0.0, dtype=np.float32):
    """One homogeneous ejectum (j' = 1), a sphere of rest-frame radius
    ``radius`` moving along sign * z with Lorentz factor ``gamma`` (a lab-frame
    spheroid of axial ratio 1 / gamma), stored over every epoch its observed
    light-cone slice needs at cadence ``c_dt`` (c = 1), viewed at theta.

    Returns (grid, j, beta, view, t_mid, kappa): the view is centred on the
    ejectum at the middle epoch time t_mid and kappa = 1 - beta cos(theta) for
    the approaching one (sign +1), 1 + beta cos(theta) for the receding one.
    Without lookback one epoch is stored, with the ejectum at the box centre.
    ``view_shift`` moves the view centre along y (the axis the view runs
    parallel to) so that no pixel's ray lies in a cell-face plane."""
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    kappa = 1.0 - sign * beta * math.cos(math.radians(theta_deg))
    span = 2.0 * radius / kappa + 3.0 * c_dt / kappa + 4.0
    M = int(math.ceil(span / c_dt)) + 1 if lookback else 1
    nxy = int(math.ceil(2 * (radius + 2)))
    zpad = radius / gamma + 2.0
    nz = int(math.ceil(beta * (M - 1) * c_dt + 2 * zpad))
    grid = Grid(n=(nxy, nxy, nz), n_epochs=M, t0=0.0, dt=c_dt)
    x = grid.cell_centres(0)[None, None, :]
    y = grid.cell_centres(1)[None, :, None]
    z = grid.cell_centres(2)[:, None, None]
    z0 = (zpad if sign > 0 else nz - zpad) if lookback else 0.5 * nz
    j = np.zeros((M, nz, nxy, nxy), dtype)
    b = np.zeros((M, nz, nxy, nxy, 3), dtype)
    for m in range(M):
        zc = z0 + sign * beta * m * c_dt
        inside = (x - nxy / 2) ** 2 + (y - nxy / 2) ** 2 + ((z - zc) * gamma) ** 2 <= radius * radius
        j[m] = inside
        b[m, ..., 2] = np.where(inside, sign * beta, 0.0)
    t_mid = 0.5 * (M - 1) * c_dt
    centre = (nxy / 2, nxy / 2 + view_shift, z0 + sign * beta * t_mid)
    v = view_from_angles(grid, theta_deg, 0.0, size=size, fov=3.2 * radius, c=1.0, beaming=True, lookback=lookback)
    return grid, j, b, v.with_(center=centre, t_obs=t_mid), t_mid, kappa


# --------------------------------------------------------------------------
# Kolmogorov fields for the turbulent-jet configurations
# --------------------------------------------------------------------------
def kolmogorov(shape, seed: int, stream: int = 0, *, slope: float = -11.0 / 3.0,
               phase_shift=None, t: float = 0.0) -> np.ndarray:
    """Periodic Gaussian random field with power spectrum P(k) ~ k^slope,
    zero mean and unit rms, from numpy PCG64(seed, stream) random phases.

    ``t`` advances every Fourier mode's phase by omega(k) t with
    omega ~ k^(2/3) (eddy turnover), for a slowly evolving series."""
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64([seed, stream]))
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz).astype(np.float32)
    k[0, 0, 0] = np.inf
    amp = k ** np.float32(slope / 2.0)
    phase = rng.random(k.shape, dtype=np.float32) * np.float32(2.0 * math.pi)
    if t != 0.0:
        kk = np.where(np.isfinite(k), k, 0.0).astype(np.float32)
        phase = phase + np.float32(t) * (kk * np.float32(max(nx, ny, nz))) ** np.float32(2.0 / 3.0)
    spec = (amp * np.exp(1j * phase)).astype(np.complex64)
    field = np.fft.irfftn(spec, s=(nz, ny, nx), axes=(0, 1, 2)).astype(np.float64)
    field -= field.mean()
    rms = field.std()
    return field / rms if rms > 0 else field


def _turbulent_jet(grid: Grid, seed: int, c_dt: float):
    """Conical jet x lognormal(0.3) Kolmogorov fluctuations + ambient floor;
    |beta| = clip(0.5 + 0.49 exp(-rho^2 / 2 sigma^2) + delta, 0.5, 0.99) with
    Kolmogorov delta (rms 0.05); direction +z tilted by a Kolmogorov transverse
    angle (rms 0.1 rad).  Epochs evolve by Kolmogorov phase advance."""
    nx, ny, nz = grid.n
    M = grid.n_epochs
    shape = (nz, ny, nx)
    apex = (grid.center[0], grid.center[1], grid.origin[2] + grid.extent[2] / 16.0)
    base = conical_jet(grid, seed, noise=0.0, apex=apex)
    x = grid.cell_centres(0)[None, None, :]
    y = grid.cell_centres(1)[None, :, None]
    z = grid.cell_centres(2)[:, None, None]
    rr = np.maximum(z - apex[2], 1.0)
    sig = rr * math.tan(math.radians(5.0))
    rho2 = (x - apex[0]) ** 2 + (y - apex[1]) ** 2
    core = np.exp(-rho2 / (2.0 * sig * sig))
    j = np.empty((M, nz, ny, nx), dtype=np.float32)
    beta = np.empty((M, nz, ny, nx, 3), dtype=np.float32)
    for m in range(M):
        tt = 0.05 * m
        dens = kolmogorov(shape, seed, 0, t=tt)
        j[m] = (base * np.exp(0.3 * dens) + 1e-3).astype(np.float32)
        delta = 0.05 * kolmogorov(shape, seed, 1, t=tt)
        mag = np.clip(0.5 + 0.49 * core + delta, 0.5, 0.99)
        tx = 0.1 * kolmogorov(shape, seed, 2, t=tt)
        ty = 0.1 * kolmogorov(shape, seed, 3, t=tt)
        # unit direction from two small tilt angles about x and y
        dxv, dyv = np.sin(tx), np.sin(ty)
        dzv = np.sqrt(np.maximum(0.0, 1.0 - dxv * dxv - dyv * dyv))
        beta[m, ..., 0] = (mag * dxv).astype(np.float32)
        beta[m, ..., 1] = (mag * dyv).astype(np.float32)
        beta[m, ..., 2] = (mag * dzv).astype(np.float32)
    return j, beta


def config_precision(seed: int = 3, n: int = 512, n_epochs: int = 8, size: int = 1024):
    """Turbulent jet, n^3 x n_epochs, c dt = n/4 so the lookback window covers
    the whole diagonal; one view at theta = 30, phi = 20, t_obs mid-window."""
    c_dt = n / 4.0
    grid = Grid(n=(n, n, n), n_epochs=n_epochs, t0=0.0, dt=c_dt)
    j, beta = _turbulent_jet(grid, seed, c_dt)
    view = view_from_angles(grid, 30.0, 20.0, size=size, c=1.0)
    t_mid = 0.5 * (n_epochs - 1) * c_dt
    return grid, j, beta, [view.with_(t_obs=t_mid)]


def config_batched(seed: int = 4, n: int = 384, n_epochs: int = 32, size: int = 256, n_views: int = 256):
    """Turbulent jet at n^3 x n_epochs (c dt = n/16), ``n_views`` orientations
    on a Fibonacci sphere, each ``size``^2, t_obs mid-window."""
    c_dt = n / 16.0
    grid = Grid(n=(n, n, n), n_epochs=n_epochs, t0=0.0, dt=c_dt)
    j, beta = _turbulent_jet(grid, seed, c_dt)
    t_mid = 0.5 * (n_epochs - 1) * c_dt
    views = [view_from_direction(grid, -d, size=size, c=1.0, t_obs=t_mid)
             for d in fibonacci_directions(n_views)]
    return grid, j, beta, views


# --------------------------------------------------------------------------
# Device-side builders for the full-size turbulent configurations
# --------------------------------------------------------------------------
def kolmogorov_torch(shape, seed: int, stream: int, *, t: float = 0.0, device="cuda", slope: float = -11.0 / 3.0):
    """Same recipe as ``kolmogorov`` (random Fourier phases, amplitude
    k^(slope/2), phase advance t (k N)^(2/3), zero mean, unit rms) built with
    torch on ``device`` from a torch generator seeded with (seed, stream).
    The numbers differ from the numpy variant; each is reproducible on its
    own device type."""
    import torch
    nz, ny, nx = shape
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1000003 + int(stream)) & 0x7FFFFFFFFFFFFFFF)
    kz = torch.fft.fftfreq(nz, device=device)[:, None, None]
    ky = torch.fft.fftfreq(ny, device=device)[None, :, None]
    kx = torch.fft.rfftfreq(nx, device=device)[None, None, :]
    k = torch.sqrt(kx * kx + ky * ky + kz * kz)
    amp = torch.where(k > 0, k.clamp_min(1e-12) ** (slope / 2.0), torch.zeros_like(k))
    phase = torch.rand(k.shape, generator=g, device=device) * (2.0 * math.pi)
    if t != 0.0:
        phase = phase + t * (k * max(nx, ny, nz)) ** (2.0 / 3.0)
    spec = torch.polar(amp, phase)
    del amp, phase, k
    field = torch.fft.irfftn(spec, s=(nz, ny, nx))
    del spec
    field -= field.mean()
    rms = field.std()
    return field / rms if float(rms) > 0 else field


def turbulent_jet_torch(grid: Grid, seed: int, device="cuda"):
    """The turbulent jet of ``config_precision`` built on ``device``:
    returns float32 tensors j[M][nz][ny][nx] and beta[M][nz][ny][nx][3]."""
    import torch
    nx, ny, nz = grid.n
    M = grid.n_epochs
    shape = (nz, ny, nx)
    apex = (float(grid.center[0]), float(grid.center[1]), float(grid.origin[2] + grid.extent[2] / 16.0))
    x = torch.tensor(grid.cell_centres(0), dtype=torch.float32, device=device)[None, None, :]
    y = torch.tensor(grid.cell_centres(1), dtype=torch.float32, device=device)[None, :, None]
    z = torch.tensor(grid.cell_centres(2), dtype=torch.float32, device=device)[:, None, None]
    r = z - apex[2]
    rr = r.clamp_min(1.0)
    sig = rr * math.tan(math.radians(5.0))
    rho2 = (x - apex[0]) ** 2 + (y - apex[1]) ** 2
    core = torch.exp(-rho2 / (2.0 * sig * sig))
    base = torch.where(r >= 0, rr ** -2.0 * core, torch.zeros_like(core))
    j = torch.empty((M, nz, ny, nx), dtype=torch.float32, device=device)
    beta = torch.empty((M, nz, ny, nx, 3), dtype=torch.float32, device=device)
    for m in range(M):
        tt = 0.05 * m
        j[m] = base * torch.exp(0.3 * kolmogorov_torch(shape, seed, 0, t=tt, device=device)) + 1e-3
        mag = (0.5 + 0.49 * core + 0.05 * kolmogorov_torch(shape, seed, 1, t=tt, device=device)).clamp(0.5, 0.99)
        dxv = torch.sin(0.1 * kolmogorov_torch(shape, seed, 2, t=tt, device=device))
        dyv = torch.sin(0.1 * kolmogorov_torch(shape, seed, 3, t=tt, device=device))
        dzv = torch.sqrt((1.0 - dxv * dxv - dyv * dyv).clamp_min(0.0))
        beta[m, ..., 0] = mag * dxv
        beta[m, ..., 1] = mag * dyv
        beta[m, ..., 2] = mag * dzv
    return j, beta


def config_precision_device(seed: int = 3, n: int = 512, n_epochs: int = 8, size: int = 1024, device="cuda"):
    """``config_precision`` at full size with the fields built on ``device``."""
    c_dt = n / 4.0
    grid = Grid(n=(n, n, n), n_epochs=n_epochs, t0=0.0, dt=c_dt)
    j, beta = turbulent_jet_torch(grid, seed, device)
    view = view_from_angles(grid, 30.0, 20.0, size=size, c=1.0)
    return grid, j, beta, [view.with_(t_obs=0.5 * (n_epochs - 1) * c_dt)]


def config_batched_device(seed: int = 4, n: int = 384, n_epochs: int = 32, size: int = 256, n_views: int = 256,
                          device="cuda"):
    """``config_batched`` at full size with the fields built on ``device``."""
    c_dt = n / 16.0
    grid = Grid(n=(n, n, n), n_epochs=n_epochs, t0=0.0, dt=c_dt)
    j, beta = turbulent_jet_torch(grid, seed, device)
    t_mid = 0.5 * (n_epochs - 1) * c_dt
    views = [view_from_direction(grid, -d, size=size, c=1.0, t_obs=t_mid) for d in fibonacci_directions(n_views)]
    return grid, j, beta, views
