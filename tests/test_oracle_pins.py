"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
chord lengths, the volume integral of a static source, a Lorentz boost of the
photon four-momentum, brute-force fine stepping, the worked cells of Fig. 2,
the apparent transverse speed (Sec. 3.2), and limits stated in Secs. 2.2-2.3.
"""
import math
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _view(grid, direction, up, *, size=1, fov=1e-3, center=None, **kw):
    d = np.asarray(direction, float)
    d = d / np.linalg.norm(d)
    c = grid.center if center is None else np.asarray(center, float)
    kw.setdefault("beaming", False)
    kw.setdefault("lookback", False)
    return gen.View(dir=tuple(d), up=tuple(up), center=tuple(c), width=size, height=size,
                    fov_u=fov, fov_v=fov, **kw)


# ---------------------------------------------------------------- P1 chords
def test_chord_axis_aligned_anisotropic_cells():
    """Rays along -z through an anisotropic box: every chord is n_z dz and
    crosses exactly n_z cells (Sec. 2.4, non-cubic cells)."""
    grid = gen.Grid(n=(5, 7, 3), dx=(1.0, 0.5, 2.0))
    j, b = gen.uniform_fields(grid, 1.0)
    # pixel pitch = cell size, so pixel centres sit on cell centres
    v = gen.View(dir=(0, 0, -1), up=(0, 1, 0), center=tuple(grid.center), width=5, height=7,
                 fov_u=5.0, fov_v=3.5, beaming=False, lookback=False)
    img, cnt = oracle.render(grid, j, b, v, counts=True)
    # e_v = +y, e_u = s x e_v = (-z) x y = +x
    assert np.allclose(img, 3 * 2.0, rtol=0, atol=1e-12)
    assert np.all(cnt == 3)


@pytest.mark.parametrize("theta", [0.0, 10.0, 30.0, 44.0])
def test_chord_tilted_through_centre(theta):
    """A ray in the x-z plane through the centre of an L-cube, tilted by
    theta < 45 deg from z, has chord L / cos(theta)."""
    L = 12
    grid = gen.Grid(n=(L, L, L))
    j, b = gen.uniform_fields(grid, 1.0)
    th = math.radians(theta)
    v = _view(grid, (-math.sin(th), 0.0, -math.cos(th)), (1.0, 0.0, 0.0) if theta == 0 else (0.0, 0.0, 1.0))
    img = oracle.render(grid, j, b, v)
    assert img[0, 0] == pytest.approx(L / math.cos(th), rel=1e-12)


def test_chord_main_diagonal():
    L = 9
    grid = gen.Grid(n=(L, L, L))
    j, b = gen.uniform_fields(grid, 1.0)
    v = _view(grid, (1.0, 1.0, 1.0), (0.0, 0.0, 1.0))
    assert oracle.render(grid, j, b, v)[0, 0] == pytest.approx(math.sqrt(3.0) * L, rel=1e-12)


@pytest.mark.parametrize("offset", [0.0, 1.3, -2.7, 4.1])
def test_chord_offset_45deg(offset):
    """Ray along (1, 0, 1)/sqrt(2) displaced by b along e_v = (-1, 0, 1)/sqrt(2):
    it runs on the line x - z = -sqrt(2) b of the square cross-section, so its
    chord is sqrt(2) L - 2 |b| (for |b| < L / sqrt(2))."""
    L = 8
    grid = gen.Grid(n=(L, 3, L))
    j, b = gen.uniform_fields(grid, 1.0)
    ev = np.array([-1.0, 0.0, 1.0]) / math.sqrt(2.0)
    v = _view(grid, (1.0, 0.0, 1.0), (0.0, 0.0, 1.0), center=grid.center + offset * ev)
    assert oracle.render(grid, j, b, v)[0, 0] == pytest.approx(math.sqrt(2.0) * L - 2.0 * abs(offset), rel=1e-12)


def test_image_orientation_single_cell():
    """A single bright cell at +x of the centre, viewed along -z with up = +y,
    lands right of centre (e_u = s x e_v = +x); at +y it lands above."""
    grid = gen.Grid(n=(8, 8, 8))
    j = np.zeros((1, 8, 8, 8))
    j[0, 4, 4, 6] = 1.0   # (z, y, x): x = 6
    j[0, 4, 7, 4] = 2.0   # y = 7
    v = gen.View(dir=(0, 0, -1), up=(0, 1, 0), center=tuple(grid.center), width=8, height=8,
                 fov_u=8.0, fov_v=8.0, beaming=False, lookback=False)
    img = oracle.render(grid, j, None, v)
    assert img[4, 6] == pytest.approx(1.0) and img[7, 4] == pytest.approx(2.0)
    assert np.count_nonzero(img) == 2


# ------------------------------------------------------ P2 static-source flux
def test_flux_equals_volume_integral_axis_aligned():
    """beta = 0: h_u h_v sum(I) = sum(j) V_cell, exactly, for views along each
    axis with pixel centres on cell centres."""
    rng = np.random.default_rng(11)
    grid = gen.Grid(n=(6, 5, 4), dx=(1.0, 0.7, 1.9))
    j = rng.random((1, 4, 5, 6))
    vol = j.sum() * np.prod(grid.dx)
    ext = grid.extent
    cases = [((0, 0, -1), (0, 1, 0), (6, 5), (ext[0], ext[1])),
             ((-1, 0, 0), (0, 0, 1), (5, 4), (ext[1], ext[2])),
             ((0, 1, 0), (0, 0, 1), (6, 4), (ext[0], ext[2]))]
    for d, up, (w, h), (fu, fv) in cases:
        v = gen.View(dir=d, up=up, center=tuple(grid.center), width=w, height=h, fov_u=fu, fov_v=fv,
                     beaming=False, lookback=False)
        img = oracle.render(grid, j, None, v)
        assert oracle.pixel_area(v) * img.sum() == pytest.approx(vol, rel=1e-12)


def test_flux_converges_to_volume_integral_oblique():
    """For an oblique view the pixel sum is a midpoint quadrature of the
    projected image, converging to the volume integral under refinement."""
    rng = np.random.default_rng(12)
    grid = gen.Grid(n=(5, 6, 4), dx=(1.0, 1.0, 1.5))
    j = rng.random((1, 4, 6, 5))
    vol = j.sum() * np.prod(grid.dx)
    errs = []
    for size in (32, 64, 128):
        v = gen.view_from_angles(grid, 37.0, 23.0, size=size, beaming=False, lookback=False)
        img = oracle.render(grid, j, None, v)
        errs.append(abs(oracle.pixel_area(v) * img.sum() - vol) / vol)
    assert errs[-1] < 2e-3
    assert errs[2] < errs[0]


# --------------------------------------------------------- P3 Doppler factor
def _doppler_by_boost(beta, n_hat):
    """nu_obs / nu_rest for a photon moving along n_hat (towards the observer),
    from a Lorentz boost of its four-momentum into the fluid frame."""
    b = np.asarray(beta, float)
    b2 = b @ b
    g = 1.0 / math.sqrt(1.0 - b2)
    lam = np.eye(4)
    lam[0, 0] = g
    lam[0, 1:] = lam[1:, 0] = -g * b
    lam[1:, 1:] += (g - 1.0) * np.outer(b, b) / b2
    k_lab = np.concatenate([[1.0], np.asarray(n_hat, float)])
    k_fluid = lam @ k_lab
    return k_lab[0] / k_fluid[0]


@pytest.mark.parametrize("beta,theta,alpha", [((0, 0, 0.9), 30.0, -0.6), ((0, 0, 0.9), 10.0, -0.6),
                                              ((0, 0, 0.9), 45.0, -0.6), ((0.3, -0.5, 0.7), 65.0, -0.6),
                                              ((0, 0, -0.95), 20.0, 0.4), ((0, 0.99, 0), 90.0, -1.0)])
def test_doppler_boost_uniform_velocity(beta, theta, alpha):
    """Uniform beta: I_beamed / I_unbeamed = D^(2 - alpha) per pixel, with D
    from a Lorentz boost of the photon travelling towards the observer."""
    grid = gen.Grid(n=(6, 6, 6))
    j, b = gen.uniform_fields(grid, 1.0, beta)
    v = gen.view_from_angles(grid, theta, 0.0, size=8, lookback=False, beaming=True, alpha=alpha)
    n_hat = -np.asarray(v.dir)
    D = _doppler_by_boost(beta, n_hat)
    on = oracle.render(grid, j, b, v)
    off = oracle.render(grid, j, b, v.with_(beaming=False))
    mask = off > 0
    assert mask.sum() > 10
    assert np.allclose(on[mask] / off[mask], D ** (2.0 - alpha), rtol=1e-12)


def test_doppler_numeric_values():
    """D = 1/(Gamma(1 - beta cos theta)) at beta = 0.9 for theta = 30, 10, 45."""
    for th, expect in ((30.0, 1.97613), (10.0, 3.83459), (45.0, 1.19880)):
        n_hat = (math.sin(math.radians(th)), 0.0, math.cos(math.radians(th)))
        assert _doppler_by_boost((0, 0, 0.9), n_hat) == pytest.approx(expect, abs=2e-5)


# ------------------------------------------------ P4 brute-force fine steps
def _brute_force_pixel(grid, j, beta, view, p, q, e_u, e_v, h=1e-4):
    """Walk the ray in steps h, look up the cell under each step midpoint and
    the fields at its own retarded time.  Independent of the oracle's plane
    enumeration; the camera basis is passed in closed form."""
    s_hat = np.asarray(view.dir, float)
    a = (p + 0.5 - view.width / 2) * view.fov_u / view.width
    bq = (q + 0.5 - view.height / 2) * view.fov_v / view.height
    r0 = np.asarray(view.center) + a * np.asarray(e_u) + bq * np.asarray(e_v)
    reach = float(np.linalg.norm(grid.extent)) + float(np.linalg.norm(r0 - grid.center))
    s = np.arange(-reach, reach, h) + 0.5 * h
    x = r0[None, :] + s[:, None] * s_hat[None, :]
    idx = np.floor((x - np.asarray(grid.origin)) / np.asarray(grid.dx)).astype(np.int64)
    ok = np.all((idx >= 0) & (idx < np.asarray(grid.n)), axis=1)
    s, idx = s[ok], idx[ok]
    M = grid.n_epochs
    tbar = view.t_obs - s / view.c if view.lookback else np.full_like(s, view.t_obs)
    u = (tbar - grid.t0) / grid.dt
    if not view.lookback:
        u = np.clip(u, 0, M - 1)
    # Eq. 9: the hat weights of Eq. 7 summed over the stored snapshots only
    total = 0.0
    n_hat = -s_hat
    for m in range(M):
        w = np.clip(1.0 - np.abs(u - m), 0.0, None)
        sel = w > 0
        if not np.any(sel):
            continue
        ii = idx[sel]
        jv = j[m, ii[:, 2], ii[:, 1], ii[:, 0]]
        if view.beaming:
            bv = beta[m, ii[:, 2], ii[:, 1], ii[:, 0]]
            D = np.array([_doppler_by_boost(bb, n_hat) if np.any(bb) else 1.0 for bb in bv])
            jv = jv * D ** (2.0 - view.alpha)
        total += float(np.sum(w[sel] * jv)) * h
    return view.nu_ratio ** view.alpha * total


def _random_tiny(seed, M=3):
    rng = np.random.default_rng(seed)
    grid = gen.Grid(n=(5, 4, 6), origin=(-1.0, 2.0, 0.5), dx=(1.0, 1.3, 0.8), n_epochs=M, t0=-0.5, dt=1.7)
    j = rng.random((M, 6, 4, 5)) + 0.1
    dirs = rng.normal(size=(M, 6, 4, 5, 3))
    dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
    beta = dirs * rng.uniform(0.0, 0.85, size=(M, 6, 4, 5, 1))
    return grid, j, beta


@pytest.mark.parametrize("lookback,beaming", [(False, False), (False, True), (True, False), (True, True)])
def test_brute_force_fine_steps(lookback, beaming):
    """The exact sum equals the limit of fine-step sampling (split at epoch
    nodes so that the piecewise-linear weight is integrated exactly)."""
    grid, j, beta = _random_tiny(5)
    th = math.radians(33.0)
    s_hat = (-math.sin(th), 0.0, -math.cos(th))
    e_v = (-math.cos(th), 0.0, math.sin(th))      # +z projected on the image plane
    e_u = (0.0, 1.0, 0.0)                          # s_hat x e_v
    v = gen.View(dir=s_hat, up=(0, 0, 1), center=tuple(grid.center), width=5, height=5, fov_u=6.0,
                 fov_v=7.0, t_obs=2.2, c=1.1, beaming=beaming, lookback=lookback, alpha=-0.6, nu_ratio=1.3)
    img = oracle.render(grid, j, beta, v, split_at_nodes=True)
    checked = 0
    for p, q in [(1, 1), (2, 2), (3, 1), (2, 3), (1, 3)]:
        ref = _brute_force_pixel(grid, j, beta, v, p, q, e_u, e_v)
        if ref == 0.0:
            continue
        assert img[q, p] == pytest.approx(ref, rel=5e-4)
        checked += 1
    assert checked >= 3


@pytest.mark.parametrize("split", [False, True])
def test_pixel_list_equals_whole_image(split):
    """The pixel-list entry point (used for sampled checks of full-size
    images) takes its pairs as (p, q) = (column, row): on a non-square image,
    a random anisotropic grid with lookback and beaming, every listed pixel
    equals the whole-image render at [q, p] bit for bit, counts included, in
    any order and with repeats; pixels off the image give 0 and no samples."""
    rng = np.random.default_rng(11)
    M = 4
    grid = gen.Grid(n=(9, 6, 7), origin=(1.5, -2.0, 0.25), dx=(0.7, 1.2, 1.0), n_epochs=M, t0=0.3, dt=1.9)
    nx, ny, nz = grid.n
    j = rng.random((M, nz, ny, nx)) + 0.05
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = d * rng.uniform(0.0, 0.9, size=(M, nz, ny, nx, 1))
    v = gen.view_from_angles(grid, 57.0, 23.0, size=13, c=1.3, t_obs=3.1, nu_ratio=1.7).with_(
        height=9, fov_v=gen.view_from_angles(grid, 57.0, 23.0, size=13).fov_v * 9 / 13)
    img, cnt = oracle.render(grid, j, beta, v, counts=True, split_at_nodes=split)
    assert np.count_nonzero(img) > img.size // 2
    pq = [(p, q) for q in range(v.height) for p in range(v.width)]
    sel = rng.permutation(len(pq))
    listed = np.array([pq[k] for k in sel] + [pq[k] for k in sel[:40]], dtype=np.int32)
    val, c = oracle.render_pixels(grid, j, beta, v, listed, counts=True, split_at_nodes=split)
    want = img[listed[:, 1], listed[:, 0]]
    assert np.array_equal(val, want)
    assert np.array_equal(c, cnt[listed[:, 1], listed[:, 0]])
    # the transposed reading would differ: the image is not symmetric
    assert not np.array_equal(img[: v.height, : v.height], img[: v.height, : v.height].T)
    off = np.array([(-1, 0), (0, -1), (v.width, 0), (0, v.height), (v.width + 5, v.height + 5),
                    (-(2 ** 31), 3), (3, 2 ** 31 - 1)], dtype=np.int32)
    val, c = oracle.render_pixels(grid, j, beta, v, off, counts=True, split_at_nodes=split)
    assert np.all(val == 0.0) and np.all(c == 0)


def test_midpoint_equals_split_without_node_crossings():
    """With the fields read at one epoch coordinate per chord, the chord
    midpoint is exact whenever no chord crosses an epoch node; fast light is
    such a case, and so is a static field."""
    grid, j, beta = _random_tiny(6)
    v = gen.view_from_angles(grid, 52.0, 17.0, size=9, t_obs=1.4, c=0.9, lookback=False)
    a = oracle.render(grid, j, beta, v)
    b = oracle.render(grid, j, beta, v, split_at_nodes=True)
    assert np.allclose(a, b, rtol=1e-13, atol=0)


# ----------------------------------------------------- P11 Fig. 2 weights
def test_fig2_worked_weights():
    """Single cell whose centre sits on the image plane (s = 0, t_bar = t_obs):
    with one-hot epochs the image value is the weight W_{n,m}."""
    rows = [list(map(float, ln.split())) for ln in open(os.path.join(GOLDEN, "fig2_weights.txt"))
            if ln.strip() and not ln.startswith("#")]
    for tbar, dt, mbar, w0, w1 in rows:
        M = 30
        grid = gen.Grid(n=(1, 1, 1), n_epochs=M, t0=0.0, dt=dt)
        v = _view(grid, (0, 0, -1), (0, 1, 0), t_obs=tbar, c=1.0, lookback=True)
        for m, expect in ((int(mbar), w0), (int(mbar) + 1, w1), (int(mbar) - 1, 0.0), (int(mbar) + 2, 0.0)):
            j = np.zeros((M, 1, 1, 1))
            j[m] = 1.0
            assert oracle.render(grid, j, None, v)[0, 0] == pytest.approx(expect, abs=1e-12)


# ------------------------------------------- P9, P10, P12 limits and scaling
def test_fast_light_limit():
    """c -> infinity: the lookback render equals the single-time render."""
    grid, j, beta = _random_tiny(7, M=4)
    v = gen.view_from_angles(grid, 61.0, 40.0, size=7, t_obs=2.9, c=math.inf)
    a = oracle.render(grid, j, beta, v)
    b = oracle.render(grid, j, beta, v.with_(lookback=False))
    assert np.array_equal(a, b)
    near = oracle.render(grid, j, beta, v.with_(c=1e9))
    assert np.allclose(near, b, rtol=1e-7)


def test_static_field_lookback_equals_fast_light():
    """Identical epochs: the weights form a partition of unity, so lookback
    equals fast light wherever the window covers the ray."""
    grid, j, beta = _random_tiny(8, M=5)
    j[:] = j[0]
    beta[:] = beta[0]
    v = gen.view_from_angles(grid, 28.0, 75.0, size=7, t_obs=20.0, c=1.0)
    # window [c(t_obs - t_{M-1}), c(t_obs - t_0)] = [13.7, 20.5] must hold the box
    v = v.with_(t_obs=grid.t0 + 2 * grid.dt + 0.0)
    v = v.with_(c=100.0)
    a = oracle.render(grid, j, beta, v)
    b = oracle.render(grid, j, beta, v.with_(lookback=False))
    assert np.allclose(a, b, rtol=1e-12, atol=0)


def test_frequency_scaling():
    grid, j, beta = _random_tiny(9)
    v = gen.view_from_angles(grid, 40.0, 10.0, size=6, t_obs=1.0, c=2.0, alpha=-0.6)
    base = oracle.render(grid, j, beta, v)
    for ratio in (0.5, 2.5, 10.0):
        scaled = oracle.render(grid, j, beta, v.with_(nu_ratio=ratio))
        assert np.allclose(scaled, ratio ** -0.6 * base, rtol=1e-13)


def test_outside_window_is_dark():
    """Lookback: a time more than one cadence outside the stored epochs
    contributes nothing."""
    grid, j, beta = _random_tiny(10)
    v = gen.view_from_angles(grid, 40.0, 10.0, size=6, t_obs=500.0, c=1.0)
    assert np.all(oracle.render(grid, j, beta, v) == 0.0)


# ------------------------------------------------------ P5 apparent speed
def blob_worldline(theta_deg, beta_z=0.95, sigma=1.5, k=3.0, c=1.0, dt=None, shift=0.65):
    """A Gaussian blob moving along +z at beta_z, stored over enough epochs
    that its whole observed light-cone slice (emission times spread by
    1/(1 - beta cos theta)) and +-1.5 ``shift`` of observer time stay inside
    the stored worldline.  Returns grid, j, beta, view and observer times."""
    kappa = 1.0 - beta_z * math.cos(math.radians(theta_deg))
    if dt is None:
        dt = 2.0 if kappa < 0.2 else 1.0
    t_half = k * sigma / (c * kappa) + 1.5 * shift / kappa + 2.0
    M = int(math.ceil(2 * t_half / dt)) + 1
    pad = k * sigma + 2.0
    nxy = int(math.ceil(2 * pad))
    nz = int(math.ceil(beta_z * c * (M - 1) * dt + 2 * pad))
    grid = gen.Grid(n=(nxy, nxy, nz), n_epochs=M, t0=0.0, dt=dt)
    start = np.array([nxy / 2, nxy / 2, pad])
    j = np.stack([gen.gaussian_blob(grid, start + [0, 0, beta_z * c * dt * m], sigma)
                  for m in range(M)]).astype(np.float32)
    beta = np.zeros(j.shape + (3,), dtype=np.float32)
    beta[..., 2] = beta_z
    view = gen.view_from_angles(grid, theta_deg, 0.0, size=64, fov=40.0, c=c, beaming=True, lookback=True)
    t_mid = 0.5 * (M - 1) * dt
    pos = start + [0, 0, beta_z * c * t_mid]
    t_obs_mid = t_mid + float(np.dot(pos - grid.center, np.asarray(view.dir))) / c
    times = [t_obs_mid + f * shift for f in (-1.5, -0.5, 0.5, 1.5)]
    return grid, j, beta, view, times


@pytest.mark.parametrize("theta,expect", [(10.0, 2.5603), (45.0, 2.0465)])
def test_apparent_superluminal_speed(theta, expect):
    """A Gaussian blob moving at beta = 0.95 along +z appears to move across
    the sky at beta sin(theta) / (1 - beta cos(theta)) (Sec. 3.2, Eq. 21)."""
    beta_z = 0.95
    assert beta_z * math.sin(math.radians(theta)) / (1 - beta_z * math.cos(math.radians(theta))) == \
        pytest.approx(expect, abs=1e-4)
    grid, j, b, v0, times = blob_worldline(theta, beta_z)
    cents = []
    q = (np.arange(v0.height) + 0.5 - v0.height / 2) * v0.fov_v / v0.height
    for t_obs in times:
        img = oracle.render(grid, j, b, v0.with_(t_obs=t_obs))
        cents.append(float((img.sum(axis=1) * q).sum() / img.sum()))
    speed = np.polyfit(times, cents, 1)[0] / v0.c
    assert speed == pytest.approx(expect, rel=0.02)


def test_no_lookback_speed_is_lab_frame():
    """Without lookback the same blob moves at beta sin(theta) on the sky
    (Table 1, routines A and B)."""
    theta, beta_z = 45.0, 0.95
    grid, j, b, v0, times = blob_worldline(theta, beta_z)
    v0 = v0.with_(lookback=False)
    q = (np.arange(v0.height) + 0.5 - v0.height / 2) * v0.fov_v / v0.height
    ts = [0.5 * (grid.n_epochs - 1) * grid.dt + d for d in (-3.0, -1.0, 1.0, 3.0)]
    cents = []
    for t_obs in ts:
        img = oracle.render(grid, j, b, v0.with_(t_obs=t_obs))
        cents.append(float((img.sum(axis=1) * q).sum() / img.sum()))
    speed = np.polyfit(ts, cents, 1)[0]
    assert speed == pytest.approx(beta_z * math.sin(math.radians(theta)), rel=0.01)


@pytest.mark.parametrize("t_obs,epoch", [(-40.0, 0), (1000.0, -1)])
def test_fast_light_clamps_to_end_epochs(t_obs, epoch):
    """Without lookback an observer time before the first (after the last)
    snapshot reads the first (last) one: the single-snapshot render of that
    epoch (reading A8 of Eq. 10's fast-light limit)."""
    grid, j, beta = _random_tiny(11, M=4)
    v = gen.view_from_angles(grid, 47.0, 12.0, size=6, t_obs=t_obs, lookback=False)
    single = gen.Grid(n=grid.n, origin=grid.origin, dx=grid.dx, n_epochs=1, t0=0.0, dt=1.0)
    a = oracle.render(grid, j, beta, v)
    b = oracle.render(single, j[epoch:][:1] if epoch >= 0 else j[-1:], beta[-1:] if epoch < 0 else beta[:1], v)
    assert np.array_equal(a, b)


def test_window_edge_fades_linearly():
    """Eq. 9 sums Eq. 7's weights over the stored snapshots, so a time just
    past the last snapshot keeps weight 1 - delta on it (continuity in t_bar)."""
    M, dt = 4, 2.0
    grid = gen.Grid(n=(1, 1, 1), n_epochs=M, t0=0.0, dt=dt)
    j = np.zeros((M, 1, 1, 1))
    j[M - 1] = 1.0
    j[0] = 10.0
    v = _view(grid, (0, 0, -1), (0, 1, 0), c=1.0, lookback=True)
    for t_obs, expect in ((6.0, 1.0), (6.5, 0.75), (7.9, 0.05), (8.0, 0.0), (-0.5, 7.5), (-2.0, 0.0)):
        assert oracle.render(grid, j, None, v.with_(t_obs=t_obs))[0, 0] == pytest.approx(expect, abs=1e-12)
