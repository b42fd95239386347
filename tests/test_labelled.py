"""Labelled mode: a scene of non-overlapping sub-domains, each with its own
Cartesian grid (the paper's second input form, Sec. 4, for mesh-refined
simulations).  A pixel's intensity is the sum over the sub-domains of its
ray's sum through each, i.e. Eq. 19 over the union of their cells.

CPU pin: the oracle is additive over any split of one grid into boxes (with
lookback and beaming), which is what makes the sum over sub-domains Eq. 19 of
the union.  GPU: a uniform emitter spread over sub-domains of different cell
sizes gives the analytic chord through the union box; random fields match the
sum of the oracle's per-sub-domain renders at 1e-5; overlapping boxes are
refused.
"""
import math

import numpy as np
import pytest

import gen
import oracle
from tests._parity import assert_parity


def _fields(rng, n, M):
    nx, ny, nz = n
    j = (rng.random((M, nz, ny, nx)) + 0.05).astype(np.float32)
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = (d * rng.uniform(0.0, 0.9, size=(M, nz, ny, nx, 1))).astype(np.float32)
    return j, beta


def _split_x(grid, j, beta, cut):
    """The grid cut at cell column `cut` along x into two sub-domains."""
    a = gen.Grid(n=(cut, grid.n[1], grid.n[2]), origin=grid.origin, dx=grid.dx, n_epochs=grid.n_epochs,
                 t0=grid.t0, dt=grid.dt)
    b = gen.Grid(n=(grid.n[0] - cut, grid.n[1], grid.n[2]),
                 origin=(grid.origin[0] + cut * grid.dx[0], grid.origin[1], grid.origin[2]), dx=grid.dx,
                 n_epochs=grid.n_epochs, t0=grid.t0, dt=grid.dt)
    return [(a, np.ascontiguousarray(j[..., :cut]), np.ascontiguousarray(beta[..., :cut, :])),
            (b, np.ascontiguousarray(j[..., cut:]), np.ascontiguousarray(beta[..., cut:, :]))]


def test_oracle_is_additive_over_sub_domains():
    rng = np.random.default_rng(3)
    grid = gen.Grid(n=(14, 9, 11), origin=(-2.0, 1.0, 0.3), dx=(1.0, 0.8, 1.3), n_epochs=4, t0=0.2, dt=1.9)
    j, beta = _fields(rng, grid.n, grid.n_epochs)
    for theta, phi, lookback in [(35.0, 20.0, True), (80.0, 200.0, True), (120.0, 45.0, False)]:
        v = gen.view_from_angles(grid, theta, phi, size=24, c=1.3, t_obs=3.1, lookback=lookback)
        whole = oracle.render(grid, j, beta, v)
        parts = sum(oracle.render(g, jj, bb, v) for g, jj, bb in _split_x(grid, j, beta, 6))
        np.testing.assert_allclose(parts, whole, rtol=1e-12, atol=1e-12 * whole.max())


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2609_09322_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _uniform(grid):
    M, (nx, ny, nz) = grid.n_epochs, grid.n
    return np.ones((M, nz, ny, nx), np.float32), np.zeros((M, nz, ny, nx, 3), np.float32)


@pytest.mark.gpu
def test_uniform_emitter_over_mixed_resolutions_gives_the_chord(ctx):
    """Box [0,16) x [0,8) x [0,8) built from a coarse half (dx = 1) and a fine
    half (dx = 0.5): with j' = 1 and beta = 0 every pixel is the length of its
    ray inside the box."""
    coarse = gen.Grid(n=(8, 8, 8), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=1)
    fine = gen.Grid(n=(16, 16, 16), origin=(8.0, 0.0, 0.0), dx=(0.5, 0.5, 0.5), n_epochs=1)
    vols = [ctx.load_snapshots(g, *_uniform(g)) for g in (coarse, fine)]
    box = gen.Grid(n=(16, 8, 8), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=1)
    for theta, phi in [(90.0, 0.0), (60.0, 30.0), (37.0, 200.0)]:
        v = gen.view_from_angles(box, theta, phi, size=48, lookback=False, beaming=False)
        img = ctx.render_labelled(vols, [v])[0].cpu().numpy()
        # analytic slab chord of every pixel's ray through the union box
        sh = np.asarray(v.dir) / np.linalg.norm(v.dir)
        up = np.asarray(v.up)
        ev = up - np.dot(up, sh) * sh
        ev /= np.linalg.norm(ev)
        eu = np.cross(sh, ev)
        hu = v.fov_u / v.width
        p = (np.arange(v.width) + 0.5 - 0.5 * v.width) * hu
        q = (np.arange(v.height) + 0.5 - 0.5 * v.height) * hu
        P, Q = np.meshgrid(p, q)
        r0 = np.asarray(v.center) + P[..., None] * eu + Q[..., None] * ev
        lo, hi = np.zeros(3), np.array([16.0, 8.0, 8.0])
        with np.errstate(divide="ignore", invalid="ignore"):
            t1, t2 = (lo - r0) / sh, (hi - r0) / sh
        s_in = np.nanmax(np.where(sh != 0, np.minimum(t1, t2), -np.inf), axis=-1)
        s_out = np.nanmin(np.where(sh != 0, np.maximum(t1, t2), np.inf), axis=-1)
        inside = np.all(np.where(sh == 0, (r0 >= lo) & (r0 < hi), True), axis=-1)
        chord = np.where(inside, np.maximum(s_out - s_in, 0.0), 0.0)
        # A ray grazing a box corner has a chord of a few thousandths whose two
        # ends are float32 crossings: they resolve about 1e-7 of a unit, so the
        # absolute floor here is 2e-7 of the peak chord (bright pixels: 1e-5).
        assert_parity(img, chord, floor_frac=0.02, what=f"labelled chord theta={theta}")
    for vol in vols:
        ctx.unload(vol)


@pytest.mark.gpu
def test_labelled_matches_the_sum_of_sub_domain_oracles(ctx):
    rng = np.random.default_rng(8)
    doms = [gen.Grid(n=(10, 12, 9), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=5, t0=0.0, dt=2.0),
            gen.Grid(n=(12, 24, 18), origin=(10.0, 0.0, 0.0), dx=(0.5, 0.5, 0.5), n_epochs=5, t0=0.0, dt=2.0),
            gen.Grid(n=(6, 6, 4), origin=(0.0, 12.0, 0.0), dx=(1.5, 1.5, 2.25), n_epochs=3, t0=2.0, dt=2.5)]
    fields = [_fields(rng, g.n, g.n_epochs) for g in doms]
    vols = [ctx.load_snapshots(g, j, b) for g, (j, b) in zip(doms, fields)]
    scene = gen.Grid(n=(16, 21, 9), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=5, t0=0.0, dt=2.0)
    views = [gen.view_from_angles(scene, th, ph, size=40, c=1.2, t_obs=5.0)
             for th, ph in [(50.0, 10.0), (100.0, 250.0), (0.0, 0.0)]]
    imgs = ctx.render_labelled(vols, views).cpu().numpy()
    for k, v in enumerate(views):
        ref = sum(oracle.render(g, j, b, v) for g, (j, b) in zip(doms, fields))
        assert_parity(imgs[k], ref, what=f"labelled view {k}")
    for vol in vols:
        ctx.unload(vol)


@pytest.mark.gpu
def test_overlapping_sub_domains_are_refused(ctx):
    import paper_2609_09322_gb300 as g
    a = gen.Grid(n=(8, 8, 8), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=1)
    b = gen.Grid(n=(8, 8, 8), origin=(7.5, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=1)
    vols = [ctx.load_snapshots(x, *_uniform(x)) for x in (a, b)]
    v = gen.view_from_angles(a, 30.0, 0.0, size=8, lookback=False)
    with pytest.raises(g.GbdError) as e:
        ctx.render_labelled(vols, [v])
    assert e.value.code == g.gbdart.ERR_INVALID
    for vol in vols:
        ctx.unload(vol)
