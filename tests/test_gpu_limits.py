"""Edge sizes of the CUDA path against the oracle: the longest grid axis the
kernels accept (4096 cells, whose march tables exceed the default 48 KB of
shared memory), the widest image (16384 pixels), a one-cell grid, and a long
series of snapshots along one ray."""
import numpy as np
import pytest

import gen
import oracle
from tests._parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_09322_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _fields(rng, n, M, bmax=0.8):
    nx, ny, nz = n
    j = (rng.random((M, nz, ny, nx)) + 0.05).astype(np.float32)
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = (d * rng.uniform(0.0, bmax, size=(M, nz, ny, nx, 1))).astype(np.float32)
    return j, beta


def _render(ctx, grid, j, beta, views, **kw):
    vol = ctx.load_snapshots(grid, j, beta, **kw)
    img = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    ctx.unload(vol)
    return img.cpu().numpy()


def test_longest_axis(ctx):
    rng = np.random.default_rng(1)
    # 4096 + 2048 + 3 cells of edges: the march tables take 49 KB of shared memory
    grid = gen.Grid(n=(4096, 2048, 3), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=2, t0=0.0, dt=900.0)
    j, beta = _fields(rng, grid.n, grid.n_epochs)
    views = [gen.view_from_direction(grid, d, size=64, c=1.0, t_obs=1000.0, fov=40.0)
             for d in ([-1.0, 0.02, 0.03], [0.999, -0.03, 0.02], [0.3, 0.6, -0.74])]
    imgs = _render(ctx, grid, j, beta, views)
    for k, v in enumerate(views):
        assert_parity(imgs[k], oracle.render(grid, j, beta, v), what=f"4096-cell axis view {k}")


def test_widest_image(ctx):
    rng = np.random.default_rng(2)
    grid = gen.Grid(n=(24, 20, 16), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=3, t0=0.0, dt=2.0)
    j, beta = _fields(rng, grid.n, grid.n_epochs)
    v = gen.view_from_angles(grid, 37.0, 21.0, size=16384, height=3, c=1.0, t_obs=2.0)
    img = _render(ctx, grid, j, beta, [v])[0]
    cols = np.arange(0, 16384, 97)
    pix = np.array([(c, r) for c in cols for r in range(3)], dtype=np.int32)
    ref = oracle.render_pixels(grid, j, beta, v, pix)
    assert_parity(img[pix[:, 1], pix[:, 0]], ref, what="16384-pixel row")


def test_one_cell_grid(ctx):
    rng = np.random.default_rng(3)
    grid = gen.Grid(n=(1, 1, 1), origin=(0.5, -0.5, 2.0), dx=(2.0, 1.5, 0.7), n_epochs=2, t0=0.0, dt=1.0)
    j, beta = _fields(rng, grid.n, grid.n_epochs)
    views = [gen.view_from_angles(grid, th, ph, size=9, c=2.0, t_obs=0.6) for th, ph in [(20, 40), (90, 0), (160, 300)]]
    imgs = _render(ctx, grid, j, beta, views)
    for k, v in enumerate(views):
        assert_parity(imgs[k], oracle.render(grid, j, beta, v), what=f"one cell view {k}")


def test_many_snapshots_along_a_ray(ctx):
    """c dt of a fifth of a cell: a ray crossing the box reads hundreds of
    snapshot pairs."""
    rng = np.random.default_rng(4)
    grid = gen.Grid(n=(40, 8, 8), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=500, t0=0.0, dt=0.2)
    j, beta = _fields(rng, grid.n, grid.n_epochs)
    views = [gen.view_from_direction(grid, d, size=24, c=1.0, t_obs=60.0)
             for d in ([-1.0, 0.1, 0.05], [0.7, 0.5, -0.5])]
    imgs = _render(ctx, grid, j, beta, views, brick=4, super_brick=2, paired=True)
    for k, v in enumerate(views):
        assert_parity(imgs[k], oracle.render(grid, j, beta, v), what=f"500 snapshots view {k}")
